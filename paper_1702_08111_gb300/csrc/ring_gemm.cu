// Legendre ring term of the boundary values as a tensor-core GEMM (split
// tiers): for every patch p and every ring-table row r of one face-plane axis
// (relative face node x in Omega_beta \ Omega_alpha, Sec. 4 eq. philocmlcII),
//   R[p][r] = sum_q c_q(p) D[r][q],   D[r][q] = (B_q - I^H B_q)(x_r)
// (the basis fields of Sec. 4 Step 1 minus their coarse interpolant), i.e.
// R = D C^T with C the [patch x npad] Legendre coefficients.  The boundary
// kernel then adds R[p][row(g - n i_p)] per ring patch instead of forming
// each npad-term dot product.
//
// tcgen05 kind::tf32 with split operands (3xTF32: x = hi + lo, both TF32;
// D_hi C_hi + D_hi C_lo + D_lo C_hi accumulated in FP32 in TMEM), M = 128
// table rows per CTA, N = NT patches, K = 8 per instruction.  Operands sit in
// shared memory in the canonical K-major layout without swizzle: 8 x 16-byte
// core matrices, 128 bytes apart along K (leading byte offset) and 256 bytes
// apart along M / N (stride byte offset), one block per (k-step, hi / lo).
// The table operand is prepared in that layout at plan time and staged with
// one bulk copy (TMA engine); the coefficients are split and laid out by the
// CTA's threads.  One thread issues the MMAs; all four warps read the
// accumulator back (tcgen05.ld, lane = table row) and store it with
// coalesced writes along the rows.
#include <cstdint>

#include "mlc_internal.h"

namespace mlc {
namespace {

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait_bounded(uint64_t *bar, unsigned parity, int tries) {
    for (int i = 0; i < tries; ++i)
        if (bar_try_wait(bar, parity)) return true;
    return false;
}
// one bulk copy global -> shared completing on bar; addresses 16-byte aligned,
// bytes a multiple of 16
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (>> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_load16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kRowsTile = 128;            // M: table rows per CTA (one TMEM lane each)
constexpr int kABlock = kRowsTile * 8 * 4;  // bytes of one (k-step, hi / lo) block of the table operand
constexpr int kWaitTries = 1 << 22;

// R[p][row] for table row tile blockIdx.x and patch tile blockIdx.y (NT
// patches), 128 threads.  aimg: the table operand of this axis, kABlock x
// 2 ksteps per row tile, in shared-memory order.  mom: [NP][npad] FP32.
template <int NT>
__global__ void __launch_bounds__(128) k_ring_gemm(const float *__restrict__ aimg, const float *__restrict__ mom,
                                                   int npad, int NP, int ksteps, float *__restrict__ R,
                                                   long rows_pad, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int kBBlock = NT * 8 * 4;  // bytes of one (k-step, hi / lo) block of the coefficients
    const int aBytes = ksteps * 2 * kABlock, bBytes = ksteps * 2 * kBBlock;
    unsigned char *sA = sm, *sB = sm + aBytes;
    uint64_t *bar = (uint64_t *)(sm + aBytes + bBytes);  // [0] table copy, [1] MMAs done
    uint32_t *tslot = (uint32_t *)(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rt = blockIdx.x, pt = blockIdx.y;
    if (tid == 0) {
        bar_init(&bar[0], 1);
        bar_init(&bar[1], 1);
    }
    __syncthreads();
    if (tid == 0) {
        bar_expect_tx(&bar[0], (unsigned)aBytes);
        bulk_copy(sA, aimg + (long)rt * (aBytes / 4), (unsigned)aBytes, &bar[0]);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(NT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // coefficients of patches pt NT + p: TF32 hi / lo in the canonical layout
    const int K8 = ksteps * 8;
    for (int e = tid; e < NT * K8; e += blockDim.x) {
        const int p = e / K8, k = e - p * K8, gp = pt * NT + p;
        const float x = (gp < NP && k < npad) ? mom[(long)gp * npad + k] : 0.f;
        const float hi = to_tf32(x), lo = to_tf32(x - hi);
        const int ks = k >> 3, off = (p >> 3) * 256 + ((k >> 2) & 1) * 128 + (p & 7) * 16 + (k & 3) * 4;
        *(float *)(sB + (ks * 2 + 0) * kBBlock + off) = hi;
        *(float *)(sB + (ks * 2 + 1) * kBBlock + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core's reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    bool ok = bar_wait_bounded(&bar[0], 0, kWaitTries);
    const bool copied = !__syncthreads_or(!ok);
    if (copied && tid == 0) {
        const uint32_t idesc = idesc_tf32(kRowsTile, NT);
        const uint32_t a0 = su32(sA), b0 = su32(sB);
        for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t ah = smem_desc(a0 + (ks * 2 + 0) * kABlock, 128, 256);
            const uint64_t al = smem_desc(a0 + (ks * 2 + 1) * kABlock, 128, 256);
            const uint64_t bh = smem_desc(b0 + (ks * 2 + 0) * kBBlock, 128, 256);
            const uint64_t bl = smem_desc(b0 + (ks * 2 + 1) * kBBlock, 128, 256);
            mma_tf32(tmem, ah, bh, idesc, ks > 0 ? 1u : 0u);
            mma_tf32(tmem, ah, bl, idesc, 1u);
            mma_tf32(tmem, al, bh, idesc, 1u);
        }
        mma_commit(&bar[1]);
    }
    bool done = false;
    if (copied) {
        done = bar_wait_bounded(&bar[1], 0, kWaitTries);
        done = !__syncthreads_or(!done);
    } else if (tid == 0) {
        bar_wait_bounded(&bar[0], 0, kWaitTries);  // one more bounded wait for the copy in flight
    }
    if (!copied || !done) {
        if (tid == 0) atomicExch(err, 1);
        if (copied && tid == 0) bar_wait_bounded(&bar[1], 0, kWaitTries);  // MMAs in flight
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const long row = (long)rt * kRowsTile + warp * 32 + lane;
        const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float v[16];
            tmem_load16(tw + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int gp = pt * NT + c0 + j;
                if (gp < NP) R[(long)gp * rows_pad + row] = v[j];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT) : "memory");
}

}  // namespace

size_t ring_gemm_smem(int ksteps, int nt) { return (size_t)ksteps * 2 * (kABlock + nt * 32) + 64; }

void configure_ring_gemm() {
    cudaFuncSetAttribute(k_ring_gemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_gemm_smem(7, 64));
    cudaFuncSetAttribute(k_ring_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_gemm_smem(7, 128));
    cudaFuncSetAttribute(k_ring_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_gemm_smem(7, 256));
}

cudaError_t launch_ring_gemm(const mlc_plan_s *pl, int axis, cudaStream_t st) {
    const Geom &g = pl->g;
    const int ks = g.ring_ksteps;
    const long tiles = g.ring_rows_pad / kRowsTile;
    const float *aimg = pl->ring_aimg + (size_t)axis * tiles * ks * 2 * (kABlock / 4);
    const int nt = g.NP >= 256 ? 256 : (g.NP >= 128 ? 128 : 64);
    dim3 grid((unsigned)tiles, (unsigned)((g.NP + nt - 1) / nt));
    const size_t smem = ring_gemm_smem(ks, nt);
    if (nt == 256)
        k_ring_gemm<256><<<grid, 128, smem, st>>>(aimg, pl->mom_f, g.npad, g.NP, ks, pl->ring_R, g.ring_rows_pad, pl->err);
    else if (nt == 128)
        k_ring_gemm<128><<<grid, 128, smem, st>>>(aimg, pl->mom_f, g.npad, g.NP, ks, pl->ring_R, g.ring_rows_pad, pl->err);
    else
        k_ring_gemm<64><<<grid, 128, smem, st>>>(aimg, pl->mom_f, g.npad, g.NP, ks, pl->ring_R, g.ring_rows_pad, pl->err);
    return cudaGetLastError();
}

// Table operand image, float offset of element (row r of axis a, k, part):
// rows of one axis in tiles of 128, each tile [k-step][hi/lo][8-row group][k
// half][row in group][k in quarter] (the shared-memory layout above).
void ring_table_image(const std::vector<double> &Dd, int nrows_axis, int npad, int ksteps, long rows_pad,
                      std::vector<float> &img) {
    const long tiles = rows_pad / kRowsTile;
    const size_t per_tile = (size_t)ksteps * 2 * (kABlock / 4);
    img.assign(3 * tiles * per_tile, 0.f);
    for (int a = 0; a < 3; ++a)
        for (long r = 0; r < nrows_axis; ++r)
            for (int k = 0; k < npad; ++k) {
                const double x = Dd[((size_t)a * nrows_axis + r) * npad + k];
                const float hi = tf32_host(x), lo = tf32_host((double)((float)x - hi));
                const long t = r / kRowsTile, rr = r % kRowsTile;
                const int ks = k >> 3;
                const size_t base = ((size_t)a * tiles + t) * per_tile;
                const size_t off = (size_t)((rr >> 3) * 64 + ((k >> 2) & 1) * 32 + (rr & 7) * 4 + (k & 3));
                img[base + (size_t)(ks * 2 + 0) * (kABlock / 4) + off] = hi;
                img[base + (size_t)(ks * 2 + 1) * (kABlock / 4) + off] = lo;
            }
}

}  // namespace mlc
