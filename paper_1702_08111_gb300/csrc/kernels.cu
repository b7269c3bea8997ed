// Solve-time kernels of the FP64 tier of the two-level MLC (Sec. 4).
//
//   moments     Legendre coefficients by composite Boole's rule (Step 1)
//   fwd_x/col/inv_x
//               Hockney convolutions (App. A.2): zero-padded periodic
//               convolution of length M, as pruned radix-2 FFTs in shared
//               memory; used for the local fields phi^{i,h} (eq.
//               initiallocalproblemsmlcII) and for the coarse solve
//               phi^H = G^H * F^H (Step 2)
//   resid       phi^{i,h} - I^H(phi^{i,h}) on the face nodes of Omega_alpha
//   assemble    F^H = sum_i F^{i,H} (eq. FDLD), a fixed-order gather
//   boundary    phi^B (eqs. philocmlcII, mlcfulldiscr) in the linear form
//               I^H(phi^H) + sum_alpha (phi^i - I^H phi^i) + sum_ring c_p (B_p - I^H B_p)
//   dirichlet   patch Dirichlet solves by DST-I (eq. last_step_fulldiscr) and
//               the Mehrstellen correction (eq. mcapplicationfulldiscr)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "mlc_internal.h"

namespace mlc {

namespace {

// Checked builds (-DMLC_CHECKED; a debugging aid standing in for a memory
// checker): computed indices into the plan's arrays are tested before use; a
// bad one is not accessed, and the plan's error word records code 2, which
// mlc_plan_status reports as MLC_ERR_INDEX.  In normal builds the test is
// compiled out.
#ifdef MLC_CHECKED
__device__ __forceinline__ bool in_range(long i, long n, int *err) {
    if (i >= 0 && i < n) return true;
    atomicCAS(err, 0, 2);
    return false;
}
#else
__device__ __forceinline__ bool in_range(long, long, int *) { return true; }
#endif

__device__ __forceinline__ int brev_bits(int i, int log2m) {
    return (int)(__brev((unsigned)i) >> (32 - log2m));
}

__device__ __forceinline__ int floordiv(int a, int b) {  // b > 0
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| a few ulp(hi) at most), about 48 significand bits.  Sums use
// the error-free two-sum of Knuth, products the FMA-based two-product; the
// FFT and DST error bounds are relative to the data norm, so no operation
// renormalises the pair.  GB300 issues FP32 on ~67x more lanes than FP64, so
// the FP64 tier's transforms and ring sums run in this arithmetic.
// ---------------------------------------------------------------------------
struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __device__ explicit dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};
struct dcx {
    dfl x, y;
};

__device__ __forceinline__ dfl df_from(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
// Sum and product are left unnormalised: (hi, lo) stays an unevaluated sum
// whose |lo| is a few ulp(hi) at most.  two_sum of the high parts is exact for
// any pair, and the product's residual is already of order 2^-24 |p|, so the
// pair keeps its ~2^-48 relative accuracy while each operation saves the
// three instructions of a fast two-sum.
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    const dfl s = two_sum(a.hi, b.hi);
    return {s.hi, s.lo + (a.lo + b.lo)};
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return {p, e};
}
__device__ __forceinline__ dcx dc_mul(dcx a, dcx w) {
    return {df_sub(df_mul(a.x, w.x), df_mul(a.y, w.y)), df_add(df_mul(a.x, w.y), df_mul(a.y, w.x))};
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) { return df_add(a, b); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return df_sub(a, b); }
__device__ __forceinline__ dfl operator-(dfl a) { return df_neg(a); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) { return df_mul(a, b); }
__device__ __forceinline__ dfl &operator*=(dfl &a, dfl b) { return a = df_mul(a, b); }
__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) { return a = df_add(a, b); }
__device__ __forceinline__ dcx cmul(dcx a, dcx w) { return dc_mul(a, w); }
// a + w x in double-float (one product, one sum)
__device__ __forceinline__ dfl df_fma(dfl w, dfl x, dfl a) { return df_add(a, df_mul(w, x)); }

// Renormalise a double-float complex value (|lo| <= ulp(hi)/2 again).  The
// transforms do it where a line is loaded (and every other radix-2 stage), so
// the unnormalised low parts grow over a few butterfly stages at most; FP32
// and FP64 values pass through.
__device__ __forceinline__ dfl renorm(dfl v) { return fast_two_sum(v.hi, v.lo); }
__device__ __forceinline__ dcx renorm(dcx v) { return {fast_two_sum(v.x.hi, v.x.lo), fast_two_sum(v.y.hi, v.y.lo)}; }
__device__ __forceinline__ float2 renorm(float2 v) { return v; }
__device__ __forceinline__ double2 renorm(double2 v) { return v; }

// Complex type of each working precision (FP64 tier: double-float; split tier: float).
template <typename R> struct Cx;
template <> struct Cx<float> {
    using T = float2;
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};
template <> struct Cx<dfl> {  // double-float complex
    using T = dcx;
    static __device__ __forceinline__ dcx mk(float a, float b) { return dcx{dfl(a, 0.f), dfl(b, 0.f)}; }
};
template <> struct Cx<double> {  // FP64 complex
    using T = double2;
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};

__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 w) {
    return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}

// Arithmetic of the steps after the local convolutions ("fine" precision):
// FP64 (the FP64 pipe) or double-float (the FP32 pipe).  Both store 8 bytes
// per value, so the arrays between these steps have one layout.
template <typename T> struct FT;
template <> struct FT<dfl> {
    static __device__ __forceinline__ dfl of(float v) { return {v, 0.f}; }
    static __device__ __forceinline__ dfl of(double v) { return df_from(v); }
    static __device__ __forceinline__ dfl of(dfl v) { return v; }
    static __device__ __forceinline__ double to(dfl v) { return df_to(v); }
    static __device__ __forceinline__ dfl rn(dfl v) { return renorm(v); }
    static __device__ __forceinline__ dfl zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ bool is0(dfl v) { return v.hi == 0.f; }
    static __device__ __forceinline__ dfl fma(dfl w, dfl x, dfl a) { return df_fma(w, x, a); }
};
template <> struct FT<double> {
    static __device__ __forceinline__ double of(float v) { return (double)v; }
    static __device__ __forceinline__ double of(double v) { return v; }
    static __device__ __forceinline__ double of(dfl v) { return df_to(v); }
    static __device__ __forceinline__ double to(double v) { return v; }
    static __device__ __forceinline__ double rn(double v) { return v; }
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ bool is0(double v) { return v == 0.0; }
    static __device__ __forceinline__ double fma(double w, double x, double a) { return ::fma(w, x, a); }
};
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// Multiply by -i (forward) or +i (inverse): a swap and a sign change, no FLOPs.
template <typename C>
__device__ __forceinline__ C mul_mi(C v, bool inv) {
    C r;
    if (inv) { r.x = -v.y; r.y = v.x; }
    else { r.x = v.y; r.y = -v.x; }
    return r;
}

// Twiddle product of a radix-2 stage with half-size hs: w = exp(-+ 2 pi i pos / (2 hs)).
// hs = 1 has w = 1 and hs = 2 has w in {1, -+i}; neither needs a multiply.
template <typename C>
__device__ __forceinline__ C twiddle(C v, int st, int pos, int tsh, const C *tw, bool inv) {
    if (st == 0) return v;
    if (st == 1) return pos ? mul_mi(v, inv) : v;
    C w = tw[pos << tsh];
    if (inv) w.y = -w.y;
    return cmul(v, w);
}

// Decimation in frequency: natural-order input, bit-reversed output.  Line l
// starts at buf + line_off(l) (lstride, plus `gap` for lines >= gap_at).
template <int LOG2M, typename C>
__device__ __forceinline__ void fft_dif(C *buf, int nlines, int lstride, int estride,
                                        const C *tw, bool inv, int gap_at = 1 << 30, int gap = 0) {
    constexpr int MH = 1 << (LOG2M - 1);
    const int total = nlines * MH;
#pragma unroll 1
    for (int st = LOG2M - 1; st >= 0; --st) {
        const int hs = 1 << st;
        const int tsh = LOG2M - 1 - st;
        for (int j = threadIdx.x; j < total; j += blockDim.x) {
            const int line = j % nlines, bf = j / nlines;
            const int grp = bf >> st, pos = bf & (hs - 1);
            const int i0 = (grp << (st + 1)) + pos;
            C *p0 = buf + line * lstride + (line >= gap_at ? gap : 0) + i0 * estride;
            C *p1 = p0 + hs * estride;
            C a = *p0, b = *p1;
            if (st & 1) { a = renorm(a); b = renorm(b); }
            *p0 = cadd(a, b);
            *p1 = twiddle(csub(a, b), st, pos, tsh, tw, inv);
        }
        __syncthreads();
    }
}

// Decimation in time: bit-reversed input, natural-order output.
template <int LOG2M, typename C>
__device__ __forceinline__ void fft_dit(C *buf, int nlines, int lstride, int estride,
                                        const C *tw, bool inv, int gap_at = 1 << 30, int gap = 0) {
    constexpr int MH = 1 << (LOG2M - 1);
    const int total = nlines * MH;
#pragma unroll 1
    for (int st = 0; st < LOG2M; ++st) {
        const int hs = 1 << st;
        const int tsh = LOG2M - 1 - st;
        for (int j = threadIdx.x; j < total; j += blockDim.x) {
            const int line = j % nlines, bf = j / nlines;
            const int grp = bf >> st, pos = bf & (hs - 1);
            const int i0 = (grp << (st + 1)) + pos;
            C *p0 = buf + line * lstride + (line >= gap_at ? gap : 0) + i0 * estride;
            C *p1 = p0 + hs * estride;
            C a = *p0, b = *p1;
            if (!(st & 1)) { a = renorm(a); b = renorm(b); }
            const C t = twiddle(b, st, pos, tsh, tw, inv);
            *p0 = cadd(a, t);
            *p1 = csub(a, t);
        }
        __syncthreads();
    }
}

// ---- TMA bulk copy (global -> shared) completing on an mbarrier -------------
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier (at most `tries` suspending
// tests); false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, int tries) {
    for (int i = 0; i < tries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Plan record and local patch index of a work item.
// Item `item` of a launch covers patch p of its plan; the item index itself
// is the slot of the item in the launch's local-convolution scratch.
__device__ __forceinline__ const PlanPtrs &item_plan(const Items &it, int item, int &p) {
    if (it.items) {
        const int2 v = it.items[item];
        p = v.y;
        return it.plans[v.x];
    }
    p = item + it.first;
    return it.plans[0];
}

template <int LOG2M, typename C>
__device__ __forceinline__ void load_twiddles(C *s_tw, const C *tw) {
    for (int t = threadIdx.x; t < (1 << (LOG2M - 1)); t += blockDim.x) s_tw[t] = tw[t];
}

// ---------------------------------------------------------------------------
// Forward real transform along axis 2 (contiguous).  Lines are rows y of the
// input; outputs kx in [0, M/2].  PATCH: input = chi-weighted charge of patch p
// read from f (nodes at index N are zero); otherwise a dense nin^3 real array.
// ---------------------------------------------------------------------------
struct FwdXArgs {
    const void *src;  // dense input (not PATCH)
    void *out;        // complex R: [slab][line][M/2+1] (not PATCH)
    int N, n, np;     // patch geometry (PATCH: n only; N, np per plan)
    int nin;          // input nodes per axis
    int lines_cta;    // lines per CTA
    const void *tw;   // complex R twiddles
    Items it;         // PATCH: work items
};

template <int LOG2M, typename TF, bool PATCH, typename R, bool SLAB = false>
__global__ void __launch_bounds__(256) k_fwd_x(FwdXArgs a) {
    using C = typename Cx<R>::T;
    constexpr int M = 1 << LOG2M, MH = M / 2 + 1, LS = M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_tw = (C *)smem_raw;
    C *buf = s_tw + M / 2;
    const int slab = blockIdx.x;  // p * nin + zi
    const int line0 = blockIdx.y * a.lines_cta;
    const int nl = min(a.lines_cta, a.nin - line0);
    load_twiddles<LOG2M>(s_tw, (const C *)a.tw);
    for (int e = threadIdx.x; e < nl * LS; e += blockDim.x) buf[e] = Cx<R>::mk(0, 0);
    __syncthreads();
    const int zi = slab % a.nin;
    int p = slab / a.nin, N = a.N, np = a.np;
    const void *src = a.src;
    void *outp = a.out;
    if constexpr (PATCH) {
        const PlanPtrs &P = item_plan(a.it, slab / a.nin, p);
        src = P.f;
        outp = a.it.a1;
        N = P.N;
        np = P.np;
    }
    for (int e = threadIdx.x; e < nl * a.nin; e += blockDim.x) {
        const int l = e / a.nin, m = e % a.nin;
        const int yi = line0 + l;
        R v;
        if constexpr (PATCH) {
            const int i2 = p % np, i1 = (p / np) % np, i0 = p / (np * np);
            const int z = i0 * a.n + zi, y = i1 * a.n + yi, x = i2 * a.n + m;
            v = R(0.0);
            if (z < N && y < N && x < N) {
                const TF *f = (const TF *)src;
                R w = (zi == 0 || zi == a.n) ? R(0.5) : R(1);
                w *= (yi == 0 || yi == a.n) ? R(0.5) : R(1);
                w *= (m == 0 || m == a.n) ? R(0.5) : R(1);
                v = w * (R)f[((long)z * N + y) * N + x];
            }
        } else {
            const double *F = (const double *)a.src;
            v = (R)F[((long)zi * a.nin + yi) * a.nin + m];
        }
        C c;
        c.x = v;
        c.y = R(0.0);
        buf[l * LS + m] = c;
    }
    __syncthreads();
    fft_dif<LOG2M>(buf, nl, LS, 1, s_tw, false);
    C *out = (C *)outp;
    if (SLAB) {  // layout [item][kx][zi][yi]: one contiguous nin x nin block per (item, kx)
        const long q = slab / a.nin;  // scratch slot: the item within this launch
        for (int e = threadIdx.x; e < nl * MH; e += blockDim.x) {
            const int kx = e / nl, l = e % nl;
            out[((q * MH + kx) * a.nin + zi) * a.nin + line0 + l] = buf[l * LS + brev_bits(kx, LOG2M)];
        }
    } else {     // layout [slab][line][kx]
        for (int e = threadIdx.x; e < nl * MH; e += blockDim.x) {
            const int l = e / MH, kx = e % MH;
            out[((long)slab * a.nin + line0 + l) * MH + kx] = buf[l * LS + brev_bits(kx, LOG2M)];
        }
    }
}

// ---------------------------------------------------------------------------
// Fused local-convolution slab: one CTA per (patch p, kx).  The (ky, kz) slab
// of the patch spectrum (M x M complex) stays in shared memory through the
// forward y and z transforms, the product with the kernel spectrum and the
// inverse z and y transforms.  In: [p][kx][zi][yi] (nin x nin); out:
// [p][zo][kx][yo] (nout x nout) from positions (out_off + t) mod M.
// Row y of the slab at S + y * (M + 1), column z contiguous.
// ---------------------------------------------------------------------------
struct SlabArgs {
    const void *tw;
    int nin, nout, out_off;
    Items it;  // per item: in = a1, out = a4, khat of its plan
    int nz;    // output z rows: zrow[j] in [0, nout), the rows the inverse-x step reads
    int zrow[128];
    int blk;   // complex entries per (patch, z row) output block (16-byte multiple)
};

template <int LOG2M, typename R>
__global__ void __launch_bounds__(256) k_slab(SlabArgs a) {
    using C = typename Cx<R>::T;
    constexpr int M = 1 << LOG2M, MH = M / 2 + 1, P = M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_tw = (C *)smem_raw;
    C *S = s_tw + M / 2;
    const int kx = blockIdx.x % MH;
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x / MH, p);
    const int nin = a.nin, W = a.nout;
    load_twiddles<LOG2M>(s_tw, (const C *)a.tw);
    for (int e = threadIdx.x; e < M * P; e += blockDim.x) S[e] = Cx<R>::mk(0, 0);
    __syncthreads();
    const long q = blockIdx.x / MH;  // scratch slot
    const C *in = (const C *)a.it.a1 + (q * MH + kx) * nin * nin;
    for (int e = threadIdx.x; e < nin * nin; e += blockDim.x) {
        const int zi = e / nin, yi = e % nin;
        S[yi * P + zi] = in[e];
    }
    __syncthreads();
    // forward y on the nin nonzero z columns (natural in, bit-reversed ky out)
    fft_dif<LOG2M>(S, nin, 1, P, s_tw, false);
    // forward z on all rows (bit-reversed kz out)
    fft_dif<LOG2M>(S, M, P, 1, s_tw, false);
    // x real-even kernel spectrum at (kx, ky, kz)
    const R *khat = (const R *)PP.khat;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
        const int r = e / M, c = e % M;
        const int ky0 = brev_bits(r, LOG2M), kz0 = brev_bits(c, LOG2M);
        const int ky = ky0 < M - ky0 ? ky0 : M - ky0;
        const int kz = kz0 < M - kz0 ? kz0 : M - kz0;
        const R k = khat[((long)kx * MH + ky) * MH + kz];
        C v = S[r * P + c];
        v.x *= k;
        v.y *= k;
        S[r * P + c] = v;
    }
    __syncthreads();
    // inverse z on all rows (bit-reversed in, natural z out)
    fft_dit<LOG2M>(S, M, P, 1, s_tw, true);
    // inverse y on the output z columns only: positions [0, hi] and [lo2, M)
    int pos0 = a.out_off % M;
    if (pos0 < 0) pos0 += M;
    // output positions (out_off + t) mod M, t < W: one wrapped range starting at pos0
    const int n1 = (pos0 + W <= M) ? W : M - pos0;  // columns pos0 .. pos0+n1-1, then 0 ..
    fft_dit<LOG2M>(S + pos0, W, 1, P, s_tw, true, n1, -(pos0 + n1));
    C *out = (C *)a.it.a4 + q * a.nz * a.blk;
    for (int e = threadIdx.x; e < a.nz * W; e += blockDim.x) {
        const int jz = e / W, yo = e % W, zo = a.zrow[jz];
        int pz = (a.out_off + zo) % M, py = (a.out_off + yo) % M;
        if (pz < 0) pz += M;
        if (py < 0) py += M;
        out[(long)jz * a.blk + kx * W + yo] = S[py * P + pz];
    }
}

// ---------------------------------------------------------------------------
// The same slab for 16-byte complex entries (FP64, double-float) at M = 128,
// whose M x M slab does not fit in shared memory: after the forward y
// transform of the nin input z columns, the ky rows go through the forward z
// transform, the kernel spectrum and the inverse z transform rb rows at a
// time in a row buffer, and each row keeps only the nz output z positions,
// written back over its own input; the inverse y transform then runs on those
// nz columns.  S: M rows of sw >= max(nin, nz) entries.  Same arithmetic per
// entry as k_slab (the z transforms of a row do not depend on the others).
// ---------------------------------------------------------------------------
template <int LOG2M, typename R>
__global__ void __launch_bounds__(256) k_slab_rows(SlabArgs a, int sw, int rb) {
    using C = typename Cx<R>::T;
    constexpr int M = 1 << LOG2M, MH = M / 2 + 1, P = M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_tw = (C *)smem_raw;
    C *S = s_tw + M / 2;
    C *B = S + M * sw;  // rb rows of P
    const int kx = blockIdx.x % MH;
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x / MH, p);
    const int nin = a.nin, W = a.nout, nz = a.nz;
    load_twiddles<LOG2M>(s_tw, (const C *)a.tw);
    for (int e = threadIdx.x; e < M * nin; e += blockDim.x) S[(e / nin) * sw + e % nin] = Cx<R>::mk(0, 0);
    __syncthreads();
    const long q = blockIdx.x / MH;  // scratch slot
    const C *in = (const C *)a.it.a1 + (q * MH + kx) * nin * nin;
    for (int e = threadIdx.x; e < nin * nin; e += blockDim.x) {
        const int zi = e / nin, yi = e % nin;
        S[yi * sw + zi] = in[e];
    }
    __syncthreads();
    // forward y on the nin z columns (natural in, bit-reversed ky rows out)
    fft_dif<LOG2M>(S, nin, 1, sw, s_tw, false);
    const R *khat = (const R *)PP.khat;
    int pos0 = a.out_off % M;
    if (pos0 < 0) pos0 += M;
    for (int r0 = 0; r0 < M; r0 += rb) {
        const int nr = min(rb, M - r0);
        for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
            const int l = e / M, c = e % M;
            B[l * P + c] = c < nin ? S[(r0 + l) * sw + c] : Cx<R>::mk(0, 0);
        }
        __syncthreads();
        fft_dif<LOG2M>(B, nr, P, 1, s_tw, false);  // forward z (bit-reversed kz)
        for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
            const int l = e / M, c = e % M;
            const int ky0 = brev_bits(r0 + l, LOG2M), kz0 = brev_bits(c, LOG2M);
            const int ky = ky0 < M - ky0 ? ky0 : M - ky0;
            const int kz = kz0 < M - kz0 ? kz0 : M - kz0;
            const R k = khat[((long)kx * MH + ky) * MH + kz];
            C v = B[l * P + c];
            v.x *= k;
            v.y *= k;
            B[l * P + c] = v;
        }
        __syncthreads();
        fft_dit<LOG2M>(B, nr, P, 1, s_tw, true);  // inverse z (natural z)
        for (int e = threadIdx.x; e < nr * nz; e += blockDim.x) {
            const int l = e / nz, jz = e % nz;
            const int pz = (pos0 + a.zrow[jz]) % M;
            S[(r0 + l) * sw + jz] = B[l * P + pz];
        }
        __syncthreads();
    }
    // inverse y on the nz output columns (bit-reversed ky in, natural y out)
    fft_dit<LOG2M>(S, nz, 1, sw, s_tw, true);
    C *out = (C *)a.it.a4 + q * a.nz * a.blk;
    for (int e = threadIdx.x; e < nz * W; e += blockDim.x) {
        const int jz = e / W, yo = e % W;
        const int py = (pos0 + yo) % M;
        out[(long)jz * a.blk + kx * W + yo] = S[py * sw + jz];
    }
}

// ---------------------------------------------------------------------------
// 64-point FFT of one line by 8 threads (radix 8 x 8, registers + one
// exchange through the line's own shared-memory storage).  n = 8 n2 + n1,
// k = k1 + 8 k2:  Y[n1][k1] = w64^(n1 k1) sum_n2 x[8 n2 + n1] w8^(n2 k1),
// X[k1 + 8 k2] = sum_n1 Y[n1][k1] w8^(n1 k2).  Input and output natural order.
// Every lane of the warp must call it (it uses __syncwarp); `valid` masks the
// memory accesses of lanes whose line does not exist.
// ---------------------------------------------------------------------------
template <typename C, typename R>
__device__ __forceinline__ C w8mul(C d, int j, bool inv) {
    const R s = (R)0.70710678118654752440;
    C r;
    switch (j) {
        case 0: r = d; break;
        case 1:
            if (!inv) { r.x = (d.x + d.y) * s; r.y = (d.y - d.x) * s; }
            else { r.x = (d.x - d.y) * s; r.y = (d.x + d.y) * s; }
            break;
        case 2: r = mul_mi(d, inv); break;
        default:
            if (!inv) { r.x = (d.y - d.x) * s; r.y = -(d.x + d.y) * s; }
            else { r.x = -(d.x + d.y) * s; r.y = (d.x - d.y) * s; }
            break;
    }
    return r;
}

// In-register 8-point DFT (natural order in and out).
template <typename C, typename R>
__device__ __forceinline__ void dft8(C (&v)[8], bool inv) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const C a = v[i], b = v[i + 4];
        v[i] = cadd(a, b);
        v[i + 4] = w8mul<C, R>(csub(a, b), i, inv);
    }
#pragma unroll
    for (int g = 0; g < 8; g += 4)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const C a = v[g + i], b = v[g + i + 2];
            v[g + i] = cadd(a, b);
            v[g + i + 2] = w8mul<C, R>(csub(a, b), 2 * i, inv);
        }
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
        const C a = v[i], b = v[i + 1];
        v[i] = cadd(a, b);
        v[i + 1] = csub(a, b);
    }
    // bit-reversed -> natural
    C t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[3]; v[3] = v[6]; v[6] = t;
}

// Exchange through `xs` (72 entries per 8-thread group, row pitch 9) when it
// is non-null, otherwise through the line's own storage.  With a line pitch of
// 4 (mod 16) complex FP32 entries, all four phases are free of bank conflicts.
template <typename C, typename R>
__device__ __forceinline__ void fft64_line(C *line, int estride, int t, bool valid, int nvalid,
                                           const C (&wt)[8], bool inv, C *xs) {
    C v[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) {
        const int pos = 8 * n2 + t;
        v[n2] = (valid && pos < nvalid) ? renorm(line[pos * estride]) : Cx<R>::mk(0, 0);
    }
    dft8<C, R>(v, inv);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) {
        C w = wt[k1];  // w64^(t k1), held in registers by the caller
        if (inv) w.y = -w.y;
        v[k1] = cmul(v[k1], w);
    }
    if (xs) {
        // no __syncwarp needed before: xs is private to the group and idle here
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) xs[9 * k1 + t] = v[k1];
        __syncwarp();
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) v[n1] = xs[9 * t + n1];
        __syncwarp();
    } else {
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1)
            if (valid) line[(8 * k1 + t) * estride] = v[k1];
        __syncwarp();
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) v[n1] = valid ? line[(8 * t + n1) * estride] : Cx<R>::mk(0, 0);
        __syncwarp();
    }
    dft8<C, R>(v, inv);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2)
        if (valid) line[(t + 8 * k2) * estride] = v[k2];
    __syncwarp();
}

// Apply fft64_line to nlines lines; line l at base + off(l) (lstride, plus
// `gap` for l >= gap_at).  xs: exchange scratch of blockDim/8 x 72 entries or
// nullptr.  Ends with __syncthreads.
template <typename C, typename R>
__device__ __forceinline__ void fft64_lines(C *base, int nlines, int lstride, int estride, int nvalid,
                                            const C *tw64, bool inv, C *xs, int gap_at = 1 << 30,
                                            int gap = 0) {
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7, ngrp = blockDim.x >> 3;
    C *gx = xs ? xs + grp * 72 : nullptr;
    C wt[8];  // this lane's twiddles w64^(t k1), k1 = 0..7
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) wt[k1] = tw64[(t * k1) & 63];
    for (int l0 = 0; l0 < nlines; l0 += ngrp) {  // uniform trip count across the CTA
        const int l = l0 + grp;
        const bool valid = l < nlines;
        C *line = base + (valid ? l * lstride + (l >= gap_at ? gap : 0) : 0);
        // every lane of a group takes the same exchange path (uniform __syncwarp
        // sites); an invalid group only writes zeros into its own scratch rows
        fft64_line<C, R>(line, estride, t, valid, nvalid, wt, inv, gx);
    }
    __syncthreads();
}

// Row pitch of the 64-point line buffers: 68 (4 mod 16) for FP32, 65 for FP64
// (both conflict-free for the line loads and stores).
template <typename R> struct Pitch64 { static constexpr int P = sizeof(R) == 4 ? 68 : 65; };
// Lines exchange through a separate padded buffer (FP32 and double-float
// complex entries); plain FP64 lines exchange in place.
template <typename R> struct UseXs { static constexpr bool v = !std::is_same<R, double>::value; };

// First radix-8 butterfly of a line whose inputs 3..7 are zero (the forward
// passes, whose n+1 <= 24 nonzero samples sit at positions 8 n2 + t, n2 < 3):
// the stage sums with a zero operand are left out (26 complex additions and
// one w8 product fewer than dft8).
template <typename C, typename R>
__device__ __forceinline__ void dft8_in3(C (&v)[8], bool inv) {
    const C v0 = v[0], v1 = v[1], v2 = v[2];
    const C u5 = w8mul<C, R>(v1, 1, inv), u6 = mul_mi(v2, inv);
    v[0] = cadd(v0, v2);
    v[2] = csub(v0, v2);
    v[1] = v1;
    v[3] = mul_mi(v1, inv);
    v[4] = cadd(v0, u6);
    v[6] = csub(v0, u6);
    v[5] = u5;
    v[7] = mul_mi(u5, inv);
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
        const C a = v[i], b = v[i + 1];
        v[i] = cadd(a, b);
        v[i + 1] = csub(a, b);
    }
    C t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[3]; v[3] = v[6]; v[6] = t;
}

// The register part of a 64-point line transform (radix 8 x 8, as fft64_line):
// lane t holds x[8 n2 + t] in v[n2] on entry and X[t + 8 k2] in v[k2] on exit,
// exchanging once through the group's padded scratch xs (row pitch 9).  The
// exit layout is the entry layout of the next transform of the same line, so
// a forward transform, a pointwise product and an inverse transform chain in
// registers.  SPARSE: v[3..7] are zero on entry.  Double-float inputs are
// renormalised first unless RENORM is false.
template <typename C, typename R, bool SPARSE, bool RENORM = true>
__device__ __forceinline__ void line64_regs(C (&v)[8], int t, const C (&wt)[8], bool inv, C *xs) {
    if (RENORM) {
#pragma unroll
        for (int n2 = 0; n2 < (SPARSE ? 3 : 8); ++n2) v[n2] = renorm(v[n2]);
    }
    if (SPARSE) dft8_in3<C, R>(v, inv);
    else dft8<C, R>(v, inv);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) {
        C w = wt[k1];
        if (inv) w.y = -w.y;
        v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) xs[9 * k1 + t] = v[k1];
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) v[n1] = xs[9 * t + n1];
    __syncwarp();
    dft8<C, R>(v, inv);
}

// Fused slab for M = 64 (same contract as k_slab), radix 8 x 8 over 8-thread
// line groups: the FP64 tier runs it with R = dfl (double-float arithmetic on
// FP64 data); the split tier uses k_slab64r instead.  The slab is S[z][y]
// (row pitch P).  Passes: forward y on the nin nonzero z rows; per y column,
// forward z, product with the real kernel spectrum and inverse z in registers
// (only the z rows the inverse-x step reads are stored back); inverse y on
// those rows only.  Requires nin <= 24.
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_slab64(SlabArgs a) {
    using C = typename Cx<R>::T;
    constexpr int M = 64, MH = 33, P = Pitch64<R>::P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw64 = (C *)smem_raw;  // 64 twiddles exp(-2 pi i j / 64)
    C *S = tw64 + M;
    C *xs = S + M * P;        // blockDim/8 x 72 exchange entries
    int *rowoff = (int *)(xs + 32 * 72);
    const int nin = a.nin, W = a.nout;
    const C *tw = (const C *)a.tw;  // M/2 entries; extend by w^(j+32) = -w^j
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        C w = tw[j & 31];
        if (j >= 32) { w.x = -w.x; w.y = -w.y; }
        tw64[j] = w;
    }
    // output z rows as slab rows (the field box starts at out_off, wrapped mod M)
    unsigned long long rowmask = 0;
    for (int j = 0; j < a.nz; ++j) {
        int pz = (a.out_off + a.zrow[j]) % M;
        if (pz < 0) pz += M;
        rowmask |= 1ull << pz;
        if (threadIdx.x == 0) rowoff[j] = pz * P;
    }
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7, ngrp = blockDim.x >> 3;
    C *gx = xs + grp * 72;
    // blockDim.x steps in (row, column) of the nin x nin input and nz x W output blocks
    const int d_in_z = blockDim.x / nin, d_in_y = blockDim.x - d_in_z * nin;
    const int d_out_z = blockDim.x / W, d_out_y = blockDim.x - d_out_z * W;
    __syncthreads();
    C wt[8];
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) wt[k1] = tw64[(t * k1) & 63];
    const C zero = Cx<R>::mk(0, 0);
    // one slab per CTA, or (persistent launch) a grid-stride loop over slabs
    const int nunits = a.it.nitems * MH;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
        const int kx = unit % MH;
        int p;
        const PlanPtrs &PP = item_plan(a.it, unit / MH, p);
        const long q = unit / MH;  // scratch slot
        const C *in = (const C *)a.it.a1 + (q * MH + kx) * nin * nin;
        // (zi, yi) of element e stepped incrementally (one division per thread)
        for (int e = threadIdx.x, zi = e / nin, yi = e - zi * nin; e < nin * nin; e += blockDim.x) {
            S[zi * P + yi] = in[e];
            yi += d_in_y;
            zi += d_in_z;
            if (yi >= nin) { yi -= nin; ++zi; }
        }
        __syncthreads();
        // forward y on the nin nonzero z rows
        for (int l0 = 0; l0 < nin; l0 += ngrp) {
            const int l = l0 + grp;
            const bool valid = l < nin;
            C *line = S + (valid ? l * P : 0);
            C v[8];
#pragma unroll
            for (int n2 = 0; n2 < 8; ++n2) {
                const int pos = 8 * n2 + t;
                v[n2] = (n2 < 3 && valid && pos < nin) ? line[pos] : zero;
            }
            line64_regs<C, R, true>(v, t, wt, false, gx);
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2)
                if (valid) line[t + 8 * k2] = v[k2];
        }
        __syncthreads();
        // per y column: forward z, kernel product, inverse z (64 columns)
        const R *khat = (const R *)PP.khat + (long)kx * MH * MH;
        for (int ky0 = grp; ky0 < M; ky0 += ngrp) {
            C *col = S + ky0;
            C v[8];
#pragma unroll
            for (int n2 = 0; n2 < 8; ++n2) {
                const int pos = 8 * n2 + t;
                v[n2] = (n2 < 3 && pos < nin) ? col[pos * P] : zero;
            }
            line64_regs<C, R, true>(v, t, wt, false, gx);
            const R *kk = khat + (ky0 < M - ky0 ? ky0 : M - ky0) * MH;
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) {
                const int kz0 = t + 8 * k2;
                const R k = kk[kz0 < M - kz0 ? kz0 : M - kz0];
                v[k2].x *= k;
                v[k2].y *= k;
            }
            // the kernel products are nearly normalised already (residual ~2^-24 |p|)
            line64_regs<C, R, false, false>(v, t, wt, true, gx);
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) {
                const int z = t + 8 * k2;
                if ((rowmask >> z) & 1ull) col[z * P] = v[k2];
            }
        }
        __syncthreads();
        // inverse y on the output z rows
        for (int l0 = 0; l0 < a.nz; l0 += ngrp) {
            const int l = l0 + grp;
            const bool valid = l < a.nz;
            C *line = S + (valid ? rowoff[l] : 0);
            C v[8];
#pragma unroll
            for (int n2 = 0; n2 < 8; ++n2) v[n2] = valid ? line[8 * n2 + t] : zero;
            line64_regs<C, R, false>(v, t, wt, true, gx);
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2)
                if (valid) line[t + 8 * k2] = v[k2];
        }
        __syncthreads();
        C *out = (C *)a.it.a4 + q * a.nz * a.blk + kx * W;
        for (int e = threadIdx.x, jz = e / W, yo = e - jz * W; jz < a.nz; e += blockDim.x) {
            out[(long)jz * a.blk + yo] = S[rowoff[jz] + ((a.out_off + yo) & (M - 1))];
            yo += d_out_y;
            jz += d_out_z;
            if (yo >= W) { yo -= W; ++jz; }
        }
        __syncthreads();  // S is rewritten by the next unit
    }
}



// ---------------------------------------------------------------------------
// Split tier slab with one 64-point line per thread: the whole transform of a
// line sits in 64 complex registers (radix 2, fully unrolled, twiddles as
// immediates), so a line pass costs one shared-memory load and one store per
// point and no exchange.  Twiddles w64^k = exp(-2 pi i k / 64), k < 32, FP32
// (cos and -sin of 2 pi k / 64 rounded to nearest); w^(k+32) = -w^k.
// ---------------------------------------------------------------------------
__device__ constexpr float kW64Re[32] = {
    1.000000000e+00f, 9.951847196e-01f, 9.807852507e-01f, 9.569403529e-01f,
    9.238795042e-01f, 8.819212914e-01f, 8.314695954e-01f, 7.730104327e-01f,
    7.071067691e-01f, 6.343932748e-01f, 5.555702448e-01f, 4.713967443e-01f,
    3.826834261e-01f, 2.902846634e-01f, 1.950903237e-01f, 9.801714122e-02f,
    6.123234263e-17f, -9.801714122e-02f, -1.950903237e-01f, -2.902846634e-01f,
    -3.826834261e-01f, -4.713967443e-01f, -5.555702448e-01f, -6.343932748e-01f,
    -7.071067691e-01f, -7.730104327e-01f, -8.314695954e-01f, -8.819212914e-01f,
    -9.238795042e-01f, -9.569403529e-01f, -9.807852507e-01f, -9.951847196e-01f,
};
__device__ constexpr float kW64Im[32] = {
    -0.000000000e+00f, -9.801714122e-02f, -1.950903237e-01f, -2.902846634e-01f,
    -3.826834261e-01f, -4.713967443e-01f, -5.555702448e-01f, -6.343932748e-01f,
    -7.071067691e-01f, -7.730104327e-01f, -8.314695954e-01f, -8.819212914e-01f,
    -9.238795042e-01f, -9.569403529e-01f, -9.807852507e-01f, -9.951847196e-01f,
    -1.000000000e+00f, -9.951847196e-01f, -9.807852507e-01f, -9.569403529e-01f,
    -9.238795042e-01f, -8.819212914e-01f, -8.314695954e-01f, -7.730104327e-01f,
    -7.071067691e-01f, -6.343932748e-01f, -5.555702448e-01f, -4.713967443e-01f,
    -3.826834261e-01f, -2.902846634e-01f, -1.950903237e-01f, -9.801714122e-02f,
};

// x * w64^k (conjugate twiddle for the inverse), k a compile-time constant
// after unrolling: k = 0 and 16 need no multiply, 8 and 24 two.
__device__ __forceinline__ float2 tw64_mul(float2 x, int k, bool inv) {
    if (k == 0) return x;
    if (k == 16) return inv ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    const float wr = kW64Re[k], wi = inv ? -kW64Im[k] : kW64Im[k];
    return make_float2(fmaf(x.x, wr, -x.y * wi), fmaf(x.x, wi, x.y * wr));
}

// One radix-2 stage of half size 2^ST over the 32 butterflies of a 64-point
// line held in registers (one loop of 32, unrolled; all indices constant).
template <int ST, bool INV, bool ZERO_HI, int NZ = 64>
__device__ __forceinline__ void dif_stage64(float2 (&v)[64]) {
    constexpr int hs = 1 << ST;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const int j = b & (hs - 1), i0 = ((b >> ST) << (ST + 1)) + j, i1 = i0 + hs, k = j << (5 - ST);
        // v[i1] is zero: the butterfly is a twiddle product.  Stage 5 with
        // ZERO_HI; stage 4 when the inputs at NZ..31 were zero as well (after
        // stage 5 entry i is zero iff i mod 32 >= NZ)
        if (ZERO_HI || (ST == 4 && NZ <= 32 && ((i1 & 31) >= NZ))) {
            v[i1] = tw64_mul(v[i0], k, INV);
        } else {
            const float2 x = v[i0], y = v[i1];
            v[i0] = make_float2(x.x + y.x, x.y + y.y);
            v[i1] = tw64_mul(make_float2(x.x - y.x, x.y - y.y), k, INV);
        }
    }
}
template <int ST, bool INV>
__device__ __forceinline__ void dit_stage64(float2 (&v)[64]) {
    constexpr int hs = 1 << ST;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const int j = b & (hs - 1), i0 = ((b >> ST) << (ST + 1)) + j, i1 = i0 + hs, k = j << (5 - ST);
        const float2 x = v[i0], y = tw64_mul(v[i1], k, INV);
        v[i0] = make_float2(x.x + y.x, x.y + y.y);
        v[i1] = make_float2(x.x - y.x, x.y - y.y);
    }
}

// Decimation in frequency, natural order in, bit-reversed out.  ZERO_HI: the
// inputs 32..63 are zero (the forward passes over n+1 <= 32 samples), so the
// first stage is a twiddle product only.
template <bool INV, bool ZERO_HI, int NZ = 64>
__device__ __forceinline__ void fft64_dif_reg(float2 (&v)[64]) {
    dif_stage64<5, INV, ZERO_HI>(v);
    dif_stage64<4, INV, false, ZERO_HI ? NZ : 64>(v);
    dif_stage64<3, INV, false>(v);
    dif_stage64<2, INV, false>(v);
    dif_stage64<1, INV, false>(v);
    dif_stage64<0, INV, false>(v);
}

// Decimation in time, bit-reversed order in, natural out.
template <bool INV>
__device__ __forceinline__ void fft64_dit_reg(float2 (&v)[64]) {
    dit_stage64<0, INV>(v);
    dit_stage64<1, INV>(v);
    dit_stage64<2, INV>(v);
    dit_stage64<3, INV>(v);
    dit_stage64<4, INV>(v);
    dit_stage64<5, INV>(v);
}

__host__ __device__ constexpr int brev6(int i) {
    return ((i & 1) << 5) | ((i & 2) << 3) | ((i & 4) << 1) | ((i & 8) >> 1) | ((i & 16) >> 3) | ((i & 32) >> 5);
}

// Same contract as k_slab64, for the split tier (FP32; 64 threads: one line each).  Passes:
// forward y on the nin nonzero z rows; per y column, forward z (bit-reversed
// result), product with the real kernel spectrum, inverse z back to natural
// order, all in registers, storing only the z rows read later; inverse y on
// those rows.  Requires nin <= NZ <= 32 (NZ: compile-time bound on the
// nonzero inputs of the forward passes; their first two stages are pruned).
template <int NZ>
__global__ void __launch_bounds__(64, 6) k_slab64r(SlabArgs a) {
    constexpr int M = 64, MH = 33, P = 65;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *S = (float2 *)smem_raw;  // S[z][y], pitch 65 (conflict-free rows and columns)
    __shared__ int rowoff[64];
    const int nin = a.nin, W = a.nout, c = threadIdx.x;
    unsigned long long rowmask = 0;
    for (int j = 0; j < a.nz; ++j) {
        int pz = (a.out_off + a.zrow[j]) % M;
        if (pz < 0) pz += M;
        rowmask |= 1ull << pz;
        if (threadIdx.x == 0) rowoff[j] = pz * P;
    }
    __syncthreads();
    const int nunits = a.it.nitems * MH;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
        const int kx = unit % MH;
        int p;
        const PlanPtrs &PP = item_plan(a.it, unit / MH, p);
        const long q = unit / MH;  // scratch slot
        const float2 *in = (const float2 *)a.it.a1 + (q * MH + kx) * nin * nin;
        float2 v[64];
        // forward y: thread c < nin takes z row c
        if (c < nin) {
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = (i < NZ && i < nin) ? in[c * nin + i] : make_float2(0.f, 0.f);
            fft64_dif_reg<false, true, NZ>(v);
#pragma unroll
            for (int i = 0; i < 64; ++i) S[c * P + brev6(i)] = v[i];
        }
        __syncthreads();
        // column ky0 = c: forward z, kernel product, inverse z
        {
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = (i < NZ && i < nin) ? S[i * P + c] : make_float2(0.f, 0.f);
            fft64_dif_reg<false, true, NZ>(v);
            const float *kk = (const float *)PP.khat + ((long)kx * MH + (c < M - c ? c : M - c)) * MH;
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                const int kz0 = brev6(i), kz = kz0 < M - kz0 ? kz0 : M - kz0;
                const float k = kk[kz];
                v[i].x *= k;
                v[i].y *= k;
            }
            fft64_dit_reg<true>(v);
#pragma unroll
            for (int i = 0; i < 64; ++i)
                if ((rowmask >> i) & 1ull) S[i * P + c] = v[i];
        }
        __syncthreads();
        // inverse y on the output z rows: thread c < nz takes row rowoff[c]
        if (c < a.nz) {
            float2 *row = S + rowoff[c];
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = row[brev6(i)];
            fft64_dit_reg<true>(v);
#pragma unroll
            for (int i = 0; i < 64; ++i) row[i] = v[i];
        }
        __syncthreads();
        float2 *out = (float2 *)a.it.a4 + q * a.nz * a.blk + kx * W;
        for (int e = threadIdx.x; e < a.nz * W; e += blockDim.x) {
            const int jz = e / W, yo = e - jz * W;
            out[(long)jz * a.blk + yo] = S[rowoff[jz] + ((a.out_off + yo) & (M - 1))];
        }
        __syncthreads();  // S is rewritten by the next unit
    }
}

// ---------------------------------------------------------------------------
// 128-point lines in FP32 by 8-lane groups, radix 16 x 8: with n = 8 n2 + n1
// and k = k1 + 16 k2, lane t = n1 forms Y[t][k1] = w128^(t k1) sum_n2
// x[8 n2 + t] w16^(n2 k1) in registers; after one exchange through the
// group's scratch, lane t takes k1 = t and t + 8 and forms X[k1 + 16 k2] =
// sum_n1 Y[n1][k1] w8^(n1 k2).  Lane t holds x[8 j + t] in v[j] on entry and
// X[8 j + t] in v[j] on exit (natural order both ways), so a forward
// transform, a pointwise product and an inverse transform chain in registers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 w16mul(float2 d, int j, bool inv) {
    // exp(-+ 2 pi i j / 16), j a compile-time constant after unrolling
    constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, c2 = 0.70710678118654752440f;
    const float cr[8] = {1.f, c1, c2, s1, 0.f, -s1, -c2, -c1};
    const float si[8] = {0.f, s1, c2, c1, 1.f, c1, c2, s1};
    if (j == 0) return d;
    const float wr = cr[j], wi = inv ? si[j] : -si[j];
    return make_float2(fmaf(d.x, wr, -d.y * wi), fmaf(d.x, wi, d.y * wr));
}

// 16-point DFT in registers, natural order in and out; SPARSE: v[8..15] zero.
template <bool SPARSE>
__device__ __forceinline__ void dft16(float2 (&v)[16], bool inv) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (SPARSE) {
            v[i + 8] = w16mul(v[i], i, inv);
        } else {
            const float2 a = v[i], b = v[i + 8];
            v[i] = make_float2(a.x + b.x, a.y + b.y);
            v[i + 8] = w16mul(make_float2(a.x - b.x, a.y - b.y), i, inv);
        }
    }
#pragma unroll
    for (int g = 0; g < 16; g += 8)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 a = v[g + i], b = v[g + i + 4];
            v[g + i] = make_float2(a.x + b.x, a.y + b.y);
            v[g + i + 4] = w16mul(make_float2(a.x - b.x, a.y - b.y), 2 * i, inv);
        }
#pragma unroll
    for (int g = 0; g < 16; g += 4)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float2 a = v[g + i], b = v[g + i + 2];
            v[g + i] = make_float2(a.x + b.x, a.y + b.y);
            v[g + i + 2] = w16mul(make_float2(a.x - b.x, a.y - b.y), 4 * i, inv);
        }
#pragma unroll
    for (int g = 0; g < 16; g += 2) {
        const float2 a = v[g], b = v[g + 1];
        v[g] = make_float2(a.x + b.x, a.y + b.y);
        v[g + 1] = make_float2(a.x - b.x, a.y - b.y);
    }
    // bit-reversed (4 bits) -> natural
    float2 t;
    t = v[1]; v[1] = v[8]; v[8] = t;
    t = v[2]; v[2] = v[4]; v[4] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[5]; v[5] = v[10]; v[10] = t;
    t = v[7]; v[7] = v[14]; v[14] = t;
    t = v[11]; v[11] = v[13]; v[13] = t;
}

// One 128-point line transform by an 8-lane group (layout above).  tw: M
// twiddles exp(-2 pi i j / 128) in shared memory, entry j at j + j / 8 (the
// padding spreads the lanes' reads of w^(t k1) over distinct banks); xs: the
// group's scratch (16 x 9 entries); gm: the group's lane mask.
template <bool SPARSE>
__device__ __forceinline__ void line128_regs(float2 (&v)[16], int t, const float2 *tw, bool inv, float2 *xs,
                                             unsigned gm) {
    dft16<SPARSE>(v, inv);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
        const int j = (t * k1) & 127;
        float2 w = tw[j + (j >> 3)];
        if (inv) w.y = -w.y;
        v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) xs[9 * k1 + t] = v[k1];
    __syncwarp(gm);
    float2 a[8], b[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
        a[n1] = xs[9 * t + n1];
        b[n1] = xs[9 * (t + 8) + n1];
    }
    __syncwarp(gm);
    dft8<float2, float>(a, inv);
    dft8<float2, float>(b, inv);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        v[2 * k2] = a[k2];
        v[2 * k2 + 1] = b[k2];
    }
}

// Split-tier slab for M = 128 (same contract as k_slab): 8-lane groups take
// one line each (forward y on the nin input z rows; per ky column forward z,
// kernel product and inverse z in registers, storing only the z positions
// read later, into compact rows in position order; inverse y on those rows);
// the slab holds max(nin, nz) rows.  Requires nin <= 64, W <= 128, 256
// threads.  Bank spreading: the two groups of a half-warp take rows or
// columns 8 apart (row pitch 129: 16 banks apart), and the groups' exchange
// scratch sits 152 entries apart (also 16 banks).
__global__ void __launch_bounds__(256, 2) k_slab128r(SlabArgs a) {
    constexpr int M = 128, MH = 65, P = 129, XP = 152;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tw = (float2 *)smem_raw;                 // M twiddles, padded (144 entries)
    float2 *xs_all = tw + 144;                       // 32 groups x XP
    float2 *S = xs_all + 32 * XP;                    // S[row][ky], pitch P
    __shared__ int rowc[128];                        // output z row jz -> compact row
    __shared__ unsigned long long mask_s[2];         // output z positions
    const int nin = a.nin, W = a.nout, nz = a.nz;
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7;
    // this group's first row / column: a bijection of 0..31 pairing the two
    // groups of each half-warp 8 apart
    const int g0 = ((grp >> 1) & 7) + 8 * (grp & 1) + 16 * (grp >> 4);
    const unsigned gm = 0xffu << (threadIdx.x & 24);
    float2 *xs = xs_all + grp * XP;
    const float2 *twg = (const float2 *)a.tw;        // M/2 entries; w^(j+64) = -w^j
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        float2 w = twg[j & 63];
        if (j >= 64) { w.x = -w.x; w.y = -w.y; }
        tw[j + (j >> 3)] = w;
    }
    if (threadIdx.x < 2) {
        unsigned long long m = 0;
        for (int j = 0; j < nz; ++j) {
            const int pz = (a.out_off + a.zrow[j]) & (M - 1);
            if ((pz >> 6) == (int)threadIdx.x) m |= 1ull << (pz & 63);
        }
        mask_s[threadIdx.x] = m;
    }
    __syncthreads();
    const unsigned long long m0 = mask_s[0], m1 = mask_s[1];
    const int c0 = __popcll(m0);
    // compact row of output position pos (position order)
    auto crow = [&](int pos) -> int {
        return pos < 64 ? __popcll(m0 & ((1ull << pos) - 1ull)) : c0 + __popcll(m1 & ((1ull << (pos - 64)) - 1ull));
    };
    for (int j = threadIdx.x; j < nz; j += blockDim.x) rowc[j] = crow((a.out_off + a.zrow[j]) & (M - 1));
    __syncthreads();
    const int nunits = a.it.nitems * MH;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
        const int kx = unit % MH;
        int p;
        const PlanPtrs &PP = item_plan(a.it, unit / MH, p);
        const long q = unit / MH;  // scratch slot
        const float2 *in = (const float2 *)a.it.a1 + (q * MH + kx) * nin * nin;
        float2 v[16];
        // forward y: one input z row per group (natural ky columns out)
        for (int r = g0; r < nin; r += 32) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int pos = 8 * j + t;
                v[j] = (j < 8 && pos < nin) ? in[r * nin + pos] : make_float2(0.f, 0.f);
            }
            line128_regs<true>(v, t, tw, false, xs, gm);
#pragma unroll
            for (int j = 0; j < 16; ++j) S[r * P + 8 * j + t] = v[j];
        }
        __syncthreads();
        // ky column c: forward z, kernel product, inverse z
        for (int c = g0; c < M; c += 32) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int pos = 8 * j + t;
                v[j] = (j < 8 && pos < nin) ? S[pos * P + c] : make_float2(0.f, 0.f);
            }
            line128_regs<true>(v, t, tw, false, xs, gm);
            const float *kk = (const float *)PP.khat + ((long)kx * MH + (c < M - c ? c : M - c)) * MH;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int kz0 = 8 * j + t, kz = kz0 < M - kz0 ? kz0 : M - kz0;
                const float k = kk[kz];
                v[j].x *= k;
                v[j].y *= k;
            }
            line128_regs<false>(v, t, tw, true, xs, gm);
            // the group's loads of column c are done (exchange above)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int pos = 8 * j + t;
                const bool need = pos < 64 ? ((m0 >> pos) & 1ull) : ((m1 >> (pos - 64)) & 1ull);
                if (need) S[crow(pos) * P + c] = v[j];
            }
        }
        __syncthreads();
        // inverse y on the output rows (compact row r)
        for (int r = g0; r < nz; r += 32) {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = S[r * P + 8 * j + t];
            line128_regs<false>(v, t, tw, true, xs, gm);
#pragma unroll
            for (int j = 0; j < 16; ++j) S[r * P + 8 * j + t] = v[j];
        }
        __syncthreads();
        float2 *out = (float2 *)a.it.a4 + q * nz * a.blk + kx * W;
        for (int e = threadIdx.x; e < nz * W; e += blockDim.x) {
            const int jz = e / W, yo = e - jz * W;
            out[(long)jz * a.blk + yo] = S[rowc[jz] * P + ((a.out_off + yo) & (M - 1))];
        }
        __syncthreads();  // S is rewritten by the next unit
    }
}

// Lane shuffles of complex values within the 8-thread line group.
__device__ __forceinline__ float2 shfl8(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src, 8), __shfl_sync(0xffffffffu, v.y, src, 8));
}
__device__ __forceinline__ double2 shfl8(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src, 8), __shfl_sync(0xffffffffu, v.y, src, 8));
}
__device__ __forceinline__ dcx shfl8(dcx v, int src) {
    dcx r;
    r.x = dfl(__shfl_sync(0xffffffffu, v.x.hi, src, 8), __shfl_sync(0xffffffffu, v.x.lo, src, 8));
    r.y = dfl(__shfl_sync(0xffffffffu, v.y.hi, src, 8), __shfl_sync(0xffffffffu, v.y.lo, src, 8));
    return r;
}

// Forward real transform along x of the patch charges for M = 64 (the first
// pass of the local convolution): one CTA per patch.  The chi-weighted
// closed-patch charge lines (zi, yi) go in pairs as the real and imaginary
// parts of one complex 64-point transform in an 8-thread group (radix 8 x 8 in
// registers, sparse first butterflies: the n+1 <= 24 nonzero samples), and
// the pair is split with X_a[k] = (Z[k] + conj Z[M-k]) / 2 and
// X_b[k] = (Z[k] - conj Z[M-k]) / 2i; the conjugate partners come from the
// group's lanes by shuffles.  Output A1 [p][kx][zi][yi], kx <= M/2.
template <typename TF, typename R>
__global__ void __launch_bounds__(256) k_fwd_x64(FwdXArgs a) {
    using C = typename Cx<R>::T;
    constexpr int M = 64, MH = 33;
    __shared__ C tw64[M];
    __shared__ C xs_all[32 * 72];
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7, ngrp = blockDim.x >> 3;
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x, p);
    const int n = a.n, nin = n + 1, N = PP.N, np = PP.np;
    const int i2 = p % np, i1 = (p / np) % np, i0 = p / (np * np);
    const TF *f = (const TF *)PP.f;
    C *out = (C *)a.it.a1 + (long)blockIdx.x * MH * nin * nin;  // scratch slot = item
    const C *tw = (const C *)a.tw;  // M/2 entries; extend by w^(j+32) = -w^j
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        C w = tw[j & 31];
        if (j >= 32) { w.x = -w.x; w.y = -w.y; }
        tw64[j] = w;
    }
    __syncthreads();
    C wt[8];
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) wt[k1] = tw64[(t * k1) & 63];
    C *gx = xs_all + grp * 72;
    const C zero = Cx<R>::mk(0, 0);
    const R half = R(0.5);
    const int nl = nin * nin, npair = (nl + 1) / 2;
    // chi-weighted charge of line l (= zi nin + yi) at x (nodes at index N are zero)
    auto charge = [&](int l, int x) -> R {
        const int zi = l / nin, yi = l - zi * nin;
        const int z = i0 * n + zi, y = i1 * n + yi, xg = i2 * n + x;
        if (z >= N || y >= N || xg >= N) return R(0.0);
        R w = R((zi == 0 || zi == n) ? 0.5 : 1.0);
        if (yi == 0 || yi == n) w = w * half;
        if (x == 0 || x == n) w = w * half;
        return w * R(f[((long)z * N + y) * N + xg]);
    };
    for (int q0 = 0; q0 < npair; q0 += ngrp) {  // uniform trip count across the CTA
        const int q = q0 + grp;
        const bool valid = q < npair;
        const int la = 2 * q, lb = 2 * q + 1;
        C v[8];
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            v[n2] = zero;
            const int x = 8 * n2 + t;
            if (n2 < 3 && valid && x < nin) {
                v[n2].x = charge(la, x);
                if (lb < nl) v[n2].y = charge(lb, x);
            }
        }
        line64_regs<C, R, true>(v, t, wt, false, gx);
        // v[k2] = Z[t + 8 k2]; Z[M - k] sits in lane (8 - t) & 7, register
        // 7 - k2 (t > 0) or (8 - k2) & 7 (t = 0)
        C w[8];
        const int src = (8 - t) & 7;
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) w[k2] = shfl8(v[k2], src);
        if (!valid) continue;
        const int zia = la / nin, yia = la - zia * nin, zib = lb / nin, yib = lb - zib * nin;
#pragma unroll
        for (int k2 = 0; k2 < 5; ++k2) {
            const int kx = t + 8 * k2;
            if (kx > M / 2) continue;
            const C Z = v[k2], Zp = (t == 0) ? w[(8 - k2) & 7] : w[7 - k2];
            C xa, xb;
            xa.x = (Z.x + Zp.x) * half;
            xa.y = (Z.y - Zp.y) * half;
            xb.x = (Z.y + Zp.y) * half;
            xb.y = (Zp.x - Z.x) * half;
            out[((long)kx * nin + zia) * nin + yia] = xa;
            if (lb < nl) out[((long)kx * nin + zib) * nin + yib] = xb;
        }
    }
}

// ---------------------------------------------------------------------------
// Inverse real transform along x of the local fields, pruned to the values
// the later steps read: the coarse lattice of the field box (for Delta^H, and
// the coarse points of the interpolation stencils) and the patch-face planes
// inside Omega_alpha (for phi^i - I^H(phi^i)).  One CTA per (patch, z row of
// the field box).  Rows that need an alpha range or the coarse x values get a
// full inverse FFT; rows that only need x on the face planes get direct sums
// over the half spectrum.
//   cl[p][k0][k1][k2]  = phi^i(4k), k in [-s/4, (n+s)/4]^3
//   fp[p][slot][u][v]  = phi^i on face plane slot (axis * npa + j, plane
//                        x_axis = pl0 + j n), (u, v) the other two coordinates
//                        in [-ga, n+ga], increasing axis order.
// ---------------------------------------------------------------------------
struct InvXPArgs {
    Items it;         // per item: in = a4 [p][zo][kx][yo], out = cl, fp of its plan
    const void *tw;   // M/2 twiddles exp(-2 pi i j / M)
    int n, s, W, ga, npa, pl0, wa, nc;
    int nz;           // z rows with outputs; zrow[j] = their index zo in [0, W)
    int zrow[128];
    int maxfft;       // most transformed rows of any z row (sizes the line buffer)
    int blk;          // complex entries per (patch, z row) input block (16-byte multiple)
    int wait_tries;   // limit of the bounded wait for the block's bulk copy
    int skip_copy;    // test hook: issue no bulk copy, so the bounded wait runs out
    int rb;           // k_inv_x_pruned: transformed rows per pass through the line buffer
    int outer;        // Q = 10 (R18): every alpha row is transformed, and the values one node
                      // off the alpha face planes go to fp2 as well
};

__device__ __forceinline__ bool in_alpha(int c, int n, int ga) { return c >= -ga && c <= n + ga; }
__device__ __forceinline__ bool on_plane(int c, int n, int ga, int pl0) {
    return in_alpha(c, n, ga) && ((c - pl0) % n) == 0;
}
// R18: slot 2 j + side of a coordinate one node off the alpha face plane
// pl0 + j n (side 0: c = plane - 1, side 1: c = plane + 1), or -1.  With 4 | n
// and 4 | ga every such c inside the alpha box has its plane inside it too.
__device__ __forceinline__ int off_slot(int c, int n, int ga, int pl0, int npa) {
    if (!in_alpha(c, n, ga)) return -1;
    int d = c + 1 - pl0;
    if (d >= 0 && d % n == 0 && d / n < npa) return 2 * (d / n);
    d = c - 1 - pl0;
    if (d >= 0 && d % n == 0 && d / n < npa) return 2 * (d / n) + 1;
    return -1;
}

template <int LOG2M, typename R, typename TO>
__global__ void __launch_bounds__(256) k_inv_x_pruned(InvXPArgs a) {
    using C = typename Cx<R>::T;
    constexpr int M = 1 << LOG2M, MH = M / 2 + 1;
    constexpr int LP = LOG2M == 6 ? Pitch64<R>::P : M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int rows[128];
    __shared__ int nfft_s;
    __shared__ unsigned wmask[4];
    const int W = a.W, n = a.n, s = a.s, ga = a.ga, pl0 = a.pl0, wa = a.wa, nc = a.nc;
    C *tw = (C *)smem_raw;        // M twiddles
    C *raw = tw + M;              // MH x W (block of a.blk entries, 16-byte aligned)
    C *buf = raw + a.blk;         // up to a.maxfft lines of LP
    C *xs = (LOG2M == 6 && UseXs<R>::v) ? buf + a.maxfft * LP : nullptr;
    const int jz = blockIdx.x % a.nz, zi = a.zrow[jz];
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x / a.nz, p);
    const int z = zi - s;
    const C *twg = (const C *)a.tw;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        C w = twg[j & (M / 2 - 1)];
        if (j >= M / 2) { w.x = -w.x; w.y = -w.y; }
        tw[j] = w;
    }
    const C *in = (const C *)a.it.a4 + ((long)(blockIdx.x / a.nz) * a.nz + jz) * a.blk;  // scratch slot = item
    // stage the contiguous block with one TMA bulk copy
    __shared__ unsigned long long bar;
    const unsigned bytes = (unsigned)(a.blk * sizeof(C));
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, bytes);
        if (!a.skip_copy) bulk_g2s(raw, in, bytes, &bar);
    }
    __syncthreads();
    const bool arrived = mbar_wait_bounded(&bar, 0, a.wait_tries);
    if (__syncthreads_or(!arrived)) {  // uniform decision for the whole CTA
        if (threadIdx.x == 0) {
            atomicExch(PP.err, 1);
            mbar_wait_bounded(&bar, 0, a.wait_tries);  // one more bounded wait for the copy in flight
        }
        return;
    }
    const bool zP = on_plane(z, n, ga, pl0), zA = in_alpha(z, n, ga), zC = (z & 3) == 0;
    // rows of this z that need a full transform, compacted with warp ballots (W <= 128)
    if (threadIdx.x < 128) {
        const int yi = threadIdx.x, y = yi - s;
        const bool yA = in_alpha(y, n, ga), yP = on_plane(y, n, ga, pl0), yC = (y & 3) == 0;
        // outer: the rows one node off a face plane too (their x values off the
        // face planes come from direct sums below, like the face-plane ones)
        const bool zQ = zP || (a.outer && off_slot(z, n, ga, pl0, a.npa) >= 0);
        const bool yQ = yP || (a.outer && off_slot(y, n, ga, pl0, a.npa) >= 0);
        const bool need = yi < W && ((zQ && yA) || (yQ && zA) || (zC && yC));
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if ((threadIdx.x & 31) == 0) wmask[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x < 128) {
        const int yi = threadIdx.x, w = yi >> 5, lane = yi & 31;
        const unsigned mine = wmask[w];
        if ((mine >> lane) & 1u) {
            int before = __popc(mine & ((1u << lane) - 1u));
            for (int q = 0; q < w; ++q) before += __popc(wmask[q]);
            rows[before] = yi;
        }
        if (yi == 0) nfft_s = __popc(wmask[0]) + __popc(wmask[1]) + __popc(wmask[2]) + __popc(wmask[3]);
    }
    __syncthreads();
    const int nfft = nfft_s;
    TO *cl = (TO *)PP.cl + (long)p * nc * nc * nc;
    TO *fp = (TO *)PP.fp + (long)p * 3 * a.npa * wa * wa;
    const int kl = -s / 4;
    // the transformed rows, a.rb at a time through the line buffer
    for (int l0 = 0; l0 < nfft; l0 += a.rb) {
    const int nl = min(a.rb, nfft - l0);
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = e / M, k = e % M, yi = rows[l0 + l];
        C v;
        if (k < MH) {
            v = raw[k * W + yi];
        } else {
            v = raw[(M - k) * W + yi];
            v.y = -v.y;
        }
        buf[l * LP + k] = v;
    }
    __syncthreads();
    if (LOG2M == 6) fft64_lines<C, R>(buf, nl, LP, 1, M, tw, true, xs);
    else fft_dif<LOG2M>(buf, nl, LP, 1, tw, true);
    // outputs of the transformed rows
    for (int e = threadIdx.x; e < nl * W; e += blockDim.x) {
        const int l = e / W, xi = e % W, yi = rows[l0 + l];
        const int x = xi - s, y = yi - s;
        const bool yA = in_alpha(y, n, ga), yP = on_plane(y, n, ga, pl0), yC = (y & 3) == 0;
        const bool xA = in_alpha(x, n, ga), xP = on_plane(x, n, ga, pl0), xC = (x & 3) == 0;
        const bool wC = zC && yC && xC, w0 = zP && yA && xA, w1 = yP && zA && xA, w2 = zA && yA && xP;
        int o0 = -1, o1 = -1, o2 = -1;
        if (a.outer && xA && yA && zA) {
            o0 = off_slot(z, n, ga, pl0, a.npa);
            o1 = off_slot(y, n, ga, pl0, a.npa);
            o2 = off_slot(x, n, ga, pl0, a.npa);
        }
        if (!(wC || w0 || w1 || w2 || o0 >= 0 || o1 >= 0 || o2 >= 0)) continue;
        int pos = x % M;
        if (pos < 0) pos += M;
        const TO v = (TO)buf[l * LP + (LOG2M == 6 ? pos : brev_bits(pos, LOG2M))].x;
        const long ncl = (long)nc * nc * nc, nfp = 3L * a.npa * wa * wa;
        if (wC) {
            const long i = ((long)((z >> 2) - kl) * nc + ((y >> 2) - kl)) * nc + ((x >> 2) - kl);
            if (in_range(i, ncl, PP.err)) cl[i] = v;
        }
        if (w0) {
            const long i = (((long)(0 * a.npa + (z - pl0) / n)) * wa + (y + ga)) * wa + (x + ga);
            if (in_range(i, nfp, PP.err)) fp[i] = v;
        }
        if (w1) {
            const long i = (((long)(1 * a.npa + (y - pl0) / n)) * wa + (z + ga)) * wa + (x + ga);
            if (in_range(i, nfp, PP.err)) fp[i] = v;
        }
        if (w2) {
            const long i = (((long)(2 * a.npa + (x - pl0) / n)) * wa + (z + ga)) * wa + (y + ga);
            if (in_range(i, nfp, PP.err)) fp[i] = v;
        }
        if (a.outer) {  // [patch][axis][j][side][u][v], in-plane (u, v) as for fp
            TO *f2 = (TO *)PP.fp2 + (long)p * 6 * a.npa * wa * wa;
            const long nf2 = 6L * a.npa * wa * wa;
            if (o0 >= 0) {
                const long i = ((long)(0 * 2 * a.npa + o0) * wa + (y + ga)) * wa + (x + ga);
                if (in_range(i, nf2, PP.err)) f2[i] = v;
            }
            if (o1 >= 0) {
                const long i = ((long)(1 * 2 * a.npa + o1) * wa + (z + ga)) * wa + (x + ga);
                if (in_range(i, nf2, PP.err)) f2[i] = v;
            }
            if (o2 >= 0) {
                const long i = ((long)(2 * 2 * a.npa + o2) * wa + (z + ga)) * wa + (y + ga);
                if (in_range(i, nf2, PP.err)) f2[i] = v;
            }
        }
    }
    __syncthreads();  // the buffer is refilled by the next pass
    }
    // rows that only need x on the face planes (outer: and one node off them):
    // direct sums over the half spectrum
    const bool zO = a.outer && off_slot(z, n, ga, pl0, a.npa) >= 0;
    const int nxs = a.outer ? 3 : 1;  // x = plane, plane - 1, plane + 1
    if (zA) {
        for (int e = threadIdx.x; e < W * a.npa * nxs; e += blockDim.x) {
            const int yi = e / (a.npa * nxs), j = (e / nxs) % a.npa, sub = e % nxs;
            const int y = yi - s;
            const bool yA = in_alpha(y, n, ga), yP = on_plane(y, n, ga, pl0), yC = (y & 3) == 0;
            const bool yO = a.outer && off_slot(y, n, ga, pl0, a.npa) >= 0;
            if (!yA || zP || yP || zO || yO || (zC && yC)) continue;  // not needed, or done by an FFT row
            const int x = pl0 + j * n + (sub == 1 ? -1 : (sub == 2 ? 1 : 0));
            if (sub && !in_alpha(x, n, ga)) continue;
            int pos = x % M;
            if (pos < 0) pos += M;
            R acc = R(0.0);
            for (int k = 0; k < MH; ++k) {
                const C X = raw[k * W + yi];
                C w = tw[(k * pos) & (M - 1)];  // exp(+2 pi i k pos / M) = conj(tw)
                const R re = X.x * w.x + X.y * w.y;
                acc += (k == 0 || 2 * k == M) ? re : R(2.0) * re;
            }
            if (sub == 0) {
                const long i = (((long)(2 * a.npa + j)) * wa + (z + ga)) * wa + (y + ga);
                if (in_range(i, 3L * a.npa * wa * wa, PP.err)) fp[i] = (TO)acc;
            } else {  // off-plane slot 2 j + side of axis 2
                TO *f2 = (TO *)PP.fp2 + (long)p * 6 * a.npa * wa * wa;
                const long i = ((long)(2 * 2 * a.npa + 2 * j + (sub == 2 ? 1 : 0)) * wa + (z + ga)) * wa + (y + ga);
                if (in_range(i, 6L * a.npa * wa * wa, PP.err)) f2[i] = (TO)acc;
            }
        }
    }
}

// Pruned inverse real transform along x for M = 64 (same contract as
// k_inv_x_pruned; local fields leave in the working precision R).  The needed
// rows go in pairs: with A, B the Hermitian half spectra of two rows,
// Z = A + iB transforms to a + ib, so one complex 64-point register transform
// (radix 8 x 8, 8-thread group) yields both real rows; the Hermitian expansion
// happens in the loads.  The per-x output classification comes from a
// 64-entry table built once per CTA.
template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 8 : 4) k_inv_x64(InvXPArgs a) {
    using C = typename Cx<R>::T;
    constexpr int M = 64, MH = 33;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int rows[64], rinfo[64];  // needed rows; their class bits (1 alpha, 2 plane, 4 coarse) | slot << 3
    __shared__ int nfft_s;
    __shared__ unsigned wmask[2];
    __shared__ int xflag[M], xplane[M], xcoarse[M];  // per x position: class bits, face-plane slot, coarse index
    const int W = a.W, n = a.n, s = a.s, ga = a.ga, pl0 = a.pl0, wa = a.wa, nc = a.nc;
    C *tw = (C *)smem_raw;        // M twiddles
    C *raw = tw + M;              // MH x W (block of a.blk entries, 16-byte aligned)
    C *xs = raw + a.blk;          // blockDim/8 groups x 72 exchange entries
    constexpr int RP = 68;           // row pitch of rbuf: 4 (mod 16) keeps the group stores conflict-free
    R *rbuf = (R *)(xs + (blockDim.x >> 3) * 72);  // transformed real rows (up to maxfft rows)
    const int jz = blockIdx.x % a.nz, zi = a.zrow[jz];
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x / a.nz, p);
    const int z = zi - s;
    const C *twg = (const C *)a.tw;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        C w = twg[j & (M / 2 - 1)];
        if (j >= M / 2) { w.x = -w.x; w.y = -w.y; }
        tw[j] = w;
    }
    const C *in = (const C *)a.it.a4 + ((long)(blockIdx.x / a.nz) * a.nz + jz) * a.blk;  // scratch slot = item
    // stage the contiguous block with one TMA bulk copy
    __shared__ unsigned long long bar;
    const unsigned bytes = (unsigned)(a.blk * sizeof(C));
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, bytes);
        if (!a.skip_copy) bulk_g2s(raw, in, bytes, &bar);
    }
    const int kl = -s / 4;
    // x classification: bit 0 in the field box, 1 in alpha, 2 on a face plane, 3 coarse
    if (threadIdx.x < M) {
        const int pos = threadIdx.x;
        const int x = pos <= n + s ? pos : pos - M;
        const bool box = x >= -s && x <= n + s;
        const bool xA = in_alpha(x, n, ga), xP = on_plane(x, n, ga, pl0), xC = (x & 3) == 0;
        xflag[pos] = box ? (1 | (xA ? 2 : 0) | (xP ? 4 : 0) | (xC ? 8 : 0)) : 0;
        xplane[pos] = xP ? (x - pl0) / n : 0;
        xcoarse[pos] = (x >> 2) - kl;
    }
    __syncthreads();
    const bool arrived = mbar_wait_bounded(&bar, 0, a.wait_tries);
    if (__syncthreads_or(!arrived)) {  // uniform decision for the whole CTA
        if (threadIdx.x == 0) {
            atomicExch(PP.err, 1);
            mbar_wait_bounded(&bar, 0, a.wait_tries);  // one more bounded wait for the copy in flight
        }
        return;
    }
    const bool zP = on_plane(z, n, ga, pl0), zA = in_alpha(z, n, ga), zC = (z & 3) == 0;
    // rows of this z that need a full transform, compacted with warp ballots (W <= 64)
    if (threadIdx.x < 64) {
        const int yi = threadIdx.x, y = yi - s;
        const bool yA = in_alpha(y, n, ga), yP = on_plane(y, n, ga, pl0), yC = (y & 3) == 0;
        // outer: the rows one node off a face plane too (their x values off the
        // face planes come from direct sums below, like the face-plane ones)
        const bool zQ = zP || (a.outer && off_slot(z, n, ga, pl0, a.npa) >= 0);
        const bool yQ = yP || (a.outer && off_slot(y, n, ga, pl0, a.npa) >= 0);
        const bool need = yi < W && ((zQ && yA) || (yQ && zA) || (zC && yC));
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if ((threadIdx.x & 31) == 0) wmask[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        const int yi = threadIdx.x;
        const unsigned m0 = wmask[0], m1 = wmask[1];
        const unsigned mine = yi < 32 ? m0 : m1;
        const int lane = yi & 31;
        if ((mine >> lane) & 1u) {
            const int before = (yi < 32 ? 0 : __popc(m0)) + __popc(mine & ((1u << lane) - 1u));
            const int y = yi - s;
            const bool yA = in_alpha(y, n, ga), yP = on_plane(y, n, ga, pl0), yC = (y & 3) == 0;
            rows[before] = yi;
            rinfo[before] = (yA ? 1 : 0) | (yP ? 2 : 0) | (yC ? 4 : 0) | ((yP ? (y - pl0) / n : 0) << 3);
        }
        if (yi == 0) nfft_s = __popc(m0) + __popc(m1);
    }
    __syncthreads();
    const int nfft = nfft_s, npair = (nfft + 1) / 2;
    R *cl = (R *)PP.cl + (long)p * nc * nc * nc;
    R *fp = (R *)PP.fp + (long)p * 3 * a.npa * wa * wa;
    const int zc = (z >> 2) - kl, jz0 = zP ? (z - pl0) / n : 0;
    const int grp = threadIdx.x >> 3, t = threadIdx.x & 7, ngrp = blockDim.x >> 3;
    C *gx = xs + grp * 72;
    C wt[8];
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) wt[k1] = tw[(t * k1) & 63];
    const C zero = Cx<R>::mk(0, 0);
    for (int q0 = 0; q0 < npair; q0 += ngrp) {  // uniform trip count across the CTA
        const int q = q0 + grp;
        const bool valid = q < npair;
        const int ya = valid ? rows[2 * q] : 0;
        const bool hasb = valid && 2 * q + 1 < nfft;
        const int yb = hasb ? rows[2 * q + 1] : 0;
        C v[8];
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            const int k = 8 * n2 + t;
            C A = zero, B = zero;
            if (valid) {
                if (k < MH) {
                    A = raw[k * W + ya];
                    if (hasb) B = raw[k * W + yb];
                } else {
                    A = raw[(M - k) * W + ya];
                    A.y = -A.y;
                    if (hasb) { B = raw[(M - k) * W + yb]; B.y = -B.y; }
                }
            }
            v[n2].x = A.x - B.y;  // Z = A + i B
            v[n2].y = A.y + B.x;
        }
        line64_regs<C, R, false>(v, t, wt, true, gx);
        if (valid) {
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) {
                rbuf[(2 * q) * RP + t + 8 * k2] = v[k2].x;
                if (hasb) rbuf[(2 * q + 1) * RP + t + 8 * k2] = v[k2].y;
            }
        }
    }
    __syncthreads();
    // outputs of the transformed rows (consecutive x per thread: coalesced stores)
    const int dl = blockDim.x / W, dxi = blockDim.x - dl * W;
    for (int e = threadIdx.x, l = e / W, xi = e - l * W; l < nfft; xi += dxi, l += dl) {
        if (xi >= W) { xi -= W; ++l; if (l >= nfft) break; }
        const int yi = rows[l], yf = rinfo[l];
        const int x = xi - s, y = yi - s;
        const int pos = x & (M - 1), xf = xflag[pos];
        const bool yA = yf & 1, yP = yf & 2, yC = yf & 4;
        const bool xA = xf & 2, xP = xf & 4, xC = xf & 8;
        const bool wC = zC && yC && xC, w0 = zP && yA && xA, w1 = yP && zA && xA, w2 = zA && yA && xP;
        int o0 = -1, o1 = -1, o2 = -1;
        if (a.outer && xA && yA && zA) {
            o0 = off_slot(z, n, ga, pl0, a.npa);
            o1 = off_slot(y, n, ga, pl0, a.npa);
            o2 = off_slot(x, n, ga, pl0, a.npa);
        }
        if (!(wC || w0 || w1 || w2 || o0 >= 0 || o1 >= 0 || o2 >= 0)) continue;
        const R val = rbuf[l * RP + pos];
        const long ncl = (long)nc * nc * nc, nfp = 3L * a.npa * wa * wa;
        if (wC) {
            const long i = ((long)zc * nc + ((y >> 2) - kl)) * nc + xcoarse[pos];
            if (in_range(i, ncl, PP.err)) cl[i] = val;
        }
        if (w0) {
            const long i = (((long)jz0) * wa + (y + ga)) * wa + (x + ga);
            if (in_range(i, nfp, PP.err)) fp[i] = val;
        }
        if (w1) {
            const long i = (((long)(a.npa + (yf >> 3))) * wa + (z + ga)) * wa + (x + ga);
            if (in_range(i, nfp, PP.err)) fp[i] = val;
        }
        if (w2) {
            const long i = (((long)(2 * a.npa + xplane[pos])) * wa + (z + ga)) * wa + (y + ga);
            if (in_range(i, nfp, PP.err)) fp[i] = val;
        }
    }
    // rows that only need x on the face planes: direct sums over the half spectrum
    if (zA) {
        for (int e = threadIdx.x; e < W * a.npa; e += blockDim.x) {
            const int yi = e / a.npa, j = e % a.npa;
            const int y = yi - s;
            const bool yA = in_alpha(y, n, ga), yP = on_plane(y, n, ga, pl0), yC = (y & 3) == 0;
            if (!yA || zP || yP || (zC && yC)) continue;  // not needed, or done by an FFT row
            const int x = pl0 + j * n;
            const int pos = x & (M - 1);
            R acc = R(0.0);
            for (int k = 0; k < MH; ++k) {
                const C X = raw[k * W + yi];
                C w = tw[(k * pos) & (M - 1)];  // exp(+2 pi i k pos / M) = conj(tw)
                const R re = X.x * w.x + X.y * w.y;
                acc += (k == 0 || 2 * k == M) ? re : R(2.0) * re;
            }
            fp[(((long)(2 * a.npa + j)) * wa + (z + ga)) * wa + (y + ga)] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Legendre coefficients c_p^i = sum_m W[m] Q^p(m) f[n i + m] (Boole, R3).
// ---------------------------------------------------------------------------
// Legendre coefficients c_p^i by composite Boole's rule, using the product
// structure of the weights and the basis: with a_k(m) = w_m q_k(2m/n - 1)
// (Boole weight times orthonormal Legendre polynomial, one axis),
//   c_p = R^{-3/2} sum_m0 a_p0(m0) sum_m1 a_p1(m1) sum_m2 a_p2(m2) f(m0,m1,m2),
// evaluated as three 1D contractions.  RM: arithmetic precision (FP64 or FP32
// for the split tier, whose last stage and output are FP64).  The charge is
// staged ns planes m0 at a time (all of them for small patches).
template <typename TF, typename RM>
__global__ void __launch_bounds__(256) k_moments(Items it, int n, int P, int npoly, int npad, int ns) {
    extern __shared__ double msm[];
    int pch;
    const PlanPtrs &PP = item_plan(it, blockIdx.x, pch);
    const int nb = n + 1, N = PP.N, np = PP.np;
    const int i2 = pch % np, i1 = (pch / np) % np, i0 = pch / (np * np);
    RM *F = (RM *)msm;                 // ns planes m0 of the closed patch's charge
    RM *T1 = F + ns * nb * nb;         // [p2][m0][m1]
    RM *T2 = T1 + P * nb * nb;         // [p1][p2][m0]
    RM *A = T2 + P * P * nb;           // [k][m] 1D weights
    const double *a1d = (const double *)PP.momw;
    for (int e = threadIdx.x; e < P * nb; e += blockDim.x) A[e] = (RM)a1d[e];
    const TF *f = (const TF *)PP.f;
    for (int s0 = 0; s0 < nb; s0 += ns) {
        const int sn = min(ns, nb - s0);
        for (int e = threadIdx.x; e < sn * nb * nb; e += blockDim.x) {
            const int m2 = e % nb, m1 = (e / nb) % nb, m0 = s0 + e / (nb * nb);
            const int z = i0 * n + m0, y = i1 * n + m1, x = i2 * n + m2;
            F[e] = (z < N && y < N && x < N) ? (RM)f[((long)z * N + y) * N + x] : (RM)0;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < P * sn * nb; e += blockDim.x) {
            const int p2 = e / (sn * nb), r = e % (sn * nb);  // r = (m0 - s0) nb + m1
            RM acc = 0;
            for (int m2 = 0; m2 < nb; ++m2) acc = fma(A[p2 * nb + m2], F[r * nb + m2], acc);
            T1[(p2 * nb + s0) * nb + r] = acc;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < P * P * nb; e += blockDim.x) {
        const int p1 = e / (P * nb), p2 = (e / nb) % P, m0 = e % nb;
        if (p1 + p2 >= P) continue;
        RM acc = 0;
        for (int m1 = 0; m1 < nb; ++m1) acc = fma(A[p1 * nb + m1], T1[(p2 * nb + m0) * nb + m1], acc);
        T2[e] = acc;
    }
    __syncthreads();
    if (threadIdx.x < npoly) {
        // index -> (p0, p1, p2) in lexicographic order, |p|_1 < P, p2 fastest
        int q = threadIdx.x, p0 = 0, p1 = 0, p2 = 0;
        for (int a0 = 0, k = 0; a0 < P; ++a0)
            for (int a1 = 0; a1 < P; ++a1)
                for (int a2 = 0; a2 < P; ++a2)
                    if (a0 + a1 + a2 < P) {
                        if (k == q) { p0 = a0; p1 = a1; p2 = a2; }
                        ++k;
                    }
        double acc = 0.0;
        for (int m0 = 0; m0 < nb; ++m0)
            acc = fma((double)A[p0 * nb + m0], (double)T2[(p1 * P + p2) * nb + m0], acc);
        acc *= PP.mom_scale;
        PP.mom[(long)pch * npad + q] = acc;
        if (PP.mom_f) PP.mom_f[(long)pch * npad + q] = (float)acc;
        if (PP.mom_df) {
            const float hi = (float)acc;
            PP.mom_df[(long)pch * npad + q] = make_float2(hi, (float)(acc - (double)hi));
        }
    }
}

// Weight table entry in the fine precision T: double-float pairs or FP64.
template <typename T> __device__ __forceinline__ T pick(const dfl &a, const double &b);
template <> __device__ __forceinline__ dfl pick<dfl>(const dfl &a, const double &) { return a; }
template <> __device__ __forceinline__ double pick<double>(const dfl &, const double &b) { return b; }

// r^i = phi^i - I^H(phi^i) on the face planes of patch i inside Omega_alpha.
// One CTA per (patch, plane); the in-plane interpolant is applied separably:
// first along v on the coarse rows u = 4k, then along u.
// resid[p][slot][u + ga][v + ga], slot = axis * npa + j for the plane
// x_axis = pl0 + j n (relative), (u, v) the other two coordinates.
struct ResArgs {
    Items it;  // per item: cl, fp -> resid of its plan
    int n, s, ga, b, npa, pl0, wa, nc;
    dfl lw[4][12];     // Lagrange weights for g mod 4 = r (row r), double-float
    double lwd[4][12]; // the same in FP64
};

// r^i = phi^i - I^H(phi^i) on the face planes inside Omega_alpha (one CTA per
// patch and plane).  TB: storage of the local fields (FP32, double-float or
// FP64 by tier); T: arithmetic of the interpolation and the difference, where
// cancellation needs the extra bits (FP64 or double-float).  The residual
// leaves in T.
template <typename TB, typename T, int K>
__global__ void __launch_bounds__(256) k_resid(ResArgs a) {
    extern __shared__ double rsm[];
    const int slot = blockIdx.y;
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x, p);
    const int axis = slot / a.npa, c4 = (a.pl0 + (slot % a.npa) * a.n) / 4;
    const int wa = a.wa, nc = a.nc, kl = -a.s / 4;  // K = 2b + 2 stencil points
    const int klo = -a.ga / 4 - a.b;  // coarse rows the stencils reach (4 | ga, 4 | n)
    const int khi = (a.n + a.ga) / 4 + a.b;
    const int nk = khi - klo + 1;
    T *Tv = (T *)rsm;                 // nk x wa: interpolated along v on coarse rows u = 4k
    T *Cv = Tv + nk * wa;             // nk x nk: phi^i at the plane's coarse points (u, v) = 4 (ka, kb)
    const TB *cl = (const TB *)PP.cl + (long)p * nc * nc * nc;
    const TB *fp = (const TB *)PP.fp + ((long)p * gridDim.y + slot) * wa * wa;
    // phi^i at the coarse point (u, v) = (4 ka, 4 kb) of this plane
    auto clp = [&](int ka, int kb) -> T {
        int i0, i1, i2;
        if (axis == 0) { i0 = c4; i1 = ka; i2 = kb; }
        else if (axis == 1) { i0 = ka; i1 = c4; i2 = kb; }
        else { i0 = ka; i1 = kb; i2 = c4; }
        if (!(in_range(i0 - kl, nc, PP.err) & in_range(i1 - kl, nc, PP.err) & in_range(i2 - kl, nc, PP.err)))
            return FT<T>::zero();
        return FT<T>::of(cl[((long)(i0 - kl) * nc + (i1 - kl)) * nc + (i2 - kl)]);
    };
    // the plane's coarse values, loaded once (independent loads, one per thread)
    for (int e = threadIdx.x; e < nk * nk; e += blockDim.x) Cv[e] = clp(klo + e / nk, klo + e % nk);
    __syncthreads();
    for (int e = threadIdx.x; e < nk * wa; e += blockDim.x) {
        const int kr = e / wa, v = e % wa - a.ga;
        const int rv = v & 3;
        const T *crow = Cv + kr * nk - klo;
        T t;
        if (rv == 0) {
            t = crow[v >> 2];
        } else {
            const int k0 = (v >> 2) - a.b;
            t = FT<T>::zero();
#pragma unroll
            for (int j = 0; j < K; ++j) t = FT<T>::fma(pick<T>(a.lw[rv][j], a.lwd[rv][j]), crow[k0 + j], t);
        }
        Tv[e] = t;
    }
    __syncthreads();
    T *out = (T *)PP.resid + ((long)p * gridDim.y + slot) * wa * wa;
    for (int e = threadIdx.x; e < wa * wa; e += blockDim.x) {
        const int u = e / wa - a.ga, v = e % wa - a.ga;
        const int ru = u & 3;
        T iv;
        if (ru == 0) {
            iv = Tv[((u >> 2) - klo) * wa + (v + a.ga)];
        } else {
            const int k0 = (u >> 2) - a.b;
            iv = FT<T>::zero();
#pragma unroll
            for (int j = 0; j < K; ++j)
                iv = FT<T>::fma(pick<T>(a.lw[ru][j], a.lwd[ru][j]), FT<T>::rn(Tv[(k0 + j - klo) * wa + (v + a.ga)]), iv);
        }
        out[e] = FT<T>::rn(FT<T>::of(fp[e]) - iv);
    }
}

// One step of a compensated dot product of double-float operands: the product
// of the high parts is split exactly (FMA residual) and added to the running
// sum s by two-sum; the rounding errors and the low-part cross terms gather in
// the FP32 compensation e (the Dot2 scheme of Ogita, Rump and Oishi, SIAM J.
// Sci. Comput. 26, 2005, with double-float inputs).  Error about n u^2 sum|x y|
// for u = 2^-24, against n u_64 sum|x y| in FP64 with u_64 = 2^-53.
__device__ __forceinline__ void dot2_step(float &s, float &e, float xh, float xl, float yh, float yl) {
    const float p = xh * yh;
    float pe = fmaf(xh, yh, -p);
    pe = fmaf(xh, yl, pe);
    pe = fmaf(xl, yh, pe);
    const float t = s + p, bb = t - s;
    e += ((s - (t - bb)) + (p - bb)) + pe;
    s = t;
}

// Ring term of one patch: dot product of two rows of n ring-table entries,
// returned in the fine precision T.  FP32 / FP64 rows accumulate in their own
// precision; double-float rows take the compensated product.
template <typename T, typename RT> __device__ __forceinline__ T ring_row(const RT *c, const RT *t, int n) {
    RT v = 0;
    for (int q = 0; q < n; ++q) v = fma(c[q], t[q], v);
    return FT<T>::of(v);
}
template <typename T> __device__ __forceinline__ T ring_row(const dfl *c, const dfl *t, int n) {
    float s = 0.f, e = 0.f;
    for (int q = 0; q < n; ++q) dot2_step(s, e, c[q].hi, c[q].lo, t[q].hi, t[q].lo);
    return FT<T>::of(two_sum(s, e));
}

// Dot product of two ring-table rows of n (a multiple of 4) elements, rows
// 16-byte aligned, added to acc.
__device__ __forceinline__ void ring_dot(const dfl *c, const dfl *d, int n, dfl &acc) {
    const float4 *c4 = (const float4 *)c, *d4 = (const float4 *)d;
    float s = 0.f, e = 0.f;
    for (int q = 0; q < n / 2; ++q) {
        const float4 x = c4[q], y = d4[q];
        dot2_step(s, e, x.x, x.y, y.x, y.y);
        dot2_step(s, e, x.z, x.w, y.z, y.w);
    }
    acc = df_add(acc, two_sum(s, e));
}
__device__ __forceinline__ void ring_dot(const float *c, const float *d, int n, float &acc) {
    const float4 *c4 = (const float4 *)c, *d4 = (const float4 *)d;
    for (int q = 0; q < n / 4; ++q) {
        const float4 x = c4[q], y = d4[q];
        acc = fmaf(x.x, y.x, acc);
        acc = fmaf(x.y, y.y, acc);
        acc = fmaf(x.z, y.z, acc);
        acc = fmaf(x.w, y.w, acc);
    }
}
__device__ __forceinline__ void ring_dot(const double *c, const double *d, int n, double &acc) {
    const double2 *c2 = (const double2 *)c, *d2 = (const double2 *)d;
    for (int q = 0; q < n / 2; ++q) {
        const double2 x = c2[q], y = d2[q];
        acc = fma(x.x, y.x, acc);
        acc = fma(x.y, y.y, acc);
    }
}

struct AsmArgs {
    int *err;                // plan error word (checked builds)
    const void *cl;          // coarse lattice of the local fields, nc^3 per patch (TB)
    const void *mom, *T;     // ring tables in the ring precision RT
    double *FH;
    int np, n, s, nc, npoly, npad, flo, nf;
    int ca_lo, ca_hi, cb_lo, cb_hi;
    dfl coef[4];      // b_k / H^2, double-float
    double coefd[4];  // the same in FP64
    int wide;         // Q = 10: the 5 x 5 x 5 operator (stencil_coef), FP64 tiers only
    double invH2;     // 1 / H^2
};

// Patches i (ascending linear index) whose coarse box C(Omega_beta(i)) holds
// the coarse node k (Sec. 2 coarsening C(D), Sec. 4 eq. FDLD), with k - n i/4
// relative to the patch and whether C(Omega_alpha(i)) holds k too:
// f(p, r0, r1, r2, in_alpha).
template <typename F>
__device__ __forceinline__ void coarse_node_patches(const int k[3], int n, int np, int ca_lo, int ca_hi,
                                                    int cb_lo, int cb_hi, F &&f) {
    const int q = n / 4;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = max(0, -floordiv(-(k[d] - cb_hi), q));  // ceil((k - cb_hi)/q)
        hi[d] = min(np - 1, floordiv(k[d] - cb_lo, q));
    }
    for (int i0 = lo[0]; i0 <= hi[0]; ++i0)
        for (int i1 = lo[1]; i1 <= hi[1]; ++i1)
            for (int i2 = lo[2]; i2 <= hi[2]; ++i2) {
                const int r0 = k[0] - q * i0, r1 = k[1] - q * i1, r2 = k[2] - q * i2;
                const long p = ((long)i0 * np + i1) * np + i2;
                const bool inA = r0 >= ca_lo && r0 <= ca_hi && r1 >= ca_lo && r1 <= ca_hi && r2 >= ca_lo &&
                                 r2 <= ca_hi;
                f(p, r0, r1, r2, inA);
            }
}

// F^H[k] = sum over patches i (ascending) of Delta^H phi^{i,h} on C(Omega_alpha(i))
// or sum_p c_p^i Delta^H(G^h * Q^p) on C(Omega_beta(i)) \ C(Omega_alpha(i)).
// TB: local-field storage, RT: ring tables, T: accumulation (FP64 or double-float).
template <typename TB, typename RT, typename T>
__global__ void __launch_bounds__(128) k_assemble(AsmArgs a) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long tot = (long)a.nf * a.nf * a.nf;
    if (idx >= tot) return;
    int k[3];
    k[2] = (int)(idx % a.nf) + a.flo;
    k[1] = (int)((idx / a.nf) % a.nf) + a.flo;
    k[0] = (int)(idx / ((long)a.nf * a.nf)) + a.flo;
    const int ncb = a.cb_hi - a.cb_lo + 1;
    const long nc = a.nc, kl = -a.s / 4;
    T acc = FT<T>::zero();
    coarse_node_patches(k, a.n, a.np, a.ca_lo, a.ca_hi, a.cb_lo, a.cb_hi,
                        [&](long p, int r0, int r1, int r2, bool inA) {
                if (inA && a.wide) {
                    const TB *bx = (const TB *)a.cl + p * nc * nc * nc;
#pragma unroll
                    for (int s0 = -2; s0 <= 2; ++s0)
#pragma unroll
                        for (int s1 = -2; s1 <= 2; ++s1)
#pragma unroll
                            for (int s2 = -2; s2 <= 2; ++s2) {
                                const double c = stencil_coef(10, s0, s1, s2);
                                if (c == 0.0) continue;
                                const long x0 = r0 + s0 - kl, x1 = r1 + s1 - kl, x2 = r2 + s2 - kl;
                                if (in_range(x0, nc, a.err) & in_range(x1, nc, a.err) & in_range(x2, nc, a.err))
                                    acc = FT<T>::fma(FT<T>::of(c * a.invH2), FT<T>::of(bx[(x0 * nc + x1) * nc + x2]), acc);
                            }
                } else if (inA) {
                    const TB *bx = (const TB *)a.cl + p * nc * nc * nc;
#pragma unroll
                    for (int s0 = -1; s0 <= 1; ++s0)
#pragma unroll
                        for (int s1 = -1; s1 <= 1; ++s1)
#pragma unroll
                            for (int s2 = -1; s2 <= 1; ++s2) {
                                const int nz = (s0 != 0) + (s1 != 0) + (s2 != 0);
                                if (a.coefd[nz] == 0.0) continue;
                                const long x0 = r0 + s0 - kl, x1 = r1 + s1 - kl, x2 = r2 + s2 - kl;
                                if (in_range(x0, nc, a.err) & in_range(x1, nc, a.err) & in_range(x2, nc, a.err))
                                    acc = FT<T>::fma(pick<T>(a.coef[nz], a.coefd[nz]), FT<T>::of(bx[(x0 * nc + x1) * nc + x2]), acc);
                            }
                } else {
                    const long t = (((long)(r0 - a.cb_lo) * ncb + (r1 - a.cb_lo)) * ncb +
                                    (r2 - a.cb_lo)) * a.npoly;
                    if (in_range(r0 - a.cb_lo, ncb, a.err) & in_range(r1 - a.cb_lo, ncb, a.err) &
                        in_range(r2 - a.cb_lo, ncb, a.err))
                        acc = acc + ring_row<T>((const RT *)a.mom + p * a.npad, (const RT *)a.T + t, a.npoly);
                }
            });
    a.FH[idx] = FT<T>::to(acc);
}

// Patches i (ascending linear index) whose Omega_beta(i) holds the
// face-lattice node g (Sec. 4, eq. philocmlcII), with g - n i relative to the
// patch and whether Omega_alpha(i) holds g too: f(p, r0, r1, r2, in_alpha).
// Regions are closed boxes; NN is the patch size n.
template <int NN, typename F>
__device__ __forceinline__ void face_node_patches(const int g[3], int np, int ga, int gb, F &&f) {
    constexpr int n = NN;
    int lo[3], hi[3], alo[3], ahi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = max(0, -floordiv(-(g[d] - n - gb), n));
        hi[d] = min(np - 1, floordiv(g[d] + gb, n));
        alo[d] = max(0, -floordiv(-(g[d] - n - ga), n));
        ahi[d] = min(np - 1, floordiv(g[d] + ga, n));
    }
    for (int i0 = lo[0]; i0 <= hi[0]; ++i0)
        for (int i1 = lo[1]; i1 <= hi[1]; ++i1)
            for (int i2 = lo[2]; i2 <= hi[2]; ++i2) {
                const long p = ((long)i0 * np + i1) * np + i2;
                const int r0 = g[0] - n * i0, r1 = g[1] - n * i1, r2 = g[2] - n * i2;
                const bool inA = i0 >= alo[0] && i0 <= ahi[0] && i1 >= alo[1] && i1 <= ahi[1] &&
                                 i2 >= alo[2] && i2 <= ahi[2];
                f(p, r0, r1, r2, inA);
            }
}

// Face-plane node idx in [axis][plane j][u][v] order -> g (plane x_axis = j n).
__device__ __forceinline__ void face_plane_node(long idx, int N, int np, int n, int g[3], int &axis, int &j) {
    const long pn = (long)(N + 1) * (N + 1);
    axis = (int)(idx / ((np + 1) * pn));
    j = (int)((idx / pn) % (np + 1));
    const int u = (int)((idx % pn) / (N + 1)), v = (int)(idx % (N + 1));
    const int jn = j * n;
    g[0] = axis == 0 ? jn : u;
    g[1] = axis == 0 ? u : (axis == 1 ? jn : v);
    g[2] = axis == 2 ? jn : v;
}

// First half of I^H(phi^H) on every face plane (R4: tensor Lagrange in the
// plane, applied separably): for plane (axis a, j) with in-plane axes u < v,
// every coarse row c_u of phi^H and every fine v in [0, N], the sum along v,
//   Tpl[a][j][c_u - olo][v] = sum_e w_{v mod 4}(e) phi^H(c_a = j n/4, c_u, v/4 - b + e)
// (or the coarse value itself when v mod 4 = 0).  The boundary kernel then
// sums K of these along u: the same operations in the same order as the
// nested sums at each node, done once per (plane, coarse row, v).
struct LagW {
    dfl lw[4][12];      // Lagrange weights for g mod 4 = r (row r), double-float
    double lwd[4][12];  // the same in FP64
};

template <typename T>
__global__ void __launch_bounds__(256) k_plane_interp(const void *phiH_, void *out_, int N, int n, int np, int b,
                                                      int olo, int no, LagW w, int *err) {
    const long tot = 3L * (np + 1) * no * (N + 1);
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const T *phiH = (const T *)phiH_;
    const int v = (int)(idx % (N + 1));
    const int cu = (int)((idx / (N + 1)) % no);
    const int pj = (int)(idx / ((long)(N + 1) * no));  // axis * (np + 1) + j
    const int axis = pj / (np + 1), j = pj % (np + 1);
    const int ca = j * n / 4 - olo, cuo = cu;  // offsets into phi^H
    // phi^H at coarse (plane, c_u, c_v) for the plane's axis order
    auto at = [&](int cv) -> T {
        const int c = cv - olo;
        if (!(in_range(c, no, err) & in_range(ca, no, err) & in_range(cuo, no, err))) return FT<T>::zero();
        long i;
        if (axis == 0) i = ((long)ca * no + cuo) * no + c;
        else if (axis == 1) i = ((long)cuo * no + ca) * no + c;
        else i = ((long)cuo * no + c) * no + ca;
        return phiH[i];
    };
    const int rv = v & 3;
    T s;
    if (rv == 0) {
        s = at(v >> 2);
    } else {
        const int kb = (v >> 2) - b, K = 2 * b + 2;
        s = FT<T>::zero();
        for (int e = 0; e < K; ++e) {
            const T x = axis == 2 ? FT<T>::rn(at(kb + e)) : at(kb + e);
            s = FT<T>::fma(pick<T>(w.lw[rv][e], w.lwd[rv][e]), x, s);
        }
    }
    ((T *)out_)[idx] = s;
}

struct BndArgs {
    int *err;                  // plan error word (checked builds)
    const void *phiH, *resid;  // fine precision T
    const void *tpl;           // k_plane_interp output, fine precision T
    const float *ringR;        // RING: [patch][ring_rows_pad] ring terms of this launch's axis
    long ring_rows_pad;
    long idx0, idx1;           // face-plane nodes of this launch: [idx0, idx1)
    const void *mom, *D;       // ring tables in the ring precision RT
    void *phiB;                // fine precision T
    int N, n, np, ga, gb, b, npoly, olo, no, wa, wbx, npa, pl0;
    int pb0, npb;     // face planes of Omega_beta (relative): pb0 + j n, j < npb
    int npad;         // row stride of the ring tables (npoly rounded up to 4; zero padding)
    dfl lw[4][12];     // Lagrange weights for g mod 4 = r (row r), 2b+2 entries
    double lwd[4][12];
};

// phi^B at every face-plane node (axis, plane j, u, v).  RT: precision of the
// Legendre ring sums (the local-convolution precision: FP32, double-float or
// FP64); T: the interpolation and the accumulation (FP64 or double-float).
// RING: the ring terms come from the ring GEMM (ringR) instead of per-node
// dot products of the ring-table rows with the coefficients.
template <typename RT, int NN, typename T, bool RING = false>
__global__ void __launch_bounds__(128, 6) k_boundary(BndArgs a) {
    constexpr int n = NN;  // patch size as a constant: the index divisions become multiplies
    const long idx = a.idx0 + (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.idx1) return;
    const T *phiH = (const T *)a.phiH;
    const T *resid = (const T *)a.resid;
    int g[3], axis, jp;
    face_plane_node(idx, a.N, a.np, n, g, axis, jp);
    // I^H(phi^H)(g): tensor Lagrange over the in-plane axes (R4), the sums
    // along v precomputed per (plane, coarse row) by k_plane_interp; here the
    // K-term sum along u (in-plane axes u < v)
    (void)phiH;
    const int K = 2 * a.b + 2;
    const int gu = axis == 0 ? g[1] : g[0], gv = axis == 2 ? g[1] : g[2];
    const T *tpl = (const T *)a.tpl + ((long)(axis * (a.np + 1) + jp) * a.no) * (a.N + 1) + gv;
    const int ru = gu & 3;
    T acc;
    if (ru == 0) {
        acc = tpl[(long)((gu >> 2) - a.olo) * (a.N + 1)];
    } else {
        acc = FT<T>::zero();
        const int kb = (gu >> 2) - a.b - a.olo;
        // unrolled to b = 3 so the K loads issue together; b = 4, 5 continue
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (e < K && in_range(kb + e, a.no, a.err))
                acc = FT<T>::fma(pick<T>(a.lw[ru][e], a.lwd[ru][e]), FT<T>::rn(tpl[(long)(kb + e) * (a.N + 1)]), acc);
        if (K > 8)
            for (int e = 8; e < K; ++e)
                if (in_range(kb + e, a.no, a.err))
                    acc = FT<T>::fma(pick<T>(a.lw[ru][e], a.lwd[ru][e]), FT<T>::rn(tpl[(long)(kb + e) * (a.N + 1)]), acc);
    }
    // local corrections of the patches whose Omega_beta holds g (ascending index);
    // the Legendre ring terms accumulate in the ring precision RT
    RT ring(0.0);
    face_node_patches<NN>(g, a.np, a.ga, a.gb, [&](long p, int r0, int r1, int r2, bool inA) {
                if (inA) {
                    // the residual plane holding r: first axis on a face plane
                    int d, uu, vv;
                    if ((r0 - a.pl0) % n == 0) { d = 0; uu = r1; vv = r2; }
                    else if ((r1 - a.pl0) % n == 0) { d = 1; uu = r0; vv = r2; }
                    else { d = 2; uu = r0; vv = r1; }
                    const int rr = d == 0 ? r0 : (d == 1 ? r1 : r2);
                    const long slot = (long)d * a.npa + (rr - a.pl0) / n;
                    if (in_range((rr - a.pl0) / n, a.npa, a.err) & in_range(uu + a.ga, a.wa, a.err) &
                        in_range(vv + a.ga, a.wa, a.err))
                        acc = acc + resid[((p * 3 * a.npa + slot) * a.wa + (uu + a.ga)) * a.wa + (vv + a.ga)];
                } else {
                    // dense ring row of (axis, plane, u, v): no index map to read
                    const int ra = axis == 0 ? r0 : (axis == 1 ? r1 : r2);
                    const int ru = axis == 0 ? r1 : r0, rv = axis == 2 ? r1 : r2;
                    const bool ok = in_range((ra - a.pb0) / n, a.npb, a.err) & in_range(ru + a.gb, a.wbx, a.err) &
                                    in_range(rv + a.gb, a.wbx, a.err);
                    if constexpr (RING) {
                        const long row = ((long)((ra - a.pb0) / n) * a.wbx + (ru + a.gb)) * a.wbx + (rv + a.gb);
                        if (ok) ring += a.ringR[p * a.ring_rows_pad + row];
                    } else {
                        const long row = (((long)axis * a.npb + (ra - a.pb0) / n) * a.wbx + (ru + a.gb)) * a.wbx + (rv + a.gb);
                        if (ok) ring_dot((const RT *)a.mom + p * a.npad, (const RT *)a.D + row * a.npad, a.npad, ring);
                    }
                }
            });
    ((T *)a.phiB)[idx] = FT<T>::rn(acc + FT<T>::of(ring));
}

// Index export (test hook): for every face-plane node ([axis][plane][u][v]
// order) the patches whose Omega_beta holds it, enumerated by
// face_node_patches -- the code the boundary kernel runs.  COUNT pass:
// cnt[node] = number of patches; fill pass: entries 2 p + (ring ? 1 : 0)
// from off[node], in enumeration (ascending patch) order.
template <int NN, bool COUNT>
__global__ void __launch_bounds__(128) k_index_face(int N, int np, int ga, int gb, long tot, int *cnt,
                                                    const long *off, int *ent) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    int g[3], axis, jp;
    face_plane_node(idx, N, np, NN, g, axis, jp);
    int c = 0;
    const long o = COUNT ? 0 : off[idx];
    face_node_patches<NN>(g, np, ga, gb, [&](long p, int, int, int, bool inA) {
        if (!COUNT) ent[o + c] = (int)(2 * p + (inA ? 0 : 1));
        ++c;
    });
    if (COUNT) cnt[idx] = c;
}

// The same for every coarse node k of the F^H extent ([k0][k1][k2] order),
// enumerated by coarse_node_patches -- the code the F^H assembly runs.
template <bool COUNT>
__global__ void __launch_bounds__(128) k_index_coarse(int n, int np, int ca_lo, int ca_hi, int cb_lo, int cb_hi,
                                                      int flo, int nf, int *cnt, const long *off, int *ent) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nf * nf * nf) return;
    const int k[3] = {(int)(idx / ((long)nf * nf)) + flo, (int)((idx / nf) % nf) + flo, (int)(idx % nf) + flo};
    int c = 0;
    const long o = COUNT ? 0 : off[idx];
    coarse_node_patches(k, n, np, ca_lo, ca_hi, cb_lo, cb_hi, [&](long p, int, int, int, bool inA) {
        if (!COUNT) ent[o + c] = (int)(2 * p + (inA ? 0 : 1));
        ++c;
    });
    if (COUNT) cnt[idx] = c;
}

struct DirArgs {
    Items it;  // per item: f, phiB, phi, lam, N, np, h of its plan
    int n;
    double b[4];
    const void *sinm;  // (n-1) x n/2: sin(pi k t / n), k in [1, n-1], t in [1, n/2], fine precision
};

template <typename T>
__device__ __forceinline__ T phiB_at(const PlanPtrs &a, int n, int g0, int g1, int g2) {
    const long pn = (long)(a.N + 1) * (a.N + 1);
    int axis, j, u, v;
    if (g0 % n == 0) {
        axis = 0; j = g0 / n; u = g1; v = g2;
    } else if (g1 % n == 0) {
        axis = 1; j = g1 / n; u = g0; v = g2;
    } else {
        axis = 2; j = g2 / n; u = g0; v = g1;
    }
    if (!(in_range(j, a.np + 1, a.err) & in_range(u, a.N + 1, a.err) & in_range(v, a.N + 1, a.err)))
        return FT<T>::zero();
    return ((const T *)a.phiB)[((long)axis * (a.np + 1) + j) * pn + (long)u * (a.N + 1) + v];
}

// sin(pi m / 16) for integer m as (index into sv[0..8] = sin(pi i / 16), sign),
// resolved at compile time.
__host__ __device__ constexpr int sin16_idx(int m) {
    return ((m % 32 + 32) % 32) % 16 <= 8 ? ((m % 32 + 32) % 32) % 16 : 16 - ((m % 32 + 32) % 32) % 16;
}
__host__ __device__ constexpr bool sin16_neg(int m) { return ((m % 32 + 32) % 32) >= 16; }
template <int M16, typename T>
__device__ __forceinline__ T mul_sin16(T v, const T (&sv)[9]) {
    const T r = v * sv[sin16_idx(M16)];
    return sin16_neg(M16) ? -r : r;
}

// DST-I of 15 values (n = 16) in the fine precision T, y_k = sum_t x_t
// sin(pi k t / 16), by symmetric splitting: with s_t = x_t + x_{16-t} and
// d_t = x_t - x_{16-t}, the even outputs are the length-7 DST-I of d (split
// once more into e_t = d_t - d_{8-t}, f_t = d_t + d_{8-t}), and the odd
// outputs pair up as y_{2j+1} = P_j + Q_j + (-1)^j x_8,
// y_{15-2j} = P_j - Q_j - (-1)^j x_8 with P_j, Q_j the sums of
// s_t sin(pi (2j+1) t / 16) over odd and even t (using
// sin(pi (16 - k) t / 16) = -(-1)^t sin(pi k t / 16)).  29 products and 68
// sums instead of 105 and 98 for the direct sums.  x[t-1] = x_t in, y_k out.
template <typename T>
__device__ __forceinline__ void dst15_fast(T (&x)[15], const T (&sv)[9]) {
    T sp[8], dm[8];
#pragma unroll
    for (int t = 1; t < 8; ++t) {
        sp[t] = x[t - 1] + x[15 - t];
        dm[t] = x[t - 1] - x[15 - t];
    }
    const T x8 = x[7];
    T y[16];
    // even outputs
    {
        T e[4], f[4];
#pragma unroll
        for (int t = 1; t < 4; ++t) {
            e[t] = dm[t] - dm[8 - t];
            f[t] = dm[t] + dm[8 - t];
        }
        const T d4 = dm[4];
        const T ec = mul_sin16<4>(e[1] + e[3], sv);
        y[4] = ec + e[2];
        y[8] = e[1] - e[3];
        y[12] = ec - e[2];
        // kk = 0: sin(pi t / 8) -> m = 2t; kk = 1: sin(3 pi t / 8) -> m = 6t
        const T po0 = mul_sin16<2>(f[1], sv) + mul_sin16<6>(f[3], sv);
        const T qe0 = mul_sin16<4>(f[2], sv);
        const T po1 = mul_sin16<6>(f[1], sv) + mul_sin16<18>(f[3], sv);
        const T qe1 = mul_sin16<12>(f[2], sv);
        y[2] = (po0 + qe0) + d4;
        y[14] = (po0 - qe0) - d4;   // kk' = 3: (-1)^3
        y[6] = (po1 + qe1) - d4;    // kk = 1
        y[10] = (po1 - qe1) + d4;   // kk' = 2
    }
    // odd outputs
    {
        const T qo0 = mul_sin16<2>(sp[2], sv) + mul_sin16<6>(sp[6], sv);
        const T qe0 = mul_sin16<4>(sp[4], sv);
        const T qo1 = mul_sin16<6>(sp[2], sv) + mul_sin16<18>(sp[6], sv);
        const T qe1 = mul_sin16<12>(sp[4], sv);
        const T Q[4] = {qo0 + qe0, qo1 + qe1, qo1 - qe1, qo0 - qe0};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = 2 * j + 1;
            T p1, p3, p5, p7;
            switch (j) {  // compile-time after unrolling
                case 0: p1 = mul_sin16<1>(sp[1], sv); p3 = mul_sin16<3>(sp[3], sv); p5 = mul_sin16<5>(sp[5], sv); p7 = mul_sin16<7>(sp[7], sv); break;
                case 1: p1 = mul_sin16<3>(sp[1], sv); p3 = mul_sin16<9>(sp[3], sv); p5 = mul_sin16<15>(sp[5], sv); p7 = mul_sin16<21>(sp[7], sv); break;
                case 2: p1 = mul_sin16<5>(sp[1], sv); p3 = mul_sin16<15>(sp[3], sv); p5 = mul_sin16<25>(sp[5], sv); p7 = mul_sin16<35>(sp[7], sv); break;
                default: p1 = mul_sin16<7>(sp[1], sv); p3 = mul_sin16<21>(sp[3], sv); p5 = mul_sin16<35>(sp[5], sv); p7 = mul_sin16<49>(sp[7], sv); break;
            }
            const T Pj = (p1 + p3) + (p5 + p7);
            const T xs = (j & 1) ? -x8 : x8;
            y[k] = (Pj + Q[j]) + xs;
            y[15 - 2 * j] = (Pj - Q[j]) - xs;
        }
    }
#pragma unroll
    for (int k = 1; k < 16; ++k) x[k - 1] = y[k];
}

// sin(pi m / 32) for integer m as (index into sv[0..16] = sin(pi i / 32), sign),
// resolved at compile time.
__host__ __device__ constexpr int sin32_idx(int m) {
    return ((m % 64 + 64) % 64) % 32 <= 16 ? ((m % 64 + 64) % 64) % 32 : 32 - ((m % 64 + 64) % 64) % 32;
}
__host__ __device__ constexpr bool sin32_neg(int m) { return ((m % 64 + 64) % 64) >= 32; }
template <int M32, typename T>
__device__ __forceinline__ T fma_sin32(T v, T acc, const T (&sv)[17]) {
    return FT<T>::fma(sv[sin32_idx(M32)], sin32_neg(M32) ? -v : v, acc);
}

// DST-I of 31 values (n = 32), y_k = sum_t x_t sin(pi k t / 32), by one
// symmetric split: with s_t = x_t + x_{32-t} and d_t = x_t - x_{32-t}
// (t = 1..15), the even outputs are the 15-point DST-I of d (dst15_fast,
// sin(pi j t / 16) = sin(pi 2 j t / 32)), and the odd outputs pair up as
// y_{2j+1} = P_j + Q_j + (-1)^j x_16, y_{31-2j} = P_j - Q_j - (-1)^j x_16
// (j = 0..7) with P_j, Q_j the sums of s_t sin(pi (2j+1) t / 32) over odd and
// even t (sin(pi (32 - k) t / 32) = -(-1)^t sin(pi k t / 32)).  120 fused
// products and about 130 sums instead of 496 products for the direct sums.
// x[t-1] = x_t in, y_k out in x[k-1].
template <int J, typename T>
__device__ __forceinline__ void dst31_odd_pair(const T (&sp)[16], T c, const T (&sv)[17], T (&x)[31]) {
    T P = FT<T>::zero(), Q = FT<T>::zero();
    P = fma_sin32<(2 * J + 1) * 1>(sp[1], P, sv);
    P = fma_sin32<(2 * J + 1) * 3>(sp[3], P, sv);
    P = fma_sin32<(2 * J + 1) * 5>(sp[5], P, sv);
    P = fma_sin32<(2 * J + 1) * 7>(sp[7], P, sv);
    P = fma_sin32<(2 * J + 1) * 9>(sp[9], P, sv);
    P = fma_sin32<(2 * J + 1) * 11>(sp[11], P, sv);
    P = fma_sin32<(2 * J + 1) * 13>(sp[13], P, sv);
    P = fma_sin32<(2 * J + 1) * 15>(sp[15], P, sv);
    Q = fma_sin32<(2 * J + 1) * 2>(sp[2], Q, sv);
    Q = fma_sin32<(2 * J + 1) * 4>(sp[4], Q, sv);
    Q = fma_sin32<(2 * J + 1) * 6>(sp[6], Q, sv);
    Q = fma_sin32<(2 * J + 1) * 8>(sp[8], Q, sv);
    Q = fma_sin32<(2 * J + 1) * 10>(sp[10], Q, sv);
    Q = fma_sin32<(2 * J + 1) * 12>(sp[12], Q, sv);
    Q = fma_sin32<(2 * J + 1) * 14>(sp[14], Q, sv);
    const T cs = (J & 1) ? -c : c;
    x[2 * J] = (P + Q) + cs;       // y_{2J+1}
    x[30 - 2 * J] = (P - Q) - cs;  // y_{31-2J}
}
template <typename T>
__device__ __forceinline__ void dst31_fast(T (&x)[31], const T (&sv)[17]) {
    T sp[16], dm[15];
#pragma unroll
    for (int t = 1; t < 16; ++t) {
        sp[t] = x[t - 1] + x[31 - t];
        dm[t - 1] = x[t - 1] - x[31 - t];
    }
    sp[0] = FT<T>::zero();
    const T c = x[15];
    dst31_odd_pair<0>(sp, c, sv, x);
    dst31_odd_pair<1>(sp, c, sv, x);
    dst31_odd_pair<2>(sp, c, sv, x);
    dst31_odd_pair<3>(sp, c, sv, x);
    dst31_odd_pair<4>(sp, c, sv, x);
    dst31_odd_pair<5>(sp, c, sv, x);
    dst31_odd_pair<6>(sp, c, sv, x);
    dst31_odd_pair<7>(sp, c, sv, x);
    T s16[9];
#pragma unroll
    for (int i = 0; i <= 8; ++i) s16[i] = sv[2 * i];  // sin(pi i / 16)
    dst15_fast(dm, s16);
#pragma unroll
    for (int j = 1; j <= 15; ++j) x[2 * j - 1] = dm[j - 1];  // y_{2j}
}

// Local Dirichlet solve of one patch (Sec. 4, final step): the (Q-th order)
// stencil problem on the closed patch with boundary data phi^B, by DST-I in
// all three axes, then phi = u + (h^2/12) f.  T: the arithmetic between the
// loads and the final FP64 store, FP64 (the FP64 pipe) or double-float (the
// FP32 pipe; GB300 issues FP64 on ~1/67 of the FP32 lanes).  TF: the charge.
// Patches up to n = 24 keep their m^3 work array in shared memory; larger
// ones (BIG) keep it in the plan's global Dirichlet workspace (the same code
// on global memory; the patch's 238 KB stay in L2 between the passes).
template <typename TF, int NN, typename T>
__global__ void __launch_bounds__(256, NN > 16 ? 1 : (std::is_same<T, double>::value ? 3 : 4))
    k_dirichlet(DirArgs a) {
    extern __shared__ double sm[];
    constexpr int n = NN, nb = n + 1, m = n - 1, h = n / 2;
    constexpr bool BIG = NN > 24;
    T *U = (T *)sm;                    // boundary values on the 6 faces, nb^2 each (face 2 axis + side)
    // boundary value at node (c0, c1, c2) of the closed patch, one coordinate 0 or n
    auto Uat = [&](int c0, int c1, int c2) -> T {
        if (c0 == 0 || c0 == n) return U[((c0 ? 1 : 0) * nb + c1) * nb + c2];
        if (c1 == 0 || c1 == n) return U[((2 + (c1 ? 1 : 0)) * nb + c0) * nb + c2];
        return U[((4 + (c2 ? 1 : 0)) * nb + c0) * nb + c1];
    };
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x, p);
    T *X = BIG ? (T *)PP.dscr + (long)p * m * m * m : U + 6 * nb * nb;  // m^3 work
    T *Sh = BIG ? U + 6 * nb * nb : X + m * m * m;                       // (n-1) x n/2 half sine table
    const int np = PP.np, N = PP.N;
    const int i2 = p % np, i1 = (p / np) % np, i0 = p / (np * np);
    const int o0 = i0 * n, o1 = i1 * n, o2 = i2 * n;
    const TF *f = (const TF *)PP.f;
    const T *sinm = (const T *)a.sinm;
    const T *lam = (const T *)PP.lam;
    for (int e = threadIdx.x; e < m * h; e += blockDim.x) Sh[e] = sinm[e];
    for (int e = threadIdx.x; e < 6 * nb * nb; e += blockDim.x) {
        const int b = e % nb, a2 = (e / nb) % nb, fc = e / (nb * nb);  // face fc: axis fc/2, side fc%2
        const int side = (fc & 1) ? n : 0;
        int m0, m1, m2;
        if (fc < 2) { m0 = side; m1 = a2; m2 = b; }
        else if (fc < 4) { m0 = a2; m1 = side; m2 = b; }
        else { m0 = a2; m1 = b; m2 = side; }
        U[e] = phiB_at<T>(PP, n, o0 + m0, o1 + m1, o2 + m2);
    }
    // stencil weights b_k / h^2 and h^2/12 of this plan (converted once per CTA)
    __shared__ T s_w[5];
    if (threadIdx.x < 5) {
        double w = PP.c2h2;
#pragma unroll
        for (int k = 0; k < 4; ++k)  // static indices: the parameter array stays out of local memory
            if (threadIdx.x == k) w = a.b[k] * PP.inv_h2;
        s_w[threadIdx.x] = FT<T>::of(w);
    }
    __syncthreads();
    T cw[4];
    bool cwz[4];  // zero weights (tested once: FP64 compares run on the slow FP64 pipe)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cw[k] = s_w[k];
        cwz[k] = a.b[k] == 0.0;
    }
    const T c2h2 = s_w[4];
    // right-hand side: f - Delta^h(boundary data).  Only the layers next to the
    // boundary see boundary values; they are subtracted in six face passes,
    // one per (axis a, side): every interior node c of the layer c_a = 1 (or
    // n - 1) and every stencil neighbour d with d_a = 0 (or n), except those
    // with a boundary coordinate on an axis before a (counted in that axis's
    // pass) -- each (node, boundary neighbour) pair once, with the threads of
    // a warp on neighbouring nodes of one layer doing the same products.
    for (int e = threadIdx.x; e < m * m * m; e += blockDim.x) {
        const int c2 = e % m + 1, c1 = (e / m) % m + 1, c0 = e / (m * m) + 1;
        const int z = o0 + c0, y = o1 + c1, x = o2 + c2;
        X[e] = (z < N && y < N && x < N) ? FT<T>::of(f[((long)z * N + y) * N + x]) : FT<T>::zero();
    }
    __syncthreads();
    for (int fc = 0; fc < 6; ++fc) {
        const int ax = fc >> 1, sa = (fc & 1) ? 1 : -1;  // neighbour offset along ax
        const int ca = (fc & 1) ? m : 1, da = (fc & 1) ? n : 0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int cb = e / m + 1, cc = e % m + 1;  // the other two coordinates, increasing axis order
            T acc = FT<T>::zero();
#pragma unroll
            for (int sb = -1; sb <= 1; ++sb)
#pragma unroll
                for (int sc = -1; sc <= 1; ++sc) {
                    const int nz = 1 + (sb != 0) + (sc != 0);
                    if (cwz[nz]) continue;
                    const int db = cb + sb, dc = cc + sc;
                    const bool bb = db == 0 || db == n, bc = dc == 0 || dc == n;
                    // other axes: b is the lower of the two, c the higher
                    const int axb = ax == 0 ? 1 : 0, axc = ax == 2 ? 1 : 2;
                    if ((axb < ax && bb) || (axc < ax && bc)) continue;  // an earlier pass has it
                    int d0, d1, d2;
                    if (ax == 0) { d0 = da; d1 = db; d2 = dc; }
                    else if (ax == 1) { d0 = db; d1 = da; d2 = dc; }
                    else { d0 = db; d1 = dc; d2 = da; }
                    acc = FT<T>::fma(cw[nz], Uat(d0, d1, d2), acc);
                }
            int c0, c1, c2;
            if (ax == 0) { c0 = ca; c1 = cb; c2 = cc; }
            else if (ax == 1) { c0 = cb; c1 = ca; c2 = cc; }
            else { c0 = cb; c1 = cc; c2 = ca; }
            T &xv = X[((c0 - 1) * m + (c1 - 1)) * m + (c2 - 1)];
            xv = xv - acc;
        }
        (void)sa;
        __syncthreads();  // the next pass may update the same edge nodes
    }
    // DST-I along axes 2, 1, 0; scale by the inverse eigenvalues; DST-I along 2, 1, 0
    if constexpr (NN == 16) {
        // n = 16: one thread per line with the split-radix DST (dst15_fast)
        T sv[9];
        sv[0] = FT<T>::zero();
#pragma unroll
        for (int i = 1; i <= 8; ++i) sv[i] = Sh[i - 1];  // sin(pi i / 16)
        for (int pass = 0; pass < 6; ++pass) {
            const int axis = 2 - (pass % 3);
            for (int l = threadIdx.x; l < m * m; l += blockDim.x) {
                const int q1 = l % m, q0 = l / m;
                int base, str;
                if (axis == 2) { base = (q0 * m + q1) * m; str = 1; }
                else if (axis == 1) { base = q0 * m * m + q1; str = m; }
                else { base = q0 * m + q1; str = m * m; }
                T x[15];
#pragma unroll
                for (int t = 0; t < 15; ++t) x[t] = FT<T>::rn(X[base + t * str]);
                dst15_fast(x, sv);
                if (pass == 2) {
#pragma unroll
                    for (int t = 0; t < 15; ++t) x[t] = x[t] * lam[base + t * str];
                }
#pragma unroll
                for (int t = 0; t < 15; ++t) X[base + t * str] = x[t];
            }
            __syncthreads();
        }
    } else if constexpr (NN == 32) {
        // n = 32: one thread per line with the split DST (dst31_fast)
        T sv[17];
        sv[0] = FT<T>::zero();
#pragma unroll
        for (int i = 1; i <= 16; ++i) sv[i] = Sh[i - 1];  // sin(pi i / 32)
        for (int pass = 0; pass < 6; ++pass) {
            const int axis = 2 - (pass % 3);
            for (int l = threadIdx.x; l < m * m; l += blockDim.x) {
                const int q1 = l % m, q0 = l / m;
                int base, str;
                if (axis == 2) { base = (q0 * m + q1) * m; str = 1; }
                else if (axis == 1) { base = q0 * m * m + q1; str = m; }
                else { base = q0 * m + q1; str = m * m; }
                T x[31];
#pragma unroll
                for (int t = 0; t < 31; ++t) x[t] = FT<T>::rn(X[base + t * str]);
                dst31_fast(x, sv);
                if (pass == 2) {
#pragma unroll
                    for (int t = 0; t < 31; ++t) x[t] = x[t] * lam[base + t * str];
                }
#pragma unroll
                for (int t = 0; t < 31; ++t) X[base + t * str] = x[t];
            }
            __syncthreads();
        }
    } else {
    // Two threads per line (adjacent lanes): lane parity 0 forms the odd
    // outputs k = 1, 3, .. from the sums x_t + x_{n-t} (and the middle node),
    // parity 1 the even outputs from the differences x_t - x_{n-t}; both run
    // the same instruction stream (the middle node enters with weight 0 for
    // even k).
    const int par = threadIdx.x & 1, ntl = blockDim.x >> 1;
    for (int pass = 0; pass < 6; ++pass) {
        const int axis = 2 - (pass % 3);
        for (int l0 = 0; l0 < m * m; l0 += ntl) {  // uniform trip count across the CTA
            const int l = l0 + (threadIdx.x >> 1);
            const bool valid = l < m * m;
            const int q1 = l % m, q0 = l / m;
            int base = 0, str = 1;
            if (axis == 2) { base = (q0 * m + q1) * m; str = 1; }
            else if (axis == 1) { base = q0 * m * m + q1; str = m; }
            else { base = q0 * m + q1; str = m * m; }
            T x[m];
#pragma unroll
            for (int t = 0; t < m; ++t) x[t] = valid ? FT<T>::rn(X[base + t * str]) : FT<T>::zero();
            T u[h + 1];
#pragma unroll
            for (int t = 1; t < h; ++t) {
                const T b = x[n - t - 1];
                u[t] = x[t - 1] + (par ? -b : b);
            }
            u[h] = par ? FT<T>::zero() : x[h - 1];
            __syncwarp();  // both lanes of the line have read it before either writes
            if (valid) {
#pragma unroll
                for (int j = 0; j < (m + 1) / 2; ++j) {
                    const int k = 2 * j + 1 + par;  // output index 1..m
                    if (k > m) break;
                    const T *row = Sh + (k - 1) * h;
                    // h products accumulated by fused multiply-adds in four
                    // independent chains (t mod 4), then summed
                    T acc[4] = {FT<T>::zero(), FT<T>::zero(), FT<T>::zero(), FT<T>::zero()};
#pragma unroll
                    for (int t = 1; t <= h; ++t) acc[(t - 1) & 3] = FT<T>::fma(row[t - 1], u[t], acc[(t - 1) & 3]);
                    T v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
                    if (pass == 2) v = v * lam[base + (k - 1) * str];
                    X[base + (k - 1) * str] = v;
                }
            }
        }
        __syncthreads();
    }
    }
    for (int e = threadIdx.x; e < n * n * n; e += blockDim.x) {
        const int m2 = e % n, m1 = (e / n) % n, m0 = e / (n * n);
        const bool bnd = m0 == 0 || m1 == 0 || m2 == 0;
        const int z = o0 + m0, y = o1 + m1, x = o2 + m2;
        const long gi = ((long)z * N + y) * N + x;
        const T u = bnd ? Uat(m0, m1, m2) : X[((m0 - 1) * m + (m1 - 1)) * m + (m2 - 1)];
        PP.phi[gi] = FT<T>::to(u + c2h2 * FT<T>::of(f[gi]));
    }
}

// ---------------------------------------------------------------------------
// Coarse Hockney convolution (Step 2, App. A.2) with mixed-radix Stockham
// FFTs: the period M is any even product of the radices 2, 3, 4, 5, so it can
// be the smallest such length that the Hockney condition allows instead of
// the next power of two (144 rather than 256 at N = 256, Q = 6).  Stockham's
// autosort form keeps natural order in and out, ping-ponging between two
// shared-memory buffers, one stage per radix.
// ---------------------------------------------------------------------------
struct RadixPlan {
    int n;       // stages
    int r[16];   // radix of each stage (product = M)
};

template <typename C, typename R>
__device__ __forceinline__ C cscale(C a, R s) {
    C r;
    r.x = a.x * s;
    r.y = a.y * s;
    return r;
}

// In-register DFT of length rad in {2, 3, 4, 5} (natural order), forward
// (exp(-2 pi i n k / rad)) or inverse (conjugate kernel).
template <typename C, typename R>
__device__ __forceinline__ void dft_small(C (&v)[5], int rad, bool inv) {
    if (rad == 2) {
        const C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (rad == 4) {
        const C a = cadd(v[0], v[2]), b = csub(v[0], v[2]), c = cadd(v[1], v[3]);
        const C d = mul_mi(csub(v[1], v[3]), inv);  // -i (x1 - x3), forward
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    } else if (rad == 3) {
        // X1,2 = x0 - (x1 + x2)/2 -+ i sin(2 pi/3) (x1 - x2)
        const R s3 = R(0.86602540378443864676), half = R(0.5);
        const C t1 = cadd(v[1], v[2]);
        const C t2 = csub(v[0], cscale(t1, half));
        const C m = mul_mi(cscale(csub(v[1], v[2]), s3), inv);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, m);
        v[2] = csub(t2, m);
    } else {  // 5: c_k = cos(2 pi k / 5), s_k = sin(2 pi k / 5)
        const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);
        const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);
        const C a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]);
        const C b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
        const C t1 = cadd(v[0], cadd(cscale(a1, c1), cscale(a2, c2)));
        const C t2 = cadd(v[0], cadd(cscale(a1, c2), cscale(a2, c1)));
        const C m1 = mul_mi(cadd(cscale(b1, s1), cscale(b2, s2)), inv);
        const C m2 = mul_mi(csub(cscale(b1, s2), cscale(b2, s1)), inv);
        v[0] = cadd(v[0], cadd(a1, a2));
        v[1] = cadd(t1, m1);
        v[4] = csub(t1, m1);
        v[2] = cadd(t2, m2);
        v[3] = csub(t2, m2);
    }
}

// Stockham FFT of nlines lines of length M in shared memory: line l at
// src + l lstride, element i at + i estride; dst is scratch of the same
// layout.  Stage with radix R and span Ns (product of the earlier radices):
// for j < M/R, k = j mod Ns, x_r = src[j + r M/R] w^(r k M/(Ns R)),
// y = DFT_R(x), dst[(j/Ns) Ns R + k + r Ns] = y_r.  tw: w^t = exp(-2 pi i t/M),
// t < M (conjugated for the inverse).  Ends with __syncthreads; returns the
// buffer that holds the result.
template <typename C, typename R>
__device__ C *fft_stockham(C *src, C *dst, int nlines, int lstride, int estride, int M, const RadixPlan &rp,
                           const C *tw, bool inv) {
    int Ns = 1;
    for (int st = 0; st < rp.n; ++st) {
        const int rad = rp.r[st], MR = M / rad, tstep = M / (Ns * rad);
        for (int e = threadIdx.x; e < nlines * MR; e += blockDim.x) {
            const int line = e % nlines, j = e / nlines;
            const C *sl = src + line * lstride;
            C *dl = dst + line * lstride;
            const int k = j % Ns;
            C v[5];
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                if (r < rad) {
                    C x = renorm(sl[(j + r * MR) * estride]);
                    if (r && k) {
                        C w = tw[(r * k * tstep) % M];
                        if (inv) w.y = -w.y;
                        x = cmul(x, w);
                    }
                    v[r] = x;
                }
            }
            dft_small<C, R>(v, rad, inv);
            const int base = (j / Ns) * Ns * rad + k;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < rad) dl[(base + r * Ns) * estride] = v[r];
        }
        __syncthreads();
        C *t = src;
        src = dst;
        dst = t;
        Ns *= rad;
    }
    return src;
}

// Full twiddle table w^t = exp(-2 pi i t / M), t < M, from the half table (t < M/2).
template <typename C>
__device__ __forceinline__ void load_twiddles_full(C *s_tw, const C *tw, int M) {
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        C w = tw[t % (M / 2)];
        if (t >= M / 2) { w.x = -w.x; w.y = -w.y; }
        s_tw[t] = w;
    }
}

struct CoarseArgs {
    const void *in;
    void *out;
    const void *tw;      // M/2 twiddles exp(-2 pi i t / M) in R
    const void *khat;    // real-even kernel spectrum octant (M/2+1)^3 in R (z pass)
    int M, MH, nin, nout, out_off;
    int lines_cta;       // x passes: lines per CTA
    int cols_cta;        // column passes: columns per CTA
    long in_sp, in_row, out_sp, out_row;  // column passes: slab and row strides (complex entries)
    RadixPlan rp;
};

// Forward real transform along x of the dense coarse charge F^H (nin^3,
// FP64): line (zi, yi) of nin samples, zero padded to M; half spectrum
// kx <= M/2 to out[(zi nin + yi) MH + kx].
template <typename R>
__global__ void __launch_bounds__(256) k_cfft_x(CoarseArgs a) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = a.M, LS = M + 1;
    C *tw = (C *)smem_raw;
    C *A = tw + M;
    C *B = A + a.lines_cta * LS;
    const int zi = blockIdx.x, y0 = blockIdx.y * a.lines_cta, nl = min(a.lines_cta, a.nin - y0);
    load_twiddles_full(tw, (const C *)a.tw, M);
    const double *F = (const double *)a.in;
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = e / M, x = e % M;
        C v = Cx<R>::mk(0, 0);
        if (x < a.nin) v.x = R(F[((long)zi * a.nin + y0 + l) * a.nin + x]);
        A[l * LS + x] = v;
    }
    __syncthreads();
    const C *res = fft_stockham<C, R>(A, B, nl, LS, 1, M, a.rp, tw, false);
    C *out = (C *)a.out;
    for (int e = threadIdx.x; e < nl * a.MH; e += blockDim.x) {
        const int l = e / a.MH, k = e % a.MH;
        out[((long)zi * a.nin + y0 + l) * a.MH + k] = res[l * LS + k];
    }
}

// Column transforms over slab blockIdx.x, columns kx of chunk blockIdx.y:
//   MODE 0: forward; rows t < nin in, all M rows out.
//   MODE 1: inverse; all M rows in; rows t < nout out from positions (out_off + t) mod M.
//   MODE 2: forward (rows t < nin in), product with the real-even kernel
//           spectrum at (kx, ky = slab, kz), inverse; rows as MODE 1.
template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_cfft_col(CoarseArgs a) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = a.M, CC = a.cols_cta;
    C *tw = (C *)smem_raw;
    C *A = tw + M;
    C *B = A + M * CC;
    const int q = blockIdx.x, c0 = blockIdx.y * CC, nc = min(CC, a.MH - c0);
    load_twiddles_full(tw, (const C *)a.tw, M);
    const C *in = (const C *)a.in + q * a.in_sp + c0;
    const int nrow_in = MODE == 1 ? M : a.nin;
    for (int e = threadIdx.x; e < M * CC; e += blockDim.x) {
        const int r = e / CC, c = e % CC;
        A[e] = (r < nrow_in && c < nc) ? in[r * a.in_row + c] : Cx<R>::mk(0, 0);
    }
    __syncthreads();
    C *res;
    if (MODE == 0) {
        res = fft_stockham<C, R>(A, B, CC, 1, CC, M, a.rp, tw, false);
        C *out = (C *)a.out + q * a.out_sp + c0;
        for (int e = threadIdx.x; e < M * nc; e += blockDim.x) {
            const int r = e / nc, c = e % nc;
            out[r * a.out_row + c] = res[r * CC + c];
        }
        return;
    }
    if (MODE == 2) {
        res = fft_stockham<C, R>(A, B, CC, 1, CC, M, a.rp, tw, false);
        const R *khat = (const R *)a.khat;
        const int ky = q < M - q ? q : M - q;
        for (int e = threadIdx.x; e < M * CC; e += blockDim.x) {
            const int r = e / CC, c = e % CC;
            const int kz = r < M - r ? r : M - r;
            const int kx0 = c0 + c, kx = kx0 < M - kx0 ? kx0 : M - kx0;
            C v = res[e];
            if (c < nc) {
                const R k = khat[((long)kx * a.MH + ky) * a.MH + kz];
                v.x = v.x * k;
                v.y = v.y * k;
            }
            res[e] = v;
        }
        __syncthreads();
        C *other = res == A ? B : A;
        res = fft_stockham<C, R>(res, other, CC, 1, CC, M, a.rp, tw, true);
    } else {
        res = fft_stockham<C, R>(A, B, CC, 1, CC, M, a.rp, tw, true);
    }
    C *out = (C *)a.out + q * a.out_sp + c0;
    for (int e = threadIdx.x; e < a.nout * nc; e += blockDim.x) {
        const int t = e / nc, c = e % nc;
        int pos = (a.out_off + t) % M;
        if (pos < 0) pos += M;
        out[t * a.out_row + c] = res[pos * CC + c];
    }
}

// Inverse real transform along x: row (zo, yo) of the half spectrum,
// extended by Hermitian symmetry; real outputs t < nout from positions
// (out_off + t) mod M to out[(zo nout + yo) nout + t] (type R).
template <typename R>
__global__ void __launch_bounds__(256) k_cifft_x(CoarseArgs a) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = a.M, LS = M + 1;
    C *tw = (C *)smem_raw;
    C *A = tw + M;
    C *B = A + a.lines_cta * LS;
    const int zo = blockIdx.x, y0 = blockIdx.y * a.lines_cta, nl = min(a.lines_cta, a.nout - y0);
    load_twiddles_full(tw, (const C *)a.tw, M);
    const C *in = (const C *)a.in + ((long)zo * a.nout + y0) * a.MH;
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = e / M, k = e % M;
        C v;
        if (k < a.MH) {
            v = in[l * a.MH + k];
        } else {
            v = in[l * a.MH + (M - k)];
            v.y = -v.y;
        }
        A[l * LS + k] = v;
    }
    __syncthreads();
    const C *res = fft_stockham<C, R>(A, B, nl, LS, 1, M, a.rp, tw, true);
    R *out = (R *)a.out + ((long)zo * a.nout + y0) * a.nout;
    for (int e = threadIdx.x; e < nl * a.nout; e += blockDim.x) {
        const int l = e / a.nout, t = e % a.nout;
        int pos = (a.out_off + t) % M;
        if (pos < 0) pos += M;
        out[l * a.nout + t] = res[l * LS + pos].x;
    }
}

// Radix plan of M: radix-4 stages first, then 2, 3, 5 (n = 0 if M has
// another factor).
RadixPlan radix_plan(int M) {
    RadixPlan rp{};
    int m = M;
    for (int r : {4, 2, 3, 5})
        while (m % r == 0 && rp.n < 16) {
            rp.r[rp.n++] = r;
            m /= r;
        }
    if (m != 1) rp.n = 0;
    return rp;
}

template <typename R>
size_t coarse_smem(int M, int lines) { return ((size_t)M + 2 * (size_t)lines) * sizeof(typename Cx<R>::T); }

template <typename R>
void set_cfft_attrs() {
    const int big = 220 * 1024;
    cudaFuncSetAttribute(k_cfft_x<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_cfft_col<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_cfft_col<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_cfft_col<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_cifft_x<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// The coarse solve phi^H = G^H * F^H (5 launches): forward x, forward y,
// z (forward, kernel spectrum, inverse), inverse y, inverse x.  b0, b1:
// spectra buffers (complex R); F^H FP64 in, phi^H in R out.
template <typename R>
cudaError_t run_coarse_t(const mlc_plan_s *pl, const void *khat, const void *tw, cudaStream_t st) {
    using C = typename Cx<R>::T;
    const Geom &g = pl->g;
    const int M = g.Mc, MH = g.Mhc, nin = g.nf, W = g.no;
    CoarseArgs a{};
    a.tw = tw;
    a.khat = khat;
    a.M = M;
    a.MH = MH;
    a.nin = nin;
    a.nout = W;
    a.out_off = g.olo - g.flo;
    a.rp = radix_plan(M);
    if (a.rp.n == 0) return cudaErrorInvalidValue;
    const size_t budget = 200 * 1024 / sizeof(C);  // complex entries of shared memory
    // rows per CTA of the x passes and columns per CTA of the column passes
    a.lines_cta = (int)std::min<size_t>(16, (budget - M) / (2 * (size_t)(M + 1)));
    a.cols_cta = (int)std::min<size_t>(16, (budget - M) / (2 * (size_t)M));
    if (a.lines_cta < 1 || a.cols_cta < 1) return cudaErrorInvalidValue;
    const int gx = (MH + a.cols_cta - 1) / a.cols_cta;
    const size_t smx = coarse_smem<R>(M, a.lines_cta * (M + 1)), smc = coarse_smem<R>(M, M * a.cols_cta);
    mark(pl, 6, st);
    {   // 1. forward x: F^H [zi][yi][x] -> b0 [zi][yi][kx]
        CoarseArgs b = a;
        b.in = pl->FH;
        b.out = pl->cbuf0;
        k_cfft_x<R><<<dim3(nin, (nin + a.lines_cta - 1) / a.lines_cta), 256, smx, st>>>(b);
    }
    mark(pl, 7, st);
    {   // 2. forward y: b0 [zi][yi][kx] -> b1 [zi][ky][kx]
        CoarseArgs b = a;
        b.in = pl->cbuf0;
        b.out = pl->cbuf1;
        b.in_sp = (long)nin * MH; b.in_row = MH;
        b.out_sp = (long)M * MH; b.out_row = MH;
        k_cfft_col<R, 0><<<dim3(nin, gx), 256, smc, st>>>(b);
    }
    mark(pl, 8, st);
    {   // 3. z: b1 [zi][ky][kx] -> b0 [zo][ky][kx]
        CoarseArgs b = a;
        b.in = pl->cbuf1;
        b.out = pl->cbuf0;
        b.in_sp = MH; b.in_row = (long)M * MH;
        b.out_sp = MH; b.out_row = (long)M * MH;
        k_cfft_col<R, 2><<<dim3(M, gx), 256, smc, st>>>(b);
    }
    mark(pl, 9, st);
    {   // 4. inverse y: b0 [zo][ky][kx] -> b1 [zo][yo][kx]
        CoarseArgs b = a;
        b.in = pl->cbuf0;
        b.out = pl->cbuf1;
        b.in_sp = (long)M * MH; b.in_row = MH;
        b.out_sp = (long)W * MH; b.out_row = MH;
        k_cfft_col<R, 1><<<dim3(W, gx), 256, smc, st>>>(b);
    }
    mark(pl, 10, st);
    {   // 5. inverse x: b1 [zo][yo][kx] -> phi^H [zo][yo][xo]
        CoarseArgs b = a;
        b.in = pl->cbuf1;
        b.out = pl->phiH;
        k_cifft_x<R><<<dim3(W, (W + a.lines_cta - 1) / a.lines_cta), 256, smx, st>>>(b);
    }
    return cudaGetLastError();
}

template <typename R>
inline size_t fft_smem_bytes(int M, int lines, int ls) {
    return ((size_t)(M / 2) + (size_t)lines * ls) * 2 * sizeof(R);
}

// Local-convolution (patch) kernels in working precision R.
// Largest dynamic shared memory of the 16-byte-entry M = 128 slab and
// inverse-x launches: the 227 KB opt-in limit of an sm_100-class SM less room
// for the kernels' static shared memory (the attribute cannot exceed the
// difference).
constexpr size_t kSlabRowsSmem = 225 * 1024;

template <int LOG2M, typename R>
void set_patch_attrs() {
    const int big = 200 * 1024;
    if constexpr (LOG2M == 7 && !std::is_same<R, float>::value) {
        cudaFuncSetAttribute(k_slab_rows<LOG2M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabRowsSmem);
        cudaFuncSetAttribute(k_inv_x_pruned<LOG2M, R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabRowsSmem);
        cudaFuncSetAttribute(k_fwd_x<LOG2M, double, true, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
        return;
    }
    cudaFuncSetAttribute(k_fwd_x<LOG2M, double, true, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fwd_x<LOG2M, float, true, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_slab<LOG2M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if constexpr (!std::is_same<R, float>::value)
        cudaFuncSetAttribute(k_slab64<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_slab64r<17>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_slab64r<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_inv_x_pruned<LOG2M, R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_inv_x64<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// Local convolutions of a set of patches: forward x (real), fused slab (y,
// z, kernel spectrum, inverse z, inverse y), pruned inverse x.  3 launches.
template <int LOG2M, typename R>
cudaError_t run_patch_conv_t(const mlc_plan_s *pl, const Items &it, bool f32, const void *tw,
                             cudaStream_t st) {
    constexpr int M = 1 << LOG2M, MH = M / 2 + 1;
    const Geom &g = pl->g;
    const int nin = g.nb, W = g.W, nb = it.nitems;
    mark(pl, 1, st);
    {
        FwdXArgs a{nullptr, nullptr, 0, g.n, 0, nin, nin, tw, it};
        if (LOG2M == 6 && nin <= 24) {  // register transform of line pairs
            if (f32) k_fwd_x64<float, R><<<nb, 256, 0, st>>>(a);
            else k_fwd_x64<double, R><<<nb, 256, 0, st>>>(a);
        } else {
            dim3 grid(nb * nin, 1);
            size_t sm = fft_smem_bytes<R>(M, nin, M + 1);
            if (f32) k_fwd_x<LOG2M, float, true, R, true><<<grid, 256, sm, st>>>(a);
            else k_fwd_x<LOG2M, double, true, R, true><<<grid, 256, sm, st>>>(a);
        }
    }
    int nz = 0, zrow[128];
    for (int zi = 0; zi < W; ++zi) {
        const int z = zi - g.s;
        if ((z >= -g.ga && z <= g.n + g.ga) || (z % 4 == 0)) zrow[nz++] = zi;
    }
    mark(pl, 2, st);
    {
        SlabArgs a{tw, nin, W, -g.s, it, nz, {}, g.a4blk};
        for (int j = 0; j < nz; ++j) a.zrow[j] = zrow[j];
        if (LOG2M == 6) {
            int dev = 0, nsm = 0, occ = 0;
            if (it.persist) {  // one wave of resident CTAs walking all slabs
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            }
            if constexpr (std::is_same<R, float>::value) {  // split tier: one line per thread
                const size_t smr = (size_t)M * 65 * sizeof(float2);
                int gr = nb * MH;
                if (it.persist) {
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_slab64r<32>, 64, smr);
                    const int wave = nsm * (occ > 0 ? occ : 1);
                    gr = gr < wave ? gr : wave;
                }
                if (nin <= 17) k_slab64r<17><<<gr, 64, smr, st>>>(a);
                else k_slab64r<32><<<gr, 64, smr, st>>>(a);
            } else if (nin > 24) {  // k_slab64's sparse forward passes take nin <= 24 (n = 24)
                k_slab<LOG2M, R><<<nb * MH, 256, fft_smem_bytes<R>(M, M, M + 1), st>>>(a);
            } else {  // FP64 and double-float: radix 8 x 8 over 8-thread groups
                const size_t sm = (size_t)(M + M * Pitch64<R>::P + 32 * 72) * sizeof(typename Cx<R>::T) + 64 * sizeof(int);
                int grid = nb * MH;
                if (it.persist) {
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_slab64<R>, 256, sm);
                    const int wave = nsm * (occ > 0 ? occ : 1);
                    grid = grid < wave ? grid : wave;
                }
                k_slab64<R><<<grid, 256, sm, st>>>(a);
            }
        }
        else {
            if constexpr (LOG2M == 7 && std::is_same<R, float>::value) {  // FP32: register lines
                const size_t sm = ((size_t)144 + 32 * 152 + (size_t)std::max(nin, nz) * (M + 1)) * sizeof(float2);
                int gr = nb * MH;
                if (it.persist) {
                    int dev = 0, nsm = 0, occ = 0;
                    cudaGetDevice(&dev);
                    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_slab128r, 256, sm);
                    const int wave = nsm * (occ > 0 ? occ : 1);
                    gr = gr < wave ? gr : wave;
                }
                k_slab128r<<<gr, 256, sm, st>>>(a);
            } else if constexpr (LOG2M == 7 && sizeof(R) == 8) {  // 16-byte entries: row-streamed slab
                const int sw = std::max(nin, nz);
                const size_t csz = 2 * sizeof(R), fixed = ((size_t)M / 2 + (size_t)M * sw) * csz;
                const int rb = (int)std::min<size_t>(M, (kSlabRowsSmem - fixed) / ((M + 1) * csz));
                if (rb < 1) return cudaErrorInvalidValue;
                k_slab_rows<LOG2M, R><<<nb * MH, 256, fixed + (size_t)rb * (M + 1) * csz, st>>>(a, sw, rb);
            } else {
                k_slab<LOG2M, R><<<nb * MH, 256, fft_smem_bytes<R>(M, M, M + 1), st>>>(a);
            }
        }
    }
    mark(pl, 3, st);
    {
        InvXPArgs a{it, tw, g.n, g.s, W, g.ga, g.npa, g.pl0, g.wa, g.nc, nz, {}, 0, g.a4blk, 1 << 22, 0};
        if (pl->fault == 1) {  // test hook: the wait must run out, quickly
            a.skip_copy = 1;
            a.wait_tries = 64;
        }
        for (int j = 0; j < nz; ++j) a.zrow[j] = zrow[j];
        a.outer = g.wide ? 1 : 0;
        // rows needing a full transform, per z row (the same rule as the kernel)
        auto inA = [&](int c) { return c >= -g.ga && c <= g.n + g.ga; };
        auto onP = [&](int c) { return inA(c) && ((c - g.pl0) % g.n) == 0; };
        auto onO = [&](int c) {  // one node off an alpha face plane (the kernel's off_slot)
            if (!g.wide || !inA(c)) return false;
            for (int d : {c + 1 - g.pl0, c - 1 - g.pl0})
                if (d >= 0 && d % g.n == 0 && d / g.n < g.npa) return true;
            return false;
        };
        for (int j = 0; j < nz; ++j) {
            const int z = zrow[j] - g.s;
            int cnt = 0;
            for (int yi = 0; yi < W; ++yi) {
                const int y = yi - g.s;
                if (((onP(z) || onO(z)) && inA(y)) || ((onP(y) || onO(y)) && inA(z)) || ((z & 3) == 0 && (y & 3) == 0))
                    ++cnt;
            }
            a.maxfft = cnt > a.maxfft ? cnt : a.maxfft;
        }
        const int LPh = LOG2M == 6 ? Pitch64<R>::P : M + 1;
        const size_t xsn = (LOG2M == 6 && UseXs<R>::v) ? 32 * 72 : 0;
        // transformed rows per pass: all of them unless the line buffer would
        // not fit beside the staged block (16-byte entries at M = 128)
        const size_t fixed = ((size_t)M + (size_t)g.a4blk + xsn) * 2 * sizeof(R);
        const size_t line = (size_t)LPh * 2 * sizeof(R);
        a.rb = a.maxfft;
        if (fixed + (size_t)a.rb * line > kSlabRowsSmem) a.rb = (int)((kSlabRowsSmem - fixed) / line);
        if (a.rb < 1) return cudaErrorInvalidValue;
        const size_t sm = fixed + (size_t)a.rb * line;
        // local fields leave in the working precision: FP32 (split tier) or
        // double-float pairs (FP64 tier)
        if (LOG2M == 6 && !g.wide) {
            const int thr = 128;  // 16 line groups: one pass over the row pairs of a z row
            const size_t sm64 = ((size_t)M + (size_t)g.a4blk + (thr / 8) * 72) * sizeof(typename Cx<R>::T) +
                                (size_t)a.maxfft * 68 * sizeof(R);
            k_inv_x64<R><<<nb * a.nz, thr, sm64, st>>>(a);
        } else {
            k_inv_x_pruned<LOG2M, R, R><<<nb * a.nz, 256, sm, st>>>(a);
        }
    }
    return cudaGetLastError();
}

void stencil_b(int Q, double b[4]) {
    if (Q == 4) {
        b[0] = -4.0; b[1] = 1.0 / 3.0; b[2] = 1.0 / 6.0; b[3] = 0.0;
    } else {
        b[0] = -64.0 / 15.0; b[1] = 7.0 / 15.0; b[2] = 1.0 / 10.0; b[3] = 1.0 / 30.0;
    }
}

}  // namespace

__global__ void k_set_ptrs(PlanPtrs *d, const void *f, double *phi) {
    d->f = f;
    d->phi = phi;
}

cudaError_t launch_set_ptrs(PlanPtrs *d, const void *f, double *phi, cudaStream_t st) {
    k_set_ptrs<<<1, 1, 0, st>>>(d, f, phi);
    return cudaGetLastError();
}

void configure_kernels() {
    set_patch_attrs<5, dfl>();
    set_patch_attrs<6, dfl>();
    set_patch_attrs<5, float>();
    set_patch_attrs<6, float>();
    set_patch_attrs<5, double>();
    set_patch_attrs<6, double>();
    set_patch_attrs<7, float>();
    cudaFuncSetAttribute(k_slab128r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabRowsSmem);
    set_patch_attrs<7, double>();
    set_patch_attrs<7, dfl>();
    set_cfft_attrs<dfl>();
    set_cfft_attrs<double>();
    configure_ring_gemm();
    const int big = 200 * 1024;
#define MLC_DIR_ATTR(NN)                                                                          \
    cudaFuncSetAttribute(k_dirichlet<double, NN, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); \
    cudaFuncSetAttribute(k_dirichlet<float, NN, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);  \
    cudaFuncSetAttribute(k_dirichlet<double, NN, dfl>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);    \
    cudaFuncSetAttribute(k_dirichlet<float, NN, dfl>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    MLC_DIR_ATTR(4)
    MLC_DIR_ATTR(8)
    MLC_DIR_ATTR(12)
    MLC_DIR_ATTR(16)
    MLC_DIR_ATTR(24)
    MLC_DIR_ATTR(32)
#undef MLC_DIR_ATTR
#define MLC_RES_ATTR(KK)                                                                            \
    cudaFuncSetAttribute(k_resid<dfl, dfl, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);    \
    cudaFuncSetAttribute(k_resid<float, dfl, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);  \
    cudaFuncSetAttribute(k_resid<float, double, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); \
    cudaFuncSetAttribute(k_resid<double, double, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    MLC_RES_ATTR(4)
    MLC_RES_ATTR(6)
    MLC_RES_ATTR(8)
    MLC_RES_ATTR(10)
    MLC_RES_ATTR(12)
#undef MLC_RES_ATTR
    cudaFuncSetAttribute(k_moments<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_moments<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    configure_wide();
}

cudaError_t launch_moments(const mlc_plan_s *pl, const Items &it, cudaStream_t st) {
    NvtxRange nvtx("mlc:moments");
    const Geom &g = pl->g;
    const int nb = g.n + 1;
    // charge planes staged at once: the whole patch while it takes <= 48 KB
    const int ns = std::max(1, std::min(nb, (int)((48u << 10) / ((g.f32in ? 4 : 8) * (size_t)nb * nb))));
    const size_t words = (size_t)ns * nb * nb + (size_t)g.P * nb * nb + (size_t)g.P * g.P * nb + (size_t)g.P * nb;
    if (g.f32in)
        k_moments<float, float><<<it.nitems, 256, words * sizeof(float), st>>>(it, g.n, g.P, g.npoly, g.npad, ns);
    else
        k_moments<double, double><<<it.nitems, 256, words * sizeof(double), st>>>(it, g.n, g.P, g.npoly, g.npad, ns);
    return cudaGetLastError();
}

// The three local-convolution launches for one launch group of items (its
// scratch in it.a1 / it.a4).
cudaError_t launch_patch_conv_group(const mlc_plan_s *pl, const Items &it, cudaStream_t st) {
    NvtxRange nvtx("mlc:local_convolutions");
    const Geom &g = pl->g;
    const bool f32 = g.f32in;
    if (g.conv == CONV_F32) {  // split tiers: FP32 (tables tw_f, khat_f)
        if (g.log2M == 5) return run_patch_conv_t<5, float>(pl, it, f32, pl->tw_f, st);
        if (g.log2M == 6) return run_patch_conv_t<6, float>(pl, it, f32, pl->tw_f, st);
        if (g.log2M == 7) return run_patch_conv_t<7, float>(pl, it, f32, pl->tw_f, st);
    } else if (g.conv == CONV_DF) {  // double-float (tables tw_df, khat_df)
        if (g.log2M == 5) return run_patch_conv_t<5, dfl>(pl, it, f32, pl->tw_df, st);
        if (g.log2M == 6) return run_patch_conv_t<6, dfl>(pl, it, f32, pl->tw_df, st);
        if (g.log2M == 7) return run_patch_conv_t<7, dfl>(pl, it, f32, pl->tw_df, st);
    } else {  // FP64 (tables tw, khat)
        if (g.log2M == 5) return run_patch_conv_t<5, double>(pl, it, f32, pl->tw, st);
        if (g.log2M == 6) return run_patch_conv_t<6, double>(pl, it, f32, pl->tw, st);
        if (g.log2M == 7) return run_patch_conv_t<7, double>(pl, it, f32, pl->tw, st);
    }
    return cudaErrorInvalidValue;
}

// Local convolutions of all items, in launch groups of g.chunk items that
// reuse one scratch (stream order keeps the groups apart).
cudaError_t launch_patch_conv(const mlc_plan_s *pl, const Items &it, cudaStream_t st) {
    const int chunk = it.chunk > 0 ? it.chunk : pl->g.chunk;
    for (int c0 = 0; c0 < it.nitems; c0 += chunk) {
        Items ic = it;
        ic.nitems = it.nitems - c0 < chunk ? it.nitems - c0 : chunk;
        if (it.items) ic.items = it.items + c0;
        else ic.first = it.first + c0;
        const cudaError_t e = launch_patch_conv_group(pl, ic, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Lagrange weights of I^H on the nodes k0-b .. k0+b+1 at t = k0 + r/4 (R4 reading).
void lagrange_rows(int b, double lw[4][12]) {
    const int K = 2 * b + 2;
    for (int r = 0; r < 4; ++r)
        for (int j = 0; j < 12; ++j) lw[r][j] = 0.0;
    for (int r = 1; r < 4; ++r)
        for (int j = 0; j < K; ++j) {
            double w = 1.0;
            const double t = r / 4.0 + b;  // position relative to the first node
            for (int l = 0; l < K; ++l)
                if (l != j) w *= (t - l) / (double)(j - l);
            lw[r][j] = w;
        }
}

// Lagrange weights as double-float pairs (host).
void lagrange_rows_df(int b, dfl out[4][12]) {
    double lw[4][12];
    lagrange_rows(b, lw);
    for (int r = 0; r < 4; ++r)
        for (int j = 0; j < 12; ++j) {
            const float hi = (float)lw[r][j];
            out[r][j] = dfl(hi, (float)(lw[r][j] - (double)hi));
        }
}
dfl host_df(double v) {
    const float hi = (float)v;
    return dfl(hi, (float)(v - (double)hi));
}

// Moments in the ring precision of the tier (the local-convolution arithmetic).
const void *ring_moments(const mlc_plan_s *pl) {
    const Geom &g = pl->g;
    return g.conv == CONV_F32 ? (const void *)pl->mom_f
           : (g.conv == CONV_DF ? (const void *)pl->mom_df : (const void *)pl->mom);
}

cudaError_t launch_resid(const mlc_plan_s *pl, const Items &it, cudaStream_t st) {
    NvtxRange nvtx("mlc:residuals");
    const Geom &g = pl->g;
    ResArgs a{};
    a.it = it; a.n = g.n; a.s = g.s; a.ga = g.ga; a.b = g.b;
    a.npa = g.npa; a.pl0 = g.pl0; a.wa = g.wa; a.nc = g.nc;
    lagrange_rows_df(g.b, a.lw);
    lagrange_rows(g.b, a.lwd);
    const int nk = (g.n + 2 * g.ga) / 4 + 2 * g.b + 1;
    const size_t sm = 8 * (size_t)nk * (g.wa + nk);
    dim3 grid(it.nitems, 3 * g.npa);
#define MLC_RES(KK)                                                                         \
    if (g.fine == FINE_F64) {                                                               \
        if (g.conv == CONV_F32) k_resid<float, double, KK><<<grid, 256, sm, st>>>(a);       \
        else k_resid<double, double, KK><<<grid, 256, sm, st>>>(a);                         \
    } else {                                                                                \
        if (g.conv == CONV_F32) k_resid<float, dfl, KK><<<grid, 256, sm, st>>>(a);          \
        else k_resid<dfl, dfl, KK><<<grid, 256, sm, st>>>(a);                               \
    }
    switch (2 * g.b + 2) {
        case 4: MLC_RES(4) break;
        case 6: MLC_RES(6) break;
        case 8: MLC_RES(8) break;
        case 10: MLC_RES(10) break;
        case 12: MLC_RES(12) break;
        default: return cudaErrorInvalidValue;
    }
#undef MLC_RES
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_resid_outer(pl, it, st);  // Q = 10: the second layer (no-op otherwise)
}

cudaError_t launch_assemble(const mlc_plan_s *pl, cudaStream_t st) {
    NvtxRange nvtx("mlc:coarse_charge");
    const Geom &g = pl->g;
    AsmArgs a{};
    a.err = pl->err;
    a.cl = pl->cl; a.FH = pl->FH;
    a.mom = ring_moments(pl);
    a.T = pl->Ttab;
    a.np = g.np; a.n = g.n; a.s = g.s; a.nc = g.nc; a.npoly = g.npoly; a.npad = g.npad; a.flo = g.flo; a.nf = g.nf;
    a.ca_lo = g.ca_lo; a.ca_hi = g.ca_hi; a.cb_lo = g.cb_lo; a.cb_hi = g.cb_hi;
    double b[4];
    stencil_b(g.Q, b);
    for (int k = 0; k < 4; ++k) {
        a.coef[k] = host_df(b[k] / (g.H * g.H));
        a.coefd[k] = b[k] / (g.H * g.H);
    }
    a.wide = g.wide ? 1 : 0;
    a.invH2 = 1.0 / (g.H * g.H);
    const long tot = (long)g.nf * g.nf * g.nf;
    const unsigned nbk = (unsigned)((tot + 127) / 128);
    if (g.conv == CONV_F32) {
        if (g.fine == FINE_F64) k_assemble<float, float, double><<<nbk, 128, 0, st>>>(a);
        else k_assemble<float, float, dfl><<<nbk, 128, 0, st>>>(a);
    } else if (g.conv == CONV_DF) {
        k_assemble<dfl, dfl, dfl><<<nbk, 128, 0, st>>>(a);
    } else {
        k_assemble<double, double, double><<<nbk, 128, 0, st>>>(a);
    }
    return cudaGetLastError();
}

// Sec. 5: F^H (nf^3 from flo) into the coarser level's charge array (node
// off = flo - c0 of its grid, side Nc), in that level's charge precision.
template <typename TF>
__global__ void __launch_bounds__(256) k_fh_to_level(const double *FH, int nf, int off, int Nc, TF *fc, int *err) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nf * nf * nf) return;
    const int x = (int)(idx % nf), y = (int)((idx / nf) % nf), z = (int)(idx / ((long)nf * nf));
    if (in_range(z + off, Nc, err) & in_range(y + off, Nc, err) & in_range(x + off, Nc, err))
        fc[((long)(z + off) * Nc + (y + off)) * Nc + (x + off)] = (TF)FH[idx];
}

// phi^H (no^3 from olo) from the coarser level's result (node off = olo - c0).
template <typename T>
__global__ void __launch_bounds__(256) k_level_to_phiH(const double *pc, int Nc, int off, int no, T *phiH, int *err) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)no * no * no) return;
    const int x = (int)(idx % no), y = (int)((idx / no) % no), z = (int)(idx / ((long)no * no));
    if (in_range(z + off, Nc, err) & in_range(y + off, Nc, err) & in_range(x + off, Nc, err))
        phiH[idx] = FT<T>::of(pc[((long)(z + off) * Nc + (y + off)) * Nc + (x + off)]);
}

// Sec. 5: the coarse solve of a multilevel plan, an MLC solve of F^H on the
// next coarser level (its own plan, on this stream).
cudaError_t run_coarse_level(const mlc_plan_s *pl, cudaStream_t st) {
    const Geom &g = pl->g;
    mlc_plan_s *ch = pl->child;
    const int Nc = ch->g.N;
    mark(pl, 6, st);
    const long nf3 = (long)g.nf * g.nf * g.nf, no3 = (long)g.no * g.no * g.no;
    const int off_f = g.flo - pl->child_c0, off_o = g.olo - pl->child_c0;
    if (g.f32in)
        k_fh_to_level<float><<<(unsigned)((nf3 + 255) / 256), 256, 0, st>>>(pl->FH, g.nf, off_f, Nc, (float *)pl->child_f, pl->err);
    else
        k_fh_to_level<double><<<(unsigned)((nf3 + 255) / 256), 256, 0, st>>>(pl->FH, g.nf, off_f, Nc, (double *)pl->child_f, pl->err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mlc_solve(ch, pl->child_f, pl->child_phi, st) != MLC_OK) {
        e = cudaGetLastError();
        return e != cudaSuccess ? e : cudaErrorUnknown;
    }
    mark(pl, 7, st);
    if (g.fine == FINE_F64)
        k_level_to_phiH<double><<<(unsigned)((no3 + 255) / 256), 256, 0, st>>>(pl->child_phi, Nc, off_o, g.no, (double *)pl->phiH, pl->err);
    else
        k_level_to_phiH<dfl><<<(unsigned)((no3 + 255) / 256), 256, 0, st>>>(pl->child_phi, Nc, off_o, g.no, (dfl *)pl->phiH, pl->err);
    mark(pl, 8, st);
    mark(pl, 9, st);
    mark(pl, 10, st);
    return cudaGetLastError();
}

cudaError_t launch_coarse(const mlc_plan_s *pl, cudaStream_t st) {
    NvtxRange nvtx("mlc:coarse_solve");
    if (pl->child) return run_coarse_level(pl, st);
    if (pl->g.fine == FINE_F64)  // coarse FFTs in FP64
        return run_coarse_t<double>(pl, pl->khat_c, pl->tw_c, st);
    return run_coarse_t<dfl>(pl, pl->khat_c_df, pl->tw_c_df, st);  // in double-float arithmetic
}

cudaError_t launch_boundary(const mlc_plan_s *pl, cudaStream_t st) {
    NvtxRange nvtx("mlc:boundary");
    const Geom &g = pl->g;
    BndArgs a{};
    a.err = pl->err;
    a.phiH = pl->phiH; a.resid = pl->resid;
    a.mom = ring_moments(pl);
    a.D = pl->Dtab;
    a.phiB = pl->phiB;
    a.pb0 = g.pb0; a.npb = g.npb;
    a.N = g.N; a.n = g.n; a.np = g.np; a.ga = g.ga; a.gb = g.gb; a.b = g.b; a.npoly = g.npoly;
    a.olo = g.olo; a.no = g.no; a.wa = g.wa; a.wbx = g.wbx; a.npa = g.npa; a.pl0 = g.pl0;
    a.npad = g.npad;
    lagrange_rows_df(g.b, a.lw);
    lagrange_rows(g.b, a.lwd);
    a.tpl = pl->tpl;
    {   // sums along v of I^H(phi^H) per (plane, coarse row)
        const long tp = 3L * (g.np + 1) * g.no * (g.N + 1);
        const unsigned nb2 = (unsigned)((tp + 255) / 256);
        LagW w;
        std::memcpy(w.lw, a.lw, sizeof(w.lw));
        std::memcpy(w.lwd, a.lwd, sizeof(w.lwd));
        if (g.fine == FINE_F64)
            k_plane_interp<double><<<nb2, 256, 0, st>>>(pl->phiH, pl->tpl, g.N, g.n, g.np, g.b, g.olo, g.no, w, pl->err);
        else
            k_plane_interp<dfl><<<nb2, 256, 0, st>>>(pl->phiH, pl->tpl, g.N, g.n, g.np, g.b, g.olo, g.no, w, pl->err);
    }
    a.ringR = pl->ring_R;
    a.ring_rows_pad = g.ring_rows_pad;
    const long per_axis = (long)(g.np + 1) * g.plane_n;
    // split tiers with a Legendre ring: one ring GEMM and one boundary launch
    // per face-plane axis (the GEMM's output holds one axis at a time)
    const bool gemm = g.conv == CONV_F32 && pl->ring_R != nullptr && pl->ring_aimg != nullptr;
    for (int axis = 0; axis < 3; ++axis) {
        if (!gemm && axis > 0) break;
        a.idx0 = gemm ? axis * per_axis : 0;
        a.idx1 = gemm ? (axis + 1) * per_axis : g.n_planes_total;
        if (gemm) {
            const cudaError_t e = launch_ring_gemm(pl, axis, st);
            if (e != cudaSuccess) return e;
        }
        const unsigned nbk = (unsigned)((a.idx1 - a.idx0 + 127) / 128);
#define MLC_BND(NN)                                                                                        \
        case NN:                                                                                           \
            if (gemm && g.fine == FINE_F64) k_boundary<float, NN, double, true><<<nbk, 128, 0, st>>>(a);   \
            else if (gemm) k_boundary<float, NN, dfl, true><<<nbk, 128, 0, st>>>(a);                        \
            else if (g.conv == CONV_F32 && g.fine == FINE_F64) k_boundary<float, NN, double><<<nbk, 128, 0, st>>>(a); \
            else if (g.conv == CONV_F32) k_boundary<float, NN, dfl><<<nbk, 128, 0, st>>>(a);                 \
            else if (g.conv == CONV_DF) k_boundary<dfl, NN, dfl><<<nbk, 128, 0, st>>>(a);                    \
            else k_boundary<double, NN, double><<<nbk, 128, 0, st>>>(a);                                     \
            break;
        switch (g.n) {
            MLC_BND(4)
            MLC_BND(8)
            MLC_BND(12)
            MLC_BND(16)
            MLC_BND(24)
            MLC_BND(32)
            default: return cudaErrorInvalidValue;
        }
#undef MLC_BND
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_boundary_outer(pl, st);  // Q = 10: the second layer (no-op otherwise)
}

cudaError_t launch_dirichlet(const mlc_plan_s *pl, const Items &it, cudaStream_t st) {
    if (pl->g.wide) return launch_dirichlet_wide(pl, it, st);
    NvtxRange nvtx("mlc:dirichlet");
    const Geom &g = pl->g;
    DirArgs a{};
    a.it = it; a.n = g.n;
    stencil_b(g.Q, a.b);
    a.sinm = pl->sinm;
    const int nb = g.n + 1, m = g.n - 1;
    const size_t sm = 8 * (6 * (size_t)nb * nb + (g.n > 24 ? 0 : (size_t)m * m * m) + (size_t)m * (g.n / 2));
#define MLC_DIR(NN)                                                                               \
    case NN:                                                                                      \
        if (g.fine == FINE_F64) {                                                                 \
            if (g.f32in) k_dirichlet<float, NN, double><<<it.nitems, 256, sm, st>>>(a);           \
            else k_dirichlet<double, NN, double><<<it.nitems, 256, sm, st>>>(a);                  \
        } else {                                                                                  \
            if (g.f32in) k_dirichlet<float, NN, dfl><<<it.nitems, 256, sm, st>>>(a);              \
            else k_dirichlet<double, NN, dfl><<<it.nitems, 256, sm, st>>>(a);                     \
        }                                                                                         \
        break;
    switch (g.n) {
        MLC_DIR(4)
        MLC_DIR(8)
        MLC_DIR(12)
        MLC_DIR(16)
        MLC_DIR(24)
        MLC_DIR(32)
        default: return cudaErrorInvalidValue;
    }
#undef MLC_DIR
    return cudaGetLastError();
}

// Index export (test hook): which = 0 face-plane nodes, 1 coarse nodes of
// the F^H extent; cnt != nullptr: count pass, else fill pass.
cudaError_t launch_index_export(const mlc_plan_s *pl, int which, int *cnt, const long *off, int *ent,
                                cudaStream_t st) {
    const Geom &g = pl->g;
    if (which == 1) {
        const long tot = (long)g.nf * g.nf * g.nf;
        const unsigned nbk = (unsigned)((tot + 127) / 128);
        if (cnt) k_index_coarse<true><<<nbk, 128, 0, st>>>(g.n, g.np, g.ca_lo, g.ca_hi, g.cb_lo, g.cb_hi, g.flo, g.nf, cnt, off, ent);
        else k_index_coarse<false><<<nbk, 128, 0, st>>>(g.n, g.np, g.ca_lo, g.ca_hi, g.cb_lo, g.cb_hi, g.flo, g.nf, cnt, off, ent);
        return cudaGetLastError();
    }
    const long tot = g.n_planes_total;
    const unsigned nbk = (unsigned)((tot + 127) / 128);
#define MLC_IDX(NN)                                                                                    \
    case NN:                                                                                           \
        if (cnt) k_index_face<NN, true><<<nbk, 128, 0, st>>>(g.N, g.np, g.ga, g.gb, tot, cnt, off, ent);  \
        else k_index_face<NN, false><<<nbk, 128, 0, st>>>(g.N, g.np, g.ga, g.gb, tot, cnt, off, ent);     \
        break;
    switch (g.n) {
        MLC_IDX(4)
        MLC_IDX(8)
        MLC_IDX(12)
        MLC_IDX(16)
        MLC_IDX(24)
        MLC_IDX(32)
        default: return cudaErrorInvalidValue;
    }
#undef MLC_IDX
    return cudaGetLastError();
}

#include "wide.cuh"

}  // namespace mlc
