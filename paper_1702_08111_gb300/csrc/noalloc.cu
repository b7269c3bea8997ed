// mlc_solve_noalloc: a solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they solve: a plugin
// whose host application owns and has already reserved the device memory, or
// code that runs while a CUDA graph is being captured in global mode, where
// allocation calls are not permitted.  For them this entry point runs the same
// steps as mlc_solve with the plan created beforehand, but takes the scratch of
// the local-convolution kernels (the patch spectra between the forward and the
// inverse transforms, the largest scratch of a solve) from a file-scope static
// device array instead of the plan's workspace, and it calls no allocating
// routine at all.
//
// The array is kNoAllocScratchBytes (64 MiB) on every GPU that loads this
// library and is held until the process exits.  Every call shares it and
// finds the previous call's contents there; nothing in it needs to start at
// zero, because each call writes every scratch element it later reads.  Calls
// that overlap on the GPU (on different streams, or with different plans)
// race on the array and must not be issued.  The first call on a device
// resolves the array's device address (cudaGetSymbolAddress) with that device
// current; make that first call before any stream capture begins.
#include <mutex>

#include "mlc_internal.h"

using namespace mlc;

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

// Scratch of the local convolutions: the x-transformed charges of every patch
// followed by the slab outputs (the layouts of the plan's own workspace).
static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];
// The per-patch kernels read their plan record from device memory.
static __device__ __align__(256) PlanPtrs g_record;

struct DevAddr {
    unsigned char *scratch = nullptr;
    PlanPtrs *record = nullptr;
};
DevAddr g_addr[kMaxDevices];
std::mutex g_addr_mu;

__global__ void k_store_record(PlanPtrs *dst, PlanPtrs rec) { *dst = rec; }

// Bytes of the two spectra buffers for this plan (as the plan sizes them),
// each rounded up to 256 bytes.
size_t scratch_bytes(const Geom &G, size_t *a1_bytes) {
    const size_t rb = conv_real_bytes(G.tier);
    const size_t A1 = (size_t)G.NP * G.nb * G.nb * G.Mh * 2 * rb;
    const size_t A4 = (size_t)G.NP * G.nzr * G.a4blk * 2 * rb;
    const size_t a1r = (A1 + 255) & ~(size_t)255;
    *a1_bytes = a1r;
    return a1r + ((A4 + 255) & ~(size_t)255);
}

}  // namespace

extern "C" mlc_status mlc_solve_noalloc(mlc_plan_t pl, const void *f, void *phi, void *stream) {
    if (!pl || !f || !phi || f == phi) return MLC_ERR_INVALID_ARG;
    size_t a1_bytes = 0;
    if (scratch_bytes(pl->g, &a1_bytes) > kNoAllocScratchBytes) return MLC_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MLC_ERR_CUDA;
    if (dev != pl->device) return MLC_ERR_INVALID_ARG;
    DevAddr addr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev].scratch) {
            void *s = nullptr, *r = nullptr;
            if (cudaGetSymbolAddress(&s, g_scratch) != cudaSuccess) return MLC_ERR_CUDA;
            if (cudaGetSymbolAddress(&r, g_record) != cudaSuccess) return MLC_ERR_CUDA;
            g_addr[dev].scratch = (unsigned char *)s;
            g_addr[dev].record = (PlanPtrs *)r;
        }
        addr = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    PlanPtrs rec = pl->hptrs;
    rec.f = f;
    rec.phi = (double *)phi;
    rec.a1 = addr.scratch;
    rec.a4 = addr.scratch + a1_bytes;
    k_store_record<<<1, 1, 0, st>>>(addr.record, rec);
    if (cudaGetLastError() != cudaSuccess) return MLC_ERR_CUDA;
    const Items it{nullptr, addr.record, pl->g.NP};
    if (launch_moments(pl, it, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_patch_conv(pl, it, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_resid(pl, it, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_assemble(pl, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_coarse(pl, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_boundary(pl, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_dirichlet(pl, it, st) != cudaSuccess) return MLC_ERR_CUDA;
    return MLC_OK;
}
