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
// routine at all.  Every step runs on the caller's stream (no side stream, so
// the moments and residuals do not overlap the convolution chain as they do in
// mlc_solve).
//
// The array is kNoAllocScratchBytes (64 MiB) on every GPU that loads this
// library and is held until the process exits.  Every call shares it and
// finds the previous call's contents there; nothing in it needs to start at
// zero, because each call writes every scratch element it later reads.  Calls
// that overlap on the GPU (on different streams, or with different plans)
// race on the array and must not be issued.  The first call on a device
// resolves the array's device address (cudaGetSymbolAddress) with that device
// current; make that first call before any stream capture begins.
#include <algorithm>
#include <mutex>

#include "mlc_internal.h"

using namespace mlc;

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

// Scratch of the local convolutions for one launch group of patches (the
// plan's group size, or all its patches if fewer): the x-transformed charges
// followed by the slab outputs (the layout of the plan's own scratch).
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

}  // namespace

extern "C" mlc_status mlc_solve_noalloc(mlc_plan_t pl, const void *f, void *phi, void *stream) {
    if (!pl || !f || !phi || f == phi) return MLC_ERR_INVALID_ARG;
    const long items = std::min<long>(pl->g.chunk, pl->g.NP);  // patches per launch group
    if (conv_scratch_bytes(pl->g, items) > kNoAllocScratchBytes) return MLC_ERR_INVALID_ARG;
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
    k_store_record<<<1, 1, 0, st>>>(addr.record, rec);
    if (cudaGetLastError() != cudaSuccess) return MLC_ERR_CUDA;
    Items it{nullptr, addr.record, pl->g.NP};
    it.a1 = addr.scratch;
    it.a4 = addr.scratch + conv_scratch_a4_offset(pl->g, items);
    if (launch_moments(pl, it, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_patch_conv(pl, it, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_resid(pl, it, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_assemble(pl, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_coarse(pl, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_boundary(pl, st) != cudaSuccess) return MLC_ERR_CUDA;
    if (launch_dirichlet(pl, it, st) != cudaSuccess) return MLC_ERR_CUDA;
    return MLC_OK;
}
