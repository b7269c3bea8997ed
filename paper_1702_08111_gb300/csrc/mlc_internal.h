// Internal declarations of the MLC library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/mlc.h"

namespace mlc {

// Launches of one solve, in order (the timing slots of mlc_debug_timing).
constexpr int kTimedLaunches = 13;

// Arithmetic of each tier (include/mlc.h): the local convolutions ("conv":
// spectra, twiddles, local fields) and the steps after them ("fine": coarse
// charge, coarse solve, residuals, boundary values, Dirichlet solves).
enum ConvPrec { CONV_F64 = 0, CONV_DF = 1, CONV_F32 = 2 };
enum FinePrec { FINE_F64 = 0, FINE_DF = 1 };
inline bool tier_valid(int t) { return t >= MLC_TIER_FP64 && t <= MLC_TIER_SPLIT_DF; }
inline int tier_conv(int t) {
    return t == MLC_TIER_FP64 ? CONV_F64 : (t == MLC_TIER_DF ? CONV_DF : CONV_F32);
}
inline int tier_fine(int t) { return (t == MLC_TIER_FP64 || t == MLC_TIER_SPLIT) ? FINE_F64 : FINE_DF; }
inline bool tier_f32_charge(int t) { return t == MLC_TIER_SPLIT || t == MLC_TIER_SPLIT_DF; }
// Bytes of one real value of the local-convolution arithmetic (complex: twice).
inline int conv_real_bytes(int t) { return tier_conv(t) == CONV_F32 ? 4 : 8; }

// ---------------------------------------------------------------------------
// Mehrstellen operators (Sec. 2, App. A.1, Sec. 8).  Q = 4 (L19) and Q = 6
// (L27) reach one node (a_j = b_{|j|}, |j| the nonzero components); Q = 10 is
// the q = 10 operator in the 5 x 5 x 5 block, one coefficient per orbit of
// offsets under the cube's symmetries (sorted absolute components):
// (0,0,0) (1,0,0) (1,1,0) (1,1,1) (2,0,0) (2,1,0), the solution of the six
// conditions of eq. mehrstellenTau with q = 10 (sum a_j = 0, sum a_j j_0^2 =
// 2, and sum a_j p(j) = 0 for the harmonic polynomials of degree 4-10).
// ---------------------------------------------------------------------------
__host__ __device__ inline int stencil_reach(int Q) { return Q == 10 ? 2 : 1; }
// C2 of the h^2 term C2 h^2 Delta^2 phi of the truncation error (the
// 4th-order correction adds C2 h^2 f): sum_j a_j j_0^4 / 4!.
inline double stencil_c2(int Q) { return Q == 10 ? 2.0 / 35.0 : 1.0 / 12.0; }
// a_j at h = 1 for |j_d| <= stencil_reach(Q) (0 off the stencil).
__host__ __device__ inline double stencil_coef(int Q, int s0, int s1, int s2) {
    int a = s0 < 0 ? -s0 : s0, b = s1 < 0 ? -s1 : s1, c = s2 < 0 ? -s2 : s2;
    if (Q != 10) {
        if (a > 1 || b > 1 || c > 1) return 0.0;
        const int nz = a + b + c;
        if (Q == 4) return nz == 0 ? -4.0 : (nz == 1 ? 1.0 / 3.0 : (nz == 2 ? 1.0 / 6.0 : 0.0));
        return nz == 0 ? -64.0 / 15.0 : (nz == 1 ? 7.0 / 15.0 : (nz == 2 ? 1.0 / 10.0 : 1.0 / 30.0));
    }
    // sort descending: a >= b >= c
    if (a < b) { const int t = a; a = b; b = t; }
    if (b < c) { const int t = b; b = c; c = t; }
    if (a < b) { const int t = a; a = b; b = t; }
    if (a == 0) return -1079.0 / 210.0;
    if (a == 1) return b == 0 ? 24.0 / 35.0 : (c == 0 ? 17.0 / 210.0 : 11.0 / 420.0);
    if (a == 2 && c == 0) return b == 0 ? -1.0 / 60.0 : (b == 1 ? -1.0 / 420.0 : 0.0);
    return 0.0;
}

// ---------------------------------------------------------------------------
// Plan geometry (Sec. 4): every size below is derived from (N, n, s, C, P, Q,
// g_beta, b) on the host and is identical for every patch.
// ---------------------------------------------------------------------------
struct Geom {
    int N, n, s, C, P, Q, b, ga, gb, np, NP, npoly, nb, W, M, log2M, Mh;
    int npad;                        // npoly rounded up to a multiple of 4 (row stride of moments, D)
    int tier, mode;
    int levels;                      // Sec. 5: 2 = two-level; > 2: the coarse solve is an MLC solve
    int conv, fine;                  // ConvPrec, FinePrec of the tier
    bool f32in;                      // FP32 charge
    double h, H, R;
    int ca_lo, ca_hi, cb_lo, cb_hi;  // coarse boxes C(Omega_alpha), C(Omega_beta), relative
    int flo, fhi, nf;                // F^H extent (union of C(Omega_beta))
    int olo, ohi, no;                // phi^H extent [-b, N/4 + b]
    int Mc, log2Mc, Mhc, Lc;         // coarse Hockney length, max coarse lag
    int L;                           // largest lag any table needs
    int nD, zeta;                    // DGF construction domain
    int S;                           // interpolation stencil size (2b+2)^2
    int wa, wbx;                     // widths of the alpha and beta boxes
    int nr_face;                     // relative face nodes in beta \ alpha
    int pb0, npb;                    // face planes of Omega_beta per axis (relative): pb0 + j n, j < npb
    int npa, pl0;                    // face planes per axis inside Omega_alpha, first at pl0
    int nc;                          // coarse points per axis of the field box, (n + 2s)/4 + 1
    int nzr;                         // z rows of the field box the pruned inverse x reads
    int a4blk;                       // complex entries per (patch, z row) block of the slab output,
                                     // (M/2+1) W rounded up to a multiple of 16 bytes
    int plane_n;                     // (N+1)^2 nodes per face plane
    long n_planes_total;             // 3 (np+1) (N+1)^2
    int ring_rows, ring_ksteps;      // split tiers: ring-table rows per face-plane axis, K / 8 of the ring GEMM
    long ring_rows_pad;              // ring_rows rounded up to the GEMM's row tile (128)
    int chunk;                       // patches per launch group of the local convolutions
    bool wide;                       // Q = 10 (s = 2): a second boundary layer one node off the
                                     // face planes (fp2, resid2, phiB2 below); R18
    size_t scr_a1, scr_a4;           // scratch bytes per patch: x-transformed charges, slab outputs
};
// Local-convolution scratch for `items` patches: the a1 part, then (from a
// 256-byte boundary) the a4 part.
inline size_t conv_scratch_a4_offset(const Geom &g, long items) {
    return ((size_t)items * g.scr_a1 + 255) & ~(size_t)255;
}
inline size_t conv_scratch_bytes(const Geom &g, long items) {
    return conv_scratch_a4_offset(g, items) + (size_t)items * g.scr_a4;
}

// Per-plan pointers and sizes read by the per-patch kernels.  A single solve
// uses its plan's record; a batch passes one record per plan plus an item
// table of (plan slot, local patch) pairs, so one launch covers the patches
// of every problem in the batch.
struct PlanPtrs {
    const void *f;        // charge, N^3 (FP64 or FP32 by tier)
    void *cl, *fp;        // local fields on the coarse lattice / alpha face planes
    const void *khat;     // patch kernel spectrum octant (working precision)
    const void *momw;     // 1D moment weights a_k(m) = w_m q_k(2m/n - 1), P x (n+1), FP64
    double mom_scale;     // R^{-3/2}
    double *mom;
    float *mom_f;         // split tiers: FP32 copy of the moments
    float2 *mom_df;       // double-float tier: moments as double-float (hi, lo) pairs
    void *resid;          // face-plane residuals (FP64 or double-float pairs, 8 bytes each)
    const void *phiB;     // boundary values on the face planes (FP64 or double-float pairs)
    double *phi;
    const void *lam;      // Dirichlet inverse eigenvalues (2/n)^3 h^2 / lambda (FP64 or double-float)
    int N, np;
    double c2h2, inv_h2;  // h^2 / 12, 1 / h^2
    void *dscr;           // Dirichlet workspace (n > 24): [patch][(n-1)^3] in the fine precision
    int *err;             // the plan's error word
    // Q = 10 (R18): local fields and residuals on the planes one node off the
    // alpha face planes, [patch][axis][j][side][u][v] (side 0: plane - 1,
    // 1: plane + 1), and the boundary values of the second layer,
    // [axis][j][side][u][v] over the global planes n j -+ 1, u, v in [0, N]
    void *fp2, *resid2;
    const double *phiB2;
};

// The items of one launch.  Item q covers patch items[q].y of plan record
// items[q].x (or, without an item table, patch first + q of plan record 0),
// and owns slot q of the local-convolution scratch a1 / a4 of the launch.
struct Items {
    const int2 *items;    // (plan slot, local patch); nullptr: plan 0, item = first + index
    const PlanPtrs *plans;
    int nitems;
    int persist = 0;      // 1: launch the slab kernel persistently (one wave of resident CTAs)
    int first = 0;        // patch of item 0 when there is no item table
    int chunk = 0;        // items per local-convolution launch group (0: the plan's conv_chunk)
    void *a1 = nullptr;   // scratch: x-transformed charges, scr_a1 bytes per item
    void *a4 = nullptr;   // scratch: slab outputs, scr_a4 bytes per item
};

}  // namespace mlc

struct mlc_plan_s;
namespace mlc {
extern thread_local bool g_capturing;
}

struct mlc_plan_s {
    mlc::Geom g;
    mlc_params params;
    int device;
    // tables (device)
    const double *dgf;       // shared octant table (L_dgf+1)^3, owned by the device cache
    int dgf_L;
    double *khat;            // patch kernel spectrum octant (Mh^3), scaled by h^2/M^3
    double *khat_c;          // coarse kernel spectrum octant (Mhc^3), scaled by H^2/Mc^3
    double *momw;            // P x nb 1D moment weights (Boole weight x orthonormal Legendre)
    // Legendre ring tables: D [axis][plane][u][v][npad] (dense over the beta
    // box face planes, zero rows off the ring), T [coarse cell][npoly], in the
    // ring precision of the tier (FP32 split tiers, double-float pairs, FP64)
    void *Dtab, *Ttab;
    double2 *tw, *tw_c;      // FFT twiddles exp(-2 pi i t / M), t < M/2 (FP64 tier)
    float *khat_f;           // split tiers: FP32 copies of the patch spectrum and twiddles
    float2 *tw_f;
    float2 *khat_c_df;       // coarse spectrum and twiddles as double-float (hi, lo) pairs
    float4 *tw_c_df;
    float2 *khat_df;         // double-float tier: patch spectrum and twiddles as double-float pairs
    float4 *tw_df;
    void *sinm;              // (n-1) x n/2 half DST-I matrix sin(pi k t / n), fine precision
    void *lam;               // (n-1)^3 (2/n)^3 h^2 / stencil eigenvalue, fine precision
    // workspace (device)
    void *scratch = nullptr;       // own local-convolution scratch, min(chunk, NP) patches (a1
                                   // then a4), allocated by the first solve that needs it
    void *user_scratch = nullptr;  // caller-owned scratch (mlc_plan_set_scratch), if any
    int fault = 0;                 // test hook (mlc_debug_set_fault)
    void *cl;                // NP x nc^3 local fields on the coarse lattice of the field box (FP32 / double-float)
    void *fpl;               // NP x 3 npa x wa^2 local fields on the face planes inside alpha (FP32 / double-float)
    double *mom;             // NP x npad
    float *mom_f;            // split tiers: FP32 copy of the moments
    float2 *mom_df;          // double-float tier: double-float copy of the moments
    double *resid;           // NP x 3 npa x wa^2 face-plane residuals (fine precision, 8 bytes)
    double *FH;              // nf^3
    double2 *cbuf0, *cbuf1;  // coarse spectra
    double *phiH;            // no^3 (fine precision, 8 bytes)
    double *phiB;            // face planes (fine precision, 8 bytes)
    double *tpl;             // 3 (np+1) no (N+1): I^H(phi^H) summed along v per plane and coarse row
    float *ring_aimg;        // split tiers: ring table as the tensor-core GEMM operand (TF32 hi/lo image)
    float *ring_R;           // split tiers: [patch][ring_rows_pad] ring terms of one face-plane axis
    void *dscr = nullptr;    // n > 24: Dirichlet workspace [patch][(n-1)^3] (fine precision)
    // Q = 10 (R18): the second boundary layer
    void *fp2 = nullptr;     // NP x 3 npa 2 x wa^2 local fields one node off the alpha face planes
    double *resid2 = nullptr;  // NP x 3 npa 2 x wa^2 their residuals (FP64)
    double *phiB2 = nullptr;   // 3 (np+1) 2 (N+1)^2 boundary values on the planes n j -+ 1
    double *tpl2 = nullptr;    // 3 (np+1) 2 no (N+1): I^H(phi^H) on those planes summed along v
    void *D2tab = nullptr;     // [axis][npb][2][wbx][wbx][npad] ring rows of the off-face nodes
    void *f_stage, *phi_stage;  // device staging for mlc_solve_host
    int *err;                // device error word: nonzero if a bounded wait in a kernel gave up
    size_t ws_bytes;
    std::vector<void *> owned;  // device allocations to free
    mlc::PlanPtrs *dptrs = nullptr;  // device copy of this plan's PlanPtrs (f, phi filled per solve)
    mlc::PlanPtrs hptrs{};
    // optional per-launch timing of the last solve (CUDA events on the solve
    // stream): (slot, event) marks in launch order; a launch's time runs from
    // its mark to the next one
    int timing = 0;
    mutable std::vector<cudaEvent_t> ev_pool;
    mutable std::vector<std::pair<int, cudaEvent_t>> marks;
    // side stream of a solve: moments, then residuals, beside the main chain
    cudaStream_t side = nullptr;
    cudaEvent_t fork[4] = {};
    // Sec. 5 (levels > 2): the plan of the next coarser level solves
    // Delta^H phi = F^H by MLC in place of the Hockney coarse solve
    mlc_plan_s *child = nullptr;
    void *child_f = nullptr;       // its charge (FP32 or FP64 by tier): F^H at offset flo - child_c0
    double *child_phi = nullptr;   // its result (child N^3)
    int child_c0 = 0;              // its node 0 in this level's coarse nodes
    double h_level = 0.0;          // mesh spacing given at creation (0: 1/N)
    bool correction = true;        // Mehrstellen correction C2 h^2 f (off on the coarser levels)
};

namespace mlc {

// NVTX range around the host code that enqueues one step (a profiler shows
// the kernels each step launched under its name, e.g. ncu --nvtx
// --nvtx-include "mlc:boundary/"); costs a function-pointer test when no tool
// is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// kernels.cu
// Record the timing event of launch slot k (no-op unless timing is enabled).
inline void mark(const mlc_plan_s *pl, int k, cudaStream_t st);
// Per-patch steps over an item set (all patches of one plan, or of a batch of
// plans with the geometry of `pl`).
cudaError_t launch_moments(const mlc_plan_s *pl, const Items &it, cudaStream_t st);
cudaError_t launch_patch_conv(const mlc_plan_s *pl, const Items &it, cudaStream_t st);
cudaError_t launch_resid(const mlc_plan_s *pl, const Items &it, cudaStream_t st);
cudaError_t launch_dirichlet(const mlc_plan_s *pl, const Items &it, cudaStream_t st);
cudaError_t launch_assemble(const mlc_plan_s *pl, cudaStream_t st);
cudaError_t launch_coarse(const mlc_plan_s *pl, cudaStream_t st);
cudaError_t launch_boundary(const mlc_plan_s *pl, cudaStream_t st);
// wide.cuh (Q = 10, R18; part of kernels.cu): residuals and boundary values of the second layer,
// and the Dirichlet solve with two boundary layers.
cudaError_t launch_resid_outer(const mlc_plan_s *pl, const Items &it, cudaStream_t st);
cudaError_t launch_boundary_outer(const mlc_plan_s *pl, cudaStream_t st);
cudaError_t launch_dirichlet_wide(const mlc_plan_s *pl, const Items &it, cudaStream_t st);
void configure_wide();
// Lagrange weights of I^H (R4) for g mod 4 = r, row r, 2b+2 <= 12 entries.
void lagrange_rows(int b, double lw[4][12]);
// ring_gemm.cu: the Legendre ring terms of one face-plane axis as a tcgen05
// GEMM (split tiers), and its plan-time operand image.
cudaError_t launch_ring_gemm(const mlc_plan_s *pl, int axis, cudaStream_t st);
void configure_ring_gemm();
void ring_table_image(const std::vector<double> &Dd, int nrows_axis, int npad, int ksteps, long rows_pad,
                      std::vector<float> &img);
// Host rounding of a value to TF32 (10 stored mantissa bits), nearest, ties away from zero.
inline float tf32_host(double v) {
    float f = (float)v;
    uint32_t b;
    std::memcpy(&b, &f, 4);
    b = (b + 0x1000u) & 0xFFFFE000u;
    std::memcpy(&f, &b, 4);
    return f;
}
// Index export (test hook): which = 0 face-plane nodes, 1 coarse nodes of the
// F^H extent; count pass (cnt != nullptr) or fill pass (off, ent).
cudaError_t launch_index_export(const mlc_plan_s *pl, int which, int *cnt, const long *off, int *ent,
                                cudaStream_t st);
void configure_kernels();
// Write f and phi into a device PlanPtrs record, in stream order.
cudaError_t launch_set_ptrs(PlanPtrs *d, const void *f, double *phi, cudaStream_t st);
// Timing marks are suppressed while a batch graph is being captured.
extern thread_local bool g_capturing;

// dgf.cu
// Build G^{h=1} on [0, L]^3 (App. A.1) into a new device array; returns nullptr on error.
cudaError_t build_dgf_octant(int Q, int nD, int zeta, int L, double **out);
// Real-even kernel spectrum: out[k] = scale * sum_m K[m] prod cos(2 pi k_d m_d / M), octant
// k in [0, M/2]^3, K[m] = G1[fold(m)] for |fold(m)| <= Lmax (else 0).
cudaError_t build_even_spectrum(const double *G1, int L_table, int M, int Lmax, double scale,
                                double *out);
// Batched strided FP64 matrix product used at plan time.
cudaError_t batched_dgemm(int I, int K, int J, int batch, const double *A, long lda,
                          const double *X, long xs_b, long xs_k, long xs_j, double *Y, long ys_b,
                          long ys_i, long ys_j, cudaStream_t st);
// Direct sum used at plan time for the basis fields: out[a*npoly + p] =
// h^2 sum_m G1[|pts[a] - m|] * charge[p][m], m over [0,n]^3.
cudaError_t basis_direct_sum(const double *G1, int L_table, const int *pts, int npts,
                             const double *charge, int npoly, int n, double h2, double *out);

}  // namespace mlc

namespace mlc {
inline void mark(const mlc_plan_s *pl, int k, cudaStream_t st) {
    if (!pl || !pl->timing || g_capturing) return;
    const size_t i = pl->marks.size();
    if (i >= pl->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        pl->ev_pool.push_back(e);
    }
    cudaEventRecord(pl->ev_pool[i], st);
    pl->marks.push_back({k, pl->ev_pool[i]});
}
}  // namespace mlc

namespace mlc {
// ---- batched launches (batch.cu): shared by mlc_batch_solve and the server ----
// Problems grouped by patch geometry and tier; record slot j (the j-th
// PlanPtrs record) is problem order[j] of the call, in group plan_group[j].
struct BatchLayout {
    struct Group {
        const mlc_plan_s *rep;  // a plan of the group (its geometry sizes the launches)
        int item0, nitems;      // the group's range of the item table
        void *a1 = nullptr, *a4 = nullptr;  // the group's local-convolution scratch
                                            // (min(chunk, nitems) patches; set by the owner)
    };
    std::vector<int> order, plan_group;
    std::vector<Group> groups;
    std::vector<int2> items;     // (record slot, local patch), group by group
    std::vector<PlanPtrs> recs;  // per record slot: the plan's pointers with its f and phi
};
// Streams and events of one batch launch sequence (created on first use).
struct BatchStreams {
    std::vector<cudaStream_t> conv, aux, side;
    std::vector<cudaEvent_t> ev;
    cudaError_t ensure(int ngroups, int nbranches);
    void release();
};
bool same_patch_geometry(const Geom &a, const Geom &b);
void batch_layout(int count, const mlc_plan_t *plans, const void *const *f, void *const *phi, BatchLayout &L);
// Enqueue every launch of a batch (all groups, all problems) after earlier
// work on st; st waits for all of it.  d_items / d_recs: device copies of
// L.items / L.recs.  plans: the problems in call order.
cudaError_t batch_enqueue(const std::vector<mlc_plan_t> &plans, const BatchLayout &L, const int2 *d_items,
                          const PlanPtrs *d_recs, BatchStreams &S, int branches, int persist,
                          cudaStream_t st, int chunk = 0);
}  // namespace mlc
