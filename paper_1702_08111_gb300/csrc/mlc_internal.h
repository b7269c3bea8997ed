// Internal declarations of the MLC library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mlc.h"

namespace mlc {

// Launches of one solve, in order (the timing slots of mlc_debug_timing).
constexpr int kTimedLaunches = 15;

// ---------------------------------------------------------------------------
// Plan geometry (Sec. 4): every size below is derived from (N, n, s, C, P, Q,
// g_beta, b) on the host and is identical for every patch.
// ---------------------------------------------------------------------------
struct Geom {
    int N, n, s, C, P, Q, b, ga, gb, np, NP, npoly, nb, W, M, log2M, Mh;
    int tier, mode;
    double h, H, R;
    int ca_lo, ca_hi, cb_lo, cb_hi;  // coarse boxes C(Omega_alpha), C(Omega_beta), relative
    int flo, fhi, nf;                // F^H extent (union of C(Omega_beta))
    int olo, ohi, no;                // phi^H extent [-b, N/4 + b]
    int Mc, log2Mc, Mhc, Lc;         // coarse Hockney length, max coarse lag
    int L;                           // largest lag any table needs
    int nD, zeta;                    // DGF construction domain
    int S;                           // interpolation stencil size (2b+2)^2
    int wa, wbx;                     // widths of the alpha and beta boxes
    int na_face, nr_face;            // relative face nodes in alpha, in beta \ alpha
    int plane_n;                     // (N+1)^2 nodes per face plane
    long n_planes_total;             // 3 (np+1) (N+1)^2
};

// Host-built relative tables, uploaded to the device.
struct HostTables {
    std::vector<double> momw;        // npoly x nb^3: Boole weight * Q^p at patch nodes
    std::vector<int> amap;           // alpha box (wa^3) -> alpha face index or -1
    std::vector<int> a_self;         // per alpha face node: field-box index of the node
    std::vector<int> a_off;          // per alpha face node: S field-box indices of 4k
    std::vector<double> a_w;         // per alpha face node: S weights
    std::vector<int> rmap;           // beta box (wbx^3) -> ring face index or -1
    std::vector<double> Dtab;        // nr_face x npoly: B_p - I(B_p) at ring face nodes
    std::vector<double> Ttab;        // ncb^3 x npoly: Delta^H B_p on C(beta) (0 inside C(alpha))
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace mlc

struct mlc_plan_s {
    mlc::Geom g;
    mlc_params params;
    int device;
    // tables (device)
    const double *dgf;       // shared octant table (L_dgf+1)^3, owned by the device cache
    int dgf_L;
    double *khat;            // patch kernel spectrum octant (Mh^3), scaled by h^2/M^3
    double *khat_c;          // coarse kernel spectrum octant (Mhc^3), scaled by H^2/Mc^3
    double *momw;            // npoly x nb^3
    int *amap, *a_self, *a_off;
    double *a_w;
    int *rmap;
    double *Dtab, *Ttab;
    double2 *tw, *tw_c;      // FFT twiddles exp(-2 pi i t / M), t < M/2
    float *khat_f;           // split tier: FP32 copies of the patch spectrum and twiddles
    float2 *tw_f;
    double *sinm;            // (n-1)^2 DST-I matrix sin(pi k m / n)
    double *lam;             // (n-1)^3 stencil eigenvalues / h^2
    // workspace (device)
    void *buf0, *buf1;       // ping-pong spectra for the patch convolutions (complex FP64 / FP32)
    void *box;               // NP x W^3 local fields phi^{i,h} (FP64 / FP32)
    double *mom;             // NP x npoly
    double *resid;           // NP x na_face
    double *FH;              // nf^3
    double2 *cbuf0, *cbuf1;  // coarse spectra
    double *phiH;            // no^3
    double *phiB;            // face planes
    void *f_stage, *phi_stage;  // device staging for mlc_solve_host
    size_t ws_bytes;
    std::vector<void *> owned;  // device allocations to free
    // optional per-launch timing of the last solve (CUDA events on the solve stream)
    int timing = 0;
    cudaEvent_t ev[mlc::kTimedLaunches + 1] = {};
};

namespace mlc {

// kernels_fp64.cu
// Record the timing event of launch slot k (no-op unless timing is enabled).
inline void mark(const mlc_plan_s *pl, int k, cudaStream_t st) {
    if (pl && pl->timing) cudaEventRecord(pl->ev[k], st);
}
cudaError_t launch_moments(const mlc_plan_s *pl, const void *f, bool f32, cudaStream_t st);
cudaError_t launch_patch_conv(const mlc_plan_s *pl, const void *f, bool f32, cudaStream_t st);
cudaError_t launch_resid(const mlc_plan_s *pl, cudaStream_t st);
cudaError_t launch_assemble(const mlc_plan_s *pl, cudaStream_t st);
cudaError_t launch_coarse(const mlc_plan_s *pl, cudaStream_t st);
cudaError_t launch_boundary(const mlc_plan_s *pl, cudaStream_t st);
cudaError_t launch_dirichlet(const mlc_plan_s *pl, const void *f, bool f32, double *phi, cudaStream_t st);
void configure_kernels();

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
