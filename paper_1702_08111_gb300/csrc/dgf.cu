// Plan-time tables: the discrete Green's function (App. A.1), the real-even
// kernel spectra used by Hockney's method (App. A.2), and the direct sums for
// the Legendre basis fields (Sec. 4, Step 1).  None of this runs inside a
// solve; it is FP64 throughout.
#include <cmath>
#include <vector>

#include "mlc_internal.h"

namespace mlc {

namespace {

// App. A.1: a_j = b_{|j|} / h^2, |j| = number of nonzero components.
void stencil_b(int Q, double b[4]) {
    if (Q == 4) {
        b[0] = -4.0; b[1] = 1.0 / 3.0; b[2] = 1.0 / 6.0; b[3] = 0.0;
    } else {
        b[0] = -64.0 / 15.0; b[1] = 7.0 / 15.0; b[2] = 1.0 / 10.0; b[3] = 1.0 / 30.0;
    }
}

// Right-hand side of the residual-correction form on the octant [0, MD-1]^3 of
// the interior of D_zeta = [-MD, MD]^3: delta_0 minus the stencil applied to the
// boundary values -1/(4 pi |y|) on |y|_inf = MD.
__global__ void k_dgf_rhs(double *r, int MD, double b0, double b1, double b2, double b3) {
    long total = (long)MD * MD * MD;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int x2 = (int)(idx % MD);
    int x1 = (int)((idx / MD) % MD);
    int x0 = (int)(idx / ((long)MD * MD));
    double acc = (x0 == 0 && x1 == 0 && x2 == 0) ? 1.0 : 0.0;
    if (x0 == MD - 1 || x1 == MD - 1 || x2 == MD - 1) {
        const double bb[4] = {b0, b1, b2, b3};
        for (int s0 = -1; s0 <= 1; ++s0)
            for (int s1 = -1; s1 <= 1; ++s1)
                for (int s2 = -1; s2 <= 1; ++s2) {
                    int y0 = x0 + s0, y1 = x1 + s1, y2 = x2 + s2;
                    if (y0 != MD && y1 != MD && y2 != MD) continue;  // y0,y1,y2 >= -1 here
                    int nz = (s0 != 0) + (s1 != 0) + (s2 != 0);
                    double c = bb[nz];
                    if (c == 0.0) continue;
                    double rr = sqrt((double)y0 * y0 + (double)y1 * y1 + (double)y2 * y2);
                    acc -= c * (-1.0 / (4.0 * M_PI * rr));
                }
    }
    r[idx] = acc;
}

// Q = 10 (R18): the reference field of the residual-correction form is the
// free-space kernel w(y) = -1/(4 pi |y|) (w(0) = 0) on the whole box, so the
// right-hand side delta_0 - L w is needed at every node of the octant; the
// stencil reads w up to two nodes beyond the boundary |y|_inf = MD.
__device__ __forceinline__ double dgf_w(int y0, int y1, int y2) {
    if (y0 == 0 && y1 == 0 && y2 == 0) return 0.0;
    return -1.0 / (4.0 * M_PI * sqrt((double)y0 * y0 + (double)y1 * y1 + (double)y2 * y2));
}
__global__ void k_dgf_rhs_wide(double *r, int MD) {
    long total = (long)MD * MD * MD;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int x2 = (int)(idx % MD);
    int x1 = (int)((idx / MD) % MD);
    int x0 = (int)(idx / ((long)MD * MD));
    double acc = 0.0;
    for (int s0 = -2; s0 <= 2; ++s0)
        for (int s1 = -2; s1 <= 2; ++s1)
            for (int s2 = -2; s2 <= 2; ++s2) {
                const double c = stencil_coef(10, s0, s1, s2);
                if (c != 0.0) acc = fma(c, dgf_w(x0 + s0, x1 + s1, x2 + s2), acc);
            }
    r[idx] = ((x0 == 0 && x1 == 0 && x2 == 0) ? 1.0 : 0.0) - acc;
}
__global__ void k_dgf_div_wide(double *u, int MD, const double *cosv) {
    long total = (long)MD * MD * MD;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const double c[3] = {cosv[idx / ((long)MD * MD)], cosv[(idx / MD) % MD], cosv[idx % MD]};
    double lam = 0.0;
    for (int s0 = -2; s0 <= 2; ++s0)
        for (int s1 = -2; s1 <= 2; ++s1)
            for (int s2 = -2; s2 <= 2; ++s2) {
                const double a = stencil_coef(10, s0, s1, s2);
                if (a == 0.0) continue;
                const int ss[3] = {s0, s1, s2};
                double t = a;
                for (int d = 0; d < 3; ++d) {
                    const int k = ss[d] < 0 ? -ss[d] : ss[d];
                    t *= k == 0 ? 1.0 : (k == 1 ? c[d] : 2.0 * c[d] * c[d] - 1.0);
                }
                lam += t;
            }
    u[idx] /= lam;
}
__global__ void k_dgf_add_w(double *G, int Lp) {
    long total = (long)Lp * Lp * Lp;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    G[idx] += dgf_w((int)(idx / ((long)Lp * Lp)), (int)((idx / Lp) % Lp), (int)(idx % Lp));
}

// Divide the cosine coefficients by the stencil's eigenvalue.
__global__ void k_dgf_div(double *u, int MD, const double *cosv, double b0, double b1, double b2,
                          double b3) {
    long total = (long)MD * MD * MD;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    double c2 = cosv[idx % MD];
    double c1 = cosv[(idx / MD) % MD];
    double c0 = cosv[idx / ((long)MD * MD)];
    double lam = b0 + 2.0 * b1 * (c0 + c1 + c2) + 4.0 * b2 * (c0 * c1 + c0 * c2 + c1 * c2) +
                 8.0 * b3 * c0 * c1 * c2;
    u[idx] /= lam;
}

// Y(b,i,j) = sum_k A(i,k) X(b,k,j); 64x64 tiles, 256 threads, 4x4 per thread.
__global__ void __launch_bounds__(256) k_dgemm(int I, int K, int J, const double *__restrict__ A,
                                               long lda, const double *__restrict__ X, long xs_b,
                                               long xs_k, long xs_j, double *__restrict__ Y,
                                               long ys_b, long ys_i, long ys_j) {
    __shared__ double As[16][65];
    __shared__ double Xs[16][65];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
    const double *Xb = X + (long)b * xs_b;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int kk = e / 64, ii = e % 64;
            int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < I && gk < K) ? A[(long)gi * lda + gk] : 0.0;
        }
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int kk = e / 64, jj = e % 64;
            int gj = j0 + jj, gk = k0 + kk;
            Xs[kk][jj] = (gj < J && gk < K) ? Xb[(long)gk * xs_k + (long)gj * xs_j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], x[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] = Xs[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], x[c], acc[r][c]);
        }
        __syncthreads();
    }
    double *Yb = Y + (long)b * ys_b;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int gi = i0 + ty * 4 + r;
        if (gi >= I) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int gj = j0 + tx * 4 + c;
            if (gj < J) Yb[(long)gi * ys_i + (long)gj * ys_j] = acc[r][c];
        }
    }
}

// Apply a (I x d_axis) matrix along one axis of a dense d0 x d1 x d2 array.
cudaError_t axis_apply(const double *A, int I, const double *X, int d0, int d1, int d2, int axis,
                       double *Y, cudaStream_t st) {
    if (axis == 2)
        return batched_dgemm(I, d2, d0 * d1, 1, A, d2, X, 0, 1, d2, Y, 0, 1, I, st);
    if (axis == 1)
        return batched_dgemm(I, d1, d2, d0, A, d1, X, (long)d1 * d2, d2, 1, Y, (long)I * d2, d2, 1,
                             st);
    return batched_dgemm(I, d0, d1 * d2, 1, A, d0, X, 0, (long)d1 * d2, 1, Y, 0, (long)d1 * d2, 1,
                         st);
}

// Long-lived device allocation helper for plan-time scratch.
struct Scratch {
    std::vector<void *> ptrs;
    cudaError_t alloc(void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
};

#define MLC_TRY(x)                            \
    do {                                      \
        cudaError_t _e = (x);                 \
        if (_e != cudaSuccess) return _e;     \
    } while (0)

}  // namespace

cudaError_t batched_dgemm(int I, int K, int J, int batch, const double *A, long lda,
                          const double *X, long xs_b, long xs_k, long xs_j, double *Y, long ys_b,
                          long ys_i, long ys_j, cudaStream_t st) {
    dim3 grid((J + 63) / 64, (I + 63) / 64, batch);
    k_dgemm<<<grid, 256, 0, st>>>(I, K, J, A, lda, X, xs_b, xs_k, xs_j, Y, ys_b, ys_i, ys_j);
    return cudaGetLastError();
}

cudaError_t build_dgf_octant(int Q, int nD, int zeta, int L, double **out) {
    *out = nullptr;
    const int MD = zeta * nD;
    if (L >= MD) return cudaErrorInvalidValue;
    double bq[4];
    stencil_b(Q, bq);
    const long vol = (long)MD * MD * MD;
    Scratch sc;
    double *r = nullptr, *t = nullptr, *dCf = nullptr, *dCi = nullptr, *dcos = nullptr;
    MLC_TRY(sc.alloc((void **)&r, vol * sizeof(double)));
    MLC_TRY(sc.alloc((void **)&t, vol * sizeof(double)));
    // forward matrix Cf[j][x] = (2/MD) w_x cos((2j+1) pi x / (2 MD)), w_0 = 1/2
    // inverse matrix Ci[x][j] = cos((2j+1) pi x / (2 MD)), x in [0, L]
    std::vector<double> Cf((size_t)MD * MD), Ci((size_t)(L + 1) * MD), cosv(MD);
    const long period = 4L * MD;  // cos(pi r / (2 MD)) has period 4 MD in r
    for (int j = 0; j < MD; ++j) {
        for (int x = 0; x < MD; ++x) {
            long rr = ((long)(2 * j + 1) * x) % period;
            double c = std::cos(M_PI * (double)rr / (2.0 * MD));
            Cf[(size_t)j * MD + x] = (2.0 / MD) * (x == 0 ? 0.5 : 1.0) * c;
            if (x <= L) Ci[(size_t)x * MD + j] = c;
        }
        cosv[j] = std::cos(M_PI * (double)(2 * j + 1) / (2.0 * MD));
    }
    MLC_TRY(sc.alloc((void **)&dCf, Cf.size() * sizeof(double)));
    MLC_TRY(sc.alloc((void **)&dCi, Ci.size() * sizeof(double)));
    MLC_TRY(sc.alloc((void **)&dcos, cosv.size() * sizeof(double)));
    MLC_TRY(cudaMemcpy(dCf, Cf.data(), Cf.size() * sizeof(double), cudaMemcpyHostToDevice));
    MLC_TRY(cudaMemcpy(dCi, Ci.data(), Ci.size() * sizeof(double), cudaMemcpyHostToDevice));
    MLC_TRY(cudaMemcpy(dcos, cosv.data(), cosv.size() * sizeof(double), cudaMemcpyHostToDevice));
    cudaStream_t st = 0;
    int threads = 256;
    long blocks = (vol + threads - 1) / threads;
    if (Q == 10) k_dgf_rhs_wide<<<(unsigned)blocks, threads, 0, st>>>(r, MD);
    else k_dgf_rhs<<<(unsigned)blocks, threads, 0, st>>>(r, MD, bq[0], bq[1], bq[2], bq[3]);
    MLC_TRY(cudaGetLastError());
    // forward cosine transform along axes 2, 1, 0
    MLC_TRY(axis_apply(dCf, MD, r, MD, MD, MD, 2, t, st));
    MLC_TRY(axis_apply(dCf, MD, t, MD, MD, MD, 1, r, st));
    MLC_TRY(axis_apply(dCf, MD, r, MD, MD, MD, 0, t, st));
    if (Q == 10) k_dgf_div_wide<<<(unsigned)blocks, threads, 0, st>>>(t, MD, dcos);
    else k_dgf_div<<<(unsigned)blocks, threads, 0, st>>>(t, MD, dcos, bq[0], bq[1], bq[2], bq[3]);
    MLC_TRY(cudaGetLastError());
    // inverse transform, keeping only x in [0, L]
    const int Lp = L + 1;
    MLC_TRY(axis_apply(dCi, Lp, t, MD, MD, MD, 2, r, st));     // MD x MD x Lp
    MLC_TRY(axis_apply(dCi, Lp, r, MD, MD, Lp, 1, t, st));     // MD x Lp x Lp
    double *res = nullptr;
    MLC_TRY(cudaMalloc((void **)&res, (size_t)Lp * Lp * Lp * sizeof(double)));
    cudaError_t e = axis_apply(dCi, Lp, t, MD, Lp, Lp, 0, res, st);  // Lp^3
    if (e == cudaSuccess && Q == 10) {  // G = w + u
        const long v3 = (long)Lp * Lp * Lp;
        k_dgf_add_w<<<(unsigned)((v3 + 255) / 256), 256, 0, st>>>(res, Lp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(res);
        return e;
    }
    *out = res;
    return cudaSuccess;
}

namespace {
__global__ void k_fold_kernel(const double *G1, int Lt, int Mh, int Lmax, double *K) {
    long total = (long)Mh * Mh * Mh;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int m2 = (int)(idx % Mh), m1 = (int)((idx / Mh) % Mh), m0 = (int)(idx / ((long)Mh * Mh));
    double v = 0.0;
    if (m0 <= Lmax && m1 <= Lmax && m2 <= Lmax)
        v = G1[((long)m0 * (Lt + 1) + m1) * (Lt + 1) + m2];
    K[idx] = v;
}
__global__ void k_scale(double *x, long n, double s) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) x[idx] *= s;
}
}  // namespace

cudaError_t build_even_spectrum(const double *G1, int L_table, int M, int Lmax, double scale,
                                double *out) {
    const int Mh = M / 2 + 1;
    if (Lmax > L_table || Lmax > M / 2) return cudaErrorInvalidValue;
    std::vector<double> E((size_t)Mh * Mh);
    for (int k = 0; k < Mh; ++k)
        for (int m = 0; m < Mh; ++m) {
            long rr = ((long)k * m) % M;
            double c = std::cos(2.0 * M_PI * (double)rr / (double)M);
            double w = (m == 0 || 2 * m == M) ? 1.0 : 2.0;
            E[(size_t)k * Mh + m] = w * c;
        }
    Scratch sc;
    double *dE = nullptr, *a = nullptr;
    const long vol = (long)Mh * Mh * Mh;
    MLC_TRY(sc.alloc((void **)&dE, E.size() * sizeof(double)));
    MLC_TRY(sc.alloc((void **)&a, vol * sizeof(double)));
    MLC_TRY(cudaMemcpy(dE, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice));
    cudaStream_t st = 0;
    unsigned blocks = (unsigned)((vol + 255) / 256);
    k_fold_kernel<<<blocks, 256, 0, st>>>(G1, L_table, Mh, Lmax, out);
    MLC_TRY(cudaGetLastError());
    MLC_TRY(axis_apply(dE, Mh, out, Mh, Mh, Mh, 2, a, st));
    MLC_TRY(axis_apply(dE, Mh, a, Mh, Mh, Mh, 1, out, st));
    MLC_TRY(axis_apply(dE, Mh, out, Mh, Mh, Mh, 0, a, st));
    MLC_TRY(cudaMemcpyAsync(out, a, vol * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_scale<<<blocks, 256, 0, st>>>(out, vol, scale);
    MLC_TRY(cudaGetLastError());
    return cudaStreamSynchronize(st);
}

namespace {
__global__ void k_basis_sum(const double *__restrict__ G1, int Lt, const int *__restrict__ pts,
                            int npts, const double *__restrict__ charge, int npoly, int n,
                            double h2, double *__restrict__ out) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= npts) return;
    const int p0 = pts[3 * a], p1 = pts[3 * a + 1], p2 = pts[3 * a + 2];
    double acc[56];
    for (int p = 0; p < npoly; ++p) acc[p] = 0.0;
    const int nb = n + 1;
    const long Lp = Lt + 1;
    for (int m0 = 0; m0 < nb; ++m0) {
        long l0 = abs(p0 - m0);
        for (int m1 = 0; m1 < nb; ++m1) {
            long l1 = abs(p1 - m1);
            const double *row = G1 + (l0 * Lp + l1) * Lp;
            for (int m2 = 0; m2 < nb; ++m2) {
                double g = row[abs(p2 - m2)];
                long m = ((long)m0 * nb + m1) * nb + m2;
                for (int p = 0; p < npoly; ++p) acc[p] = fma(g, charge[(long)p * nb * nb * nb + m], acc[p]);
            }
        }
    }
    for (int p = 0; p < npoly; ++p) out[(long)a * npoly + p] = h2 * acc[p];
}
}  // namespace

cudaError_t basis_direct_sum(const double *G1, int L_table, const int *pts, int npts,
                             const double *charge, int npoly, int n, double h2, double *out) {
    if (npoly > 56) return cudaErrorInvalidValue;
    k_basis_sum<<<(npts + 127) / 128, 128>>>(G1, L_table, pts, npts, charge, npoly, n, h2, out);
    MLC_TRY(cudaGetLastError());
    return cudaDeviceSynchronize();
}

}  // namespace mlc
