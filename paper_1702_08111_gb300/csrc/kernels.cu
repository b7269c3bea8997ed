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
#include <cmath>

#include "mlc_internal.h"

namespace mlc {

namespace {

__device__ __forceinline__ int brev_bits(int i, int log2m) {
    return (int)(__brev((unsigned)i) >> (32 - log2m));
}

__device__ __forceinline__ int floordiv(int a, int b) {  // b > 0
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Complex type of each working precision (FP64 tier: double; split tier: float).
template <typename R> struct Cx;
template <> struct Cx<double> {
    using T = double2;
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};
template <> struct Cx<float> {
    using T = float2;
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};

__device__ __forceinline__ double2 cmul(double2 a, double2 w) {
    return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// Decimation in frequency: natural-order input, bit-reversed output.
template <int LOG2M, typename C>
__device__ __forceinline__ void fft_dif(C *buf, int nlines, int lstride, int estride,
                                        const C *tw, bool inv) {
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
            C *p0 = buf + line * lstride + i0 * estride;
            C *p1 = p0 + hs * estride;
            C w = tw[pos << tsh];
            if (inv) w.y = -w.y;
            const C a = *p0, b = *p1;
            *p0 = cadd(a, b);
            *p1 = cmul(csub(a, b), w);
        }
        __syncthreads();
    }
}

// Decimation in time: bit-reversed input, natural-order output.
template <int LOG2M, typename C>
__device__ __forceinline__ void fft_dit(C *buf, int nlines, int lstride, int estride,
                                        const C *tw, bool inv) {
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
            C *p0 = buf + line * lstride + i0 * estride;
            C *p1 = p0 + hs * estride;
            C w = tw[pos << tsh];
            if (inv) w.y = -w.y;
            const C a = *p0;
            const C t = cmul(*p1, w);
            *p0 = cadd(a, t);
            *p1 = csub(a, t);
        }
        __syncthreads();
    }
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
    const void *src;
    void *out;        // complex R: [slab][line][M/2+1]
    int N, n, np;     // patch geometry (PATCH)
    int nin;          // input nodes per axis
    int lines_cta;    // lines per CTA
    const void *tw;   // complex R twiddles
};

template <int LOG2M, typename TF, bool PATCH, typename R>
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
    const int zi = slab % a.nin, p = slab / a.nin;
    for (int e = threadIdx.x; e < nl * a.nin; e += blockDim.x) {
        const int l = e / a.nin, m = e % a.nin;
        const int yi = line0 + l;
        R v;
        if (PATCH) {
            const int i2 = p % a.np, i1 = (p / a.np) % a.np, i0 = p / (a.np * a.np);
            const int z = i0 * a.n + zi, y = i1 * a.n + yi, x = i2 * a.n + m;
            v = 0;
            if (z < a.N && y < a.N && x < a.N) {
                const TF *f = (const TF *)a.src;
                R w = (zi == 0 || zi == a.n) ? R(0.5) : R(1);
                w *= (yi == 0 || yi == a.n) ? R(0.5) : R(1);
                w *= (m == 0 || m == a.n) ? R(0.5) : R(1);
                v = w * (R)f[((long)z * a.N + y) * a.N + x];
            }
        } else {
            const double *F = (const double *)a.src;
            v = (R)F[((long)zi * a.nin + yi) * a.nin + m];
        }
        buf[l * LS + m] = Cx<R>::mk(v, 0);
    }
    __syncthreads();
    fft_dif<LOG2M>(buf, nl, LS, 1, s_tw, false);
    C *out = (C *)a.out;
    for (int e = threadIdx.x; e < nl * MH; e += blockDim.x) {
        const int l = e / MH, kx = e % MH;
        out[((long)slab * a.nin + line0 + l) * MH + kx] = buf[l * LS + brev_bits(kx, LOG2M)];
    }
}

// ---------------------------------------------------------------------------
// Transform along a strided axis; lines are contiguous columns.
//   MODE 0: forward; input rows t < nin at positions t; all M rows out.
//   MODE 1: inverse; all M rows in; rows t < nout out from positions
//           (out_off + t) mod M.
//   MODE 2: forward, multiply by the real-even kernel spectrum, inverse.
// slab = blockIdx.x = p * S2 + q; blockIdx.y = column chunk.
// ---------------------------------------------------------------------------
struct ColArgs {
    const void *in;
    void *out;
    int S2;
    long in_sp, in_sq, in_row, out_sp, out_sq, out_row;
    int ncols, cols_cta, nin, nout, out_off;
    const void *khat;  // MODE 2: real R octant (M/2+1)^3, index (kx, ky = q, kz = row)
    const void *tw;
};

template <int LOG2M, int MODE, typename R>
__global__ void __launch_bounds__(256) k_col(ColArgs a) {
    using C = typename Cx<R>::T;
    constexpr int M = 1 << LOG2M, MH = M / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_tw = (C *)smem_raw;
    C *buf = s_tw + M / 2;
    const int slab = blockIdx.x;
    const int p = slab / a.S2, q = slab % a.S2;
    const int c0 = blockIdx.y * a.cols_cta;
    const int nc = min(a.cols_cta, a.ncols - c0);
    const int CC = a.cols_cta;  // row stride in shared memory
    load_twiddles<LOG2M>(s_tw, (const C *)a.tw);
    const C *in = (const C *)a.in + p * a.in_sp + q * a.in_sq + c0;
    if (MODE != 1)
        for (int e = threadIdx.x; e < M * CC; e += blockDim.x) buf[e] = Cx<R>::mk(0, 0);
    __syncthreads();
    const int nrow_in = (MODE == 1) ? M : a.nin;
    for (int e = threadIdx.x; e < nrow_in * nc; e += blockDim.x) {
        const int r = e / nc, c = e % nc;
        buf[r * CC + c] = in[r * a.in_row + c];
    }
    __syncthreads();
    C *out = (C *)a.out + p * a.out_sp + q * a.out_sq + c0;
    if (MODE == 0) {
        fft_dif<LOG2M>(buf, nc, 1, CC, s_tw, false);
        for (int e = threadIdx.x; e < M * nc; e += blockDim.x) {
            const int r = e / nc, c = e % nc;
            out[r * a.out_row + c] = buf[brev_bits(r, LOG2M) * CC + c];
        }
        return;
    }
    if (MODE == 1) {
        fft_dif<LOG2M>(buf, nc, 1, CC, s_tw, true);
    } else {
        fft_dif<LOG2M>(buf, nc, 1, CC, s_tw, false);
        const R *khat = (const R *)a.khat;
        const int ky = q < M - q ? q : M - q;
        for (int e = threadIdx.x; e < M * nc; e += blockDim.x) {
            const int r = e / nc, c = e % nc;
            const int kz0 = brev_bits(r, LOG2M);
            const int kz = kz0 < M - kz0 ? kz0 : M - kz0;
            const int kx0 = c0 + c;
            const int kx = kx0 < M - kx0 ? kx0 : M - kx0;
            const R k = khat[((long)kx * MH + ky) * MH + kz];
            C v = buf[r * CC + c];
            v.x *= k;
            v.y *= k;
            buf[r * CC + c] = v;
        }
        __syncthreads();
        fft_dit<LOG2M>(buf, nc, 1, CC, s_tw, true);
    }
    for (int e = threadIdx.x; e < a.nout * nc; e += blockDim.x) {
        const int t = e / nc, c = e % nc;
        int pos = (a.out_off + t) % M;
        if (pos < 0) pos += M;
        const int sr = (MODE == 1) ? brev_bits(pos, LOG2M) : pos;
        out[t * a.out_row + c] = buf[sr * CC + c];
    }
}

// ---------------------------------------------------------------------------
// Inverse real transform along axis 2: lines are rows; the half spectrum
// kx in [0, M/2] is extended by Hermitian symmetry; outputs t < nout from
// positions (out_off + t) mod M.  out[(slab * nrow + row) * nout + t] (type TO).
// ---------------------------------------------------------------------------
struct InvXArgs {
    const void *in;
    void *out;
    int nrow, nout, out_off, lines_cta;
    const void *tw;
};

template <int LOG2M, typename R, typename TO>
__global__ void __launch_bounds__(256) k_inv_x(InvXArgs a) {
    using C = typename Cx<R>::T;
    constexpr int M = 1 << LOG2M, MH = M / 2 + 1, LS = M + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s_tw = (C *)smem_raw;
    C *buf = s_tw + M / 2;
    const int slab = blockIdx.x;
    const int r0 = blockIdx.y * a.lines_cta;
    const int nl = min(a.lines_cta, a.nrow - r0);
    load_twiddles<LOG2M>(s_tw, (const C *)a.tw);
    const C *in = (const C *)a.in + ((long)slab * a.nrow + r0) * MH;
    for (int e = threadIdx.x; e < nl * M; e += blockDim.x) {
        const int l = e / M, k = e % M;
        C v;
        if (k < MH) {
            v = in[l * MH + k];
        } else {
            v = in[l * MH + (M - k)];
            v.y = -v.y;
        }
        buf[l * LS + k] = v;
    }
    __syncthreads();
    fft_dif<LOG2M>(buf, nl, LS, 1, s_tw, true);
    TO *out = (TO *)a.out + ((long)slab * a.nrow + r0) * a.nout;
    for (int e = threadIdx.x; e < nl * a.nout; e += blockDim.x) {
        const int l = e / a.nout, t = e % a.nout;
        int pos = (a.out_off + t) % M;
        if (pos < 0) pos += M;
        out[l * a.nout + t] = (TO)buf[l * LS + brev_bits(pos, LOG2M)].x;
    }
}

// ---------------------------------------------------------------------------
// Legendre coefficients c_p^i = sum_m W[m] Q^p(m) f[n i + m] (Boole, R3).
// ---------------------------------------------------------------------------
template <typename TF>
__global__ void __launch_bounds__(256) k_moments(const TF *__restrict__ f, int N, int n, int np,
                                                 int npoly, const double *__restrict__ momw,
                                                 double *__restrict__ mom) {
    __shared__ double red[8][56];
    const int p = blockIdx.x;
    const int i2 = p % np, i1 = (p / np) % np, i0 = p / (np * np);
    const int nb = n + 1, nb3 = nb * nb * nb;
    double acc[56];
    for (int k = 0; k < npoly; ++k) acc[k] = 0.0;
    for (int m = threadIdx.x; m < nb3; m += blockDim.x) {
        const int m2 = m % nb, m1 = (m / nb) % nb, m0 = m / (nb * nb);
        const int z = i0 * n + m0, y = i1 * n + m1, x = i2 * n + m2;
        if (z >= N || y >= N || x >= N) continue;
        const double v = (double)f[((long)z * N + y) * N + x];
        for (int k = 0; k < npoly; ++k) acc[k] = fma(momw[(long)k * nb3 + m], v, acc[k]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < npoly; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < npoly) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        mom[(long)p * npoly + threadIdx.x] = v;
    }
}

// r^i[a] = phi^i[g_a] - I^H(phi^i)(g_a) on the face nodes of Omega_alpha.
template <typename TB>
__global__ void __launch_bounds__(256) k_resid(const TB *__restrict__ box, long W3, int na,
                                               int S, const int *__restrict__ a_self,
                                               const int *__restrict__ a_off,
                                               const double *__restrict__ a_w,
                                               double *__restrict__ resid) {
    const int p = blockIdx.x;
    const int a = blockIdx.y * blockDim.x + threadIdx.x;
    if (a >= na) return;
    const TB *bx = box + (long)p * W3;
    double acc = 0.0;
    for (int j = 0; j < S; ++j) acc = fma(a_w[(long)a * S + j], (double)bx[a_off[(long)a * S + j]], acc);
    resid[(long)p * na + a] = (double)bx[a_self[a]] - acc;
}

struct AsmArgs {
    const void *box;
    const double *mom, *T;
    double *FH;
    int np, n, s, W, npoly, flo, nf;
    int ca_lo, ca_hi, cb_lo, cb_hi;
    double coef[4];  // b_k / H^2
};

// F^H[k] = sum over patches i (ascending) of Delta^H phi^{i,h} on C(Omega_alpha(i))
// or sum_p c_p^i Delta^H(G^h * Q^p) on C(Omega_beta(i)) \ C(Omega_alpha(i)).
template <typename TB>
__global__ void __launch_bounds__(128) k_assemble(AsmArgs a) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long tot = (long)a.nf * a.nf * a.nf;
    if (idx >= tot) return;
    int k[3];
    k[2] = (int)(idx % a.nf) + a.flo;
    k[1] = (int)((idx / a.nf) % a.nf) + a.flo;
    k[0] = (int)(idx / ((long)a.nf * a.nf)) + a.flo;
    const int q = a.n / 4;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = max(0, -floordiv(-(k[d] - a.cb_hi), q));  // ceil((k - cb_hi)/q)
        hi[d] = min(a.np - 1, floordiv(k[d] - a.cb_lo, q));
    }
    const int ncb = a.cb_hi - a.cb_lo + 1;
    const long W = a.W;
    double acc = 0.0;
    for (int i0 = lo[0]; i0 <= hi[0]; ++i0)
        for (int i1 = lo[1]; i1 <= hi[1]; ++i1)
            for (int i2 = lo[2]; i2 <= hi[2]; ++i2) {
                const int r0 = k[0] - q * i0, r1 = k[1] - q * i1, r2 = k[2] - q * i2;
                const long p = ((long)i0 * a.np + i1) * a.np + i2;
                const bool inA = r0 >= a.ca_lo && r0 <= a.ca_hi && r1 >= a.ca_lo &&
                                 r1 <= a.ca_hi && r2 >= a.ca_lo && r2 <= a.ca_hi;
                if (inA) {
                    const TB *bx = (const TB *)a.box + p * W * W * W;
                    double lap = 0.0;
                    for (int s0 = -1; s0 <= 1; ++s0)
                        for (int s1 = -1; s1 <= 1; ++s1)
                            for (int s2 = -1; s2 <= 1; ++s2) {
                                const int nz = (s0 != 0) + (s1 != 0) + (s2 != 0);
                                const double c = a.coef[nz];
                                if (c == 0.0) continue;
                                const long x0 = 4 * (r0 + s0) + a.s, x1 = 4 * (r1 + s1) + a.s,
                                           x2 = 4 * (r2 + s2) + a.s;
                                lap = fma(c, (double)bx[(x0 * W + x1) * W + x2], lap);
                            }
                    acc += lap;
                } else {
                    const long t = (((long)(r0 - a.cb_lo) * ncb + (r1 - a.cb_lo)) * ncb +
                                    (r2 - a.cb_lo)) * a.npoly;
                    const double *c = a.mom + p * a.npoly;
                    double v = 0.0;
                    for (int pp = 0; pp < a.npoly; ++pp) v = fma(c[pp], a.T[t + pp], v);
                    acc += v;
                }
            }
    a.FH[idx] = acc;
}

struct BndArgs {
    const double *phiH, *resid, *mom, *D;
    const int *amap, *rmap;
    double *phiB;
    int N, n, np, ga, gb, b, npoly, na, olo, no, wa, wbx;
    double lw[4][8];  // Lagrange weights for g mod 4 = r (row r), 2b+2 entries
};

// phi^B at every face-plane node (axis, plane j, u, v).
__global__ void __launch_bounds__(128) k_boundary(BndArgs a) {
    const long pn = (long)(a.N + 1) * (a.N + 1);
    const long tot = 3L * (a.np + 1) * pn;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int axis = (int)(idx / ((a.np + 1) * pn));
    const int j = (int)((idx / pn) % (a.np + 1));
    const int u = (int)((idx % pn) / (a.N + 1)), v = (int)(idx % (a.N + 1));
    int g[3];
    g[axis] = j * a.n;
    g[axis == 0 ? 1 : 0] = u;
    g[axis == 2 ? 1 : 2] = v;
    // I^H(phi^H)(g): tensor Lagrange over the in-plane axes (R4)
    const int K = 2 * a.b + 2;
    int kb[3], cnt[3], rr[3];
    for (int d = 0; d < 3; ++d) {
        rr[d] = g[d] & 3;
        if (rr[d] == 0) {
            kb[d] = g[d] >> 2;
            cnt[d] = 1;
        } else {
            kb[d] = (g[d] >> 2) - a.b;
            cnt[d] = K;
        }
    }
    double acc = 0.0;
    for (int e0 = 0; e0 < cnt[0]; ++e0) {
        const double w0 = rr[0] ? a.lw[rr[0]][e0] : 1.0;
        for (int e1 = 0; e1 < cnt[1]; ++e1) {
            const double w1 = w0 * (rr[1] ? a.lw[rr[1]][e1] : 1.0);
            const long base = ((long)(kb[0] + e0 - a.olo) * a.no + (kb[1] + e1 - a.olo)) * a.no;
            for (int e2 = 0; e2 < cnt[2]; ++e2) {
                const double w = w1 * (rr[2] ? a.lw[rr[2]][e2] : 1.0);
                acc = fma(w, a.phiH[base + (kb[2] + e2 - a.olo)], acc);
            }
        }
    }
    // local corrections of the patches whose Omega_beta holds g (ascending index)
    int lo[3], hi[3], alo[3], ahi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = max(0, -floordiv(-(g[d] - a.n - a.gb), a.n));
        hi[d] = min(a.np - 1, floordiv(g[d] + a.gb, a.n));
        alo[d] = max(0, -floordiv(-(g[d] - a.n - a.ga), a.n));
        ahi[d] = min(a.np - 1, floordiv(g[d] + a.ga, a.n));
    }
    for (int i0 = lo[0]; i0 <= hi[0]; ++i0)
        for (int i1 = lo[1]; i1 <= hi[1]; ++i1)
            for (int i2 = lo[2]; i2 <= hi[2]; ++i2) {
                const long p = ((long)i0 * a.np + i1) * a.np + i2;
                const int r0 = g[0] - a.n * i0, r1 = g[1] - a.n * i1, r2 = g[2] - a.n * i2;
                const bool inA = i0 >= alo[0] && i0 <= ahi[0] && i1 >= alo[1] && i1 <= ahi[1] &&
                                 i2 >= alo[2] && i2 <= ahi[2];
                if (inA) {
                    const int ai = a.amap[((long)(r0 + a.ga) * a.wa + (r1 + a.ga)) * a.wa + (r2 + a.ga)];
                    acc += a.resid[p * a.na + ai];
                } else {
                    const int ri = a.rmap[((long)(r0 + a.gb) * a.wbx + (r1 + a.gb)) * a.wbx + (r2 + a.gb)];
                    const double *c = a.mom + p * a.npoly;
                    const double *Dr = a.D + (long)ri * a.npoly;
                    double vv = 0.0;
                    for (int pp = 0; pp < a.npoly; ++pp) vv = fma(c[pp], Dr[pp], vv);
                    acc += vv;
                }
            }
    a.phiB[idx] = acc;
}

struct DirArgs {
    const void *f;
    const double *phiB;
    double *phi;
    int N, n, np;
    double h2, c2h2;
    double b[4];
    const double *sinm;  // (n-1)^2: sin(pi k m / n), k, m in [1, n-1]
    const double *lam;   // (n-1)^3 eigenvalues (already / h^2)
};

__device__ __forceinline__ double phiB_at(const DirArgs &a, int g0, int g1, int g2) {
    const long pn = (long)(a.N + 1) * (a.N + 1);
    int axis, j, u, v;
    if (g0 % a.n == 0) {
        axis = 0; j = g0 / a.n; u = g1; v = g2;
    } else if (g1 % a.n == 0) {
        axis = 1; j = g1 / a.n; u = g0; v = g2;
    } else {
        axis = 2; j = g2 / a.n; u = g0; v = g1;
    }
    return a.phiB[((long)axis * (a.np + 1) + j) * pn + (long)u * (a.N + 1) + v];
}

template <typename TF>
__global__ void __launch_bounds__(256) k_dirichlet(DirArgs a) {
    extern __shared__ double sm[];
    const int n = a.n, nb = n + 1, m = n - 1;
    double *U = sm;                  // nb^3 boundary values (interior 0)
    double *X = U + nb * nb * nb;    // m^3 work
    double *Y = X + m * m * m;       // m^3 work
    double *S = Y + m * m * m;       // m^2 sine matrix
    const int p = blockIdx.x;
    const int i2 = p % a.np, i1 = (p / a.np) % a.np, i0 = p / (a.np * a.np);
    const int o0 = i0 * n, o1 = i1 * n, o2 = i2 * n;
    const TF *f = (const TF *)a.f;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) S[e] = a.sinm[e];
    for (int e = threadIdx.x; e < nb * nb * nb; e += blockDim.x) {
        const int m2 = e % nb, m1 = (e / nb) % nb, m0 = e / (nb * nb);
        const bool bnd = m0 == 0 || m0 == n || m1 == 0 || m1 == n || m2 == 0 || m2 == n;
        U[e] = bnd ? phiB_at(a, o0 + m0, o1 + m1, o2 + m2) : 0.0;
    }
    __syncthreads();
    // right-hand side on the interior: f - Delta^h(boundary data)
    for (int e = threadIdx.x; e < m * m * m; e += blockDim.x) {
        const int c2 = e % m + 1, c1 = (e / m) % m + 1, c0 = e / (m * m) + 1;
        double lap = 0.0;
        for (int s0 = -1; s0 <= 1; ++s0)
            for (int s1 = -1; s1 <= 1; ++s1)
                for (int s2 = -1; s2 <= 1; ++s2) {
                    const int nz = (s0 != 0) + (s1 != 0) + (s2 != 0);
                    const double c = a.b[nz];
                    if (c == 0.0) continue;
                    lap = fma(c, U[((c0 + s0) * nb + (c1 + s1)) * nb + (c2 + s2)], lap);
                }
        const int z = o0 + c0, y = o1 + c1, x = o2 + c2;
        const double fv = (z < a.N && y < a.N && x < a.N) ? (double)f[((long)z * a.N + y) * a.N + x] : 0.0;
        X[e] = fv - lap / a.h2;
    }
    __syncthreads();
    // DST-I along axes 2, 1, 0; divide; DST-I back along 2, 1, 0
    for (int pass = 0; pass < 6; ++pass) {
        const int axis = 2 - (pass % 3);
        double *src = (pass % 2 == 0) ? X : Y;
        double *dst = (pass % 2 == 0) ? Y : X;
        for (int e = threadIdx.x; e < m * m * m; e += blockDim.x) {
            const int c2 = e % m, c1 = (e / m) % m, c0 = e / (m * m);
            int kk, base, str;
            if (axis == 2) { kk = c2; base = (c0 * m + c1) * m; str = 1; }
            else if (axis == 1) { kk = c1; base = c0 * m * m + c2; str = m; }
            else { kk = c0; base = c1 * m + c2; str = m * m; }
            double v = 0.0;
            for (int t = 0; t < m; ++t) v = fma(S[kk * m + t], src[base + t * str], v);
            dst[e] = v;
        }
        __syncthreads();
        if (pass == 2) {
            for (int e = threadIdx.x; e < m * m * m; e += blockDim.x) Y[e] /= a.lam[e];
            __syncthreads();
        }
    }
    // after 6 passes the result is in X (passes alternate X->Y->X...; pass 5 writes X)
    const double norm = (2.0 / n) * (2.0 / n) * (2.0 / n);
    for (int e = threadIdx.x; e < n * n * n; e += blockDim.x) {
        const int m2 = e % n, m1 = (e / n) % n, m0 = e / (n * n);
        const bool bnd = m0 == 0 || m1 == 0 || m2 == 0;
        const double u = bnd ? U[(m0 * nb + m1) * nb + m2]
                             : X[((m0 - 1) * m + (m1 - 1)) * m + (m2 - 1)] * norm;
        const int z = o0 + m0, y = o1 + m1, x = o2 + m2;
        const long gi = ((long)z * a.N + y) * a.N + x;
        a.phi[gi] = u + a.c2h2 * (double)f[gi];
    }
}

template <typename R>
inline size_t fft_smem_bytes(int M, int lines, int ls) {
    return ((size_t)(M / 2) + (size_t)lines * ls) * 2 * sizeof(R);
}

template <int LOG2M, typename R>
void set_smem_attrs() {
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_fwd_x<LOG2M, double, true, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fwd_x<LOG2M, float, true, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fwd_x<LOG2M, double, false, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_col<LOG2M, 0, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_col<LOG2M, 1, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_col<LOG2M, 2, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_inv_x<LOG2M, R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// One Hockney convolution pipeline (5 launches) for `nbatch` problems with
// nin input nodes per axis at positions [0, nin) and nout outputs per axis
// from positions out_off + t.  R: working precision; output array of type R.
struct ConvDesc {
    int M, log2M, nbatch, nin, nout, out_off;
    const void *src;     // fwd_x input (patch gather or dense FP64)
    bool patch, f32;
    int N, n, np;
    void *b0, *b1;       // ping-pong spectra (complex R)
    void *out;           // nbatch x nout^3, type R
    const void *khat;    // real R
    const void *tw;      // complex R
    const mlc_plan_s *pl;  // timing events (slots ev0 .. ev0+4)
    int ev0;
};

template <int LOG2M, typename R>
cudaError_t run_conv_t(const ConvDesc &d, cudaStream_t st) {
    constexpr int M = 1 << LOG2M, MH = M / 2 + 1;
    const int nin = d.nin, W = d.nout;
    mark(d.pl, d.ev0 + 0, st);
    // 1. forward x: out A1[p][zi][yi][kx]
    {
        FwdXArgs a{d.src, d.b0, d.N, d.n, d.np, nin, 0, d.tw};
        a.lines_cta = (M <= 64) ? nin : 16;
        a.lines_cta = a.lines_cta > nin ? nin : a.lines_cta;
        dim3 grid(d.nbatch * nin, (nin + a.lines_cta - 1) / a.lines_cta);
        size_t sm = fft_smem_bytes<R>(M, a.lines_cta, M + 1);
        if (d.patch) {
            if (d.f32) k_fwd_x<LOG2M, float, true, R><<<grid, 256, sm, st>>>(a);
            else k_fwd_x<LOG2M, double, true, R><<<grid, 256, sm, st>>>(a);
        } else {
            k_fwd_x<LOG2M, double, false, R><<<grid, 256, sm, st>>>(a);
        }
    }
    const int CC = (M <= 64) ? MH : 16;
    const int gx = (MH + CC - 1) / CC;
    const size_t smc = fft_smem_bytes<R>(M, M, CC);
    mark(d.pl, d.ev0 + 1, st);
    // 2. forward y: A1[p][zi][yi][kx] -> A2[p][zi][ky][kx]
    {
        ColArgs a{};
        a.in = d.b0; a.out = d.b1; a.S2 = nin;
        a.in_sp = (long)nin * nin * MH; a.in_sq = (long)nin * MH; a.in_row = MH;
        a.out_sp = (long)nin * M * MH; a.out_sq = (long)M * MH; a.out_row = MH;
        a.ncols = MH; a.cols_cta = CC; a.nin = nin; a.nout = M; a.out_off = 0; a.tw = d.tw;
        k_col<LOG2M, 0, R><<<dim3(d.nbatch * nin, gx), 256, smc, st>>>(a);
    }
    mark(d.pl, d.ev0 + 2, st);
    // 3. z: forward, x kernel, inverse: A2[p][zi][ky][kx] -> A3[p][zo][ky][kx]
    {
        ColArgs a{};
        a.in = d.b1; a.out = d.b0; a.S2 = M;
        a.in_sp = (long)nin * M * MH; a.in_sq = MH; a.in_row = (long)M * MH;
        a.out_sp = (long)W * M * MH; a.out_sq = MH; a.out_row = (long)M * MH;
        a.ncols = MH; a.cols_cta = CC; a.nin = nin; a.nout = W; a.out_off = d.out_off;
        a.khat = d.khat; a.tw = d.tw;
        k_col<LOG2M, 2, R><<<dim3(d.nbatch * M, gx), 256, smc, st>>>(a);
    }
    mark(d.pl, d.ev0 + 3, st);
    // 4. inverse y: A3[p][zo][ky][kx] -> A4[p][zo][yo][kx]
    {
        ColArgs a{};
        a.in = d.b0; a.out = d.b1; a.S2 = W;
        a.in_sp = (long)W * M * MH; a.in_sq = (long)M * MH; a.in_row = MH;
        a.out_sp = (long)W * W * MH; a.out_sq = (long)W * MH; a.out_row = MH;
        a.ncols = MH; a.cols_cta = CC; a.nin = M; a.nout = W; a.out_off = d.out_off; a.tw = d.tw;
        k_col<LOG2M, 1, R><<<dim3(d.nbatch * W, gx), 256, smc, st>>>(a);
    }
    mark(d.pl, d.ev0 + 4, st);
    // 5. inverse x (real): A4[p][zo][yo][kx] -> out[p][zo][yo][xo]
    {
        InvXArgs a{d.b1, d.out, W, W, d.out_off, 0, d.tw};
        a.lines_cta = (M <= 64) ? W : 16;
        dim3 grid(d.nbatch * W, (W + a.lines_cta - 1) / a.lines_cta);
        k_inv_x<LOG2M, R, R><<<grid, 256, fft_smem_bytes<R>(M, a.lines_cta, M + 1), st>>>(a);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t run_conv(const ConvDesc &d, cudaStream_t st) {
    switch (d.log2M) {
        case 5: return run_conv_t<5, R>(d, st);
        case 6: return run_conv_t<6, R>(d, st);
        case 7: return run_conv_t<7, R>(d, st);
        case 8: return run_conv_t<8, R>(d, st);
        default: return cudaErrorInvalidValue;
    }
}

void stencil_b(int Q, double b[4]) {
    if (Q == 4) {
        b[0] = -4.0; b[1] = 1.0 / 3.0; b[2] = 1.0 / 6.0; b[3] = 0.0;
    } else {
        b[0] = -64.0 / 15.0; b[1] = 7.0 / 15.0; b[2] = 1.0 / 10.0; b[3] = 1.0 / 30.0;
    }
}

}  // namespace

void configure_kernels() {
    set_smem_attrs<5, double>();
    set_smem_attrs<6, double>();
    set_smem_attrs<7, double>();
    set_smem_attrs<8, double>();
    set_smem_attrs<5, float>();
    set_smem_attrs<6, float>();
    cudaFuncSetAttribute(k_dirichlet<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_dirichlet<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_moments(const mlc_plan_s *pl, const void *f, bool f32, cudaStream_t st) {
    const Geom &g = pl->g;
    if (f32)
        k_moments<float><<<g.NP, 256, 0, st>>>((const float *)f, g.N, g.n, g.np, g.npoly, pl->momw, pl->mom);
    else
        k_moments<double><<<g.NP, 256, 0, st>>>((const double *)f, g.N, g.n, g.np, g.npoly, pl->momw, pl->mom);
    return cudaGetLastError();
}

cudaError_t launch_patch_conv(const mlc_plan_s *pl, const void *f, bool f32, cudaStream_t st) {
    const Geom &g = pl->g;
    ConvDesc d{};
    d.M = g.M; d.log2M = g.log2M; d.nbatch = g.NP; d.nin = g.nb; d.nout = g.W; d.out_off = -g.s;
    d.src = f; d.patch = true; d.f32 = f32; d.N = g.N; d.n = g.n; d.np = g.np;
    d.b0 = pl->buf0; d.b1 = pl->buf1; d.out = pl->box; d.pl = pl; d.ev0 = 1;
    if (pl->g.tier == MLC_TIER_SPLIT) {
        d.khat = pl->khat_f; d.tw = pl->tw_f;
        return run_conv<float>(d, st);
    }
    d.khat = pl->khat; d.tw = pl->tw;
    return run_conv<double>(d, st);
}

cudaError_t launch_resid(const mlc_plan_s *pl, cudaStream_t st) {
    const Geom &g = pl->g;
    dim3 grid(g.NP, (g.na_face + 255) / 256);
    if (g.tier == MLC_TIER_SPLIT)
        k_resid<float><<<grid, 256, 0, st>>>((const float *)pl->box, (long)g.W * g.W * g.W, g.na_face,
                                             g.S, pl->a_self, pl->a_off, pl->a_w, pl->resid);
    else
        k_resid<double><<<grid, 256, 0, st>>>((const double *)pl->box, (long)g.W * g.W * g.W, g.na_face,
                                              g.S, pl->a_self, pl->a_off, pl->a_w, pl->resid);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const mlc_plan_s *pl, cudaStream_t st) {
    const Geom &g = pl->g;
    AsmArgs a{};
    a.box = pl->box; a.mom = pl->mom; a.T = pl->Ttab; a.FH = pl->FH;
    a.np = g.np; a.n = g.n; a.s = g.s; a.W = g.W; a.npoly = g.npoly; a.flo = g.flo; a.nf = g.nf;
    a.ca_lo = g.ca_lo; a.ca_hi = g.ca_hi; a.cb_lo = g.cb_lo; a.cb_hi = g.cb_hi;
    double b[4];
    stencil_b(g.Q, b);
    for (int k = 0; k < 4; ++k) a.coef[k] = b[k] / (g.H * g.H);
    const long tot = (long)g.nf * g.nf * g.nf;
    if (g.tier == MLC_TIER_SPLIT)
        k_assemble<float><<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(a);
    else
        k_assemble<double><<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_coarse(const mlc_plan_s *pl, cudaStream_t st) {
    const Geom &g = pl->g;
    ConvDesc d{};
    d.M = g.Mc; d.log2M = g.log2Mc; d.nbatch = 1; d.nin = g.nf; d.nout = g.no;
    d.out_off = g.olo - g.flo;
    d.src = pl->FH; d.patch = false; d.f32 = false;
    d.b0 = pl->cbuf0; d.b1 = pl->cbuf1; d.out = pl->phiH; d.khat = pl->khat_c; d.tw = pl->tw_c;
    d.pl = pl; d.ev0 = 8;
    return run_conv<double>(d, st);
}

cudaError_t launch_boundary(const mlc_plan_s *pl, cudaStream_t st) {
    const Geom &g = pl->g;
    BndArgs a{};
    a.phiH = pl->phiH; a.resid = pl->resid; a.mom = pl->mom; a.D = pl->Dtab;
    a.amap = pl->amap; a.rmap = pl->rmap; a.phiB = pl->phiB;
    a.N = g.N; a.n = g.n; a.np = g.np; a.ga = g.ga; a.gb = g.gb; a.b = g.b; a.npoly = g.npoly;
    a.na = g.na_face; a.olo = g.olo; a.no = g.no; a.wa = g.wa; a.wbx = g.wbx;
    // Lagrange weights on the nodes k0-b .. k0+b+1 at t = k0 + r/4 (R4)
    const int K = 2 * g.b + 2;
    for (int r = 0; r < 4; ++r)
        for (int j = 0; j < 8; ++j) a.lw[r][j] = 0.0;
    for (int r = 1; r < 4; ++r)
        for (int j = 0; j < K; ++j) {
            double w = 1.0;
            const double t = r / 4.0 + g.b;  // position relative to the first node
            for (int l = 0; l < K; ++l)
                if (l != j) w *= (t - l) / (double)(j - l);
            a.lw[r][j] = w;
        }
    const long tot = g.n_planes_total;
    k_boundary<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dirichlet(const mlc_plan_s *pl, const void *f, bool f32, double *phi,
                             cudaStream_t st) {
    const Geom &g = pl->g;
    DirArgs a{};
    a.f = f; a.phiB = pl->phiB; a.phi = phi; a.N = g.N; a.n = g.n; a.np = g.np;
    a.h2 = g.h * g.h; a.c2h2 = g.h * g.h / 12.0;
    stencil_b(g.Q, a.b);
    a.sinm = pl->sinm; a.lam = pl->lam;
    const int nb = g.n + 1, m = g.n - 1;
    const size_t sm = sizeof(double) * ((size_t)nb * nb * nb + 2 * (size_t)m * m * m + (size_t)m * m);
    if (f32) k_dirichlet<float><<<g.NP, 256, sm, st>>>(a);
    else k_dirichlet<double><<<g.NP, 256, sm, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mlc
