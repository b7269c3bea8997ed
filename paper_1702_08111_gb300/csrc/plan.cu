// Host side of the MLC library: parameter checks, plan geometry and index
// tables (Sec. 4 regions), plan-time tables, the solve sequence and the C ABI.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mlc_internal.h"

using namespace mlc;

thread_local bool mlc::g_capturing = false;
void mlc_batch_forget(mlc_plan_t plan);

namespace {

int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
int ceildiv(int a, int b) { return -floordiv(-a, b); }
int fmod_pos(int a, int b) { int r = a % b; return r < 0 ? r + b : r; }

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

void stencil_b(int Q, double b[4]) {
    if (Q == 4) {
        b[0] = -4.0; b[1] = 1.0 / 3.0; b[2] = 1.0 / 6.0; b[3] = 0.0;
    } else {
        b[0] = -64.0 / 15.0; b[1] = 7.0 / 15.0; b[2] = 1.0 / 10.0; b[3] = 1.0 / 30.0;
    }
}

double symbol(int Q, double c0, double c1, double c2) {
    if (Q == 10) {  // sum_j a_j prod_d cos(j_d theta_d), cos(2 theta) = 2 c^2 - 1
        const double c[3] = {c0, c1, c2};
        double lam = 0.0;
        for (int s0 = -2; s0 <= 2; ++s0)
            for (int s1 = -2; s1 <= 2; ++s1)
                for (int s2 = -2; s2 <= 2; ++s2) {
                    const double a = stencil_coef(10, s0, s1, s2);
                    if (a == 0.0) continue;
                    double t = a;
                    const int ss[3] = {s0, s1, s2};
                    for (int d = 0; d < 3; ++d) {
                        const int k = std::abs(ss[d]);
                        t *= k == 0 ? 1.0 : (k == 1 ? c[d] : 2.0 * c[d] * c[d] - 1.0);
                    }
                    lam += t;
                }
        return lam;
    }
    double b[4];
    stencil_b(Q, b);
    return b[0] + 2.0 * b[1] * (c0 + c1 + c2) + 4.0 * b[2] * (c0 * c1 + c0 * c2 + c1 * c2) +
           8.0 * b[3] * c0 * c1 * c2;
}

// Orthonormal Legendre polynomial sqrt((2k+1)/2) P_k(t) by the three-term recurrence.
double legendre(int k, double t) {
    double p0 = 1.0, p1 = t;
    if (k == 0) return std::sqrt(0.5);
    for (int j = 1; j < k; ++j) {
        double p2 = ((2.0 * j + 1.0) * t * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return std::sqrt((2.0 * k + 1.0) / 2.0) * p1;
}

// 1D factor of the interpolant I^H at fine coordinate x (R4 reading of Sec. 4, Step 3).
void axis_stencil(int x, int b, std::vector<int> &nodes, std::vector<double> &w) {
    nodes.clear();
    w.clear();
    if (fmod_pos(x, 4) == 0) {
        nodes.push_back(floordiv(x, 4));
        w.push_back(1.0);
        return;
    }
    const int k0 = floordiv(x, 4), K = 2 * b + 2;
    const double t = (double)(x - 4 * k0) / 4.0 + b;
    for (int j = 0; j < K; ++j) {
        double v = 1.0;
        for (int l = 0; l < K; ++l)
            if (l != j) v *= (t - l) / (double)(j - l);
        nodes.push_back(k0 - b + j);
        w.push_back(v);
    }
}

// Full stencil of I^H at a face-lattice point: tensor product of the axis factors.
void face_stencil(const int g[3], int b, std::vector<std::array<int, 3>> &pts, std::vector<double> &w) {
    std::vector<int> n0, n1, n2;
    std::vector<double> w0, w1, w2;
    axis_stencil(g[0], b, n0, w0);
    axis_stencil(g[1], b, n1, w1);
    axis_stencil(g[2], b, n2, w2);
    pts.clear();
    w.clear();
    for (size_t a = 0; a < n0.size(); ++a)
        for (size_t c = 0; c < n1.size(); ++c)
            for (size_t e = 0; e < n2.size(); ++e) {
                pts.push_back({n0[a], n1[c], n2[e]});
                w.push_back(w0[a] * w1[c] * w2[e]);
            }
}

bool on_face(const int g[3], int n) {
    return fmod_pos(g[0], n) == 0 || fmod_pos(g[1], n) == 0 || fmod_pos(g[2], n) == 0;
}

// ---- per-device DGF table cache (tables stay resident until process exit) ----
struct DgfEntry {
    double *ptr;
    int L;
};
std::mutex g_dgf_mu;
std::map<std::tuple<int, int, int, int>, DgfEntry> g_dgf;
std::once_flag g_cfg_once;

mlc_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return MLC_OK;
    if (e == cudaErrorMemoryAllocation) return MLC_ERR_OOM;
    return MLC_ERR_CUDA;
}

#define TRY_CUDA(x)                               \
    do {                                          \
        cudaError_t _e = (x);                     \
        if (_e != cudaSuccess) return to_status(_e); \
    } while (0)

template <typename T>
mlc_status dev_upload(mlc_plan_s *pl, T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return MLC_OK;
    void *p = nullptr;
    TRY_CUDA(cudaMalloc(&p, src.size() * sizeof(T)));
    pl->owned.push_back(p);
    TRY_CUDA(cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = (T *)p;
    return MLC_OK;
}

template <typename T>
mlc_status dev_alloc(mlc_plan_s *pl, T **dst, size_t count, bool workspace = true) {
    *dst = nullptr;
    if (count == 0) return MLC_OK;
    void *p = nullptr;
    TRY_CUDA(cudaMalloc(&p, count * sizeof(T)));
    pl->owned.push_back(p);
    if (workspace) pl->ws_bytes += count * sizeof(T);
    *dst = (T *)p;
    return MLC_OK;
}

#define TRY(x)                             \
    do {                                   \
        mlc_status _s = (x);               \
        if (_s != MLC_OK) return _s;       \
    } while (0)

mlc_status derive_geometry(const mlc_params &pp, Geom &g) {
    g = Geom{};
    g.N = pp.N; g.n = pp.n; g.s = pp.s; g.C = pp.C; g.P = pp.P; g.Q = pp.Q;
    if (g.C != 4) return MLC_ERR_INVALID_ARG;
    if (g.Q != 4 && g.Q != 6 && g.Q != 10) return MLC_ERR_INVALID_ARG;
    g.wide = stencil_reach(g.Q) > 1;
    if (g.N <= 0 || g.n <= 0 || g.s < 0 || g.P < 1 || g.P > 6) return MLC_ERR_INVALID_ARG;
    if (g.N % g.n || g.n % 4 || g.s % 4) return MLC_ERR_INVALID_ARG;
    // q_I = 2b + 2 = q + 2 for L19 and L27 (Sec. 7); b = 4 for Q = 10 (R18)
    g.b = pp.b < 0 ? (g.Q == 4 ? 2 : (g.Q == 6 ? 3 : 4)) : pp.b;
    if (g.b < 1 || g.b > 5) return MLC_ERR_INVALID_ARG;
    g.ga = g.s - g.C * g.b;
    if (g.ga < 0) return MLC_ERR_INVALID_ARG;
    g.mode = pp.mode < 0 ? MLC_MODE_MLC : pp.mode;
    g.levels = pp.levels < 0 ? 2 : pp.levels;
    if (g.levels < 2 || g.levels > 6) return MLC_ERR_INVALID_ARG;
    g.tier = pp.tier < 0 ? MLC_TIER_FP64 : pp.tier;
    if (!tier_valid(g.tier)) return MLC_ERR_INVALID_ARG;
    g.conv = tier_conv(g.tier);
    g.fine = tier_fine(g.tier);
    g.f32in = tier_f32_charge(g.tier);
    if (g.mode == MLC_MODE_MLC0) {
        g.gb = g.ga;
    } else if (pp.g_beta >= 0) {
        g.gb = pp.g_beta;
    } else {
        // beta = 3 (Q = 4) or 13/4 (Q = 6, and Q = 10 by R18): g_beta = ceil((beta - 1) n / 2)
        g.gb = (g.Q == 4) ? g.n : ceildiv(9 * g.n, 8);
    }
    if (g.gb < g.ga) return MLC_ERR_INVALID_ARG;
    g.h = 1.0 / g.N;
    g.H = g.C * g.h;
    g.R = g.n * g.h / 2.0;
    g.np = g.N / g.n;
    g.NP = g.np * g.np * g.np;
    g.npoly = 0;
    for (int a = 0; a < g.P; ++a)
        for (int c = 0; c < g.P; ++c)
            for (int e = 0; e < g.P; ++e)
                if (a + c + e < g.P) ++g.npoly;
    g.npad = (g.npoly + 3) & ~3;
    g.nb = g.n + 1;
    g.W = g.n + 2 * g.s + 1;
    g.M = next_pow2(2 * (g.n + g.s));
    g.log2M = ilog2(g.M);
    g.Mh = g.M / 2 + 1;
    g.ca_lo = floordiv(-g.ga, 4); g.ca_hi = ceildiv(g.n + g.ga, 4);
    g.cb_lo = floordiv(-g.gb, 4); g.cb_hi = ceildiv(g.n + g.gb, 4);
    g.flo = g.cb_lo;
    g.fhi = (g.np - 1) * (g.n / 4) + g.cb_hi;
    g.nf = g.fhi - g.flo + 1;
    // R6; R18: the second boundary layer's stencils reach one coarse node further
    g.olo = -g.b - (g.wide ? 1 : 0); g.ohi = g.N / 4 + g.b + (g.wide ? 1 : 0);
    g.no = g.ohi - g.olo + 1;
    g.Lc = std::max(g.fhi - g.olo, g.ohi - g.flo);
    // coarse Hockney period: the smallest even length >= 2 Lc (and >= the
    // extents) whose only prime factors are 2, 3 and 5 (mixed-radix FFTs)
    {
        auto smooth = [](int m) {
            for (int r : {2, 3, 5})
                while (m % r == 0) m /= r;
            return m == 1;
        };
        int mc = std::max(2 * g.Lc, std::max(g.nf, g.no));
        mc += mc & 1;
        while (!smooth(mc)) mc += 2;
        g.Mc = mc;
    }
    g.log2Mc = 0;
    g.Mhc = g.Mc / 2 + 1;
    // patch sizes with a Dirichlet kernel instantiation; patch periods 32 to
    // 128 (at 128 the FP64 and double-float slabs stream their rows)
    if (g.n != 4 && g.n != 8 && g.n != 12 && g.n != 16 && g.n != 24 && g.n != 32) return MLC_ERR_UNSUPPORTED;
    // (a multilevel plan's own coarse period is never used: its coarse solve
    // is the next level's MLC solve)
    if (g.M < 32 || g.M > 128 || (g.levels <= 2 && g.Mc > 512)) return MLC_ERR_UNSUPPORTED;
    // Q = 10 (R18): two levels, FP64 boundary and Dirichlet steps (tiers FP64
    // and SPLIT), and patches whose two-layer Dirichlet arrays fit shared memory
    if (g.wide && (g.levels != 2 || g.fine != FINE_F64)) return MLC_ERR_UNSUPPORTED;
    if (g.wide && g.b < 2) return MLC_ERR_INVALID_ARG;  // Delta^H reaches two coarse nodes past C(alpha)
    g.S = (2 * g.b + 2) * (2 * g.b + 2);
    g.nc = (g.n + 2 * g.s) / 4 + 1;
    g.nzr = 0;
    for (int zi = 0; zi < g.W; ++zi) {
        const int z = zi - g.s;
        if ((z >= -g.ga && z <= g.n + g.ga) || (z % 4 == 0)) ++g.nzr;
    }
    {
        const int cb = 2 * conv_real_bytes(g.tier);         // bytes per complex entry
        const int per16 = 16 / cb;                          // entries per 16 bytes
        g.a4blk = ((g.Mh * g.W + per16 - 1) / per16) * per16;
    }
    {
        const size_t cb = 2 * (size_t)conv_real_bytes(g.tier);
        g.scr_a1 = (size_t)g.Mh * g.nb * g.nb * cb;
        g.scr_a4 = (size_t)g.nzr * g.a4blk * cb;
        g.chunk = pp.conv_chunk > 0 ? pp.conv_chunk : 1024;
    }
    g.wa = g.n + 2 * g.ga + 1;
    g.wbx = g.n + 2 * g.gb + 1;
    g.plane_n = (g.N + 1) * (g.N + 1);
    g.n_planes_total = 3L * (g.np + 1) * (long)g.plane_n;
    g.zeta = pp.dgf_zeta < 0 ? 2 : pp.dgf_zeta;
    g.nD = pp.dgf_nD < 0 ? 128 : pp.dgf_nD;
    return MLC_OK;
}

// Host tables for one plan; basis fields need the DGF on the device.
mlc_status build_tables(mlc_plan_s *pl) {
    Geom &g = pl->g;
    const int n = g.n, nb = g.nb, nb3 = nb * nb * nb, W = g.W;
    // Legendre basis at the patch nodes (R3), Boole weights, chi
    std::vector<std::array<int, 3>> pidx;
    for (int a = 0; a < g.P; ++a)
        for (int c = 0; c < g.P; ++c)
            for (int e = 0; e < g.P; ++e)
                if (a + c + e < g.P) pidx.push_back({a, c, e});
    std::vector<double> bw(nb, 0.0), chi1(nb, 1.0);
    const double panel[5] = {7.0, 32.0, 12.0, 32.0, 7.0};
    for (int pn = 0; pn < n / 4; ++pn)
        for (int k = 0; k < 5; ++k) bw[4 * pn + k] += (2.0 * g.h / 45.0) * panel[k];
    chi1[0] = chi1[n] = 0.5;
    std::vector<double> leg((size_t)g.P * nb);
    for (int k = 0; k < g.P; ++k)
        for (int m = 0; m < nb; ++m) leg[(size_t)k * nb + m] = legendre(k, 2.0 * m / n - 1.0);
    const double rs = std::pow(g.R, -1.5);
    std::vector<double> lcharge((size_t)g.npoly * nb3);
    for (int p = 0; p < g.npoly; ++p)
        for (int m0 = 0; m0 < nb; ++m0)
            for (int m1 = 0; m1 < nb; ++m1)
                for (int m2 = 0; m2 < nb; ++m2) {
                    const double q = rs * leg[(size_t)pidx[p][0] * nb + m0] *
                                     leg[(size_t)pidx[p][1] * nb + m1] *
                                     leg[(size_t)pidx[p][2] * nb + m2];
                    const size_t m = ((size_t)m0 * nb + m1) * nb + m2;
                    lcharge[(size_t)p * nb3 + m] = chi1[m0] * chi1[m1] * chi1[m2] * q;
                }
    // moments are separable: 1D weights a_k(m) = w_m q_k(m), R^{-3/2} applied in the kernel
    std::vector<double> a1d((size_t)g.P * nb);
    for (int k = 0; k < g.P; ++k)
        for (int m = 0; m < nb; ++m) a1d[(size_t)k * nb + m] = bw[m] * leg[(size_t)k * nb + m];
    TRY(dev_upload(pl, &pl->momw, a1d));

    // face planes of the patch lattice inside Omega_alpha (relative x = pl0 + j n)
    g.pl0 = g.n * ceildiv(-g.ga, g.n);
    g.npa = 0;
    for (int c = g.pl0; c <= n + g.ga; c += n) ++g.npa;
    // every interpolation stencil of a face node of Omega_alpha stays in the field box
    if (4 * (-g.ga / 4 - g.b) < -g.s || 4 * ((n + g.ga) / 4 + g.b) > n + g.s) return MLC_ERR_INVALID_ARG;
    (void)W;

    // ring: face nodes in Omega_beta \ Omega_alpha and coarse nodes C(beta) \ C(alpha)
    std::vector<std::array<int, 3>> sp;
    std::vector<double> sw;
    std::vector<int> rmap((size_t)g.wbx * g.wbx * g.wbx, -1);
    std::vector<std::array<int, 3>> ring_nodes;
    std::vector<std::vector<std::array<int, 3>>> ring_st;
    std::vector<std::vector<double>> ring_w;
    const bool ring = g.gb > g.ga;
    const int ncb = g.cb_hi - g.cb_lo + 1;
    std::vector<double> Ttab;
    std::vector<double> Dtab;
    // R18 (Q = 10): ring rows of the nodes one node off the face planes
    std::vector<int> omap(g.wide ? (size_t)g.wbx * g.wbx * g.wbx : 0, -1), oself;
    std::vector<std::vector<int>> ost;
    std::vector<std::vector<double>> ow;
    std::vector<double> Dout;
    if (ring) {
        for (int x0 = -g.gb; x0 <= n + g.gb; ++x0)
            for (int x1 = -g.gb; x1 <= n + g.gb; ++x1)
                for (int x2 = -g.gb; x2 <= n + g.gb; ++x2) {
                    const int gg[3] = {x0, x1, x2};
                    if (!on_face(gg, n)) continue;
                    const bool inA = x0 >= -g.ga && x0 <= n + g.ga && x1 >= -g.ga &&
                                     x1 <= n + g.ga && x2 >= -g.ga && x2 <= n + g.ga;
                    if (inA) continue;
                    rmap[((size_t)(x0 + g.gb) * g.wbx + (x1 + g.gb)) * g.wbx + (x2 + g.gb)] =
                        (int)ring_nodes.size();
                    ring_nodes.push_back({x0, x1, x2});
                    face_stencil(gg, g.b, sp, sw);
                    ring_st.push_back(sp);
                    ring_w.push_back(sw);
                }
        // basis-field evaluation points: ring nodes, their stencils, and the
        // fine nodes under Delta^H on the coarse ring
        const int pad = 4 * g.b + 12;
        const int blo = -g.gb - pad, bhi = n + g.gb + pad, bw_ = bhi - blo + 1;
        std::vector<int> pmap((size_t)bw_ * bw_ * bw_, -1);
        std::vector<int> pts;
        auto add = [&](int y0, int y1, int y2) -> int {
            int &slot = pmap[((size_t)(y0 - blo) * bw_ + (y1 - blo)) * bw_ + (y2 - blo)];
            if (slot < 0) {
                slot = (int)(pts.size() / 3);
                pts.push_back(y0); pts.push_back(y1); pts.push_back(y2);
            }
            return slot;
        };
        std::vector<int> rn_self(ring_nodes.size());
        std::vector<std::vector<int>> rn_st(ring_nodes.size());
        for (size_t r = 0; r < ring_nodes.size(); ++r) {
            rn_self[r] = add(ring_nodes[r][0], ring_nodes[r][1], ring_nodes[r][2]);
            for (auto &k : ring_st[r]) rn_st[r].push_back(add(4 * k[0], 4 * k[1], 4 * k[2]));
        }
        // R18: ring nodes one node off the face planes (the second boundary
        // layer of Q = 10), with the interpolation stencil on every axis
        if (g.wide) {
            for (int x0 = -g.gb; x0 <= n + g.gb; ++x0)
                for (int x1 = -g.gb; x1 <= n + g.gb; ++x1)
                    for (int x2 = -g.gb; x2 <= n + g.gb; ++x2) {
                        const int gg[3] = {x0, x1, x2};
                        bool off = false;
                        for (int d = 0; d < 3; ++d) {
                            const int m = fmod_pos(gg[d], n);
                            off = off || m == 1 || m == n - 1;
                        }
                        if (!off) continue;
                        const bool inA = x0 >= -g.ga && x0 <= n + g.ga && x1 >= -g.ga &&
                                         x1 <= n + g.ga && x2 >= -g.ga && x2 <= n + g.ga;
                        if (inA) continue;
                        omap[((size_t)(x0 + g.gb) * g.wbx + (x1 + g.gb)) * g.wbx + (x2 + g.gb)] =
                            (int)oself.size();
                        oself.push_back(add(x0, x1, x2));
                        face_stencil(gg, g.b, sp, sw);
                        std::vector<int> st_;
                        for (auto &k : sp) st_.push_back(add(4 * k[0], 4 * k[1], 4 * k[2]));
                        ost.push_back(st_);
                        ow.push_back(sw);
                    }
        }
        const int reach = stencil_reach(g.Q);
        std::vector<std::vector<std::pair<int, double>>> lapT((size_t)ncb * ncb * ncb);
        for (int k0 = g.cb_lo; k0 <= g.cb_hi; ++k0)
            for (int k1 = g.cb_lo; k1 <= g.cb_hi; ++k1)
                for (int k2 = g.cb_lo; k2 <= g.cb_hi; ++k2) {
                    const bool inA = k0 >= g.ca_lo && k0 <= g.ca_hi && k1 >= g.ca_lo &&
                                     k1 <= g.ca_hi && k2 >= g.ca_lo && k2 <= g.ca_hi;
                    if (inA) continue;
                    auto &lst = lapT[((size_t)(k0 - g.cb_lo) * ncb + (k1 - g.cb_lo)) * ncb + (k2 - g.cb_lo)];
                    for (int s0 = -reach; s0 <= reach; ++s0)
                        for (int s1 = -reach; s1 <= reach; ++s1)
                            for (int s2 = -reach; s2 <= reach; ++s2) {
                                const double c = stencil_coef(g.Q, s0, s1, s2);
                                if (c == 0.0) continue;
                                lst.push_back({add(4 * (k0 + s0), 4 * (k1 + s1), 4 * (k2 + s2)),
                                               c / (g.H * g.H)});
                            }
                }
        // lag extent needed by the basis sums
        int Lb = 0;
        for (size_t a = 0; a < pts.size(); ++a) {
            const int v = pts[a];
            Lb = std::max(Lb, std::max(std::abs(v), std::abs(v - n)));
        }
        g.L = std::max(g.L, Lb);
        if (g.L > pl->dgf_L) return MLC_ERR_INVALID_ARG;
        const int npts = (int)(pts.size() / 3);
        int *dpts = nullptr;
        double *dch = nullptr, *dB = nullptr;
        TRY_CUDA(cudaMalloc((void **)&dpts, pts.size() * sizeof(int)));
        TRY_CUDA(cudaMalloc((void **)&dch, lcharge.size() * sizeof(double)));
        TRY_CUDA(cudaMalloc((void **)&dB, (size_t)npts * g.npoly * sizeof(double)));
        cudaMemcpy(dpts, pts.data(), pts.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(dch, lcharge.data(), lcharge.size() * sizeof(double), cudaMemcpyHostToDevice);
        cudaError_t e = basis_direct_sum(pl->dgf, pl->dgf_L, dpts, npts, dch, g.npoly, n,
                                         g.h * g.h, dB);
        std::vector<double> B((size_t)npts * g.npoly);
        if (e == cudaSuccess)
            e = cudaMemcpy(B.data(), dB, B.size() * sizeof(double), cudaMemcpyDeviceToHost);
        cudaFree(dpts);
        cudaFree(dch);
        cudaFree(dB);
        TRY_CUDA(e);
        const int np_ = g.npoly;
        Ttab.assign((size_t)ncb * ncb * ncb * np_, 0.0);
        for (size_t t = 0; t < lapT.size(); ++t)
            for (auto &pr : lapT[t])
                for (int p = 0; p < np_; ++p)
                    Ttab[t * np_ + p] += pr.second * B[(size_t)pr.first * np_ + p];
        Dtab.assign(ring_nodes.size() * g.npad, 0.0);  // rows padded with zeros to npad
        for (size_t r = 0; r < ring_nodes.size(); ++r)
            for (int p = 0; p < np_; ++p) {
                double iv = 0.0;
                for (size_t j = 0; j < rn_st[r].size(); ++j)
                    iv += ring_w[r][j] * B[(size_t)rn_st[r][j] * np_ + p];
                Dtab[r * g.npad + p] = B[(size_t)rn_self[r] * np_ + p] - iv;
            }
        Dout.assign(oself.size() * g.npad, 0.0);
        for (size_t r = 0; r < oself.size(); ++r)
            for (int p = 0; p < np_; ++p) {
                double iv = 0.0;
                for (size_t j = 0; j < ost[r].size(); ++j) iv += ow[r][j] * B[(size_t)ost[r][j] * np_ + p];
                Dout[r * g.npad + p] = B[(size_t)oself[r] * np_ + p] - iv;
            }
    }
    g.nr_face = (int)ring_nodes.size();
    // dense ring table per face-plane axis: rows [axis][plane j][u][v] (relative
    // plane coordinate pb0 + j n, in-plane offsets u, v in [-gb, n+gb], v the
    // faster axis), npad coefficients each; zero rows where a position is no
    // ring node.  Consecutive v are consecutive rows and no index map is read.
    g.pb0 = g.n * ceildiv(-g.gb, g.n);
    g.npb = 0;
    for (int c = g.pb0; c <= n + g.gb; c += n) ++g.npb;
    if (ring) {
        std::vector<double> Dd((size_t)3 * g.npb * g.wbx * g.wbx * g.npad, 0.0);
        for (int ax = 0; ax < 3; ++ax)
            for (int j = 0; j < g.npb; ++j)
                for (int u = 0; u < g.wbx; ++u)
                    for (int v = 0; v < g.wbx; ++v) {
                        int r[3];
                        r[ax] = g.pb0 + j * n;
                        r[ax == 0 ? 1 : 0] = u - g.gb;
                        r[ax == 2 ? 1 : 2] = v - g.gb;
                        const int ri = rmap[((size_t)(r[0] + g.gb) * g.wbx + (r[1] + g.gb)) * g.wbx + (r[2] + g.gb)];
                        if (ri < 0) continue;
                        const size_t row = (((size_t)ax * g.npb + j) * g.wbx + u) * g.wbx + v;
                        for (int k = 0; k < g.npad; ++k) Dd[row * g.npad + k] = Dtab[(size_t)ri * g.npad + k];
                    }
        Dtab.swap(Dd);
    }
    // split tiers: the ring table as the operand of the tensor-core ring GEMM
    g.ring_rows = g.npb * g.wbx * g.wbx;
    g.ring_ksteps = (g.npad + 7) / 8;
    g.ring_rows_pad = ((long)g.ring_rows + 127) / 128 * 128;
    if (ring && g.conv == CONV_F32) {
        std::vector<float> img;
        ring_table_image(Dtab, g.ring_rows, g.npad, g.ring_ksteps, g.ring_rows_pad, img);
        TRY(dev_upload(pl, &pl->ring_aimg, img));
        TRY(dev_alloc(pl, &pl->ring_R, (size_t)g.NP * g.ring_rows_pad));
    }
    auto to_df = [](const std::vector<double> &v) {  // double-float (hi, lo) pairs
        std::vector<float2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) {
            const float hi = (float)v[i];
            o[i] = make_float2(hi, (float)(v[i] - (double)hi));
        }
        return o;
    };
    // R18: dense rows [axis][j][side][u][v] of the off-face ring nodes, plane
    // pb0 + (j - 1) n for j in [0, npb + 2) (a node of Omega_beta one step off
    // a face plane can belong to the plane just outside it), normal coordinate
    // plane - 1 (side 0) or plane + 1 (side 1)
    if (ring && g.wide) {
        std::vector<double> Do((size_t)6 * (g.npb + 2) * g.wbx * g.wbx * g.npad, 0.0);
        for (int ax = 0; ax < 3; ++ax)
            for (int j = 0; j < g.npb + 2; ++j)
                for (int sd = 0; sd < 2; ++sd)
                    for (int u = 0; u < g.wbx; ++u)
                        for (int v = 0; v < g.wbx; ++v) {
                            int r[3];
                            r[ax] = g.pb0 + (j - 1) * n + (sd ? 1 : -1);
                            r[ax == 0 ? 1 : 0] = u - g.gb;
                            r[ax == 2 ? 1 : 2] = v - g.gb;
                            if (r[ax] < -g.gb || r[ax] > n + g.gb) continue;
                            const int ri = omap[((size_t)(r[0] + g.gb) * g.wbx + (r[1] + g.gb)) * g.wbx + (r[2] + g.gb)];
                            if (ri < 0) continue;
                            const size_t row = ((((size_t)ax * (g.npb + 2) + j) * 2 + sd) * g.wbx + u) * g.wbx + v;
                            for (int k = 0; k < g.npad; ++k) Do[row * g.npad + k] = Dout[(size_t)ri * g.npad + k];
                        }
        if (g.conv == CONV_F32) {
            float *d = nullptr;
            TRY(dev_upload(pl, &d, std::vector<float>(Do.begin(), Do.end())));
            pl->D2tab = d;
        } else {
            double *d = nullptr;
            TRY(dev_upload(pl, &d, Do));
            pl->D2tab = d;
        }
    }
    // ring tables in the ring precision: the local-convolution arithmetic
    if (g.conv == CONV_F32) {
        float *d = nullptr, *t = nullptr;
        TRY(dev_upload(pl, &d, std::vector<float>(Dtab.begin(), Dtab.end())));
        TRY(dev_upload(pl, &t, std::vector<float>(Ttab.begin(), Ttab.end())));
        pl->Dtab = d;
        pl->Ttab = t;
    } else if (g.conv == CONV_DF) {
        float2 *d = nullptr, *t = nullptr;
        TRY(dev_upload(pl, &d, to_df(Dtab)));
        TRY(dev_upload(pl, &t, to_df(Ttab)));
        pl->Dtab = d;
        pl->Ttab = t;
    } else {
        double *d = nullptr, *t = nullptr;
        TRY(dev_upload(pl, &d, Dtab));
        TRY(dev_upload(pl, &t, Ttab));
        pl->Dtab = d;
        pl->Ttab = t;
    }

    // FFT twiddles
    auto twiddles = [](int M) {
        std::vector<double2> tw(M / 2);
        for (int t = 0; t < M / 2; ++t) {
            const double a = 2.0 * M_PI * (double)t / (double)M;
            tw[t] = make_double2(std::cos(a), -std::sin(a));
        }
        return tw;
    };
    TRY(dev_upload(pl, &pl->tw, twiddles(g.M)));
    if (g.levels <= 2) TRY(dev_upload(pl, &pl->tw_c, twiddles(g.Mc)));  // coarse Hockney solve

    // Dirichlet tables: half DST-I matrix and eigenvalues of the stencil / h^2
    const int m = n - 1, hn = n / 2;
    std::vector<double> sinm((size_t)m * hn), lam((size_t)m * m * m);
    std::vector<double> cth(m);
    for (int k = 0; k < m; ++k) {
        cth[k] = std::cos(M_PI * (k + 1) / (double)n);
        for (int t = 0; t < hn; ++t) {
            const long r = ((long)(k + 1) * (t + 1)) % (2L * n);
            sinm[(size_t)k * hn + t] = std::sin(M_PI * (double)r / (double)n);
        }
    }
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c)
            for (int e = 0; e < m; ++e)
                lam[((size_t)a * m + c) * m + e] = (g.h * g.h) / symbol(g.Q, cth[a], cth[c], cth[e]);
    // in the fine precision (FP64 or double-float pairs); the DST-I
    // normalisation (2/n)^3 is folded into lam
    const double dnorm = std::pow(2.0 / n, 3);
    for (double &v : lam) v *= dnorm;
    if (g.fine == FINE_DF) {
        float2 *a = nullptr, *c = nullptr;
        TRY(dev_upload(pl, &a, to_df(sinm)));
        TRY(dev_upload(pl, &c, to_df(lam)));
        pl->sinm = a;
        pl->lam = c;
    } else {
        double *a = nullptr, *c = nullptr;
        TRY(dev_upload(pl, &a, sinm));
        TRY(dev_upload(pl, &c, lam));
        pl->sinm = a;
        pl->lam = c;
    }
    return MLC_OK;
}

mlc_status get_dgf(int device, int Q, int nD, int zeta, int L, const double **ptr, int *Lout) {
    std::lock_guard<std::mutex> lk(g_dgf_mu);
    auto key = std::make_tuple(device, Q, nD, zeta);
    auto it = g_dgf.find(key);
    if (it != g_dgf.end() && it->second.L >= L) {
        *ptr = it->second.ptr;
        *Lout = it->second.L;
        return MLC_OK;
    }
    // build with some headroom so later plans reuse the table
    int Lb = std::max(L, std::min(zeta * nD - 1, 128));
    double *p = nullptr;
    cudaError_t e = build_dgf_octant(Q, nD, zeta, Lb, &p);
    if (e != cudaSuccess) return to_status(e);
    g_dgf[key] = DgfEntry{p, Lb};  // an older, smaller table stays allocated for its plans
    *ptr = p;
    *Lout = Lb;
    return MLC_OK;
}

void free_plan(mlc_plan_s *pl) {
    if (!pl) return;
    free_plan(pl->child);
    for (void *p : pl->owned) cudaFree(p);
    for (auto &e : pl->ev_pool) cudaEventDestroy(e);
    for (auto &e : pl->fork)
        if (e) cudaEventDestroy(e);
    if (pl->side) cudaStreamDestroy(pl->side);
    delete pl;
}

// Point a plan (and its coarser levels) at another error word.
mlc_status share_error_word(mlc_plan_s *pl, int *err) {
    for (; pl; pl = pl->child) {
        pl->err = err;
        pl->hptrs.err = err;
        TRY_CUDA(cudaMemcpy(pl->dptrs, &pl->hptrs, sizeof(PlanPtrs), cudaMemcpyHostToDevice));
    }
    return MLC_OK;
}

// What a solve needs besides the plan's tables: the local-convolution
// scratch (unless the caller gave one) and the side stream with its events.
mlc_status prepare_solve(mlc_plan_s *pl) {
    if (!pl->user_scratch && !pl->scratch) {
        char *sc = nullptr;
        TRY(dev_alloc(pl, &sc, conv_scratch_bytes(pl->g, std::min<long>(pl->g.chunk, pl->g.NP))));
        pl->scratch = sc;
    }
    if (!pl->side) {
        TRY_CUDA(cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking));
        for (auto &e : pl->fork) TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    return MLC_OK;
}

}  // namespace

extern "C" {

const char *mlc_status_string(mlc_status s) {
    switch (s) {
        case MLC_OK: return "ok";
        case MLC_ERR_INVALID_ARG: return "invalid argument";
        case MLC_ERR_UNSUPPORTED: return "unsupported configuration";
        case MLC_ERR_OOM: return "out of memory";
        case MLC_ERR_CUDA: return "CUDA error";
        case MLC_ERR_ADMISSION: return "request exceeds the memory budget";
        case MLC_ERR_TIMEOUT: return "timed out";
        case MLC_ERR_INDEX: return "index out of range (checked build)";
    }
    return "unknown status";
}

mlc_status mlc_params_init(mlc_params *p, int N, int n, int s, int P, int Q) {
    if (!p) return MLC_ERR_INVALID_ARG;
    p->N = N; p->n = n; p->s = s; p->C = 4; p->P = P; p->Q = Q;
    p->g_beta = -1; p->b = -1; p->tier = MLC_TIER_FP64; p->mode = MLC_MODE_MLC;
    p->dgf_nD = -1; p->dgf_zeta = -1; p->conv_chunk = -1; p->levels = -1; p->coarse_s = -1;
    return MLC_OK;
}

}  // extern "C"

namespace {

// Plan creation; dgf_host (optional): the caller's DGF octant [0, dgf_Lh]^3
// in place of the device's cached table.
mlc_status make_coarser_level(mlc_plan_s *pl, const double *dgf_host, int dgf_Lh);

// h_level > 0: the mesh spacing of a coarser level of a multilevel solve (in
// place of 1/N); correction: add the Mehrstellen correction C2 h^2 f.
mlc_status create_plan(const mlc_params *params, const double *dgf_host, int dgf_Lh, mlc_plan_t *out,
                       double h_level = 0.0, bool correction = true) {
    if (!params || !out) return MLC_ERR_INVALID_ARG;
    *out = nullptr;
    Geom g;
    TRY(derive_geometry(*params, g));
    if (h_level > 0.0) {
        g.h = h_level;
        g.H = g.C * g.h;
        g.R = g.n * g.h / 2.0;
    }
    std::call_once(g_cfg_once, configure_kernels);
    int device = 0;
    TRY_CUDA(cudaGetDevice(&device));
    mlc_plan_s *pl = new (std::nothrow) mlc_plan_s();
    if (!pl) return MLC_ERR_OOM;
    pl->g = g;
    pl->params = *params;
    pl->device = device;
    pl->h_level = h_level;
    pl->correction = correction;
    // lag extent: local fields n + s, coarse Lc, basis fields (checked in build_tables)
    Geom &G = pl->g;
    G.L = std::max(G.n + G.s, G.levels > 2 ? 0 : G.Lc);  // a multilevel plan convolves no coarse lags
    const int Lbasis_bound = G.n + G.gb + 4 * G.b + 12;
    int Lneed = std::max(G.L, G.gb > G.ga ? Lbasis_bound : 0);
    if (Lneed >= G.zeta * G.nD) G.nD = (Lneed + G.zeta) / G.zeta + 1;
    mlc_status st = MLC_OK;
    if (dgf_host) {
        if (dgf_Lh < Lneed) {
            st = MLC_ERR_INVALID_ARG;
        } else {
            const size_t cnt = (size_t)(dgf_Lh + 1) * (dgf_Lh + 1) * (dgf_Lh + 1);
            double *d = nullptr;
            st = dev_upload(pl, &d, std::vector<double>(dgf_host, dgf_host + cnt));
            pl->dgf = d;
            pl->dgf_L = dgf_Lh;
        }
    } else {
        st = get_dgf(pl->device, G.Q, G.nD, G.zeta, Lneed, &pl->dgf, &pl->dgf_L);
    }
    if (st == MLC_OK) st = build_tables(pl);
    auto alloc_all = [&]() -> mlc_status {
        TRY(dev_alloc(pl, &pl->khat, (size_t)G.Mh * G.Mh * G.Mh, false));
        TRY_CUDA(build_even_spectrum(pl->dgf, pl->dgf_L, G.M, std::min(G.n + G.s, G.M / 2),
                                     G.h * G.h / ((double)G.M * G.M * G.M), pl->khat));
        const bool hockney = G.levels <= 2;  // this plan runs the coarse Hockney solve itself
        if (hockney) {
            TRY(dev_alloc(pl, &pl->khat_c, (size_t)G.Mhc * G.Mhc * G.Mhc, false));
            TRY_CUDA(build_even_spectrum(pl->dgf, pl->dgf_L, G.Mc, G.Lc,
                                         G.H * G.H / ((double)G.Mc * G.Mc * G.Mc), pl->khat_c));
        }
        if (hockney && G.fine == FINE_DF) {   // double-float copies for the coarse convolution: v = hi + lo
            auto split = [](double v) {
                const float h = (float)v;
                return make_float2(h, (float)(v - (double)h));
            };
            const size_t nk = (size_t)G.Mhc * G.Mhc * G.Mhc;
            std::vector<double> kd(nk);
            TRY_CUDA(cudaMemcpy(kd.data(), pl->khat_c, nk * sizeof(double), cudaMemcpyDeviceToHost));
            std::vector<float2> kf(nk);
            for (size_t i = 0; i < nk; ++i) kf[i] = split(kd[i]);
            TRY(dev_upload(pl, &pl->khat_c_df, kf));
            std::vector<float4> tf(G.Mc / 2);
            for (int t = 0; t < G.Mc / 2; ++t) {
                const double a = 2.0 * M_PI * (double)t / (double)G.Mc;
                const float2 re = split(std::cos(a)), im = split(-std::sin(a));
                tf[t] = make_float4(re.x, re.y, im.x, im.y);
            }
            TRY(dev_upload(pl, &pl->tw_c_df, tf));
        }
        const size_t NP = G.NP;
        const size_t rb = conv_real_bytes(G.tier);
        // the local-convolution scratch (a1 [item][kx][zi][yi], a4 [item][z
        // row][kx][yo] for one launch group) is allocated by the first solve
        // that needs it, unless the caller provides one (mlc_plan_set_scratch)
        char *bc = nullptr, *bf = nullptr;
        TRY(dev_alloc(pl, &bc, NP * (size_t)G.nc * G.nc * G.nc * rb));
        TRY(dev_alloc(pl, &bf, NP * 3 * (size_t)G.npa * G.wa * G.wa * rb));
        pl->cl = bc;
        pl->fpl = bf;
        if (G.conv == CONV_DF) {
            // double-float copies of the patch kernel spectrum and twiddles
            auto split = [](double v) {
                const float h = (float)v;
                return make_float2(h, (float)(v - (double)h));
            };
            const size_t nk = (size_t)G.Mh * G.Mh * G.Mh;
            std::vector<double> kd(nk);
            TRY_CUDA(cudaMemcpy(kd.data(), pl->khat, nk * sizeof(double), cudaMemcpyDeviceToHost));
            std::vector<float2> kf(nk);
            for (size_t i = 0; i < nk; ++i) kf[i] = split(kd[i]);
            TRY(dev_upload(pl, &pl->khat_df, kf));
            std::vector<float4> tf(G.M / 2);
            for (int t = 0; t < G.M / 2; ++t) {
                const double a = 2.0 * M_PI * (double)t / (double)G.M;
                const float2 re = split(std::cos(a)), im = split(-std::sin(a));
                tf[t] = make_float4(re.x, re.y, im.x, im.y);
            }
            TRY(dev_upload(pl, &pl->tw_df, tf));
        }
        if (G.conv == CONV_F32) {
            // FP32 copies of the patch kernel spectrum and twiddles
            const size_t nk = (size_t)G.Mh * G.Mh * G.Mh;
            std::vector<double> kd(nk);
            TRY_CUDA(cudaMemcpy(kd.data(), pl->khat, nk * sizeof(double), cudaMemcpyDeviceToHost));
            std::vector<float> kf(kd.begin(), kd.end());
            std::vector<float2> tf(G.M / 2);
            for (int t = 0; t < G.M / 2; ++t) {
                const double a = 2.0 * M_PI * (double)t / (double)G.M;
                tf[t] = make_float2((float)std::cos(a), (float)-std::sin(a));
            }
            TRY(dev_upload(pl, &pl->khat_f, kf));
            TRY(dev_upload(pl, &pl->tw_f, tf));
        }
        TRY(dev_alloc(pl, &pl->mom, NP * G.npad));  // padding stays zero (memset below)
        TRY_CUDA(cudaMemset(pl->mom, 0, NP * G.npad * sizeof(double)));
        TRY(dev_alloc(pl, &pl->resid, NP * 3 * (size_t)G.npa * G.wa * G.wa));
        if (G.conv == CONV_F32) {
            TRY(dev_alloc(pl, &pl->mom_f, NP * G.npad));
            TRY_CUDA(cudaMemset(pl->mom_f, 0, NP * G.npad * sizeof(float)));
        } else if (G.conv == CONV_DF) {
            TRY(dev_alloc(pl, &pl->mom_df, NP * G.npad));
            TRY_CUDA(cudaMemset(pl->mom_df, 0, NP * G.npad * sizeof(float2)));
        }
        const size_t nf = G.nf, no = G.no, Mc = G.Mc, Mhc = G.Mhc;
        TRY(dev_alloc(pl, &pl->FH, nf * nf * nf));
        if (hockney) {
            TRY(dev_alloc(pl, &pl->cbuf0, std::max(nf * nf * Mhc, no * Mc * Mhc)));
            TRY(dev_alloc(pl, &pl->cbuf1, std::max(nf * Mc * Mhc, no * no * Mhc)));
        }
        TRY(dev_alloc(pl, &pl->phiH, no * no * no));
        TRY(dev_alloc(pl, &pl->phiB, (size_t)G.n_planes_total));
        TRY(dev_alloc(pl, &pl->tpl, 3 * (size_t)(G.np + 1) * G.no * (G.N + 1)));
        if (G.wide) {  // R18: the second boundary layer
            char *f2 = nullptr;
            const size_t per = NP * 6 * (size_t)G.npa * G.wa * G.wa;
            TRY(dev_alloc(pl, &f2, per * rb));
            pl->fp2 = f2;
            TRY(dev_alloc(pl, &pl->resid2, per));
            TRY(dev_alloc(pl, &pl->phiB2, 2 * (size_t)G.n_planes_total));
            TRY(dev_alloc(pl, &pl->tpl2, 6 * (size_t)(G.np + 1) * G.no * (G.N + 1)));
        }
        if (G.n > 24 || (G.wide && G.n > 16)) {  // Dirichlet workspace of patches too large for shared memory
            double *d = nullptr;                     // (Q = 10: right-hand side, iterate and work array)
            TRY(dev_alloc(pl, &d, NP * (G.wide ? 3 : 1) * (size_t)(G.n - 1) * (G.n - 1) * (G.n - 1)));
            pl->dscr = d;
        }
        TRY(dev_alloc(pl, &pl->err, 1, false));
        TRY_CUDA(cudaMemset(pl->err, 0, sizeof(int)));
        return MLC_OK;
    };
    if (st == MLC_OK) st = alloc_all();
    if (st == MLC_OK) {
        PlanPtrs &h = pl->hptrs;
        h.f = nullptr;
        h.phi = nullptr;
        h.cl = pl->cl;
        h.fp = pl->fpl;
        h.khat = G.conv == CONV_F32 ? (const void *)pl->khat_f
                 : (G.conv == CONV_DF ? (const void *)pl->khat_df : (const void *)pl->khat);
        h.momw = pl->momw;
        h.mom_scale = std::pow(G.R, -1.5);
        h.mom = pl->mom;
        h.mom_f = pl->mom_f;
        h.mom_df = pl->mom_df;
        h.resid = pl->resid;
        h.phiB = pl->phiB;
        h.lam = pl->lam;
        h.N = G.N;
        h.np = G.np;
        h.c2h2 = correction ? stencil_c2(G.Q) * G.h * G.h : 0.0;
        h.inv_h2 = 1.0 / (G.h * G.h);
        h.err = pl->err;
        h.dscr = pl->dscr;
        h.fp2 = pl->fp2;
        h.resid2 = pl->resid2;
        h.phiB2 = pl->phiB2;
        st = dev_upload(pl, &pl->dptrs, std::vector<PlanPtrs>{h});
    }
    if (st == MLC_OK && G.levels > 2) st = make_coarser_level(pl, dgf_host, dgf_Lh);
    if (st == MLC_OK) st = to_status(cudaDeviceSynchronize());
    if (st != MLC_OK) {
        free_plan(pl);
        return st;
    }
    *out = pl;
    return MLC_OK;
}

// Sec. 5: the next coarser level of a multilevel solve.  Its problem is
// Delta^H phi = F^H on a box of whole patches (spacing H) starting at
// min(flo, olo) that holds the support of F^H and the nodes phi^H is read
// on; same n, s, P, Q, b, g_beta, mode, tier; no Mehrstellen correction.  Its
// charge array stays zero outside the F^H box (written once here), and its
// scratch and side stream exist before the first solve, so that solves
// allocate nothing (and can be captured in a graph).
mlc_status make_coarser_level(mlc_plan_s *pl, const double *dgf_host, int dgf_Lh) {
    const Geom &G = pl->g;
    const int c0 = std::min(G.flo, G.olo), top = std::max(G.fhi, G.ohi);
    const int Nc = G.n * ((top - c0 + G.n) / G.n);
    mlc_params cp = pl->params;
    cp.N = Nc;
    cp.levels = G.levels - 1;
    if (cp.coarse_s > 0) cp.s = cp.coarse_s;  // the coarser levels' inner radius
    mlc_plan_t ch = nullptr;
    TRY(create_plan(&cp, dgf_host, dgf_Lh, &ch, G.H, false));
    pl->child = ch;
    pl->child_c0 = c0;
    const size_t n3 = (size_t)Nc * Nc * Nc;
    if (G.f32in) {
        float *f = nullptr;
        TRY(dev_alloc(pl, &f, n3));
        pl->child_f = f;
    } else {
        double *f = nullptr;
        TRY(dev_alloc(pl, &f, n3));
        pl->child_f = f;
    }
    TRY_CUDA(cudaMemset(pl->child_f, 0, n3 * (G.f32in ? sizeof(float) : sizeof(double))));
    TRY(dev_alloc(pl, &pl->child_phi, n3));
    TRY(prepare_solve(ch));
    TRY(share_error_word(ch, pl->err));  // a coarser level's failures show on this plan
    pl->ws_bytes += ch->ws_bytes;
    return MLC_OK;
}

}  // namespace

extern "C" {

mlc_status mlc_plan_create_ex(const mlc_params *params, mlc_plan_t *out) {
    return create_plan(params, nullptr, 0, out);
}

mlc_status mlc_plan_set_dgf(mlc_plan_t pl, const double *table, int L) {
    if (!pl || !table || L < 1) return MLC_ERR_INVALID_ARG;
    int dev = -1;
    TRY_CUDA(cudaGetDevice(&dev));
    if (dev != pl->device) return MLC_ERR_INVALID_ARG;
    mlc_plan_t np = nullptr;
    TRY(create_plan(&pl->params, table, L, &np, pl->h_level, pl->correction));
    TRY_CUDA(cudaDeviceSynchronize());
    mlc_batch_forget(pl);
    np->user_scratch = pl->user_scratch;
    np->fault = pl->fault;
    np->timing = pl->timing;
    std::swap(*pl, *np);  // the handle keeps its identity; np now holds the old tables
    free_plan(np);
    return MLC_OK;
}

mlc_status mlc_plan_create(int N, int patch, int support, int coarsening, int P, int Q,
                           mlc_plan_t *out) {
    mlc_params p;
    mlc_params_init(&p, N, patch, support, P, Q);
    p.C = coarsening;
    return mlc_plan_create_ex(&p, out);
}

mlc_status mlc_plan_destroy(mlc_plan_t plan) {
    if (!plan) return MLC_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    mlc_batch_forget(plan);
    free_plan(plan);
    return to_status(e);
}

mlc_status mlc_plan_workspace_bytes(mlc_plan_t plan, size_t *bytes) {
    if (!plan || !bytes) return MLC_ERR_INVALID_ARG;
    *bytes = plan->ws_bytes;
    return MLC_OK;
}

mlc_status mlc_plan_info(mlc_plan_t plan, int *o) {
    if (!plan || !o) return MLC_ERR_INVALID_ARG;
    const Geom &g = plan->g;
    const int v[16] = {g.N, g.n, g.s, g.b, g.ga, g.gb, g.P, g.npoly, g.flo, g.fhi,
                       g.olo, g.ohi, g.M, g.Mc, plan->dgf_L, g.nD};
    std::memcpy(o, v, sizeof(v));
    return MLC_OK;
}

mlc_status mlc_plan_scratch_bytes(mlc_plan_t pl, size_t *bytes) {
    if (!pl || !bytes) return MLC_ERR_INVALID_ARG;
    *bytes = conv_scratch_bytes(pl->g, std::min<long>(pl->g.chunk, pl->g.NP));
    return MLC_OK;
}

mlc_status mlc_plan_set_scratch(mlc_plan_t pl, void *scratch, size_t bytes) {
    if (!pl) return MLC_ERR_INVALID_ARG;
    if (scratch) {
        size_t need = 0;
        mlc_plan_scratch_bytes(pl, &need);
        if (bytes < need || ((uintptr_t)scratch & 255)) return MLC_ERR_INVALID_ARG;
    }
    pl->user_scratch = scratch;
    return MLC_OK;
}

mlc_status mlc_solve(mlc_plan_t pl, const void *f, void *phi, void *stream) {
    if (!pl || !f || !phi || f == phi) return MLC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    TRY(prepare_solve(pl));  // first solve: the plan's own scratch and side stream
    NvtxRange nvtx(pl->correction ? "mlc:solve" : "mlc:coarser_level_solve");
    void *scr = pl->user_scratch ? pl->user_scratch : pl->scratch;
    if (pl->hptrs.f != f || pl->hptrs.phi != phi) {
        TRY_CUDA(launch_set_ptrs(pl->dptrs, f, (double *)phi, st));
        pl->hptrs.f = f;
        pl->hptrs.phi = (double *)phi;
    }
    Items it{nullptr, pl->dptrs, pl->g.NP};
    it.a1 = scr;
    it.a4 = (char *)scr + conv_scratch_a4_offset(pl->g, std::min<long>(pl->g.chunk, pl->g.NP));
    if (!pl->timing) {
        // Two streams: the moments (they read only f) and, once the local
        // fields exist, the face-plane residuals run on a side stream beside
        // the local convolutions and the coarse-charge assembly and coarse
        // solve; the boundary step joins both.
        cudaStream_t s2 = pl->side;
        TRY_CUDA(cudaEventRecord(pl->fork[0], st));
        TRY_CUDA(cudaStreamWaitEvent(s2, pl->fork[0], 0));
        TRY_CUDA(launch_moments(pl, it, s2));
        TRY_CUDA(cudaEventRecord(pl->fork[1], s2));
        TRY_CUDA(launch_patch_conv(pl, it, st));
        TRY_CUDA(cudaEventRecord(pl->fork[2], st));
        TRY_CUDA(cudaStreamWaitEvent(s2, pl->fork[2], 0));
        TRY_CUDA(launch_resid(pl, it, s2));
        TRY_CUDA(cudaEventRecord(pl->fork[3], s2));
        TRY_CUDA(cudaStreamWaitEvent(st, pl->fork[1], 0));
        TRY_CUDA(launch_assemble(pl, st));
        TRY_CUDA(launch_coarse(pl, st));
        TRY_CUDA(cudaStreamWaitEvent(st, pl->fork[3], 0));
        TRY_CUDA(launch_boundary(pl, st));
        TRY_CUDA(launch_dirichlet(pl, it, st));
        return MLC_OK;
    }
    // per-launch timing: the same launches in sequence on one stream
    pl->marks.clear();
    mark(pl, 0, st);
    TRY_CUDA(launch_moments(pl, it, st));
    TRY_CUDA(launch_patch_conv(pl, it, st));       // slots 1-3 (per launch group)
    mark(pl, 4, st);
    TRY_CUDA(launch_resid(pl, it, st));
    mark(pl, 5, st);
    TRY_CUDA(launch_assemble(pl, st));
    TRY_CUDA(launch_coarse(pl, st));               // slots 6-10
    mark(pl, 11, st);
    TRY_CUDA(launch_boundary(pl, st));
    mark(pl, 12, st);
    TRY_CUDA(launch_dirichlet(pl, it, st));
    mark(pl, 13, st);
    return MLC_OK;
}

mlc_status mlc_solve_host(mlc_plan_t pl, const void *f_host, void *phi_host, void *stream) {
    if (!pl || !f_host || !phi_host) return MLC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N3 = (size_t)pl->g.N * pl->g.N * pl->g.N;
    const size_t fbytes = N3 * (pl->g.f32in ? sizeof(float) : sizeof(double));
    if (!pl->f_stage) {
        char *fs = nullptr;
        double *ps = nullptr;
        TRY(dev_alloc(pl, &fs, fbytes));
        TRY(dev_alloc(pl, &ps, N3));
        pl->f_stage = fs;
        pl->phi_stage = ps;
    }
    TRY_CUDA(cudaMemcpyAsync(pl->f_stage, f_host, fbytes, cudaMemcpyHostToDevice, st));
    TRY(mlc_solve(pl, pl->f_stage, pl->phi_stage, stream));
    TRY_CUDA(cudaMemcpyAsync(phi_host, pl->phi_stage, N3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    // the plan's error word, read in stream order (no device-wide synchronisation)
    int e = 0;
    TRY_CUDA(cudaMemcpyAsync(&e, pl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY_CUDA(cudaStreamSynchronize(st));
    if (e) {
        TRY_CUDA(cudaMemsetAsync(pl->err, 0, sizeof(int), st));
        TRY_CUDA(cudaStreamSynchronize(st));
        return e == 2 ? MLC_ERR_INDEX : MLC_ERR_TIMEOUT;
    }
    return MLC_OK;
}

mlc_status mlc_plan_status(mlc_plan_t pl) {
    if (!pl) return MLC_ERR_INVALID_ARG;
    TRY_CUDA(cudaDeviceSynchronize());
    int e = 0;
    TRY_CUDA(cudaMemcpy(&e, pl->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        TRY_CUDA(cudaMemset(pl->err, 0, sizeof(int)));
        return e == 2 ? MLC_ERR_INDEX : MLC_ERR_TIMEOUT;
    }
    return MLC_OK;
}

mlc_status mlc_debug_set_fault(mlc_plan_t pl, int kind) {
    if (!pl || kind < 0 || kind > 1) return MLC_ERR_INVALID_ARG;
    pl->fault = kind;
    return MLC_OK;
}

mlc_status mlc_debug_set_timing(mlc_plan_t pl, int enable) {
    if (!pl) return MLC_ERR_INVALID_ARG;
    pl->timing = enable ? 1 : 0;
    pl->marks.clear();
    return MLC_OK;
}

mlc_status mlc_debug_timing(mlc_plan_t pl, float *ms, int count) {
    if (!pl || !ms || count < kTimedLaunches || !pl->timing || pl->marks.size() < 2) return MLC_ERR_INVALID_ARG;
    TRY_CUDA(cudaEventSynchronize(pl->marks.back().second));
    for (int k = 0; k < kTimedLaunches; ++k) ms[k] = 0.f;
    for (size_t i = 0; i + 1 < pl->marks.size(); ++i) {
        float t = 0.f;
        TRY_CUDA(cudaEventElapsedTime(&t, pl->marks[i].second, pl->marks[i + 1].second));
        const int k = pl->marks[i].first;
        if (k >= 0 && k < kTimedLaunches) ms[k] += t;
    }
    return MLC_OK;
}

// Patch counts of the index stages (count pass on the device) as offsets.
mlc_status index_offsets(mlc_plan_t pl, int which, std::vector<long> &off) {
    const Geom &g = pl->g;
    const long nodes = which ? (long)g.nf * g.nf * g.nf : g.n_planes_total;
    int *cnt = nullptr;
    TRY_CUDA(cudaMalloc((void **)&cnt, nodes * sizeof(int)));
    cudaError_t e = launch_index_export(pl, which, cnt, nullptr, nullptr, 0);
    std::vector<int> h(nodes);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cnt, nodes * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(cnt);
    TRY_CUDA(e);
    off.assign(nodes + 1, 0);
    for (long k = 0; k < nodes; ++k) off[k + 1] = off[k] + h[k];
    if (off[nodes] > INT32_MAX) return MLC_ERR_UNSUPPORTED;
    return MLC_OK;
}

mlc_status mlc_debug_stage_bytes(mlc_plan_t pl, int stage, size_t *bytes) {
    if (!pl || !bytes) return MLC_ERR_INVALID_ARG;
    const Geom &g = pl->g;
    switch (stage) {
        case MLC_STAGE_MOMENTS: *bytes = (size_t)g.NP * g.npoly * 8; break;
        case MLC_STAGE_FH: *bytes = (size_t)g.nf * g.nf * g.nf * 8; break;
        case MLC_STAGE_PHIH: *bytes = (size_t)g.no * g.no * g.no * 8; break;
        case MLC_STAGE_PHIB: *bytes = (size_t)g.n_planes_total * 8; break;
        case MLC_STAGE_PHIB_OUTER:
            if (!g.wide) return MLC_ERR_INVALID_ARG;
            *bytes = 2 * (size_t)g.n_planes_total * 8;
            break;
        case MLC_STAGE_DGF: *bytes = (size_t)(pl->dgf_L + 1) * (pl->dgf_L + 1) * (pl->dgf_L + 1) * 8; break;
        case MLC_STAGE_COARSE_SAMPLES: *bytes = (size_t)g.NP * g.nc * g.nc * g.nc * 8; break;
        case MLC_STAGE_FACE_INDEX:
        case MLC_STAGE_COARSE_INDEX: {
            std::vector<long> off;
            TRY(index_offsets(pl, stage == MLC_STAGE_COARSE_INDEX, off));
            *bytes = (off.size() + (size_t)off.back()) * sizeof(int32_t);
            break;
        }
        default: return MLC_ERR_INVALID_ARG;
    }
    return MLC_OK;
}

mlc_status mlc_debug_export(mlc_plan_t pl, int stage, void *host, size_t bytes) {
    size_t need = 0;
    TRY(mlc_debug_stage_bytes(pl, stage, &need));
    if (!host || bytes != need) return MLC_ERR_INVALID_ARG;
    if (stage == MLC_STAGE_FACE_INDEX || stage == MLC_STAGE_COARSE_INDEX) {
        const int which = stage == MLC_STAGE_COARSE_INDEX;
        std::vector<long> off;
        TRY(index_offsets(pl, which, off));
        const long nodes = (long)off.size() - 1, total = off.back();
        long *doff = nullptr;
        int *dent = nullptr;
        TRY_CUDA(cudaMalloc((void **)&doff, off.size() * sizeof(long)));
        cudaError_t e = cudaMalloc((void **)&dent, std::max<long>(total, 1) * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(doff, off.data(), off.size() * sizeof(long), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_index_export(pl, which, nullptr, doff, dent, 0);
        int32_t *out = (int32_t *)host;
        for (long k = 0; k <= nodes; ++k) out[k] = (int32_t)off[k];
        if (e == cudaSuccess) e = cudaMemcpy(out + nodes + 1, dent, total * sizeof(int), cudaMemcpyDeviceToHost);
        cudaFree(doff);
        cudaFree(dent);
        TRY_CUDA(e);
        return MLC_OK;
    }
    const void *src = nullptr;
    switch (stage) {
        case MLC_STAGE_COARSE_SAMPLES: src = pl->cl; break;
        case MLC_STAGE_MOMENTS: src = pl->mom; break;
        case MLC_STAGE_FH: src = pl->FH; break;
        case MLC_STAGE_PHIH: src = pl->phiH; break;
        case MLC_STAGE_PHIB: src = pl->phiB; break;
        case MLC_STAGE_PHIB_OUTER: src = pl->phiB2; break;
        case MLC_STAGE_DGF: src = pl->dgf; break;
        default: return MLC_ERR_INVALID_ARG;
    }
    TRY_CUDA(cudaDeviceSynchronize());
    if (stage == MLC_STAGE_MOMENTS) {  // rows are stored with stride npad
        TRY_CUDA(cudaMemcpy2D(host, pl->g.npoly * sizeof(double), src, pl->g.npad * sizeof(double),
                              pl->g.npoly * sizeof(double), pl->g.NP, cudaMemcpyDeviceToHost));
        return MLC_OK;
    }
    if (stage == MLC_STAGE_COARSE_SAMPLES && pl->g.conv != CONV_F64) {  // FP32 or double-float storage
        const size_t cnt = bytes / sizeof(double);
        double *out = (double *)host;
        if (pl->g.conv == CONV_F32) {
            std::vector<float> tmp(cnt);
            TRY_CUDA(cudaMemcpy(tmp.data(), src, cnt * sizeof(float), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < cnt; ++i) out[i] = tmp[i];
        } else {
            std::vector<float2> tmp(cnt);
            TRY_CUDA(cudaMemcpy(tmp.data(), src, cnt * sizeof(float2), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < cnt; ++i) out[i] = (double)tmp[i].x + (double)tmp[i].y;
        }
        return MLC_OK;
    }
    if ((stage == MLC_STAGE_PHIH || stage == MLC_STAGE_PHIB) && pl->g.fine == FINE_DF) {
        // double-float pairs on the device
        std::vector<float2> tmp(bytes / sizeof(double));
        TRY_CUDA(cudaMemcpy(tmp.data(), src, tmp.size() * sizeof(float2), cudaMemcpyDeviceToHost));
        double *out = (double *)host;
        for (size_t i = 0; i < tmp.size(); ++i) out[i] = (double)tmp[i].x + (double)tmp[i].y;
        return MLC_OK;
    }
    TRY_CUDA(cudaMemcpy(host, src, bytes, cudaMemcpyDeviceToHost));
    return MLC_OK;
}

}  // extern "C"
