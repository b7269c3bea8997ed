// The q = 10 operator's second boundary layer (Sec. 8; reading R18).
//
// An operator that reaches two nodes (s = 2) needs, in the final Dirichlet
// step (eq. last_step_fulldiscr), boundary data on the closed faces and on
// the layer one node outside them.  Those outer nodes lie on the planes
// n j -+ 1, which are not coarse planes, so I^H there is R4's tensor-product
// Lagrange factor on all three axes; the boundary values keep the linear form
// of eq. mlcfulldiscr (I^H(phi^H) + the alpha patches' residuals phi^i -
// I^H(phi^i) + the ring patches' Legendre terms).  The Dirichlet problem with
// two boundary layers is not diagonalised by DST-I: its operator on the
// interior is the odd-extension operator that DST-I inverts plus a term E
// that couples the layer next to each face to its mirror image, and the
// fixed point u = L_odd^-1 (b - E u) converges by a factor of about 0.025 per
// step (the spectral radius of L_odd^-1 E for this stencil at n = 8 to 32).
//
// Included by kernels.cu inside namespace mlc, after its kernels: the kernels
// below reuse its helpers (FT, item_plan, in_range, face_node_patches,
// ring_dot, lagrange_rows_df).  FP64 arithmetic throughout (tiers FP64 and
// SPLIT; the plan refuses the double-float tiers for Q = 10).

namespace {

// Residuals r^i = phi^i - I^H(phi^i) one node off the face planes of patch i
// inside Omega_alpha (one CTA per patch and off-plane).  The plane's
// coordinate c = pl0 + j n -+ 1 is not a coarse coordinate, so the coarse
// values on the plane are first interpolated along the normal from the 2b+2
// coarse planes around it; the in-plane interpolation then runs as in
// k_resid (along v on the coarse rows, then along u).
struct ResOutArgs {
    Items it;
    int n, s, ga, b, npa, pl0, wa, nc;
    double lwd[4][12];
};

template <typename TB, int K>
__global__ void __launch_bounds__(256) k_resid_outer(ResOutArgs a) {
    extern __shared__ double rsm[];
    const int slot = blockIdx.y;  // axis * 2 npa + 2 j + side
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x, p);
    const int axis = slot / (2 * a.npa), o = slot % (2 * a.npa);
    const int c = a.pl0 + (o / 2) * a.n + ((o & 1) ? 1 : -1);
    if (c < -a.ga || c > a.n + a.ga) return;  // off the alpha box: never read
    const int wa = a.wa, nc = a.nc, kl = -a.s / 4;
    const int klo = -a.ga / 4 - a.b, khi = (a.n + a.ga) / 4 + a.b, nk = khi - klo + 1;
    const int rn = c & 3, kn0 = (c >> 2) - a.b;  // normal stencil: coarse planes kn0 .. kn0 + K - 1
    double *Tv = rsm;           // nk x wa
    double *Cv = Tv + nk * wa;  // nk x nk: phi^i interpolated along the normal to the plane
    const TB *cl = (const TB *)PP.cl + (long)p * nc * nc * nc;
    auto clp = [&](int kn, int ka, int kb) -> double {
        int i0, i1, i2;
        if (axis == 0) { i0 = kn; i1 = ka; i2 = kb; }
        else if (axis == 1) { i0 = ka; i1 = kn; i2 = kb; }
        else { i0 = ka; i1 = kb; i2 = kn; }
        if (!(in_range(i0 - kl, nc, PP.err) & in_range(i1 - kl, nc, PP.err) & in_range(i2 - kl, nc, PP.err)))
            return 0.0;
        return (double)cl[((long)(i0 - kl) * nc + (i1 - kl)) * nc + (i2 - kl)];
    };
    for (int e = threadIdx.x; e < nk * nk; e += blockDim.x) {
        const int ka = klo + e / nk, kb = klo + e % nk;
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < K; ++j) t = fma(a.lwd[rn][j], clp(kn0 + j, ka, kb), t);
        Cv[e] = t;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nk * wa; e += blockDim.x) {
        const int kr = e / wa, v = e % wa - a.ga;
        const int rv = v & 3;
        const double *crow = Cv + kr * nk - klo;
        double t;
        if (rv == 0) {
            t = crow[v >> 2];
        } else {
            const int k0 = (v >> 2) - a.b;
            t = 0.0;
#pragma unroll
            for (int j = 0; j < K; ++j) t = fma(a.lwd[rv][j], crow[k0 + j], t);
        }
        Tv[e] = t;
    }
    __syncthreads();
    const long off = ((long)p * 6 * a.npa + slot) * wa * wa;
    const TB *fp = (const TB *)PP.fp2 + off;
    double *out = (double *)PP.resid2 + off;
    for (int e = threadIdx.x; e < wa * wa; e += blockDim.x) {
        const int u = e / wa - a.ga, v = e % wa - a.ga;
        const int ru = u & 3;
        double iv;
        if (ru == 0) {
            iv = Tv[((u >> 2) - klo) * wa + (v + a.ga)];
        } else {
            const int k0 = (u >> 2) - a.b;
            iv = 0.0;
#pragma unroll
            for (int j = 0; j < K; ++j) iv = fma(a.lwd[ru][j], Tv[(k0 + j - klo) * wa + (v + a.ga)], iv);
        }
        out[e] = (double)fp[e] - iv;
    }
}

// First half of I^H(phi^H) on the planes n j -+ 1 (j in [0, np]): for every
// coarse row c_u and fine v in [0, N],
//   tpl2[a][j][side][c_u - olo][v] = sum_e w_{v mod 4}(e) Phi(c_u, v/4 - b + e),
// Phi(c_u, c_v) = sum_t w_{c mod 4}(t) phi^H(c/4 - b + t, c_u, c_v) along the
// normal (the coarse value itself when v mod 4 = 0).
__global__ void __launch_bounds__(256) k_plane_interp_outer(const double *phiH, double *out, int N, int n, int np,
                                                            int b, int olo, int no, LagW w, int *err) {
    const long tot = 6L * (np + 1) * no * (N + 1);
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int v = (int)(idx % (N + 1));
    const int cu = (int)((idx / (N + 1)) % no);
    const int pjs = (int)(idx / ((long)(N + 1) * no));  // (axis * (np + 1) + j) * 2 + side
    const int side = pjs & 1, axis = (pjs >> 1) / (np + 1), j = (pjs >> 1) % (np + 1);
    const int c = j * n + (side ? 1 : -1);
    const int rn = c & 3, kn0 = (c >> 2) - b, K = 2 * b + 2;
    auto at = [&](int kn, int cv) -> double {
        const int a0 = kn - olo, c1 = cv - olo;
        if (!(in_range(a0, no, err) & in_range(c1, no, err) & in_range(cu, no, err))) return 0.0;
        long i;
        if (axis == 0) i = ((long)a0 * no + cu) * no + c1;
        else if (axis == 1) i = ((long)cu * no + a0) * no + c1;
        else i = ((long)cu * no + c1) * no + a0;
        return phiH[i];
    };
    auto Phi = [&](int cv) -> double {
        double t = 0.0;
        for (int q = 0; q < K; ++q) t = fma(w.lwd[rn][q], at(kn0 + q, cv), t);
        return t;
    };
    const int rv = v & 3;
    double s;
    if (rv == 0) {
        s = Phi(v >> 2);
    } else {
        const int kb = (v >> 2) - b;
        s = 0.0;
        for (int e = 0; e < K; ++e) s = fma(w.lwd[rv][e], Phi(kb + e), s);
    }
    out[idx] = s;
}

// phi^B on the planes n j -+ 1 of every axis, in-plane coordinates [0, N]
// ([axis][j][side][u][v], side 0: n j - 1, side 1: n j + 1).  The in-plane
// sum along u of I^H(phi^H) reads tpl2; each alpha patch adds its residual
// on the off-plane slot of the node's own axis (the node's coordinate there
// is that patch's face plane -+ 1), each ring patch its Legendre term from
// the off-face ring rows.  RT: the ring precision (the tier's convolution
// arithmetic: FP32 or FP64).
struct BndOutArgs {
    int *err;
    const double *tpl2, *resid2;
    const void *mom, *D2;
    double *phiB2;
    int N, n, np, ga, gb, b, olo, no, wa, wbx, npa, pl0, pb0, npb, npad;
    double lwd[4][12];
};

template <typename RT, int NN>
__global__ void __launch_bounds__(128) k_boundary_outer(BndOutArgs a) {
    constexpr int n = NN;
    const long pn = (long)(a.N + 1) * (a.N + 1);
    const long tot = 6L * (a.np + 1) * pn;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int pjs = (int)(idx / pn);
    const int side = pjs & 1, axis = (pjs >> 1) / (a.np + 1), jp = (pjs >> 1) % (a.np + 1);
    const int u = (int)((idx % pn) / (a.N + 1)), v = (int)(idx % (a.N + 1));
    const int sg = side ? 1 : -1, c = jp * n + sg;
    int g[3];
    g[axis] = c;
    g[axis == 0 ? 1 : 0] = u;
    g[axis == 2 ? 1 : 2] = v;
    // I^H(phi^H): sum along u of the along-v sums on this plane
    const double *tpl = a.tpl2 + (long)pjs * a.no * (a.N + 1) + v;
    const int K = 2 * a.b + 2, ru = u & 3;
    double acc;
    if (ru == 0) {
        const int k = (u >> 2) - a.olo;
        acc = in_range(k, a.no, a.err) ? tpl[(long)k * (a.N + 1)] : 0.0;
    } else {
        acc = 0.0;
        const int kb = (u >> 2) - a.b - a.olo;
        for (int e = 0; e < K; ++e)
            if (in_range(kb + e, a.no, a.err)) acc = fma(a.lwd[ru][e], tpl[(long)(kb + e) * (a.N + 1)], acc);
    }
    RT ring(0.0);
    face_node_patches<NN>(g, a.np, a.ga, a.gb, [&](long p, int r0, int r1, int r2, bool inA) {
        const int ra = axis == 0 ? r0 : (axis == 1 ? r1 : r2);
        const int ru_ = axis == 0 ? r1 : r0, rv_ = axis == 2 ? r1 : r2;
        if (inA) {
            const int j = (ra - sg - a.pl0) / n;
            const long slot = (long)axis * 2 * a.npa + 2 * j + side;
            if (in_range(j, a.npa, a.err) & in_range(ru_ + a.ga, a.wa, a.err) & in_range(rv_ + a.ga, a.wa, a.err))
                acc += a.resid2[((p * 6 * a.npa + slot) * a.wa + (ru_ + a.ga)) * a.wa + (rv_ + a.ga)];
        } else {
            const int j = (ra - sg - (a.pb0 - n)) / n;  // rows from the plane pb0 - n
            const bool ok = in_range(j, a.npb + 2, a.err) & in_range(ru_ + a.gb, a.wbx, a.err) &
                            in_range(rv_ + a.gb, a.wbx, a.err);
            const long row = ((((long)axis * (a.npb + 2) + j) * 2 + side) * a.wbx + (ru_ + a.gb)) * a.wbx + (rv_ + a.gb);
            if (ok) ring_dot((const RT *)a.mom + p * a.npad, (const RT *)a.D2 + row * a.npad, a.npad, ring);
        }
    });
    a.phiB2[idx] = acc + (double)ring;
}

// Dirichlet step of a Q = 10 patch (eq. last_step_fulldiscr with the second
// layer): Delta^h u = f on the interior [1, n-1]^3 with u = phi^B on the
// closed faces and on the layer one node outside them, then phi = u + C2 h^2
// f (eq. mcapplicationfulldiscr).  With the boundary data moved to the
// right-hand side b, the interior operator is L = L_odd + E: L_odd is the
// stencil with the odd continuation across the faces (diagonal in DST-I), and
// E u(g) = sum over the offsets that leave the layer next to a face through
// it of a_s u(mirror(g + s)) (L reads zero there, L_odd minus the mirrored
// value).  u_0 = L_odd^-1 b, u_{k+1} = L_odd^-1 (b - E u_k).  One CTA per
// patch; b, u and the work array in shared memory up to n = 16, in the
// plan's workspace above; each DST pass gives a line of m = n-1 values to one
// thread (n = 16: the split-radix 15-point DST; n = 32: the split 31-point
// DST; other n: dense m x m sums with the matrix in shared memory).
struct DirWArgs {
    Items it;
    const double *sinm;  // (n-1) x n/2 half DST-I matrix sin(pi k t / n), t in [1, n/2]
    int iters;           // fixed-point steps after the first solve
};

template <typename TF, int NN>
__global__ void __launch_bounds__(256) k_dirichlet_wide(DirWArgs a) {
    constexpr int n = NN, m = n - 1, m3 = m * m * m, h = n / 2;
    constexpr bool BIG = NN > 16;  // the three arrays in the plan's global workspace (L2-resident)
    extern __shared__ double smw[];
    int p;
    const PlanPtrs &PP = item_plan(a.it, blockIdx.x, p);
    double *B, *U, *X, *S;  // right-hand side, current iterate, transform work array, DST-I matrix
    if constexpr (BIG) {
        B = (double *)PP.dscr + (long)p * 3 * m3;
        U = B + m3;
        X = U + m3;
        S = smw;
    } else {
        B = smw;
        U = B + m3;
        X = U + m3;
        S = X + m3;
    }
    const int N = PP.N, np = PP.np;
    const int i0 = p / (np * np), i1 = (p / np) % np, i2 = p % np;
    const int o0 = i0 * n, o1 = i1 * n, o2 = i2 * n;
    const TF *f = (const TF *)PP.f;
    const double ih2 = PP.inv_h2;
    const double *lam = (const double *)PP.lam;
    for (int e = threadIdx.x; e < m * m && NN != 16 && NN != 32; e += blockDim.x) {  // dense lines only
        const int k = e / m, T = e % m + 1;
        // sin(pi K (n - T') / n) = (-1)^(K+1) sin(pi K T' / n), K = k + 1
        S[e] = T <= h ? a.sinm[k * h + (T - 1)] : ((k & 1) ? -1.0 : 1.0) * a.sinm[k * h + (n - T - 1)];
    }
    // boundary value at the relative node q (a face node, or one coordinate -1 or n+1)
    auto bval = [&](int q0, int q1, int q2) -> double {
        const int G[3] = {o0 + q0, o1 + q1, o2 + q2}, q[3] = {q0, q1, q2}, ip[3] = {i0, i1, i2};
        for (int d = 0; d < 3; ++d)
            if (q[d] == -1 || q[d] == n + 1) {
                const int side = q[d] == n + 1 ? 1 : 0, j = ip[d] + side;
                const int u = d == 0 ? G[1] : G[0], v = d == 2 ? G[1] : G[2];
                if (!(in_range(j, np + 1, PP.err) & in_range(u, N + 1, PP.err) & in_range(v, N + 1, PP.err)))
                    return 0.0;
                return PP.phiB2[(((long)(d * (np + 1) + j) * 2 + side) * (N + 1) + u) * (N + 1) + v];
            }
        return phiB_at<double>(PP, n, G[0], G[1], G[2]);
    };
    for (int e = threadIdx.x; e < m3; e += blockDim.x) {
        const int q2 = e % m + 1, q1 = (e / m) % m + 1, q0 = e / (m * m) + 1;
        double r = (double)f[((long)(o0 + q0) * N + (o1 + q1)) * N + (o2 + q2)];
        const bool near = q0 <= 2 || q0 >= n - 2 || q1 <= 2 || q1 >= n - 2 || q2 <= 2 || q2 >= n - 2;
        if (near) {
#pragma unroll
            for (int s0 = -2; s0 <= 2; ++s0)
#pragma unroll
                for (int s1 = -2; s1 <= 2; ++s1)
#pragma unroll
                    for (int s2 = -2; s2 <= 2; ++s2) {
                        const double c = stencil_coef(10, s0, s1, s2);
                        if (c == 0.0) continue;
                        const int t0 = q0 + s0, t1 = q1 + s1, t2 = q2 + s2;
                        if (t0 >= 1 && t0 <= m && t1 >= 1 && t1 <= m && t2 >= 1 && t2 <= m) continue;
                        r -= c * ih2 * bval(t0, t1, t2);
                    }
        }
        B[e] = r;
    }
    __syncthreads();
    // X <- L_odd^-1 X: three DST-I passes, the eigenvalue scaling (lam holds
    // (2/n)^3 h^2 / lambda), three more passes
    double sv16[9];  // n = 16: sin(pi i / 16), i = 0..8
    sv16[0] = 0.0;
#pragma unroll
    for (int i = 1; i <= 8; ++i) sv16[i] = NN == 16 ? a.sinm[i - 1] : 0.0;
    double sv32[17];  // n = 32: sin(pi i / 32), i = 0..16
    sv32[0] = 0.0;
#pragma unroll
    for (int i = 1; i <= 16; ++i) sv32[i] = NN == 32 ? a.sinm[i - 1] : 0.0;
    auto solve = [&]() {
        for (int pass = 0; pass < 6; ++pass) {
            const int axis = 2 - (pass % 3);
            for (int l = threadIdx.x; l < m * m; l += blockDim.x) {
                const int qa = l / m, qb = l % m;
                int base, str;
                if (axis == 2) { base = (qa * m + qb) * m; str = 1; }
                else if (axis == 1) { base = qa * m * m + qb; str = m; }
                else { base = qa * m + qb; str = m * m; }
                double x[m];
#pragma unroll
                for (int t = 0; t < m; ++t) x[t] = X[base + t * str];
                if constexpr (NN == 16 || NN == 32) {  // the split-radix 15-point / split 31-point DST-I
                    if constexpr (NN == 16) dst15_fast(x, sv16);
                    else dst31_fast(x, sv32);
#pragma unroll
                    for (int k = 0; k < m; ++k) X[base + k * str] = pass == 2 ? x[k] * lam[base + k * str] : x[k];
                } else {
#pragma unroll
                    for (int k = 0; k < m; ++k) {
                        double acc = 0.0;
#pragma unroll
                        for (int t = 0; t < m; ++t) acc = fma(S[k * m + t], x[t], acc);
                        if (pass == 2) acc *= lam[base + k * str];
                        X[base + k * str] = acc;
                    }
                }
            }
            __syncthreads();
        }
    };
    for (int e = threadIdx.x; e < m3; e += blockDim.x) X[e] = B[e];
    __syncthreads();
    solve();
    for (int e = threadIdx.x; e < m3; e += blockDim.x) U[e] = X[e];
    __syncthreads();
    // E u on the layer next to a face: the offsets that leave the interior
    // through the face are (-+2, 0, 0) and (-+2, +-1, 0), (-+2, 0, +-1) along
    // its normal; their mirror images lie in the same layer, at the node
    // itself and its four in-layer neighbours (zero on the faces)
    const double e200 = stencil_coef(10, 2, 0, 0) * ih2, e210 = stencil_coef(10, 2, 1, 0) * ih2;
    auto Uin = [&](int q0, int q1, int q2) -> double {
        return (q0 < 1 || q0 > m || q1 < 1 || q1 > m || q2 < 1 || q2 > m) ? 0.0
                                                                         : U[((q0 - 1) * m + (q1 - 1)) * m + (q2 - 1)];
    };
    for (int it = 0; it < a.iters; ++it) {
        for (int e = threadIdx.x; e < m3; e += blockDim.x) {
            const int q2 = e % m + 1, q1 = (e / m) % m + 1, q0 = e / (m * m) + 1;
            double r = B[e];
            if (q0 == 1 || q0 == m)
                r -= e200 * U[e] + e210 * (Uin(q0, q1 - 1, q2) + Uin(q0, q1 + 1, q2) + Uin(q0, q1, q2 - 1) +
                                           Uin(q0, q1, q2 + 1));
            if (q1 == 1 || q1 == m)
                r -= e200 * U[e] + e210 * (Uin(q0 - 1, q1, q2) + Uin(q0 + 1, q1, q2) + Uin(q0, q1, q2 - 1) +
                                           Uin(q0, q1, q2 + 1));
            if (q2 == 1 || q2 == m)
                r -= e200 * U[e] + e210 * (Uin(q0 - 1, q1, q2) + Uin(q0 + 1, q1, q2) + Uin(q0, q1 - 1, q2) +
                                           Uin(q0, q1 + 1, q2));
        X[e] = r;
        }
        __syncthreads();
        solve();
        for (int e = threadIdx.x; e < m3; e += blockDim.x) U[e] = X[e];
        __syncthreads();
    }
    const double c2h2 = PP.c2h2;
    for (int e = threadIdx.x; e < n * n * n; e += blockDim.x) {
        const int m2 = e % n, m1 = (e / n) % n, m0 = e / (n * n);
        const bool bnd = m0 == 0 || m1 == 0 || m2 == 0;
        const int z = o0 + m0, y = o1 + m1, x = o2 + m2;
        const long gi = ((long)z * N + y) * N + x;
        const double u = bnd ? phiB_at<double>(PP, n, z, y, x) : U[((m0 - 1) * m + (m1 - 1)) * m + (m2 - 1)];
        PP.phi[gi] = u + c2h2 * (double)f[gi];
    }
}

}  // namespace

cudaError_t launch_resid_outer(const mlc_plan_s *pl, const Items &it, cudaStream_t st) {
    const Geom &g = pl->g;
    if (!g.wide) return cudaSuccess;
    NvtxRange nvtx("mlc:residuals_outer");
    ResOutArgs a{};
    a.it = it; a.n = g.n; a.s = g.s; a.ga = g.ga; a.b = g.b;
    a.npa = g.npa; a.pl0 = g.pl0; a.wa = g.wa; a.nc = g.nc;
    lagrange_rows(g.b, a.lwd);
    const int nk = (g.n + 2 * g.ga) / 4 + 2 * g.b + 1;
    const size_t sm = 8 * (size_t)nk * (g.wa + nk);
    dim3 grid(it.nitems, 6 * g.npa);
#define MLC_RESO(KK)                                                                   \
    case KK:                                                                           \
        if (g.conv == CONV_F32) k_resid_outer<float, KK><<<grid, 256, sm, st>>>(a);    \
        else k_resid_outer<double, KK><<<grid, 256, sm, st>>>(a);                      \
        break;
    switch (2 * g.b + 2) {
        MLC_RESO(4)
        MLC_RESO(6)
        MLC_RESO(8)
        MLC_RESO(10)
        MLC_RESO(12)
        default: return cudaErrorInvalidValue;
    }
#undef MLC_RESO
    return cudaGetLastError();
}

cudaError_t launch_boundary_outer(const mlc_plan_s *pl, cudaStream_t st) {
    const Geom &g = pl->g;
    if (!g.wide) return cudaSuccess;
    NvtxRange nvtx("mlc:boundary_outer");
    LagW w{};
    lagrange_rows(g.b, w.lwd);
    {
        const long tp = 6L * (g.np + 1) * g.no * (g.N + 1);
        k_plane_interp_outer<<<(unsigned)((tp + 255) / 256), 256, 0, st>>>(pl->phiH, pl->tpl2, g.N, g.n, g.np, g.b,
                                                                          g.olo, g.no, w, pl->err);
    }
    BndOutArgs a{};
    a.err = pl->err;
    a.tpl2 = pl->tpl2; a.resid2 = pl->resid2;
    a.mom = ring_moments(pl); a.D2 = pl->D2tab;
    a.phiB2 = pl->phiB2;
    a.N = g.N; a.n = g.n; a.np = g.np; a.ga = g.ga; a.gb = g.gb; a.b = g.b; a.olo = g.olo; a.no = g.no;
    a.wa = g.wa; a.wbx = g.wbx; a.npa = g.npa; a.pl0 = g.pl0; a.pb0 = g.pb0; a.npb = g.npb; a.npad = g.npad;
    std::memcpy(a.lwd, w.lwd, sizeof(a.lwd));
    const long tot = 6L * (g.np + 1) * (g.N + 1) * (g.N + 1);
    const unsigned nbk = (unsigned)((tot + 127) / 128);
#define MLC_BNDO(NN)                                                                     \
    case NN:                                                                             \
        if (g.conv == CONV_F32) k_boundary_outer<float, NN><<<nbk, 128, 0, st>>>(a);     \
        else k_boundary_outer<double, NN><<<nbk, 128, 0, st>>>(a);                       \
        break;
    switch (g.n) {
        MLC_BNDO(4)
        MLC_BNDO(8)
        MLC_BNDO(12)
        MLC_BNDO(16)
        MLC_BNDO(24)
        MLC_BNDO(32)
        default: return cudaErrorInvalidValue;
    }
#undef MLC_BNDO
    return cudaGetLastError();
}

// Fixed-point steps of the two-layer Dirichlet solve after the first: the
// error contracts by about 0.025 per step, so ten take it below 1e-16.
constexpr int kWideDirichletIters = 10;

cudaError_t launch_dirichlet_wide(const mlc_plan_s *pl, const Items &it, cudaStream_t st) {
    NvtxRange nvtx("mlc:dirichlet_wide");
    const Geom &g = pl->g;
    DirWArgs a{};
    a.it = it;
    a.sinm = (const double *)pl->sinm;
    a.iters = kWideDirichletIters;
    const int m = g.n - 1;
    // n > 16: the arrays live in the plan's workspace; shared memory holds the dense DST-I matrix
    const size_t sm = 8 * ((g.n > 16 ? 0 : 3 * (size_t)m * m * m) + (size_t)m * m);
#define MLC_DIRW(NN)                                                                                      \
    case NN:                                                                                              \
        if (g.f32in) k_dirichlet_wide<float, NN><<<it.nitems, 256, sm, st>>>(a);                          \
        else k_dirichlet_wide<double, NN><<<it.nitems, 256, sm, st>>>(a);                                 \
        break;
    switch (g.n) {
        MLC_DIRW(4)
        MLC_DIRW(8)
        MLC_DIRW(12)
        MLC_DIRW(16)
        MLC_DIRW(24)
        MLC_DIRW(32)
        default: return cudaErrorInvalidValue;
    }
#undef MLC_DIRW
    return cudaGetLastError();
}

void configure_wide() {
    const int big = 200 * 1024;
#define MLC_DIRW_ATTR(NN)                                                                                   \
    cudaFuncSetAttribute(k_dirichlet_wide<float, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);   \
    cudaFuncSetAttribute(k_dirichlet_wide<double, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    MLC_DIRW_ATTR(4)
    MLC_DIRW_ATTR(8)
    MLC_DIRW_ATTR(12)
    MLC_DIRW_ATTR(16)
    MLC_DIRW_ATTR(24)
    MLC_DIRW_ATTR(32)
#undef MLC_DIRW_ATTR
#define MLC_RESO_ATTR(KK)                                                                                   \
    cudaFuncSetAttribute(k_resid_outer<float, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);      \
    cudaFuncSetAttribute(k_resid_outer<double, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    MLC_RESO_ATTR(4)
    MLC_RESO_ATTR(6)
    MLC_RESO_ATTR(8)
    MLC_RESO_ATTR(10)
    MLC_RESO_ATTR(12)
#undef MLC_RESO_ATTR
}
