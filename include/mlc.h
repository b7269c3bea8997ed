/*
 * mlc.h -- C ABI of the GB300 two-level Method of Local Corrections (MLC)
 * solver for the free-space Poisson equation (Kavouklis & Colella,
 * arXiv:1702.08111, Sec. 4 "Fully-Discrete Two-Level Algorithm").
 *
 * Problem (Sec. 1, eqs. poisson/potential): Delta phi = f on R^3 with
 * phi(x) ~ -(int f) / (4 pi |x|) at infinity, so a positive charge gives a
 * negative potential.  The charge is sampled on the unit cube at the nodes
 * x = g h, h = 1/N, g in [0, N)^3 (axis 2 contiguous in memory); the nodes at
 * index N carry zero charge (the charge must vanish on the faces x_d = 1).
 * The result phi^{MLC,h} (Sec. 4, eq. mcapplicationfulldiscr) is returned on
 * the same N^3 nodes.
 *
 * Ownership: the caller owns every array passed in (f, phi, host buffers);
 * the library never frees them.  A plan owns its tables and its device
 * workspace and frees them in mlc_plan_destroy.  Discrete Green's function
 * tables are built once per (Q, nD, zeta) on each device and stay resident
 * until the process exits.
 *
 * Errors: every call returns an mlc_status; no exception crosses the ABI.
 * CUDA errors raised by kernels that run asynchronously are reported by the
 * next call that synchronises or checks the stream (MLC_ERR_CUDA).
 *
 * Threads: a plan may be used by one host thread at a time; different plans
 * may be used concurrently on different streams.
 */
#ifndef MLC_H
#define MLC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MLC_OK = 0,
    MLC_ERR_INVALID_ARG = 1, /* a size or pointer breaks a stated precondition */
    MLC_ERR_UNSUPPORTED = 2, /* legal for the method, not built in this library */
    MLC_ERR_OOM = 3,         /* a device or host allocation failed */
    MLC_ERR_CUDA = 4,        /* a CUDA runtime call or kernel failed */
    MLC_ERR_ADMISSION = 5,   /* server: request exceeds the memory budget */
    MLC_ERR_TIMEOUT = 6,     /* server: wait timed out / request cancelled; a bounded wait
                                inside a kernel gave up                                    */
    MLC_ERR_INDEX = 7        /* checked builds only (-DMLC_CHECKED): a computed index fell
                                outside its array; the access was skipped                  */
} mlc_status;

/* Arithmetic of a plan.  "Double-float" is an unevaluated sum hi + lo of two
 * FP32 numbers (about 48 significand bits, FP32's exponent range) computed on
 * the FP32 pipe; GB300 issues FP64 on about 1/67 of its FP32 lanes. */
typedef enum {
    MLC_TIER_FP64 = 0,     /* FP64 charge and result; every step in FP64 arithmetic on
                              the FP64 pipe (the plain FP64 solve)                        */
    MLC_TIER_SPLIT = 1,    /* FP32 charge; local convolutions (FFTs on the CUDA cores) and
                              the Legendre ring sums in FP32, the moments in FP32 with an
                              FP64 last contraction; coarse charge, coarse solve, boundary
                              values (subtract, interpolate, accumulate) and Dirichlet
                              solves in FP64; FP64 result                                 */
    MLC_TIER_DF = 2,       /* FP64 charge and result; moments in FP64, every other step in
                              double-float arithmetic                                     */
    MLC_TIER_SPLIT_DF = 3  /* as MLC_TIER_SPLIT with double-float in place of FP64 in the
                              steps after the local convolutions                          */
} mlc_tier;

typedef enum {
    MLC_MODE_MLC = 0,    /* inner radius alpha < outer radius beta, Legendre ring (Sec. 4) */
    MLC_MODE_MLC0 = 1    /* alpha = beta, no Legendre ring (Sec. 7, "MLC-0") */
} mlc_mode;

/* Parameters of a plan.  Fields set to -1 take the defaults listed. */
typedef struct {
    int N;          /* nodes per axis, h = 1/N                                          */
    int n;          /* patch side in cells (patches n i + [0,n]^3, Sec. 4); 4 | n, n | N */
    int s;          /* support: the local field box G(Omega_alpha, C b) is the patch
                       grown by s nodes (eq. initiallocalproblemsmlcII); 4 | s, s >= C b */
    int C;          /* coarsening ratio N_ref; must be 4 (Sec. 2)                       */
    int P;          /* Legendre orders: |p|_1 <= P-1 (eq. led3d); 1 <= P <= 6           */
    int Q;          /* Mehrstellen order: 4 -> 19-point, 6 -> 27-point (App. A.1),
                       10 -> the 57-point q = 10 operator in the 5x5x5 block (Sec. 8):
                       a_j by orbit of j (sorted |j_d|): (0,0,0) -1079/210, (1,0,0)
                       24/35, (1,1,0) 17/210, (1,1,1) 11/420, (2,0,0) -1/60, (2,1,0)
                       -1/420; C2 = 2/35.  Its Dirichlet step has a second boundary
                       layer one node outside the faces (MLC_STAGE_PHIB_OUTER)          */
    int g_beta;     /* outer growth ceil((beta-1) n/2) (Sec. 4); -1: beta = 3 (Q=4),
                       3.25 (Q=6, Q=10)                                                  */
    int b;          /* interpolation stencil radius, 1..5 (q_I = 2b+2); -1: 2 for Q=4,
                       3 for Q=6 (q_I = q + 2, Sec. 7), 4 for Q=10                       */
    int tier;       /* mlc_tier                                                         */
    int mode;       /* mlc_mode                                                         */
    int dgf_nD;     /* DGF table built on [-zeta nD, zeta nD]^3 (App. A.1); -1: 128,
                       raised automatically to the largest lag the plan needs           */
    int dgf_zeta;   /* -1: 2                                                            */
    int conv_chunk; /* patches per launch group of the local convolutions: their spectra
                       (the scratch between the forward and inverse transforms) exist
                       for one group at a time; -1: the library's choice (1024)        */
    int levels;     /* number of levels of the multilevel MLC (Sec. 5); -1: 2, the
                       two-level algorithm of Sec. 4.  With levels > 2 the global coarse
                       solve phi^H = G^H * F^H becomes the MLC solve of F^H on the next
                       coarser level (spacing H = C h; the same n, s, P, Q, b, g_beta,
                       mode and tier; a box of whole patches from min(F^H low corner,
                       phi^H low corner) that holds the support of F^H and the nodes
                       phi^H is read on), recursively, down to a two-level solve whose
                       coarse solve is Hockney's; the Mehrstellen correction
                       (eq. mcapplicationfullmultipole) is added on the finest level
                       only.  2 <= levels <= 6                                         */
    int coarse_s;   /* support s of the coarser levels' patches, i.e. their inner radius
                       (g_alpha = coarse_s - C b; Sec. 7.2 raises alpha at coarser levels);
                       -1: s.  Same rules as s                                          */
} mlc_params;

typedef struct mlc_plan_s *mlc_plan_t;

/* Fill *p with N, n, s, P, Q as given, C = 4 and every other field -1 (default). */
mlc_status mlc_params_init(mlc_params *p, int N, int n, int s, int P, int Q);

/*
 * Create a plan on the current CUDA device (Sec. 4 with the regions
 * Omega_alpha = G(Omega_i, s - C b), Omega_beta = G(Omega_i, g_beta)).  Builds
 * the DGF table (App. A.1) if this device has none for (Q, nD, zeta), the
 * kernel spectra for the Hockney convolutions (App. A.2), the Legendre
 * basis-field tables Delta^H(G^h * Q^p) (Sec. 4, Step 1) and the index tables,
 * and allocates the workspace.  Synchronises the device.
 * INVALID_ARG if: out is NULL; N, n, s, C, P, Q, levels break the rules
 * above; g_beta < s - C b.  UNSUPPORTED if: n is not one of 4, 8, 12, 16, 24,
 * 32; the patch FFT length (the power of two >= 2(n+s)) is above 128; the
 * coarse FFT length (the smallest even 2^a 3^b 5^c >= twice the largest
 * coarse lag) is above 512; Q = 10 with levels > 2 or a double-float tier
 * (its boundary and Dirichlet steps run in FP64: tiers FP64 and SPLIT).  With levels > 2 the plan of the next coarser
 * level is created with it, with its scratch, so that no solve allocates.
 */
mlc_status mlc_plan_create(int N, int patch, int support, int coarsening, int P, int Q,
                           mlc_plan_t *out);
mlc_status mlc_plan_create_ex(const mlc_params *params, mlc_plan_t *out);
mlc_status mlc_plan_destroy(mlc_plan_t plan);

/*
 * Replace the plan's discrete Green's function G^{h=1} (Sec. 2 eq. dgf, App.
 * A.1) by a caller-given table and rebuild every table derived from it (the
 * Hockney kernel spectra of the local and coarse convolutions, App. A.2; the
 * Legendre basis fields Delta^H(G^h * Q^p) of Sec. 4 Step 1), so that another
 * implementation's table can be used as data for isolated parity checks.
 * table: host array of (L+1)^3 FP64 values G^{h=1}[i][j][k] on the octant
 * [0, L]^3, k fastest (the layout of MLC_STAGE_DGF); copied, the caller keeps
 * it.  L must reach every lag the plan needs (the L that mlc_plan_info reports
 * for the library's own table is enough), else INVALID_ARG and the plan is
 * unchanged.  Synchronises the device; the handle stays valid.
 */
mlc_status mlc_plan_set_dgf(mlc_plan_t plan, const double *table, int L);

/* Synchronise the device and report kernel-side failures of this plan's
 * solves since the last check: TIMEOUT if a bounded wait inside a kernel (the
 * staging of a block by an asynchronous bulk copy) gave up, so the result of
 * that solve is not valid; the flag is then cleared.  mlc_solve_host calls it
 * before returning. */
mlc_status mlc_plan_status(mlc_plan_t plan);
/* (In a library built with -DMLC_CHECKED the kernels test their computed
 * indices before use: a bad one is skipped and mlc_plan_status reports
 * MLC_ERR_INDEX; normal builds compile the tests out.) */

/* Bytes of device workspace the plan holds now (tables excluded; the plan's
 * own local-convolution scratch counts once a solve has allocated it). */
mlc_status mlc_plan_workspace_bytes(mlc_plan_t plan, size_t *bytes);

/*
 * Scratch of the local convolutions (Sec. 4, Step 1: the patch spectra
 * between the forward and the inverse transforms of Hockney's method, App.
 * A.2).  The convolutions run in launch groups of conv_chunk patches, so a
 * solve needs scratch for min(conv_chunk, patches) patches: *bytes.  By
 * default the first mlc_solve with a plan allocates it and the plan keeps it.
 * mlc_plan_set_scratch hands the plan caller-owned device memory instead
 * (scratch: 256-byte aligned, at least mlc_plan_scratch_bytes bytes, owned by
 * the caller and alive while solves that use it run; NULL returns to the
 * plan's own scratch).  Contents need no initialisation and are not kept.
 * Solves that share one scratch must not overlap on the GPU.  INVALID_ARG if
 * scratch is too small or misaligned.
 */
mlc_status mlc_plan_scratch_bytes(mlc_plan_t plan, size_t *bytes);
mlc_status mlc_plan_set_scratch(mlc_plan_t plan, void *scratch, size_t bytes);

/*
 * Solve Delta phi = f in free space by the two-level MLC (Sec. 4, Steps 1-3,
 * Dirichlet solves and the Mehrstellen correction).  f: device array of N^3
 * values (FP32 for the split tiers, FP64 for the others), x = g h, axis 2
 * contiguous.  phi: device array of N^3 FP64 values, same layout; may not
 * alias f.  Work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 * default stream); the call returns without synchronising.  The first call
 * with a plan that has no caller-owned scratch allocates the plan's
 * local-convolution scratch (see mlc_plan_set_scratch).  Two steps that
 * do not depend on the local convolutions' chain (the moments, then the
 * face-plane residuals) run on a stream the plan owns, forked from and joined
 * back to `stream` with events, so all of the solve's work follows earlier
 * work on `stream` and precedes later work on it.  Calls with the same plan
 * must not overlap on the GPU (they share the plan's workspace).
 */
mlc_status mlc_solve(mlc_plan_t plan, const void *f, void *phi, void *stream);

/*
 * As mlc_solve, for callers that must not allocate device memory when they
 * solve (for example a plugin whose host application has already reserved the
 * device memory, or code running while a CUDA graph is captured in global
 * mode, where allocation calls are not permitted).  The paper has no
 * counterpart: this is an engineering variant of mlc_solve.  The plan is
 * created beforehand; this call allocates nothing and takes the scratch of the
 * local convolutions (the patch spectra) from one static device array of
 * 64 MiB that every GPU loading the library holds until the process exits,
 * instead of from the plan's workspace.  Same f, phi, stream contract and the
 * same result as mlc_solve, but every step runs on `stream` (no side stream:
 * the moments and residuals do not overlap the convolution chain).
 * INVALID_ARG if the spectra of one launch group (min(conv_chunk, patches)
 * patches) need more than 64 MiB (about 1.1 MB per patch of 16^3 with support
 * 16 in the FP64 and double-float tiers, half that in the split tiers: some
 * 60 and 120 patches; lower conv_chunk to fit more) or the current device is
 * not the plan's.  The first call on a device looks
 * up the array's device address with that device current: make it before any
 * stream capture.  All calls share the array and see the last call's
 * contents (every element a call reads it has written first, so nothing needs
 * clearing); calls that overlap on the GPU race on it and must not be issued.
 */
mlc_status mlc_solve_noalloc(mlc_plan_t plan, const void *f, void *phi, void *stream);

/*
 * As mlc_solve with host arrays: copies f (host, pinned or pageable) to the
 * plan's device staging buffer, solves, copies phi back to the host array and
 * synchronises the stream (not the device) before returning.  Reports TIMEOUT
 * like mlc_plan_status if a bounded wait of this solve gave up.
 */
mlc_status mlc_solve_host(mlc_plan_t plan, const void *f_host, void *phi_host, void *stream);

/*
 * Solve `count` independent problems in one call (no counterpart in the
 * paper: each problem is the solve of Sec. 4).  Problems are grouped by patch
 * geometry and tier; the per-patch work of all problems of a group runs in
 * shared launches (moments, local convolutions, residuals, Dirichlet steps),
 * the groups concurrently, and each problem's coarse charge, coarse solve and
 * boundary values on parallel branches.  The launch sequence is captured as a
 * CUDA graph per set of plans, tuned on the first call (branches, slab launch
 * shape, patches per convolution launch group) and replayed on later calls;
 * a later call with other f / phi arrays for the same plans rewrites the
 * graph's problem records on `stream` (after the earlier replays finish) and
 * replays the same graph.  plans[k], f[k], phi[k] as in mlc_solve; plans must
 * be distinct (INVALID_ARG otherwise) and on the current device.  The first
 * call with a set of plans allocates its item tables and convolution scratch.
 */
mlc_status mlc_batch_solve(int count, const mlc_plan_t *plans, const void *const *f,
                           void *const *phi, void *stream);

/* Stage exports for testing: copy an intermediate result of the last solve
 * (or, for the index stages, the plan's indexing as the kernels compute it)
 * to host memory (FP64 unless noted).  `bytes` must equal the stage's size,
 * returned by mlc_debug_stage_bytes.  Both synchronise the device. */
typedef enum {
    MLC_STAGE_MOMENTS = 0,  /* Legendre coefficients c_p^i, [patch][p] (Sec. 4, Step 1)      */
    MLC_STAGE_FH = 1,       /* coarse charge F^H on its extent [lo,hi]^3 (Step 2)            */
    MLC_STAGE_PHIH = 2,     /* coarse potential phi^H on [-b, N/4+b]^3 (Step 2)              */
    MLC_STAGE_PHIB = 3,     /* boundary values phi^B on the face planes,
                               [axis][plane j][u][v], plane x_axis = j n, (u,v) the other
                               two coordinates in increasing axis order (Step 3)             */
    MLC_STAGE_DGF = 4,      /* the DGF octant G^{h=1}[0..L]^3, L = entry 14 of mlc_plan_info  */
    MLC_STAGE_COARSE_SAMPLES = 5, /* local fields phi^{i,h} at the coarse points of each patch's
                               field box: [patch][k0][k1][k2], k in [-s/4, (n+s)/4] relative
                               to the patch's coarse origin n i / 4 (Step 1, eq. FDLD)      */
    MLC_STAGE_FACE_INDEX = 6, /* int32 (not FP64): the patch indexing of Step 3 (eq.
                               philocmlcII) for every face-plane node, nodes in the order of
                               MLC_STAGE_PHIB: offsets[nodes + 1], then entries; node k owns
                               entries offsets[k] .. offsets[k+1]-1, each 2 i + 0 if
                               Omega_alpha(i) holds the node, 2 i + 1 if only Omega_beta(i)
                               does (i the patch's linear index), ascending i               */
    MLC_STAGE_COARSE_INDEX = 7, /* int32: the same for every coarse node of the F^H extent
                               ([k0][k1][k2] order) and the coarse boxes C(Omega_alpha(i)),
                               C(Omega_beta(i)) (eq. FDLD)                                */
    MLC_STAGE_PHIB_OUTER = 8 /* Q = 10 only: boundary values on the second layer, the planes
                               one node off the face planes, [axis][plane j][side][u][v],
                               x_axis = j n - 1 (side 0) or j n + 1 (side 1), j in [0, N/n],
                               (u,v) in [0, N]^2 as for MLC_STAGE_PHIB (Sec. 8)            */
} mlc_stage;

mlc_status mlc_debug_stage_bytes(mlc_plan_t plan, int stage, size_t *bytes);
/* Per-launch timing of later solves with this plan: when enabled, mlc_solve
 * runs its 13 launches in sequence on its stream (no side stream) and records
 * a CUDA event before each launch and after the last.  mlc_debug_timing waits for the last solve's final event and
 * writes the 13 durations (ms) in launch order: moments; local convolutions:
 * forward x, fused slab (forward y and z, kernel spectrum, inverse z and y),
 * inverse x; residuals; assembly of F^H; coarse convolution x, y, z (forward,
 * kernel, inverse), inverse y, inverse x; boundary values; Dirichlet solves.
 * count must be >= 13. */
mlc_status mlc_debug_set_timing(mlc_plan_t plan, int enable);
/* Test hook for the failure path of the bounded waits (no counterpart in the
 * paper): kind 1 makes later solves with this plan skip the bulk copy that the
 * local-convolution inverse-x kernel waits for, with the wait limited to 64
 * tests, so every such wait runs out, the kernel records the failure and
 * returns, and mlc_plan_status reports TIMEOUT (the potential is then not
 * valid).  kind 0 restores normal solves.  INVALID_ARG for other kinds. */
mlc_status mlc_debug_set_fault(mlc_plan_t plan, int kind);
mlc_status mlc_debug_timing(mlc_plan_t plan, float *ms_out, int count);
/* Configuration the batch autotuner chose for this set of plans (f, phi as
 * passed to mlc_batch_solve; the choice does not depend on them): 2 x
 * (parallel branches of the per-problem coarse steps) + 1 if the
 * local-convolution slab kernel runs persistently; 0 if this set has not been
 * solved yet. */
int mlc_debug_batch_choice(int count, const mlc_plan_t *plans, const void *const *f, void *const *phi);
/* Patches per local-convolution launch group (the number of patches whose
 * pencils one set of convolution launches transforms) that the autotuner
 * chose for this set of plans, from {512, 1024, 2048}; 0 if not solved yet. */
int mlc_debug_batch_chunk(int count, const mlc_plan_t *plans, const void *const *f, void *const *phi);
mlc_status mlc_debug_export(mlc_plan_t plan, int stage, void *host, size_t bytes);
/* Geometry of the plan: out[0..15] = N, n, s, b, g_alpha, g_beta, P, npoly,
 * fh_lo, fh_hi, phih_lo, phih_hi, M (patch FFT), Mc (coarse FFT), L (DGF
 * extent), nD. */
mlc_status mlc_plan_info(mlc_plan_t plan, int *out16);

/* ---------------- continuous-batching server ---------------- */
typedef struct mlc_server_s *mlc_server_t;

typedef struct {
    mlc_params params;   /* problem definition (N, n, s, P, Q, tier, ...)          */
    const void *f;       /* device charge, as in mlc_solve; must stay alive until done */
    void *phi;           /* device result, as in mlc_solve; must stay alive until done */
} mlc_request;

typedef struct {
    mlc_status status;   /* outcome of the solve                                     */
    double latency_ms;   /* enqueue -> completion                                    */
    double queue_ms;     /* enqueue -> start of its batch                            */
} mlc_result;

/* Create a server on the current device with a device-memory budget (bytes)
 * for the plans and workspaces of admitted requests, and at most `max_batch`
 * requests per launch group. */
mlc_status mlc_server_create(size_t hbm_budget_bytes, int max_batch, mlc_server_t *out);
mlc_status mlc_server_destroy(mlc_server_t srv);
/* Enqueue a request (copied); returns a ticket.  ADMISSION if the request
 * alone can never fit the budget; INVALID_ARG for bad parameters. */
mlc_status mlc_server_enqueue(mlc_server_t srv, const mlc_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (<0: forever) for a ticket; TIMEOUT if not done. */
mlc_status mlc_server_wait(mlc_server_t srv, uint64_t ticket, int timeout_ms, mlc_result *res);

const char *mlc_status_string(mlc_status s);

#ifdef __cplusplus
}
#endif
#endif /* MLC_H */
