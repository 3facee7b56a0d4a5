/*
 * tdbem.h -- C ABI of the GB300 time-domain boundary element library.
 *
 * The library solves transient electromagnetic scattering off perfect
 * electric conductors by marching on in time (paper section 2): the surface
 * current J = n x H (n pointing into the conductor, section 2.1) is expanded in
 * RWG basis functions f_j (one per mesh edge) and an order-2 B-spline in time
 * (section 2.2),
 *
 *     J(x, t) = sum_j sum_beta J_j^beta f_j(x) N^{beta,2}(t),
 *
 * and the Galerkin-tested CFIE (eq. cfie, built from the time-differentiated
 * EFIE, the time-differentiated MFIE and the MFIE) becomes, at every step
 * alpha = 1 .. Nt-1 (eqs. system, solve and R),
 *
 *     Z0 J^{alpha-1} = R^{alpha-1},
 *     R^{alpha-1}   = V^{alpha-1} - sum_{m >= 2} Zt^(m) J^{alpha-m},
 *
 * where Zt^(m) is the interaction matrix of time lag m (eq. z_ij with the
 * B-spline of eq. J), Z0 = Zt^(1) and V is the tested incident field (eq. v_i).
 * Two modes evaluate the history sum R:
 *   TDBEM_DIRECT : every edge pair, FP64 (the conventional method, section
 *                  3.6.3).  Coefficients are assembled and Z0 solved in FP64;
 *                  with one right-hand side the history products run in
 *                  double-float arithmetic (each operand a pair of FP32
 *                  numbers, 46 significant bits per term, compensated sums),
 *                  which needs coefficients and currents inside FP32's normal
 *                  range (about 1e-38 .. 3e38);
 *   TDBEM_FAST   : near pairs directly and far pairs by the space-time
 *                  interpolation-based FMM (section 3: P2M, M2M, M2L, L2L, L2P
 *                  over an octree with per-level time intervals).
 *
 * Conventions shared by every entry point
 *   * Units are normalised through eps and mu (c = 1/sqrt(eps mu)).
 *   * Edges are numbered in increasing (min vertex, max vertex) order.  The
 *     "+" triangle of an edge is the one whose winding runs from its smaller
 *     to its larger vertex; f_j = +l/(2A+) (x - o+) there and -l/(2A-) (x - o-)
 *     on the other triangle.  Triangles must be wound consistently.
 *   * J^beta (beta = 0 .. Nt-2) multiplies f_j N^{beta,2}; step alpha produces
 *     J^{alpha-1}.  Vectors are [ne] doubles in edge order.
 *   * Every pointer argument is a HOST pointer unless the name ends in _dev.
 *     The caller owns all arrays; the library copies what it needs during
 *     the call and keeps no pointer to caller memory.
 *   * Errors are returned, never thrown or trapped.  tdbem_last_error gives a
 *     one-line description.  After TDBEM_ECUDA or TDBEM_ETIMEOUT the context
 *     can only be destroyed.
 *   * Calls on one context are not thread-safe; distinct contexts are.
 */
#ifndef TDBEM_H
#define TDBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdbem_ctx tdbem_ctx;

typedef enum {
  TDBEM_OK = 0,
  TDBEM_EINVAL = 1,      /* bad argument (NULL pointer, size out of range, unsupported order) */
  TDBEM_EMESH = 2,       /* mesh not a closed consistently-wound 2-manifold, or degenerate triangle */
  TDBEM_EBREAKDOWN = 3,  /* time interval of the finest level holds no whole step (section 3.4.1 Remark 1) */
  TDBEM_ENOMEM = 4,      /* device or host allocation failed */
  TDBEM_ENOCONV = 5,     /* Z0 solve did not reach the tolerance within solve_maxit; best iterate kept */
  TDBEM_ETIMEOUT = 6,    /* a bounded device wait expired */
  TDBEM_ESTATE = 7,      /* call out of order (e.g. step beyond Nt-1, no incident field set) */
  TDBEM_ECUDA = 8        /* CUDA runtime error */
} tdbem_status;

typedef enum { TDBEM_DIRECT = 0, TDBEM_FAST = 1 } tdbem_mode;

/* arithmetic of the M2L contraction (fast mode, m2l_prec) and of the direct
   history sum (p2p_prec) */
typedef enum {
  TDBEM_P_FP32 = 0,   /* FP32 CUDA cores */
  TDBEM_P_TF32 = 1,   /* TF32 tensor cores, FP32 accumulate */
  TDBEM_P_BF16 = 2,   /* BF16 tensor cores, FP32 accumulate */
  TDBEM_P_BF16X3 = 3, /* split-precision BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulate */
  TDBEM_P_TF32X3 = 4, /* split-precision TF32 (hi*hi + hi*lo + lo*hi), FP32 accumulate */
  TDBEM_P_F16X3 = 5,  /* split-precision FP16 (hi*hi + hi*lo + lo*hi), FP32 accumulate, on the FP16 rate
                         (twice TF32's): each operator and each moment column is scaled by a power of two
                         (exact) that brings its largest magnitude into [2^14, 2^15), and the products are
                         unscaled in FP32.  hi + lo carry 22 significand bits, as in TF32 x 3 */
  TDBEM_P_FP64 = 6,   /* FP64: for p2p_prec, the default (see there) */
  TDBEM_P_FP24 = 7    /* p2p_prec only: FP32 with the significand rounded to 16 bits, 3 bytes (see there) */
} tdbem_prec;

typedef struct {
  int32_t d;            /* temporal B-spline order; only 2 is supported (paper's choice) */
  int32_t p_s, p_t;     /* interpolation points per axis in space and time (fast mode), 2..8 */
  int32_t n_leaf;       /* an octree cell is split while it holds more than n_leaf edges */
  double theta, zeta;   /* CFIE coupling parameters of eq. cfie (paper: 1, 1) */
  double eps, mu;       /* permittivity and permeability */
  double s_jump;        /* weight of the MFIE identity term (+1: exterior limit, 0: omitted) */
  int32_t mode;         /* tdbem_mode */
  int32_t m2l_prec;     /* tdbem_prec */
  double solve_tol;     /* relative residual of the Z0 solve */
  int32_t solve_maxit;  /* iteration cap of the Z0 solve */
  int32_t warm_start;   /* 0: zero initial guess, 1: cubic extrapolation of past currents */
  int32_t n_rhs;        /* right-hand sides marched together, 1 .. TDBEM_MAX_RHS (batched form) */
  int32_t jacobi_sweeps; /* Z0 solve: at most this many FP64 Jacobi sweeps before the Krylov refinement
                            (0: Krylov only); a sweep that does not cut the residual by 0.7 ends them */
  int32_t m2l_tile_rows; /* tensor-core M2L: rows of the product per CTA, 128 or 256; 0 (default) times
                            both at setup on each level and keeps the faster, with the resident-operator
                            kernel as a third candidate for the FP16 form (see tdbem_info.m2l_resident);
                            1 forces the resident-operator kernel where it applies (128 elsewhere) */
  int32_t precond;       /* Z0 solve preconditioner: 0 Jacobi; 1 (default) triangle blocks (the inverses of the 3 x 3
                            blocks of Z0 among the RWG functions of each triangle, summed) */
  int32_t far_overlap;   /* 1 (default): the steps overlap.  Fast mode: the M2L products of a gating event with
                            lag q >= 2, whose local coefficients are first read one interval later, run on a
                            lowest-priority second stream of the context while the next steps proceed; with
                            one right-hand side, the near-field lags >= 3 of step alpha + 2 are summed on a
                            middle-priority third stream while step alpha's solve runs.  Direct mode with one
                            right-hand side: likewise the history lags >= 3 of step alpha + 2 (which need the
                            currents up to J^{alpha-1} only) are summed on a middle-priority side stream during
                            step alpha + 1; the step then adds the lag-2 coefficients and V.  Both orders do
                            the same arithmetic there, so the currents are bitwise equal.  0: every kernel on the context's
                            stream in program 1's order.  The library's own stream has the highest priority (a
                            caller's stream keeps its own) */
  int32_t solve_grid;    /* single-RHS Z0 solve: 0 (default) one thread-block cluster below 49152 RWG functions
                            and a cooperative grid of every SM from there on; 1 always the cluster; 2 always
                            the grid */
  double chi;            /* weight of the time-differentiated MFIE inside the coupling: the tested equation is
                            dtEFIE + theta eta (chi dtMFIE + zeta MFIE).  1 (default): the paper's CFIE of
                            eq. cfie (CFIE1); zeta = 0: CFIE2; chi = 0: CFIE3 (section 4.3) */
  int32_t far_kernel;    /* fast mode, kernel of the far field (for checks of the FMM's exactness):
                              0 (default): the truncated-power kernels of the method, K_phi = (c tau - r)_+^2/(r (c dt)^2)
                                 and K_A = dK_phi/dt (tau = t - s, r = |x - y|; eq. U and section 3.3);
                              1: the polynomial K_phi = (1 + r^2) T3(tau/ts - 1), T3(x) = 4x^3 - 3x the
                                 Chebyshev cubic, ts = 64 dt (lengths in the mesh's unit), with K_A = dK_phi/dt.
                                 It has degree 2 in each coordinate and 3 in t and s, so the space-time
                                 interpolation reproduces it exactly for p_s >= 3 and p_t >= 4: the far field
                                 then equals its plain windowed sum up to rounding, whatever the tree;
                              2: zero (no far field: the history sum is the near field alone);
                              3: as 1 with the Chebyshev quadratic T2(x) = 2x^2 - 1 for T3: degree 2 in every
                                 variable, reproduced exactly by both interpolants (s_interp, t_interp) for
                                 p_s, p_t >= 3.
                            The window of source intervals, the truncated J-hat and the time gating are the
                            same for every choice. */
  int32_t s_interp;      /* fast mode, interpolation in space: 0 (default) Lagrange on p_s Chebyshev nodes per
                            direction of each cell; 1 the paper's CHI (section 3.2): piecewise cubic Hermite on
                            p_s >= 2 uniformly spaced nodes per direction (the cell's faces included), the node
                            derivatives finite differences of the node values (central inside, second-order
                            one-sided at the faces, first-order when p_s = 2).  CHI reproduces quadratics */
  int32_t t_interp;      /* fast mode, interpolation in time, the same two choices on the p_t nodes of each
                            interval.  far_kernel = 1 (cubic in time) is reproduced exactly by t_interp = 0 only */
  int32_t a_deriv;       /* fast mode, where the far field's vector potential takes its two time derivatives
                            (section 4.3.2): 0 (default) the paper's split, one on the interpolated kernel
                            (dU/dt) and one on the target's time factor; 1 both on the target factor (U
                            interpolated); 2 both on the kernel (d^2U/dt^2, a step in time, interpolated) */
  int32_t solve_cluster;  /* CTAs of the single-RHS cluster solve: 1, 2, 4, 8 or 16 caps it; 0 (default) the
                             largest cluster the device schedules (16 on GB300), except in the pipelined direct
                             march with a history sum streaming at least 3 GB per step, where it is 4: the
                             solve overlaps that sum there, and a smaller cluster leaves SMs to it */
  int64_t max_device_bytes; /* device memory budget of the context's own allocations (0: none).  An allocation
                               that would exceed it fails as if the device were full: tdbem_create returns
                               TDBEM_ENOMEM with nothing left allocated.  Per-call temporaries of
                               tdbem_history_eval and the learned warm start's buffers (tdbem_mlp_*) are
                               outside it. */
  int32_t p2p_prec;      /* direct mode, precision of the stored coefficients Zt^(m) of the lags m >= 3 in the
                            history sum of eq. R (the instantaneous Z0 of the solve, the lag-2 coefficients,
                            the currents and every sum stay in FP64 or double-float):
                              TDBEM_P_FP64 (default): each coefficient held as an unevaluated sum of two FP32
                                 numbers (hi + lo, 8 bytes, 48 significand bits), products and sums in
                                 double-float; the currents equal the FP64 oracle's to about 1e-10;
                              TDBEM_P_FP32: the P2P arithmetic of the paper's FP32 form: each coefficient
                                 rounded to FP32 (4 bytes, half the memory traffic of the history sum),
                                 multiplied by the FP32-rounded history and summed over the lags of one
                                 edge pair with FP32 FMAs; the per-pair sums are added in double-float and
                                 the currents stay FP64.  With u = 2^-24 and n the longest lag window, the
                                 history sum of row i moves by at most about (2 + n) u sum |Zt^(m)_ij|
                                 |J_j|.  Needs n_rhs = 1 and a history ring of at most 128 steps (EINVAL
                                 otherwise);
                              TDBEM_P_FP24: as FP32, with each stored coefficient's significand further
                                 rounded to 16 bits (relative 2^-16, 3 bytes: a quarter less traffic than
                                 FP32); the bound gains 2^-16 sum |Zt^(m)_ij| |J_j|.  Same conditions.
                            Fast mode stores its near field in FP32 whatever the value (every value is
                            accepted). */
} tdbem_params;

/* Largest n_rhs.  The R right-hand sides of a context (incident waves on one
   scatterer) share every stored operator: the near field becomes a sparse
   matrix times an R-column block, the M2L products gain R times more columns
   per operator, and the R Z0 solves run in one launch. */
#define TDBEM_MAX_RHS 64

/* Fills defaults: d=2, p_s=p_t=4, n_leaf=64, theta=zeta=1, eps=mu=1, s_jump=1,
   DIRECT, FP32, solve_tol=1e-13, solve_maxit=1000, warm_start=1, n_rhs=1,
   jacobi_sweeps=0, m2l_tile_rows=0, precond=1, far_overlap=1, solve_grid=0, chi=1, far_kernel=0,
   s_interp=0, t_interp=0, a_deriv=0, solve_cluster=0, max_device_bytes=0, p2p_prec=FP64. */
void tdbem_default_params(tdbem_params* p);

/* Builds the context for a closed triangle mesh: verts [nv][3] (float64),
   tris [ntri][3] (int32, consistently wound), time step dt > 0 and Nt >= 2 time
   levels (paper Program 1 inputs).  Validates the mesh, builds the RWG edge
   table and, in fast mode, the space-time hierarchy (section 3.4.1); assembles
   on the device every coefficient the chosen mode stores.  Allocates device
   memory on the current device.  Returns EMESH, EBREAKDOWN, ENOMEM, ECUDA or
   EINVAL on failure with *out = NULL. */
tdbem_status tdbem_create(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri, double dt,
                          int32_t Nt, const tdbem_params* params, tdbem_ctx** out);

tdbem_status tdbem_num_edges(const tdbem_ctx* ctx, int64_t* ne);

/* edge_vert [ne][2] (min, max vertex), edge_tri [ne][2] (+ triangle, - triangle) */
tdbem_status tdbem_edges(const tdbem_ctx* ctx, int32_t* edge_vert, int32_t* edge_tri);

/* CUDA stream (a cudaStream_t passed as void*) on which every later kernel of
   this context is launched; NULL selects the library's own stream.  With
   far_overlap on, the deferred M2L products run on a second stream owned by
   the context, ordered after this one by events; every call that marches to
   completion (march, march_dev, march_many), resets, evaluates a history or
   reads the profile makes this stream wait for them. */
tdbem_status tdbem_set_stream(tdbem_ctx* ctx, void* stream);

/* Incident plane wave for right-hand side `rhs` (0 <= rhs < n_rhs; a
   right-hand side never set has zero incident field):
   pulse = {k[3], pol[3], f0, sigma, t0, z_min}; E = pol g(u), H = k x E / eta,
   u = t - (k.x - z_min)/c, and
     sigma > 0: the modulated Gaussian g(u) = cos(2 pi f0 (u - t0)) exp(-(u-t0)^2/(2 sigma^2));
     sigma < 0: the Sin^2 pulse of the paper's test problem (section 4.1) with
                length Lambda = f0 > 0 and amplitude A = -sigma:
                g(u) = A sin^2(2 pi c (u - t0) / Lambda) while 0 <= 2 pi c (u - t0) / Lambda <= 2 pi, else 0.
   V^{alpha-1} (eq. v_i) is then evaluated on the device at every step.
   EINVAL for sigma = 0 or a Sin^2 length <= 0. */
tdbem_status tdbem_set_incident_plane(tdbem_ctx* ctx, int32_t rhs, const double* pulse);

/* Use caller-supplied right-hand sides instead: V[(alpha-1)*ne + i] for
   alpha = 1 .. Nt-1 (host, copied to the device) is right-hand side `rhs`.
   Once any caller table exists it replaces the plane-wave tables of every
   right-hand side (columns never supplied are zero). */
tdbem_status tdbem_set_rhs(tdbem_ctx* ctx, int32_t rhs, const double* V);

/* History evaluation without solving (eq. R): for a given history
   J_hist[(b*n_rhs + r)*ne + j] = J_j^b of right-hand side r (b = 0 .. n_hist-1;
   J^b = 0 outside) returns R_out[r*ne + i] = V_i^{alpha-1} - sum_{m >= 2}
   Zt^(m)_ij J_j^{alpha-m}, evaluated exactly as tdbem_step evaluates it (far
   field through the FMM in fast mode, with the same time gating).  V is the
   incident field of each right-hand side (zero where none is set).  Does not
   change the marching state. */
tdbem_status tdbem_history_eval(tdbem_ctx* ctx, int32_t alpha, const double* J_hist, int32_t n_hist,
                                double* R_out);

/* Capacity, in doubles, of the fixed device scratch array used by
   tdbem_history_eval_noalloc (16 MiB). */
#define TDBEM_NOALLOC_SCRATCH_DOUBLES (2 * 1024 * 1024)

/* Same result as tdbem_history_eval, for callers that must not allocate
   device memory at the time of the call: code running while another library
   captures the stream into a CUDA graph, real-time loops whose allocator is
   frozen, or hosts that own the whole device pool.  tdbem_history_eval
   allocates a temporary device ring for the supplied history on every call;
   this variant stages the history in a file-scope static device array of
   TDBEM_NOALLOC_SCRATCH_DOUBLES doubles instead (reserved on every GPU that
   loads the library, until exit), and calls no cudaMalloc, cudaFree or other
   allocating routine.  The paper has no counterpart: it is a deployment
   convenience.
     * Needs ne * n_rhs * (L + K) <= TDBEM_NOALLOC_SCRATCH_DOUBLES, where L is the
       context's history ring length and K the number of history steps used
       (at most the largest lag); larger problems get TDBEM_EINVAL.
     * Direct mode only (TDBEM_EINVAL otherwise).
     * The context's device must be the current device.
     * The first call on a device resolves the array's device address
       (cudaGetSymbolAddress) once; make that first call before any stream
       capture.  The address is kept for the life of the process, so it does
       not survive a cudaDeviceReset of that device (the array's storage does
       not either).
     * Every call shares the one array and rewrites all of it that it reads, so
       no state carries over between calls; calls that overlap on the GPU (two
       streams, or two contexts on one device) race on it.
   Arguments, ownership and errors as for tdbem_history_eval. */
tdbem_status tdbem_history_eval_noalloc(tdbem_ctx* ctx, int32_t alpha, const double* J_hist, int32_t n_hist,
                                        double* R_out);

/* One step of Program 1: adds V^{alpha-1}, evaluates the history sum, solves
   Z0 J^{alpha-1} = R^{alpha-1} and, in fast mode at gating steps, pushes the far
   field of the finished time intervals into future right-hand sides.  J_out
   ([n_rhs][ne], may be NULL) receives J^{alpha-1}; iters (may be NULL) the
   solver iterations.  ESTATE after Nt-1 steps. */
tdbem_status tdbem_step(tdbem_ctx* ctx, double* J_out, int32_t* iters);

/* One step with a caller-supplied right-hand side for this step only:
   V ([n_rhs][ne], host) is V^{alpha-1} (eq. v_i), copied to the device during
   the call; J_out as in tdbem_step.  Used for end-to-end streaming where the
   incident field is produced on the host. */
tdbem_status tdbem_step_v(tdbem_ctx* ctx, const double* V, double* J_out, int32_t* iters);

/* The same, without waiting: the copy of V, the step and the copy of J^{alpha-1} into J_out are enqueued
   on the context's stream and the call returns.  Up to 4 steps may be outstanding (a fifth call first
   waits for the oldest).  With V and J_out in pinned host memory (cudaMallocHost) the copies overlap the
   computation; V may be reused when the call returns, J_out is written once the step has been waited
   for.  tdbem_step_wait waits for the oldest outstanding step and returns its status (ENOCONV when its
   solve missed the tolerance; iters, may be NULL, its solver iterations; OK with iters 0 when none is
   outstanding).  tdbem_reset and tdbem_save first wait for every outstanding step. */
tdbem_status tdbem_step_v_async(tdbem_ctx* ctx, const double* V, double* J_out);
tdbem_status tdbem_step_wait(tdbem_ctx* ctx, int32_t* iters);

/* n_steps steps; J_all ([n_steps][n_rhs][ne], may be NULL) receives every J.
   Host arrays of every entry point keep the right-hand side index outside
   the edge index ([n_rhs][ne]); on the device the library stores it innermost
   ([ne][n_rhs]) and converts on the way in and out. */
tdbem_status tdbem_march(tdbem_ctx* ctx, int32_t n_steps, double* J_all);

/* Same with the result written to device memory J_all_dev (may be NULL). */
tdbem_status tdbem_march_dev(tdbem_ctx* ctx, int32_t n_steps, double* J_all_dev);

/* March several scatterers together.  Context i (its own mesh, dt, tree and
   right-hand sides) takes n_steps[i] steps; the steps are issued in rounds,
   one step of every context that still has steps in each round, each context
   on its own stream (tdbem_set_stream, or the library's stream per context),
   so that the kernels of different scatterers overlap on the GPU where one
   scatterer alone leaves SMs idle (the Z0 solve of one context occupies one
   16-SM cluster).  It is an interleave issued from the host, not a single
   persistent launch.  J_all_dev (array of n device pointers, each
   [n_steps[i]][n_rhs][ne] or NULL; the array itself may be NULL) receives
   every current, as in tdbem_march_dev.  All contexts must live on the current
   device and be distinct.  On an error, failed (may be NULL) receives the
   index of the context that reported it (-1 for invalid arguments) and the
   others may have taken some of their steps. */
tdbem_status tdbem_march_many(tdbem_ctx* const* ctxs, int32_t n, const int32_t* n_steps, double* const* J_all_dev,
                              int32_t* failed);

/* Restart the march at alpha = 1 (history and future right-hand sides cleared). */
tdbem_status tdbem_reset(tdbem_ctx* ctx);

/* Checkpoint and resume.  tdbem_save writes the march state to the file at
   `path`: the step counter alpha, the history ring of the currents (every
   J^beta a later step reads), the current solution and, in fast mode, the
   far field in flight -- per octree level the moments of the recent source
   intervals and the local coefficients of the target intervals not yet
   reached, and the far right-hand sides ahead of the current step.  Deferred
   work is waited for first.  tdbem_load reads such a file into a context
   created with the same mesh, dt, Nt and parameters (checked against a header
   and a hash of the mesh: EINVAL otherwise, with the state unchanged); the
   march then continues from the saved step.  The incident fields or
   caller-supplied right-hand sides, and the learned warm start's network, are
   inputs and are not in the file: set them on the loading context as on the
   saving one.  A direct march resumed this way is bit-identical to an
   uninterrupted one; in fast mode the far field's FP32 atomic accumulation
   already makes two uninterrupted marches differ in the last bits.  The
   paper has no counterpart (its marches run in one go).  File errors give
   EINVAL with tdbem_last_error naming the path. */
tdbem_status tdbem_save(tdbem_ctx* ctx, const char* path);
tdbem_status tdbem_load(tdbem_ctx* ctx, const char* path);

/* Current step alpha (the next tdbem_step solves J^{alpha-1}). */
tdbem_status tdbem_alpha(const tdbem_ctx* ctx, int32_t* alpha);

/* Sizes and counters for reporting: see tdbem_info fields. */
typedef struct {
  int64_t ne, n_tri;
  int32_t lmax, n_levels;          /* octree depth (fast mode) */
  int32_t mt_leaf;                 /* steps per time interval at the finest level */
  int64_t n_near_pairs;            /* edge pairs handled directly */
  int64_t near_coef_bytes;         /* bytes of the near-field coefficients as assembled in FP64 (direct mode: every
                                      pair; with one right-hand side the history sum then streams its own store,
                                      history_bytes) */
  int64_t device_bytes;            /* device memory held by the context */
  double setup_seconds;            /* wall time of tdbem_create */
  int64_t total_solver_iters;
  int32_t solver_cluster;          /* CTAs of the single-RHS Z0 solve: one thread-block cluster, or for meshes of
                                      49152 RWG functions or more a cooperative grid of every SM (0 before the
                                      first solve) */
  int64_t n_far_pairs;             /* interaction-list cluster pairs over all levels (fast mode) */
  double m2l_flops_per_step;       /* M2L flops per step, averaged over the gating cycle (fast mode) */
  int64_t total_jacobi_sweeps;     /* FP64 Jacobi sweeps of the Z0 solves (per-cluster maximum when batched) */
  int32_t m2l_tile_rows[8];        /* per octree level: rows of the M2L product per tensor-core CTA (128 or
                                      256), chosen at setup by timing both shapes; 0 where no tensor-core M2L runs */
  int64_t z0_nnz;                  /* stored non-zeros of Z0 (the solver's sparse matrix) */
  int32_t max_lag;                 /* largest time lag m with a stored coefficient: from step alpha = max_lag + 1 on,
                                      every history step a coefficient can reach is inside the march (the steady
                                      state of the history sum) */
  int32_t m2l_resident;            /* bit l set where level l's M2L runs the resident-operator kernel (FP16 form,
                                      P <= 256: the operator's 128-row tiles stay in shared memory over runs of
                                      column tiles), chosen at setup against the tiled shapes by timing */
  int64_t device_bytes_peak;       /* the most device memory the context held at once, setup included (a
                                      max_device_bytes at least this large lets tdbem_create succeed) */
  int64_t history_bytes;           /* direct mode: bytes the history sum of the lags >= 3 streams per step (its
                                      coefficient store and lag windows); 0 where it runs untiled */
} tdbem_info;
tdbem_status tdbem_get_info(const tdbem_ctx* ctx, tdbem_info* info);

/* Kernel timing for reports.  While enabled, the library records CUDA events
   on its stream around every launch of each kernel class; tdbem_profile_read
   synchronises and returns, per class, the number of launches and the summed
   device time in milliseconds since the last enable.  Classes (index):
   0 incident RHS, 1 history/near field, 2 Z0 solve, 3 P2M, 4 M2M, 5 M2L,
   6 L2L, 7 L2P, 8 M2L moment packing (the symmetry-permuted copy of the
   moments that the tensor-core M2L reads), 9 history split (direct mode, one
   right-hand side, the untiled history sum: the current history converted to
   FP32 hi/lo pairs before it), 10 history reduction (direct mode, one
   right-hand side, the tiled history sum: the per-column-block partial sums of
   a row added in a fixed order with the lag-2 entries and V; class 1 is then
   the row-tile sum of the lags >= 3, launched ahead on the side stream when
   the steps overlap).  n_classes receives the number of classes (<= 16). */
tdbem_status tdbem_profile_enable(tdbem_ctx* ctx, int32_t on);
tdbem_status tdbem_profile_read(tdbem_ctx* ctx, int64_t* launches, double* ms, int32_t* n_classes);

/* ------------------------------------------------------------------------
   Learned warm start of the Z0 solve.  Not in the paper: the paper solves
   with GMRES from the previous data (section 2.6).  Here a small network
   predicts each step's current from local data; the solve to solve_tol
   still decides the result, so the network changes the work, never the
   answer.

   Features of edge i at step alpha (TDBEM_MLP_FEATURES = 25):
     J_i^{alpha-1-k} for k = 1..4 (4 values);
     sigma_n J_{j_n}^{alpha-1-k} for its 4 RWG neighbours j_n (16 values),
       where the neighbours are the other two sides of the + triangle, then of
       the - triangle, in winding order, and sigma_n = (sign of i) x (sign of
       j_n) in the shared triangle;
     g_i = b_i / Z0_ii and sigma_n g_{j_n} (5 values), b = R^{alpha-1}.
   With s_i = RMS of the 25 values and xc_i = 4J^{a-2} - 6J^{a-3} + 4J^{a-4}
   - J^{a-5} (cubic extrapolation), the prediction is
     x0_i = xc_i + s_i y(f_i / s_i),
   y an odd perceptron F -> H -> H -> 1 with tanh and no biases (H =
   TDBEM_MLP_WIDTH).  Parameters, flattened: W1 [H][F], W2 [H][H], w3 [H].
   When the network is in use, each solve also forms xc and starts from
   whichever of x0 and xc has the smaller FP64 residual (the fallback; a
   non-finite x0 always loses). */
#define TDBEM_MLP_FEATURES 25
#define TDBEM_MLP_WIDTH 64
#define TDBEM_MLP_NPARAM (TDBEM_MLP_WIDTH * TDBEM_MLP_FEATURES + TDBEM_MLP_WIDTH * TDBEM_MLP_WIDTH + TDBEM_MLP_WIDTH)
#define TDBEM_MLP_NPARAM_OF(H) ((H) * TDBEM_MLP_FEATURES + (H) * (H) + (H))

/* Width of the network: TDBEM_MLP_WIDTH (64, the default; FP32 arithmetic on the CUDA cores) or 256.  At
   width 256 the dense layers of inference and training and the weight gradients run as products on the
   tensor cores (BF16 operands, FP32 accumulation; FP32 parameters and Adam), the parameter count being
   TDBEM_MLP_NPARAM_OF(256).  Discards the weights, Adam's moments and the use flag (set the weights
   again); recorded samples are kept. */
tdbem_status tdbem_mlp_set_width(tdbem_ctx* ctx, int32_t width);

/* Set (host array of TDBEM_MLP_NPARAM_OF(width) floats, copied) or read the network's
   parameters.  The first set allocates the network; Adam's moments are reset. */
tdbem_status tdbem_mlp_set_weights(tdbem_ctx* ctx, const float* theta);
tdbem_status tdbem_mlp_get_weights(tdbem_ctx* ctx, float* theta);

/* Training samples.  With capacity > 0 every later step appends, for every
   edge and right-hand side, its scaled features f/s, target
   t = (J^{alpha-1} - xc)/s (edges with s = 0 are stored as zeros) and weight
   w = s^2 / (mean over that step's samples of s^2 t^2) to a device buffer
   of `capacity` samples, until it is full; capacity = 0 stops recording and
   frees the buffer.  A step's mean of w (y - t)^2 is the squared error of
   the network's guess divided by that of the plain extrapolation (1 for
   y = 0; steps whose extrapolation is exact get zero weight).
   tdbem_mlp_samples reads back samples [first, first+n) (X [n][F], T [n],
   W [n], host; any may be NULL) and the number stored so far (count may be
   NULL). */
tdbem_status tdbem_mlp_record(tdbem_ctx* ctx, int64_t capacity);
/* Record only the steps alpha with alpha % every == 0 (default 1: every step), so that a buffer of a
   given capacity spans more trajectories. */
tdbem_status tdbem_mlp_record_every(tdbem_ctx* ctx, int32_t every);
tdbem_status tdbem_mlp_samples(tdbem_ctx* ctx, int64_t first, int64_t n, float* X, float* T, float* W,
                               int64_t* count);

/* Train on the recorded samples (weighted loss) with Adam (beta1 0.9, beta2 0.999, eps 1e-8,
   step size lr) for `epochs` passes in minibatches of `batch` samples (a
   multiple of 128), visiting samples in an order shuffled per epoch from
   `seed`.  Forward, backward and update run in the library's kernels.
   loss ([epochs], may be NULL) receives each epoch's mean minibatch loss. */
tdbem_status tdbem_mlp_train(tdbem_ctx* ctx, int32_t epochs, int32_t batch, float lr, uint64_t seed, float* loss);

/* Loss (1/n) sum w (y - t)^2 and its gradient for the current parameters
   on a caller batch (X [n][F], T [n], W [n] or NULL for unit weights, host),
   computed by the training kernels (for gradient checks). */
tdbem_status tdbem_mlp_grad(tdbem_ctx* ctx, const float* X, const float* T, const float* W, int64_t n, float* loss,
                            float* grad);

/* Network output y for the rows of X ([n][F], host) by the inference kernel. */
tdbem_status tdbem_mlp_forward(tdbem_ctx* ctx, const float* X, int64_t n, float* Y);

/* Use the network as the warm start of every later solve (on != 0), or the
   cubic extrapolation alone (on = 0).  Needs weights.  used / fallback (may
   be NULL) receive how many solves (per right-hand side) since the last
   reset started from the network's and from the extrapolation's guess. */
tdbem_status tdbem_mlp_use(tdbem_ctx* ctx, int32_t on);
tdbem_status tdbem_mlp_stats(tdbem_ctx* ctx, int64_t* used, int64_t* fallback);

const char* tdbem_last_error(const tdbem_ctx* ctx);

void tdbem_destroy(tdbem_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TDBEM_H */
