/*
 * rt.h — C ABI of the GB300 (sm_103a) library for one time step of the
 * spatially truncated density matrix in a non-orthogonal, atom-blocked basis
 * (O'Rourke & Bowler, "Linear scaling density matrix real time TDDFT:
 * propagator unitarity & matrix truncation", arXiv:1404.5776).
 *
 * The method (paper Sec. II.A-II.B, Sec. IV, Sec. V.A):
 *   rho(r,r') = sum phi_ia(r) K_ia,jb phi_jb(r')            (density matrix K)
 *   S_ab = <phi_a|phi_b>                                     (overlap)
 *   i dK/dt = S^-1 H K - K H S^-1,  K(t) = U K(t0) U^dagger  (Liouville equation)
 *   U_EM(t+dt,t) = exp(-i S^-1 H(t+dt/2) dt)                 (eq. EM, Taylor, 6 terms)
 *   S^-1 by Hotelling's iteration X <- X(2I - S X) at t = 0  (Sec. V.A)
 *   H(t) = H0 - E_j(t) D_j,  D_j = <phi|r_j|phi>             (Sec. II.B, dv = -E r)
 *   charge Tr(K S), dipole Tr(K D_j)                          (Sec. IV, Sec. II.B)
 *   every matrix cut to a spatial radius                      (Sec. II.A)
 * An added propagator mode uses the Crank-Nicolson form
 *   U = (S + i dt/2 H)^-1 (S - i dt/2 H)
 * with the inverse by Hotelling's iteration warm-started from the previous step.
 * The paper's other two propagators (Sec. II.A) are available as well:
 *   U_ETRS = exp(-i dt/2 T(t+dt)) exp(-i dt/2 T(t)),  T = S^-1 H
 *   U_M4   = exp(-i dt/2 [T(t1) + T(t2)] - sqrt(3) dt^2/12 [T(t2), T(t1)]),
 *            t_{2,1} = t + (1/2 +- sqrt(3)/6) dt
 * every exponential by the same truncated Taylor series.
 *
 * Conventions of every entry point:
 *   - Pointers named h_* or documented "host" are host memory; the library
 *     copies from them before returning and keeps no reference.
 *   - Atom positions, cell lengths and radii are in Angstrom; matrix values,
 *     energies, time and field in atomic units.
 *   - Block-CSR: rowptr[n_atoms+1], col[nnzb] ascending within each row, values
 *     as consecutive row-major b_i x b_j blocks in row order (b_i = bsize[i]).
 *     Complex values are interleaved (re, im) doubles.
 *   - A block (i,j) of a pattern with radius r exists iff the minimum-image
 *     distance of atoms i and j is strictly below r, evaluated in FP64 as
 *       dx = x_j - x_i; dx -= L*rint(dx/L); d2 = (dx*dx + dy*dy) + dz*dz; d2 < r*r
 *     with every operation separately rounded.
 *   - All GPU work is enqueued on the stream given to rt_create.  Functions
 *     that return data to the host synchronise that stream.
 *   - Every call returns an rt_status; rt_last_error(ctx) gives the reason of the
 *     last failure.  After RT_ECUDA, RT_ETIMEOUT or RT_EINTERNAL the context is
 *     poisoned: every later call except rt_last_error, rt_set_state and
 *     rt_destroy returns RT_ESTATE; rt_set_state (a checkpoint of this context)
 *     clears the poisoned state and the device error word.
 *   - Device memory comes from the allocator passed to rt_create (cudaMalloc
 *     when it is NULL) and is owned by the context until rt_destroy.
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RT_API __attribute__((visibility("default")))
#else
#define RT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_ctx rt_ctx;

typedef enum {
  RT_OK = 0,
  RT_EINVAL = 1,     /* invalid argument (message says which)             */
  RT_ENOMEM = 2,     /* device allocation failed                         */
  RT_ECUDA = 3,      /* CUDA runtime error (poisons the context)         */
  RT_ENOTCONV = 4,   /* Hotelling iteration diverged or hit max_iter     */
  RT_ENUMERIC = 5,   /* NaN/Inf in an observable                         */
  RT_ETIMEOUT = 6,   /* a bounded device wait gave up (poisons)          */
  RT_EINTERNAL = 7,  /* internal consistency check failed (poisons)      */
  RT_ESTATE = 8      /* call not valid in the context's current state    */
} rt_status;

enum { RT_PROP_EM = 0, RT_PROP_CN = 1, RT_PROP_ETRS = 2, RT_PROP_M4 = 3 };
enum { RT_FP64 = 0, RT_FP32 = 1 };
enum { RT_FIELD_NONE = 0, RT_FIELD_GAUSSIAN = 1, RT_FIELD_CONSTANT = 2 };

/* matrices readable with rt_get_matrix */
enum {
  RT_MAT_S = 0, RT_MAT_H0 = 1, RT_MAT_DX = 2, RT_MAT_DY = 3, RT_MAT_DZ = 4,
  RT_MAT_SINV = 5, /* Hotelling S^-1 on P_Sinv                             */
  RT_MAT_T = 6,    /* last T = cut(S^-1 H) on P_T formed by a step: EM at
                      t+dt/2, ETRS at t+dt, M4 at t1 (not formed per step by
                      the field polynomial)                                */
  RT_MAT_U = 7,    /* last propagator on P_U (the FP32 EM, ETRS and M4 modes
                      hold U - I in FP32; it is returned as I + (U - I))   */
  RT_MAT_K = 8,    /* density matrix of (sys, kick) on P_K                 */
  RT_MAT_X = 9     /* CN warm-start inverse (S + i dt/2 H)^-1 on P_U       */
};
/* patterns readable with rt_get_pattern */
enum {
  RT_PAT_S = 0, RT_PAT_H = 1, RT_PAT_SINV = 2, RT_PAT_T = 3, RT_PAT_U = 4,
  RT_PAT_K = 5, RT_PAT_M = 6, RT_PAT_A = 7, RT_PAT_W = 8
};
/* observables per step, per (system, kick): RT_NOBS doubles */
enum {
  RT_OBS_T = 0,          /* time at the end of the step (a.u.)            */
  RT_OBS_TRKS_RE = 1, RT_OBS_TRKS_IM = 2,
  RT_OBS_TRKDX_RE = 3, RT_OBS_TRKDX_IM = 4,
  RT_OBS_TRKDY_RE = 5, RT_OBS_TRKDY_IM = 6,
  RT_OBS_TRKDZ_RE = 7, RT_OBS_TRKDZ_IM = 8,
  RT_OBS_HERM = 9,       /* max |K_ii - K_ii^dagger| before symmetrising   */
  RT_OBS_HOT_ITERS = 10, /* CN Hotelling iterations this step              */
  RT_OBS_HOT_RESID = 11, /* ||I - A X||_F / sqrt(n) of the last iteration  */
  RT_NOBS = 12
};

/* Device allocator hook: return `bytes` of device memory usable on `stream`, or
 * NULL on failure.  The free hook gets the same pointer back. */
typedef void* (*rt_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*rt_free_fn)(void* ptr, void* stream, void* user);

/* One system (host arrays, copied by rt_create). */
typedef struct {
  int32_t n_atoms;
  const double* pos;        /* [n_atoms*3] Angstrom, wrapped into [0, cell)      */
  const double* cell;       /* [3] orthorhombic cell lengths, NULL = open system  */
  const int32_t* bsize;     /* [n_atoms] functions per atom, 1..13               */
  double r_S, r_H;          /* radii of the given S and H/D patterns             */
  const int32_t* s_rowptr;  /* S on P_{r_S} (symmetric, values real)             */
  const int32_t* s_col;
  const double* s_val;
  const int32_t* h_rowptr;  /* H0 and D_x,y,z on P_{r_H}                          */
  const int32_t* h_col;
  const double* h_val;
  const double* d_val[3];
} rt_system;

typedef struct {
  double r_Sinv, r_T, r_U, r_K, r_M; /* truncation radii (Angstrom)                 */
  double dt;                /* time step (a.u.)                                   */
  int32_t prop;             /* RT_PROP_EM (paper, default), RT_PROP_CN, RT_PROP_ETRS
                               or RT_PROP_M4 (both Sec. II.A); ETRS and M4 build
                               U in FP64 in either precision                      */
  int32_t taylor_terms;     /* terms of every exponential series in total (EM,
                               ETRS, M4; 6 in the paper), 1..32                  */
  double hot_tol;           /* Hotelling tolerance on ||I - S X||_F / sqrt(n)     */
  int32_t hot_maxit;        /* Hotelling iteration cap for rt_inverse             */
  int32_t hot_step_iters;   /* CN: Hotelling iterations per step                  */
  int32_t precision;        /* RT_FP64 or RT_FP32 (block products in FP32, K,
                               reductions and the last CN iteration in FP64;
                               EM, ETRS and M4 build U - I in FP32 from
                               T(t) = S^-1 H0 - E(t) S^-1 D, both cut to r_T
                               and formed once in FP64)                          */
  int32_t full_step;        /* 1: rebuild U for every step; 0: reuse U            */
  int32_t n_kick;           /* density matrices per system sharing U (1..3)       */
  int32_t kick_terms;       /* Taylor terms of the kick exponential               */
  int32_t obs_capacity;     /* steps kept in the observables buffer               */
  int32_t use_graph;        /* capture the step in a CUDA graph and replay it     */
  int32_t incremental;      /* reference split (RT_FP32, systems of block size 4 or 13):
                               K = K_ref + dK, K_ref = K at the first step after
                               K changed (or, with full_step = 0, U changed).  The
                               part of the step acting on K_ref,
                               R = sym(cut(cut(U K_ref) U^dagger)) - K_ref, is
                               FP64: once for a constant U (full_step = 0, U
                               built in FP64 by rt_propagator, any propagator),
                               or, with full_step = 1 and the EM field
                               polynomial (field_poly = 1), per step as
                               R(E) = sum_p E^p B_p at E = E(t + dt/2), the
                               B_p = sum_{m+m'=p} sym(cut(cut(V_m K_ref) V_m'^dagger))
                               formed in FP64 when the reference is set (every
                               cut is linear; exact for H = H0 - E D).  The FP32
                               block products act on the small dK only, with
                               U - I stochastically rounded to FP32 afresh at
                               every step (counter-based draws keyed on the step
                               and element; an unbiased rounding, so its error
                               does not accumulate as a drift).  Memory with
                               full_step = 1: (2 taylor_terms - 1) complex FP64
                               matrices on P_K per kick, taylor_terms on P_M    */
  int32_t field_poly;       /* EM only: build U(t) each step as the polynomial
                               U = sum_m E^m V_m in the field value E = E(t+dt/2).
                               H = H0 - E D and every cut being linear, the
                               truncated powers are T^n(E) = sum_m E^m Q_{n,m}
                               with Q_{1,0} = cut(S^-1 H0), Q_{1,1} = -cut(S^-1 D),
                               Q_{n,m} = cut(Q_{1,0} Q_{n-1,m}) + cut(Q_{1,1} Q_{n-1,m-1});
                               V_m = sum_n c_n Q_{n,m} (+ I in V_0) are formed in
                               FP64 once by rt_inverse (and again when the field
                               axis changes).  The same U as the literal series up
                               to rounding, in FP64 in either precision; holds
                               (taylor_terms + 1) complex FP64 matrices on P_U and
                               twice that many real ones while they are formed  */
  int32_t hot_fp64_iters;   /* CN with RT_FP32: how many of the hot_step_iters
                               iterations of each step (the last ones, with the
                               reported residual) run in FP64; the earlier ones
                               run as FP32 block products (Hotelling converges
                               quadratically: an FP64 iteration squares the FP32
                               error away).  1..hot_step_iters; default 1       */
  int32_t tensor_cores;     /* with RT_FP32, 1: the sandwich's complex products of
                               13-function blocks (M = dU K, K' = W dU^dagger)
                               run on the tensor cores (tcgen05, TF32 parts and
                               FP32 remainders of both operands, three MMAs per
                               K step, the partial sum of every k added in FP32
                               registers).  Agrees with the CUDA cores to FP32
                               level per step, but the tensor cores' own
                               accumulation is coarser than round-to-nearest
                               FP32 and its error adds up coherently over long
                               runs; 0 (default): FP32 CUDA cores              */
  int32_t packed_fma;       /* reference split (incremental = 1) on the CUDA
                               cores with 13-function blocks: 1 (default) keeps
                               U - I and W = dK + M column-planar and runs the
                               complex products with packed two-lane FMAs
                               (fma.rn.f32x2, rows in pairs; measured 8 %
                               faster); 0: the row-layout kernel with scalar
                               FMAs.  Same sums, in a different order          */
} rt_params;

typedef struct {
  int32_t kind;             /* RT_FIELD_*                                         */
  int32_t dir;              /* polarisation axis 0,1,2                            */
  double E0, t0, sigma, omega; /* E(t) = E0 exp(-(t-t0)^2/(2 sigma^2)) cos(omega(t-t0)) */
} rt_field;

/* Fills the defaults: radii 8 A, dt 0.05, EM, 6 Taylor terms, tol 1e-10,
 * maxit 100, 2 CN iterations per step, FP64, full step, 1 kick, 12 kick terms,
 * 4096 observable steps, graphs on, incremental form and field polynomial off,
 * 1 FP64 CN iteration per step in the mixed mode, CUDA-core FP32 products. */
RT_API rt_status rt_default_params(rt_params* p);

/* Creates a context for n_sys systems: validates and copies the host inputs,
 * builds every pattern (S, H, S^-1, T, U, K, M, A = P_{max(r_S,r_H)},
 * W = P_{r_U+r_S}) on the device with cell lists, and the triple lists of every
 * product of the step.  Paper: spatial cut-off of Sec. II.A; atoms are
 * stationary, so patterns are built once (Sec. V.A).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * alloc/free/alloc_user: device allocator (NULL = cudaMalloc/cudaFree).
 * Errors: RT_EINVAL (inputs), RT_ENOMEM, RT_ECUDA. */
RT_API rt_status rt_create(rt_ctx** ctx, const rt_system* sys, int32_t n_sys, const rt_params* p,
                    void* cuda_stream, rt_alloc_fn alloc, rt_free_fn free_fn, void* alloc_user);

/* External field E(t) along dir (Sec. II.B: dv_ext = -E_j(t) r, so H(t) =
 * H0 - E(t) D_j; a Gaussian profile as in Sec. IV.A).  Default: none. */
RT_API rt_status rt_set_field(rt_ctx* ctx, const rt_field* f);

/* S^-1 for every system by Hotelling's iteration X <- X(2I - S X) from
 * X0 = I/||S||_inf, each product cut to r_Sinv (Sec. V.A).  Stops when the
 * residual ||I - S X||_F/sqrt(n) < hot_tol, or when it shrinks by less than a
 * factor 0.9 (truncation floor; returns RT_OK).  RT_ENOTCONV when it grows
 * above 1 or hot_maxit is reached.  iters/residual: host outputs of the
 * system `sys` (may be NULL).  Synchronises. */
RT_API rt_status rt_inverse(rt_ctx* ctx, int32_t sys, int32_t* iters, double* residual);

/* Sets K of (sys, kick) from host values on P_K (complex interleaved, true
 * block sizes; rt_pattern_size/rt_get_pattern give P_K). Resets time to 0. */
RT_API rt_status rt_set_density(rt_ctx* ctx, int32_t sys, int32_t kick, const double* h_k_re_im);

/* Ground-state K0 = f(S^-1 H0) S^-1 with the Fermi function f of chemical
 * potential mu and temperature kT, by a Chebyshev expansion of `order` on the
 * spectral interval [e_lo, e_hi] (set-up step, not part of the paper's
 * propagation; needs rt_inverse).  Products cut to r_K; result symmetrised.
 * Written to every kick slot of system `sys`. */
RT_API rt_status rt_ground_state(rt_ctx* ctx, int32_t sys, int32_t order, double mu, double kT,
                          double e_lo, double e_hi);

/* Delta kick: K <- V K V^dagger, V = exp(+i kappa S^-1 D_dir) (H = H0 -
 * kappa delta(t) D_dir, Sec. II.B), Taylor series of kick_terms terms with
 * powers cut to r_U. Needs rt_inverse. */
RT_API rt_status rt_kick(rt_ctx* ctx, int32_t sys, int32_t kick, int32_t dir, double kappa);

/* Builds U for [t, t+dt] for every system with the context's propagator
 * (EM at the midpoint, its field polynomial, ETRS, M4 or the CN form) and
 * keeps it for steps with full_step = 0 (in the reference split in FP64).
 * Synchronises. */
RT_API rt_status rt_propagator(rt_ctx* ctx, double t);

/* n time steps K <- U K U^dagger for every (system, kick), each followed by the
 * observables.  With full_step, U is rebuilt at each step's midpoint.
 * In the reference split on the CUDA cores (incremental = 1, tensor_cores = 0)
 * the two block products of the step (M and K', Sec. II.A) run as one launch
 * per product and block size over every (system, kick) pair, the pairs with
 * the most block triples first. */
RT_API rt_status rt_step(rt_ctx* ctx, int32_t n);

/* Launch-shape tuner of the grouped products of the reference split (no
 * counterpart in the paper: a property of the GPU kernels).  Stages: 0 = M of
 * the 13-function systems, 1 = their K', 2 = M of the 4-function systems,
 * 3 = their K'.  For every stage present it times each candidate shape -
 * stages per warp of the 13-function kernel (2 or 3) and a one-shot grid or a
 * persistent one (one resident wave of CTAs walking the items) - on the
 * context's own products: one warm-up launch, then `reps` (1..100) launches
 * between CUDA events, and keeps the fastest.  The densities are not changed
 * (the K' launches write into scratch copies of their outputs; the M
 * launches write only M and W, which every step forms again).  Allocates the
 * scratch through the context's allocator and synchronises.  rows: host
 * [max_rows][4] of (stage, stages per warp, persistent, chosen 0/1) and ms:
 * host [max_rows], milliseconds per launch; n_rows: rows produced (may exceed
 * max_rows; may be NULL).  RT_ESTATE when the context has no such products. */
RT_API rt_status rt_autotune(rt_ctx* ctx, int32_t reps, int32_t max_rows, int32_t* n_rows, int32_t* rows,
                             double* ms);

/* Sets (or reads) the launch shape of one stage (as in rt_autotune), e.g. a
 * shape a caller cached from an earlier tuning run: stages per warp 2 or 3
 * (3 only for stages 0 and 1), persistent 0 or 1.  Default: 2, 0. */
RT_API rt_status rt_set_launch_shape(rt_ctx* ctx, int32_t stage, int32_t stages, int32_t persistent);
RT_API rt_status rt_get_launch_shape(rt_ctx* ctx, int32_t stage, int32_t* stages, int32_t* persistent);

/* Copies the observables recorded since the previous call for (sys, kick) to
 * host `out` [max_steps][RT_NOBS] in step order; *n_out = steps copied.
 * RT_ENUMERIC if any copied value is NaN/Inf (data still copied). */
RT_API rt_status rt_observables(rt_ctx* ctx, int32_t sys, int32_t kick, double* out, int32_t max_steps,
                         int32_t* n_out);

/* Number of blocks of pattern `which` (RT_PAT_*) of system `sys`. */
RT_API rt_status rt_pattern_size(rt_ctx* ctx, int32_t sys, int32_t which, int64_t* nnzb);
/* Copies the pattern to host rowptr[n_atoms+1], col[nnzb]. */
RT_API rt_status rt_get_pattern(rt_ctx* ctx, int32_t sys, int32_t which, int32_t* rowptr, int32_t* col);
/* Number of doubles rt_get_matrix writes for `which` (2 per matrix element). */
RT_API rt_status rt_matrix_size(rt_ctx* ctx, int32_t sys, int32_t which, int64_t* n_doubles);
/* Copies matrix `which` (RT_MAT_*) of (sys, kick) to host, complex interleaved,
 * true block sizes, on its pattern. capacity = doubles available in vals. */
RT_API rt_status rt_get_matrix(rt_ctx* ctx, int32_t sys, int32_t kick, int32_t which, double* vals,
                        int64_t capacity);

/* Unitarity of the last propagator of `sys` (paper Sec. IV, eq. s_unit):
 * with metric_S = 1, E = cut_{P_U}(U^dagger cut_{P_W}(S U)) - S (the conserved
 * form in a non-orthogonal basis); with 0, E = cut_{P_U}(U^dagger U) - I (the
 * printed form).  Host outputs max|E| and mean|E| over the entries of P_U.
 * In the FP32 EM, ETRS and M4 modes the propagator is held as U - I in FP32;
 * it is promoted to U = I + (U - I) in FP64 first, so E measures the mixed
 * propagator. */
RT_API rt_status rt_unitarity(rt_ctx* ctx, int32_t sys, int32_t metric_S, double* maxabs, double* meanabs);

/* Algorithmic work of one step summed over systems and kicks:
 * flops = sum over products of triples * (8 b^3 complex, 2 b^3 real), counted
 * with the true block sizes (padding excluded); bytes = block values read
 * and written by those products once each. */
RT_API rt_status rt_step_work(rt_ctx* ctx, double* flops, double* bytes);

/* Number of kernels one step launches (the nodes of the captured step graph). */
RT_API rt_status rt_step_kernels(rt_ctx* ctx, int64_t* kernels);

/* Per-kernel-class timing: enable=1 makes later rt_step calls launch without
 * a graph and bracket each kernel with CUDA events on the context stream;
 * rt_profile_read returns, per class c < *n_classes (<= max), the launch
 * count, total milliseconds, and algorithmic flops and bytes, with a name. */
RT_API rt_status rt_profile(rt_ctx* ctx, int32_t enable);
RT_API rt_status rt_profile_read(rt_ctx* ctx, int32_t max, int32_t* n_classes, int64_t* launches,
                          double* ms, double* flops, double* bytes, char* names /* [max][32] */);

/* Checkpoint: every K, U, the CN warm start, the device step state (time,
 * field samples), the step counter and the observables cursor.  With buf
 * NULL, *bytes receives the size.  Where only U - I is current (FP32 EM, ETRS,
 * M4) the state holds U = I + (U - I).  rt_set_state restores it, forms the
 * FP32 parts of U that the mixed sandwich uses from it, and clears the
 * poisoned state and the device error word. */
RT_API rt_status rt_get_state(rt_ctx* ctx, void* buf, size_t* bytes);
RT_API rt_status rt_set_state(rt_ctx* ctx, const void* buf, size_t bytes);

/* Allocation-free traces.  The paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory when they need the
 * observables -- code running while a stream is being captured into a CUDA
 * graph (allocation is not allowed there) or a host framework that owns all
 * device memory.  It allocates nothing (no cudaMalloc, cudaFree or
 * allocating library call) and needs no context.
 *
 * Computes out[0..7] = (Re, Im) of Tr(K S), Tr(K Dx), Tr(K Dy), Tr(K Dz) for a
 * hermitian K and real symmetric S, D (the imaginary parts are then 0), from
 * the upper blocks of K, exactly as rt_observables does.  All pointers are
 * device memory owned by the caller:
 *   K       nnzb blocks of B x B complex values (interleaved re, im doubles),
 *           row-major, in pattern order; rowidx[q], col[q] = block (i,j)
 *   bsize   [n_atoms] true functions per atom (<= B; the rest is padding)
 *   S       real B x B blocks; ks_map[q] = index in S of block (j,i), or -1
 *   Dx,Dy,Dz real B x B blocks on one pattern; kd_map[q] = index of (j,i), or -1
 *   out     [8] doubles
 * n_ctas: CTAs of the partial-sum pass (0 = automatic); at most
 * RT_NOALLOC_MAX_CTAS, larger values are rejected with RT_EINVAL.
 * Scratch: a fixed device array of RT_NOALLOC_MAX_CTAS * 8 doubles (64 KiB)
 * inside the library, held by every GPU that loads it until the process
 * exits; nothing in it needs to start at zero.  All calls share it, so calls
 * that overlap on the GPU race: serialise them.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and should come
 * before any stream capture.  Work is enqueued on cuda_stream (NULL = legacy
 * default stream); the call does not synchronise.  Errors: RT_EINVAL, RT_ECUDA
 * (reason printed on stderr); a CUDA error already pending from the caller's
 * earlier work is reported as RT_ECUDA and left pending, not consumed. */
#define RT_NOALLOC_MAX_CTAS 1024
RT_API rt_status rt_traces_noalloc(const double* K, int64_t nnzb, const int32_t* rowidx, const int32_t* col,
                                   const int32_t* bsize, int32_t B, const double* S, const int32_t* ks_map,
                                   const double* Dx, const double* Dy, const double* Dz, const int32_t* kd_map,
                                   int32_t n_ctas, double* out, void* cuda_stream);

/* Waits for all work of the context's stream. */
RT_API rt_status rt_synchronize(rt_ctx* ctx);

/* Host-side fault injection for tests (no counterpart in the paper; nothing
 * is made to fault or hang on the GPU).  Flags (or-ed):
 *   RT_FAULT_HOTELLING_MAXITER1  the next rt_inverse runs with hot_maxit = 1,
 *                                so it ends with RT_ENOTCONV;
 *   RT_FAULT_NAN_IN_H            writes a NaN into the first element of H0 of
 *                                system 0 (and of the precomputed S^-1 H0 of
 *                                the FP32 EM, ETRS and M4 modes, if formed): the next step's
 *                                observables are NaN and rt_observables returns
 *                                RT_ENUMERIC.  Permanent for this context;
 *   RT_FAULT_WAIT_TIMEOUT_0      the next rt_step gives its bounded waits
 *                                (FP32 13-function kernels) a zero budget: they
 *                                give up at once, drain the copies in flight and
 *                                set the error word, and the step returns
 *                                RT_ETIMEOUT; the context is then refused
 *                                (RT_ESTATE) until rt_set_state.
 * Errors: RT_EINVAL for unknown flags. */
enum { RT_FAULT_HOTELLING_MAXITER1 = 1, RT_FAULT_NAN_IN_H = 2, RT_FAULT_WAIT_TIMEOUT_0 = 4 };
RT_API rt_status rt_debug_inject(rt_ctx* ctx, uint32_t flags);

/* Structural check of one block product's triple list against its patterns
 * (host arrays; no device work, no context): the contract every block-product
 * kernel relies on for in-bounds operand loads and race-free stores.  The
 * truncated product C = cut_{P_C}(op(A) op(B)) (Sec. II.A) is evaluated per
 * output block (i,j) of P_C as sum over k of op(A)_ik op(B)_kj; a triple list
 * names, per output item, the operand blocks of each k.
 *   Patterns: symmetric block-CSR over n_atoms atoms, rowptr[n_atoms+1] from
 *   0 and non-decreasing, col[] in range and strictly ascending in a row.
 *   Items: item_blk[n_items] lists the blocks of P_C (with upper_only, the
 *   blocks with col >= row) in increasing order, one item each, so every
 *   output block has exactly one writer and an upper-only product never has
 *   a mirrored (lower) block as an item.
 *   ptr[n_items+1]: ptr[0] = 0, non-decreasing, ptr[n_items] = n_triples.
 *   ab[n_triples][2]: for the item's block (i,j), a indexes the stored block
 *   (i,k) of A ((k,i) when a_dag), b the stored block (k,j) of B ((j,k) when
 *   b_dag), both within their pattern; k strictly ascending within an item;
 *   complete: one triple for every k with (i,k) in P_A and (k,j) in P_B.
 * Returns RT_OK, RT_EINTERNAL if a condition fails (*bad_item, if not NULL,
 * receives the first failing item, or -1 when the failure is not tied to an
 * item), or RT_EINVAL for NULL arrays or negative counts. */
RT_API rt_status rt_check_triples(int32_t n_atoms, const int32_t* a_rowptr, const int32_t* a_col, int32_t a_dag,
                                  const int32_t* b_rowptr, const int32_t* b_col, int32_t b_dag,
                                  const int32_t* c_rowptr, const int32_t* c_col, int32_t upper_only,
                                  int64_t n_items, const int32_t* item_blk, const int64_t* ptr, const int32_t* ab,
                                  int64_t n_triples, int64_t* bad_item);

/* Debug check of a live context: copies every pattern and every triple list
 * that the context has built (all systems) back to the host and applies the
 * checks of rt_check_triples to each.  Synchronises the context stream.
 * *n_checked (may be NULL) receives the number of triple lists checked.  A
 * failing list returns RT_EINTERNAL (the product is named in rt_last_error)
 * and, like every internal error, leaves the context refused until
 * rt_set_state. */
RT_API rt_status rt_debug_check(rt_ctx* ctx, int64_t* n_checked);

/* Reason of the last failure (never NULL; "" after success). */
RT_API const char* rt_last_error(rt_ctx* ctx);

RT_API void rt_destroy(rt_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RT_H */
