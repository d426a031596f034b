/*
 * dafmm.h -- C-ABI of the GB300 (sm_103a) library for the Directional
 * Algebraic FMM (DAFMM) matrix-vector product of Gujjula & Ambikasaran,
 * arXiv 2204.00326, applied to the discretised Lippmann-Schwinger equation.
 *
 * The operator.  On a uniform quadtree over [x0,x1]^2 with p x p first-kind
 * Chebyshev nodes per leaf (Section 2, Eq. 7-9), the unknowns are psi at the
 * N = n_side^2 nodes and the discrete system is A psi = f (Eq. 12a) with
 *     A = I + kappa^2 diag(q) K,
 *     K_ij = int_{B(j)} G(x_i, y) L_{j'}(y) dy,  G = (i/4) H0^(1)(kappa|x-y|),
 * L_{j'} the least-squares cardinal function of leaf B(j) (Eq. 11, Eq. 13).
 * dafmm_matvec applies the NCA-compressed K (Section 4-5) and the diagonal
 * epilogue.
 *
 * Conventions for every call:
 *   - Return value: DAFMM_OK (0) or one of the DAFMM_E* codes below; the text
 *     of the last error on the calling thread is available from
 *     dafmm_last_error().  No call aborts the process.
 *   - Handles (dafmm_tree, dafmm_ops) are opaque, owned by the library and
 *     released with tree_destroy / ops_destroy.  An ops handle keeps a
 *     reference to its tree: destroy the ops before the tree.
 *   - Arrays named *_dev are device pointers in the current CUDA device's
 *     memory, owned by the caller; *_host are host pointers.  Complex vectors
 *     are interleaved (re, im) doubles.  Vectors with several right-hand sides
 *     are stored [N][nrhs] (right-hand side fastest).
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream enqueue their kernels on it and do
 *     not synchronise the device unless stated.
 *   - Unknowns are ordered leaf by leaf in Morton (Z) order of the leaves
 *     (x bit below y bit); inside a leaf, node i' = k1 + p*k2 sits at
 *     alpha + beta (zeta_k1, zeta_k2), zeta_k = -cos((2k+1) pi / (2p)).
 *   - There is no CPU fallback: without a CUDA device every call that needs
 *     one returns DAFMM_ECUDA.
 */
#ifndef DAFMM_H
#define DAFMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define DAFMM_OK 0
#define DAFMM_EBADARG 1     /* invalid argument or unsupported configuration */
#define DAFMM_ENOMEM 2      /* host or device allocation failed */
#define DAFMM_ENOTCONV 3    /* iterative solver stopped before the tolerance */
#define DAFMM_EBREAKDOWN 4  /* numerical breakdown (singular pivot block, ...) */
#define DAFMM_ETIMEOUT 5    /* a bounded device-side wait gave up */
#define DAFMM_ECUDA 6       /* CUDA runtime error or no device */

/* Arithmetic of an operator application. */
#define DAFMM_FP64 0        /* complex128 operators and vectors, computed in
                               double-float (float pairs, unit roundoff 2^-48:
                               FP64 issues at 1/64 of the FP32 rate on GB300)
                               with results rounded to double; the epilogue
                               v + kappa^2 q (K v) is FP64 */
#define DAFMM_MIXED 1       /* complex64 operators and coefficients, FP32 math;
                               boundary vectors stay complex128 */

/* Parameters of the discretisation and of the compression (Section 3-4). */
typedef struct dafmm_params {
    int p;            /* Chebyshev nodes per leaf side; the library supports p = 4 */
    double kappa;     /* wavenumber kappa > 0 (Eq. 1) */
    double T;         /* a box of half-width w is high-frequency iff (kappa w)^2 > T
                         (Section 3; the paper leaves T open, 16 is the default) */
    double eps_nca;   /* tolerance of the partially pivoted ACA that picks the
                         NCA pivots (Section 4.2.2, Rjasanow's stopping rule) */
    int max_rank;     /* cap on every NCA rank; 0 = no cap */
    int kernel;       /* the matrix K the DAFMM compresses: DAFMM_KERNEL_LS (0) or
                         DAFMM_KERNEL_POINTS (1), see below */
    int reserved[6];  /* must be zero */
} dafmm_params;

/*
 * Kernels.  DAFMM_KERNEL_LS: K_ij = int_{B(j)} G(x_i, y) L_{j'}(y) dy, the
 * discretised volume integral of Eq. 13 (the Lippmann-Schwinger operator).
 * DAFMM_KERNEL_POINTS: K_ij = G(x_i, x_j) for j != i and K_ii = 0, the point
 * N-body operator of Experiment 1 (Section 6.2) with charges at the same
 * Chebyshev nodes; dafmm_potential then returns u = K v, and
 * dafmm_nbody_direct gives the same sum by direct summation.
 */
#define DAFMM_KERNEL_LS 0
#define DAFMM_KERNEL_POINTS 1

/* Shape of a built tree (filled by tree_info). */
typedef struct dafmm_tree_info {
    long N;           /* number of unknowns n_side^2 */
    int n_side;       /* nodes per side */
    int levels;       /* L + 1: levels 0 (root) .. L (leaves) */
    int top;          /* coarsest level with a non-empty interaction list
                         (levels > L when there is no far field) */
    int hf[32];       /* per level: 1 if high-frequency (Section 3.2) */
    int cones[32];    /* per level: number of cones (1 for low frequency) */
    long il_pairs[32];/* per level: number of interaction-list pairs */
} dafmm_tree_info;

/* Realised sizes of a built operator (filled by dafmm_stats). */
typedef struct dafmm_stats_t {
    int rank_in_max[32];    /* per level: largest incoming rank */
    int rank_out_max[32];   /* per level: largest outgoing rank */
    double rank_in_mean[32];
    double rank_out_mean[32];
    long slots[32];         /* per level: active (box, cone) pairs */
    double operator_bytes_fp64;   /* stored operators, complex128 */
    double operator_bytes_fp32;   /* stored operators, complex64 */
    double vector_bytes_per_rhs;  /* algorithmic vector/coefficient traffic of
                                     one application, complex128, per RHS */
    double cmacs_per_rhs;         /* complex multiply-adds of one application */
    double setup_seconds_table;   /* entry-table kernel */
    double setup_seconds_nca;     /* pivots and operators */
    long p2p_cmacs_per_rhs;       /* part of cmacs_per_rhs spent in the near field */
    double cmacs_up;              /* per RHS: P2M, M2M, directional M2M */
    double cmacs_m2l;             /* per RHS: M2L, directional M2L */
    double cmacs_down;            /* per RHS: directional L2L, L2L (not L2P) */
    double cmacs_leaf;            /* per RHS: L2P + near field */
    double coef_bytes_per_rhs;    /* multipole/local coefficients written and
                                     read once each, complex128 */
    int launches_per_call;        /* kernels one dafmm_matvec launches (mixed) */
    int launches_per_call_fp64;   /* ... in FP64 */
    double cmacs_far_fused;       /* per application with one RHS: complex multiply-adds of the
                                     far-field kernel (its level L-1 up pass reads the leaf values
                                     through the P2M; the last L2L is left to the leaf kernel) */
    double cmacs_leaf_fused;      /* ... of the leaf kernel: near field, L2P, L2L composed with L2P */
} dafmm_stats_t;

/*
 * Device time of the passes of the profiled dafmm_matvec calls (ms, summed).
 * A single-right-hand-side call runs every tree pass (P2M, M2M, M2L, L2L) in
 * one kernel: it adds to ms_far only.  A call with several right-hand sides
 * launches the passes separately: it adds to ms_up, ms_m2l and ms_down, and
 * their sum to ms_far.
 */
typedef struct dafmm_profile_t {
    long calls;
    double ms_total;  /* first to last kernel of each call */
    double ms_up;     /* P2M + M2M (+ the complex64 conversion in mixed mode) */
    double ms_m2l;    /* M2L at every level */
    double ms_down;   /* L2L into the leaves' locals */
    double ms_leaf;   /* L2P + near field + epilogue */
    double ms_far;    /* every tree pass: P2M, M2M, M2L, L2L */
} dafmm_profile_t;

typedef struct dafmm_tree dafmm_tree;
typedef struct dafmm_ops dafmm_ops;
typedef struct dafmm_hodlr dafmm_hodlr;

/* Options of gmres_solve. */
typedef struct gmres_opts {
    int restart;        /* Krylov dimension m of one cycle (1..128); 50 is typical */
    int max_iters;      /* cap on inner iterations over all cycles */
    double tol;         /* stop when |f - A x| / |f| <= tol (FP64 residual, Section 6) */
    int precision;      /* DAFMM_FP64, or DAFMM_MIXED: inner cycles use complex64
                           operators and each outer step refines in FP64 */
    double inner_tol;   /* mixed precision: relative tolerance of one correction
                           solve (1e-5 is typical) */
    double* history;    /* optional host array: relative residuals (true residual at
                           each restart, least-squares estimate in between) */
    int history_len;    /* its length */
    int side;           /* side of the preconditioner M: DAFMM_PREC_RIGHT (0,
                           default; GMRES minimises the residual the stopping
                           rule measures) or DAFMM_PREC_LEFT (1; the paper's
                           M^{-1} A x = M^{-1} f, Eq. hybrid, with the same
                           FP64 true-residual stopping rule at every restart) */
    int reserved[5];    /* must be zero */
} gmres_opts;

#define DAFMM_PREC_RIGHT 0
#define DAFMM_PREC_LEFT 1

/* What gmres_solve did. */
typedef struct gmres_stats {
    int iterations;        /* inner iterations (one operator application each) */
    int outer_iterations;  /* true-residual checks after the first */
    int matvecs;           /* dafmm_matvec calls, including the FP64 residuals */
    int precond_applies;   /* hodlr_solve calls */
    int converged;         /* 1 if the tolerance was met */
    double rel_residual;   /* final |f - A x| / |f|, FP64 */
    double seconds;        /* wall time of the call (it synchronises the stream) */
} gmres_stats;

/* Copy the message of the last failed call on this thread into buf (always
 * NUL-terminated when size > 0).  Returns the status code of that call. */
int dafmm_last_error(char* buf, size_t size);

/*
 * build_tree -- uniform quadtree on [x0,x1]^2 with n_side nodes per side
 * (n_side = p * 2^L), its high/low-frequency regimes (Section 3), cones
 * (Section 3.2.1, angle 2 pi / 2^ceil(log2(2 pi kappa w)) at the finest
 * high-frequency level, doubling per level up), neighbour and interaction
 * lists (Table 1).  Host work only; no device memory is used.
 * Errors: DAFMM_EBADARG for p != 4, n_side not p times a power of two,
 * x1 <= x0, kappa <= 0, eps_nca outside (0, 1), or leaves in the
 * high-frequency regime.
 */
int build_tree(const dafmm_params* params, int n_side, double x0, double x1, dafmm_tree** out);

/* Coordinates of the N unknowns (xy_host: N x 2 doubles, caller-owned). */
int tree_nodes(const dafmm_tree* tree, double* xy_host);

/* The same coordinates into device memory (xy_dev: N x 2 doubles,
 * caller-owned), copied on stream; synchronises the stream.  Errors:
 * DAFMM_EBADARG for NULL arguments, DAFMM_ECUDA. */
int tree_nodes_dev(const dafmm_tree* tree, double* xy_dev, void* stream);

/* Shape of the tree (see dafmm_tree_info). */
int tree_info(const dafmm_tree* tree, dafmm_tree_info* info);

/*
 * tree_check -- self-check of the lists (host only).  Counts, into *bad, the
 * ordered leaf pairs that are not covered exactly once by the near field
 * (same-level neighbours at the leaves) plus the interaction lists of their
 * ancestors (Section 5: every interaction is either near or transferred at
 * exactly one level), and the directional list entries whose mirror entry
 * is missing (Table 1: B lies in the cone of A that points back at B).
 * Cost O(nleaf^2 L): meant for small trees.
 */
int tree_check(const dafmm_tree* tree, long* bad);

/* Release a tree.  NULL is accepted. */
int tree_destroy(dafmm_tree* tree);

/*
 * build_nca_operators -- setup of the DAFMM operator for the contrast q.
 *   1. On the device, tabulates K for every leaf offset of the uniform grid
 *      (the near-field singular integrals and the far-field Gauss-Legendre
 *      integrals of Section 2.3 are translation invariant per level).
 *   2. Traverses the tree upwards and picks the nested pivots by partially
 *      pivoted ACA (Section 4.2.2), forming the P2M/M2M, L2L/L2P (Section
 *      4.2.1, all four cases) and M2L operators (Section 5 step 4).  K, not
 *      A, is compressed; kappa^2 q enters in the epilogue (Eq. 13).
 *   3. Uploads complex128 and complex64 copies of every operator.
 * q_dev: N doubles on the device (copied; the caller may free it after the
 * call returns).  The call synchronises the stream.
 * Errors: DAFMM_EBADARG, DAFMM_ENOMEM, DAFMM_EBREAKDOWN (a singular pivot
 * block), DAFMM_ECUDA.
 */
int build_nca_operators(dafmm_tree* tree, const double* q_dev, void* stream, dafmm_ops** out);

/*
 * dafmm_matvec -- out = A v = v + kappa^2 q .* (K~ v) for nrhs right-hand
 * sides, K~ the DAFMM approximation of K: upward pass (P2M, M2M, directional
 * M2M), transverse pass (M2L, directional M2L), downward pass (directional
 * L2L, L2L, L2P) and near field (Section 5 steps 3-6).
 * v_dev, out_dev: N x nrhs complex128 (interleaved) on the device; they must
 * not overlap.  precision: DAFMM_FP64 or DAFMM_MIXED.  Asynchronous on stream.
 * Calls on one ops handle must not overlap in time (they share its scratch).
 * Errors: DAFMM_EBADARG (nrhs < 1, NULL pointers, unknown precision),
 * DAFMM_ENOMEM (growing scratch for a larger nrhs), DAFMM_ECUDA.
 */
int dafmm_matvec(const dafmm_ops* ops, int nrhs, const double* v_dev, double* out_dev, int precision, void* stream);

/*
 * dafmm_potential -- out = K~ v: the volume potential V[v] of Eq. 5 at the N
 * nodes, discretised as in Eq. 13 and applied by the same DAFMM passes (the
 * scattered field u_scat = V[psi] from the solution psi, as the paper
 * evaluates it on the grid).  No identity and no kappa^2 q.  Arguments,
 * layouts and errors as dafmm_matvec; launched directly (no graph replay).
 */
int dafmm_potential(const dafmm_ops* ops, int nrhs, const double* v_dev, double* out_dev, int precision, void* stream);

/*
 * gmres_solve -- solve A psi = f (Eq. 12a) with restarted flexible GMRES
 * (Saad), right-preconditioned by the HODLR approximation M when M != NULL
 * (the Hybrid solver, Eq. hybrid; right rather than left preconditioning so
 * that GMRES minimises the unpreconditioned residual the paper's stopping
 * rule measures).  Every outer step forms the true residual f - A x with the
 * FP64 DAFMM; inner cycles apply A (and M) in opts->precision.  The
 * Hessenberg matrix, Givens rotations, preconditioned basis and x are FP64
 * on the device; the Arnoldi basis is complex128 in FP64 cycles and
 * complex64 in the inner cycles of DAFMM_MIXED.  A zero initial guess takes
 * r = f without an application.  f_dev: N x nrhs complex128 (not modified);
 * x_dev: N x nrhs complex128, in: initial guess, out: solution (both
 * [N][nrhs], right-hand side fastest).  nrhs in 1..64: several right-hand
 * sides are solved together by nrhs independent GMRES processes in lockstep,
 * each step applying A (and M) to all columns in one batched application;
 * every column has its own Hessenberg matrix, rotations, inner tolerance and
 * FP64 true-residual stopping rule (a column that has converged stops
 * contributing; its later basis vectors are zero).  st: nrhs entries, one
 * per column (matvecs and precond_applies count batched applications,
 * iterations the steps that column used).  With several right-hand sides,
 * opts->history receives the largest relative residual over the columns.
 * Its Krylov workspace is kept on the ops handle between calls (grown when
 * N, nrhs or m grows); calls on one handle must be ordered.  Synchronises
 * the stream.
 * Returns DAFMM_OK when every column converged, DAFMM_ENOTCONV when
 * max_iters was reached (x holds the last iterates, st the residuals),
 * DAFMM_EBADARG (nrhs outside 1..64, ...), DAFMM_ENOMEM, DAFMM_ECUDA.
 */
int gmres_solve(dafmm_ops* ops, const dafmm_hodlr* M, int nrhs, const double* f_dev, double* x_dev, const gmres_opts* opts, gmres_stats* st,
                void* stream);

/*
 * hodlr_factor -- HODLR approximation A~ of A (Ambikasaran & Darve; the
 * preconditioner of the paper's Hybrid solver, Section 6 and Eq. hybrid).
 * The Morton-ordered index set is halved recursively down to leaves of
 * leaf_size unknowns (a power of two, 32..1024; 64 is typical); at every node
 * the two off-diagonal blocks of A are compressed by partially pivoted ACA,
 * to the fixed rank `rank` (rank > 0, the paper's preconditioner with r = 5,
 * 15, 25) or to relative accuracy tol (rank = 0).  The factorisation
 * (recursive Sherman-Morrison-Woodbury, FP64 on the host; leaf blocks
 * inverted by Gauss-Jordan with partial pivoting) is uploaded in complex128
 * and complex64.  Uses the entries tabulated by build_nca_operators, so the
 * ops handle must outlive nothing here: A~ is self-contained once built.
 * Synchronous.  Errors: DAFMM_EBADARG, DAFMM_ENOMEM, DAFMM_EBREAKDOWN
 * (singular leaf block or Woodbury system), DAFMM_ECUDA.
 */
int hodlr_factor(const dafmm_ops* ops, int rank, double tol, int leaf_size, dafmm_hodlr** out);

/*
 * hodlr_solve -- x = A~^{-1} b for nrhs right-hand sides (1..64): leaf
 * inverses, then per level from the leaves up t = W x, s = S^{-1} t,
 * x -= Ut s (recursive Sherman-Morrison-Woodbury, Section 6).  Cost
 * O(r N log N) per right-hand side.  One right-hand side: one cooperative
 * launch whose CTAs meet at a grid barrier per level; each barrier wait has
 * a limit (about 0.2 s), after which the launch sets the handle's error flag
 * and returns (see hodlr_sync).  Several: ordinary launches per level (no
 * device waits), the factors read once for all columns; ranks up to 256.
 * b_dev, x_dev: N x nrhs complex128 on the device, [N][nrhs] (right-hand side
 * fastest); x_dev == b_dev is allowed.
 * precision: DAFMM_FP64 (factors as float pairs, double-float arithmetic,
 * result rounded to double), or DAFMM_MIXED (complex64 factors and
 * arithmetic); boundary vectors are complex128.  Asynchronous on stream.  Calls on one
 * handle must be ordered (one stream): they share work buffers.
 */
int hodlr_solve(const dafmm_hodlr* M, int nrhs, const double* b_dev, double* x_dev, int precision, void* stream);

/*
 * hodlr_sync -- synchronise the stream, then report whether an application
 * on this handle gave up a barrier wait since the last check
 * (DAFMM_ETIMEOUT; the flag is cleared and the barrier re-armed; the result
 * of that application is undefined).  gmres_solve checks this itself.
 * Errors: DAFMM_EBADARG for NULL, DAFMM_ECUDA.
 */
int hodlr_sync(const dafmm_hodlr* M, void* stream);

/*
 * hodlr_set_ctas -- width of the hodlr_solve launch (CTAs; each owns N / ctas
 * consecutive unknowns).  0 restores the width chosen at factorisation (a
 * power of two, all CTAs resident at once, at most one per leaf, about 256
 * unknowns per CTA on large problems and at least 128 CTAs).  Otherwise ctas
 * must be a power of two, at most N / leaf_size and at most the number of
 * CTAs the device holds at once.  A tuning and test knob; the result does
 * not depend on it beyond rounding.  Errors: DAFMM_EBADARG.
 */
int hodlr_set_ctas(dafmm_hodlr* M, int ctas);

/*
 * hodlr_debug_stall -- test support for the timeout path (the paper has no
 * counterpart): the next hodlr_solve on this handle waits at its first grid
 * barrier for one CTA more than the launch has, so every wait gives up and
 * hodlr_sync returns DAFMM_ETIMEOUT.  Errors: DAFMM_EBADARG for NULL.
 */
int hodlr_debug_stall(const dafmm_hodlr* M);

/*
 * hodlr_export -- the dense N x N matrix A~ assembled from the factors
 * (dense leaf blocks plus U V products off the diagonal), row-major complex
 * interleaved, into dense_host (caller-owned, 16 N^2 bytes).  For checking
 * hodlr_solve against a dense solve; meant for small N.
 */
int hodlr_export(const dafmm_hodlr* M, double* dense_host);

/* Shape of a HODLR factorisation. */
int hodlr_info(const dafmm_hodlr* M, long* N, int* levels, int* leaf_size, int* rank_max, double* factor_seconds);

/* Release a HODLR factorisation.  NULL is accepted. */
int hodlr_destroy(dafmm_hodlr* M);

/* Size of the static device scratch used by dafmm_matvec_noalloc. */
#define DAFMM_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * dafmm_matvec_noalloc -- the same application as dafmm_matvec for one
 * right-hand side (out = A v), for callers that cannot have memory allocated
 * on their behalf at call time: processes whose device memory is owned by
 * their own pool, hot loops that cannot absorb cudaMalloc's implicit device
 * synchronisation, and deployments that fix all memory up front.  The paper
 * has no counterpart; this is a library convenience.
 *
 * The call allocates nothing.  Its coefficient scratch is a file-scope static
 * device array of DAFMM_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading
 * the library holds until the process exits.  The first call on a device
 * resolves that array's device address (cudaGetSymbolAddress) with the device
 * current; make that first call before any stream capture.  The address is
 * cached for the life of the process: it stays valid while the device's
 * primary context lives, so do not call this entry point after the caller has
 * reset the device (cudaDeviceReset) or torn its primary context down.  Every call on a
 * device shares the array and clears the part it uses, so calls whose kernels
 * overlap in time on one device race and must be ordered by the caller (one
 * stream, or events).  The call also uses the ops handle's pass counters,
 * like dafmm_matvec: on one handle, a dafmm_matvec_noalloc and a dafmm_matvec
 * must not overlap in time either.  The operator itself (built by build_nca_operators)
 * must already exist; v_dev and out_dev are the caller's N complex128 device
 * vectors and must not overlap.
 * Errors: DAFMM_EBADARG when the problem needs more scratch than the array
 * holds (the message states both sizes), for NULL pointers or an unknown
 * precision; DAFMM_ECUDA for CUDA errors.
 */
int dafmm_matvec_noalloc(const dafmm_ops* ops, const double* v_dev, double* out_dev, int precision, void* stream);

/*
 * dafmm_sync -- synchronise the stream, then report whether any kernel of
 * this handle gave up a bounded wait on the device since the last check
 * (DAFMM_ETIMEOUT; the flag is cleared).  Otherwise DAFMM_OK, or DAFMM_ECUDA
 * for a CUDA error.  The apply kernels wait with a limit instead of an
 * unbounded spin: on the arrival of their own bulk copies (an iteration
 * limit) and, in the single-right-hand-side launch, on the rows of the tree
 * passes they read (about 0.2 s each).  After a timeout the result of the
 * application is undefined; the handle stays usable.
 */
int dafmm_sync(dafmm_ops* ops, void* stream);

/*
 * dafmm_set_contrast -- replace the contrast q of an operator (N doubles on
 * the device, copied on `stream`).  The NCA compresses K, which does not
 * depend on q (q enters A = I + kappa^2 diag(q) K only in the epilogue), so
 * one tree and one set of operators serve any number of contrasts.  A HODLR
 * preconditioner factored earlier keeps the q it was built with.  Errors:
 * DAFMM_EBADARG for NULL arguments, DAFMM_ECUDA.
 */
int dafmm_set_contrast(dafmm_ops* ops, const double* q_dev, void* stream);

/*
 * dafmm_debug_stall -- test support for the timeout path (the paper has no
 * counterpart).  The next single-right-hand-side dafmm_matvec on this handle
 * runs without graph replay and its kernel waits for one more row of tree
 * pass `pass` (0 = the leaf-level P2M) than the pass writes, so that wait
 * and the waits behind it give up; dafmm_sync then returns DAFMM_ETIMEOUT.
 * pass = -1 cancels.  Errors: DAFMM_EBADARG for a NULL handle or a pass
 * outside -1 .. (passes - 1).
 */
int dafmm_debug_stall(dafmm_ops* ops, int pass);

/*
 * dafmm_debug_leaf_staging -- test support (no counterpart in the paper).
 * The leaf kernel of a single-right-hand-side application copies its
 * far-field blocks (the L2L from level L-1 composed with L2P, and L2P:
 * Section 4's downward pass) into shared memory before it waits for the far
 * field, when every leaf has at most 8 composed blocks, one L2P block and
 * 64 columns of each; else it reads them from global memory.  enable = 0
 * forces the global-memory path, 1 restores the planned one (both give the
 * same result bit for bit: the same products in the same order).  Drops the
 * handle's captured graphs.  Errors: DAFMM_EBADARG for a NULL handle or
 * enable outside 0 .. 1.
 */
int dafmm_debug_leaf_staging(dafmm_ops* ops, int enable);

/*
 * dafmm_set_batched_kernel -- which kernel runs the tree passes (P2M, M2M,
 * M2L, L2L) of a complex64 (DAFMM_MIXED) application with several
 * right-hand sides: 0 automatic (currently the CUDA cores: faster at the
 * chunk shapes of these operators), 1 CUDA cores (FP32 FMA), 2 tensor cores.
 * The tensor-core kernel computes each block product as a real GEMM on
 * tcgen05.mma (kind::tf32) with every FP32 value split exactly into three
 * tf32 parts, and drains each chunk's accumulator into FP32 registers;
 * results differ from the CUDA-core kernel by FP32 rounding only.  Complex128 applications and single right-hand sides are
 * not affected.  Cached application graphs are dropped when the mode
 * changes.  Errors: DAFMM_EBADARG for a NULL handle or a mode outside 0..2.
 */
int dafmm_set_batched_kernel(dafmm_ops* ops, int mode);

/*
 * dafmm_field_eval -- the solution's fields at m arbitrary points x_k (Section
 * 6.1, the error function E(x)): psi(x_k) = sum_l Q^+(l,:) psi_vec^B b_l((x_k
 * - alpha^B) / beta) on the leaf B containing x_k (Eq. 7; zero outside the
 * domain), and the volume potential u(x_k) = int_Omega G(x_k, y) psi(y) dy
 * of that interpolant (Eq. 5), summed over every leaf with the quadrature of
 * the entry table (the near rule within one box width of x_k, the 16 x 16
 * rule beyond).  With them E(x) = |psi(x) + kappa^2 q(x) u(x) - f(x)| /
 * kappa^2 for the caller's q and f.  O(m N): one CTA per point.
 * psi_dev: N complex128 (the grid values); pts_dev: m x 2 doubles; u_dev: m
 * complex128; psi_at_dev: m complex128 or NULL; all on the device.  The
 * volume integral whatever the ops handle's kernel.  Allocates the N_p
 * coefficients per leaf for the call (stream-ordered).  Asynchronous on
 * stream.  Errors: DAFMM_EBADARG, DAFMM_ENOMEM, DAFMM_ECUDA.
 */
int dafmm_field_eval(const dafmm_ops* ops, const double* psi_dev, long m, const double* pts_dev, double* u_dev, double* psi_at_dev,
                     void* stream);

/*
 * dafmm_nbody_direct -- u_i = sum_{j != i} G(x_i, x_j) v_j over the tree's N
 * nodes by direct summation, O(N^2) (the reference of Experiment 1, Section
 * 6.2): one warp per target, the Hankel function H0^(1) = J0 + i Y0
 * evaluated in registers for every source (FP64), the partial sums of the
 * lanes combined by warp shuffles.  Uses the tree's kappa whatever its
 * kernel.  v_dev, out_dev: N complex128 on the device (must not overlap).
 * Allocates N x 2 doubles of node coordinates for the call (stream-ordered)
 * and synchronises the stream once, after copying them; the sum itself is
 * asynchronous on stream.  Errors: DAFMM_EBADARG, DAFMM_ENOMEM, DAFMM_ECUDA.
 */
int dafmm_nbody_direct(const dafmm_tree* tree, const double* v_dev, double* out_dev, void* stream);

/*
 * Tuning of the several-right-hand-side passes (see dafmm_tune_batched).
 * kernel: 1 CUDA cores, 2 tensor cores; ctas_per_sm: cap on the CTAs per SM
 * of the CUDA-core pass grids (0: as many as fit).
 */
typedef struct dafmm_tuning {
    int nrhs;              /* right-hand sides it was tuned for */
    int precision;         /* DAFMM_FP64 or DAFMM_MIXED */
    int kernel;            /* the choice */
    int ctas_per_sm;       /* the choice */
    double best_ms;        /* time of one application with the choice */
    int ncand;             /* candidates timed */
    int cand_kernel[16];
    int cand_ctas[16];
    double cand_ms[16];    /* each candidate's time of one application */
    int reserved[8];
} dafmm_tuning;

/*
 * dafmm_tune_batched -- time the candidate configurations of the tree passes
 * of an application with nrhs (2..64) right-hand sides in the given
 * precision: the CUDA-core kernel with 0 (all that fit), 1, 2 and 4 CTAs per
 * SM, and in DAFMM_MIXED the tensor-core kernel; each candidate runs two
 * untimed and five timed applications (CUDA events) on a private stream with
 * a fixed input.  The fastest is kept on the handle (as by
 * dafmm_set_batched_kernel and dafmm_set_batched_grid) and recorded in *out
 * with every candidate's time.  Results do not depend on the choice beyond
 * rounding.  Allocates two N x nrhs vectors for the call; synchronises.
 * Errors: DAFMM_EBADARG, DAFMM_ENOMEM, DAFMM_ECUDA.
 */
int dafmm_tune_batched(dafmm_ops* ops, int nrhs, int precision, dafmm_tuning* out);

/* Cap the CTAs per SM of the CUDA-core several-right-hand-side pass grids
 * (0: as many as fit, else 1..32).  Cached application graphs are dropped
 * when it changes.  Errors: DAFMM_EBADARG. */
int dafmm_set_batched_grid(dafmm_ops* ops, int ctas_per_sm);

/*
 * Several problems (operators of different sizes, each with its own tree)
 * applied together.  dafmm_batch_matvec computes out[i] = A_i v[i] for every
 * problem i, nrhs right-hand sides each, in one CUDA graph: with several
 * right-hand sides every problem's kernels on a stream of its own forked
 * from the graph's start, so the problems' kernels overlap (with one, the
 * problems run in order: the single-right-hand-side kernel needs the whole
 * GPU); the graph is captured on the first call for a
 * given (nrhs, precision, pointers) and replayed by one cudaGraphLaunch
 * after that (at most four such sets are kept).  v_dev, out_dev: host arrays
 * of n device pointers, each vector N_i x nrhs complex128.  The handles must
 * outlive the batch and must not be used concurrently elsewhere.
 * Errors: DAFMM_EBADARG, DAFMM_ENOMEM, DAFMM_ECUDA.
 */
typedef struct dafmm_batch dafmm_batch;
int dafmm_batch_create(int n, dafmm_ops* const* ops, dafmm_batch** out);
int dafmm_batch_matvec(dafmm_batch* batch, int nrhs, const double* const* v_dev, double* const* out_dev, int precision, void* stream);
int dafmm_batch_destroy(dafmm_batch* batch);

/* Realised ranks, operator bytes and work of one application. */
int dafmm_stats(const dafmm_ops* ops, dafmm_stats_t* stats);

/*
 * dafmm_entries -- the library's own entries K(rows[a], cols[b]) of Eq. 13,
 * read from the device-built offset table, into out_host (nr x nc complex,
 * interleaved, row-major).  For checking the setup against an independent
 * quadrature.
 */
int dafmm_entries(const dafmm_ops* ops, long nr, const long* rows_host, long nc, const long* cols_host, double* out_host);

/*
 * dafmm_profile -- enable (1) or disable (0) CUDA-event timing of the passes
 * of subsequent dafmm_matvec calls on this handle (events recorded on the
 * call's stream; at most 65536 calls are kept).  Enabling clears earlier
 * records.  dafmm_profile_read synchronises on the recorded events and sums
 * the pass times into *out.  Profiled calls replay graphs captured with
 * event-record nodes at the pass marks (each adds about 2.5 us of latency to
 * the application); unprofiled calls replay graphs without them.
 */
int dafmm_profile(dafmm_ops* ops, int enable);
int dafmm_profile_read(dafmm_ops* ops, dafmm_profile_t* out);

/* Release an operator and its device memory.  NULL is accepted. */
int ops_destroy(dafmm_ops* ops);

/* ------------------------------------------------------------------------
 * Learned initial guess and coarse correction.  Not part of the paper: a
 * convolutional U-Net maps (q, f) on the node grid to an approximation of
 * the solution psi of Eq. 13, trained on the library's own solutions.  The
 * node grid is the n_side x n_side image whose pixel (x, y) holds node
 * (4 lx + k1, 4 ly + k2) of leaf (lx, ly) (Morton order) at local index
 * k1 + 4 k2.
 * Network: `levels` resolution levels with base * 2^l channels at level l;
 * per level two 3x3 convolutions (bias, ReLU), 2 x 2 average pooling
 * between levels, nearest 2x upsampling, a 3x3 up-convolution, the
 * concatenation [skip, up] and two 3x3 convolutions on the way up, a final
 * 1x1 convolution.  Zero padding.  Activations and weights are rounded to
 * BF16 for the products, sums are FP32; FP32 master weights, Adam.
 * Parameters, flattened: for every convolution in the order (encoder level
 * 0..levels-1: first, second), (decoder level levels-2..0: up, first,
 * second), (output), the weights [ky][kx][c_in][c_out] then the bias
 * [c_out].
 * ------------------------------------------------------------------------ */
typedef struct unet_params {
    int levels;               /* 1..6 (4 is typical) */
    int base;                 /* channels at full resolution, 1..256 (32 is typical) */
    int in_ch;                /* 3: q, Re f / s, Im f / s */
    int out_ch;               /* 2: Re psi / s, Im psi / s */
    unsigned long long seed;  /* He-normal weight initialisation (SplitMix64, Box-Muller) */
    int reserved[8];          /* must be zero */
} unet_params;

typedef struct dafmm_unet dafmm_unet;

/* Create a network with freshly initialised weights.  DAFMM_EBADARG for
 * parameters outside the ranges above, DAFMM_ENOMEM, DAFMM_ECUDA. */
int unet_create(const unet_params* p, dafmm_unet** out);
int unet_destroy(dafmm_unet* net);
/* Number of FP32 parameters. */
int unet_num_params(const dafmm_unet* net, long* n);
/* Copy the FP32 parameters (layout above) to / from a host array. */
int unet_get_params(const dafmm_unet* net, float* host);
int unet_set_params(dafmm_unet* net, const float* host);

/*
 * unet_forward -- out = N(in) for `batch` images of height x width
 * (multiples of 2^(levels-1)).  in_dev: [batch][height][width][in_ch] FP32,
 * out_dev: [batch][height][width][out_ch] FP32, both device, caller-owned.
 * Activations are kept in the handle (grown on demand; not thread-safe).
 */
int unet_forward(dafmm_unet* net, int batch, int height, int width, const float* in_dev, float* out_dev, void* stream);

/*
 * unet_backward -- forward, mean squared error against target_dev (same
 * shape as out_dev), and the gradient of that error with respect to every
 * parameter, kept in the handle (replacing the previous one).  out_dev
 * receives the forward output; *loss_host the error.  Synchronises.
 */
int unet_backward(dafmm_unet* net, int batch, int height, int width, const float* in_dev, const float* target_dev, float* out_dev,
                  double* loss_host, void* stream);
/* The gradient of the last unet_backward (layout of the parameters). */
int unet_get_grads(const dafmm_unet* net, float* host);
/* One Adam step (Kingma and Ba, with bias correction) with that gradient. */
int unet_adam(dafmm_unet* net, float lr, float beta1, float beta2, float eps, void* stream);

/*
 * unet_guess -- x = s N(q, f / s) on the operator's node grid, s = max |f|
 * (q: the contrast the operator was built with).  f_dev, x_dev: N complex128.
 */
int unet_guess(dafmm_unet* net, const dafmm_ops* ops, const double* f_dev, double* x_dev, void* stream);

/* What gmres_solve_learned adds to gmres_stats. */
typedef struct learned_stats {
    int guess_used;          /* 1: the network's guess was accepted as x0 */
    double guess_residual;   /* |f - A x_guess| / |f| (FP64), or -1 when no guess was made */
    int corrections;         /* applications of the learned coarse correction */
} learned_stats;

/*
 * gmres_solve_learned -- gmres_solve with the network's help.  flags bit 0:
 * start from x0 = unet_guess(f) when |f - A x0| < |f| (FP64 residual),
 * else from the caller's x.  Bit 1: right preconditioner
 * z = M^-1 r + alpha s N(q, r / s), s = max |r| (a nonlinear coarse
 * correction added to the HODLR solve, or to the identity when M is NULL;
 * flexible GMRES keeps the preconditioned vectors).  Otherwise as
 * gmres_solve.
 */
int gmres_solve_learned(dafmm_ops* ops, const dafmm_hodlr* M, dafmm_unet* net, int flags, double alpha, const double* f_dev,
                        double* x_dev, const gmres_opts* opts, gmres_stats* st, learned_stats* ls, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DAFMM_H */
