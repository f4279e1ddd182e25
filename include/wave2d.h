/*
 * wave2d: explicit time marching of the 2D acoustic wave equation with the
 * 5-, 9- and 13-point schemes generated by Poisson's formula
 * (N. Khutoryansky, arXiv:1904.04048), on one NVIDIA GB300 (sm_103a).
 *
 * Problem (Section 2, Eq. we1): u_tt = c^2 (u_x1x1 + u_x2x2), u(.,0) = u0,
 * u_t(.,0) = v0, on a uniform grid of spacing h with time step tau and
 * Courant number lambda = c tau / h (Eq. Courant).
 *
 * Time-stepping algorithm (Section 3):
 *   first step  (Eq. A1):  u^1 = u^0 + tau v^0 + 1/2 Lambda_a(u^0) + tau Lambda_b(v^0)
 *   two-step    (Eq. A2):  u^{k+1} = 2 u^k - u^{k-1} + Lambda_a(u^k),  k >= 1
 * with Lambda_a(w) = a10 delta_w(1,0) + a11 delta_w(1,1) + a20 delta_w(2,0),
 * delta_w(q1,q2) = the sum of w over the four 90-degree rotations of the
 * offset (q1,q2) minus four times the centre (Eq. notations2), and the
 * coefficients of Section 6 (Eq. comp5.1/5.2, comp9.1/9.2, comp13.1/13.2):
 *   scheme 5:  a10 = l^2                    b10 = l^2/6
 *   scheme 9:  a10 = l^2 (1 - l^2/3)        b10 = l^2/6 (1 - l^2/5)
 *              a11 = l^4/6                  b11 = l^4/60
 *   scheme 13: a10 = l^2 (4 - 2 l^2)/3      b10 = l^2/6 (4/3 - 2 l^2/5)
 *              a11 = l^4/6                  b11 = l^4/60
 *              a20 = l^2 (l^2 - 1)/12       b20 = l^2/6 (l^2/20 - 1/12)
 * (l = lambda; all other coefficients zero).  WAVE2D_CONVENTIONAL selects the
 * comparison schemes of Section 6: b = 0 (central-difference first step,
 * Eq. comp5.1a, comp9.1b) and, for scheme 9, a10 = 2 l^2/3, a11 = l^2/6
 * (Eq. comp9.2b).
 *
 * Stability (Eq. stability5, stability9, Section 6.3): lambda <= lambda_max
 * with lambda_max = 1/sqrt2 (schemes 5, 13), sqrt((3 - sqrt3)/2) (scheme 9;
 * the printed value is read this way), sqrt3/2 (conventional 9).
 *
 * Conventions of every function below
 *   Fields are row-major nx-by-ny arrays of double: node (i, j), i along x1,
 *   j along x2, at index j*nx + i.  Boundary (Section 6.1.2, Section 6.3):
 *   WAVE2D_BC_ZERO     nodes outside the nx-by-ny set hold 0 at every level
 *                      (the grid boundary condition u = 0 of Section 6.1.2,
 *                      a zero ring of width 2 for scheme 13);
 *   WAVE2D_BC_PERIODIC indices wrap modulo nx and ny (Section 6.3).
 *   WAVE2D_BC_ODD      the zero boundary's node set and boundary nodes
 *                      (u = 0 at i = -1, i = nx and likewise in j), with the
 *                      field continued beyond them as an odd function,
 *                      u(-1 - k) = -u(-1 + k), u(nx + k) = -u(nx - k): for
 *                      radius-1 stencils the same as WAVE2D_BC_ZERO, for the
 *                      13-point and derived schemes a Dirichlet condition the
 *                      paper leaves open (it is exact for sine modes).  One-
 *                      node and TMA kernels (no temporal blocking, no batches).
 *   Errors: every int function returns WAVE2D_OK (0) or a negative status;
 *   wave2d_last_error() then gives a message (thread-local).  Kernels run
 *   asynchronously on the handle's stream; a device-side failure surfaces as
 *   WAVE2D_ERR_CUDA at the next call that synchronises (sync, norms, state).
 *   Ownership: the library owns all device memory of a handle (allocated at
 *   create through the allocator hook, freed by destroy).  Input arrays are
 *   copied before the call returns; outputs go to caller buffers.
 *   Thread safety: a handle is used by one host thread at a time.
 */
#ifndef WAVE2D_H
#define WAVE2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    WAVE2D_OK = 0,
    WAVE2D_ERR_ARG = -1,       /* invalid argument                              */
    WAVE2D_ERR_UNSTABLE = -2,  /* lambda above the scheme's stability limit     */
    WAVE2D_ERR_OOM = -3,       /* device allocation failed                      */
    WAVE2D_ERR_CUDA = -4,      /* CUDA runtime / kernel error                   */
    WAVE2D_ERR_NONFINITE = -5, /* a norm found NaN or Inf in the field          */
    WAVE2D_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up            */
    WAVE2D_ERR_STATE = -7      /* call out of order (e.g. stepping before init) */
};

enum { WAVE2D_BC_ZERO = 0, WAVE2D_BC_PERIODIC = 1, WAVE2D_BC_ODD = 2 };

/* Storage / arithmetic type of the time levels.  The first step always
 * computes in FP64 and rounds into the storage type; norms reduce in FP64.
 * WAVE2D_F32X2 keeps each value as an unevaluated sum hi + lo of two floats
 * (double-float arithmetic, about 48 significant bits). */
enum { WAVE2D_F64 = 0, WAVE2D_F32 = 1, WAVE2D_F32X2 = 2 };

/* grid.flags */
enum {
    WAVE2D_ALLOW_UNSTABLE = 1, /* accept lambda > lambda_max (for instability tests) */
    WAVE2D_CONVENTIONAL = 2,   /* comparison schemes: central-difference first step,
                                  isotropic 9-point Laplacian (Eq. comp9.2b)        */
    WAVE2D_DIFF_SUMS = 4,      /* form each stencil sum of the two-step from the
                                  differences u_q - u_ij (exact for neighbouring
                                  values of a smooth field): the same operator
                                  with less cancellation in the sums (measured
                                  3-4x lower FP32 error for mid-length waves; the
                                  longest waves need WAVE2D_DIFF_FORM).  F32 and
                                  F64 storage; one-node and TMA kernels only (no
                                  temporal blocking, no batches).                */
    WAVE2D_DIFF_FORM = 8,      /* F32 only: keep u^k and d^k = u^k - u^{k-1} and
                                  step d^{k+1} = d^k + Lambda(u^k),
                                  u^{k+1} = u^k + d^{k+1} (the same recursion,
                                  Eq. A2) with difference sums: the rounding of
                                  u enters once instead of being integrated
                                  twice.  Three planes, 16 B per node-update;
                                  one-node and TMA kernels.  get/set_state
                                  convert to and from (u^{k-1}, u^k) in FP64;
                                  the raw layout is [d^k][u^k].                 */
    WAVE2D_CANARY = 16         /* debug: fill the plane cells no one-level kernel
                                  writes and no result depends on (ghost cells
                                  more than R rows or R + 4 columns outside the
                                  grid, row padding) with a NaN pattern;
                                  wave2d_canary_check counts cells that changed.
                                  Such handles use the temporal kernels on the
                                  zero boundary only (periodic images fill the
                                  whole ring there) and no batches.             */
};

/* Exact solutions for wave2d_error_vs_exact / wave2d_track_error.
 *   STANDING: amp sin(2 pi m x1) sin(2 pi m x2) sin(2 sqrt2 pi m c t)
 *             (Eq. "exact sol" for amp = m = 1)
 *   PLANE:    amp cos(k1 x1 + k2 x2 - c |k| t)
 *   NONE:     u_e = 0 (the norms then measure the field itself)
 * Node (i, j) sits at x = ((i + x_off) h, (j + x_off) h); the paper's
 * Dirichlet node set {0 < i < n} is x_off = 1, its periodic one x_off = 0. */
enum { WAVE2D_EXACT_NONE = 0, WAVE2D_EXACT_STANDING = 1, WAVE2D_EXACT_PLANE = 2 };

typedef struct {
    int32_t kind;
    int32_t reserved;
    double amp;
    double m;      /* STANDING mode number */
    double k1, k2; /* PLANE wave vector    */
    double x_off;
} wave2d_exact;

typedef struct {
    int32_t nx, ny; /* updated nodes along x1 and x2 (1 .. 65536 each)          */
    int32_t bc;     /* WAVE2D_BC_*                                             */
    int32_t dtype;  /* WAVE2D_F64 | WAVE2D_F32 | WAVE2D_F32X2                  */
    int32_t flags;  /* WAVE2D_ALLOW_UNSTABLE | WAVE2D_CONVENTIONAL | WAVE2D_DIFF_SUMS |
                       WAVE2D_DIFF_FORM                                         */
    int32_t reserved;
    void *stream;   /* cudaStream_t the handle launches on; NULL = default stream */
} wave2d_grid;

typedef struct wave2d *wave2d_t;

/* Kernel selection for the two-step.  Zero-initialised = automatic: the
 * one-node kernel below 65536 nodes and for FP64 / FP32x2; from 65536 nodes
 * in FP32 the streaming kernel where it applies (below: the Section 6 schemes
 * and class chains of one to three classes), else the TMA kernel. */
enum {
    WAVE2D_KERNEL_AUTO = 0,
    WAVE2D_KERNEL_SIMPLE = 1,   /* one thread per node, global loads (FP32x2
                                   above 2^20 nodes without per-step norms: two
                                   nodes per thread in packed double-float
                                   arithmetic, the same result)              */
    WAVE2D_KERNEL_TMA = 2,      /* TMA-staged shared-memory tiles, one step      */
    WAVE2D_KERNEL_TEMPORAL = 3, /* TMA tiles advanced T steps in shared memory   */
    WAVE2D_KERNEL_STREAM = 4,   /* T steps per launch with the levels in
                                   registers: one warp walks down a strip of 128
                                   columns, halo columns by warp shuffles       */
    WAVE2D_KERNEL_PERSISTENT = 5 /* every level of a step_n call in one
                                   cooperative launch (one node per thread per
                                   pass, a grid barrier between levels, each wait
                                   bounded): for grids too small to fill the GPU,
                                   where a launch per level costs more than the
                                   level; the Section 6 schemes with plain sums,
                                   any storage type and boundary               */
};
/* The two multi-level kernels (TEMPORAL, STREAM) take FP32 handles on the
 * zero and periodic boundaries (with WAVE2D_CANARY the zero boundary only):
 * TEMPORAL the 5-, 9- and 13-point schemes with plain sums; STREAM those and
 * every class chain of one to three classes (WAVE2D_DIFF_SUMS,
 * WAVE2D_DIFF_FORM, derived schemes of up to 13 points), the difference form
 * on a periodic grid only with nx a multiple of 4 and ny >= 16.  They write
 * out of place (the handle's second pair of level planes; the difference
 * form alternates u^k and d^k between two planes each) and finish a run
 * whose length is not a multiple of T with TMA single steps.  Every kernel
 * evaluates each node identically, so the choice changes no result bit. */

typedef struct {
    int32_t kernel;       /* WAVE2D_KERNEL_*                                      */
    int32_t tile_h;       /* output rows per tile of WAVE2D_KERNEL_TEMPORAL: 16,
                             24, 32 or 64 (0 = 24 for 9 points, else 32); output
                             rows per strip of WAVE2D_KERNEL_STREAM: 8 .. 4096
                             (0 = the most of 64, 32 and 16 that makes at
                             least 6 strips per SM)                               */
    int32_t temporal_t;   /* steps per launch of the multi-level kernels: 2, 3 or
                             4 for WAVE2D_KERNEL_TEMPORAL (0 = 4); 2, 3, 4 or 6
                             for WAVE2D_KERNEL_STREAM (0 = 4 for 13 points, 6
                             for 5 and 9 points), 2, 3 or 4 in the difference
                             form (0 = 3 for 13 points, else 4)                   */
    int32_t use_graph;    /* capture runs of steps in a CUDA graph: 1 on, 0 off,
                             -1 automatic                                         */
    int32_t ctas_per_sm;  /* resident CTAs per SM for the TMA kernels; 0 = auto:
                             as many as fit while both levels nearly fit in L2,
                             else one (measured: wider residency starves some
                             CTAs once the levels stream from HBM)               */
} wave2d_tune;

typedef struct {
    double lambda, h, tau, c;
    double a[3];     /* a10, a11, a20 as used (FP64)                          */
    double b[3];     /* b10, b11, b20 as used (FP64)                          */
    double lambda_max;
    int64_t k;       /* index of the current time level u^k (0 before any step) */
    int32_t scheme, radius, dtype, bc;
    int32_t nx, ny, pitch, ghost;
    int64_t device_bytes;
    int32_t kernel;  /* two-step kernel currently selected (WAVE2D_KERNEL_*)  */
    int32_t temporal_t;
    int32_t n_classes;  /* derived schemes: classes in use (0 for scheme 5/9/13) */
    int32_t n_points;   /* stencil nodes, centre included                        */
    double class_a[8];  /* derived schemes: a_c as used, in chain order          */
    double class_b[8];  /* derived schemes: b_c as used                          */
} wave2d_info_t;

/* ------------------------------------------------------------------------ */
/* Allocation hook (process-wide).  alloc returns a device pointer with at   */
/* least 256-byte alignment or NULL; free releases it.  Passing NULL for both */
/* restores cudaMalloc / cudaFree.  Handles keep the hook they were created   */
/* with.                                                                      */
/* ------------------------------------------------------------------------ */
typedef void *(*wave2d_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*wave2d_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int wave2d_set_allocator(wave2d_alloc_fn alloc, wave2d_free_fn release, void *ctx);

/* Create a simulation of `scheme` (5, 9 or 13) on `grid` with spacing h,
 * time step tau and speed c (Section 3; lambda = c tau / h, Eq. Courant).
 * Allocates the two time levels (plus a halo ring) and the reduction scratch
 * on the current device.  Errors: WAVE2D_ERR_ARG (bad sizes / scheme / h,
 * tau, c not positive and finite), WAVE2D_ERR_UNSTABLE (lambda above
 * lambda_max * (1 + 1e-12) without WAVE2D_ALLOW_UNSTABLE), WAVE2D_ERR_OOM. */
int wave2d_create(const wave2d_grid *grid, double h, double tau, double c, int scheme,
                  wave2d_t *out);

/* ------------------------------------------------------------------------ */
/* Derived schemes.  Sections 4-5 build a stencil from any initial segment    */
/* M*_{<=m} of the monomials ordered by Eq. g: the nodes are the McKinney      */
/* images (Eq. alpha / invMcKinney) of the monomials, the weights A phi_q and  */
/* B phi_q of the Lagrange basis of Eq. Lagrange follow from the inverse of    */
/* the matrix D of Eq. matrix1 and the exact integrals of Eq. exact1 / exact2.*/
/* m = 6, 11, 15 give the 5-, 9- and 13-point schemes of Section 6; larger     */
/* segments give further schemes.  When the weights are symmetric under the   */
/* eight symmetries of the square they group into classes: class (q1, q2),    */
/* q1 > 0, 0 <= q2 <= q1, is the set of nodes (+-q1, +-q2), (+-q2, +-q1)       */
/* (4 nodes if q2 == 0 or q2 == q1, else 8), and                              */
/*   Lambda_a(w) = sum_c a_c delta_c(w),  delta_c(w) = sum_{q in c} w_{.+q} - n_c w. */
/* Segments up to m = 49 use the classes of the chain, in this order:         */
/*   c = 0..7:  (1,0) (1,1) (2,0) (2,1) (3,0) (2,2) (3,1) (4,0)                */
/* (m = 24: 21 points, 28: 25, 37: 29, 41: 37, 45: 41); a scheme uses the     */
/* first n_classes of them, a class it lacks having zero coefficients.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t segment;    /* m of the segment it was derived from; 0 if supplied   */
    int32_t n_classes;  /* 1..8: the first n_classes classes of the chain        */
    int32_t radius;     /* stencil radius (largest q1 in use)                    */
    int32_t n_points;   /* stencil nodes with a non-zero weight, centre included */
    double a[8][9];     /* a_c(lambda) = sum_p a[c][p] lambda^p  (two-step)      */
    double b[8][9];     /* b_c(lambda) = sum_p b[c][p] lambda^p  (first step, v) */
} wave2d_scheme;

/* Derive the scheme of the segment M*_{<=m} (host only, no GPU needed): the
 * derivation above in FP64 (Gaussian elimination with partial pivoting and
 * two rounds of refinement whose residuals are computed with compensated
 * products and sums; the entries of D are small integers, held exactly),
 * a_c = 2 A phi_q and
 * b_c = B phi_q / tau as polynomials in lambda, coefficients below 1e-13 of
 * the largest dropped to zero.  Errors: WAVE2D_ERR_ARG for m outside 1..49,
 * a segment whose nodes are not distinct or whose D is singular, weights
 * that are not symmetric (e.g. m = 14, 23, 27, 40, 44) or a segment with no
 * class at all (m <= 4). */
int wave2d_derive_scheme(int32_t m, wave2d_scheme *out);

/* Stability limit of a scheme (host only): the largest lambda such that for
 * every lambda' <= lambda the symbol S(theta) = sum_c a_c(lambda') sigma_c(theta),
 * sigma_c(theta) = sum_{q in c} (cos(q . theta) - 1), stays in [-4, 0] on a
 * 129 x 129 grid of theta in [0, pi]^2 (von Neumann: the roots of
 * g^2 - (2 + S) g + 1 then lie on the unit circle), found by a scan in steps
 * of 1/512 up to lambda = 2 and 60 bisections.  For m = 6, 11, 15 it returns
 * the Section 6 limits to 1e-12.  *out = 0 if even lambda = 1/512 is unstable. */
int wave2d_scheme_lambda_max(const wave2d_scheme *s, double *out);

/* Create a simulation of a derived (or caller-supplied) scheme; otherwise as
 * wave2d_create.  The coefficients are evaluated at lambda = c tau / h in
 * FP64.  The two-step runs on the one-node kernel or the TMA kernel
 * (WAVE2D_KERNEL_TEMPORAL is not available: WAVE2D_ERR_ARG from
 * wave2d_set_tuning); grid.flags may hold WAVE2D_ALLOW_UNSTABLE,
 * WAVE2D_DIFF_SUMS and WAVE2D_DIFF_FORM, not WAVE2D_CONVENTIONAL.  Errors as
 * wave2d_create, with the stability limit of wave2d_scheme_lambda_max. */
int wave2d_create_scheme(const wave2d_grid *grid, double h, double tau, double c,
                         const wave2d_scheme *s, wave2d_t *out);

/* First time step (Eq. A1 in the discrete forms comp5.1, comp9.1, comp13.1):
 * u0, v0 are nx*ny FP64 arrays, in host memory (on_device = 0) or device
 * memory (on_device = 1).  Computes u^1 in FP64 and stores u^0, u^1 in the
 * storage type; afterwards k = 1.  Resets any spacetime error accumulation
 * and, if tracking is on (wave2d_track_error), adds the k = 1 term. */
int wave2d_first_step(wave2d_t h, const double *u0, const double *v0, int on_device);

/* n two-steps (Eq. A2 in the forms comp5.2, comp9.2, comp13.2), in place,
 * asynchronous on the handle's stream; k += n.  n = 0 is a no-op; n < 0 is
 * WAVE2D_ERR_ARG; before first_step / set_state it is WAVE2D_ERR_STATE. */
int wave2d_step_n(wave2d_t h, int64_t n);

/* Error of the current level u^k against an exact solution at t = k tau,
 * reduced in FP64 on the device:
 *   rel_l2   = sqrt(sum (u - u_e)^2 / sum u_e^2)  (for kind NONE: sqrt(sum u^2))
 *   rel_linf = max |u - u_e| / max |u_e|           (for kind NONE: max |u|)
 * spacetime_E (may be NULL) receives the paper's relative space-time error
 * E(n, n_t) of Eq. error, sum over k = 1..n_t, accumulated since first_step
 * when tracking is enabled, else NaN.  Any output pointer may be NULL.
 * Synchronises the stream.  Returns WAVE2D_ERR_NONFINITE (outputs still
 * written) if the field holds NaN or Inf. */
int wave2d_error_vs_exact(wave2d_t h, const wave2d_exact *ex, double *rel_l2, double *rel_linf,
                          double *spacetime_E);

/* The current levels of two handles of the same grid size and level index k
 * (any storage types, same device) compared in FP64 on the device:
 *   rel_l2   = sqrt(sum (u_a - u_b)^2 / sum u_b^2)
 *   rel_linf = max |u_a - u_b| / max |u_b|
 * b is the reference (e.g. an FP64 run of the same problem: the error of a
 * lower-precision run against it).  Orders a's stream after b's; synchronises
 * a's stream.  WAVE2D_ERR_ARG for different sizes or devices,
 * WAVE2D_ERR_STATE for different k. */
int wave2d_diff_norms(wave2d_t a, wave2d_t b, double *rel_l2, double *rel_linf);

/* Enable (ex != NULL) or disable (NULL) accumulation of the sums of Eq. error
 * after every step from the next first_step on.  Tracking uses the one-node-
 * per-thread kernel with the reduction fused into the step. */
int wave2d_track_error(wave2d_t h, const wave2d_exact *ex);

/* Checkpoint: copy u^{k-1}, u^k (as FP64; exact for FP64 and FP32 storage,
 * hi + lo rounded to FP64 for FP32X2) and k to host buffers of nx*ny doubles.
 * Any pointer may be NULL.  Synchronises. */
int wave2d_get_state(wave2d_t h, double *u_prev, double *u_cur, int64_t *k);

/* Resume: load u^{k-1}, u^k (host or device FP64 arrays, rounded to the
 * storage type) and the level index k (k >= 1). */
int wave2d_set_state(wave2d_t h, const double *u_prev, const double *u_cur, int64_t k,
                     int on_device);

/* Raw storage copy of the two current levels to host memory, for bitwise
 * checkpoints in every storage type.  bytes must be >= wave2d_raw_bytes(). */
int64_t wave2d_raw_bytes(wave2d_t h);
int wave2d_get_raw(wave2d_t h, void *dst, int64_t bytes, int64_t *k);
int wave2d_set_raw(wave2d_t h, const void *src, int64_t bytes, int64_t k);

int wave2d_set_tuning(wave2d_t h, const wave2d_tune *tune);

/* Autotuner: time every candidate two-step configuration for `steps` levels
 * on a copy of the current state (FP32: the TMA one-step kernel at 1 and 2
 * CTAs per SM, the temporal kernel with T in {2, 3, 4} and 16, 24, 32 or 64
 * rows per tile, and the streaming kernel with T in {2, 3, 4} and 16, 24, 32
 * or 48 rows per strip; derived FP32 schemes: the TMA kernel at 1 and 2 CTAs per SM
 * and the one-node kernel; FP64: TMA at 1 and 2 CTAs per SM and the one-node
 * kernel), restore
 * the state exactly (levels, k) and keep the fastest configuration, which is
 * also written to *best (may be NULL).  Results do not depend on the choice:
 * every configuration evaluates each node identically.  Needs an initialised
 * handle (WAVE2D_ERR_STATE) and steps >= 1; allocates a snapshot of two
 * levels for the duration of the call.  Synchronises the stream. */
int wave2d_autotune(wave2d_t h, int64_t steps, wave2d_tune *best);
int wave2d_get_info(wave2d_t h, wave2d_info_t *info);
int wave2d_sync(wave2d_t h);

/* Row access for domain decomposition.  Eq. A2 updates a node from the
 * nodes within the stencil radius R of it (Section 4, the stencil Q_m around
 * node (i, j)), so a band of rows advanced T levels stays exact R T rows in
 * from its edges: a partition of the grid into row slabs, each extended by
 * R T halo rows and refreshed from its neighbours every T levels, reproduces
 * the undivided run bit for bit.  These calls move the halo rows.
 *   get_rows: copy rows [j0, j0 + nrows) of the two state planes of h to
 *             prev (u^{k-1}; d^k for WAVE2D_DIFF_FORM) and cur (u^k), each a
 *             packed block of nrows * nx values of the storage type (F64:
 *             double; F32: float; F32X2: nrows * nx hi floats followed by
 *             nrows * nx lo floats), row r of the block at r * nx.
 *   set_rows: the reverse; the ghost-ring images (periodic, odd) of h are
 *             rewritten afterwards.
 * on_device = 1: prev / cur are device memory and the copies are queued on
 * the handle's stream (synchronise it before other streams use the buffer);
 * 0: host memory, the call returns when the copy is done.  The caller owns
 * the buffers.  WAVE2D_ERR_ARG for rows outside 0 .. ny or a null buffer,
 * WAVE2D_ERR_STATE before the first step. */
int wave2d_get_rows(wave2d_t h, int j0, int nrows, void *prev, void *cur, int on_device);
int wave2d_set_rows(wave2d_t h, int j0, int nrows, const void *prev, const void *cur, int on_device);

/* The unnormalised terms of the error norms (wave2d_error_vs_exact) over rows
 * [j0, j0 + nrows) of u^k, with the exact solution evaluated as if local row
 * j were row j + row_shift of a larger grid (a slab's offset in the whole
 * grid): sums[0] = sum (u - u_e)^2, sums[1] = sum u_e^2, sums[2] =
 * max |u - u_e|, sums[3] = max |u_e|, reduced in FP64 on the device.  Slabs
 * combine them by a sum (0, 1) and a maximum (2, 3) into the norms of
 * Eq. error.  Synchronises the stream; WAVE2D_ERR_NONFINITE if the rows hold
 * NaN or Inf. */
int wave2d_error_sums(wave2d_t h, const wave2d_exact *ex, int j0, int nrows, int64_t row_shift,
                      double *sums);

/* Failure-detection self-test: launch, on the handle's stream, a kernel that
 * waits on an mbarrier nothing ever completes, through the same bounded wait
 * every pipelined kernel uses, and one that waits at the persistent kernel's
 * grid barrier for an arrival that never comes, each with a limit of
 * limit_cycles SM clocks (1 .. 2^31).  The waits give up and raise the
 * handle's timeout status, which the next synchronising call (wave2d_sync,
 * norms, state) reports as WAVE2D_ERR_TIMEOUT and clears; the GPU stays
 * usable. */
int wave2d_selftest_timeout(wave2d_t h, int64_t limit_cycles);

/* Guard-band check of a handle created with WAVE2D_CANARY: *changed receives
 * the number of canary cells (see WAVE2D_CANARY) whose bits differ from the
 * pattern written at create and after wave2d_set_raw — 0 unless a kernel
 * wrote outside the part of the planes it owns.  Synchronises the stream.
 * WAVE2D_ERR_STATE for a handle without the flag. */
int wave2d_canary_check(wave2d_t h, int64_t *changed);
void wave2d_destroy(wave2d_t h);
const char *wave2d_last_error(void);

/* Allocation-free variant of the FP64 norms of wave2d_error_vs_exact, for
 * callers that cannot allocate device memory: code whose GPU memory is owned
 * and budgeted by another allocator (a serving process that hands its whole
 * memory pool to a framework), and latency-critical loops where a cudaMalloc
 * would synchronise the device.  The paper has no counterpart; it is a
 * service of this library.
 *   field   device array of nx*ny values (F32 or F64 per dtype), row j at
 *           field + j*ld elements; owned by the caller, only read.
 *   h, c, t grid spacing, wave speed and time of the exact solution; ex as
 *           for wave2d_error_vs_exact (NULL = WAVE2D_EXACT_NONE).
 *   rel_l2, rel_linf  host outputs with the meaning of wave2d_error_vs_exact.
 *   stream  cudaStream_t to run on (NULL = default stream); the call
 *           synchronises it before returning.
 * No device memory is allocated: the scratch (partial sums, result slots,
 * exact-solution tables) is one file-scope __device__ array of about 320 KiB
 * that every GPU loading the library holds until the process exits.  Limits:
 * 1 <= nx, ny <= 8192, else WAVE2D_ERR_ARG.  The first call on each device
 * looks up the array's address (cudaGetSymbolAddress) and caches it: make
 * that first call before any stream capture.  The cached address belongs to
 * the device's context of that moment: after cudaDeviceReset (or anything
 * else that destroys the primary context) it is stale, so do not call this
 * function again in that process.  All calls share the array and
 * it keeps the last call's contents (the call clears what must start at
 * zero): calls that overlap on the GPU, from any thread or stream, race and
 * must be serialised by the caller. */
int wave2d_error_norms_noalloc(const void *field, int dtype, int nx, int ny, int64_t ld, double h,
                               double c, double t, const wave2d_exact *ex, double *rel_l2,
                               double *rel_linf, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched stepping of many independent simulations (FP32 storage, one       */
/* boundary type and one device for the whole batch).  A run advances every  */
/* instance by its own number of two-steps (Eq. A2) in quanta of Tq <= 4     */
/* levels; each quantum is one launch over the tiles of all instances still  */
/* running, the quanta of a run are replayed from one CUDA graph, and every  */
/* instance ends bit for bit where the same steps on its own handle end.     */
/* The handles stay owned by the caller and must outlive the batch; they may  */
/* be stepped, checkpointed or queried individually between batch calls.     */
/* ------------------------------------------------------------------------ */
typedef struct wave2d_batch *wave2d_batch_t;

/* Group n handles; opt (may be NULL) chooses the kernel: 0 or
 * WAVE2D_KERNEL_TEMPORAL for shared-memory regions (any boundary; tile_h 32
 * or 64 rows), WAVE2D_KERNEL_STREAM for register streaming (zero boundary;
 * one warp per strip of 8..1024 rows, tile_h, default 64, over the strips of
 * all instances of a scheme, the three schemes as concurrent branches), and
 * fixes the quantum (temporal_t, 1..4 levels per launch); zero fields keep
 * the defaults (regions, 4 levels, 32 rows) until wave2d_batch_autotune
 * chooses; use_graph = 0 launches the quanta of every run directly (for runs
 * used once) instead of capturing a graph.  WAVE2D_ERR_ARG for non-F32
 * handles, mixed boundaries or devices, a repeated handle, or streaming on a
 * periodic batch. */
int wave2d_batch_create(wave2d_t *handles, int n, const wave2d_tune *opt, wave2d_batch_t *out);

/* First step (Eq. A1) of every instance in one launch: u0[i], v0[i] are the
 * nx*ny FP64 arrays of instance i, all on the host (on_device = 0) or all on
 * the device (1).  Afterwards every instance is at k = 1. */
int wave2d_batch_first_step(wave2d_batch_t b, const double *const *u0, const double *const *v0,
                            int on_device);

/* Advance instance i by steps[i] >= 0 levels, asynchronously on the first
 * handle's stream.  The captured run is reused while the step counts and the
 * handles' plane pairs repeat. */
int wave2d_batch_run(wave2d_batch_t b, const int64_t *steps);

/* Time the run for min(steps[i], probe_steps) levels with the candidate
 * configurations on a snapshot of every instance, restore every instance
 * exactly and keep the fastest (written to *best, may be NULL): regions with
 * quanta 2 and 4 and tiles of 32 and 64 rows, and for the zero boundary
 * register streaming with 2, 3 or 4 levels per launch (which also sets the
 * strips' halo width, R T columns) and strips of 16, 32 or 64 rows. */
int wave2d_batch_autotune(wave2d_batch_t b, const int64_t *steps, int64_t probe_steps,
                          wave2d_tune *best);

/* FP64 L2 norm sqrt(sum u^2) and max |u| of every instance's current level:
 * out[2i], out[2i+1].  Synchronises. */
int wave2d_batch_norms(wave2d_batch_t b, double *out);

void wave2d_batch_destroy(wave2d_batch_t b);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of independent simulations (FP32 storage,    */
/* zero boundary).  A scheduler thread admits queued requests in arrival     */
/* order while the device-memory budget and the slot limit allow, runs the   */
/* first step (Eq. A1) of the newly admitted ones in one batched launch,     */
/* advances every resident simulation by up to `quantum` two-steps (Eq. A2)  */
/* per round in one batched run (the batch kept while its members stay), and */
/* retires finished ones: their FP64 norms in one launch, copied to pinned   */
/* host memory and collected once the copy has passed, their memory released */
/* in stream order.  The host queues each round without waiting for the GPU  */
/* and runs at most two rounds ahead of it.  Requests that arrive while       */
/* others run join at the next round.  A result does not depend on what else  */
/* was resident (same per-node arithmetic as a single handle).               */
/* ------------------------------------------------------------------------ */
typedef struct wave2d_server *wave2d_server_t;

typedef struct {
    int32_t nx, ny, scheme, flags; /* flags: WAVE2D_CONVENTIONAL, WAVE2D_ALLOW_UNSTABLE        */
    double h, tau, c;
    int64_t steps;                 /* two-steps after the first step (levels = steps + 1)    */
    const double *u0, *v0;         /* host FP64 nx*ny initial data (copied at submit), or     */
                                   /* both NULL for the Gaussian pulse below                 */
    double pulse_amp, pulse_cx, pulse_cy, pulse_sigma; /* u0 = amp exp(-|x-c|^2/(2 sigma^2)),
                                      v0 = 0, nodes at x = ((i+1) h, (j+1) h)               */
    double *out_field;             /* optional host buffer of nx*ny doubles that receives the
                                      final level; must stay valid until its completion is
                                      polled                                               */
    uint64_t tag;                  /* returned in the completion                             */
} wave2d_request;

typedef struct {
    uint64_t tag;
    int32_t status;                /* WAVE2D_OK, or the error of a step that failed for this
                                      request: its l2 / linf are NaN and its levels are not
                                      counted in node_updates                              */
    int32_t reserved;
    double l2, linf;               /* FP64 sqrt(sum u^2) and max |u| of the final level      */
    int64_t k;                     /* index of the final level                              */
    double t_submit, t_admit, t_done; /* library steady clock, seconds                       */
} wave2d_completion;

typedef struct {
    int64_t submitted, completed, queued, node_updates, rounds, used_bytes;
    int32_t max_resident_seen, reserved;
    double gpu_busy_s;             /* device time of the rounds (CUDA events around each
                                      round's work on the server stream), seconds        */
} wave2d_server_stats_t;

/* Device bytes a handle of this size and type holds (the admission cost). */
int64_t wave2d_required_bytes(int nx, int ny, int dtype);

/* Start a server on the current device.  budget_bytes: device memory that
 * resident simulations may hold (their handles, wave2d_required_bytes each;
 * the transient FP64 initial data of a round's pulse requests, 16 nx ny bytes
 * each, and the batch tables are allocated on top of it for the duration of
 * the round); max_resident: slot limit; quantum: two-steps per round; opt
 * (may be NULL): kernel of the batched runs (WAVE2D_KERNEL_STREAM, the
 * default, or WAVE2D_KERNEL_TEMPORAL), temporal_t (1..4 levels per launch)
 * and tile_h (strip rows 8..1024 for streaming, else chosen per round as the
 * tallest of 64, 32, 16 that gives a full wave of warps; 32 | 64 for
 * regions); stream: cudaStream_t to use, NULL = a new one.
 * Failures: a request whose step fails is completed with that status.  A
 * failed allocation of a round's initial-data staging fails that round's
 * pulse requests with WAVE2D_ERR_OOM and the server keeps serving; a CUDA
 * error also latches a server-wide error that poll and drain return. */
int wave2d_server_create(int64_t budget_bytes, int max_resident, int quantum, const wave2d_tune *opt,
                         void *stream, wave2d_server_t *out);

/* Queue a request (thread-safe).  Errors: WAVE2D_ERR_ARG (bad request),
 * WAVE2D_ERR_UNSTABLE, WAVE2D_ERR_OOM (larger than the whole budget),
 * WAVE2D_ERR_STATE (server shutting down). */
int wave2d_server_submit(wave2d_server_t s, const wave2d_request *r);

/* Move up to max completions to out (thread-safe, non-blocking). */
int wave2d_server_poll(wave2d_server_t s, wave2d_completion *out, int max, int *n_out);

/* Wait until every submitted request has completed (WAVE2D_ERR_TIMEOUT
 * after timeout_s seconds). */
int wave2d_server_drain(wave2d_server_t s, double timeout_s);

int wave2d_server_stats(wave2d_server_t s, wave2d_server_stats_t *st);

/* Finish all queued and running requests, then stop the scheduler. */
void wave2d_server_destroy(wave2d_server_t s);

/* Number of kernels the library has launched in this process (graph
 * launches count every kernel node).  For launch accounting in benchmarks. */
int64_t wave2d_launch_count(void);

/* Stability limit of a scheme (conventional = 1 for the comparison scheme). */
double wave2d_lambda_max(int scheme, int conventional);

/* Arithmetic throughput of the current device, measured: the denominators of
 * the ALU rooflines of this library's kernels (the paper has no counterpart;
 * it is a measurement service).  Every field except sms and clock_khz is in
 * lane operations per second, one lane operation being one add or one fused
 * multiply-add of one lane (a packed f32x2 FMA counts two): many independent
 * chains per thread, 4 blocks of 512 threads per SM, best of 5 timed
 * launches after 3 warm-ups (CUDA events on `stream`, NULL = default
 * stream; the call synchronises it).  Allocates a small scratch buffer
 * through the allocator hook for the duration of the call. */
typedef struct {
    double fp32_fma;   /* scalar FP32 fused multiply-add                    */
    double fp32_fma2;  /* packed fma.rn.f32x2 (the temporal kernels' form)  */
    double fp32_add;   /* scalar FP32 add                                   */
    double fp64_fma;   /* FP64 fused multiply-add                           */
    int32_t sms;       /* streaming multiprocessors                         */
    int32_t clock_khz; /* the device's maximum SM clock attribute           */
} wave2d_alu_peaks_t;
int wave2d_alu_peaks(wave2d_alu_peaks_t *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* WAVE2D_H */
