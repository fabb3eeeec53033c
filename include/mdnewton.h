/*
 * mdnewton.h -- C ABI of the GB300 library for the power-series Newton step
 * in multiple-double arithmetic (Verschelde, "Parallel Software to Offset the
 * Cost of Higher Precision", arXiv 2012.06607).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Numbers.  A multiple-double (md) number is an unevaluated sum of K doubles,
 *   K = limbs in {1, 2, 3, 4, 5, 8, 10} (double, double double, triple, quad,
 *   penta, octo, deca double; Section 2).  Complex numbers have two planes
 *   (P = 2: real part, imaginary part); real ones one plane (P = 1).
 * Layouts (structure of arrays, limbs outermost; all row-major C indices):
 *   md array of count values .......... [P][K][count]
 *   series vector (n series, degree d)  [P][K][n][d+1]    coefficient fastest
 *   matrix series A_0..A_d ............ [P][K][d+1][n][n] each A_k column-major:
 *                                       element (row r, col c) of A_k at
 *                                       [p][l][k][c][r]
 * Memory.  "device" pointers are CUDA global memory owned by the caller; "host"
 *   pointers are host memory owned by the caller.  The library allocates no
 *   device memory: every call that needs scratch space takes a caller-owned
 *   device workspace `ws` of at least the queried number of bytes, 256-byte
 *   aligned.  A workspace must not be shared by calls that may run
 *   concurrently.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls enqueue work and return without synchronising, except
 *   where stated.  Argument errors are returned synchronously; errors found on
 *   the device (singular A_0, non-finite results) set a sticky word inside the
 *   workspace, read with md_get_device_status().
 * Threads.  Entry points are re-entrant for distinct workspaces.
 */
#ifndef MDNEWTON_H
#define MDNEWTON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum md_status {
  MD_OK = 0,
  MD_ERR_ARG = 1,         /* invalid argument (sizes, limbs, pointers, system)  */
  MD_ERR_WORKSPACE = 2,   /* workspace NULL, misaligned or too small            */
  MD_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed        */
  MD_ERR_SINGULAR = 4,    /* A_0 is singular (a Householder column norm is 0)   */
  MD_ERR_NONFINITE = 5,   /* an update contains Inf or NaN                      */
  MD_ERR_NOCONV = 6,      /* reserved for drivers that iterate to a tolerance   */
  MD_ERR_TIMEOUT = 7,     /* a bounded device wait ran out (md_wait_selftest, the
                             batched form's placement gate; results unaffected) */
  MD_ERR_UNSUPPORTED = 8, /* valid request this build does not implement        */
  MD_ERR_CHECK = 9        /* MD_FLAG_CHECK: a plan table or layout out of bounds */
} md_status;

/* Maximum number of (variable, exponent) pairs per monomial. */
#define MD_MAXV 4

/*
 * A polynomial system f(x) = 0 of N polynomials in the n unknowns
 * x_0..x_{n-1} and the series parameter t, which has variable index n
 * (Section 4: systems with one more variable than equations have power series
 * solutions; t is the extra variable).  N = n unless neq > n: then the linear
 * systems of every Newton step are solved in the least squares sense with the
 * QR of the N x n matrix A_0 (Section 4, N > n).  Polynomial i is
 * cst[i] + sum over its monomials m in [poly_ptr[i], poly_ptr[i+1]) of
 * coef[m] * prod_q var(idx[m][q])^expo[m][q].
 *
 *   structure (HOST pointers, read during the call):
 *     poly_ptr [N+1]            CSR offsets, poly_ptr[0] = 0, poly_ptr[N] = nmono
 *     nvar     [nmono]          number of used pairs, 0..MD_MAXV
 *     idx      [nmono*MD_MAXV]  distinct variable indices in 0..n (n = t)
 *     expo     [nmono*MD_MAXV]  exponents >= 1 for the used pairs
 *   values (DEVICE pointers):
 *     coef     [P][K][nmono]    monomial coefficients
 *     cst      [P][K][N]        constant terms
 *   neq: N (0 means N = n; otherwise N >= n).  N > n is not available with
 *        MD_FLAG_LU (MD_ERR_ARG), MD_FLAG_OZAKI or the batched form
 *        (MD_ERR_UNSUPPORTED).
 */
typedef struct md_system {
  int limbs;
  int is_complex;
  int n;
  int degree;
  int nmono;
  const int *poly_ptr;
  const int *nvar;
  const int *idx;
  const int *expo;
  const double *coef;
  const double *cst;
  int neq;
} md_system;

/* flags */
#define MD_FLAG_PLAIN 0x0 /* plain multiple-double kernels for every step        */
/*
 * Split-product form.
 *   - The block Toeplitz update r_k = b_k - sum_j A_{k-j} dx_j: every md number
 *     of a row of A_i (and of dx_j) is cut into signed 8-bit integer slices
 *     relative to a shared power of two; all slice products are exact BF16
 *     tensor-core products with exact fp32 accumulation (K <= 1024 per
 *     product), and the terms of r_k are added exactly in a fixed-point integer
 *     before one conversion to K limbs.  Error: 2^(12 - 8S) of the largest term
 *     (S slices per number, 8S >= 53K + 24 bits).  Needs the larger workspace
 *     reported for this flag.
 *   - In md_newton_series_step, the series products of the evaluation
 *     (K >= 3): each term on 32-bit word slices of the md operands, exact word
 *     products and column sums, the coefficient kept in W-word fixed point
 *     (53K bits and two guard words) and rounded to K limbs once; and the
 *     accumulation of f and A_k the same way (each contribution an exact
 *     word-slice product, each entry's sum rounded once).  A_0 still comes
 *     from the md products and sums of coefficient 0.
 *   - In md_newton_series_step_batched (K >= 3), the same series products and
 *     accumulation and, in place of the 8-bit slices above, the chunk sums of
 *     the block Toeplitz update on 32-bit word slices, each chunk rounded to
 *     K limbs once.
 * Non-finite values propagate as in md arithmetic (an output with a
 * non-finite input limb is NaN).  At one and two limbs the flag leaves the
 * series products in md arithmetic, which is faster there.  Results are within the plain form's tolerance, not
 * its bits.  (In every form, from three limbs on, the QR of A_0,
 * W = R^-1 Q^H, the finish of r_k and dx_k = W r_k run in the same W-word
 * fixed point.)
 */
#define MD_FLAG_OZAKI 0x1
/* batched form: pick threads per CTA and CTAs per SM per precision class, and
   the threads of the whole-SM CTAs, by timing trial steps (first call only;
   trial steps do not update x).
   single step (md_newton_series_step, without MD_FLAG_SERIAL): pick how many
   SMs the factorisation of A_0 keeps while the evaluation runs, per plan and
   form: after one untimed call, the next 14 calls outside a stream capture
   each time one of seven counts (4 to 48; events on the caller's stream,
   read later without waiting), and once all are read the fastest is kept
   (md_plan_factor_sms reports it).  Results do not depend on it; calls
   before then use the default (4). */
#define MD_FLAG_AUTOTUNE 0x2
/* batched form: capture the step (plan upload + persistent launches) in a CUDA
   graph on the first call and replay it on later calls with the same arguments
   (needs a non-default stream) */
#define MD_FLAG_GRAPH 0x4
/* single-system step: run every phase on `stream` in order.  By default the
   factorisation of A_0 runs on a second (library-owned, highest-priority)
   stream on a few SMs while the higher coefficients are evaluated on the rest;
   results are identical either way.  Batched form: no whole-SM systems (every
   launch on `stream`, see md_newton_series_step_batched); results are
   identical either way. */
#define MD_FLAG_SERIAL 0x8
/* factor A_0 by LU with partial pivoting (Section 4: for N = n "an LU
   factorization can be applied") instead of Householder QR.  Pivot: the first
   row of largest |re| + |im| of the leading limbs; multipliers by the
   reciprocal of the pivot.  Single-system calls only (the batched form
   returns MD_ERR_UNSUPPORTED). */
#define MD_FLAG_LU 0x10
/* batched form: `times` holds MD_PHASE_STAMPS global-timer stamps per system
   instead of 2: the start of its step, then the end of each phase -- x loaded
   and coefficients scaled, series products, accumulation of f and A, QR
   set-up, Householder QR, reciprocals of R's diagonal, W = R^-1 Q^H, degree
   loop -- and the end (x updated).  Adds a few barriers per system. */
#define MD_FLAG_PHASE_TIMES 0x20
#define MD_PHASE_STAMPS 10
/* Bounds mode: before any launch, check on the host every index the kernels
   follow from the plan's tables and the workspace layout: each product's
   operands are series made before it, and each product and coefficient index
   is in range. Each accumulation group and contribution points inside its
   tables, and every workspace region lies in order within the workspace.
   Failure returns MD_ERR_CHECK without device work.  The kernels compute
   every other address from (N, n, d, K, P).  Costs one pass over the tables
   per call. */
#define MD_FLAG_CHECK 0x40

/* Version of this ABI (major*100 + minor). */
int md_version(void);

/* Human-readable name of a status code (static string). */
const char *md_status_string(md_status st);

/*
 * Workspace bytes needed by md_eval_diff / md_newton_series_step for `sys`
 * (reads only the host structure arrays).  Returns 0 if `sys` is invalid.
 */
size_t md_workspace_bytes(const md_system *sys, int flags);

/* Workspace bytes needed by md_linsolve_series. */
size_t md_linsolve_workspace_bytes(int limbs, int is_complex, int n, int degree, int flags);

/*
 * Elementwise md arithmetic on `count` values (Section 2, Table 1 operations).
 *   op: 0 add (z = x + y), 1 sub (z = x - y), 2 mul, 3 div, 4 sqrt (real only,
 *       y unused), 5 multiply by a double (y: DEVICE double[count]).
 *   x, y, z: DEVICE [P][K][count] (z may alias x or y).
 * Results are identical to a sequential evaluation of the same operation
 * sequence in IEEE binary64 round-to-nearest (see the library's design notes
 * for the algorithms).
 */
md_status md_elementwise(int op, int limbs, int is_complex, long long count, const double *x, const double *y,
                         double *z, void *stream);

/*
 * Products of `count` pairs of truncated power series (Section 3):
 * z_k = sum_{i=0..k} x_i y_{k-i}, k = 0..degree, summed in ascending i.
 *   x, y, z: DEVICE [P][K][count][degree+1]; z must not alias x or y.
 */
md_status md_series_conv(int limbs, int is_complex, int degree, long long count, const double *x, const double *y,
                         double *z, void *stream);

/*
 * Evaluate and differentiate the system at the series vector x (Section 4):
 *   f[i](t)   = f_i(x(t), t) truncated at degree d,
 *   A_k[i][j] = coefficient k of d f_i / d x_j (x(t), t),  j < n (no t column).
 *   x: DEVICE [P][K][n][d+1]     input series
 *   f: DEVICE [P][K][N][d+1]     output
 *   A: DEVICE [P][K][d+1][n][N]  output (column-major N x n blocks)
 *   ws: DEVICE workspace of md_workspace_bytes(sys, 0) bytes.
 * Monomials are evaluated with Speelpenning products (value and all partials
 * at about three times the cost of the value); every sum is taken in the order
 * of the definition, so f and A are the same bits on every run.
 */
md_status md_eval_diff(const md_system *sys, const double *x, double *f, double *A, void *ws, size_t ws_bytes,
                       void *stream);

/*
 * Solve the lower triangular block Toeplitz system A(t) dx(t) = b(t) of
 * Section 4: A_0 dx_k = b_k - sum_{j<k} A_{k-j} dx_j, k = 0..d, with a
 * Householder QR of A_0.
 *   A : DEVICE [P][K][d+1][n][n]  (read only)
 *   b : DEVICE [P][K][n][d+1]
 *   dx: DEVICE [P][K][n][d+1]     output
 *   ws: DEVICE workspace of md_linsolve_workspace_bytes(...) bytes.
 * A singular A_0 sets MD_ERR_SINGULAR in the workspace status word.
 */
md_status md_linsolve_series(int limbs, int is_complex, int n, int degree, const double *A, const double *b,
                             double *dx, void *ws, size_t ws_bytes, int flags, void *stream);

/*
 * The same for an N x n A_0 with N >= n equations (Section 4: for N > n the
 * linear systems are solved in the least squares sense, with QR): per degree
 * dx_k minimises ||A_0 dx_k - r_k||_2, r_k = b_k - sum_{j<k} A_{k-j} dx_j,
 * through dx_k = R^-1 (Q^H r_k)[0:n].
 *   A : DEVICE [P][K][d+1][n][N]  (read only, column-major N x n blocks)
 *   b : DEVICE [P][K][N][d+1]
 *   dx: DEVICE [P][K][n][d+1]     output
 *   ws: DEVICE workspace of md_lstsq_workspace_bytes(...) bytes (0 = invalid).
 * neq < n is MD_ERR_ARG; with neq > n, MD_FLAG_LU is MD_ERR_ARG and
 * MD_FLAG_OZAKI is MD_ERR_UNSUPPORTED.  md_linsolve_series is neq = n.
 */
size_t md_lstsq_workspace_bytes(int limbs, int is_complex, int neq, int n, int degree, int flags);
md_status md_lstsq_series(int limbs, int is_complex, int neq, int n, int degree, const double *A, const double *b,
                          double *dx, void *ws, size_t ws_bytes, int flags, void *stream);

/*
 * One Newton step on truncated power series (Section 4): x <- x + dx where
 * A(t) dx(t) = -f(x(t)).
 *   x:       DEVICE [P][K][n][d+1], updated in place
 *   dx_norm: DEVICE double[2] or NULL: [0] = max_i |dx_{d,i}| (the size of
 *            the update of the degree-d coefficient, the convergence measure
 *            of Section 6), [1] = max over all coefficients; both from the
 *            leading limbs.
 *   ws:      DEVICE workspace of md_workspace_bytes(sys, flags) bytes.
 *   flags:   MD_FLAG_OZAKI, MD_FLAG_LU, MD_FLAG_SERIAL, MD_FLAG_CHECK,
 *            MD_FLAG_AUTOTUNE
 */
md_status md_newton_series_step(const md_system *sys, double *x, double *dx_norm, void *ws, size_t ws_bytes,
                                int flags, void *stream);

/*
 * One Newton step for each of `nsys` independent systems (uneven n, degree and
 * precision), as in md_newton_series_step, in one persistent launch per
 * precision class: each CTA takes the next system from an atomic job counter
 * (most expensive first) and runs its whole step; there are no waits between
 * CTAs.  Every system gets the same bits as md_newton_series_step on it alone.
 * The classes run one after another; a class runs at most a set number of
 * CTAs per SM (autotuned, else 2).  When that number is above one, the
 * systems of the first class whose step on a shared SM would outlast an even
 * share of the batch over the SMs each run in a CTA that holds a whole SM, on
 * `stream`, while the others share the remaining SMs from a second
 * (library-owned) stream that `stream` waits for.
 *   sys:     HOST array of nsys systems (structure host, values device)
 *   x:       HOST array of nsys DEVICE pointers, each [P][K][n][d+1], updated
 *   dx_norm: DEVICE double[nsys][2] or NULL (per system, as in the single step)
 *   times:   DEVICE unsigned long long[nsys][2] or NULL: global-timer
 *            nanoseconds at the start and end of each system's step
 *            ([nsys][MD_PHASE_STAMPS] with MD_FLAG_PHASE_TIMES)
 *   ws:      DEVICE workspace of md_batched_workspace_bytes(nsys, sys, flags)
 *            bytes (MD_FLAG_OZAKI adds fixed-point copies of the series pool,
 *            A and dx for systems of three or more limbs); the status word
 *            covers the whole batch
 *   flags:   MD_FLAG_AUTOTUNE, MD_FLAG_GRAPH, MD_FLAG_SERIAL, MD_FLAG_PHASE_TIMES,
 *            MD_FLAG_CHECK, MD_FLAG_OZAKI (series products and update sums on
 *            32-bit word slices; the bit-equality with md_newton_series_step
 *            holds for the plain form).  The two forms keep separate plans,
 *            tunings and graphs.
 */
size_t md_batched_workspace_bytes(int nsys, const md_system *sys, int flags);
md_status md_newton_series_step_batched(int nsys, const md_system *sys, double *const *x, double *dx_norm,
                                        unsigned long long *times, void *ws, size_t ws_bytes, int flags,
                                        void *stream);

/*
 * The bounds mode's checks of MD_FLAG_CHECK on the plan of one system, host
 * only (no device work): MD_OK, MD_ERR_CHECK, or MD_ERR_ARG for an invalid
 * system.  flags: MD_FLAG_OZAKI selects that form's workspace layout.
 */
md_status md_plan_check(const md_system *sys, int flags);

/*
 * Host-side cost estimate of each system's Newton step: the estimate the
 * batched form orders its job queue by (most expensive first) and the one to
 * partition a batch across GPUs by (longest processing time first).  It
 * counts multiply-adds: series products (d+1)(d+2)/2 per product, 2 n^3 for
 * the QR and W, n^2 d (d+1)/2 for the block Toeplitz update, one per
 * coefficient and contribution for the accumulation; times K^2, and times 4
 * for complex.  Host only (no device work); plans structures not seen before.
 *   cost: HOST double[nsys], written
 * Returns MD_ERR_ARG for nsys < 1, NULL pointers or an invalid system (cost
 * is then unspecified).
 */
md_status md_batched_job_costs(int nsys, const md_system *sys, double *cost);

/*
 * Synchronise `stream`, read the sticky device status word of `ws` (written by
 * the calls above that used this workspace), clear it and return it
 * (MD_OK, MD_ERR_SINGULAR, MD_ERR_NONFINITE or MD_ERR_TIMEOUT, in that order
 * of precedence).  MD_ERR_TIMEOUT from a batched step means that its
 * placement gate (a one-thread kernel waiting, at most about 0.1 s, until the
 * whole-SM CTAs are resident) gave up: the step's results are unaffected, only
 * the order in which CTAs were placed was not enforced.
 */
md_status md_get_device_status(void *ws, void *stream);

/*
 * Failure-detection check of the library's one bounded device wait (no
 * counterpart in the paper).  Clears the first 256 bytes of `ws` (the status
 * word and the batched form's counters) and runs the batched form's placement
 * gate on `stream` against a counter there that nothing increments, with the
 * given target.  target = 0: the wait ends at once, the status stays MD_OK.
 * target >= 1: the wait runs out after about 0.1 s and sets the timeout bit,
 * so that md_get_device_status(ws, stream) returns MD_ERR_TIMEOUT.  The
 * context stays usable either way.
 *   ws: DEVICE, >= 256 bytes, 256-byte aligned (MD_ERR_WORKSPACE otherwise).
 * Errors: MD_ERR_ARG (target < 0), MD_ERR_WORKSPACE, MD_ERR_CUDA.
 */
md_status md_wait_selftest(void *ws, size_t ws_bytes, int target, void *stream);

/*
 * Allocation-free block Toeplitz solve.  The paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory for a workspace
 * -- applications whose device memory belongs to another allocator or is
 * reserved up to the limit, latency-critical code where cudaMalloc/cudaFree
 * would synchronise the device, plug-in or callback contexts that forbid
 * allocation.
 *
 * Same computation, arguments and layouts as md_linsolve_series, without `ws`:
 * the scratch space is a static device array of MD_STATIC_WS_BYTES (16 MiB)
 * inside the library, which every GPU that loads the library holds until the
 * process exits.  Requests whose md_linsolve_workspace_bytes() exceeds it are
 * rejected with MD_ERR_WORKSPACE before any device work (16 MiB holds, e.g.,
 * n = 64, d = 64 in quad double complex).  The call allocates nothing.
 *   - The array is claimed on a device when the CUDA runtime loads the
 *     library's module there.  With lazy module loading (the default since
 *     CUDA 12.2) that can be this entry point's first call on the device,
 *     which then returns MD_ERR_CUDA if the device has no 16 MiB left.  Callers
 *     that reserve device memory up to the limit should make one call (or set
 *     CUDA_MODULE_LOADING=EAGER) before reserving the rest.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it; make that
 *     first call before any stream capture on the device.  The address belongs
 *     to the context current at that call (the runtime's primary context of
 *     the device); after cudaDeviceReset, or from another context on the same
 *     device, do not call this entry point again in the same process.
 *   - Every call on a device shares the one array and it keeps the last call's
 *     contents; calls whose work may overlap on the GPU (different streams,
 *     host threads) race on it and must be serialised by the caller.
 *   - The device status word lives in that array too, so device-detected
 *     conditions (singular A_0) are not readable through
 *     md_get_device_status; a singular A_0 (QR: a zero Householder column
 *     norm; LU: a zero pivot) shows as non-finite entries of dx, because the
 *     reciprocal of the zero pivot spreads into every later column.
 */
#define MD_STATIC_WS_BYTES (16u << 20)
md_status md_linsolve_series_static(int limbs, int is_complex, int n, int degree, const double *A, const double *b,
                                    double *dx, int flags, void *stream);

/*
 * Reciprocal condition number of A_0 in the 1-norm, 1 / (||A_0||_1 ||A_0^-1||_1)
 * (Section 6 quotes such an estimate, 4.6E-6, for the cyclic 128-roots
 * system).  The solve forms A_0^-1 = R^-1 Q^H (or U^-1 L^-1 P) explicitly, so
 * the value is that of the computed inverse, from the moduli of the leading
 * limbs summed in double.  It reads the factorisation left in the workspace:
 *   md_rcond_a0:       after md_newton_series_step(sys, ..., ws, ..., flags)
 *                      (A_0 of that step's linearisation);
 *   md_linsolve_rcond: after md_linsolve_series(limbs, ..., A, ..., ws, ...)
 *                      with the same A.
 *   rcond: DEVICE double, written on `stream` (no synchronisation).
 * Errors: MD_ERR_ARG, MD_ERR_WORKSPACE, MD_ERR_CUDA.
 */
md_status md_rcond_a0(const md_system *sys, void *ws, size_t ws_bytes, int flags, double *rcond, void *stream);
md_status md_linsolve_rcond(int limbs, int is_complex, int n, int degree, const double *A, void *ws,
                            size_t ws_bytes, int flags, double *rcond, void *stream);
/* N x n A_0 after md_lstsq_series: 1 / (||A_0||_1 ||A_0^+||_1), A_0^+ the
   pseudo-inverse R^-1 (Q^H)[0:n, :] that the solve forms. */
md_status md_lstsq_rcond(int limbs, int is_complex, int neq, int n, int degree, const double *A, void *ws,
                         size_t ws_bytes, int flags, double *rcond, void *stream);

/*
 * Newton's method with degree continuation (the cyclic 128-roots experiment
 * of Section 6): levels l = 0..nlevels-1 at truncation degrees degree[l]
 * (nondecreasing, each <= sys->degree).  Level l runs Newton steps on the
 * coefficients 0..degree[l] of x, at most max_iter[l] of them, and stops as soon
 * as ||dx|| <= tol, where ||dx|| = max_i |dx_{degree[l],i}| is the size of the
 * update of the last coefficient (leading limbs).  The next level starts from
 * this level's series (its higher coefficients are those of x on entry).
 * After a level that ends with ||dx|| > too_large the ladder stops ("once the
 * update is too large for one degree, the next degrees are not computed"; the
 * paper gives no threshold, the caller does).
 *   sys:   the system at its largest degree D = sys->degree (coefficient arrays
 *          do not depend on the degree).
 *   x:     DEVICE [P][K][n][D+1], updated in place.
 *   sched: HOST schedule; rep: HOST report (may be NULL).
 *   ws:    DEVICE workspace of md_newton_run_workspace_bytes(sys, sched, flags).
 *   flags: as for md_newton_series_step.
 * The call waits for the GPU after every step (it reads ||dx|| to decide).
 * Errors: MD_ERR_ARG (bad schedule), MD_ERR_WORKSPACE, MD_ERR_SINGULAR /
 * MD_ERR_NONFINITE when a step's device status reports it (x then holds the
 * series after that step and rep, if given, the levels up to it), MD_ERR_CUDA.
 */
#define MD_MAX_LEVELS 16
typedef struct {
  int nlevels;                    /* 1..MD_MAX_LEVELS                         */
  int degree[MD_MAX_LEVELS];      /* truncation degree of each level          */
  int max_iter[MD_MAX_LEVELS];    /* at most this many steps per level (>= 1) */
  double tol;                     /* level converged when ||dx|| <= tol       */
  double too_large;               /* ladder stops after ||dx|| > too_large    */
} md_newton_schedule;

typedef struct {
  int levels_done;                /* levels run (the last may not have converged) */
  int converged;                  /* 1 if every level run ended with ||dx|| <= tol */
  int iterations[MD_MAX_LEVELS];  /* steps taken per level                        */
  double dx_norm[MD_MAX_LEVELS];  /* ||dx|| after the last step of each level     */
  double dx_max[MD_MAX_LEVELS];   /* max |dx| over all coefficients, same step    */
} md_newton_report;

size_t md_newton_run_workspace_bytes(const md_system *sys, const md_newton_schedule *sched, int flags);
md_status md_newton_series_run(const md_system *sys, double *x, const md_newton_schedule *sched,
                               md_newton_report *rep, void *ws, size_t ws_bytes, int flags, void *stream);

/*
 * Test hook of the plan cache (no counterpart in the paper).  The library
 * caches the product schedule of each system structure under a 64-bit hash of
 * the structure and, on a hit, compares the stored structure with the
 * caller's, so that a colliding structure gets its own plan.  To let tests
 * exercise that path, this narrows every structure hash to `mask` (so that
 * structures collide); 0 restores the full hash.  Results never depend on
 * it; only the cache's hit rate does.  Host only.
 */
void md_plan_cache_hash_mask(unsigned long long mask);

/*
 * The number of SMs the factorisation of A_0 keeps while the evaluation runs
 * (MD_FLAG_AUTOTUNE) in the cached plan of this system's structure and form
 * (MD_FLAG_OZAKI in flags selects the split-product form; no counterpart in
 * the paper).  Returns the tuned count once the tuning has ended, 0 while it
 * has not (the step then uses the default of 4), -1 when no plan of this
 * structure and form is cached (md_newton_series_step has not run on it) or
 * the structure is invalid.  Host only; results never depend on it.
 */
int md_plan_factor_sms(const md_system *sys, int flags);

/*
 * Optional timing of the library's own kernels (tracing support; not part of
 * the computation).  While enabled, every kernel launch of every call in this
 * process is bracketed by two CUDA events on its stream.
 *   md_profile_enable(1|0)   switch on / off (host only, no synchronisation).
 *   md_profile_read(ms, launches, nkinds): waits for the recorded events, adds
 *     their elapsed milliseconds and launch counts per kernel class into
 *     HOST arrays ms[nkinds], launches[nkinds] (either may be NULL), clears the
 *     record and returns the number of classes (or -1 if an event failed).
 *   md_profile_kind_name(k): static name of class k.
 */
void md_profile_enable(int on);
int md_profile_read(double *ms, long long *launches, int nkinds);
const char *md_profile_kind_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* MDNEWTON_H */
