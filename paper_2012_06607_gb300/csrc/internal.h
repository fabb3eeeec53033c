// Host-side descriptors passed from the C ABI layer to the templated launchers.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace mdk {

enum : int { ST_SINGULAR = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

// Virtual lanes of the CTA-level row reductions, and threads of the
// Householder-vector block (kernels.cuh, house_fx.cuh).
constexpr int kRowLanes = 128;
constexpr int kHouseThreads = 128;

// Limb counts from which the factorisation chain (QR, R^-1, W, the finish of
// r_k and dx_k = W r_k) runs in W-word fixed point, and from which the
// split-product form puts the series products (and the batched form's update
// sums) on 32-bit word slices.  The md forms' cost grows as K^2 and the
// fixed-point forms' fixed part (conversions, renormalisation, values passed
// through the call stack) does not shrink with K: on GB300 double double is
// faster in md arithmetic in every phase (the n = 64, d = 64 step 10.9 ms in
// md against 13.8 ms with the fixed-point chain; series products 0.64x in
// fixed point), and from three limbs on the fixed-point forms are faster
// (products 2.2x at K = 3, 3.9x at K = 10).
constexpr int kFxMinLimbs = 3;
constexpr int kFxConvMinLimbs = 3;

// 32-bit words of one value of the split-product form's fixed-point pool:
// packed_words(words_for(K)) of conv_fx.cuh, for the host's workspace layout.
__host__ __device__ constexpr int fx_packed_words_for(int K) { return ((53 * K + 31) / 32 + 2 + 4) & ~3; }

// Kernel classes for the optional per-launch timing (md_profile_*).
enum ProfKind : int {
  PK_POOL = 0, PK_SCAL, PK_CONV, PK_ACCUM, PK_QR_HOUSE, PK_QR_APPLY, PK_RINV, PK_BACKSUB,
  PK_RHS_PARTIAL, PK_RHS_FINISH, PK_WMV, PK_FINISH, PK_ELEMENTWISE, PK_SERIES, PK_OZ_SPLIT, PK_OZ_UPDATE,
  PK_LU, PK_COUNT
};
bool prof_enabled();
int prof_begin(int kind, cudaStream_t s);
void prof_end(int id, cudaStream_t s);

struct ProfScope {
  int id;
  cudaStream_t s;
  ProfScope(int kind, cudaStream_t st) : id(prof_enabled() ? prof_begin(kind, st) : -1), s(st) {}
  ~ProfScope() {
    if (id >= 0) prof_end(id, s);
  }
};

// Lanes targeted by one split launch: 152 SMs x 4 sub-partitions x 2 warps x 32.
constexpr int kTargetLanes = 152 * 4 * 2 * 32;

struct EvalDev {
  int n = 0, d = 0, nmono = 0;
  int N = 0;  // polynomials (rows of f and A), N >= n
  const double *x = nullptr;
  double *f = nullptr;
  double *A = nullptr;
  const double *coef = nullptr;
  const double *cst = nullptr;
  double *pool = nullptr;
  double *scal = nullptr;
  const int *tasks = nullptr;
  const int *stage_off = nullptr;  // HOST array, nstages + 1 entries
  int nstages = 0;
  const int *scal_src = nullptr;
  int nscal = 0;
  const int *tasks0 = nullptr;      // coefficient-0 tasks (single jobs), stage-major
  const int *stage_off0 = nullptr;  // HOST array, nstages + 1 entries
  int resident_ctas = 0;            // > 0: run the full stages on this many SM-filling CTAs
  int resident_smem = 0;            // dynamic shared memory those CTAs reserve (keeps other CTAs off their SMs)
  int split = 0;                    // series products in fixed point (the split-product form), K >= 3
  unsigned *fxpool = nullptr;       // with split: the pool's values in packed fixed point (conv_fx.cuh)
  unsigned *fxscal = nullptr;       // with split: the scaled coefficients, packed
  unsigned *fxprod = nullptr;       // with split: the contribution values [ncontrib][d+1], packed
  const int *groups = nullptr;
  int ngroups = 0;
  const int *contrib = nullptr;
  int ncontrib = 0;
  double *prod = nullptr;  // contribution values, AoS [ncontrib][d+1]
};

struct SolveDev {
  int n = 0, d = 0;
  int N = 0;                  // rows of A_0 (N >= n; N > n: least squares)
  const double *A = nullptr;  // caller layout [P][K][d+1][n][N]
  const double *b = nullptr;  // caller layout [P][K][N][d+1]
  double sgn = 1.0;           // r_k = sgn * b_k - ...
  double *dx_out = nullptr;   // caller layout, may be null
  double *x = nullptr;        // x += dx when not null
  double *nrm = nullptr;      // device double[2] or null
  double *M = nullptr, *Y = nullptr, *W = nullptr;
  double *vd = nullptr, *beta = nullptr, *rinv = nullptr;
  double *r = nullptr, *dxw = nullptr, *part = nullptr;
  int *status = nullptr;
  int maxchunk = 1;
  int lu = 0;                 // factor A_0 by LU with partial pivoting instead of QR
  double *rcond = nullptr;    // rcond kernel output (device double)
  // split-product form (ozaki != 0)
  int ozaki = 0;
  void *oz_As = nullptr, *oz_Xs = nullptr;  // bf16 slices
  int *oz_eA = nullptr, *oz_ex = nullptr;
  unsigned long long *oz_acc = nullptr;     // fixed-point accumulators, n P outputs
};

// Terms j*n + col (j < k) of one of the N rows of r_k, cut into nchunk
// chunks of C so that N * nchunk is about kTargetLanes.
__host__ __device__ inline void rhs_chunking(int N, int n, int k, int &C, int &nchunk) {
  const long long terms = (long long)k * n;
  if (terms == 0) {
    C = 1;
    nchunk = 0;
    return;
  }
  long long c = (terms * N + kTargetLanes - 1) / kTargetLanes;
  if (c < 1) c = 1;
  C = (int)c;
  nchunk = (int)((terms + c - 1) / c);
}

// Stamps per system of the batched form with phase times: start, then after
// loading x, the series products, the accumulation of f and A, the QR set-up,
// the Householder QR, the reciprocals of R's diagonal, W = R^-1 Q^H and the
// degree loop, then the end.  Without phase times: start and end.
constexpr int kPhaseStamps = 10;

// Largest limb count of the batched form (larger ones use the per-system step).
constexpr int kBatchMaxLimbs = 5;

// One system of a batched step (offsets into the batch workspace).
struct BatchJob {
  int n, d, nstages, ngroups;
  int nscal, nmono, nops, pad;
  long long ops;        // ibase offset: 3 ints per product (out, a, b), stage-major
  long long stage_off;  // ibase offset: nstages+1 product offsets
  long long scal_src;   // ibase offset: 2 ints per scaling entry
  long long groups;     // ibase offset: 4 ints per group (16-byte aligned)
  long long contrib;    // ibase offset: 4 ints per contribution (16-byte aligned)
  long long pool, scal, f, A, M, Y, W, vd, beta, rinv, r, dxw, part;  // dbase offsets (doubles)
  // the split-product form's packed fixed-point copies of the pool, A and dx
  // (dbase offsets in doubles, 16-byte aligned; laid out only for that form)
  long long fxpool, fxA, fxdx, fxscal;
  const double *coef;
  const double *cst;
  double *x;
};

struct BatchDev {
  const BatchJob *jobs = nullptr;
  const int *order = nullptr;
  int njobs = 0;
  int *counter = nullptr;
  const int *ibase = nullptr;
  double *dbase = nullptr;
  double *nrm = nullptr;
  unsigned long long *times = nullptr;
  int *status = nullptr;
  int update_x = 1;
  int grid = 1;
  int threads = 128;
  int ctas_per_sm = 0;      // > 0: dynamic shared memory lets at most this many CTAs share an SM
  int *resident = nullptr;  // if set, every CTA adds 1 here when it starts
  int times_stride = 2;     // stamps per system in times: 2 or kPhaseStamps
  int split = 0;            // series products in fixed point (MD_FLAG_OZAKI), K >= 3
};

template <int K, int P>
struct Impl {
  static cudaError_t batched(const BatchDev &b, cudaStream_t s);
  static cudaError_t batched_setup();  // shared-memory attributes of the batched kernel (outside stream capture)
  static cudaError_t elementwise(int op, long long count, const double *x, const double *y, double *z,
                                 cudaStream_t s);
  static cudaError_t series_conv(int d, long long count, const double *x, const double *y, double *z,
                                 cudaStream_t s);
  static cudaError_t eval(const EvalDev &e, cudaStream_t s);
  static cudaError_t eval0(const EvalDev &e, cudaStream_t s);      // prologue + coefficient 0 of f, A
  static cudaError_t eval_rest(const EvalDev &e, cudaStream_t s);  // all products, coefficients >= 1
  static cudaError_t solve(const SolveDev &v, cudaStream_t s);
  static cudaError_t factor(const SolveDev &v, cudaStream_t s);    // QR, Q^H, W = R^-1 Q^H
  static cudaError_t degrees(const SolveDev &v, cudaStream_t s);   // degree loop and update
  static cudaError_t rcond(const SolveDev &v, cudaStream_t s);     // 1-norm rcond of A_0 from A_0 and W
  static cudaError_t backsub(const SolveDev &v, int N, cudaStream_t s);  // W = R^-1 Y[0:n, :]
};

}  // namespace mdk
