// Series products in W-word fixed point: the evaluation of the split-product
// form (MD_FLAG_OZAKI).
//
// Coefficient k of z = x * y is sum_{i<=k} x_i y_{k-i} (Section 3).  Here
// every term is formed on 32-bit word slices of the md operands -- exact word
// products with exact 64-bit column sums (fixp.cuh) -- and the sum is kept in
// the same W-word format (53K bits and two guard words), then written back
// to K limbs once.  That is the split-product idea applied to the series
// products, on the integer multiplier: on GB300 the integer pipe retires ~30
// times the FP64 pipe's lanes per cycle, and a quad double complex
// multiply-add costs 712 FP64 instructions in md arithmetic.  The result is
// at least as accurate as the md form (one truncation to K limbs instead of
// a rounding in every operation) but not its bits: the split-product form is
// checked against the oracle by tolerance, the plain form keeps the bits.
#pragma once
#include "house_fx.cuh"

namespace mdk {

// Two output coefficients of series products as conv_pair (same task layout
// and term order), in fixed point.  The W-word operations are called out of
// line (inlined, they needed ~156 registers a thread and the kernel ran 25%
// slower at 384 threads than called at 512, despite the call stack's traffic).
template <int K, int P>
__device__ __forceinline__ void conv_pair_fx(double *pool, int d, int outA, int xA, int yA, int kA, int outB, int xB,
                                             int yB) {
  using namespace fxp;
  constexpr int W = words_for(K);
  const int kB = d - kA;
  const long long VS = P * K, SS = (long long)(d + 1) * VS;
  const int total = (outB >= 0) ? (d + 2) : (kA + 1);
  bf<W> acc[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = zero<W>();
  for (int it = 0; it < total; ++it) {
    const bool first = it <= kA;
    const int i = first ? it : it - kA - 1;
    const double *xp = pool + (first ? xA : xB) * SS + i * VS;
    const double *yp = pool + (first ? yA : yB) * SS + ((first ? kA : kB) - i) * VS;
    bf<W> a[P], b[P], t[P];
    fx_ld_val<W, K, P>(xp, a);
    fx_ld_val<W, K, P>(yp, b);
    fx_cmul<W, P>(a, b, t);
    if (it == kA + 1) {
#pragma unroll
      for (int p = 0; p < P; ++p) acc[p] = zero<W>();
    }
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = add<W>(acc[p], t[p]);
    if (it == kA) fx_st_val<W, K, P>(pool + outA * SS + kA * VS, acc);
  }
  if (outB >= 0) fx_st_val<W, K, P>(pool + outB * SS + kB * VS, acc);
}

// One chunk of a row of the block Toeplitz update sum_{j<k} A_{k-j} dx_j
// (Section 3.2; rhs_partial_item's terms in its order) in fixed point: every
// term an exact product of word slices, the chunk's sum rounded to K limbs
// once.  A: [P][K][d+1][n][N] (column-major blocks), dx: [d+1][n] values of
// P*K doubles, part: [N][nchunk] values.
template <int K, int P>
__device__ __forceinline__ void rhs_partial_item_fx(const double *A, const double *dx, double *part, int N, int n,
                                                    int d, int k, int C, int nchunk, long long e) {
  using namespace fxp;
  constexpr int W = words_for(K);
  const int row = (int)(e % N), chunk = (int)(e / N);
  const long long nn = (long long)N * n, VS = P * K, stride = (long long)(d + 1) * nn;
  const int t0 = chunk * C, t1 = min(t0 + C, k * n);
  bf<W> acc[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = zero<W>();
  for (int t = t0; t < t1; ++t) {
    const int j = t / n, col = t % n;
    const double *ap = A + (long long)(k - j) * nn + (long long)col * N + row;
    bf<W> a[P], x[P], prod[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      double v[K];
#pragma unroll
      for (int l = 0; l < K; ++l) v[l] = ap[(long long)(p * K + l) * stride];
      a[p] = from_md<W, K>(v);
    }
    fx_ld_val<W, K, P>(dx + ((long long)j * n + col) * VS, x);
    fx_cmul<W, P>(a, x, prod);
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = add<W>(acc[p], prod[p]);
  }
  fx_st_val<W, K, P>(part + ((long long)row * nchunk + chunk) * VS, acc);
}

// The resident stage launch of conv_stage_resident_kernel in fixed point
// (same grid and task numbering; ~90 registers a thread: 16 warps an SM).
template <int K>
__host__ __device__ constexpr int conv_fx_threads() {
  return 512;
}

template <int K, int P>
__global__ void __launch_bounds__(conv_fx_threads<K>(), 1)
    conv_stage_fx_kernel(const int *__restrict__ tasks, int ntask, double *pool, int d) {
  for (int t = threadIdx.x * gridDim.x + blockIdx.x; t < ntask; t += gridDim.x * blockDim.x) {
    const int4 t0 = __ldg(reinterpret_cast<const int4 *>(tasks) + 2 * t);
    const int4 t1 = __ldg(reinterpret_cast<const int4 *>(tasks) + 2 * t + 1);
    conv_pair_fx<K, P>(pool, d, t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z);
  }
}

}  // namespace mdk
