// Householder QR steps in W-word fixed-point arithmetic (fixp.cuh).
//
// Same steps as house_block / house_apply_col / house_apply_col_cta in
// kernels.cuh (Golub-Van Loan: alpha = ||x||, phase e = x_0/|x_0|,
// v = x + e alpha e_1, beta = 1/(alpha (alpha + |x_0|)), R_jj = -e alpha;
// t <- t - beta (v^H t) v), with every dot product, square root, reciprocal
// and update formed on multiword integer mantissas and converted back to K
// limbs once.  On GB300 an FP64 warp instruction costs ~64 cycles of its SM
// sub-partition and an integer one ~2, and these steps are latency-bound
// chains; their W-word arithmetic carries 53K bits and two guard words, so
// the results stay within the same tolerance (they are not the md forms'
// bits).
//
// Reductions run over fixed lane sets (a warp, or 128 virtual lanes of a
// CTA, rows assigned in order), so the result does not depend on how many
// threads run the body: the single-system kernels and the batched kernel get
// the same bits.
#pragma once
#include "fixp.cuh"
#include "internal.h"
#include "md.cuh"

namespace mdk {

template <int W>
__device__ __forceinline__ fxp::bf<W> fx_shfl_xor(const fxp::bf<W> &a, int off) {
  fxp::bf<W> o;
#pragma unroll
  for (int i = 0; i < W; ++i) o.m[i] = __shfl_xor_sync(0xffffffffu, a.m[i], off);
  o.e = __shfl_xor_sync(0xffffffffu, a.e, off);
  o.neg = __shfl_xor_sync(0xffffffffu, a.neg, off);
  return o;
}

// Sum over the 32 lanes of a warp (xor tree); every lane gets it.
template <int W>
__device__ __forceinline__ void fx_warp_sum(fxp::bf<W> &a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a = fxp::add<W>(a, fx_shfl_xor<W>(a, off));
}

template <int W, int K>
__device__ __forceinline__ fxp::bf<W> fx_ld(const double *src) {
  double v[K];
#pragma unroll
  for (int l = 0; l < K; ++l) v[l] = src[l];
  return fxp::from_md<W, K>(v);
}

template <int K, int W>
__device__ __forceinline__ void fx_st(double *dst, const fxp::bf<W> &a) {
  double v[K];
  fxp::to_md<K, W>(a, v);
#pragma unroll
  for (int l = 0; l < K; ++l) dst[l] = v[l];
}

// conj(v) t (P = 2) or v t (P = 1), accumulated into (dr, di).
template <int W, int P>
__device__ __forceinline__ void fx_cdot_acc(const fxp::bf<W> (&v)[P], const fxp::bf<W> (&t)[P], fxp::bf<W> &dr,
                                            fxp::bf<W> &di) {
  using namespace fxp;
  if constexpr (P == 1) {
    dr = add<W>(dr, mul<W>(v[0], t[0]));
  } else {
    dr = add<W>(dr, add<W>(mul<W>(v[0], t[0]), mul<W>(v[1], t[1])));
    di = add<W>(di, add<W>(mul<W>(v[0], t[1]), neg<W>(mul<W>(v[1], t[0]))));
  }
}

// t - tau v for complex (P = 2) or real tau, v, t.
template <int W, int P>
__device__ __forceinline__ void fx_axpy(const fxp::bf<W> (&tau)[P], const fxp::bf<W> (&v)[P], fxp::bf<W> (&t)[P]) {
  using namespace fxp;
  if constexpr (P == 1) {
    t[0] = add<W>(t[0], neg<W>(mul<W>(tau[0], v[0])));
  } else {
    const bf<W> pr = add<W>(mul<W>(tau[0], v[0]), neg<W>(mul<W>(tau[1], v[1])));
    const bf<W> pi = add<W>(mul<W>(tau[0], v[1]), mul<W>(tau[1], v[0]));
    t[0] = add<W>(t[0], neg<W>(pr));
    t[1] = add<W>(t[1], neg<W>(pi));
  }
}

// Element i of the Householder vector of column j (v_j from vd, the rest
// below the diagonal of M).
template <int W, int K, int P>
__device__ __forceinline__ void fx_ld_v(const double *M, const double *vd, int N, int j, int i, fxp::bf<W> (&v)[P]) {
  const long long VS = P * K;
  const double *src = (i == j) ? vd + (long long)j * VS : M + ((long long)j * N + i) * VS;
#pragma unroll
  for (int p = 0; p < P; ++p) v[p] = fx_ld<W, K>(src + p * K);
}

// Householder vector of column j (block body, kHouseThreads threads take
// part; other threads of a larger CTA only pass the barriers).
template <int K, int P>
__device__ __forceinline__ void house_block_fx(double *M, double *vd, double *beta, int *status, int N, int j) {
  using namespace fxp;
  constexpr int W = words_for(K), ST = newton_steps(K);
  __shared__ bf<W> s_red[kHouseThreads / 32];
  __shared__ bf<W> s_alpha, s_a0, s_e[P];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long VS = P * K;
  const bool act = tid < kHouseThreads;
  bf<W> acc = zero<W>();
  for (int i = j + tid; act && i < N; i += kHouseThreads) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const bf<W> x = fx_ld<W, K>(M + ((long long)j * N + i) * VS + p * K);
      acc = add<W>(acc, mul<W>(x, x));
    }
  }
  if (act) {
    fx_warp_sum<W>(acc);
    if (lane == 0) s_red[warp] = acc;
  }
  __syncthreads();
  const double *x0p = M + ((long long)j * N + j) * VS;
  if (tid == 0) {
    bf<W> A = s_red[0];
#pragma unroll
    for (int w = 1; w < kHouseThreads / 32; ++w) A = add<W>(A, s_red[w]);
    bf<W> al = zero<W>();
    if (is_zero(A))
      atomicOr(status, ST_SINGULAR);
    else
      al = mul<W>(A, rsqrt<W, ST>(A));
    s_alpha = al;
  }
  if (tid == 32) {  // |x_0| and the phase e = x_0 / |x_0| (1 for x_0 = 0)
    bf<W> xs[P];
#pragma unroll
    for (int p = 0; p < P; ++p) xs[p] = fx_ld<W, K>(x0p + p * K);
    if constexpr (P == 1) {
      const bool ng = xs[0].neg != 0;
      bf<W> a0 = xs[0];
      a0.neg = 0;
      s_a0 = a0;
      bf<W> e = from_double<W>(ng ? -1.0 : 1.0);
      s_e[0] = e;
    } else {
      const bf<W> S = add<W>(mul<W>(xs[0], xs[0]), mul<W>(xs[1], xs[1]));
      if (is_zero(S)) {
        s_a0 = zero<W>();
        s_e[0] = from_double<W>(1.0);
        s_e[1] = zero<W>();
      } else {
        const bf<W> rs = rsqrt<W, ST>(S);
        s_a0 = mul<W>(S, rs);
        s_e[0] = mul<W>(xs[0], rs);
        s_e[1] = mul<W>(xs[1], rs);
      }
    }
  }
  __syncthreads();
  if (tid == 0) {  // beta = 1 / (alpha (alpha + |x_0|)); not finite for a zero column
    const bf<W> den = mul<W>(s_alpha, add<W>(s_alpha, s_a0));
    double bt[K];
    if (is_zero(den)) {
#pragma unroll
      for (int l = 0; l < K; ++l) bt[l] = __longlong_as_double(0x7ff8000000000000LL);  // NaN
    } else {
      to_md<K, W>(recip<W, ST>(den), bt);
    }
#pragma unroll
    for (int l = 0; l < K; ++l) beta[(long long)j * K + l] = bt[l];
  }
  if (tid >= 32 && tid < 32 + 32 * P && lane == 0) {  // plane p = warp - 1: v_0 = x_0 + e alpha, R_jj = -e alpha
    const int p = warp - 1;
    const bf<W> pa = mul<W>(s_e[p], s_alpha);
    const bf<W> x = fx_ld<W, K>(x0p + p * K);
    fx_st<K, W>(vd + (long long)j * VS + p * K, add<W>(x, pa));
    fx_st<K, W>(M + ((long long)j * N + j) * VS + p * K, neg<W>(pa));
  }
  __syncthreads();
}

// H_j applied to target column w (warp body; targets as in house_apply_col).
template <int K, int P>
__device__ __forceinline__ void house_apply_col_fx(double *M, double *Y, const double *vd, const double *beta, int N,
                                                   int n, int j, int w, int lane) {
  using namespace fxp;
  constexpr int W = words_for(K);
  const int nm = n - j - 1;
  double *T = (w < nm) ? M : Y;
  const int c = (w < nm) ? j + 1 + w : w - nm;
  const long long VS = P * K;
  bf<W> dr = zero<W>(), di = zero<W>();
  for (int i = j + lane; i < N; i += 32) {
    bf<W> v[P], t[P];
    fx_ld_v<W, K, P>(M, vd, N, j, i, v);
#pragma unroll
    for (int p = 0; p < P; ++p) t[p] = fx_ld<W, K>(T + ((long long)c * N + i) * VS + p * K);
    fx_cdot_acc<W, P>(v, t, dr, di);
  }
  fx_warp_sum<W>(dr);
  if constexpr (P == 2) fx_warp_sum<W>(di);
  const bf<W> bt = fx_ld<W, K>(beta + (long long)j * K);
  bf<W> tau[P];
  tau[0] = mul<W>(bt, dr);
  if constexpr (P == 2) tau[1] = mul<W>(bt, di);
  for (int i = j + lane; i < N; i += 32) {
    bf<W> v[P], t[P];
    fx_ld_v<W, K, P>(M, vd, N, j, i, v);
    double *dst = T + ((long long)c * N + i) * VS;
#pragma unroll
    for (int p = 0; p < P; ++p) t[p] = fx_ld<W, K>(dst + p * K);
    fx_axpy<W, P>(tau, v, t);
#pragma unroll
    for (int p = 0; p < P; ++p) fx_st<K, W>(dst + p * K, t[p]);
  }
}

// The same application by a CTA over kRowLanes virtual lanes (lane q takes
// rows j+q, j+q+kRowLanes, ...), warp trees and then the four warp sums in
// order.  All threads of the CTA call it.
template <int K, int P>
__device__ __forceinline__ void house_apply_col_cta_fx(double *M, double *Y, const double *vd, const double *beta,
                                                       int N, int n, int j, int w) {
  using namespace fxp;
  constexpr int W = words_for(K);
  __shared__ bf<W> s_dot[kRowLanes / 32][P];
  __shared__ bf<W> s_tau[P];
  const int nm = n - j - 1;
  double *T = (w < nm) ? M : Y;
  const int c = (w < nm) ? j + 1 + w : w - nm;
  const long long VS = P * K;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool act = tid < kRowLanes;
  bf<W> dr = zero<W>(), di = zero<W>();
  for (int i = j + tid; act && i < N; i += kRowLanes) {
    bf<W> v[P], t[P];
    fx_ld_v<W, K, P>(M, vd, N, j, i, v);
#pragma unroll
    for (int p = 0; p < P; ++p) t[p] = fx_ld<W, K>(T + ((long long)c * N + i) * VS + p * K);
    fx_cdot_acc<W, P>(v, t, dr, di);
  }
  if (act) {
    fx_warp_sum<W>(dr);
    if constexpr (P == 2) fx_warp_sum<W>(di);
    if (lane == 0) {
      s_dot[warp][0] = dr;
      if constexpr (P == 2) s_dot[warp][1] = di;
    }
  }
  __syncthreads();
  if (tid < P) {
    bf<W> d = s_dot[0][tid];
#pragma unroll
    for (int q = 1; q < kRowLanes / 32; ++q) d = add<W>(d, s_dot[q][tid]);
    s_tau[tid] = mul<W>(fx_ld<W, K>(beta + (long long)j * K), d);
  }
  __syncthreads();
  bf<W> tau[P];
#pragma unroll
  for (int p = 0; p < P; ++p) tau[p] = s_tau[p];
  for (int i = j + tid; act && i < N; i += kRowLanes) {
    bf<W> v[P], t[P];
    fx_ld_v<W, K, P>(M, vd, N, j, i, v);
    double *dst = T + ((long long)c * N + i) * VS;
#pragma unroll
    for (int p = 0; p < P; ++p) t[p] = fx_ld<W, K>(dst + p * K);
    fx_axpy<W, P>(tau, v, t);
#pragma unroll
    for (int p = 0; p < P; ++p) fx_st<K, W>(dst + p * K, t[p]);
  }
  __syncthreads();
}

}  // namespace mdk
