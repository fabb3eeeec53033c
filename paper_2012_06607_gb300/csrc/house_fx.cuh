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

// The sum over the 32 lanes of a warp of NV values per lane; every lane gets
// it.  Every value is shifted once to the largest exponent among them, into
// a frame of W + 2 words (a word of headroom for the sign and the carries,
// the W mantissa words, a guard word; bits below the frame are dropped); the
// frames are added as two's-complement integers, within the lane and then
// over the lanes by an xor tree (integer addition is exact, so every lane
// gets the same total whatever the order), and the total is normalized
// once.  A NaN anywhere gives NaN.  (A tree of W-word additions would
// align, truncate and renormalise at each of its levels: about 20 times the
// instructions on the chains that wait for this sum.)
template <int W, int NV>
__device__ __forceinline__ fxp::bf<W> fx_warp_sum_n(const fxp::bf<W> (&v)[NV]) {
  using namespace fxp;
  constexpr int F = W + 2;
  constexpr unsigned kAll = 0xffffffffu;
  bool nan = false;
  int emax = kZeroExp;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    nan = nan || is_nan(v[q]);
    if (!is_zero(v[q])) emax = max(emax, v[q].e);
  }
  if (__any_sync(kAll, nan)) return nan_value<W>();
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(kAll, emax, off));
  if (emax == kZeroExp) return zero<W>();
  uint32_t S[F];
#pragma unroll
  for (int i = 0; i < F; ++i) S[i] = 0u;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    if (is_zero(v[q])) continue;
    uint32_t X[F];
    X[0] = 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) X[i + 1] = v[q].m[i];
    X[F - 1] = 0u;
    shr_bits<F>(X, emax - v[q].e);
    uint64_t c = v[q].neg ? 1u : 0u;  // two's complement: invert and add one
#pragma unroll
    for (int i = F - 1; i >= 0; --i) {
      const uint64_t t = (uint64_t)S[i] + (v[q].neg ? (uint32_t)~X[i] : X[i]) + c;
      S[i] = (uint32_t)t;
      c = t >> 32;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    uint32_t T[F];
#pragma unroll
    for (int i = 0; i < F; ++i) T[i] = __shfl_xor_sync(kAll, S[i], off);
    uint64_t c = 0;
#pragma unroll
    for (int i = F - 1; i >= 0; --i) {
      const uint64_t t = (uint64_t)S[i] + T[i] + c;
      S[i] = (uint32_t)t;
      c = t >> 32;
    }
  }
  bf<W> z;
  z.neg = (int)(S[0] >> 31);
  if (z.neg) {  // magnitude
    uint64_t c = 1;
#pragma unroll
    for (int i = F - 1; i >= 0; --i) {
      const uint64_t t = (uint64_t)(uint32_t)~S[i] + c;
      S[i] = (uint32_t)t;
      c = t >> 32;
    }
  }
  int lead = 32 * F;  // position of the first set bit from the top of word 0
#pragma unroll
  for (int i = F - 1; i >= 0; --i)
    if (S[i]) lead = 32 * i + clz32(S[i]);
  if (lead >= 32 * F) return zero<W>();
  shl_bits<F>(S, lead);
#pragma unroll
  for (int i = 0; i < W; ++i) z.m[i] = S[i];
  // the total is S 2^(emax - 32(W+1)); after the shift its top W words are m
  z.e = emax + 32 - lead;
  return z;
}

// Sum over the 32 lanes of a warp; every lane gets it.
template <int W>
__device__ __forceinline__ void fx_warp_sum(fxp::bf<W> &a) {
  const fxp::bf<W> v[1] = {a};
  a = fx_warp_sum_n<W, 1>(v);
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

// H_j applied to target column w (targets as in house_apply_col: w < n-j-1
// is column j+1+w of M, otherwise column w-(n-j-1) of Y) over 128 virtual
// lanes: lane q takes rows j+q, j+q+128, ... in order and holds their partial
// dot product p_q; the column's dot product is the exact aligned sum of the
// 128 values (fx_warp_sum_n, lane l holding p_l, p_{l+32}, p_{l+64},
// p_{l+96}).  CTA = true: 128 threads of a CTA, one virtual lane each (all
// threads of the CTA call it); CTA = false: one warp, lane l running virtual
// lanes l, l+32, l+64, l+96.  Both forms sum the same values exactly, so they
// give the same bits.
template <int K, int P, bool CTA, bool CACHE = true>
__device__ __forceinline__ void house_apply_col_v128(double *M, double *Y, const double *vd, const double *beta,
                                                     int N, int n, int j, int w) {
  using namespace fxp;
  constexpr int W = words_for(K);
  const int nm = n - j - 1;
  double *T = (w < nm) ? M : Y;
  const int c = (w < nm) ? j + 1 + w : w - nm;
  const long long VS = P * K;
  const int tid = CTA ? (int)threadIdx.x : (int)(threadIdx.x & 31);
  auto partial = [&](int q, bf<W> (&d)[P]) {
#pragma unroll
    for (int p = 0; p < P; ++p) d[p] = zero<W>();
    for (int i = j + q; i < N; i += kRowLanes) {
      bf<W> v[P], t[P];
      fx_ld_v<W, K, P>(M, vd, N, j, i, v);
#pragma unroll
      for (int p = 0; p < P; ++p) t[p] = fx_ld<W, K>(T + ((long long)c * N + i) * VS + p * K);
      if constexpr (P == 1) {
        fx_cdot_acc<W, P>(v, t, d[0], d[0]);
      } else {
        fx_cdot_acc<W, P>(v, t, d[0], d[1]);
      }
    }
  };
  bf<W> u[P];
  // CTA form: the lane's first row keeps its converted (v, t) for the update
  // (where they fit in registers: up to 30 words a row)
  constexpr bool kCache = CACHE && CTA && P * (W + 2) <= 30;  // same values either way
  bf<W> cv[P], ct[P];
  if constexpr (CTA) {
    __shared__ bf<W> s_p[kRowLanes][P];
    __shared__ bf<W> s_tau[P];
    if (tid < kRowLanes) {
      bf<W> d[P];
#pragma unroll
      for (int p = 0; p < P; ++p) d[p] = zero<W>();
      for (int i = j + tid; i < N; i += kRowLanes) {
        bf<W> v[P], t[P];
        fx_ld_v<W, K, P>(M, vd, N, j, i, v);
#pragma unroll
        for (int p = 0; p < P; ++p) t[p] = fx_ld<W, K>(T + ((long long)c * N + i) * VS + p * K);
        if constexpr (P == 1) {
          fx_cdot_acc<W, P>(v, t, d[0], d[0]);
        } else {
          fx_cdot_acc<W, P>(v, t, d[0], d[1]);
        }
        if (kCache && i == j + tid) {
#pragma unroll
          for (int p = 0; p < P; ++p) {
            cv[p] = v[p];
            ct[p] = t[p];
          }
        }
      }
#pragma unroll
      for (int p = 0; p < P; ++p) s_p[tid][p] = d[p];
    }
    __syncthreads();
    if (tid < 32) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const bf<W> v4[4] = {s_p[tid][p], s_p[tid + 32][p], s_p[tid + 64][p], s_p[tid + 96][p]};
        u[p] = fx_warp_sum_n<W, 4>(v4);
      }
      if (tid == 0) {
        const bf<W> bt = fx_ld<W, K>(beta + (long long)j * K);
#pragma unroll
        for (int p = 0; p < P; ++p) s_tau[p] = mul<W>(bt, u[p]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < P; ++p) u[p] = s_tau[p];
  } else {
    bf<W> q0[P], q1[P], q2[P], q3[P];
    partial(tid, q0);
    partial(tid + 32, q1);
    partial(tid + 64, q2);
    partial(tid + 96, q3);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const bf<W> v4[4] = {q0[p], q1[p], q2[p], q3[p]};
      u[p] = fx_warp_sum_n<W, 4>(v4);
    }
    const bf<W> bt = fx_ld<W, K>(beta + (long long)j * K);
#pragma unroll
    for (int p = 0; p < P; ++p) u[p] = mul<W>(bt, u[p]);
  }
  // t_i <- t_i - tau v_i on every virtual lane's rows
  const int qs = CTA ? kRowLanes : 32;
  for (int q = tid; q < kRowLanes; q += qs) {
    for (int i = j + q; i < N; i += kRowLanes) {
      bf<W> v[P], t[P];
      double *dst = T + ((long long)c * N + i) * VS;
      if (kCache && i == j + q) {  // converted in the first pass
#pragma unroll
        for (int p = 0; p < P; ++p) {
          v[p] = cv[p];
          t[p] = ct[p];
        }
      } else {
        fx_ld_v<W, K, P>(M, vd, N, j, i, v);
#pragma unroll
        for (int p = 0; p < P; ++p) t[p] = fx_ld<W, K>(dst + p * K);
      }
      fx_axpy<W, P>(u, v, t);
#pragma unroll
      for (int p = 0; p < P; ++p) fx_st<K, W>(dst + p * K, t[p]);
    }
  }
  if constexpr (CTA) __syncthreads();
}

// ------------------------------------------------- back substitution, W = R^-1 Q^H
// The element bodies of rinv_entry / backsub_entry / the lookahead kernels in
// fixed point: w = y r_cc^-1, y_i <- y_i - R_ic w.  Every element takes the
// same operations in the same order in the lookahead kernels and in the
// batched kernel, so both get the same bits.

// z = a b (complex for P = 2)
template <int W, int P>
__device__ __forceinline__ void fx_cmul(const fxp::bf<W> (&a)[P], const fxp::bf<W> (&b)[P], fxp::bf<W> (&z)[P]) {
  using namespace fxp;
  if constexpr (P == 1) {
    z[0] = mul<W>(a[0], b[0]);
  } else {
    z[0] = add<W>(mul<W>(a[0], b[0]), neg<W>(mul<W>(a[1], b[1])));
    z[1] = add<W>(mul<W>(a[0], b[1]), mul<W>(a[1], b[0]));
  }
}

template <int W, int K, int P>
__device__ __forceinline__ void fx_ld_val(const double *src, fxp::bf<W> (&v)[P]) {
#pragma unroll
  for (int p = 0; p < P; ++p) v[p] = fx_ld<W, K>(src + p * K);
}

template <int W, int K, int P>
__device__ __forceinline__ void fx_st_val(double *dst, const fxp::bf<W> (&v)[P]) {
#pragma unroll
  for (int p = 0; p < P; ++p) fx_st<K, W>(dst + p * K, v[p]);
}

// rinv[j] = 1 / R_jj (conj(r) / |r|^2 for complex r); not finite for r = 0.
template <int K, int P>
__device__ __forceinline__ void rinv_entry_fx(const double *M, double *rinv, int N, int j) {
  using namespace fxp;
  constexpr int W = words_for(K), ST = newton_steps(K);
  const long long VS = P * K;
  bf<W> r[P], z[P];
  fx_ld_val<W, K, P>(M + ((long long)j * N + j) * VS, r);
  bf<W> S = mul<W>(r[0], r[0]);
  if constexpr (P == 2) S = add<W>(S, mul<W>(r[1], r[1]));
  double *dst = rinv + (long long)j * VS;
  if (is_zero(S)) {
#pragma unroll
    for (int l = 0; l < P * K; ++l) dst[l] = __longlong_as_double(0x7ff8000000000000LL);  // NaN
    return;
  }
  const bf<W> rs = recip<W, ST>(S);
  z[0] = mul<W>(r[0], rs);
  if constexpr (P == 2) z[1] = neg<W>(mul<W>(r[1], rs));
  fx_st_val<W, K, P>(dst, z);
}

// y <- y - R_ic w at Y[(col, i)], w the K-limb value at wsrc (W[c][col] or
// the same value formed in registers).
template <int K, int P>
__device__ __forceinline__ void fx_bs_update(const double *M, double *Y, const double *wsrc, int N, int c, int col,
                                             int i) {
  using namespace fxp;
  constexpr int W = words_for(K);
  const long long VS = P * K;
  bf<W> w[P], rc[P], y[P], t[P];
  fx_ld_val<W, K, P>(wsrc, w);
  fx_ld_val<W, K, P>(M + ((long long)c * N + i) * VS, rc);
  double *yp = Y + ((long long)col * N + i) * VS;
  fx_ld_val<W, K, P>(yp, y);
  fx_cmul<W, P>(rc, w, t);
#pragma unroll
  for (int p = 0; p < P; ++p) y[p] = add<W>(y[p], neg<W>(t[p]));
  fx_st_val<W, K, P>(yp, y);
}

// dst (P K doubles) = Y[(col, c)] rinv[c], rounded to K limbs: the value of W[c][col]
template <int K, int P>
__device__ __forceinline__ void fx_bs_w(const double *Y, const double *rinv, int N, int c, int col, double *dst) {
  using namespace fxp;
  constexpr int W = words_for(K);
  const long long VS = P * K;
  bf<W> y[P], ri[P], w[P];
  fx_ld_val<W, K, P>(Y + ((long long)col * N + c) * VS, y);
  fx_ld_val<W, K, P>(rinv + (long long)c * VS, ri);
  fx_cmul<W, P>(y, ri, w);
  fx_st_val<W, K, P>(dst, w);
}

// backsub_entry in fixed point: element e = (i, col) of step c.
template <int K, int P>
__device__ __forceinline__ void backsub_entry_fx(const double *M, double *Y, double *Wm, const double *rinv, int N,
                                                 int c, long long e) {
  const int i = (int)(e / N), col = (int)(e % N);
  if (i == c) {
    fx_bs_w<K, P>(Y, rinv, N, c, col, Wm + ((long long)c * N + col) * (P * K));
  } else {
    double w[P * K];
    fx_bs_w<K, P>(Y, rinv, N, c, col, w);
    fx_bs_update<K, P>(M, Y, w, N, c, col, i);
  }
}

// ------------------------------------------------------ dx_k = W r_k, one row
// Warps of one CTA at most (the batched kernel's largest CTA: 384 threads).
constexpr int kFxMaxWarps = 12;

// Row `row` of dx_k = W r_k in fixed point, over the kRowLanes virtual lanes
// of wmv_row (lane v: plane p = v / Vc, column slot cs = v % Vc, Vc =
// kRowLanes / P; slot cs sums columns cs, cs + Vc, ... in order): each warp
// reduces its 32 lanes by an xor tree, then the warp sums of a plane are
// added in warp order.  Called by every thread of the CTA; the group of
// kRowLanes threads with index gt (active when act) handles the row, the
// others only pass the barriers.
template <int K, int P>
__device__ __forceinline__ void wmv_row_fx(const double *Wm, const double *r, double *dx, int N, int n, int k,
                                           int row, int gt, bool act) {
  using namespace fxp;
  constexpr int W = words_for(K), Vc = kRowLanes / P, WPP = Vc / 32;  // warps per plane
  __shared__ bf<W> s_wsum[kFxMaxWarps];
  const long long VS = P * K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bf<W> acc = zero<W>();
  if (act) {
    const int p = gt / Vc, cs = gt % Vc;
    for (int c = cs; c < N; c += Vc) {
      bf<W> w[P], x[P];
      fx_ld_val<W, K, P>(Wm + ((long long)row * N + c) * VS, w);
      fx_ld_val<W, K, P>(r + ((long long)k * N + c) * VS, x);
      bf<W> t;
      if constexpr (P == 1) {
        t = mul<W>(w[0], x[0]);
      } else if (p == 0) {  // real part: w_re x_re - w_im x_im
        t = add<W>(mul<W>(w[0], x[0]), neg<W>(mul<W>(w[1], x[1])));
      } else {  // imaginary part: w_re x_im + w_im x_re
        t = add<W>(mul<W>(w[0], x[1]), mul<W>(w[1], x[0]));
      }
      acc = add<W>(acc, t);
    }
    fx_warp_sum<W>(acc);
    if (lane == 0) s_wsum[warp] = acc;
  }
  __syncthreads();
  if (act && gt < P) {  // lane gt = plane: the plane's warp sums in order
    const int w0 = warp - (gt >> 5) + gt * WPP;  // first warp of the plane within this group
    bf<W> z = s_wsum[w0];
#pragma unroll
    for (int q = 1; q < WPP; ++q) z = add<W>(z, s_wsum[w0 + q]);
    fx_st<K, W>(dx + ((long long)k * n + row) * VS + gt * K, z);
  }
  __syncthreads();
}

// ----------------------------------------- r_k = sgn b_k - (sum of the partials)
// The finish of the block Toeplitz update in fixed point: the partial sums
// that rhs_partial left in md (one per chunk of terms) are added in W-word
// fixed point over the virtual lanes of rhs_finish_row (lane v: plane
// p = v / Vc, chunk slot cs = v % Vc, slot cs takes chunks cs, cs + Vc, ...
// in order), each warp's lanes by an xor tree, the warp sums of a plane in
// warp order, and sgn b_k minus that sum is rounded to K limbs once.  Same
// calling convention as wmv_row_fx.
template <int K, int P>
__device__ __forceinline__ void rhs_finish_row_fx(const double *b, double sgn, const double *part, double *r, int N,
                                                  int d, int k, int nchunk, int row, int gt, bool act) {
  using namespace fxp;
  constexpr int W = words_for(K), Vc = kRowLanes / P, WPP = Vc / 32;
  __shared__ bf<W> s_fsum[kFxMaxWarps];
  const long long VS = P * K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bf<W> acc = zero<W>();
  if (act) {
    const int p = gt / Vc, cs = gt % Vc;
    for (int c = cs; c < nchunk; c += Vc)
      acc = add<W>(acc, fx_ld<W, K>(part + ((long long)row * nchunk + c) * VS + p * K));
    fx_warp_sum<W>(acc);
    if (lane == 0) s_fsum[warp] = acc;
  }
  __syncthreads();
  if (act && gt < P) {  // lane gt = plane
    const int w0 = warp - (gt >> 5) + gt * WPP;
    bf<W> z = s_fsum[w0];
#pragma unroll
    for (int q = 1; q < WPP; ++q) z = add<W>(z, s_fsum[w0 + q]);
    const long long stride = (long long)N * (d + 1);
    double bv[K];
#pragma unroll
    for (int l = 0; l < K; ++l) bv[l] = b[(long long)row * (d + 1) + k + (long long)(gt * K + l) * stride];
    bf<W> bb = from_md<W, K>(bv);
    if (sgn < 0.0) bb = neg<W>(bb);
    fx_st<K, W>(r + ((long long)k * N + row) * VS + gt * K, add<W>(bb, neg<W>(z)));
  }
  __syncthreads();
}

}  // namespace mdk
