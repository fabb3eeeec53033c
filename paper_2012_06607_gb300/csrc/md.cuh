// Multiple-double (md) arithmetic on the FP64 pipe, sm_103a.
//
// An md number is an unevaluated sum of K doubles (Section 2 of the paper,
// K in {1,2,3,4,5,8,10}: double, double double, ..., deca double).  The
// algorithms are fixed as follows (the paper cites QDlib and CAMPARY but does
// not write them out):
//   * error-free transformations: TwoSum, FastTwoSum, TwoProd with an fma;
//   * K = 2 addition: AccurateDWPlusDW (Joldes, Muller, Popescu 2017);
//   * K = 2 multiplication: TwoProd(x0,y0) plus the cross products, then
//     FastTwoSum (Hida, Li, Bailey 2001);
//   * K >= 3: terms of order 2^(-53 n) (level n) are summed by a TwoSum chain
//     whose errors move to level n+1; level K is summed with plain additions;
//     products x_i y_j use TwoProd when i+j <= K-1 and a plain product when
//     i+j = K; the K+1 level sums are renormalised into K limbs by a
//     bottom-up TwoSum sweep followed by a top-down sweep that skips zero
//     errors;
//   * division: long division with K+1 quotient limbs;
//   * square root: hardware sqrt of the leading limb and ceil(log2 K)+1
//     Heron steps s <- (s + a/s)/2.
//
// GB300 specifics.  The FP64 pipe issues one warp instruction per ~64 cycles
// per SM sub-partition, so FP64 instruction count is the cost.  TwoSum is done
// as "order the operands by exponent (32-bit integer compare of the high words,
// integer selects), then FastTwoSum": 3 FP64 instructions instead of 6, with
// the identical sum and exact error.  Zero tests use the integer pipe too.
// Build with -fmad=false: every +,-,* is separately rounded and fmas appear
// only where __fma_rn is written (dadd, dsub, dmul below are single-rounding
// fma forms of the plain operations).
#pragma once
#include <cstdint>

namespace mdk {

// a + b = fma(a, 1, b), a - b = fma(a, 1, -b), a * b = fma(a, b, -0): a*1 is
// exact and the product inside an fma is exact, so each form rounds once to
// the same double as DADD / DSUB / DMUL, signed zeros included.  On sm_103a the
// FP64 pipe retires DFMA faster than DADD and DMUL (measured: the resident
// series-product kernel ran 15% faster, pipe 99.6% busy).  The unit and the
// zero come from constant memory so that the compiler cannot fold the forms
// back into DADD / DMUL.
static __constant__ double c_fma_unit[2] = {1.0, 0.0};
__device__ __forceinline__ double dadd(double a, double b) { return __fma_rn(a, c_fma_unit[0], b); }
__device__ __forceinline__ double dsub(double a, double b) { return __fma_rn(a, c_fma_unit[0], -b); }
__device__ __forceinline__ double dmul(double a, double b) { return __fma_rn(a, b, -c_fma_unit[1]); }
// -a by flipping the sign bit on the integer pipe (a negation that cannot be
// folded into the consumer would otherwise cost an FP64 instruction).
__device__ __forceinline__ double dneg(double a) {
  return __hiloint2double(__double2hiint(a) ^ (int)0x80000000u, __double2loint(a));
}
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// Exponent order for FastTwoSum (Dekker needs exponent(hi) >= exponent(lo)):
// compare the high words with the sign cleared.  32-bit integer ops only, so
// that nothing lands on the FP64 pipe.
__device__ __forceinline__ bool exp_ge(double a, double b) {
  const unsigned ha = (unsigned)__double2hiint(a) & 0x7fffffffu;
  const unsigned hb = (unsigned)__double2hiint(b) & 0x7fffffffu;
  return ha >= hb;
}

__device__ __forceinline__ bool nonzero(double a) {
  return (((unsigned)__double2hiint(a) & 0x7fffffffu) | (unsigned)__double2loint(a)) != 0u;
}

// s = fl(a + b), e = (a + b) - s exactly.
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
  const bool ge = exp_ge(a, b);
  const double hi = ge ? a : b;
  const double lo = ge ? b : a;
  const double ss = dadd(hi, lo);
  e = dsub(lo, dsub(ss, hi));
  s = ss;
}

__device__ __forceinline__ void fast_two_sum(double a, double b, double &s, double &e) {
  const double ss = dadd(a, b);
  e = dsub(b, dsub(ss, a));
  s = ss;
}

__device__ __forceinline__ void two_prod(double a, double b, double &p, double &e) {
  const double pp = dmul(a, b);
  e = __fma_rn(a, b, -pp);
  p = pp;
}

// M terms t (roughly by decreasing order) -> K non-overlapping limbs.
template <int M, int K>
__device__ __forceinline__ void renorm(const double (&t)[M], double (&z)[K]) {
  double c[M];
  double s = t[M - 1];
#pragma unroll
  for (int i = M - 2; i >= 0; --i) two_sum(t[i], s, s, c[i + 1]);
  c[0] = s;
#pragma unroll
  for (int q = 0; q < K; ++q) z[q] = 0.0;
  int j = 0;
  double e = c[0];
#pragma unroll
  for (int i = 1; i < M; ++i) {
    if (j < K - 1) {
      double r, f;
      two_sum(e, c[i], r, f);
      const bool nz = nonzero(f);
#pragma unroll
      for (int q = 0; q < K - 1; ++q)
        if (nz && q == j) z[q] = r;
      e = nz ? f : r;
      j += nz ? 1 : 0;
    } else {
      e = dadd(e, c[i]);
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q == j) z[q] = e;
}

template <int K>
__device__ __forceinline__ void md_add(const double (&x)[K], const double (&y)[K], double (&z)[K]) {
  if constexpr (K == 1) {
    z[0] = dadd(x[0], y[0]);
  } else if constexpr (K == 2) {
    double sh, sl, th, tl, vh, vl;
    two_sum(x[0], y[0], sh, sl);
    two_sum(x[1], y[1], th, tl);
    const double c = dadd(sl, th);
    fast_two_sum(sh, c, vh, vl);
    const double w = dadd(tl, vl);
    fast_two_sum(vh, w, z[0], z[1]);
  } else {
    double lv[K + 1];
    double carry[K], nc[K];
    two_sum(x[0], y[0], lv[0], carry[0]);
#pragma unroll
    for (int n = 1; n < K; ++n) {
      double s;
      two_sum(x[n], y[n], s, nc[0]);
#pragma unroll
      for (int i = 0; i < n; ++i) two_sum(s, carry[i], s, nc[i + 1]);
      lv[n] = s;
#pragma unroll
      for (int i = 0; i <= n; ++i) carry[i] = nc[i];
    }
    double s = carry[0];
#pragma unroll
    for (int i = 1; i < K; ++i) s = dadd(s, carry[i]);
    lv[K] = s;
    renorm<K + 1, K>(lv, z);
  }
}

template <int K>
__device__ __forceinline__ void md_neg(const double (&x)[K], double (&z)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) z[i] = dneg(x[i]);
}

template <int K>
__device__ __forceinline__ void md_sub(const double (&x)[K], const double (&y)[K], double (&z)[K]) {
  double ny[K];
  md_neg<K>(y, ny);
  md_add<K>(x, ny, z);
}

template <int K>
__device__ __forceinline__ void md_mul(const double (&x)[K], const double (&y)[K], double (&z)[K]) {
  if constexpr (K == 1) {
    z[0] = dmul(x[0], y[0]);
  } else if constexpr (K == 2) {
    double p, e;
    two_prod(x[0], y[0], p, e);
    const double t1 = dmul(x[0], y[1]);
    const double t2 = dmul(x[1], y[0]);
    e = dadd(e, dadd(t1, t2));
    fast_two_sum(p, e, z[0], z[1]);
  } else {
    constexpr int MC = K * (K - 1);
    double lv[K + 1];
    double carry[MC], nc[MC];
    double low[K], nlow[K], hi[K];
    // all loops run to fixed bounds with compile-time guards, so that every
    // array index is a constant and the arrays stay in registers
#pragma unroll
    for (int n = 0; n < K; ++n) {
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i <= n) two_prod(x[i], y[n - i], hi[i], nlow[i]);
      double s = hi[0];
#pragma unroll
      for (int i = 1; i < K; ++i)
        if (i <= n) two_sum(s, hi[i], s, nc[i - 1]);
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i < n) two_sum(s, low[i], s, nc[n + i]);
#pragma unroll
      for (int i = 0; i < MC; ++i)
        if (i < (n - 1) * n) two_sum(s, carry[i], s, nc[2 * n + i]);
      lv[n] = s;
#pragma unroll
      for (int i = 0; i < MC; ++i)
        if (i < n * (n + 1)) carry[i] = nc[i];
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i <= n) low[i] = nlow[i];
    }
    double s = dmul(x[1], y[K - 1]);
#pragma unroll
    for (int i = 2; i <= K - 1; ++i) s = dadd(s, dmul(x[i], y[K - i]));
#pragma unroll
    for (int i = 0; i < K; ++i) s = dadd(s, low[i]);
#pragma unroll
    for (int i = 0; i < MC; ++i) s = dadd(s, carry[i]);
    lv[K] = s;
    renorm<K + 1, K>(lv, z);
  }
}

// md times double
template <int K>
__device__ __forceinline__ void md_mul_d(const double (&x)[K], double b, double (&z)[K]) {
  if constexpr (K == 1) {
    z[0] = dmul(x[0], b);
  } else if constexpr (K == 2) {
    double p, e;
    two_prod(x[0], b, p, e);
    e = dadd(e, dmul(x[1], b));
    fast_two_sum(p, e, z[0], z[1]);
  } else {
    double lv[K + 1];
    double carry[K], nc[K];
    double lo_prev;
    two_prod(x[0], b, lv[0], lo_prev);
#pragma unroll
    for (int n = 1; n < K; ++n) {
      double h, l, s;
      two_prod(x[n], b, h, l);
      s = h;
      two_sum(s, lo_prev, s, nc[0]);
#pragma unroll
      for (int i = 0; i < n - 1; ++i) two_sum(s, carry[i], s, nc[i + 1]);
      lv[n] = s;
#pragma unroll
      for (int i = 0; i < n; ++i) carry[i] = nc[i];
      lo_prev = l;
    }
    double s = lo_prev;
#pragma unroll
    for (int i = 0; i < K - 1; ++i) s = dadd(s, carry[i]);
    lv[K] = s;
    renorm<K + 1, K>(lv, z);
  }
}

template <int K>
__device__ __forceinline__ void md_div(const double (&x)[K], const double (&y)[K], double (&z)[K]) {
  if constexpr (K == 1) {
    z[0] = ddiv(x[0], y[0]);
  } else {
    double q[K + 1], r[K], t[K];
#pragma unroll
    for (int i = 0; i < K; ++i) r[i] = x[i];
#pragma unroll
    for (int i = 0; i <= K; ++i) {
      q[i] = ddiv(r[0], y[0]);
      if (i < K) {
        md_mul_d<K>(y, q[i], t);
        md_sub<K>(r, t, r);
      }
    }
    renorm<K + 1, K>(q, z);
  }
}

template <int K>
__host__ __device__ constexpr int sqrt_iters() {
  int l = 0;
  while ((1 << l) < K) ++l;
  return l + 1;
}

template <int K>
__device__ __forceinline__ void md_sqrt(const double (&a)[K], double (&z)[K]) {
  if constexpr (K == 1) {
    z[0] = __dsqrt_rn(a[0]);
  } else {
    if (!nonzero(a[0])) {
#pragma unroll
      for (int i = 0; i < K; ++i) z[i] = 0.0;
      return;
    }
    double s[K], t[K];
    s[0] = __dsqrt_rn(a[0]);
#pragma unroll
    for (int i = 1; i < K; ++i) s[i] = 0.0;
    constexpr int iters = sqrt_iters<K>();
#pragma unroll 1
    for (int k = 0; k < iters; ++k) {
      md_div<K>(a, s, t);
      md_add<K>(s, t, s);
#pragma unroll
      for (int i = 0; i < K; ++i) s[i] = dmul(s[i], 0.5);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) z[i] = s[i];
  }
}

// ------------------------------------------ precision-doubling iterations
// For the latency-bound chain of Householder vectors: Newton iterations whose
// early steps run at 2, 4, 8 limbs (each step doubles the correct bits, so a
// step needs only the precision it produces) and whose last step runs at K
// limbs.  Same accuracy as md_sqrt / md_div, about a third of the sequential
// FP64 instructions for the square root; not bit-identical to them.

// s <- (s + a/s) / 2 on the leading L limbs (s's limbs from L on are zero).
template <int L, int K>
__device__ __forceinline__ void heron_step(const double (&a)[K], double (&s)[K]) {
  double aL[L], sL[L], q[L], t[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    aL[l] = a[l];
    sL[l] = s[l];
  }
  md_div<L>(aL, sL, q);
  md_add<L>(sL, q, t);
#pragma unroll
  for (int l = 0; l < L; ++l) s[l] = dmul(t[l], 0.5);  // exact halving
}

template <int K>
__device__ __forceinline__ void md_sqrt_pd(const double (&a)[K], double (&z)[K]) {
  if constexpr (K == 1) {
    z[0] = __dsqrt_rn(a[0]);
  } else {
    double s[K];
#pragma unroll
    for (int l = 0; l < K; ++l) s[l] = 0.0;
    if (nonzero(a[0])) {
      s[0] = __dsqrt_rn(a[0]);
      heron_step<2, K>(a, s);
      if constexpr (K > 2) heron_step<(K < 4 ? K : 4), K>(a, s);
      if constexpr (K > 4) heron_step<(K < 8 ? K : 8), K>(a, s);
      if constexpr (K > 8) heron_step<K, K>(a, s);
    }
#pragma unroll
    for (int l = 0; l < K; ++l) z[l] = s[l];
  }
}

// y <- y + y (1 - a y) on the leading L limbs.
template <int L, int K>
__device__ __forceinline__ void recip_step(const double (&a)[K], double (&y)[K]) {
  double aL[L], yL[L], t[L], e[L], u[L], one[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    aL[l] = a[l];
    yL[l] = y[l];
    one[l] = l == 0 ? 1.0 : 0.0;
  }
  md_mul<L>(aL, yL, t);
  md_sub<L>(one, t, e);
  md_mul<L>(yL, e, u);
  md_add<L>(yL, u, t);
#pragma unroll
  for (int l = 0; l < L; ++l) y[l] = t[l];
}

// 1 / a (a != 0) by Newton steps at 2, 4, 8 and K limbs from 1 / a_0.
template <int K>
__device__ __forceinline__ void md_recip_pd(const double (&a)[K], double (&z)[K]) {
  double y[K];
#pragma unroll
  for (int l = 0; l < K; ++l) y[l] = 0.0;
  y[0] = ddiv(1.0, a[0]);
  if constexpr (K > 1) {
    recip_step<2, K>(a, y);
    if constexpr (K > 2) recip_step<(K < 4 ? K : 4), K>(a, y);
    if constexpr (K > 4) recip_step<(K < 8 ? K : 8), K>(a, y);
    if constexpr (K > 8) recip_step<K, K>(a, y);
  }
#pragma unroll
  for (int l = 0; l < K; ++l) z[l] = y[l];
}

// ----------------------------------------------------------------- complex
// P = 1: real, P = 2: complex (v[0] real part, v[1] imaginary part).
template <int K, int P>
struct mdv {
  double v[P][K];
};

template <int K, int P>
__device__ __forceinline__ void c_zero(mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) z.v[p][l] = 0.0;
}

template <int K, int P>
__device__ __forceinline__ void c_add(const mdv<K, P> &a, const mdv<K, P> &b, mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p) md_add<K>(a.v[p], b.v[p], z.v[p]);
}

template <int K, int P>
__device__ __forceinline__ void c_sub(const mdv<K, P> &a, const mdv<K, P> &b, mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p) md_sub<K>(a.v[p], b.v[p], z.v[p]);
}

template <int K, int P>
__device__ __forceinline__ void c_mul(const mdv<K, P> &a, const mdv<K, P> &b, mdv<K, P> &z) {
  if constexpr (P == 1) {
    md_mul<K>(a.v[0], b.v[0], z.v[0]);
  } else {
    double ac[K], bd[K], ad[K], bc[K];
    md_mul<K>(a.v[0], b.v[0], ac);
    md_mul<K>(a.v[1], b.v[1], bd);
    md_mul<K>(a.v[0], b.v[1], ad);
    md_mul<K>(a.v[1], b.v[0], bc);
    md_sub<K>(ac, bd, z.v[0]);
    md_add<K>(ad, bc, z.v[1]);
  }
}

template <int K, int P>
__device__ __forceinline__ void c_mul_real(const mdv<K, P> &a, const double (&r)[K], mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p) md_mul<K>(a.v[p], r, z.v[p]);
}

template <int K, int P>
__device__ __forceinline__ void c_mul_d(const mdv<K, P> &a, double b, mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p) md_mul_d<K>(a.v[p], b, z.v[p]);
}

template <int K, int P>
__device__ __forceinline__ void c_conj(const mdv<K, P> &a, mdv<K, P> &z) {
  z = a;
  if constexpr (P == 2) md_neg<K>(a.v[1], z.v[1]);
}

template <int K, int P>
__device__ __forceinline__ void c_abs2(const mdv<K, P> &a, double (&z)[K]) {
  if constexpr (P == 1) {
    md_mul<K>(a.v[0], a.v[0], z);
  } else {
    double t1[K], t2[K];
    md_mul<K>(a.v[0], a.v[0], t1);
    md_mul<K>(a.v[1], a.v[1], t2);
    md_add<K>(t1, t2, z);
  }
}

template <int K, int P>
__device__ __forceinline__ void c_div(const mdv<K, P> &a, const mdv<K, P> &b, mdv<K, P> &z) {
  if constexpr (P == 1) {
    md_div<K>(a.v[0], b.v[0], z.v[0]);
  } else {
    double cc[K], dd[K], den[K], t1[K], t2[K], nr[K], ni[K];
    md_mul<K>(b.v[0], b.v[0], cc);
    md_mul<K>(b.v[1], b.v[1], dd);
    md_add<K>(cc, dd, den);
    md_mul<K>(a.v[0], b.v[0], t1);
    md_mul<K>(a.v[1], b.v[1], t2);
    md_add<K>(t1, t2, nr);
    md_mul<K>(a.v[1], b.v[0], t1);
    md_mul<K>(a.v[0], b.v[1], t2);
    md_sub<K>(t1, t2, ni);
    md_div<K>(nr, den, z.v[0]);
    md_div<K>(ni, den, z.v[1]);
  }
}

// ------------------------------------------------------ loads and stores
// AoS value: P*K consecutive doubles, plane-major ([p][l]).
template <int K, int P>
__device__ __forceinline__ void ld_aos(const double *src, mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) z.v[p][l] = src[p * K + l];
}

template <int K, int P>
__device__ __forceinline__ void ld_aos_nc(const double *src, mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) z.v[p][l] = __ldg(src + p * K + l);
}

template <int K, int P>
__device__ __forceinline__ void st_aos(double *dst, const mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) dst[p * K + l] = z.v[p][l];
}

// SoA value: limb l of plane p at src[(p*K + l) * plane_stride].
template <int K, int P>
__device__ __forceinline__ void ld_soa(const double *src, long long stride, mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) z.v[p][l] = src[(long long)(p * K + l) * stride];
}

template <int K, int P>
__device__ __forceinline__ void st_soa(double *dst, long long stride, const mdv<K, P> &z) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) dst[(long long)(p * K + l) * stride] = z.v[p][l];
}

template <int K, int P>
__device__ __forceinline__ void shfl_xor(mdv<K, P> &z, int lanemask, mdv<K, P> &out) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) out.v[p][l] = __shfl_xor_sync(0xffffffffu, z.v[p][l], lanemask);
}

template <int K, int P>
__device__ __forceinline__ void shfl_idx(mdv<K, P> &z, int src, mdv<K, P> &out) {
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) out.v[p][l] = __shfl_sync(0xffffffffu, z.v[p][l], src);
}

}  // namespace mdk
