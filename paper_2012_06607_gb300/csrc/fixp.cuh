// Binary floating-point numbers with a W-word (32-bit words) integer
// mantissa, for the scalar chain of the Householder QR (norm, square root,
// reciprocal, phase).
//
// Why: that chain is a sequence of dependent md operations on one warp, and on
// GB300 every FP64 warp instruction holds its SM sub-partition's FP64 unit for
// about 64 cycles, while an integer warp instruction takes about 2.  An md
// square root or reciprocal at 8 limbs is several thousand FP64 instructions;
// the same quantity from Newton steps on a multiword integer mantissa takes a
// few thousand integer instructions.  The results are accurate to the last of
// the 53K bits the caller converts back to K limbs (a few units of
// 2^(-32(W-1)) relative), not bit-identical to the md forms.
//
// A number is (-1)^neg m 2^(e - 32W) with m = sum_i m[i] 2^(32(W-1-i)), m[0]
// the most significant word; normalized numbers have the top bit of m[0] set,
// so the value lies in [2^(e-1), 2^e).  Zero has m = 0 (and e = kZeroExp).
#pragma once
#include <cstdint>
#include <cstring>

// FXP_HD: small helpers, inlined.  FXP_NI: the W-word operations, called (not
// inlined) on the device: fully unrolled over up to 20 words, inlining them at
// every use multiplied the build time of the QR kernels several times over.
#ifdef __CUDACC__
#define FXP_HD __host__ __device__ __forceinline__
#define FXP_NI __host__ __device__ __noinline__
#else
#define FXP_HD inline
#define FXP_NI inline
#endif

namespace mdk {
namespace fxp {

constexpr int kZeroExp = -100000;
constexpr int kNanExp = 100000;  // not a number: from a non-finite input, or 1/0

// words for K limbs: 53K bits and two guard words
FXP_HD constexpr int words_for(int K) { return (53 * K + 31) / 32 + 2; }

template <int W>
struct bf {
  uint32_t m[W];
  int e;
  int neg;
};

FXP_HD uint64_t dbits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}

FXP_HD double dfrom(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}

FXP_HD int clz32(uint32_t v) {  // v != 0
#ifdef __CUDA_ARCH__
  return __clz((int)v);
#else
  return __builtin_clz(v);
#endif
}

template <int W>
FXP_HD bool is_zero(const bf<W> &a) {
  return a.m[0] == 0u;
}

template <int W>
FXP_HD bool is_nan(const bf<W> &a) {
  return a.e == kNanExp;
}

// NaN: nonzero mantissa (so that is_zero is false) and the NaN exponent; every
// operation with a NaN operand returns NaN and to_md writes NaN limbs, as the
// md forms propagate non-finite values.
template <int W>
FXP_HD bf<W> nan_value() {
  bf<W> z;
#pragma unroll
  for (int i = 0; i < W; ++i) z.m[i] = i == 0 ? 0x80000000u : 0u;
  z.e = kNanExp;
  z.neg = 0;
  return z;
}

template <int W>
FXP_HD bf<W> zero() {
  bf<W> z;
#pragma unroll
  for (int i = 0; i < W; ++i) z.m[i] = 0u;
  z.e = kZeroExp;
  z.neg = 0;
  return z;
}

// Funnel shift: the high 32 bits of (hi:lo) << s, 0 <= s < 32.
FXP_HD uint32_t fshl(uint32_t hi, uint32_t lo, int s) {
#ifdef __CUDA_ARCH__
  return __funnelshift_l(lo, hi, s);
#else
  return s ? (hi << s) | (lo >> (32 - s)) : hi;
#endif
}

// t (N words, t[0] the most significant) shifted left by s bits, 0 <= s,
// zeros shifted in: word shifts by binary stages (selects), then a funnel
// shift -- O(N log N) instead of a select per (word, offset) pair.
template <int N>
FXP_HD void shl_bits(uint32_t (&t)[N], int s) {
  const int ws = s >> 5;
#pragma unroll
  for (int b = 1; b < N; b <<= 1) {
    const bool on = (ws & b) != 0;
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = on ? (i + b < N ? t[i + b] : 0u) : t[i];
  }
  if (ws >= N) {
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = 0u;
  }
  const int bs = s & 31;
#pragma unroll
  for (int i = 0; i < N; ++i) t[i] = fshl(t[i], i + 1 < N ? t[i + 1] : 0u, bs);
}

// t shifted right by s bits, 0 <= s, zeros shifted in.
template <int N>
FXP_HD void shr_bits(uint32_t (&t)[N], int s) {
  const int ws = s >> 5;
#pragma unroll
  for (int b = 1; b < N; b <<= 1) {
    const bool on = (ws & b) != 0;
#pragma unroll
    for (int i = N - 1; i >= 0; --i) t[i] = on ? (i - b >= 0 ? t[i - b] : 0u) : t[i];
  }
  if (ws >= N) {
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = 0u;
  }
  const int bs = s & 31;
  // word i gets the low bits of word i-1 on top
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    const uint32_t prev = i > 0 ? t[i - 1] : 0u;
    t[i] = bs ? fshl(prev, t[i], 32 - bs) : t[i];
  }
}

// Shift the (W+1)-word magnitude t left until its top bit is set and keep the
// top W words; returns the shift (0 if t is zero, which the caller checks).
template <int W>
FXP_HD int normalize_words(uint32_t (&t)[W + 1], uint32_t (&out)[W]) {
  int lead = 32 * (W + 1);  // position of the first set bit
#pragma unroll
  for (int i = W; i >= 0; --i)
    if (t[i]) lead = 32 * i + clz32(t[i]);
  if (lead >= 32 * (W + 1)) lead = 0;
  shl_bits<W + 1>(t, lead);
#pragma unroll
  for (int i = 0; i < W; ++i) out[i] = t[i];
  return lead;
}

// Exact value of the K-limb md number x (rounded down in magnitude below the
// last word when its limbs span more than W words).
template <int W, int K>
FXP_HD bf<W> from_md_impl(const double (&x)[K]) {
  const uint64_t b0 = dbits(x[0]);
  const int B0 = (int)(b0 >> 52) & 0x7ff;
  bool finite = true;
#pragma unroll
  for (int l = 0; l < K; ++l) finite = finite && (((int)(dbits(x[l]) >> 52) & 0x7ff) != 0x7ff);
  if (!finite) return nan_value<W>();
  if (((b0 << 1) == 0) || B0 == 0) return zero<W>();  // zero (subnormal leads: treated as zero)
  // |x| < 2^(B0 - 1022) (1 + 2^-52) < 2^T with T = B0 - 1021: digit q of the
  // signed accumulator has weight 2^(T - 32(q+1)), q = 0..W+1
  const int T = B0 - 1021;
  int64_t acc[W + 2];
#pragma unroll
  for (int q = 0; q < W + 2; ++q) acc[q] = 0;
#pragma unroll
  for (int l = 0; l < K; ++l) {
    const uint64_t b = dbits(x[l]);
    const int B = (int)(b >> 52) & 0x7ff;
    if ((b << 1) == 0 || B == 0) continue;
    const uint64_t mant = (b & ((1ULL << 52) - 1)) | (1ULL << 52);
    const bool sgn = (b >> 63) != 0;
    // x_l = mant 2^(B - 1075): the mantissa's LSB lies `below` bits under 2^T
    const int below = T - (B - 1075);
    // split mant into its bits by 32-bit digit positions
#pragma unroll
    for (int piece = 0; piece < 2; ++piece) {
      const uint64_t chunk = piece == 0 ? (mant & 0xffffffffULL) : (mant >> 32);
      const int lsb = below - 32 * piece;  // chunk * 2^(T - lsb)
      if (lsb <= 0) continue;              // cannot happen: |x_l| < 2^T
      int q = (lsb + 31) / 32 - 1;
      const int r = 32 * (q + 1) - lsb;  // chunk << r sits in digits q (low part) and q-1 (high part)
      int64_t lo, hi;
      if (q >= W + 2) {  // below the last digit: shifted down into it (truncated)
        const int drop = lsb - 32 * (W + 2);
        lo = drop >= 64 ? 0 : (int64_t)(chunk >> drop);
        hi = 0;
        q = W + 1;
      } else {
        const uint64_t v = chunk << r;  // < 2^64 since chunk < 2^32 and r < 32
        lo = (int64_t)(v & 0xffffffffULL);
        hi = (int64_t)(v >> 32);
      }
      if (sgn) {
        lo = -lo;
        hi = -hi;
      }
      // predicated adds over the digits: no runtime index, the digits stay in registers
#pragma unroll
      for (int dg = 0; dg < W + 2; ++dg) acc[dg] += (dg == q ? lo : 0) + (dg == q - 1 ? hi : 0);
    }
  }
  // carries: digits 1..W+1 into [0, 2^32), digit 0 signed
#pragma unroll
  for (int q = W + 1; q > 0; --q) {
    const int64_t c = acc[q] >> 32;
    acc[q] -= c * 4294967296LL;
    acc[q - 1] += c;
  }
  bf<W> z;
  z.neg = acc[0] < 0;
  if (z.neg) {  // two's complement negate of the whole number
    int64_t carry = 1;
#pragma unroll
    for (int q = W + 1; q > 0; --q) {
      const int64_t v = (~acc[q] & 0xffffffffLL) + carry;
      carry = v >> 32;
      acc[q] = v & 0xffffffffLL;
    }
    acc[0] = -acc[0] - 1 + carry;
  }
  // digit 0 is below 2^32 here (|x| < 2^T); keep W+1 words, then normalize
  uint32_t t[W + 1];
#pragma unroll
  for (int q = 0; q <= W; ++q) t[q] = (uint32_t)acc[q];
  if (t[0] == 0u && t[1] == 0u && t[2] == 0u) {
    bool nz = false;
#pragma unroll
    for (int q = 0; q <= W; ++q) nz = nz || t[q] != 0u;
    if (!nz) return zero<W>();
  }
  const int s = normalize_words<W>(t, z.m);
  // value = t 2^(T - 32(W+1)) = m 2^(T - 32(W+1) - s + 32) = m 2^(e - 32W)
  z.e = T - s;
  return z;
}

// Bit p (from the top, p >= 0) of the mantissa onwards: the first set bit at
// or after p, or -1.
template <int W>
FXP_HD int first_set(const bf<W> &a, int p) {
  int r = -1;
#pragma unroll
  for (int i = W - 1; i >= 0; --i) {
    uint32_t v = a.m[i];
    const int lo = 32 * i;  // word i covers bits [32 i, 32 i + 32)
    if (p > lo + 31) v = 0u;
    else if (p > lo) v &= 0xffffffffu >> (p - lo);
    if (v) r = lo + clz32(v);
  }
  return r;
}

// K-limb md value: each limb is the 53 bits of the mantissa from the first set
// bit after the previous limb, so no limb overlaps the next; the last limb is
// rounded to nearest on the next bit (a truncation would bias every result
// toward zero, and those biases add up along the degrees of the solve).
template <int K, int W>
FXP_HD void to_md_impl(const bf<W> &a, double (&z)[K]) {
#pragma unroll
  for (int l = 0; l < K; ++l) z[l] = is_nan(a) ? dfrom(0x7ff8000000000000ULL) : 0.0;
  if (is_zero(a) || is_nan(a)) return;
  int p = 0;  // the top bit is set
  int plast = -1, last = -1;
#pragma unroll
  for (int l = 0; l < K; ++l) {
    if (p < 0 || p >= 32 * W) break;
    const int w = p >> 5, o = p & 31;
    uint32_t w0 = 0u, w1 = 0u, w2 = 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      if (i == w) w0 = a.m[i];
      if (i == w + 1) w1 = a.m[i];
      if (i == w + 2) w2 = a.m[i];
    }
    uint64_t win = (((uint64_t)w0 << 32) | w1) << o;
    if (o) win |= (uint64_t)w2 >> (32 - o);
    const uint64_t mant = win >> 11;  // 53 bits, bit 52 set (bit p is set)
    // bit p has weight 2^(e - 1 - p): value = mant 2^(e - 1 - p - 52)
    const int Be = a.e - 1 - p - 52 + 1075;
    if (Be <= 0 || Be >= 2047) break;  // outside the double range: dropped
    z[l] = dfrom(((uint64_t)a.neg << 63) | ((uint64_t)Be << 52) | (mant & ((1ULL << 52) - 1)));
    plast = p;
    last = l;
    p = first_set<W>(a, p + 53);
  }
  if (last == K - 1) {  // round the last limb on the bit below it
    const int q = plast + 53;
    if (q < 32 * W) {
      uint32_t wq = 0u;
#pragma unroll
      for (int i = 0; i < W; ++i)
        if (i == (q >> 5)) wq = a.m[i];
      const int Bu = a.e - 1 - plast - 52 + 1023;  // the last limb's unit in the last place
      if (((wq >> (31 - (q & 31))) & 1u) && Bu > 0) {
        const double ulp = dfrom((uint64_t)Bu << 52);
        z[K - 1] = z[K - 1] + (a.neg ? -ulp : ulp);  // exact: (mant + 1) 2^(exp), at most a power of two
      }
    }
  }
}

template <int W>
FXP_HD bf<W> from_double(double x) {
  double v[1] = {x};
  return from_md_impl<W, 1>(v);
}

// Truncated product: the top W words of the 2W-word product (partial
// products of words i + j <= W), normalized.
template <int W>
FXP_HD bf<W> mul_impl(const bf<W> &a, const bf<W> &b) {
  if (is_nan(a) || is_nan(b)) return nan_value<W>();
  if (is_zero(a) || is_zero(b)) return zero<W>();
  uint64_t col[W + 2];
#pragma unroll
  for (int k = 0; k < W + 2; ++k) col[k] = 0ULL;
#pragma unroll
  for (int i = 0; i < W; ++i)
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (i + j <= W) {
        const uint64_t p = (uint64_t)a.m[i] * b.m[j];
        col[i + j] += p >> 32;
        col[i + j + 1] += p & 0xffffffffULL;
      }
#pragma unroll
  for (int k = W + 1; k > 0; --k) {
    col[k - 1] += col[k] >> 32;
    col[k] &= 0xffffffffULL;
  }
  // product = col 2^(ea + eb - 64W) with col[0] the word of weight 2^(32(2W-1)) ...;
  // its top bit is bit 31 or 30 of col[0] (both mantissas >= 2^(32W-1))
  bf<W> z;
  const int s = (col[0] >> 31) ? 0 : 1;  // the top bit is bit 31 or 30 of word 0
#pragma unroll
  for (int k = 0; k < W; ++k)
    z.m[k] = s ? (((uint32_t)col[k] << 1) | ((uint32_t)col[k + 1] >> 31)) : (uint32_t)col[k];
  z.e = a.e + b.e - s;
  z.neg = a.neg ^ b.neg;
  return z;
}

// |a| >= |b| for normalized numbers.
template <int W>
FXP_HD bool mag_ge(const bf<W> &a, const bf<W> &b) {
  if (a.e != b.e) return a.e > b.e;
  int r = 0;  // first differing word decides
#pragma unroll
  for (int i = W - 1; i >= 0; --i) r = a.m[i] > b.m[i] ? 1 : (a.m[i] < b.m[i] ? -1 : r);
  return r >= 0;
}

// a + b (signs included), truncated to W words.
template <int W>
FXP_HD bf<W> add_impl(const bf<W> &a, const bf<W> &b) {
  if (is_nan(a) || is_nan(b)) return nan_value<W>();
  if (is_zero(b)) return a;
  if (is_zero(a)) return b;
  const bool a_big = mag_ge<W>(a, b);
  const bf<W> &x = a_big ? a : b;
  const bf<W> &y = a_big ? b : a;
  const int d = x.e - y.e;  // >= 0
  if (d >= 32 * W + 32) return x;
  // y's mantissa shifted right by d into W+1 words (one guard word); x's words
  // shifted right by one word position as well so that a carry fits
  // a (W+2)-word frame: word 0 takes a carry, words 1..W hold x, word W+1 is
  // a guard word; y is shifted right by d bits into the same frame
  uint32_t xs[W + 2], ys[W + 2];
  xs[0] = 0u;
  ys[0] = 0u;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    xs[i + 1] = x.m[i];
    ys[i + 1] = y.m[i];
  }
  xs[W + 1] = 0u;
  ys[W + 1] = 0u;
  shr_bits<W + 2>(ys, d);
  uint32_t r[W + 2];
  if (x.neg == y.neg) {
    uint64_t carry = 0;
#pragma unroll
    for (int i = W + 1; i >= 0; --i) {
      const uint64_t s = (uint64_t)xs[i] + ys[i] + carry;
      r[i] = (uint32_t)s;
      carry = s >> 32;
    }
  } else {
    int64_t borrow = 0;
#pragma unroll
    for (int i = W + 1; i >= 0; --i) {
      const int64_t s = (int64_t)xs[i] - ys[i] - borrow;
      r[i] = (uint32_t)s;
      borrow = s < 0 ? 1 : 0;
    }
  }
  uint32_t t[W + 1];
#pragma unroll
  for (int i = 0; i <= W; ++i) t[i] = r[i];
  bool nz = false;
#pragma unroll
  for (int i = 0; i <= W; ++i) nz = nz || t[i] != 0u;
  if (!nz) return zero<W>();
  bf<W> z;
  const int s = normalize_words<W>(t, z.m);
  z.e = x.e + 32 - s;
  z.neg = x.neg;
  return z;
}

// The W-word operations as called (not inlined) on the device; a kernel that
// needs them inlined (the series products, where passing W-word values through
// the call stack cost more than the arithmetic) calls the *_impl forms.
template <int W, int K>
FXP_NI bf<W> from_md(const double (&x)[K]) {
  return from_md_impl<W, K>(x);
}

template <int K, int W>
FXP_NI void to_md(const bf<W> &a, double (&z)[K]) {
  to_md_impl<K, W>(a, z);
}

template <int W>
FXP_NI bf<W> mul(const bf<W> &a, const bf<W> &b) {
  return mul_impl<W>(a, b);
}

template <int W>
FXP_NI bf<W> add(const bf<W> &a, const bf<W> &b) {
  return add_impl<W>(a, b);
}

template <int W>
FXP_HD bf<W> neg(bf<W> a) {
  a.neg ^= 1;
  return a;
}

// a 2^k
template <int W>
FXP_HD bf<W> ldexp(bf<W> a, int k) {
  if (!is_zero(a) && !is_nan(a)) a.e += k;
  return a;
}

// Leading double of a (truncated), for Newton seeds; a must be in the double range.
template <int W>
FXP_HD double lead_double(const bf<W> &a) {
  double z[1];
  to_md<1, W>(a, z);
  return z[0];
}

// Newton steps for K limbs from a 50-bit seed: 53K + 16 bits.
FXP_HD constexpr int newton_steps(int K) {
  return K <= 1 ? 0 : (53 * K + 16 <= 100 ? 1 : (53 * K + 16 <= 200 ? 2 : (53 * K + 16 <= 400 ? 3 : 4)));
}

// a with W2 words (the top min(W, W2) words; zeros below, or the low words
// dropped: truncation toward zero).
template <int W2, int W>
FXP_HD bf<W2> resize(const bf<W> &a) {
  bf<W2> z;
#pragma unroll
  for (int i = 0; i < W2; ++i) z.m[i] = i < W ? a.m[i] : 0u;
  z.e = a.e;
  z.neg = a.neg;
  return z;
}

// Words for Newton step s of STEPS: the step doubles the accuracy to
// 50 2^(s+1) bits (from a ~50-bit seed), so it is carried out on that many
// bits, 16 more and a guard word; the last step on all W words.
FXP_HD constexpr int stage_words(int W, int s, int STEPS) {
  return s + 1 >= STEPS ? W : ((((50 << (s + 1)) + 16 + 31) / 32 + 1) < W ? ((50 << (s + 1)) + 16 + 31) / 32 + 1 : W);
}

// One step y <- y + y (1 - a y^2) / 2 on WS words.
template <int W, int WS>
FXP_HD void rsqrt_step(const bf<W> &a, bf<W> &y) {
  const bf<WS> as = resize<WS>(a), ys = resize<WS>(y), one = from_double<WS>(1.0);
  const bf<WS> t = mul<WS>(mul<WS>(as, ys), ys);
  const bf<WS> r = add<WS>(one, neg<WS>(t));
  y = resize<W>(add<WS>(ys, ldexp<WS>(mul<WS>(ys, r), -1)));
}

// One step y <- y + y (1 - a y) on WS words.
template <int W, int WS>
FXP_HD void recip_step(const bf<W> &a, bf<W> &y) {
  const bf<WS> as = resize<WS>(a), ys = resize<WS>(y), one = from_double<WS>(1.0);
  const bf<WS> r = add<WS>(one, neg<WS>(mul<WS>(as, ys)));
  y = resize<W>(add<WS>(ys, mul<WS>(ys, r)));
}

// 1 / sqrt(a), a > 0: y <- y + y (1 - a y^2) / 2, each step on the words its
// accuracy needs (stage_words).  The seed comes from the leading bits of a
// scaled into [1/4, 1) by an even power of two.
template <int W, int STEPS>
FXP_NI bf<W> rsqrt(const bf<W> &a) {
  static_assert(STEPS <= 4, "at most four Newton steps");
  if (is_nan(a) || is_zero(a) || a.neg) return nan_value<W>();  // as 1/sqrt(0) is not finite
  bf<W> as = a;
  const int ee = (a.e % 2 == 0) ? a.e : a.e + 1;  // a = as 2^ee with as in [1/4, 1)
  as.e -= ee;
  double s = lead_double<W>(as);
#ifdef __CUDA_ARCH__
  const double y0 = 1.0 / __dsqrt_rn(s);
#else
  const double y0 = 1.0 / __builtin_sqrt(s);
#endif
  bf<W> y = from_double<W>(y0);
  if constexpr (STEPS > 0) rsqrt_step<W, stage_words(W, 0, STEPS)>(as, y);
  if constexpr (STEPS > 1) rsqrt_step<W, stage_words(W, 1, STEPS)>(as, y);
  if constexpr (STEPS > 2) rsqrt_step<W, stage_words(W, 2, STEPS)>(as, y);
  if constexpr (STEPS > 3) rsqrt_step<W, stage_words(W, 3, STEPS)>(as, y);
  return ldexp<W>(y, -ee / 2);
}

// 1 / a, a != 0: y <- y + y (1 - a y), each step on the words its accuracy
// needs.
template <int W, int STEPS>
FXP_NI bf<W> recip(const bf<W> &a) {
  static_assert(STEPS <= 4, "at most four Newton steps");
  if (is_nan(a) || is_zero(a)) return nan_value<W>();  // as 1/0 is not finite
  bf<W> as = a;
  as.e = 0;  // as in [1/2, 1)
  as.neg = 0;
  const double s = lead_double<W>(as);
  bf<W> y = from_double<W>(1.0 / s);
  if constexpr (STEPS > 0) recip_step<W, stage_words(W, 0, STEPS)>(as, y);
  if constexpr (STEPS > 1) recip_step<W, stage_words(W, 1, STEPS)>(as, y);
  if constexpr (STEPS > 2) recip_step<W, stage_words(W, 2, STEPS)>(as, y);
  if constexpr (STEPS > 3) recip_step<W, stage_words(W, 3, STEPS)>(as, y);
  y.e -= a.e;
  y.neg = a.neg;
  return y;
}

}  // namespace fxp
}  // namespace mdk
