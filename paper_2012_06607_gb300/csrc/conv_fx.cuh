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
// at least as accurate as the md form (one rounding to K limbs, to nearest,
// instead of a rounding in every operation) but not its bits: the
// split-product form is checked against the oracle by tolerance, the plain
// form keeps the bits.  Used from kFxConvMinLimbs limbs on: at double double
// the md form is faster.
#pragma once
#include "house_fx.cuh"

namespace mdk {

// The fixed-point copy of the series pool: every value of the md pool
// [series][d+1][P][K] as a W-word number, stored in packed_words(W) 32-bit
// words (the mantissa words, then the exponent shifted left by one with the
// sign in bit 0, zeros to a multiple of four words), so that a value moves in
// 16-byte loads.  The products convert each operand once, where it is made,
// instead of at every term that reads it (a K-limb conversion costs about as
// much as two W-word products).
__host__ __device__ constexpr int packed_words(int W) { return (W + 4) & ~3; }
static_assert(packed_words(fxp::words_for(3)) == fx_packed_words_for(3) &&
                  packed_words(fxp::words_for(10)) == fx_packed_words_for(10),
              "the host's workspace layout uses the same packed size");

template <int W>
__device__ __forceinline__ void fx_st_packed(uint32_t *dst, const fxp::bf<W> &a) {
  constexpr int PW = packed_words(W);
  uint32_t w[PW];
#pragma unroll
  for (int i = 0; i < PW; ++i) w[i] = i < W ? a.m[i] : 0u;
  w[W] = ((uint32_t)a.e << 1) | (uint32_t)(a.neg & 1);
#pragma unroll
  for (int q = 0; q < PW / 4; ++q)
    reinterpret_cast<uint4 *>(dst)[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

template <int W>
__device__ __forceinline__ fxp::bf<W> fx_ld_packed(const uint32_t *src) {
  constexpr int PW = packed_words(W);
  uint32_t w[PW];
#pragma unroll
  for (int q = 0; q < PW / 4; ++q) {
    const uint4 v = reinterpret_cast<const uint4 *>(src)[q];
    w[4 * q] = v.x;
    w[4 * q + 1] = v.y;
    w[4 * q + 2] = v.z;
    w[4 * q + 3] = v.w;
  }
  fxp::bf<W> a;
#pragma unroll
  for (int i = 0; i < W; ++i) a.m[i] = w[i];
  a.e = (int)w[W] >> 1;
  a.neg = (int)(w[W] & 1u);
  return a;
}

// A value of P planes rounded to K limbs, stored in the md pool and, as the
// exact value of those limbs, in the fixed-point pool.
template <int W, int K, int P>
__device__ __forceinline__ void fx_st_both(double *dst, uint32_t *pdst, const fxp::bf<W> (&v)[P]) {
  constexpr int PW = packed_words(W);
#pragma unroll
  for (int p = 0; p < P; ++p) {
    double z[K];
    fxp::to_md<K, W>(v[p], z);
#pragma unroll
    for (int l = 0; l < K; ++l) dst[p * K + l] = z[l];
    fx_st_packed<W>(pdst + p * PW, fxp::from_md<W, K>(z));
  }
}

// One md value of P planes (limb l of plane p at src[(p K + l) stride]) into
// the packed fixed-point form at dst (P packed values).
template <int K, int P>
__device__ __forceinline__ void fx_pack_value(const double *src, long long stride, uint32_t *dst) {
  constexpr int W = fxp::words_for(K), PW = packed_words(W);
#pragma unroll
  for (int p = 0; p < P; ++p) {
    double v[K];
#pragma unroll
    for (int l = 0; l < K; ++l) v[l] = src[(long long)(p * K + l) * stride];
    fx_st_packed<W>(dst + p * PW, fxp::from_md<W, K>(v));
  }
}

// The inputs' series into both pools (pool_load_entry, and each value
// converted once for the fixed-point products).
template <int K, int P>
__device__ __forceinline__ void pool_load_entry_fx(const double *x, double *pool, uint32_t *fxpool, int n, int d,
                                                   long long e) {
  constexpr int PW = packed_words(fxp::words_for(K));
  const long long stride = (long long)n * (d + 1);
  fx_pack_value<K, P>(x + e, stride, fxpool + e * P * PW);
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) pool[e * (P * K) + p * K + l] = x[e + (long long)(p * K + l) * stride];
}

template <int K, int P>
__global__ void pool_load_x_fx_kernel(const double *__restrict__ x, double *__restrict__ pool,
                                      uint32_t *__restrict__ fxpool, int n, int d) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * (d + 1)) return;
  pool_load_entry_fx<K, P>(x, pool, fxpool, n, d, e);
}

// acc += a b (complex for P = 2) with the W-word products and sums inlined:
// the values stay in registers (the out-of-line forms pass every operand and
// result through the call stack, and that local-memory traffic, not the
// integer arithmetic, bounded the products).  The same operations in the same
// order as fx_cmul followed by add.
template <int W, int P>
__device__ __forceinline__ void fx_cmac_inl(fxp::bf<W> (&acc)[P], const fxp::bf<W> (&a)[P],
                                            const fxp::bf<W> (&b)[P]) {
  using namespace fxp;
  if constexpr (P == 1) {
    acc[0] = add_impl<W>(acc[0], mul_impl<W>(a[0], b[0]));
  } else {
    const bf<W> re = add_impl<W>(mul_impl<W>(a[0], b[0]), neg<W>(mul_impl<W>(a[1], b[1])));
    const bf<W> im = add_impl<W>(mul_impl<W>(a[0], b[1]), mul_impl<W>(a[1], b[0]));
    acc[0] = add_impl<W>(acc[0], re);
    acc[1] = add_impl<W>(acc[1], im);
  }
}

// Two output coefficients of series products as conv_pair (same task layout
// and term order), in fixed point: the operands from the fixed-point pool,
// every term inlined (fx_cmac_inl), the outputs rounded to K limbs into the
// md pool and, as the exact values of those limbs, into the fixed-point pool.
template <int K, int P>
__device__ __forceinline__ void conv_pair_fx(double *pool, uint32_t *fxpool, int d, int outA, int xA, int yA, int kA,
                                             int outB, int xB, int yB) {
  using namespace fxp;
  constexpr int W = words_for(K), PW = packed_words(W);
  const int kB = d - kA;
  const long long VS = P * K, SS = (long long)(d + 1) * VS;
  const long long FS = (long long)(d + 1) * P * PW, FV = (long long)P * PW;  // fixed-point pool strides
  const int total = (outB >= 0) ? (d + 2) : (kA + 1);
  bf<W> acc[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = zero<W>();
  for (int it = 0; it < total; ++it) {
    const bool first = it <= kA;
    const int i = first ? it : it - kA - 1;
    const int sx = first ? xA : xB, sy = first ? yA : yB, iy = (first ? kA : kB) - i;
    bf<W> a[P], b[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      a[p] = fx_ld_packed<W>(fxpool + sx * FS + i * FV + p * PW);
      b[p] = fx_ld_packed<W>(fxpool + sy * FS + iy * FV + p * PW);
    }
    if (it == kA + 1) {
#pragma unroll
      for (int p = 0; p < P; ++p) acc[p] = zero<W>();
    }
    fx_cmac_inl<W, P>(acc, a, b);
    if (it == kA) fx_st_both<W, K, P>(pool + outA * SS + kA * VS, fxpool + outA * FS + kA * FV, acc);
  }
  if (outB >= 0) fx_st_both<W, K, P>(pool + outB * SS + kB * VS, fxpool + outB * FS + kB * FV, acc);
}

// z = a b (complex for P = 2) with the W-word products and sums inlined (the
// operations of fx_cmul).
template <int W, int P>
__device__ __forceinline__ void fx_cmul_inl(const fxp::bf<W> (&a)[P], const fxp::bf<W> (&b)[P],
                                            fxp::bf<W> (&z)[P]) {
  using namespace fxp;
  if constexpr (P == 1) {
    z[0] = mul_impl<W>(a[0], b[0]);
  } else {
    z[0] = add_impl<W>(mul_impl<W>(a[0], b[0]), neg<W>(mul_impl<W>(a[1], b[1])));
    z[1] = add_impl<W>(mul_impl<W>(a[0], b[1]), mul_impl<W>(a[1], b[0]));
  }
}

// ------------------------------------------------- accumulation of f and A_k
// The split-product form's accumulation (Section 4, the linearization): the
// steps of accum_contrib_value / accum_entry on the packed fixed-point copies
// of the coefficients (fxscal: nscal values of P packed planes) and of the
// series pool, each contribution value an exact word-slice product, each
// entry's sum (constant term, then the contributions in list order) kept in
// W-word fixed point and rounded to K limbs once.

// Coefficient k of one contribution: c s_{k-a} for a product slot s, c at
// k = a for the unit series, zero for k < a.
template <int K, int P>
__device__ __forceinline__ void accum_contrib_value_fx(const int4 C, const uint32_t *fxpool, const uint32_t *fxscal,
                                                       int d, int k, fxp::bf<fxp::words_for(K)> (&v)[P]) {
  using namespace fxp;
  constexpr int W = words_for(K), PW = packed_words(W);
#pragma unroll
  for (int p = 0; p < P; ++p) v[p] = zero<W>();
  if (k < C.z) return;
  bf<W> c[P];
#pragma unroll
  for (int p = 0; p < P; ++p) c[p] = fx_ld_packed<W>(fxscal + ((long long)C.y * P + p) * PW);
  if (C.x < 0) {
    if (k == C.z) {
#pragma unroll
      for (int p = 0; p < P; ++p) v[p] = c[p];
    }
    return;
  }
  bf<W> sv[P];
#pragma unroll
  for (int p = 0; p < P; ++p)
    sv[p] = fx_ld_packed<W>(fxpool + (((long long)C.x * (d + 1) + (k - C.z)) * P + p) * PW);
  fx_cmul_inl<W, P>(c, sv, v);
}

// The sum of one entry (group g, coefficient k) from its constant term and
// the contribution values get(q), q < G.w, rounded to K limbs into f or A.
template <int K, int P, class Get>
__device__ __forceinline__ void accum_finish_fx(const int4 G, const double *cst, double *f, double *A, int N, int n,
                                                int d, int k, Get get) {
  using namespace fxp;
  constexpr int W = words_for(K);
  bf<W> acc[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = zero<W>();
  if (G.y < 0 && k == 0) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      double c[K];
#pragma unroll
      for (int l = 0; l < K; ++l) c[l] = cst[G.x + (long long)(p * K + l) * N];
      acc[p] = from_md<W, K>(c);
    }
  }
  for (int q = 0; q < G.w; ++q) {
    bf<W> v[P];
    get(q, v);
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = add_impl<W>(acc[p], v[p]);
  }
  // f: [P][K][N][d+1]; A: [P][K][d+1][n][N]
  double *dst;
  long long stride;
  if (G.y < 0) {
    dst = f + (long long)G.x * (d + 1) + k;
    stride = (long long)N * (d + 1);
  } else {
    const long long nn = (long long)N * n;
    dst = A + (long long)k * nn + (long long)G.y * N + G.x;
    stride = (long long)(d + 1) * nn;
  }
#pragma unroll
  for (int p = 0; p < P; ++p) {
    double z[K];
    to_md<K, W>(acc[p], z);
#pragma unroll
    for (int l = 0; l < K; ++l) dst[(long long)(p * K + l) * stride] = z[l];
  }
}

// One entry in one pass (the batched kernel's form of accum_entry).
template <int K, int P>
__device__ __forceinline__ void accum_entry_fx(const int4 *groups, const int4 *contrib, const uint32_t *fxpool,
                                               const uint32_t *fxscal, const double *cst, double *f, double *A, int N,
                                               int n, int d, int g, int k) {
  const int4 G = groups[g];
  accum_finish_fx<K, P>(G, cst, f, A, N, n, d, k, [&](int q, fxp::bf<fxp::words_for(K)>(&v)[P]) {
    accum_contrib_value_fx<K, P>(contrib[G.z + q], fxpool, fxscal, d, k, v);
  });
}

// Two passes, as accum_prod_kernel / accum_sum_kernel: every contribution
// value (packed) to fxprod [contribution][k], then each entry's sum.
template <int K, int P>
__global__ void __launch_bounds__(128) accum_prod_fx_kernel(const int4 *__restrict__ contrib, int ncontrib,
                                                            const uint32_t *__restrict__ fxpool,
                                                            const uint32_t *__restrict__ fxscal,
                                                            uint32_t *__restrict__ fxprod, int d) {
  constexpr int W = fxp::words_for(K), PW = packed_words(W);
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)ncontrib * (d + 1)) return;
  const int q = (int)(e / (d + 1)), k = (int)(e % (d + 1));
  fxp::bf<W> v[P];
  accum_contrib_value_fx<K, P>(contrib[q], fxpool, fxscal, d, k, v);
#pragma unroll
  for (int p = 0; p < P; ++p) fx_st_packed<W>(fxprod + (e * P + p) * PW, v[p]);
}

// Entries (group, k); the A groups at k = 0 are skipped when skip_A0 is set
// (coefficient 0 of A comes from the md pre-pass).
template <int K, int P>
__global__ void __launch_bounds__(128) accum_sum_fx_kernel(const int4 *__restrict__ groups, int ngroups,
                                                           const uint32_t *__restrict__ fxprod,
                                                           const double *__restrict__ cst, double *__restrict__ f,
                                                           double *__restrict__ A, int N, int n, int d, int skip_A0) {
  constexpr int W = fxp::words_for(K), PW = packed_words(W);
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)ngroups * (d + 1)) return;
  const int g = (int)(e / (d + 1)), k = (int)(e % (d + 1));
  const int4 G = groups[g];
  if (skip_A0 && k == 0 && G.y >= 0) return;
  accum_finish_fx<K, P>(G, cst, f, A, N, n, d, k, [&](int q, fxp::bf<W>(&v)[P]) {
#pragma unroll
    for (int p = 0; p < P; ++p)
      v[p] = fx_ld_packed<W>(fxprod + (((long long)(G.z + q) * (d + 1) + k) * P + p) * PW);
  });
}

// One chunk of a row of the block Toeplitz update sum_{j<k} A_{k-j} dx_j
// (Section 3.2; rhs_partial_item's terms in its order) in fixed point: the
// operands from packed fixed-point copies of A (fxA: the values of A in A's
// order [d+1][n][N], P packed values each) and of dx (fxdx: [d+1][n]), every
// term an exact product of word slices, the chunk's sum rounded to K limbs
// once into part ([N][nchunk] values).
template <int K, int P>
__device__ __forceinline__ void rhs_partial_item_fx(const uint32_t *fxA, const uint32_t *fxdx, double *part, int N,
                                                    int n, int k, int C, int nchunk, long long e) {
  using namespace fxp;
  constexpr int W = words_for(K), PW = packed_words(W);
  const int row = (int)(e % N), chunk = (int)(e / N);
  const long long nn = (long long)N * n, VS = P * K;
  const int t0 = chunk * C, t1 = min(t0 + C, k * n);
  bf<W> acc[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = zero<W>();
  for (int t = t0; t < t1; ++t) {
    const int j = t / n, col = t % n;
    const uint32_t *ap = fxA + ((long long)(k - j) * nn + (long long)col * N + row) * P * PW;
    const uint32_t *xp = fxdx + ((long long)j * n + col) * P * PW;
    bf<W> a[P], x[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      a[p] = fx_ld_packed<W>(ap + p * PW);
      x[p] = fx_ld_packed<W>(xp + p * PW);
    }
    fx_cmac_inl<W, P>(acc, a, x);
  }
  fx_st_val<W, K, P>(part + ((long long)row * nchunk + chunk) * VS, acc);
}

// The resident stage launch of conv_stage_resident_kernel in fixed point
// (same grid and task numbering).  Threads per CTA by limb count so that the
// inlined terms fit in registers without spilling: 512 threads (128
// registers) up to three limbs, 384 (168) at four, 256 (255) from five on.
template <int K>
__host__ __device__ constexpr int conv_fx_threads() {
  return K <= 3 ? 512 : (K == 4 ? 384 : 256);
}

template <int K, int P>
__global__ void __launch_bounds__(conv_fx_threads<K>(), 1)
    conv_stage_fx_kernel(const int *__restrict__ tasks, int ntask, double *pool, uint32_t *fxpool, int d) {
  for (int t = threadIdx.x * gridDim.x + blockIdx.x; t < ntask; t += gridDim.x * blockDim.x) {
    const int4 t0 = __ldg(reinterpret_cast<const int4 *>(tasks) + 2 * t);
    const int4 t1 = __ldg(reinterpret_cast<const int4 *>(tasks) + 2 * t + 1);
    conv_pair_fx<K, P>(pool, fxpool, d, t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z);
  }
}

}  // namespace mdk
