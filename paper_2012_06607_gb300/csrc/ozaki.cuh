// Split-product ("Ozaki") form of the block Toeplitz update
//   r_k = b_k - sum_{j<k} A_{k-j} dx_j          (Section 4)
// on the BF16 tensor pipe.
//
// Every md number v of a row of a block A_i (or of a vector dx_j) is written
// relative to a shared exponent e as  v ~ sum_{s<S} v_s 2^(e - 8(s+1))  with
// integer slices v_s in [-128, 128] (bf16 holds them exactly); the truncation is
// below 2^(e - 8S), i.e. 2^-8S relative to the largest entry.  Products of
// slices are integers below 2^14; K <= 1024 of them sum below 2^24, so the
// tensor core's fp32 accumulation of a BF16 mma is exact.  For each pair
// (row of block A_{k-j}, vector dx_j) the S x S slice products
// C[s][t] = sum_col A_s x_t (K = n) are formed on the tensor pipe inside the
// update kernel.  The terms of r_k -- the C values with their power-of-two
// weights and the limbs of b_k -- are added exactly into a fixed-point integer
// (int64 digits of 32 bits in shared memory) and converted to K limbs once.  The only rounding is the slicing
// (normwise 2^(12 - 8S) relative to the largest term) and the final K-limb
// truncation; the plain path rounds at every md multiply-add.
#pragma once
#include <cuda_bf16.h>

#include <cmath>

#include "md.cuh"

namespace mdk {

// Slices per real number: 53K + 24 bits, rounded up to a multiple of 16 slices
// (so that n P S rows tile by 16 for any n).
__host__ __device__ constexpr int oz_slices(int K) { return (((53 * K + 24 + 7) / 8) + 15) / 16 * 16; }
// Fixed-point accumulator digits (32 bits each): 53K + 24 bits of precision,
// 64 bits of headroom above the largest term and 64 guard bits.
__host__ __device__ constexpr int oz_digits(int K) { return (53 * K + 24 + 128 + 31) / 32 + 1; }

__host__ __device__ inline int oz_kpad(int n) { return (n + 15) / 16 * 16; }

// The exponent that marks a row, a vector or a right-hand side holding a
// non-finite limb: it puts the output's accumulator top above
// kOzNonFiniteTop, every finite term then falls below the accumulator (and
// is dropped), and oz_finish_kernel writes NaN limbs, as md arithmetic
// propagates non-finite values.
constexpr int kOzNonFinite = 1 << 20;
constexpr int kOzNonFiniteTop = kOzNonFinite / 2;

__device__ __forceinline__ bool oz_finite(double x) {
  return (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffULL) != 0x7ffULL;
}

// exponent e with |v| < 2^(e-1) for the md number whose leading limb is x0
// (-2000 for zero, kOzNonFinite for a non-finite limb).
__device__ __forceinline__ int oz_exp_bound(double x0) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x0) & 0x7fffffffffffffffULL;
  if (b == 0ULL) return -2000;
  int ex = (int)(b >> 52);
  if (ex == 0x7ff) return kOzNonFinite;
  if (ex == 0) {  // subnormal: frexp exponent
    ex = -1022 - (__clzll((long long)b) - 12) + 1;
    return ex + 1;
  }
  return ex - 1022 + 1;  // |x0| < 2^(ex-1022); one more bit covers the lower limbs
}

// Signed fixed-point integer with W 32-bit digits held in int64 (carry-save);
// digit 0 is the most significant and has weight 2^(top - 32).
template <int W>
struct oz_fix {
  long long d[W];
};

// Add the double x (exactly) into a fixed-point number whose digit 0 covers
// bits [top-32, top); bits below the last digit are dropped (truncated).
template <int W>
__device__ __forceinline__ void oz_add_double(oz_fix<W> &a, int top, double x, int sign) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = b & 0x7fffffffffffffffULL;
  if (mag == 0ULL) return;
  const int ex = (int)(mag >> 52);
  unsigned long long m = mag & 0xfffffffffffffULL;
  int e2;  // x = +-m * 2^e2
  if (ex == 0) {
    e2 = -1074;
  } else {
    m |= 1ULL << 52;
    e2 = ex - 1075;
  }
  const bool neg = ((b >> 63) != 0ULL) != (sign < 0);
  // bit position of the mantissa's LSB counted down from `top`
  const int below = top - e2;  // m*2^e2 = m * 2^(top - below)
  // place m (53 bits) as 32-bit chunks at the right digits
  for (int piece = 0; piece < 2; ++piece) {
    const unsigned long long chunk = piece == 0 ? (m & 0xffffffffULL) : (m >> 32);
    const int lsb_below = below - 32 * piece;  // chunk * 2^(top - lsb_below)
    // digit q has weight 2^(top - 32(q+1)); chunk*2^(top - lsb_below) = chunk*2^r * 2^(top-32(q+1))
    int q = (lsb_below + 31) / 32 - 1;  // digit containing the LSB when r >= 0
    int r = 32 * (q + 1) - lsb_below;   // 0..31
    if (lsb_below <= 0) continue;       // above the top: cannot happen with proper headroom
    if (q >= W) {
      // LSB below the accumulator: shift the chunk down and drop the bits
      const int drop = lsb_below - 32 * W;
      if (drop >= 64) continue;
      const unsigned long long c = chunk >> drop;
      q = W - 1;
      r = 0;
      const long long v = (long long)c;
      a.d[q] += neg ? -v : v;
      continue;
    }
    const unsigned long long v = chunk << r;  // < 2^63
    const long long lo = (long long)(v & 0xffffffffULL), hi = (long long)(v >> 32);
    a.d[q] += neg ? -lo : lo;
    if (q > 0) a.d[q - 1] += neg ? -hi : hi;
  }
}

// Propagate carries: afterwards d[1..W-1] in [0, 2^32), d[0] signed.
template <int W>
__device__ __forceinline__ void oz_normalize(oz_fix<W> &a) {
#pragma unroll
  for (int q = W - 1; q > 0; --q) {
    const long long c = a.d[q] >> 32;  // arithmetic shift: floor division
    a.d[q] -= c << 32;
    a.d[q - 1] += c;
  }
}

// K-limb md value of the fixed-point number (top as in oz_add_double): limbs
// are consecutive 53-bit chunks of the magnitude (truncated), each starting at
// the first set bit after the previous one.  Word operations only: the
// magnitude is a stream of 32-bit words, MSB first.
template <int W, int K>
__device__ __forceinline__ void oz_to_md(oz_fix<W> a, int top, double (&z)[K]) {
  oz_normalize<W>(a);
  const bool neg = a.d[0] < 0;
  if (neg) {  // two's complement negate
    long long carry = 1;
#pragma unroll
    for (int q = W - 1; q > 0; --q) {
      long long v = (~a.d[q] & 0xffffffffLL) + carry;
      carry = v >> 32;
      a.d[q] = v & 0xffffffffLL;
    }
    a.d[0] = -a.d[0] - 1 + carry;
  }
#pragma unroll
  for (int l = 0; l < K; ++l) z[l] = 0.0;
  // stream words: the 64-bit head d[0] (units of 2^(top-32)) as two words, then d[1..W-1]
  constexpr int NWD = W + 1;
  unsigned wd[NWD];
  const unsigned long long head = (unsigned long long)a.d[0];
  wd[0] = (unsigned)(head >> 32);
  wd[1] = (unsigned)head;
#pragma unroll
  for (int q = 1; q < W; ++q) wd[q + 1] = (unsigned)a.d[q];
  // stream bit p (p = 0 is the MSB of wd[0]) has weight 2^(top - 32 + 63 - p)
  auto first_set = [&](int p) -> int {  // first set bit at or after p, or -1
    for (int w = p >> 5; w < NWD; ++w) {
      unsigned v = wd[w];
      if (w == (p >> 5)) v &= 0xffffffffu >> (p & 31);
      if (v) return 32 * w + __clz((int)v);
    }
    return -1;
  };
  auto bits53 = [&](int p) -> unsigned long long {  // stream bits [p, p + 53), zero past the end
    unsigned long long win = 0;  // 64 bits starting at p
    const int w = p >> 5, o = p & 31;
    const unsigned w0 = w < NWD ? wd[w] : 0u, w1 = w + 1 < NWD ? wd[w + 1] : 0u, w2 = w + 2 < NWD ? wd[w + 2] : 0u;
    win = ((unsigned long long)w0 << 32 | w1) << o;
    if (o) win |= (unsigned long long)w2 >> (32 - o);
    return win >> 11;
  };
  int p = first_set(0);
#pragma unroll 1
  for (int l = 0; l < K && p >= 0; ++l) {
    const unsigned long long m = bits53(p);
    const int lsb_weight = top - 32 + 63 - (p + 52);
    const double v = scalbn((double)m, lsb_weight);
    z[l] = neg ? -v : v;
    p = (p + 53 < 32 * NWD) ? first_set(p + 53) : -1;
  }
}

// ------------------------------------------------------------------ kernels
// Slices of one md value v (planes handled by the caller) relative to e:
// v 2^-e in (-1/2, 1/2) -> S balanced base-256 digits.
template <int K, int S>
__device__ __forceinline__ void oz_slice_value(const double (&v)[K], int e, __nv_bfloat16 *out, long long stride) {
  constexpr int W = (8 * S + 64) / 32 + 1;
  oz_fix<W> a;
#pragma unroll
  for (int q = 0; q < W; ++q) a.d[q] = 0;
  // digit 0 covers bits [e - 32, e): top = e
#pragma unroll
  for (int l = 0; l < K; ++l) oz_add_double<W>(a, e, v[l], 1);
  oz_normalize<W>(a);
  // value = sum_q d[q] 2^(e - 32(q+1)); slice s has weight 2^(e - 8(s+1)).
  // Take 8-bit digits from the least significant slice upwards with balancing.
  int carry = 0;
  for (int s = S - 1; s >= 0; --s) {
    const int bitpos = 8 * (s + 1);  // slice s occupies bits [e - 8(s+1), e - 8s)
    const int q = (bitpos - 1) / 32, off = 32 * (q + 1) - bitpos;  // within digit q, from its LSB
    int dig;
    if (q == 0) {
      dig = (int)((a.d[0] >> off) & 0xff);
      if (s == 0) dig = (int)(a.d[0] >> off);  // signed head (|value| < 1/2 -> small)
    } else {
      dig = (int)(((unsigned long long)a.d[q] >> off) & 0xffULL);
    }
    dig += carry;
    carry = 0;
    if (s > 0 && dig >= 128) {
      dig -= 256;
      carry = 1;
    }
    out[(long long)s * stride] = __int2bfloat16_rn(dig);
  }
}

// Slices of the rows of the blocks A_1..A_d.  One warp per (block i >= 1, row).
// As[((i*n + row)*P + p)*S + s][kpad] bf16; eA[i*n + row].
template <int K, int P>
__global__ void oz_split_rows_kernel(const double *__restrict__ A, __nv_bfloat16 *__restrict__ As,
                                     int *__restrict__ eA, int n, int d) {
  constexpr int S = oz_slices(K);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= d * n) return;
  const int i = 1 + warp / n, row = warp % n;
  const int kp = oz_kpad(n);
  const long long nn = (long long)n * n, stride = (long long)(d + 1) * nn;
  int e = -2000;
  for (int c = lane; c < n; c += 32)
#pragma unroll
    for (int p = 0; p < P; ++p) {
      e = max(e, oz_exp_bound(A[(long long)(p * K) * stride + (long long)i * nn + (long long)c * n + row]));
#pragma unroll
      for (int l = 1; l < K; ++l)
        if (!oz_finite(A[(long long)(p * K + l) * stride + (long long)i * nn + (long long)c * n + row]))
          e = kOzNonFinite;
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
  if (lane == 0) eA[i * n + row] = e;
  for (int c = lane; c < kp; c += 32) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      __nv_bfloat16 *out = As + ((((long long)i * n + row) * P + p) * S) * kp + c;
      if (c < n) {
        double v[K];
#pragma unroll
        for (int l = 0; l < K; ++l) v[l] = A[(long long)(p * K + l) * stride + (long long)i * nn + (long long)c * n + row];
        oz_slice_value<K, S>(v, e, out, kp);
      } else {
        for (int s = 0; s < S; ++s) out[(long long)s * kp] = __int2bfloat16_rn(0);
      }
    }
  }
}

// Slices of dx_j (AoS [j][i][P*K]); one block of 128 threads per vector j.
// Xs[(j*P + p)*S + t][kpad] bf16; ex[j].
template <int K, int P>
__global__ void oz_split_vec_kernel(const double *__restrict__ dxw, __nv_bfloat16 *__restrict__ Xs,
                                    int *__restrict__ ex, int n, int j) {
  constexpr int S = oz_slices(K);
  __shared__ int s_e[4];
  const int tid = threadIdx.x, kp = oz_kpad(n);
  const long long VS = P * K;
  int e = -2000;
  for (int c = tid; c < n; c += blockDim.x)
#pragma unroll
    for (int p = 0; p < P; ++p) {
      e = max(e, oz_exp_bound(dxw[((long long)j * n + c) * VS + p * K]));
#pragma unroll
      for (int l = 1; l < K; ++l)
        if (!oz_finite(dxw[((long long)j * n + c) * VS + p * K + l])) e = kOzNonFinite;
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
  if ((tid & 31) == 0) s_e[tid >> 5] = e;
  __syncthreads();
  e = max(max(s_e[0], s_e[1]), max(s_e[2], s_e[3]));
  if (tid == 0) ex[j] = e;
  for (int c = tid; c < kp; c += blockDim.x) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      __nv_bfloat16 *out = Xs + (((long long)j * P + p) * S) * kp + c;
      if (c < n) {
        double v[K];
#pragma unroll
        for (int l = 0; l < K; ++l) v[l] = dxw[((long long)j * n + c) * VS + p * K + l];
        oz_slice_value<K, S>(v, e, out, kp);
      } else {
        for (int s = 0; s < S; ++s) out[(long long)s * kp] = __int2bfloat16_rn(0);
      }
    }
  }
}

__device__ __forceinline__ unsigned oz_pack(const __nv_bfloat16 *p) {
  return *reinterpret_cast<const unsigned *>(p);
}

// The update of one degree k on the tensor pipe; no slice product leaves the
// SM.  For each output (row, plane q), G CTAs of oz_warps(K) warps share the
// j range (warp number gw = group * warps + w takes j = gw, gw + G warps, ...).
// For each j and each plane pair (pa, px) of the complex product a warp stages
// the slices of (row of A_{k-j}, plane pa) and of (dx_j, plane px) in shared
// memory, 64 columns at a time (rows padded to 72 bf16 so that fragment loads
// hit 32 distinct banks), with cp.async into two buffers so that the next
// stage loads while the current one is multiplied.  It forms the S x S slice
// products with m16n8k16 BF16 mma on ldmatrix fragments, a 32-row (S <= 32) or
// 16-row band of tiles at a time (exact in fp32: at most 64 terms of < 2^14
// per chunk), sums each lane's values of
// equal level L = s + t in registers and then in shared int32 bins (at most
// S * kpad terms of < 2^14: below 2^31 for kpad <= 1024), and adds each
// nonzero level, weighted 2^(eA + ex - 8(L+2)), into a fixed-point
// accumulator: the CTA's in shared memory, then (atomically, in int64 digits
// of 32 bits) the output's in global memory.  Integer additions are exact in
// any order, so neither the split over warps and CTAs nor the chunking
// changes the result: the exact sum of the terms, rounded once to K limbs by
// oz_finish_kernel.
constexpr int kOzChunk = 64;             // columns staged per step
constexpr int kOzPitch = kOzChunk + 8;   // bf16 per staged row
constexpr int kOzSmemBudget = 96 * 1024;  // per CTA, so that two CTAs share an SM

__host__ __device__ constexpr int oz_warp_smem(int K) {
  return 2 * 2 * oz_slices(K) * kOzPitch * 2;  // bytes: two buffers of A and X slices
}
__host__ __device__ constexpr int oz_warps(int K) {
  return kOzSmemBudget / oz_warp_smem(K) < 1 ? 1 : (kOzSmemBudget / oz_warp_smem(K) < 4 ? kOzSmemBudget / oz_warp_smem(K) : 4);
}
__host__ __device__ constexpr int oz_update_smem(int K) { return oz_warps(K) * oz_warp_smem(K); }

__device__ __forceinline__ void oz_cp16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// top of the accumulator of (row, q) at degree k: 64 bits above the largest
// term and above b_k (the same in every CTA and in the finish).
template <int K, int P>
__device__ __forceinline__ int oz_top(const int *eA, const int *ex, const double *b, int n, int d, int k, int row,
                                      int q, int lane) {
  int etop = -4000;
  for (int j = lane; j < k; j += 32) etop = max(etop, eA[(k - j) * n + row] + ex[j]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) etop = max(etop, __shfl_xor_sync(0xffffffffu, etop, off));
  etop = max(etop, oz_exp_bound(b[((long long)(q * K) * n + row) * (d + 1) + k]));
#pragma unroll
  for (int l = 1; l < K; ++l)
    if (!oz_finite(b[((long long)(q * K + l) * n + row) * (d + 1) + k])) etop = kOzNonFinite;
  return etop + 64;
}

template <int K, int P>
__global__ void __launch_bounds__(4 * 32) oz_update_kernel(const __nv_bfloat16 *__restrict__ As,
                                                           const __nv_bfloat16 *__restrict__ Xs,
                                                           const int *__restrict__ eA, const int *__restrict__ ex,
                                                           const double *__restrict__ b,
                                                           unsigned long long *__restrict__ gacc, int n, int d,
                                                           int k, int G) {
  constexpr int S = oz_slices(K), W = oz_digits(K), NW = oz_warps(K);
  constexpr int MB = S <= 32 ? S / 16 : 1;  // 16-row bands multiplied together
  constexpr int NU = 2 * (S / 16) + S / 8;  // slots u = 2 mt + nt (+1)
  static_assert(NW >= 1 && S % 16 == 0, "split sizes");
  extern __shared__ __align__(16) unsigned char oz_smem[];
  __shared__ long long acc[W];
  __shared__ int bins[NW][2 * S];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16 *buf = reinterpret_cast<__nv_bfloat16 *>(oz_smem) + (long long)wib * 4 * S * kOzPitch;
  const int out = blockIdx.x / G, grp = blockIdx.x % G;
  const int row = out / P, q = out % P;
  const int kp = oz_kpad(n), nchunk = kp / kOzChunk + (kp % kOzChunk ? 1 : 0);
  const int npairs = (P == 2) ? 2 : 1;
  const int g = lane >> 2, t4 = lane & 3;
  for (int i = threadIdx.x; i < W; i += blockDim.x) acc[i] = 0;
  for (int i = lane; i < 2 * S; i += 32) bins[wib][i] = 0;
  const int top = oz_top<K, P>(eA, ex, b, n, d, k, row, q, lane);
  __syncthreads();
  const int gw = grp * NW + wib, TW = G * NW;
  const int myj = (k > gw) ? (k - gw + TW - 1) / TW : 0;
  const int nstage = myj * npairs * nchunk;
  auto plane_pair = [&](int pr, int &pa, int &px, int &sg) {
    if (P == 1) {
      pa = 0; px = 0; sg = 1;
    } else if (q == 0) {  // real part: (re, re) - (im, im)
      pa = pr; px = pr; sg = pr == 0 ? 1 : -1;
    } else {  // imaginary part: (re, im) + (im, re)
      pa = pr; px = 1 - pr; sg = 1;
    }
  };
  auto issue = [&](int st) {  // start loading stage st into buffer st & 1
    const int c = st % nchunk, pr = (st / nchunk) % npairs, j = gw + TW * (st / (nchunk * npairs));
    int pa, px, sg;
    plane_pair(pr, pa, px, sg);
    const __nv_bfloat16 *Ab = As + ((((long long)(k - j) * n + row) * P + pa) * S) * kp;
    const __nv_bfloat16 *Bb = Xs + (((long long)j * P + px) * S) * kp;
    __nv_bfloat16 *sA = buf + (st & 1) * 2 * S * kOzPitch, *sX = sA + S * kOzPitch;
    const int c0 = c * kOzChunk, pieces = min(kOzChunk, kp - c0) / 8;
    if (pieces == kOzChunk / 8) {  // full chunk: lane = (row mod 4, 16-byte piece)
      const int cc = (lane & 7) * 8;
#pragma unroll 4
      for (int rr = lane >> 3; rr < S; rr += 4) {
        oz_cp16(sA + rr * kOzPitch + cc, Ab + (long long)rr * kp + c0 + cc);
        oz_cp16(sX + rr * kOzPitch + cc, Bb + (long long)rr * kp + c0 + cc);
      }
    } else {
      for (int e = lane; e < S * pieces; e += 32) {
        const int rr = e / pieces, cc = (e % pieces) * 8;
        oz_cp16(sA + rr * kOzPitch + cc, Ab + (long long)rr * kp + c0 + cc);
        oz_cp16(sX + rr * kOzPitch + cc, Bb + (long long)rr * kp + c0 + cc);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (nstage > 0) issue(0);
  for (int st = 0; st < nstage; ++st) {
    if (st + 1 < nstage) {
      issue(st + 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncwarp();
    const int c = st % nchunk, pr = (st / nchunk) % npairs, j = gw + TW * (st / (nchunk * npairs));
    const __nv_bfloat16 *sA = buf + (st & 1) * 2 * S * kOzPitch, *sX = sA + S * kOzPitch;
    const int cw = min(kOzChunk, kp - c * kOzChunk);  // a multiple of 16
    // per-lane sums of equal levels: slot u holds L = g + 2 t4 + 8u (e0) and +1 (e1)
    int e0[NU + 1], e1[NU + 1];
#pragma unroll
    for (int u = 0; u <= NU; ++u) e0[u] = e1[u] = 0;
    // tile groups: all tiles when S <= 32, else one 16-row band (S/8 tiles)
#pragma unroll
    for (int mg = 0; mg < S / 16; mg += MB) {
      float cf[MB][S / 8][4];
#pragma unroll
      for (int a = 0; a < MB; ++a)
#pragma unroll
        for (int t = 0; t < S / 8; ++t) cf[a][t][0] = cf[a][t][1] = cf[a][t][2] = cf[a][t][3] = 0.f;
      for (int k0 = 0; k0 < cw; k0 += 16) {
        // fragments with ldmatrix: A rows 16 (mg + a) + (lane & 15), columns k0 + 8 (lane >> 4);
        // B rows 8 t + (lane & 7), columns k0 + 8 ((lane >> 3) & 1)
        unsigned af[MB][4], bf[S / 8][2];
#pragma unroll
        for (int a = 0; a < MB; ++a) {
          const __nv_bfloat16 *pa = sA + (16 * (mg + a) + (lane & 15)) * kOzPitch + k0 + 8 * (lane >> 4);
          const unsigned sa = (unsigned)__cvta_generic_to_shared(pa);
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                       : "=r"(af[a][0]), "=r"(af[a][1]), "=r"(af[a][2]), "=r"(af[a][3])
                       : "r"(sa));
        }
#pragma unroll
        for (int t = 0; t < S / 8; ++t) {
          const __nv_bfloat16 *pb = sX + (8 * t + (lane & 7)) * kOzPitch + k0 + 8 * ((lane >> 3) & 1);
          const unsigned sb = (unsigned)__cvta_generic_to_shared(pb);
          asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                       : "=r"(bf[t][0]), "=r"(bf[t][1])
                       : "r"(sb));
        }
#pragma unroll
        for (int a = 0; a < MB; ++a)
#pragma unroll
          for (int t = 0; t < S / 8; ++t)
            asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(cf[a][t][0]), "+f"(cf[a][t][1]), "+f"(cf[a][t][2]), "+f"(cf[a][t][3])
                : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bf[t][0]), "r"(bf[t][1]));
      }
#pragma unroll
      for (int a = 0; a < MB; ++a)
#pragma unroll
        for (int t = 0; t < S / 8; ++t) {
          const int u = 2 * (mg + a) + t;
          // values at (16 mt + g, 8 nt + 2 t4) + {(0,0), (0,1), (8,0), (8,1)}: L = g + 2 t4 + 8u + {0, 1, 8, 9}
          e0[u] += __float2int_rn(cf[a][t][0]);
          e1[u] += __float2int_rn(cf[a][t][1]);
          e0[u + 1] += __float2int_rn(cf[a][t][2]);
          e1[u + 1] += __float2int_rn(cf[a][t][3]);
        }
    }
    const int Lb = g + 2 * t4;
#pragma unroll
    for (int u = 0; u <= NU; ++u) {
      if (e0[u] != 0) atomicAdd(&bins[wib][Lb + 8 * u], e0[u]);
      if (e1[u] != 0) atomicAdd(&bins[wib][Lb + 8 * u + 1], e1[u]);
    }
    __syncwarp();  // the buffer is free and the bins are complete for this chunk
    if (c == nchunk - 1) {  // last chunk of (j, pr): add the levels
      int pa, px, sg;
      plane_pair(pr, pa, px, sg);
      const int base = eA[(k - j) * n + row] + ex[j];
      for (int Lv = lane; Lv <= 2 * S - 2; Lv += 32) {
        const long long lv = bins[wib][Lv];
        bins[wib][Lv] = 0;
        if (lv == 0) continue;
        // r = b - term: the term lv 2^(base - 8(Lv+2)) enters with sign -sg
        const int lsb_below = top - (base - 8 * (Lv + 2));
        const bool neg = (lv < 0) != (sg < 0);
        const unsigned long long mag = (unsigned long long)(lv < 0 ? -lv : lv);  // < 2^31
        if (lsb_below <= 0) continue;
        int qd = (lsb_below + 31) / 32 - 1;
        if (qd >= W) {
          const int drop = lsb_below - 32 * W;
          if (drop >= 64) continue;
          const long long sv = (long long)(mag >> drop);
          atomicAdd((unsigned long long *)&acc[W - 1], (unsigned long long)(neg ? sv : -sv));
          continue;
        }
        const int rr = 32 * (qd + 1) - lsb_below;
        const unsigned long long v = mag << rr;
        const long long lo = (long long)(v & 0xffffffffULL), hi = (long long)(v >> 32);
        atomicAdd((unsigned long long *)&acc[qd], (unsigned long long)(neg ? lo : -lo));
        if (qd > 0) atomicAdd((unsigned long long *)&acc[qd - 1], (unsigned long long)(neg ? hi : -hi));
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < W; w += blockDim.x)
    if (acc[w] != 0) atomicAdd(gacc + (long long)out * W + w, (unsigned long long)acc[w]);
}

// r_k[row] (plane q) from the output's fixed-point accumulator and b_k; the
// accumulator is cleared for the next degree.  One thread per (row, q).
template <int K, int P>
__global__ void oz_finish_kernel(const int *__restrict__ eA, const int *__restrict__ ex,
                                 const double *__restrict__ b, double sgn, unsigned long long *__restrict__ gacc,
                                 double *__restrict__ r, int n, int d, int k) {
  constexpr int W = oz_digits(K);
  const int out = blockIdx.x, lane = threadIdx.x;  // one warp per output
  const int row = out / P, q = out % P;
  const int top = oz_top<K, P>(eA, ex, b, n, d, k, row, q, lane);
  if (lane != 0) return;
  oz_fix<W> a;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    a.d[w] = (long long)gacc[(long long)out * W + w];
    gacc[(long long)out * W + w] = 0ULL;
  }
#pragma unroll
  for (int l = 0; l < K; ++l)
    oz_add_double<W>(a, top, b[((long long)(q * K + l) * n + row) * (d + 1) + k], sgn < 0.0 ? -1 : 1);
  double z[K];
  if (top >= kOzNonFiniteTop) {  // a non-finite limb among the inputs of this output
#pragma unroll
    for (int l = 0; l < K; ++l) z[l] = __longlong_as_double(0x7ff8000000000000LL);
  } else {
    oz_to_md<W, K>(a, top, z);
  }
  const long long VS = P * K;
#pragma unroll
  for (int l = 0; l < K; ++l) r[((long long)k * n + row) * VS + q * K + l] = z[l];
}

}  // namespace mdk
