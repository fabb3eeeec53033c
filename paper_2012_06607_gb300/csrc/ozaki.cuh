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
// (block A_{k-j}, vector dx_j) one GEMM gives C[row, s][t] = sum_col A_s x_t for
// all slice pairs at once (M = n P S, N = P S, K = n).  The terms of r_k -- the
// C values with their power-of-two weights and the limbs of b_k -- are then
// added exactly into a fixed-point integer (int64 digits of 32 bits in shared
// memory) and converted to K limbs once.  The only rounding is the slicing
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

// exponent e with |v| < 2^(e-1) for the md number whose leading limb is x0
// (-2000 for zero).
__device__ __forceinline__ int oz_exp_bound(double x0) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x0) & 0x7fffffffffffffffULL;
  if (b == 0ULL) return -2000;
  int ex = (int)(b >> 52);
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

// K-limb md value of the normalised fixed-point number (top as in oz_add_double):
// limbs are consecutive 53-bit chunks of the magnitude (truncated).
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
  // magnitude digits: d[0] may exceed 32 bits; handle it as a 64-bit head
#pragma unroll
  for (int l = 0; l < K; ++l) z[l] = 0.0;
  // find the leading set bit
  int lead = -1;  // bit index counted from the top: position p has weight 2^(top - 1 - p) for p >= 0
  // head digit (possibly > 32 bits): weight 2^(top-32) per unit
  const unsigned long long head = (unsigned long long)a.d[0];
  int hb = head ? 64 - __clzll((long long)head) : 0;  // bits in head
  // bit stream: head bits (hb of them, MSB first) then W-1 digits of 32 bits
  // value = sum of bits; emit 53-bit chunks
  auto bit_at = [&](int p) -> unsigned {  // p = 0 is the MSB of the stream
    if (p < hb) return (unsigned)((head >> (hb - 1 - p)) & 1ULL);
    const int q = 1 + (p - hb) / 32, o = (p - hb) % 32;
    if (q >= W) return 0u;
    return (unsigned)(((unsigned long long)a.d[q] >> (31 - o)) & 1ULL);
  };
  const int nbits = hb + 32 * (W - 1);
  for (int p = 0; p < nbits; ++p)
    if (bit_at(p)) {
      lead = p;
      break;
    }
  if (lead < 0) return;
  // weight of stream bit p: 2^(top - 32 + hb - 1 - p)
  int p = lead;
#pragma unroll 1
  for (int l = 0; l < K && p < nbits; ++l) {
    unsigned long long m = 0;
    const int first = p;
    for (int i = 0; i < 53; ++i) m = (m << 1) | (p + i < nbits ? bit_at(p + i) : 0u);
    const int lsb_weight = top - 32 + hb - 1 - (first + 52);
    const double v = scalbn((double)m, lsb_weight);
    z[l] = neg ? -v : v;
    p = first + 53;
    while (p < nbits && !bit_at(p)) ++p;  // next limb starts at the next set bit
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
    for (int p = 0; p < P; ++p) e = max(e, oz_exp_bound(A[(long long)(p * K) * stride + (long long)i * nn + (long long)c * n + row]));
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
    for (int p = 0; p < P; ++p) e = max(e, oz_exp_bound(dxw[((long long)j * n + c) * VS + p * K]));
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

// C[j][m][nn] = sum_c As_{k-j}[m][c] * Xs_j[nn][c]  for j < k (exact fp32).
// One warp per 16 x 8 tile; grid covers (j, m tiles, n tiles).
__device__ __forceinline__ unsigned oz_pack(const __nv_bfloat16 *p) {
  return *reinterpret_cast<const unsigned *>(p);
}

template <int S, int P>
__global__ void oz_gemm_kernel(const __nv_bfloat16 *__restrict__ As, const __nv_bfloat16 *__restrict__ Xs,
                               float *__restrict__ C, int n, int k) {
  const int M = n * P * S, N = P * S, kp = oz_kpad(n);
  const int mt = M / 16, nt = N / 8;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)k * mt * nt) return;
  const int j = (int)(warp / ((long long)mt * nt));
  const int rem = (int)(warp % ((long long)mt * nt));
  const int tm = rem / nt, tn = rem % nt;
  const int i = k - j;
  const __nv_bfloat16 *Ab = As + ((long long)i * M + tm * 16) * kp;
  const __nv_bfloat16 *Bb = Xs + ((long long)j * N + tn * 8) * kp;
  const int g = lane >> 2, t = lane & 3;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
  for (int k0 = 0; k0 < kp; k0 += 16) {
    const unsigned a0 = oz_pack(Ab + (long long)g * kp + k0 + 2 * t);
    const unsigned a1 = oz_pack(Ab + (long long)(g + 8) * kp + k0 + 2 * t);
    const unsigned a2 = oz_pack(Ab + (long long)g * kp + k0 + 2 * t + 8);
    const unsigned a3 = oz_pack(Ab + (long long)(g + 8) * kp + k0 + 2 * t + 8);
    const unsigned b0 = oz_pack(Bb + (long long)g * kp + k0 + 2 * t);
    const unsigned b1 = oz_pack(Bb + (long long)g * kp + k0 + 2 * t + 8);
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float *Cb = C + ((long long)j * M + tm * 16) * N + tn * 8;
  Cb[(long long)g * N + 2 * t] = c0;
  Cb[(long long)g * N + 2 * t + 1] = c1;
  Cb[(long long)(g + 8) * N + 2 * t] = c2;
  Cb[(long long)(g + 8) * N + 2 * t + 1] = c3;
}

// r_k[row] (plane q) = sgn b_k[row] - sum_{j<k} A_{k-j}[row,:] dx_j, exactly into a
// fixed-point accumulator, then to K limbs.  One warp per (row, q).
template <int K, int P>
__global__ void __launch_bounds__(128) oz_accum_kernel(const float *__restrict__ C, const int *__restrict__ eA,
                                                       const int *__restrict__ ex, const double *__restrict__ b,
                                                       double sgn, double *__restrict__ r, int n, int d, int k) {
  constexpr int S = oz_slices(K), W = oz_digits(K);
  __shared__ long long acc[4][W];
  __shared__ int s_top[4];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int warp = blockIdx.x * 4 + wib;
  const bool active = warp < n * P;
  const int row = active ? warp / P : 0, q = active ? warp % P : 0;
  const int M = n * P * S, N = P * S;
  // top of the accumulator: 64 bits above the largest term and above b_k
  int etop = -4000;
  if (active) {
    for (int j = lane; j < k; j += 32) etop = max(etop, eA[(k - j) * n + row] + ex[j]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) etop = max(etop, __shfl_xor_sync(0xffffffffu, etop, off));
  double bl[K];
  if (active) {
#pragma unroll
    for (int l = 0; l < K; ++l) bl[l] = b[((long long)(q * K + l) * n + row) * (d + 1) + k];
    etop = max(etop, oz_exp_bound(bl[0]));
  }
  const int top = etop + 64;
  for (int w = lane; w < W; w += 32) acc[wib][w] = 0;
  __syncwarp();
  if (active) {
    // products: C-values of slice pair (s, t) have weight 2^(eA + ex - 8(s+1) - 8(t+1))
    // real part: (re,re) - (im,im); imaginary part: (re,im) + (im,re)
    const int npairs = (P == 2) ? 2 : 1;
    for (int j = 0; j < k; ++j) {
      const int base = eA[(k - j) * n + row] + ex[j];
      for (int pr = 0; pr < npairs; ++pr) {
        int pa, px, sg;
        if (P == 1) {
          pa = 0; px = 0; sg = 1;
        } else if (q == 0) {
          pa = pr; px = pr; sg = pr == 0 ? 1 : -1;
        } else {
          pa = pr; px = 1 - pr; sg = 1;
        }
        const float *Crow = C + ((long long)j * M + ((long long)row * P + pa) * S) * N + px * S;
        // level sums over s + t = L, then one exact add per level
        for (int L = lane; L <= 2 * S - 2; L += 32) {
          long long lv = 0;
          const int s0 = max(0, L - (S - 1)), s1 = min(S - 1, L);
          for (int s = s0; s <= s1; ++s) lv += (long long)Crow[(long long)s * N + (L - s)];
          if (lv == 0) continue;
          // lv * 2^(base - 8(L+2)) subtracted (sg * -1 for r = b - sum)
          const int lsb_below = top - (base - 8 * (L + 2));
          const bool neg = (lv < 0) != (sg < 0);  // sign of the term before the minus
          unsigned long long mag = (unsigned long long)(lv < 0 ? -lv : lv);
          // place mag (< 2^40) in 32-bit chunks
          for (int piece = 0; piece < 2 && mag; ++piece) {
            const unsigned long long chunk = mag & 0xffffffffULL;
            mag >>= 32;
            const int lb = lsb_below - 32 * piece;
            if (lb <= 0) continue;
            int qd = (lb + 31) / 32 - 1;
            unsigned long long v;
            if (qd >= W) {
              const int drop = lb - 32 * W;
              if (drop >= 64) continue;
              v = chunk >> drop;
              qd = W - 1;
              const long long sv = (long long)v;
              atomicAdd((unsigned long long *)&acc[wib][qd], (unsigned long long)(neg ? sv : -sv));
              continue;
            }
            const int rr = 32 * (qd + 1) - lb;
            v = chunk << rr;
            const long long lo = (long long)(v & 0xffffffffULL), hi = (long long)(v >> 32);
            // r = b - term: add -term
            atomicAdd((unsigned long long *)&acc[wib][qd], (unsigned long long)(neg ? lo : -lo));
            if (qd > 0) atomicAdd((unsigned long long *)&acc[wib][qd - 1], (unsigned long long)(neg ? hi : -hi));
          }
        }
      }
    }
  }
  __syncwarp();
  if (active && lane == 0) {
    oz_fix<W> a;
#pragma unroll
    for (int w = 0; w < W; ++w) a.d[w] = acc[wib][w];
#pragma unroll
    for (int l = 0; l < K; ++l) oz_add_double<W>(a, top, bl[l], sgn < 0.0 ? -1 : 1);
    double z[K];
    oz_to_md<W, K>(a, top, z);
    const long long VS = P * K;
#pragma unroll
    for (int l = 0; l < K; ++l) r[((long long)k * n + row) * VS + q * K + l] = z[l];
  }
  (void)s_top;
}

}  // namespace mdk
