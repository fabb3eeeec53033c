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

__device__ __forceinline__ unsigned oz_pack(const __nv_bfloat16 *p) {
  return *reinterpret_cast<const unsigned *>(p);
}

// The update of one degree k on the tensor pipe; no slice product leaves the
// SM.  One CTA of kOzWarps warps per (row, plane q); warp w takes
// j = w, w + kOzWarps, ... < k.  For each j and each plane pair (pa, px) of the
// complex product the warp stages the slices of (row of A_{k-j}, plane pa) and
// of (dx_j, plane px) in shared memory, 64 columns at a time (rows padded to 72
// bf16 so that fragment loads hit 32 distinct banks), forms the S x S slice
// products with m16n8k16 BF16 mma (exact in fp32: at most 64 terms of < 2^14
// per chunk), sums them by level L = s + t into shared int32 bins (at most
// S * kpad terms of < 2^14: below 2^31 for kpad <= 1024), and adds each nonzero
// level, weighted 2^(eA + ex - 8(L+2)), into the CTA's fixed-point
// accumulator.  Integer additions are exact in any order, so neither the split
// over warps nor the chunking changes the result: the exact sum of the terms,
// rounded once to K limbs.
constexpr int kOzWarps = 8;
constexpr int kOzChunk = 64;             // columns staged per step
constexpr int kOzPitch = kOzChunk + 8;   // bf16 per staged row

__host__ __device__ constexpr int oz_update_smem(int K) {
  return kOzWarps * 2 * oz_slices(K) * kOzPitch * 2;  // bytes: A and X slices per warp
}

template <int K, int P>
__global__ void __launch_bounds__(kOzWarps * 32) oz_update_kernel(const __nv_bfloat16 *__restrict__ As,
                                                                  const __nv_bfloat16 *__restrict__ Xs,
                                                                  const int *__restrict__ eA,
                                                                  const int *__restrict__ ex,
                                                                  const double *__restrict__ b, double sgn,
                                                                  double *__restrict__ r, int n, int d, int k) {
  constexpr int S = oz_slices(K), W = oz_digits(K);
  extern __shared__ __align__(16) unsigned char oz_smem[];
  __shared__ long long acc[W];
  __shared__ int bins[kOzWarps][2 * S];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(oz_smem) + (long long)wib * 2 * S * kOzPitch;
  __nv_bfloat16 *sX = sA + S * kOzPitch;
  const int row = blockIdx.x / P, q = blockIdx.x % P;
  const int kp = oz_kpad(n);
  const int g = lane >> 2, t4 = lane & 3;
  for (int i = threadIdx.x; i < W; i += blockDim.x) acc[i] = 0;
  for (int i = lane; i < 2 * S; i += 32) bins[wib][i] = 0;
  // top of the accumulator: 64 bits above the largest term and above b_k
  int etop = -4000;
  for (int j = lane; j < k; j += 32) etop = max(etop, eA[(k - j) * n + row] + ex[j]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) etop = max(etop, __shfl_xor_sync(0xffffffffu, etop, off));
  double bl[K];
#pragma unroll
  for (int l = 0; l < K; ++l) bl[l] = b[((long long)(q * K + l) * n + row) * (d + 1) + k];
  etop = max(etop, oz_exp_bound(bl[0]));
  const int top = etop + 64;
  __syncthreads();
  const int npairs = (P == 2) ? 2 : 1;
  for (int j = wib; j < k; j += kOzWarps) {
    const int base = eA[(k - j) * n + row] + ex[j];
    for (int pr = 0; pr < npairs; ++pr) {
      int pa, px, sg;
      if (P == 1) {
        pa = 0; px = 0; sg = 1;
      } else if (q == 0) {  // real part: (re, re) - (im, im)
        pa = pr; px = pr; sg = pr == 0 ? 1 : -1;
      } else {  // imaginary part: (re, im) + (im, re)
        pa = pr; px = 1 - pr; sg = 1;
      }
      const __nv_bfloat16 *Ab = As + ((((long long)(k - j) * n + row) * P + pa) * S) * kp;
      const __nv_bfloat16 *Bb = Xs + (((long long)j * P + px) * S) * kp;
      for (int c0 = 0; c0 < kp; c0 += kOzChunk) {
        const int cw = min(kOzChunk, kp - c0);  // a multiple of 16
        // stage S rows x cw columns of both operands (16-byte pieces)
        const int pieces = cw / 8;
        for (int e = lane; e < S * pieces; e += 32) {
          const int rr = e / pieces, cc = (e % pieces) * 8;
          *reinterpret_cast<uint4 *>(sA + rr * kOzPitch + cc) =
              *reinterpret_cast<const uint4 *>(Ab + (long long)rr * kp + c0 + cc);
          *reinterpret_cast<uint4 *>(sX + rr * kOzPitch + cc) =
              *reinterpret_cast<const uint4 *>(Bb + (long long)rr * kp + c0 + cc);
        }
        __syncwarp();
        for (int mt = 0; mt < S / 16; ++mt) {
          for (int nt = 0; nt < S / 8; ++nt) {
            float c0f = 0.f, c1f = 0.f, c2f = 0.f, c3f = 0.f;
            const __nv_bfloat16 *Am = sA + (mt * 16) * kOzPitch, *Bn = sX + (nt * 8) * kOzPitch;
            for (int k0 = 0; k0 < cw; k0 += 16) {
              const unsigned a0 = oz_pack(Am + g * kOzPitch + k0 + 2 * t4);
              const unsigned a1 = oz_pack(Am + (g + 8) * kOzPitch + k0 + 2 * t4);
              const unsigned a2 = oz_pack(Am + g * kOzPitch + k0 + 2 * t4 + 8);
              const unsigned a3 = oz_pack(Am + (g + 8) * kOzPitch + k0 + 2 * t4 + 8);
              const unsigned b0 = oz_pack(Bn + g * kOzPitch + k0 + 2 * t4);
              const unsigned b1 = oz_pack(Bn + g * kOzPitch + k0 + 2 * t4 + 8);
              asm volatile(
                  "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                  "{%0,%1,%2,%3};"
                  : "+f"(c0f), "+f"(c1f), "+f"(c2f), "+f"(c3f)
                  : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
            // (s, t) of the four values: (16 mt + g, 8 nt + 2 t4) and neighbours
            const int L = mt * 16 + g + nt * 8 + 2 * t4;
            if (c0f != 0.f) atomicAdd(&bins[wib][L], __float2int_rn(c0f));
            if (c1f != 0.f) atomicAdd(&bins[wib][L + 1], __float2int_rn(c1f));
            if (c2f != 0.f) atomicAdd(&bins[wib][L + 8], __float2int_rn(c2f));
            if (c3f != 0.f) atomicAdd(&bins[wib][L + 9], __float2int_rn(c3f));
          }
        }
        __syncwarp();
      }
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
  if (threadIdx.x == 0) {
    oz_fix<W> a;
#pragma unroll
    for (int w = 0; w < W; ++w) a.d[w] = acc[w];
#pragma unroll
    for (int l = 0; l < K; ++l) oz_add_double<W>(a, top, bl[l], sgn < 0.0 ? -1 : 1);
    double z[K];
    oz_to_md<W, K>(a, top, z);
    const long long VS = P * K;
#pragma unroll
    for (int l = 0; l < K; ++l) r[((long long)k * n + row) * VS + q * K + l] = z[l];
  }
}

}  // namespace mdk
