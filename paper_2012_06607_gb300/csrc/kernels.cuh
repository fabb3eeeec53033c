// Kernels of the power-series Newton step (templated on limbs K and planes P).
//
// Evaluate and differentiate (Section 4, algorithmic differentiation):
//   the host plans every series product of every monomial (common factor,
//   Speelpenning forward / backward / cross products, factor times product) and
//   groups them in dependency stages; one launch per stage computes all
//   products of that stage across all monomials.  A product z = x * y of two
//   series truncated at degree d has output coefficient k = sum_{i<=k} x_i y_{k-i}
//   (Section 3), summed in ascending i; a thread owns two output coefficients
//   whose term counts add up to d+2 (k and d-k, or two middle coefficients of
//   two products), so every lane of a warp runs the same d+2 iterations.
//   A second kernel accumulates f_i = cst_i + sum c_m G_m and
//   A_k[i][j] = sum (c_m a_j) D_mj in the order of the monomials.  Both keep
//   the summation order of the definition, so they agree with a sequential
//   evaluation bit for bit.
//
// Solve (Section 4, lower triangular block Toeplitz system):
//   Householder QR of A_0, one launch per column for the reflector and one
//   for its application to the trailing columns and to the identity (which
//   builds Q^H alongside); column-oriented back substitution of R W = Q^H for
//   all n columns at once gives W = R^-1 Q^H = A_0^-1; then degree by degree
//   r_k = b_k - sum_{j<k} A_{k-j} dx_j (split into chunks over all lanes) and
//   dx_k = W r_k.  Reductions here are trees across lanes.
#pragma once
#include <cuda_runtime.h>

#include "conv_fx.cuh"
#include "house_fx.cuh"
#include "internal.h"
#include "md.cuh"

namespace mdk {

// ------------------------------------------------------------------ helpers
template <int K, int P>
__device__ __forceinline__ void warp_sum(mdv<K, P> &v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mdv<K, P> o;
    shfl_xor<K, P>(v, off, o);
    c_add<K, P>(v, o, v);
  }
}

// Sum over the first `active` threads of the block (all threads must call it;
// the others contribute nothing); every thread gets the result.  smem: active/32 values.
template <int K, int P>
__device__ __forceinline__ void block_sum(mdv<K, P> &v, mdv<K, P> *smem, int active) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (active + 31) >> 5;
  if (warp < nw) warp_sum<K, P>(v);
  if (lane == 0 && warp < nw) smem[warp] = v;
  __syncthreads();
  if (warp == 0) {
    mdv<K, P> t;
    if (lane < nw)
      t = smem[lane];
    else
      c_zero<K, P>(t);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      if (off < nw) {  // uniform across the warp; lanes >= nw hold zero
        mdv<K, P> o;
        shfl_xor<K, P>(t, off, o);
        c_add<K, P>(t, o, t);
      }
    }
    if (lane == 0) smem[0] = t;
  }
  __syncthreads();
  v = smem[0];
  __syncthreads();
}

// ------------------------------------------------ row reductions (CTA level)
// The finish of r_k and the product dx_k = W r_k reduce one row at a time over
// a fixed set of kRowLanes virtual lanes: lane v handles plane p = v / Vc
// (P = 2: real, imaginary part) and column slot cs = v % Vc, Vc = kRowLanes / P.
// Slot cs sums the row's items cs, cs + Vc, cs + 2 Vc, ... in ascending order;
// the slots are then added pairwise in shared memory (slot i and slot i + s for
// s = 1, 2, 4, ...).  The result depends on the row only, never on how many
// threads run the virtual lanes, so the per-system kernels (one CTA of
// kRowLanes threads per row) and the batched kernel (its CTA walks the rows)
// produce the same bits.  An FP64 warp instruction costs the same with one or
// 32 active lanes, so spreading a row over four warps (one per SM
// sub-partition) and splitting complex products by plane is what shortens
// these latency-bound steps.  (kRowLanes: internal.h.)

template <int K>
__device__ __forceinline__ void ld_limbs(const double *src, double (&z)[K]) {
#pragma unroll
  for (int l = 0; l < K; ++l) z[l] = src[l];
}

template <int K>
__device__ __forceinline__ void st_limbs(double *dst, const double (&z)[K]) {
#pragma unroll
  for (int l = 0; l < K; ++l) dst[l] = z[l];
}

// Pairwise sum of the first nleaf slots of every plane.  All threads of the
// CTA call it; the gn threads of a group (gt = index in the group) work on
// the group's sm, and groups with act false only take the barriers.
template <int K, int P>
__device__ __forceinline__ void row_tree(double (*sm)[K], int nleaf, int gt, int gn, bool act) {
  constexpr int Vc = kRowLanes / P;
  for (int s = 1; s < nleaf; s <<= 1) {
    for (int v = gt; act && v < kRowLanes; v += gn) {
      const int cs = v % Vc;
      if ((cs & (2 * s - 1)) == 0 && cs + s < nleaf) {
        double a[K], b[K], z[K];
        ld_limbs<K>(sm[v], a);
        ld_limbs<K>(sm[v + s], b);
        md_add<K>(a, b, z);
        st_limbs<K>(sm[v], z);
      }
    }
    __syncthreads();
  }
}

template <int K, int P>
__device__ __forceinline__ void row_tree(double (*sm)[K], int nleaf) {
  row_tree<K, P>(sm, nleaf, threadIdx.x, blockDim.x, true);
}

// Plane p of the product a * b, computed as the complex product does it:
// real part a_re b_re - a_im b_im, imaginary part a_re b_im + a_im b_re.
template <int K, int P>
__device__ __forceinline__ void plane_prod_v(const mdv<K, P> &a, const mdv<K, P> &b, int p, double (&z)[K]) {
  if constexpr (P == 1) {
    md_mul<K>(a.v[0], b.v[0], z);
  } else {
    double b1[K], b2[K], t1[K], t2[K];
#pragma unroll
    for (int l = 0; l < K; ++l) {
      b1[l] = p == 0 ? b.v[0][l] : b.v[1][l];  // b_re or b_im
      b2[l] = p == 0 ? b.v[1][l] : b.v[0][l];  // b_im or b_re
    }
    md_mul<K>(a.v[0], b1, t1);
    md_mul<K>(a.v[1], b2, t2);
    if (p == 0) md_neg<K>(t2, t2);  // a - b is a + (-b)
    md_add<K>(t1, t2, z);
  }
}

template <int K, int P>
__device__ __forceinline__ void plane_prod(const double *w, const double *x, int p, double (&z)[K]) {
  mdv<K, P> a, b;
  ld_aos<K, P>(w, a);
  ld_aos<K, P>(x, b);
  plane_prod_v<K, P>(a, b, p, z);
}


template <int K>
__device__ __forceinline__ void real_to(const double (&r)[K], mdv<K, 1> &z) {
#pragma unroll
  for (int l = 0; l < K; ++l) z.v[0][l] = r[l];
}

// ---------------------------------------------------------------- elementwise
// op: 0 add, 1 sub, 2 mul, 3 div, 4 sqrt (real), 5 multiply by a double.
template <int K, int P, int OP>
__global__ void elementwise_kernel(long long count, const double *__restrict__ x, const double *__restrict__ y,
                                   double *__restrict__ z) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= count) return;
  mdv<K, P> a, b, c;
  ld_soa<K, P>(x + i, count, a);
  if constexpr (OP <= 3) ld_soa<K, P>(y + i, count, b);
  if constexpr (OP == 0) c_add<K, P>(a, b, c);
  if constexpr (OP == 1) c_sub<K, P>(a, b, c);
  if constexpr (OP == 2) c_mul<K, P>(a, b, c);
  if constexpr (OP == 3) c_div<K, P>(a, b, c);
  if constexpr (OP == 4) {
    md_sqrt<K>(a.v[0], c.v[0]);
    if constexpr (P == 2) {
#pragma unroll
      for (int l = 0; l < K; ++l) c.v[1][l] = 0.0;
    }
  }
  if constexpr (OP == 5) c_mul_d<K, P>(a, y[i], c);
  st_soa<K, P>(z + i, count, c);
}

// series products of `count` independent pairs, SoA layout [P][K][count][d+1];
// one thread per output coefficient (the reference form of a series product).
template <int K, int P>
__global__ void series_conv_kernel(int d, long long count, const double *__restrict__ x, const double *__restrict__ y,
                                   double *__restrict__ z) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= count * (d + 1)) return;
  const long long c = e / (d + 1);
  const int k = (int)(e % (d + 1));
  const long long stride = count * (d + 1);
  const double *xs = x + c * (d + 1);
  const double *ys = y + c * (d + 1);
  mdv<K, P> acc, a, b, t;
  ld_soa<K, P>(xs, stride, a);
  ld_soa<K, P>(ys + k, stride, b);
  c_mul<K, P>(a, b, acc);
  for (int i = 1; i <= k; ++i) {
    ld_soa<K, P>(xs + i, stride, a);
    ld_soa<K, P>(ys + (k - i), stride, b);
    c_mul<K, P>(a, b, t);
    c_add<K, P>(acc, t, acc);
  }
  st_soa<K, P>(z + e, stride, acc);
}

// -------------------------------------------------------------------- eval
// Pool of series, AoS: value (slot s, coefficient k) at pool[(s*(d+1) + k)*P*K].
template <int K, int P>
__device__ __forceinline__ void pool_load_entry(const double *x, double *pool, int n, int d,
                                                long long e) {
  mdv<K, P> v;
  ld_soa<K, P>(x + e, (long long)n * (d + 1), v);
  st_aos<K, P>(pool + e * (P * K), v);
}

template <int K, int P>
__global__ void pool_load_x_kernel(const double *__restrict__ x, double *__restrict__ pool, int n, int d) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * (d + 1)) return;
  pool_load_entry<K, P>(x, pool, n, d, e);
}

// scal[i] = c_mono (a == 1) or c_mono * a (exponent factor of a derivative).
template <int K, int P>
__device__ __forceinline__ void prep_scal_entry(const int *src, const double *coef, int nmono,
                                                double *scal, int i) {
  const int mono = src[2 * i], a = src[2 * i + 1];
  mdv<K, P> c, z;
  ld_soa<K, P>(coef + mono, nmono, c);
  if (a == 1)
    z = c;
  else
    c_mul_d<K, P>(c, (double)a, z);
  st_aos<K, P>(scal + (long long)i * (P * K), z);
}

template <int K, int P>
__global__ void prep_scal_kernel(const int *__restrict__ src, int nscal, const double *__restrict__ coef, int nmono,
                                 double *__restrict__ scal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nscal) return;
  prep_scal_entry<K, P>(src, coef, nmono, scal, i);
}

// The scaled coefficients of prep_scal_entry, also in packed fixed point.
template <int K, int P>
__device__ __forceinline__ void prep_scal_entry_fx(const int *src, const double *coef, int nmono, double *scal,
                                                   uint32_t *fxscal, int i) {
  constexpr int PW = packed_words(fxp::words_for(K));
  prep_scal_entry<K, P>(src, coef, nmono, scal, i);
  fx_pack_value<K, P>(scal + (long long)i * (P * K), 1, fxscal + (long long)i * P * PW);
}

template <int K, int P>
__global__ void prep_scal_fx_kernel(const int *__restrict__ src, int nscal, const double *__restrict__ coef, int nmono,
                                    double *__restrict__ scal, uint32_t *__restrict__ fxscal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nscal) return;
  prep_scal_entry_fx<K, P>(src, coef, nmono, scal, fxscal, i);
}

// Two output coefficients of series products: the first job computes
// coefficient kA of product (outA = xA * yA), the second coefficient kB of
// (outB = xB * yB); kA + kB = d, so the loop has d+2 iterations (outB < 0: only
// the first job).  Coefficient k is sum_{i<=k} x_i y_{k-i}, ascending i.
// NC: read through the read-only data path (only when nothing written in the
// same kernel is read, i.e. one stage per launch).
template <int K, int P, bool NC = true>
__device__ __forceinline__ void conv_pair(double *pool, int d, int outA, int xA, int yA, int kA, int outB, int xB,
                                          int yB) {
  const int kB = d - kA;
  const long long VS = P * K, SS = (long long)(d + 1) * VS;
  const int total = (outB >= 0) ? (d + 2) : (kA + 1);
  mdv<K, P> acc, a, b, prod;
  auto addr = [&](int it, const double *&xp, const double *&yp) {
    const bool first = it <= kA;
    const int i = first ? it : it - kA - 1;
    xp = pool + (first ? xA : xB) * SS + i * VS;
    yp = pool + (first ? yA : yB) * SS + ((first ? kA : kB) - i) * VS;
  };
  auto load = [&](const double *src, mdv<K, P> &z) {
    if constexpr (NC)
      ld_aos_nc<K, P>(src, z);
    else
      ld_aos<K, P>(src, z);
  };
  // No prefetch: an iteration is ~(cmul + cadd) FP64 instructions, i.e. tens of
  // thousands of cycles of pipe time per warp, so load latency is hidden by
  // the other resident warps; the registers go to occupancy instead.
  const double *xp, *yp;
  for (int it = 0; it < total; ++it) {
    addr(it, xp, yp);
    load(xp, a);
    load(yp, b);
    c_mul<K, P>(a, b, prod);
    if (it == 0 || it == kA + 1)
      acc = prod;
    else
      c_add<K, P>(acc, prod, acc);
    if (it == kA) st_aos<K, P>(pool + outA * SS + kA * VS, acc);
  }
  if (outB >= 0) st_aos<K, P>(pool + outB * SS + kB * VS, acc);
}

// One launch per stage.  task = {outA, xA, yA, kA, outB, xB, yB, -}.
template <int K, int P>
__global__ void __launch_bounds__(64) conv_stage_kernel(const int *__restrict__ tasks, int ntask,
                                                         double *pool, int d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntask) return;
  const int4 t0 = __ldg(reinterpret_cast<const int4 *>(tasks) + 2 * t);
  const int4 t1 = __ldg(reinterpret_cast<const int4 *>(tasks) + 2 * t + 1);
  conv_pair<K, P>(pool, d, t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z);
}

// Same work with a fixed grid of CTAs (one per SM)
// that stride over the tasks, so that a grid of SMs - R CTAs leaves R SMs to
// kernels that run concurrently on another stream.  Thread numbering is
// interleaved across CTAs (t = tid * grid + cta): all tasks cost the same, and
// the last, partial round of tasks is then spread over every SM instead of
// going whole to the first CTAs, so the SMs end together.
// Up to five limbs a task fits in the 168 registers a 384-thread CTA leaves
// per thread; eight and ten limbs get 256 threads and up to 255 registers
// (two warps per SM sub-partition still keep the FP64 pipe busy).
template <int K>
constexpr int conv_resident_threads() {
  return K <= 5 ? 384 : 256;
}

template <int K, int P>
__global__ void __launch_bounds__(conv_resident_threads<K>(), 1)
    conv_stage_resident_kernel(const int *__restrict__ tasks, int ntask, double *pool, int d) {
  for (int t = threadIdx.x * gridDim.x + blockIdx.x; t < ntask; t += gridDim.x * blockDim.x) {
    const int4 t0 = __ldg(reinterpret_cast<const int4 *>(tasks) + 2 * t);
    const int4 t1 = __ldg(reinterpret_cast<const int4 *>(tasks) + 2 * t + 1);
    conv_pair<K, P>(pool, d, t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z);
  }
}

// group = {row, col (-1: f_row), first contribution, count};
// contribution = {slot (-1: the unit series), scal index, shift a_t, -}.
// Coefficient k of one contribution: c * s_{k - a} for a product slot s, c at
// k = a for the unit series, zero for k < a.
template <int K, int P>
__device__ __forceinline__ void accum_contrib_value(const int4 C, const double *pool, const double *scal, int d, int k,
                                                    mdv<K, P> &v) {
  const long long VS = P * K, SS = (long long)(d + 1) * VS;
  mdv<K, P> c, s;
  c_zero<K, P>(v);
  if (k >= C.z) {
    ld_aos<K, P>(scal + (long long)C.y * VS, c);
    if (C.x < 0) {
      if (k == C.z) v = c;
    } else {
      ld_aos<K, P>(pool + C.x * SS + (k - C.z) * VS, s);
      c_mul<K, P>(c, s, v);
    }
  }
}

// f: [P][K][N][d+1]; A: [P][K][d+1][n][N] (column-major N x n blocks).
template <int K, int P>
__device__ __forceinline__ void accum_store(const int4 G, const mdv<K, P> &acc, double *f, double *A, int N, int n,
                                            int d, int k) {
  if (G.y < 0) {
    st_soa<K, P>(f + (long long)G.x * (d + 1) + k, (long long)N * (d + 1), acc);
  } else {
    const long long nn = (long long)N * n;
    st_soa<K, P>(A + (long long)k * nn + (long long)G.y * N + G.x, (long long)(d + 1) * nn, acc);
  }
}

// Coefficient k of one group: the constant term (f rows, k = 0), then the
// contributions added one by one in list order.
template <int K, int P>
__device__ __forceinline__ void accum_entry(const int4 *groups, const int4 *contrib,
                                            const double *pool, const double *scal,
                                            const double *cst, double *f,
                                            double *A, int N, int n, int d, int g, int k) {
  const int4 G = groups[g];
  mdv<K, P> acc, v;
  c_zero<K, P>(acc);
  if (G.y < 0 && k == 0) ld_soa<K, P>(cst + G.x, N, acc);
  for (int q = 0; q < G.w; ++q) {
    accum_contrib_value<K, P>(contrib[G.z + q], pool, scal, d, k, v);
    c_add<K, P>(acc, v, acc);
  }
  accum_store<K, P>(G, acc, f, A, N, n, d, k);
}

// Entries (group, k) for k in [k0, k0 + nk); only_A: skip the f rows.
template <int K, int P>
__global__ void accum_kernel(const int4 *__restrict__ groups, int ngroups, const int4 *__restrict__ contrib,
                             const double *__restrict__ pool, const double *__restrict__ scal,
                             const double *__restrict__ cst, double *__restrict__ f, double *__restrict__ A, int N,
                             int n, int d, int k0, int nk, int only_A) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)ngroups * nk) return;
  const int g = (int)(e / nk);
  if (only_A && groups[g].y < 0) return;
  accum_entry<K, P>(groups, contrib, pool, scal, cst, f, A, N, n, d, g, k0 + (int)(e % nk));
}

// The same accumulation in two passes, so that long groups (the f rows sum
// one contribution per monomial) do not serialise the products: every
// contribution value goes to prod (AoS [contribution][k]), then each entry
// adds its group's values in the same order as accum_entry, which makes the
// result bit-identical to it.
template <int K, int P>
__global__ void accum_prod_kernel(const int4 *__restrict__ contrib, int ncontrib, const double *__restrict__ pool,
                                  const double *__restrict__ scal, double *__restrict__ prod, int d) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)ncontrib * (d + 1)) return;
  const int q = (int)(e / (d + 1)), k = (int)(e % (d + 1));
  mdv<K, P> v;
  accum_contrib_value<K, P>(contrib[q], pool, scal, d, k, v);
  st_aos<K, P>(prod + e * (P * K), v);
}

// Entries (group, k), k in [0, d]; the A groups at k = 0 are skipped when
// skip_A0 is set (coefficient 0 of A is accumulated beforehand).
template <int K, int P>
__global__ void accum_sum_kernel(const int4 *__restrict__ groups, int ngroups, const double *__restrict__ prod,
                                 const double *__restrict__ cst, double *__restrict__ f, double *__restrict__ A,
                                 int N, int n, int d, int skip_A0) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)ngroups * (d + 1)) return;
  const int g = (int)(e / (d + 1)), k = (int)(e % (d + 1));
  const int4 G = groups[g];
  if (skip_A0 && k == 0 && G.y >= 0) return;
  const long long VS = P * K;
  mdv<K, P> acc, v;
  c_zero<K, P>(acc);
  if (G.y < 0 && k == 0) ld_soa<K, P>(cst + G.x, N, acc);
  for (int q = 0; q < G.w; ++q) {
    ld_aos<K, P>(prod + ((long long)(G.z + q) * (d + 1) + k) * VS, v);
    c_add<K, P>(acc, v, acc);
  }
  accum_store<K, P>(G, acc, f, A, N, n, d, k);
}

// ------------------------------------------------------------------- solve
// A_0 is N x n (N >= n equations; N > n: least squares).  Work matrices are
// AoS, column-major with N rows: element (r, c) of M (N x n, becomes R and the
// reflectors) and of Y (N x N, becomes Q^H) at [(c*N + r)*P*K]; W (n x N) is
// row-major.  Every body below is shared by the one-launch-per-step kernels and
// by the batched kernel (one CTA per system, N = n); the reduction trees are the
// same in both.
template <int K, int P>
__device__ __forceinline__ void solve_init_entry(const double *A, double *M, double *Y, int N, int n, int d,
                                                 long long e) {
  const long long nn = (long long)N * n;
  mdv<K, P> v;
  if (e < nn) {
    ld_soa<K, P>(A + e, (long long)(d + 1) * nn, v);  // A_0, column-major, e = c*N + r
    st_aos<K, P>(M + e * (P * K), v);
  }
  c_zero<K, P>(v);
  const long long r = e % N, c = e / N;
  if (r == c) v.v[0][0] = 1.0;
  st_aos<K, P>(Y + e * (P * K), v);
}

template <int K, int P>
__global__ void solve_init_kernel(const double *__restrict__ A, double *__restrict__ M, double *__restrict__ Y, int N,
                                  int n, int d) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)N * N) return;
  solve_init_entry<K, P>(A, M, Y, N, n, d, e);
}

// Householder vector of column j (Golub-Van Loan): alpha = ||x||, phase
// e = x_0/|x_0|, v = x + e alpha e_1, beta = 1/(alpha (alpha + |x_0|)), R_jj = -e alpha.
// The square roots and the reciprocal use the precision-doubling iterations
// (this chain bounds the factorisation).  Block-level body for kHouseThreads
// threads.
template <int K, int P>
__device__ __forceinline__ void house_block(double *M, double *vd,
                                            double *beta, int *status, int N, int j) {
  __shared__ mdv<K, 1> red[kHouseThreads / 32];
  __shared__ double s_alpha[K], s_a0[K], s_beta[K];
  __shared__ mdv<K, P> s_ph;
  const int tid = threadIdx.x;
  const long long VS = P * K;
  mdv<K, 1> acc;
  c_zero<K, 1>(acc);
  bool have = false;
  for (int i = j + tid; tid < kHouseThreads && i < N; i += kHouseThreads) {
    mdv<K, P> x;
    ld_aos<K, P>(M + ((long long)j * N + i) * VS, x);
    double a2[K];
    c_abs2<K, P>(x, a2);
    if (!have) {
      real_to<K>(a2, acc);
      have = true;
    } else {
      mdv<K, 1> t;
      real_to<K>(a2, t);
      c_add<K, 1>(acc, t, acc);
    }
  }
  block_sum<K, 1>(acc, red, kHouseThreads);
  mdv<K, P> x0;
  ld_aos<K, P>(M + ((long long)j * N + j) * VS, x0);
  if (tid == 0) {
    double al[K];
    md_sqrt_pd<K>(acc.v[0], al);
#pragma unroll
    for (int l = 0; l < K; ++l) s_alpha[l] = al[l];
  }
  if (tid == 32) {
    double a0[K];
    if constexpr (P == 1) {
      const bool neg = x0.v[0][0] < 0.0;
#pragma unroll
      for (int l = 0; l < K; ++l) a0[l] = neg ? -x0.v[0][l] : x0.v[0][l];
    } else {
      double s2[K];
      c_abs2<K, P>(x0, s2);
      md_sqrt_pd<K>(s2, a0);
    }
#pragma unroll
    for (int l = 0; l < K; ++l) s_a0[l] = a0[l];
  }
  __syncthreads();
  if (tid == 0) {
    double al[K], a0[K], t[K], den[K], bt[K];
#pragma unroll
    for (int l = 0; l < K; ++l) {
      al[l] = s_alpha[l];
      a0[l] = s_a0[l];
    }
    if (!nonzero(al[0])) atomicOr(status, ST_SINGULAR);
    md_add<K>(al, a0, t);
    md_mul<K>(al, t, den);
    md_recip_pd<K>(den, bt);
#pragma unroll
    for (int l = 0; l < K; ++l) s_beta[l] = bt[l];
  }
  if (P == 1 && tid == 32) {
    mdv<K, P> ph;
    c_zero<K, P>(ph);
    ph.v[0][0] = (x0.v[0][0] < 0.0) ? -1.0 : 1.0;
    s_ph = ph;
  }
  if constexpr (P == 2) {
    if (tid == 32 || tid == 64) {
      const int p = (tid == 32) ? 0 : 1;
      double a0[K], q[K];
#pragma unroll
      for (int l = 0; l < K; ++l) a0[l] = s_a0[l];
      if (!nonzero(a0[0])) {
#pragma unroll
        for (int l = 0; l < K; ++l) q[l] = 0.0;
        if (p == 0) q[0] = 1.0;
      } else {
        md_div<K>(x0.v[p], a0, q);
      }
#pragma unroll
      for (int l = 0; l < K; ++l) s_ph.v[p][l] = q[l];
    }
  }
  __syncthreads();
  if (tid == 0) {
    double al[K];
#pragma unroll
    for (int l = 0; l < K; ++l) al[l] = s_alpha[l];
    mdv<K, P> ph = s_ph, pa, v0, rjj;
    c_mul_real<K, P>(ph, al, pa);
    c_add<K, P>(x0, pa, v0);
#pragma unroll
    for (int p = 0; p < P; ++p) md_neg<K>(pa.v[p], rjj.v[p]);
    st_aos<K, P>(vd + (long long)j * VS, v0);
    st_aos<K, P>(M + ((long long)j * N + j) * VS, rjj);
#pragma unroll
    for (int l = 0; l < K; ++l) beta[(long long)j * K + l] = s_beta[l];
  }
  __syncthreads();
}

// The QR steps as the kernels run them: in W-word fixed point (house_fx.cuh)
// from kFxMinLimbs limbs on, in md arithmetic below.
template <int K, int P>
__device__ __forceinline__ void qr_house(double *M, double *vd, double *beta, int *status, int N, int j) {
  if constexpr (K >= kFxMinLimbs)
    house_block_fx<K, P>(M, vd, beta, status, N, j);
  else
    house_block<K, P>(M, vd, beta, status, N, j);
}

template <int K, int P>
__global__ void __launch_bounds__(kHouseThreads) house_kernel(double *__restrict__ M, double *__restrict__ vd,
                                                              double *__restrict__ beta, int *__restrict__ status,
                                                              int N, int j) {
  qr_house<K, P>(M, vd, beta, status, N, j);
}

// Apply H_j = I - beta_j v v^H to target column w: w < n-j-1 is column j+1+w of
// M (trailing columns), otherwise column w-(n-j-1) of Y (accumulating Q^H).
// Warp-level body.
template <int K, int P>
__device__ __forceinline__ void house_apply_col(double *M, double *Y,
                                                const double *vd, const double *beta, int N,
                                                int n, int j, int w, int lane) {
  const int nm = n - j - 1;
  double *T;
  int c;
  if (w < nm) {
    T = M;
    c = j + 1 + w;
  } else {
    T = Y;
    c = w - nm;
  }
  const long long VS = P * K;
  mdv<K, P> acc, v, cv, t, prod;
  c_zero<K, P>(acc);
  bool have = false;
  for (int i = j + lane; i < N; i += 32) {
    if (i == j)
      ld_aos<K, P>(vd + (long long)j * VS, v);
    else
      ld_aos<K, P>(M + ((long long)j * N + i) * VS, v);
    c_conj<K, P>(v, cv);
    ld_aos<K, P>(T + ((long long)c * N + i) * VS, t);
    c_mul<K, P>(cv, t, prod);
    if (!have) {
      acc = prod;
      have = true;
    } else {
      c_add<K, P>(acc, prod, acc);
    }
  }
  warp_sum<K, P>(acc);
  double bt[K];
#pragma unroll
  for (int l = 0; l < K; ++l) bt[l] = beta[(long long)j * K + l];
  mdv<K, P> tau;
  c_mul_real<K, P>(acc, bt, tau);
  for (int i = j + lane; i < N; i += 32) {
    if (i == j)
      ld_aos<K, P>(vd + (long long)j * VS, v);
    else
      ld_aos<K, P>(M + ((long long)j * N + i) * VS, v);
    ld_aos<K, P>(T + ((long long)c * N + i) * VS, t);
    c_mul<K, P>(tau, v, prod);
    c_sub<K, P>(t, prod, t);
    st_aos<K, P>(T + ((long long)c * N + i) * VS, t);
  }
}

template <int K, int P>
__global__ void __launch_bounds__(128) house_apply_kernel(double *__restrict__ M, double *__restrict__ Y,
                                                          const double *__restrict__ vd,
                                                          const double *__restrict__ beta, int N, int n, int j) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= (n - j - 1) + N) return;
  house_apply_col<K, P>(M, Y, vd, beta, N, n, j, warp, lane);
}

// The same application by a whole CTA over kRowLanes virtual lanes (plane,
// row slot): plane products of conj(v_i) t_i summed per plane with the
// shared-memory tree, tau = beta * dot, then t_i -= tau v_i plane by plane
// (each element updated exactly as in house_apply_col).  CTA body.
template <int K, int P>
__device__ __forceinline__ void house_apply_col_cta(double *M, double *Y, const double *vd, const double *beta, int N,
                                                    int n, int j, int w, double (*sm)[K]) {
  constexpr int Vc = kRowLanes / P;
  const int nm = n - j - 1;
  double *T = (w < nm) ? M : Y;
  const int c = (w < nm) ? j + 1 + w : w - nm;
  const long long VS = P * K;
  const int nleaf = min(N - j, Vc);
  auto ld_v = [&](int i, mdv<K, P> &v) {
    if (i == j)
      ld_aos<K, P>(vd + (long long)j * VS, v);
    else
      ld_aos<K, P>(M + ((long long)j * N + i) * VS, v);
  };
  for (int q = threadIdx.x; q < kRowLanes; q += blockDim.x) {
    const int p = q / Vc, cs = q % Vc;
    if (cs < nleaf) {
      double acc[K], t[K];
      bool have = false;
      for (int i = j + cs; i < N; i += Vc) {
        mdv<K, P> v, cv, x;
        ld_v(i, v);
        c_conj<K, P>(v, cv);
        ld_aos<K, P>(T + ((long long)c * N + i) * VS, x);
        if (!have) {
          plane_prod_v<K, P>(cv, x, p, acc);
          have = true;
        } else {
          plane_prod_v<K, P>(cv, x, p, t);
          md_add<K>(acc, t, acc);
        }
      }
      st_limbs<K>(sm[q], acc);
    }
  }
  __syncthreads();
  row_tree<K, P>(sm, nleaf);
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double dt[K], bt[K], z[K];
    ld_limbs<K>(sm[p * Vc], dt);
    ld_limbs<K>(beta + (long long)j * K, bt);
    md_mul<K>(dt, bt, z);
    st_limbs<K>(sm[p * Vc], z);
  }
  __syncthreads();
  mdv<K, P> tau;
#pragma unroll
  for (int p = 0; p < P; ++p) ld_limbs<K>(sm[p * Vc], tau.v[p]);
  for (int q = threadIdx.x; q < kRowLanes; q += blockDim.x) {
    const int p = q / Vc, cs = q % Vc;
    for (int i = j + cs; i < N; i += Vc) {
      mdv<K, P> v;
      ld_v(i, v);
      double pr[K], t[K];
      plane_prod_v<K, P>(tau, v, p, pr);
      double *dst = T + ((long long)c * N + i) * VS + p * K;
      ld_limbs<K>(dst, t);
      md_sub<K>(t, pr, t);
      st_limbs<K>(dst, t);
    }
  }
  __syncthreads();
}

// One step of the QR with lookahead: CTA 0 applies H_j to column j+1 and then
// builds the Householder vector of column j+1, while the other CTAs apply H_j
// to columns j+2.. of M and to Y (one CTA per column in fixed point, one warp
// per column in plain double).  The next step needs
// both, and column j+1 is touched by CTA 0 only, so the step's critical path is
// the larger of (column j+1 + Householder vector) and the rest of the update,
// not their sum.
template <int K, int P, bool CACHE = true>
__device__ __forceinline__ void qr_apply_cta(double *M, double *Y, const double *vd, const double *beta, int N, int n,
                                             int j, int w, double (*sm)[K]) {
  if constexpr (K >= kFxMinLimbs)
    house_apply_col_v128<K, P, true, CACHE>(M, Y, vd, beta, N, n, j, w);
  else
    house_apply_col_cta<K, P>(M, Y, vd, beta, N, n, j, w, sm);
}

template <int K, int P>
__device__ __forceinline__ void qr_apply_warp(double *M, double *Y, const double *vd, const double *beta, int N,
                                              int n, int j, int w, int lane) {
  if constexpr (K >= kFxMinLimbs) {
    (void)lane;
    house_apply_col_v128<K, P, false>(M, Y, vd, beta, N, n, j, w);
  } else {
    house_apply_col<K, P>(M, Y, vd, beta, N, n, j, w, lane);
  }
}

// CTAs of house_step_kernel after CTA 0: one per trailing target (fixed
// point, K >= kFxMinLimbs) or one warp per target (md arithmetic).
template <int K>
__host__ __device__ constexpr bool qr_cta_per_target() {
  return K >= kFxMinLimbs;
}

template <int K, int P>
__global__ void __launch_bounds__(kHouseThreads) house_step_kernel(double *M, double *Y, double *vd, double *beta,
                                                                   int *status, int N, int n, int j) {
  __shared__ double sm[K >= kFxMinLimbs ? 1 : kRowLanes][K];
  const bool ahead = j + 1 < n;
  if (blockIdx.x == 0) {
    if (ahead) {
      qr_apply_cta<K, P>(M, Y, vd, beta, N, n, j, 0, sm);
      qr_house<K, P>(M, vd, beta, status, N, j + 1);
    }
    return;
  }
  if constexpr (qr_cta_per_target<K>()) {
    const int w = (int)blockIdx.x - 1 + (ahead ? 1 : 0);
    if (w >= (n - j - 1) + N) return;  // uniform over the CTA
    qr_apply_cta<K, P>(M, Y, vd, beta, N, n, j, w, sm);
  } else {
    const int warp = ((blockIdx.x - 1) * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int w = warp + (ahead ? 1 : 0);
    if (w >= (n - j - 1) + N) return;
    qr_apply_warp<K, P>(M, Y, vd, beta, N, n, j, w, lane);
  }
}

// rinv[j] = 1 / R_jj
template <int K, int P>
__device__ __forceinline__ void rinv_entry(const double *M, double *rinv, int N, int j) {
  if constexpr (K >= kFxMinLimbs) {  // fixed point, as the QR (house_fx.cuh)
    rinv_entry_fx<K, P>(M, rinv, N, j);
    return;
  }
  const long long VS = P * K;
  mdv<K, P> r, one, z;
  ld_aos<K, P>(M + ((long long)j * N + j) * VS, r);
  c_zero<K, P>(one);
  one.v[0][0] = 1.0;
  c_div<K, P>(one, r, z);
  st_aos<K, P>(rinv + (long long)j * VS, z);
}

template <int K, int P>
__global__ void rinv_kernel(const double *__restrict__ M, double *__restrict__ rinv, int N, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  rinv_entry<K, P>(M, rinv, N, j);
}

// Column-oriented back substitution step c of R W = Y[0:n, :] (all N
// right-hand sides; R is the top n x n block): W[c][:] = Y[c][:] / R_cc;
// Y[i][:] -= R_ic W[c][:] for i < c.  W (n x N) is row-major.
template <int K, int P>
__device__ __forceinline__ void backsub_entry(const double *M, double *Y,
                                              double *W, const double *rinv, int N, int c,
                                              long long e) {
  if constexpr (K >= kFxMinLimbs) {  // fixed point, as the QR (house_fx.cuh)
    backsub_entry_fx<K, P>(M, Y, W, rinv, N, c, e);
    return;
  }
  const int i = (int)(e / N), col = (int)(e % N);
  const long long VS = P * K;
  mdv<K, P> y, ri, w;
  ld_aos<K, P>(Y + ((long long)col * N + c) * VS, y);
  ld_aos<K, P>(rinv + (long long)c * VS, ri);
  c_mul<K, P>(y, ri, w);
  if (i == c) {
    st_aos<K, P>(W + ((long long)c * N + col) * VS, w);
  } else {
    mdv<K, P> rc, t, yi;
    ld_aos<K, P>(M + ((long long)c * N + i) * VS, rc);
    ld_aos<K, P>(Y + ((long long)col * N + i) * VS, yi);
    c_mul<K, P>(rc, w, t);
    c_sub<K, P>(yi, t, yi);
    st_aos<K, P>(Y + ((long long)col * N + i) * VS, yi);
  }
}

template <int K, int P>
__global__ void backsub_kernel(const double *__restrict__ M, double *__restrict__ Y, double *__restrict__ W,
                               const double *__restrict__ rinv, int N, int c) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)(c + 1) * N) return;
  backsub_entry<K, P>(M, Y, W, rinv, N, c, e);
}

// ------------------------------------------------------------ LU (N = n)
// Gaussian elimination with partial pivoting, the factorisation Section 4
// allows when N = n.  Column j: pivot row p = the first row i >= j with the
// largest |re| + |im| of the leading limbs; rows j and p are swapped in M and
// in Y (Y starts as I and so ends as the permutation P); multipliers
// l_ij = M_ij * (1 / M_jj); trailing update M_ik -= l_ij M_jk.  Afterwards
// L Z = P (unit lower triangular, forward) overwrites Y, and U W = Z is the
// back substitution of the QR path with U in the upper triangle of M, so that
// W = U^-1 L^-1 P = A_0^-1 feeds the same degree loop.
template <int P>
__device__ __forceinline__ double cabs1_lead(const double *v, int K) {
  return fabs(v[0]) + (P == 2 ? fabs(v[K]) : 0.0);
}

template <int K, int P>
__global__ void __launch_bounds__(128) lu_pivot_kernel(double *M, double *Y, double *rinv, int *status, int n, int j) {
  __shared__ double s_val[128];
  __shared__ int s_idx[128];
  const int tid = threadIdx.x;
  const long long VS = P * K;
  double best = -1.0;
  int bi = j;
  for (int i = j + tid; i < n; i += blockDim.x) {
    const double v = cabs1_lead<P>(M + ((long long)j * n + i) * VS, K);
    if (v > best) {  // rows visited in increasing order: ties keep the first
      best = v;
      bi = i;
    }
  }
  s_val[tid] = best;
  s_idx[tid] = bi;
  __syncthreads();
  for (int off = 64; off > 0; off >>= 1) {
    if (tid < off) {
      const double a = s_val[tid], b = s_val[tid + off];
      const int ia = s_idx[tid], ib = s_idx[tid + off];
      if (b > a || (b == a && ib < ia)) {
        s_val[tid] = b;
        s_idx[tid] = ib;
      }
    }
    __syncthreads();
  }
  const int p = s_idx[0];
  if (tid == 0 && !(s_val[0] > 0.0)) atomicOr(status, ST_SINGULAR);
  if (p != j) {
    for (int c = tid; c < 2 * n; c += blockDim.x) {
      double *T = c < n ? M : Y;
      const int cc = c < n ? c : c - n;
      mdv<K, P> a, b;
      ld_aos<K, P>(T + ((long long)cc * n + j) * VS, a);
      ld_aos<K, P>(T + ((long long)cc * n + p) * VS, b);
      st_aos<K, P>(T + ((long long)cc * n + j) * VS, b);
      st_aos<K, P>(T + ((long long)cc * n + p) * VS, a);
    }
  }
  __syncthreads();
  __shared__ mdv<K, P> s_ri;
  if (tid == 0) {
    mdv<K, P> piv, one, ri;
    ld_aos<K, P>(M + ((long long)j * n + j) * VS, piv);
    c_zero<K, P>(one);
    one.v[0][0] = 1.0;
    c_div<K, P>(one, piv, ri);
    st_aos<K, P>(rinv + (long long)j * VS, ri);
    s_ri = ri;
  }
  __syncthreads();
  const mdv<K, P> ri = s_ri;
  for (int i = j + 1 + tid; i < n; i += blockDim.x) {
    mdv<K, P> a, l;
    ld_aos<K, P>(M + ((long long)j * n + i) * VS, a);
    c_mul<K, P>(a, ri, l);
    st_aos<K, P>(M + ((long long)j * n + i) * VS, l);
  }
}

// Trailing update of column j: M_ik -= l_ij M_jk for i, k > j.
template <int K, int P>
__global__ void lu_update_kernel(double *__restrict__ M, int n, int j) {
  const int m = n - j - 1;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)m * m) return;
  const int i = j + 1 + (int)(e % m), k = j + 1 + (int)(e / m);
  const long long VS = P * K;
  mdv<K, P> l, u, a, t;
  ld_aos<K, P>(M + ((long long)j * n + i) * VS, l);
  ld_aos<K, P>(M + ((long long)k * n + j) * VS, u);
  ld_aos<K, P>(M + ((long long)k * n + i) * VS, a);
  c_mul<K, P>(l, u, t);
  c_sub<K, P>(a, t, a);
  st_aos<K, P>(M + ((long long)k * n + i) * VS, a);
}

// Forward substitution step j of L Z = Y (unit diagonal): Y_ic -= L_ij Y_jc, i > j.
template <int K, int P>
__global__ void lu_forward_kernel(const double *__restrict__ M, double *__restrict__ Y, int n, int j) {
  const int m = n - j - 1;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  const int i = j + 1 + (int)(e % m), c = (int)(e / m);
  const long long VS = P * K;
  mdv<K, P> l, z, y, t;
  ld_aos<K, P>(M + ((long long)j * n + i) * VS, l);
  ld_aos<K, P>(Y + ((long long)c * n + j) * VS, z);
  ld_aos<K, P>(Y + ((long long)c * n + i) * VS, y);
  c_mul<K, P>(l, z, t);
  c_sub<K, P>(y, t, y);
  st_aos<K, P>(Y + ((long long)c * n + i) * VS, y);
}

// 1 / (||A_0||_1 ||W||_1) from the leading limbs (moduli in double): the
// reciprocal condition number of A_0 in the 1-norm, W = A_0^-1 (the
// pseudo-inverse when N > n) being formed by the solve.  A: caller layout
// [P][K][d+1][n][N] (coefficient 0, column-major); W: n x N row-major AoS.
// One CTA.
template <int K, int P>
__global__ void __launch_bounds__(256) rcond_kernel(const double *__restrict__ A, const double *__restrict__ W,
                                                    double *__restrict__ out, int N, int n, int d) {
  __shared__ double s_max[2][256];
  const int tid = threadIdx.x;
  const long long nn = (long long)N * n, pstride = (long long)K * (d + 1) * nn, VS = P * K;
  double ma = 0.0, mw = 0.0;
  for (int c = tid; c < n; c += blockDim.x) {  // ||A_0||_1: N rows of column c
    double sa = 0.0;
    for (int r = 0; r < N; ++r) {
      const double are = A[(long long)c * N + r];
      const double aim = P == 2 ? A[pstride + (long long)c * N + r] : 0.0;
      sa += sqrt(are * are + aim * aim);
    }
    ma = fmax(ma, sa);
  }
  for (int c = tid; c < N; c += blockDim.x) {  // ||W||_1: n rows of column c
    double sw = 0.0;
    for (int r = 0; r < n; ++r) {
      const double *w = W + ((long long)r * N + c) * VS;
      const double wre = w[0], wim = P == 2 ? w[K] : 0.0;
      sw += sqrt(wre * wre + wim * wim);
    }
    mw = fmax(mw, sw);
  }
  s_max[0][tid] = ma;
  s_max[1][tid] = mw;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (tid < off) {
      s_max[0][tid] = fmax(s_max[0][tid], s_max[0][tid + off]);
      s_max[1][tid] = fmax(s_max[1][tid], s_max[1][tid + off]);
    }
    __syncthreads();
  }
  if (tid == 0) out[0] = 1.0 / (s_max[0][0] * s_max[1][0]);
}

// The same back substitution with lookahead: row c of W is known when step c
// starts (W[c][:] = Y[c][:] / R_cc).  The first gA CTAs update row c-1 of Y
// with it and form row c-1 of W (the next step's row); the other CTAs update
// rows 0..c-2.  Each element gets the same operations as in backsub_entry, so
// W is the same; the chain per step is one row instead of the whole step.
template <int K, int P>
__global__ void backsub_row0_kernel(const double *__restrict__ Y, double *__restrict__ W,
                                    const double *__restrict__ rinv, int N, int c) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= N) return;
  const long long VS = P * K;
  if constexpr (K >= kFxMinLimbs) {
    fx_bs_w<K, P>(Y, rinv, N, c, col, W + ((long long)c * N + col) * VS);
    return;
  }
  mdv<K, P> y, ri, w;
  ld_aos<K, P>(Y + ((long long)col * N + c) * VS, y);
  ld_aos<K, P>(rinv + (long long)c * VS, ri);
  c_mul<K, P>(y, ri, w);
  st_aos<K, P>(W + ((long long)c * N + col) * VS, w);
}

template <int K, int P>
__global__ void backsub_step_kernel(const double *__restrict__ M, double *__restrict__ Y, double *__restrict__ W,
                                    const double *__restrict__ rinv, int N, int c, int gA) {
  const long long VS = P * K;
  if ((int)blockIdx.x < gA) {  // row c-1, then W[c-1][:]
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= N) return;
    if constexpr (K >= kFxMinLimbs) {
      fx_bs_update<K, P>(M, Y, W + ((long long)c * N + col) * VS, N, c, col, c - 1);
      fx_bs_w<K, P>(Y, rinv, N, c - 1, col, W + ((long long)(c - 1) * N + col) * VS);
      return;
    }
    mdv<K, P> w, rc, t, yi, ri;
    ld_aos<K, P>(W + ((long long)c * N + col) * VS, w);
    ld_aos<K, P>(M + ((long long)c * N + (c - 1)) * VS, rc);
    ld_aos<K, P>(Y + ((long long)col * N + (c - 1)) * VS, yi);
    c_mul<K, P>(rc, w, t);
    c_sub<K, P>(yi, t, yi);
    st_aos<K, P>(Y + ((long long)col * N + (c - 1)) * VS, yi);
    ld_aos<K, P>(rinv + (long long)(c - 1) * VS, ri);
    c_mul<K, P>(yi, ri, w);
    st_aos<K, P>(W + ((long long)(c - 1) * N + col) * VS, w);
    return;
  }
  // rows 0..c-2: e = col * (c-1) + i
  const long long e = (blockIdx.x - gA) * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)(c - 1) * N) return;
  const int i = (int)(e % (c - 1)), col = (int)(e / (c - 1));
  if constexpr (K >= kFxMinLimbs) {
    fx_bs_update<K, P>(M, Y, W + ((long long)c * N + col) * VS, N, c, col, i);
    return;
  }
  mdv<K, P> w, rc, t, yi;
  ld_aos<K, P>(W + ((long long)c * N + col) * VS, w);
  ld_aos<K, P>(M + ((long long)c * N + i) * VS, rc);
  ld_aos<K, P>(Y + ((long long)col * N + i) * VS, yi);
  c_mul<K, P>(rc, w, t);
  c_sub<K, P>(yi, t, yi);
  st_aos<K, P>(Y + ((long long)col * N + i) * VS, yi);
}

// Partial sums of sum_{j<k} A_{k-j} dx_j for item e = (row, chunk); term index
// t = j*n + col over [chunk*C, min((chunk+1)*C, k*n)).  A is the caller's
// SoA [P][K][d+1][n][n] (column-major blocks); dx is AoS [k][i].
template <int K, int P>
__device__ __forceinline__ void rhs_partial_item(const double *A, const double *dx,
                                                 double *part, int N, int n, int d, int k, int C, int nchunk,
                                                 long long e) {
  const int row = (int)(e % N), chunk = (int)(e / N);
  const long long nn = (long long)N * n, VS = P * K, stride = (long long)(d + 1) * nn;
  const int t0 = chunk * C, t1 = min(t0 + C, k * n);
  mdv<K, P> acc, a, x, prod;
  c_zero<K, P>(acc);
  for (int t = t0; t < t1; ++t) {
    const int j = t / n, col = t % n;
    ld_soa<K, P>(A + (long long)(k - j) * nn + (long long)col * N + row, stride, a);
    ld_aos<K, P>(dx + ((long long)j * n + col) * VS, x);
    c_mul<K, P>(a, x, prod);
    if (t == t0)
      acc = prod;
    else
      c_add<K, P>(acc, prod, acc);
  }
  st_aos<K, P>(part + ((long long)row * nchunk + chunk) * VS, acc);
}

template <int K, int P>
__global__ void rhs_partial_kernel(const double *__restrict__ A, const double *__restrict__ dx,
                                   double *__restrict__ part, int N, int n, int d, int k, int C, int nchunk) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)N * nchunk) return;
  rhs_partial_item<K, P>(A, dx, part, N, n, d, k, C, nchunk, e);
}

// r_k[row] = sgn * b_k[row] - (sum of the row's nchunk partials), row < N.
// b: [P][K][N][d+1].  CTA body: a group of gn threads (gt = index in the
// group) per row, as in row_tree.
template <int K, int P>
__device__ __forceinline__ void rhs_finish_row(const double *b, double sgn, const double *part, double *r, int N,
                                               int d, int k, int nchunk, int row, double (*sm)[K], int gt, int gn,
                                               bool act) {
  if constexpr (K >= kFxMinLimbs) {  // the partials summed in fixed point (house_fx.cuh)
    (void)sm;
    (void)gn;  // groups are kRowLanes threads
    rhs_finish_row_fx<K, P>(b, sgn, part, r, N, d, k, nchunk, row, gt, act);
    return;
  }
  constexpr int Vc = kRowLanes / P;
  const long long VS = P * K;
  const int nleaf = min(nchunk, Vc);
  for (int v = gt; act && v < kRowLanes; v += gn) {
    const int p = v / Vc, cs = v % Vc;
    if (cs < nleaf) {
      double acc[K], t[K];
      ld_limbs<K>(part + ((long long)row * nchunk + cs) * VS + p * K, acc);
      for (int c = cs + Vc; c < nchunk; c += Vc) {
        ld_limbs<K>(part + ((long long)row * nchunk + c) * VS + p * K, t);
        md_add<K>(acc, t, acc);
      }
      st_limbs<K>(sm[v], acc);
    }
  }
  __syncthreads();
  row_tree<K, P>(sm, nleaf, gt, gn, act);
  for (int p = gt; act && p < P; p += gn) {
    double bv[K], a[K], z[K];
    const long long stride = (long long)N * (d + 1);
#pragma unroll
    for (int l = 0; l < K; ++l) bv[l] = b[(long long)row * (d + 1) + k + (long long)(p * K + l) * stride];
    if (sgn < 0.0) md_neg<K>(bv, bv);
    if (nleaf > 0) {
      ld_limbs<K>(sm[p * Vc], a);
      md_sub<K>(bv, a, z);
    } else {
#pragma unroll
      for (int l = 0; l < K; ++l) z[l] = bv[l];
    }
    st_limbs<K>(r + ((long long)k * N + row) * VS + p * K, z);
  }
  __syncthreads();
}

template <int K, int P>
__device__ __forceinline__ void rhs_finish_row(const double *b, double sgn, const double *part, double *r, int N,
                                               int d, int k, int nchunk, int row, double (*sm)[K]) {
  rhs_finish_row<K, P>(b, sgn, part, r, N, d, k, nchunk, row, sm, threadIdx.x, blockDim.x, true);
}

template <int K, int P>
__global__ void __launch_bounds__(kRowLanes) rhs_finish_kernel(const double *__restrict__ b, double sgn,
                                                               const double *__restrict__ part,
                                                               double *__restrict__ r, int N, int d, int k,
                                                               int nchunk) {
  __shared__ double sm[kRowLanes][K];
  rhs_finish_row<K, P>(b, sgn, part, r, N, d, k, nchunk, blockIdx.x, sm);
}

// dx_k[row] = sum_{col < N} W[row][col] r_k[col], row < n.  CTA body, with
// groups as in rhs_finish_row.
template <int K, int P>
__device__ __forceinline__ void wmv_row(const double *W, const double *r, double *dx, int N, int n, int k, int row,
                                        double (*sm)[K], int gt, int gn, bool act) {
  if constexpr (K >= kFxMinLimbs) {  // W = A_0^-1 applied in fixed point, as it was formed (house_fx.cuh)
    (void)sm;
    (void)gn;  // groups are kRowLanes threads
    wmv_row_fx<K, P>(W, r, dx, N, n, k, row, gt, act);
    return;
  }
  constexpr int Vc = kRowLanes / P;
  const long long VS = P * K;
  const int nleaf = min(N, Vc);
  for (int v = gt; act && v < kRowLanes; v += gn) {
    const int p = v / Vc, cs = v % Vc;
    if (cs < nleaf) {
      double acc[K], t[K];
      plane_prod<K, P>(W + ((long long)row * N + cs) * VS, r + ((long long)k * N + cs) * VS, p, acc);
      for (int c = cs + Vc; c < N; c += Vc) {
        plane_prod<K, P>(W + ((long long)row * N + c) * VS, r + ((long long)k * N + c) * VS, p, t);
        md_add<K>(acc, t, acc);
      }
      st_limbs<K>(sm[v], acc);
    }
  }
  __syncthreads();
  row_tree<K, P>(sm, nleaf, gt, gn, act);
  for (int p = gt; act && p < P; p += gn) {
    double z[K];
    ld_limbs<K>(sm[p * Vc], z);
    st_limbs<K>(dx + ((long long)k * n + row) * VS + p * K, z);
  }
  __syncthreads();
}

template <int K, int P>
__device__ __forceinline__ void wmv_row(const double *W, const double *r, double *dx, int N, int n, int k, int row,
                                        double (*sm)[K]) {
  wmv_row<K, P>(W, r, dx, N, n, k, row, sm, threadIdx.x, blockDim.x, true);
}

template <int K, int P>
__global__ void __launch_bounds__(kRowLanes) wmv_kernel(const double *__restrict__ W, const double *__restrict__ r,
                                                        double *__restrict__ dx, int N, int n, int k) {
  __shared__ double sm[kRowLanes][K];
  wmv_row<K, P>(W, r, dx, N, n, k, blockIdx.x, sm);
}

// dx (AoS [k][i]) -> SoA [P][K][n][d+1]; optionally x += dx and the norms
// nrm[0] = max_i |dx_{d,i}|, nrm[1] = max |dx| from the leading limbs.
template <int K, int P>
__device__ __forceinline__ void finish_entry(const double *dxw, double *dx_out,
                                             double *x, double *nrm,
                                             int *status, int n, int d, long long e) {
  const int j = (int)(e / (d + 1)), k = (int)(e % (d + 1));
  const long long VS = P * K, stride = (long long)n * (d + 1);
  mdv<K, P> v;
  ld_aos<K, P>(dxw + ((long long)k * n + j) * VS, v);
  bool finite = true;
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int l = 0; l < K; ++l) finite = finite && isfinite(v.v[p][l]);
  if (!finite) atomicOr(status, ST_NONFINITE);
  if (dx_out) st_soa<K, P>(dx_out + e, stride, v);
  if (x) {
    mdv<K, P> xv;
    ld_soa<K, P>(x + e, stride, xv);
    c_add<K, P>(xv, v, xv);
    st_soa<K, P>(x + e, stride, xv);
  }
  if (nrm) {
    const double re = v.v[0][0];
    const double im = (P == 2) ? v.v[P - 1][0] : 0.0;
    const double mod = __dsqrt_rn(__dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im)));
    if (finite) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(mod);
      atomicMax(reinterpret_cast<unsigned long long *>(nrm) + 1, bits);
      if (k == d) atomicMax(reinterpret_cast<unsigned long long *>(nrm), bits);
    }
  }
}

template <int K, int P>
__global__ void finish_dx_kernel(const double *__restrict__ dxw, double *__restrict__ dx_out, double *__restrict__ x,
                                 double *__restrict__ nrm, int *__restrict__ status, int n, int d) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * (d + 1)) return;
  finish_entry<K, P>(dxw, dx_out, x, nrm, status, n, d, e);
}

}  // namespace mdk
