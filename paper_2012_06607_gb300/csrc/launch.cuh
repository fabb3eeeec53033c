// Templated launchers; explicitly instantiated once per limb count (inst_k*.cu).
#pragma once
#include "internal.h"
#include "kernels.cuh"
#include <algorithm>

#include "ozaki.cuh"
#include "batched.cuh"

namespace mdk {

inline unsigned blocks_for(long long work, int threads) { return (unsigned)((work + threads - 1) / threads); }

template <int K, int P>
cudaError_t Impl<K, P>::elementwise(int op, long long count, const double *x, const double *y, double *z,
                                    cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int T = 128;
  const unsigned B = blocks_for(count, T);
  ProfScope prof(PK_ELEMENTWISE, s);
  switch (op) {
    case 0: elementwise_kernel<K, P, 0><<<B, T, 0, s>>>(count, x, y, z); break;
    case 1: elementwise_kernel<K, P, 1><<<B, T, 0, s>>>(count, x, y, z); break;
    case 2: elementwise_kernel<K, P, 2><<<B, T, 0, s>>>(count, x, y, z); break;
    case 3: elementwise_kernel<K, P, 3><<<B, T, 0, s>>>(count, x, y, z); break;
    case 4: elementwise_kernel<K, P, 4><<<B, T, 0, s>>>(count, x, y, z); break;
    case 5: elementwise_kernel<K, P, 5><<<B, T, 0, s>>>(count, x, y, z); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int K, int P>
cudaError_t Impl<K, P>::series_conv(int d, long long count, const double *x, const double *y, double *z,
                                    cudaStream_t s) {
  const long long work = count * (d + 1);
  if (work <= 0) return cudaSuccess;
  const int T = 64;
  ProfScope prof(PK_SERIES, s);
  series_conv_kernel<K, P><<<blocks_for(work, T), T, 0, s>>>(d, count, x, y, z);
  return cudaGetLastError();
}

template <int K, int P>
cudaError_t Impl<K, P>::batched(const BatchDev &b, cudaStream_t s) {
  if constexpr (K > kBatchMaxLimbs) {
    (void)b;
    (void)s;
    return cudaErrorNotSupported;
  } else {
    if (b.njobs <= 0) return cudaSuccess;
    // the kernel splits its threads into groups of kRowLanes
    if (b.threads < kRowLanes || b.threads % kRowLanes != 0 || b.threads > kBatchMaxThreads)
      return cudaErrorInvalidValue;
    const int smem = b.ctas_per_sm > 0 ? batched_cap_bytes<K, P>(b.ctas_per_sm) : 0;
    batched_step_kernel<K, P><<<b.grid, b.threads, smem, s>>>(b.jobs, b.order, b.njobs, b.counter, b.ibase, b.dbase,
                                                                  b.nrm, b.times, b.status, b.update_x, b.resident,
                                                                  b.times_stride, b.split);
    return cudaGetLastError();
  }
}

template <int K, int P>
cudaError_t Impl<K, P>::batched_setup() {
  if constexpr (K > kBatchMaxLimbs) {
    return cudaErrorNotSupported;
  } else {
    // room for the largest cap (one CTA per SM), and the largest shared-memory
    // carveout, so that cps CTAs with their share fit on one SM
    const cudaError_t e = cudaFuncSetAttribute(batched_step_kernel<K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               batched_cap_bytes<K, P>(1));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batched_step_kernel<K, P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
  }
}

template <int K, int P>
cudaError_t Impl<K, P>::eval0(const EvalDev &e, cudaStream_t s) {
  const int n = e.n, d = e.d;
  cudaError_t err;
  const long long nx = (long long)n * (d + 1);
  {
    ProfScope prof(PK_POOL, s);
    if constexpr (K >= kFxConvMinLimbs) {
      if (e.split) {  // both pools: the fixed-point products read the converted copy
        pool_load_x_fx_kernel<K, P><<<blocks_for(nx, 128), 128, 0, s>>>(e.x, e.pool, e.fxpool, n, d);
      } else {
        pool_load_x_kernel<K, P><<<blocks_for(nx, 128), 128, 0, s>>>(e.x, e.pool, n, d);
      }
    } else {
      pool_load_x_kernel<K, P><<<blocks_for(nx, 128), 128, 0, s>>>(e.x, e.pool, n, d);
    }
  }
  if (e.nscal > 0) {
    ProfScope prof(PK_SCAL, s);
    bool fx = false;
    if constexpr (K >= kFxConvMinLimbs) fx = e.split != 0;
    if (fx)  // also packed, for the fixed-point accumulation
      prep_scal_fx_kernel<K, P><<<blocks_for(e.nscal, 64), 64, 0, s>>>(e.scal_src, e.nscal, e.coef, e.nmono, e.scal,
                                                                       e.fxscal);
    else
      prep_scal_kernel<K, P><<<blocks_for(e.nscal, 64), 64, 0, s>>>(e.scal_src, e.nscal, e.coef, e.nmono, e.scal);
  }
  const size_t Abytes = sizeof(double) * P * K * (size_t)(d + 1) * e.N * n;
  if ((err = cudaMemsetAsync(e.A, 0, Abytes, s)) != cudaSuccess) return err;
  // coefficient 0 of every product is the single product of the inputs' coefficients 0
  for (int st = 0; st < e.nstages; ++st) {
    const int t0 = e.stage_off0[st], t1 = e.stage_off0[st + 1];
    if (t1 > t0) {
      ProfScope prof(PK_CONV, s);
      conv_stage_kernel<K, P><<<blocks_for(t1 - t0, 64), 64, 0, s>>>(e.tasks0 + 8LL * t0, t1 - t0, e.pool, d);
    }
  }
  // coefficient 0 of A (what the factorisation of A_0 needs); f_0 comes with the rest
  if (e.ngroups > 0) {
    ProfScope prof(PK_ACCUM, s);
    accum_kernel<K, P><<<blocks_for(e.ngroups, 128), 128, 0, s>>>(reinterpret_cast<const int4 *>(e.groups), e.ngroups,
                                                                  reinterpret_cast<const int4 *>(e.contrib), e.pool,
                                                                  e.scal, e.cst, e.f, e.A, e.N, n, d, 0, 1, 1);
  }
  return cudaGetLastError();
}

template <int K, int P>
cudaError_t Impl<K, P>::eval_rest(const EvalDev &e, cudaStream_t s) {
  const int n = e.n, d = e.d;
  for (int st = 0; st < e.nstages; ++st) {
    const int t0 = e.stage_off[st], t1 = e.stage_off[st + 1];
    if (t1 <= t0) continue;
    ProfScope prof(PK_CONV, s);
    if constexpr (K >= kFxConvMinLimbs) {
      if (e.split) {  // the split-product form: every term on 32-bit word slices
        // No shared memory reserved: the CTAs' registers (threads x registers
        // of conv_fx_threads) fill the SM's register file, which keeps the
        // factorisation's CTAs off their SMs as well, and the L1 left to the
        // kernel holds the operands it re-reads.
        auto kern = conv_stage_fx_kernel<K, P>;
        const int smem = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0) != cudaSuccess)
          (void)cudaGetLastError();
        constexpr int T = conv_fx_threads<K>();
        const unsigned grid = e.resident_ctas > 0 ? (unsigned)e.resident_ctas : blocks_for(t1 - t0, T);
        kern<<<grid, T, smem, s>>>(e.tasks + 8LL * t0, t1 - t0, e.pool, e.fxpool, d);
        continue;
      }
    }
    if (e.resident_ctas > 0) {
      // The CTAs reserve all the shared memory an SM offers (the kernel does
      // not use it), so that kernels on the other stream cannot share their
      // SMs and stay on the SMs left free.
      int smem = e.resident_smem;
      if (smem > 0 &&
          cudaFuncSetAttribute(conv_stage_resident_kernel<K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
              cudaSuccess) {
        (void)cudaGetLastError();
        smem = 0;
      }
      conv_stage_resident_kernel<K, P><<<e.resident_ctas, conv_resident_threads<K>(), smem, s>>>(e.tasks + 8LL * t0,
                                                                                           t1 - t0, e.pool, d);
    } else {
      conv_stage_kernel<K, P><<<blocks_for(t1 - t0, 64), 64, 0, s>>>(e.tasks + 8LL * t0, t1 - t0, e.pool, d);
    }
  }
  if constexpr (K >= kFxConvMinLimbs) {
    if (e.split) {  // the split-product form: contribution values and sums in fixed point
      if (e.ncontrib > 0) {
        ProfScope prof(PK_ACCUM, s);
        const long long work = (long long)e.ncontrib * (d + 1);
        accum_prod_fx_kernel<K, P><<<blocks_for(work, 128), 128, 0, s>>>(reinterpret_cast<const int4 *>(e.contrib),
                                                                         e.ncontrib, e.fxpool, e.fxscal, e.fxprod, d);
      }
      if (e.ngroups > 0) {
        ProfScope prof(PK_ACCUM, s);
        const long long work = (long long)e.ngroups * (d + 1);
        accum_sum_fx_kernel<K, P><<<blocks_for(work, 128), 128, 0, s>>>(reinterpret_cast<const int4 *>(e.groups),
                                                                        e.ngroups, e.fxprod, e.cst, e.f, e.A, e.N, n,
                                                                        d, 1);
      }
      return cudaGetLastError();
    }
  }
  if (e.ncontrib > 0) {
    ProfScope prof(PK_ACCUM, s);
    const long long work = (long long)e.ncontrib * (d + 1);
    accum_prod_kernel<K, P><<<blocks_for(work, 128), 128, 0, s>>>(reinterpret_cast<const int4 *>(e.contrib),
                                                                  e.ncontrib, e.pool, e.scal, e.prod, d);
  }
  if (e.ngroups > 0) {
    ProfScope prof(PK_ACCUM, s);
    const long long work = (long long)e.ngroups * (d + 1);
    accum_sum_kernel<K, P><<<blocks_for(work, 128), 128, 0, s>>>(reinterpret_cast<const int4 *>(e.groups),
                                                                 e.ngroups, e.prod, e.cst, e.f, e.A, e.N, n, d, 1);
  }
  return cudaGetLastError();
}

template <int K, int P>
cudaError_t Impl<K, P>::eval(const EvalDev &e, cudaStream_t s) {
  cudaError_t err = eval0(e, s);
  if (err != cudaSuccess) return err;
  return eval_rest(e, s);
}

template <int K, int P>
cudaError_t Impl<K, P>::solve(const SolveDev &v, cudaStream_t s) {
  cudaError_t err = factor(v, s);
  if (err != cudaSuccess) return err;
  return degrees(v, s);
}

template <int K, int P>
cudaError_t Impl<K, P>::factor(const SolveDev &v, cudaStream_t s) {
  const int n = v.n, N = v.N, d = v.d;
  {
    ProfScope prof(PK_QR_HOUSE, s);
    solve_init_kernel<K, P><<<blocks_for((long long)N * N, 128), 128, 0, s>>>(v.A, v.M, v.Y, N, n, d);
  }
  if (v.lu) {  // N = n
    // LU with partial pivoting, L Z = P, then the shared back substitution
    for (int j = 0; j < n; ++j) {
      ProfScope prof(PK_LU, s);
      lu_pivot_kernel<K, P><<<1, 128, 0, s>>>(v.M, v.Y, v.rinv, v.status, n, j);
      const long long m = n - j - 1;
      if (m > 0) lu_update_kernel<K, P><<<blocks_for(m * m, 128), 128, 0, s>>>(v.M, n, j);
    }
    for (int j = 0; j + 1 < n; ++j) {
      ProfScope prof(PK_LU, s);
      const long long m = n - j - 1;
      lu_forward_kernel<K, P><<<blocks_for(m * n, 128), 128, 0, s>>>(v.M, v.Y, n, j);
    }
    return backsub(v, n, s);
  }
  {
    ProfScope prof(PK_QR_HOUSE, s);
    house_kernel<K, P><<<1, kHouseThreads, 0, s>>>(v.M, v.vd, v.beta, v.status, N, 0);
  }
  for (int j = 0; j < n; ++j) {
    // H_j on every target, and the Householder vector of column j+1 (lookahead)
    ProfScope prof(PK_QR_APPLY, s);
    const int rest = (n - j - 1) + N - (j + 1 < n ? 1 : 0);
    const int grid = 1 + (qr_cta_per_target<K>() ? rest : (int)blocks_for((long long)rest * 32, kHouseThreads));
    house_step_kernel<K, P><<<grid, kHouseThreads, 0, s>>>(v.M, v.Y, v.vd, v.beta, v.status, N, n, j);
  }
  {
    ProfScope prof(PK_RINV, s);
    rinv_kernel<K, P><<<blocks_for(n, 64), 64, 0, s>>>(v.M, v.rinv, N, n);
  }
  return backsub(v, N, s);
}

// W = R^-1 Y[0:n, :] (N columns), lookahead form: row c of W is ready when
// step c starts.
template <int K, int P>
cudaError_t Impl<K, P>::backsub(const SolveDev &v, int N, cudaStream_t s) {
  const int n = v.n;
  {
    ProfScope prof(PK_BACKSUB, s);
    backsub_row0_kernel<K, P><<<blocks_for(N, 64), 64, 0, s>>>(v.Y, v.W, v.rinv, N, n - 1);
  }
  for (int c = n - 1; c >= 1; --c) {
    ProfScope prof(PK_BACKSUB, s);
    const int gA = (int)blocks_for(N, 64);
    const long long rest = (long long)(c - 1) * N;
    backsub_step_kernel<K, P><<<gA + (int)blocks_for(rest, 64), 64, 0, s>>>(v.M, v.Y, v.W, v.rinv, N, c, gA);
  }
  return cudaGetLastError();
}

template <int K, int P>
cudaError_t Impl<K, P>::rcond(const SolveDev &v, cudaStream_t s) {
  rcond_kernel<K, P><<<1, 256, 0, s>>>(v.A, v.W, v.rcond, v.N, v.n, v.d);
  return cudaGetLastError();
}

template <int K, int P>
cudaError_t Impl<K, P>::degrees(const SolveDev &v, cudaStream_t s) {
  const int n = v.n, N = v.N, d = v.d;  // the split-product form needs N = n
  __nv_bfloat16 *As = static_cast<__nv_bfloat16 *>(v.oz_As), *Xs = static_cast<__nv_bfloat16 *>(v.oz_Xs);
  constexpr int oz_smem = oz_update_smem(K);
  static_assert(oz_smem <= kOzSmemBudget, "staged slices exceed the shared memory of an SM");
  int oz_slots = 0;  // update CTAs resident on the whole GPU
  if (v.ozaki) {
    cudaError_t e = cudaFuncSetAttribute(oz_update_kernel<K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, oz_smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oz_update_kernel<K, P>, oz_warps(K) * 32,
                                                           oz_smem)) != cudaSuccess)
      return e;
    oz_slots = std::max(1, sms * per_sm);
    e = cudaMemsetAsync(v.oz_acc, 0, sizeof(unsigned long long) * (size_t)n * P * oz_digits(K), s);
    if (e != cudaSuccess) return e;
  }
  if (v.ozaki && d >= 1) {
    ProfScope prof(PK_OZ_SPLIT, s);
    oz_split_rows_kernel<K, P><<<blocks_for((long long)d * n * 32, 128), 128, 0, s>>>(v.A, As, v.oz_eA, n, d);
  }
  for (int k = 0; k <= d; ++k) {
    if (v.ozaki) {
      if (k >= 1) {
        ProfScope prof(PK_OZ_SPLIT, s);
        oz_split_vec_kernel<K, P><<<1, 128, 0, s>>>(v.dxw, Xs, v.oz_ex, n, k - 1);
      }
      {
        ProfScope prof(PK_OZ_UPDATE, s);
        // G CTAs per output: as many as fit on the GPU at once (one wave)
        const int nw = oz_warps(K), outs = n * P;
        const int G = std::max(1, std::min((k + nw - 1) / nw, oz_slots / outs));
        oz_update_kernel<K, P><<<outs * G, nw * 32, oz_smem, s>>>(As, Xs, v.oz_eA, v.oz_ex, v.b, v.oz_acc, n, d, k,
                                                                   G);
        oz_finish_kernel<K, P><<<outs, 32, 0, s>>>(v.oz_eA, v.oz_ex, v.b, v.sgn, v.oz_acc, v.r, n, d, k);
      }
      ProfScope prof(PK_WMV, s);
      wmv_kernel<K, P><<<n, kRowLanes, 0, s>>>(v.W, v.r, v.dxw, n, n, k);
      continue;
    }
    int C, nchunk;
    rhs_chunking(N, n, k, C, nchunk);
    if (nchunk > 0) {
      ProfScope prof(PK_RHS_PARTIAL, s);
      rhs_partial_kernel<K, P><<<blocks_for((long long)N * nchunk, 64), 64, 0, s>>>(v.A, v.dxw, v.part, N, n, d, k,
                                                                                    C, nchunk);
    }
    {
      ProfScope prof(PK_RHS_FINISH, s);
      rhs_finish_kernel<K, P><<<N, kRowLanes, 0, s>>>(v.b, v.sgn, v.part, v.r, N, d, k, nchunk);
    }
    ProfScope prof(PK_WMV, s);
    wmv_kernel<K, P><<<n, kRowLanes, 0, s>>>(v.W, v.r, v.dxw, N, n, k);
  }
  const long long nx = (long long)n * (d + 1);
  ProfScope prof(PK_FINISH, s);
  finish_dx_kernel<K, P><<<blocks_for(nx, 128), 128, 0, s>>>(v.dxw, v.dx_out, v.x, v.nrm, v.status, n, d);
  return cudaGetLastError();
}

}  // namespace mdk
