// Batched form: many independent systems of uneven dimension n and degree d,
// one Newton step each, in persistent launches per precision class.
//
// Every CTA (128 to 384 threads) takes the next system from an atomic job
// counter (systems listed longest first) and runs that system's whole step:
// series products stage by stage, accumulation of f and A, Householder QR of
// A_0 with Q^H, W = R^-1 Q^H, the degree loop of the block Toeplitz solve and
// the update of x -- with __syncthreads between phases and no waiting on other
// CTAs, so nothing can hang.  The per-item bodies and reduction trees are
// those of the one-system kernels, so every system gets the same bits as a
// single-system step.  The most expensive systems may run in a launch whose
// CTAs each hold a whole SM (see batched_cap_bytes); the others share SMs.

#pragma once
#include "kernels.cuh"

namespace mdk {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Called by every thread of the CTA at a phase boundary that all of them have
// passed (after a __syncthreads); thread 0 writes the global timer.
__device__ __forceinline__ void phase_stamp(bool on, unsigned long long *times, long long at) {
  if (on && threadIdx.x == 0) times[at] = global_ns();
}

// CTA sizes of the batched kernel: kBatchThreads (default) up to kBatchMaxThreads.
constexpr int kBatchThreads = 128;
constexpr int kBatchMaxThreads = 384;
static_assert(kBatchMaxThreads / 32 <= kFxMaxWarps, "fixed-point row sums keep one slot per warp");

template <int K, int P>
__global__ void batched_step_kernel(const BatchJob *__restrict__ jobs, const int *__restrict__ order, int njobs,
                                    int *__restrict__ counter, const int *ibase, double *dbase,
                                    double *__restrict__ nrm, unsigned long long *__restrict__ times,
                                    int *__restrict__ status, int update_x, int *__restrict__ resident, int tstride,
                                    int split);

// Dynamic shared memory per CTA of the batched kernel that lets at most
// `cps` CTAs share an SM: the SM's shared memory split cps ways, less the
// per-CTA reserve and the kernel's static shared memory (cps = 1: the CTA
// holds a whole SM).  The kernel does not use it; it only bounds residency,
// which registers alone would leave at up to four CTAs per SM.
template <int K, int P>
inline int batched_cap_bytes(int cps) {
  int dev = 0, per_sm = 0, resv = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cps < 1 || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, batched_step_kernel<K, P>) != cudaSuccess)
    return 0;
  const int room = optin - (int)fa.sharedSizeBytes;
  const int b = per_sm / cps - resv - (int)fa.sharedSizeBytes;
  return b <= 0 ? 0 : (b < room ? b : room);
}

template <int K, int P>
__global__ void __launch_bounds__(kBatchMaxThreads) batched_step_kernel(const BatchJob *__restrict__ jobs,
                                                                     const int *__restrict__ order, int njobs,
                                                                     int *__restrict__ counter,
                                                                     const int *ibase, double *dbase,
                                                                     double *__restrict__ nrm,
                                                                     unsigned long long *__restrict__ times,
                                                                     int *__restrict__ status, int update_x,
                                                                     int *__restrict__ resident, int tstride,
                                                                     int split) {
  __shared__ int s_job;
  // one reduction buffer per group of kRowLanes threads: the degree loop
  // reduces that many rows at once
  __shared__ double s_rows[kBatchMaxThreads / kRowLanes][kRowLanes][K];
  double(*s_row)[K] = s_rows[0];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x, nwarp = NT / 32;
  const int G = NT / kRowLanes, grp = tid / kRowLanes, gt = tid % kRowLanes;
  if (resident && tid == 0) atomicAdd(resident, 1);
  // times: tstride stamps per system; with kPhaseStamps, one after each phase
  const bool phases = times && tstride == kPhaseStamps;
  for (;;) {
    if (tid == 0) s_job = atomicAdd(counter, 1);
    __syncthreads();
    const int q = s_job;
    __syncthreads();
    if (q >= njobs) return;
    const int job = order[q];
    const BatchJob J = jobs[job];
    const int n = J.n, d = J.d;
    if (tid == 0) {
      if (times) times[(long long)tstride * job] = global_ns();
      if (nrm) {
        nrm[2 * job] = 0.0;
        nrm[2 * job + 1] = 0.0;
      }
    }
    double *pool = dbase + J.pool;
    double *scal = dbase + J.scal;
    double *f = dbase + J.f;
    double *A = dbase + J.A;
    // the split-product form (uniform over the launch): products and update
    // sums on 32-bit word slices, operands from packed fixed-point copies
    const bool fx = K >= kFxConvMinLimbs && split;
    uint32_t *fxpool = reinterpret_cast<uint32_t *>(dbase + J.fxpool);
    uint32_t *fxA = reinterpret_cast<uint32_t *>(dbase + J.fxA);
    uint32_t *fxdx = reinterpret_cast<uint32_t *>(dbase + J.fxdx);
    constexpr int PW = packed_words(fxp::words_for(K));
    // ---- evaluate and differentiate
    for (long long e = tid; e < (long long)n * (d + 1); e += NT) {
      if (fx)
        pool_load_entry_fx<K, P>(J.x, pool, fxpool, n, d, e);
      else
        pool_load_entry<K, P>(J.x, pool, n, d, e);
    }
    uint32_t *fxscal = reinterpret_cast<uint32_t *>(dbase + J.fxscal);
    for (int i = tid; i < J.nscal; i += NT) {
      if (fx)
        prep_scal_entry_fx<K, P>(ibase + J.scal_src, J.coef, J.nmono, scal, fxscal, i);
      else
        prep_scal_entry<K, P>(ibase + J.scal_src, J.coef, J.nmono, scal, i);
    }
    const long long Awords = (long long)P * K * (d + 1) * n * n;
    for (long long e = tid; e < Awords; e += NT) A[e] = 0.0;
    __syncthreads();
    phase_stamp(phases, times, (long long)tstride * job + 1);
    const int *ops = ibase + J.ops;
    const int *soff = ibase + J.stage_off;
    const int npairs = (d + 2) / 2;  // coefficient pairs (k, d-k); the middle one alone when d is even
    for (int st = 0; st < J.nstages; ++st) {
      const int o0 = soff[st], o1 = soff[st + 1];
      const long long items = (long long)(o1 - o0) * npairs;
      for (long long it = tid; it < items; it += NT) {
        const int o = o0 + (int)(it / npairs), p = (int)(it % npairs);
        const int out = ops[3 * o], a = ops[3 * o + 1], b = ops[3 * o + 2];
        // one call for both kinds of item: two inlined copies would run one
        // after the other in a warp that holds both
        const bool pair = 2 * p < d;
        if (fx)
          conv_pair_fx<K, P>(pool, fxpool, d, out, a, b, p, pair ? out : -1, pair ? a : -1, pair ? b : -1);
        else
          conv_pair<K, P, false>(pool, d, out, a, b, p, pair ? out : -1, pair ? a : -1, pair ? b : -1);
      }
      __syncthreads();
    }
    phase_stamp(phases, times, (long long)tstride * job + 2);
    const int4 *groups = reinterpret_cast<const int4 *>(ibase + J.groups);
    const int4 *contrib = reinterpret_cast<const int4 *>(ibase + J.contrib);
    for (long long e = tid; e < (long long)J.ngroups * (d + 1); e += NT) {
      if (fx)
        accum_entry_fx<K, P>(groups, contrib, fxpool, fxscal, J.cst, f, A, n, n, d, (int)(e / (d + 1)),
                             (int)(e % (d + 1)));
      else
        accum_entry<K, P>(groups, contrib, pool, scal, J.cst, f, A, n, n, d, (int)(e / (d + 1)), (int)(e % (d + 1)));
    }
    __syncthreads();
    if (fx) {  // A's values converted once for the update sums of every degree
      const long long cnt = (long long)(d + 1) * n * n;
      for (long long e = tid; e < cnt; e += NT) fx_pack_value<K, P>(A + e, cnt, fxA + e * P * PW);
      __syncthreads();
    }
    phase_stamp(phases, times, (long long)tstride * job + 3);
    // ---- solve A(t) dx(t) = -f(t)
    double *M = dbase + J.M, *Y = dbase + J.Y, *W = dbase + J.W;
    double *vd = dbase + J.vd, *beta = dbase + J.beta, *rinv = dbase + J.rinv;
    double *r = dbase + J.r, *dxw = dbase + J.dxw, *part = dbase + J.part;
    for (long long e = tid; e < (long long)n * n; e += NT) solve_init_entry<K, P>(A, M, Y, n, n, d, e);
    __syncthreads();
    phase_stamp(phases, times, (long long)tstride * job + 4);
    // QR in the order of the lookahead form (same arithmetic per column): H_j
    // on column j+1 by the whole CTA, on the other targets by warps, then the
    // Householder vector of column j+1
    qr_house<K, P>(M, vd, beta, status, n, 0);
    for (int j = 0; j < n; ++j) {
      const bool ahead = j + 1 < n;
      // (no register caching of converted rows here: the batched kernel's
      // register bound would spill them; the values and bits are the same)
      if (ahead) qr_apply_cta<K, P, false>(M, Y, vd, beta, n, n, j, 0, s_row);
      for (int w = warp + (ahead ? 1 : 0); w < (n - j - 1) + n; w += nwarp)
        qr_apply_warp<K, P>(M, Y, vd, beta, n, n, j, w, lane);
      __syncthreads();
      if (ahead) qr_house<K, P>(M, vd, beta, status, n, j + 1);
    }
    if (phases) __syncthreads();
    phase_stamp(phases, times, (long long)tstride * job + 5);
    for (int j = tid; j < n; j += NT) rinv_entry<K, P>(M, rinv, n, j);
    __syncthreads();
    phase_stamp(phases, times, (long long)tstride * job + 6);
    for (int c = n - 1; c >= 0; --c) {
      if constexpr (K >= kFxMinLimbs) {
        // row c of W once, then the rows above it read it: the values that
        // backsub_entry forms in every element (the same bits)
        for (int col = tid; col < n; col += NT)
          fx_bs_w<K, P>(Y, rinv, n, c, col, W + ((long long)c * n + col) * (P * K));
        __syncthreads();
        for (long long e = tid; e < (long long)c * n; e += NT) {
          const int i = (int)(e / n), col = (int)(e % n);
          fx_bs_update<K, P>(M, Y, W + ((long long)c * n + col) * (P * K), n, c, col, i);
        }
      } else {
        for (long long e = tid; e < (long long)(c + 1) * n; e += NT) backsub_entry<K, P>(M, Y, W, rinv, n, c, e);
      }
      __syncthreads();
    }
    phase_stamp(phases, times, (long long)tstride * job + 7);
    for (int k = 0; k <= d; ++k) {
      int C, nchunk;
      rhs_chunking(n, n, k, C, nchunk);
      for (long long e = tid; e < (long long)n * nchunk; e += NT) {
        if (fx)
          rhs_partial_item_fx<K, P>(fxA, fxdx, part, n, n, k, C, nchunk, e);
        else
          rhs_partial_item<K, P>(A, dxw, part, n, n, d, k, C, nchunk, e);
      }
      __syncthreads();
      // G rows at a time, one per group; every row's tree is the one-row tree
      for (int row0 = 0; row0 < n; row0 += G) {
        const bool act = grp < G && row0 + grp < n;
        rhs_finish_row<K, P>(f, -1.0, part, r, n, d, k, nchunk, act ? row0 + grp : 0, s_rows[act ? grp : 0], gt,
                             kRowLanes, act);
      }
      for (int row0 = 0; row0 < n; row0 += G) {
        const bool act = grp < G && row0 + grp < n;
        wmv_row<K, P>(W, r, dxw, n, n, k, act ? row0 + grp : 0, s_rows[act ? grp : 0], gt, kRowLanes, act);
      }
      if (fx && k < d) {  // dx_k for the update sums of the later degrees (wmv_row ends with a barrier)
        for (int e = tid; e < n; e += NT)
          fx_pack_value<K, P>(dxw + ((long long)k * n + e) * (P * K), 1, fxdx + ((long long)k * n + e) * P * PW);
        __syncthreads();
      }
    }
    phase_stamp(phases, times, (long long)tstride * job + 8);
    for (long long e = tid; e < (long long)n * (d + 1); e += NT)
      finish_entry<K, P>(dxw, nullptr, update_x ? J.x : nullptr, nrm ? nrm + 2 * job : nullptr, status, n, d, e);
    __syncthreads();
    if (tid == 0 && times) times[(long long)tstride * job + tstride - 1] = global_ns();
  }
}

}  // namespace mdk
