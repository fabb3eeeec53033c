// C ABI of the library (declared in include/mdnewton.h): argument checks,
// host planning of the evaluation schedule, workspace layout and dispatch to
// the templated launchers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mdnewton.h"
#include "internal.h"

namespace {

using mdk::EvalDev;
using mdk::SolveDev;

bool valid_limbs(int K) { return K == 1 || K == 2 || K == 3 || K == 4 || K == 5 || K == 8 || K == 10; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------ dispatch
template <int K>
cudaError_t dispatch_p(int P, int what, const void *a, cudaStream_t s, int op = 0, long long count = 0, int d = 0,
                       const double *x = nullptr, const double *y = nullptr, double *z = nullptr) {
  if (P == 1) {
    switch (what) {
      case 0: return mdk::Impl<K, 1>::elementwise(op, count, x, y, z, s);
      case 1: return mdk::Impl<K, 1>::series_conv(d, count, x, y, z, s);
      case 2: return mdk::Impl<K, 1>::eval(*static_cast<const EvalDev *>(a), s);
      case 3: return mdk::Impl<K, 1>::solve(*static_cast<const SolveDev *>(a), s);
      case 4:
        if constexpr (K <= mdk::kBatchMaxLimbs) return mdk::Impl<K, 1>::batched(*static_cast<const mdk::BatchDev *>(a), s);
        return cudaErrorNotSupported;
      case 5: return mdk::Impl<K, 1>::eval0(*static_cast<const EvalDev *>(a), s);
      case 6: return mdk::Impl<K, 1>::eval_rest(*static_cast<const EvalDev *>(a), s);
      case 7: return mdk::Impl<K, 1>::factor(*static_cast<const SolveDev *>(a), s);
      case 8: return mdk::Impl<K, 1>::degrees(*static_cast<const SolveDev *>(a), s);
      case 9: return mdk::Impl<K, 1>::rcond(*static_cast<const SolveDev *>(a), s);
      case 10:
        if constexpr (K <= mdk::kBatchMaxLimbs) return mdk::Impl<K, 1>::batched_setup();
        return cudaErrorNotSupported;
    }
  } else {
    switch (what) {
      case 0: return mdk::Impl<K, 2>::elementwise(op, count, x, y, z, s);
      case 1: return mdk::Impl<K, 2>::series_conv(d, count, x, y, z, s);
      case 2: return mdk::Impl<K, 2>::eval(*static_cast<const EvalDev *>(a), s);
      case 3: return mdk::Impl<K, 2>::solve(*static_cast<const SolveDev *>(a), s);
      case 4:
        if constexpr (K <= mdk::kBatchMaxLimbs) return mdk::Impl<K, 2>::batched(*static_cast<const mdk::BatchDev *>(a), s);
        return cudaErrorNotSupported;
      case 5: return mdk::Impl<K, 2>::eval0(*static_cast<const EvalDev *>(a), s);
      case 6: return mdk::Impl<K, 2>::eval_rest(*static_cast<const EvalDev *>(a), s);
      case 7: return mdk::Impl<K, 2>::factor(*static_cast<const SolveDev *>(a), s);
      case 8: return mdk::Impl<K, 2>::degrees(*static_cast<const SolveDev *>(a), s);
      case 9: return mdk::Impl<K, 2>::rcond(*static_cast<const SolveDev *>(a), s);
      case 10:
        if constexpr (K <= mdk::kBatchMaxLimbs) return mdk::Impl<K, 2>::batched_setup();
        return cudaErrorNotSupported;
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t dispatch(int K, int P, int what, const void *a, cudaStream_t s, int op = 0, long long count = 0, int d = 0,
                     const double *x = nullptr, const double *y = nullptr, double *z = nullptr) {
  switch (K) {
    case 1: return dispatch_p<1>(P, what, a, s, op, count, d, x, y, z);
    case 2: return dispatch_p<2>(P, what, a, s, op, count, d, x, y, z);
    case 3: return dispatch_p<3>(P, what, a, s, op, count, d, x, y, z);
    case 4: return dispatch_p<4>(P, what, a, s, op, count, d, x, y, z);
    case 5: return dispatch_p<5>(P, what, a, s, op, count, d, x, y, z);
    case 8: return dispatch_p<8>(P, what, a, s, op, count, d, x, y, z);
    case 10: return dispatch_p<10>(P, what, a, s, op, count, d, x, y, z);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------- solve layout
struct SolveLayout {
  size_t off_M, off_Y, off_W, off_vd, off_beta, off_rinv, off_r, off_dxw, off_part, bytes;
  size_t off_As = 0, off_Xs = 0, off_eA = 0, off_ex = 0, off_acc = 0;
  int maxchunk;
  int ozaki = 0;
};

// slices and accumulator sizes of the split-product form (must match ozaki.cuh)
int oz_slices_host(int K) { return (((53 * K + 24 + 7) / 8) + 15) / 16 * 16; }
int oz_kpad_host(int n) { return (n + 15) / 16 * 16; }

// N x n A_0 (N >= n): M is N x n, Y (Q^H) N x N, W n x N, r has N rows.
SolveLayout solve_layout(int K, int P, int N, int n, int d, size_t base, int flags = 0) {
  SolveLayout L;
  const size_t VS = sizeof(double) * P * K;
  const size_t Nn = (size_t)N * n, NN = (size_t)N * N;
  int maxchunk = 1;
  for (int k = 0; k <= d; ++k) {
    int C, nc;
    mdk::rhs_chunking(N, n, k, C, nc);
    maxchunk = std::max(maxchunk, nc);
  }
  L.maxchunk = maxchunk;
  size_t o = base;
  L.off_M = o; o = align256(o + Nn * VS);
  L.off_Y = o; o = align256(o + NN * VS);
  L.off_W = o; o = align256(o + Nn * VS);
  L.off_vd = o; o = align256(o + n * VS);
  L.off_beta = o; o = align256(o + n * sizeof(double) * K);
  L.off_rinv = o; o = align256(o + n * VS);
  L.off_r = o; o = align256(o + (size_t)(d + 1) * N * VS);
  L.off_dxw = o; o = align256(o + (size_t)(d + 1) * n * VS);
  L.off_part = o; o = align256(o + (size_t)N * maxchunk * VS);
  if (flags & MD_FLAG_OZAKI) {
    const size_t S = oz_slices_host(K), kp = oz_kpad_host(n), MA = (size_t)n * P * S, NX = (size_t)P * S;
    L.ozaki = 1;
    L.off_As = o; o = align256(o + (size_t)(d + 1) * MA * kp * 2);
    L.off_Xs = o; o = align256(o + (size_t)(d + 1) * NX * kp * 2);
    L.off_eA = o; o = align256(o + sizeof(int) * (size_t)(d + 1) * n);
    L.off_ex = o; o = align256(o + sizeof(int) * (size_t)(d + 1));
    const size_t W = (53 * K + 24 + 128 + 31) / 32 + 1;  // digits per output, as oz_digits
    L.off_acc = o; o = align256(o + sizeof(unsigned long long) * (size_t)n * P * W);
  }
  L.bytes = o - base;
  return L;
}

// --------------------------------------------------------- eval planning
struct Plan {
  int K = 0, P = 0, n = 0, N = 0, d = 0, nmono = 0;
  int nslots = 0;
  std::vector<int> tasks;      // 8 ints per task, stage-major
  std::vector<int> stage_off;  // nstages + 1
  std::vector<int> tasks0;     // coefficient-0 tasks (single jobs), stage-major
  std::vector<int> stage_off0; // nstages + 1
  std::vector<int> scal_src;   // (monomial, exponent factor)
  std::vector<int> groups;     // (row, col or -1, first contribution, count)
  std::vector<int> contrib;    // (slot or -1, scal index, t shift, 0)
  std::vector<int> ops3;          // (out, a, b) per product, stage-major (batched form)
  std::vector<int> op_stage_off;  // nstages + 1 product offsets
  // workspace offsets (bytes)
  size_t off_pool = 0, off_scal = 0, off_tasks = 0, off_scalsrc = 0, off_groups = 0, off_contrib = 0, off_tasks0 = 0;
  size_t off_f = 0, off_A = 0, off_prod = 0, off_solve = 0, total = 0;
  // the split-product form's packed fixed-point copies (pool, coefficients,
  // contribution values), one region; fxpool_bytes = 0 when not laid out
  size_t off_fxpool = 0, off_fxscal = 0, off_fxprod = 0, fxpool_bytes = 0;
  SolveLayout sl{};
  uint64_t checksum = 0;
  // the planned structure itself, compared with the caller's on every cache
  // hit (a 64-bit hash can collide)
  int hdr[6] = {0, 0, 0, 0, 0, 0};
  std::vector<int> s_poly, s_nvar, s_idx, s_expo;
  int oz = 0;  // laid out for the split-product form
};

uint64_t fnv(uint64_t h, const void *p, size_t bytes) {
  const unsigned char *c = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= c[i];
    h *= 1099511628211ULL;
  }
  return h;
}

// Number of polynomials N >= n (neq = 0 means N = n).
int neq_of(const md_system *s) { return s->neq ? s->neq : s->n; }

// Hash of a byte range, eight bytes at a time in four independent
// multiply-xorshift lanes (the FNV prime as multiplier), folded with the
// length: the structure of a large batch is hashed on every call, and byte-wise
// FNV took tenths of a second there.
uint64_t hash_bytes(uint64_t h, const void *p, size_t bytes) {
  const unsigned char *c = static_cast<const unsigned char *>(p);
  const uint64_t prime = 1099511628211ULL;
  uint64_t l[4] = {h, h ^ 0x9e3779b97f4a7c15ULL, h ^ 0xbf58476d1ce4e5b9ULL, h ^ 0x94d049bb133111ebULL};
  size_t i = 0;
  for (; i + 32 <= bytes; i += 32)
    for (int k = 0; k < 4; ++k) {
      uint64_t w;
      std::memcpy(&w, c + i + 8 * k, 8);
      l[k] = (l[k] ^ w) * prime;
      l[k] ^= l[k] >> 29;
    }
  uint64_t r = fnv(l[0], c + i, bytes - i);
  for (int k = 1; k < 4; ++k) {
    r = (r ^ l[k]) * prime;
    r ^= r >> 29;
  }
  return (r ^ (uint64_t)bytes) * prime;
}

// Mask applied to every structure checksum (all ones; tests narrow it with
// md_plan_cache_hash_mask to make different structures collide).
std::atomic<uint64_t> g_hash_mask{~0ULL};

uint64_t structure_checksum(const md_system *s) {
  uint64_t h = 1469598103934665603ULL;
  const int hdr[6] = {s->limbs, s->is_complex, s->n, s->degree, s->nmono, neq_of(s)};
  h = fnv(h, hdr, sizeof(hdr));
  h = hash_bytes(h, s->poly_ptr, sizeof(int) * (neq_of(s) + 1));
  h = hash_bytes(h, s->nvar, sizeof(int) * s->nmono);
  h = hash_bytes(h, s->idx, sizeof(int) * s->nmono * MD_MAXV);
  h = hash_bytes(h, s->expo, sizeof(int) * s->nmono * MD_MAXV);
  return (h & g_hash_mask.load(std::memory_order_relaxed)) | 1;  // never 0 (0 marks "not computed")
}

void structure_header(const md_system *s, int (&hdr)[6]) {
  hdr[0] = s->limbs;
  hdr[1] = s->is_complex;
  hdr[2] = s->n;
  hdr[3] = s->degree;
  hdr[4] = s->nmono;
  hdr[5] = neq_of(s);
}

template <class T>
bool same_ints(const std::vector<int> &v, const T *a, size_t count) {
  return v.size() == count && (count == 0 || std::memcmp(v.data(), a, sizeof(int) * count) == 0);
}

// Is `p` the plan of the structure of `s` (header and every structure array)?
bool same_structure(const Plan &p, const md_system *s) {
  int hdr[6];
  structure_header(s, hdr);
  if (std::memcmp(hdr, p.hdr, sizeof(hdr)) != 0) return false;
  const size_t nm = (size_t)s->nmono;
  return same_ints(p.s_poly, s->poly_ptr, (size_t)neq_of(s) + 1) && same_ints(p.s_nvar, s->nvar, nm) &&
         same_ints(p.s_idx, s->idx, nm * MD_MAXV) && same_ints(p.s_expo, s->expo, nm * MD_MAXV);
}

// Sizes, pointers and polynomial offsets (what the structure hash needs).
md_status check_system_header(const md_system *s) {
  if (!s || !valid_limbs(s->limbs) || s->n < 1 || s->degree < 0 || s->nmono < 0) return MD_ERR_ARG;
  if (s->neq != 0 && s->neq < s->n) return MD_ERR_ARG;
  if (!s->poly_ptr || (s->nmono > 0 && (!s->nvar || !s->idx || !s->expo || !s->coef)) || !s->cst) return MD_ERR_ARG;
  const int N = neq_of(s);
  if (s->poly_ptr[0] != 0 || s->poly_ptr[N] != s->nmono) return MD_ERR_ARG;
  for (int i = 0; i < N; ++i)
    if (s->poly_ptr[i + 1] < s->poly_ptr[i]) return MD_ERR_ARG;
  return MD_OK;
}

md_status check_system(const md_system *s) {
  const md_status st = check_system_header(s);
  if (st != MD_OK) return st;
  for (int m = 0; m < s->nmono; ++m) {
    if (s->nvar[m] < 0 || s->nvar[m] > MD_MAXV) return MD_ERR_ARG;
    for (int q = 0; q < s->nvar[m]; ++q) {
      const int v = s->idx[m * MD_MAXV + q], e = s->expo[m * MD_MAXV + q];
      if (v < 0 || v > s->n || e < 1) return MD_ERR_ARG;
      for (int q2 = 0; q2 < q; ++q2)
        if (s->idx[m * MD_MAXV + q2] == v) return MD_ERR_ARG;
    }
  }
  return MD_OK;
}

// Builds the product schedule of every monomial in the order of the
// definition (common factor, Speelpenning forward / backward / cross products,
// F*P and F*partials), the stage of each product and the accumulation lists.
// Flags that need a square A_0 (N = n).
md_status flags_for_shape(int N, int n, int flags) {
  if (N != n && (flags & MD_FLAG_LU)) return MD_ERR_ARG;
  if (N != n && (flags & MD_FLAG_OZAKI)) return MD_ERR_UNSUPPORTED;
  return MD_OK;
}

md_status build_plan(const md_system *s, Plan &p, int flags = 0) {
  md_status st = check_system(s);
  if (st != MD_OK) return st;
  if ((st = flags_for_shape(neq_of(s), s->n, flags)) != MD_OK) return st;
  const int n = s->n, N = neq_of(s), d = s->degree;
  p.K = s->limbs;
  p.P = s->is_complex ? 2 : 1;
  p.n = n;
  p.N = N;
  p.d = d;
  p.nmono = s->nmono;
  p.nslots = n;
  std::vector<int> stage(n, 0);
  struct Op {
    int out, a, b, st;
  };
  std::vector<Op> ops;
  auto conv = [&](int a, int b) {
    const int out = p.nslots++;
    const int sg = 1 + std::max(stage[a], stage[b]);
    stage.push_back(sg);
    ops.push_back({out, a, b, sg});
    return out;
  };
  // -1 is the unit series
  auto conv_or_copy = [&](int a, int b) {
    if (a < 0) return b;
    if (b < 0) return a;
    return conv(a, b);
  };
  std::vector<int> fcon;  // f contributions, 4 ints each, polynomial-major
  std::vector<int> alist;  // A contributions, 4 ints each
  std::map<std::pair<int, int>, std::vector<int>> acon;  // (row, col) -> indices into alist
  std::vector<int> fgroup_first(N), fgroup_count(N);
  for (int i = 0; i < N; ++i) {
    fgroup_first[i] = (int)fcon.size() / 4;
    fgroup_count[i] = s->poly_ptr[i + 1] - s->poly_ptr[i];
    for (int mo = s->poly_ptr[i]; mo < s->poly_ptr[i + 1]; ++mo) {
      int m = 0, at = 0, vj[MD_MAXV], va[MD_MAXV];
      for (int q = 0; q < s->nvar[mo]; ++q) {
        const int v = s->idx[mo * MD_MAXV + q], e = s->expo[mo * MD_MAXV + q];
        if (v == n) {
          at = e;
        } else {
          vj[m] = v;
          va[m] = e;
          ++m;
        }
      }
      // common factor F = prod x_j^(a_j - 1)
      int F = -1;
      for (int q = 0; q < m; ++q)
        for (int e = 1; e < va[q]; ++e) F = (F < 0) ? vj[q] : conv(F, vj[q]);
      // Speelpenning products
      int pf[MD_MAXV], sb[MD_MAXV];
      int Pser = -1;
      if (m >= 1) {
        pf[0] = vj[0];
        for (int q = 1; q < m; ++q) pf[q] = conv(pf[q - 1], vj[q]);
        sb[m - 1] = vj[m - 1];
        for (int q = m - 2; q >= 1; --q) sb[q] = conv(vj[q], sb[q + 1]);
        Pser = pf[m - 1];
      }
      const int G = conv_or_copy(F, Pser);
      const int sv = (int)p.scal_src.size() / 2;
      p.scal_src.push_back(mo);
      p.scal_src.push_back(1);
      fcon.insert(fcon.end(), {G, sv, at, 0});
      for (int q = 0; q < m; ++q) {
        int der;
        if (m == 1)
          der = -1;
        else if (q == 0)
          der = sb[1];
        else if (q == m - 1)
          der = pf[m - 2];
        else
          der = conv(pf[q - 1], sb[q + 1]);
        const int D = conv_or_copy(F, der);
        const int sq = (int)p.scal_src.size() / 2;
        p.scal_src.push_back(mo);
        p.scal_src.push_back(va[q]);
        acon[{i, vj[q]}].push_back((int)alist.size() / 4);
        alist.insert(alist.end(), {D, sq, at, 0});
      }
    }
  }
  // f groups first, then one group per (row, col) with its contributions in monomial order
  p.contrib = fcon;
  for (int i = 0; i < N; ++i) p.groups.insert(p.groups.end(), {i, -1, fgroup_first[i], fgroup_count[i]});
  for (auto &kv : acon) {
    const int first = (int)p.contrib.size() / 4;
    for (int a : kv.second) p.contrib.insert(p.contrib.end(), alist.begin() + 4 * a, alist.begin() + 4 * a + 4);
    p.groups.insert(p.groups.end(), {kv.first.first, kv.first.second, first, (int)kv.second.size()});
  }
  // stages and tasks
  int nst = 0;
  for (const Op &o : ops) nst = std::max(nst, o.st);
  p.op_stage_off.assign(1, 0);
  for (int sg = 1; sg <= nst; ++sg) {
    for (const Op &o : ops)
      if (o.st == sg) p.ops3.insert(p.ops3.end(), {o.out, o.a, o.b});
    p.op_stage_off.push_back((int)p.ops3.size() / 3);
  }
  p.stage_off0.assign(1, 0);
  for (int sg = 1; sg <= nst; ++sg) {
    for (const Op &o : ops)
      if (o.st == sg) p.tasks0.insert(p.tasks0.end(), {o.out, o.a, o.b, 0, -1, -1, -1, 0});
    p.stage_off0.push_back((int)p.tasks0.size() / 8);
  }
  p.stage_off.assign(1, 0);
  for (int sg = 1; sg <= nst; ++sg) {
    std::vector<int> middles;  // ops whose middle coefficient is left
    for (const Op &o : ops) {
      if (o.st != sg) continue;
      for (int k = 0; 2 * k < d; ++k) p.tasks.insert(p.tasks.end(), {o.out, o.a, o.b, k, o.out, o.a, o.b, 0});
      if (d % 2 == 0) middles.push_back((int)(&o - ops.data()));
    }
    for (size_t q = 0; q < middles.size(); q += 2) {
      const Op &A = ops[middles[q]];
      if (q + 1 < middles.size()) {
        const Op &B = ops[middles[q + 1]];
        p.tasks.insert(p.tasks.end(), {A.out, A.a, A.b, d / 2, B.out, B.a, B.b, 0});
      } else {
        p.tasks.insert(p.tasks.end(), {A.out, A.a, A.b, d / 2, -1, -1, -1, 0});
      }
    }
    p.stage_off.push_back((int)p.tasks.size() / 8);
  }
  // workspace layout
  const size_t VS = sizeof(double) * p.P * p.K;
  size_t o = 256;  // header: status word
  p.off_pool = o; o = align256(o + (size_t)p.nslots * (d + 1) * VS);
  const int nscal = (int)p.scal_src.size() / 2;
  p.off_scal = o; o = align256(o + (size_t)std::max(nscal, 1) * VS);
  p.off_tasks = o; o = align256(o + sizeof(int) * std::max<size_t>(p.tasks.size(), 8));
  p.off_scalsrc = o; o = align256(o + sizeof(int) * std::max<size_t>(p.scal_src.size(), 2));
  p.off_groups = o; o = align256(o + sizeof(int) * std::max<size_t>(p.groups.size(), 4));
  p.off_contrib = o; o = align256(o + sizeof(int) * std::max<size_t>(p.contrib.size(), 4));
  p.off_tasks0 = o; o = align256(o + sizeof(int) * std::max<size_t>(p.tasks0.size(), 8));
  p.off_f = o; o = align256(o + (size_t)N * (d + 1) * VS);
  p.off_A = o; o = align256(o + (size_t)(d + 1) * N * n * VS);
  p.off_prod = o; o = align256(o + (p.contrib.size() / 4) * (size_t)(d + 1) * VS);
  // the split-product form's fixed-point copies (K >= kFxConvMinLimbs)
  p.off_fxpool = o;
  if ((flags & MD_FLAG_OZAKI) && p.K >= mdk::kFxConvMinLimbs) {
    const size_t FV = sizeof(unsigned) * p.P * mdk::fx_packed_words_for(p.K);  // bytes per value
    size_t q = o;
    q = align256(q + (size_t)p.nslots * (d + 1) * FV);
    p.off_fxscal = q;
    q = align256(q + (size_t)std::max(nscal, 1) * FV);
    p.off_fxprod = q;
    q = align256(q + (size_t)std::max<size_t>(p.contrib.size() / 4, 1) * (d + 1) * FV);
    p.fxpool_bytes = q - o;
    o = q;
  }
  p.off_solve = o;
  p.sl = solve_layout(p.K, p.P, N, n, d, o, flags);
  p.total = o + p.sl.bytes;
  p.checksum = structure_checksum(s);
  p.oz = (flags & MD_FLAG_OZAKI) ? 1 : 0;
  structure_header(s, p.hdr);
  p.s_poly.assign(s->poly_ptr, s->poly_ptr + N + 1);
  if (s->nmono > 0) {
    p.s_nvar.assign(s->nvar, s->nvar + s->nmono);
    p.s_idx.assign(s->idx, s->idx + (size_t)s->nmono * MD_MAXV);
    p.s_expo.assign(s->expo, s->expo + (size_t)s->nmono * MD_MAXV);
  }
  return MD_OK;
}

// MD_FLAG_CHECK: every index the kernels follow from the plan's tables, and
// the workspace layout, checked on the host before any launch.  The kernels
// compute all other addresses from (N, n, d, K, P), which the parity tests
// cover shape by shape.
md_status check_plan(const Plan &p) {
  const int ns = p.nslots, n = p.n, N = p.N, d = p.d;
  const int nscal = (int)p.scal_src.size() / 2, ncon = (int)p.contrib.size() / 4;
  auto in = [](long long v, long long lo, long long hi) { return v >= lo && v < hi; };
  // a product's operands are series made before it (slots are numbered in order)
  auto product = [&](int out, int a, int b) { return in(out, n, ns) && in(a, 0, out) && in(b, 0, out); };
  auto stages = [&](const std::vector<int> &off, size_t count) {
    if (off.empty() || off.front() != 0 || (size_t)off.back() != count) return false;
    for (size_t i = 1; i < off.size(); ++i)
      if (off[i] < off[i - 1]) return false;
    return true;
  };
  if (p.tasks.size() % 8 || p.tasks0.size() % 8 || p.ops3.size() % 3 || p.scal_src.size() % 2 ||
      p.groups.size() % 4 || p.contrib.size() % 4)
    return MD_ERR_CHECK;
  if (!stages(p.stage_off, p.tasks.size() / 8) || !stages(p.stage_off0, p.tasks0.size() / 8) ||
      !stages(p.op_stage_off, p.ops3.size() / 3))
    return MD_ERR_CHECK;
  for (size_t t = 0; t < p.tasks.size(); t += 8) {
    const int *q = &p.tasks[t];
    if (!product(q[0], q[1], q[2]) || !in(q[3], 0, d + 1)) return MD_ERR_CHECK;
    if (q[4] >= 0 ? !product(q[4], q[5], q[6]) || 2 * q[3] > d : q[5] != -1 || q[6] != -1) return MD_ERR_CHECK;
  }
  for (size_t t = 0; t < p.tasks0.size(); t += 8)
    if (!product(p.tasks0[t], p.tasks0[t + 1], p.tasks0[t + 2]) || p.tasks0[t + 3] != 0 || p.tasks0[t + 4] != -1)
      return MD_ERR_CHECK;
  for (size_t t = 0; t < p.ops3.size(); t += 3)
    if (!product(p.ops3[t], p.ops3[t + 1], p.ops3[t + 2])) return MD_ERR_CHECK;
  for (int i = 0; i < nscal; ++i)
    if (!in(p.scal_src[2 * i], 0, p.nmono) || p.scal_src[2 * i + 1] < 1) return MD_ERR_CHECK;
  for (size_t g = 0; g < p.groups.size(); g += 4) {
    const int *q = &p.groups[g];
    if (!in(q[0], 0, N) || !in(q[1], -1, n) || q[2] < 0 || q[3] < 0 || (long long)q[2] + q[3] > ncon)
      return MD_ERR_CHECK;
  }
  for (int c = 0; c < ncon; ++c) {
    const int *q = &p.contrib[4 * c];
    if (!in(q[0], -1, ns) || !in(q[1], 0, nscal) || q[2] < 0) return MD_ERR_CHECK;
  }
  // regions in order, each within the next offset, the solve area last
  const size_t VS = sizeof(double) * p.P * p.K;
  const size_t ends[][2] = {
      {p.off_pool, (size_t)ns * (d + 1) * VS},
      {p.off_scal, (size_t)std::max(nscal, 1) * VS},
      {p.off_tasks, sizeof(int) * std::max<size_t>(p.tasks.size(), 8)},
      {p.off_scalsrc, sizeof(int) * std::max<size_t>(p.scal_src.size(), 2)},
      {p.off_groups, sizeof(int) * std::max<size_t>(p.groups.size(), 4)},
      {p.off_contrib, sizeof(int) * std::max<size_t>(p.contrib.size(), 4)},
      {p.off_tasks0, sizeof(int) * std::max<size_t>(p.tasks0.size(), 8)},
      {p.off_f, (size_t)N * (d + 1) * VS},
      {p.off_A, (size_t)(d + 1) * N * n * VS},
      {p.off_prod, (size_t)ncon * (d + 1) * VS},
      {p.off_fxpool, p.fxpool_bytes},
      {p.off_solve, p.sl.bytes}};
  size_t prev_end = 256;  // the status header
  for (const auto &r : ends) {
    if (r[0] < prev_end || r[0] % 256) return MD_ERR_CHECK;
    prev_end = r[0] + r[1];
  }
  if (prev_end > p.total) return MD_ERR_CHECK;
  const SolveLayout &L = p.sl;
  const size_t solve[] = {L.off_M, L.off_Y, L.off_W, L.off_vd, L.off_beta, L.off_rinv, L.off_r, L.off_dxw, L.off_part};
  for (size_t i = 0; i < sizeof(solve) / sizeof(solve[0]); ++i)
    if (solve[i] < (i ? solve[i - 1] + 1 : p.off_solve) || solve[i] >= p.off_solve + L.bytes) return MD_ERR_CHECK;
  return MD_OK;
}

// Plans are cached per system structure (checksum) together with a pinned host
// image of their integer tables; every call copies that image into its
// workspace with one asynchronous copy, so a workspace needs no state between
// calls.  A hit is taken only if the stored structure equals the caller's
// (a colliding structure gets its own plan).  Beyond kPlanCache structures
// the least recently used plans are dropped; a call holds its plan by
// shared_ptr, and a dropped image is freed once the copies enqueued from it
// have run (an event per stream), which is skipped while the calling stream
// is being captured.  A plan used inside a capture is never dropped: the
// caller's graph copies from its image on every replay.
// Events recorded on each stream after a use of a pinned image (one per
// stream), so that dropping the image waits for its own copies only.
struct UseEvents {
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> ev;
  // after an enqueue on s (not during a capture)
  cudaError_t record(cudaStream_t s) {
    for (auto &p : ev)
      if (p.first == s) return cudaEventRecord(p.second, s);
    cudaEvent_t e = nullptr;
    cudaError_t err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (err != cudaSuccess) return err;
    ev.emplace_back(s, e);
    return cudaEventRecord(e, s);
  }
  void wait_and_release() {
    for (auto &p : ev) {
      cudaEventSynchronize(p.second);
      cudaEventDestroy(p.second);
    }
    ev.clear();
  }
};

// MD_FLAG_AUTOTUNE of the single step: how many SMs the factorisation keeps
// while the evaluation's resident CTAs run.  The results do not depend on it
// (the same kernels and task numbering on any grid); the time does, by the
// balance of evaluation and factorisation.  The first call of a plan is not
// timed (it uploads the plan and loads the kernels, and its two streams
// interleave unlike later calls: measured, it could come out shorter than any
// later call at the same count).  The next 2 kN calls each run one candidate
// between two timing events on the caller's stream; a later call reads them
// (without waiting) and keeps the fastest.
struct FactorTune {
  static constexpr int kN = 7;
  static constexpr int kCand[kN] = {4, 8, 12, 16, 24, 32, 48};
  std::mutex mu;
  int best = 0;       // the chosen count, once tuned
  bool warm = false;  // the first (untimed) call has run
  int next = 0;       // measurements started
  int dev = -1;  // the device the events belong to
  float ms[kN];
  bool done[2 * kN] = {};
  cudaEvent_t a[2 * kN] = {}, b[2 * kN] = {};
  FactorTune() {
    for (float &v : ms) v = 1e30f;
  }
  void release() {
    for (int i = 0; i < 2 * kN; ++i) {
      if (a[i]) cudaEventDestroy(a[i]);
      if (b[i]) cudaEventDestroy(b[i]);
      a[i] = b[i] = nullptr;
    }
  }
  ~FactorTune() { release(); }
};

struct PlanEntry {
  Plan plan;
  int *pinned = nullptr;  // tables laid out exactly as in the workspace, from off_tasks
  size_t image_bytes = 0;
  UseEvents uses;
  FactorTune tune;
  // used while a stream was being captured: a caller's graph may copy from
  // the pinned image whenever it is replayed, so the entry is never dropped
  bool captured = false;
  ~PlanEntry() {
    if (pinned) {
      uses.wait_and_release();
      cudaFreeHost(pinned);
    }
  }
};
constexpr size_t kPlanCache = 4096;  // a batch plans one structure per system
std::mutex g_mu;

// A cache of shared values by 64-bit key with least-recently-used order
// (touch and insert in O(log n)); not locked itself.
template <class V>
struct LruCache {
  struct Slot {
    std::shared_ptr<V> v;
    std::list<uint64_t>::iterator pos;
  };
  std::map<uint64_t, Slot> map;
  std::list<uint64_t> order;  // most recently used first

  std::shared_ptr<V> find(uint64_t key) const {
    auto it = map.find(key);
    return it == map.end() ? nullptr : it->second.v;
  }
  void put(uint64_t key, std::shared_ptr<V> v) {
    auto it = map.find(key);
    if (it != map.end()) {
      it->second.v = std::move(v);
    } else {
      order.push_front(key);
      map.emplace(key, Slot{std::move(v), order.begin()});
    }
  }
  void touch(uint64_t key) {
    auto it = map.find(key);
    if (it != map.end()) order.splice(order.begin(), order, it->second.pos);
  }
  // drops the least recently used entries beyond `bound`, except `keep` and
  // those `pinned(v)` says must stay
  template <class Pinned>
  void evict(size_t bound, uint64_t keep, Pinned pinned) {
    for (auto it = order.end(); map.size() > bound && it != order.begin();) {
      --it;
      auto e = map.find(*it);
      if (*it == keep || pinned(*e->second.v)) continue;
      map.erase(e);
      it = order.erase(it);
    }
  }
};

// Never destroyed: entries free pinned memory with CUDA calls, which must not
// run from static destructors after the runtime has unloaded.
LruCache<PlanEntry> &g_plans = *new LruCache<PlanEntry>;

// Under g_mu: mark `key` used, then drop the least recently used plans beyond
// the bound (those with a pinned image only if may_sync; never one used in a
// capture).
void plans_touch(uint64_t key, bool may_sync) {
  g_plans.touch(key);
  g_plans.evict(kPlanCache, key, [&](const PlanEntry &e) { return e.captured || (!may_sync && e.pinned); });
}

// Under g_mu: the cached plan of structure `s` with checksum `cs`, planned
// (and cached under `cs`) if there is none or if the cached one belongs to a
// different structure whose checksum collides with this one's.
md_status plan_cached(const md_system *s, uint64_t cs, int flags, std::shared_ptr<PlanEntry> &hold) {
  hold = g_plans.find(cs);
  if (hold && same_structure(hold->plan, s) && hold->plan.oz == ((flags & MD_FLAG_OZAKI) ? 1 : 0)) return MD_OK;
  md_status st = check_system(s);  // a cached structure passed it when it was planned
  if (st != MD_OK) return st;
  std::shared_ptr<PlanEntry> e = std::make_shared<PlanEntry>();
  if ((st = build_plan(s, e->plan, flags)) != MD_OK) return st;
  if (hold && hold->captured) {  // keep the captured entry alive: hold this one uncached
    hold = e;
    return MD_OK;
  }
  g_plans.put(cs, e);
  hold = e;
  return MD_OK;
}

bool not_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
}

// Plan of `s` (cached), its tables uploaded into ws on `stream`.  `hold`
// keeps the plan alive for the caller; `out` points into it.
md_status prepare(const md_system *s, void *ws, size_t ws_bytes, cudaStream_t stream, Plan *&out,
                  std::shared_ptr<PlanEntry> &hold, int flags = 0) {
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return MD_ERR_WORKSPACE;
  md_status st = check_system_header(s);
  if (st != MD_OK) return st;
  const uint64_t cs = structure_checksum(s) ^ (0x9e3779b97f4a7c15ULL * (uint64_t)(flags & MD_FLAG_OZAKI));
  const bool may_sync = not_capturing(stream);
  std::lock_guard<std::mutex> lk(g_mu);
  if ((st = plan_cached(s, cs, flags, hold)) != MD_OK) return st;
  plans_touch(cs, may_sync);
  PlanEntry *pe = hold.get();
  if ((flags & MD_FLAG_CHECK) && (st = check_plan(pe->plan)) != MD_OK) return st;
  const Plan &p = pe->plan;
  // the cached plan does not depend on MD_FLAG_LU: check the shape every call
  if ((st = flags_for_shape(p.N, p.n, flags)) != MD_OK) return st;
  if (p.total > ws_bytes) return MD_ERR_WORKSPACE;
  if (!pe->pinned) {  // pinned image of the integer tables, created at the first upload
    const size_t bytes = p.off_f - p.off_tasks;
    void *h = nullptr;
    if (cudaHostAlloc(&h, bytes, cudaHostAllocDefault) != cudaSuccess) return MD_ERR_CUDA;
    std::memset(h, 0, bytes);
    auto put = [&](size_t off, const std::vector<int> &v) {
      if (!v.empty()) std::memcpy(static_cast<char *>(h) + (off - p.off_tasks), v.data(), sizeof(int) * v.size());
    };
    put(p.off_tasks, p.tasks);
    put(p.off_scalsrc, p.scal_src);
    put(p.off_groups, p.groups);
    put(p.off_contrib, p.contrib);
    put(p.off_tasks0, p.tasks0);
    pe->image_bytes = bytes;
    pe->pinned = static_cast<int *>(h);
  }
  if (cudaMemcpyAsync(static_cast<char *>(ws) + p.off_tasks, pe->pinned, pe->image_bytes, cudaMemcpyHostToDevice,
                      stream) != cudaSuccess)
    return MD_ERR_CUDA;
  if (!may_sync)
    pe->captured = true;
  else if (pe->uses.record(stream) != cudaSuccess)
    return MD_ERR_CUDA;
  out = &pe->plan;
  return MD_OK;
}


// ------------------------------------------------------------ batched form
// Host plans of single systems, cached by structure checksum (no pinned image).
// A structure already in the cache passed the full check when it was planned:
// only the header is checked again.  `hold` keeps the plan alive.
// cs: the structure checksum if already computed (the header then checked), else 0.
Plan *plan_of(const md_system *s, md_status &st, std::shared_ptr<PlanEntry> &hold, bool may_sync, uint64_t cs = 0) {
  if (!cs) {
    st = check_system_header(s);
    if (st != MD_OK) return nullptr;
    cs = structure_checksum(s);
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if ((st = plan_cached(s, cs, 0, hold)) != MD_OK) return nullptr;
  plans_touch(cs, may_sync);
  return &hold->plan;
}

struct BatchClass {
  int K = 0, P = 0;
  std::vector<int> order;    // job indices, most expensive first
  std::vector<double> cost;  // job_cost of order[q]
  size_t order_off = 0;      // int offset from off_orders
  int cps = 2;               // CTAs per SM (autotuned)
  int threads = 128;         // threads per CTA (autotuned)
  int big_threads = 384;     // threads of the whole-SM CTAs (autotuned)
};

struct BatchPlan {
  int nsys = 0;
  double total_cost = 0;  // sum of job_cost over the batch
  std::vector<mdk::BatchJob> jobs;
  std::vector<BatchClass> classes;
  size_t off_jobs = 0, off_orders = 0, off_ibase = 0, off_dbase = 0, total = 0;
  char *pinned = nullptr;  // [jobs | orders | ibase] as laid out in the workspace from off_jobs
  size_t image_bytes = 0;
  bool tuned = false;
  cudaGraphExec_t exec = nullptr;
  const void *exec_ws = nullptr, *exec_nrm = nullptr, *exec_times = nullptr;
  cudaStream_t exec_stream = nullptr;
  bool exec_split = false;
  int exec_tstride = 2;
  UseEvents uses;         // after each step enqueued on a stream
  bool captured = false;  // enqueued into a caller's capture: never dropped
  int oz = 0;             // laid out for MD_FLAG_OZAKI (a plan of its own per form)
  ~BatchPlan() {
    // a step in flight may still read the pinned image, directly or from the
    // graph: wait for the steps enqueued with this plan, not the device
    uses.wait_and_release();
    if (exec) cudaGraphExecDestroy(exec);
    if (pinned) cudaFreeHost(pinned);
  }
};

// Batch plans, keyed by the structures and the coefficient and x pointers.
// Beyond kBatchPlanCache the least recently used are dropped, so that callers
// who pass new buffers on every call do not accumulate pinned images; a call
// holds its plan by shared_ptr.  Dropping a plan with a pinned image or a
// graph waits for the steps enqueued with it (events), so it is skipped while
// the calling stream is being captured (the cache may then exceed the bound
// for a while); a plan enqueued into a caller's capture is never dropped.
constexpr size_t kBatchPlanCache = 16;
LruCache<BatchPlan> &g_batch = *new LruCache<BatchPlan>;  // never destroyed (as g_plans)

// Under g_mu: mark `key` used and drop the least recently used batch plans
// beyond the bound (those with a pinned image or a graph only if may_sync).
void batch_touch(uint64_t key, bool may_sync) {
  g_batch.touch(key);
  g_batch.evict(kBatchPlanCache, key,
                [&](const BatchPlan &b) { return b.captured || (!may_sync && (b.pinned || b.exec)); });
}

double job_cost(const Plan &p) {
  const double n = p.n, d = p.d, D1 = d + 1;
  const double convs = (double)p.ops3.size() / 3;
  const double macs = convs * D1 * (D1 + 1) / 2 + 2 * n * n * n + n * n * d * D1 / 2 + (double)p.contrib.size() / 4 * D1;
  const double per = p.K * p.K * (p.P == 2 ? 4.0 : 1.0);
  return macs * per;
}

md_status batch_prepare(int nsys, const md_system *sys, double *const *x, std::shared_ptr<BatchPlan> &out,
                        bool need_image, bool may_sync, bool check = false, int oz = 0) {
  if (nsys < 1 || !sys) return MD_ERR_ARG;
  std::vector<Plan *> plans(nsys);
  std::vector<std::shared_ptr<PlanEntry>> holds(nsys);
  // the structures are hashed on every call: on several host threads
  for (int i = 0; i < nsys; ++i)
    if (check_system_header(&sys[i]) != MD_OK) return MD_ERR_ARG;
  std::vector<uint64_t> sums(nsys);
  {
    const int nt = nsys < 64 ? 1 : std::max(1, std::min(8, (int)std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    auto work = [&] {
      for (int i; (i = next.fetch_add(1)) < nsys;) sums[i] = structure_checksum(&sys[i]);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (std::thread &t : pool) t.join();
  }
  uint64_t key = 1469598103934665603ULL;
  for (int i = 0; i < nsys; ++i) {
    md_status st;
    plans[i] = plan_of(&sys[i], st, holds[i], may_sync, sums[i]);
    if (!plans[i]) return st;
    if (check && (st = check_plan(*plans[i])) != MD_OK) return st;
    if (plans[i]->N != plans[i]->n) return MD_ERR_UNSUPPORTED;  // the batched form is for square systems
    const uint64_t cs = plans[i]->checksum;
    key = fnv(key, &cs, sizeof(cs));
    const void *ptrs[3] = {sys[i].coef, sys[i].cst, x ? (const void *)x[i] : nullptr};
    key = fnv(key, ptrs, sizeof(ptrs));
  }
  key = fnv(key, &oz, sizeof(oz));  // each form has its own layout (and tuning and graph)
  {
    std::lock_guard<std::mutex> lk(g_mu);
    std::shared_ptr<BatchPlan> hit = g_batch.find(key);
    if (hit && (!need_image || hit->pinned)) {
      out = hit;
      batch_touch(key, may_sync);
      return MD_OK;
    }
  }
  std::shared_ptr<BatchPlan> bp = std::make_shared<BatchPlan>();
  bp->nsys = nsys;
  bp->oz = oz;
  bp->jobs.resize(nsys);
  // classes by (K, P), jobs ordered by decreasing cost
  std::map<int, int> cls_of;
  for (int i = 0; i < nsys; ++i) {
    const int key2 = plans[i]->K * 4 + plans[i]->P;
    if (!cls_of.count(key2)) {
      cls_of[key2] = (int)bp->classes.size();
      BatchClass c;
      c.K = plans[i]->K;
      c.P = plans[i]->P;
      bp->classes.push_back(c);
    }
    bp->classes[cls_of[key2]].order.push_back(i);
  }
  for (BatchClass &c : bp->classes) {
    std::stable_sort(c.order.begin(), c.order.end(),
                     [&](int a, int b) { return job_cost(*plans[a]) > job_cost(*plans[b]); });
    for (int j : c.order) {
      c.cost.push_back(job_cost(*plans[j]));
      bp->total_cost += c.cost.back();
    }
  }
  // the class holding the most expensive job first (its largest systems start first; only it gets whole-SM CTAs)
  std::stable_sort(bp->classes.begin(), bp->classes.end(), [&](const BatchClass &a, const BatchClass &b) {
    return job_cost(*plans[a.order.front()]) > job_cost(*plans[b.order.front()]);
  });
  // layout
  size_t o = 256;
  bp->off_jobs = o;
  o = align256(o + sizeof(mdk::BatchJob) * nsys);
  bp->off_orders = o;
  size_t oo = 0;
  for (BatchClass &c : bp->classes) {
    c.order_off = oo;
    oo += c.order.size();
  }
  o = align256(o + sizeof(int) * oo);
  bp->off_ibase = o;
  size_t ni = 0, nd = 0;
  auto a4 = [](size_t v) { return (v + 3) & ~(size_t)3; };
  auto a32 = [](size_t v) { return (v + 31) & ~(size_t)31; };
  for (int i = 0; i < nsys; ++i) {
    const Plan &p = *plans[i];
    mdk::BatchJob &J = bp->jobs[i];
    std::memset(&J, 0, sizeof(J));
    const long long VS = (long long)p.P * p.K, n = p.n, D1 = p.d + 1;
    J.n = p.n;
    J.d = p.d;
    J.nstages = (int)p.op_stage_off.size() - 1;
    J.ngroups = (int)p.groups.size() / 4;
    J.nscal = (int)p.scal_src.size() / 2;
    J.nmono = p.nmono;
    J.nops = (int)p.ops3.size() / 3;
    ni = a4(ni);
    J.ops = ni; ni += p.ops3.size();
    J.stage_off = ni; ni += p.op_stage_off.size();
    J.scal_src = ni; ni += p.scal_src.size();
    ni = a4(ni);
    J.groups = ni; ni += p.groups.size();
    ni = a4(ni);
    J.contrib = ni; ni += p.contrib.size();
    nd = a32(nd);
    J.pool = nd; nd += (size_t)p.nslots * D1 * VS;
    J.scal = nd; nd += (size_t)std::max(J.nscal, 1) * VS;
    J.f = nd; nd += (size_t)n * D1 * VS;
    J.A = nd; nd += (size_t)D1 * n * n * VS;
    J.M = nd; nd += (size_t)n * n * VS;
    J.Y = nd; nd += (size_t)n * n * VS;
    J.W = nd; nd += (size_t)n * n * VS;
    J.vd = nd; nd += (size_t)n * VS;
    J.beta = nd; nd += (size_t)n * p.K;
    J.rinv = nd; nd += (size_t)n * VS;
    J.r = nd; nd += (size_t)D1 * n * VS;
    J.dxw = nd; nd += (size_t)D1 * n * VS;
    J.part = nd; nd += (size_t)n * p.sl.maxchunk * VS;
    if (oz && p.K >= mdk::kFxConvMinLimbs) {  // packed fixed-point copies, in doubles (PW is a multiple of 4)
      const size_t FV = (size_t)p.P * mdk::fx_packed_words_for(p.K) / 2;
      nd = a32(nd);
      J.fxpool = nd; nd += (size_t)p.nslots * D1 * FV;
      J.fxA = nd; nd += (size_t)D1 * n * n * FV;
      J.fxdx = nd; nd += (size_t)D1 * n * FV;
      J.fxscal = nd; nd += (size_t)std::max(J.nscal, 1) * FV;
    }
    J.coef = sys[i].coef;
    J.cst = sys[i].cst;
    J.x = x ? x[i] : nullptr;
  }
  o = align256(o + sizeof(int) * ni);
  bp->off_dbase = o;
  bp->total = o + sizeof(double) * nd;
  if (need_image) {
    bp->image_bytes = bp->off_dbase - bp->off_jobs;
    void *h = nullptr;
    if (cudaHostAlloc(&h, bp->image_bytes, cudaHostAllocDefault) != cudaSuccess) return MD_ERR_CUDA;
    std::memset(h, 0, bp->image_bytes);
    bp->pinned = static_cast<char *>(h);
    std::memcpy(bp->pinned, bp->jobs.data(), sizeof(mdk::BatchJob) * nsys);
    int *ord = reinterpret_cast<int *>(bp->pinned + (bp->off_orders - bp->off_jobs));
    for (const BatchClass &c : bp->classes)
      for (size_t q = 0; q < c.order.size(); ++q) ord[c.order_off + q] = c.order[q];
    int *ib = reinterpret_cast<int *>(bp->pinned + (bp->off_ibase - bp->off_jobs));
    for (int i = 0; i < nsys; ++i) {
      const Plan &p = *plans[i];
      const mdk::BatchJob &J = bp->jobs[i];
      std::copy(p.ops3.begin(), p.ops3.end(), ib + J.ops);
      std::copy(p.op_stage_off.begin(), p.op_stage_off.end(), ib + J.stage_off);
      std::copy(p.scal_src.begin(), p.scal_src.end(), ib + J.scal_src);
      std::copy(p.groups.begin(), p.groups.end(), ib + J.groups);
      std::copy(p.contrib.begin(), p.contrib.end(), ib + J.contrib);
    }
  }
  std::lock_guard<std::mutex> lk(g_mu);
  std::shared_ptr<BatchPlan> old = g_batch.find(key);
  if (!old || (!old->pinned && bp->pinned)) {
    g_batch.put(key, bp);  // new, or replaces a size-only plan
    out = bp;
  } else {
    out = old;
  }
  batch_touch(key, may_sync);
  return MD_OK;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 152;
  return sms > 0 ? sms : 152;
}

// Largest dynamic shared memory one CTA may opt into (0 if unknown).
int device_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return v;
}

// Job counters of the batched launches: ints at base + 64 (cleared with the
// status word by the 256-byte memset of every step).  Class ci's shared-SM
// launch counts at [ci] (at most 20 classes), the whole-SM launch at
// [kBigCounter]; its CTAs count themselves in at [kResidentCounter].
constexpr int kBigCounter = 24, kResidentCounter = 25;
static_assert(MD_PHASE_STAMPS == mdk::kPhaseStamps, "phase stamps of the ABI and the kernel differ");

// Launch of class c over its jobs order[first, first + count): `grid` CTAs
// of `threads`, at most `cps` of them on one SM.
mdk::BatchDev batch_dev(const BatchPlan &bp, const BatchClass &c, int ctr, int first, int count, char *base,
                        double *nrm, unsigned long long *times, int update_x, int grid, int threads, int cps) {
  mdk::BatchDev b;
  b.jobs = reinterpret_cast<const mdk::BatchJob *>(base + bp.off_jobs);
  b.order = reinterpret_cast<const int *>(base + bp.off_orders) + c.order_off + first;
  b.njobs = count;
  b.counter = reinterpret_cast<int *>(base + 64) + ctr;
  b.ibase = reinterpret_cast<const int *>(base + bp.off_ibase);
  b.dbase = reinterpret_cast<double *>(base + bp.off_dbase);
  b.nrm = nrm;
  b.times = times;
  b.status = reinterpret_cast<int *>(base);
  b.update_x = update_x;
  b.grid = grid;
  b.threads = threads;
  b.ctas_per_sm = cps;
  b.split = bp.oz;
  return b;
}

// Systems of the first class (the one holding the most expensive system)
// that get a whole SM each: the leading ones whose step on a shared SM
// (cps CTAs) would take longer than an even share of the whole batch over
// the SMs, cps * cost > total / sms.  At most sms - 1, so that one SM stays
// for the gate and the shared CTAs; none when the class runs one CTA per SM
// anyway.
int big_jobs(const BatchPlan &bp, int sms) {
  const BatchClass &c = bp.classes[0];
  if (c.cps <= 1) return 0;
  const double share = bp.total_cost / sms;
  int nb = 0;
  while (nb < (int)c.order.size() && nb < sms - 1 && c.cps * c.cost[nb] > share) ++nb;
  return nb;
}

// Holds back the launches after it on its stream until `target` CTAs have
// counted themselves in at `resident`, so that the whole-SM CTAs are placed
// before CTAs that share SMs take the rest.  It only orders placement (no
// result depends on it) and gives up after about a tenth of a second; giving
// up sets ST_TIMEOUT in the status word (md_get_device_status then reports
// MD_ERR_TIMEOUT: the results stand, the placement was not enforced).
__global__ void batch_gate_kernel(const int *resident, int target, int *status) {
  if (threadIdx.x != 0) return;
  for (int it = 0; it < 100000; ++it) {
    if (*reinterpret_cast<const volatile int *>(resident) >= target) return;
    __nanosleep(1000);
  }
  atomicOr(status, mdk::ST_TIMEOUT);
}

struct DevAux;
DevAux *aux_for_current_device();
std::mutex *aux_mutex(DevAux *a);
cudaStream_t aux_stream(DevAux *a);
cudaEvent_t aux_event(DevAux *a, int i);

// One step of the batch.  Every class runs in turn, in launches of
// sms x cps CTAs with at most cps of them on one SM.  With `split` and
// whole-SM systems in the first class (big_jobs), those run on the caller's
// stream in CTAs that each hold a whole SM, and on the library's second
// stream a gate waits until those CTAs are placed before the shared-SM
// launches take the other SMs (and each SM a whole-SM CTA leaves).
cudaError_t batch_enqueue(const BatchPlan &bp, char *base, double *nrm, unsigned long long *times, cudaStream_t s,
                          int sms, bool split, int tstride) {
  cudaError_t e = cudaMemcpyAsync(base + bp.off_jobs, bp.pinned, bp.image_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(base, 0, 256, s)) != cudaSuccess) return e;
  const int nbig = split ? big_jobs(bp, sms) : 0;
  DevAux *ax = nbig > 0 ? aux_for_current_device() : nullptr;
  if (!ax) {
    for (size_t ci = 0; ci < bp.classes.size(); ++ci) {
      const BatchClass &c = bp.classes[ci];
      mdk::BatchDev b =
          batch_dev(bp, c, (int)ci, 0, (int)c.order.size(), base, nrm, times, 1, sms * c.cps, c.threads, c.cps);
      b.times_stride = tstride;
      if ((e = dispatch(c.K, c.P, 4, &b, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  std::lock_guard<std::mutex> lk(*aux_mutex(ax));
  cudaStream_t s2 = aux_stream(ax);
  if ((e = cudaEventRecord(aux_event(ax, 0), s)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(s2, aux_event(ax, 0), 0)) != cudaSuccess)
    return e;
  {
    const BatchClass &c = bp.classes[0];
    int *ctr = reinterpret_cast<int *>(base + 64);
    mdk::BatchDev b = batch_dev(bp, c, kBigCounter, 0, nbig, base, nrm, times, 1, nbig, c.big_threads, 1);
    b.resident = ctr + kResidentCounter;
    b.times_stride = tstride;
    if ((e = dispatch(c.K, c.P, 4, &b, s)) != cudaSuccess) return e;
    batch_gate_kernel<<<1, 32, 0, s2>>>(ctr + kResidentCounter, nbig, reinterpret_cast<int *>(base));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (size_t ci = 0; ci < bp.classes.size(); ++ci) {
    const BatchClass &c = bp.classes[ci];
    const int first = ci == 0 ? nbig : 0;
    mdk::BatchDev b = batch_dev(bp, c, (int)ci, first, (int)c.order.size() - first, base, nrm, times, 1, sms * c.cps,
                                c.threads, c.cps);
    b.times_stride = tstride;
    if ((e = dispatch(c.K, c.P, 4, &b, s2)) != cudaSuccess) return e;
  }
  if ((e = cudaEventRecord(aux_event(ax, 1), s2)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(s, aux_event(ax, 1), 0);
}

// Per precision class, picks the shape (threads per CTA, CTAs per SM) by
// timing trial steps that do not update x on the same first 4 x SMs of the
// class's jobs (the most expensive ones) for every shape, then, if whole-SM
// systems result, their threads by timing one launch over those.  Only
// shapes whose registers fit on an SM are tried.  Shapes are tried from the
// fewest CTAs per SM (the shortest time per system, hence the shortest
// tail); one with more CTAs per SM must be 3% faster per system to be taken.
md_status batch_autotune(BatchPlan &bp, char *base, cudaStream_t s, int sms, bool split) {
  struct Events {  // destroyed on every return
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) return MD_ERR_CUDA;
  cudaEvent_t a = ev.a, b = ev.b;
  if (cudaMemcpyAsync(base + bp.off_jobs, bp.pinned, bp.image_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MD_ERR_CUDA;
  auto trial = [&](const BatchClass &c, mdk::BatchDev &d, float &ms) -> md_status {
    ms = -1.f;
    if (cudaMemsetAsync(base, 0, 256, s) != cudaSuccess) return MD_ERR_CUDA;
    cudaEventRecord(a, s);
    if (dispatch(c.K, c.P, 4, &d, s) != cudaSuccess) {  // shape does not fit: skip it
      cudaGetLastError();
      return MD_OK;
    }
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) return MD_ERR_CUDA;
    cudaEventElapsedTime(&ms, a, b);
    return MD_OK;
  };
  const int shapes[][2] = {{384, 1}, {256, 1}, {128, 1}, {128, 2}, {128, 3}};
  for (size_t ci = 0; ci < bp.classes.size(); ++ci) {
    BatchClass &c = bp.classes[ci];
    const int first = 0;
    const int avail = (int)c.order.size();
    float best = 1e30f;
    int best_t = c.threads, best_cps = c.cps;
    for (const auto &sh : shapes) {
      if (avail <= 0) break;
      c.threads = sh[0];
      c.cps = sh[1];
      mdk::BatchDev d = batch_dev(bp, c, (int)ci, first, std::min(avail, 4 * sms), base, nullptr, nullptr, 0,
                                  sms * c.cps, c.threads, c.cps);
      float ms;
      if (trial(c, d, ms) != MD_OK) return MD_ERR_CUDA;
      if (ms < 0.f) continue;
      const float per_job = ms / (float)std::max(1, d.njobs);
      if (per_job < (c.cps > best_cps ? 0.97f : 1.0f) * best) {
        best = per_job;
        best_t = c.threads;
        best_cps = c.cps;
      }
    }
    c.threads = best_t;
    c.cps = best_cps;
  }
  const int nbig2 = split ? big_jobs(bp, sms) : 0;
  if (nbig2 > 0) {
    BatchClass &c = bp.classes[0];
    float best = 1e30f;
    int best_t = c.big_threads;
    for (int t : {256, 384}) {
      c.big_threads = t;
      mdk::BatchDev d = batch_dev(bp, c, kBigCounter, 0, nbig2, base, nullptr, nullptr, 0, nbig2, t, 1);
      float ms;
      if (trial(c, d, ms) != MD_OK) return MD_ERR_CUDA;
      if (ms >= 0.f && ms < best) {
        best = ms;
        best_t = t;
      }
    }
    c.big_threads = best_t;
  }
  bp.tuned = true;
  bp.exec_ws = nullptr;  // configuration changed: recapture any graph
  return MD_OK;
}

EvalDev make_eval(const Plan &p, const md_system *s, const double *x, double *f, double *A, char *base) {
  EvalDev e;
  e.n = p.n;
  e.N = p.N;
  e.d = p.d;
  e.nmono = p.nmono;
  e.x = x;
  e.f = f;
  e.A = A;
  e.coef = s->coef;
  e.cst = s->cst;
  e.pool = reinterpret_cast<double *>(base + p.off_pool);
  e.scal = reinterpret_cast<double *>(base + p.off_scal);
  e.tasks = reinterpret_cast<const int *>(base + p.off_tasks);
  e.stage_off = p.stage_off.data();
  e.nstages = (int)p.stage_off.size() - 1;
  e.scal_src = reinterpret_cast<const int *>(base + p.off_scalsrc);
  e.nscal = (int)p.scal_src.size() / 2;
  e.groups = reinterpret_cast<const int *>(base + p.off_groups);
  e.ngroups = (int)p.groups.size() / 4;
  e.contrib = reinterpret_cast<const int *>(base + p.off_contrib);
  e.ncontrib = (int)p.contrib.size() / 4;
  e.prod = reinterpret_cast<double *>(base + p.off_prod);
  e.tasks0 = reinterpret_cast<const int *>(base + p.off_tasks0);
  e.stage_off0 = p.stage_off0.data();
  if (p.fxpool_bytes) {
    e.fxpool = reinterpret_cast<unsigned *>(base + p.off_fxpool);
    e.fxscal = reinterpret_cast<unsigned *>(base + p.off_fxscal);
    e.fxprod = reinterpret_cast<unsigned *>(base + p.off_fxprod);
  }
  return e;
}

SolveDev make_solve(const SolveLayout &L, int N, int n, int d, char *base) {
  SolveDev v;
  v.N = N;
  v.n = n;
  v.d = d;
  v.M = reinterpret_cast<double *>(base + L.off_M);
  v.Y = reinterpret_cast<double *>(base + L.off_Y);
  v.W = reinterpret_cast<double *>(base + L.off_W);
  v.vd = reinterpret_cast<double *>(base + L.off_vd);
  v.beta = reinterpret_cast<double *>(base + L.off_beta);
  v.rinv = reinterpret_cast<double *>(base + L.off_rinv);
  v.r = reinterpret_cast<double *>(base + L.off_r);
  v.dxw = reinterpret_cast<double *>(base + L.off_dxw);
  v.part = reinterpret_cast<double *>(base + L.off_part);
  v.status = reinterpret_cast<int *>(base);
  v.maxchunk = L.maxchunk;
  if (L.ozaki) {
    v.ozaki = 1;
    v.oz_As = base + L.off_As;
    v.oz_Xs = base + L.off_Xs;
    v.oz_eA = reinterpret_cast<int *>(base + L.off_eA);
    v.oz_ex = reinterpret_cast<int *>(base + L.off_ex);
    v.oz_acc = reinterpret_cast<unsigned long long *>(base + L.off_acc);
  }
  return v;
}

md_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MD_OK : MD_ERR_CUDA; }

// Per-device second stream (highest priority) and events for running the
// factorisation of A_0 alongside the evaluation of the higher coefficients.
struct DevAux {
  std::mutex mu;
  cudaStream_t s2 = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};
DevAux g_aux[64];

DevAux *aux_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  DevAux &a = g_aux[dev];
  std::lock_guard<std::mutex> lk(a.mu);
  if (!a.s2) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&a.s2, cudaStreamNonBlocking, hi) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&a.e0, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&a.e1, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  }
  return &a;
}

std::mutex *aux_mutex(DevAux *a) { return &a->mu; }
cudaStream_t aux_stream(DevAux *a) { return a->s2; }
cudaEvent_t aux_event(DevAux *a, int i) { return i == 0 ? a->e0 : a->e1; }

// SMs left to the factorisation while the evaluation runs resident.  With
// the factorisation in fixed point (about 15 ms of QR and W at quad double
// n = 64 on six SMs, against 45 ms of evaluation) four suffice: measured
// 15.81 (6), 16.04 (4) and 16.04 (3) steps/s at n = 64, d = 64, and
// 21.03 / 20.88 / 20.79 steps/s at octo double n = 128, whose step waits on
// the factorisation.
#ifndef MDK_FACTOR_SMS
#define MDK_FACTOR_SMS 4
#endif
constexpr int kFactorSms = MDK_FACTOR_SMS;
// Other balances want more (measured: the split-product form at n = 64,
// d = 64, whose fixed-point products now take less time than the
// factorisation on four SMs, 19.2 ms with 4 and 15.1 with 16; the octo double
// n = 128 plain step 41.8 ms with 4 and 35.1 with 48): MD_FLAG_AUTOTUNE picks
// the count per plan (FactorTune).

// The count for this call of the step, and the timing events to record
// around it (null: untimed).  Under MD_FLAG_AUTOTUNE, outside a capture.
md_status factor_sms_for(FactorTune &t, int flags, cudaStream_t s, int &fsms, cudaEvent_t &ta, cudaEvent_t &tb) {
  fsms = kFactorSms;
  ta = tb = nullptr;
  if (!(flags & MD_FLAG_AUTOTUNE) || !not_capturing(s)) return MD_OK;
  std::lock_guard<std::mutex> lk(t.mu);
  if (t.best) {
    fsms = t.best;
    return MD_OK;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MD_ERR_CUDA;
  if (t.dev >= 0 && t.dev != dev) return MD_OK;  // tuning on another device: the default here
  t.dev = dev;
  if (!t.warm) {  // the plan's first call: untimed
    t.warm = true;
    return MD_OK;
  }
  constexpr int kM = 2 * FactorTune::kN;
  if (t.next < kM) {
    const int i = t.next;
    if ((!t.a[i] && cudaEventCreate(&t.a[i]) != cudaSuccess) || (!t.b[i] && cudaEventCreate(&t.b[i]) != cudaSuccess))
      return MD_ERR_CUDA;
    t.next++;
    fsms = FactorTune::kCand[i % FactorTune::kN];
    ta = t.a[i];
    tb = t.b[i];
    return MD_OK;
  }
  bool all = true;
  for (int i = 0; i < kM; ++i) {
    if (t.done[i]) continue;
    const cudaError_t q = cudaEventQuery(t.b[i]);
    if (q == cudaErrorNotReady) {
      all = false;
      continue;
    }
    float ms = 0.f;
    if (q != cudaSuccess || cudaEventElapsedTime(&ms, t.a[i], t.b[i]) != cudaSuccess) return MD_ERR_CUDA;
    t.ms[i % FactorTune::kN] = std::min(t.ms[i % FactorTune::kN], ms);
    t.done[i] = true;
  }
  if (!all) return MD_OK;
  int bi = 0;
  for (int c = 1; c < FactorTune::kN; ++c)
    if (t.ms[c] < t.ms[bi]) bi = c;
  t.best = FactorTune::kCand[bi];
  t.release();
  fsms = t.best;
  return MD_OK;
}

// ------------------------------------------------------------- profiling
// Optional per-launch timing: when enabled, every launch is bracketed by a
// pair of CUDA events recorded on its stream; md_profile_read sums the
// elapsed times per kernel class.
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_free;

cudaEvent_t prof_event() {
  if (!g_prof_free.empty()) {
    cudaEvent_t e = g_prof_free.back();
    g_prof_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

namespace mdk {
bool prof_enabled() { return g_prof_on.load(std::memory_order_relaxed); }
int prof_begin(int kind, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r{kind, prof_event(), prof_event()};
  cudaEventRecord(r.a, s);
  g_prof_recs.push_back(r);
  return (int)g_prof_recs.size() - 1;
}
void prof_end(int id, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (id >= 0 && id < (int)g_prof_recs.size()) cudaEventRecord(g_prof_recs[id].b, s);
}
}  // namespace mdk

namespace {
const char *kProfNames[mdk::PK_COUNT] = {"pool_load_x", "prep_scal", "conv_stage", "accum", "qr_house", "qr_apply",
                                         "rinv", "backsub", "rhs_partial", "rhs_finish", "wmv", "finish_dx",
                                         "elementwise", "series_conv", "oz_split", "oz_update", "lu"};

md_status check_schedule(const md_system *s, const md_newton_schedule *sc) {
  if (!sc || sc->nlevels < 1 || sc->nlevels > MD_MAX_LEVELS) return MD_ERR_ARG;
  if (!(sc->tol >= 0.0) || !(sc->too_large >= 0.0)) return MD_ERR_ARG;  // also rejects NaN
  for (int l = 0; l < sc->nlevels; ++l) {
    if (sc->degree[l] < 0 || sc->degree[l] > s->degree || sc->max_iter[l] < 1) return MD_ERR_ARG;
    if (l > 0 && sc->degree[l] < sc->degree[l - 1]) return MD_ERR_ARG;
  }
  return MD_OK;
}

md_system at_degree(const md_system *s, int d) {
  md_system t = *s;
  t.degree = d;
  return t;
}

// Workspace of the driver: [step workspace of the largest level | x at that
// level's degree | dx norms].
struct RunLayout {
  size_t step = 0, off_x = 0, off_nrm = 0, total = 0;
};

RunLayout run_layout(const md_system *s, const md_newton_schedule *sc, int flags) {
  RunLayout L;
  int dmax = 0;
  for (int l = 0; l < sc->nlevels; ++l) {
    md_system t = at_degree(s, sc->degree[l]);
    Plan p;
    if (build_plan(&t, p, flags) != MD_OK) return RunLayout{};
    L.step = std::max(L.step, p.total);
    dmax = std::max(dmax, sc->degree[l]);
  }
  const size_t P = s->is_complex ? 2 : 1;
  L.off_x = align256(L.step);
  L.off_nrm = align256(L.off_x + sizeof(double) * P * s->limbs * (size_t)s->n * (dmax + 1));
  L.total = L.off_nrm + 256;
  return L;
}

}  // namespace

extern "C" {

int md_version(void) { return 101; }

const char *md_status_string(md_status st) {
  switch (st) {
    case MD_OK: return "ok";
    case MD_ERR_ARG: return "invalid argument";
    case MD_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case MD_ERR_CUDA: return "CUDA error";
    case MD_ERR_SINGULAR: return "A_0 is singular";
    case MD_ERR_NONFINITE: return "non-finite update";
    case MD_ERR_NOCONV: return "no convergence";
    case MD_ERR_TIMEOUT: return "device wait timed out";
    case MD_ERR_UNSUPPORTED: return "unsupported";
    case MD_ERR_CHECK: return "bounds check failed";
  }
  return "unknown status";
}

md_status md_plan_check(const md_system *sys, int flags) {
  Plan p;
  const md_status st = build_plan(sys, p, flags);
  return st != MD_OK ? st : check_plan(p);
}

size_t md_workspace_bytes(const md_system *sys, int flags) {
  Plan p;
  if (build_plan(sys, p, flags) != MD_OK) return 0;
  return p.total;
}

size_t md_lstsq_workspace_bytes(int limbs, int is_complex, int neq, int n, int degree, int flags) {
  if (!valid_limbs(limbs) || n < 1 || neq < n || degree < 0 || flags_for_shape(neq, n, flags) != MD_OK) return 0;
  return 256 + solve_layout(limbs, is_complex ? 2 : 1, neq, n, degree, 256, flags).bytes;
}

size_t md_linsolve_workspace_bytes(int limbs, int is_complex, int n, int degree, int flags) {
  return md_lstsq_workspace_bytes(limbs, is_complex, n, n, degree, flags);
}

md_status md_elementwise(int op, int limbs, int is_complex, long long count, const double *x, const double *y,
                         double *z, void *stream) {
  if (!valid_limbs(limbs) || op < 0 || op > 5 || count < 0 || (op == 4 && is_complex)) return MD_ERR_ARG;
  if (count > 0 && (!x || !z || (op != 4 && !y))) return MD_ERR_ARG;
  return cuda_status(dispatch(limbs, is_complex ? 2 : 1, 0, nullptr, static_cast<cudaStream_t>(stream), op, count, 0,
                              x, y, z));
}

md_status md_series_conv(int limbs, int is_complex, int degree, long long count, const double *x, const double *y,
                         double *z, void *stream) {
  if (!valid_limbs(limbs) || degree < 0 || count < 0) return MD_ERR_ARG;
  if (count > 0 && (!x || !y || !z)) return MD_ERR_ARG;
  return cuda_status(dispatch(limbs, is_complex ? 2 : 1, 1, nullptr, static_cast<cudaStream_t>(stream), 0, count,
                              degree, x, y, z));
}

md_status md_eval_diff(const md_system *sys, const double *x, double *f, double *A, void *ws, size_t ws_bytes,
                       void *stream) {
  if (!x || !f || !A) return MD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Plan *p = nullptr;
  std::shared_ptr<PlanEntry> hold;
  md_status st = prepare(sys, ws, ws_bytes, s, p, hold);
  if (st != MD_OK) return st;
  char *base = static_cast<char *>(ws);
  if (cudaMemsetAsync(base, 0, 256, s) != cudaSuccess) return MD_ERR_CUDA;
  EvalDev e = make_eval(*p, sys, x, f, A, base);
  return cuda_status(dispatch(p->K, p->P, 2, &e, s));
}

md_status md_lstsq_series(int limbs, int is_complex, int neq, int n, int degree, const double *A, const double *b,
                           double *dx, void *ws, size_t ws_bytes, int flags, void *stream) {
  if (!valid_limbs(limbs) || n < 1 || neq < n || degree < 0 || !A || !b || !dx) return MD_ERR_ARG;
  md_status st = flags_for_shape(neq, n, flags);
  if (st != MD_OK) return st;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return MD_ERR_WORKSPACE;
  const int P = is_complex ? 2 : 1;
  SolveLayout L = solve_layout(limbs, P, neq, n, degree, 256, flags);
  if (256 + L.bytes > ws_bytes) return MD_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char *base = static_cast<char *>(ws);
  if (cudaMemsetAsync(base, 0, 256, s) != cudaSuccess) return MD_ERR_CUDA;
  SolveDev v = make_solve(L, neq, n, degree, base);
  v.A = A;
  v.b = b;
  v.sgn = 1.0;
  v.dx_out = dx;
  v.lu = (flags & MD_FLAG_LU) ? 1 : 0;
  return cuda_status(dispatch(limbs, P, 3, &v, s));
}

md_status md_linsolve_series(int limbs, int is_complex, int n, int degree, const double *A, const double *b,
                             double *dx, void *ws, size_t ws_bytes, int flags, void *stream) {
  return md_lstsq_series(limbs, is_complex, n, n, degree, A, b, dx, ws, ws_bytes, flags, stream);
}

md_status md_newton_series_step(const md_system *sys, double *x, double *dx_norm, void *ws, size_t ws_bytes, int flags,
                                void *stream) {
  if (!x) return MD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Plan *p = nullptr;
  std::shared_ptr<PlanEntry> hold;
  md_status st = prepare(sys, ws, ws_bytes, s, p, hold, flags);
  if (st != MD_OK) return st;
  char *base = static_cast<char *>(ws);
  if (cudaMemsetAsync(base, 0, 256, s) != cudaSuccess) return MD_ERR_CUDA;
  if (dx_norm && cudaMemsetAsync(dx_norm, 0, 2 * sizeof(double), s) != cudaSuccess) return MD_ERR_CUDA;
  double *f = reinterpret_cast<double *>(base + p->off_f);
  double *A = reinterpret_cast<double *>(base + p->off_A);
  EvalDev e = make_eval(*p, sys, x, f, A, base);
  // series products as split products too (from kFxConvMinLimbs limbs on,
  // where the plan holds the fixed-point pool)
  e.split = ((flags & MD_FLAG_OZAKI) && e.fxpool) ? 1 : 0;
  SolveDev v = make_solve(p->sl, p->N, p->n, p->d, base);
  v.A = A;
  v.b = f;
  v.sgn = -1.0;
  v.x = x;
  v.nrm = dx_norm;
  v.lu = (flags & MD_FLAG_LU) ? 1 : 0;
  DevAux *ax = (flags & MD_FLAG_SERIAL) ? nullptr : aux_for_current_device();
  if (!ax) {
    if (dispatch(p->K, p->P, 2, &e, s) != cudaSuccess) return MD_ERR_CUDA;
    return cuda_status(dispatch(p->K, p->P, 3, &v, s));
  }
  // evaluation prologue and coefficient 0 (gives A_0) -> factorisation on the
  // second stream, concurrently with the remaining products on SMs - fsms
  // resident CTAs -> degree loop once both are done
  int fsms = kFactorSms;
  cudaEvent_t ta = nullptr, tb = nullptr;
  if ((st = factor_sms_for(hold->tune, flags, s, fsms, ta, tb)) != MD_OK) return st;
  e.resident_ctas = std::max(1, device_sms() - fsms);
  e.resident_smem = device_smem_optin();
  std::lock_guard<std::mutex> lk(ax->mu);
  if (ta && cudaEventRecord(ta, s) != cudaSuccess) return MD_ERR_CUDA;
  if (dispatch(p->K, p->P, 5, &e, s) != cudaSuccess) return MD_ERR_CUDA;
  if (cudaEventRecord(ax->e0, s) != cudaSuccess || cudaStreamWaitEvent(ax->s2, ax->e0, 0) != cudaSuccess)
    return MD_ERR_CUDA;
  if (dispatch(p->K, p->P, 7, &v, ax->s2) != cudaSuccess) return MD_ERR_CUDA;
  if (cudaEventRecord(ax->e1, ax->s2) != cudaSuccess) return MD_ERR_CUDA;
  if (dispatch(p->K, p->P, 6, &e, s) != cudaSuccess) return MD_ERR_CUDA;
  if (cudaStreamWaitEvent(s, ax->e1, 0) != cudaSuccess) return MD_ERR_CUDA;
  if (dispatch(p->K, p->P, 8, &v, s) != cudaSuccess) return MD_ERR_CUDA;
  return cuda_status(tb ? cudaEventRecord(tb, s) : cudaSuccess);
}

md_status md_rcond_a0(const md_system *sys, void *ws, size_t ws_bytes, int flags, double *rcond, void *stream) {
  if (!rcond) return MD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Plan *p = nullptr;
  std::shared_ptr<PlanEntry> hold;
  md_status st = prepare(sys, ws, ws_bytes, s, p, hold, flags);
  if (st != MD_OK) return st;
  char *base = static_cast<char *>(ws);
  SolveDev v = make_solve(p->sl, p->N, p->n, p->d, base);
  v.A = reinterpret_cast<const double *>(base + p->off_A);
  v.rcond = rcond;
  return cuda_status(dispatch(p->K, p->P, 9, &v, s));
}

md_status md_lstsq_rcond(int limbs, int is_complex, int neq, int n, int degree, const double *A, void *ws,
                          size_t ws_bytes, int flags, double *rcond, void *stream) {
  if (!valid_limbs(limbs) || n < 1 || neq < n || degree < 0 || !A || !rcond) return MD_ERR_ARG;
  md_status st = flags_for_shape(neq, n, flags);
  if (st != MD_OK) return st;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return MD_ERR_WORKSPACE;
  const int P = is_complex ? 2 : 1;
  SolveLayout L = solve_layout(limbs, P, neq, n, degree, 256, flags);
  if (256 + L.bytes > ws_bytes) return MD_ERR_WORKSPACE;
  SolveDev v = make_solve(L, neq, n, degree, static_cast<char *>(ws));
  v.A = A;
  v.rcond = rcond;
  return cuda_status(dispatch(limbs, P, 9, &v, static_cast<cudaStream_t>(stream)));
}

md_status md_linsolve_rcond(int limbs, int is_complex, int n, int degree, const double *A, void *ws,
                            size_t ws_bytes, int flags, double *rcond, void *stream) {
  return md_lstsq_rcond(limbs, is_complex, n, n, degree, A, ws, ws_bytes, flags, rcond, stream);
}

size_t md_newton_run_workspace_bytes(const md_system *sys, const md_newton_schedule *sched, int flags) {
  if (check_system(sys) != MD_OK || check_schedule(sys, sched) != MD_OK) return 0;
  return run_layout(sys, sched, flags).total;
}

md_status md_newton_series_run(const md_system *sys, double *x, const md_newton_schedule *sched,
                               md_newton_report *rep, void *ws, size_t ws_bytes, int flags, void *stream) {
  md_status st = check_system(sys);
  if (st != MD_OK) return st;
  if (!x || (st = check_schedule(sys, sched)) != MD_OK) return MD_ERR_ARG;
  const RunLayout L = run_layout(sys, sched, flags);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || L.total == 0 || ws_bytes < L.total) return MD_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char *base = static_cast<char *>(ws);
  double *xl = reinterpret_cast<double *>(base + L.off_x);
  double *nrm = reinterpret_cast<double *>(base + L.off_nrm);
  const size_t rows = (size_t)(sys->is_complex ? 2 : 1) * sys->limbs * sys->n;
  const size_t pitch = sizeof(double) * (sys->degree + 1);
  md_newton_report r;
  std::memset(&r, 0, sizeof(r));
  r.converged = 1;
  for (int l = 0; l < sched->nlevels; ++l) {
    const int d = sched->degree[l];
    const md_system t = at_degree(sys, d);
    const size_t w = sizeof(double) * (d + 1);
    // coefficients 0..d of every component, packed as the degree-d layout
    if (cudaMemcpy2DAsync(xl, w, x, pitch, w, rows, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return MD_ERR_CUDA;
    double h[2] = {0.0, 0.0};
    md_status fail = MD_OK;
    for (int it = 1; it <= sched->max_iter[l]; ++it) {
      if ((st = md_newton_series_step(&t, xl, nrm, ws, L.step, flags, stream)) != MD_OK) return st;
      if (cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MD_ERR_CUDA;
      fail = md_get_device_status(ws, stream);  // waits for the step
      r.iterations[l] = it;
      r.dx_norm[l] = h[0];
      r.dx_max[l] = h[1];
      if (fail != MD_OK || h[0] <= sched->tol) break;
    }
    if (cudaMemcpy2DAsync(x, pitch, xl, w, w, rows, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return MD_ERR_CUDA;
    r.levels_done = l + 1;
    if (!(r.dx_norm[l] <= sched->tol)) r.converged = 0;
    if (fail != MD_OK) {
      if (rep) *rep = r;
      return cudaStreamSynchronize(s) == cudaSuccess ? fail : MD_ERR_CUDA;
    }
    if (!(r.dx_norm[l] <= sched->too_large)) break;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return MD_ERR_CUDA;
  if (rep) *rep = r;
  return MD_OK;
}

md_status md_batched_job_costs(int nsys, const md_system *sys, double *cost) {
  if (nsys < 1 || !sys || !cost) return MD_ERR_ARG;
  for (int i = 0; i < nsys; ++i) {
    md_status st;
    std::shared_ptr<PlanEntry> hold;
    const Plan *p = plan_of(&sys[i], st, hold, false);
    if (!p) return st;
    cost[i] = job_cost(*p);
  }
  return MD_OK;
}

size_t md_batched_workspace_bytes(int nsys, const md_system *sys, int flags) {
  std::shared_ptr<BatchPlan> bp;
  if (batch_prepare(nsys, sys, nullptr, bp, false, false, false, (flags & MD_FLAG_OZAKI) ? 1 : 0) != MD_OK) return 0;
  return bp->total;
}

md_status md_newton_series_step_batched(int nsys, const md_system *sys, double *const *x, double *dx_norm,
                                        unsigned long long *times, void *ws, size_t ws_bytes, int flags,
                                        void *stream) {
  if (flags & MD_FLAG_LU) return MD_ERR_UNSUPPORTED;
  if (nsys < 1 || !sys || !x) return MD_ERR_ARG;
  for (int i = 0; i < nsys; ++i)
    if (!x[i]) return MD_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return MD_ERR_WORKSPACE;
  for (int i = 0; i < nsys; ++i)
    if (sys[i].limbs > mdk::kBatchMaxLimbs) return MD_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return MD_ERR_CUDA;
  std::shared_ptr<BatchPlan> bp;
  md_status st = batch_prepare(nsys, sys, x, bp, true, cap == cudaStreamCaptureStatusNone, flags & MD_FLAG_CHECK,
                               (flags & MD_FLAG_OZAKI) ? 1 : 0);
  if (st != MD_OK) return st;
  if (bp->total > ws_bytes) return MD_ERR_WORKSPACE;
  char *base = static_cast<char *>(ws);
  const int sms = device_sms();
  const bool split = !(flags & MD_FLAG_SERIAL);
  const int tstride = (flags & MD_FLAG_PHASE_TIMES) ? mdk::kPhaseStamps : 2;
  // shared-memory attributes of the batched kernels (not stream operations: kept out of any capture)
  for (const BatchClass &c : bp->classes)
    if (dispatch(c.K, c.P, 10, nullptr, s) != cudaSuccess) return MD_ERR_CUDA;
  if ((flags & MD_FLAG_AUTOTUNE) && !bp->tuned) {
    st = batch_autotune(*bp, base, s, sms, split);
    if (st != MD_OK) return st;
  }
  if ((flags & MD_FLAG_GRAPH) && s != nullptr) {
    if (!bp->exec || bp->exec_ws != ws || bp->exec_nrm != dx_norm || bp->exec_times != times || bp->exec_stream != s ||
        bp->exec_split != split || bp->exec_tstride != tstride) {
      if (bp->exec) cudaGraphExecDestroy(bp->exec);
      bp->exec = nullptr;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MD_ERR_CUDA;
      const cudaError_t e = batch_enqueue(*bp, base, dx_norm, times, s, sms, split, tstride);
      if (cudaStreamEndCapture(s, &g) != cudaSuccess || e != cudaSuccess) return MD_ERR_CUDA;
      if (cudaGraphInstantiate(&bp->exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        bp->exec = nullptr;
        return MD_ERR_CUDA;
      }
      cudaGraphDestroy(g);
      bp->exec_ws = ws;
      bp->exec_nrm = dx_norm;
      bp->exec_times = times;
      bp->exec_stream = s;
      bp->exec_split = split;
      bp->exec_tstride = tstride;
    }
    if (cudaGraphLaunch(bp->exec, s) != cudaSuccess) return MD_ERR_CUDA;
  } else if (batch_enqueue(*bp, base, dx_norm, times, s, sms, split, tstride) != cudaSuccess) {
    return MD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap != cudaStreamCaptureStatusNone) {
    bp->captured = true;
    return MD_OK;
  }
  return cuda_status(bp->uses.record(s));
}

void md_plan_cache_hash_mask(unsigned long long mask) { g_hash_mask.store(mask ? mask : ~0ULL); }

int md_plan_factor_sms(const md_system *sys, int flags) {
  if (check_system_header(sys) != MD_OK) return -1;
  const uint64_t cs = structure_checksum(sys) ^ (0x9e3779b97f4a7c15ULL * (uint64_t)(flags & MD_FLAG_OZAKI));
  std::shared_ptr<PlanEntry> hold;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    hold = g_plans.find(cs);
  }
  if (!hold || !same_structure(hold->plan, sys) || hold->plan.oz != ((flags & MD_FLAG_OZAKI) ? 1 : 0)) return -1;
  std::lock_guard<std::mutex> lk(hold->tune.mu);
  return hold->tune.best;
}

void md_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on.store(on != 0);
}

int md_profile_read(double *ms, long long *launches, int nkinds) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (ms)
    for (int k = 0; k < nkinds; ++k) ms[k] = 0.0;
  if (launches)
    for (int k = 0; k < nkinds; ++k) launches[k] = 0;
  int bad = 0;
  for (ProfRec &r : g_prof_recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) ++bad;
    if (r.kind < nkinds) {
      if (ms) ms[r.kind] += t;
      if (launches) launches[r.kind] += 1;
    }
    g_prof_free.push_back(r.a);
    g_prof_free.push_back(r.b);
  }
  g_prof_recs.clear();
  return bad ? -1 : (int)mdk::PK_COUNT;
}

const char *md_profile_kind_name(int kind) {
  if (kind < 0 || kind >= mdk::PK_COUNT) return "unknown";
  return kProfNames[kind];
}

md_status md_get_device_status(void *ws, void *stream) {
  if (!ws) return MD_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MD_ERR_CUDA;
  int word = 0;
  if (cudaMemcpy(&word, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MD_ERR_CUDA;
  if (cudaMemset(ws, 0, sizeof(int)) != cudaSuccess) return MD_ERR_CUDA;
  if (word & mdk::ST_SINGULAR) return MD_ERR_SINGULAR;
  if (word & mdk::ST_NONFINITE) return MD_ERR_NONFINITE;
  if (word & mdk::ST_TIMEOUT) return MD_ERR_TIMEOUT;
  return MD_OK;
}

md_status md_wait_selftest(void *ws, size_t ws_bytes, int target, void *stream) {
  if (!ws || ws_bytes < 256 || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return MD_ERR_WORKSPACE;
  if (target < 0) return MD_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char *base = static_cast<char *>(ws);
  cudaError_t e = cudaMemsetAsync(base, 0, 256, s);
  if (e != cudaSuccess) return MD_ERR_CUDA;
  int *ctr = reinterpret_cast<int *>(base + 64);
  batch_gate_kernel<<<1, 32, 0, s>>>(ctr + kResidentCounter, target, reinterpret_cast<int *>(base));
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
