// Host build of the fixed-point scalar arithmetic (csrc/fixp.cuh) for the CPU
// tests: every operation on K-limb md inputs, results as K-limb md values.
#include <cstdint>

#include "../paper_2012_06607_gb300/csrc/fixp.cuh"

using namespace mdk::fxp;

template <int K>
static void run(int op, const double *x, const double *y, double *out) {
  constexpr int W = words_for(K);
  constexpr int ST = newton_steps(K);
  double xv[K], yv[K], z[K];
  for (int l = 0; l < K; ++l) {
    xv[l] = x[l];
    yv[l] = y ? y[l] : 0.0;
  }
  const bf<W> a = from_md<W, K>(xv), b = from_md<W, K>(yv);
  bf<W> r;
  switch (op) {
    case 0: r = a; break;                           // round trip
    case 1: r = mul<W>(a, b); break;                // product
    case 2: r = add<W>(a, b); break;                // sum
    case 3: r = rsqrt<W, ST>(a); break;             // 1 / sqrt(a)
    case 4: r = mul<W>(a, rsqrt<W, ST>(a)); break;  // sqrt(a)
    default: r = recip<W, ST>(a); break;            // 1 / a
  }
  to_md<K, W>(r, z);
  for (int l = 0; l < K; ++l) out[l] = z[l];
}

extern "C" int fxp_op(int K, int op, long count, const double *x, const double *y, double *out) {
  for (long i = 0; i < count; ++i) {
    const double *yi = y ? y + i * K : nullptr;
    switch (K) {
      case 2: run<2>(op, x + i * K, yi, out + i * K); break;
      case 3: run<3>(op, x + i * K, yi, out + i * K); break;
      case 4: run<4>(op, x + i * K, yi, out + i * K); break;
      case 5: run<5>(op, x + i * K, yi, out + i * K); break;
      case 8: run<8>(op, x + i * K, yi, out + i * K); break;
      case 10: run<10>(op, x + i * K, yi, out + i * K); break;
      default: return 1;
    }
  }
  return 0;
}
