// Explicit instantiation of one part of the launchers for MDK_K limbs and
// MDK_P planes (compiled once per (K, P, part) by the build script, so that
// the translation units compile in parallel).
#include "launch.cuh"

#if MDK_PART == 0
template cudaError_t mdk::Impl<MDK_K, MDK_P>::elementwise(int, long long, const double *, const double *, double *,
                                                          cudaStream_t);
template cudaError_t mdk::Impl<MDK_K, MDK_P>::series_conv(int, long long, const double *, const double *, double *,
                                                          cudaStream_t);
#elif MDK_PART == 1
template cudaError_t mdk::Impl<MDK_K, MDK_P>::eval(const mdk::EvalDev &, cudaStream_t);
template cudaError_t mdk::Impl<MDK_K, MDK_P>::eval0(const mdk::EvalDev &, cudaStream_t);
template cudaError_t mdk::Impl<MDK_K, MDK_P>::eval_rest(const mdk::EvalDev &, cudaStream_t);
#elif MDK_PART == 2
template cudaError_t mdk::Impl<MDK_K, MDK_P>::solve(const mdk::SolveDev &, cudaStream_t);
template cudaError_t mdk::Impl<MDK_K, MDK_P>::factor(const mdk::SolveDev &, cudaStream_t);
template cudaError_t mdk::Impl<MDK_K, MDK_P>::degrees(const mdk::SolveDev &, cudaStream_t);
template cudaError_t mdk::Impl<MDK_K, MDK_P>::rcond(const mdk::SolveDev &, cudaStream_t);
#elif MDK_PART == 3
template cudaError_t mdk::Impl<MDK_K, MDK_P>::batched(const mdk::BatchDev &, cudaStream_t);
template cudaError_t mdk::Impl<MDK_K, MDK_P>::batched_setup();
#endif
