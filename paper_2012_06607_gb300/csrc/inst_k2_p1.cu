// Kernels and launchers for 2-limb real numbers.
#include "launch.cuh"
template struct mdk::Impl<2, 1>;
