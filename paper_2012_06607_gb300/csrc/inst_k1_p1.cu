// Kernels and launchers for 1-limb real numbers.
#include "launch.cuh"
template struct mdk::Impl<1, 1>;
