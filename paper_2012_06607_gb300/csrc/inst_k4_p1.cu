// Kernels and launchers for 4-limb real numbers.
#include "launch.cuh"
template struct mdk::Impl<4, 1>;
