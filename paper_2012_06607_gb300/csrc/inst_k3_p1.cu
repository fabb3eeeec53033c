// Kernels and launchers for 3-limb real numbers.
#include "launch.cuh"
template struct mdk::Impl<3, 1>;
