// Kernels and launchers for 8-limb real numbers.
#include "launch.cuh"
template struct mdk::Impl<8, 1>;
