// Kernels and launchers for 10-limb real numbers.
#include "launch.cuh"
template struct mdk::Impl<10, 1>;
