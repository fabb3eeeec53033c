// Kernels and launchers for 5-limb real numbers.
#include "launch.cuh"
template struct mdk::Impl<5, 1>;
