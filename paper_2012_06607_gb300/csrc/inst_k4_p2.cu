// Kernels and launchers for 4-limb complex numbers.
#include "launch.cuh"
template struct mdk::Impl<4, 2>;
