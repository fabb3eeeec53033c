// Kernels and launchers for 1-limb complex numbers.
#include "launch.cuh"
template struct mdk::Impl<1, 2>;
