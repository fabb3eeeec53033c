// Kernels and launchers for 3-limb complex numbers.
#include "launch.cuh"
template struct mdk::Impl<3, 2>;
