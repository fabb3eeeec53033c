// Kernels and launchers for 2-limb complex numbers.
#include "launch.cuh"
template struct mdk::Impl<2, 2>;
