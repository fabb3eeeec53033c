// Kernels and launchers for 8-limb complex numbers.
#include "launch.cuh"
template struct mdk::Impl<8, 2>;
