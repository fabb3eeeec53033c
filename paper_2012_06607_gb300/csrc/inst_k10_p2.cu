// Kernels and launchers for 10-limb complex numbers.
#include "launch.cuh"
template struct mdk::Impl<10, 2>;
