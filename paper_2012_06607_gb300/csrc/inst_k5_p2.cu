// Kernels and launchers for 5-limb complex numbers.
#include "launch.cuh"
template struct mdk::Impl<5, 2>;
