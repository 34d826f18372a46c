// Kernels and launchers for int32_t keys.
#include "cr_keyops_impl.cuh"

template struct cr::KeyOps<int32_t>;
