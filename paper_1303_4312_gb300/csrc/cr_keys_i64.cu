// Kernels and launchers for int64_t keys.
#include "cr_keyops_impl.cuh"

template struct cr::KeyOps<int64_t>;
