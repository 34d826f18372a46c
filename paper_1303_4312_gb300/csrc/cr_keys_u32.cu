// Kernels and launchers for uint32_t keys.
#include "cr_keyops_impl.cuh"

template struct cr::KeyOps<uint32_t>;
