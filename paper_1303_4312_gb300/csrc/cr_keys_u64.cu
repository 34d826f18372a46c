// Kernels and launchers for uint64_t keys.
#include "cr_keyops_impl.cuh"

template struct cr::KeyOps<uint64_t>;
