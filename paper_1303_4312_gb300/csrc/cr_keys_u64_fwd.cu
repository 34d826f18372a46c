// Forward tile-merge kernels for uint64_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_FORWARD(uint64_t)
