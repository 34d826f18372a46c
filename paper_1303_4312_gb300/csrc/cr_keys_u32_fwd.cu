// Forward tile-merge kernels for uint32_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_FORWARD(uint32_t)
