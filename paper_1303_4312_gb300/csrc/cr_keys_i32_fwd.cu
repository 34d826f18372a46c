// Forward tile-merge kernels for int32_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_FORWARD(int32_t)
