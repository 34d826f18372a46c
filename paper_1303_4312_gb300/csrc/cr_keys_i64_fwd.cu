// Forward tile-merge kernels for int64_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_FORWARD(int64_t)
