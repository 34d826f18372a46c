// Backward kernels, partitions and co-rank kernels for int32_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_REST(int32_t)
