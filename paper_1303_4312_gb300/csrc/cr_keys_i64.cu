// Backward kernels, partitions and co-rank kernels for int64_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_REST(int64_t)
