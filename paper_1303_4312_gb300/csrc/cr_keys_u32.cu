// Backward kernels, partitions and co-rank kernels for uint32_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_REST(uint32_t)
