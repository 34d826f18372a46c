// Recording forward tile-merge kernels (merge passes whose backward reads
// no keys) for int32_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_RECORD(int32_t)
