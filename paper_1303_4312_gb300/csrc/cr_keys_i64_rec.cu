// Recording forward tile-merge kernels (merge passes whose backward reads
// no keys) for int64_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_RECORD(int64_t)
