// Recording forward tile-merge kernels (merge passes whose backward reads
// no keys) for uint64_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_RECORD(uint64_t)
