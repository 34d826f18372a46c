// Recording forward tile-merge kernels (merge passes whose backward reads
// no keys) for uint32_t keys.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_RECORD(uint32_t)
