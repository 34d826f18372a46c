// Tile-merge kernels (forward, recording forward, backward) for uint32_t keys in
// descending order (comparisons reversed; keys neither mapped nor mapped back).
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_DESC(uint32_t)
