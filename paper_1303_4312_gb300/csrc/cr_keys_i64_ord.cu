// Tile-merge kernels (forward, recording forward, backward) for int64_t keys in
// another order than their own (descending; float total order).
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_ORDER(int64_t)
