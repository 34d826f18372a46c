// Tile-merge kernels (forward, recording forward, backward) for float keys in
// IEEE-754 totalOrder stored as int64_t, ascending and descending, with the
// order map fixed at compile time.
#include "cr_keyops_impl.cuh"

CR_INSTANTIATE_FLOAT(int64_t)
