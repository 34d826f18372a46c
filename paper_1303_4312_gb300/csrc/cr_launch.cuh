// cr_launch.cuh -- host-side launchers for one key type K.  Each key type is
// instantiated in its own translation unit (cr_keys_*.cu) so the kernels
// compile in parallel; cr_abi.cu only sees the declarations below.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "cr_device.cuh"

namespace cr {

// Tile shape per key size and payload width: consumer threads NT and items per
// thread IPT (odd, so that a warp's stride-IPT shared-memory accesses fall in
// distinct banks).  TILE = NT * IPT is the same for the forward and the
// backward kernel of a (key, payload) pair.
template <int KS, int VB> struct TileShape { static constexpr int NT = 256, IPT = 7; };
template <> struct TileShape<4, 0> { static constexpr int NT = 256, IPT = 15; };

// Stages in the shared-memory ring and the CTAs per SM they leave room for:
// four stages when a stage is at most 16 KB (three CTAs per SM), else three.
template <int KS, int VB, bool TAG, bool BWD> struct Stages {
    static constexpr int TILE = TileShape<KS, VB>::NT * TileShape<KS, VB>::IPT;
    static constexpr int BYTES = TILE * (KS + VB + (TAG && !BWD ? 4 : 0));
    static constexpr int NS = BYTES <= 16384 ? 4 : 3;
    static constexpr int MINB = NS == 4 ? 3 : 2;
};

template <int KS, int VB> constexpr int64_t tile_of() {
    return int64_t(TileShape<KS, VB>::NT) * TileShape<KS, VB>::IPT;
}

inline int64_t tile_for(int key_bytes, int vb) {
    if (key_bytes == 4) {
        if (vb == 0) return tile_of<4, 0>();
        if (vb == 4) return tile_of<4, 4>();
        if (vb == 8) return tile_of<4, 8>();
    } else if (key_bytes == 8) {
        if (vb == 0) return tile_of<8, 0>();
        if (vb == 4) return tile_of<8, 4>();
        if (vb == 8) return tile_of<8, 8>();
    }
    return 0;
}

template <class K>
struct KeyOps {
    // Forward merge of the tiles listed in the workspace.  vb in {0,4,8}.
    static cudaError_t merge_fwd(int vb, bool tag, const MergeArgs& a, int64_t max_tiles,
                                 cudaStream_t st);
    // Payload backward (vb in {4,8}).
    static cudaError_t merge_bwd(int vb, const MergeArgs& a, int64_t max_tiles, cudaStream_t st);
    static cudaError_t partition_single(const void* A, int64_t m, const void* B, int64_t n,
                                        int64_t tile, int64_t ntiles, void* ws, cudaStream_t st);
    static cudaError_t partition_pass(const void* X, int64_t N, int64_t w, int64_t tile,
                                      void* ws, int64_t* ntiles_out, cudaStream_t st);
    static cudaError_t partition_batched(const void* A, const void* B, const int64_t* a_off,
                                         const int64_t* b_off, int64_t nseg, int64_t a_total,
                                         int64_t b_total, int64_t tile, int64_t max_tiles,
                                         void* ws, int64_t* prefix, cudaStream_t st);
    static cudaError_t co_rank_many(const void* A, int64_t m, const void* B, int64_t n,
                                    const int64_t* ranks, int64_t cnt, int64_t* oi, int64_t* oj,
                                    cudaStream_t st);
    static cudaError_t co_rank_one(const void* A, int64_t m, const void* B, int64_t n, int64_t r,
                                   int64_t* out, cudaStream_t st);
};

// Tiles of a merge pass over N elements with run width w.
inline int64_t pass_tiles(int64_t N, int64_t w, int64_t tile, int64_t* tpp_out,
                          int64_t* npairs_out) {
    if (N <= 0) {
        if (tpp_out) *tpp_out = 1;
        if (npairs_out) *npairs_out = 0;
        return 0;
    }
    const int64_t npairs = (N + 2 * w - 1) / (2 * w);
    const int64_t tpp = (2 * w + tile - 1) / tile;
    const int64_t last = N - 2 * w * (npairs - 1);
    if (tpp_out) *tpp_out = tpp;
    if (npairs_out) *npairs_out = npairs;
    return (npairs - 1) * tpp + (last + tile - 1) / tile;
}

}  // namespace cr
