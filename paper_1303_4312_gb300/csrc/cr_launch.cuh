// cr_launch.cuh -- host-side launchers for one key type K.  Each key type is
// instantiated in its own translation unit (cr_keys_*.cu) so the kernels
// compile in parallel; cr_abi.cu only sees the declarations below.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/corank.h"
#include "cr_device.cuh"

namespace cr {

// Tile shapes: NT consumer threads, each merging ILP interleaved chains of IPT
// items (IPT odd, so that a warp's stride-IPT shared-memory accesses fall in
// distinct banks); TILE = NT * IPT * ILP.
// Every shape is compiled for every key and payload width it fits; which one
// a call uses is a runtime choice per (key size, payload width), set through
// cr_set_tile_shape (the autotuner sweeps them).  TILE = NT * IPT is shared
// by the forward and the backward kernel of a (key, payload) pair, so one
// tile table serves both.
struct ShapeDesc {
    int nt, ipt, ilp;   // consumer threads, items per chain, chains per thread
};
constexpr int kNumShapes = 6;
constexpr ShapeDesc kShapes[kNumShapes] = {{256, 15, 1}, {128, 31, 1}, {256, 7, 1},
                                           {128, 15, 1}, {128, 15, 2}, {256, 31, 1}};

template <int S> struct ShapeAt {
    static constexpr int NT = kShapes[S].nt;
    static constexpr int IPT = kShapes[S].ipt;
    static constexpr int ILP = kShapes[S].ilp;
    static constexpr int TILE = NT * IPT * ILP;
};

// Shared-memory stages of a (key, payload, tag, direction, shape) kernel and
// the CTAs per SM they leave room for: four stages when four fit in about a
// third of the SM's shared memory, else three; FITS is false when even three
// exceed a CTA's 227 KB.
template <int KS, int VB, bool TAG, bool BWD, int S> struct Stages {
    static constexpr int TILE = ShapeAt<S>::TILE;
    static constexpr int BYTES = (TILE + 32) * (KS + VB + (TAG && !BWD ? 4 : 0));
    static constexpr int NS = 4 * BYTES <= 75 * 1024 ? 4 : 3;
    static constexpr int MINB = NS == 4 ? 3 : (3 * BYTES <= 110 * 1024 ? 2 : 1);
    static constexpr bool FITS = NS * BYTES <= 220 * 1024;
};

// A shape is offered for (KS, VB) when the forward kernel with tags and, for
// payloads, the backward kernel fit.
template <int KS, int VB, int S> constexpr bool shape_fits() {
    return Stages<KS, VB, true, false, S>::FITS && (VB == 0 || Stages<KS, VB, false, true, S>::FITS);
}

inline bool shape_available(int key_bytes, int vb, int s) {
    if (s < 0 || s >= kNumShapes) return false;
#define CR_FIT(KS, VB)                                                                       \
    if (key_bytes == KS && vb == VB) {                                                        \
        constexpr bool f[kNumShapes] = {shape_fits<KS, VB, 0>(), shape_fits<KS, VB, 1>(),     \
                                        shape_fits<KS, VB, 2>(), shape_fits<KS, VB, 3>(),     \
                                        shape_fits<KS, VB, 4>(), shape_fits<KS, VB, 5>()};    \
        return f[s];                                                                          \
    }
    CR_FIT(4, 0) CR_FIT(4, 4) CR_FIT(4, 8) CR_FIT(8, 0) CR_FIT(8, 4) CR_FIT(8, 8)
#undef CR_FIT
    return false;
}

// Geometry class of a merge: small (2) when m + n <= kSmallClassElems --
// few tiles per CTA slot, where smaller tiles balance the grid better and
// the partition is cheap; else skewed (1) when one input is more than 16
// times longer than the other (nearly whole tiles come from one input);
// else balanced (0).  Each class has its own tile shape.
constexpr int64_t kSmallClassElems = int64_t(1) << 23;
// Batched calls (3) and merge passes (4) have classes of their own: their
// segments or runs are not known on the host, and their best shapes differ
// from a single merge's.
constexpr int kClassBatched = 3;
constexpr int kClassPass = 4;
constexpr int kNumClasses = 5;
// Recorded merge passes keep a tile's source flags in one CTA of the
// routing backward: their tiles hold at most this many elements.
constexpr int64_t kMaxRecordTile = 4096;
inline int geometry_class(int64_t m, int64_t n) {
    if (m + n <= kSmallClassElems) return 2;
    const int64_t lo = m < n ? m : n, hi = m < n ? n : m;
    return 16 * lo < hi ? 1 : 0;
}

// Current shape per (key size, payload width, geometry class) (cr_abi.cu
// owns the table).
int current_shape(int key_bytes, int vb, int cls);

// Single merges with at most this many tiles co-rank every tile start with
// its own 16-lane group (fewer dependent rounds; the probes of all tile
// starts stay within a few MB).
constexpr int64_t kSmallMergeTiles = 4096;

// Run formation: the chunk of the shared-memory merge stage (cr_block.cu).
constexpr int64_t kSortRun = 4096;

// Round an array pointer down to its 16-byte boundary; *sh receives the
// array's start from there in elements of `elem` bytes (the pointer must be
// aligned to `elem`).
template <class P>
inline P* align16_base(P* p, int elem, int32_t* sh) {
    const uintptr_t u = reinterpret_cast<uintptr_t>(p);
    *sh = elem > 0 ? int32_t((u & 15u) / uintptr_t(elem)) : 0;
    return reinterpret_cast<P*>(u & ~uintptr_t(15));
}

// Apply align16_base to every data array of a tile-merge call (keys of ks
// bytes; payloads and gradients of vb bytes; tags of 4).  flags and ws are
// left as they are (they must be 16-byte aligned themselves).
inline void align_merge_args(MergeArgs& a, int ks, int vb) {
    a.ak = align16_base(a.ak, ks, &a.sh_ak);
    a.bk = align16_base(a.bk, ks, &a.sh_bk);
    a.av = align16_base(a.av, vb, &a.sh_av);
    a.bv = align16_base(a.bv, vb, &a.sh_bv);
    a.gc_in = align16_base(a.gc_in, vb, &a.sh_gc);
    a.ck = align16_base(a.ck, ks, &a.sh_ck);
    a.cv = align16_base(a.cv, vb, &a.sh_cv);
    a.cv2 = align16_base(a.cv2, vb, &a.sh_cv2);
    a.ctag = align16_base(a.ctag, 4, &a.sh_tag);
}

inline int64_t tile_of_shape(int s) {
    return int64_t(kShapes[s].nt) * kShapes[s].ipt * kShapes[s].ilp;
}

template <class K>
struct KeyOps {
    // Forward merge of the tiles listed in the workspace.  vb in {0,4,8};
    // shape: index into kShapes (must match the tile size of the table).
    static cudaError_t merge_fwd(int shape, int vb, bool tag, const MergeArgs& a,
                                 int64_t max_tiles, cudaStream_t st);
    // Forward merge with payloads (vb in {4,8}) that also records every
    // output's source run as one bit per output (a.flags, per tile).
    static cudaError_t merge_fwd_rec(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                     cudaStream_t st);
    // Payload backward (vb in {4,8}).
    static cudaError_t merge_bwd(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                 cudaStream_t st);
    // The same three for keys in another order than their storage type's
    // (a.order != 0); the calls above forward to these.
    static cudaError_t merge_fwd_ord(int shape, int vb, bool tag, const MergeArgs& a,
                                     int64_t max_tiles, cudaStream_t st);
    static cudaError_t merge_fwd_rec_ord(int shape, int vb, const MergeArgs& a,
                                         int64_t max_tiles, cudaStream_t st);
    static cudaError_t merge_bwd_ord(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                     cudaStream_t st);
    // The same three for the descending order of the storage type
    // (a.order == 1): the comparisons reversed, keys neither mapped nor
    // mapped back.
    static cudaError_t merge_fwd_desc(int shape, int vb, bool tag, const MergeArgs& a,
                                      int64_t max_tiles, cudaStream_t st);
    static cudaError_t merge_fwd_rec_desc(int shape, int vb, const MergeArgs& a,
                                          int64_t max_tiles, cudaStream_t st);
    static cudaError_t merge_bwd_desc(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                      cudaStream_t st);
    // And for IEEE-754 totalOrder floats stored in a signed K (a.order 2
    // ascending, 3 descending), with the order map fixed at compile time.
    static cudaError_t merge_fwd_flt(int shape, int vb, bool tag, const MergeArgs& a,
                                     int64_t max_tiles, cudaStream_t st);
    static cudaError_t merge_fwd_rec_flt(int shape, int vb, const MergeArgs& a,
                                         int64_t max_tiles, cudaStream_t st);
    static cudaError_t merge_bwd_flt(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                     cudaStream_t st);
    // order: key order of the call (order_key in cr_device.cuh).
    static cudaError_t partition_single(const void* A, int64_t m, const void* B, int64_t n,
                                        int64_t tile, int64_t ntiles, void* ws, int order,
                                        cudaStream_t st);
    // Same table, every tile co-ranking both of its ends (Algorithm 1).
    static cudaError_t partition_single_free(const void* A, int64_t m, const void* B, int64_t n,
                                             int64_t tile, int64_t ntiles, void* ws, int order,
                                             cudaStream_t st);
    static cudaError_t partition_pass(const void* X, int64_t N, int64_t w, int64_t tile,
                                      void* ws, int64_t* ntiles_out, int order, cudaStream_t st);
    static cudaError_t partition_batched(const void* A, const void* B, const int64_t* a_off,
                                         const int64_t* b_off, int64_t nseg, int64_t a_total,
                                         int64_t b_total, int64_t tile, int64_t max_tiles,
                                         void* ws, int64_t* prefix, int order, cudaStream_t st);
    static cudaError_t co_rank_many(const void* A, int64_t m, const void* B, int64_t n,
                                    const int64_t* ranks, int64_t cnt, int64_t* oi, int64_t* oj,
                                    int order, cudaStream_t st);
    static cudaError_t co_rank_one(const void* A, int64_t m, const void* B, int64_t n, int64_t r,
                                   int64_t* out, int order, cudaStream_t st);
};

// Backward of a recorded merge pass (vb in {4,8}) over N elements with run
// width w (1 <= w <= N): gX from gY, routed by the tile table in ws and the
// per-tile source flags, without keys.  tile: the table's tile size (the
// table's header and records are checked against it and the pass geometry).
cudaError_t route_recorded(int vb, void* ws, const uint32_t* flags, int64_t flag_words,
                           int64_t N, int64_t w, int64_t tile, const void* gY, void* gX,
                           cudaStream_t st);

// Run formation (cr_block.cu): the shared-memory merge stage from width 1
// stably sorts every run of kSortRun elements.  mode 0: forward (vb 0, 4,
// 8); 1: forward that also writes each run's permutation (vb 4, 8); 2:
// backward that replays the sort on X and routes gY to gX through the
// recovered permutation (vb 4, 8; Xv, Y, Yv, perm unused).
cudaError_t block_sort_runs(int key_type, int vb, int mode, const void* X, const void* Xv,
                            int64_t N, void* Y, void* Yv, uint16_t* perm, const void* gY,
                            void* gX, cudaStream_t st);

// Backward of a recorded run formation (vb in {4,8}): within every run of
// kSortRun elements, gX[base + perm[base + x]] = gY[base + x].
cudaError_t sort_route_recorded(int vb, int64_t N, const uint16_t* perm, const void* gY, void* gX,
                                cudaStream_t st);

// C-ABI key types: storage width, storage type and order (order_key).
// F32/F64 are stored and compared as the signed integer of their width after
// the float total-order map; key pairs as uint64 (signed halves after the
// pair map); CR_KEY_DESC adds the complement.
inline int key_base(int key_type) { return key_type & ~int(CR_KEY_DESC); }

inline int key_type_bytes(int key_type) {
    if (key_type < 0 || (key_type & ~(int(CR_KEY_DESC) | 0xFF)) != 0) return 0;
    switch (key_base(key_type)) {
        case CR_KEY_I32:
        case CR_KEY_U32:
        case CR_KEY_F32: return 4;
        case CR_KEY_I64:
        case CR_KEY_U64:
        case CR_KEY_F64:
        case CR_KEY_PAIR_U32:
        case CR_KEY_PAIR_I32: return 8;
        default: return 0;
    }
}

inline int key_type_order(int key_type) {
    const int b = key_base(key_type);
    return ((b == CR_KEY_F32 || b == CR_KEY_F64) ? 2 : 0) | (b == CR_KEY_PAIR_I32 ? 4 : 0) |
           ((key_type & CR_KEY_DESC) ? 1 : 0);
}

template <class F>
cudaError_t with_key_ops(int key_type, F&& f) {
    if (key_type_bytes(key_type) == 0) return cudaErrorInvalidValue;
    switch (key_base(key_type)) {
        case CR_KEY_I32:
        case CR_KEY_F32: return f(KeyOps<int32_t>{});
        case CR_KEY_U32: return f(KeyOps<uint32_t>{});
        case CR_KEY_I64:
        case CR_KEY_F64: return f(KeyOps<int64_t>{});
        case CR_KEY_U64:
        case CR_KEY_PAIR_U32:
        case CR_KEY_PAIR_I32: return f(KeyOps<uint64_t>{});
        default: return cudaErrorInvalidValue;
    }
}

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
