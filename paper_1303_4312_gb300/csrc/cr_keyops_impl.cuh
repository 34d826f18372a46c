// cr_keyops_impl.cuh -- definitions of KeyOps<K>; included by exactly one
// translation unit per key type.
#pragma once

#include <mutex>

#include "cr_launch.cuh"
#include "cr_merge.cuh"
#include "cr_partition.cuh"

namespace cr {

constexpr int kMaxDevices = 64;

// Per-device launch shape of one merge kernel instantiation: CTAs per SM
// (from the occupancy calculator, after raising the shared-memory limit) and
// the SM count.  Computed once per device.
struct LaunchShape {
    int blocks_per_sm = 0;
    int sms = 0;
};

template <class Kern>
cudaError_t launch_shape(Kern kern, int threads, size_t smem, LaunchShape* cache,
                         std::once_flag* once, LaunchShape& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaError_t err = cudaSuccess;
    std::call_once(once[dev], [&] {
        LaunchShape s;
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (err == cudaSuccess)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.blocks_per_sm, kern, threads,
                                                                smem);
        if (err == cudaSuccess)
            err = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
        if (err == cudaSuccess) cache[dev] = s;
    });
    if (err != cudaSuccess) return err;
    out = cache[dev];
    if (out.sms <= 0 || out.blocks_per_sm <= 0) return cudaErrorInvalidConfiguration;
    return cudaSuccess;
}

template <class K, int VB, bool TAG, bool BWD, int S, bool REC, int ORD>
cudaError_t launch_merge_shape(const MergeArgs& a, int64_t max_tiles, cudaStream_t st) {
    constexpr int KS = int(sizeof(K));
    if constexpr (!Stages<KS, VB, TAG, BWD, S>::FITS) {
        return cudaErrorInvalidConfiguration;
    } else {
        constexpr int NT = ShapeAt<S>::NT;
        constexpr int IPT = ShapeAt<S>::IPT;
        constexpr int ILP = ShapeAt<S>::ILP;
        constexpr int NS = Stages<KS, VB, TAG, BWD, S>::NS;
        constexpr int MINB = Stages<KS, VB, TAG, BWD, S>::MINB;
        using L = Layout<K, VB, TAG, NT, IPT, ILP, NS, BWD, REC>;
        auto kern = merge_tiles_kernel<K, VB, TAG, NT, IPT, ILP, NS, MINB, BWD, REC, ORD>;
        static LaunchShape cache[kMaxDevices];
        static std::once_flag once[kMaxDevices];
        LaunchShape sh;
        constexpr int THREADS = merge_block_threads<NT>();
        cudaError_t e = launch_shape(kern, THREADS, L::TOTAL, cache, once, sh);
        if (e != cudaSuccess) return e;
        if (max_tiles <= 0) return cudaSuccess;
        int64_t grid = int64_t(sh.sms) * sh.blocks_per_sm;
        if (grid > max_tiles) grid = max_tiles;
        MergeArgs aa = a;
        align_merge_args(aa, KS, VB);
        kern<<<unsigned(grid), THREADS, L::TOTAL, st>>>(aa);
        return cudaGetLastError();
    }
}

template <class K, int VB, bool TAG, bool BWD, bool REC = false, int ORD = 0>
cudaError_t launch_merge(int shape, const MergeArgs& a, int64_t max_tiles, cudaStream_t st) {
    static_assert(kNumShapes == 6, "dispatch below lists every shape");
    switch (shape) {
        case 0: return launch_merge_shape<K, VB, TAG, BWD, 0, REC, ORD>(a, max_tiles, st);
        case 1: return launch_merge_shape<K, VB, TAG, BWD, 1, REC, ORD>(a, max_tiles, st);
        case 2: return launch_merge_shape<K, VB, TAG, BWD, 2, REC, ORD>(a, max_tiles, st);
        case 3: return launch_merge_shape<K, VB, TAG, BWD, 3, REC, ORD>(a, max_tiles, st);
        case 4: return launch_merge_shape<K, VB, TAG, BWD, 4, REC, ORD>(a, max_tiles, st);
        case 5: return launch_merge_shape<K, VB, TAG, BWD, 5, REC, ORD>(a, max_tiles, st);
        default: return cudaErrorInvalidValue;
    }
}

// The forward tile merges of one key type, for its own order (ORD 0),
// another one through the order map (ORD 1) or its own order descending
// (ORD 2, the comparison reversed).
template <class K, int ORD>
cudaError_t merge_fwd_impl(int shape, int vb, bool tag, const MergeArgs& a, int64_t max_tiles,
                           cudaStream_t st) {
    switch (vb * 2 + (tag ? 1 : 0)) {
        case 0: return launch_merge<K, 0, false, false, false, ORD>(shape, a, max_tiles, st);
        case 1: return launch_merge<K, 0, true, false, false, ORD>(shape, a, max_tiles, st);
        case 8: return launch_merge<K, 4, false, false, false, ORD>(shape, a, max_tiles, st);
        case 9: return launch_merge<K, 4, true, false, false, ORD>(shape, a, max_tiles, st);
        case 16: return launch_merge<K, 8, false, false, false, ORD>(shape, a, max_tiles, st);
        case 17: return launch_merge<K, 8, true, false, false, ORD>(shape, a, max_tiles, st);
        default: return cudaErrorInvalidValue;
    }
}

template <class K, int ORD>
cudaError_t merge_fwd_rec_impl(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                               cudaStream_t st) {
    if (vb == 4) return launch_merge<K, 4, false, false, true, ORD>(shape, a, max_tiles, st);
    if (vb == 8) return launch_merge<K, 8, false, false, true, ORD>(shape, a, max_tiles, st);
    return cudaErrorInvalidValue;
}

template <class K, int ORD>
cudaError_t merge_bwd_impl(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                           cudaStream_t st) {
    if (vb == 4) return launch_merge<K, 4, false, true, false, ORD>(shape, a, max_tiles, st);
    if (vb == 8) return launch_merge<K, 8, false, true, false, ORD>(shape, a, max_tiles, st);
    return cudaErrorInvalidValue;
}

template <class K>
cudaError_t KeyOps<K>::merge_fwd(int shape, int vb, bool tag, const MergeArgs& a,
                                 int64_t max_tiles, cudaStream_t st) {
    if (a.order == 1) return merge_fwd_desc(shape, vb, tag, a, max_tiles, st);
    if constexpr (std::is_signed<K>::value)
        if (a.order == 2 || a.order == 3) return merge_fwd_flt(shape, vb, tag, a, max_tiles, st);
    if (a.order != 0) return merge_fwd_ord(shape, vb, tag, a, max_tiles, st);
    return merge_fwd_impl<K, 0>(shape, vb, tag, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_fwd_rec(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                     cudaStream_t st) {
    if (a.order == 1) return merge_fwd_rec_desc(shape, vb, a, max_tiles, st);
    if constexpr (std::is_signed<K>::value)
        if (a.order == 2 || a.order == 3) return merge_fwd_rec_flt(shape, vb, a, max_tiles, st);
    if (a.order != 0) return merge_fwd_rec_ord(shape, vb, a, max_tiles, st);
    return merge_fwd_rec_impl<K, 0>(shape, vb, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_bwd(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                 cudaStream_t st) {
    if (a.order == 1) return merge_bwd_desc(shape, vb, a, max_tiles, st);
    if constexpr (std::is_signed<K>::value)
        if (a.order == 2 || a.order == 3) return merge_bwd_flt(shape, vb, a, max_tiles, st);
    if (a.order != 0) return merge_bwd_ord(shape, vb, a, max_tiles, st);
    return merge_bwd_impl<K, 0>(shape, vb, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_fwd_ord(int shape, int vb, bool tag, const MergeArgs& a,
                                     int64_t max_tiles, cudaStream_t st) {
    return merge_fwd_impl<K, 1>(shape, vb, tag, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_fwd_rec_ord(int shape, int vb, const MergeArgs& a,
                                         int64_t max_tiles, cudaStream_t st) {
    return merge_fwd_rec_impl<K, 1>(shape, vb, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_bwd_ord(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                     cudaStream_t st) {
    return merge_bwd_impl<K, 1>(shape, vb, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_fwd_desc(int shape, int vb, bool tag, const MergeArgs& a,
                                      int64_t max_tiles, cudaStream_t st) {
    return merge_fwd_impl<K, 2>(shape, vb, tag, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_fwd_rec_desc(int shape, int vb, const MergeArgs& a,
                                          int64_t max_tiles, cudaStream_t st) {
    return merge_fwd_rec_impl<K, 2>(shape, vb, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_bwd_desc(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                      cudaStream_t st) {
    return merge_bwd_impl<K, 2>(shape, vb, a, max_tiles, st);
}

// Float keys (signed storage types only): order 2 ascending, 3 descending.
template <class K>
cudaError_t KeyOps<K>::merge_fwd_flt(int shape, int vb, bool tag, const MergeArgs& a,
                                     int64_t max_tiles, cudaStream_t st) {
    return a.order == 3 ? merge_fwd_impl<K, 4>(shape, vb, tag, a, max_tiles, st)
                        : merge_fwd_impl<K, 3>(shape, vb, tag, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_fwd_rec_flt(int shape, int vb, const MergeArgs& a,
                                         int64_t max_tiles, cudaStream_t st) {
    return a.order == 3 ? merge_fwd_rec_impl<K, 4>(shape, vb, a, max_tiles, st)
                        : merge_fwd_rec_impl<K, 3>(shape, vb, a, max_tiles, st);
}

template <class K>
cudaError_t KeyOps<K>::merge_bwd_flt(int shape, int vb, const MergeArgs& a, int64_t max_tiles,
                                     cudaStream_t st) {
    return a.order == 3 ? merge_bwd_impl<K, 4>(shape, vb, a, max_tiles, st)
                        : merge_bwd_impl<K, 3>(shape, vb, a, max_tiles, st);
}

static inline unsigned blocks_for(int64_t n, int threads) {
    return unsigned((n + threads - 1) / threads);
}

template <class K>
cudaError_t KeyOps<K>::partition_single(const void* A, int64_t m, const void* B, int64_t n,
                                        int64_t tile, int64_t ntiles, void* ws, int order,
                                        cudaStream_t st) {
    if (ntiles <= kSmallMergeTiles) {
        // 16 lanes per tile start, 15 tiles per block
        const unsigned g = unsigned(((ntiles > 0 ? ntiles : 1) + 14) / 15);
        partition_single_small_kernel<K><<<g, 256, 0, st>>>(
            static_cast<const K*>(A), m, static_cast<const K*>(B), n, tile, ntiles, ws, order);
        return cudaGetLastError();
    }
    // 256 threads search 256 consecutive boundaries = 255 tiles per block
    const unsigned g = unsigned(((ntiles > 0 ? ntiles : 1) + 254) / 255);
    partition_single_kernel<K><<<g, 256, 0, st>>>(static_cast<const K*>(A), m,
                                                   static_cast<const K*>(B), n, tile, ntiles, ws,
                                                   order);
    return cudaGetLastError();
}

template <class K>
cudaError_t KeyOps<K>::partition_single_free(const void* A, int64_t m, const void* B, int64_t n,
                                             int64_t tile, int64_t ntiles, void* ws, int order,
                                             cudaStream_t st) {
    const unsigned g = blocks_for(ntiles > 0 ? ntiles : 1, 256);
    partition_single_free_kernel<K><<<g, 256, 0, st>>>(static_cast<const K*>(A), m,
                                                        static_cast<const K*>(B), n, tile, ntiles,
                                                        ws, order);
    return cudaGetLastError();
}

template <class K>
cudaError_t KeyOps<K>::partition_pass(const void* X, int64_t N, int64_t w, int64_t tile,
                                      void* ws, int64_t* ntiles_out, int order, cudaStream_t st) {
    int64_t tpp = 1, npairs = 0;
    const int64_t ntiles = pass_tiles(N, w, tile, &tpp, &npairs);
    if (ntiles_out) *ntiles_out = ntiles;
    // 256 threads co-rank 256 consecutive tile starts = 255 tiles per block
    const unsigned g = unsigned(((ntiles > 0 ? ntiles : 1) + 254) / 255);
    partition_pass_kernel<K><<<g, 256, 0, st>>>(static_cast<const K*>(X), N, w, tile, tpp,
                                                 npairs, ntiles, ws, order);
    return cudaGetLastError();
}

template <class K>
cudaError_t KeyOps<K>::partition_batched(const void* A, const void* B, const int64_t* a_off,
                                         const int64_t* b_off, int64_t nseg, int64_t a_total,
                                         int64_t b_total, int64_t tile, int64_t max_tiles,
                                         void* ws, int64_t* prefix, int order, cudaStream_t st) {
    segment_scan_kernel<<<1, 1024, 0, st>>>(a_off, b_off, nseg, a_total, b_total, tile, ws,
                                            prefix);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || max_tiles <= 0) return e;
    partition_batched_kernel<K><<<blocks_for(max_tiles, 255), 256, 0, st>>>(
        static_cast<const K*>(A), static_cast<const K*>(B), a_off, b_off, nseg, tile, prefix, ws,
        order);
    return cudaGetLastError();
}

template <class K>
cudaError_t KeyOps<K>::co_rank_many(const void* A, int64_t m, const void* B, int64_t n,
                                    const int64_t* ranks, int64_t cnt, int64_t* oi, int64_t* oj,
                                    int order, cudaStream_t st) {
    if (cnt <= 0) return cudaSuccess;
    co_rank_many_kernel<K><<<blocks_for(cnt, 256), 256, 0, st>>>(
        static_cast<const K*>(A), m, static_cast<const K*>(B), n, ranks, cnt, oi, oj, order);
    return cudaGetLastError();
}

template <class K>
cudaError_t KeyOps<K>::co_rank_one(const void* A, int64_t m, const void* B, int64_t n, int64_t r,
                                   int64_t* out, int order, cudaStream_t st) {
    co_rank_one_kernel<K><<<1, 1, 0, st>>>(static_cast<const K*>(A), m,
                                           static_cast<const K*>(B), n, r, out, order);
    return cudaGetLastError();
}

}  // namespace cr

// Explicit instantiation, split so that the forward kernels and the rest of a
// key type compile in separate translation units.
#define CR_INSTANTIATE_FORWARD(K)                                                              \
    template cudaError_t cr::KeyOps<K>::merge_fwd(int, int, bool, const cr::MergeArgs&,        \
                                                  int64_t, cudaStream_t);
#define CR_INSTANTIATE_ORDER(K)                                                                \
    template cudaError_t cr::KeyOps<K>::merge_fwd_ord(int, int, bool, const cr::MergeArgs&,    \
                                                      int64_t, cudaStream_t);                  \
    template cudaError_t cr::KeyOps<K>::merge_fwd_rec_ord(int, int, const cr::MergeArgs&,      \
                                                          int64_t, cudaStream_t);              \
    template cudaError_t cr::KeyOps<K>::merge_bwd_ord(int, int, const cr::MergeArgs&, int64_t, \
                                                      cudaStream_t);
#define CR_INSTANTIATE_DESC(K)                                                                 \
    template cudaError_t cr::KeyOps<K>::merge_fwd_desc(int, int, bool, const cr::MergeArgs&,   \
                                                       int64_t, cudaStream_t);                 \
    template cudaError_t cr::KeyOps<K>::merge_fwd_rec_desc(int, int, const cr::MergeArgs&,     \
                                                           int64_t, cudaStream_t);             \
    template cudaError_t cr::KeyOps<K>::merge_bwd_desc(int, int, const cr::MergeArgs&, int64_t,\
                                                       cudaStream_t);
#define CR_INSTANTIATE_FLOAT(K)                                                                \
    template cudaError_t cr::KeyOps<K>::merge_fwd_flt(int, int, bool, const cr::MergeArgs&,    \
                                                      int64_t, cudaStream_t);                  \
    template cudaError_t cr::KeyOps<K>::merge_fwd_rec_flt(int, int, const cr::MergeArgs&,      \
                                                          int64_t, cudaStream_t);              \
    template cudaError_t cr::KeyOps<K>::merge_bwd_flt(int, int, const cr::MergeArgs&, int64_t, \
                                                      cudaStream_t);
#define CR_INSTANTIATE_RECORD(K)                                                               \
    template cudaError_t cr::KeyOps<K>::merge_fwd_rec(int, int, const cr::MergeArgs&, int64_t, \
                                                      cudaStream_t);
#define CR_INSTANTIATE_REST(K)                                                                 \
    template cudaError_t cr::KeyOps<K>::merge_bwd(int, int, const cr::MergeArgs&, int64_t,     \
                                                  cudaStream_t);                               \
    template cudaError_t cr::KeyOps<K>::partition_single(const void*, int64_t, const void*,    \
                                                         int64_t, int64_t, int64_t, void*,     \
                                                         int, cudaStream_t);                   \
    template cudaError_t cr::KeyOps<K>::partition_single_free(                                 \
        const void*, int64_t, const void*, int64_t, int64_t, int64_t, void*, int,              \
        cudaStream_t);                                                                         \
    template cudaError_t cr::KeyOps<K>::partition_pass(const void*, int64_t, int64_t, int64_t, \
                                                       void*, int64_t*, int, cudaStream_t);    \
    template cudaError_t cr::KeyOps<K>::partition_batched(                                     \
        const void*, const void*, const int64_t*, const int64_t*, int64_t, int64_t, int64_t,   \
        int64_t, int64_t, void*, int64_t*, int, cudaStream_t);                                 \
    template cudaError_t cr::KeyOps<K>::co_rank_many(const void*, int64_t, const void*,        \
                                                     int64_t, const int64_t*, int64_t,         \
                                                     int64_t*, int64_t*, int, cudaStream_t);   \
    template cudaError_t cr::KeyOps<K>::co_rank_one(const void*, int64_t, const void*,         \
                                                    int64_t, int64_t, int64_t*, int,           \
                                                    cudaStream_t);
