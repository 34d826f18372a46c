// cr_partition.cuh -- kernels that place the output tiles: for every tile,
// the co-ranks of its first and last output rank over the arrays in HBM,
// written as a TileRec.  These are the "grid-level" co-rank passes; the
// merge kernel reads the records.  Single merges and merge passes share each
// tile boundary between its two tiles (block-level searches, then
// bisection); the batched partition searches each tile start once with
// Algorithm 1; the sync-free form gives every tile both of its ends, as each
// processing element does in Algorithm 2, with the two searches in lock step
// so that one round trip to memory serves both.  The list-of-ranks and
// single-rank co-rank kernels of the C ABI are here too.
#pragma once

#include "cr_device.cuh"

namespace cr {

// Algorithm 1 (Section 2), one iteration per call.  Paper notation: rank i,
// co-ranks j (into A) and k (into B), j + k = i (the C ABI calls the same
// triple (k; i, j)).  Starting from j = min(i, m) the search keeps j + k = i
// and lower bounds j_low, k_low, and halves [j_low, j] while the first
// Lemma-1 condition fails (A[j-1] > B[k]) or [k_low, k] while the second
// fails (B[k-1] >= A[j]).  The "conditional and" becomes index guards; the
// four candidate keys of an iteration are loaded together, one memory round
// trip per iteration.  k_low starts at the first k: the paper shows it is
// written before it is read (the first move is on the first condition).
// Callers cap the loop at 128 iterations (Proposition 1 bounds it by about
// log2 min(m, n) + 1 <= 64 for any int64 size) and every load is
// range-checked, so unsorted input can give a wrong split but never an
// out-of-range access or an endless loop; co_rank_end clamps the result to
// [max(0, i-n), min(i, m)].
struct CoRankState {
    int64_t j, k, j_low, k_low, j_min, j_max;
    bool done;
};

__device__ __forceinline__ CoRankState co_rank_begin(int64_t i, int64_t m, int64_t n) {
    CoRankState s;
    s.j = i < m ? i : m;
    s.k = i - s.j;
    s.j_low = i - n > 0 ? i - n : 0;
    s.k_low = s.k;
    s.j_min = s.j_low;
    s.j_max = s.j;
    s.done = false;
    return s;
}

// A and B are key views (KeyView: keys mapped into the call's order).
template <class V>
__device__ __forceinline__ void co_rank_step(CoRankState& s, V A, int64_t m, V B, int64_t n) {
    using K = typename V::key_type;
    if (s.done) return;
    const int64_t j = s.j, k = s.k;
    const bool okA1 = j > 0 && j - 1 < m;
    const bool okB0 = k >= 0 && k < n;
    const bool okB1 = k > 0 && k - 1 < n;
    const bool okA0 = j >= 0 && j < m;
    const K a1 = okA1 ? A[j - 1] : K(0);
    const K b0 = okB0 ? B[k] : K(0);
    const K b1 = okB1 ? B[k - 1] : K(0);
    const K a0 = okA0 ? A[j] : K(0);
    if (okA1 && okB0 && a1 > b0) {             // first Lemma condition violated
        const int64_t d = (j - s.j_low + 1) >> 1;
        s.k_low = k;
        s.j = j - d;
        s.k = k + d;
    } else if (okB1 && okA0 && b1 >= a0) {     // second Lemma condition violated
        const int64_t d = (k - s.k_low + 1) >> 1;
        s.j_low = j;
        s.j = j + d;
        s.k = k - d;
    } else {
        s.done = true;
    }
}

__device__ __forceinline__ int64_t co_rank_end(const CoRankState& s) {
    int64_t j = s.j < s.j_min ? s.j_min : s.j;
    return j > s.j_max ? s.j_max : j;
}

// Co-ranks of ranks r0 and r1 of one merge problem, searched together.
template <class V>
__device__ __forceinline__ void co_rank_pair(int64_t r0, int64_t r1, V A, int64_t m, V B,
                                             int64_t n, int64_t& j0, int64_t& j1) {
    CoRankState s0 = co_rank_begin(r0, m, n);
    CoRankState s1 = co_rank_begin(r1, m, n);
#pragma unroll 1
    for (int it = 0; it < 128 && !(s0.done && s1.done); ++it) {
        co_rank_step(s0, A, m, B, n);
        co_rank_step(s1, A, m, B, n);
    }
    j0 = co_rank_end(s0);
    j1 = co_rank_end(s1);
}

__device__ __forceinline__ TileRec make_rec(int64_t a_base, int64_t b_base, int64_t c_base,
                                            int64_t r0, int64_t r1, int64_t j0, int64_t j1) {
    TileRec r;
    r.ga = a_base + j0;
    r.gb = b_base + (r0 - j0);
    r.gc = c_base + r0;
    r.alen = int32_t(j1 - j0);
    r.blen = int32_t((r1 - j1) - (r0 - j0));
    return r;
}

// Co-rank of output rank i by a group of G lanes (mask `gmask`, this lane's
// index `l` in the group): the largest j in [max(0, i-n), min(i, m)] for
// which the first Lemma-1 condition holds (A[j-1] <= B[i-j], with B[n] =
// +inf); the condition holds exactly for j <= j*, so G probes per round cut
// the interval (G+1)-fold.
template <class V, int G>
__device__ __forceinline__ int64_t co_rank_group(V A, int64_t m, V B, int64_t n, int64_t i,
                                                 int l, unsigned gmask, int gshift) {
    int64_t lo = i - n > 0 ? i - n : 0;
    int64_t hi = i < m ? i : m;
#pragma unroll 1
    for (int round = 0; round < 64 && hi > lo; ++round) {
        const int64_t w = hi - lo;
        const int64_t p = lo + ((int64_t(l) + 1) * w + G - 1) / G;   // in (lo, hi]
        const int64_t k = i - p;                                     // in [0, n]
        const bool c1 = (k >= n) || !(B[k] < A[p - 1]);
        const unsigned ball = (__ballot_sync(gmask, c1) >> gshift) & ((1u << G) - 1u);
        const int cnt = __popc(ball);   // the condition holds on a prefix of the probes
        if (cnt == 0) {
            hi = lo + (w + G - 1) / G - 1;
        } else {
            const int64_t plast = lo + (int64_t(cnt) * w + G - 1) / G;
            if (cnt < G) hi = lo + ((int64_t(cnt) + 1) * w + G - 1) / G - 1;
            lo = plast;
        }
    }
    return lo;
}

// Single merge: tile t covers output ranks [t*tile, min((t+1)*tile, m+n)).
// A block of 256 threads handles 256 consecutive tile boundaries (255 tiles;
// neighbouring blocks share one boundary), in two steps:
//  1. the producer-style warp 0 co-ranks the block's first and last boundary
//     (16 lanes each, co_rank_group), giving the block's A interval
//     [jb0, jb1] that contains every co-rank the block needs;
//  2. every thread bisects that common interval for its own boundary on the
//     first Lemma-1 condition.  All threads start from the same interval, so
//     the top levels of their searches probe the same few positions (L1 and
//     L2 hits) and only the last levels touch distinct DRAM sectors.
template <class K>
__global__ void __launch_bounds__(256) partition_single_kernel(const K* Ap, int64_t m,
                                                               const K* Bp, int64_t n,
                                                               int64_t tile, int64_t ntiles,
                                                               void* ws, int order) {
    const KeyView<K> A{Ap, order}, B{Bp, order};
    __shared__ int64_t s_j[256];
    __shared__ int64_t s_jb[2];
    const int64_t mn = m + n;
    const int64_t tb = int64_t(blockIdx.x) * 255;
    const int64_t t = tb + threadIdx.x;   // boundary index
    if (t == 0) {
        WsHeader* h = static_cast<WsHeader*>(ws);
        h->status = kDevOk;
        h->tile = int32_t(tile);
        h->ntiles = ntiles;
    }
    if (threadIdx.x < 32) {
        const int grp = threadIdx.x >> 4;
        const int64_t tt = grp == 0 ? tb : (tb + 255 < ntiles ? tb + 255 : ntiles);
        const int64_t i = tt * tile < mn ? tt * tile : mn;
        const int64_t j = co_rank_group<KeyView<K>, 16>(A, m, B, n, i, threadIdx.x & 15,
                                                        0xFFFFu << (16 * grp), 16 * grp);
        if ((threadIdx.x & 15) == 0) s_jb[grp] = j;
    }
    __syncthreads();
    if (t <= ntiles) {
        const int64_t i = t * tile < mn ? t * tile : mn;
        // largest j in [jb0, jb1] with the first condition true at (j, i-j);
        // k > n counts as true (B[n] = +inf), k < 0 as false (j > i).
        int64_t lo = s_jb[0], hi = s_jb[1];
#pragma unroll 1
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;   // > lo >= 0
            const int64_t k = i - mid;
            const bool c1 = k >= n || (k >= 0 && !(B[k] < A[mid - 1]));
            if (c1) lo = mid; else hi = mid - 1;
        }
        s_j[threadIdx.x] = lo;
    }
    __syncthreads();
    if (threadIdx.x < 255 && t < ntiles) {
        const int64_t r0 = t * tile;
        const int64_t r1 = r0 + tile < mn ? r0 + tile : mn;
        ws_recs(ws)[t] = make_rec(0, 0, 0, r0, r1, s_j[threadIdx.x], s_j[threadIdx.x + 1]);
    }
}

// Single merge with few tiles: every tile start is co-ranked by its own
// group of 16 lanes (co_rank_group over the whole range), so the search takes
// about log17 of the range in dependent rounds instead of the block-end
// search followed by a bisection.  A block of 256 threads (16 groups) owns
// tiles tb .. tb+14 and the 16 starts tb .. tb+15.  Used when the merge has
// few tiles (the extra probes are then a few MB at most); same records as
// partition_single_kernel.
template <class K>
__global__ void __launch_bounds__(256) partition_single_small_kernel(const K* Ap, int64_t m,
                                                                     const K* Bp, int64_t n,
                                                                     int64_t tile, int64_t ntiles,
                                                                     void* ws, int order) {
    const KeyView<K> A{Ap, order}, B{Bp, order};
    __shared__ int64_t s_j[16];
    const int64_t mn = m + n;
    const int grp = threadIdx.x >> 4;
    const int64_t tb = int64_t(blockIdx.x) * 15;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        WsHeader* h = static_cast<WsHeader*>(ws);
        h->status = kDevOk;
        h->tile = int32_t(tile);
        h->ntiles = ntiles;
    }
    const int64_t tt = tb + grp < ntiles ? tb + grp : ntiles;   // boundary of this group
    const int64_t i = tt * tile < mn ? tt * tile : mn;
    const unsigned gmask = 0xFFFFu << (16 * (grp & 1));
    const int64_t j = co_rank_group<KeyView<K>, 16>(A, m, B, n, i, threadIdx.x & 15, gmask,
                                                    16 * (grp & 1));
    if ((threadIdx.x & 15) == 0) s_j[grp] = j;
    __syncthreads();
    const int64_t t = tb + threadIdx.x;
    if (threadIdx.x < 15 && t < ntiles) {
        const int64_t r0 = t * tile;
        const int64_t r1 = r0 + tile < mn ? r0 + tile : mn;
        ws_recs(ws)[t] = make_rec(0, 0, 0, r0, r1, s_j[threadIdx.x], s_j[threadIdx.x + 1]);
    }
}

// Single merge, sync-free form of Algorithm 2: tile t co-ranks both of its
// ends itself with Algorithm 1 as printed (the two searches in lock step),
// sharing nothing with other tiles.  Same records as partition_single_kernel.
template <class K>
__global__ void __launch_bounds__(256) partition_single_free_kernel(const K* Ap, int64_t m,
                                                                    const K* Bp, int64_t n,
                                                                    int64_t tile, int64_t ntiles,
                                                                    void* ws, int order) {
    const KeyView<K> A{Ap, order}, B{Bp, order};
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t == 0) {
        WsHeader* h = static_cast<WsHeader*>(ws);
        h->status = kDevOk;
        h->tile = int32_t(tile);
        h->ntiles = ntiles;
    }
    if (t >= ntiles) return;
    const int64_t r0 = t * tile;
    const int64_t r1 = r0 + tile < m + n ? r0 + tile : m + n;
    int64_t j0, j1;
    co_rank_pair(r0, r1, A, m, B, n, j0, j1);
    ws_recs(ws)[t] = make_rec(0, 0, 0, r0, r1, j0, j1);
}

// One bottom-up merge-sort pass over X[0, N): pair q merges the runs
// X[2qw, 2qw+w) and X[2qw+w, 2qw+2w) (cut at N).  Tiles never straddle pairs;
// every pair but the last has tpp = ceil(2w / tile) tiles.
//
// The two steps of partition_single_kernel, applied pair by pair: a block of
// 256 threads owns tiles tb .. tb+254 and the 256 tile starts tb .. tb+255.
//  1. warp 0 co-ranks the first and the last of those starts inside their
//     own pairs (16 lanes each, co_rank_group);
//  2. every thread bisects for its own start between the trivial bounds of
//     its pair, [max(0, r-n), min(r, m)], narrowed by step 1's co-ranks when
//     it shares their pair (co-ranks grow with the rank inside a pair).
// A tile ends where the next tile of its pair starts, or at the pair's end,
// whose co-rank is m.
struct PassPos {
    int64_t q, r, m, n;   // pair, rank inside the pair, run lengths
};

__device__ __forceinline__ PassPos pass_locate(int64_t tt, int64_t N, int64_t w, int64_t tile,
                                               int64_t tpp, int64_t npairs) {
    PassPos p;
    p.q = tt / tpp;
    if (p.q > npairs - 1) p.q = npairs - 1;   // tt == ntiles: end of the last pair
    const int64_t a0 = 2 * p.q * w;
    p.m = w < N - a0 ? w : N - a0;
    const int64_t nb = N - a0 - p.m;
    p.n = w < nb ? w : nb;
    p.r = (tt - p.q * tpp) * tile;
    if (p.r > p.m + p.n) p.r = p.m + p.n;
    return p;
}

template <class K>
__global__ void __launch_bounds__(256) partition_pass_kernel(const K* Xp, int64_t N, int64_t w,
                                                             int64_t tile, int64_t tpp,
                                                             int64_t npairs, int64_t ntiles,
                                                             void* ws, int order) {
    const KeyView<K> X{Xp, order};
    __shared__ int64_t s_j[256];
    __shared__ int64_t s_jb[2];
    __shared__ int64_t s_qb[2];
    const int64_t tb = int64_t(blockIdx.x) * 255;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        WsHeader* h = static_cast<WsHeader*>(ws);
        h->status = kDevOk;
        h->tile = int32_t(tile);
        h->ntiles = ntiles;
    }
    if (threadIdx.x < 32) {
        const int grp = threadIdx.x >> 4;
        const int64_t tt = grp == 0 ? tb : (tb + 255 < ntiles ? tb + 255 : ntiles);
        const PassPos p = pass_locate(tt, N, w, tile, tpp, npairs);
        const KeyView<K> A = X + 2 * p.q * w;
        const int64_t j = co_rank_group<KeyView<K>, 16>(A, p.m, A + p.m, p.n, p.r,
                                                        threadIdx.x & 15,
                                                        0xFFFFu << (16 * grp), 16 * grp);
        if ((threadIdx.x & 15) == 0) {
            s_jb[grp] = j;
            s_qb[grp] = p.q;
        }
    }
    __syncthreads();
    const int64_t tt = tb + threadIdx.x;
    if (tt <= ntiles) {
        const PassPos p = pass_locate(tt, N, w, tile, tpp, npairs);
        const KeyView<K> A = X + 2 * p.q * w;
        const KeyView<K> B = A + p.m;
        int64_t lo = p.r - p.n > 0 ? p.r - p.n : 0;
        int64_t hi = p.r < p.m ? p.r : p.m;
        if (p.q == s_qb[0] && s_jb[0] > lo) lo = s_jb[0];
        if (p.q == s_qb[1] && s_jb[1] < hi) hi = s_jb[1];
        // largest j in [lo, hi] with the first condition true at (j, r-j)
#pragma unroll 1
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;   // > lo >= 0
            const int64_t k = p.r - mid;
            const bool c1 = k >= p.n || (k >= 0 && !(B[k] < A[mid - 1]));
            if (c1) lo = mid; else hi = mid - 1;
        }
        s_j[threadIdx.x] = lo;
    }
    __syncthreads();
    if (threadIdx.x < 255 && tt < ntiles) {
        const PassPos p = pass_locate(tt, N, w, tile, tpp, npairs);
        const int64_t r1 = p.r + tile < p.m + p.n ? p.r + tile : p.m + p.n;
        const int64_t j1 = r1 == p.m + p.n ? p.m : s_j[threadIdx.x + 1];
        const int64_t a0 = 2 * p.q * w;
        ws_recs(ws)[tt] = make_rec(a0, a0 + p.m, a0, p.r, r1, s_j[threadIdx.x], j1);
    }
}

// Batched merge, step 1 (one CTA of 1024 threads): validate the segment
// tables and write prefix[s] = number of tiles of segments 0..s-1 (tiles of
// segment s: ceil((m_s + n_s) / tile)), prefix[nseg] = total tiles.  On an
// invalid table the status word becomes kDevBadSeg and the tile count 0.
static __global__ void __launch_bounds__(1024) segment_scan_kernel(const int64_t* a_off,
                                                            const int64_t* b_off, int64_t nseg,
                                                            int64_t a_total, int64_t b_total,
                                                            int64_t tile, void* ws,
                                                            int64_t* prefix) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t s_carry;
    __shared__ int s_bad;
    constexpr int IT = 8;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_carry = 0;
        s_bad = (a_off[0] != 0 || b_off[0] != 0 || a_off[nseg] > a_total ||
                 b_off[nseg] > b_total) ? 1 : 0;
    }
    __syncthreads();
    for (int64_t base = 0; base < nseg; base += 1024 * IT) {
        int64_t cnt[IT];
        int64_t mine = 0;
        bool bad = false;   // kept in a register: no shared store between the loads
#pragma unroll
        for (int e = 0; e < IT; ++e) {
            const int64_t s = base + int64_t(tid) * IT + e;
            cnt[e] = 0;
            if (s < nseg) {
                const int64_t ms = a_off[s + 1] - a_off[s];
                const int64_t ns = b_off[s + 1] - b_off[s];
                if (ms < 0 || ns < 0) bad = true;
                else cnt[e] = (ms + ns + tile - 1) / tile;
            }
            mine += cnt[e];
        }
        if (bad) s_bad = 1;
        // block-wide exclusive scan of `mine`
        int64_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((tid & 31) >= o) incl += v;
        }
        if ((tid & 31) == 31) warp_tot[tid >> 5] = incl;
        __syncthreads();
        if (tid < 32) {
            int64_t w = warp_tot[tid];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t v = __shfl_up_sync(0xffffffffu, w, o);
                if (tid >= o) w += v;
            }
            warp_tot[tid] = w;   // inclusive over warps
        }
        __syncthreads();
        int64_t run = s_carry + (incl - mine) + ((tid >> 5) ? warp_tot[(tid >> 5) - 1] : 0);
#pragma unroll
        for (int e = 0; e < IT; ++e) {
            const int64_t s = base + int64_t(tid) * IT + e;
            if (s < nseg) prefix[s] = run;
            run += cnt[e];
        }
        __syncthreads();
        if (tid == 0) s_carry += warp_tot[31];
        __syncthreads();
    }
    if (tid == 0) {
        prefix[nseg] = s_carry;
        WsHeader* h = static_cast<WsHeader*>(ws);
        h->status = s_bad ? kDevBadSeg : kDevOk;
        h->tile = int32_t(tile);
        h->ntiles = s_bad ? 0 : s_carry;
    }
}

// Batched merge, step 2: a block of 256 threads owns tiles tb .. tb+254
// (tb = 255 * blockIdx.x) and the 256 tile starts tb .. tb+255.  Thread i
// finds the segment of tile tb + i in the tile prefix (binary search) and
// co-ranks that tile's start inside its segment with Algorithm 1 as printed;
// a tile ends where the next tile of its segment starts (the neighbouring
// thread's co-rank) or at its segment's end, whose co-rank is m.  So every
// tile start is searched once.
template <class K>
__global__ void __launch_bounds__(256) partition_batched_kernel(
    const K* Ap, const K* Bp, const int64_t* a_off, const int64_t* b_off, int64_t nseg,
    int64_t tile, const int64_t* prefix, void* ws, int order) {
    const KeyView<K> A{Ap, order}, B{Bp, order};
    __shared__ int64_t s_j[256];
    __shared__ int64_t s_seg[256];
    const int64_t ntiles = static_cast<const WsHeader*>(ws)->ntiles;
    const int64_t t = int64_t(blockIdx.x) * 255 + threadIdx.x;
    int64_t seg = -1, a0 = 0, b0 = 0, m = 0, n = 0, r0 = 0;
    if (t < ntiles) {
        // largest s < nseg with prefix[s] <= t (empty segments are skipped)
        int64_t lo = 0, hi = nseg;   // invariant: prefix[lo] <= t < prefix[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (prefix[mid] <= t) lo = mid; else hi = mid;
        }
        seg = lo;
        a0 = a_off[seg];
        b0 = b_off[seg];
        m = a_off[seg + 1] - a0;
        n = b_off[seg + 1] - b0;
        r0 = (t - prefix[seg]) * tile;
        CoRankState st = co_rank_begin(r0, m, n);
#pragma unroll 1
        for (int it = 0; it < 128 && !st.done; ++it) co_rank_step(st, A + a0, m, B + b0, n);
        s_j[threadIdx.x] = co_rank_end(st);
    }
    s_seg[threadIdx.x] = seg;   // -1: no tile starts here
    __syncthreads();
    if (threadIdx.x < 255 && t < ntiles) {
        // tile t + 1 exists and lies in this segment: it starts where t ends
        const bool next_same = s_seg[threadIdx.x + 1] == seg;
        const int64_t r1 = next_same ? r0 + tile : m + n;
        const int64_t j1 = next_same ? s_j[threadIdx.x + 1] : m;
        ws_recs(ws)[t] = make_rec(a0, b0, a0 + b0, r0, r1, s_j[threadIdx.x], j1);
    }
}

// co_rank for a list of ranks (C-ABI names: rank k -> (i, j)).
template <class K>
__global__ void co_rank_many_kernel(const K* Ap, int64_t m, const K* Bp, int64_t n,
                                    const int64_t* ranks, int64_t cnt, int64_t* out_i,
                                    int64_t* out_j, int order) {
    const KeyView<K> A{Ap, order}, B{Bp, order};
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    const int64_t r = ranks[q];
    if (r < 0 || r > m + n) {
        out_i[q] = -1;
        out_j[q] = -1;
        return;
    }
    CoRankState s = co_rank_begin(r, m, n);
#pragma unroll 1
    for (int it = 0; it < 128 && !s.done; ++it) co_rank_step(s, A, m, B, n);
    const int64_t j = co_rank_end(s);
    out_i[q] = j;
    out_j[q] = r - j;
}

// One rank, result as two int64 (i, j) in device memory.
template <class K>
__global__ void co_rank_one_kernel(const K* Ap, int64_t m, const K* Bp, int64_t n, int64_t r,
                                   int64_t* out_ij, int order) {
    const KeyView<K> A{Ap, order}, B{Bp, order};
    CoRankState s = co_rank_begin(r, m, n);
#pragma unroll 1
    for (int it = 0; it < 128 && !s.done; ++it) co_rank_step(s, A, m, B, n);
    const int64_t j = co_rank_end(s);
    out_ij[0] = j;
    out_ij[1] = r - j;
}

}  // namespace cr
