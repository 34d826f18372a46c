// cr_sort.cuh -- run formation for the bottom-up stable merge sort: every
// CTA stably sorts one run of R = NT*IPT consecutive elements (keys with
// their payloads) in shared memory, so that the merge passes can take over
// from runs of R.
//
//  1. coalesced load of the run's keys (and payloads) into shared memory;
//     every key is paired with its index inside the run (16 bits);
//  2. each thread sorts its IPT consecutive (key, index) pairs in registers
//     by odd-even transposition (adjacent swaps only when strictly greater:
//     stable);
//  3. log2(NT) rounds of in-block merges: round r merges neighbouring sorted
//     runs of IPT*2^r; each thread produces IPT outputs, co-ranking its
//     diagonal inside its pair of runs (the split of Lemma 1, binary lifting)
//     and merging serially with one index-selected load per step (ties take
//     the left run, which holds the earlier elements: stable);
//  4. coalesced store of the keys; the payloads are gathered once through
//     the carried indices (they never move during the rounds).
// Keys are mapped into the call's order on load and back on store
// (order_key).
//
// MODE 0: forward.  MODE 1: forward that also writes the run's permutation
// (perm[base + x] = input index inside the run of output x), for a backward
// that needs no keys.  MODE 2: backward by replay: the same sort on the
// input keys recovers the permutation, then gX[perm[x]] = gY[x] inside the
// run, scattered through shared memory.
#pragma once

#include "cr_device.cuh"
#include "cr_merge.cuh"

namespace cr {

template <class K, int VB, int MODE, int NT, int IPT>
struct SortLayout {
    static constexpr int R = NT * IPT;
    static_assert(R <= 65536, "run indices are 16-bit");
    // one element of slack: a merge step may read one past its pair
    static constexpr size_t KEYS = align_up_sz(size_t(R + 1) * sizeof(K), 128);
    static constexpr bool IDX = VB != 0 || MODE != 0;
    static constexpr size_t INDEX = IDX ? align_up_sz(size_t(R + 1) * 2, 128) : 0;
    // MODE 0/1: the input payloads; MODE 2: gradient staging
    static constexpr size_t VALS = VB ? align_up_sz(size_t(R) * VB, 128) : 0;
    static constexpr size_t TOTAL = 2 * (KEYS + INDEX) + VALS;
    static_assert(TOTAL <= 232448, "run does not fit shared memory");
};

template <class K, int VB, int MODE, int NT, int IPT>
__global__ void __launch_bounds__(NT) sort_runs_kernel(const K* __restrict__ X,
                                                       const void* __restrict__ Xv, int64_t N,
                                                       K* __restrict__ Y, void* __restrict__ Yv,
                                                       uint16_t* __restrict__ perm,
                                                       const void* __restrict__ gY,
                                                       void* __restrict__ gX, int order) {
    using L = SortLayout<K, VB, MODE, NT, IPT>;
    using V = typename VBits<VB>::T;
    constexpr bool IDX = L::IDX;
    constexpr int R = L::R;
    extern __shared__ __align__(128) unsigned char smem[];
    K* const sk0 = reinterpret_cast<K*>(smem);
    K* const sk1 = reinterpret_cast<K*>(smem + L::KEYS);
    uint16_t* const si0 = reinterpret_cast<uint16_t*>(smem + 2 * L::KEYS);
    uint16_t* const si1 = reinterpret_cast<uint16_t*>(smem + 2 * L::KEYS + L::INDEX);
    V* const sv = reinterpret_cast<V*>(smem + 2 * (L::KEYS + L::INDEX));

    const int tid = threadIdx.x;
    const int64_t base = int64_t(blockIdx.x) * R;
    const int len = int(N - base < R ? N - base : R);

    // 1. load
    for (int x = tid; x < len; x += NT) {
        sk0[x] = order_key(X[base + x], order);
        if constexpr (IDX) si0[x] = uint16_t(x);
        if constexpr (VB != 0 && MODE != 2) sv[x] = static_cast<const V*>(Xv)[base + x];
    }
    __syncthreads();

    // 2. per-thread stable sort of IPT elements (odd-even transposition)
    const int d0 = tid * IPT;
    const int cnt = d0 < len ? (len - d0 < IPT ? len - d0 : IPT) : 0;
    {
        K rk[IPT];
        uint16_t ri[IDX ? IPT : 1];
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (q < cnt) {
                rk[q] = sk0[d0 + q];
                if constexpr (IDX) ri[q] = si0[d0 + q];
            }
        }
#pragma unroll
        for (int round = 0; round < IPT; ++round) {
#pragma unroll
            for (int q = round & 1; q + 1 < IPT; q += 2) {
                if (q + 1 < cnt && rk[q + 1] < rk[q]) {
                    const K tk = rk[q];
                    rk[q] = rk[q + 1];
                    rk[q + 1] = tk;
                    if constexpr (IDX) {
                        const uint16_t tp = ri[q];
                        ri[q] = ri[q + 1];
                        ri[q + 1] = tp;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (q < cnt) {
                sk0[d0 + q] = rk[q];
                if constexpr (IDX) si0[d0 + q] = ri[q];
            }
        }
    }
    __syncthreads();

    // 3. merge rounds: runs of w -> 2w (2w is a multiple of IPT, so a
    //    thread's IPT outputs never straddle two pairs)
    int cur = 0;
    for (int w = IPT; w < len; w *= 2) {
        const K* ik = cur ? sk1 : sk0;
        const uint16_t* ii = cur ? si1 : si0;
        K* ok = cur ? sk0 : sk1;
        uint16_t* oi = cur ? si0 : si1;
        if (cnt > 0) {
            const int ps = (d0 / (2 * w)) * (2 * w);      // pair start
            const int alen = min(w, len - ps);
            const int blen = max(0, min(w, len - ps - alen));
            const int bs = ps + alen;                      // B run start
            const int dd[1] = {d0 - ps};
            int jj[1];
            split_in_tile<Log2Ceil<R + 1>::v>(ik + ps, alen, ik + bs, blen, dd, jj);
            int j = jj[0], k = dd[0] - j;
            // ik[bs + blen] is at most ik[len] <= ik[R]: inside the slack
            K a = ik[ps + j];
            K b = ik[bs + k];
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (q < cnt) {
                    const bool takeA = (k >= blen) || (j < alen && !(b < a));
                    const int src = takeA ? ps + j : bs + k;
                    ok[d0 + q] = takeA ? a : b;
                    if constexpr (IDX) oi[d0 + q] = ii[src];
                    j += takeA ? 1 : 0;
                    k += takeA ? 0 : 1;
                    const K nx = ik[takeA ? ps + j : bs + k];   // never taken when past a run
                    a = takeA ? nx : a;
                    b = takeA ? b : nx;
                }
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    const K* fk = cur ? sk1 : sk0;
    const uint16_t* fi = cur ? si1 : si0;

    // 4. store
    if constexpr (MODE != 2) {
        for (int x = tid; x < len; x += NT) {
            Y[base + x] = order_key_inverse(fk[x], order);
            if constexpr (VB != 0) static_cast<V*>(Yv)[base + x] = sv[fi[x]];
            if constexpr (MODE == 1) perm[base + x] = fi[x];
        }
    } else {
        // gradient: gX[perm[x]] = gY[x] within the run
        const V* gy = static_cast<const V*>(gY);
        for (int x = tid; x < len; x += NT) sv[fi[x]] = gy[base + x];
        __syncthreads();
        V* gx = static_cast<V*>(gX);
        for (int x = tid; x < len; x += NT) gx[base + x] = sv[x];
    }
}

}  // namespace cr
