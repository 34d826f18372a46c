// cr_sort.cuh -- run formation for the bottom-up stable merge sort: every
// CTA stably sorts one run of R = NT*IPT consecutive elements (keys with
// their payloads) in shared memory, so that the merge passes can take over
// from runs of R.
//
//  1. coalesced load of the run into shared memory;
//  2. each thread sorts its IPT consecutive elements in registers by odd-even
//     transposition (adjacent swaps only when strictly greater: stable);
//  3. log2(NT) rounds of in-block merges: round r merges neighbouring sorted
//     runs of IPT*2^r; each thread produces IPT outputs, co-ranking its
//     diagonal inside its pair of runs (the split of Lemma 1, binary lifting)
//     and merging serially (ties take the left run, which holds the earlier
//     elements: stable);
//  4. coalesced store.
//
// Backward (payload gradient of the run sort): the same sort is replayed on
// (key, local index) pairs to recover the permutation, then gX[perm[x]] =
// gY[x] inside the run, scattered through shared memory.
#pragma once

#include "cr_device.cuh"
#include "cr_merge.cuh"

namespace cr {

template <class K, int VB, bool BWD, int NT, int IPT>
struct SortLayout {
    static constexpr int R = NT * IPT;
    // payload carried through the rounds: the values (forward) or the
    // element's index inside the run (backward)
    using P = typename std::conditional<BWD, uint32_t, typename VBits<VB>::T>::type;
    static constexpr bool CARRY = BWD || VB != 0;
    static constexpr size_t KEYS = align_up_sz(size_t(R) * sizeof(K), 128);
    static constexpr size_t PAY = CARRY ? align_up_sz(size_t(R) * sizeof(P), 128) : 0;
    static constexpr size_t GRAD = BWD ? align_up_sz(size_t(R) * (VB ? VB : 4), 128) * 2 : 0;
    static constexpr size_t TOTAL = 2 * (KEYS + PAY) + GRAD + 128;
    static_assert(TOTAL <= 232448, "run does not fit shared memory");
};

template <class K, int VB, bool BWD, int NT, int IPT>
__global__ void __launch_bounds__(NT) sort_runs_kernel(const K* __restrict__ X,
                                                       const void* __restrict__ Xv, int64_t N,
                                                       K* __restrict__ Y, void* __restrict__ Yv,
                                                       const void* __restrict__ gY,
                                                       void* __restrict__ gX) {
    using L = SortLayout<K, VB, BWD, NT, IPT>;
    using P = typename L::P;
    using V = typename VBits<VB>::T;
    constexpr int R = L::R;
    extern __shared__ __align__(128) unsigned char smem[];
    K* sk[2] = {reinterpret_cast<K*>(smem), reinterpret_cast<K*>(smem + L::KEYS)};
    P* sp[2] = {reinterpret_cast<P*>(smem + 2 * L::KEYS),
                reinterpret_cast<P*>(smem + 2 * L::KEYS + L::PAY)};

    const int tid = threadIdx.x;
    const int64_t base = int64_t(blockIdx.x) * R;
    const int len = int(N - base < R ? N - base : R);

    // 1. load
    for (int x = tid; x < len; x += NT) {
        sk[0][x] = X[base + x];
        if constexpr (L::CARRY) {
            if constexpr (BWD) sp[0][x] = uint32_t(x);
            else sp[0][x] = static_cast<const V*>(Xv)[base + x];
        }
    }
    __syncthreads();

    // 2. per-thread stable sort of IPT elements (odd-even transposition)
    const int d0 = tid * IPT;
    const int cnt = d0 < len ? (len - d0 < IPT ? len - d0 : IPT) : 0;
    {
        K rk[IPT];
        P rp[L::CARRY ? IPT : 1];
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (q < cnt) {
                rk[q] = sk[0][d0 + q];
                if constexpr (L::CARRY) rp[q] = sp[0][d0 + q];
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
                    if constexpr (L::CARRY) {
                        const P tp = rp[q];
                        rp[q] = rp[q + 1];
                        rp[q + 1] = tp;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (q < cnt) {
                sk[0][d0 + q] = rk[q];
                if constexpr (L::CARRY) sp[0][d0 + q] = rp[q];
            }
        }
    }
    __syncthreads();

    // 3. merge rounds: runs of w -> 2w (2w is a multiple of IPT, so a
    //    thread's IPT outputs never straddle two pairs)
    int cur = 0;
    for (int w = IPT; w < len; w *= 2) {
        const K* ik = sk[cur];
        const P* ip = sp[cur];
        K* ok = sk[cur ^ 1];
        P* op = sp[cur ^ 1];
        if (cnt > 0) {
            const int ps = (d0 / (2 * w)) * (2 * w);      // pair start
            const int alen = min(w, len - ps);
            const int blen = max(0, min(w, len - ps - alen));
            const K* sA = ik + ps;
            const K* sB = ik + ps + alen;
            const int dd[1] = {d0 - ps};
            int jj[1];
            split_in_tile<Log2Ceil<R + 1>::v>(sA, alen, sB, blen, dd, jj);
            int j = jj[0], k = dd[0] - j;
            K a = j < alen ? sA[j] : K(0);
            K b = k < blen ? sB[k] : K(0);
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (q < cnt) {
                    const bool takeA = (k >= blen) || (j < alen && !(b < a));
                    ok[d0 + q] = takeA ? a : b;
                    if constexpr (L::CARRY) op[d0 + q] = takeA ? ip[ps + j] : ip[ps + alen + k];
                    j += takeA ? 1 : 0;
                    k += takeA ? 0 : 1;
                    if (takeA) {
                        if (j < alen) a = sA[j];
                    } else {
                        if (k < blen) b = sB[k];
                    }
                }
            }
        }
        __syncthreads();
        cur ^= 1;
    }

    // 4. store
    if constexpr (!BWD) {
        for (int x = tid; x < len; x += NT) {
            Y[base + x] = sk[cur][x];
            if constexpr (VB != 0) static_cast<V*>(Yv)[base + x] = sp[cur][x];
        }
    } else {
        // gradient: gX[perm[x]] = gY[x] within the run
        V* g0 = reinterpret_cast<V*>(smem + 2 * (L::KEYS + L::PAY));
        V* g1 = reinterpret_cast<V*>(smem + 2 * (L::KEYS + L::PAY) + L::GRAD / 2);
        const V* gy = static_cast<const V*>(gY);
        for (int x = tid; x < len; x += NT) g0[x] = gy[base + x];
        __syncthreads();
        for (int x = tid; x < len; x += NT) g1[sp[cur][x]] = g0[x];
        __syncthreads();
        V* gx = static_cast<V*>(gX);
        for (int x = tid; x < len; x += NT) gx[base + x] = g1[x];
    }
}

}  // namespace cr
