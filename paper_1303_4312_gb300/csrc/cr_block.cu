// cr_block.cu -- the first passes of a bottom-up merge sort whose runs are
// short, merged inside shared memory: each CTA loads a chunk of R = 4096
// consecutive elements (R / w runs of a power-of-two width w <= R/2), runs
// the passes w -> 2w -> ... -> R in shared memory, and stores the chunk once,
// instead of one pass over HBM per width.  Same result as those passes
// (stable merges of neighbouring runs; ties take the left run).
//
// Work split: thread t of NT = R / IPT owns the outputs [t IPT, (t+1) IPT)
// of every round (IPT = 8); since 2w is a multiple of IPT they lie in one
// pair of runs.  A thread co-ranks the start of its range inside its pair
// (the split of Lemma 1, binary lifting) and merges IPT steps serially.  Keys
// carry their 16-bit index in the chunk; the payloads are gathered once at
// the end through those indices, and with `perm` the indices are written
// out, so that the backward routes gradients through them without keys.
//
// Shared-memory layout: element i of a key array sits at slot
// i + i / 16 (8-byte keys) or i + i / 32 (4-byte keys), element i of an index
// array at i + 2 (i / 64).  With those gaps the IPT-strided writes of a warp
// (and its linear loads and stores) fall in distinct banks, although the
// stride IPT and the chunk length are powers of two.
//
// Run formation (w < IPT, FORM): every thread first sorts its own group of
// IPT consecutive elements stably in registers (odd-even transposition,
// swaps only on strictly smaller), which equals the merges of widths
// w .. IPT/2 (a stable merge's result is unique), and the rounds start at
// IPT; with w = 1 this sorts any input into sorted runs of R.
//
// MODE 0: forward.  MODE 1: forward that also writes the chunk permutation.
// MODE 2 (run formation only): backward by replay -- the same sort of the
// input keys recovers the permutation, and gX[base + perm[x]] = gY[base + x]
// is scattered through shared memory.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/corank.h"
#include "cr_launch.cuh"
#include "cr_merge.cuh"

namespace cr {
namespace {

constexpr int kBlockR = 4096;
constexpr int kBlockIPT = 8;
constexpr int kBlockNT = kBlockR / kBlockIPT;   // 512
// merge rounds start at width >= IPT (below it, FORM sorts groups of IPT),
// so 2w is a multiple of IPT and a thread's outputs lie in one pair
static_assert(kBlockR == kSortRun, "run formation sorts chunks of the merge stage");

template <class K>
struct BlockSlots {
    static constexpr int SHIFT = sizeof(K) == 8 ? 4 : 5;
    static __device__ __forceinline__ int key(int i) { return i + (i >> SHIFT); }
    static __device__ __forceinline__ int idx(int i) { return i + ((i >> 6) << 1); }
    // slot of element R included: a merge step may read one past its pair
    static constexpr int KEYS = kBlockR + (kBlockR >> SHIFT) + 1;
    static constexpr int IDX = kBlockR + ((kBlockR >> 6) << 1) + 1;
    static_assert((1 << SHIFT) % kBlockIPT == 0 && 64 % kBlockIPT == 0,
                  "the IPT outputs of a thread never straddle a gap");
};

template <class K, int VB>
struct BlockLayout {
    using S = BlockSlots<K>;
    static constexpr size_t KEYS = align_up_sz(size_t(S::KEYS) * sizeof(K), 128);
    static constexpr size_t INDEX = align_up_sz(size_t(S::IDX) * 2, 128);
    static constexpr size_t VALS = VB ? align_up_sz(size_t(kBlockR) * VB, 128) : 0;
    static constexpr size_t TOTAL = 2 * (KEYS + INDEX) + VALS;
    static_assert(TOTAL <= 232448, "chunk does not fit shared memory");
};

// Largest j in [max(0, d - blen), min(d, alen)] with A[j-1] <= B[d-j]
// (Lemma 1's first condition; A = s[pa ..], B = s[pb ..] in logical
// indices), by binary lifting with steps w, w/2, ..., 1: the interval is at
// most w long (alen, blen <= w, a power of two), so a round of width w
// takes log2(w) + 1 steps, the same for every thread of the round.
template <class K>
__device__ __forceinline__ int split_pair(const K* s, int pa, int alen, int pb, int blen, int d,
                                          int w) {
    using S = BlockSlots<K>;
    int pos = d - blen > 0 ? d - blen : 0;
    const int hi = d < alen ? d : alen;
#pragma unroll 4
    for (int step = w; step > 0; step >>= 1) {
        const int np = pos + step;
        if (np <= hi && !(s[S::key(pb + d - np)] < s[S::key(pa + np - 1)])) pos = np;
    }
    return pos;
}

template <class K, int VB, int MODE, bool FORM>
__global__ void __launch_bounds__(kBlockNT, 2) merge_runs_block_kernel(
    const K* __restrict__ X, const void* __restrict__ Xv, int64_t N, int w0, K* __restrict__ Y,
    void* __restrict__ Yv, uint16_t* __restrict__ perm, const void* __restrict__ gY,
    void* __restrict__ gX, int order) {
    static_assert(MODE != 2 || (FORM && VB != 0), "replay backward: run formation, payloads");
    using L = BlockLayout<K, VB>;
    using S = BlockSlots<K>;
    using V = typename VBits<VB>::T;
    constexpr int IPT = kBlockIPT;
    // Chunk positions ride along with the keys only when something reads
    // them at the end: payloads, the permutation or the replay backward.
    constexpr bool IDX = VB != 0 || MODE != 0;
    extern __shared__ __align__(128) unsigned char smem[];
    K* const sk0 = reinterpret_cast<K*>(smem);
    K* const sk1 = reinterpret_cast<K*>(smem + L::KEYS);
    uint16_t* const si0 = reinterpret_cast<uint16_t*>(smem + 2 * L::KEYS);
    uint16_t* const si1 = reinterpret_cast<uint16_t*>(smem + 2 * L::KEYS + L::INDEX);
    V* const sv = reinterpret_cast<V*>(smem + 2 * (L::KEYS + L::INDEX));

    const int tid = threadIdx.x;
    const int64_t base = int64_t(blockIdx.x) * kBlockR;
    const int len = int(N - base < kBlockR ? N - base : kBlockR);

    for (int x = tid; x < len; x += kBlockNT) {
        sk0[S::key(x)] = order_key(X[base + x], order);
        if constexpr (IDX) si0[S::idx(x)] = uint16_t(x);
        if constexpr (VB != 0 && MODE != 2) sv[x] = static_cast<const V*>(Xv)[base + x];
    }
    __syncthreads();

    const int d0 = tid * IPT;
    const int cnt = d0 < len ? (len - d0 < IPT ? len - d0 : IPT) : 0;
    if constexpr (FORM) {
        K rk[IPT];
        uint16_t ri[IPT];
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (q < cnt) {
                rk[q] = sk0[S::key(d0 + q)];
                ri[q] = uint16_t(d0 + q);
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
                        const uint16_t ti = ri[q];
                        ri[q] = ri[q + 1];
                        ri[q + 1] = ti;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (q < cnt) {
                sk0[S::key(d0 + q)] = rk[q];
                if constexpr (IDX) si0[S::idx(d0 + q)] = ri[q];
            }
        }
        __syncthreads();
    }

    int cur = 0;
    for (int w = FORM ? IPT : w0; w < len; w *= 2) {
        const K* ik = cur ? sk1 : sk0;
        const uint16_t* ii = cur ? si1 : si0;
        K* ok = cur ? sk0 : sk1;
        uint16_t* oi = cur ? si0 : si1;
        if (cnt > 0) {
            const int ps = (d0 / (2 * w)) * (2 * w);     // pair start
            const int alen = min(w, len - ps);
            const int blen = max(0, min(w, len - ps - alen));
            const int bs = ps + alen;
            const int d = d0 - ps;
            int j = split_pair<K>(ik, ps, alen, bs, blen, d, w);
            int k = d - j;
            K a = ik[S::key(ps + j)];     // at most element len <= R: the slack slot
            K b = ik[S::key(bs + k)];
            // a thread's IPT outputs are consecutive slots (no gap inside them)
            K* const okt = ok + S::key(d0);
            uint16_t* const oit = oi + S::idx(d0);
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (q < cnt) {
                    const bool takeA = (k >= blen) || (j < alen && !(b < a));
                    const int src = takeA ? ps + j : bs + k;
                    okt[q] = takeA ? a : b;
                    if constexpr (IDX) oit[q] = ii[S::idx(src)];
                    j += takeA ? 1 : 0;
                    k += takeA ? 0 : 1;
                    const K nx = ik[S::key(takeA ? ps + j : bs + k)];   // unused past a run
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
    if constexpr (MODE != 2) {
        for (int x = tid; x < len; x += kBlockNT) {
            Y[base + x] = order_key_inverse(fk[S::key(x)], order);
            if constexpr (IDX) {
                const uint16_t src = fi[S::idx(x)];
                if constexpr (VB != 0) static_cast<V*>(Yv)[base + x] = sv[src];
                if constexpr (MODE == 1) perm[base + x] = src;
            }
        }
    } else {
        const V* gy = static_cast<const V*>(gY);
        for (int x = tid; x < len; x += kBlockNT) sv[fi[S::idx(x)]] = gy[base + x];
        __syncthreads();
        V* gx = static_cast<V*>(gX);
        for (int x = tid; x < len; x += kBlockNT) gx[base + x] = sv[x];
    }
}

template <class K, int VB, int MODE, bool FORM>
cudaError_t launch_block(const void* X, const void* Xv, int64_t N, int w0, void* Y, void* Yv,
                         uint16_t* perm, const void* gY, void* gX, int order, cudaStream_t st) {
    using L = BlockLayout<K, VB>;
    auto kern = merge_runs_block_kernel<K, VB, MODE, FORM>;
    static std::once_flag once[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(L::TOTAL));
    });
    if (e != cudaSuccess) return e;
    const int64_t chunks = (N + kBlockR - 1) / kBlockR;
    kern<<<unsigned(chunks), kBlockNT, L::TOTAL, st>>>(static_cast<const K*>(X), Xv, N, w0,
                                                        static_cast<K*>(Y), Yv, perm, gY, gX,
                                                        order);
    return cudaGetLastError();
}

template <class K, bool FORM>
cudaError_t block_dispatch_form(int vb, const void* X, const void* Xv, int64_t N, int w0,
                                void* Y, void* Yv, uint16_t* perm, int order, cudaStream_t st) {
    const bool rec = perm != nullptr;
    switch (vb * 2 + (rec ? 1 : 0)) {
        case 0: return launch_block<K, 0, 0, FORM>(X, Xv, N, w0, Y, Yv, perm, nullptr, nullptr,
                                                   order, st);
        case 8: return launch_block<K, 4, 0, FORM>(X, Xv, N, w0, Y, Yv, perm, nullptr, nullptr,
                                                   order, st);
        case 9: return launch_block<K, 4, 1, FORM>(X, Xv, N, w0, Y, Yv, perm, nullptr, nullptr,
                                                   order, st);
        case 16: return launch_block<K, 8, 0, FORM>(X, Xv, N, w0, Y, Yv, perm, nullptr, nullptr,
                                                    order, st);
        case 17: return launch_block<K, 8, 1, FORM>(X, Xv, N, w0, Y, Yv, perm, nullptr, nullptr,
                                                    order, st);
        default: return cudaErrorInvalidValue;
    }
}

template <class K>
cudaError_t block_dispatch(int vb, const void* X, const void* Xv, int64_t N, int w0, void* Y,
                           void* Yv, uint16_t* perm, int order, cudaStream_t st) {
    return w0 < kBlockIPT
               ? block_dispatch_form<K, true>(vb, X, Xv, N, w0, Y, Yv, perm, order, st)
               : block_dispatch_form<K, false>(vb, X, Xv, N, w0, Y, Yv, perm, order, st);
}

template <class K>
cudaError_t block_replay(int vb, const void* X, int64_t N, const void* gY, void* gX, int order,
                         cudaStream_t st) {
    if (vb == 4)
        return launch_block<K, 4, 2, true>(X, nullptr, N, 1, nullptr, nullptr, nullptr, gY, gX,
                                           order, st);
    if (vb == 8)
        return launch_block<K, 8, 2, true>(X, nullptr, N, 1, nullptr, nullptr, nullptr, gY, gX,
                                           order, st);
    return cudaErrorInvalidValue;
}

// Storage type of a key type (float keys are ordered as the signed integer
// of their width after order_key).
template <class F>
cudaError_t by_storage(int key_type, F&& f) {
    switch (key_base(key_type)) {
        case CR_KEY_I32:
        case CR_KEY_F32: return f(int32_t(0));
        case CR_KEY_U32: return f(uint32_t(0));
        case CR_KEY_I64:
        case CR_KEY_F64: return f(int64_t(0));
        default: return f(uint64_t(0));
    }
}

bool overlaps(const void* p, int64_t pb, const void* q, int64_t qb) {
    if (pb <= 0 || qb <= 0) return false;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p), b = reinterpret_cast<uintptr_t>(q);
    return a < b + uintptr_t(qb) && b < a + uintptr_t(pb);
}

}  // namespace

cudaError_t block_sort_runs(int key_type, int vb, int mode, const void* X, const void* Xv,
                            int64_t N, void* Y, void* Yv, uint16_t* perm, const void* gY,
                            void* gX, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int order = key_type_order(key_type);
    return by_storage(key_type, [&](auto k) {
        using K = decltype(k);
        if (mode == 2) return block_replay<K>(vb, X, N, gY, gX, order, st);
        if ((mode == 1) != (perm != nullptr)) return cudaErrorInvalidValue;
        return block_dispatch_form<K, true>(vb, X, Xv, N, 1, Y, Yv, perm, order, st);
    });
}

// Backward of a recorded block: the chunk permutation routes gY to gX
// (cr_route.cu, shared with run formation's recorded backward).
cudaError_t chunk_route_recorded(int vb, int64_t N, int64_t chunk, const uint16_t* perm,
                                 const void* gY, void* gX, cudaStream_t st);

void set_last_error(const char* msg);   // cr_abi.cu

namespace {
// Status with its cr_last_error() detail ("" on success).
cr_status block_fail(cr_status st, const char* msg) {
    set_last_error(msg);
    return st;
}
cr_status block_done(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return block_fail(CR_OK, "");
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return block_fail(CR_ECUDA, buf);
}
}  // namespace

}  // namespace cr

extern "C" int64_t cr_merge_runs_block_length(void) { return cr::kBlockR; }

extern "C" cr_status cr_merge_runs_block(int key_type, int val_bytes, const void* X,
                                         const void* Xv, int64_t N, int64_t width, void* Y,
                                         void* Yv, uint16_t* perm, cr_stream stream) {
    const int ks = cr::key_type_bytes(key_type);
    if (ks == 0) return cr::block_fail(CR_EINVAL, "unknown key type");
    if (N < 0 || N > (int64_t(1) << 59))
        return cr::block_fail(CR_EINVAL, "negative or too large size");
    if (!(val_bytes == 0 || val_bytes == 4 || val_bytes == 8))
        return cr::block_fail(CR_EINVAL, "payload width must be 0, 4 or 8");
    if (perm != nullptr && val_bytes == 0)
        return cr::block_fail(CR_EINVAL, "a permutation needs payloads");
    if (width < 1 || width > cr::kBlockR / 2 || (width & (width - 1)) != 0)
        return cr::block_fail(CR_EINVAL, "width must be a power of two in [1, 2048]");
    if (N == 0) return cr::block_fail(CR_OK, "");
    const void* arrs[5] = {X, Y, val_bytes ? Xv : nullptr, val_bytes ? Yv : nullptr, perm};
    const bool need[5] = {true, true, val_bytes != 0, val_bytes != 0, perm != nullptr};
    const uintptr_t elem[5] = {uintptr_t(ks), uintptr_t(ks), uintptr_t(val_bytes),
                               uintptr_t(val_bytes), 2};
    for (int i = 0; i < 5; ++i) {
        if (!need[i]) continue;
        if (arrs[i] == nullptr) return cr::block_fail(CR_EINVAL, "NULL array");
        if (reinterpret_cast<uintptr_t>(arrs[i]) % elem[i])
            return cr::block_fail(CR_EALIGN, "array not aligned to its element size");
    }
    const int64_t kb = N * ks, vbb = N * val_bytes, pb = perm ? N * 2 : 0;
    if (cr::overlaps(Y, kb, X, kb) || (val_bytes && cr::overlaps(Y, kb, Xv, vbb)) ||
        (val_bytes && cr::overlaps(Yv, vbb, X, kb)) ||
        (val_bytes && cr::overlaps(Yv, vbb, Xv, vbb)) || (val_bytes && cr::overlaps(Yv, vbb, Y, kb)) ||
        (perm && (cr::overlaps(perm, pb, X, kb) || cr::overlaps(perm, pb, Y, kb) ||
                  (val_bytes && (cr::overlaps(perm, pb, Xv, vbb) ||
                                 cr::overlaps(perm, pb, Yv, vbb))))))
        return cr::block_fail(CR_EALIAS, "an output overlaps another array");
    const int order = cr::key_type_order(key_type);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int w0 = int(width);
    const cudaError_t e = cr::by_storage(key_type, [&](auto k) {
        using K = decltype(k);
        return cr::block_dispatch<K>(val_bytes, X, Xv, N, w0, Y, Yv, perm, order, st);
    });
    return cr::block_done(e, "merge block launch");
}

extern "C" cr_status cr_merge_runs_block_backward_recorded(int val_bytes, int64_t N,
                                                           const uint16_t* perm, const void* gY,
                                                           void* gX, cr_stream stream) {
    if (!(val_bytes == 4 || val_bytes == 8))
        return cr::block_fail(CR_EINVAL, "payload width must be 4 or 8");
    if (N < 0 || N > (int64_t(1) << 59))
        return cr::block_fail(CR_EINVAL, "negative or too large size");
    if (N == 0) return cr::block_fail(CR_OK, "");
    if (!perm || !gY || !gX) return cr::block_fail(CR_EINVAL, "NULL array");
    if ((reinterpret_cast<uintptr_t>(perm) & 1u) ||
        ((reinterpret_cast<uintptr_t>(gY) | reinterpret_cast<uintptr_t>(gX)) %
         uintptr_t(val_bytes)))
        return cr::block_fail(CR_EALIGN, "array not aligned to its element size");
    const int64_t b = N * val_bytes;
    if (cr::overlaps(gX, b, gY, b) || cr::overlaps(gX, b, perm, N * 2))
        return cr::block_fail(CR_EALIAS, "gX overlaps another array");
    const cudaError_t e = cr::chunk_route_recorded(val_bytes, N, cr::kBlockR, perm, gY, gX,
                                                   static_cast<cudaStream_t>(stream));
    return cr::block_done(e, "merge block backward launch");
}
