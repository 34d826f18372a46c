// cr_merge.cuh -- the persistent tile-merge kernel (forward and payload
// backward) for sm_103a, driven by a table of tile records.
//
// Each CTA runs one producer warp and NT consumer threads and walks the
// output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...  Every tile
// carries exactly TILE = NT*IPT output elements (the last one of a merge or
// segment fewer), so the static round-robin schedule is balanced
// (Algorithm 2 with equal blocks, Proposition 2).
//
//  producer (one lane): reads the tile record (A window, B window, output
//      offset; prefetched one tile ahead), then stages the windows into an
//      NS-deep ring of shared-memory stages with bulk copies (TMA engine,
//      cp.async.bulk completing on the stage's mbarrier).  Windows start at
//      arbitrary element offsets: the copy covers the 16-byte aligned
//      superset and the consumers index from the head offset.
//  consumers (NT threads): thread s finds the split of diagonal s*IPT of
//      the tile inside the shared-memory windows, merges exactly IPT
//      elements serially into registers (ties take A), and after a barrier
//      writes them back into the same stage, which then serves as the output
//      staging buffer; one thread issues bulk stores of the 16-byte aligned
//      interior and a few threads store the ragged ends.  A stage is handed
//      back to the producer one tile later, once its bulk store has read it.
//
// The in-tile split is the unique co-rank of Lemma 1, found by binary lifting
// on the first Lemma condition (A[j-1] <= B[d-j] holds exactly for j <= j*):
// one comparison per step instead of Algorithm 1's two-sided test, which
// matters here because every consumer thread runs it once per tile.
#pragma once

#include "cr_device.cuh"

namespace cr {

template <int VB> struct VBits { using T = uint32_t; };
template <bool B> struct BoolC { static constexpr bool value = B; };
template <> struct VBits<8> { using T = uint64_t; };

__host__ __device__ constexpr size_t align_up_sz(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-stage description written by the producer for the consumers.
struct StageInfo {
    int64_t ga, gb, gc;      // window starts (elements) in A, B and output
    int32_t alen, blen;      // window lengths
    int32_t ak, bk;          // smem element offset of A[ga] / B[gb] in the key stage
    int32_t av, bv;          // same in the payload stage (forward) / head of gC (backward)
};
static_assert(sizeof(StageInfo) == 48, "StageInfo size");

// Shared-memory layout of one kernel instantiation (host and device agree).
// A stage holds the input windows and, after the consumers have read them,
// the tile's output (forward: keys, payloads, tags; backward: gA, gB).
template <class K, int VB, bool TAG, int NT, int IPT, int NS, bool BWD>
struct Layout {
    static constexpr int TILE = NT * IPT;
    static constexpr int KS = sizeof(K);
    static constexpr int EK = 16 / KS;
    static constexpr int VS = VB ? VB : 4;
    static constexpr int EV = 16 / VS;
    static constexpr int SK = TILE + 4 * EK;                      // A and B key windows
    static constexpr int SV = (VB && !BWD) ? TILE + 4 * EV : 0;   // A and B payload windows
    static constexpr int ST = (TAG && !BWD) ? TILE + 8 : 0;       // output tags
    static constexpr int SG = BWD ? TILE + 4 * EV : 0;            // gC window, then gA | gB
    static constexpr size_t STAGE_K = align_up_sz(size_t(SK) * KS, 128);
    static constexpr size_t STAGE_V = align_up_sz(size_t(SV) * VS, 128);
    static constexpr size_t STAGE_T = align_up_sz(size_t(ST) * 4, 128);
    static constexpr size_t STAGE_G = align_up_sz(size_t(SG) * VS, 128);
    static constexpr size_t STAGE = STAGE_K + STAGE_V + STAGE_T + STAGE_G;
    static constexpr size_t BAR_OFF = 0;                       // full[NS], empty[NS], flags
    static constexpr size_t INFO_OFF = 256;
    static constexpr size_t STAGE_OFF = align_up_sz(INFO_OFF + NS * sizeof(StageInfo), 128);
    static constexpr size_t TOTAL = STAGE_OFF + NS * STAGE + 128;  // + slack for one-past reads
    static_assert(NS >= 3, "the consumers hold two stages at a time");
    static_assert(2 * NS * 8 + 16 <= INFO_OFF, "barrier area");
    static_assert(TILE % EK == 0 && TILE % EV == 0 && TILE % 4 == 0, "tile alignment");
    static_assert(TOTAL <= 232448, "exceeds 227 KB of shared memory per CTA");
};

// Plan for staging one window [g0, g0+len) of an array of `total` elements
// with 16-byte chunks of E elements: the bulk copy covers
// [s0, min(s1, floor_E(total))) and elements beyond the last full chunk of
// the array are loaded one by one (only windows touching the array's end).
struct WinPlan {
    int64_t s0;        // first element copied (aligned down)
    int64_t bulk;      // elements moved by the bulk copy
    int64_t plain0;    // [plain0, plain1): elements loaded one by one
    int64_t plain1;
    int32_t head;      // g0 - s0
    int32_t sup;       // aligned superset length (smem footprint)
};

__device__ __forceinline__ WinPlan plan_window(int64_t g0, int32_t len, int64_t total, int E) {
    WinPlan w;
    const int64_t mask = ~int64_t(E - 1);
    w.s0 = g0 & mask;
    const int64_t s1 = (g0 + len + E - 1) & mask;
    const int64_t tot_al = total & mask;
    const int64_t bulk_end = s1 < tot_al ? s1 : tot_al;
    w.bulk = bulk_end > w.s0 ? bulk_end - w.s0 : 0;
    const int64_t covered = w.s0 + w.bulk;
    w.plain0 = covered > g0 ? covered : g0;
    w.plain1 = g0 + len;
    w.head = int32_t(g0 - w.s0);
    w.sup = int32_t(s1 - w.s0);
    return w;
}

template <class T>
__device__ __forceinline__ void window_plain(T* region, const T* gbase, const WinPlan& w) {
    for (int64_t g = w.plain0; g < w.plain1; ++g) region[g - w.s0] = gbase[g];
}

template <class T>
__device__ __forceinline__ void window_bulk(T* region, const T* gbase, const WinPlan& w,
                                            uint64_t* bar) {
    if (w.bulk > 0) bulk_g2s(region, gbase + w.s0, uint32_t(w.bulk * sizeof(T)), bar);
}

// Store the staged output window buf[ph + x] (x < len) to gbase[g0 + x],
// ph = g0 mod E.  store_bulk: the whole 16-byte chunks (one thread);
// store_edges: the ragged ends, one element per `lane` in [0, 2E).
template <class T>
__device__ __forceinline__ void store_bulk(T* gbase, const T* buf, int64_t g0, int32_t len, int E) {
    const int64_t mask = ~int64_t(E - 1);
    const int64_t a0 = (g0 + E - 1) & mask;
    const int64_t a1 = (g0 + len) & mask;
    if (a1 > a0) {
        const int64_t ph = g0 & (E - 1);
        bulk_s2g(gbase + a0, buf + ph + (a0 - g0), uint32_t((a1 - a0) * sizeof(T)));
    }
}

template <class T>
__device__ __forceinline__ void store_edges(T* gbase, const T* buf, int64_t g0, int32_t len, int E,
                                            int lane) {
    const int64_t mask = ~int64_t(E - 1);
    const int64_t a0 = (g0 + E - 1) & mask;
    const int64_t a1 = (g0 + len) & mask;
    const int64_t ph = g0 & (E - 1);
    int64_t g = -1;
    if (a1 > a0) {
        const int hc = int(a0 - g0);
        const int tc = int(g0 + len - a1);
        if (lane < hc) g = g0 + lane;
        else if (lane - hc < tc) g = a1 + (lane - hc);
    } else if (lane < len) {
        g = g0 + lane;
    }
    if (g >= 0) gbase[g] = buf[ph + (g - g0)];
}

// Number of A elements among the first d outputs of the stable merge of
// sA[0, alen) and sB[0, blen): the co-rank j of Lemma 1, found on its first
// condition (A[x] <= B[d-1-x] holds exactly for x < j) by binary lifting:
// LOG fixed steps of decreasing size, so all threads of a warp run the same
// instruction stream.  Loads are issued only for in-range probes.
template <int LOG, class K>
__device__ __forceinline__ int split_in_tile(const K* sA, int alen, const K* sB, int blen, int d) {
    const int lo = d - blen > 0 ? d - blen : 0;
    const int hi = d < alen ? d : alen;
    int pos = lo;
#pragma unroll
    for (int step = 1 << (LOG - 1); step > 0; step >>= 1) {
        const int np = pos + step;
        if (np <= hi && !(sB[d - np] < sA[np - 1])) pos = np;
    }
    return pos;
}

template <int X> struct Log2Ceil { static constexpr int v = 1 + Log2Ceil<(X + 1) / 2>::v; };
template <> struct Log2Ceil<1> { static constexpr int v = 0; };

// ---------------------------------------------------------------------------
// Forward (BWD = false): C keys [+ payloads] [+ tags].
// Backward (BWD = true): gA / gB from gC, routed by the same merge decisions.
// ---------------------------------------------------------------------------
template <class K, int VB, bool TAG, int NT, int IPT, int NS, int MINB, bool BWD>
__global__ void __launch_bounds__(NT + 32, MINB) merge_tiles_kernel(const MergeArgs p) {
    using L = Layout<K, VB, TAG, NT, IPT, NS, BWD>;
    using V = typename VBits<VB>::T;
    constexpr int TILE = L::TILE;
    constexpr int EK = L::EK;
    constexpr int EV = L::EV;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    uint64_t* empty = full + NS;
    // s_abort: written only by consumer threads between their two named
    // barriers of an iteration and read by all of them after the second one,
    // so every consumer takes the same exit decision.
    volatile int32_t* s_abort = reinterpret_cast<volatile int32_t*>(empty + NS);
    volatile int32_t* s_issued = s_abort + 1;
    StageInfo* info = reinterpret_cast<StageInfo*>(smem + L::INFO_OFF);

    auto base = [&](int s) { return smem + L::STAGE_OFF + size_t(s) * L::STAGE; };
    auto stage_k = [&](int s) { return reinterpret_cast<K*>(base(s)); };
    auto stage_v = [&](int s) { return reinterpret_cast<V*>(base(s) + L::STAGE_K); };
    auto stage_t = [&](int s) {
        return reinterpret_cast<uint32_t*>(base(s) + L::STAGE_K + L::STAGE_V);
    };
    auto stage_g = [&](int s) {
        return reinterpret_cast<V*>(base(s) + L::STAGE_K + L::STAGE_V + L::STAGE_T);
    };

    WsHeader* hdr = reinterpret_cast<WsHeader*>(p.ws);
    const TileRec* recs = ws_recs(p.ws);
    const int tid = threadIdx.x;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        *s_abort = 0;
        *s_issued = 0;
        fence_barrier_init();
    }
    __syncthreads();

    // A table made for another tile size (the shape was changed between the
    // partition and this launch) is refused as a whole.
    if (hdr->tile != TILE) {
        if (tid == 0) set_status(&hdr->status, kDevInternal);
        return;
    }
    const int64_t ntiles = hdr->ntiles;

    if (tid >= NT) {
        // ------------------------------------------------------------ producer
        if (tid != NT) return;
        const K* A = static_cast<const K*>(p.ak);
        const K* B = static_cast<const K*>(p.bk);
        int64_t t = blockIdx.x;
        int it = 0;
        TileRec cur;
        if (t < ntiles) cur = recs[t];
        for (; t < ntiles; t += gridDim.x, ++it) {
            const int s = it % NS;
            TileRec nxt = cur;
            if (t + gridDim.x < ntiles) nxt = recs[t + gridDim.x];
            if (it >= NS && !mbar_wait(&empty[s], ((it / NS) - 1) & 1)) {
                // Consumers then time out on the stage they wait for.
                set_status(&hdr->status, kDevTimeout);
                break;
            }
            const bool ok = cur.alen >= 0 && cur.blen >= 0 && cur.alen + cur.blen <= TILE &&
                            cur.ga >= 0 && cur.gb >= 0 && cur.gc >= 0 &&
                            cur.ga + cur.alen <= p.a_total && cur.gb + cur.blen <= p.b_total &&
                            cur.gc + cur.alen + cur.blen <= p.c_total;
            if (!ok) {
                set_status(&hdr->status, kDevInternal);
                cur.alen = 0;
                cur.blen = 0;
            }
            const int32_t len = cur.alen + cur.blen;
            K* sk = stage_k(s);
            const WinPlan wa = plan_window(cur.ga, cur.alen, p.a_total, EK);
            const WinPlan wb = plan_window(cur.gb, cur.blen, p.b_total, EK);
            StageInfo in;
            in.ga = cur.ga;
            in.gb = cur.gb;
            in.gc = cur.gc;
            in.alen = cur.alen;
            in.blen = cur.blen;
            in.ak = wa.head;
            in.bk = wa.sup + wb.head;
            uint32_t bytes = uint32_t((wa.bulk + wb.bulk) * sizeof(K));
            WinPlan va{}, vb{}, wg{};
            if (!BWD && VB) {
                va = plan_window(cur.ga, cur.alen, p.a_total, EV);
                vb = plan_window(cur.gb, cur.blen, p.b_total, EV);
                in.av = va.head;
                in.bv = va.sup + vb.head;
                bytes += uint32_t((va.bulk + vb.bulk) * sizeof(V));
            } else if (BWD) {
                wg = plan_window(cur.gc, len, p.c_total, EV);
                in.av = wg.head;
                in.bv = 0;
                bytes += uint32_t(wg.bulk * sizeof(V));
            } else {
                in.av = 0;
                in.bv = 0;
            }
            info[s] = in;
            // rare: elements past the last full 16-byte chunk of an array
            window_plain(sk, A, wa);
            window_plain(sk + wa.sup, B, wb);
            if (!BWD && VB) {
                window_plain(stage_v(s), static_cast<const V*>(p.av), va);
                window_plain(stage_v(s) + va.sup, static_cast<const V*>(p.bv), vb);
            } else if (BWD) {
                window_plain(stage_g(s), static_cast<const V*>(p.gc_in), wg);
            }
            mbar_arrive_expect_tx(&full[s], bytes);
            window_bulk(sk, A, wa, &full[s]);
            window_bulk(sk + wa.sup, B, wb, &full[s]);
            if (!BWD && VB) {
                window_bulk(stage_v(s), static_cast<const V*>(p.av), va, &full[s]);
                window_bulk(stage_v(s) + va.sup, static_cast<const V*>(p.bv), vb, &full[s]);
            } else if (BWD) {
                window_bulk(stage_g(s), static_cast<const V*>(p.gc_in), wg, &full[s]);
            }
            *s_issued = it + 1;
            cur = nxt;
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    int it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = it % NS;
        const bool ready = mbar_wait(&full[s], (it / NS) & 1);
        if (!ready) {
            set_status(&hdr->status, kDevTimeout);
            *s_abort = 1;
        }
        const StageInfo in = info[s];
        const int alen = ready ? in.alen : 0;
        const int blen = ready ? in.blen : 0;
        const int len = alen + blen;
        const int d = min(tid * IPT, len);
        const int cnt = min(IPT, len - d);
        K* sk = stage_k(s);
        const K* sA = sk + in.ak;
        const K* sB = sk + in.bk;
        int j = split_in_tile<Log2Ceil<TILE + 1>::v>(sA, alen, sB, blen, d);
        int k = d - j;
        K a = K(0), b = K(0);
        if (cnt > 0) {
            a = sA[j];   // may be one past A's window: never taken then
            b = sB[k];
        }
        if constexpr (!BWD) {
            K okey[IPT];
            V oval[VB ? IPT : 1];
            uint32_t otag[TAG ? IPT : 1];
            const V* sv = stage_v(s);
            const int avo = in.av, bvo = in.bv;
            // One merge step (ties take A).  GUARD: some side may run out
            // within this thread's IPT steps (only near the windows' ends).
            auto step = [&](int q, auto guard) {
                const bool takeA = decltype(guard)::value
                                       ? (k >= blen) || (j < alen && !(b < a))
                                       : !(b < a);
                okey[q] = takeA ? a : b;
                if constexpr (VB != 0) oval[q] = sv[takeA ? avo + j : bvo + k];
                if constexpr (TAG)
                    otag[q] = takeA ? uint32_t(in.ga + j) : uint32_t(p.tag_b + in.gb + k);
                j += takeA ? 1 : 0;
                k += takeA ? 0 : 1;
                const K nx = takeA ? sA[j] : sB[k];
                a = takeA ? nx : a;
                b = takeA ? b : nx;
            };
            if (cnt == IPT && j + IPT <= alen && k + IPT <= blen) {
#pragma unroll
                for (int q = 0; q < IPT; ++q) step(q, BoolC<false>{});
            } else {
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if (q < cnt) step(q, BoolC<true>{});
            }
            named_sync(1, NT);   // every input of stage s has been read
            const int ph = int(in.gc & (EK - 1));
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                if (q < cnt) sk[ph + d + q] = okey[q];
            if constexpr (VB != 0) {
                V* ov = stage_v(s);
                const int phv = int(in.gc & (EV - 1));
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if (q < cnt) ov[phv + d + q] = oval[q];
            }
            if constexpr (TAG) {
                uint32_t* ot = stage_t(s);
                const int pht = int(in.gc & 3);
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if (q < cnt) ot[pht + d + q] = otag[q];
            }
        } else {
            V gval[IPT];
            int dst[IPT];
            const V* sg = stage_g(s) + in.av;
            const int pha = int(in.ga & (EV - 1));
            const int boff = ((pha + alen + EV - 1) / EV) * EV + int(in.gb & (EV - 1));
            auto step = [&](int q, auto guard) {
                const bool takeA = decltype(guard)::value
                                       ? (k >= blen) || (j < alen && !(b < a))
                                       : !(b < a);
                gval[q] = sg[d + q];
                dst[q] = takeA ? pha + j : boff + k;
                j += takeA ? 1 : 0;
                k += takeA ? 0 : 1;
                const K nx = takeA ? sA[j] : sB[k];
                a = takeA ? nx : a;
                b = takeA ? b : nx;
            };
            if (cnt == IPT && j + IPT <= alen && k + IPT <= blen) {
#pragma unroll
                for (int q = 0; q < IPT; ++q) step(q, BoolC<false>{});
            } else {
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if (q < cnt) step(q, BoolC<true>{});
            }
            named_sync(1, NT);   // every input of stage s has been read
            V* og = stage_g(s);
#pragma unroll
            for (int q = 0; q < IPT; ++q)
                if (q < cnt) og[dst[q]] = gval[q];
        }
        fence_proxy_async_smem();
        named_sync(1, NT);       // the tile's output is staged
        if (*s_abort) break;
        if constexpr (!BWD) {
            K* C = static_cast<K*>(p.ck);
            if (tid == 0) {
                store_bulk(C, sk, in.gc, len, EK);
                if constexpr (VB != 0) store_bulk(static_cast<V*>(p.cv), stage_v(s), in.gc, len, EV);
                if constexpr (TAG) store_bulk(p.ctag, stage_t(s), in.gc, len, 4);
                bulk_commit();
            } else if (tid <= 2 * EK) {
                store_edges(C, sk, in.gc, len, EK, tid - 1);
            } else if (VB != 0 && tid >= 32 && tid < 32 + 2 * EV) {
                store_edges(static_cast<V*>(p.cv), stage_v(s), in.gc, len, EV, tid - 32);
            } else if (TAG && tid >= 64 && tid < 64 + 8) {
                store_edges(p.ctag, stage_t(s), in.gc, len, 4, tid - 64);
            }
        } else {
            V* gA = static_cast<V*>(p.cv);
            V* gB = static_cast<V*>(p.cv2);
            const int pha = int(in.ga & (EV - 1));
            const int ob = ((pha + in.alen + EV - 1) / EV) * EV;
            if (tid == 0) {
                store_bulk(gA, stage_g(s), in.ga, in.alen, EV);
                store_bulk(gB, stage_g(s) + ob, in.gb, in.blen, EV);
                bulk_commit();
            } else if (tid <= 2 * EV) {
                store_edges(gA, stage_g(s), in.ga, in.alen, EV, tid - 1);
            } else if (tid >= 32 && tid < 32 + 2 * EV) {
                store_edges(gB, stage_g(s) + ob, in.gb, in.blen, EV, tid - 32);
            }
        }
        if (tid == 0) {
            // Hand the previous tile's stage back once its bulk store has read
            // it (its edge stores finished before this iteration's barriers).
            bulk_wait_read<1>();
            if (it > 0) mbar_arrive(&empty[(it - 1) % NS]);
        }
    }
    if (*s_abort && tid == 0) {
        // Let copies that were issued but never consumed land before exit.
        const int issued = *s_issued;
        for (int q = it; q < issued; ++q) mbar_wait(&full[q % NS], (q / NS) & 1, 100000000ull);
    }
    if (tid == 0) bulk_wait_all<0>();
}

}  // namespace cr
