// cr_merge.cuh -- the persistent tile-merge kernel (forward and payload
// backward) for sm_103a, driven by a table of tile records.
//
// Each CTA runs NT consumer threads, one producer warp and one storer warp,
// and walks the output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// Every tile carries exactly TILE = NT*IPT*ILP output elements (the last one of a merge or
// segment fewer), so the static round-robin schedule is balanced
// (Algorithm 2 with equal blocks, Proposition 2).
//
//  producer (one lane): reads the tile record (A window, B window, output
//      offset; prefetched one tile ahead), then stages the windows into an
//      NS-deep ring of shared-memory stages with bulk copies (TMA engine,
//      cp.async.bulk completing on the stage's mbarrier).  Windows start at
//      arbitrary element offsets: the copy covers the 16-byte aligned
//      superset and the consumers index from the head offset.
//  consumers (NT threads): each thread owns ILP diagonals of the tile
//      (chain c of thread s starts at (c*NT + s)*IPT), finds their splits
//      inside the shared-memory windows, merges exactly IPT elements per
//      chain serially into registers (ties take A; the chains interleave
//      so their shared-memory latencies overlap), and after a barrier
//      writes them back into the same stage, which then serves as the output
//      staging buffer, and signals the stage's "staged" mbarrier.  In the
//      forward with payloads and at least 15 merge steps per thread and
//      tile the barrier is an mbarrier and a warp finds its splits in the
//      next tile's stage between arriving and waiting on it.
//  storer (one warp): waits for a staged tile, issues the bulk store of its
//      16-byte aligned interior, stores the ragged ends with plain stores,
//      and hands the stage back to the producer as soon as the bulk store has
//      read it.  The consumers never wait on stores.
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
// the tile's output (forward: keys, payloads, tags, and with REC the tile's
// source-flag words; backward: gA, gB).
template <class K, int VB, bool TAG, int NT, int IPT, int ILP, int NS, bool BWD, bool REC = false>
struct Layout {
    static constexpr int TILE = NT * IPT * ILP;
    static constexpr int KS = sizeof(K);
    static constexpr int EK = 16 / KS;
    static constexpr int VS = VB ? VB : 4;
    static constexpr int EV = 16 / VS;
    static constexpr int SK = TILE + 4 * EK;                      // A and B key windows
    static constexpr int SV = (VB && !BWD) ? TILE + 4 * EV : 0;   // A and B payload windows
    static constexpr int ST = (TAG && !BWD) ? TILE + 8 : 0;       // output tags
    static constexpr int SG = BWD ? TILE + 4 * EV : 0;            // gC window, then gA | gB
    static constexpr int WPT = TILE / 32;                         // source-flag words (REC)
    static constexpr size_t STAGE_K = align_up_sz(size_t(SK) * KS, 128);
    static constexpr size_t STAGE_V = align_up_sz(size_t(SV) * VS, 128);
    static constexpr size_t STAGE_T = align_up_sz(size_t(ST) * 4, 128);
    static constexpr size_t STAGE_G = align_up_sz(size_t(SG) * VS, 128);
    static constexpr size_t STAGE_F = REC ? align_up_sz(size_t(WPT) * 4, 128) : 0;
    static constexpr size_t STAGE = STAGE_K + STAGE_V + STAGE_T + STAGE_G + STAGE_F;
    static constexpr size_t BAR_OFF = 0;              // full, staged, empty, consumed [NS]; flags
    static constexpr size_t INFO_OFF = 256;
    static constexpr size_t STAGE_OFF = align_up_sz(INFO_OFF + NS * sizeof(StageInfo), 128);
    static constexpr size_t TOTAL = STAGE_OFF + NS * STAGE + 128;  // + slack for one-past reads
    static_assert(NS >= 2, "at least one stage can load while another is merged");
    static_assert(4 * NS * 8 + 20 <= INFO_OFF, "barrier area");
    static_assert(TILE % EK == 0 && TILE % EV == 0 && TILE % 4 == 0, "tile alignment");
    // a tile's flag words form whole 16-byte chunks (bulk store at t * WPT)
    static_assert(!REC || (!BWD && TILE % 32 == 0 && (WPT * 4) % 16 == 0 && WPT <= NT),
                  "source flags need TILE % 128 == 0 and at most one word per consumer");
    static_assert(TOTAL <= 232448, "exceeds 227 KB of shared memory per CTA");
};

// Plan for staging one window [g0, g0+len) of an array that occupies
// [lo, total) (element indices from a 16-byte boundary at or below the
// array's start, lo < E) with 16-byte chunks of E elements: the stage holds
// the aligned superset [s0, s1) of the window; the bulk copy moves the whole
// chunks of it that lie inside the array, [bb, bb + bulk), and the elements
// of the window in the array's partial first or last chunk are loaded one by
// one (only windows touching either end of the array have any).  Nothing
// outside the array is read.
struct WinPlan {
    int64_t s0;        // first element of the superset (aligned down)
    int64_t bb;        // first element moved by the bulk copy
    int64_t bulk;      // elements moved by the bulk copy
    int64_t front0;    // [front0, front1): loaded one by one (array's first chunk)
    int64_t front1;
    int64_t plain0;    // [plain0, plain1): loaded one by one (array's last chunk)
    int64_t plain1;
    int32_t head;      // g0 - s0
    int32_t sup;       // aligned superset length (smem footprint)
};

__device__ __forceinline__ WinPlan plan_window(int64_t g0, int32_t len, int64_t lo,
                                               int64_t total, int E) {
    WinPlan w;
    const int64_t mask = ~int64_t(E - 1);
    w.s0 = g0 & mask;
    const int64_t s1 = (g0 + len + E - 1) & mask;
    const int64_t lo_al = (lo + E - 1) & mask;   // first chunk wholly inside the array
    const int64_t hi_al = total & mask;          // end of the last whole chunk
    const int64_t bb = w.s0 > lo_al ? w.s0 : lo_al;
    const int64_t be = s1 < hi_al ? s1 : hi_al;
    if (be > bb) {
        // bb <= g0 + len and be > g0: the copied chunks overlap the window
        w.bb = bb;
        w.bulk = be - bb;
        w.front0 = g0;
        w.front1 = bb > g0 ? bb : g0;
        w.plain0 = be;
    } else {
        w.bb = w.s0;
        w.bulk = 0;
        w.front0 = g0;
        w.front1 = g0;
        w.plain0 = g0;
    }
    w.plain1 = g0 + len;
    w.head = int32_t(g0 - w.s0);
    w.sup = int32_t(s1 - w.s0);
    return w;
}

template <class T>
__device__ __forceinline__ void window_plain(T* region, const T* gbase, const WinPlan& w) {
    for (int64_t g = w.front0; g < w.front1; ++g) region[g - w.s0] = gbase[g];
    for (int64_t g = w.plain0; g < w.plain1; ++g) region[g - w.s0] = gbase[g];
}

template <class T>
__device__ __forceinline__ void window_bulk(T* region, const T* gbase, const WinPlan& w,
                                            uint64_t* bar) {
    if (w.bulk > 0)
        bulk_g2s(region + (w.bb - w.s0), gbase + w.bb, uint32_t(w.bulk * sizeof(T)), bar);
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
// instruction stream.  Loads are issued only for in-range probes.  ILP
// independent diagonals are searched in lock step (their loads overlap).
struct KeyIdentity {
    template <class K>
    __device__ __forceinline__ K operator()(K x) const { return x; }
};

// Key comparison of the merge: `<` of the storage type, or reversed (for a
// descending order, whose order map is the complement: ~x < ~y exactly when
// y < x, so comparing the stored keys with the operands swapped needs no
// per-key work).
template <bool REV>
struct KeyLess {
    template <class K>
    __device__ __forceinline__ bool operator()(K x, K y) const { return REV ? (y < x) : (x < y); }
};

// `key` maps every key read before it is compared (the call's key order;
// the identity for the storage type's own order); `less` compares mapped keys.
template <int LOG, int ILP, class K, class KeyMap = KeyIdentity, class Less = KeyLess<false>>
__device__ __forceinline__ void split_in_tile(const K* sA, int alen, const K* sB, int blen,
                                              const int (&d)[ILP], int (&pos)[ILP],
                                              KeyMap key = KeyMap(), Less less = Less()) {
    int hi[ILP];
#pragma unroll
    for (int c = 0; c < ILP; ++c) {
        pos[c] = d[c] - blen > 0 ? d[c] - blen : 0;
        hi[c] = d[c] < alen ? d[c] : alen;
    }
#pragma unroll
    for (int step = 1 << (LOG - 1); step > 0; step >>= 1) {
#pragma unroll
        for (int c = 0; c < ILP; ++c) {
            const int np = pos[c] + step;
            if (np <= hi[c] && !less(key(sB[d[c] - np]), key(sA[np - 1]))) pos[c] = np;
        }
    }
}

template <int X> struct Log2Ceil { static constexpr int v = 1 + Log2Ceil<(X + 1) / 2>::v; };
template <> struct Log2Ceil<1> { static constexpr int v = 0; };

// ---------------------------------------------------------------------------
// Forward (BWD = false): C keys [+ payloads] [+ tags].
// Backward (BWD = true): gA / gB from gC, routed by the same merge decisions.
// ---------------------------------------------------------------------------
// Block: NT consumer threads, then one producer warp, then one storer warp.
template <int NT> constexpr int merge_block_threads() { return NT + 64; }

// REC (forward only): also record, per output, whether it came from B, as
// bit x % 32 of word x / 32 of the tile's WPT flag words, stored at
// p.flags + t * WPT for tile t (the backward then routes gradients from
// these bits and the tile table without reading keys).
//
// ORD: the key order.  0: the storage type's own (plain `<`).  1: another
// order (p.order, order_key): every key read from shared memory is mapped
// before it is compared and the output keys are mapped back.  2: the
// descending order of the storage type, by comparing with the operands
// swapped (keys are neither mapped nor mapped back).  3 and 4: IEEE-754
// totalOrder of floats stored in the signed integer of their width, with
// the map's masks known at compile time, ascending (3) or descending (4,
// the comparison reversed).
template <class K, int VB, bool TAG, int NT, int IPT, int ILP, int NS, int MINB, bool BWD,
          bool REC, int ORD>
__global__ void __launch_bounds__(NT + 64, MINB) merge_tiles_kernel(const MergeArgs p) {
    using L = Layout<K, VB, TAG, NT, IPT, ILP, NS, BWD, REC>;
    using V = typename VBits<VB>::T;
    constexpr int TILE = L::TILE;
    constexpr int EK = L::EK;
    constexpr int EV = L::EV;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
    uint64_t* staged = full + NS;
    uint64_t* empty = staged + NS;
    uint64_t* consumed = empty + NS;   // PIPE: one arrival per consumer warp
    // s_abort[it & 1] (s_abort[it & 3] with PIPE): written only by consumer
    // threads before the barrier that separates iteration it's reads from
    // its writes (with PIPE, also while preparing iteration it in iteration
    // it - 1) and read by all of them after it (the other slots belong to
    // the neighbouring iterations), so every consumer takes the same exit
    // decision.
    volatile int32_t* s_abort = reinterpret_cast<volatile int32_t*>(consumed + NS);
    volatile int32_t* s_issued = s_abort + 4;
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
    auto stage_f = [&](int s) {
        return reinterpret_cast<uint32_t*>(base(s) + L::STAGE_K + L::STAGE_V + L::STAGE_T +
                                           L::STAGE_G);
    };

    WsHeader* hdr = reinterpret_cast<WsHeader*>(p.ws);
    const TileRec* recs = ws_recs(p.ws);
    const int tid = threadIdx.x;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&staged[s], NT);
            mbar_init(&empty[s], 1);
            mbar_init(&consumed[s], NT / 32);
        }
        for (int q = 0; q < 4; ++q) s_abort[q] = 0;
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

    if (tid >= NT + 32) {
        // -------------------------------------------------------------- storer
        const int lane = tid - NT - 32;
        int it = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int s = it % NS;
            // the decision is made warp-uniform so that every lane reaches
            // the __syncwarp below
            if (!__all_sync(0xffffffffu, mbar_wait(&staged[s], (it / NS) & 1))) {
                if (lane == 0) set_status(&hdr->status, kDevTimeout);
                break;
            }
            const StageInfo in = info[s];
            const int len = in.alen + in.blen;
            if constexpr (!BWD) {
                K* C = static_cast<K*>(p.ck);
                if (lane == 0) {
                    store_bulk(C, stage_k(s), in.gc + p.sh_ck, len, EK);
                    if constexpr (VB != 0)
                        store_bulk(static_cast<V*>(p.cv), stage_v(s), in.gc + p.sh_cv, len, EV);
                    if constexpr (TAG) store_bulk(p.ctag, stage_t(s), in.gc + p.sh_tag, len, 4);
                    if constexpr (REC) bulk_s2g(p.flags + t * L::WPT, stage_f(s), L::WPT * 4);
                    bulk_commit();
                } else if (lane <= 2 * EK) {
                    store_edges(C, stage_k(s), in.gc + p.sh_ck, len, EK, lane - 1);
                } else if (VB != 0 && lane >= 9 && lane < 9 + 2 * EV) {
                    store_edges(static_cast<V*>(p.cv), stage_v(s), in.gc + p.sh_cv, len, EV,
                                lane - 9);
                } else if (TAG && lane >= 17 && lane < 17 + 8) {
                    store_edges(p.ctag, stage_t(s), in.gc + p.sh_tag, len, 4, lane - 17);
                }
            } else {
                V* gA = static_cast<V*>(p.cv);
                V* gB = static_cast<V*>(p.cv2);
                const int64_t ga = in.ga + p.sh_cv, gb = in.gb + p.sh_cv2;
                const int pha = int(ga & (EV - 1));
                const int ob = ((pha + in.alen + EV - 1) / EV) * EV;
                if (lane == 0) {
                    store_bulk(gA, stage_g(s), ga, in.alen, EV);
                    store_bulk(gB, stage_g(s) + ob, gb, in.blen, EV);
                    bulk_commit();
                } else if (lane <= 2 * EV) {
                    store_edges(gA, stage_g(s), ga, in.alen, EV, lane - 1);
                } else if (lane >= 9 && lane < 9 + 2 * EV) {
                    store_edges(gB, stage_g(s) + ob, gb, in.blen, EV, lane - 9);
                }
            }
            if (lane == 0) bulk_wait_read<0>();   // the bulk store has read the stage
            __syncwarp();                          // and so have the edge stores
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (lane == 0) bulk_wait_all<0>();
        return;
    }
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
            const WinPlan wa = plan_window(cur.ga + p.sh_ak, cur.alen, p.sh_ak,
                                           p.a_total + p.sh_ak, EK);
            const WinPlan wb = plan_window(cur.gb + p.sh_bk, cur.blen, p.sh_bk,
                                           p.b_total + p.sh_bk, EK);
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
                va = plan_window(cur.ga + p.sh_av, cur.alen, p.sh_av, p.a_total + p.sh_av, EV);
                vb = plan_window(cur.gb + p.sh_bv, cur.blen, p.sh_bv, p.b_total + p.sh_bv, EV);
                in.av = va.head;
                in.bv = va.sup + vb.head;
                bytes += uint32_t((va.bulk + vb.bulk) * sizeof(V));
            } else if (BWD) {
                wg = plan_window(cur.gc + p.sh_gc, len, p.sh_gc, p.c_total + p.sh_gc, EV);
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
    constexpr bool MAPPED = ORD == 1 || ORD >= 3;
    const OrderMap<K> om(ORD == 1 ? p.order : (ORD >= 3 ? 2 : 0));
    const auto km = [om](K x) { return MAPPED ? om(x) : x; };
    const KeyLess<ORD == 2 || ORD == 4> lt;
    constexpr bool PIPE = VB != 0 && !BWD && !REC && IPT * ILP >= 15;
    // Thread tid merges ILP chains; chain c starts at diagonal (c*NT + tid)*IPT
    // and the chains run interleaved, so each thread has ILP independent
    // dependency chains of shared-memory loads in flight.
    int it = 0;
    if constexpr (PIPE) {
        // Forward with payloads, whose merge steps also gather a payload
        // from the stage, and at least 15 merge steps per thread and tile
        // (with fewer the extra arrivals and polls outweigh the overlap):
        // the consumers run one tile ahead.  After merging
        // tile it into registers a warp arrives on consumed[s] (its lanes
        // have read their inputs), waits for the next tile's stage and finds
        // its splits there, and only then waits for every warp's arrival
        // before its outputs overwrite stage s, so warps that finish a merge
        // early search the next tile instead of idling at a barrier.  One
        // lane per warp arrives and polls; the others wait at __syncwarp.
        struct Split {
            int alen, blen;
            int j[ILP];
            K a[ILP], b[ILP];
            bool fast;
        };
        bool timed_out = false;
        // Wait for the stage of iteration q and find this thread's splits in it.
        auto prepare = [&](int q, Split& P) {
            const int s = q % NS;
            const bool ready = !timed_out && mbar_wait(&full[s], (q / NS) & 1);
            if (!ready) {
                if (!timed_out) set_status(&hdr->status, kDevTimeout);
                timed_out = true;
                s_abort[q & 3] = 1;
            }
            P.alen = ready ? info[s].alen : 0;
            P.blen = ready ? info[s].blen : 0;
            const int len = P.alen + P.blen;
            const K* sk = stage_k(s);
            const K* sA = sk + info[s].ak;
            const K* sB = sk + info[s].bk;
            int d[ILP];
#pragma unroll
            for (int c = 0; c < ILP; ++c) d[c] = min((c * NT + tid) * IPT, len);
            split_in_tile<Log2Ceil<TILE + 1>::v>(sA, P.alen, sB, P.blen, d, P.j, km, lt);
            P.fast = true;
#pragma unroll
            for (int c = 0; c < ILP; ++c) {
                const int k = d[c] - P.j[c];
                const int cnt = min(IPT, len - d[c]);
                P.a[c] = K(0);
                P.b[c] = K(0);
                if (cnt > 0) {
                    P.a[c] = km(sA[P.j[c]]);   // may be one past A's window: never taken then
                    P.b[c] = km(sB[k]);
                }
                P.fast = P.fast && cnt == IPT && P.j[c] + IPT <= P.alen && k + IPT <= P.blen;
            }
            P.fast = __all_sync(0xffffffffu, P.fast);
        };
        const int lane = tid & 31;
        Split P;
        if (blockIdx.x < ntiles) prepare(0, P);
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int s = it % NS;
            const StageInfo in = info[s];
            const int alen = P.alen, blen = P.blen, len = alen + blen;
            K* sk = stage_k(s);
            const V* sv = stage_v(s);
            const int ao = in.ak, bo = in.bk, avo = in.av, bvo = in.bv;
            int d[ILP], cnt[ILP], j[ILP], k[ILP];
            K a[ILP], b[ILP];
            const bool fast = P.fast;
#pragma unroll
            for (int c = 0; c < ILP; ++c) {
                d[c] = min((c * NT + tid) * IPT, len);
                cnt[c] = min(IPT, len - d[c]);
                j[c] = P.j[c];
                k[c] = d[c] - j[c];
                a[c] = P.a[c];
                b[c] = P.b[c];
            }
            K okey[ILP][IPT];
            V oval[ILP][IPT];
            uint32_t otag[ILP][TAG ? IPT : 1];
            auto step = [&](int c, int q, auto guard) {
                const bool takeA = decltype(guard)::value
                                       ? (k[c] >= blen) || (j[c] < alen && !lt(b[c], a[c]))
                                       : !lt(b[c], a[c]);
                okey[c][q] = takeA ? a[c] : b[c];
                oval[c][q] = sv[takeA ? avo + j[c] : bvo + k[c]];
                if constexpr (TAG)
                    otag[c][q] = takeA ? uint32_t(in.ga + j[c]) : uint32_t(p.tag_b + in.gb + k[c]);
                j[c] += takeA ? 1 : 0;
                k[c] += takeA ? 0 : 1;
                const K nx = km(sk[takeA ? ao + j[c] : bo + k[c]]);
                a[c] = takeA ? nx : a[c];
                b[c] = takeA ? b[c] : nx;
            };
            if (fast) {
#pragma unroll
                for (int q = 0; q < IPT; ++q)
#pragma unroll
                    for (int c = 0; c < ILP; ++c) step(c, q, BoolC<false>{});
            } else {
#pragma unroll
                for (int q = 0; q < IPT; ++q)
#pragma unroll
                    for (int c = 0; c < ILP; ++c)
                        if (q < cnt[c]) step(c, q, BoolC<true>{});
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&consumed[s]);
            if (t + gridDim.x < ntiles) prepare(it + 1, P);
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&consumed[s], (it / NS) & 1);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();   // every input of stage s has been read
            if (!ok) {
                if (lane == 0) set_status(&hdr->status, kDevTimeout);
                s_abort[it & 3] = 1;
            }
            const int ph = int((in.gc + p.sh_ck) & (EK - 1));
            const int phv = int((in.gc + p.sh_cv) & (EV - 1));
            V* ov = stage_v(s);
#pragma unroll
            for (int c = 0; c < ILP; ++c)
#pragma unroll
                for (int q = 0; q < IPT; ++q)
                    if (q < cnt[c]) {
                        sk[ph + d[c] + q] = MAPPED ? om.inverse(okey[c][q]) : okey[c][q];
                        ov[phv + d[c] + q] = oval[c][q];
                    }
            if constexpr (TAG) {
                uint32_t* ot = stage_t(s);
                const int pht = int((in.gc + p.sh_tag) & 3);
#pragma unroll
                for (int c = 0; c < ILP; ++c)
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
                        if (q < cnt[c]) ot[pht + d[c] + q] = otag[c][q];
            }
            fence_proxy_async_smem();   // the outputs are read by the bulk-store engine
            mbar_arrive(&staged[s]);
            if (s_abort[it & 3]) break;
        }
    } else {
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int s = it % NS;
            const bool ready = mbar_wait(&full[s], (it / NS) & 1);
            if (!ready) {
                set_status(&hdr->status, kDevTimeout);
                s_abort[it & 1] = 1;
            }
            const StageInfo in = info[s];
            const int alen = ready ? in.alen : 0;
            const int blen = ready ? in.blen : 0;
            const int len = alen + blen;
            K* sk = stage_k(s);
            const int ao = in.ak, bo = in.bk;   // A[0] and B[0] of the tile in the stage
            const K* sA = sk + ao;
            const K* sB = sk + bo;
            int d[ILP], cnt[ILP], j[ILP], k[ILP];
            K a[ILP], b[ILP];
            bool fast = true;
#pragma unroll
            for (int c = 0; c < ILP; ++c) {
                d[c] = min((c * NT + tid) * IPT, len);
                cnt[c] = min(IPT, len - d[c]);
            }
            split_in_tile<Log2Ceil<TILE + 1>::v>(sA, alen, sB, blen, d, j, km, lt);
#pragma unroll
            for (int c = 0; c < ILP; ++c) {
                k[c] = d[c] - j[c];
                a[c] = K(0);
                b[c] = K(0);
                if (cnt[c] > 0) {
                    a[c] = km(sA[j[c]]);   // may be one past A's window: never taken then
                    b[c] = km(sB[k[c]]);
                }
                fast = fast && cnt[c] == IPT && j[c] + IPT <= alen && k[c] + IPT <= blen;
            }
            // One loop version per warp: a warp whose threads disagree would run both.
            fast = __all_sync(0xffffffffu, fast);
            if constexpr (!BWD) {
                K okey[ILP][IPT];
                V oval[ILP][VB ? IPT : 1];
                uint32_t otag[ILP][TAG ? IPT : 1];
                uint32_t obit[ILP];   // REC: bit q set when output q of chain c came from B
                const V* sv = stage_v(s);
                const int avo = in.av, bvo = in.bv;
                if constexpr (REC) {
#pragma unroll
                    for (int c = 0; c < ILP; ++c) obit[c] = 0;
                    // cleared before the barrier below, set after it
                    if (tid < L::WPT) stage_f(s)[tid] = 0;
                }
                // One merge step of chain c (ties take A).  GUARD: some side may
                // run out within the chain's IPT steps (only near the windows' ends).
                auto step = [&](int c, int q, auto guard) {
                    const bool takeA = decltype(guard)::value
                                           ? (k[c] >= blen) || (j[c] < alen && !lt(b[c], a[c]))
                                           : !lt(b[c], a[c]);
                    okey[c][q] = takeA ? a[c] : b[c];
                    if constexpr (VB != 0) oval[c][q] = sv[takeA ? avo + j[c] : bvo + k[c]];
                    if constexpr (TAG)
                        otag[c][q] = takeA ? uint32_t(in.ga + j[c]) : uint32_t(p.tag_b + in.gb + k[c]);
                    if constexpr (REC) obit[c] |= (takeA ? 0u : 1u) << q;
                    j[c] += takeA ? 1 : 0;
                    k[c] += takeA ? 0 : 1;
                    const K nx = km(sk[takeA ? ao + j[c] : bo + k[c]]);   // one load from either window
                    a[c] = takeA ? nx : a[c];
                    b[c] = takeA ? b[c] : nx;
                };
                if (fast) {
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
#pragma unroll
                        for (int c = 0; c < ILP; ++c) step(c, q, BoolC<false>{});
                } else {
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
#pragma unroll
                        for (int c = 0; c < ILP; ++c)
                            if (q < cnt[c]) step(c, q, BoolC<true>{});
                }
                named_sync(1, NT);   // every input of stage s has been read
                const int ph = int((in.gc + p.sh_ck) & (EK - 1));
#pragma unroll
                for (int c = 0; c < ILP; ++c)
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
                        if (q < cnt[c])
                            sk[ph + d[c] + q] = MAPPED ? om.inverse(okey[c][q]) : okey[c][q];
                if constexpr (VB != 0) {
                    V* ov = stage_v(s);
                    const int phv = int((in.gc + p.sh_cv) & (EV - 1));
#pragma unroll
                    for (int c = 0; c < ILP; ++c)
#pragma unroll
                        for (int q = 0; q < IPT; ++q)
                            if (q < cnt[c]) ov[phv + d[c] + q] = oval[c][q];
                }
                if constexpr (TAG) {
                    uint32_t* ot = stage_t(s);
                    const int pht = int((in.gc + p.sh_tag) & 3);
#pragma unroll
                    for (int c = 0; c < ILP; ++c)
#pragma unroll
                        for (int q = 0; q < IPT; ++q)
                            if (q < cnt[c]) ot[pht + d[c] + q] = otag[c][q];
                }
                if constexpr (REC) {
                    // a chain's IPT (< 32) bits straddle at most two words
                    uint32_t* sf = stage_f(s);
#pragma unroll
                    for (int c = 0; c < ILP; ++c) {
                        if (cnt[c] > 0 && obit[c] != 0) {
                            const int w = d[c] >> 5, o = d[c] & 31;
                            atomicOr(&sf[w], obit[c] << o);
                            if (o + cnt[c] > 32) atomicOr(&sf[w + 1], obit[c] >> (32 - o));
                        }
                    }
                }
            } else {
                V gval[ILP][IPT];
                int dst[ILP][IPT];
                const V* sg = stage_g(s) + in.av;
                const int pha = int((in.ga + p.sh_cv) & (EV - 1));
                const int boff =
                    ((pha + alen + EV - 1) / EV) * EV + int((in.gb + p.sh_cv2) & (EV - 1));
                auto step = [&](int c, int q, auto guard) {
                    const bool takeA = decltype(guard)::value
                                           ? (k[c] >= blen) || (j[c] < alen && !lt(b[c], a[c]))
                                           : !lt(b[c], a[c]);
                    gval[c][q] = sg[d[c] + q];
                    dst[c][q] = takeA ? pha + j[c] : boff + k[c];
                    j[c] += takeA ? 1 : 0;
                    k[c] += takeA ? 0 : 1;
                    const K nx = km(sk[takeA ? ao + j[c] : bo + k[c]]);   // one load from either window
                    a[c] = takeA ? nx : a[c];
                    b[c] = takeA ? b[c] : nx;
                };
                if (fast) {
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
#pragma unroll
                        for (int c = 0; c < ILP; ++c) step(c, q, BoolC<false>{});
                } else {
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
#pragma unroll
                        for (int c = 0; c < ILP; ++c)
                            if (q < cnt[c]) step(c, q, BoolC<true>{});
                }
                named_sync(1, NT);   // every input of stage s has been read
                V* og = stage_g(s);
#pragma unroll
                for (int c = 0; c < ILP; ++c)
#pragma unroll
                    for (int q = 0; q < IPT; ++q)
                        if (q < cnt[c]) og[dst[c][q]] = gval[c][q];
            }
            fence_proxy_async_smem();   // the outputs are read by the bulk-store engine
            mbar_arrive(&staged[s]);
            if (s_abort[it & 1]) break;
        }
    }
    if ((s_abort[0] || s_abort[1] || s_abort[2] || s_abort[3]) && tid == 0) {
        // Let copies that were issued but never consumed land before exit.
        const int issued = *s_issued;
        for (int q = it; q < issued; ++q) mbar_wait(&full[q % NS], (q / NS) & 1, 100000000ull);
    }
}

}  // namespace cr
