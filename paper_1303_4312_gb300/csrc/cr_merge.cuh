// cr_merge.cuh -- the persistent tile-merge kernels (forward and payload
// backward) for sm_103a.
//
// Each CTA runs one producer warp and NT consumer threads and walks the
// output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...  Because every
// tile carries exactly TILE = NT*IPT output elements (Algorithm 2 with equal
// blocks, Proposition 2), the static round-robin schedule is balanced.
//
//  producer (one lane):  reads the tile record (A window, B window, output
//      offset) written by a partition kernel, then stages the windows into
//      an NS-deep ring of shared-memory buffers with bulk copies (TMA
//      engine, cp.async.bulk + mbarrier transaction counts).  Windows start
//      at arbitrary element offsets: the copy covers the 16-byte aligned
//      superset and the consumers index from the head offset.
//  consumers (NT threads): thread s co-ranks diagonal s*IPT inside the two
//      shared-memory windows (Algorithm 1 again, now over a tile), then merges
//      exactly IPT elements serially (ties take A) and writes them to an
//      output staging buffer in shared memory; one thread then issues bulk
//      stores of the whole tile (the 16-byte aligned interior) and a few
//      threads store the ragged ends with plain stores.
#pragma once

#include "cr_device.cuh"

namespace cr {

template <int VB> struct VBits { using T = uint32_t; };
template <> struct VBits<8> { using T = uint64_t; };

__host__ __device__ constexpr size_t align_up_sz(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Per-stage description written by the producer for the consumers.
struct StageInfo {
    int64_t ga, gb, gc;      // window starts (elements) in A, B and output
    int32_t alen, blen;      // window lengths
    int32_t ak, bk;          // smem element offset of A[ga] / B[gb] in the key stage
    int32_t av, bv;          // same in the payload / gradient stage
};
static_assert(sizeof(StageInfo) == 48, "StageInfo size");

// Shared-memory layout of one kernel instantiation (host and device agree).
template <class K, int VB, bool TAG, int NT, int IPT, int NS, bool BWD>
struct Layout {
    static constexpr int TILE = NT * IPT;
    static constexpr int KS = sizeof(K);
    static constexpr int EK = 16 / KS;
    static constexpr int VS = VB ? VB : 4;
    static constexpr int EV = 16 / VS;
    // stage buffers (elements)
    static constexpr int SK = TILE + 4 * EK;                      // A and B key windows
    static constexpr int SV = (VB && !BWD) ? TILE + 4 * EV : 0;   // A and B payload windows
    static constexpr int SG = BWD ? TILE + 2 * EV : 0;            // gradient window of C
    static constexpr size_t STAGE_K = align_up_sz(size_t(SK) * KS, 128);
    static constexpr size_t STAGE_V = align_up_sz(size_t(SV) * VS, 128);
    static constexpr size_t STAGE_G = align_up_sz(size_t(SG) * VS, 128);
    static constexpr size_t STAGE = STAGE_K + STAGE_V + STAGE_G;
    // output buffers
    static constexpr int OK = BWD ? 0 : TILE + 2 * EK;
    static constexpr int OV = BWD ? TILE + 4 * EV : (VB ? TILE + 2 * EV : 0);
    static constexpr int OT = (TAG && !BWD) ? TILE + 8 : 0;
    static constexpr size_t OUT_K = align_up_sz(size_t(OK) * KS, 128);
    static constexpr size_t OUT_V = align_up_sz(size_t(OV) * VS, 128);
    static constexpr size_t OUT_T = align_up_sz(size_t(OT) * 4, 128);
    static constexpr size_t OUT = OUT_K + OUT_V + OUT_T;
    // regions
    static constexpr size_t BAR_OFF = 0;                       // full[NS], empty[NS], flags
    static constexpr size_t INFO_OFF = 256;
    static constexpr size_t STAGE_OFF = align_up_sz(INFO_OFF + NS * sizeof(StageInfo), 128);
    static constexpr size_t OUT_OFF = STAGE_OFF + NS * STAGE;
    static constexpr size_t TOTAL = OUT_OFF + 2 * OUT + 128;  // + slack for one-past reads
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
// ph = g0 mod E.  bulk part (whole 16-byte chunks): issued by the caller
// thread; edge elements: thread `lane` in [0, 2E) of a helper group.
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


// ---------------------------------------------------------------------------
// Forward (BWD = false): C keys [+ payloads] [+ tags].
// Backward (BWD = true): gA / gB from gC, routed by the same merge decisions.
// ---------------------------------------------------------------------------
template <class K, int VB, bool TAG, int NT, int IPT, int NS, bool BWD>
__global__ void __launch_bounds__(NT + 32, 1) merge_tiles_kernel(const MergeArgs p) {
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

    auto stage_k = [&](int s) { return reinterpret_cast<K*>(smem + L::STAGE_OFF + s * L::STAGE); };
    auto stage_v = [&](int s) {
        return reinterpret_cast<V*>(smem + L::STAGE_OFF + s * L::STAGE + L::STAGE_K);
    };
    auto stage_g = [&](int s) {
        return reinterpret_cast<V*>(smem + L::STAGE_OFF + s * L::STAGE + L::STAGE_K + L::STAGE_V);
    };
    auto out_k = [&](int b) { return reinterpret_cast<K*>(smem + L::OUT_OFF + b * L::OUT); };
    auto out_v = [&](int b) {
        return reinterpret_cast<V*>(smem + L::OUT_OFF + b * L::OUT + L::OUT_K);
    };
    auto out_t = [&](int b) {
        return reinterpret_cast<uint32_t*>(smem + L::OUT_OFF + b * L::OUT + L::OUT_K + L::OUT_V);
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
        const int ob = it & 1;
        if (tid == 0) bulk_wait_read<1>();   // output buffer `ob` (tile it-2) drained
        named_sync(1, NT);
        bool ready = mbar_wait(&full[s], (it / NS) & 1);
        if (!ready) {
            set_status(&hdr->status, kDevTimeout);
            *s_abort = 1;
        }
        const StageInfo in = info[s];
        const int len = ready ? in.alen + in.blen : 0;
        const int d = min(tid * IPT, len);
        const int cnt = min(IPT, len - d);
        const K* sk = stage_k(s);
        const int ao = in.ak, bo = in.bk;
        const int alen = in.alen, blen = in.blen;
        int j = 0;
        if (cnt > 0) {
            j = co_rank<K, int>(d, alen, blen, [&](int x) { return sk[ao + x]; },
                                [&](int x) { return sk[bo + x]; });
        }
        int k = d - j;
        K a = K(0), b = K(0);
        if (cnt > 0) {
            a = sk[ao + j];   // may be one past A's window: unused then
            b = sk[bo + k];
        }
        if (!BWD) {
            K* ok = out_k(ob);
            const int ph = int(in.gc & (EK - 1));
            V* ov = out_v(ob);
            const int phv = int(in.gc & (EV - 1));
            uint32_t* ot = out_t(ob);
            const int pht = int(in.gc & 3);
            const V* sv = stage_v(s);
            const int avo = in.av, bvo = in.bv;
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (q < cnt) {
                    const bool takeB = (k < blen) && (j >= alen || b < a);
                    ok[ph + d + q] = takeB ? b : a;
                    if constexpr (VB != 0) ov[phv + d + q] = sv[takeB ? bvo + k : avo + j];
                    if constexpr (TAG)
                        ot[pht + d + q] = takeB ? uint32_t(p.tag_b + in.gb + k) : uint32_t(in.ga + j);
                    const K nx = sk[takeB ? bo + k + 1 : ao + j + 1];
                    if (takeB) { b = nx; ++k; } else { a = nx; ++j; }
                }
            }
        } else {
            V* oa = out_v(ob);
            const int pha = int(in.ga & (EV - 1));
            const int ob_off = int(((pha + alen + EV - 1) / EV) * EV);
            V* obb = oa + ob_off;
            const int phb = int(in.gb & (EV - 1));
            const V* sg = stage_g(s) + in.av;
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                if (q < cnt) {
                    const bool takeB = (k < blen) && (j >= alen || b < a);
                    const V g = sg[d + q];
                    if (takeB) obb[phb + k] = g; else oa[pha + j] = g;
                    const K nx = sk[takeB ? bo + k + 1 : ao + j + 1];
                    if (takeB) { b = nx; ++k; } else { a = nx; ++j; }
                }
            }
        }
        fence_proxy_async_smem();
        named_sync(1, NT);
        if (*s_abort) break;
        // Stage s is consumed; output buffer ob is complete.
        if (!BWD) {
            K* C = static_cast<K*>(p.ck);
            if (tid == 0) {
                mbar_arrive(&empty[s]);
                store_bulk(C, out_k(ob), in.gc, len, EK);
                if constexpr (VB != 0) store_bulk(static_cast<V*>(p.cv), out_v(ob), in.gc, len, EV);
                if constexpr (TAG) store_bulk(p.ctag, out_t(ob), in.gc, len, 4);
                bulk_commit();
            } else if (tid <= 2 * EK) {
                store_edges(C, out_k(ob), in.gc, len, EK, tid - 1);
            } else if (VB != 0 && tid >= 32 && tid < 32 + 2 * EV) {
                store_edges(static_cast<V*>(p.cv), out_v(ob), in.gc, len, EV, tid - 32);
            } else if (TAG && tid >= 64 && tid < 64 + 8) {
                store_edges(p.ctag, out_t(ob), in.gc, len, 4, tid - 64);
            }
        } else {
            V* gA = static_cast<V*>(p.cv);
            V* gB = static_cast<V*>(p.cv2);
            const int pha = int(in.ga & (EV - 1));
            const int ob_off = int(((pha + in.alen + EV - 1) / EV) * EV);
            if (tid == 0) {
                mbar_arrive(&empty[s]);
                store_bulk(gA, out_v(ob), in.ga, in.alen, EV);
                store_bulk(gB, out_v(ob) + ob_off, in.gb, in.blen, EV);
                bulk_commit();
            } else if (tid <= 2 * EV) {
                store_edges(gA, out_v(ob), in.ga, in.alen, EV, tid - 1);
            } else if (tid >= 32 && tid < 32 + 2 * EV) {
                store_edges(gB, out_v(ob) + ob_off, in.gb, in.blen, EV, tid - 32);
            }
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
