// cr_route.cu -- backward of a recorded merge pass: the payload gradient is
// routed by the merge decisions the forward recorded, without reading keys.
//
// The forward (merge_tiles_kernel with REC) left, per tile t of the pass, the
// tile record (A window at ga, B window at gb, output at gc; alen + blen
// outputs) and WPT = TILE/32 flag words, bit x set when output gc + x came
// from B.  By the prefix property of Lemma 1 the outputs taken from A are
// A[ga], A[ga+1], ... in output order, and likewise for B, so output x is
// B[gb + rb] with rb = number of set bits before x, or A[ga + x - rb]:
//     gX[gb + rb] = gY[gc + x]   or   gX[ga + x - rb] = gY[gc + x].
// Every input position belongs to exactly one tile window, so each gX
// element is written once.  Traffic per element: gY read, gX written, one bit
// of flags, and a 32-byte record per tile.  A tile's output window follows
// from its index and the pass geometry (pair q = t / tpp starts at 2qw; the
// tile at (t - q*tpp) * TILE inside it), so the gradient and flag loads are
// issued together with the record load instead of after it; the record's
// own output window is then checked against it.
#include "cr_launch.cuh"
#include "cr_merge.cuh"

namespace cr {

namespace {

constexpr int kRouteThreads = 128;
constexpr int kRouteMaxTile = 4096;   // the largest tile a recorded pass may use
static_assert(kRouteMaxTile == kMaxRecordTile, "recorded-pass tile limit");
constexpr int kRouteMaxWords = kRouteMaxTile / 32;

// Asynchronous global -> shared copies (no registers held while in flight).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src),
                     "n"(BYTES)
                     : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// One CTA per tile; dynamic shared memory holds the tile's gradients
// (tile * VB bytes, 16-byte aligned).
template <int VB>
__global__ void __launch_bounds__(kRouteThreads) route_recorded_kernel(
    void* ws, const uint32_t* __restrict__ flags, int64_t flag_words, int64_t N, int64_t w,
    int64_t tile, int64_t tpp, int64_t ntiles, const void* __restrict__ gY,
    void* __restrict__ gX) {
    using V = typename VBits<VB>::T;
    extern __shared__ __align__(16) unsigned char route_smem[];
    V* s_val = reinterpret_cast<V*>(route_smem);
    __shared__ uint32_t s_word[kRouteMaxWords + 1];
    __shared__ int32_t s_pre[kRouteMaxWords + 1];   // set bits in the words before
    __shared__ int32_t s_wsum[kRouteThreads / 32];

    WsHeader* hdr = static_cast<WsHeader*>(ws);
    const int tid = threadIdx.x;
    const int64_t t = blockIdx.x;
    // A table for another tile size or tile count is refused as a whole.
    if (hdr->tile != tile || hdr->ntiles != ntiles) {
        if (t == 0 && tid == 0) set_status(&hdr->status, kDevInternal);
        return;
    }
    const int wpt = int(tile / 32);
    if ((t + 1) * wpt > flag_words) {
        if (tid == 0) set_status(&hdr->status, kDevInternal);
        return;
    }
    // output window of tile t from the pass geometry (t < ntiles, so q is a
    // pair of the pass and gc + len <= N); t < 2^31 (one CTA per tile)
    const int64_t q = int64_t(uint32_t(t) / uint32_t(tpp));
    const int64_t a0 = 2 * q * w;
    const int64_t pair = (N - a0 < 2 * w) ? N - a0 : 2 * w;
    const int64_t r0 = (t - q * tpp) * tile;
    const int64_t gc = a0 + r0;
    const int len = int(pair - r0 < tile ? pair - r0 : tile);

    // stage the tile's gradients and flag words (16-byte chunks when the
    // window starts on a 16-byte boundary; whole chunks only, so nothing past
    // gY[gc + len) is read), while the record loads
    const V* gy = static_cast<const V*>(gY) + gc;
    constexpr int E = 16 / VB;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(gy) & 15u) == 0) {
        const int chunks = len / E;
        for (int k = tid; k < chunks; k += kRouteThreads) cp_async<16>(s_val + k * E, gy + k * E);
        done = chunks * E;
    }
    for (int x = done + tid; x < len; x += kRouteThreads) cp_async<VB>(s_val + x, gy + x);
    for (int k = tid; k < wpt; k += kRouteThreads) cp_async<4>(s_word + k, flags + t * wpt + k);
    const TileRec r = ws_recs(ws)[t];
    cp_async_wait_all();
    __syncthreads();

    const bool ok = len > 0 && r.gc == gc && r.alen >= 0 && r.blen >= 0 &&
                    r.alen + r.blen == len && r.ga >= 0 && r.gb >= 0 &&
                    r.ga + r.alen <= N && r.gb + r.blen <= N;
    if (!ok) {
        if (tid == 0) set_status(&hdr->status, kDevInternal);
        return;
    }

    // exclusive prefix of the flag words' bit counts (one word per thread,
    // then up to one more: wpt <= 128 = kRouteThreads)
    const uint32_t fw = tid < wpt ? s_word[tid] : 0u;
    const int c = __popc(fw);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if ((tid & 31) >= o) incl += u;
    }
    if ((tid & 31) == 31) s_wsum[tid >> 5] = incl;
    __syncthreads();
    int off = 0;
    for (int k = 0; k < (tid >> 5); ++k) off += s_wsum[k];
    s_pre[tid] = off + incl - c;
    if (tid == 0) {
        s_pre[kRouteMaxWords] = s_wsum[0] + s_wsum[1] + s_wsum[2] + s_wsum[3];
        if (wpt <= kRouteMaxWords) s_word[wpt] = 0u;   // read below only when len == tile
    }
    __syncthreads();
    // The record must take exactly blen outputs from B; then every rank
    // below stays inside its window.  A tile that does not is refused.
    {
        const int lw = len >> 5, lb = len & 31;
        const int before = lw < kRouteMaxWords ? s_pre[lw] : s_pre[kRouteMaxWords];
        const int nb = before + (lb ? __popc(s_word[lw] & ((1u << lb) - 1u)) : 0);
        if (nb != r.blen) {
            if (tid == 0) set_status(&hdr->status, kDevInternal);
            return;
        }
    }

    // x = tid + 128 i: a warp's 32 outputs are exactly flag word x / 32
    // (warp-uniform loads), and output x's bit is the lane's bit
    V* const pa = static_cast<V*>(gX) + r.ga;
    V* const pb = static_cast<V*>(gX) + r.gb;
    const int lane = tid & 31;
    const uint32_t below = (1u << lane) - 1u;
    for (int x = tid; x < len; x += kRouteThreads) {
        const uint32_t word = s_word[x >> 5];
        const int rb = s_pre[x >> 5] + __popc(word & below);
        V* const dst = ((word >> lane) & 1u) ? pb + rb : pa + (x - rb);
        *dst = s_val[x];
    }
}

// Backward of a recorded run formation or merge block: one CTA per chunk of
// `chunk` elements scatters the chunk's gradients through its permutation
// in shared memory (gX[perm[x]] = gY[x]) and stores them coalesced.  Entries
// outside the chunk are skipped (the permutation comes from the forward).
constexpr int kSortRouteThreads = 256;
constexpr int64_t kRouteMaxChunk = 4096;

template <int VB>
__global__ void __launch_bounds__(kSortRouteThreads) sort_route_kernel(
    int64_t N, int64_t chunk, const uint16_t* __restrict__ perm, const void* __restrict__ gY,
    void* __restrict__ gX) {
    using V = typename VBits<VB>::T;
    extern __shared__ __align__(16) unsigned char route_smem[];
    V* s = reinterpret_cast<V*>(route_smem);
    const int64_t base = int64_t(blockIdx.x) * chunk;
    const int len = int(N - base < chunk ? N - base : chunk);
    const V* gy = static_cast<const V*>(gY) + base;
    for (int x = threadIdx.x; x < len; x += kSortRouteThreads) {
        const int p = perm[base + x];
        if (p < len) s[p] = gy[x];
    }
    __syncthreads();
    V* gx = static_cast<V*>(gX) + base;
    for (int x = threadIdx.x; x < len; x += kSortRouteThreads) gx[x] = s[x];
}

}  // namespace

cudaError_t chunk_route_recorded(int vb, int64_t N, int64_t chunk, const uint16_t* perm,
                                 const void* gY, void* gX, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    if (chunk <= 0 || chunk > kRouteMaxChunk) return cudaErrorInvalidValue;
    const int64_t runs = (N + chunk - 1) / chunk;
    if (runs > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t smem = size_t(chunk) * size_t(vb);   // 32 KB at most
    if (vb == 4)
        sort_route_kernel<4><<<unsigned(runs), kSortRouteThreads, smem, st>>>(N, chunk, perm, gY,
                                                                             gX);
    else if (vb == 8)
        sort_route_kernel<8><<<unsigned(runs), kSortRouteThreads, smem, st>>>(N, chunk, perm, gY,
                                                                             gX);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t sort_route_recorded(int vb, int64_t N, const uint16_t* perm, const void* gY, void* gX,
                                cudaStream_t st) {
    return chunk_route_recorded(vb, N, kSortRun, perm, gY, gX, st);
}

cudaError_t route_recorded(int vb, void* ws, const uint32_t* flags, int64_t flag_words, int64_t N,
                           int64_t w, int64_t tile, const void* gY, void* gX, cudaStream_t st) {
    if (tile <= 0 || tile > kRouteMaxTile || tile % 32 != 0 || w < 1 || w > N)
        return cudaErrorInvalidValue;
    int64_t tpp = 1, npairs = 0;
    const int64_t ntiles = pass_tiles(N, w, tile, &tpp, &npairs);
    if (ntiles <= 0) return cudaSuccess;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned grid = unsigned(ntiles);
    const size_t smem = size_t(tile) * size_t(vb);   // <= 32 KB: no opt-in needed
    if (vb == 4)
        route_recorded_kernel<4><<<grid, kRouteThreads, smem, st>>>(ws, flags, flag_words, N, w,
                                                                    tile, tpp, ntiles, gY, gX);
    else if (vb == 8)
        route_recorded_kernel<8><<<grid, kRouteThreads, smem, st>>>(ws, flags, flag_words, N, w,
                                                                    tile, tpp, ntiles, gY, gX);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace cr
