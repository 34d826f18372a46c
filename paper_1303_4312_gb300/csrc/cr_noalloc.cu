// cr_noalloc.cu -- cr_stable_merge_noalloc: the keys-only stable merge for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden
// -- for example a host callback or a library hook invoked while the
// application owns every allocation and has none to lend, a real-time loop
// that must not enter the allocator, or a plug-in whose host framework gives
// it buffers for inputs and outputs but no scratch space.  The regular entry
// point cr_stable_merge needs a caller-provided workspace for its tile table;
// this one keeps that table in a fixed-size array that is part of the
// library's device image instead.
//
// The array (kNoAllocScratchBytes, 4 MiB) is a file-scope __device__ symbol:
// every GPU on which the library is loaded holds it until the process exits.
// In host code the symbol's name is only a host-side stand-in, so the device
// address is looked up with cudaGetSymbolAddress on the first call on each
// device (with that device current) and then passed to the kernels.  Only a
// successful lookup is kept; a failed one is retried by the next call.  That
// first call should be made before any stream capture begins.  The kept
// address belongs to the device context it was looked up in: after
// cudaDeviceReset the library must not be called again in this process.
//
// All calls share the one array: two calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on it and may produce
// wrong output.  Serialise them on one stream.  The array keeps whatever the
// last call left there; the only field that must start at zero, the status
// word, is reset by the first kernel of every call, and every tile record is
// written before it is read.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/corank.h"
#include "cr_launch.cuh"

namespace cr {
void set_last_error(const char* msg);   // cr_abi.cu
}

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_scratch_mu[kMaxDev];
void* g_scratch_ptr[kMaxDev];   // nullptr until a lookup on that device succeeded

cr_status na_fail(cr_status st, const char* fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    cr::set_last_error(buf);
    return st;
}

// Device address of the scratch array on the current device.  A successful
// lookup is kept for later calls; a failed one is not, so the next call
// tries again.
cr_status scratch_on_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return na_fail(CR_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDev) return na_fail(CR_EUNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu[dev]);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            if (e != cudaSuccess) (void)cudaGetLastError();   // not sticky: clear it
            return na_fail(CR_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                           cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CR_OK;
}

bool ranges_overlap(const void* a, int64_t abytes, const void* b, int64_t bbytes) {
    if (abytes <= 0 || bbytes <= 0) return false;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
    return a0 < b0 + uintptr_t(bbytes) && b0 < a0 + uintptr_t(abytes);
}

}  // namespace

extern "C" cr_status cr_stable_merge_noalloc(int key_type, const void* A, int64_t m,
                                             const void* B, int64_t n, void* C,
                                             uint32_t* C_tag, cr_stream stream) {
    const int ks = cr::key_type_bytes(key_type);
    if (ks == 0) return na_fail(CR_EINVAL, "unknown key type %d", key_type);
    if (m < 0 || n < 0) return na_fail(CR_EINVAL, "negative size");
    const int64_t max_tiles =
        int64_t((kNoAllocScratchBytes - size_t(cr::kHeaderBytes)) / sizeof(cr::TileRec));
    // Refused before m + n is formed: no table of any tile shape could hold
    // more than max_tiles * largest_tile elements (far below 2^63), so the
    // sum and the tile count below cannot overflow.
    int64_t largest_tile = 0;
    for (int s = 0; s < cr::kNumShapes; ++s)
        largest_tile = cr::tile_of_shape(s) > largest_tile ? cr::tile_of_shape(s) : largest_tile;
    const int64_t cap = max_tiles * largest_tile;
    if (m > cap || n > cap - m)
        return na_fail(CR_EINVAL,
                       "m + n exceeds the %lld elements the fixed %zu-byte scratch array can "
                       "plan with any tile shape; use cr_stable_merge with a workspace",
                       static_cast<long long>(cap), kNoAllocScratchBytes);
    const int64_t mn = m + n;
    const int shape = cr::current_shape(ks, 0, cr::geometry_class(m, n));
    const int64_t tile = cr::tile_of_shape(shape);
    const int64_t ntiles = (mn + tile - 1) / tile;
    if (ntiles > max_tiles)
        return na_fail(CR_EINVAL,
                       "m + n = %lld exceeds the %lld elements the fixed %zu-byte scratch "
                       "array can plan for this key type; use cr_stable_merge with a workspace",
                       static_cast<long long>(mn), static_cast<long long>(max_tiles * tile),
                       kNoAllocScratchBytes);
    // Arrays need only be aligned to their element size (the kernels
    // address whole 16-byte chunks from the boundary below each start).
    struct { const void* p; int64_t count; int elem; const char* name; } arrs[4] = {
        {A, m, ks, "A"}, {B, n, ks, "B"}, {C, mn, ks, "C"}, {C_tag, C_tag ? mn : 0, 4, "C tag"}};
    for (auto& a : arrs) {
        if (a.count == 0) continue;
        if (a.p == nullptr) return na_fail(CR_EINVAL, "%s is NULL", a.name);
        if (reinterpret_cast<uintptr_t>(a.p) % uintptr_t(a.elem))
            return na_fail(CR_EALIGN, "%s is not aligned to %d bytes", a.name, a.elem);
    }
    if (ranges_overlap(C, mn * ks, A, m * ks) || ranges_overlap(C, mn * ks, B, n * ks) ||
        (C_tag && (ranges_overlap(C_tag, mn * 4, A, m * ks) ||
                   ranges_overlap(C_tag, mn * 4, B, n * ks) ||
                   ranges_overlap(C_tag, mn * 4, C, mn * ks))))
        return na_fail(CR_EALIAS, "an output overlaps an input");
    if (C_tag && mn > (int64_t(1) << 32)) return na_fail(CR_EINVAL, "tags need m + n <= 2^32");
    if (mn == 0) {
        cr::set_last_error("");
        return CR_OK;
    }
    void* scratch = nullptr;
    const cr_status s = scratch_on_current_device(&scratch);
    if (s != CR_OK) return s;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cr::MergeArgs a{};
    a.order = cr::key_type_order(key_type);
    a.ak = A;
    a.bk = B;
    a.ck = C;
    a.ctag = C_tag;
    a.a_total = m;
    a.b_total = n;
    a.c_total = mn;
    a.tag_b = m;
    a.ws = scratch;
    auto run = [&](auto ops) {
        cudaError_t e = ops.partition_single(A, m, B, n, tile, ntiles, scratch, a.order, st);
        if (e != cudaSuccess) return e;
        return ops.merge_fwd(shape, 0, C_tag != nullptr, a, ntiles, st);
    };
    const cudaError_t e = cr::with_key_ops(key_type, run);
    if (e != cudaSuccess)
        return na_fail(CR_ECUDA, "merge launch: %s", cudaGetErrorString(e));
    cr::set_last_error("");
    return CR_OK;
}
