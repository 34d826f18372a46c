// cr_abi.cu -- the extern "C" entry points declared in include/corank.h:
// argument validation, workspace sizing, and stream-ordered launches of the
// partition (co-rank) and tile-merge kernels.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <atomic>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/corank.h"
#include "cr_launch.cuh"

using cr::KeyOps;

namespace {

thread_local std::string g_last_error;

cr_status fail(cr_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

cr_status ok() {
    g_last_error.clear();
    return CR_OK;
}

cr_status cuda_fail(cudaError_t e, const char* what) {
    return fail(CR_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

int key_bytes(int key_type) { return cr::key_type_bytes(key_type); }
int key_order(int key_type) { return cr::key_type_order(key_type); }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// A device array argument: `count` elements of `elem` bytes.  Data arrays
// (keys, payloads, tags, gradients) may start at any multiple of their
// element size, so that a window of a larger array can be passed as it is;
// library-format buffers (source flags) set `align` to 16.
struct Arr {
    const void* p;
    int64_t count;
    int64_t elem;
    const char* name;
    int64_t align = 0;   // 0: the element size
    int64_t bytes() const { return count * elem; }
};

// Largest element count accepted for one array: every sum of two counts and
// every count times an element width (at most 8 bytes) stays inside int64.
constexpr int64_t kMaxElems = int64_t(1) << 59;

bool bad_size(int64_t x) { return x < 0 || x > kMaxElems; }

cr_status check_arr(const Arr& a) {
    if (a.count < 0) return fail(CR_EINVAL, "%s: negative length", a.name);
    if (a.count == 0) return CR_OK;
    if (a.p == nullptr) return fail(CR_EINVAL, "%s is NULL with %lld elements", a.name,
                                    static_cast<long long>(a.count));
    const int64_t al = a.align > 0 ? a.align : a.elem;
    if (a.count > INT64_MAX / a.elem)
        return fail(CR_EINVAL, "%s: %lld elements of %lld bytes overflow the address space",
                    a.name, static_cast<long long>(a.count), static_cast<long long>(a.elem));
    if (reinterpret_cast<uintptr_t>(a.p) % uintptr_t(al) != 0)
        return fail(CR_EALIGN, "%s is not aligned to %lld bytes", a.name,
                    static_cast<long long>(al));
    return CR_OK;
}

bool overlap(const Arr& x, const Arr& y) {
    if (x.count <= 0 || y.count <= 0) return false;
    const uintptr_t x0 = reinterpret_cast<uintptr_t>(x.p), x1 = x0 + uintptr_t(x.bytes());
    const uintptr_t y0 = reinterpret_cast<uintptr_t>(y.p), y1 = y0 + uintptr_t(y.bytes());
    return x0 < y1 && y0 < x1;
}

cr_status check_no_alias(const Arr* outs, int nout, const Arr* ins, int nin) {
    for (int o = 0; o < nout; ++o) {
        for (int i = 0; i < nin; ++i)
            if (overlap(outs[o], ins[i]))
                return fail(CR_EALIAS, "output %s overlaps input %s", outs[o].name, ins[i].name);
        for (int q = o + 1; q < nout; ++q)
            if (overlap(outs[o], outs[q]))
                return fail(CR_EALIAS, "outputs %s and %s overlap", outs[o].name, outs[q].name);
    }
    return CR_OK;
}

// Result slot of the host-result cr_co_rank: one pair per device, in this
// library's device image (the call allocates nothing).  Its device address is
// looked up once per device; calls on one device take turns on it.
constexpr int kMaxResultDevices = 64;
__device__ int64_t g_co_rank_result[2];
std::mutex g_result_mu[kMaxResultDevices];
int64_t* g_result_ptr[kMaxResultDevices];

constexpr size_t kRecBytes = sizeof(cr::TileRec);

size_t single_ws_bytes(int64_t ntiles) {
    return size_t(cr::kHeaderBytes) + size_t(ntiles) * kRecBytes;
}

int64_t batched_max_tiles(int64_t tile, int64_t nseg, int64_t a_total, int64_t b_total) {
    return (a_total + b_total + tile - 1) / tile + nseg;
}

size_t batched_ws_bytes(int64_t max_tiles, int64_t nseg) {
    return size_t(cr::kHeaderBytes) + size_t(max_tiles) * kRecBytes +
           size_t(nseg + 1) * sizeof(int64_t);
}

cr_status check_ws(const void* ws, size_t have, size_t need) {
    if (ws == nullptr) return fail(CR_EINVAL, "workspace is NULL");
    if (!aligned16(ws)) return fail(CR_EALIGN, "workspace is not 16-byte aligned");
    if (have < need)
        return fail(CR_ENOSPACE, "workspace has %zu bytes, needs %zu", have, need);
    return CR_OK;
}

template <class F>
cudaError_t by_key(int key_type, F&& f) {
    return cr::with_key_ops(key_type, static_cast<F&&>(f));
}

#define CR_TRY(expr)                       \
    do {                                   \
        const cr_status _s = (expr);       \
        if (_s != CR_OK) return _s;        \
    } while (0)

cr_status check_key_type(int key_type) {
    if (key_bytes(key_type) == 0) return fail(CR_EINVAL, "unknown key type %d", key_type);
    return CR_OK;
}

cr_status check_vb(int vb, bool allow_zero) {
    if (vb == 4 || vb == 8 || (allow_zero && vb == 0)) return CR_OK;
    return fail(CR_EINVAL, "payload width %d not supported (4 or 8%s)", vb,
                allow_zero ? ", or 0 for keys only" : "");
}

// Validation shared by every forward single-merge entry point.
cr_status check_forward(int key_type, int vb, const void* Ak, const void* Av, int64_t m,
                        const void* Bk, const void* Bv, int64_t n, const void* Ck,
                        const void* Cv, const uint32_t* tag) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(vb, true));
    if (bad_size(m) || bad_size(n)) return fail(CR_EINVAL, "bad size (m=%lld, n=%lld)",
                                    static_cast<long long>(m), static_cast<long long>(n));
    const int ks = key_bytes(key_type);
    const int64_t mn = m + n;
    const Arr ins[4] = {{Ak, m, ks, "A"}, {Bk, n, ks, "B"},
                        {vb ? Av : nullptr, vb ? m : 0, vb, "A payload"},
                        {vb ? Bv : nullptr, vb ? n : 0, vb, "B payload"}};
    const Arr outs[3] = {{Ck, mn, ks, "C"},
                         {vb ? Cv : nullptr, vb ? mn : 0, vb, "C payload"},
                         {tag, tag ? mn : 0, 4, "C tag"}};
    for (const Arr& a : ins) CR_TRY(check_arr(a));
    for (const Arr& a : outs) CR_TRY(check_arr(a));
    CR_TRY(check_no_alias(outs, 3, ins, 4));
    if (tag && mn > (int64_t(1) << 32))
        return fail(CR_EINVAL, "source tags need m + n <= 2^32");
    return CR_OK;
}

cr_status check_backward(int key_type, int vb, const void* Ak, int64_t m, const void* Bk,
                         int64_t n, const void* gC, const void* gA, const void* gB) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(vb, false));
    if (bad_size(m) || bad_size(n)) return fail(CR_EINVAL, "negative or too large size");
    const int ks = key_bytes(key_type);
    const Arr ins[3] = {{Ak, m, ks, "A"}, {Bk, n, ks, "B"}, {gC, m + n, vb, "gC"}};
    const Arr outs[2] = {{gA, m, vb, "gA"}, {gB, n, vb, "gB"}};
    for (const Arr& a : ins) CR_TRY(check_arr(a));
    for (const Arr& a : outs) CR_TRY(check_arr(a));
    return check_no_alias(outs, 2, ins, 3);
}

// Shape of a single merge of m and n elements (its geometry class).
int shape_of(int key_type, int vb, int64_t m, int64_t n) {
    return cr::current_shape(key_bytes(key_type), vb, cr::geometry_class(m, n));
}

// Shapes of batched and merge-pass calls: classes of their own (their
// segments and runs are not known on the host).
int shape_batched(int key_type, int vb) {
    return cr::current_shape(key_bytes(key_type), vb, cr::kClassBatched);
}
int shape_pass(int key_type, int vb) {
    return cr::current_shape(key_bytes(key_type), vb, cr::kClassPass);
}

int64_t single_tiles(int shape, int64_t m, int64_t n, int64_t* tile_out) {
    const int64_t tile = cr::tile_of_shape(shape);
    if (tile_out) *tile_out = tile;
    return (m + n + tile - 1) / tile;
}

// Grid-level co-rank pass of a single merge (writes the tile table).
cr_status launch_partition(int shape, int key_type, const void* Ak, int64_t m, const void* Bk,
                           int64_t n, void* ws, size_t ws_bytes, cudaStream_t st) {
    int64_t tile = 0;
    const int64_t ntiles = single_tiles(shape, m, n, &tile);
    CR_TRY(check_ws(ws, ws_bytes, single_ws_bytes(ntiles)));
    cudaError_t e = by_key(key_type, [&](auto ops) {
        return ops.partition_single(Ak, m, Bk, n, tile, ntiles, ws, key_order(key_type), st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "partition launch");
    return CR_OK;
}

cr_status launch_tiles(int shape, int key_type, int vb, const void* Ak, const void* Av, int64_t m,
                       const void* Bk, const void* Bv, int64_t n, void* Ck, void* Cv,
                       uint32_t* tag, void* ws, size_t ws_bytes, cudaStream_t st) {
    const int64_t ntiles = single_tiles(shape, m, n, nullptr);
    CR_TRY(check_ws(ws, ws_bytes, single_ws_bytes(ntiles)));
    cr::MergeArgs a{};
    a.order = key_order(key_type);
    a.ak = Ak;
    a.bk = Bk;
    a.av = Av;
    a.bv = Bv;
    a.ck = Ck;
    a.cv = Cv;
    a.ctag = tag;
    a.a_total = m;
    a.b_total = n;
    a.c_total = m + n;
    a.tag_b = m;
    a.ws = ws;
    cudaError_t e = by_key(key_type, [&](auto ops) {
        return ops.merge_fwd(shape, vb, tag != nullptr, a, ntiles, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "tile merge launch");
    return CR_OK;
}

cr_status launch_tiles_backward(int shape, int key_type, int vb, const void* Ak, int64_t m,
                                const void* Bk, int64_t n, const void* gC, void* gA, void* gB,
                                void* ws, size_t ws_bytes, cudaStream_t st) {
    const int64_t ntiles = single_tiles(shape, m, n, nullptr);
    CR_TRY(check_ws(ws, ws_bytes, single_ws_bytes(ntiles)));
    cr::MergeArgs a{};
    a.order = key_order(key_type);
    a.ak = Ak;
    a.bk = Bk;
    a.gc_in = gC;
    a.cv = gA;
    a.cv2 = gB;
    a.a_total = m;
    a.b_total = n;
    a.c_total = m + n;
    a.ws = ws;
    cudaError_t e =
        by_key(key_type, [&](auto ops) { return ops.merge_bwd(shape, vb, a, ntiles, st); });
    if (e != cudaSuccess) return cuda_fail(e, "tile backward launch");
    return CR_OK;
}

}  // namespace

// Lets other translation units of the library report through cr_last_error().
namespace cr {
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

// Selected tile shape per (key size 4|8, payload width 0|4|8, class
// balanced|skewed|small|batched|pass).  Defaults: 256 x 15 for keys without payload
// (128 x 31 for skewed 8-byte merges), 256 x 7 otherwise.
static std::atomic<int> g_shape[2][3][kNumClasses] = {
    {{{0}, {0}, {0}, {0}, {0}}, {{2}, {2}, {2}, {2}, {2}}, {{2}, {2}, {2}, {2}, {2}}},
    {{{0}, {1}, {0}, {0}, {0}}, {{2}, {2}, {2}, {2}, {2}}, {{2}, {2}, {2}, {2}, {2}}}};

int current_shape(int key_bytes, int vb, int cls) {
    return g_shape[key_bytes == 8 ? 1 : 0][vb / 4][cls].load(std::memory_order_relaxed);
}
}  // namespace cr

extern "C" {

const char* cr_status_string(int status) {
    switch (status) {
        case CR_OK: return "CR_OK";
        case CR_EINVAL: return "CR_EINVAL";
        case CR_EALIAS: return "CR_EALIAS";
        case CR_EALIGN: return "CR_EALIGN";
        case CR_ENOSPACE: return "CR_ENOSPACE";
        case CR_ECUDA: return "CR_ECUDA";
        case CR_ETIMEOUT: return "CR_ETIMEOUT";
        case CR_EUNSUPPORTED: return "CR_EUNSUPPORTED";
        case CR_EINTERNAL: return "CR_EINTERNAL";
        case CR_EBADSEG: return "CR_EBADSEG";
        default: return "CR_UNKNOWN";
    }
}

const char* cr_last_error(void) { return g_last_error.c_str(); }

int cr_abi_version(void) { return 200; }

int64_t cr_tile_size(int key_type, int val_bytes) {
    const int ks = key_bytes(key_type);
    if (ks == 0) return 0;
    if (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) return 0;
    return cr::tile_of_shape(cr::current_shape(ks, val_bytes, 0));
}

int cr_tile_shape_count(void) { return cr::kNumShapes; }

cr_status cr_tile_shape_info(int shape, int* nt, int* ipt, int* ilp) {
    if (shape < 0 || shape >= cr::kNumShapes) return fail(CR_EINVAL, "no tile shape %d", shape);
    if (nt) *nt = cr::kShapes[shape].nt;
    if (ipt) *ipt = cr::kShapes[shape].ipt;
    if (ilp) *ilp = cr::kShapes[shape].ilp;
    return ok();
}

cr_status cr_set_tile_shape(int key_type, int val_bytes, int shape) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, true));
    const int ks = key_bytes(key_type);
    if (!cr::shape_available(ks, val_bytes, shape))
        return fail(CR_EUNSUPPORTED, "tile shape %d does not fit %d-byte keys with %d-byte payloads",
                    shape, ks, val_bytes);
    const bool pass_ok = val_bytes == 0 || cr::tile_of_shape(shape) <= cr::kMaxRecordTile;
    for (int cls = 0; cls < cr::kNumClasses; ++cls)
        if (cls != cr::kClassPass || pass_ok)
            cr::g_shape[ks == 8 ? 1 : 0][val_bytes / 4][cls].store(shape, std::memory_order_relaxed);
    return ok();
}

int cr_get_tile_shape(int key_type, int val_bytes) {
    return cr_get_tile_shape_for(key_type, val_bytes, 0);
}

cr_status cr_set_tile_shape_for(int key_type, int val_bytes, int cls, int shape) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, true));
    if (cls < 0 || cls >= cr::kNumClasses) return fail(CR_EINVAL, "no geometry class %d", cls);
    const int ks = key_bytes(key_type);
    if (!cr::shape_available(ks, val_bytes, shape))
        return fail(CR_EUNSUPPORTED, "tile shape %d does not fit %d-byte keys with %d-byte payloads",
                    shape, ks, val_bytes);
    if (cls == cr::kClassPass && val_bytes != 0 && cr::tile_of_shape(shape) > cr::kMaxRecordTile)
        return fail(CR_EUNSUPPORTED,
                    "tile shape %d: merge passes with payloads are recorded in tiles of at most "
                    "%lld elements", shape, static_cast<long long>(cr::kMaxRecordTile));
    cr::g_shape[ks == 8 ? 1 : 0][val_bytes / 4][cls].store(shape, std::memory_order_relaxed);
    return ok();
}

int cr_get_tile_shape_for(int key_type, int val_bytes, int cls) {
    const int ks = key_bytes(key_type);
    if (ks == 0 || (val_bytes != 0 && val_bytes != 4 && val_bytes != 8)) return -1;
    if (cls < 0 || cls >= cr::kNumClasses) return -1;
    return cr::current_shape(ks, val_bytes, cls);
}

int64_t cr_tile_size_class(int key_type, int val_bytes, int cls) {
    const int ks = key_bytes(key_type);
    if (ks == 0 || (val_bytes != 0 && val_bytes != 4 && val_bytes != 8)) return 0;
    if (cls < 0 || cls >= cr::kNumClasses) return 0;
    return cr::tile_of_shape(cr::current_shape(ks, val_bytes, cls));
}

int64_t cr_tile_size_for(int key_type, int val_bytes, int64_t m, int64_t n) {
    const int ks = key_bytes(key_type);
    if (ks == 0 || (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) || bad_size(m) || bad_size(n))
        return 0;
    return cr::tile_of_shape(cr::current_shape(ks, val_bytes, cr::geometry_class(m, n)));
}

cr_status cr_co_rank_async(int key_type, const void* A, int64_t m, const void* B, int64_t n,
                           int64_t k, int64_t* d_ij, cr_stream stream) {
    CR_TRY(check_key_type(key_type));
    const int ks = key_bytes(key_type);
    if (bad_size(m) || bad_size(n)) return fail(CR_EINVAL, "negative or too large size");
    if (k < 0 || k > m + n)
        return fail(CR_EINVAL, "rank %lld outside [0, %lld]", static_cast<long long>(k),
                    static_cast<long long>(m + n));
    CR_TRY(check_arr({A, m, ks, "A"}));
    CR_TRY(check_arr({B, n, ks, "B"}));
    if (d_ij == nullptr) return fail(CR_EINVAL, "result pointer is NULL");
    if ((reinterpret_cast<uintptr_t>(d_ij) & 7u) != 0)
        return fail(CR_EALIGN, "result pointer is not 8-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = by_key(key_type,
                           [&](auto ops) { return ops.co_rank_one(A, m, B, n, k, d_ij, key_order(key_type), st); });
    if (e != cudaSuccess) return cuda_fail(e, "co_rank launch");
    return ok();
}

cr_status cr_co_rank(int key_type, const void* A, int64_t m, const void* B, int64_t n, int64_t k,
                     int64_t* i_out, int64_t* j_out, cr_stream stream) {
    if (i_out == nullptr || j_out == nullptr) return fail(CR_EINVAL, "result pointer is NULL");
    CR_TRY(check_key_type(key_type));
    if (bad_size(m) || bad_size(n)) return fail(CR_EINVAL, "negative or too large size");
    if (k < 0 || k > m + n)
        return fail(CR_EINVAL, "rank %lld outside [0, %lld]", static_cast<long long>(k),
                    static_cast<long long>(m + n));
    // trivial ranks need no search
    if (k == 0 || k == m + n || m == 0 || n == 0) {
        CR_TRY(check_arr({A, m, key_bytes(key_type), "A"}));
        CR_TRY(check_arr({B, n, key_bytes(key_type), "B"}));
        *i_out = k == 0 ? 0 : (k == m + n ? m : (m == 0 ? 0 : k));
        *j_out = k - *i_out;
        return ok();
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxResultDevices)
        return fail(CR_EUNSUPPORTED, "device %d out of range", dev);
    // The kernel writes into this library's one result slot of the device;
    // the lock keeps it to one call at a time from launch to read-back.
    std::lock_guard<std::mutex> lock(g_result_mu[dev]);
    if (g_result_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_co_rank_result);
        if (e != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return cuda_fail(e, "result slot lookup");
        }
        g_result_ptr[dev] = static_cast<int64_t*>(p);
    }
    CR_TRY(cr_co_rank_async(key_type, A, m, B, n, k, g_result_ptr[dev], stream));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t ij[2] = {-1, -1};
    e = cudaMemcpyAsync(ij, g_result_ptr[dev], sizeof(ij), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "co_rank result read");
    if (ij[0] < 0 || ij[1] < 0 || ij[0] + ij[1] != k)
        return fail(CR_EINTERNAL, "co_rank result (%lld, %lld) is not a split of rank %lld",
                    static_cast<long long>(ij[0]), static_cast<long long>(ij[1]),
                    static_cast<long long>(k));
    *i_out = ij[0];
    *j_out = ij[1];
    return ok();
}

cr_status cr_co_rank_many(int key_type, const void* A, int64_t m, const void* B, int64_t n,
                          const int64_t* d_k, int64_t cnt, int64_t* d_i, int64_t* d_j,
                          cr_stream stream) {
    CR_TRY(check_key_type(key_type));
    const int ks = key_bytes(key_type);
    if (bad_size(m) || bad_size(n) || bad_size(cnt))
        return fail(CR_EINVAL, "negative or too large size");
    CR_TRY(check_arr({A, m, ks, "A"}));
    CR_TRY(check_arr({B, n, ks, "B"}));
    if (cnt == 0) return ok();
    if (!d_k || !d_i || !d_j) return fail(CR_EINVAL, "rank or result array is NULL");
    const Arr outs[2] = {{d_i, cnt, 8, "i"}, {d_j, cnt, 8, "j"}};
    const Arr ins[3] = {{d_k, cnt, 8, "k"}, {A, m, ks, "A"}, {B, n, ks, "B"}};
    CR_TRY(check_no_alias(outs, 2, ins, 3));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = by_key(key_type, [&](auto ops) {
        return ops.co_rank_many(A, m, B, n, d_k, cnt, d_i, d_j, key_order(key_type), st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "co_rank_many launch");
    return ok();
}

cr_status cr_merge_workspace_size(int key_type, int val_bytes, int64_t m, int64_t n,
                                  size_t* bytes) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, true));
    if (bad_size(m) || bad_size(n)) return fail(CR_EINVAL, "negative or too large size");
    if (!bytes) return fail(CR_EINVAL, "bytes is NULL");
    *bytes = single_ws_bytes(single_tiles(shape_of(key_type, val_bytes, m, n), m, n, nullptr));
    return ok();
}

cr_status cr_stable_merge(int key_type, const void* A, int64_t m, const void* B, int64_t n,
                          void* C, uint32_t* C_tag, void* ws, size_t ws_bytes, cr_stream stream) {
    return cr_stable_merge_kv(key_type, 0, A, nullptr, m, B, nullptr, n, C, nullptr, C_tag, ws,
                              ws_bytes, stream);
}

cr_status cr_stable_merge_kv(int key_type, int val_bytes, const void* Ak, const void* Av,
                             int64_t m, const void* Bk, const void* Bv, int64_t n, void* Ck,
                             void* Cv, uint32_t* C_tag, void* ws, size_t ws_bytes,
                             cr_stream stream) {
    CR_TRY(check_forward(key_type, val_bytes, Ak, Av, m, Bk, Bv, n, Ck, Cv, C_tag));
    if (m + n == 0) return ok();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int shape = shape_of(key_type, val_bytes, m, n);
    CR_TRY(launch_partition(shape, key_type, Ak, m, Bk, n, ws, ws_bytes, st));
    CR_TRY(launch_tiles(shape, key_type, val_bytes, Ak, Av, m, Bk, Bv, n, Ck, Cv, C_tag, ws,
                        ws_bytes, st));
    return ok();
}

cr_status cr_stable_merge_kv_backward(int key_type, int val_bytes, const void* Ak, int64_t m,
                                      const void* Bk, int64_t n, const void* gC, void* gA,
                                      void* gB, void* ws, size_t ws_bytes, cr_stream stream) {
    CR_TRY(check_backward(key_type, val_bytes, Ak, m, Bk, n, gC, gA, gB));
    if (m + n == 0) return ok();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int shape = shape_of(key_type, val_bytes, m, n);
    CR_TRY(launch_partition(shape, key_type, Ak, m, Bk, n, ws, ws_bytes, st));
    CR_TRY(launch_tiles_backward(shape, key_type, val_bytes, Ak, m, Bk, n, gC, gA, gB, ws,
                                 ws_bytes, st));
    return ok();
}

cr_status cr_merge_partition(int key_type, int val_bytes, const void* A, int64_t m, const void* B,
                             int64_t n, void* ws, size_t ws_bytes, cr_stream stream) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, true));
    if (bad_size(m) || bad_size(n)) return fail(CR_EINVAL, "negative or too large size");
    const int ks = key_bytes(key_type);
    CR_TRY(check_arr({A, m, ks, "A"}));
    CR_TRY(check_arr({B, n, ks, "B"}));
    if (m + n == 0) return ok();
    CR_TRY(launch_partition(shape_of(key_type, val_bytes, m, n), key_type, A, m, B, n, ws, ws_bytes,
                            static_cast<cudaStream_t>(stream)));
    return ok();
}

cr_status cr_merge_partition_alg2(int key_type, int val_bytes, const void* A, int64_t m,
                                  const void* B, int64_t n, void* ws, size_t ws_bytes,
                                  cr_stream stream) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, true));
    if (bad_size(m) || bad_size(n)) return fail(CR_EINVAL, "negative or too large size");
    const int ks = key_bytes(key_type);
    CR_TRY(check_arr({A, m, ks, "A"}));
    CR_TRY(check_arr({B, n, ks, "B"}));
    if (m + n == 0) return ok();
    int64_t tile = 0;
    const int64_t ntiles = single_tiles(shape_of(key_type, val_bytes, m, n), m, n, &tile);
    CR_TRY(check_ws(ws, ws_bytes, single_ws_bytes(ntiles)));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = by_key(key_type, [&](auto ops) {
        return ops.partition_single_free(A, m, B, n, tile, ntiles, ws, key_order(key_type), st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "partition launch");
    return ok();
}

cr_status cr_merge_tiles(int key_type, int val_bytes, const void* Ak, const void* Av, int64_t m,
                         const void* Bk, const void* Bv, int64_t n, void* Ck, void* Cv,
                         uint32_t* C_tag, void* ws, size_t ws_bytes, cr_stream stream) {
    CR_TRY(check_forward(key_type, val_bytes, Ak, Av, m, Bk, Bv, n, Ck, Cv, C_tag));
    if (m + n == 0) return ok();
    CR_TRY(launch_tiles(shape_of(key_type, val_bytes, m, n), key_type, val_bytes, Ak, Av, m, Bk, Bv, n,
                        Ck, Cv, C_tag, ws, ws_bytes, static_cast<cudaStream_t>(stream)));
    return ok();
}

cr_status cr_merge_tiles_backward(int key_type, int val_bytes, const void* Ak, int64_t m,
                                  const void* Bk, int64_t n, const void* gC, void* gA, void* gB,
                                  void* ws, size_t ws_bytes, cr_stream stream) {
    CR_TRY(check_backward(key_type, val_bytes, Ak, m, Bk, n, gC, gA, gB));
    if (m + n == 0) return ok();
    CR_TRY(launch_tiles_backward(shape_of(key_type, val_bytes, m, n), key_type, val_bytes, Ak, m, Bk,
                                 n, gC, gA, gB, ws, ws_bytes, static_cast<cudaStream_t>(stream)));
    return ok();
}

cr_status cr_batched_workspace_size(int key_type, int val_bytes, int64_t nseg, int64_t a_total,
                                    int64_t b_total, size_t* bytes) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, true));
    if (bad_size(nseg) || bad_size(a_total) || bad_size(b_total))
        return fail(CR_EINVAL, "negative or too large size");
    if (!bytes) return fail(CR_EINVAL, "bytes is NULL");
    const int64_t tile = cr::tile_of_shape(shape_batched(key_type, val_bytes));
    *bytes = batched_ws_bytes(batched_max_tiles(tile, nseg, a_total, b_total), nseg);
    return ok();
}

namespace {

cr_status batched_common(bool backward, int key_type, int val_bytes, int64_t nseg,
                         const int64_t* a_off, const int64_t* b_off, const void* Ak,
                         const void* Av, int64_t a_total, const void* Bk, const void* Bv,
                         int64_t b_total, const void* gC, void* Ck, void* Cv, void* gA, void* gB,
                         void* ws, size_t ws_bytes, cr_stream stream) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, !backward));
    if (bad_size(nseg) || bad_size(a_total) || bad_size(b_total))
        return fail(CR_EINVAL, "negative or too large size");
    const int ks = key_bytes(key_type);
    const int vb = val_bytes;
    const int64_t ct = a_total + b_total;
    if (nseg == 0) return ok();
    if (!a_off || !b_off) return fail(CR_EINVAL, "segment offset table is NULL");
    if ((reinterpret_cast<uintptr_t>(a_off) & 7u) || (reinterpret_cast<uintptr_t>(b_off) & 7u))
        return fail(CR_EALIGN, "segment offset tables must be 8-byte aligned");
    if (!backward) {
        const Arr ins[4] = {{Ak, a_total, ks, "A"}, {Bk, b_total, ks, "B"},
                            {vb ? Av : nullptr, vb ? a_total : 0, vb, "A payload"},
                            {vb ? Bv : nullptr, vb ? b_total : 0, vb, "B payload"}};
        const Arr outs[2] = {{Ck, ct, ks, "C"}, {vb ? Cv : nullptr, vb ? ct : 0, vb, "C payload"}};
        for (const Arr& a : ins) CR_TRY(check_arr(a));
        for (const Arr& a : outs) CR_TRY(check_arr(a));
        CR_TRY(check_no_alias(outs, 2, ins, 4));
    } else {
        const Arr ins[3] = {{Ak, a_total, ks, "A"}, {Bk, b_total, ks, "B"}, {gC, ct, vb, "gC"}};
        const Arr outs[2] = {{gA, a_total, vb, "gA"}, {gB, b_total, vb, "gB"}};
        for (const Arr& a : ins) CR_TRY(check_arr(a));
        for (const Arr& a : outs) CR_TRY(check_arr(a));
        CR_TRY(check_no_alias(outs, 2, ins, 3));
    }
    const int shape = shape_batched(key_type, vb);
    const int64_t tile = cr::tile_of_shape(shape);
    const int64_t max_tiles = batched_max_tiles(tile, nseg, a_total, b_total);
    CR_TRY(check_ws(ws, ws_bytes, batched_ws_bytes(max_tiles, nseg)));
    int64_t* prefix = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + cr::kHeaderBytes +
                                                 size_t(max_tiles) * kRecBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cr::MergeArgs a{};
    a.order = key_order(key_type);
    a.ak = Ak;
    a.bk = Bk;
    a.av = Av;
    a.bv = Bv;
    a.gc_in = gC;
    a.ck = Ck;
    a.cv = backward ? gA : Cv;
    a.cv2 = gB;
    a.a_total = a_total;
    a.b_total = b_total;
    a.c_total = ct;
    a.ws = ws;
    cudaError_t e = by_key(key_type, [&](auto ops) {
        cudaError_t r = ops.partition_batched(Ak, Bk, a_off, b_off, nseg, a_total, b_total, tile,
                                              max_tiles, ws, prefix, key_order(key_type), st);
        if (r != cudaSuccess) return r;
        return backward ? ops.merge_bwd(shape, vb, a, max_tiles, st)
                        : ops.merge_fwd(shape, vb, false, a, max_tiles, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "batched merge launch");
    return ok();
}

// Merge-pass modes: plain forward, backward that re-merges the keys,
// forward that records source flags, backward from those flags.
enum class Pass { kForward, kBackward, kRecord, kReplay };

cr_status pass_common(Pass mode, int key_type, int val_bytes, const void* X, const void* Xv,
                      int64_t N, int64_t width, const void* gY, void* Y, void* Yv, void* gX,
                      uint32_t* flags, size_t flag_words, void* ws, size_t ws_bytes,
                      cr_stream stream) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, mode == Pass::kForward));
    if (bad_size(N)) return fail(CR_EINVAL, "negative or too large size");
    if (width < 1) return fail(CR_EINVAL, "run width must be >= 1");
    if (flag_words > size_t(INT64_MAX / 4)) return fail(CR_EINVAL, "flag_words too large");
    const int ks = key_bytes(key_type);
    const int vb = val_bytes;
    const bool rec = mode == Pass::kRecord || mode == Pass::kReplay;
    const Arr fl = {rec ? flags : nullptr, rec ? int64_t(flag_words) : 0, 4, "flags", 16};
    if (mode == Pass::kForward || mode == Pass::kRecord) {
        const Arr ins[2] = {{X, N, ks, "X"}, {vb ? Xv : nullptr, vb ? N : 0, vb, "X payload"}};
        const Arr outs[3] = {{Y, N, ks, "Y"}, {vb ? Yv : nullptr, vb ? N : 0, vb, "Y payload"},
                             fl};
        for (const Arr& a : ins) CR_TRY(check_arr(a));
        for (const Arr& a : outs) CR_TRY(check_arr(a));
        CR_TRY(check_no_alias(outs, 3, ins, 2));
    } else if (mode == Pass::kBackward) {
        const Arr ins[2] = {{X, N, ks, "X"}, {gY, N, vb, "gY"}};
        const Arr outs[1] = {{gX, N, vb, "gX"}};
        for (const Arr& a : ins) CR_TRY(check_arr(a));
        CR_TRY(check_arr(outs[0]));
        CR_TRY(check_no_alias(outs, 1, ins, 2));
    } else {
        const Arr ins[2] = {{gY, N, vb, "gY"}, fl};
        const Arr outs[1] = {{gX, N, vb, "gX"}};
        for (const Arr& a : ins) CR_TRY(check_arr(a));
        CR_TRY(check_arr(outs[0]));
        CR_TRY(check_no_alias(outs, 1, ins, 2));
    }
    if (N == 0) return ok();
    if (width > N) width = N;   // one pair with an empty second run: the same result
    const int shape = shape_pass(key_type, vb);
    const int64_t tile = cr::tile_of_shape(shape);
    if (rec && tile > cr::kMaxRecordTile)
        return fail(CR_EUNSUPPORTED, "recorded passes need tiles of at most %lld elements",
                    static_cast<long long>(cr::kMaxRecordTile));
    const int64_t ntiles = cr::pass_tiles(N, width, tile, nullptr, nullptr);
    CR_TRY(check_ws(ws, ws_bytes, single_ws_bytes(ntiles)));
    if (rec) {
        const size_t need = size_t(ntiles) * size_t(tile / 32);
        if (flag_words < need)
            return fail(CR_ENOSPACE, "flags hold %zu words, need %zu", flag_words, need);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mode == Pass::kReplay) {
        const cudaError_t e =
            cr::route_recorded(vb, ws, flags, int64_t(flag_words), N, width, tile, gY, gX, st);
        if (e != cudaSuccess) return cuda_fail(e, "recorded pass backward launch");
        return ok();
    }
    cr::MergeArgs a{};
    a.order = key_order(key_type);
    a.ak = X;
    a.bk = X;
    a.av = Xv;
    a.bv = Xv;
    a.gc_in = gY;
    a.ck = Y;
    a.cv = mode == Pass::kBackward ? gX : Yv;
    a.cv2 = gX;
    a.flags = flags;
    a.a_total = N;
    a.b_total = N;
    a.c_total = N;
    a.ws = ws;
    cudaError_t e = by_key(key_type, [&](auto ops) {
        int64_t nt = 0;
        cudaError_t r = ops.partition_pass(X, N, width, tile, ws, &nt, key_order(key_type), st);
        if (r != cudaSuccess) return r;
        switch (mode) {
            case Pass::kBackward: return ops.merge_bwd(shape, vb, a, nt, st);
            case Pass::kRecord: return ops.merge_fwd_rec(shape, vb, a, nt, st);
            default: return ops.merge_fwd(shape, vb, false, a, nt, st);
        }
    });
    if (e != cudaSuccess) return cuda_fail(e, "merge pass launch");
    return ok();
}

}  // namespace

cr_status cr_batched_merge_kv(int key_type, int val_bytes, int64_t nseg, const int64_t* d_a_off,
                              const int64_t* d_b_off, const void* Ak, const void* Av,
                              int64_t a_total, const void* Bk, const void* Bv, int64_t b_total,
                              void* Ck, void* Cv, void* ws, size_t ws_bytes, cr_stream stream) {
    return batched_common(false, key_type, val_bytes, nseg, d_a_off, d_b_off, Ak, Av, a_total,
                          Bk, Bv, b_total, nullptr, Ck, Cv, nullptr, nullptr, ws, ws_bytes,
                          stream);
}

cr_status cr_batched_merge_kv_backward(int key_type, int val_bytes, int64_t nseg,
                                       const int64_t* d_a_off, const int64_t* d_b_off,
                                       const void* Ak, int64_t a_total, const void* Bk,
                                       int64_t b_total, const void* gC, void* gA, void* gB,
                                       void* ws, size_t ws_bytes, cr_stream stream) {
    return batched_common(true, key_type, val_bytes, nseg, d_a_off, d_b_off, Ak, nullptr,
                          a_total, Bk, nullptr, b_total, gC, nullptr, nullptr, gA, gB, ws,
                          ws_bytes, stream);
}

cr_status cr_merge_pass_workspace_size(int key_type, int val_bytes, int64_t N, int64_t width,
                                       size_t* bytes) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, true));
    if (bad_size(N) || width < 1) return fail(CR_EINVAL, "bad size or width");
    if (!bytes) return fail(CR_EINVAL, "bytes is NULL");
    const int64_t tile = cr::tile_of_shape(shape_pass(key_type, val_bytes));
    if (width > N) width = N > 0 ? N : 1;
    *bytes = single_ws_bytes(cr::pass_tiles(N, width, tile, nullptr, nullptr));
    return ok();
}

cr_status cr_merge_pass(int key_type, int val_bytes, const void* X, const void* Xv, int64_t N,
                        int64_t width, void* Y, void* Yv, void* ws, size_t ws_bytes,
                        cr_stream stream) {
    return pass_common(Pass::kForward, key_type, val_bytes, X, Xv, N, width, nullptr, Y, Yv,
                       nullptr, nullptr, 0, ws, ws_bytes, stream);
}

cr_status cr_merge_pass_backward(int key_type, int val_bytes, const void* X, int64_t N,
                                 int64_t width, const void* gY, void* gX, void* ws,
                                 size_t ws_bytes, cr_stream stream) {
    return pass_common(Pass::kBackward, key_type, val_bytes, X, nullptr, N, width, gY, nullptr,
                       nullptr, gX, nullptr, 0, ws, ws_bytes, stream);
}

cr_status cr_merge_pass_record_size(int key_type, int val_bytes, int64_t N, int64_t width,
                                    size_t* ws_bytes, size_t* flag_words) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, false));
    if (bad_size(N) || width < 1) return fail(CR_EINVAL, "bad size or width");
    if (!ws_bytes || !flag_words) return fail(CR_EINVAL, "output pointer is NULL");
    const int64_t tile = cr::tile_of_shape(shape_pass(key_type, val_bytes));
    if (width > N) width = N > 0 ? N : 1;
    const int64_t nt = cr::pass_tiles(N, width, tile, nullptr, nullptr);
    *ws_bytes = single_ws_bytes(nt);
    *flag_words = size_t(nt) * size_t(tile / 32);
    return ok();
}

cr_status cr_merge_pass_record(int key_type, int val_bytes, const void* X, const void* Xv,
                               int64_t N, int64_t width, void* Y, void* Yv, uint32_t* flags,
                               size_t flag_words, void* ws, size_t ws_bytes, cr_stream stream) {
    return pass_common(Pass::kRecord, key_type, val_bytes, X, Xv, N, width, nullptr, Y, Yv,
                       nullptr, flags, flag_words, ws, ws_bytes, stream);
}

cr_status cr_merge_pass_backward_recorded(int key_type, int val_bytes, int64_t N, int64_t width,
                                          const uint32_t* flags, size_t flag_words,
                                          const void* gY, void* gX, void* ws, size_t ws_bytes,
                                          cr_stream stream) {
    return pass_common(Pass::kReplay, key_type, val_bytes, nullptr, nullptr, N, width, gY,
                       nullptr, nullptr, gX, const_cast<uint32_t*>(flags), flag_words, ws,
                       ws_bytes, stream);
}

int64_t cr_sort_run_length(void) { return cr::kSortRun; }

namespace {

cr_status sort_runs_common(int key_type, int val_bytes, const void* X, const void* Xv, int64_t N,
                           void* Y, void* Yv, uint16_t* perm, cr_stream stream) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, perm == nullptr));
    if (bad_size(N)) return fail(CR_EINVAL, "negative or too large size");
    const int ks = key_bytes(key_type);
    const int vb = val_bytes;
    const Arr ins[2] = {{X, N, ks, "X"}, {vb ? Xv : nullptr, vb ? N : 0, vb, "X payload"}};
    const Arr outs[3] = {{Y, N, ks, "Y"}, {vb ? Yv : nullptr, vb ? N : 0, vb, "Y payload"},
                         {perm, perm ? N : 0, 2, "perm"}};
    for (const Arr& a : ins) CR_TRY(check_arr(a));
    for (const Arr& a : outs) CR_TRY(check_arr(a));
    CR_TRY(check_no_alias(outs, 3, ins, 2));
    if (N == 0) return ok();
    const cudaError_t e = cr::block_sort_runs(key_type, vb, perm ? 1 : 0, X, Xv, N, Y, Yv, perm,
                                              nullptr, nullptr, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "run sort launch");
    return ok();
}

}  // namespace

cr_status cr_sort_runs(int key_type, int val_bytes, const void* X, const void* Xv, int64_t N,
                       void* Y, void* Yv, cr_stream stream) {
    return sort_runs_common(key_type, val_bytes, X, Xv, N, Y, Yv, nullptr, stream);
}

cr_status cr_sort_runs_record(int key_type, int val_bytes, const void* X, const void* Xv,
                              int64_t N, void* Y, void* Yv, uint16_t* perm, cr_stream stream) {
    CR_TRY(check_vb(val_bytes, false));
    if (perm == nullptr && N > 0) return fail(CR_EINVAL, "perm is NULL");
    return sort_runs_common(key_type, val_bytes, X, Xv, N, Y, Yv, perm, stream);
}

cr_status cr_sort_runs_backward_recorded(int val_bytes, int64_t N, const uint16_t* perm,
                                         const void* gY, void* gX, cr_stream stream) {
    CR_TRY(check_vb(val_bytes, false));
    if (bad_size(N)) return fail(CR_EINVAL, "negative or too large size");
    const Arr ins[2] = {{perm, N, 2, "perm"}, {gY, N, val_bytes, "gY"}};
    const Arr outs[1] = {{gX, N, val_bytes, "gX"}};
    for (const Arr& a : ins) CR_TRY(check_arr(a));
    CR_TRY(check_arr(outs[0]));
    CR_TRY(check_no_alias(outs, 1, ins, 2));
    if (N == 0) return ok();
    const cudaError_t e = cr::sort_route_recorded(val_bytes, N, perm, gY, gX,
                                                  static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "recorded run sort backward launch");
    return ok();
}

cr_status cr_sort_runs_backward(int key_type, int val_bytes, const void* X, int64_t N,
                                const void* gY, void* gX, cr_stream stream) {
    CR_TRY(check_key_type(key_type));
    CR_TRY(check_vb(val_bytes, false));
    if (bad_size(N)) return fail(CR_EINVAL, "negative or too large size");
    const int ks = key_bytes(key_type);
    const Arr ins[2] = {{X, N, ks, "X"}, {gY, N, val_bytes, "gY"}};
    const Arr outs[1] = {{gX, N, val_bytes, "gX"}};
    for (const Arr& a : ins) CR_TRY(check_arr(a));
    CR_TRY(check_arr(outs[0]));
    CR_TRY(check_no_alias(outs, 1, ins, 2));
    if (N == 0) return ok();
    const cudaError_t e = cr::block_sort_runs(key_type, val_bytes, 2, X, nullptr, N, nullptr,
                                              nullptr, nullptr, gY, gX,
                                              static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "run sort backward launch");
    return ok();
}

cr_status cr_workspace_status(const void* ws, cr_stream stream) {
    if (ws == nullptr) return fail(CR_EINVAL, "workspace is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int32_t code = 0;
    e = cudaMemcpy(&code, ws, sizeof(code), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    switch (code) {
        case cr::kDevOk: return ok();
        case cr::kDevTimeout: return fail(CR_ETIMEOUT, "a device-side wait gave up");
        case cr::kDevInternal: return fail(CR_EINTERNAL, "inconsistent tile record");
        case cr::kDevBadSeg: return fail(CR_EBADSEG, "invalid segment offset table");
        default: return fail(CR_EINTERNAL, "unknown device status %d", code);
    }
}

}  // extern "C"
