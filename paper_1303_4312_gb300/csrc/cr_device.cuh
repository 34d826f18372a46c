// cr_device.cuh -- device-side building blocks of the co-rank / stable-merge
// kernels for sm_103a: the tile record, the workspace header, Algorithm 1,
// and inline-PTX wrappers for mbarriers and bulk (TMA engine) copies.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace cr {

// ---------------------------------------------------------------------------
// Workspace layout (caller-owned device memory, 16-byte aligned):
//   [0, 256)                 header: status word, tile count
//   [256, 256 + 32*ntiles)   one TileRec per output tile
//   [..., + 8*(nseg+1))      batched calls only: tile prefix per segment
// ---------------------------------------------------------------------------
constexpr int kHeaderBytes = 256;

struct WsHeader {
    int32_t status;      // device status (kDev*), 0 = ok
    int32_t tile;        // TILE the table was made for (checked by the merge kernel)
    int64_t ntiles;      // tiles of the current call (written by the partition kernel)
};

// Device status codes: equal to the public cr_status values they map to.
constexpr int32_t kDevOk = 0;
constexpr int32_t kDevTimeout = 6;
constexpr int32_t kDevInternal = 8;
constexpr int32_t kDevBadSeg = 9;

// One output tile: it merges A[ga, ga+alen) with B[gb, gb+blen) into
// C[gc, gc+alen+blen).  alen + blen <= TILE; ga/gb/gc are element indices
// into the full arrays (segment offsets already applied).
struct __align__(16) TileRec {
    int64_t ga, gb, gc;
    int32_t alen, blen;
};
static_assert(sizeof(TileRec) == 32, "TileRec is two 16-byte words");

// Kernel arguments shared by the forward and backward tile-merge kernels.
struct MergeArgs {
    const void* ak;      // A keys
    const void* bk;      // B keys
    const void* av;      // fwd: A payloads
    const void* bv;      // fwd: B payloads
    const void* gc_in;   // bwd: gradient of C
    void* ck;            // fwd: C keys
    void* cv;            // fwd: C payloads / bwd: gradient of A
    void* cv2;           // bwd: gradient of B
    uint32_t* ctag;      // fwd: source tags (nullable)
    uint32_t* flags;     // fwd, recording kernels: per-tile source flags
    int64_t a_total;     // length of the A array
    int64_t b_total;     // length of the B array
    int64_t c_total;     // length of the C array
    int64_t tag_b;       // tag of B[0]
    void* ws;            // workspace: header + tile records
    int32_t order;       // key order (order_key): 0 = the key type's own
    // Array starts need only be aligned to their element size.  The pointers
    // above are the 16-byte boundaries at or below each array's start (bulk
    // copies address whole 16-byte chunks), and sh_* is the array's start
    // measured from there in elements: element x of A is ak[x + sh_ak].
    // flags and ws are library-format buffers and stay 16-byte aligned.
    int32_t sh_ak, sh_bk, sh_av, sh_bv, sh_gc, sh_ck, sh_cv, sh_cv2, sh_tag;
};

// ---------------------------------------------------------------------------
// Key orders.  The merge compares keys with `<` of their storage type; other
// orders are reached through an order-preserving bijection applied to every
// key before it is compared (and undone on the keys written out):
//   bit 1: IEEE-754 totalOrder of a float stored in the signed integer of
//          its width (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN):
//          negative values have their magnitude bits flipped, after which
//          the signed integer order is the float total order;
//   bit 2: a pair of signed 32-bit keys stored in one 64-bit word (major key
//          in the high half), ordered lexicographically: both halves' sign
//          bits flipped, after which the unsigned 64-bit order is that order;
//   bit 0: descending: the bitwise complement reverses any integer order.
// All steps are involutions; order 0 is the identity.
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ K order_flip_float(K x) {
    using S = typename std::make_signed<K>::type;
    const S s = S(x);
    constexpr S mag = S(~(typename std::make_unsigned<K>::type(1)
                          << (8 * sizeof(K) - 1)));     // all bits but the sign
    return K(s ^ ((s >> (8 * int(sizeof(K)) - 1)) & mag));
}

template <class K>
__host__ __device__ constexpr K pair_sign_bits() {
    return sizeof(K) == 8 ? K(0x8000000080000000ull) : K(0);
}

template <class K>
__device__ __forceinline__ K order_key(K x, int order) {
    if (order & 2) x = order_flip_float(x);
    if (order & 4) x = K(x ^ pair_sign_bits<K>());
    if (order & 1) x = K(~x);
    return x;
}

template <class K>
__device__ __forceinline__ K order_key_inverse(K x, int order) {
    if (order & 1) x = K(~x);
    if (order & 4) x = K(x ^ pair_sign_bits<K>());
    if (order & 2) x = order_flip_float(x);
    return x;
}

// order_key / order_key_inverse without branches, for hot loops: with
// F = the magnitude bits when bit 1 of the order is set (else 0) and M = all
// ones when bit 0 is set (else 0), xor the pair sign bits when bit 2 is set,
// map(x) = x ^ ((sign(x) & F) ^ M), where sign(x) is x's sign bit replicated
// (bits 1 and 2 are never set together); the inverse undoes M first.
template <class K>
struct OrderMap {
    using S = typename std::make_signed<K>::type;
    using U = typename std::make_unsigned<K>::type;
    static constexpr int SH = 8 * int(sizeof(K)) - 1;
    K flt, neg;
    __device__ __forceinline__ explicit OrderMap(int order)
        : flt((order & 2) ? K(U(~U(0)) >> 1) : K(0)),
          neg(K(((order & 1) ? K(~U(0)) : K(0)) ^ ((order & 4) ? pair_sign_bits<K>() : K(0)))) {}
    __device__ __forceinline__ K operator()(K x) const {
        return K(x ^ ((K(S(x) >> SH) & flt) ^ neg));
    }
    __device__ __forceinline__ K inverse(K u) const {
        const K v = K(u ^ neg);
        return K(v ^ (K(S(v) >> SH) & flt));
    }
};

// Read-only view of a key array in a given order: v[i] is key i mapped by
// order_key, so searches written with `<` on v[i] follow that order.
template <class K>
struct KeyView {
    using key_type = K;
    const K* p;
    int order;
    __device__ __forceinline__ K operator[](int64_t i) const { return order_key(p[i], order); }
    __device__ __forceinline__ KeyView operator+(int64_t off) const { return {p + off, order}; }
};

__host__ __device__ inline TileRec* ws_recs(void* ws) {
    return reinterpret_cast<TileRec*>(static_cast<char*>(ws) + kHeaderBytes);
}

// ---------------------------------------------------------------------------
// PTX wrappers (sm_90+ forms, valid on sm_103a).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make mbarrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking probe: has the phase with the given parity completed?
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void sleep_ns(uint32_t ns) {
    asm volatile("nanosleep.u32 %0;" ::"r"(ns));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity to complete.  Gives up
// after about `limit_ns` nanoseconds of wall time and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
#pragma unroll 1
    for (uint32_t spin = 1; spin < (1u << 26); ++spin) {   // hard cap as a backstop
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 255u) == 0 && global_timer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Bulk copy global -> this CTA's shared memory, completion counted in bytes
// on `bar`.  dst, src 16-byte aligned; bytes a nonzero multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bulk copy shared -> global (bulk-group completion).  Same alignment rules.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_addr(src)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until at most N committed bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until at most N committed bulk groups are incomplete.
template <int N>
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Order this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) reads of the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier over `count` threads (a multiple of 32).
__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    atomicCAS(status, 0, code);
}

}  // namespace cr
