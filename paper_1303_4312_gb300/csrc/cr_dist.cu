// cr_dist.cu -- Algorithm 1 (Section 2) for inputs that no single processor
// holds: the co-ranks of a batch of output ranks when A and B are
// block-distributed over the processing elements of Algorithm 2 (Section 3,
// its distributed-memory remark).  Every search needs four keys per
// iteration, A[i-1], A[i], B[j-1] and B[j]; these kernels split one
// iteration into the parts a process group runs between its collectives:
//
//   probes  -- the positions every live search reads next (-1: none),
//   answer  -- the keys of those positions that fall in this rank's blocks
//              (0 elsewhere, so a sum over the ranks delivers each key),
//   step    -- one iteration of Algorithm 1 on the delivered keys.
//
// The state of cnt searches is an int64 array of 6 * cnt entries, one
// column per field: [k | i | j | i_low | j_low | done] (ABI naming: rank k,
// co-ranks i into A and j into B; paper (i; j, k)).  Keys travel as int64
// carriers holding the key's bits (zero-extended for 4-byte keys).
#include <cuda_runtime.h>

#include "../../include/corank.h"
#include "cr_launch.cuh"

namespace cr {
void set_last_error(const char* msg);   // cr_abi.cu
}

namespace {

constexpr int kThreads = 256;

struct State {
    int64_t* k;
    int64_t* i;
    int64_t* j;
    int64_t* ilo;
    int64_t* jlo;
    int64_t* done;
    __device__ __forceinline__ explicit State(int64_t* st, int64_t cnt)
        : k(st), i(st + cnt), j(st + 2 * cnt), ilo(st + 3 * cnt), jlo(st + 4 * cnt),
          done(st + 5 * cnt) {}
};

// Algorithm 1's starting point: i = min(k, m), j = k - i.  Both low bounds
// start at their smallest possible value (the printed algorithm leaves the
// second unset and argues it is set before it is read).  A rank outside
// [0, m + n] gives a finished search with i = j = -1.
__global__ void __launch_bounds__(kThreads) dist_init_kernel(int64_t m, int64_t n,
                                                             const int64_t* __restrict__ ranks,
                                                             int64_t cnt, int64_t* st) {
    const int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (q >= cnt) return;
    State s(st, cnt);
    const int64_t k = ranks[q];
    s.k[q] = k;
    if (k < 0 || k > m + n) {
        s.i[q] = s.j[q] = -1;
        s.ilo[q] = s.jlo[q] = 0;
        s.done[q] = 1;
        return;
    }
    const int64_t i = k < m ? k : m;
    s.i[q] = i;
    s.j[q] = k - i;
    s.ilo[q] = k - n > 0 ? k - n : 0;
    s.jlo[q] = k - m > 0 ? k - m : 0;
    s.done[q] = 0;
}

// Positions read by the next iteration: pa[2q] = i-1, pa[2q+1] = i (into A),
// pb[2q] = j-1, pb[2q+1] = j (into B); -1 where the iteration's conditions
// do not need that key (out of range, or the search has finished).
__global__ void __launch_bounds__(kThreads) dist_probes_kernel(int64_t m, int64_t n,
                                                               const int64_t* st, int64_t cnt,
                                                               int64_t* __restrict__ pa,
                                                               int64_t* __restrict__ pb) {
    const int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (q >= cnt) return;
    State s(const_cast<int64_t*>(st), cnt);
    const bool live = s.done[q] == 0;
    const int64_t i = s.i[q], j = s.j[q];
    // first condition: A[i-1] against B[j]; second: B[j-1] against A[i]
    const bool c1 = live && i > 0 && j < n;
    const bool c2 = live && j > 0 && i < m;
    pa[2 * q] = c1 ? i - 1 : -1;
    pa[2 * q + 1] = c2 ? i : -1;
    pb[2 * q] = c2 ? j - 1 : -1;
    pb[2 * q + 1] = c1 ? j : -1;
}

// out[q] = bits of blk[idx[q] - lo] when lo <= idx[q] < hi, else 0.
template <class K>
__global__ void __launch_bounds__(kThreads) dist_answer_kernel(const K* __restrict__ blk,
                                                               int64_t lo, int64_t hi,
                                                               const int64_t* __restrict__ idx,
                                                               int64_t cnt,
                                                               int64_t* __restrict__ out) {
    const int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (q >= cnt) return;
    const int64_t x = idx[q];
    using U = typename std::make_unsigned<K>::type;
    out[q] = (x >= lo && x < hi) ? int64_t(uint64_t(U(blk[x - lo]))) : 0;
}

template <class K>
__device__ __forceinline__ K carried(int64_t v, int order) {
    using U = typename std::make_unsigned<K>::type;
    return cr::order_key(K(U(uint64_t(v))), order);
}

// One iteration of Algorithm 1 for every live search, with the keys the
// probes asked for: va[2q] = A[i-1], va[2q+1] = A[i], vb[2q] = B[j-1],
// vb[2q+1] = B[j] (entries for unrequested positions are ignored).
template <class K>
__global__ void __launch_bounds__(kThreads) dist_step_kernel(int64_t m, int64_t n,
                                                             const int64_t* __restrict__ va,
                                                             const int64_t* __restrict__ vb,
                                                             int64_t* st, int64_t cnt,
                                                             int order) {
    const int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (q >= cnt) return;
    State s(st, cnt);
    if (s.done[q]) return;
    const int64_t i = s.i[q], j = s.j[q];
    if (i > 0 && j < n && carried<K>(vb[2 * q + 1], order) < carried<K>(va[2 * q], order)) {
        // A[i-1] > B[j]: the split lies further left in A
        const int64_t d = (i - s.ilo[q] + 1) / 2;
        s.jlo[q] = j;
        s.i[q] = i - d;
        s.j[q] = j + d;
    } else if (j > 0 && i < m &&
               !(carried<K>(vb[2 * q], order) < carried<K>(va[2 * q + 1], order))) {
        // B[j-1] >= A[i]: the split lies further right in A
        const int64_t d = (j - s.jlo[q] + 1) / 2;
        s.ilo[q] = i;
        s.i[q] = i + d;
        s.j[q] = j - d;
    } else {
        s.done[q] = 1;   // both conditions of Lemma 1 hold
    }
}

// d_i[q], d_j[q] from the state; *d_live = number of unfinished searches.
__global__ void __launch_bounds__(kThreads) dist_result_kernel(const int64_t* st, int64_t cnt,
                                                               int64_t* __restrict__ oi,
                                                               int64_t* __restrict__ oj,
                                                               unsigned long long* live) {
    const int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    bool open = false;
    if (q < cnt) {
        State s(const_cast<int64_t*>(st), cnt);
        oi[q] = s.i[q];
        oj[q] = s.j[q];
        open = s.done[q] == 0;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, open);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(live, (unsigned long long)__popc(ballot));
}

__global__ void dist_zero_kernel(unsigned long long* p) { *p = 0; }

cr_status dist_fail(cr_status st, const char* msg) {
    cr::set_last_error(msg);
    return st;
}

bool bad_count(int64_t x) { return x < 0 || x > (int64_t(1) << 36); }
bool bad_size(int64_t x) { return x < 0 || x > (int64_t(1) << 59); }
bool al8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

unsigned grid_of(int64_t cnt) { return unsigned((cnt + kThreads - 1) / kThreads); }

cr_status launched() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dist_fail(CR_ECUDA, cudaGetErrorString(e));
    return dist_fail(CR_OK, "");
}

template <class F>
cudaError_t by_storage(int key_type, F&& f) {
    switch (cr::key_base(key_type)) {
        case CR_KEY_I32:
        case CR_KEY_F32: return f(int32_t(0));
        case CR_KEY_U32: return f(uint32_t(0));
        case CR_KEY_I64:
        case CR_KEY_F64: return f(int64_t(0));
        default: return f(uint64_t(0));
    }
}

}  // namespace

extern "C" {

cr_status cr_dist_co_rank_init(int64_t m, int64_t n, const int64_t* d_ranks, int64_t cnt,
                               int64_t* d_state, cr_stream stream) {
    if (bad_size(m) || bad_size(n) || bad_count(cnt))
        return dist_fail(CR_EINVAL, "negative or too large size");
    if (cnt == 0) return dist_fail(CR_OK, "");
    if (!d_ranks || !d_state) return dist_fail(CR_EINVAL, "NULL array");
    if (!al8(d_ranks) || !al8(d_state)) return dist_fail(CR_EALIGN, "arrays must be 8-byte aligned");
    dist_init_kernel<<<grid_of(cnt), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        m, n, d_ranks, cnt, d_state);
    return launched();
}

cr_status cr_dist_co_rank_probes(int64_t m, int64_t n, const int64_t* d_state, int64_t cnt,
                                 int64_t* d_probe_a, int64_t* d_probe_b, cr_stream stream) {
    if (bad_size(m) || bad_size(n) || bad_count(cnt))
        return dist_fail(CR_EINVAL, "negative or too large size");
    if (cnt == 0) return dist_fail(CR_OK, "");
    if (!d_state || !d_probe_a || !d_probe_b) return dist_fail(CR_EINVAL, "NULL array");
    if (!al8(d_state) || !al8(d_probe_a) || !al8(d_probe_b))
        return dist_fail(CR_EALIGN, "arrays must be 8-byte aligned");
    dist_probes_kernel<<<grid_of(cnt), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        m, n, d_state, cnt, d_probe_a, d_probe_b);
    return launched();
}

cr_status cr_dist_co_rank_answer(int key_type, const void* blk, int64_t lo, int64_t hi,
                                 const int64_t* d_idx, int64_t cnt, int64_t* d_vals,
                                 cr_stream stream) {
    const int ks = cr::key_type_bytes(key_type);
    if (ks == 0) return dist_fail(CR_EINVAL, "unknown key type");
    if (bad_size(lo) || bad_size(hi) || hi < lo || bad_count(cnt))
        return dist_fail(CR_EINVAL, "bad block bounds or count");
    if (cnt == 0) return dist_fail(CR_OK, "");
    if (!d_idx || !d_vals || (hi > lo && !blk)) return dist_fail(CR_EINVAL, "NULL array");
    if (!al8(d_idx) || !al8(d_vals) || (reinterpret_cast<uintptr_t>(blk) % uintptr_t(ks)))
        return dist_fail(CR_EALIGN, "misaligned array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    by_storage(key_type, [&](auto k) {
        using K = decltype(k);
        dist_answer_kernel<K><<<grid_of(cnt), kThreads, 0, st>>>(static_cast<const K*>(blk), lo,
                                                                 hi, d_idx, cnt, d_vals);
        return cudaSuccess;
    });
    return launched();
}

cr_status cr_dist_co_rank_step(int key_type, int64_t m, int64_t n, const int64_t* d_vals_a,
                               const int64_t* d_vals_b, int64_t* d_state, int64_t cnt,
                               cr_stream stream) {
    if (cr::key_type_bytes(key_type) == 0) return dist_fail(CR_EINVAL, "unknown key type");
    if (bad_size(m) || bad_size(n) || bad_count(cnt))
        return dist_fail(CR_EINVAL, "negative or too large size");
    if (cnt == 0) return dist_fail(CR_OK, "");
    if (!d_vals_a || !d_vals_b || !d_state) return dist_fail(CR_EINVAL, "NULL array");
    if (!al8(d_vals_a) || !al8(d_vals_b) || !al8(d_state))
        return dist_fail(CR_EALIGN, "arrays must be 8-byte aligned");
    const int order = cr::key_type_order(key_type);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    by_storage(key_type, [&](auto k) {
        using K = decltype(k);
        dist_step_kernel<K><<<grid_of(cnt), kThreads, 0, st>>>(m, n, d_vals_a, d_vals_b, d_state,
                                                               cnt, order);
        return cudaSuccess;
    });
    return launched();
}

cr_status cr_dist_co_rank_result(const int64_t* d_state, int64_t cnt, int64_t* d_i, int64_t* d_j,
                                 uint64_t* d_live, cr_stream stream) {
    if (bad_count(cnt)) return dist_fail(CR_EINVAL, "bad count");
    if (!d_live) return dist_fail(CR_EINVAL, "NULL live counter");
    if (!al8(d_live)) return dist_fail(CR_EALIGN, "live counter must be 8-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto* live = reinterpret_cast<unsigned long long*>(d_live);
    dist_zero_kernel<<<1, 1, 0, st>>>(live);
    if (cnt > 0) {
        if (!d_state || !d_i || !d_j) return dist_fail(CR_EINVAL, "NULL array");
        if (!al8(d_state) || !al8(d_i) || !al8(d_j))
            return dist_fail(CR_EALIGN, "arrays must be 8-byte aligned");
        dist_result_kernel<<<grid_of(cnt), kThreads, 0, st>>>(d_state, cnt, d_i, d_j, live);
    }
    return launched();
}

}  // extern "C"
