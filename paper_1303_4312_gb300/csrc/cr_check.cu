// cr_check.cu -- debug check of the merge's precondition: an input array is
// sorted in its key type's order (the hot path does not check it).  One
// grid-stride pass compares every neighbouring pair in that order
// (order_key) and keeps the smallest position p with key[p] < key[p-1].
#include <cuda_runtime.h>

#include "../../include/corank.h"
#include "cr_launch.cuh"

namespace {

constexpr unsigned long long kNone = ~0ull;

__global__ void check_init_kernel(unsigned long long* first) { *first = kNone; }

template <class K>
__global__ void __launch_bounds__(256) check_sorted_kernel(const K* __restrict__ A, int64_t m,
                                                           int order,
                                                           unsigned long long* first) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x + 1; p < m; p += stride) {
        if (cr::order_key(A[p], order) < cr::order_key(A[p - 1], order))
            atomicMin(first, static_cast<unsigned long long>(p));
    }
}

__global__ void check_final_kernel(const unsigned long long* first, int64_t* out) {
    *out = *first == kNone ? -1 : static_cast<int64_t>(*first);
}

template <class K>
cudaError_t run_check(const void* A, int64_t m, int order, unsigned long long* scratch,
                      int64_t* out, cudaStream_t st) {
    check_init_kernel<<<1, 1, 0, st>>>(scratch);
    if (m > 1) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t want = (m + 255) / 256;
        const int64_t cap = int64_t(sms > 0 ? sms : 1) * 8;
        check_sorted_kernel<K><<<unsigned(want < cap ? want : cap), 256, 0, st>>>(
            static_cast<const K*>(A), m, order, scratch);
    }
    check_final_kernel<<<1, 1, 0, st>>>(scratch, out);
    return cudaGetLastError();
}

}  // namespace

namespace cr {
void set_last_error(const char* msg);   // cr_abi.cu
}

namespace {
cr_status check_fail(cr_status st, const char* msg) {
    cr::set_last_error(msg);
    return st;
}
}  // namespace

extern "C" cr_status cr_check_sorted(int key_type, const void* A, int64_t m, int64_t* d_first,
                                     void* ws, size_t ws_bytes, cr_stream stream) {
    if (cr::key_type_bytes(key_type) == 0) return check_fail(CR_EINVAL, "unknown key type");
    if (m < 0) return check_fail(CR_EINVAL, "negative size");
    if ((m > 0 && A == nullptr) || d_first == nullptr || ws == nullptr)
        return check_fail(CR_EINVAL, "NULL array");
    if (ws_bytes < 16) return check_fail(CR_EINVAL, "scratch smaller than 16 bytes");
    if ((reinterpret_cast<uintptr_t>(A) % uintptr_t(cr::key_type_bytes(key_type))) ||
        (reinterpret_cast<uintptr_t>(ws) & 15u) || (reinterpret_cast<uintptr_t>(d_first) & 7u))
        return check_fail(CR_EALIGN,
                          "A not aligned to its key size, the scratch not 16-byte aligned, or "
                          "d_first not 8-byte aligned");
    const int order = cr::key_type_order(key_type);
    auto* scratch = static_cast<unsigned long long*>(ws);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaErrorInvalidValue;
    switch (cr::key_base(key_type)) {
        case CR_KEY_I32:
        case CR_KEY_F32: e = run_check<int32_t>(A, m, order, scratch, d_first, st); break;
        case CR_KEY_U32: e = run_check<uint32_t>(A, m, order, scratch, d_first, st); break;
        case CR_KEY_I64:
        case CR_KEY_F64: e = run_check<int64_t>(A, m, order, scratch, d_first, st); break;
        default: e = run_check<uint64_t>(A, m, order, scratch, d_first, st); break;
    }
    if (e != cudaSuccess) return check_fail(CR_ECUDA, cudaGetErrorString(e));
    return check_fail(CR_OK, "");
}
