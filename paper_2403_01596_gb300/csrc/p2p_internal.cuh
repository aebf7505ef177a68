// Internal declarations of the GB300 P2P library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "p2p.h"

#define P2P_FULL_MASK 0xffffffffu

// Device status word bits (set with atomicOr by kernels, read by p2p_last_async_status).
enum : unsigned int {
    P2P_DEV_BAD_INPUT = 1u,    // non-finite coordinate or out-of-range structure index
    P2P_DEV_TIMEOUT = 2u,      // a bounded wait ran out
    P2P_DEV_TC_FAULTED = 4u    // tensor-core path bailed out (its results are not valid)
};

struct p2p_plan {
    // sizes and parameters
    int64_t n;
    int32_t nb;
    int64_t nnz;
    int64_t sources;        // sum over boxes of S_b
    int64_t packed;         // padded packed size (redundant layout), 0 otherwise
    p2p_kernel kernel;
    float k;
    p2p_layout layout;
    int32_t max_nrhs;
    p2p_tuning tune;
    // caller arrays (not owned)
    const float* pts;
    const int32_t* perm;
    const int32_t* box_ptr;
    const int32_t* nbr_ptr;
    const int32_t* nbr_idx;
    // carved from the caller's workspace
    float4* xs;             // [n] box-sorted coordinates (w = 0)
    int32_t* box_src;       // [nb] S_b, sources in the neighbourhood of box b
    int32_t* box_self;      // [nb] position of box b's own sources inside its concatenated neighbourhood
    int4* items;            // [n_items] (box, source begin, target begin, 0)
    int64_t n_items;
    int32_t max_chunks;     // max over boxes of ceil(S_b / chunk)
    int32_t max_box;        // largest box occupancy
    int32_t* pk_off;        // [nb + 1] packed offsets (redundant layout)
    float4* pk_xyz;         // [packed] per-box neighbourhood coordinates
    int32_t* pk_src;        // [packed] original index of each packed source, -1 for padding
    float2* lam_buf;        // [max(n, packed) * max_nrhs] sorted / packed strengths
    float2* g_buf;          // [n * max_nrhs] sorted upstream gradient (coordinate gradient)
    unsigned int* status;   // device status word
    long long* scratch64;   // small device scratch (pair count)
};

namespace p2p_detail {

// thread-local message of the last CUDA failure
void set_cuda_error(cudaError_t e, const char* where);
void set_message(const char* msg);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves 256-byte aligned sub-buffers out of one workspace.
struct Carver {
    char* base;
    size_t off;
    size_t cap;
    template <typename T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    bool ok() const { return off <= cap; }
};

// Device-wide exclusive scan of int32 (total written to *total_dev if non-null).
size_t scan_workspace_bytes(int64_t n);
cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev, void* work,
                               cudaStream_t s);

// Stable LSD radix sort of (uint64 key, int32 value) pairs on the low `bits` bits.
size_t radix_workspace_bytes(int64_t n);
cudaError_t radix_sort_pairs(uint64_t* keys, int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, int64_t n,
                             int bits, void* work, cudaStream_t s, bool* result_in_alt);

}  // namespace p2p_detail

#define P2P_TRY_CUDA(expr, where)                        \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) {                         \
            p2p_detail::set_cuda_error(e_, where);       \
            return P2P_ERR_CUDA;                         \
        }                                                \
    } while (0)

#define P2P_CHECK_LAUNCH(where) P2P_TRY_CUDA(cudaGetLastError(), where)

// ----------------------------------------------------------- device helpers --

// Spreads the low 21 bits of v so that bit i lands at bit 3i.
__device__ __forceinline__ uint64_t p2p_spread3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Inverse of p2p_spread3: gathers bits 0, 3, 6, ... into the low 21 bits.
__device__ __forceinline__ uint32_t p2p_compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

__device__ __forceinline__ uint64_t p2p_morton(uint32_t cx, uint32_t cy, uint32_t cz) {
    return p2p_spread3(cx) | (p2p_spread3(cy) << 1) | (p2p_spread3(cz) << 2);
}
