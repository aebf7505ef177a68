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

// One work item of the FP32 pair kernels: target box b against one chunk of
// its concatenated neighbourhood (own box first).  Built and sorted by
// decreasing cost (targets x sources) at plan time.
struct ItemRec {
    int32_t src_off;   // first entry of the chunk in the per-box source lists (pk_off[b] + chunk start)
    int32_t ns;        // sources in the chunk
    int32_t tb;        // first target (box-sorted index)
    int32_t nt;        // targets of the box
    int32_t m_end;     // low 16 bits: the chunk's first m_end sources belong to the box itself (r = 0
                       // possible); bit 16: the chunk starts at the list's first entry, so the box's
                       // targets t < m_end are the staged sources 0 .. m_end - 1
    int32_t map_full;  // lane map of a full target group (see p2p_lane_map)
    int32_t map_last;  // lane map of the last (possibly partial) target group
    int32_t b;         // box id
};

// Lane map of a target group of nt targets against ns sources on `lanes` lanes
// (32, or the 16 / 8 lanes of a box in the direct kernel): TT targets per lane
// (1, 2 or 4), G = ceil(nt / TT) target slots, Q = lanes / G source slices, and
// mG = ceil(65536 / G) so that x / G == (x * mG) >> 16 for x < 128.  TT
// minimises the lane's instruction count: ceil(ns / Q) iterations of TT pair
// evaluations (~20 instructions each) plus the per-iteration source loads and
// loop control (`per_iter`).  Packed as TT | G << 3 | Q << 9 | (mG - 1) << 15.
__host__ __device__ inline int32_t p2p_lane_map(int nt, int ns, int lanes = 32, int per_iter = 4) {
    int best = 4, best_cost = 0x7fffffff;
    for (int tt = 1; tt <= 4; tt <<= 1) {
        const int g = (nt + tt - 1) / tt;
        if (g > lanes || g < 1) continue;
        const int q = lanes / g;
        const int cost = (20 * tt + per_iter) * ((ns + q - 1) / q);
        if (cost < best_cost) {
            best_cost = cost;
            best = tt;
        }
    }
    int g = (nt + best - 1) / best;
    if (g < 1) g = 1;
    const int q = lanes / g;
    const int mg = (65536 + g - 1) / g;
    return best | (g << 3) | (q << 9) | ((mg - 1) << 15);
}

struct p2p_plan {
    // sizes and parameters.  n, nb, pts, perm, box_ptr and xs describe the TARGET points and their boxes (work
    // items, outputs); the src_* fields describe the SOURCE points.  A one-set plan (sources = targets) has
    // src_* equal to the target fields; a two-set plan (p2p_plan_create_st) has its own.
    int64_t n;
    int32_t nb;
    int32_t two_sets;       // 1: separate target and source point sets
    int64_t n_src;          // source points
    int32_t nbs;            // source boxes
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
    const float* src_pts;
    const int32_t* src_perm;
    const int32_t* src_box_ptr;
    const int32_t* nbr_self;  // two-set plans: position in each target box's list of the source box of the same
                              // cell, -1 if none (NULL for one-set plans: the box itself)
    // carved from the caller's workspace
    float4* xs;             // [n] box-sorted target coordinates (w = 0)
    float4* xs_src;         // [n_src] box-sorted source coordinates (= xs for one-set plans)
    int32_t* box_src;       // [nb] S_b, sources in the neighbourhood of box b
    ItemRec* items;         // [n_items] work items, heaviest first
    int64_t n_items;
    int32_t max_chunks;     // max over boxes of ceil(S_b / chunk)
    int32_t max_box;        // largest box occupancy
    int32_t* pk_off;        // [nb + 1] offsets of the per-box source lists (each padded to 4 entries)
    int32_t* nb_src;        // [packed] box-sorted index of every listed source, -1 for padding
    float4* pk_xyz;         // [packed] redundant layout: per-box copy of the listed coordinates
    int32_t* pk_src;        // [packed] redundant layout: original index of every listed source, -1 for padding
    // repetition layout (Sec. 3.3): one record per target -- its coordinates, then its neighbourhood's sources
    int64_t records;        // entries of all records (sum over boxes of n_b (1 + S_b)), 0 for other layouts
    int32_t* rec_off;       // [n + 1] first entry of the record of every target (box-sorted order)
    float4* rec_xyz;        // [records] coordinates: the target, then its sources
    int32_t* rec_src;       // [records] original index of every source entry, -1 for the target entry
    int32_t* rec_boff;      // [nb + 1] first record entry of every box
    int32_t direct_k;       // boxes per warp of the direct kernel (1, 2 or 4); 0: the staged pipeline
    ItemRec* ditems;        // [nb] direct kernel: one item per target box (whole source list, lane maps for
                            // 32 / direct_k lanes), heaviest first
    int32_t direct_grid;    // persistent grid of the direct kernel (blocks of kDirectWarps warps)
    int32_t grid[3];        // persistent grid of the pair kernel for R = 1, 2, 4 right-hand sides per pass
    int32_t grid_warps[3];  // warps per block of that grid (the tuning's, halved until a block fits)
    float2* lam_buf;        // [max(n, packed) * max_nrhs] sorted / packed strengths
    float2* g_buf;          // [n * max_nrhs] sorted upstream gradient (coordinate gradient)
    unsigned int* status;   // device status word
    long long* scratch64;   // small device scratch (pair count)
    // tensor-core path (plans with max_nrhs >= 16)
    int32_t* tc_gstart;     // [nb + 1] first 16-source group of every box (exclusive scan of ceil(n_b / 16))
    int32_t tc_groups;      // number of 16-source groups
    int32_t* tc_glist_off;  // [nb + 1] offsets of the per-box group lists
    int32_t* tc_glist;      // per box: the groups of its neighbour boxes (ascending box id), -1 padding to a
                            // multiple of 4 entries
    int32_t* tc_gcount;     // [nb] groups in the list of every box (without padding)
    unsigned char* tc_pack; // per-apply group records: BF16 hi/lo strength images (one per block of 64 RHS)
                            // followed by the group's 16 source coordinates
    int32_t tc_wait_polls;  // poll bound of the tensor-core pipeline's waits, -1: the default (a self-check
                            // lowers it to make the abort path run)
    // box-group kernel (p2p_group.cu; indexed layout, one right-hand side): kGroupBoxes consecutive target boxes
    // stage the union of their neighbour boxes once
    int32_t group_k;        // 1: one-RHS applies run the box-group kernel
    int32_t n_groups;       // ceil(nb / kGroupBoxes)
    int32_t group_cap;      // largest union (sources): the kernel's coordinate and strength buffers
    int32_t group_pos_cap;  // largest sum of a group's padded list lengths: its position buffer
    int32_t group_grid;     // persistent grid (blocks of 8 warps)
    int32_t* g_union;       // [n_groups * kGroupBoxes * 27] union boxes of every group, ascending
    int32_t* g_nunion;      // [n_groups]
    int32_t* g_order;       // [n_groups] groups, heaviest first
    int16_t* g_pos;         // [list entries, at pk_off] every box's source list as positions in its group's buffer
    int32_t* g_mend;        // [nb] own-box prefix of every list
    int32_t* g_map;         // [2 nb] lane maps (full 128-target pass, last pass) of every box
    int32_t* g_morder;      // [n_groups * kGroupBoxes] members of every group by decreasing cost
    int4* g_copy;           // [n_groups * kGroupBoxes * 27] union copies: source start, buffer offset, length
};

// Bytes of the tensor-core group records for n points in nb boxes (0 when max_nrhs < 16).
size_t p2p_tc_pack_bytes(int64_t n, int32_t nb, int32_t max_nrhs);
// Entries of the tensor-core group lists: at most sources / 16 + nnz + 3 nb.
inline size_t p2p_tc_list_bound(int64_t sources, int64_t nnz, int32_t nb) {
    return (size_t)(sources / 16 + nnz + 3 * (int64_t)nb + 4);
}

namespace p2p_detail {

// Target boxes per group of the box-group kernel (consecutive in Morton order; at most 32).
#ifndef P2P_GROUP_BOXES
#define P2P_GROUP_BOXES 16
#endif
constexpr int kGroupBoxes = P2P_GROUP_BOXES;

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

// Persistent grid sizes of the pair kernel for the plan's kernel, layout and
// tuning (resident blocks per SM x SMs), one per right-hand-side block width.
cudaError_t p2p_pair_configure(p2p_plan* plan);

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
