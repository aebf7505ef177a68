// Box-group kernel: the one-right-hand-side FP32 sum with the sources of
// several target boxes staged once.
//
// Why.  Neighbouring target boxes share most of their neighbourhoods (Sec. 3.1:
// the 27 boxes around a leaf).  The staged pipeline (p2p_pair.cuh) stages every
// box's list for that box alone, and the direct kernel (p2p_direct.cuh) loads
// each source through the L1 once per target box.  Here a group of kGroupBoxes
// consecutive target boxes (Morton order keeps them close) stages the union of
// their neighbour boxes' sources in shared memory once -- every union box's
// sources contiguous -- together with every member's source list rewritten as
// 16-bit positions in that buffer (own box first, as in the plan's lists), and
// each member then sweeps its list from shared memory only.  Each result is
// stored once (no atomics, no zeroing).
//
// Plan time (k_group_build, one warp per group): the members' neighbour lists
// (contiguous in the CSR) are sorted and made unique into the union, a prefix of
// the union boxes' sizes places them in the buffer, the members' lists become
// buffer positions, and the members are ranked by cost.  Groups are ordered by
// cost (targets x sources), heaviest first.
//
// Apply (k_pair_group, 8 warps per block, persistent): per group, the warps
// copy the union boxes' coordinates and staged strengths and the members'
// position lists (cp.async) following the group's copy list, which was read
// into shared memory while the previous group was swept; meanwhile every warp
// loads its first member's lane map (built at plan time), targets and output
// rows; then each warp sweeps the group's costliest member not yet taken (the
// first eight one each, the rest from a shared counter): TT targets per lane, Q
// source slices, the next source read ahead, the slice partials summed through
// shared memory.
//
// Build parameters (measured on the sphere at 16 points per box): groups of 16
// boxes, 8 warps per block, 80 registers (3 blocks per SM); groups of 24 or 32,
// blocks of 4 warps, 64 registers or two buffers per block measured slower.
#include <algorithm>

#include "p2p_pair.cuh"

using namespace p2p_detail;
using namespace p2p_pair;

namespace {

// Launch shape and lane-map cost of the apply kernel (build parameters).
#ifndef P2P_GROUP_MIN_BLOCKS
#define P2P_GROUP_MIN_BLOCKS 3
#endif
#ifndef P2P_GROUP_PER_ITER
#define P2P_GROUP_PER_ITER 4
#endif

#ifndef P2P_GROUP_WARPS
#define P2P_GROUP_WARPS 8
#endif

constexpr int kGroupWarps = P2P_GROUP_WARPS;  // warps of the apply kernel's blocks
constexpr int kBuildWarps = 4;
constexpr int kUnionMax = kGroupBoxes * 27;  // union entries of a group at most
constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }
constexpr int kSortSlots = pow2_at_least(kUnionMax);
constexpr int kPass = 4 * 32;    // targets of one pass of a member
static_assert(kGroupBoxes >= 1 && kGroupBoxes <= 32, "members are ranked by one warp");

// One warp per group g: union of the members' neighbour boxes, its buffer
// offsets, the members' position lists, lane maps and cost ranks.  maxes[0]:
// largest union (sources), maxes[1]: largest sum of the members' padded list
// lengths.
__global__ void __launch_bounds__(kBuildWarps * 32)
    k_group_build(const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                  const int32_t* __restrict__ nbr_self, const int32_t* __restrict__ box_ptr,
                  const int32_t* __restrict__ src_box_ptr, const int32_t* __restrict__ box_src,
                  const int32_t* __restrict__ pk_off, int32_t nb, int32_t n_groups, int32_t* __restrict__ g_union,
                  int32_t* __restrict__ g_nunion, int16_t* __restrict__ g_pos, int32_t* __restrict__ g_mend,
                  int32_t* __restrict__ g_map, int32_t* __restrict__ g_morder, int4* __restrict__ g_copy,
                  uint64_t* __restrict__ keys, int32_t* __restrict__ vals, int32_t* __restrict__ maxes) {
    __shared__ int32_t buf_all[kBuildWarps][kSortSlots];
    __shared__ int32_t off_all[kBuildWarps][kUnionMax + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * kBuildWarps + warp;
    if (g >= n_groups) return;
    int32_t* buf = buf_all[warp];
    int32_t* uoff = off_all[warp];
    const int32_t b0 = (int32_t)g * kGroupBoxes, b1 = min(nb, b0 + kGroupBoxes);
    const int32_t e0 = nbr_ptr[b0], ne = nbr_ptr[b1] - e0;  // <= kUnionMax (lists hold <= 27 entries)
    for (int i = lane; i < kSortSlots; i += 32) buf[i] = i < ne ? nbr_idx[e0 + i] : INT32_MAX;
    __syncwarp();
    // bitonic sort of the slots, ascending
    for (int k = 2; k <= kSortSlots; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < kSortSlots; i += 32) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t x = buf[i], y = buf[l];
                    const bool up = (i & k) == 0;
                    if (up ? x > y : x < y) {
                        buf[i] = y;
                        buf[l] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
    // unique entries, compacted into the union (kSortSlots / 32 consecutive slots per lane)
    constexpr int kPer = kSortSlots / 32;
    int32_t v[kPer];
    int cnt = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = lane * kPer + u;
        v[u] = buf[i];
        const bool keep = v[u] != INT32_MAX && (i == 0 || buf[i - 1] != v[u]);
        if (!keep) v[u] = -1;
        cnt += keep;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(P2P_FULL_MASK, incl, o);
        if (lane >= o) incl += y;
    }
    const int nu = __shfl_sync(P2P_FULL_MASK, incl, 31);
    __syncwarp();
    int pos = incl - cnt;
    int32_t* U = g_union + g * kUnionMax;
#pragma unroll
    for (int u = 0; u < kPer; ++u)
        if (v[u] >= 0) {
            U[pos] = v[u];
            buf[pos] = v[u];  // the union stays in shared memory for the lookups below (pos <= slot index)
            ++pos;
        }
    __syncwarp();
    // buffer offsets of the union boxes: exclusive prefix of their sizes
    int sz[kPer];
    int tot = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = lane * kPer + u;
        sz[u] = i < nu ? src_box_ptr[buf[i] + 1] - src_box_ptr[buf[i]] : 0;
        tot += sz[u];
    }
    int run = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(P2P_FULL_MASK, run, o);
        if (lane >= o) run += y;
    }
    int acc = run - tot;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = lane * kPer + u;
        if (i <= nu && i < kUnionMax + 1) uoff[i] = acc;
        acc += sz[u];
    }
    const int total = __shfl_sync(P2P_FULL_MASK, run, 31);
    if (lane == 0) {
        g_nunion[g] = nu;
        uoff[nu] = total;
        atomicMax(&maxes[0], total);
        atomicMax(&maxes[1], pk_off[b1] - pk_off[b0]);
    }
    __syncwarp();
    // the copies that stage the union: source start, buffer offset and length of every union box
    for (int i = lane; i < nu; i += 32)
        g_copy[g * kUnionMax + i] = make_int4(src_box_ptr[buf[i]], uoff[i], uoff[i + 1] - uoff[i], 0);
    // members: their lists (own box first, then the others ascending, as the plan's source lists) as buffer
    // positions; lane = entry of the member's neighbour list, moved to its place in that order
    int64_t cost = 0;
    for (int32_t b = b0; b < b1; ++b) {
        const int32_t f0 = nbr_ptr[b], ne_b = nbr_ptr[b + 1] - f0;  // <= 27
        const int32_t c = lane < ne_b ? nbr_idx[f0 + lane] : -1;
        int sp;
        if (nbr_self) {
            sp = nbr_self[b];  // -1: no source box in the own cell
        } else {
            const unsigned selfm = __ballot_sync(P2P_FULL_MASK, c == b);
            sp = selfm ? __ffs(selfm) - 1 : 0;
        }
        const int from = sp < 0 ? lane : (lane == 0 ? sp : (lane <= sp ? lane - 1 : lane));
        const int32_t cs = __shfl_sync(P2P_FULL_MASK, c, from);
        int start = 0, len = 0;
        if (lane < ne_b) {
            int lo = 0, hi = nu - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (buf[mid] < cs) lo = mid + 1;
                else hi = mid;
            }
            start = uoff[lo];
            len = uoff[lo + 1] - start;
        }
        int li = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(P2P_FULL_MASK, li, o);
            if (lane >= o) li += y;
        }
        int16_t* list = g_pos + pk_off[b] + (li - len);
        for (int e = 0; e < len; ++e) list[e] = (int16_t)(start + e);
        const int own_len = __shfl_sync(P2P_FULL_MASK, len, 0);
        if (lane == 0) {
            const int32_t nt = box_ptr[b + 1] - box_ptr[b], S = box_src[b];
            g_mend[b] = sp < 0 ? 0 : own_len;
            cost += (int64_t)nt * S;
            // lane maps of a full pass and of the last pass
            g_map[2 * (int64_t)b] = p2p_lane_map(min(nt, kPass), S, 32, P2P_GROUP_PER_ITER);
            g_map[2 * (int64_t)b + 1] = p2p_lane_map(nt - ((nt - 1) / kPass) * kPass, S, 32, P2P_GROUP_PER_ITER);
        }
    }
    if (lane == 0) {
        keys[g] = 0xFFFFFFFFull - (uint64_t)min(cost, (int64_t)0xFFFFFFFF);
        vals[g] = (int32_t)g;
    }
    // members by decreasing cost (ties by position)
    const int nm = b1 - b0;
    int64_t mc = -1;
    if (lane < nm) mc = (int64_t)(box_ptr[b0 + lane + 1] - box_ptr[b0 + lane]) * box_src[b0 + lane];
    int rank = 0;
    for (int j = 0; j < nm; ++j) {
        const int64_t cj = __shfl_sync(P2P_FULL_MASK, mc, j);
        rank += (cj > mc) || (cj == mc && j < lane);
    }
    if (lane < nm) g_morder[g * kGroupBoxes + rank] = lane;
}

struct GroupArgs {
    const int32_t* order;   // groups, heaviest first
    int32_t n_groups;
    int32_t nb;
    int32_t cap;            // largest union (sources): the coordinate and strength buffers
    int32_t pos_cap;        // largest sum of a group's padded list lengths: the position buffer
    const int32_t* g_union;
    const int32_t* g_nunion;
    const int16_t* g_pos;   // members' lists as buffer positions, at the plan's list offsets pk_off
    const int32_t* g_mend;  // own-box prefix of every list
    const int32_t* g_map;   // lane maps of a full pass and of the last pass of every box
    const int32_t* g_morder;  // members of every group by decreasing cost
    const int4* g_copy;     // per group and union box: source start, buffer offset, length
    const int32_t* pk_off;
    const int32_t* box_ptr;
    const int32_t* box_src;
    const int32_t* src_box_ptr;
    const float4* xs;       // box-sorted source coordinates
    const float4* xt;       // box-sorted target coordinates
    const float2* lam;      // staged strengths, box-sorted source order
    const int32_t* perm;
    float2* out;
    int64_t ld;
    float k;
};

// Targets of a pass (lane map `map`, nt targets from tb) into tx, and the lane's output row.
__device__ __forceinline__ void load_pass(const GroupArgs& a, int tb, int nt, int32_t map, int lane, float4 (&tx)[4],
                                          int32_t& perm0) {
    const int G = map_g(map), Q = map_q(map), TT = map_tt(map);
    const int q = map_div(map, lane);
    const int g = lane - q * G;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int t = g + u * G;
        tx[u] = (u < TT && q < Q && t < nt) ? __ldg(a.xt + tb + t) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    perm0 = lane < nt ? __ldg(a.perm + tb + lane) : 0;
}

// One pass of a member (targets tb .. tb + nt - 1, coordinates in tx4) against its list pl[0 .. S) of buffer
// positions, the first m_end of them its own box's sources (r = 0 possible).
template <int KERN, int TT>
__device__ __forceinline__ void member_pass(const GroupArgs& a, const float4* __restrict__ sx,
                                            const float2* __restrict__ sl, const int16_t* __restrict__ pl, int S,
                                            int m_end, float2* red, int tb, int nt, int32_t map,
                                            const float4 (&tx4)[4], int32_t perm0, int lane) {
    const int G = map_g(map), Q = map_q(map);
    const int q = map_div(map, lane);
    float4 tx[TT];
    float2 acc[TT][1];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        tx[u] = tx4[u];
        acc[u][0] = make_float2(0.f, 0.f);
    }
    const float k = a.k;
    if (q < Q) {
        int s = q;
        if constexpr (TT % 2 == 0) {
            float2 nx[TT / 2], ny[TT / 2], nz[TT / 2], ax[TT / 2][1], ay[TT / 2][1];
#pragma unroll
            for (int v = 0; v < TT / 2; ++v) {
                nx[v] = make_float2(-tx[2 * v].x, -tx[2 * v + 1].x);
                ny[v] = make_float2(-tx[2 * v].y, -tx[2 * v + 1].y);
                nz[v] = make_float2(-tx[2 * v].z, -tx[2 * v + 1].z);
                ax[v][0] = ay[v][0] = make_float2(0.f, 0.f);
            }
            const float2 k2 = make_float2(k, k);
            for (; s < m_end; s += Q) {
                const int j = pl[s];
                const float2 l[1] = {sl[j]};
                pair_core_x2<KERN, 1, TT, true>(sx[j], l, nx, ny, nz, ax, ay, k2);
            }
            // the next source's position and data are read before this one is evaluated
            if (s < S) {
                int j = pl[s];
                float4 p = sx[j];
                float2 l[1] = {sl[j]};
                for (; s < S; s += Q) {
                    const int sn = s + Q;
                    const int jn = sn < S ? pl[sn] : j;
                    const float4 pn = sx[jn];
                    const float2 ln = sl[jn];
                    pair_core_x2<KERN, 1, TT, false>(p, l, nx, ny, nz, ax, ay, k2);
                    p = pn;
                    l[0] = ln;
                }
            }
#pragma unroll
            for (int v = 0; v < TT / 2; ++v) {
                acc[2 * v][0] = make_float2(ax[v][0].x, ay[v][0].x);
                acc[2 * v + 1][0] = make_float2(ax[v][0].y, ay[v][0].y);
            }
        } else {
            for (; s < m_end; s += Q) {
                const int j = pl[s];
                const float2 l[1] = {sl[j]};
                pair_core<KERN, 1, TT, true>(sx[j], l, tx, acc, k);
            }
            if (s < S) {
                int j = pl[s];
                float4 p = sx[j];
                float2 l[1] = {sl[j]};
                for (; s < S; s += Q) {
                    const int sn = s + Q;
                    const int jn = sn < S ? pl[sn] : j;
                    const float4 pn = sx[jn];
                    const float2 ln = sl[jn];
                    pair_core<KERN, 1, TT, false>(p, l, tx, acc, k);
                    p = pn;
                    l[0] = ln;
                }
            }
        }
    }
    // slice partials -> one sum per target
#pragma unroll
    for (int u = 0; u < TT; ++u) red[u * 32 + lane] = acc[u][0];
    __syncwarp();
    for (int t = lane; t < nt; t += 32) {
        const int u = map_div(map, t);
        const int gg = t - u * G;
        float2 v = make_float2(0.f, 0.f);
        for (int qq = 0; qq < Q; ++qq) {
            const float2 w = red[u * 32 + qq * G + gg];
            v.x += w.x;
            v.y += w.y;
        }
        const int64_t row = (int64_t)(t == lane ? perm0 : __ldg(a.perm + tb + t)) * a.ld;
        a.out[row] = make_float2(v.x * kInv4Pi, v.y * kInv4Pi);
    }
    __syncwarp();
}

template <int KERN>
__device__ __forceinline__ void run_pass(const GroupArgs& a, const float4* sx, const float2* sl, const int16_t* pl,
                                         int S, int m_end, float2* red, int tb, int nt, int32_t map,
                                         const float4 (&tx)[4], int32_t perm0, int lane) {
    const int tt = map_tt(map);
    if (tt == 1) member_pass<KERN, 1>(a, sx, sl, pl, S, m_end, red, tb, nt, map, tx, perm0, lane);
    else if (tt == 2) member_pass<KERN, 2>(a, sx, sl, pl, S, m_end, red, tb, nt, map, tx, perm0, lane);
    else member_pass<KERN, 4>(a, sx, sl, pl, S, m_end, red, tb, nt, map, tx, perm0, lane);
}

// Member box b: the lane map of its first pass, that pass's targets and output rows.
struct Member {
    int32_t b, map, perm0;
    int tb, ntb;
    float4 tx[4];
};

__device__ __forceinline__ void load_member(const GroupArgs& a, int32_t b, int lane, Member& m) {
    m.b = b;
    m.tb = __ldg(a.box_ptr + b);
    m.ntb = __ldg(a.box_ptr + b + 1) - m.tb;
    m.map = __ldg(a.g_map + 2 * (int64_t)b + (m.ntb <= kPass ? 1 : 0));
    load_pass(a, m.tb, min(m.ntb, kPass), m.map, lane, m.tx, m.perm0);
}

template <int KERN>
__device__ __forceinline__ void sweep_member(const GroupArgs& a, const float4* sx, const float2* sl,
                                             const int16_t* pos, int32_t pos0, float2* red, Member& m, int lane) {
    const int16_t* pl = pos + (__ldg(a.pk_off + m.b) - pos0);
    const int S = __ldg(a.box_src + m.b), m_end = __ldg(a.g_mend + m.b);
    run_pass<KERN>(a, sx, sl, pl, S, m_end, red, m.tb, min(m.ntb, kPass), m.map, m.tx, m.perm0, lane);
    // boxes of more than 128 targets: further passes (the last one with its own lane map)
    for (int t0 = kPass; t0 < m.ntb; t0 += kPass) {
        const int nt = min(kPass, m.ntb - t0);
        m.map = __ldg(a.g_map + 2 * (int64_t)m.b + (t0 + kPass >= m.ntb ? 1 : 0));
        load_pass(a, m.tb + t0, nt, m.map, lane, m.tx, m.perm0);
        run_pass<KERN>(a, sx, sl, pl, S, m_end, red, m.tb + t0, nt, m.map, m.tx, m.perm0, lane);
    }
}

// Shared memory of a block: coordinates and strengths of the union (cap entries), the members' positions
// (pos_cap 16-bit entries), the next group's union copies, the member counter and the warps' slice-reduction
// buffers.
struct GroupSmem {
    float4* sx;
    float2* sl;
    int16_t* pos;
    int4* ents;
    int32_t* next;
    float2* red;
};

__host__ __device__ inline size_t pos_bytes(int pos_cap) { return ((size_t)pos_cap * 2 + 15) / 16 * 16; }

__host__ __device__ inline size_t group_smem_bytes(int cap, int pos_cap) {
    return (size_t)cap * 24 + pos_bytes(pos_cap) + 16 * kUnionMax + 16 + (size_t)kGroupWarps * kMaxTT * 32 * 8;
}

__device__ __forceinline__ GroupSmem group_smem(unsigned char* smem, int cap, int pos_cap) {
    GroupSmem m;
    m.sx = reinterpret_cast<float4*>(smem);
    m.sl = reinterpret_cast<float2*>(smem + (size_t)cap * 16);
    m.pos = reinterpret_cast<int16_t*>(smem + (size_t)cap * 24);
    unsigned char* q = smem + (size_t)cap * 24 + pos_bytes(pos_cap);
    m.ents = reinterpret_cast<int4*>(q);
    m.next = reinterpret_cast<int32_t*>(q + 16 * kUnionMax);
    m.red = reinterpret_cast<float2*>(q + 16 * kUnionMax + 16);
    return m;
}

// Group g's copy list (one int4 per union box) into shared memory, as its own cp.async group.
__device__ __forceinline__ void prefetch_copies(const GroupArgs& a, int32_t g, int4* ents) {
    const int nu = __ldg(a.g_nunion + g);
    const int4* src = a.g_copy + (int64_t)g * kUnionMax;
    for (int i = threadIdx.x; i < nu; i += kGroupWarps * 32) cp_async16(ents + i, src + i);
    cp_async_commit();
}

// Block = one group at a time: warp w takes the group's w-th costliest member, then further members from a
// shared counter as it finishes.
template <int KERN>
__global__ void __launch_bounds__(kGroupWarps * 32, P2P_GROUP_MIN_BLOCKS) k_pair_group(const __grid_constant__ GroupArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const GroupSmem sm = group_smem(smem, a.cap, a.pos_cap);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* red = sm.red + warp * kMaxTT * 32;
    // the first group's union copies, read ahead into shared memory like every later group's
    if (blockIdx.x < a.n_groups) prefetch_copies(a, __ldg(a.order + blockIdx.x), sm.ents);
    for (int64_t gi = blockIdx.x; gi < a.n_groups; gi += gridDim.x) {
        const int32_t g = __ldg(a.order + gi);
        const int nu = __ldg(a.g_nunion + g);
        const int32_t b0 = g * kGroupBoxes;
        const int nm = min(a.nb - b0, kGroupBoxes);
        const int32_t* order = a.g_morder + (int64_t)g * kGroupBoxes;
        const int32_t pos0 = __ldg(a.pk_off + b0), npos = __ldg(a.pk_off + b0 + nm) - pos0;
        // this group's copy list has arrived, and every warp has finished the previous group
        cp_async_wait<0>();
        __syncthreads();
        // the union: one warp per union box, its sources contiguous in the buffer; the members' position lists
        // contiguous from the group's first list (every list padded to 4 entries, so 8-byte copies)
        for (int u = warp; u < nu; u += kGroupWarps) {
            const int4 c = sm.ents[u];
            for (int e = lane; e < c.z; e += 32) {
                cp_async16(sm.sx + c.y + e, a.xs + c.x + e);
                cp_async8(sm.sl + c.y + e, a.lam + c.x + e);
            }
        }
        for (int e = threadIdx.x; e < npos / 4; e += kGroupWarps * 32)
            cp_async8(sm.pos + 4 * e, a.g_pos + pos0 + 4 * e);
        cp_async_commit();
        // this warp's first member, loaded while the union is staged
        Member m;
        const bool has = warp < nm;
        if (has) load_member(a, b0 + __ldg(order + warp), lane, m);
        if (threadIdx.x == 0) *sm.next = kGroupWarps;
        cp_async_wait<0>();
        __syncthreads();
        // the next group's copy list, in flight while this group is swept
        if (gi + gridDim.x < a.n_groups) prefetch_copies(a, __ldg(a.order + gi + gridDim.x), sm.ents);
        if (has) {
            sweep_member<KERN>(a, sm.sx, sm.sl, sm.pos, pos0, red, m, lane);
            while (true) {
                int idx = 0;
                if (lane == 0) idx = atomicAdd(sm.next, 1);
                idx = __shfl_sync(P2P_FULL_MASK, idx, 0);
                if (idx >= nm) break;
                load_member(a, b0 + __ldg(order + idx), lane, m);
                sweep_member<KERN>(a, sm.sx, sm.sl, sm.pos, pos0, red, m, lane);
            }
        }
    }
}

}  // namespace

// Plan time: builds the groups of a plan (g_* arrays carved by the plan) and orders them heaviest first.
// keys / vals / keys_alt / vals_alt / radix_ws: sort scratch of at least n_groups entries.  Returns the
// largest union and the largest group list total in cap[0], cap[1].
cudaError_t p2p_group_build(p2p_plan* p, const int32_t* nbr_ptr, const int32_t* nbr_idx, uint64_t* keys,
                            int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, void* radix_ws, int32_t* maxes,
                            cudaStream_t s, int32_t* cap) {
    cap[0] = cap[1] = 0;
    const int32_t ng = p->n_groups;
    if (ng == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(maxes, 0, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_group_build<<<(unsigned)((ng + kBuildWarps - 1) / kBuildWarps), kBuildWarps * 32, 0, s>>>(
        nbr_ptr, nbr_idx, p->two_sets ? p->nbr_self : nullptr, p->box_ptr, p->src_box_ptr, p->box_src, p->pk_off,
        p->nb, ng, p->g_union, p->g_nunion, p->g_pos, p->g_mend, p->g_map, p->g_morder, p->g_copy, keys, vals,
        maxes);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bool in_alt = false;
    e = radix_sort_pairs(keys, vals, keys_alt, vals_alt, ng, 32, radix_ws, s, &in_alt);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(p->g_order, in_alt ? vals_alt : vals, (size_t)ng * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(cap, maxes, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// Persistent grid of the group kernel for the plan's buffer sizes (0: no block fits).
cudaError_t p2p_group_configure(p2p_plan* p) {
    p->group_grid = 0;
    if (!p->group_k) return cudaSuccess;
    int dev = 0, sms = 0, optin = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = group_smem_bytes(p->group_cap, p->group_pos_cap);
    if (smem > (size_t)optin) return cudaSuccess;
    auto kern = p->kernel == P2P_LAPLACE ? k_pair_group<P2P_LAPLACE> : k_pair_group<P2P_HELMHOLTZ>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGroupWarps * 32, smem);
    if (e == cudaSuccess) p->group_grid = per_sm * sms;
    return e;
}

// Apply: one right-hand side from the staged strengths (box-sorted source order) into out.
p2p_status p2p_group_launch(const p2p_plan* p, float2* out, int64_t ld, float k, cudaStream_t s) {
    GroupArgs a;
    a.order = p->g_order;
    a.n_groups = p->n_groups;
    a.nb = p->nb;
    a.cap = p->group_cap;
    a.pos_cap = p->group_pos_cap;
    a.g_union = p->g_union;
    a.g_nunion = p->g_nunion;
    a.g_pos = p->g_pos;
    a.g_mend = p->g_mend;
    a.g_map = p->g_map;
    a.g_morder = p->g_morder;
    a.g_copy = p->g_copy;
    a.pk_off = p->pk_off;
    a.box_ptr = p->box_ptr;
    a.box_src = p->box_src;
    a.src_box_ptr = p->src_box_ptr;
    a.xs = p->xs_src;
    a.xt = p->xs;
    a.lam = p->lam_buf;
    a.perm = p->perm;
    a.out = out;
    a.ld = ld;
    a.k = k;
    const size_t smem = group_smem_bytes(p->group_cap, p->group_pos_cap);
    auto kern = p->kernel == P2P_LAPLACE ? k_pair_group<P2P_LAPLACE> : k_pair_group<P2P_HELMHOLTZ>;
    P2P_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "p2p_apply/group");
    const int grid = (int)std::min<int64_t>(p->group_grid, p->n_groups);
    kern<<<grid, kGroupWarps * 32, smem, s>>>(a);
    P2P_CHECK_LAUNCH("p2p_apply/group");
    return P2P_OK;
}
