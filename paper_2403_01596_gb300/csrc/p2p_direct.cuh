// Device code of the direct pair kernel: the near-field sum for plans whose
// boxes hold few targets (a handful to a few dozen points per box).
//
// Why a second kernel.  The staged pipeline (p2p_pair.cuh) spends a fixed
// amount of work per item -- record, bulk / cp.async staging, waits, slice
// reduction -- that a box of ~8 targets against ~100 sources cannot amortise:
// each lane then sweeps only a dozen sources.  Here a warp serves K boxes at
// once (K = 1, 2, 4, 8, 16 or 32; 32 / K lanes per box, down to one lane per box
// for boxes of a point or two), an item is one whole box (its
// complete source list, so every result is written once, without atomics), and
// the sources are read straight from global memory through the L1, with the
// next sources prefetched into registers, instead of being staged in shared
// memory.  The redundant layout (Sec. 3.3) reads the box's contiguous tile of
// coordinates and repacked strengths; the indexed layout (Sec. 3.2) reads the
// box's source list and gathers through it.  The sources are swept in blocks of
// two per lane with the next block's loads in flight; 64 registers per thread
// keep 32 warps per SM resident, which is what hides the L2 latency (deeper
// blocks cost occupancy and measured slower).
//
// Lanes.  A pass over up to 4 * 32 / K targets of the box maps lane l of the
// box's lanes to (g, q) with the lane map of the item (TT targets per lane,
// G target slots, Q = lanes / G source slices); the Q slice partials of a
// target are summed through shared memory within the box's lanes.
#pragma once

#include "p2p_pair.cuh"

namespace p2p_direct {

using p2p_pair::kInv4Pi;
using p2p_pair::map_div;
using p2p_pair::map_g;
using p2p_pair::map_q;
using p2p_pair::map_tt;

constexpr int kDirectWarps = 8;  // warps per block

struct DirectArgs {
    const ItemRec* items;   // one per target box, heaviest first; lane maps for 32 / K lanes
    int64_t n_items;
    const float4* xs;       // box-sorted source coordinates (indexed layout)
    const float4* xt;       // box-sorted target coordinates
    const float4* pk_xyz;   // redundant layout: per-box source tiles
    const int32_t* nb_src;  // indexed layout: per-box source lists (box-sorted source indices)
    const float2* lam;      // staged strengths of one right-hand side: sorted rows or packed rows
    const int32_t* perm;    // target permutation (sorted position -> original index)
    float2* out;
    int64_t ld;
    float k;
};

#ifndef P2P_DIRECT_BLOCK
#define P2P_DIRECT_BLOCK 2
#endif
constexpr int kBlock = P2P_DIRECT_BLOCK;  // sources per lane per block of the software pipeline

// The lane's sources s0, s0 + Q, ... < ns in blocks of kBlock: while a block is
// evaluated (pair(p, l, own) per source, own = s < m_end: a source of the box's
// own cell, where r = 0 is possible) the next block's coordinates and strengths
// are already being loaded, and for the indexed layout the list entries of the
// block after that as well.  The own cell's sources (the list's prefix) go
// through the same pipeline as the rest.
template <bool RED, typename Pair>
__device__ __forceinline__ void sweep_blocks(const DirectArgs& a, int32_t off, int s0, int Q, int ns, int m_end,
                                             Pair pair) {
    if (s0 >= ns) return;
    const int stride = kBlock * Q;
    float4 p[kBlock];
    float2 l[kBlock];
    int j[kBlock];  // indexed layout: list entries of the next block to load
    auto load_idx = [&](int base) {
#pragma unroll
        for (int u = 0; u < kBlock; ++u) {
            const int s = base + u * Q;
            j[u] = (!RED && s < ns) ? __ldg(a.nb_src + off + s) : 0;
        }
    };
    auto load_data = [&](int base, float4 (&pp)[kBlock], float2 (&ll)[kBlock]) {
#pragma unroll
        for (int u = 0; u < kBlock; ++u) {
            const int s = base + u * Q;
            pp[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            ll[u] = make_float2(0.f, 0.f);
            if (s < ns) {
                if (RED) {
                    pp[u] = __ldg(a.pk_xyz + off + s);
                    ll[u] = __ldg(a.lam + off + s);
                } else {
                    pp[u] = __ldg(a.xs + j[u]);
                    ll[u] = __ldg(a.lam + j[u]);
                }
            }
        }
    };
    load_idx(s0);
    load_data(s0, p, l);
    load_idx(s0 + stride);
    for (int base = s0; base < ns; base += stride) {
        float4 pn[kBlock];
        float2 ln[kBlock];
        load_data(base + stride, pn, ln);
        load_idx(base + 2 * stride);
#pragma unroll
        for (int u = 0; u < kBlock; ++u)
            if (base + u * Q < ns) pair(p[u], l[u], base + u * Q < m_end);
#pragma unroll
        for (int u = 0; u < kBlock; ++u) {
            p[u] = pn[u];
            l[u] = ln[u];
        }
    }
}

// One pass of one box's lanes over targets t0 .. t0 + nt - 1 against the box's
// whole source list; results stored to out.  red: the box's 4 * GS partials.
template <int KERN, int TT, bool RED, int GS>
__device__ __forceinline__ void box_pass(const DirectArgs& a, const ItemRec& r, int t0, int nt, int32_t map, int ll,
                                         float2* red, unsigned gmask) {
    const int G = map_g(map), Q = map_q(map);
    const int q = map_div(map, ll);
    const int g = ll - q * G;
    const int tb = r.tb + t0;
    const int ns = r.ns, m_end = r.m_end & 0xFFFF;
    const int32_t perm0 = ll < nt ? __ldg(a.perm + tb + ll) : 0;  // loaded early, used after the sweep
    float4 tx[TT];
    float2 acc[TT][1];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const int t = g + u * G;
        tx[u] = (q < Q && t < nt) ? __ldg(a.xt + tb + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        acc[u][0] = make_float2(0.f, 0.f);
    }
    if (q < Q) {
        const float k = a.k;
        const int32_t off = r.src_off;
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
            // blocks of kBlock sources per lane, the next block's loads in flight; own cell first (r = 0 possible)
            sweep_blocks<RED>(a, off, q, Q, ns, m_end, [&](const float4& p, const float2& l, bool own) {
                const float2 lv[1] = {l};
                if (own) p2p_pair::pair_core_x2<KERN, 1, TT, true>(p, lv, nx, ny, nz, ax, ay, k2);
                else p2p_pair::pair_core_x2<KERN, 1, TT, false>(p, lv, nx, ny, nz, ax, ay, k2);
            });
#pragma unroll
            for (int v = 0; v < TT / 2; ++v) {
                acc[2 * v][0] = make_float2(ax[v][0].x, ay[v][0].x);
                acc[2 * v + 1][0] = make_float2(ax[v][0].y, ay[v][0].y);
            }
        } else {
            sweep_blocks<RED>(a, off, q, Q, ns, m_end, [&](const float4& p, const float2& l, bool own) {
                const float2 lv[1] = {l};
                if (own) p2p_pair::pair_core<KERN, 1, TT, true>(p, lv, tx, acc, k);
                else p2p_pair::pair_core<KERN, 1, TT, false>(p, lv, tx, acc, k);
            });
        }
    }
    // slice partials of the box's lanes -> one sum per target
#pragma unroll
    for (int u = 0; u < TT; ++u) red[u * GS + ll] = acc[u][0];
    __syncwarp(gmask);
    for (int t = ll; t < nt; t += GS) {
        const int u = map_div(map, t);
        const int gg = t - u * G;
        float2 v = make_float2(0.f, 0.f);
        for (int qq = 0; qq < Q; ++qq) {
            const float2 w = red[u * GS + qq * G + gg];
            v.x += w.x;
            v.y += w.y;
        }
        const int64_t row = (int64_t)(t == ll ? perm0 : __ldg(a.perm + tb + t)) * a.ld;
        a.out[row] = make_float2(v.x * kInv4Pi, v.y * kInv4Pi);
    }
    __syncwarp(gmask);
}

__device__ __forceinline__ ItemRec load_item(const ItemRec* p) {
    const int4 u = __ldg(reinterpret_cast<const int4*>(p));
    const int4 w = __ldg(reinterpret_cast<const int4*>(p) + 1);
    ItemRec r;
    r.src_off = u.x;
    r.ns = u.y;
    r.tb = u.z;
    r.nt = u.w;
    r.m_end = w.x;
    r.map_full = w.y;
    r.map_last = w.z;
    r.b = w.w;
    return r;
}

// Warp w of the persistent grid takes the K items w K .. w K + K - 1, then
// those W K further (W = warps in the grid); lanes j * 32 / K .. serve item j.
template <int KERN, bool RED, int K>
__device__ __forceinline__ void run_direct(const DirectArgs& a, float2* red_warp, int warp_global, int64_t warps_total,
                                           int lane) {
    constexpr int GS = 32 / K;
    constexpr int kPass = 4 * GS;  // targets per pass (TT <= 4 on GS lanes)
    const int grp = lane / GS, ll = lane - grp * GS;
    const unsigned gmask = (GS == 32) ? 0xffffffffu : (((1u << GS) - 1u) << (grp * GS));
    float2* red = red_warp + grp * 4 * GS;
    const int64_t step = warps_total * K;
    int64_t idx = (int64_t)warp_global * K + grp;
    ItemRec r = idx < a.n_items ? load_item(a.items + idx) : ItemRec{};
    while (idx < a.n_items) {
        const int64_t nidx = idx + step;
        const ItemRec rn = nidx < a.n_items ? load_item(a.items + nidx) : ItemRec{};  // next item in flight
        for (int t0 = 0; t0 < r.nt; t0 += kPass) {
            const int nt = min(kPass, r.nt - t0);
            const int32_t map = (t0 + kPass >= r.nt) ? r.map_last : r.map_full;
            const int tt = map_tt(map);
            if (tt == 1) box_pass<KERN, 1, RED, GS>(a, r, t0, nt, map, ll, red, gmask);
            else if (tt == 2) box_pass<KERN, 2, RED, GS>(a, r, t0, nt, map, ll, red, gmask);
            else box_pass<KERN, 4, RED, GS>(a, r, t0, nt, map, ll, red, gmask);
        }
        idx = nidx;
        r = rn;
    }
}

}  // namespace p2p_direct
