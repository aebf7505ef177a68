// Device code of the FP32 pair kernel shared by the per-plan launch
// (p2p_apply.cu) and the persistent batched launch (p2p_batch.cu).
//
// Work decomposition.  A work item is one target box b and one chunk of at
// most `chunk` sources of b's concatenated neighbourhood.  One warp owns one
// item: it stages the chunk's coordinates and strengths into its own
// shared-memory region and then sweeps every target of b against them.
// Inside the warp a target group of nt <= 128 targets is mapped to lanes as
// (g, q): lane g + q*G holds TT targets {g, g+G, ...} (G = ceil(nt/TT)) and the
// q-th of Q = 32/G interleaved slices of the chunk, so the idle-lane fraction
// stays small for any box occupancy; slice partials are combined through
// shared memory.  Items of boxes with more than one chunk add into the zeroed
// output with float2 atomics; single-chunk plans store directly.
#pragma once

#include "p2p_internal.cuh"

// Unroll factor of the per-lane source loop, and the minimum number of
// resident 512-thread blocks the pair kernel is compiled for (its register
// budget: 65536 / (512 * P2P_PAIR_MIN_BLOCKS) registers per thread).
#ifndef P2P_PAIR_UNROLL
#define P2P_PAIR_UNROLL 2
#endif
#ifndef P2P_PAIR_MIN_BLOCKS
#define P2P_PAIR_MIN_BLOCKS 1
#endif

namespace p2p_pair {

constexpr int kPairUnroll = P2P_PAIR_UNROLL;

constexpr float kInv4Pi = 0.0795774715459476679f;  // 1 / (4 pi)
constexpr int kMaxTT = 4;

struct PairArgs {
    const int4* items;
    int64_t n_items;
    const float4* xs;       // box-sorted coordinates (targets, and sources of the indexed layout)
    const float4* src_xyz;  // sources: xs (indexed) or the packed tiles (redundant)
    const float2* lam;      // staged strengths, row stride nrhs: sorted (indexed) or packed (redundant)
    const float2* gsrc;     // staged upstream gradient (coordinate gradient only), row stride nrhs
    const int32_t* box_ptr;
    const int32_t* nbr_ptr;
    const int32_t* nbr_idx;
    const int32_t* box_src;
    const int32_t* pk_off;
    const int32_t* perm;
    float2* out;
    float* grad;
    int64_t ld;
    int32_t nrhs;
    float k;
    int32_t chunk;
    int32_t tg;
    int32_t atomic_out;
};

__host__ __device__ inline int warp_smem_bytes(int chunk, int R) {
    // coords + strengths (R per source) + staged source index + segment table + reduction
    return chunk * 16 + chunk * R * 8 + chunk * 4 + 64 * 4 + 32 * kMaxTT * R * 8;
}

// Stages the coordinates of sources [s0, s0 + ns) of box b's neighbourhood and
// records, for each, the row of the strength arrays it reads.  The
// neighbourhood is concatenated with the box's own sources first (its n_b
// sources occupy positions [0, n_b)), then the other neighbour boxes in
// ascending id; only the own box can hold r = 0 pairs.  The redundant layout
// packs its tiles in the same order.
template <bool RED>
__device__ __forceinline__ void stage_sources(const PairArgs& a, int b, int s0, int ns, float4* sx, int* sj, int* seg,
                                              int lane) {
    if (RED) {
        const int base = a.pk_off[b] + s0;
        for (int p = lane; p < ns; p += 32) {
            sj[p] = base + p;
            sx[p] = a.src_xyz[base + p];
        }
    } else {
        const int e0 = a.nbr_ptr[b];
        const int ne = a.nbr_ptr[b + 1] - e0;
        const int c = lane < ne ? a.nbr_idx[e0 + lane] : -1;
        const unsigned selfm = __ballot_sync(P2P_FULL_MASK, c == b);
        const int sp = selfm ? __ffs(selfm) - 1 : 0;
        // slot 0 <- the own box, slots 1..sp <- entries 0..sp-1, later slots unchanged
        const int from = lane == 0 ? sp : (lane <= sp ? lane - 1 : lane);
        const int cs = __shfl_sync(P2P_FULL_MASK, c, from);
        int start = 0, len = 0;
        if (lane < ne) {
            start = a.box_ptr[cs];
            len = a.box_ptr[cs + 1] - start;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(P2P_FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        seg[lane] = incl - len;     // exclusive prefix: first concatenated position of slot lane
        seg[32 + lane] = start;     // first sorted index of slot lane
        __syncwarp();
        for (int p = lane; p < ns; p += 32) {
            const int pp = s0 + p;
            int lo = 0, hi = ne - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg[mid] <= pp) lo = mid;
                else hi = mid - 1;
            }
            const int j = seg[32 + lo] + (pp - seg[lo]);
            sj[p] = j;
            sx[p] = a.xs[j];
        }
    }
}

// Chooses targets-per-lane TT in {1, 2, 4} minimising the lane's instruction
// count: ceil(ns / Q) iterations of TT pair evaluations (~20 instructions
// each) plus the per-iteration source loads and loop control (~4).
__device__ __forceinline__ int choose_tt(int nt, int ns) {
    int best = 4, best_cost = 0x7fffffff;
#pragma unroll
    for (int tt = 1; tt <= 4; tt <<= 1) {
        const int g = (nt + tt - 1) / tt;
        if (g > 32) continue;
        const int q = 32 / g;
        const int cost = (20 * tt + 4) * ((ns + q - 1) / q);
        if (cost < best_cost) {
            best_cost = cost;
            best = tt;
        }
    }
    return best;
}

// One staged source against the lane's TT targets.  MASK: the source may
// coincide with a target (own box) and r = 0 pairs are skipped; otherwise r > 0
// and the guard only keeps an underflowed r^2 finite.
template <int KERN, int R, int TT, bool MASK>
__device__ __forceinline__ void pair_step(const float4* __restrict__ sx, const float2* __restrict__ sl, int s,
                                          const float4 (&tx)[TT], float2 (&acc)[TT][R], float k) {
    const float4 p = sx[s];
    float2 l[R];
#pragma unroll
    for (int r = 0; r < R; ++r) l[r] = sl[s * R + r];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const float dx = p.x - tx[u].x, dy = p.y - tx[u].y, dz = p.z - tx[u].z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float inv;
        if (MASK) {
            inv = rsqrtf(r2);
            inv = r2 > 0.f ? inv : 0.f;
        } else {
            inv = rsqrtf(fmaxf(r2, 1.17549435e-38f));
        }
        if (KERN == P2P_HELMHOLTZ) {
            float sn, cs;
            __sincosf(k * (r2 * inv), &sn, &cs);
            const float gr = cs * inv, gi = sn * inv;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                acc[u][r].x = fmaf(gr, l[r].x, fmaf(-gi, l[r].y, acc[u][r].x));
                acc[u][r].y = fmaf(gr, l[r].y, fmaf(gi, l[r].x, acc[u][r].y));
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                acc[u][r].x = fmaf(inv, l[r].x, acc[u][r].x);
                acc[u][r].y = fmaf(inv, l[r].y, acc[u][r].y);
            }
        }
    }
}

// Sweeps the staged chunk for one target group and writes / adds the results.
template <int KERN, int R, int TT>
__device__ __forceinline__ void sweep_targets(const PairArgs& a, const float4* __restrict__ sx,
                                              const float2* __restrict__ sl, float2* red, int ns, int m_end,
                                              int tbase, int nt, int rb, int lane) {
    const int G = (nt + TT - 1) / TT;
    const int Q = 32 / G;
    const int g = lane % G, q = lane / G;
    float4 tx[TT];
    float2 acc[TT][R];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const int t = g + u * G;
        tx[u] = t < nt ? a.xs[tbase + t] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[u][r] = make_float2(0.f, 0.f);
    }
    if (q < Q) {
        const float k = a.k;
        int s = q;
        for (; s < m_end; s += Q) pair_step<KERN, R, TT, true>(sx, sl, s, tx, acc, k);   // own box: r = 0 possible
#pragma unroll kPairUnroll
        for (; s < ns; s += Q) pair_step<KERN, R, TT, false>(sx, sl, s, tx, acc, k);     // other boxes: r > 0
    }
#pragma unroll
    for (int u = 0; u < TT; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) red[(lane * TT + u) * R + r] = acc[u][r];
    __syncwarp();
    for (int t = lane; t < nt; t += 32) {
        const int gg = t % G, u = t / G;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
        for (int qq = 0; qq < Q; ++qq) {
            const int l2 = qq * G + gg;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 w = red[(l2 * TT + u) * R + r];
                v[r].x += w.x;
                v[r].y += w.y;
            }
        }
        const int64_t row = (int64_t)a.perm[tbase + t] * a.ld + rb;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (rb + r < a.nrhs) {
                const float2 o = make_float2(v[r].x * kInv4Pi, v[r].y * kInv4Pi);
                if (a.atomic_out) atomicAdd(a.out + row + r, o);
                else a.out[row + r] = o;
            }
        }
    }
    __syncwarp();
}

// Processes one work item (target box, source chunk) with the calling warp:
// stage the chunk into the warp's shared-memory region `ws`, then sweep every
// target group of the box against it for every block of R right-hand sides.
template <int KERN, int R, bool RED>
__device__ __forceinline__ void process_item(const PairArgs& a, int64_t item, unsigned char* ws, int lane) {
    const int chunk = a.chunk;
    float4* sx = reinterpret_cast<float4*>(ws);
    float2* sl = reinterpret_cast<float2*>(ws + chunk * 16);
    int* sj = reinterpret_cast<int*>(ws + chunk * 16 + chunk * R * 8);
    int* seg = sj + chunk;
    float2* red = reinterpret_cast<float2*>(seg + 64);

    const int4 it = a.items[item];
    const int b = it.x, s0 = it.y;
    const int ns = min(chunk, a.box_src[b] - s0);
    stage_sources<RED>(a, b, s0, ns, sx, sj, seg, lane);
    const int tb = a.box_ptr[b];
    const int nt_all = a.box_ptr[b + 1] - tb;
    const int m_end = max(0, min(ns, nt_all - s0));  // own-box sources of this chunk come first
    for (int rb = 0; rb < a.nrhs; rb += R) {
        __syncwarp();
        for (int p = lane; p < ns; p += 32) {
            const int64_t row = (int64_t)sj[p] * a.nrhs + rb;
#pragma unroll
            for (int r = 0; r < R; ++r) sl[p * R + r] = (rb + r < a.nrhs) ? a.lam[row + r] : make_float2(0.f, 0.f);
        }
        __syncwarp();
        for (int t0 = 0; t0 < nt_all; t0 += a.tg) {
            const int nt = min(a.tg, nt_all - t0);
            const int tt = choose_tt(nt, ns);
            if (tt == 1) sweep_targets<KERN, R, 1>(a, sx, sl, red, ns, m_end, tb + t0, nt, rb, lane);
            else if (tt == 2) sweep_targets<KERN, R, 2>(a, sx, sl, red, ns, m_end, tb + t0, nt, rb, lane);
            else sweep_targets<KERN, R, 4>(a, sx, sl, red, ns, m_end, tb + t0, nt, rb, lane);
        }
    }
    __syncwarp();
}

inline PairArgs base_args(const p2p_plan* p) {
    PairArgs a;
    a.items = p->items;
    a.n_items = p->n_items;
    a.xs = p->xs;
    a.src_xyz = p->layout == P2P_LAYOUT_REDUNDANT ? p->pk_xyz : p->xs;
    a.lam = p->lam_buf;
    a.gsrc = p->g_buf;
    a.box_ptr = p->box_ptr;
    a.nbr_ptr = p->nbr_ptr;
    a.nbr_idx = p->nbr_idx;
    a.box_src = p->box_src;
    a.pk_off = p->pk_off;
    a.perm = p->perm;
    a.out = nullptr;
    a.grad = nullptr;
    a.ld = 0;
    a.nrhs = 1;
    a.k = p->k;
    a.chunk = p->tune.chunk;
    a.tg = p->tune.target_group;
    a.atomic_out = p->max_chunks > 1;
    return a;
}

}  // namespace p2p_pair
