// Device code of the FP32 pair kernel shared by the per-plan launch
// (p2p_apply.cu) and the persistent batched launch (p2p_batch.cu).
//
// Work.  A work item (ItemRec, built at plan time and sorted heaviest first)
// is one target box against one chunk of at most `chunk` entries of the box's
// source list: the box's own sources first, then those of its other neighbour
// boxes in ascending id.  The indexed layout (Sec. 3.2) lists box-sorted
// indices and gathers coordinates and strengths through them; the redundant
// layout (Sec. 3.3) holds a per-box copy of the coordinates and a per-apply
// repack of the strengths, so a chunk is one contiguous tile.
//
// Pipeline.  The kernel is persistent: warp w of W takes items w, w + W, ... of
// the heaviest-first list (a fixed stride, so the records of the next items can be
// loaded ahead) and keeps two shared-memory stages.  While it sweeps
// the targets of item i against stage i % 2, the sources of item i + 1 are
// already on their way into the other stage -- with cp.async (per-lane 16/8 B
// asynchronous copies) for the indexed gather, or with one or two TMA bulk
// copies (cp.async.bulk, completion on an mbarrier) for the redundant tile.
// Waits on an mbarrier are bounded; on expiry the warp sets the status word,
// drains its copies (bounded) and stops.
//
// Lanes.  A target group of nt <= 128 targets is mapped to lanes as (g, q):
// lane g + q*G holds TT targets {g, g + G, ...} (G = ceil(nt / TT)) and sweeps
// the q-th of Q = 32 / G interleaved slices of the chunk; the slice partials
// are combined through shared memory.  The map (TT, G, Q and a reciprocal for
// the divisions by G) is precomputed per item.  Items of boxes with more than
// one chunk add into the zeroed output with float2 atomics; single-chunk
// plans store directly.
#pragma once

#include "p2p_internal.cuh"

// Unroll factor of the per-lane source loop, and the launch bounds the pair
// kernel is compiled for: blocks of at most P2P_PAIR_MAX_THREADS threads, at
// least P2P_PAIR_MIN_BLOCKS of them resident (its register budget:
// 65536 / (P2P_PAIR_MAX_THREADS * P2P_PAIR_MIN_BLOCKS) registers per thread).
#ifndef P2P_PAIR_UNROLL
#define P2P_PAIR_UNROLL 2
#endif
#ifndef P2P_PAIR_MAX_THREADS
#define P2P_PAIR_MAX_THREADS 512
#endif
#ifndef P2P_PAIR_MIN_BLOCKS
#define P2P_PAIR_MIN_BLOCKS 1
#endif

namespace p2p_pair {

constexpr int kPairUnroll = P2P_PAIR_UNROLL;
constexpr float kInv4Pi = 0.0795774715459476679f;  // 1 / (4 pi)
constexpr int kMaxTT = 4;
constexpr uint32_t kBulkWaitLimit = 1u << 24;

struct PairArgs {
    const ItemRec* items;
    int64_t n_items;
    const float4* xs;       // box-sorted source coordinates (indexed layout)
    const float4* xt;       // box-sorted target coordinates (= xs when sources are the targets)
    const float4* pk_xyz;   // redundant layout: per-box source tiles
    const int32_t* nb_src;  // per-box source lists (box-sorted indices)
    const float2* lam;      // staged strengths, row stride nrhs: sorted (indexed) or packed (redundant)
    const float2* gsrc;     // staged upstream gradient (coordinate gradient only), row stride nrhs
    const int32_t* perm;
    float2* out;
    float* grad;
    unsigned int* status;
    int64_t ld;
    int32_t nrhs;
    float k;
    int32_t chunk;
    int32_t tg;
    int32_t atomic_out;
    int32_t kernel;
    int32_t red;
    int32_t sym;            // symmetric layout: unordered pairs of different boxes once, added to both ends
};

// Per-warp shared memory: two data stages (coordinates + R strengths per
// source), three index stages (the chunk's source list; an item's list stays
// until its results are scattered), the slice-reduction buffer, the source-side
// accumulator (symmetric layout only), and five mbarriers (two for data, three
// for indices).
__host__ __device__ inline int stage_bytes(int chunk, int R) { return chunk * 16 + chunk * R * 8; }
__host__ __device__ inline int warp_smem_bytes(int chunk, int R, bool sym) {
    return 2 * stage_bytes(chunk, R) + 3 * chunk * 4 + 32 * kMaxTT * R * 8 + (sym ? chunk * R * 8 : 0) + 48;
}

// ------------------------------------------------------------ async copies --

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kBulkWaitLimit) {
    const uint32_t addr = smem_addr(bar);
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ------------------------------------------------------------------ stages --

struct Stage {
    float4* sx;  // chunk coordinates
    float2* sl;  // chunk * R strengths
};

struct WarpSmem {
    unsigned char* data;  // two data stages
    int* idx;             // three index stages of `chunk` ints
    float2* red;
    float2* src_acc;      // chunk * R source-side sums (symmetric layout)
    uint64_t* bar;        // bar[0..1]: data stages, bar[2..4]: index stages
    int chunk;
    int R;
    __device__ __forceinline__ Stage stage(int i) const {
        unsigned char* b = data + i * stage_bytes(chunk, R);
        return Stage{reinterpret_cast<float4*>(b), reinterpret_cast<float2*>(b + chunk * 16)};
    }
    __device__ __forceinline__ int* index(int i) const { return idx + i * chunk; }
};

__device__ __forceinline__ WarpSmem warp_smem(unsigned char* ws, int chunk, int R, bool sym) {
    WarpSmem w;
    w.chunk = chunk;
    w.R = R;
    w.data = ws;
    unsigned char* q = ws + 2 * stage_bytes(chunk, R);
    w.idx = reinterpret_cast<int*>(q);
    q += 3 * chunk * 4;
    w.red = reinterpret_cast<float2*>(q);
    q += 32 * kMaxTT * R * 8;
    w.src_acc = reinterpret_cast<float2*>(q);
    if (sym) q += chunk * R * 8;
    w.bar = reinterpret_cast<uint64_t*>(q);
    return w;
}

// Indexed layout, two items ahead: one TMA bulk copy of the chunk's source
// list (box-sorted indices) into index stage `i` (lane 0 only).
__device__ __forceinline__ void issue_index_copy(const PairArgs& a, const ItemRec& r, const WarpSmem& w, int i) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const uint32_t n4 = (uint32_t)((r.ns + 3) & ~3);
    mbar_expect_tx(&w.bar[2 + i], n4 * 4u);
    bulk_g2s(w.index(i), a.nb_src + r.src_off, n4 * 4u, &w.bar[2 + i]);
}

// One item ahead: the chunk's coordinates and (when one pass covers every
// right-hand side, nrhs == R) strengths into data stage `i`.  Redundant: two
// TMA bulk copies of the contiguous tile (lane 0).  Indexed: per-lane cp.async
// gathers through index stage `ii`, which the caller has waited for.
template <int R>
__device__ __forceinline__ void issue_data(const PairArgs& a, const ItemRec& r, const WarpSmem& w, int i, int ii,
                                           int lane) {
    const Stage st = w.stage(i);
    const bool lam_async = a.nrhs == R;
    if (a.red) {
        if (lane == 0) {
            // the stage was last read through the generic proxy; order those reads before the bulk write
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const uint32_t n4 = (uint32_t)((r.ns + 3) & ~3);
            const uint32_t bytes = n4 * 16u + (lam_async ? n4 * (uint32_t)R * 8u : 0u);
            mbar_expect_tx(&w.bar[i], bytes);
            bulk_g2s(st.sx, a.pk_xyz + r.src_off, n4 * 16u, &w.bar[i]);
            if (lam_async) bulk_g2s(st.sl, a.lam + (int64_t)r.src_off * R, n4 * (uint32_t)R * 8u, &w.bar[i]);
        }
    } else {
        const int* idx = w.index(ii);
        for (int p = lane; p < r.ns; p += 32) {
            const int j = idx[p];
            cp_async16(st.sx + p, a.xs + j);
            if (lam_async) {
                if (R == 1) cp_async8(st.sl + p, a.lam + j);
                else {
#pragma unroll
                    for (int h = 0; h < R; h += 2) cp_async16(st.sl + p * R + h, a.lam + (int64_t)j * R + h);
                }
            }
        }
    }
    cp_async_commit();  // one group per item and lane, possibly empty
}

// Strengths of right-hand sides [rb, rb + R) for the staged chunk (the
// synchronous path used when nrhs > R).
template <int R>
__device__ __forceinline__ void load_lam_block(const PairArgs& a, const ItemRec& r, float2* sl, int rb, int lane) {
    for (int p = lane; p < r.ns; p += 32) {
        const int64_t row = (int64_t)(a.red ? r.src_off + p : a.nb_src[r.src_off + p]) * a.nrhs + rb;
#pragma unroll
        for (int q = 0; q < R; ++q) sl[p * R + q] = (rb + q < a.nrhs) ? a.lam[row + q] : make_float2(0.f, 0.f);
    }
}

// ------------------------------------------------------------------- sweep --

// One source (coordinates p, strengths l) against the lane's TT targets.  MASK:
// the source may coincide with a target (own box) and r = 0 pairs are skipped;
// otherwise r > 0 and the guard only keeps an underflowed r^2 finite.
template <int KERN, int R, int TT, bool MASK>
__device__ __forceinline__ void pair_core(const float4 p, const float2 (&l)[R], const float4 (&tx)[TT],
                                          float2 (&acc)[TT][R], float k) {
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const float dx = p.x - tx[u].x, dy = p.y - tx[u].y, dz = p.z - tx[u].z;
        float r2, inv;
        if (MASK) {
            r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            inv = rsqrtf(r2);
            inv = r2 > 0.f ? inv : 0.f;
        } else {
            // sources of other boxes are never at r = 0; starting the sum at the
            // smallest normal float keeps r^2 positive (rsqrt finite) even when the
            // squares of a very close pair underflow, at no extra instruction
            r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1.17549435e-38f)));
            inv = rsqrtf(r2);
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

// One staged source s against the lane's TT targets (pair_core on shared memory).
template <int KERN, int R, int TT, bool MASK>
__device__ __forceinline__ void pair_step(const float4* __restrict__ sx, const float2* __restrict__ sl, int s,
                                          const float4 (&tx)[TT], float2 (&acc)[TT][R], float k) {
    const float4 p = sx[s];
    float2 l[R];
#pragma unroll
    for (int r = 0; r < R; ++r) l[r] = sl[s * R + r];
    pair_core<KERN, R, TT, MASK>(p, l, tx, acc, k);
}

// pair_core for an even number of targets per lane with the packed two-lane
// FP32 instructions (add/mul/fma.f32x2): targets u and u + 1 share one register
// pair in every operand, so coordinate differences, r^2, the phase, the
// amplitude and the complex multiply-add issue once for two pairs; rsqrt and
// sincos stay per pair.  Each packed operation rounds as its scalar
// counterpart in pair_core, in the same order (the targets are kept negated so
// that p - t is one add).
template <int KERN, int R, int TT, bool MASK>
__device__ __forceinline__ void pair_core_x2(const float4 p, const float2 (&lv)[R], const float2 (&nx)[TT / 2],
                                             const float2 (&ny)[TT / 2], const float2 (&nz)[TT / 2],
                                             float2 (&ax)[TT / 2][R], float2 (&ay)[TT / 2][R], float2 k2) {
    const float2 px = make_float2(p.x, p.x), py = make_float2(p.y, p.y), pz = make_float2(p.z, p.z);
    float2 lx[R], ly[R], nly[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 l = lv[r];
        lx[r] = make_float2(l.x, l.x);
        ly[r] = make_float2(l.y, l.y);
        nly[r] = make_float2(-l.y, -l.y);
    }
#pragma unroll
    for (int v = 0; v < TT / 2; ++v) {
        const float2 dx = __fadd2_rn(px, nx[v]), dy = __fadd2_rn(py, ny[v]), dz = __fadd2_rn(pz, nz[v]);
        float2 r2, inv;
        if (MASK) {
            r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
            inv.x = r2.x > 0.f ? inv.x : 0.f;
            inv.y = r2.y > 0.f ? inv.y : 0.f;
        } else {
            const float2 tiny = make_float2(1.17549435e-38f, 1.17549435e-38f);
            r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, tiny)));
            inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        }
        if (KERN == P2P_HELMHOLTZ) {
            const float2 ph = __fmul2_rn(k2, __fmul2_rn(r2, inv));
            float2 sn, cs;
            __sincosf(ph.x, &sn.x, &cs.x);
            __sincosf(ph.y, &sn.y, &cs.y);
            const float2 gr = __fmul2_rn(cs, inv), gi = __fmul2_rn(sn, inv);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ax[v][r] = __ffma2_rn(gr, lx[r], __ffma2_rn(gi, nly[r], ax[v][r]));
                ay[v][r] = __ffma2_rn(gr, ly[r], __ffma2_rn(gi, lx[r], ay[v][r]));
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ax[v][r] = __ffma2_rn(inv, lx[r], ax[v][r]);
                ay[v][r] = __ffma2_rn(inv, ly[r], ay[v][r]);
            }
        }
    }
}

// pair_core_x2 on staged source s.
template <int KERN, int R, int TT, bool MASK>
__device__ __forceinline__ void pair_step_x2(const float4* __restrict__ sx, const float2* __restrict__ sl, int s,
                                             const float2 (&nx)[TT / 2], const float2 (&ny)[TT / 2],
                                             const float2 (&nz)[TT / 2], float2 (&ax)[TT / 2][R],
                                             float2 (&ay)[TT / 2][R], float2 k2) {
    const float4 p = sx[s];
    float2 l[R];
#pragma unroll
    for (int r = 0; r < R; ++r) l[r] = sl[s * R + r];
    pair_core_x2<KERN, R, TT, MASK>(p, l, nx, ny, nz, ax, ay, k2);
}

__device__ __forceinline__ int map_tt(int32_t m) { return m & 7; }
__device__ __forceinline__ int map_g(int32_t m) { return (m >> 3) & 63; }
__device__ __forceinline__ int map_q(int32_t m) { return (m >> 9) & 63; }
__device__ __forceinline__ int map_div(int32_t m, int x) { return (x * ((int)(((uint32_t)m) >> 15) + 1)) >> 16; }

// Sweeps the staged chunk for one target group and writes / adds the results.
template <int KERN, int R, int TT>
__device__ __forceinline__ void sweep_targets(const PairArgs& a, const float4* __restrict__ sx,
                                              const float2* __restrict__ sl, float2* red, int ns, int m_end,
                                              int tsm, int tbase, int nt, int32_t map, int rb, int lane) {
    const int G = map_g(map), Q = map_q(map);
    const int q = map_div(map, lane);
    const int g = lane - q * G;
    // output row of the lane's first target, loaded now so the sweep hides its latency
    const int32_t perm0 = lane < nt ? a.perm[tbase + lane] : 0;
    float4 tx[TT];
    float2 acc[TT][R];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const int t = g + u * G;
        // targets staged with the chunk (own box first) come from shared memory
        tx[u] = t < nt ? (tsm >= 0 && tsm + t < m_end ? sx[tsm + t] : a.xt[tbase + t]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[u][r] = make_float2(0.f, 0.f);
    }
    if (q < Q) {
        const float k = a.k;
        int s = q;
        if constexpr (TT % 2 == 0) {
            // targets in pairs for the packed two-lane instructions, accumulators (Re, Im) split by component
            float2 nx[TT / 2], ny[TT / 2], nz[TT / 2], ax[TT / 2][R], ay[TT / 2][R];
#pragma unroll
            for (int v = 0; v < TT / 2; ++v) {
                nx[v] = make_float2(-tx[2 * v].x, -tx[2 * v + 1].x);
                ny[v] = make_float2(-tx[2 * v].y, -tx[2 * v + 1].y);
                nz[v] = make_float2(-tx[2 * v].z, -tx[2 * v + 1].z);
#pragma unroll
                for (int r = 0; r < R; ++r) ax[v][r] = ay[v][r] = make_float2(0.f, 0.f);
            }
            const float2 k2 = make_float2(k, k);
            for (; s < m_end; s += Q) pair_step_x2<KERN, R, TT, true>(sx, sl, s, nx, ny, nz, ax, ay, k2);
#pragma unroll kPairUnroll
            for (; s < ns; s += Q) pair_step_x2<KERN, R, TT, false>(sx, sl, s, nx, ny, nz, ax, ay, k2);
#pragma unroll
            for (int v = 0; v < TT / 2; ++v)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    acc[2 * v][r] = make_float2(ax[v][r].x, ay[v][r].x);
                    acc[2 * v + 1][r] = make_float2(ax[v][r].y, ay[v][r].y);
                }
        } else {
            for (; s < m_end; s += Q) pair_step<KERN, R, TT, true>(sx, sl, s, tx, acc, k);  // own box: r = 0 possible
#pragma unroll kPairUnroll
            for (; s < ns; s += Q) pair_step<KERN, R, TT, false>(sx, sl, s, tx, acc, k);    // other boxes: r > 0
        }
    }
#pragma unroll
    for (int u = 0; u < TT; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) red[(u * 32 + lane) * R + r] = acc[u][r];
    __syncwarp();
    for (int t = lane; t < nt; t += 32) {
        const int u = map_div(map, t);
        const int gg = t - u * G;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
        for (int qq = 0; qq < Q; ++qq) {
            const int l2 = qq * G + gg;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 w = red[(u * 32 + l2) * R + r];
                v[r].x += w.x;
                v[r].y += w.y;
            }
        }
        const int64_t row = (int64_t)(t == lane ? perm0 : a.perm[tbase + t]) * a.ld + rb;
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

// Symmetric layout: sources of the own box (the chunk's first m_end) are swept
// as in the plain layout; every other source s meets the lane's TT targets
// once, adding G lambda_s to the targets and G lambda_t to s.  The source-side
// partials of the G lanes that share a slice are summed with a segmented
// shuffle reduction and lane g = 0 adds them to src_acc[s].  Rounds over the
// chunk run the same number of times in every lane so the shuffles converge.
template <int KERN, int R, int TT>
__device__ __forceinline__ void sweep_targets_sym(const PairArgs& a, const float4* __restrict__ sx,
                                                  const float2* __restrict__ sl, float2* red, float2* src_acc, int ns,
                                                  int m_end, int tsm, int tbase, int nt, int32_t map, int rb,
                                                  int lane) {
    const int G = map_g(map), Q = map_q(map);
    const int q = map_div(map, lane);
    const int g = lane - q * G;
    float4 tx[TT];
    float2 tl[TT][R];
    float2 acc[TT][R];
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const int t = g + u * G;
        const bool ok = t < nt && q < Q;
        const bool staged = tsm >= 0 && tsm + t < m_end;  // target staged with the chunk
        tx[u] = ok ? (staged ? sx[tsm + t] : a.xt[tbase + t]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            tl[u][r] = (ok && rb + r < a.nrhs)
                           ? (staged ? sl[(tsm + t) * R + r] : a.lam[(int64_t)(tbase + t) * a.nrhs + rb + r])
                           : make_float2(0.f, 0.f);
            acc[u][r] = make_float2(0.f, 0.f);
        }
    }
    const float k = a.k;
    if (q < Q) {
        for (int s = q; s < m_end; s += Q) pair_step<KERN, R, TT, true>(sx, sl, s, tx, acc, k);
    }
    const int m0 = m_end / Q, m1 = (ns + Q - 1) / Q;
    for (int m = m0; m < m1; ++m) {
        const int s = m * Q + q;
        const bool active = q < Q && s >= m_end && s < ns;
        float2 ps[R];
#pragma unroll
        for (int r = 0; r < R; ++r) ps[r] = make_float2(0.f, 0.f);
        if (active) {
            const float4 p = sx[s];
            float2 l[R];
#pragma unroll
            for (int r = 0; r < R; ++r) l[r] = sl[s * R + r];
#pragma unroll
            for (int u = 0; u < TT; ++u) {
                const float dx = p.x - tx[u].x, dy = p.y - tx[u].y, dz = p.z - tx[u].z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1.17549435e-38f)));
                const float inv = rsqrtf(r2);
                float gr = inv, gi = 0.f;
                if (KERN == P2P_HELMHOLTZ) {
                    float sn, cs;
                    __sincosf(k * (r2 * inv), &sn, &cs);
                    gr = cs * inv;
                    gi = sn * inv;
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    acc[u][r].x = fmaf(gr, l[r].x, fmaf(-gi, l[r].y, acc[u][r].x));
                    acc[u][r].y = fmaf(gr, l[r].y, fmaf(gi, l[r].x, acc[u][r].y));
                    ps[r].x = fmaf(gr, tl[u][r].x, fmaf(-gi, tl[u][r].y, ps[r].x));
                    ps[r].y = fmaf(gr, tl[u][r].y, fmaf(gi, tl[u][r].x, ps[r].y));
                }
            }
        }
        for (int off = 1; off < G; off <<= 1) {
            const bool take = g + off < G;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float x = __shfl_down_sync(P2P_FULL_MASK, ps[r].x, off);
                const float y = __shfl_down_sync(P2P_FULL_MASK, ps[r].y, off);
                if (take) {
                    ps[r].x += x;
                    ps[r].y += y;
                }
            }
        }
        if (active && g == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 v = src_acc[s * R + r];
                v.x += ps[r].x;
                v.y += ps[r].y;
                src_acc[s * R + r] = v;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < TT; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) red[(u * 32 + lane) * R + r] = acc[u][r];
    __syncwarp();
    for (int t = lane; t < nt; t += 32) {
        const int u = map_div(map, t);
        const int gg = t - u * G;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = make_float2(0.f, 0.f);
        for (int qq = 0; qq < Q; ++qq) {
            const int l2 = qq * G + gg;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 w = red[(u * 32 + l2) * R + r];
                v[r].x += w.x;
                v[r].y += w.y;
            }
        }
        const int64_t row = (int64_t)a.perm[tbase + t] * a.ld + rb;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (rb + r < a.nrhs) atomicAdd(a.out + row + r, make_float2(v[r].x * kInv4Pi, v[r].y * kInv4Pi));
    }
    __syncwarp();
}

template <int KERN, int R>
__device__ __forceinline__ void compute_item_sym(const PairArgs& a, const ItemRec& r, const Stage& st, const int* idx,
                                                 float2* red, float2* src_acc, int lane) {
    for (int rb = 0; rb < a.nrhs; rb += R) {
        if (a.nrhs != R) {
            __syncwarp();
            load_lam_block<R>(a, r, st.sl, rb, lane);
        }
        for (int p = lane; p < r.ns * R; p += 32) src_acc[p] = make_float2(0.f, 0.f);
        __syncwarp();
        const int m_end = r.m_end & 0xFFFF;
        const bool first = (r.m_end >> 16) & 1;
        for (int t0 = 0; t0 < r.nt; t0 += a.tg) {
            const int nt = min(a.tg, r.nt - t0);
            const int32_t map = (t0 + a.tg >= r.nt) ? r.map_last : r.map_full;
            const int tt = map_tt(map);
            const int tsm = first ? t0 : -1;
            if (tt == 1) sweep_targets_sym<KERN, R, 1>(a, st.sx, st.sl, red, src_acc, r.ns, m_end, tsm, r.tb + t0, nt, map, rb, lane);
            else if (tt == 2) sweep_targets_sym<KERN, R, 2>(a, st.sx, st.sl, red, src_acc, r.ns, m_end, tsm, r.tb + t0, nt, map, rb, lane);
            else sweep_targets_sym<KERN, R, 4>(a, st.sx, st.sl, red, src_acc, r.ns, m_end, tsm, r.tb + t0, nt, map, rb, lane);
        }
        // scatter the source-side sums of the sources outside the own box
        for (int p = (r.m_end & 0xFFFF) + lane; p < r.ns; p += 32) {
            const int64_t row = (int64_t)a.perm[idx[p]] * a.ld + rb;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (rb + q < a.nrhs) {
                    const float2 v = src_acc[p * R + q];
                    atomicAdd(a.out + row + q, make_float2(v.x * kInv4Pi, v.y * kInv4Pi));
                }
            }
        }
        __syncwarp();
    }
}

// Sweeps every target group of item `r` against its staged chunk, for every
// block of R right-hand sides.
template <int KERN, int R>
__device__ __forceinline__ void compute_item(const PairArgs& a, const ItemRec& r, const Stage& st, float2* red,
                                             int lane) {
    for (int rb = 0; rb < a.nrhs; rb += R) {
        if (a.nrhs != R) {
            __syncwarp();
            load_lam_block<R>(a, r, st.sl, rb, lane);
            __syncwarp();
        }
        const int m_end = r.m_end & 0xFFFF;
        const bool first = (r.m_end >> 16) & 1;
        for (int t0 = 0; t0 < r.nt; t0 += a.tg) {
            const int nt = min(a.tg, r.nt - t0);
            const int32_t map = (t0 + a.tg >= r.nt) ? r.map_last : r.map_full;
            const int tt = map_tt(map);
            const int tsm = first ? t0 : -1;
            if (tt == 1) sweep_targets<KERN, R, 1>(a, st.sx, st.sl, red, r.ns, m_end, tsm, r.tb + t0, nt, map, rb, lane);
            else if (tt == 2) sweep_targets<KERN, R, 2>(a, st.sx, st.sl, red, r.ns, m_end, tsm, r.tb + t0, nt, map, rb, lane);
            else sweep_targets<KERN, R, 4>(a, st.sx, st.sl, red, r.ns, m_end, tsm, r.tb + t0, nt, map, rb, lane);
        }
    }
}

template <int R>
__device__ __forceinline__ void compute_dispatch(const PairArgs& a, const ItemRec& r, const Stage& st, const int* idx,
                                                 float2* red, float2* src_acc, int lane) {
    if (a.sym) {
        if (a.kernel == P2P_HELMHOLTZ) compute_item_sym<P2P_HELMHOLTZ, R>(a, r, st, idx, red, src_acc, lane);
        else compute_item_sym<P2P_LAPLACE, R>(a, r, st, idx, red, src_acc, lane);
    } else {
        if (a.kernel == P2P_HELMHOLTZ) compute_item<P2P_HELMHOLTZ, R>(a, r, st, red, lane);
        else compute_item<P2P_LAPLACE, R>(a, r, st, red, lane);
    }
}

// Item record distributed over lanes 0..7 of a warp (field f in lane f).
__device__ __forceinline__ int32_t load_rec_lane(const ItemRec* items, int64_t idx, int64_t n, int lane) {
    return (idx < n && lane < 8) ? reinterpret_cast<const int32_t*>(items + idx)[lane] : 0;
}

__device__ __forceinline__ ItemRec gather_rec(int32_t v) {
    ItemRec r;
    r.src_off = __shfl_sync(P2P_FULL_MASK, v, 0);
    r.ns = __shfl_sync(P2P_FULL_MASK, v, 1);
    r.tb = __shfl_sync(P2P_FULL_MASK, v, 2);
    r.nt = __shfl_sync(P2P_FULL_MASK, v, 3);
    r.m_end = __shfl_sync(P2P_FULL_MASK, v, 4);
    r.map_full = __shfl_sync(P2P_FULL_MASK, v, 5);
    r.map_last = __shfl_sync(P2P_FULL_MASK, v, 6);
    r.b = __shfl_sync(P2P_FULL_MASK, v, 7);
    return r;
}

// The per-warp pipeline over the items first, first + stride, ... of `items`
// (n of them).  `args_of(rec)` points to the PairArgs an item belongs to.  At the
// top of iteration k the warp holds records k .. k+2 (lane-distributed) and
// starts loading record k+3; it issues the index copy of item k+2 (index stage
// (k+2) % 3, indexed layouts) and the data copies of item k+1 (data stage
// (k+1) % 2), then waits for item k's data and sweeps it.  Every mbarrier wait
// is bounded.
template <int R, typename ArgsOf>
__device__ __forceinline__ void run_pipeline(unsigned char* ws, int chunk, bool sym, int lane, const ItemRec* items, int64_t n,
                                             int64_t first, int64_t stride, unsigned int* status, ArgsOf args_of) {
    const WarpSmem w = warp_smem(ws, chunk, R, sym);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 5; ++i) mbar_init(&w.bar[i]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (first >= n) return;
    uint32_t parity[5] = {0u, 0u, 0u, 0u, 0u};
    bool failed = false;
    // prologue: records 0..2, index copies of items 0 and 1, data of item 0
    int32_t v0 = load_rec_lane(items, first, n, lane);
    int32_t v1 = load_rec_lane(items, first + stride, n, lane);
    int32_t v2 = load_rec_lane(items, first + 2 * stride, n, lane);
    ItemRec r0 = gather_rec(v0), r1 = gather_rec(v1);
    const bool has1 = first + stride < n;
    const PairArgs* a0 = args_of(r0);
    const PairArgs* a1 = has1 ? args_of(r1) : nullptr;
    if (lane == 0) {
        if (!a0->red) issue_index_copy(*a0, r0, w, 0);
        if (a1 && !a1->red) issue_index_copy(*a1, r1, w, 1);
    }
    if (!a0->red) {
        failed |= !mbar_wait(&w.bar[2], parity[2]);
        parity[2] ^= 1u;
    }
    failed = !__all_sync(P2P_FULL_MASK, !failed);
    if (!failed) issue_data<R>(*a0, r0, w, 0, 0, lane);
    int64_t k = 0;
    while (!failed) {
        const int cur = (int)(k & 1), nxt = cur ^ 1;
        const int i0 = (int)(k % 3), i1s = (int)((k + 1) % 3), i2s = (int)((k + 2) % 3);  // index stages
        const int64_t i1 = first + (k + 1) * stride, i2 = first + (k + 2) * stride, i3 = first + (k + 3) * stride;
        const int32_t v3 = load_rec_lane(items, i3, n, lane);  // consumed two iterations later
        const ItemRec r2 = gather_rec(v2);
        const PairArgs* a2 = i2 < n ? args_of(r2) : nullptr;
        // index copy of item k+2 (item k's list stays in its own stage until it is scattered)
        if (a2 && !a2->red && lane == 0) issue_index_copy(*a2, r2, w, i2s);
        // data of item k+1
        if (a1) {
            if (!a1->red) {
                failed |= !mbar_wait(&w.bar[2 + i1s], parity[2 + i1s]);
                parity[2 + i1s] ^= 1u;
                failed = !__all_sync(P2P_FULL_MASK, !failed);
                if (failed) break;
            }
            issue_data<R>(*a1, r1, w, nxt, i1s, lane);
        }
        // wait for item k's data
        if (a0->red) {
            failed |= !mbar_wait(&w.bar[cur], parity[cur]);
            parity[cur] ^= 1u;
        }
        if (a1) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncwarp();
        failed = !__all_sync(P2P_FULL_MASK, !failed);
        if (failed) break;
        compute_dispatch<R>(*a0, r0, w.stage(cur), w.index(i0), w.red, w.src_acc, lane);
        __syncwarp();
        if (!a1) break;
        r0 = r1;
        a0 = a1;
        r1 = r2;
        a1 = a2;
        v2 = v3;
        ++k;
        (void)i1;
    }
    if (failed) {
        if (lane == 0) atomicOr(status, P2P_DEV_TIMEOUT);
        // drain every bulk copy that may still be in flight (bounded), then the cp.async groups
        for (int i = 0; i < 5; ++i) mbar_wait(&w.bar[i], parity[i], 1u << 20);
        cp_async_wait<0>();
        __syncwarp();
    }
}

inline PairArgs base_args(const p2p_plan* p) {
    PairArgs a;
    a.items = p->items;
    a.n_items = p->n_items;
    a.xs = p->xs_src;
    a.xt = p->xs;
    a.pk_xyz = p->pk_xyz;
    a.nb_src = p->nb_src;
    a.lam = p->lam_buf;
    a.gsrc = p->g_buf;
    a.perm = p->perm;
    a.out = nullptr;
    a.grad = nullptr;
    a.status = p->status;
    a.ld = 0;
    a.nrhs = 1;
    a.k = p->k;
    a.chunk = p->tune.chunk;
    a.tg = p->tune.target_group;
    a.atomic_out = p->max_chunks > 1;
    a.kernel = p->kernel;
    a.red = p->layout == P2P_LAYOUT_REDUNDANT;
    a.sym = p->layout == P2P_LAYOUT_SYMMETRIC;
    if (a.sym) a.atomic_out = 1;  // sources scatter into other boxes' targets
    return a;
}

}  // namespace p2p_pair
