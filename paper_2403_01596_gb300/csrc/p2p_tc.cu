// Multi-RHS P2P on the 5th-generation tensor cores (tcgen05, TMEM accumulator).
//
// Contraction.  A unit of work is one target box b and a group of nt <= TG of
// its targets (T = nt rounded up to 8).  For every group of 16 consecutive
// box-sorted sources of a neighbour box, one real MMA chain adds
//
//     D[128 x 2T] += A[128 x 16] . B[16 x 2T],
//     A[r, s] = Re lambda[s, r],  A[64 + r, s] = Im lambda[s, r]   (r: RHS within a block of 64)
//     B[s, t] = Re G(x_t, y_s),   B[s, T + t]  = Im G(x_t, y_s),
//
// so that Re out[t, r] = D[r, t] - D[64 + r, T + t] and Im out[t, r] =
// D[r, T + t] + D[64 + r, t] (the four real products of a complex product; no
// padded M rows and no negated copy).  G is formed on the CUDA cores in FP32
// (rsqrt, sincos), both operands are split x = hi + lo into BF16, and three MMAs
// (hi.hi + hi.lo + lo.hi, kind::f16, FP32 accumulation in TMEM) keep the product
// error near 2^-16.  With NP = 3 parts (hi + mid + lo, ~24 bits) six MMAs take
// every part product p.q with p + q < 3, and the product error is near 2^-24.
//
// Group records.  The A operand of a source group does not depend on the target
// box, so a pass per apply (k_tc_pack) writes every group's hi and lo images,
// already in the operand's shared-memory layout, followed by the group's source
// coordinates; the main kernel moves a record with one TMA bulk copy.  The plan
// keeps, per box, the list of the groups of its neighbour boxes (ascending box
// id), padded with -1 to a multiple of four entries.
//
// Main kernel (k_p2p_tc): persistent, one CTA per SM, units (box, target group)
// round robin over the CTAs in Morton order (neighbouring CTAs share records in
// L2).  Warp roles:
//   warps 0-3    one producer per G set: walks a unit's group list four entries (a quad) at a time and
//                issues entry 4q + s into a slot of set s (metadata, TMA bulk copy of the record, the
//                unit's targets with the first quad)
//   warps 4-19   four G sets of four warps: G tile in FP32, BF16 hi/lo split into the slot's B operand
//   warps 20-23  one MMA issuer per set (one thread): once the set has written B, the three MMAs (per RHS
//                block) into the set's own accumulator, committed to the slot's release barrier
//   warps 24-27  epilogue: sums the sets' accumulators (TMEM -> registers), combines Re/Im through
//                shared memory and writes out[perm[t]]
// (with P2P_TC_SETS = 2: two producers, two sets of eight warps, entries taken in pairs)
// Four independent issue chains (one per set) keep the tensor core fed with the
// small (N = 2T) MMAs.  With the hi/lo split (units of up to 32 targets) two TMEM
// buffers alternate between a CTA's units so the epilogue of one unit overlaps
// the MMAs of the next; the three-part split takes units of up to 64 targets in
// one buffer.
//
// Every wait is bounded: a wait that runs out sets the plan's status word and an
// abort flag; every role then stops (the epilogue warps decide together through
// a barrier reduction), the producer waits (bounded) for the bulk copies it
// issued, each MMA issuer for its MMAs, and the CTA frees its TMEM and returns.
//
// Operands use the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices, the two K-adjacent cores of a 16-wide K slice 128 bytes apart
// (leading byte offset) and 8-row groups 256 bytes apart (stride byte offset).
#include <cuda_bf16.h>
#include <math.h>

#include "p2p_internal.cuh"

using namespace p2p_detail;

namespace {

constexpr float kInv4Pi = 0.0795774715459476679f;
constexpr int kSrcGroup = 16;          // sources per stage (MMA K)
constexpr int kPart = 4096;            // one BF16 image of a 128 x 16 A operand
constexpr int kImage = 2 * kPart;      // hi + lo images (the operand self-check)
constexpr int kLbo = 128, kSbo = 256;  // core-matrix strides (K direction, 8-row groups)
constexpr int kSetCols = 256;          // TMEM columns of a unit buffer of 32-target units (an accumulator per set)
// G sets (independent producer -> G -> MMA chains; 2 or 4, the group lists are
// padded to multiples of 4).  On the 2^21-point ellipsoid at 64 RHS four sets of
// four warps measured 5.1 ms against 5.3 for two sets of eight with units of up
// to 64 targets; two sets would also halve the accumulators of the three-part
// split, whose error grows with the accumulation chains.
#ifndef P2P_TC_SETS
#define P2P_TC_SETS 4
#endif
constexpr int kSets = P2P_TC_SETS;     // G sets; set s takes list entries s, s + kSets, ... of a unit
constexpr int kSetWarps = 16 / kSets;  // warps of one G set
constexpr int kSetThreads = 32 * kSetWarps;
constexpr int kGWarp0 = kSets, kMmaWarp0 = kGWarp0 + kSetWarps * kSets, kEpiWarp0 = kMmaWarp0 + kSets;
constexpr int kWarps = kEpiWarp0 + 4;
constexpr int kThreads = kWarps * 32;
// A waiting thread is suspended (up to kSuspendNs per poll) until the phase
// completes, so idle roles do not take issue slots from the working warps.
// kWaitLimit polls bound every wait to a few seconds at most.
constexpr uint32_t kSuspendNs = 10000;
constexpr uint32_t kWaitLimit = 1u << 18;
constexpr uint32_t kDrainLimit = 1u << 14;

// --------------------------------------------------------------- PTX helpers --

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading and stride byte offsets (>> 4),
// descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kLbo >> 4) << 16) | ((uint64_t)(kSbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N, M = 128.
__host__ __device__ inline uint32_t idesc_bf16_f32(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return done != 0;
}

// Bounded wait; gives up early once *abort is set.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (abort && (i & 15u) == 15u && *abort) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Named barrier 5 for the epilogue warps (0 is __syncthreads).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 5, 128;" ::: "memory"); }
// Barrier of the 128 epilogue threads that also ORs a condition over them.
__device__ __forceinline__ bool epi_any(bool c) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 5, 128, q;\n\t"
        "selp.s32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((int)c)
        : "memory");
    return r != 0;
}

// 32 lanes x 8 consecutive 32-bit columns of TMEM into registers.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 16 consecutive 32-bit columns of TMEM into registers.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo with hi, lo BF16 (round to nearest), two values per 32-bit word.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    float2 hf = __bfloat1622float2(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

// x = hi + mid + lo with three BF16 parts (each the round-to-nearest of what the
// previous parts leave), two values per 32-bit word: the parts carry ~24 bits.
__device__ __forceinline__ void split3(float a, float b, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const float ra = a - hf.x, rb = b - hf.y;
    __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
    const float2 mf = __bfloat1622float2(m);
    __nv_bfloat162 l = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
    hi = *reinterpret_cast<uint32_t*>(&h);
    mid = *reinterpret_cast<uint32_t*>(&m);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

__device__ __forceinline__ void split1(float a, uint16_t& hi, uint16_t& lo) {
    __nv_bfloat16 h = __float2bfloat16_rn(a);
    __nv_bfloat16 l = __float2bfloat16_rn(a - __bfloat162float(h));
    hi = *reinterpret_cast<uint16_t*>(&h);
    lo = *reinterpret_cast<uint16_t*>(&l);
}

// Byte offset of element (row, k) of a K-major operand with 16-wide K slices.
__host__ __device__ inline int op_off(int row, int k) {
    return (row >> 3) * kSbo + (k >> 3) * kLbo + (row & 7) * 16 + (k & 7) * 2;
}

// Splits n values (n = 1, 2, 4 or 8, consecutive K elements of one row) and
// stores the hi and lo parts.
template <int N>
__device__ __forceinline__ void store_split(unsigned char* hi, unsigned char* lo, int off, const float (&v)[N]) {
    if constexpr (N == 1) {
        uint16_t h, l;
        split1(v[0], h, l);
        *reinterpret_cast<uint16_t*>(hi + off) = h;
        *reinterpret_cast<uint16_t*>(lo + off) = l;
    } else if constexpr (N == 2) {
        uint32_t h, l;
        split2(v[0], v[1], h, l);
        *reinterpret_cast<uint32_t*>(hi + off) = h;
        *reinterpret_cast<uint32_t*>(lo + off) = l;
    } else if constexpr (N == 4) {
        uint2 h, l;
        split2(v[0], v[1], h.x, l.x);
        split2(v[2], v[3], h.y, l.y);
        *reinterpret_cast<uint2*>(hi + off) = h;
        *reinterpret_cast<uint2*>(lo + off) = l;
    } else {
        uint4 h, l;
        split2(v[0], v[1], h.x, l.x);
        split2(v[2], v[3], h.y, l.y);
        split2(v[4], v[5], h.z, l.z);
        split2(v[6], v[7], h.w, l.w);
        *reinterpret_cast<uint4*>(hi + off) = h;
        *reinterpret_cast<uint4*>(lo + off) = l;
    }
}

// Splits n values (n = 2, 4 or 8, consecutive K elements of one row) into NP
// BF16 parts (2: hi, lo; 3: hi, mid, lo) stored at `off` in the images starting
// at part0, part_bytes apart.
template <int NP, int N>
__device__ __forceinline__ void store_parts(unsigned char* part0, int part_bytes, int off, const float (&v)[N]) {
    if constexpr (NP == 2) {
        store_split<N>(part0, part0 + part_bytes, off, v);
    } else if constexpr (N == 1) {
        uint32_t h, m, l;
        split3(v[0], 0.f, h, m, l);
        *reinterpret_cast<uint16_t*>(part0 + off) = (uint16_t)(h & 0xffffu);
        *reinterpret_cast<uint16_t*>(part0 + part_bytes + off) = (uint16_t)(m & 0xffffu);
        *reinterpret_cast<uint16_t*>(part0 + 2 * part_bytes + off) = (uint16_t)(l & 0xffffu);
    } else {
        uint32_t h[N / 2], m[N / 2], l[N / 2];
#pragma unroll
        for (int i = 0; i < N / 2; ++i) split3(v[2 * i], v[2 * i + 1], h[i], m[i], l[i]);
        unsigned char* dst[3] = {part0, part0 + part_bytes, part0 + 2 * part_bytes};
        const uint32_t* src[3] = {h, m, l};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if constexpr (N == 2) {
                *reinterpret_cast<uint32_t*>(dst[q] + off) = src[q][0];
            } else if constexpr (N == 4) {
                *reinterpret_cast<uint2*>(dst[q] + off) = make_uint2(src[q][0], src[q][1]);
            } else {
                *reinterpret_cast<uint4*>(dst[q] + off) = make_uint4(src[q][0], src[q][1], src[q][2], src[q][3]);
            }
        }
    }
}

// ----------------------------------------------------------- strength pre-pack --

// Bytes of one group record: the NP BF16 part images of every block of 64 RHS,
// then the group's 16 source coordinates (w = 1 marks a padding slot).
__host__ __device__ inline int record_bytes(int rb_count, int np) { return rb_count * np * kPart + kSrcGroup * 16; }

// The records of one launch (a chunk of rb_launch RHS blocks) are contiguous:
// chunk c starts chunk_bytes * c into the buffer, group g's record
// record_bytes(rb_launch, NP) * g into the chunk.
//
// Block (group g, RHS block rb), 128 threads: thread (r = tid % 64, o = tid / 64)
// splits Re and Im lambda of RHS rb * 64 + r for sources 8o .. 8o + 7 of the
// group into rows r and 64 + r of the group's NP part images in its chunk's
// record.  Sources past the box's end and RHS past nrhs are zero.  The first
// block of each chunk also writes the record's coordinates.
template <int NP>
__global__ void __launch_bounds__(128) k_tc_pack(const float2* __restrict__ lam, int64_t ld, int32_t nrhs,
                                                 const int32_t* __restrict__ perm, const int32_t* __restrict__ box_ptr,
                                                 const float4* __restrict__ xs, const int32_t* __restrict__ gstart,
                                                 int32_t nb, int32_t rb_launch, int64_t chunk_bytes,
                                                 unsigned char* __restrict__ pack) {
    const int g = blockIdx.x, rb = blockIdx.y;
    // box of group g: the last c with gstart[c] <= g
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gstart[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const int c = lo;
    const int j = g - gstart[c];
    const int s0 = box_ptr[c] + j * kSrcGroup;
    const int cnt = min(kSrcGroup, box_ptr[c + 1] - s0);
    const int lb = rb % rb_launch;
    unsigned char* rec = pack + (rb / rb_launch) * chunk_bytes + (int64_t)g * record_bytes(rb_launch, NP);
    if (lb == 0 && threadIdx.x < kSrcGroup) {
        const int k = threadIdx.x;
        reinterpret_cast<float4*>(rec + rb_launch * NP * kPart)[k] =
            k < cnt ? xs[s0 + k] : make_float4(0.f, 0.f, 0.f, 1.f);
    }
    const int r = threadIdx.x & 63, o = threadIdx.x >> 6;
    const int rr = rb * 64 + r;
    float re[8], im[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = 8 * o + e;
        float2 v = make_float2(0.f, 0.f);
        if (k < cnt && rr < nrhs) v = lam[(int64_t)perm[s0 + k] * ld + rr];
        re[e] = v.x;
        im[e] = v.y;
    }
    unsigned char* img = rec + lb * NP * kPart;
    store_parts<NP, 8>(img, kPart, op_off(r, 8 * o), re);
    store_parts<NP, 8>(img, kPart, op_off(64 + r, 8 * o), im);
}

// ------------------------------------------------------------------ main kernel --

struct TcArgs {
    const float4* xs;              // box-sorted coordinates
    const unsigned char* pack;     // group records
    const int32_t* box_ptr;
    const int32_t* glist_off;      // per-box group lists (padded to multiples of kSets)
    const int32_t* glist;
    const int32_t* gcount;
    const int32_t* perm;
    float2* out;
    int64_t ld;
    int32_t nrhs;
    int32_t rb_count;              // RHS blocks of 64
    int32_t tg;                    // targets per unit (multiple of 8)
    int32_t ngrp;                  // units per box: ceil(max_box / tg)
    int32_t nb;
    int32_t slots;                 // pipeline slots per G set
    int32_t slot_bytes;
    int32_t np;                    // BF16 parts per operand: 2 (hi, lo) or 3 (hi, mid, lo)
    int32_t nbuf;                  // unit buffers in TMEM (512 / (kSets x 2 tg x rb_count)): 2, or 1 at 64 targets
    float k;
    unsigned int* status;
    uint32_t wait_limit;           // polls of every pipeline wait (kWaitLimit unless a self-check lowers it)
};

// Slot layout: group record (A part images, source coordinates), the unit's
// targets, the NP parts of B (2T rows each, T <= tg), metadata.
__host__ __device__ inline int slot_t_off(int rb_count, int np) { return record_bytes(rb_count, np); }
__host__ __device__ inline int slot_b_off(int rb_count, int tg, int np) { return record_bytes(rb_count, np) + tg * 16; }
__host__ __device__ inline int slot_b_half(int tg) { return (2 * tg / 8) * kSbo; }  // bytes of one B part
__host__ __device__ inline int slot_meta_off(int rb_count, int tg, int np) {
    return slot_b_off(rb_count, tg, np) + np * slot_b_half(tg);
}
__host__ __device__ inline int slot_bytes_for(int rb_count, int tg, int np) {
    return (slot_meta_off(rb_count, tg, np) + 16 + 1023) / 1024 * 1024;
}
constexpr int kEpiBytes = 8 * 64 * 8;  // epilogue exchange: 8 targets x 64 RHS x complex
__host__ __device__ inline int tc_smem_bytes(int slots, int slot_bytes) {
    return kSets * slots * slot_bytes + kEpiBytes + 1024;  // barriers: (3 kSets slots + 4) x 8 bytes <= 1024
}

// Metadata of a stage (int4): x = group (-1: padding, nothing to do), y = flags,
// z = targets of the unit.  Flags: first quad of the unit (the stage carries the
// unit's targets, the set's accumulator starts), last quad, done.
constexpr int kFirst = 1, kLast = 2, kDone = 4;

struct TcSmem {
    unsigned char* slots;  // kSets x slots
    float2* epi;
    uint64_t* full;        // [kSets * slots] TMA bytes + producer arrival
    uint64_t* full_b;      // [kSets * slots] the G set's threads (B operand written)
    uint64_t* empty;       // [kSets * slots] MMA commit
    uint64_t* acc_full;    // [2] one commit per set after a unit's last quad
    uint64_t* acc_empty;   // [2] the epilogue's 128 threads
    uint32_t* tmem_slot;
    int* abort;
};

__device__ __forceinline__ TcSmem carve(unsigned char* smem, int slots, int slot_bytes) {
    TcSmem s;
    const int n = kSets * slots;
    s.slots = smem;
    s.epi = reinterpret_cast<float2*>(smem + (size_t)n * slot_bytes);
    uint64_t* b = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(s.epi) + kEpiBytes);
    s.full = b;
    s.full_b = b + n;
    s.empty = b + 2 * n;
    s.acc_full = b + 3 * n;
    s.acc_empty = b + 3 * n + 2;
    s.tmem_slot = reinterpret_cast<uint32_t*>(b + 3 * n + 4);
    s.abort = reinterpret_cast<int*>(s.tmem_slot + 1);
    return s;
}

__device__ __forceinline__ void set_abort(const TcArgs& a, const TcSmem& sm) {
    *(volatile int*)sm.abort = 1;
    atomicOr(a.status, P2P_DEV_TIMEOUT | P2P_DEV_TC_FAULTED);
}

// Unit u of the round-robin sequence: target box, first target, target count (0: empty unit).  Units run box
// by box in Morton order, a box's ngrp target groups next to each other (CTAs serving neighbouring units share
// records in L2).  When the grid is a multiple of ngrp, each round of the grid covers whole boxes and a CTA
// would take the same group of every box it serves -- the CTAs of the first group carrying most of the work --
// so round k rotates the groups of its boxes by k.
__device__ __forceinline__ void unit_of(const TcArgs& a, int64_t u, int& b, int& t0, int& nt) {
    b = (int)(u / a.ngrp);
    int j = (int)(u - (int64_t)b * a.ngrp);
    if (gridDim.x % (unsigned)a.ngrp == 0) j = (int)((j + u / gridDim.x) % a.ngrp);
    t0 = j * a.tg;
    const int n_b = a.box_ptr[b + 1] - a.box_ptr[b];
    nt = max(0, min(a.tg, n_b - t0));
}

// Ring of one set's slots: slot index and the parity of its round.
struct Ring {
    int slot;
    uint32_t phase;
    __device__ __forceinline__ void advance(int slots) {
        if (++slot == slots) {
            slot = 0;
            phase ^= 1u;
        }
    }
};

// ---- producer of set s (one warp; lane 0 issues) ----
// A unit's group list is walked four entries (a quad) at a time, entry 4q + s going to set s.
template <bool LIMITED>
__device__ void run_producer(const TcArgs& a, const TcSmem& sm, int64_t units, int set, int lane) {
    volatile int* abort = sm.abort;
    const uint32_t wlim = LIMITED ? a.wait_limit : kWaitLimit;
    const bool active = lane == 0;
    Ring r{0, 0u};
    int64_t staged = 0;  // stages this producer has armed (their copies may still be in flight)
    const uint32_t rec = (uint32_t)record_bytes(a.rb_count, a.np);
    const int t_off = slot_t_off(a.rb_count, a.np), meta_off = slot_meta_off(a.rb_count, a.tg, a.np);
    bool failed = false;
    auto slot_base = [&](int slot) { return sm.slots + (size_t)(set * a.slots + slot) * a.slot_bytes; };
    for (int64_t u = blockIdx.x; u < units && !failed; u += gridDim.x) {
        int b, t0, nt;
        unit_of(a, u, b, t0, nt);
        if (nt == 0) continue;
        const int off = a.glist_off[b], len = a.glist_off[b + 1] - off;
        const float4* tsrc = a.xs + a.box_ptr[b] + t0;
        for (int w0 = 0; w0 < len && !failed; w0 += 32) {
            // 32 entries of the list (8 quads) in the warp's lanes
            const int gl = w0 + lane < len ? a.glist[off + w0 + lane] : -1;
            const int nq = min(32 / kSets, (len - w0) / kSets);
            for (int q = 0; q < nq; ++q) {
                const int g = __shfl_sync(P2P_FULL_MASK, gl, q * kSets + set);
                bool ok = true;
                if (active) ok = mbar_wait(&sm.empty[set * a.slots + r.slot], r.phase ^ 1u, abort, wlim);
                if (!__all_sync(P2P_FULL_MASK, ok)) {
                    if (!ok && !*abort) set_abort(a, sm);
                    failed = true;
                    break;
                }
                if (active) {
                    unsigned char* base = slot_base(r.slot);
                    const int qq = w0 / kSets + q;
                    const bool first = qq == 0, last = w0 + (q + 1) * kSets == len;
                    *reinterpret_cast<int4*>(base + meta_off) =
                        make_int4(g, (first ? kFirst : 0) | (last ? kLast : 0), nt, 0);
                    uint64_t* bar = &sm.full[set * a.slots + r.slot];
                    if (g >= 0) {
                        fence_async_smem();  // the slot was last read through the generic proxy
                        mbar_expect_tx(bar, rec + (first ? (uint32_t)nt * 16u : 0u));
                        bulk_g2s(base, a.pack + (int64_t)g * rec, rec, bar);
                        if (first) bulk_g2s(base + t_off, tsrc, (uint32_t)nt * 16u, bar);
                    } else {
                        mbar_arrive(bar);
                    }
                }
                ++staged;
                r.advance(a.slots);
            }
        }
    }
    // a terminal stage for each set
    if (!failed) {
        bool ok = true;
        if (active) ok = mbar_wait(&sm.empty[set * a.slots + r.slot], r.phase ^ 1u, abort, wlim);
        if (__all_sync(P2P_FULL_MASK, ok)) {
            if (active) {
                *reinterpret_cast<int4*>(slot_base(r.slot) + meta_off) = make_int4(-1, kDone, 0, 0);
                mbar_arrive(&sm.full[set * a.slots + r.slot]);
            }
        } else {
            if (!ok && !*abort) set_abort(a, sm);
            failed = true;
        }
    }
    if (failed && active) {
        // wait (bounded) for the bulk copies of this set's latest round of slots (the ones it has armed)
        const int armed = (int)(staged < a.slots ? staged : a.slots);
        for (int i = 0; i < armed; ++i) {
            if (--r.slot < 0) {
                r.slot += a.slots;
                r.phase ^= 1u;
            }
            mbar_wait(&sm.full[set * a.slots + r.slot], r.phase, nullptr, kDrainLimit);
        }
    }
}

// ---- G sets (128 threads each); the set's first thread issues its MMAs ----
// G tile part of one thread: target tx against sources h SP .. h SP + SP - 1.
// For SP >= 2 the sources go in pairs through the packed two-lane FP32
// instructions (each rounding as its scalar counterpart); rsqrt and sincos
// stay per pair.  r = 0 and padding slots (w = 1) give 0.
template <int KERN, int SP, int NP>
__device__ __forceinline__ void g_tile(const float4* __restrict__ sx, float4 tx, int t, int h, int T,
                                       unsigned char* b_part0, int b_part_bytes, float k) {
    float re[SP], im[SP];
    if constexpr (SP == 1) {
        const float4 p = sx[h];
        const float dx = p.x - tx.x, dy = p.y - tx.y, dz = p.z - tx.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float inv = rsqrtf(r2);
        const bool ok = r2 > 0.f && p.w == 0.f;
        if (KERN == P2P_LAPLACE) {
            re[0] = ok ? inv : 0.f;
            im[0] = 0.f;
        } else {
            float sn, cs;
            __sincosf(k * (r2 * inv), &sn, &cs);
            re[0] = ok ? cs * inv : 0.f;
            im[0] = ok ? sn * inv : 0.f;
        }
    } else {
        const float2 ntx = make_float2(-tx.x, -tx.x), nty = make_float2(-tx.y, -tx.y), ntz = make_float2(-tx.z, -tx.z);
        const float2 k2 = make_float2(k, k);
#pragma unroll
        for (int e = 0; e < SP; e += 2) {
            const float4 p0 = sx[h * SP + e], p1 = sx[h * SP + e + 1];
            const float2 dx = __fadd2_rn(make_float2(p0.x, p1.x), ntx);
            const float2 dy = __fadd2_rn(make_float2(p0.y, p1.y), nty);
            const float2 dz = __fadd2_rn(make_float2(p0.z, p1.z), ntz);
            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
            const bool ok0 = r2.x > 0.f && p0.w == 0.f, ok1 = r2.y > 0.f && p1.w == 0.f;
            if (KERN == P2P_LAPLACE) {
                re[e] = ok0 ? inv.x : 0.f;
                re[e + 1] = ok1 ? inv.y : 0.f;
                im[e] = im[e + 1] = 0.f;
            } else {
                const float2 ph = __fmul2_rn(k2, __fmul2_rn(r2, inv));
                float2 sn, cs;
                __sincosf(ph.x, &sn.x, &cs.x);
                __sincosf(ph.y, &sn.y, &cs.y);
                const float2 gr = __fmul2_rn(cs, inv), gi = __fmul2_rn(sn, inv);
                re[e] = ok0 ? gr.x : 0.f;
                re[e + 1] = ok1 ? gr.y : 0.f;
                im[e] = ok0 ? gi.x : 0.f;
                im[e + 1] = ok1 ? gi.y : 0.f;
            }
        }
    }
    store_parts<NP, SP>(b_part0, b_part_bytes, op_off(t, h * SP), re);
    store_parts<NP, SP>(b_part0, b_part_bytes, op_off(T + t, h * SP), im);
}

template <int KERN, bool LIMITED, int NP>
__device__ void run_gset(const TcArgs& a, const TcSmem& sm, int set, int i) {
    volatile int* abort = sm.abort;
    const uint32_t wlim = LIMITED ? a.wait_limit : kWaitLimit;
    const int t_off = slot_t_off(a.rb_count, NP), b_off = slot_b_off(a.rb_count, a.tg, NP);
    const int b_half = slot_b_half(a.tg), meta_off = slot_meta_off(a.rb_count, a.tg, NP);
    // this thread's task in the current unit: target t, sources h sp .. h sp + sp - 1 (set at the unit's first quad)
    float4 tx = make_float4(0.f, 0.f, 0.f, 0.f);
    int T = 8, sp = 1, t = 0, h = 0;
    bool act = false;
    Ring r{0, 0u};
    while (true) {
        const int idx = set * a.slots + r.slot;
        unsigned char* base = sm.slots + (size_t)idx * a.slot_bytes;
        if (!mbar_wait(&sm.full[idx], r.phase, abort, wlim)) {
            if (!*abort) set_abort(a, sm);
            break;
        }
        const int4 m = *reinterpret_cast<const int4*>(base + meta_off);
        if (m.y & kDone) break;
        if (m.y & kFirst) {
            T = (m.z + 7) & ~7;
            // sources per task: the smallest power of two with 16 T / SP <= kSetThreads tasks
            sp = 1;
            while (kSrcGroup * T > sp * kSetThreads) sp <<= 1;
            // eight consecutive threads take eight consecutive targets (rows of one 8-row core matrix) and the
            // next bits the source slices, so a warp's B stores fill whole core matrices (no bank conflicts)
            const int rest = i >> 3, H = kSrcGroup / sp;
            h = rest % H;
            t = (rest / H) * 8 + (i & 7);
            act = t < T;
            // the targets travel with the real stages of the first quad
            if (m.x >= 0) {
                const float4* st = reinterpret_cast<const float4*>(base + t_off);
                tx = t < m.z ? st[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (m.x >= 0) {
            const float4* sx = reinterpret_cast<const float4*>(base + NP * kPart * a.rb_count);
            if (act) {
                unsigned char* b0 = base + b_off;
                if (sp == 8) g_tile<KERN, 8, NP>(sx, tx, t, h, T, b0, b_half, a.k);
                else if (sp == 4) g_tile<KERN, 4, NP>(sx, tx, t, h, T, b0, b_half, a.k);
                else if (sp == 2) g_tile<KERN, 2, NP>(sx, tx, t, h, T, b0, b_half, a.k);
                else g_tile<KERN, 1, NP>(sx, tx, t, h, T, b0, b_half, a.k);
            }
            fence_async_smem();
        }
        mbar_arrive(&sm.full_b[idx]);
        r.advance(a.slots);
    }
}

// ---- MMA issuer of a set (one thread) ----
template <bool LIMITED, int NP>
__device__ void run_mma(const TcArgs& a, const TcSmem& sm, uint32_t tmem, int set) {
    volatile int* abort = sm.abort;
    const uint32_t wlim = LIMITED ? a.wait_limit : kWaitLimit;
    const int b_off = slot_b_off(a.rb_count, a.tg, NP), b_half = slot_b_half(a.tg);
    const int meta_off = slot_meta_off(a.rb_count, a.tg, NP);
    const uint32_t acc_cols = (uint32_t)(a.rb_count * 2 * a.tg), bufcols = 512u / (uint32_t)a.nbuf;
    // The issuing thread is on every stage's critical path: per stage it only adds the slot's offset to
    // descriptors and accumulator addresses prepared here (a descriptor's start address is its low 14 bits, in
    // 16-byte units, and shared memory stays below 2^18 bytes, so the sum never carries out of the field).
    const uint32_t set_base = smem_u32(sm.slots + (size_t)set * a.slots * a.slot_bytes);
    const uint64_t da_set = smem_desc(set_base), db_set = smem_desc(set_base + (uint32_t)b_off);
    const uint32_t d_set = tmem + (uint32_t)set * acc_cols;
    Ring r{0, 0u}, ab{0, 0u};  // pipeline slot; accumulator buffer of the current unit
    bool acc_started = false, issued = false;
    while (true) {
        const int idx = set * a.slots + r.slot;
        unsigned char* base = sm.slots + (size_t)idx * a.slot_bytes;
        if (!mbar_wait(&sm.full[idx], r.phase, abort, wlim)) {
            if (!*abort) set_abort(a, sm);
            break;
        }
        const int4 m = *reinterpret_cast<const int4*>(base + meta_off);
        if (m.y & kDone) break;
        const uint32_t ub = (uint32_t)ab.slot;
        if (m.y & kFirst) {
            // the epilogue has released this accumulator buffer (unit - nbuf)
            if (!mbar_wait(&sm.acc_empty[ub], ab.phase ^ 1u, abort, wlim)) {
                if (!*abort) set_abort(a, sm);
                break;
            }
            acc_started = false;
        }
        if (!mbar_wait(&sm.full_b[idx], r.phase, abort, wlim)) {
            if (!*abort) set_abort(a, sm);
            break;
        }
        tc_fence_after();
        if (m.x >= 0) {
            const int T = (m.z + 7) & ~7;
            const uint32_t idesc = idesc_bf16_f32(2 * T);
            // descriptors address 16-byte units: part p of an operand is p * bytes-per-part / 16 further
            const uint64_t slot16 = (uint64_t)(((uint32_t)r.slot * (uint32_t)a.slot_bytes) >> 4);
            const uint64_t db0 = db_set + slot16;
            const uint64_t db_step = (uint64_t)(b_half >> 4);
            const uint32_t d0 = d_set + ub * bufcols;
            for (int rb = 0; rb < a.rb_count; ++rb) {
                const uint64_t da0 = da_set + slot16 + (uint64_t)((rb * NP * kPart) >> 4);
                const uint64_t da_step = (uint64_t)(kPart >> 4);
                const uint32_t d = d0 + (uint32_t)(rb * 2 * a.tg);
                // every product of parts p (of lambda) and q (of G) with p + q < NP: 3 MMAs for hi / lo,
                // 6 for hi / mid / lo (the dropped products are below 2^-8 NP of the leading one)
                mma_bf16(d, da0, db0, idesc, acc_started ? 1u : 0u);
                mma_bf16(d, da0, db0 + db_step, idesc, 1u);
                mma_bf16(d, da0 + da_step, db0, idesc, 1u);
                if constexpr (NP == 3) {
                    mma_bf16(d, da0, db0 + 2 * db_step, idesc, 1u);
                    mma_bf16(d, da0 + da_step, db0 + db_step, idesc, 1u);
                    mma_bf16(d, da0 + 2 * da_step, db0, idesc, 1u);
                }
            }
            acc_started = true;
        }
        mma_commit(&sm.empty[idx]);
        issued = true;
        if (m.y & kLast) {
            mma_commit(&sm.acc_full[ub]);
            ab.advance(a.nbuf);
        }
        r.advance(a.slots);
    }
    if (*abort && issued) {
        // the latest commit arrives once every MMA issued before it has completed
        if (--r.slot < 0) {
            r.slot += a.slots;
            r.phase ^= 1u;
        }
        mbar_wait(&sm.empty[set * a.slots + r.slot], r.phase, nullptr, kDrainLimit);
    }
}

// ---- epilogue (128 threads, TMEM lanes by warp quadrant) ----
template <bool LIMITED>
__device__ void run_epilogue(const TcArgs& a, const TcSmem& sm, uint32_t tmem, int64_t units, int warp, int lane) {
    volatile int* abort = sm.abort;
    const uint32_t wlim = LIMITED ? a.wait_limit : kWaitLimit;
    const int q = warp & 3;
    const int m = q * 32 + lane;  // accumulator row
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    const uint32_t acc_cols = (uint32_t)(a.rb_count * 2 * a.tg);
    const uint32_t bufcols = 512u / (uint32_t)a.nbuf;
    Ring eb{0, 0u};  // accumulator buffer of the next unit
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        int b, t0, nt;
        unit_of(a, u, b, t0, nt);
        // a box without any source group (two point sets, no source nearby) has no stages and no accumulator:
        // the producer skips it too, and its results stay at the zeros written before the launch
        if (nt == 0 || a.gcount[b] == 0) continue;
        // sets with work in this unit: entries 0 .. gcount - 1 of the list go to sets 0, 1, 2, 3, 0, ...
        const int used = min(kSets, a.gcount[b]);
        const int T = (nt + 7) & ~7;
        const int tb = a.box_ptr[b] + t0;
        const uint32_t ub = (uint32_t)eb.slot, par = eb.phase;
        eb.advance(a.nbuf);
        const bool ok = mbar_wait(&sm.acc_full[ub], par, abort, wlim);
        // the 128 threads leave together (they meet at named barriers below)
        if (epi_any(!ok)) {
            if (!ok && !*abort) set_abort(a, sm);
            return;
        }
        tc_fence_after();
        for (int rb = 0; rb < a.rb_count; ++rb) {
            const int r = rb * 64 + (m & 63);
            for (int c0 = 0; c0 < T; c0 += 8) {
                __syncwarp();
                int prow[8];
                if (m < 64) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) prow[j] = c0 + j < nt ? a.perm[tb + c0 + j] : 0;
                }
                const uint32_t col = lane_addr + ub * bufcols + (uint32_t)(rb * 2 * a.tg + c0);
                float x[8], y[8];
                tmem_ld8(col, x);
                tmem_ld8(col + (uint32_t)T, y);
                for (int s = 1; s < used; ++s) {
                    float x1[8], y1[8];
                    tmem_ld8(col + (uint32_t)s * acc_cols, x1);
                    tmem_ld8(col + (uint32_t)s * acc_cols + (uint32_t)T, y1);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        x[j] += x1[j];
                        y[j] += y1[j];
                    }
                }
                // rows 64..127 (Im lambda) hand (-D[., T + t], D[., t]) to rows 0..63
                if (m >= 64) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) sm.epi[j * 64 + (m - 64)] = make_float2(-y[j], x[j]);
                }
                epi_sync();
                if (m < 64 && r < a.nrhs) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (c0 + j < nt) {
                            const float2 w = sm.epi[j * 64 + m];
                            a.out[(int64_t)prow[j] * a.ld + r] =
                                make_float2((x[j] + w.x) * kInv4Pi, (y[j] + w.y) * kInv4Pi);
                        }
                    }
                }
                epi_sync();
            }
        }
        tc_fence_before();
        mbar_arrive(&sm.acc_empty[ub]);
    }
}

// LIMITED: the waits poll at most a.wait_limit times (the abort-path self-check); otherwise kWaitLimit.
// NP: BF16 parts per operand (2: three MMAs per stage, 3: six).
template <int KERN, bool LIMITED, int NP>
__global__ void __launch_bounds__(kThreads, 1) k_p2p_tc(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const TcSmem sm = carve(smem, a.slots, a.slot_bytes);
    if (warp == 0) tmem_alloc(sm.tmem_slot, 512u);
    if (tid == 32) {
        for (int i = 0; i < kSets * a.slots; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.full_b[i], kSetThreads);
            mbar_init(&sm.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.acc_full[i], kSets);
            mbar_init(&sm.acc_empty[i], 128);
        }
        *sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_slot;
    const int64_t units = (int64_t)a.nb * a.ngrp;
    if (warp < kGWarp0) {
        run_producer<LIMITED>(a, sm, units, warp, lane);
    } else if (warp < kMmaWarp0) {
        const int gw = warp - kGWarp0;
        run_gset<KERN, LIMITED, NP>(a, sm, gw / kSetWarps, (gw % kSetWarps) * 32 + lane);
    } else if (warp < kEpiWarp0) {
        if (lane == 0) run_mma<LIMITED, NP>(a, sm, tmem, warp - kMmaWarp0);
    } else {
        run_epilogue<LIMITED>(a, sm, tmem, units, warp, lane);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 512u);
    }
}

// ------------------------------------------------- operand-layout self-check --

// D[128 x N] = A[128 x K] . B[N x K]^T with A, B split into BF16 hi + lo (3 MMAs
// per 16-wide K slice), through the same operand layout, descriptors and
// instruction descriptor as k_p2p_tc.
__global__ void __launch_bounds__(128, 1) k_tc_gemm_check(const float* __restrict__ A, const float* __restrict__ B,
                                                          float* __restrict__ D, int K, int n, int tmem_cols,
                                                          unsigned int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* a_hi = smem;
    unsigned char* a_lo = a_hi + kImage / 2;
    unsigned char* b_hi = smem + kImage;
    unsigned char* b_lo = b_hi + (n / 8) * kSbo;
    uint64_t* bar = reinterpret_cast<uint64_t*>(b_lo + (n / 8) * kSbo);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    if (warp == 0) tmem_alloc(slot, (uint32_t)tmem_cols);
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t idesc = idesc_bf16_f32(n);
    bool ok = true;
    for (int ks = 0; ks < K / kSrcGroup && ok; ++ks) {
        for (int c = tid; c < 128 * 2; c += 128) {
            const int row = c >> 1, half = c & 1;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = A[(int64_t)row * K + ks * 16 + half * 8 + i];
            store_split<8>(a_hi, a_lo, op_off(row, half * 8), v);
        }
        for (int c = tid; c < n * 2; c += 128) {
            const int row = c >> 1, half = c & 1;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = B[(int64_t)row * K + ks * 16 + half * 8 + i];
            store_split<8>(b_hi, b_lo, op_off(row, half * 8), v);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            mma_bf16(tmem, smem_desc(smem_u32(a_hi)), smem_desc(smem_u32(b_hi)), idesc, ks == 0 ? 0u : 1u);
            mma_bf16(tmem, smem_desc(smem_u32(a_hi)), smem_desc(smem_u32(b_lo)), idesc, 1u);
            mma_bf16(tmem, smem_desc(smem_u32(a_lo)), smem_desc(smem_u32(b_hi)), idesc, 1u);
            mma_commit(bar);
        }
        // the operands are rewritten next slice: wait for these MMAs
        bool done = true;
        if (tid == 0) done = mbar_wait(bar, (uint32_t)(ks & 1), nullptr);
        ok = __syncthreads_and(done);
        tc_fence_after();
    }
    if (ok) {
        tc_fence_after();
        for (int c0 = 0; c0 < n; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(int64_t)(warp * 32 + lane) * n + c0 + i] = v[i];
        }
    } else if (tid == 0) {
        atomicOr(status, P2P_DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)tmem_cols);
    }
}

int tmem_cols_for(int n) {
    int c = 32;
    while (c < n) c <<= 1;
    return c;
}

// Launch shape for nrhs right-hand sides: RHS blocks, targets per unit, slots per set.
struct TcShape {
    int rb_count, tg, slots, slot_bytes, smem;
};

TcShape tc_shape(int32_t nrhs, int optin, int np) {
    TcShape s;
    s.rb_count = (nrhs + 63) / 64;
    // One accumulator per G set (rb_count blocks x 2T columns) in each unit buffer.  The hi/lo split keeps two
    // buffers of 32-target units, so the epilogue of one unit overlaps the MMAs of the next.  The three-part
    // split takes 64-target units in one buffer (all 512 columns): a box of 33 - 64 targets is one unit instead
    // of two walking the same list, and its six MMAs per stage leave the epilogue's wait a smaller share (the
    // ellipsoid at 64 RHS: 7.14 ms against 7.64; hi/lo with the same shape 5.46 against 5.11).
    const int units_in_tmem = np == 3 ? 1 : 2;
    s.tg = (2 * kSetCols / (units_in_tmem * 2 * kSets * s.rb_count)) / 8 * 8;
    if (s.tg > 64) s.tg = 64;
    s.slot_bytes = slot_bytes_for(s.rb_count, s.tg, np);
    s.slots = 8;
    while (s.slots > 1 && tc_smem_bytes(s.slots, s.slot_bytes) > optin) --s.slots;
    s.smem = tc_smem_bytes(s.slots, s.slot_bytes);
    // more than half an SM's shared memory keeps one CTA (and one 512-column TMEM allocation) per SM
    const int half = 116 * 1024;
    if (s.smem < half) s.smem = half;
    return s;
}

}  // namespace

// RHS blocks of 64 per launch.  One block per launch keeps units of 32 targets
// (the TMEM accumulators of four G sets x two unit buffers hold 2 T x 64 RHS
// each); a launch over two blocks must halve the unit to 16 targets and measured
// 15.4 ms on the 2^21-point ellipsoid at 128 RHS against 2 x 5.2 ms for two
// launches of one block (G is formed once per launch: its share is small).
constexpr int kRbLaunch = 1;

// Room for the records of either split (sized for three parts), chunk by chunk.
size_t p2p_tc_pack_bytes(int64_t n, int32_t nb, int32_t max_nrhs) {
    if (max_nrhs < 16) return 0;
    const int64_t groups = n / kSrcGroup + nb;
    const int chunks = (max_nrhs + 64 * kRbLaunch - 1) / (64 * kRbLaunch);
    return (size_t)chunks * (size_t)groups * (size_t)record_bytes(kRbLaunch, 3);
}

bool p2p_tc_supported(const p2p_plan* plan, int32_t nrhs) {
    if (!plan || !plan->tc_pack || nrhs < 1 || nrhs > 256 || nrhs > plan->max_nrhs) return false;
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return false;
    return major == 10 && minor == 3;
}

// Stage: the group records (strength images from original-order lambda via perm, coordinates).
p2p_status p2p_tc_stage(const p2p_plan* plan, const float2* lam, int32_t nrhs, int64_t ld, int np,
                        cudaStream_t s) {
    if (plan->n == 0 || plan->tc_groups == 0) return P2P_OK;
    const int rb_count = (nrhs + 63) / 64;
    dim3 grid((unsigned)plan->tc_groups, (unsigned)rb_count);
    const int64_t chunk_bytes = (int64_t)plan->tc_groups * record_bytes(kRbLaunch, np);
    // the group records are built over the SOURCE boxes
    auto pack = np == 3 ? k_tc_pack<3> : k_tc_pack<2>;
    pack<<<grid, 128, 0, s>>>(lam, ld, nrhs, plan->src_perm, plan->src_box_ptr, plan->xs_src, plan->tc_gstart,
                              plan->nbs, kRbLaunch, chunk_bytes, plan->tc_pack);
    P2P_CHECK_LAUNCH("p2p_apply_stage/tc_pack");
    return P2P_OK;
}

p2p_status p2p_apply_tc(const p2p_plan* plan, float2* out, int32_t nrhs, int64_t ld, int32_t adjoint, int np,
                        cudaStream_t s) {
    if (plan->n == 0) return P2P_OK;
    int dev = 0, optin = 0, sms = 0;
    P2P_TRY_CUDA(cudaGetDevice(&dev), "p2p_apply_tc");
    P2P_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "p2p_apply_tc");
    P2P_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "p2p_apply_tc");
    // one launch per chunk of kRbLaunch RHS blocks, each on its own records
    const int chunk_rhs = 64 * kRbLaunch;
    const TcShape sh = tc_shape(std::min(nrhs, chunk_rhs), optin, np);
    if (sh.smem > optin) {
        set_message("p2p_apply_tc: the tensor-core pipeline does not fit in shared memory");
        return P2P_ERR_UNSUPPORTED;
    }
    TcArgs a;
    a.xs = plan->xs;
    a.pack = plan->tc_pack;
    a.box_ptr = plan->box_ptr;
    a.glist_off = plan->tc_glist_off;
    a.glist = plan->tc_glist;
    a.gcount = plan->tc_gcount;
    a.perm = plan->perm;
    a.ld = ld;
    a.rb_count = sh.rb_count;
    a.tg = sh.tg;
    a.ngrp = (plan->max_box + sh.tg - 1) / sh.tg;
    a.nb = plan->nb;
    a.slots = sh.slots;
    a.slot_bytes = sh.slot_bytes;
    a.np = np;
    a.nbuf = 512 / (kSets * 2 * sh.tg * sh.rb_count);
    a.k = adjoint ? -plan->k : plan->k;
    a.status = plan->status;
    a.wait_limit = plan->tc_wait_polls < 0 ? kWaitLimit : (uint32_t)plan->tc_wait_polls;
    const bool limited = plan->tc_wait_polls >= 0;
    void (*kern)(TcArgs) = nullptr;
    const bool lap = plan->kernel == P2P_LAPLACE;
    if (np == 3) {
        kern = lap ? (limited ? k_p2p_tc<P2P_LAPLACE, true, 3> : k_p2p_tc<P2P_LAPLACE, false, 3>)
                   : (limited ? k_p2p_tc<P2P_HELMHOLTZ, true, 3> : k_p2p_tc<P2P_HELMHOLTZ, false, 3>);
    } else {
        kern = lap ? (limited ? k_p2p_tc<P2P_LAPLACE, true, 2> : k_p2p_tc<P2P_LAPLACE, false, 2>)
                   : (limited ? k_p2p_tc<P2P_HELMHOLTZ, true, 2> : k_p2p_tc<P2P_HELMHOLTZ, false, 2>);
    }
    P2P_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem), "p2p_apply_tc");
    const int64_t units = (int64_t)a.nb * a.ngrp;
    const int grid = (int)std::min<int64_t>(units, sms);
    const int64_t chunk_bytes = (int64_t)plan->tc_groups * record_bytes(kRbLaunch, np);
    for (int c = 0; c * chunk_rhs < nrhs; ++c) {
        a.pack = plan->tc_pack + c * chunk_bytes;
        a.out = out + (int64_t)c * chunk_rhs;
        a.nrhs = std::min(chunk_rhs, nrhs - c * chunk_rhs);
        kern<<<grid, kThreads, sh.smem, s>>>(a);
        P2P_CHECK_LAUNCH("p2p_apply_tc");
    }
    return P2P_OK;
}

extern "C" P2P_API p2p_status p2p_diag_tc_gemm(const float* A, const float* B, float* D, int32_t K, int32_t n,
                                               unsigned int* status, p2p_stream_t stream) {
    if (!A || !B || !D || !status || K < 16 || K % 16 != 0 || n < 16 || n > 256 || n % 16 != 0)
        return P2P_ERR_INVALID;
    const int smem = kImage + 2 * (n / 8) * kSbo + 64;
    P2P_TRY_CUDA(cudaFuncSetAttribute(k_tc_gemm_check, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                 "p2p_diag_tc_gemm");
    k_tc_gemm_check<<<1, 128, smem, (cudaStream_t)stream>>>(A, B, D, K, n, tmem_cols_for(n), status);
    P2P_CHECK_LAUNCH("p2p_diag_tc_gemm");
    return P2P_OK;
}

// Self-check of the tensor-core path's abort handling: every pipeline wait of the plan's later tensor-core
// launches polls at most `polls` times (negative: the normal bound).
extern "C" P2P_API p2p_status p2p_diag_tc_wait_limit(p2p_plan* plan, int32_t polls) {
    if (!plan) return P2P_ERR_INVALID;
    plan->tc_wait_polls = polls < 0 ? -1 : polls;
    return P2P_OK;
}
