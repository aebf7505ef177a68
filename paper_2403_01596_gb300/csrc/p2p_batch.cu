// Persistent batched P2P over several independent geometries (plans).
//
// One batched apply is two kernel launches, both safe to capture in a CUDA
// graph (no allocation, no host synchronisation, every pointer passed by
// value):
//   k_batch_stage   one block row per geometry: writes the geometry's output
//                   pointer into the device geometry table, gathers its
//                   strengths into its plan's staging buffer (sorted or packed
//                   rows) and zeroes its outputs when they are accumulated with
//                   atomics;
//   k_pair_batched  a persistent grid (resident blocks x SMs) whose warps take
//                   work items (geometry, box, source chunk) from one combined
//                   list, warp w taking items w, w + W, ... (W warps).  The list
//                   is the plans' own item lists (each heaviest first) one after
//                   the other in the order the plans were given, so the warps work
//                   on one geometry's data at a time and the last geometry's light
//                   items fill the tail (measured 4 % faster on eight geometries
//                   than one list ordered by cost across all of them, which mixes
//                   every geometry's data in flight).  Warps never wait on each
//                   other.
// The per-item work is the same device code as the per-plan pair kernel.
#include <string.h>

#include <algorithm>

#include "p2p_pair.cuh"

using namespace p2p_detail;
using namespace p2p_pair;

namespace {

constexpr int kMaxBatch = 16;

struct BatchGeom {
    PairArgs a;
    int64_t n;
    int64_t nrows;         // staged rows (points or packed entries)
    const int32_t* rows;   // original index of every staged row (-1: padding)
};

struct BatchIO {
    const float2* lam[kMaxBatch];
    float2* out[kMaxBatch];
    int64_t row_off[kMaxBatch + 1];  // prefix over geometries of staged rows * nrhs
    int64_t out_off[kMaxBatch + 1];  // prefix over atomic geometries of n * nrhs (0 for the others)
    int32_t count;
    int32_t nrhs;
    int64_t ld;
};

struct ItemOffsets {
    int64_t off[kMaxBatch + 1];
    int32_t count;
};

__device__ __forceinline__ int find_geom(const int64_t* off, int count, int64_t i) {
    int g = 0;
    while (g + 1 < count && off[g + 1] <= i) ++g;
    return g;
}

// Block row blockIdx.y stages geometry blockIdx.y: its output pointer into the
// geometry table, its strengths into the plan's staging buffer, and zeros for
// its outputs when they are accumulated with atomics.
__global__ void k_batch_stage(BatchGeom* __restrict__ geoms, const BatchIO io) {
    const int g = blockIdx.y;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        geoms[g].a.out = io.out[g];
        geoms[g].a.ld = io.ld;
        geoms[g].a.nrhs = io.nrhs;
    }
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int32_t* __restrict__ rows = geoms[g].rows;
    float2* __restrict__ dst = const_cast<float2*>(geoms[g].a.lam);
    const float2* __restrict__ src = io.lam[g];
    const int64_t n_el = io.row_off[g + 1] - io.row_off[g];
    for (int64_t i = tid; i < n_el; i += stride) {
        const int64_t s = i / io.nrhs;
        const int q = (int)(i - s * io.nrhs);
        const int32_t r = rows[s];
        dst[i] = r >= 0 ? src[(int64_t)r * io.ld + q] : make_float2(0.f, 0.f);
    }
    const int64_t n_out = io.out_off[g + 1] - io.out_off[g];
    float2* __restrict__ out = io.out[g];
    for (int64_t i = tid; i < n_out; i += stride) {
        const int64_t row = i / io.nrhs;
        const int q = (int)(i - row * io.nrhs);
        out[row * io.ld + q] = make_float2(0.f, 0.f);
    }
}

template <int R>
__global__ void __launch_bounds__(P2P_PAIR_MAX_THREADS, R == 1 ? P2P_PAIR_MIN_BLOCKS : 1)
    k_pair_batched(const BatchGeom* __restrict__ geoms, const ItemRec* __restrict__ recs, int64_t total, int chunk_max,
                   int sym_any) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    unsigned char* ws = smem_raw + (size_t)warp * warp_smem_bytes(chunk_max, R, sym_any != 0);
    run_pipeline<R>(ws, chunk_max, sym_any != 0, lane, recs, total, (int64_t)blockIdx.x * warps + warp, (int64_t)gridDim.x * warps,
                    geoms[0].a.status, [&](const ItemRec& r) -> const PairArgs* { return &geoms[r.b].a; });
}

// Combined item list: plan after plan, each in its own (heaviest first) order; the
// record's last field names its geometry.
__global__ void k_batch_order(const BatchGeom* __restrict__ geoms, const ItemOffsets off, ItemRec* __restrict__ recs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= off.off[off.count]) return;
    const int g = find_geom(off.off, off.count, i);
    ItemRec r = geoms[g].a.items[i - off.off[g]];
    r.b = g;
    recs[i] = r;
}

struct BatchLayout {
    BatchGeom* geoms;
    ItemRec* order;
    size_t bytes;
};

BatchLayout batch_layout(int64_t total, void* ws) {
    Carver c{static_cast<char*>(ws), 0, (size_t)-1};
    BatchLayout L;
    size_t m = (size_t)(total > 0 ? total : 1);
    L.geoms = c.take<BatchGeom>(kMaxBatch);
    L.order = c.take<ItemRec>(m);
    L.bytes = align_up(c.off, 256);
    return L;
}

// warp_bytes: per-warp shared memory.  The kernel's dynamic shared-memory
// limit is raised once to the device's opt-in maximum (the attribute is shared
// by every batch).
template <int R>
cudaError_t configure(int warps, int warp_bytes, int* ctas_per_sm) {
    const int smem = warps * warp_bytes;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_pair_batched<R>);
    if (e != cudaSuccess) return e;
    if (smem > optin || warps * 32 > fa.maxThreadsPerBlock) {
        *ctas_per_sm = 0;
        return cudaSuccess;
    }
    e = cudaFuncSetAttribute(k_pair_batched<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_pair_batched<R>, warps * 32, smem);
}

}  // namespace

struct p2p_batch {
    int32_t count;
    int32_t nrhs;
    int32_t R;
    int32_t warps;
    int32_t warp_bytes;
    int32_t chunk_max;
    int32_t sym_any;        // some geometry uses the symmetric layout (per-warp source accumulator)
    int32_t grid;
    int64_t total;
    const p2p_plan* plans[kMaxBatch];
    BatchLayout L;
    BatchIO io;  // row/output prefixes (pointers filled per apply)
    cudaStream_t capture_stream;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

static p2p_status check_plans(const p2p_plan* const* plans, int32_t count, int32_t nrhs, int64_t* total) {
    if (!plans || count < 1 || count > kMaxBatch || nrhs < 1 || nrhs > 256) return P2P_ERR_INVALID;
    int64_t t = 0;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || plans[i]->n == 0 || nrhs > plans[i]->max_nrhs) return P2P_ERR_INVALID;
        t += plans[i]->n_items;
    }
    if (t >= INT32_MAX) return P2P_ERR_UNSUPPORTED;
    *total = t;
    return P2P_OK;
}

static p2p_status batch_launch(const p2p_batch* b, const void* const* lambdas, void* const* outs, int64_t ld,
                               cudaStream_t s) {
    BatchIO io = b->io;
    for (int g = 0; g < b->count; ++g) {
        if (!lambdas[g] || !outs[g] || ((uintptr_t)lambdas[g] & 7) || ((uintptr_t)outs[g] & 7))
            return P2P_ERR_INVALID;
        io.lam[g] = static_cast<const float2*>(lambdas[g]);
        io.out[g] = static_cast<float2*>(outs[g]);
    }
    io.ld = ld;
    int64_t most = 0;
    for (int g = 0; g < b->count; ++g) {
        most = std::max(most, io.row_off[g + 1] - io.row_off[g]);
        most = std::max(most, io.out_off[g + 1] - io.out_off[g]);
    }
    const int threads = 256;
    int64_t blocks = (most + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_batch_stage<<<dim3((unsigned)blocks, (unsigned)b->count), threads, 0, s>>>(b->L.geoms, io);
    P2P_CHECK_LAUNCH("p2p_batch_apply/stage");
    const int smem = b->warps * b->warp_bytes;
    if (b->R == 1)
        k_pair_batched<1><<<b->grid, b->warps * 32, smem, s>>>(b->L.geoms, b->L.order, b->total, b->chunk_max, b->sym_any);
    else if (b->R == 2)
        k_pair_batched<2><<<b->grid, b->warps * 32, smem, s>>>(b->L.geoms, b->L.order, b->total, b->chunk_max, b->sym_any);
    else
        k_pair_batched<4><<<b->grid, b->warps * 32, smem, s>>>(b->L.geoms, b->L.order, b->total, b->chunk_max, b->sym_any);
    P2P_CHECK_LAUNCH("p2p_batch_apply/pair");
    return P2P_OK;
}

extern "C" {

P2P_API p2p_status p2p_batch_workspace_size(const p2p_plan* const* plans, int32_t count, int32_t nrhs,
                                            size_t* bytes) {
    int64_t total = 0;
    if (!bytes) return P2P_ERR_INVALID;
    p2p_status st = check_plans(plans, count, nrhs, &total);
    if (st != P2P_OK) return st;
    *bytes = batch_layout(total, nullptr).bytes;
    return P2P_OK;
}

P2P_API p2p_status p2p_batch_create(p2p_batch** batch, const p2p_plan* const* plans, int32_t count, int32_t nrhs,
                                    int32_t warps_per_cta, void* workspace, size_t workspace_bytes,
                                    p2p_stream_t stream) {
    if (!batch) return P2P_ERR_INVALID;
    *batch = nullptr;
    int64_t total = 0;
    p2p_status st = check_plans(plans, count, nrhs, &total);
    if (st != P2P_OK) return st;
    if (warps_per_cta == 0) warps_per_cta = 8;
    if (warps_per_cta < 1 || warps_per_cta > 16) return P2P_ERR_INVALID;
    if (!workspace || ((uintptr_t)workspace & 255)) return P2P_ERR_INVALID;
    BatchLayout L = batch_layout(total, workspace);
    if (workspace_bytes < L.bytes) return P2P_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    p2p_batch* b = (p2p_batch*)calloc(1, sizeof(p2p_batch));
    if (!b) return P2P_ERR_ALLOC;
    b->count = count;
    b->nrhs = nrhs;
    b->R = nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1);
    b->warps = warps_per_cta;
    b->total = total;
    b->L = L;
    int max_chunk = 32;
    BatchGeom host[kMaxBatch];
    ItemOffsets off;
    memset(&off, 0, sizeof(off));
    memset(&b->io, 0, sizeof(b->io));
    off.count = count;
    b->io.count = count;
    b->io.nrhs = nrhs;
    for (int g = 0; g < count; ++g) {
        const p2p_plan* p = plans[g];
        b->plans[g] = p;
        host[g].a = base_args(p);
        host[g].a.nrhs = nrhs;
        host[g].n = p->n;
        host[g].nrows = host[g].a.red ? p->packed : p->n_src;   // staged strengths live on the sources
        host[g].rows = host[g].a.red ? p->pk_src : p->src_perm;
        max_chunk = std::max(max_chunk, p->tune.chunk);
        if (host[g].a.sym) b->sym_any = 1;
        off.off[g + 1] = off.off[g] + p->n_items;
        b->io.row_off[g + 1] = b->io.row_off[g] + host[g].nrows * nrhs;
        // outputs accumulated with atomics, and two-set plans (targets without nearby sources get no item),
        // are zeroed by the staging kernel
        b->io.out_off[g + 1] = b->io.out_off[g] + ((host[g].a.atomic_out || p->two_sets) ? p->n * nrhs : 0);
    }
    b->chunk_max = max_chunk;
    b->warp_bytes = warp_smem_bytes(max_chunk, b->R, b->sym_any != 0);
#define FAIL(expr, where)                 \
    do {                                  \
        cudaError_t e_ = (expr);          \
        if (e_ != cudaSuccess) {          \
            set_cuda_error(e_, where);    \
            free(b);                      \
            return P2P_ERR_CUDA;          \
        }                                 \
    } while (0)
    int ctas_per_sm = 0, dev = 0, sms = 0;
    // the requested warps per block, halved until one block's shared memory fits
    for (; b->warps >= 1; b->warps >>= 1) {
        cudaError_t e = b->R == 1 ? configure<1>(b->warps, b->warp_bytes, &ctas_per_sm)
                      : b->R == 2 ? configure<2>(b->warps, b->warp_bytes, &ctas_per_sm)
                                  : configure<4>(b->warps, b->warp_bytes, &ctas_per_sm);
        FAIL(e, "p2p_batch_create/occupancy");
        if (ctas_per_sm > 0) break;
    }
    FAIL(cudaGetDevice(&dev), "p2p_batch_create");
    FAIL(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "p2p_batch_create");
    if (ctas_per_sm < 1) {
        free(b);
        return P2P_ERR_UNSUPPORTED;
    }
    b->grid = ctas_per_sm * sms;
    FAIL(cudaMemcpyAsync(L.geoms, host, sizeof(BatchGeom) * count, cudaMemcpyHostToDevice, s), "p2p_batch_create");
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (blocks) {
        k_batch_order<<<blocks, 256, 0, s>>>(L.geoms, off, L.order);
        FAIL(cudaGetLastError(), "p2p_batch_create/order");
    }
    FAIL(cudaStreamSynchronize(s), "p2p_batch_create");
#undef FAIL
    *batch = b;
    return P2P_OK;
}

P2P_API p2p_status p2p_batch_apply(const p2p_batch* batch, const void* const* lambdas, void* const* outs, int64_t ld,
                                   p2p_stream_t stream) {
    if (!batch || !lambdas || !outs || ld < batch->nrhs) return P2P_ERR_INVALID;
    return batch_launch(batch, lambdas, outs, ld, (cudaStream_t)stream);
}

P2P_API p2p_status p2p_batch_graph_create(p2p_batch* batch, const void* const* lambdas, void* const* outs,
                                          int64_t ld) {
    if (!batch || !lambdas || !outs || ld < batch->nrhs) return P2P_ERR_INVALID;
    if (batch->exec) return P2P_ERR_INVALID;
    cudaStream_t cs = nullptr;
    P2P_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "p2p_batch_graph_create");
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        set_cuda_error(e, "p2p_batch_graph_create/begin");
        return P2P_ERR_CUDA;
    }
    p2p_status st = batch_launch(batch, lambdas, outs, ld, cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (st != P2P_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (st != P2P_OK) return st;
        set_cuda_error(e, "p2p_batch_graph_create/end");
        return P2P_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        set_cuda_error(e, "p2p_batch_graph_create/instantiate");
        return P2P_ERR_CUDA;
    }
    batch->capture_stream = cs;
    batch->graph = graph;
    batch->exec = exec;
    return P2P_OK;
}

P2P_API p2p_status p2p_batch_graph_launch(const p2p_batch* batch, p2p_stream_t stream) {
    if (!batch || !batch->exec) return P2P_ERR_INVALID;
    P2P_TRY_CUDA(cudaGraphLaunch(batch->exec, (cudaStream_t)stream), "p2p_batch_graph_launch");
    return P2P_OK;
}

P2P_API p2p_status p2p_batch_info(const p2p_batch* batch, int64_t* work_items, int32_t* grid, int32_t* warps_per_cta) {
    if (!batch) return P2P_ERR_INVALID;
    if (work_items) *work_items = batch->total;
    if (grid) *grid = batch->grid;
    if (warps_per_cta) *warps_per_cta = batch->warps;
    return P2P_OK;
}

P2P_API p2p_status p2p_batch_destroy(p2p_batch* batch) {
    if (!batch) return P2P_OK;
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    if (batch->capture_stream) cudaStreamDestroy(batch->capture_stream);
    free(batch);
    return P2P_OK;
}

}  // extern "C"
