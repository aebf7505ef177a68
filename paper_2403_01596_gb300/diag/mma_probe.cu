// tcgen05.mma throughput microbenchmark (kind::f16, BF16 operands, FP32 accumulation, M = 128, K = 16).
//
// One block per SM; `issuers` threads (lane 0 of warps 0 .. issuers-1) each issue `iters` MMAs of width N back
// to back into their own TMEM columns, then commit to an mbarrier and wait for it (bounded). B is in shared
// memory (zero-filled, the canonical K-major layout without swizzle that the multi-RHS kernel uses: 8-row x
// 16-byte core matrices, LBO 128 B, SBO 256 B); A is in shared memory the same way, or (second half of the
// run) in tensor memory. clock64 around the issue loop and the wait gives cycles per MMA per issuer for block 0.
// Operand bytes read from shared memory per MMA: 4 KB (A, when there) + N x 32 B (B).
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_at(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
                 ::"r"(d), "r"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(128, 1) k_bench(int n, int iters, int issuers, int a_tmem, long long* out, unsigned* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // A: 128 x 16 bf16 = 4 KB; B: 256 x 16 bf16 = 8 KB (max N)
    unsigned char* A = smem;
    unsigned char* Bm = smem + 4096;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 4096 + 8192);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 4);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (4096 + 8192) / 4; i += 128) reinterpret_cast<uint32_t*>(smem)[i] = 0u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(512u) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    if ((tid & 31) == 0 && warp < issuers) {
        const uint64_t da = smem_desc(smem_u32(A)), db = smem_desc(smem_u32(Bm));
        const uint32_t id = idesc(n);
        const uint32_t d = tmem + (uint32_t)(warp * ((a_tmem ? 256 : 512) / issuers));  // disjoint columns per issuer
        const uint32_t at = tmem + 256u + (uint32_t)(warp * 16);                       // A operand columns (TMEM mode)
        long long t0 = clock64();
        if (a_tmem) {
            for (int i = 0; i < iters; ++i) mma_at(d, at, db, id, i > 0 ? 1u : 0u);
        } else {
            for (int i = 0; i < iters; ++i) mma(d, da, db, id, i > 0 ? 1u : 0u);
        }
        long long t1 = clock64();
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar[warp])) : "memory");
        bool ok = mbar_wait(&bar[warp], 0);
        long long t2 = clock64();
        if (!ok) atomicOr(status, 1u);
        if (blockIdx.x == 0) {
            out[warp * 2 + 0] = t1 - t0;
            out[warp * 2 + 1] = t2 - t0;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

int main() {
    long long* out; unsigned* status;
    cudaMalloc(&out, 64 * sizeof(long long));
    cudaMalloc(&status, 4);
    cudaMemset(status, 0, 4);
    const int smem = 4096 + 8192 + 64;
    cudaFuncSetAttribute(k_bench, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int iters = 256;
    int ns[] = {32, 64, 128, 256};
    for (int a_tmem : {0, 1})
    for (int issuers : {1, 2, 4}) {
        for (int n : ns) {
            const int cols = a_tmem ? 256 : 512;
            if (n > cols / issuers) continue;
            for (int rep = 0; rep < 2; ++rep) {
                cudaMemset(out, 0, 64 * sizeof(long long));
                k_bench<<<sms, 128, smem>>>(n, iters, issuers, a_tmem, out, status);
                cudaError_t e = cudaDeviceSynchronize();
                if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return 1; }
                long long h[8]; unsigned st;
                cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
                cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost);
                if (rep == 1) {
                    printf("A in %s issuers %d N %3d: per-MMA issue", a_tmem ? "TMEM" : "smem", issuers, n);
                    for (int w = 0; w < issuers; ++w) printf(" %.1f", (double)h[2 * w] / iters);
                    printf(" | issue+complete per MMA");
                    for (int w = 0; w < issuers; ++w) printf(" %.1f", (double)h[2 * w + 1] / iters);
                    printf(" | status %u\n", st);
                }
            }
        }
    }
    return 0;
}
