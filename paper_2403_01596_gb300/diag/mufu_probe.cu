// Microbenchmark behind the roofline denominator: MUFU throughput of rsqrtf and
// __sincosf, and the bare Helmholtz / Laplace pair loop with sources in shared
// memory.  Standalone (not part of libp2p.so); build and run with
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -ftz=true -o probe mufu_probe.cu && ./probe
#include <cstdio>
#include <cuda_runtime.h>

__global__ void k_rsqrt(float* out, int iters) {
    float a0 = 1.f + threadIdx.x * 1e-3f, a1 = a0 + 0.5f, a2 = a0 + 0.25f, a3 = a0 + 0.125f;
    float c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    for (int i = 0; i < iters; ++i) {
        c0 += rsqrtf(a0); c1 += rsqrtf(a1); c2 += rsqrtf(a2); c3 += rsqrtf(a3);
        a0 += 1e-3f; a1 += 1e-3f; a2 += 1e-3f; a3 += 1e-3f;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + c2 + c3;
}

__global__ void k_sincos(float* out, int iters) {
    float a0 = 1.f + threadIdx.x * 1e-3f, a1 = a0 + 0.5f, a2 = a0 + 0.25f, a3 = a0 + 0.125f;
    float c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    for (int i = 0; i < iters; ++i) {
        float s, c;
        __sincosf(a0, &s, &c); c0 += s + c;
        __sincosf(a1, &s, &c); c1 += s + c;
        __sincosf(a2, &s, &c); c2 += s + c;
        __sincosf(a3, &s, &c); c3 += s + c;
        a0 += 1e-3f; a1 += 1e-3f; a2 += 1e-3f; a3 += 1e-3f;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + c2 + c3;
}

// One target per thread against 256 sources staged in shared memory (the
// inner loop of the pair kernel with one target per lane).
template <int VARIANT>
__global__ void k_pairs(float2* out, int reps, float k) {
    __shared__ float4 sx[256];
    __shared__ float2 sl[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        sx[i] = make_float4(0.01f * (i % 17), 0.013f * (i % 13), 0.007f * (i % 11), 0.f);
        sl[i] = make_float2(1.f + 0.001f * i, -0.5f + 0.002f * i);
    }
    __syncthreads();
    const float tx = 0.05f + 1e-4f * threadIdx.x, ty = 0.031f, tz = 0.077f;
    float ar = 0.f, ai = 0.f;
    for (int rep = 0; rep < reps; ++rep) {
        for (int s = 0; s < 256; ++s) {
            const float4 p = sx[s];
            const float2 l = sl[s];
            const float dx = p.x - tx, dy = p.y - ty, dz = p.z - tz;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float inv;
            if (VARIANT == 0) { inv = rsqrtf(r2); inv = r2 > 0.f ? inv : 0.f; }
            else { inv = rsqrtf(r2); }
            if (VARIANT == 2) {
                ar = fmaf(inv, l.x, ar);
                ai = fmaf(inv, l.y, ai);
            } else {
                float sn, cs;
                __sincosf(k * (r2 * inv), &sn, &cs);
                const float gr = cs * inv, gi = sn * inv;
                ar = fmaf(gr, l.x, fmaf(-gi, l.y, ar));
                ai = fmaf(gr, l.y, fmaf(gi, l.x, ai));
            }
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = make_float2(ar, ai);
}

int main() {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    const int blocks = sms * 8, threads = 256;
    float* out;
    float2* out2;
    cudaMalloc(&out, blocks * threads * sizeof(float));
    cudaMalloc(&out2, blocks * threads * sizeof(float2));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 4096;
    for (int w = 0; w < 2; ++w) {
        float ms;
        k_rsqrt<<<blocks, threads>>>(out, iters);
        cudaEventRecord(e0);
        k_rsqrt<<<blocks, threads>>>(out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        double ops = 4.0 * iters * blocks * threads;
        if (w) printf("rsqrt: %.3f ms, %.2f Gop/s, %.2f per SM per clk (at %d MHz attr)\n", ms, ops / ms / 1e6,
                      ops / (ms * 1e-3) / sms / (clk * 1e3), clk / 1000);
        k_sincos<<<blocks, threads>>>(out, iters);
        cudaEventRecord(e0);
        k_sincos<<<blocks, threads>>>(out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        ops = 4.0 * iters * blocks * threads;
        if (w) printf("sincos: %.3f ms, %.2f G sincos/s, %.2f sincos per SM per clk\n", ms, ops / ms / 1e6,
                      ops / (ms * 1e-3) / sms / (clk * 1e3));
        const int reps = 16;
        double pairs = 256.0 * reps * blocks * threads;
        k_pairs<0><<<blocks, threads>>>(out2, reps, 10.f);
        cudaEventRecord(e0);
        k_pairs<0><<<blocks, threads>>>(out2, reps, 10.f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (w) printf("pairs masked: %.3f ms, %.1f Gpair/s, %.3f pair per SM per clk\n", ms, pairs / ms / 1e6,
                      pairs / (ms * 1e-3) / sms / (clk * 1e3));
        k_pairs<1><<<blocks, threads>>>(out2, reps, 10.f);
        cudaEventRecord(e0);
        k_pairs<1><<<blocks, threads>>>(out2, reps, 10.f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (w) printf("pairs unmasked: %.3f ms, %.1f Gpair/s, %.3f pair per SM per clk\n", ms, pairs / ms / 1e6,
                      pairs / (ms * 1e-3) / sms / (clk * 1e3));
        k_pairs<2><<<blocks, threads>>>(out2, reps, 10.f);
        cudaEventRecord(e0);
        k_pairs<2><<<blocks, threads>>>(out2, reps, 10.f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (w) printf("pairs laplace: %.3f ms, %.1f Gpair/s, %.3f pair per SM per clk\n", ms, pairs / ms / 1e6,
                      pairs / (ms * 1e-3) / sms / (clk * 1e3));
    }
    cudaError_t e = cudaDeviceSynchronize();
    printf("status %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
