// bench_atomics.cu -- a standalone measurement of the atomic throughputs the backward and raster kernels
// depend on, for their atomic rooflines: global FP64 / FP32 reductions into an L2-resident array (the
// vertex-gradient flush), and shared-memory adds of FP32, int32, FP64 and u64 (the per-tile triangle table,
// the z-buffer) without and with address conflicts.  Not part of the library.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 paper_2405_02508_gb300/csrc/bench_atomics.cu -o bench_atomics
//   ./bench_atomics
#include <cstdio>

#include <cuda_runtime.h>

template <typename T>
__global__ void global_red(T* buf, unsigned mask, int iters) {
    unsigned h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    for (int it = 0; it < iters; ++it) {
        h = h * 1664525u + 1013904223u;
        atomicAdd(buf + (h & mask), (T)1);
    }
}

template <typename T>
__global__ void shared_add(T* out, int iters, int conflict) {
    __shared__ T s[512];
    for (int i = threadIdx.x; i < 512; i += blockDim.x) s[i] = (T)0;
    __syncthreads();
    unsigned h = threadIdx.x * 2654435761u + blockIdx.x;
    for (int it = 0; it < iters; ++it) {
        h = h * 1664525u + 1013904223u;
        const int slot = conflict ? (int)((h >> 20) & 7u) : (int)((h >> 20) & 511u);  // 8 or 512 targets
        atomicAdd(&s[slot], (T)1);
    }
    __syncthreads();
    if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

template <typename K>
static float time_ms(K launch) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return t;
}

int main() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned n = 1u << 21;  // 2M entries: 16 MB of doubles, resident in L2
    double* gd = nullptr;
    float* gf = nullptr;
    cudaMalloc(&gd, n * sizeof(double));
    cudaMalloc(&gf, n * sizeof(float));
    cudaMemset(gd, 0, n * sizeof(double));
    cudaMemset(gf, 0, n * sizeof(float));
    const int blocks = sms * 8, threads = 256, iters = 256;
    const double ops = (double)blocks * threads * iters;
    float t = time_ms([&] { global_red<double><<<blocks, threads>>>(gd, n - 1, iters); });
    printf("global RED.F64, random addresses in 16 MB: %.1f G/s\n", ops / t / 1e6);
    t = time_ms([&] { global_red<float><<<blocks, threads>>>(gf, n - 1, iters); });
    printf("global RED.F32, random addresses in 8 MB: %.1f G/s\n", ops / t / 1e6);
    void* out = nullptr;
    cudaMalloc(&out, (size_t)blocks * 8);
    const int siters = 1024;
    const double sops = (double)blocks * threads * siters;
    for (int conflict = 0; conflict < 2; ++conflict) {
        const float tf = time_ms([&] { shared_add<float><<<blocks, threads>>>((float*)out, siters, conflict); });
        const float ti = time_ms([&] { shared_add<int><<<blocks, threads>>>((int*)out, siters, conflict); });
        const float td = time_ms([&] { shared_add<double><<<blocks, threads>>>((double*)out, siters, conflict); });
        const float tu = time_ms([&] {
            shared_add<unsigned long long><<<blocks, threads>>>((unsigned long long*)out, siters, conflict);
        });
        printf("shared add, %s targets per CTA: f32 %.0f G/s, i32 %.0f G/s, f64 %.0f G/s, u64 %.0f G/s\n",
               conflict ? "8" : "512", sops / tf / 1e6, sops / ti / 1e6, sops / td / 1e6, sops / tu / 1e6);
    }
    const cudaError_t e = cudaGetLastError();
    printf("%s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
