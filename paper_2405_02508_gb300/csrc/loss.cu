// loss.cu -- the L2 image loss of inverse-rendering loops and its gradient in one pass:
// grad = 2 (image - target), *loss += sum (image - target)^2 (FP64).  Grid-stride over float4 groups
// when the buffers allow it, one block reduction and one FP64 atomic per block.
#include <cuda_runtime.h>

#include <cstdint>

#include "mer_device.cuh"

namespace mer {

__global__ void k_l2_loss_grad(const float* __restrict__ image, const float* __restrict__ target, long long n,
                               float* __restrict__ grad, double* __restrict__ loss) {
    __shared__ double sh[8];
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(target) |
                       reinterpret_cast<uintptr_t>(grad)) & 15u) == 0;
    long long done = 0;
    if (vec) {
        const long long n4 = n / 4;
        const float4* a4 = reinterpret_cast<const float4*>(image);
        const float4* b4 = reinterpret_cast<const float4*>(target);
        float4* g4 = reinterpret_cast<float4*>(grad);
        // FP32 partial sums of 32 groups go to the FP64 total (the FP64 pipe is narrow on this GPU)
        float part = 0.f;
        int k = 0;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 a = a4[i], b = b4[i];
            const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
            g4[i] = make_float4(2.f * d0, 2.f * d1, 2.f * d2, 2.f * d3);
            part += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
            if (++k == 32) {
                acc += (double)part;
                part = 0.f;
                k = 0;
            }
        }
        acc += (double)part;
        done = n4 * 4;
    }
    for (long long i = done + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float d = image[i] - target[i];
        grad[i] = 2.f * d;
        acc += (double)(d * d);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        atomicAdd(loss, s);
    }
}

}  // namespace mer

using namespace mer;

extern "C" int mer_l2_loss_grad(const float* image, const float* target, int64_t n, float* grad, double* loss,
                                void* stream) {
    if (n < 0) return MER_EINVAL;
    if (n == 0) return MER_OK;
    if (!image || !target || !grad || !loss) return MER_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MER_ECUDA;
    const long long want = (n / 4 + 255) / 256 + 1;
    const unsigned grid = (unsigned)(want < 8LL * sms ? want : 8LL * sms);
    k_l2_loss_grad<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(image, target, n, grad, loss);
    return cudaGetLastError() == cudaSuccess ? MER_OK : MER_ECUDA;
}
