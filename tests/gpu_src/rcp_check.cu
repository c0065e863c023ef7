// Checks rcp_nr (one Newton step from the hardware reciprocal estimate) against the correctly rounded
// reciprocal on every float of the chosen exponent range: how many differ, and the largest difference in
// units in the last place.  Built and run by tests/test_gpu_rcp.py.
#include <cstdio>
#include <cstdlib>

#include "../../paper_2405_02508_gb300/csrc/mer_device.cuh"

__global__ void k_check(unsigned lo, unsigned hi, unsigned long long* out) {
    unsigned long long diff = 0ull, worst = 0ull;
    for (unsigned b = lo + blockIdx.x * blockDim.x + threadIdx.x; b < hi; b += gridDim.x * blockDim.x) {
        const float x = __uint_as_float(b);
        const float a = mer::rcp_nr(x), c = __frcp_rn(x);
        const unsigned ua = __float_as_uint(a), uc = __float_as_uint(c);
        if (ua != uc) {
            ++diff;
            const unsigned long long d = ua > uc ? ua - uc : uc - ua;
            if (d > worst) worst = d;
        }
    }
    atomicAdd(&out[0], diff);
    atomicMax(&out[1], worst);
}

int main(int argc, char** argv) {
    // all positive normal floats with exponents in [2^-60, 2^60] (both signs by symmetry of the method)
    const unsigned lo = 0x21800000u, hi = 0x5D800000u;
    unsigned long long* out = nullptr;
    if (cudaMalloc(&out, 2 * sizeof(unsigned long long)) != cudaSuccess) return 2;
    if (cudaMemset(out, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return 2;
    k_check<<<4096, 256>>>(lo, hi, out);
    unsigned long long h[2] = {0ull, 0ull};
    if (cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
    printf("%llu %llu %u\n", h[0], h[1], hi - lo);
    cudaFree(out);
    return 0;
}
