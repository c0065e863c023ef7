// shade.cu -- barycentrics + interpolation modules and deferred shading (Supp. B).
//
// One thread per pixel: re-derive the screen barycentrics of the pixel centre
// from the index image and the projected vertex records, make them perspective
// correct, and write the shaded channels (interpolated attributes or bilinear
// texture, coverage mask, depth) as one contiguous NHWC run per pixel.
#include <cuda_runtime.h>

#include <cstdint>

#include "shade_device.cuh"

namespace mer {

// Pixel (x, y) of an item: vb / tris / attr are the item's bases, p the global pixel.  PRECISE: FP64
// arithmetic, one rounding per value (the precise shading option).
template <bool PRECISE>
__device__ __forceinline__ void shade_pixel(const mer_vertex* __restrict__ vb, int V, const int* __restrict__ tris,
                                            int T, int x, int y, size_t p, const int* __restrict__ index,
                                            const float* __restrict__ attr, const float* __restrict__ tex,
                                            const ShadeArgs& a, float* __restrict__ image, void* ws) {
    if (PRECISE)
        shade_fragment_f64(vb, V, tris, T, index[p], x, y, attr, tex, a, image + p * a.sh.C, ws);
    else
        shade_fragment(vb, V, tris, T, index[p], x, y, attr, tex, a, image + p * a.sh.C, ws);
}

template <bool PRECISE>
__global__ void k_shade(const mer_vertex* __restrict__ vpix, int V, const int* __restrict__ tris, int T, int n, int H,
                        int W, const int* __restrict__ index, const float* __restrict__ attr,
                        const float* __restrict__ tex, ShadeArgs a, float* __restrict__ image, void* ws) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long npix = (long long)n * H * W;
    if (p >= npix) return;
    const int view = (int)(p / ((long long)H * W));
    const int rem = (int)(p % ((long long)H * W));
    shade_pixel<PRECISE>(vpix + (size_t)view * V, V, tris, T, rem % W, rem / W, (size_t)p, index, attr, tex, a, image, ws);
}

template <bool PRECISE>
__global__ void k_shade_batch(const mer_vertex* __restrict__ vpix, const int* __restrict__ tris,
                              const mer_item* __restrict__ items, int n_items, long long pixels,
                              const int* __restrict__ index, const float* __restrict__ attr,
                              const float* __restrict__ tex, ShadeArgs a, float* __restrict__ image, void* ws) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = block_find_item(items, n_items, (long long)blockIdx.x * blockDim.x, p, kFieldPix);
    if (p >= pixels) return;
    const mer_item m = items[k];
    const int rem = (int)(p - m.pix);
    shade_pixel<PRECISE>(vpix + m.vrec, m.V, tris + 3 * m.tri, m.T, rem % m.W, rem / m.W, (size_t)p, index,
                attr ? attr + (size_t)m.vert * a.sh.C_attr : nullptr, tex, a, image, ws);
}

}  // namespace mer

using namespace mer;


extern "C" int mer_launch_shade_batch(const mer_vertex* vpix, const int* tris, const mer_item* items, int n_items,
                                      long long pixels, const int* index, const float* attr, const float* tex,
                                      const float* bg, const mer_shading* sh, float* image, void* ws, cudaStream_t s) {
    if (pixels == 0) return 0;
    const ShadeArgs a = make_shade_args(tex, bg, sh);
    const unsigned blocks = (unsigned)((pixels + 255) / 256);
    if (sh->precise)
        k_shade_batch<true><<<blocks, 256, 0, s>>>(vpix, tris, items, n_items, pixels, index, attr, tex, a, image, ws);
    else
        k_shade_batch<false><<<blocks, 256, 0, s>>>(vpix, tris, items, n_items, pixels, index, attr, tex, a, image, ws);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int mer_launch_shade(const mer_vertex* vpix, int V, const int* tris, int T, int n, int H, int W,
                                const int* index, const float* attr, const float* tex, const float* bg,
                                const mer_shading* sh, float* image, void* ws, cudaStream_t s) {
    const long long npix = (long long)n * H * W;
    if (npix == 0) return 0;
    const ShadeArgs a = make_shade_args(tex, bg, sh);
    const unsigned blocks = (unsigned)((npix + 255) / 256);
    if (sh->precise)
        k_shade<true><<<blocks, 256, 0, s>>>(vpix, V, tris, T, n, H, W, index, attr, tex, a, image, ws);
    else
        k_shade<false><<<blocks, 256, 0, s>>>(vpix, V, tris, T, n, H, W, index, attr, tex, a, image, ws);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
