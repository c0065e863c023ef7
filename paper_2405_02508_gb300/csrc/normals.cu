// normals.cu -- area-weighted vertex normals of triangle meshes and their backward, for inverse rendering
// loops that shade with normals recomputed from the current positions (the paper's normal supervision,
// Supp. B).  n_v = a_v / |a_v| with a_v = sum over the triangles at v of (p1 - p0) x (p2 - p0); |a_v| is
// clamped below at 1e-20 (an isolated vertex gets a zero normal and the gradient of a / 1e-20).
//
// Forward: one thread per triangle adds its face normal to its three vertices (FP32 atomics), then one
// thread per vertex normalises.  Backward: one thread per vertex forms dL/da_v = (g - n (n . g)) / |a_v|,
// then one thread per triangle sums it over its vertices (dL/d(face normal)) and adds the cross-product
// derivatives to the three positions.
#include <cuda_runtime.h>

#include <cstdint>

#include "mer_device.cuh"

namespace mer {

constexpr float kNormalFloor = 1e-20f;

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ bool tri_fetch(const int* __restrict__ tris, long long t, int V, int v[3]) {
    v[0] = tris[3 * t];
    v[1] = tris[3 * t + 1];
    v[2] = tris[3 * t + 2];
    return (unsigned)v[0] < (unsigned)V && (unsigned)v[1] < (unsigned)V && (unsigned)v[2] < (unsigned)V;
}

__global__ void k_face_accumulate(const float* __restrict__ verts, const int* __restrict__ tris, long long T, int V,
                                  float* __restrict__ acc, void* ws) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int v[3];
    if (!tri_fetch(tris, t, V, v)) {
        set_status(ws, kStatusRange);
        return;
    }
    float p[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) p[k][c] = verts[3 * (size_t)v[k] + c];
    const float e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
    const float e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
    float fn[3];
    cross3(e1, e2, fn);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(acc + 3 * (size_t)v[k] + c, fn[c]);
}

__global__ void k_normalize(const float* __restrict__ acc, long long V, float* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    const float a0 = acc[3 * i], a1 = acc[3 * i + 1], a2 = acc[3 * i + 2];
    const float inv = 1.0f / fmaxf(sqrtf(a0 * a0 + a1 * a1 + a2 * a2), kNormalFloor);
    out[3 * i] = a0 * inv;
    out[3 * i + 1] = a1 * inv;
    out[3 * i + 2] = a2 * inv;
}

// dL/da_v in place of dL/dn_v.
__global__ void k_normalize_backward(const float* __restrict__ acc, long long V, float* __restrict__ g) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    const float a[3] = {acc[3 * i], acc[3 * i + 1], acc[3 * i + 2]};
    const float gi[3] = {g[3 * i], g[3 * i + 1], g[3 * i + 2]};
    const float len = sqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (!(len > kNormalFloor)) {  // clamped: n = a / floor
#pragma unroll
        for (int c = 0; c < 3; ++c) g[3 * i + c] = gi[c] / kNormalFloor;
        return;
    }
    const float inv = 1.0f / len;
    const float n[3] = {a[0] * inv, a[1] * inv, a[2] * inv};
    const float ng = n[0] * gi[0] + n[1] * gi[1] + n[2] * gi[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) g[3 * i + c] = (gi[c] - n[c] * ng) * inv;
}

// Face normal fn = e1 x e2 (e1 = p1 - p0, e2 = p2 - p0) with dL/dfn = sum of dL/da over its vertices:
// dL/dp1 = e2 x G, dL/dp2 = G x e1, dL/dp0 = -(dL/dp1 + dL/dp2).
__global__ void k_face_backward(const float* __restrict__ verts, const int* __restrict__ tris, long long T, int V,
                                const float* __restrict__ ga, float* __restrict__ grad_verts, void* ws) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int v[3];
    if (!tri_fetch(tris, t, V, v)) {
        set_status(ws, kStatusRange);
        return;
    }
    float p[3][3], G[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p[k][c] = verts[3 * (size_t)v[k] + c];
            G[c] += ga[3 * (size_t)v[k] + c];
        }
    const float e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
    const float e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
    float g1[3], g2[3];
    cross3(e2, G, g1);
    cross3(G, e1, g2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        atomicAdd(grad_verts + 3 * (size_t)v[1] + c, g1[c]);
        atomicAdd(grad_verts + 3 * (size_t)v[2] + c, g2[c]);
        atomicAdd(grad_verts + 3 * (size_t)v[0] + c, -(g1[c] + g2[c]));
    }
}

}  // namespace mer

using namespace mer;

namespace {
inline unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }
}  // namespace

extern "C" int mer_vertex_normals(const float* verts, int V, const int32_t* tris, int64_t T, float* acc,
                                  float* normals, void* status_ws, void* stream) {
    if (V < 0 || T < 0) return MER_EINVAL;
    if (V == 0) return MER_OK;
    if (!verts || !acc || !normals || (T > 0 && !tris) || acc == normals) return MER_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(acc, 0, (size_t)V * 3 * sizeof(float), s) != cudaSuccess) return MER_ECUDA;
    if (T > 0) k_face_accumulate<<<blocks(T), 256, 0, s>>>(verts, tris, T, V, acc, status_ws);
    k_normalize<<<blocks(V), 256, 0, s>>>(acc, V, normals);
    return cudaGetLastError() == cudaSuccess ? MER_OK : MER_ECUDA;
}

extern "C" int mer_vertex_normals_backward(const float* verts, int V, const int32_t* tris, int64_t T,
                                           const float* acc, float* grad_normals, float* grad_verts,
                                           void* status_ws, void* stream) {
    if (V < 0 || T < 0) return MER_EINVAL;
    if (V == 0) return MER_OK;
    if (!verts || !acc || !grad_normals || !grad_verts || (T > 0 && !tris)) return MER_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_normalize_backward<<<blocks(V), 256, 0, s>>>(acc, V, grad_normals);
    if (T > 0) k_face_backward<<<blocks(T), 256, 0, s>>>(verts, tris, T, V, grad_normals, grad_verts, status_ws);
    return cudaGetLastError() == cudaSuccess ? MER_OK : MER_ECUDA;
}
