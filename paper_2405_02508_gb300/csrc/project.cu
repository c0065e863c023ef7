// project.cu -- vertex transform module (Supp. B) and its backward.
//
// Forward in FP64 with a fixed operation order and correctly rounded intrinsics
// (no contraction into FMA), so the snapped screen positions X = rint(256 x_s)
// are reproducible bit for bit by any IEEE FP64 implementation of the same
// formula.  Backward in FP32.
#include <cuda_runtime.h>

#include "mer_device.cuh"

namespace mer {

__device__ __forceinline__ void write_vertex(double xs, double ys, double zeta, bool front, mer_vertex* out) {
    mer_vertex r;
    r.X = 0; r.Y = 0; r.rx = 0.f; r.ry = 0.f; r.zeta = 0.f; r.zeta_lo = 0.f; r.flags = 0u; r.pad = 0.f;
    if (front) {
        r.flags = 1u;
        const double X = __dmul_rn(xs, 256.0), Y = __dmul_rn(ys, 256.0);  // exact (power of two)
        if (fabs(X) <= kGuard && fabs(Y) <= kGuard) {
            r.flags |= 2u;
            const long long sx = __double2ll_rn(X), sy = __double2ll_rn(Y);  // ties to even
            r.X = (int)sx;
            r.Y = (int)sy;
            r.rx = __double2float_rn(__dsub_rn(xs, __dmul_rn((double)sx, 1.0 / 256.0)));
            r.ry = __double2float_rn(__dsub_rn(ys, __dmul_rn((double)sy, 1.0 / 256.0)));
        }
        r.zeta = __double2float_rn(zeta);
        r.zeta_lo = __double2float_rn(__dsub_rn(zeta, (double)r.zeta));
    }
    *out = r;
}

__device__ __forceinline__ void project_one(const float* __restrict__ w, const mer_camera& c, mer_vertex* out) {
    const double x = w[0], y = w[1], z = w[2];
    const double* R = c.R;
    const double Xc = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[0], x), __dmul_rn(R[1], y)), __dmul_rn(R[2], z)), c.t[0]);
    const double Yc = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[3], x), __dmul_rn(R[4], y)), __dmul_rn(R[5], z)), c.t[1]);
    const double Zc = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[6], x), __dmul_rn(R[7], y)), __dmul_rn(R[8], z)), c.t[2]);
    const bool front = Zc > c.znear;
    double zeta = 0.0, xs = 0.0, ys = 0.0;
    if (front) {
        zeta = __drcp_rn(Zc);
        xs = __dadd_rn(__dmul_rn(__dmul_rn(c.fx, Xc), zeta), c.cx);
        ys = __dadd_rn(__dmul_rn(__dmul_rn(c.fy, Yc), zeta), c.cy);
    }
    write_vertex(xs, ys, zeta, front, out);
}

__global__ void k_project(const float* __restrict__ verts, int V, const mer_camera* __restrict__ cams, int n,
                          mer_vertex* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)V * n) return;
    const int view = (int)(i / V), v = (int)(i % V);
    project_one(verts + 3 * (size_t)v, cams[view], out + i);
}

__global__ void k_project_batch(const float* __restrict__ verts, const mer_camera* __restrict__ cams,
                                const mer_item* __restrict__ items, int n_items, long long vrecs,
                                mer_vertex* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = block_find_item(items, n_items, (long long)blockIdx.x * blockDim.x, i, kFieldVrec);
    if (i >= vrecs) return;
    const mer_item m = items[k];
    project_one(verts + 3 * (size_t)(m.vert + (i - m.vrec)), cams[m.cam], out + i);
}

__global__ void k_project_screen(const double* __restrict__ scr, int V, int n, mer_vertex* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)V * n) return;
    const double xs = scr[3 * i], ys = scr[3 * i + 1], zeta = scr[3 * i + 2];
    write_vertex(xs, ys, zeta, zeta > 0.0, out + i);
}

// R^T J^T g for one projected vertex, J = d(x_s, y_s, zeta)/d(X_c, Y_c, Z_c)
// = [[fx z, 0, -(x_s-cx) z], [0, fy z, -(y_s-cy) z], [0, 0, -z^2]]; false if the vertex is behind the camera.
__device__ __forceinline__ bool world_grad(const mer_vertex& r, const mer_camera& c, const double* g3, float out[3]) {
    if ((r.flags & 1u) == 0u) return false;
    const float gx = (float)g3[0], gy = (float)g3[1], gz = (float)g3[2];
    const float z = r.zeta;
    const float xs = (float)((double)r.X * (1.0 / 256.0) - c.cx) + r.rx;
    const float ys = (float)((double)r.Y * (1.0 / 256.0) - c.cy) + r.ry;
    const float gX = gx * (float)c.fx * z;
    const float gY = gy * (float)c.fy * z;
    const float gZ = -z * (gx * xs + gy * ys + gz * z);
    out[0] = (float)c.R[0] * gX + (float)c.R[3] * gY + (float)c.R[6] * gZ;
    out[1] = (float)c.R[1] * gX + (float)c.R[4] * gY + (float)c.R[7] * gZ;
    out[2] = (float)c.R[2] * gX + (float)c.R[5] * gY + (float)c.R[8] * gZ;
    return true;
}

// Batched: one thread per (item, vertex); items sharing a mesh add into the same rows.
__global__ void k_project_backward_batch(const mer_camera* __restrict__ cams, const mer_item* __restrict__ items,
                                         int n_items, long long vrecs, const mer_vertex* __restrict__ vpix,
                                         const double* __restrict__ grad_vpix, float* __restrict__ grad_verts) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = block_find_item(items, n_items, (long long)blockIdx.x * blockDim.x, i, kFieldVrec);
    if (i >= vrecs) return;
    const mer_item m = items[k];
    float w[3];
    if (!world_grad(vpix[i], cams[m.cam], grad_vpix + 3 * i, w)) return;
    float* o = grad_verts + 3 * (size_t)(m.vert + (i - m.vrec));
    atomicAdd(o, w[0]);
    atomicAdd(o + 1, w[1]);
    atomicAdd(o + 2, w[2]);
}

// One thread per vertex, looping over the views: grad_world = sum_views R^T J^T g.
__global__ void k_project_backward(int V, const mer_camera* __restrict__ cams, int n,
                                   const mer_vertex* __restrict__ vpix, const double* __restrict__ grad_vpix,
                                   float* __restrict__ grad_verts) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;  // sum over views in FP64, products in FP32
    for (int view = 0; view < n; ++view) {
        const size_t k = (size_t)view * V + v;
        float w[3];
        if (!world_grad(vpix[k], cams[view], grad_vpix + 3 * k, w)) continue;
        a0 += (double)w[0];
        a1 += (double)w[1];
        a2 += (double)w[2];
    }
    grad_verts[3 * (size_t)v] += (float)a0;
    grad_verts[3 * (size_t)v + 1] += (float)a1;
    grad_verts[3 * (size_t)v + 2] += (float)a2;
}

}  // namespace mer

using namespace mer;

extern "C" int mer_launch_project(const float* verts, int V, const mer_camera* cams, int n, mer_vertex* vpix,
                                  cudaStream_t s) {
    const long long N = (long long)V * n;
    if (N == 0) return 0;
    k_project<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(verts, V, cams, n, vpix);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int mer_launch_project_screen(const double* scr, int V, int n, mer_vertex* vpix, cudaStream_t s) {
    const long long N = (long long)V * n;
    if (N == 0) return 0;
    k_project_screen<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(scr, V, n, vpix);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int mer_launch_project_backward(int V, const mer_camera* cams, int n, const mer_vertex* vpix,
                                           const double* grad_vpix, float* grad_verts, cudaStream_t s) {
    if (V == 0 || n == 0) return 0;
    k_project_backward<<<(V + 255) / 256, 256, 0, s>>>(V, cams, n, vpix, grad_vpix, grad_verts);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int mer_launch_project_batch(const float* verts, const mer_camera* cams, const mer_item* items, int n_items,
                                        long long vrecs, mer_vertex* vpix, cudaStream_t s) {
    if (vrecs == 0) return 0;
    k_project_batch<<<(unsigned)((vrecs + 255) / 256), 256, 0, s>>>(verts, cams, items, n_items, vrecs, vpix);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int mer_launch_project_backward_batch(const mer_camera* cams, const mer_item* items, int n_items,
                                                 long long vrecs, const mer_vertex* vpix, const double* grad_vpix,
                                                 float* grad_verts, cudaStream_t s) {
    if (vrecs == 0) return 0;
    k_project_backward_batch<<<(unsigned)((vrecs + 255) / 256), 256, 0, s>>>(cams, items, n_items, vrecs, vpix,
                                                                             grad_vpix, grad_verts);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
