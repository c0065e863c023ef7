// project.cu -- vertex transform module (Supp. B) and its backward.
//
// Forward in FP64 with a fixed operation order and correctly rounded intrinsics
// (no contraction into FMA), so the snapped screen positions X = rint(256 x_s)
// are reproducible bit for bit by any IEEE FP64 implementation of the same
// formula.  Backward: the per-view kernel in FP64 (sums over the views in a fixed order); the batched one
// in FP32 with atomics, or, given a workspace, in FP64 with fixed-point sums (bitwise reproducible).
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

// world_grad in FP64 (vertex position from the exact snapped part plus the residual, zeta from its hi + lo
// split).
__device__ __forceinline__ bool world_grad_f64(const mer_vertex& r, const mer_camera& c, const double* g3,
                                               double out[3]) {
    if ((r.flags & 1u) == 0u) return false;
    const double gx = g3[0], gy = g3[1], gz = g3[2];
    const double z = (double)r.zeta + (double)r.zeta_lo;
    const double xs = ((double)r.X * (1.0 / 256.0) - c.cx) + (double)r.rx;
    const double ys = ((double)r.Y * (1.0 / 256.0) - c.cy) + (double)r.ry;
    const double gX = gx * c.fx * z;
    const double gY = gy * c.fy * z;
    const double gZ = -z * (gx * xs + gy * ys + gz * z);
    out[0] = c.R[0] * gX + c.R[3] * gY + c.R[6] * gZ;
    out[1] = c.R[1] * gX + c.R[4] * gY + c.R[7] * gZ;
    out[2] = c.R[2] * gX + c.R[5] * gY + c.R[8] * gZ;
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

// Batched, reproducible: FP64 products rounded once to fixed point with 52 fractional bits, held as two
// 64-bit words (hi = floor(w 2^20), lo = the remainder in units of 2^-52, in [0, 2^32]), and added with
// integer atomics into acc [mesh rows, 3, 2] (exact, so the order does not matter); k_world_finalize converts.
__global__ void k_project_backward_batch_fixed(const mer_camera* __restrict__ cams, const mer_item* __restrict__ items,
                                               int n_items, long long vrecs, const mer_vertex* __restrict__ vpix,
                                               const double* __restrict__ grad_vpix, unsigned long long* acc,
                                               void* ws) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = block_find_item(items, n_items, (long long)blockIdx.x * blockDim.x, i, kFieldVrec);
    if (i >= vrecs) return;
    const mer_item m = items[k];
    double w[3];
    if (!world_grad_f64(vpix[i], cams[m.cam], grad_vpix + 3 * i, w)) return;
    unsigned long long* o = acc + 6 * (size_t)(m.vert + (i - m.vrec));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (!(fabs(w[c]) < 8589934592.0)) {  // 2^33
            set_status(ws, kStatusFixed);
            continue;
        }
        const double h = floor(w[c] * 1048576.0);
        const long long hi = (long long)h;
        const long long lo = __double2ll_rn((w[c] - h * (1.0 / 1048576.0)) * 4503599627370496.0);
        if (hi != 0) atomicAdd(o + 2 * c, (unsigned long long)hi);
        if (lo != 0) atomicAdd(o + 2 * c + 1, (unsigned long long)lo);
    }
}

__global__ void k_world_finalize(const unsigned long long* __restrict__ acc, long long n, float* __restrict__ grad_verts) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long lo = (long long)acc[2 * i + 1];
    const long long hi = (long long)acc[2 * i] + (lo >> 32);
    grad_verts[i] += __double2float_rn((double)hi * (1.0 / 1048576.0) + (double)(lo & 0xffffffffll) * (1.0 / 4503599627370496.0));
}

// One thread per vertex, looping over the views: grad_world = sum_views R^T J^T g (FP64).
__global__ void k_project_backward(int V, const mer_camera* __restrict__ cams, int n,
                                   const mer_vertex* __restrict__ vpix, const double* __restrict__ grad_vpix,
                                   float* __restrict__ grad_verts) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int view = 0; view < n; ++view) {
        const size_t k = (size_t)view * V + v;
        double w[3];
        if (!world_grad_f64(vpix[k], cams[view], grad_vpix + 3 * k, w)) continue;
        a0 += w[0];
        a1 += w[1];
        a2 += w[2];
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

// ws: null for the FP32 atomic path; else a workspace whose bytes after the 256-byte header hold
// mesh_rows * 3 two-word fixed-point sums (the reproducible FP64 path).
extern "C" int mer_launch_project_backward_batch(const mer_camera* cams, const mer_item* items, int n_items,
                                                 long long vrecs, long long mesh_rows, const mer_vertex* vpix,
                                                 const double* grad_vpix, float* grad_verts, void* ws,
                                                 cudaStream_t s) {
    if (vrecs == 0) return 0;
    if (ws) {
        unsigned long long* acc = reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + 256);
        if (cudaMemsetAsync(acc, 0, (size_t)mesh_rows * 48, s) != cudaSuccess) return 2;
        k_project_backward_batch_fixed<<<(unsigned)((vrecs + 255) / 256), 256, 0, s>>>(cams, items, n_items, vrecs,
                                                                                       vpix, grad_vpix, acc, ws);
        const long long n = 3 * mesh_rows;
        if (n > 0) k_world_finalize<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc, n, grad_verts);
        return cudaGetLastError() == cudaSuccess ? 0 : 2;
    }
    k_project_backward_batch<<<(unsigned)((vrecs + 255) / 256), 256, 0, s>>>(cams, items, n_items, vrecs, vpix,
                                                                             grad_vpix, grad_verts);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
