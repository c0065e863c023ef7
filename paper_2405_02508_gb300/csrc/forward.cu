// forward.cu -- forward gradients (Sec. 5): the per-pixel derivative of the shaded image along one scene
// parameter theta, given its tangent on the projected vertices t_v = d(x_s, y_s, zeta)/d theta.  This is the
// transpose of the backward pass (for every cotangent image g, sum_p g_p . out_p = sum_v grad_v(g) . t_v):
//
//  * interior: screen barycentrics of a fixed pixel centre move as d lambda_i = -grad(lambda_i) . T, with
//    T = sum_j lambda_j t_j (x, y) the motion of the fragment point; zeta tangents enter the perspective
//    correction b_k = lambda_k zeta_k / s; the shaded channels follow (attribute differences, bilinear texture
//    derivative, depth 1/s);
//  * edge: for every neighbour pair with differing ids the classification of Sec. 4.3 (the same exact
//    predicates as the raster), the micro-edge position p (increasing from the left/top pixel A to B) moves
//    by dp/dtheta = the pair-axis motion of the foreground fragment (overhang), or the sum over both
//    fragments of Eq. 12's dp/dr times the slice normal dotted with the fragment's (axis, zeta) motion
//    (intersection); Eq. 11 then changes both pixels by 1/2 (I_A - I_B) dp/dtheta.
//
// One thread per pixel (32 x 8 tiles, index tile with a one-pixel halo in shared memory), no atomics: each
// pixel evaluates its own four pairs.
#include <cuda_runtime.h>

#include <cstdint>

#include "mer_device.cuh"

namespace mer {

constexpr int kFTW = 32, kFTH = 8;

struct FwdArgs {
    mer_shading sh;
    int terms;
    int n, H, W, V, T;
    int tex_stride;
    bool tex_vec4;
};

__device__ __forceinline__ bool fwd_tri_ids(const int* __restrict__ tris, int t, int V, int v[3]) {
    v[0] = __ldg(tris + 3 * (size_t)t);
    v[1] = __ldg(tris + 3 * (size_t)t + 1);
    v[2] = __ldg(tris + 3 * (size_t)t + 2);
    return (unsigned)v[0] < (unsigned)V && (unsigned)v[1] < (unsigned)V && (unsigned)v[2] < (unsigned)V;
}

__device__ __forceinline__ void load_tangent(const float* __restrict__ tb, int v, float t[3]) {
    t[0] = __ldg(tb + 3 * (size_t)v);
    t[1] = __ldg(tb + 3 * (size_t)v + 1);
    t[2] = __ldg(tb + 3 * (size_t)v + 2);
}

// Motion dr = sum_i lambda_i t_i of the fragment of triangle (vid, rv) at pixel (x, y).
__device__ __forceinline__ void frag_motion(const VRec rv[3], const int vid[3], const float* __restrict__ tb, int x,
                                            int y, float dr[3]) {
    const Bary B = screen_bary(rv, x, y);
    dr[0] = dr[1] = dr[2] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float t[3];
        load_tangent(tb, vid[k], t);
        dr[0] += B.lam[k] * t[0];
        dr[1] += B.lam[k] * t[1];
        dr[2] += B.lam[k] * t[2];
    }
}

// dp/dtheta of an overhang pair: the pair-axis motion of the foreground fragment (triangle rv / vid, pixel
// (fx, fy)), or with the exact-crossing option that of the crossing on its exit edge towards pixel (ox, oy).
__device__ __forceinline__ float overhang_rate(const VRec rv[3], const int vid[3], const float* __restrict__ tb,
                                               int fx, int fy, int ox, int oy, int axis, bool exact) {
    if (exact) {
        const int X[3] = {rv[0].X, rv[1].X, rv[2].X}, Y[3] = {rv[0].Y, rv[1].Y, rv[2].Y};
        const int k = exit_edge(X, Y, 256 * fx + 128, 256 * fy + 128, 256 * ox + 128, 256 * oy + 128);
        if (k >= 0) {
            const int j = (k + 1) % 3, l = (k + 2) % 3;
            const float u = axis == 0 ? crossing_u(rv[j].Y, rv[j].ry, rv[l].Y, rv[l].ry, 256 * fy + 128)
                                      : crossing_u(rv[j].X, rv[j].rx, rv[l].X, rv[l].rx, 256 * fx + 128);
            float tj[3], tl[3];
            load_tangent(tb, vid[j], tj);
            load_tangent(tb, vid[l], tl);
            return (1.0f - u) * tj[axis] + u * tl[axis];
        }
    }
    float dr[3];
    frag_motion(rv, vid, tb, fx, fy, dr);
    return dr[axis];
}

__device__ __forceinline__ void plane_normal(const VRec r[3], float N[3]) {
    float p[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k][0] = (float)r[k].X * (1.0f / 256.0f) + r[k].rx;
        p[k][1] = (float)r[k].Y * (1.0f / 256.0f) + r[k].ry;
        p[k][2] = r[k].zeta;
    }
    const float u[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], (r[1].zeta - r[0].zeta) + (r[1].zeta_lo - r[0].zeta_lo)};
    const float w[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], (r[2].zeta - r[0].zeta) + (r[2].zeta_lo - r[0].zeta_lo)};
    N[0] = diff_of_products(u[1], w[2], u[2], w[1]);
    N[1] = diff_of_products(u[2], w[0], u[0], w[2]);
    N[2] = diff_of_products(u[0], w[1], u[1], w[0]);
}

__global__ void __launch_bounds__(kFTW * kFTH) k_forward_grad(const mer_vertex* __restrict__ vpix,
                                                            const int* __restrict__ tris,
                                                            const int* __restrict__ index,
                                                            const float* __restrict__ image,
                                                            const float* __restrict__ tangent,
                                                            const float* __restrict__ attr,
                                                            const float* __restrict__ tex, FwdArgs a,
                                                            float* __restrict__ out, void* ws) {
    __shared__ int sidx[kFTH + 2][kFTW + 2];
    const int view = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = blockIdx.x * kFTW + tx, y = blockIdx.y * kFTH + ty;
    const size_t plane = (size_t)a.H * a.W;
    const int* idx = index + (size_t)view * plane;
    for (int i = ty * kFTW + tx; i < (kFTH + 2) * (kFTW + 2); i += kFTW * kFTH) {
        const int hy = i / (kFTW + 2), hx = i % (kFTW + 2);
        const int gx = blockIdx.x * kFTW + hx - 1, gy = blockIdx.y * kFTH + hy - 1;
        sidx[hy][hx] = (gx >= 0 && gx < a.W && gy >= 0 && gy < a.H) ? __ldg(idx + (size_t)gy * a.W + gx) : -2;
    }
    __syncthreads();
    if (x >= a.W || y >= a.H) return;
    const int C = a.sh.C;
    const mer_vertex* vb = vpix + (size_t)view * a.V;
    const float* tb = tangent + (size_t)view * a.V * 3;
    const float* img = image + (size_t)view * plane * C;
    const size_t p = (size_t)y * a.W + x;
    float acc[kMaxC];
#pragma unroll
    for (int c = 0; c < kMaxC; ++c) acc[c] = 0.f;

    int t = sidx[ty + 1][tx + 1];
    int vid[3] = {0, 0, 0};
    if (t >= a.T || (t >= 0 && !fwd_tri_ids(tris, t, a.V, vid))) {
        set_status(ws, kStatusRange);
        t = -1;
    }
    VRec rv[3];
    if (t >= 0) {
        rv[0] = load_vrec(vb + vid[0]);
        rv[1] = load_vrec(vb + vid[1]);
        rv[2] = load_vrec(vb + vid[2]);
    }

    if (t >= 0 && (a.terms & MER_INTERIOR)) {
        const Bary B = screen_bary(rv, x, y);
        float tv[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) load_tangent(tb, vid[k], tv[k]);
        const float Tx = B.lam[0] * tv[0][0] + B.lam[1] * tv[1][0] + B.lam[2] * tv[2][0];
        const float Ty = B.lam[0] * tv[0][1] + B.lam[1] * tv[1][1] + B.lam[2] * tv[2][1];
        float dl[3], z[3];
        float s = 0.f, ds = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dl[k] = -(B.gx[k] * Tx + B.gy[k] * Ty);
            z[k] = rv[k].zeta;
            s += B.lam[k] * z[k];
            ds += dl[k] * z[k] + B.lam[k] * tv[k][2];
        }
        const float is = rcp_nr(s);
        float b[3], db[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            b[k] = B.lam[k] * z[k] * is;
            db[k] = (dl[k] * z[k] + B.lam[k] * tv[k][2]) * is - b[k] * ds * is;
        }
        const int Ca = a.sh.C_attr;
        if (a.sh.uv_offset < 0) {
#pragma unroll
            for (int c = 0; c < kMaxC; ++c) {
                if (c >= a.sh.n_main) break;
                const float a0 = __ldg(attr + (size_t)vid[0] * Ca + c);
                const float a1 = __ldg(attr + (size_t)vid[1] * Ca + c);
                const float a2 = __ldg(attr + (size_t)vid[2] * Ca + c);
                acc[c] += db[1] * (a1 - a0) + db[2] * (a2 - a0);  // sum_k db_k = 0
            }
        } else {
            float uk[3], vk[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                uk[k] = __ldg(attr + (size_t)vid[k] * Ca + a.sh.uv_offset);
                vk[k] = __ldg(attr + (size_t)vid[k] * Ca + a.sh.uv_offset + 1);
            }
            const float du = db[1] * (uk[1] - uk[0]) + db[2] * (uk[2] - uk[0]);
            const float dv = db[1] * (vk[1] - vk[0]) + db[2] * (vk[2] - vk[0]);
            const TexCoord cx = tex_coord(uk[0], uk[1], uk[2], b[1], b[2], a.sh.tex_w);
            const TexCoord cy = tex_coord(vk[0], vk[1], vk[2], b[1], b[2], a.sh.tex_h);
            const TexTaps taps = tex_taps(a.sh.tex_h, a.sh.tex_w, cx, cy);
            const float dfx = (float)a.sh.tex_w * du, dfy = taps.clamped ? 0.f : (float)a.sh.tex_h * dv;
#pragma unroll
            for (int c = 0; c < kMaxC; ++c) {
                if (c >= a.sh.n_main) break;
                const float* r0 = tex + (size_t)taps.j0 * a.sh.tex_w * a.tex_stride;
                const float* r1 = tex + (size_t)taps.j1 * a.sh.tex_w * a.tex_stride;
                const float t00 = __ldg(r0 + (size_t)taps.i0 * a.tex_stride + c);
                const float t10 = __ldg(r0 + (size_t)taps.i1 * a.tex_stride + c);
                const float t01 = __ldg(r1 + (size_t)taps.i0 * a.tex_stride + c);
                const float t11 = __ldg(r1 + (size_t)taps.i1 * a.tex_stride + c);
                const float dTx = (1.0f - taps.fy) * (t10 - t00) + taps.fy * (t11 - t01);
                const float lo = t00 + taps.fx * (t10 - t00), hi = t01 + taps.fx * (t11 - t01);
                acc[c] += dTx * dfx + (hi - lo) * dfy;
            }
        }
        if (a.sh.depth_ch >= 0) {
#pragma unroll
            for (int c = 0; c < kMaxC; ++c)
                if (c == a.sh.depth_ch) acc[c] += -ds * is * is;
        }
    }

    if (a.terms & MER_EDGE) {
        const bool exact = (a.terms & MER_EXACT_CROSSING) != 0;
#pragma unroll 1
        for (int d = 0; d < 4; ++d) {
            const int ddx = d == 0 ? -1 : (d == 1 ? 1 : 0);
            const int ddy = d == 2 ? -1 : (d == 3 ? 1 : 0);
            int tq = sidx[ty + 1 + ddy][tx + 1 + ddx];
            if (tq == -2 || tq == t) continue;  // outside the image, or the same triangle
            const int qx = x + ddx, qy = y + ddy;
            int vq[3] = {0, 0, 0};
            VRec rq[3];
            if (tq >= 0) {
                if (tq >= a.T || !fwd_tri_ids(tris, tq, a.V, vq)) {
                    set_status(ws, kStatusRange);
                    continue;
                }
                rq[0] = load_vrec(vb + vq[0]);
                rq[1] = load_vrec(vb + vq[1]);
                rq[2] = load_vrec(vb + vq[2]);
            }
            if (t < 0 && tq < 0) continue;
            float dpdt = 0.f;
            if (t >= 0 && tq >= 0) {
                const int Xp[3] = {rv[0].X, rv[1].X, rv[2].X}, Yp[3] = {rv[0].Y, rv[1].Y, rv[2].Y};
                const int Xq[3] = {rq[0].X, rq[1].X, rq[2].X}, Yq[3] = {rq[0].Y, rq[1].Y, rq[2].Y};
                const bool p_in_q = covers_xy(Xq, Yq, 256 * x + 128, 256 * y + 128);
                const bool q_in_p = covers_xy(Xp, Yp, 256 * qx + 128, 256 * qy + 128);
                if (!p_in_q && !q_in_p) continue;  // adjacent
                const int axis = ddx != 0 ? 0 : 1;
                if (p_in_q && q_in_p) {
                    if (!(a.terms & MER_INTERSECT)) continue;
                    // Eq. 12 on both fragments, slice (axis, zeta)
                    float Np[3], Nq[3], drp[3], drq[3];
                    plane_normal(rv, Np);
                    plane_normal(rq, Nq);
                    const float np0 = Np[axis], np1 = Np[2], nq0 = Nq[axis], nq1 = Nq[2];
                    const float den_p = diff_of_products(nq0, np1, nq1, np0);  // v = p, f = q
                    const float mag = sqrtf((np0 * np0 + np1 * np1) * (nq0 * nq0 + nq1 * nq1));
                    if (!(fabsf(den_p) > 1e-12f * mag)) continue;
                    const float den_q = -den_p;  // v = q, f = p
                    frag_motion(rv, vid, tb, x, y, drp);
                    frag_motion(rq, vq, tb, qx, qy, drq);
                    dpdt = (-nq1 / den_p) * (np0 * drp[axis] + np1 * drp[2]) +
                           (-np1 / den_q) * (nq0 * drq[axis] + nq1 * drq[2]);
                } else {
                    dpdt = p_in_q ? overhang_rate(rv, vid, tb, x, y, qx, qy, axis, exact)
                                  : overhang_rate(rq, vq, tb, qx, qy, x, y, axis, exact);
                }
            } else {
                const int axis = ddx != 0 ? 0 : 1;
                dpdt = t >= 0 ? overhang_rate(rv, vid, tb, x, y, qx, qy, axis, exact)
                              : overhang_rate(rq, vq, tb, qx, qy, x, y, axis, exact);
            }
            // Eq. 11 transposed: both pixels of the pair change by 1/2 (I_A - I_B) dp/dtheta, A = left/top
            const size_t q = (size_t)qy * a.W + qx;
            const float* ia = (ddx > 0 || ddy > 0) ? img + p * C : img + q * C;
            const float* ib = (ddx > 0 || ddy > 0) ? img + q * C : img + p * C;
#pragma unroll
            for (int c = 0; c < kMaxC; ++c) {
                if (c >= C) break;
                acc[c] += 0.5f * (__ldg(ia + c) - __ldg(ib + c)) * dpdt;
            }
        }
    }
    float* o = out + ((size_t)view * plane + p) * C;
#pragma unroll
    for (int c = 0; c < kMaxC; ++c)
        if (c < C) o[c] = acc[c];
}

// Tangent of the projected vertices for a world-space vertex tangent (shared by all views):
// d(x_s, y_s, zeta) = J(X_c) R d(X_w), J as in the projection backward.
__global__ void k_project_jvp(const float* __restrict__ tw, int V, const mer_camera* __restrict__ cams, int n,
                              const mer_vertex* __restrict__ vpix, float* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)V * n) return;
    const int view = (int)(i / V), v = (int)(i % V);
    const mer_vertex r = vpix[i];
    const mer_camera& c = cams[view];
    float* o = out + 3 * i;
    if ((r.flags & 1u) == 0u) {
        o[0] = o[1] = o[2] = 0.f;
        return;
    }
    const float d0 = tw[3 * (size_t)v], d1 = tw[3 * (size_t)v + 1], d2 = tw[3 * (size_t)v + 2];
    const float dX = (float)c.R[0] * d0 + (float)c.R[1] * d1 + (float)c.R[2] * d2;
    const float dY = (float)c.R[3] * d0 + (float)c.R[4] * d1 + (float)c.R[5] * d2;
    const float dZ = (float)c.R[6] * d0 + (float)c.R[7] * d1 + (float)c.R[8] * d2;
    const float z = r.zeta;
    const float xs = (float)((double)r.X * (1.0 / 256.0) - c.cx) + r.rx;
    const float ys = (float)((double)r.Y * (1.0 / 256.0) - c.cy) + r.ry;
    o[0] = (float)c.fx * z * dX - xs * z * dZ;
    o[1] = (float)c.fy * z * dY - ys * z * dZ;
    o[2] = -z * z * dZ;
}

}  // namespace mer

using namespace mer;

extern "C" int mer_launch_forward_grad(const mer_vertex* vpix, int V, const int* tris, int T, int n, int H, int W,
                                       const int* index, const float* image, const float* tangent, const float* attr,
                                       const float* tex, const mer_shading* sh, int terms, float* out, void* ws,
                                       cudaStream_t s) {
    FwdArgs a;
    a.sh = *sh;
    a.terms = terms;
    a.n = n; a.H = H; a.W = W; a.V = V; a.T = T;
    a.tex_stride = sh->tex_c > 0 ? sh->tex_c : sh->n_main;
    a.tex_vec4 = false;
    const dim3 grid((unsigned)((W + kFTW - 1) / kFTW), (unsigned)((H + kFTH - 1) / kFTH), (unsigned)n);
    k_forward_grad<<<grid, dim3(kFTW, kFTH), 0, s>>>(vpix, tris, index, image, tangent, attr, tex, a, out, ws);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int mer_launch_project_jvp(const float* tangent_world, int V, const mer_camera* cams, int n,
                                      const mer_vertex* vpix, float* out, cudaStream_t s) {
    const long long N = (long long)V * n;
    k_project_jvp<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(tangent_world, V, cams, n, vpix, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
