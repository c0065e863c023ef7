// backward.cu -- EdgeGrad module backward (Sec. 4.2-4.4, Supp. A.2-A.3) fused with
// the interior term Omega (Eq. 5) and the interpolation / barycentrics backward.
//
// One CTA per 16x16 pixel tile of one view; the tile's index image plus a
// one-pixel halo sits in shared memory.  Each covered pixel p owns the fragment
// of its triangle t at its centre and accumulates that fragment's gradient
// dL/dr (a 3-vector in x_s, y_s, zeta):
//   * interior: -grad_P(L) in x, y from the barycentric derivatives, plus the
//     direct zeta derivative of the perspective weights and depth;
//   * edge: for each of its 4 neighbours q with a different id, Eq. 11 for the
//     pair (oriented left->right / top->bottom), then the Sec. 4.3 rule (p on
//     top -> dp/dr = 1 on the pair axis) or Eq. 12 (intersection) for p's side.
// The fragment gradient is gathered to the 3 vertices with p's screen
// barycentrics (dL/dv_i = lambda_i dL/dr), with FP64 atomics into grad_vpix (the
// per-pixel terms are FP32; the sums over pixels are kept in FP64).
#include <cuda_runtime.h>

#include "mer_device.cuh"

namespace mer {

constexpr int kBT = 16;  // tile edge
constexpr int kHalo = kBT + 2;

struct BwdArgs {
    mer_shading sh;
    int terms;
    int n, H, W, V, T;
    int ntx, nty;
};

// Vertex records of triangle t; false (nothing read) if a vertex id is out of range.
__device__ __forceinline__ bool load_tri_xy(const mer_vertex* vb, const int* tris, int t, int V, int X[3], int Y[3],
                                            const mer_vertex** rec) {
    int id[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        id[k] = __ldg(tris + 3 * (size_t)t + k);
        if ((unsigned)id[k] >= (unsigned)V) return false;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const mer_vertex* r = vb + id[k];
        rec[k] = r;
        X[k] = r->X;
        Y[k] = r->Y;
    }
    return true;
}

// Plane normal (v1 - v0) x (v2 - v0) in (x_s, y_s, zeta) from accurate differences.
__device__ __forceinline__ void tri_normal(const mer_vertex* const r[3], float N[3]) {
    float e[2][3];
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        e[k - 1][0] = __int2float_rn(r[k]->X - r[0]->X) * (1.0f / 256.0f) + (r[k]->rx - r[0]->rx);
        e[k - 1][1] = __int2float_rn(r[k]->Y - r[0]->Y) * (1.0f / 256.0f) + (r[k]->ry - r[0]->ry);
        e[k - 1][2] = (r[k]->zeta - r[0]->zeta) + (r[k]->zeta_lo - r[0]->zeta_lo);
    }
    N[0] = diff_of_products(e[0][1], e[1][2], e[0][2], e[1][1]);
    N[1] = diff_of_products(e[0][2], e[1][0], e[0][0], e[1][2]);
    N[2] = diff_of_products(e[0][0], e[1][1], e[0][1], e[1][0]);
}

__global__ void __launch_bounds__(kBT* kBT) k_backward(const mer_vertex* __restrict__ vpix, const int* __restrict__ tris,
                                                      const int* __restrict__ index, const float* __restrict__ image,
                                                      const float* __restrict__ grad, const float* __restrict__ attr,
                                                      const float* __restrict__ tex, BwdArgs a,
                                                      double* __restrict__ grad_vpix, float* __restrict__ grad_attr,
                                                      void* ws) {
    __shared__ int sidx[kHalo][kHalo];
    const int tiles_per_view = a.ntx * a.nty;
    const int view = blockIdx.x / tiles_per_view;
    const int local = blockIdx.x % tiles_per_view;
    const int tx = local % a.ntx, ty = local / a.ntx;
    const size_t plane = (size_t)a.H * a.W;
    const int* idx_v = index + (size_t)view * plane;
    for (int i = threadIdx.x; i < kHalo * kHalo; i += kBT * kBT) {
        const int hy = i / kHalo, hx = i % kHalo;
        const int gx = tx * kBT + hx - 1, gy = ty * kBT + hy - 1;
        sidx[hy][hx] = (gx >= 0 && gx < a.W && gy >= 0 && gy < a.H) ? idx_v[(size_t)gy * a.W + gx] : -2;
    }
    __syncthreads();
    const int lx = threadIdx.x % kBT, ly = threadIdx.x / kBT;
    const int x = tx * kBT + lx, y = ty * kBT + ly;
    if (x >= a.W || y >= a.H) return;
    const int t = sidx[ly + 1][lx + 1];
    if (t < 0) return;  // background: no fragment of its own
    if (t >= a.T) {
        set_status(ws, kStatusRange);
        return;
    }
    const int C = a.sh.C;
    const size_t p = (size_t)view * plane + (size_t)y * a.W + x;
    const mer_vertex* vb = vpix + (size_t)view * a.V;
    int X[3], Y[3], vid[3];
    const mer_vertex* rv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) vid[k] = __ldg(tris + 3 * (size_t)t + k);
    if (!load_tri_xy(vb, tris, t, a.V, X, Y, rv)) {
        set_status(ws, kStatusRange);
        return;
    }
    const Bary B = screen_bary(rv, x, y);
    float g[kMaxC], img[kMaxC];
#pragma unroll
    for (int c = 0; c < kMaxC; ++c) {
        g[c] = c < C ? __ldg(grad + p * C + c) : 0.f;
        img[c] = 0.f;
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float hz[3] = {0.f, 0.f, 0.f};

    if (a.terms & MER_INTERIOR) {
        const float z[3] = {rv[0]->zeta, rv[1]->zeta, rv[2]->zeta};
        const float s = B.lam[0] * z[0] + B.lam[1] * z[1] + B.lam[2] * z[2];
        const float is = 1.0f / s;
        float b[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k] = B.lam[k] * z[k] * is;
        // G_k = dL/db_k.  Only the differences G_k - G_i enter (sum_i b_i = 1), so they are formed
        // from attribute differences: D01 = G_0 - G_1, D02 = G_0 - G_2, D12 = G_1 - G_2.
        float D01 = 0.f, D02 = 0.f, D12 = 0.f;
        const int Ca = a.sh.C_attr;
        if (a.sh.uv_offset < 0) {
            for (int c = 0; c < a.sh.n_main; ++c) {
                const float a0 = __ldg(attr + (size_t)vid[0] * Ca + c);
                const float a1 = __ldg(attr + (size_t)vid[1] * Ca + c);
                const float a2 = __ldg(attr + (size_t)vid[2] * Ca + c);
                D01 += g[c] * (a0 - a1);
                D02 += g[c] * (a0 - a2);
                D12 += g[c] * (a1 - a2);
            }
            if (grad_attr) {
                for (int k = 0; k < 3; ++k)
                    for (int c = 0; c < a.sh.n_main; ++c) atomicAdd(grad_attr + (size_t)vid[k] * Ca + c, b[k] * g[c]);
            }
        } else {
            float uk[3], vk[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                uk[k] = __ldg(attr + (size_t)vid[k] * Ca + a.sh.uv_offset);
                vk[k] = __ldg(attr + (size_t)vid[k] * Ca + a.sh.uv_offset + 1);
            }
            const TexCoord cx = tex_coord(uk[0], uk[1], uk[2], b[1], b[2], a.sh.tex_w);
            const TexCoord cy = tex_coord(vk[0], vk[1], vk[2], b[1], b[2], a.sh.tex_h);
            float val[kMaxC], du[kMaxC], dv[kMaxC];
            tex_sample(tex, a.sh.tex_h, a.sh.tex_w, a.sh.n_main, cx, cy, val, du, dv);
            float gu = 0.f, gv = 0.f;
            for (int c = 0; c < a.sh.n_main; ++c) {
                gu += g[c] * du[c];
                gv += g[c] * dv[c];
            }
            D01 = gu * (uk[0] - uk[1]) + gv * (vk[0] - vk[1]);
            D02 = gu * (uk[0] - uk[2]) + gv * (vk[0] - vk[2]);
            D12 = gu * (uk[1] - uk[2]) + gv * (vk[1] - vk[2]);
            if (grad_attr) {
                for (int k = 0; k < 3; ++k) {
                    atomicAdd(grad_attr + (size_t)vid[k] * Ca + a.sh.uv_offset, b[k] * gu);
                    atomicAdd(grad_attr + (size_t)vid[k] * Ca + a.sh.uv_offset + 1, b[k] * gv);
                }
            }
        }
        // G_k - Gbar = sum_i b_i (G_k - G_i)
        const float GmG[3] = {b[1] * D01 + b[2] * D02, b[2] * D12 - b[0] * D01, -(b[0] * D02 + b[1] * D12)};
        const float gZ = a.sh.depth_ch >= 0 ? g[a.sh.depth_ch] : 0.f;
        // w = sum_k (dL/d lambda_k) grad lambda_k with dL/d lambda_k = zeta_k is (GmG_k - gZ is).  The depth
        // part -gZ is^2 sum_k zeta_k grad lambda_k equals -gZ is^2 sum_k (zeta_k - zeta_0) grad lambda_k
        // (the gradients sum to zero); the zeta differences come from the hi + lo split, so the near
        // cancellation of an almost constant zeta across the triangle costs no accuracy.
        const float dz1 = (z[1] - z[0]) + (rv[1]->zeta_lo - rv[0]->zeta_lo);
        const float dz2 = (z[2] - z[0]) + (rv[2]->zeta_lo - rv[0]->zeta_lo);
        float wx = 0.f, wy = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            hz[k] = is * (GmG[k] - gZ * is);  // (dL/d zeta_k) / lambda_k
            const float dl = z[k] * is * GmG[k];
            wx += dl * B.gx[k];
            wy += dl * B.gy[k];
        }
        const float dep = gZ * is * is;
        wx -= dep * (dz1 * B.gx[1] + dz2 * B.gx[2]);
        wy -= dep * (dz1 * B.gy[1] + dz2 * B.gy[2]);
        fx -= wx;
        fy -= wy;
    }

    if (a.terms & MER_EDGE) {
        bool own_loaded = false;
        const int ddx[4] = {-1, 1, 0, 0}, ddy[4] = {0, 0, -1, 1};
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int tq = sidx[ly + 1 + ddy[d]][lx + 1 + ddx[d]];
            if (tq == t || tq == -2) continue;
            const int qx = x + ddx[d], qy = y + ddy[d];
            const int axis = ddx[d] != 0 ? 0 : 1;
            bool inter = false;
            int Xq[3], Yq[3];
            const mer_vertex* rq[3];
            if (tq >= 0) {
                if (tq >= a.T) {
                    set_status(ws, kStatusRange);
                    continue;
                }
                if (!load_tri_xy(vb, tris, tq, a.V, Xq, Yq, rq)) {
                    set_status(ws, kStatusRange);
                    continue;
                }
                const bool q_in_t = covers_pts(X, Y, 256 * qx + 128, 256 * qy + 128);
                const bool p_in_q = covers_pts(Xq, Yq, 256 * x + 128, 256 * y + 128);
                if (!p_in_q) continue;  // adjacent, or q's triangle on top: p's fragment gets nothing
                if (q_in_t) {
                    if (!(a.terms & MER_INTERSECT)) continue;
                    inter = true;
                }
            }
            // Eq. 11 with A = left/top pixel, B = right/bottom pixel
            if (!own_loaded) {
                for (int c = 0; c < C; ++c) img[c] = __ldg(image + p * C + c);
                own_loaded = true;
            }
            const size_t q = (size_t)view * plane + (size_t)qy * a.W + qx;
            const bool p_is_a = ddx[d] > 0 || ddy[d] > 0;
            float dLdp = 0.f;
            for (int c = 0; c < C; ++c) {
                const float gq = __ldg(grad + q * C + c), iq = __ldg(image + q * C + c);
                const float diff = p_is_a ? (img[c] - iq) : (iq - img[c]);
                dLdp += 0.5f * (g[c] + gq) * diff;
            }
            if (!inter) {
                if (axis == 0) fx += dLdp; else fy += dLdp;
                continue;
            }
            // Eq. 12: p's triangle varies (v), q's triangle is fixed (f), slice (axis, zeta)
            float Nv[3], Nf[3];
            tri_normal(rv, Nv);
            tri_normal(rq, Nf);
            const float nv0 = Nv[axis], nv1 = Nv[2], nf0 = Nf[axis], nf1 = Nf[2];
            const float den = diff_of_products(nf0, nv1, nf1, nv0);
            const float mag = sqrtf((nv0 * nv0 + nv1 * nv1) * (nf0 * nf0 + nf1 * nf1));
            if (!(fabsf(den) > 1e-12f * mag)) continue;
            const float k = dLdp * (-nf1 / den);
            if (axis == 0) fx += k * nv0; else fy += k * nv0;
            fz += k * nv1;
        }
    }

    double* gv = grad_vpix + (size_t)view * a.V * 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float l = B.lam[k];
        const float cx = l * fx, cy = l * fy, cz = l * (fz + hz[k]);
        if (cx != 0.f) atomicAdd(gv + 3 * (size_t)vid[k], (double)cx);
        if (cy != 0.f) atomicAdd(gv + 3 * (size_t)vid[k] + 1, (double)cy);
        if (cz != 0.f) atomicAdd(gv + 3 * (size_t)vid[k] + 2, (double)cz);
    }
}

}  // namespace mer

using namespace mer;

extern "C" int mer_launch_backward(const mer_vertex* vpix, int V, const int* tris, int T, int n, int H, int W,
                                   const int* index, const float* image, const float* grad_image, const float* attr,
                                   const float* tex, const mer_shading* sh, int terms, double* grad_vpix,
                                   float* grad_attr, void* ws, cudaStream_t s) {
    BwdArgs a;
    a.sh = *sh;
    a.terms = terms;
    a.n = n; a.H = H; a.W = W; a.V = V; a.T = T;
    a.ntx = (W + kBT - 1) / kBT;
    a.nty = (H + kBT - 1) / kBT;
    const long long blocks = (long long)a.ntx * a.nty * n;
    if (blocks == 0) return 0;
    k_backward<<<(unsigned)blocks, kBT * kBT, 0, s>>>(vpix, tris, index, image, grad_image, attr, tex, a, grad_vpix,
                                                     grad_attr, ws);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
