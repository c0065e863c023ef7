// backward_det.cu -- the deterministic option of the backward pass (MER_DETERMINISTIC): the micro-edge term
// (Eq. 11, the Sec. 4.3 classification, Eq. 12 at intersections) and the interior term (Eq. 5) with every
// per-pixel quantity in FP64, and sums that do not depend on the order of the additions.
//
// One thread per pixel p of the index image.  If p is covered by triangle t, the thread forms the gradient
// of p's fragment (a 3-vector in x_s, y_s, zeta) from the interior term and from the pairs with its four
// neighbours in which p's fragment scatters, gathers it to t's vertices with p's screen barycentrics, and
// rounds each of the nine vertex contributions (and the attribute-gradient ones) once to a 64-bit
// fixed-point number with 52 fractional bits, held as two 64-bit integers (a part with 20 fractional bits
// and the non-negative remainder in units of 2^-52).  Integer sums are exact, so the warp's run sums (a
// segmented scan over equal triangles) and the 64-bit integer atomics into the fixed-point accumulators give
// the same bits in any order.  A last pass adds the accumulators to grad_vpix (FP64) and grad_attr (FP32).
// The per-pixel formulas are those of the default path in backward.cu, evaluated in FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "shade_device.cuh"

namespace mer {
namespace {

// A contribution v (|v| < 2^33) is split exactly into hi = floor(v 2^20) and lo = round((v - hi 2^-20) 2^52)
// in [0, 2^32]: v = hi 2^-20 + lo 2^-52 to within 2^-53.
constexpr double kHiScale = 1048576.0;                 // 2^20
constexpr double kHiInv = 1.0 / 1048576.0;
constexpr double kLoScale = 4503599627370496.0;        // 2^52
constexpr double kLoInv = 1.0 / 4503599627370496.0;
constexpr double kFixLimit = 8589934592.0;             // 2^33: largest contribution kept
constexpr int kDetThreads = 256;
constexpr int kDetMaxA = 4;                  // attribute-gradient channels carried

struct DetArgs {
    mer_shading sh;
    int terms;
    int tex_stride;
    int A;   // attribute-gradient channels (0: none)
    int a0;  // first attribute channel they belong to
};

// One item: a mesh seen by one camera.
struct DetItem {
    const mer_vertex* vb;
    const int* tris;
    const int* index;
    const float* image;
    const float* grad;
    const float* attr;
    unsigned long long* acc_v;  // [V, 3] fixed point (the item's vertex-record rows)
    unsigned long long* acc_a;  // [V, A] fixed point (the item's mesh rows) or null
    int V, T, H, W;
};

struct Fix {
    long long hi, lo;
};

__device__ __forceinline__ Fix to_fixed(double v, void* ws) {
    Fix f;
    f.hi = 0;
    f.lo = 0;
    if (!(fabs(v) < kFixLimit)) {
        set_status(ws, kStatusFixed);
        return f;
    }
    const double h = floor(v * kHiScale);  // exact: v 2^20 scales by a power of two
    f.hi = (long long)h;
    f.lo = __double2ll_rn((v - h * kHiInv) * kLoScale);  // v - h 2^-20 is exact and lies in [0, 2^-20)
    return f;
}

__device__ __forceinline__ void fix_add(Fix& a, const Fix& b) {
    a.hi += b.hi;
    a.lo += b.lo;
}

// The value of a sum of fixed-point numbers (the carry of the low word folded into the high word first).
__device__ __forceinline__ double fix_value(long long hi, long long lo) {
    const long long h = hi + (lo >> 32);
    const long long l = lo & 0xffffffffll;
    return (double)h * kHiInv + (double)l * kLoInv;
}

// Crossing position u in [0, 1] along the edge v_j -> v_l measured on axis o (the axis orthogonal to the pair
// axis), in FP64 on the unsnapped geometry; 1/2 for an edge parallel to the pair axis.
__device__ __forceinline__ double crossing_u_f64(int Sj, float rj, int Sl, float rl, int Fo_snapped) {
    const double num = (double)(Fo_snapped - Sj) * (1.0 / 256.0) - (double)rj;
    const double den = (double)(Sl - Sj) * (1.0 / 256.0) + ((double)rl - (double)rj);
    double u = den != 0.0 ? num / den : 0.5;
    return fmin(fmax(u, 0.0), 1.0);
}

// (v1 - v0) x (v2 - v0) in (x_s, y_s, zeta), FP64.
__device__ __forceinline__ void tri_normal_f64(const VRec r[3], double N[3]) {
    double e[2][3];
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        e[k - 1][0] = (double)(r[k].X - r[0].X) * (1.0 / 256.0) + ((double)r[k].rx - (double)r[0].rx);
        e[k - 1][1] = (double)(r[k].Y - r[0].Y) * (1.0 / 256.0) + ((double)r[k].ry - (double)r[0].ry);
        e[k - 1][2] = zeta_f64(r[k]) - zeta_f64(r[0]);
    }
    N[0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
    N[1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
    N[2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
}

__device__ __forceinline__ bool ids_of(const int* __restrict__ tris, int t, int V, int id[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        id[k] = __ldg(tris + 3 * (size_t)t + k);
        if ((unsigned)id[k] >= (unsigned)V) return false;
    }
    return true;
}

// The contributions of pixel (x, y) of an item: returns its triangle (or -1) with its vertex ids and the
// fixed-point contributions cv[k][c] to vertex k's gradient component c and ca[k][j] to its attribute
// gradient channel j.
__device__ int det_pixel(const DetItem& it, const DetArgs& a, const float* __restrict__ tex, int x, int y, void* ws,
                         int vid[3], Fix cv[3][3], Fix ca[3][kDetMaxA]) {
    const size_t p = (size_t)y * it.W + x;
    int t = __ldg(it.index + p);
    if (t < 0) return -1;
    if (t >= it.T || !ids_of(it.tris, t, it.V, vid)) {
        set_status(ws, kStatusRange);
        return -1;
    }
    const int C = a.sh.C;
    const VRec rv[3] = {load_vrec(it.vb + vid[0]), load_vrec(it.vb + vid[1]), load_vrec(it.vb + vid[2])};
    const DBary B = screen_bary_f64(rv, x, y);
    const float* gp = it.grad + p * C;
    double f[3] = {0.0, 0.0, 0.0};             // fragment gradient dL/dr (x_s, y_s, zeta)
    double hz[3] = {0.0, 0.0, 0.0};            // interior zeta derivative of vertex k over lambda_k
    double ev[3][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};  // exact-crossing parts per vertex (x, y)
    double cat[3][kDetMaxA];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < kDetMaxA; ++j) cat[k][j] = 0.0;

    if (a.terms & MER_INTERIOR) {
        const double z[3] = {zeta_f64(rv[0]), zeta_f64(rv[1]), zeta_f64(rv[2])};
        const double s = B.lam[0] * z[0] + B.lam[1] * z[1] + B.lam[2] * z[2];
        const double is = 1.0 / s;
        double b[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k] = B.lam[k] * z[k] * is;
        // G_k = dL/db_k enters through its differences (sum_k b_k = 1)
        double D01 = 0.0, D02 = 0.0, D12 = 0.0;
        const int Ca = a.sh.C_attr;
        if (a.sh.uv_offset < 0) {
            for (int c = 0; c < a.sh.n_main; ++c) {
                const double gc = (double)__ldg(gp + c);
                const double a0 = __ldg(it.attr + (size_t)vid[0] * Ca + c);
                const double a1 = __ldg(it.attr + (size_t)vid[1] * Ca + c);
                const double a2 = __ldg(it.attr + (size_t)vid[2] * Ca + c);
                D01 += gc * (a0 - a1);
                D02 += gc * (a0 - a2);
                D12 += gc * (a1 - a2);
                if (c < a.A && c < kDetMaxA) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) cat[k][c] = b[k] * gc;
                }
            }
        } else {
            float uk[3], vk[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                uk[k] = __ldg(it.attr + (size_t)vid[k] * Ca + a.sh.uv_offset);
                vk[k] = __ldg(it.attr + (size_t)vid[k] * Ca + a.sh.uv_offset + 1);
            }
            const DTexCoord cx = tex_coord_f64(uk[0], uk[1], uk[2], b[1], b[2], a.sh.tex_w);
            const DTexCoord cy = tex_coord_f64(vk[0], vk[1], vk[2], b[1], b[2], a.sh.tex_h);
            const DTexTaps taps = tex_taps_f64(a.sh.tex_h, a.sh.tex_w, cx, cy);
            double gu, gv;
            tex_grad_uv_f64(tex, a.sh.tex_h, a.sh.tex_w, a.tex_stride, a.sh.n_main, taps, gp, gu, gv);
            const double u0 = uk[0], u1 = uk[1], u2 = uk[2], v0 = vk[0], v1 = vk[1], v2 = vk[2];
            D01 = gu * (u0 - u1) + gv * (v0 - v1);
            D02 = gu * (u0 - u2) + gv * (v0 - v2);
            D12 = gu * (u1 - u2) + gv * (v1 - v2);
            if (a.A >= 2) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    cat[k][0] = b[k] * gu;
                    cat[k][1] = b[k] * gv;
                }
            }
        }
        const double GmG[3] = {b[1] * D01 + b[2] * D02, b[2] * D12 - b[0] * D01, -(b[0] * D02 + b[1] * D12)};
        const double gZ = a.sh.depth_ch >= 0 ? (double)__ldg(gp + a.sh.depth_ch) : 0.0;
        const double dz1 = z[1] - z[0], dz2 = z[2] - z[0];
        double wx = 0.0, wy = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            hz[k] = is * (GmG[k] - gZ * is);
            const double dl = z[k] * is * GmG[k];
            wx += dl * B.gx[k];
            wy += dl * B.gy[k];
        }
        const double dep = gZ * is * is;
        wx -= dep * (dz1 * B.gx[1] + dz2 * B.gx[2]);
        wy -= dep * (dz1 * B.gy[1] + dz2 * B.gy[2]);
        f[0] -= wx;
        f[1] -= wy;
    }

    if (a.terms & MER_EDGE) {
        int Xs[3], Ys[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Xs[k] = rv[k].X;
            Ys[k] = rv[k].Y;
        }
        const int pxs = 256 * x + 128, pys = 256 * y + 128;
        for (int d = 0; d < 4; ++d) {  // left, right, up, down: a fixed order
            const int ddx = d == 0 ? -1 : (d == 1 ? 1 : 0);
            const int ddy = d == 2 ? -1 : (d == 3 ? 1 : 0);
            const int qx = x + ddx, qy = y + ddy;
            if (qx < 0 || qx >= it.W || qy < 0 || qy >= it.H) continue;  // no pair across the image border
            const size_t q = (size_t)qy * it.W + qx;
            const int tq = __ldg(it.index + q);
            if (tq == t) continue;
            const int axis = ddx != 0 ? 0 : 1;
            bool inter = false;
            int vq[3] = {0, 0, 0};
            if (tq >= 0) {
                if (tq >= it.T || !ids_of(it.tris, tq, it.V, vq)) {
                    set_status(ws, kStatusRange);
                    continue;
                }
                int Xq[3], Yq[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int2 xy = __ldg(reinterpret_cast<const int2*>(it.vb + vq[k]));
                    Xq[k] = xy.x;
                    Yq[k] = xy.y;
                }
                // Sec. 4.3: p's fragment scatters only if p's centre lies inside q's triangle (p on top), or
                // both centres lie inside each other's triangles (an intersection)
                if (!covers_xy(Xq, Yq, pxs, pys)) continue;
                if (covers_xy(Xs, Ys, 256 * qx + 128, 256 * qy + 128)) {
                    if (!(a.terms & MER_INTERSECT)) continue;
                    inter = true;
                }
            }
            // Eq. 11 with A = the left / top pixel of the pair, B = the right / bottom one
            const float *gq = it.grad + q * C, *ip = it.image + p * C, *iq = it.image + q * C;
            const bool p_is_a = ddx > 0 || ddy > 0;
            double dLdp = 0.0;
            for (int c = 0; c < C; ++c) {
                const double diff = (double)__ldg(ip + c) - (double)__ldg(iq + c);
                dLdp += 0.5 * ((double)__ldg(gp + c) + (double)__ldg(gq + c)) * (p_is_a ? diff : -diff);
            }
            if (!inter) {
                if (a.terms & MER_EXACT_CROSSING) {
                    const int e = exit_edge(Xs, Ys, pxs, pys, 256 * qx + 128, 256 * qy + 128);
                    if (e >= 0) {
                        const int j = (e + 1) % 3, l = (e + 2) % 3;
                        const double u = axis == 0 ? crossing_u_f64(Ys[j], rv[j].ry, Ys[l], rv[l].ry, pys)
                                                   : crossing_u_f64(Xs[j], rv[j].rx, Xs[l], rv[l].rx, pxs);
                        ev[j][axis] += (1.0 - u) * dLdp;
                        ev[l][axis] += u * dLdp;
                        continue;
                    }
                }
                f[axis] += dLdp;
            } else {
                // Eq. 12 in the (axis, zeta) slice: p's triangle moves (v), q's is fixed (f)
                const VRec rq[3] = {load_vrec(it.vb + vq[0]), load_vrec(it.vb + vq[1]), load_vrec(it.vb + vq[2])};
                double Nv[3], Nf[3];
                tri_normal_f64(rv, Nv);
                tri_normal_f64(rq, Nf);
                const double nv0 = Nv[axis], nv1 = Nv[2], nf0 = Nf[axis], nf1 = Nf[2];
                const double den = nf0 * nv1 - nf1 * nv0;
                const double mag = sqrt((nv0 * nv0 + nv1 * nv1) * (nf0 * nf0 + nf1 * nf1));
                if (!(fabs(den) > 1e-12 * mag)) continue;
                const double kk = dLdp * (-nf1 / den);
                f[axis] += kk * nv0;
                f[2] += kk * nv1;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double l = B.lam[k];
        cv[k][0] = to_fixed(l * f[0] + ev[k][0], ws);
        cv[k][1] = to_fixed(l * f[1] + ev[k][1], ws);
        cv[k][2] = to_fixed(l * (f[2] + hz[k]), ws);
#pragma unroll
        for (int j = 0; j < kDetMaxA; ++j) {
            ca[k][j].hi = 0;
            ca[k][j].lo = 0;
            if (j < a.A) ca[k][j] = to_fixed(cat[k][j], ws);
        }
    }
    return t;
}

__device__ __forceinline__ void shfl_up_add(Fix& v, int dlt, bool take) {
    const unsigned full = 0xffffffffu;
    const long long h = __shfl_up_sync(full, v.hi, dlt);
    const long long l = __shfl_up_sync(full, v.lo, dlt);
    if (take) {
        v.hi += h;
        v.lo += l;
    }
}

__device__ __forceinline__ void atomic_fix(unsigned long long* p, const Fix& v) {
    if (v.hi != 0) atomicAdd(p, (unsigned long long)v.hi);
    if (v.lo != 0) atomicAdd(p + 1, (unsigned long long)v.lo);
}

// Adds the contributions of a warp's pixels: runs of lanes with the same (item, triangle) are summed by a
// segmented scan (exact integer sums) and each run's last lane adds the totals to the accumulators (two
// 64-bit words per component: the high and low parts).
__device__ __forceinline__ void det_warp_add(const DetItem& it, const DetArgs& a, int key_item, int t,
                                             const int vid[3], Fix cv[3][3], Fix ca[3][kDetMaxA]) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int tprev = __shfl_up_sync(full, t, 1), iprev = __shfl_up_sync(full, key_item, 1);
    const bool head = lane == 0 || tprev != t || iprev != key_item;
    const unsigned heads = __ballot_sync(full, head);
    const int seg = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    const bool with_attr = a.A > 0 && it.acc_a != nullptr;
#pragma unroll
    for (int dlt = 1; dlt < 32; dlt <<= 1) {
        const bool take = lane - dlt >= seg;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int c = 0; c < 3; ++c) shfl_up_add(cv[k][c], dlt, take);
            if (with_attr) {
#pragma unroll
                for (int j = 0; j < kDetMaxA; ++j) shfl_up_add(ca[k][j], dlt, take);
            }
        }
    }
    const int tnext = __shfl_down_sync(full, t, 1), inext = __shfl_down_sync(full, key_item, 1);
    const bool tail = lane == 31 || tnext != t || inext != key_item;
    if (!tail || t < 0) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) atomic_fix(it.acc_v + 2 * (3 * (size_t)vid[k] + c), cv[k][c]);
        if (with_attr) {
            for (int j = 0; j < a.A; ++j) atomic_fix(it.acc_a + 2 * ((size_t)vid[k] * a.A + j), ca[k][j]);
        }
    }
}

// Per-view launch: n views of one mesh, pixels of all views in order.
__global__ void __launch_bounds__(kDetThreads) k_backward_det(const mer_vertex* __restrict__ vpix,
                                                              const int* __restrict__ tris, const int* __restrict__ index,
                                                              const float* __restrict__ image,
                                                              const float* __restrict__ grad,
                                                              const float* __restrict__ attr,
                                                              const float* __restrict__ tex, DetArgs a, int n, int H,
                                                              int W, int V, int T, unsigned long long* acc_v,
                                                              unsigned long long* acc_a, void* ws) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long plane = (long long)H * W;
    const bool live = g < (long long)n * plane;
    const int view = live ? (int)(g / plane) : -1;
    const int rem = live ? (int)(g % plane) : 0;
    DetItem it;
    it.vb = vpix + (size_t)(view < 0 ? 0 : view) * V;
    it.tris = tris;
    it.index = index + (size_t)(view < 0 ? 0 : view) * plane;
    it.image = image ? image + (size_t)(view < 0 ? 0 : view) * plane * a.sh.C : nullptr;
    it.grad = grad + (size_t)(view < 0 ? 0 : view) * plane * a.sh.C;
    it.attr = attr;
    it.acc_v = acc_v + 6 * (size_t)(view < 0 ? 0 : view) * V;
    it.acc_a = acc_a;
    it.V = V; it.T = T; it.H = H; it.W = W;
    int vid[3] = {0, 0, 0};
    Fix cv[3][3] = {};
    Fix ca[3][kDetMaxA] = {};
    const int t = live ? det_pixel(it, a, tex, rem % W, rem / W, ws, vid, cv, ca) : -1;
    det_warp_add(it, a, view, t, vid, cv, ca);
}

// Batched launch: the pixels of all items in order (item.pix).
__global__ void __launch_bounds__(kDetThreads) k_backward_det_batch(const mer_vertex* __restrict__ vpix,
                                                                    const int* __restrict__ tris,
                                                                    const mer_item* __restrict__ items, int n_items,
                                                                    long long pixels, const int* __restrict__ index,
                                                                    const float* __restrict__ image,
                                                                    const float* __restrict__ grad,
                                                                    const float* __restrict__ attr,
                                                                    const float* __restrict__ tex, DetArgs a,
                                                                    unsigned long long* acc_v,
                                                                    unsigned long long* acc_a, void* ws) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = block_find_item(items, n_items, (long long)blockIdx.x * blockDim.x, g, kFieldPix);
    const bool live = g < pixels;
    const mer_item m = items[k];
    const int C = a.sh.C, Ca = a.sh.C_attr;
    DetItem it;
    it.vb = vpix + m.vrec;
    it.tris = tris + 3 * m.tri;
    it.index = index + m.pix;
    it.image = image ? image + (size_t)m.pix * C : nullptr;
    it.grad = grad + (size_t)m.pix * C;
    it.attr = attr ? attr + (size_t)m.vert * Ca : nullptr;
    it.acc_v = acc_v + 6 * (size_t)m.vrec;
    it.acc_a = acc_a ? acc_a + 2 * (size_t)m.vert * a.A : nullptr;
    it.V = m.V; it.T = m.T; it.H = m.H; it.W = m.W;
    int vid[3] = {0, 0, 0};
    Fix cv[3][3] = {};
    Fix ca[3][kDetMaxA] = {};
    int t = -1;
    if (live && m.W > 0) {
        const int rem = (int)(g - m.pix);
        t = det_pixel(it, a, tex, rem % m.W, rem / m.W, ws, vid, cv, ca);
    }
    det_warp_add(it, a, k, t, vid, cv, ca);
}

// grad_vpix += the accumulated sums (FP64); grad_attr[:, a0 + j] += those of acc_a (rounded to FP32).
__global__ void k_det_finalize(const unsigned long long* __restrict__ acc_v, long long nv, double* __restrict__ grad_vpix,
                               const unsigned long long* __restrict__ acc_a, long long arows, int A, int a0, int Ca,
                               float* __restrict__ grad_attr) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv) grad_vpix[i] += fix_value((long long)acc_v[2 * i], (long long)acc_v[2 * i + 1]);
    if (grad_attr && i < arows * A) {
        const long long r = i / A;
        const int j = (int)(i % A);
        grad_attr[(size_t)r * Ca + a0 + j] +=
            __double2float_rn(fix_value((long long)acc_a[2 * i], (long long)acc_a[2 * i + 1]));
    }
}

DetArgs det_args(const mer_shading* sh, int terms, const float* grad_attr) {
    DetArgs a;
    a.sh = *sh;
    a.terms = terms;
    a.tex_stride = sh->tex_c > 0 ? sh->tex_c : sh->n_main;
    a.A = grad_attr ? (sh->uv_offset < 0 ? sh->n_main : 2) : 0;
    a.a0 = sh->uv_offset < 0 ? 0 : sh->uv_offset;
    return a;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace mer

using namespace mer;

// 256-byte header, then two 64-bit words per vertex-gradient and per attribute-gradient component.
extern "C" size_t mer_det_workspace_size(long long vertex_rows, long long attr_rows, int attr_channels) {
    return 256 + round256((size_t)vertex_rows * 3 * 16) + round256((size_t)attr_rows * (size_t)attr_channels * 16);
}

namespace {
int det_finish(unsigned long long* acc_v, long long vrows, double* grad_vpix, unsigned long long* acc_a, long long arows,
               const DetArgs& a, float* grad_attr, cudaStream_t s) {
    const long long nv = 3 * vrows, na = grad_attr ? arows * a.A : 0;
    const long long m = nv > na ? nv : na;
    if (m > 0)
        k_det_finalize<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(acc_v, nv, grad_vpix, acc_a, arows, a.A, a.a0,
                                                                  a.sh.C_attr, grad_attr);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
}  // namespace

extern "C" int mer_launch_backward_det(const mer_vertex* vpix, int V, const int* tris, int T, int n, int H, int W,
                                       const int* index, const float* image, const float* grad_image, const float* attr,
                                       const float* tex, const mer_shading* sh, int terms, double* grad_vpix,
                                       float* grad_attr, void* ws, cudaStream_t s) {
    const DetArgs a = det_args(sh, terms, grad_attr);
    if (a.A > kDetMaxA) return 1;
    const long long vrows = (long long)n * V;
    char* base = static_cast<char*>(ws);
    unsigned long long* acc_v = reinterpret_cast<unsigned long long*>(base + 256);
    unsigned long long* acc_a = grad_attr ? reinterpret_cast<unsigned long long*>(base + 256 + round256((size_t)vrows * 48))
                                          : nullptr;
    const size_t bytes = mer_det_workspace_size(vrows, grad_attr ? V : 0, a.A) - 256;
    if (bytes > 0 && cudaMemsetAsync(acc_v, 0, bytes, s) != cudaSuccess) return 2;
    const long long npix = (long long)n * H * W;
    if (npix > 0)
        k_backward_det<<<(unsigned)((npix + kDetThreads - 1) / kDetThreads), kDetThreads, 0, s>>>(
            vpix, tris, index, image, grad_image, attr, tex, a, n, H, W, V, T, acc_v, acc_a, ws);
    if (cudaGetLastError() != cudaSuccess) return 2;
    return det_finish(acc_v, vrows, grad_vpix, acc_a, V, a, grad_attr, s);
}

extern "C" int mer_launch_backward_det_batch(const mer_vertex* vpix, const int* tris, const mer_item* items, int n_items,
                                             long long pixels, long long vrecs, long long mesh_rows, const int* index,
                                             const float* image, const float* grad_image, const float* attr,
                                             const float* tex, const mer_shading* sh, int terms, double* grad_vpix,
                                             float* grad_attr, void* ws, cudaStream_t s) {
    const DetArgs a = det_args(sh, terms, grad_attr);
    if (a.A > kDetMaxA) return 1;
    char* base = static_cast<char*>(ws);
    unsigned long long* acc_v = reinterpret_cast<unsigned long long*>(base + 256);
    unsigned long long* acc_a = grad_attr ? reinterpret_cast<unsigned long long*>(base + 256 + round256((size_t)vrecs * 48))
                                          : nullptr;
    const size_t bytes = mer_det_workspace_size(vrecs, grad_attr ? mesh_rows : 0, a.A) - 256;
    if (bytes > 0 && cudaMemsetAsync(acc_v, 0, bytes, s) != cudaSuccess) return 2;
    if (pixels > 0)
        k_backward_det_batch<<<(unsigned)((pixels + kDetThreads - 1) / kDetThreads), kDetThreads, 0, s>>>(
            vpix, tris, items, n_items, pixels, index, image, grad_image, attr, tex, a, acc_v, acc_a, ws);
    if (cudaGetLastError() != cudaSuccess) return 2;
    return det_finish(acc_v, vrecs, grad_vpix, acc_a, mesh_rows, a, grad_attr, s);
}
