// shade_device.cuh -- per-fragment shading shared by the deferred shading kernels and the fused raster +
// shade pass: perspective-correct barycentrics of the pixel centre, interpolated attributes or a bilinear
// texture lookup at the interpolated uv, coverage mask and depth (Supp. B, barycentrics and interpolation
// modules).
#pragma once

#include <cstdint>

#include "mer_device.cuh"

namespace mer {

struct ShadeArgs {
    mer_shading sh;
    float bg[kMaxC];
    int tex_stride;  // floats per texel
    bool tex_vec4;   // stride 4 and 16-byte aligned: 128-bit texel loads
};

inline ShadeArgs make_shade_args(const float* tex, const float* bg, const mer_shading* sh) {
    ShadeArgs a;
    a.sh = *sh;
    for (int c = 0; c < kMaxC; ++c) a.bg[c] = (bg && c < sh->C) ? bg[c] : 0.f;
    a.tex_stride = sh->tex_c > 0 ? sh->tex_c : sh->n_main;
    a.tex_vec4 = a.tex_stride == 4 && tex && (reinterpret_cast<uintptr_t>(tex) & 15u) == 0;
    return a;
}

// The C channels of pixel (x, y) covered by triangle t (t < 0: background), written to o[0..C).  vb / tris /
// attr are the item's bases.
__device__ __forceinline__ void shade_fragment(const mer_vertex* __restrict__ vb, int V, const int* __restrict__ tris,
                                               int T, int t, int x, int y, const float* __restrict__ attr,
                                               const float* __restrict__ tex, const ShadeArgs& a,
                                               float* __restrict__ o, void* ws) {
    const int C = a.sh.C;
    if (t >= T) set_status(ws, kStatusRange);
    int i0 = 0, i1 = 0, i2 = 0;
    bool ok = t >= 0 && t < T;
    if (ok) {
        i0 = tris[3 * (size_t)t];
        i1 = tris[3 * (size_t)t + 1];
        i2 = tris[3 * (size_t)t + 2];
        if ((unsigned)i0 >= (unsigned)V || (unsigned)i1 >= (unsigned)V || (unsigned)i2 >= (unsigned)V) {
            set_status(ws, kStatusRange);
            ok = false;
        }
    }
    if (!ok) {
#pragma unroll
        for (int c = 0; c < kMaxC; ++c)  // static indices keep the arguments out of local memory
            if (c < C) o[c] = a.bg[c];
        return;
    }
    const VRec v[3] = {load_vrec(vb + i0), load_vrec(vb + i1), load_vrec(vb + i2)};
    const int vid[3] = {i0, i1, i2};
    const Bary B = screen_bary(v, x, y);
    float b[3];
    const float s = B.lam[0] * v[0].zeta + B.lam[1] * v[1].zeta + B.lam[2] * v[2].zeta;
    const float is = rcp_nr(s);
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] = B.lam[k] * v[k].zeta * is;
    const int Ca = a.sh.C_attr;
    if (a.sh.uv_offset < 0) {
        for (int c = 0; c < a.sh.n_main; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc += b[k] * __ldg(attr + (size_t)vid[k] * Ca + c);
            o[c] = acc;
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
        const TexTaps taps = tex_taps(a.sh.tex_h, a.sh.tex_w, cx, cy);
        if (a.sh.n_main <= 4) {
            float v4[4];
            tex_values(tex, a.sh.tex_w, a.tex_stride, a.tex_vec4, a.sh.n_main, taps, v4);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < a.sh.n_main) o[c] = v4[c];
        } else {
            float vk_[kMaxC];
            tex_values(tex, a.sh.tex_w, a.tex_stride, false, a.sh.n_main, taps, vk_);
            for (int c = 0; c < a.sh.n_main && c < kMaxC; ++c) o[c] = vk_[c];
        }
    }
    if (a.sh.mask_ch >= 0) o[a.sh.mask_ch] = 1.0f;
    if (a.sh.depth_ch >= 0) o[a.sh.depth_ch] = is;
    if (a.sh.backface_ch >= 0) {
        // back-face image: the exact sign of the snapped screen area (positive = facing away, y down)
        const int64_t area = (int64_t)(v[1].X - v[0].X) * (v[2].Y - v[0].Y) - (int64_t)(v[1].Y - v[0].Y) * (v[2].X - v[0].X);
        o[a.sh.backface_ch] = area > 0 ? 1.0f : 0.0f;
    }
}

// ---- FP64 counterparts: the precise shading option and the deterministic backward ----

// Screen barycentrics of the pixel centre and their screen gradients in FP64.  The vertex position relative
// to the centre, (X - P)/256 + rx, is formed from the exact integer difference and the FP32 residual.
struct DBary {
    double lam[3];
    double gx[3], gy[3];  // d lambda_i / d P_x, d lambda_i / d P_y
    double d;             // twice the signed area
};

__device__ __forceinline__ DBary screen_bary_f64(const VRec v[3], int x, int y) {
    const int pxf = 256 * x + 128, pyf = 256 * y + 128;
    double ax[3], ay[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ax[i] = (double)(v[i].X - pxf) * (1.0 / 256.0) + (double)v[i].rx;
        ay[i] = (double)(v[i].Y - pyf) * (1.0 / 256.0) + (double)v[i].ry;
    }
    double e[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        e[i] = ax[j] * ay[k] - ay[j] * ax[k];
    }
    DBary B;
    B.d = (e[0] + e[1]) + e[2];
    const double inv = 1.0 / B.d;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        B.lam[i] = e[i] * inv;
        B.gx[i] = (ay[j] - ay[k]) * inv;
        B.gy[i] = (ax[k] - ax[j]) * inv;
    }
    return B;
}

__device__ __forceinline__ double zeta_f64(const VRec& v) { return (double)v.zeta + (double)v.zeta_lo; }

// Texel coordinate x = u N - 1/2 of u = u0 + b1 (u1 - u0) + b2 (u2 - u0) in FP64, split into cell and
// fraction; the base u0 N - 1/2 and its integer part are exact, the offset carries the rounding.
// Non-finite or |u| >= 1024 samples at u = 0.
struct DTexCoord {
    long long cell;
    double frac;
};

__device__ __forceinline__ DTexCoord tex_coord_f64(float u0, float u1, float u2, double b1, double b2, int N) {
    const double U0 = u0, U1 = u1, U2 = u2, Nd = (double)N;
    const double u = U0 + (b1 * (U1 - U0) + b2 * (U2 - U0));
    DTexCoord t;
    if (!(fabs(u) < 1024.0)) {
        t.cell = -1;
        t.frac = 0.5;
        return t;
    }
    const double xb = U0 * Nd - 0.5;
    const double fl = floor(xb);
    const double f = (xb - fl) + (b1 * (U1 * Nd - U0 * Nd) + b2 * (U2 * Nd - U0 * Nd));
    const double ci = floor(f);
    t.cell = (long long)fl + (long long)ci;
    t.frac = f - ci;
    return t;
}

// Bilinear taps of FP64 texel coordinates: u wraps, v clamps to the edge texels (a clamped v has zero
// derivative), as tex_taps.
struct DTexTaps {
    int i0, i1, j0, j1;
    double fx, fy;
    bool clamped;
};

__device__ __forceinline__ DTexTaps tex_taps_f64(int TH, int TW, DTexCoord cx, DTexCoord cy) {
    DTexTaps t;
    long long i0 = cx.cell % TW;
    if (i0 < 0) i0 += TW;
    t.i0 = (int)i0;
    t.i1 = (t.i0 + 1 == TW) ? 0 : t.i0 + 1;
    t.fx = cx.frac;
    t.clamped = false;
    if (cy.cell < 0) {
        t.j0 = 0; t.j1 = TH > 1 ? 1 : 0; t.fy = 0.0; t.clamped = true;
    } else if (cy.cell > TH - 1 || (cy.cell == TH - 1 && cy.frac > 0.0)) {
        t.j0 = TH - 1; t.j1 = TH - 1; t.fy = 0.0; t.clamped = true;
    } else {
        t.j0 = (int)cy.cell; t.j1 = t.j0 + 1 < TH ? t.j0 + 1 : TH - 1; t.fy = cy.frac;
    }
    return t;
}

__device__ __forceinline__ double texel_f64(const float* __restrict__ tex, int TW, int stride, int j, int i, int c) {
    return (double)__ldg(tex + ((size_t)j * TW + i) * stride + c);
}

// Bilinear value of channel c in FP64.
__device__ __forceinline__ double tex_value_f64(const float* __restrict__ tex, int TW, int stride, const DTexTaps& t,
                                                int c) {
    const double t00 = texel_f64(tex, TW, stride, t.j0, t.i0, c), t10 = texel_f64(tex, TW, stride, t.j0, t.i1, c);
    const double t01 = texel_f64(tex, TW, stride, t.j1, t.i0, c), t11 = texel_f64(tex, TW, stride, t.j1, t.i1, c);
    const double a = t00 + t.fx * (t10 - t00);
    const double b = t01 + t.fx * (t11 - t01);
    return a + t.fy * (b - a);
}

// sum_c g_c dT_c/du and sum_c g_c dT_c/dv in FP64 (g: the pixel's upstream gradient, nc channels).
__device__ __forceinline__ void tex_grad_uv_f64(const float* __restrict__ tex, int TH, int TW, int stride, int nc,
                                                const DTexTaps& t, const float* __restrict__ g, double& gu,
                                                double& gv) {
    double su = 0.0, sv = 0.0;
    for (int c = 0; c < nc; ++c) {
        const double t00 = texel_f64(tex, TW, stride, t.j0, t.i0, c), t10 = texel_f64(tex, TW, stride, t.j0, t.i1, c);
        const double t01 = texel_f64(tex, TW, stride, t.j1, t.i0, c), t11 = texel_f64(tex, TW, stride, t.j1, t.i1, c);
        const double gc = (double)__ldg(g + c);
        su += gc * ((1.0 - t.fy) * (t10 - t00) + t.fy * (t11 - t01));
        const double a = t00 + t.fx * (t10 - t00);
        const double b = t01 + t.fx * (t11 - t01);
        sv += gc * (b - a);
    }
    gu = (double)TW * su;
    gv = t.clamped ? 0.0 : (double)TH * sv;
}

// shade_fragment with FP64 arithmetic and one rounding per output value (the precise shading option).
__device__ __forceinline__ void shade_fragment_f64(const mer_vertex* __restrict__ vb, int V,
                                                   const int* __restrict__ tris, int T, int t, int x, int y,
                                                   const float* __restrict__ attr, const float* __restrict__ tex,
                                                   const ShadeArgs& a, float* __restrict__ o, void* ws) {
    const int C = a.sh.C;
    if (t >= T) set_status(ws, kStatusRange);
    int vid[3] = {0, 0, 0};
    bool ok = t >= 0 && t < T;
    if (ok) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            vid[k] = tris[3 * (size_t)t + k];
            if ((unsigned)vid[k] >= (unsigned)V) ok = false;
        }
        if (!ok) set_status(ws, kStatusRange);
    }
    if (!ok) {
#pragma unroll
        for (int c = 0; c < kMaxC; ++c)
            if (c < C) o[c] = a.bg[c];
        return;
    }
    const VRec v[3] = {load_vrec(vb + vid[0]), load_vrec(vb + vid[1]), load_vrec(vb + vid[2])};
    const DBary B = screen_bary_f64(v, x, y);
    const double z[3] = {zeta_f64(v[0]), zeta_f64(v[1]), zeta_f64(v[2])};
    const double s = B.lam[0] * z[0] + B.lam[1] * z[1] + B.lam[2] * z[2];
    const double is = 1.0 / s;
    double b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] = B.lam[k] * z[k] * is;
    const int Ca = a.sh.C_attr;
    if (a.sh.uv_offset < 0) {
        for (int c = 0; c < a.sh.n_main; ++c) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc += b[k] * (double)__ldg(attr + (size_t)vid[k] * Ca + c);
            o[c] = __double2float_rn(acc);
        }
    } else {
        float uk[3], vk[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uk[k] = __ldg(attr + (size_t)vid[k] * Ca + a.sh.uv_offset);
            vk[k] = __ldg(attr + (size_t)vid[k] * Ca + a.sh.uv_offset + 1);
        }
        const DTexCoord cx = tex_coord_f64(uk[0], uk[1], uk[2], b[1], b[2], a.sh.tex_w);
        const DTexCoord cy = tex_coord_f64(vk[0], vk[1], vk[2], b[1], b[2], a.sh.tex_h);
        const DTexTaps taps = tex_taps_f64(a.sh.tex_h, a.sh.tex_w, cx, cy);
        for (int c = 0; c < a.sh.n_main && c < kMaxC; ++c)
            o[c] = __double2float_rn(tex_value_f64(tex, a.sh.tex_w, a.tex_stride, taps, c));
    }
    if (a.sh.mask_ch >= 0) o[a.sh.mask_ch] = 1.0f;
    if (a.sh.depth_ch >= 0) o[a.sh.depth_ch] = __double2float_rn(is);
    if (a.sh.backface_ch >= 0) {
        const int64_t area = (int64_t)(v[1].X - v[0].X) * (v[2].Y - v[0].Y) - (int64_t)(v[1].Y - v[0].Y) * (v[2].X - v[0].X);
        o[a.sh.backface_ch] = area > 0 ? 1.0f : 0.0f;
    }
}

}  // namespace mer
