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
    const float is = 1.0f / s;
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

}  // namespace mer
