// mer_device.cuh -- device-side building blocks shared by the kernels of libmer.
//
// Exact coverage (snapped int64 edge functions with the top-left rule), the
// FP32 depth key of the z-buffer, accurate screen barycentrics from the
// snapped-plus-residual vertex records, and the bilinear texture sampler.
#pragma once

#include <cstdint>

#include "../../include/mer.h"

namespace mer {

constexpr int kMaxDim = 8192;
constexpr double kGuard = 536870912.0;  // 2^29 (snapped units)
constexpr uint32_t kValid = 3u;         // in front of the near plane and inside the guard band
constexpr int kMaxC = 16;               // channels of a shaded image handled per pixel

// Workspace header, first 256 bytes of every workspace / status buffer.
struct WsHeader {
    int status;          // bit 0: bin overflow, bit 1: triangle / index out of range
    int pad0;
    long long total_bins;
    long long capacity;
    unsigned long long queue_raster;    // work-queue counters of the persistent kernels
    unsigned long long queue_backward;
    int pad[54];
};
static_assert(sizeof(WsHeader) == 256, "header");
constexpr int kStatusOverflow = 1;
constexpr int kStatusRange = 2;
constexpr int kStatusFixed = 4;  // a deterministic-mode contribution beyond the fixed-point range

// Backward tile: 32 x 16 pixels, one CTA of 8 warps (two rows each); the batch plan counts items in these.
constexpr int kBwdTileW = 32, kBwdTileH = 16;

// Per (view, triangle) raster record written by the binning pass, 64 bytes.
// A small triangle (flag bit 4: snapped box extent below 2^14) keeps its three edge functions instead of its
// vertices: with s the sign of the area and tl_i the top-left bit of edge i, X[i] x + Y[i] y + K[i] equals
// s e_i(pixel centre of (x, y)) + tl_i - 1 modulo 2^32 for pixel indices (x, y), and inside the box that value
// fits 31 bits, so the wrapped 32-bit evaluation is exact and the centre is covered iff all three are >= 0.
struct __align__(16) TriRaster {  // 16-byte aligned: copied with 128-bit loads and stores
    int X[3], Y[3];   // snapped vertex positions; small triangle: edge i's coefficients of x and y
    float zd[3];      // zeta_i / |E_0 + E_1 + E_2|, FP32
    int flags;        // bits 0..2: edge i is top-left; bit 3: negative area; bit 4: small (32-bit path); bit 31: culled
    short bx0, bx1, by0, by1;  // inclusive pixel bounding box of the covered centres
    float zmax;       // largest vertex zeta: no fragment of the triangle has a larger depth key
    int K[3];         // small triangle: edge i's constant term (unused otherwise)
};
static_assert(sizeof(TriRaster) == 64, "TriRaster");

__device__ __forceinline__ int64_t edge_fn(int xj, int yj, int xk, int yk, int px, int py) {
    // cross(v_j - P, v_k - P); every factor fits int32 (|X| <= 2^29, P < 2^22)
    return (int64_t)(xj - px) * (int64_t)(yk - py) - (int64_t)(yj - py) * (int64_t)(xk - px);
}

// Exact-crossing gather option (overhang pairs): the edge k (opposite vertex k) through which the segment from
// pixel centre F to pixel centre O (snapped units) leaves the triangle: among the edges with O on or beyond
// them (s E_k(O) <= 0, s the area sign) the one reached first, i.e. the smallest
// t_k = s E_k(F) / (s E_k(F) - s E_k(O)), compared exactly (128-bit products); ties go to the lower k.
// -1 if the triangle is degenerate or no edge qualifies.
__device__ __forceinline__ int exit_edge(const int X[3], const int Y[3], int Fx, int Fy, int Ox, int Oy) {
    const int64_t a2 = (int64_t)(X[1] - X[0]) * (Y[2] - Y[0]) - (int64_t)(Y[1] - Y[0]) * (X[2] - X[0]);
    if (a2 == 0) return -1;
    const int64_t sg = a2 > 0 ? 1 : -1;
    int best = -1;
    int64_t bnum = 0, bden = 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int j = (k + 1) % 3, l = (k + 2) % 3;
        const int64_t eF = sg * edge_fn(X[j], Y[j], X[l], Y[l], Fx, Fy);
        const int64_t eO = sg * edge_fn(X[j], Y[j], X[l], Y[l], Ox, Oy);
        if (eO > 0 || eF - eO <= 0) continue;
        if (best < 0 || (__int128)eF * bden < (__int128)bnum * (eF - eO)) {
            best = k;
            bnum = eF;
            bden = eF - eO;
        }
    }
    return best;
}

// Position u in [0, 1] of the crossing along the edge v_j -> v_l, measured on the axis o orthogonal to the
// pair axis (o = 1: y, for a horizontal pair): u = (F_o - v_j,o) / (v_l,o - v_j,o) on the unsnapped geometry
// (v = snapped/256 + residual), differences of the integer parts taken exactly; 1/2 for an edge parallel to
// the pair axis.  Fo_snapped = 256 * pixel + 128 on axis o.
__device__ __forceinline__ float crossing_u(int Sj, float rj, int Sl, float rl, int Fo_snapped) {
    const float num = (float)(Fo_snapped - Sj) * (1.0f / 256.0f) - rj;
    const float den = (float)(Sl - Sj) * (1.0f / 256.0f) + (rl - rj);
    float u = den != 0.0f ? num / den : 0.5f;
    return fminf(fmaxf(u, 0.0f), 1.0f);
}

// Exact coverage of the pixel centre (px, py) (snapped units) by a raster record.
__device__ __forceinline__ bool covers(const TriRaster& t, int px, int py, int64_t E[3]) {
    const bool neg = (t.flags & 8) != 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        int64_t e = edge_fn(t.X[j], t.Y[j], t.X[k], t.Y[k], px, py);
        E[i] = e;
        if (neg) e = -e;
        // covered iff e > 0, or e == 0 on a top-left edge: e + tl > 0
        if (e + (int64_t)((t.flags >> i) & 1) <= 0) return false;
    }
    return true;
}

// The same predicate for a "small" triangle (snapped bbox extent < 2^14) at the centre of pixel (x, y) inside
// its box, from the record's edge functions: |e_i| < 2^29 there, so the wrapped evaluation is exact.  E[i] is
// s e_i, as covers would give it after the sign flip.
__device__ __forceinline__ bool covers_small(const TriRaster& t, int x, int y, int E[3]) {
    int e[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        e[i] = (int)((unsigned)t.K[i] + (unsigned)t.X[i] * (unsigned)x + (unsigned)t.Y[i] * (unsigned)y);
    if ((e[0] | e[1] | e[2]) < 0) return false;  // covered iff s e_i + tl_i > 0 for every edge
#pragma unroll
    for (int i = 0; i < 3; ++i) E[i] = e[i] + 1 - ((t.flags >> i) & 1);
    return true;
}

// Same predicate from three vertex records (used by the classification).
__device__ __forceinline__ bool covers_pts(const int X[3], const int Y[3], int px, int py) {
    const int64_t a2 = (int64_t)(X[1] - X[0]) * (Y[2] - Y[0]) - (int64_t)(Y[1] - Y[0]) * (X[2] - X[0]);
    if (a2 == 0) return false;
    const int64_t s = a2 > 0 ? 1 : -1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        const int64_t e = s * edge_fn(X[j], Y[j], X[k], Y[k], px, py);
        if (e > 0) continue;
        if (e < 0) return false;
        const int64_t ga = s * (int64_t)(Y[j] - Y[k]);
        const int64_t gb = s * (int64_t)(X[k] - X[j]);
        if (!(ga > 0 || (ga == 0 && gb > 0))) return false;
    }
    return true;
}

// int64 -> float, round to nearest even, with integer instructions only (the hardware conversion of a
// 64-bit integer runs on the FP64 pipe, which is narrow on GB300).  Normalise so the leading one is bit
// 63, keep 24 bits, round on the next 8 bits plus a sticky bit for everything below.
__device__ __forceinline__ float ll2f_rn(long long v) {
    if (v == 0) return 0.0f;
    unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)a);
    a <<= lz;
    const unsigned top = (unsigned)(a >> 32);
    const bool sticky = (unsigned)a != 0u;
    unsigned m = top >> 8;
    const unsigned rem = top & 0xFFu;
    if (rem > 0x80u || (rem == 0x80u && (sticky || (m & 1u)))) ++m;
    unsigned e = 127u + 63u - (unsigned)lz;
    if (m >> 24) {
        m >>= 1;
        ++e;
    }
    return __uint_as_float((e << 23) | (m & 0x7FFFFFu) | (v < 0 ? 0x80000000u : 0u));
}

// int -> float (exact below 2^24 in magnitude, correctly rounded above), and floor(x) as an int (saturating,
// 0 for NaN): single hardware conversions.  They issue on the conversion pipe, which these kernels leave
// mostly idle; the bias tricks they replaced took four to six issue slots on the busy FP32 and integer pipes
// (measured: backward and fused raster 2-4 % faster with the same results).
__device__ __forceinline__ float i2f_exact(int v) { return __int2float_rn(v); }

__device__ __forceinline__ int floor_i(float x) { return __float2int_rd(x); }

// 1 / x: the hardware's approximate reciprocal r0 (about one ulp) refined by one Newton-Raphson step,
// r1 = r0 + r0 (1 - x r0) with both operations fused (the quadratic convergence of Newton's iteration for the
// reciprocal; the residual is formed exactly by the FMA), so r1 is within about half an ulp of 1 / x and in
// almost every case the correctly rounded value.  Zero, infinite and NaN inputs keep r0 (the residual of
// 0 * inf is NaN there).  Three instructions instead of the correctly rounded reciprocal's longer sequence.
__device__ __forceinline__ float rcp_nr(float x) {
    const float r0 = __fdividef(1.0f, x);
    const float r1 = __fmaf_rn(r0, __fmaf_rn(-x, r0, 1.0f), r0);
    return isfinite(r1) ? r1 : r0;
}

// Non-negative int64 -> float, exact below 2^23 with one integer add and one float subtract (the bits of
// 2^23 + v read as a float are exactly 2^23 + v); the general conversion otherwise.
__device__ __forceinline__ float nonneg_ll2f_rn(long long v) {
    if ((unsigned long long)v < (1ull << 23)) return __uint_as_float(0x4B000000u + (unsigned)v) - 8388608.0f;
    return ll2f_rn(v);
}

__device__ __forceinline__ float signed_ll2f_rn(long long v) {
    const float f = nonneg_ll2f_rn(v < 0 ? -v : v);
    return v < 0 ? -f : f;
}

// covers_pts with a 32-bit path: when every |X_j - px|, |Y_j - py| < 2^15 each product fits 30 bits and each
// edge function 31 bits; the area is their sum (taken in 64 bits).  Falls back to 64-bit arithmetic.
__device__ __forceinline__ bool covers_xy(const int X[3], const int Y[3], int px, int py) {
    int dx[3], dy[3];
    bool small = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dx[i] = X[i] - px;
        dy[i] = Y[i] - py;
        small &= (unsigned)(dx[i] + 32768) < 65536u && (unsigned)(dy[i] + 32768) < 65536u;
    }
    if (!small) return covers_pts(X, Y, px, py);
    int E[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        E[i] = dx[j] * dy[k] - dy[j] * dx[k];
    }
    const long long a2 = (long long)E[0] + E[1] + E[2];
    if (a2 == 0) return false;
    const bool pos = a2 > 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int e = pos ? E[i] : -E[i];
        if (e > 0) continue;
        if (e < 0) return false;
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        const int ga = pos ? (Y[j] - Y[k]) : (Y[k] - Y[j]);
        const int gb = pos ? (X[k] - X[j]) : (X[j] - X[k]);
        if (!(ga > 0 || (ga == 0 && gb > 0))) return false;
    }
    return true;
}

// FP32 depth key: sum_i E_i * (zeta_i / sum E) with correctly rounded conversions
// and an FMA chain (relative error <= 7 * 2^-24, see the design notes).
// Non-negative int32 -> float, correctly rounded.
__device__ __forceinline__ float nonneg_i2f_rn(int v) { return __int2float_rn(v); }

// Depth key of a small triangle from the sign-normalised 32-bit edge functions (same rounding as below).
__device__ __forceinline__ float depth_key_small(const TriRaster& t, const int E[3]) {
    float z = __fmul_rn(nonneg_i2f_rn(E[0]), t.zd[0]);
    z = __fmaf_rn(nonneg_i2f_rn(E[1]), t.zd[1], z);
    z = __fmaf_rn(nonneg_i2f_rn(E[2]), t.zd[2], z);
    return z;
}

// zd_i = zeta_i / |sum E| and |E_i| (E_i has the sign of the area at a covered pixel), so every term is >= 0.
__device__ __forceinline__ float depth_key(const TriRaster& t, const int64_t E[3]) {
    const bool neg = (t.flags & 8) != 0;
    const long long e0 = neg ? -E[0] : E[0], e1 = neg ? -E[1] : E[1], e2 = neg ? -E[2] : E[2];
    float z = __fmul_rn(nonneg_ll2f_rn(e0), t.zd[0]);
    z = __fmaf_rn(nonneg_ll2f_rn(e1), t.zd[1], z);
    z = __fmaf_rn(nonneg_ll2f_rn(e2), t.zd[2], z);
    return z;
}

// a*d - b*c with one rounding error less (Kahan's product difference, FMA based).
__device__ __forceinline__ float diff_of_products(float a, float d, float b, float c) {
    const float w = b * c;
    const float e = __fmaf_rn(-b, c, w);
    const float f = __fmaf_rn(a, d, -w);
    return f + e;
}

// A projected vertex record loaded with two 128-bit loads (records are 32-byte aligned).
struct VRec {
    int X, Y;
    float rx, ry, zeta, zeta_lo;
};

__device__ __forceinline__ VRec load_vrec(const mer_vertex* p) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float2 b = __ldg(reinterpret_cast<const float2*>(p) + 2);
    VRec r;
    r.X = __float_as_int(a.x);
    r.Y = __float_as_int(a.y);
    r.rx = a.z;
    r.ry = a.w;
    r.zeta = b.x;
    r.zeta_lo = b.y;
    return r;
}

// Screen barycentrics of a pixel centre and their screen gradients.
struct Bary {
    float lam[3];
    float gx[3], gy[3];  // d lambda_i / d P_x, d lambda_i / d P_y
    float d;             // twice the signed area
};

// Barycentrics on the unsnapped geometry v = (X/256 + rx, Y/256 + ry).  With
// a = (X - Px)/256, r = rx (and b, s for y) the edge function
//   e_i = cross(v_j - P, v_k - P) = [a_j b_k - b_j a_k] + [a_j s_k + r_j b_k - b_j r_k - s_j a_k] + [r_j s_k - s_j r_k]
// has an exact integer first bracket (the snapped edge function / 65536), so
// e_i is accurate to about one ulp of itself even where it is small.
__device__ __forceinline__ Bary screen_bary(const VRec v[3], int x, int y) {
    const int pxf = 256 * x + 128, pyf = 256 * y + 128;
    int ix[3], iy[3];
    float r[3], s[3];
    unsigned span = 0u;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ix[i] = v[i].X - pxf;
        iy[i] = v[i].Y - pyf;
        r[i] = v[i].rx;
        s[i] = v[i].ry;
        span |= (unsigned)(ix[i] + 32768) | (unsigned)(iy[i] + 32768);
    }
    Bary B;
    float e[3], a[3], b[3];
    if ((span >> 16) == 0u) {
        // Every vertex within 128 px of the centre (the common case): |ix|, |iy| < 2^15, so the integer edge
        // functions fit 32 bits, the coordinates convert exactly, and differences of the converted
        // coordinates are exact.  The same values as the general path below.
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            a[i] = __int2float_rn(ix[i]) * (1.0f / 256.0f);
            b[i] = __int2float_rn(iy[i]) * (1.0f / 256.0f);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int j = (i + 1) % 3, k = (i + 2) % 3;
            const int E = ix[j] * iy[k] - iy[j] * ix[k];
            const float lin = (a[j] * s[k] - s[j] * a[k]) + (r[j] * b[k] - b[j] * r[k]);
            const float quad = r[j] * s[k] - s[j] * r[k];
            e[i] = __fmaf_rn(__int2float_rn(E), 1.0f / 65536.0f, lin + quad);
        }
        B.d = (e[0] + e[1]) + e[2];
        const float inv = rcp_nr(B.d);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int j = (i + 1) % 3, k = (i + 2) % 3;
            B.lam[i] = e[i] * inv;
            B.gx[i] = ((b[j] - b[k]) + (s[j] - s[k])) * inv;
            B.gy[i] = ((a[k] - a[j]) + (r[k] - r[j])) * inv;
        }
        return B;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        a[i] = i2f_exact(ix[i]) * (1.0f / 256.0f);
        b[i] = i2f_exact(iy[i]) * (1.0f / 256.0f);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        const int64_t E = (int64_t)ix[j] * iy[k] - (int64_t)iy[j] * ix[k];
        const float lin = (a[j] * s[k] - s[j] * a[k]) + (r[j] * b[k] - b[j] * r[k]);
        const float quad = r[j] * s[k] - s[j] * r[k];
        e[i] = __fmaf_rn(signed_ll2f_rn(E), 1.0f / 65536.0f, lin + quad);
    }
    B.d = (e[0] + e[1]) + e[2];
    const float inv = rcp_nr(B.d);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        B.lam[i] = e[i] * inv;
        // dy_j - dy_k and dx_k - dx_j from exact integer differences plus residuals
        B.gx[i] = (i2f_exact(iy[j] - iy[k]) * (1.0f / 256.0f) + (s[j] - s[k])) * inv;
        B.gy[i] = (i2f_exact(ix[k] - ix[j]) * (1.0f / 256.0f) + (r[k] - r[j])) * inv;
    }
    return B;
}

// Texel coordinate x = u*N - 1/2 of the interpolated u = u0 + b1 (u1 - u0) + b2 (u2 - u0), split into an
// integer cell and a fraction in [0, 1).  The base x0 = u0*N - 1/2 is formed exactly (for N a power of two)
// and only the small offset sum_i b_i (x_i - x0) carries rounding, so the fraction is accurate to far below
// the FP32 resolution of u itself.  Non-finite or |u| >= 1024 samples at u = 0.
struct TexCoord {
    int cell;
    float frac;
};

__device__ __forceinline__ TexCoord tex_coord(float u0, float u1, float u2, float b1, float b2, int N) {
    const float u = u0 + (b1 * (u1 - u0) + b2 * (u2 - u0));
    TexCoord t;
    if (!(fabsf(u) < 1024.0f)) {
        t.cell = -1;
        t.frac = 0.5f;
        return t;
    }
    const float Nf = (float)N;
    const float xb = u0 * Nf - 0.5f;
    const float d = b1 * ((u1 * Nf - 0.5f) - xb) + b2 * ((u2 * Nf - 0.5f) - xb);
    const int fli = floor_i(xb);
    const float fl = i2f_exact(fli);
    const float f = (xb - fl) + d;  // xb - fl is exact
    const int ci = floor_i(f);
    float fr = f - i2f_exact(ci);
    int cell = fli + ci;
    if (fr >= 1.0f) {  // f just below an integer rounded up: the next cell at fraction 0
        fr = 0.0f;
        cell += 1;
    }
    t.cell = cell;
    t.frac = fr;
    return t;
}

// The four taps and weights of a bilinear lookup at texel coordinates (cx, cy): u wraps, v clamps to the
// edge texels (a clamped v has zero derivative).
struct TexTaps {
    int i0, i1, j0, j1;
    float fx, fy;
    bool clamped;
};

__device__ __forceinline__ TexTaps tex_taps(int TH, int TW, TexCoord cx, TexCoord cy) {
    TexTaps t;
    if ((unsigned)cx.cell < (unsigned)TW) {
        t.i0 = cx.cell;
    } else {
        t.i0 = cx.cell % TW;
        if (t.i0 < 0) t.i0 += TW;
    }
    t.i1 = (t.i0 + 1 == TW) ? 0 : t.i0 + 1;
    t.fx = cx.frac;
    t.clamped = false;
    if (cy.cell < 0) {
        t.j0 = 0; t.j1 = TH > 1 ? 1 : 0; t.fy = 0.0f; t.clamped = true;
    } else if (cy.cell > TH - 1 || (cy.cell == TH - 1 && cy.frac > 0.0f)) {
        t.j0 = TH - 1; t.j1 = TH - 1; t.fy = 0.0f; t.clamped = true;
    } else {
        t.j0 = cy.cell; t.j1 = t.j0 + 1 < TH ? t.j0 + 1 : TH - 1; t.fy = cy.frac;
    }
    return t;
}

// Texel (j, i) of a texture with `stride` floats per texel; vec4: stride == 4 and 16-byte aligned (one
// 128-bit load per texel).
__device__ __forceinline__ float4 texel4(const float* __restrict__ tex, int TW, int stride, bool vec4, int nc, int j,
                                         int i) {
    const float* q = tex + ((size_t)j * TW + i) * stride;
    if (vec4) return __ldg(reinterpret_cast<const float4*>(q));
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    r.x = __ldg(q);
    if (nc > 1) r.y = __ldg(q + 1);
    if (nc > 2) r.z = __ldg(q + 2);
    if (nc > 3) r.w = __ldg(q + 3);
    return r;
}

__device__ __forceinline__ float comp(const float4& v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w)); }

// Bilinear values of channels 0..nc-1 written to out[0..nc-1].
__device__ __forceinline__ void tex_values(const float* __restrict__ tex, int TW, int stride, bool vec4, int nc,
                                           const TexTaps& t, float* out) {
    if (nc <= 4) {
        const float4 a00 = texel4(tex, TW, stride, vec4, nc, t.j0, t.i0), a10 = texel4(tex, TW, stride, vec4, nc, t.j0, t.i1);
        const float4 a01 = texel4(tex, TW, stride, vec4, nc, t.j1, t.i0), a11 = texel4(tex, TW, stride, vec4, nc, t.j1, t.i1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c >= nc) break;
            const float t00 = comp(a00, c), t10 = comp(a10, c), t01 = comp(a01, c), t11 = comp(a11, c);
            const float a = t00 + t.fx * (t10 - t00);
            const float b = t01 + t.fx * (t11 - t01);
            out[c] = a + t.fy * (b - a);
        }
        return;
    }
    const float* r0 = tex + (size_t)t.j0 * TW * stride;
    const float* r1 = tex + (size_t)t.j1 * TW * stride;
    for (int c = 0; c < nc; ++c) {
        const float t00 = __ldg(r0 + (size_t)t.i0 * stride + c), t10 = __ldg(r0 + (size_t)t.i1 * stride + c);
        const float t01 = __ldg(r1 + (size_t)t.i0 * stride + c), t11 = __ldg(r1 + (size_t)t.i1 * stride + c);
        const float a = t00 + t.fx * (t10 - t00);
        const float b = t01 + t.fx * (t11 - t01);
        out[c] = a + t.fy * (b - a);
    }
}

// sum_c g_c dT_c/du and sum_c g_c dT_c/dv (g read from global memory, nc channels).
__device__ __forceinline__ void tex_grad_uv(const float* __restrict__ tex, int TH, int TW, int stride, bool vec4,
                                            int nc, const TexTaps& t, const float* __restrict__ g, float& gu,
                                            float& gv) {
    float su = 0.f, sv = 0.f;
    if (nc <= 4) {
        const float4 a00 = texel4(tex, TW, stride, vec4, nc, t.j0, t.i0), a10 = texel4(tex, TW, stride, vec4, nc, t.j0, t.i1);
        const float4 a01 = texel4(tex, TW, stride, vec4, nc, t.j1, t.i0), a11 = texel4(tex, TW, stride, vec4, nc, t.j1, t.i1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c >= nc) break;
            const float t00 = comp(a00, c), t10 = comp(a10, c), t01 = comp(a01, c), t11 = comp(a11, c);
            const float gc = __ldg(g + c);
            su += gc * ((1.0f - t.fy) * (t10 - t00) + t.fy * (t11 - t01));
            const float a = t00 + t.fx * (t10 - t00);
            const float b = t01 + t.fx * (t11 - t01);
            sv += gc * (b - a);
        }
    } else {
        const float* r0 = tex + (size_t)t.j0 * TW * stride;
        const float* r1 = tex + (size_t)t.j1 * TW * stride;
        for (int c = 0; c < nc; ++c) {
            const float t00 = __ldg(r0 + (size_t)t.i0 * stride + c), t10 = __ldg(r0 + (size_t)t.i1 * stride + c);
            const float t01 = __ldg(r1 + (size_t)t.i0 * stride + c), t11 = __ldg(r1 + (size_t)t.i1 * stride + c);
            const float gc = __ldg(g + c);
            su += gc * ((1.0f - t.fy) * (t10 - t00) + t.fy * (t11 - t01));
            const float a = t00 + t.fx * (t10 - t00);
            const float b = t01 + t.fx * (t11 - t01);
            sv += gc * (b - a);
        }
    }
    gu = (float)TW * su;
    gv = t.clamped ? 0.0f : (float)TH * sv;
}

// Item of a batch that holds global element g of one offset field (largest i with key(i) <= g; items
// with an empty range share their key with the next item and are never returned for a valid g).
enum ItemField { kFieldVrec = 0, kFieldTrec, kFieldPix, kFieldTile, kFieldBtile };

__device__ __forceinline__ long long item_key(const mer_item& it, int f) {
    switch (f) {
        case kFieldVrec: return it.vrec;
        case kFieldTrec: return it.trec;
        case kFieldPix: return it.pix;
        case kFieldTile: return it.tile;
        default: return it.btile;
    }
}

__device__ __forceinline__ int find_item(const mer_item* __restrict__ items, int n, long long g, int f) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item_key(items[mid], f) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// find_item for one element per thread of a 1-D block: one search for the block's first element g0, then
// each thread steps forward over the (few) item boundaries inside the block.  All threads of the block
// must call it (it holds a barrier), also those whose element is past the end.
__device__ __forceinline__ int block_find_item(const mer_item* __restrict__ items, int n, long long g0, long long g,
                                               int f) {
    __shared__ int s_k;
    if (threadIdx.x == 0) s_k = find_item(items, n, g0, f);
    __syncthreads();
    int k = s_k;
    while (k + 1 < n && item_key(items[k + 1], f) <= g) ++k;
    return k;
}

__device__ __forceinline__ void set_status(void* ws, int bit) {
    if (ws) atomicOr(&reinterpret_cast<WsHeader*>(ws)->status, bit);
}

}  // namespace mer
