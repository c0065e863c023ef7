/*
 * oracle.c -- FP64 CPU oracle of the micro-edge rasterizer-gradient method
 * ("Rasterized Edge Gradients: Handling Discontinuities Differentiably",
 * arXiv 2405.02508, called EdgeGrad in the paper).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  The CUDA product path never
 * calls it, links it or shares code with it.
 *
 * Plain, slow, obviously correct: one view per call, nested loops over
 * triangles, pixels and pixel pairs, FP64 arithmetic and exact int64 coverage.
 * Each function names the passage of the paper it follows.  Conventions the
 * paper leaves open (camera model, fill rule, snapping, depth tie-break, which
 * barycentrics gather fragment gradients) are stated where they are used.
 *
 * Compile with -ffp-contract=off: the projection must round exactly as written
 * (no fused multiply-add), because the snapped integer screen positions decide
 * coverage and must be reproducible.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double R[9];   /* world -> camera rotation, row-major */
    double t[3];   /* world -> camera translation */
    double fx, fy, cx, cy;
    double znear;  /* triangles with any vertex at Z <= znear are culled */
} orc_camera;

typedef struct {
    int n_main;    /* channels [0, n_main): interpolated attributes or texture */
    int C;         /* total channels of the shaded image */
    int uv_offset; /* texture mode: attribute channel of u (v = u + 1); -1: interpolation mode */
    int mask_ch;   /* channel holding the coverage mask, or -1 */
    int depth_ch;  /* channel holding depth Z, or -1 */
    int C_attr;    /* attribute channels per vertex */
    int tex_h, tex_w;
    int tex_c;     /* floats per texel in memory (>= n_main) */
    int backface_ch; /* channel holding the back-face image (1 where the visible triangle faces away from the
                        camera, else 0), or -1 */
} orc_shading;

enum { ORC_VALID_FRONT = 1, ORC_VALID_GUARD = 2, ORC_VALID = 3 };

/* Snapped positions are integers in 1/256 px; the guard band keeps every
 * coverage product inside int64. */
#define ORC_SUBPIX 256.0
#define ORC_GUARD 536870912.0 /* 2^29 */
#define ORC_TIE_REL 1e-6

/* ------------------------------------------------------------------------
 * Vertex transform module (Supp. B, "transforms the vertices to the camera
 * frame and then projects them onto the image plane").
 * Camera frame X_c = R X_w + t; x_s = fx X_c/Z_c + cx, y_s = fy Y_c/Z_c + cy,
 * zeta = 1/Z_c.  The operation order below is the definition: left-to-right
 * sums, one reciprocal, no fused operations.  Snap: X = round-half-even(256 x_s).
 * ------------------------------------------------------------------------ */
void orc_project(const float* verts, int V, const orc_camera* cam,
                 double* scr /* [V,3]: x_s, y_s, zeta */,
                 int64_t* snap /* [V,2] */, int32_t* flags /* [V] */)
{
    for (int v = 0; v < V; ++v) {
        double x = verts[3 * v + 0], y = verts[3 * v + 1], z = verts[3 * v + 2];
        const double* R = cam->R;
        double Xc = ((R[0] * x + R[1] * y) + R[2] * z) + cam->t[0];
        double Yc = ((R[3] * x + R[4] * y) + R[5] * z) + cam->t[1];
        double Zc = ((R[6] * x + R[7] * y) + R[8] * z) + cam->t[2];
        int32_t fl = 0;
        double xs = 0.0, ys = 0.0, zeta = 0.0;
        int64_t sx = 0, sy = 0;
        if (Zc > cam->znear) {
            fl |= ORC_VALID_FRONT;
            zeta = 1.0 / Zc;
            xs = (cam->fx * Xc) * zeta + cam->cx;
            ys = (cam->fy * Yc) * zeta + cam->cy;
            double X = xs * ORC_SUBPIX, Y = ys * ORC_SUBPIX;
            if (fabs(X) <= ORC_GUARD && fabs(Y) <= ORC_GUARD) {
                fl |= ORC_VALID_GUARD;
                sx = (int64_t)nearbyint(X); /* default rounding mode: nearest, ties to even */
                sy = (int64_t)nearbyint(Y);
            }
        }
        scr[3 * v + 0] = xs;
        scr[3 * v + 1] = ys;
        scr[3 * v + 2] = zeta;
        snap[2 * v + 0] = sx;
        snap[2 * v + 1] = sy;
        flags[v] = fl;
    }
}

/* ------------------------------------------------------------------------
 * Coverage (rasterization module, Supp. B: the z-buffered rasterizer whose
 * output is the index image).  The paper uses an unmodified rasterizer and
 * fixes no fill rule; this library's rule:
 *   pixel (x, y) has its centre at (x + 1/2, y + 1/2), i.e. (256x+128, 256y+128)
 *   in snapped units; E_i(P) = cross(v_j - P, v_k - P) for (i,j,k) cyclic, so
 *   E_0 + E_1 + E_2 = cross(v1 - v0, v2 - v0) = twice the signed area A2.
 *   Both windings are drawn (s = sign A2; A2 == 0 draws nothing).  P is covered
 *   iff every s*E_i > 0, or s*E_i == 0 on a top or left edge (y points down):
 *   with (a, b) = s * grad E_i, the edge is top-left iff a > 0 or (a == 0, b > 0).
 * ------------------------------------------------------------------------ */
static int64_t edge_fn(int64_t xj, int64_t yj, int64_t xk, int64_t yk, int64_t px, int64_t py)
{
    return (xj - px) * (yk - py) - (yj - py) * (xk - px);
}

static int covers(const int64_t X[3], const int64_t Y[3], int64_t px, int64_t py)
{
    int64_t a2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
    if (a2 == 0) return 0;
    int64_t s = a2 > 0 ? 1 : -1;
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        int64_t e = s * edge_fn(X[j], Y[j], X[k], Y[k], px, py);
        if (e > 0) continue;
        if (e < 0) return 0;
        int64_t ga = s * (Y[j] - Y[k]); /* dE_i/dPx */
        int64_t gb = s * (X[k] - X[j]); /* dE_i/dPy */
        if (!(ga > 0 || (ga == 0 && gb > 0))) return 0;
    }
    return 1;
}

static int64_t floordiv(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

static int tri_fetch(const int64_t* snap, const int32_t* flags, const int32_t* tris, int t,
                     int64_t X[3], int64_t Y[3])
{
    for (int i = 0; i < 3; ++i) {
        int v = tris[3 * t + i];
        if ((flags[v] & ORC_VALID) != ORC_VALID) return 0; /* near-plane or guard-band cull */
        X[i] = snap[2 * v];
        Y[i] = snap[2 * v + 1];
    }
    return 1;
}

/* Exact coverage test exposed for tests: is pixel (x, y)'s centre in triangle t? */
int orc_covers_pixel(const int64_t* snap, const int32_t* flags, const int32_t* tris, int t, int x, int y)
{
    int64_t X[3], Y[3];
    if (!tri_fetch(snap, flags, tris, t, X, Y)) return 0;
    return covers(X, Y, 256 * (int64_t)x + 128, 256 * (int64_t)y + 128);
}

/* ------------------------------------------------------------------------
 * Rasterization module with z-buffer (Supp. B: index image + depth image).
 * Depth test: zeta_test = sum_i E_i zeta_i / sum_i E_i with the exact integer
 * E_i of the coverage test (a convex combination of the vertices' 1/Z); the
 * nearest fragment has the largest zeta_test; an exact tie goes to the lower
 * triangle id.  A pixel is flagged as a near-tie when the winner and the next
 * covering fragment differ by at most 1e-6 relative.
 * Per-triangle bounding-box loops.
 * ------------------------------------------------------------------------ */
int orc_rasterize(const double* scr, const int64_t* snap, const int32_t* flags, int V,
                  const int32_t* tris, int T, int H, int W,
                  int32_t* index /* [H,W], -1 background */,
                  double* zbest /* [H,W] or NULL */, uint8_t* tie /* [H,W] or NULL */)
{
    (void)V;
    size_t npix = (size_t)H * W;
    double* z1 = (double*)malloc(npix * sizeof(double));
    double* z2 = (double*)malloc(npix * sizeof(double));
    if (!z1 || !z2) { free(z1); free(z2); return -1; }
    for (size_t p = 0; p < npix; ++p) { index[p] = -1; z1[p] = -1.0; z2[p] = -1.0; }
    for (int t = 0; t < T; ++t) {
        int64_t X[3], Y[3];
        if (!tri_fetch(snap, flags, tris, t, X, Y)) continue;
        int64_t a2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
        if (a2 == 0) continue;
        int64_t mnx = X[0], mxx = X[0], mny = Y[0], mxy = Y[0];
        for (int i = 1; i < 3; ++i) {
            if (X[i] < mnx) mnx = X[i];
            if (X[i] > mxx) mxx = X[i];
            if (Y[i] < mny) mny = Y[i];
            if (Y[i] > mxy) mxy = Y[i];
        }
        int64_t x0 = -floordiv(-(mnx - 128), 256), x1 = floordiv(mxx - 128, 256);
        int64_t y0 = -floordiv(-(mny - 128), 256), y1 = floordiv(mxy - 128, 256);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > W - 1) x1 = W - 1;
        if (y1 > H - 1) y1 = H - 1;
        double zt[3];
        for (int i = 0; i < 3; ++i) zt[i] = scr[3 * tris[3 * t + i] + 2];
        for (int64_t y = y0; y <= y1; ++y) {
            for (int64_t x = x0; x <= x1; ++x) {
                int64_t px = 256 * x + 128, py = 256 * y + 128;
                if (!covers(X, Y, px, py)) continue;
                double num = 0.0, den = 0.0;
                for (int i = 0; i < 3; ++i) {
                    int j = (i + 1) % 3, k = (i + 2) % 3;
                    double e = (double)edge_fn(X[j], Y[j], X[k], Y[k], px, py);
                    num += e * zt[i];
                    den += e;
                }
                double z = num / den;
                size_t p = (size_t)y * W + x;
                if (z > z1[p] || (z == z1[p] && t < index[p])) {
                    if (z1[p] > z2[p]) z2[p] = z1[p];
                    z1[p] = z;
                    index[p] = t;
                } else if (z > z2[p]) {
                    z2[p] = z;
                }
            }
        }
    }
    for (size_t p = 0; p < npix; ++p) {
        if (zbest) zbest[p] = z1[p];
        if (tie) tie[p] = (index[p] >= 0 && z2[p] > 0.0 && z1[p] - z2[p] <= ORC_TIE_REL * z1[p]) ? 1 : 0;
    }
    free(z1);
    free(z2);
    return 0;
}

/* ------------------------------------------------------------------------
 * Barycentrics module (Supp. B: index image + geometry -> barycentric image).
 * Values use the unsnapped screen positions: lambda_i = e_i / d with
 * e_i = cross(v_j - P, v_k - P), d = e_0 + e_1 + e_2 at the pixel centre P;
 * perspective-correct b_i = lambda_i zeta_i / s, s = sum_j lambda_j zeta_j,
 * depth Z = 1/s (distance along the principal axis).
 * ------------------------------------------------------------------------ */
static void screen_lambda(const double* scr, const int32_t* tri, double px, double py, double lam[3])
{
    double x[3], y[3];
    for (int i = 0; i < 3; ++i) { x[i] = scr[3 * tri[i]] - px; y[i] = scr[3 * tri[i] + 1] - py; }
    double e[3];
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        e[i] = x[j] * y[k] - y[j] * x[k];
    }
    double d = e[0] + e[1] + e[2];
    for (int i = 0; i < 3; ++i) lam[i] = e[i] / d;
}

int orc_pixel_values(const double* scr, const int32_t* tris, const int32_t* index, int H, int W,
                     double* lam_out /* [H,W,3] or NULL */, double* bary /* [H,W,3] or NULL */,
                     double* depth /* [H,W] or NULL */)
{
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            int t = index[p];
            double lam[3] = {0, 0, 0}, b[3] = {0, 0, 0}, Z = 0.0;
            if (t >= 0) {
                const int32_t* tri = tris + 3 * (size_t)t;
                screen_lambda(scr, tri, x + 0.5, y + 0.5, lam);
                double s = 0.0;
                for (int i = 0; i < 3; ++i) s += lam[i] * scr[3 * tri[i] + 2];
                for (int i = 0; i < 3; ++i) b[i] = lam[i] * scr[3 * tri[i] + 2] / s;
                Z = 1.0 / s;
            }
            for (int i = 0; i < 3; ++i) {
                if (lam_out) lam_out[3 * p + i] = lam[i];
                if (bary) bary[3 * p + i] = b[i];
            }
            if (depth) depth[p] = Z;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Dual numbers with 9 tangents (x_s, y_s, zeta of the triangle's 3 vertices):
 * forward-mode derivatives of a pixel's shaded value, used for the smooth
 * (interior) term Omega of Eq. 5 / Eq. 11.
 * ------------------------------------------------------------------------ */
#define ND 9
/* v: value, d: derivatives.  m: magnitudes of the derivatives -- the same chain
 * rule with every sum replaced by a sum of absolute values -- used only to report
 * how strongly each derivative cancels (the conditioning the tests scale
 * tolerances with); d never depends on m. */
typedef struct { double v; double d[ND]; double m[ND]; } dual;

static dual dconst(double v) { dual r; r.v = v; memset(r.d, 0, sizeof r.d); memset(r.m, 0, sizeof r.m); return r; }
static dual dvar(double v, int k) { dual r = dconst(v); r.d[k] = 1.0; r.m[k] = 1.0; return r; }
static dual dadd(dual a, dual b)
{
    dual r;
    r.v = a.v + b.v;
    for (int k = 0; k < ND; ++k) { r.d[k] = a.d[k] + b.d[k]; r.m[k] = a.m[k] + b.m[k]; }
    return r;
}
static dual dsub(dual a, dual b)
{
    dual r;
    r.v = a.v - b.v;
    for (int k = 0; k < ND; ++k) { r.d[k] = a.d[k] - b.d[k]; r.m[k] = a.m[k] + b.m[k]; }
    return r;
}
static dual dmul(dual a, dual b)
{
    dual r;
    r.v = a.v * b.v;
    for (int k = 0; k < ND; ++k) {
        r.d[k] = a.d[k] * b.v + a.v * b.d[k];
        r.m[k] = a.m[k] * fabs(b.v) + fabs(a.v) * b.m[k];
    }
    return r;
}
static dual ddiv(dual a, dual b)
{
    dual r;
    r.v = a.v / b.v;
    for (int k = 0; k < ND; ++k) {
        r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
        r.m[k] = (a.m[k] + fabs(r.v) * b.m[k]) / fabs(b.v);
    }
    return r;
}
static dual dscale(dual a, double c)
{
    dual r;
    r.v = a.v * c;
    for (int k = 0; k < ND; ++k) { r.d[k] = a.d[k] * c; r.m[k] = a.m[k] * fabs(c); }
    return r;
}

/* Bilinear texture lookup, texel centres at ((i + 1/2)/TW, (j + 1/2)/TH):
 * u wraps, v clamps to the edge texels.  Value and derivatives through (u, v). */
static void tex_bilinear(const float* tex, int TH, int TW, int nc, int stride, dual u, dual v, dual* out)
{
    /* non-finite or far-out coordinates (|u| or |v| >= 1024) sample at 0 */
    if (!(fabs(u.v) < 1024.0)) u = dconst(0.0);
    if (!(fabs(v.v) < 1024.0)) v = dconst(0.0);
    dual x = dsub(dscale(u, (double)TW), dconst(0.5));
    double x0 = floor(x.v);
    dual fx = dsub(x, dconst(x0));
    long long i0 = (long long)x0 % TW;
    if (i0 < 0) i0 += TW;
    long long i1 = (i0 + 1) % TW;
    dual y = dsub(dscale(v, (double)TH), dconst(0.5));
    if (y.v < 0.0) y = dconst(0.0);
    if (y.v > TH - 1) y = dconst((double)(TH - 1));
    double y0 = floor(y.v);
    dual fy = dsub(y, dconst(y0));
    long long j0 = (long long)y0;
    long long j1 = j0 + 1 < TH ? j0 + 1 : TH - 1;
    dual one = dconst(1.0);
    dual w00 = dmul(dsub(one, fx), dsub(one, fy)), w10 = dmul(fx, dsub(one, fy));
    dual w01 = dmul(dsub(one, fx), fy), w11 = dmul(fx, fy);
    for (int c = 0; c < nc; ++c) {
        double t00 = tex[((size_t)j0 * TW + i0) * stride + c], t10 = tex[((size_t)j0 * TW + i1) * stride + c];
        double t01 = tex[((size_t)j1 * TW + i0) * stride + c], t11 = tex[((size_t)j1 * TW + i1) * stride + c];
        out[c] = dadd(dadd(dscale(w00, t00), dscale(w10, t10)), dadd(dscale(w01, t01), dscale(w11, t11)));
    }
}

/* Facing of a triangle (Supp. B back-face image).  With the camera looking down +Z, x right and y down, a
 * triangle whose world normal (v1 - v0) x (v2 - v0) points away from the camera projects with a positive
 * signed area (x1 - x0)(y2 - y0) - (y1 - y0)(x2 - x0).  Taken on the snapped coordinates, exactly, like the
 * coverage test. */
static int back_facing(const int64_t* snap, const int32_t* tri)
{
    const int64_t X0 = snap[2 * tri[0]], Y0 = snap[2 * tri[0] + 1];
    const int64_t X1 = snap[2 * tri[1]], Y1 = snap[2 * tri[1] + 1];
    const int64_t X2 = snap[2 * tri[2]], Y2 = snap[2 * tri[2] + 1];
    return (X1 - X0) * (Y2 - Y0) - (Y1 - Y0) * (X2 - X0) > 0;
}

/* Shaded channels of one covered pixel as duals in the 9 vertex coordinates. */
static void shade_pixel_dual(const double* scr, const int64_t* snap, const int32_t* tri, double px, double py,
                             const float* attr, const float* tex, const orc_shading* sh, dual* I)
{
    dual x[3], y[3], z[3];
    for (int i = 0; i < 3; ++i) {
        x[i] = dsub(dvar(scr[3 * tri[i]], 3 * i + 0), dconst(px));
        y[i] = dsub(dvar(scr[3 * tri[i] + 1], 3 * i + 1), dconst(py));
        z[i] = dvar(scr[3 * tri[i] + 2], 3 * i + 2);
    }
    dual e[3];
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        e[i] = dsub(dmul(x[j], y[k]), dmul(y[j], x[k]));
    }
    dual d = dadd(dadd(e[0], e[1]), e[2]);
    dual lam[3], s = dconst(0.0), b[3];
    for (int i = 0; i < 3; ++i) { lam[i] = ddiv(e[i], d); s = dadd(s, dmul(lam[i], z[i])); }
    for (int i = 0; i < 3; ++i) b[i] = ddiv(dmul(lam[i], z[i]), s);
    for (int c = 0; c < sh->C; ++c) I[c] = dconst(0.0);
    if (sh->uv_offset < 0) {
        for (int c = 0; c < sh->n_main; ++c)
            for (int i = 0; i < 3; ++i)
                I[c] = dadd(I[c], dscale(b[i], attr[(size_t)tri[i] * sh->C_attr + c]));
    } else {
        dual u = dconst(0.0), v = dconst(0.0);
        for (int i = 0; i < 3; ++i) {
            u = dadd(u, dscale(b[i], attr[(size_t)tri[i] * sh->C_attr + sh->uv_offset]));
            v = dadd(v, dscale(b[i], attr[(size_t)tri[i] * sh->C_attr + sh->uv_offset + 1]));
        }
        tex_bilinear(tex, sh->tex_h, sh->tex_w, sh->n_main, sh->tex_c, u, v, I);
    }
    if (sh->mask_ch >= 0) I[sh->mask_ch] = dconst(1.0);
    if (sh->depth_ch >= 0) I[sh->depth_ch] = ddiv(dconst(1.0), s);
    /* a binary image: constant on each triangle, so only the edge term differentiates it */
    if (sh->backface_ch >= 0) I[sh->backface_ch] = dconst(back_facing(snap, tri) ? 1.0 : 0.0);
}

/* ------------------------------------------------------------------------
 * Interpolation module + deferred shading (Supp. B): shaded image [H,W,C].
 * ------------------------------------------------------------------------ */
/* Rows [y0, y1) only (the other rows of `image` are left as they are); orc_shade is all rows.  A view's
 * rows are independent, so callers may shade bands of rows on separate threads. */
int orc_shade_rows(const double* scr, const int64_t* snap, const int32_t* tris, const int32_t* index, int H, int W,
                   const float* attr, const float* tex, const float* bg, const orc_shading* sh,
                   double* image /* [H,W,C] */, int y0, int y1)
{
    dual I[64];
    if (sh->C > 64) return -1;
    if (sh->backface_ch >= 0 && !snap) return -1;
    if (y0 < 0) y0 = 0;
    if (y1 > H) y1 = H;
    for (int y = y0; y < y1; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            int t = index[p];
            if (t < 0) {
                for (int c = 0; c < sh->C; ++c) image[p * sh->C + c] = bg[c];
                continue;
            }
            shade_pixel_dual(scr, snap, tris + 3 * (size_t)t, x + 0.5, y + 0.5, attr, tex, sh, I);
            for (int c = 0; c < sh->C; ++c) image[p * sh->C + c] = I[c].v;
        }
    }
    return 0;
}

int orc_shade(const double* scr, const int64_t* snap, const int32_t* tris, const int32_t* index, int H, int W,
              const float* attr, const float* tex, const float* bg, const orc_shading* sh,
              double* image /* [H,W,C] */)
{
    return orc_shade_rows(scr, snap, tris, index, H, W, attr, tex, bg, sh, image, 0, H);
}

/* ------------------------------------------------------------------------
 * Backward pass: EdgeGrad module (Sec. 4.2-4.4, Supp. A.2-A.3) plus the smooth
 * term Omega (Eq. 5, Eq. 11), into gradients w.r.t. the projected vertex
 * positions (x_s, y_s, zeta).
 *
 * counts[0] differing pairs, [1] overhang (incl. background), [2] adjacent,
 * [3] intersection, [4] intersection skipped (parallel slice normals),
 * [5] intersection skipped because intersections are disabled.
 * ------------------------------------------------------------------------ */
enum { ORC_EDGE = 1, ORC_INTERIOR = 2, ORC_INTERSECT = 4, ORC_EXACT_CROSSING = 8 };

/* Exact-crossing gather weights for an overhang pair (an option; the default gathers with lambda at the
 * foreground pixel centre).  The micro-edge of the pair is where the foreground triangle's outline crosses
 * the segment from the foreground pixel centre F to the other centre O.  That crossing lies on the edge
 * through which the segment leaves the triangle: among the edges with O on or beyond them (s E(O) <= 0 with
 * s the area sign), the one reached first, i.e. the smallest t_k = e_k(F) / (e_k(F) - e_k(O)), compared
 * exactly in integer arithmetic on the snapped coordinates (ties: lower k).  Along the pair axis the crossing
 * moves with the edge's endpoints v_j, v_l (j = k+1, l = k+2) with weights 1 - u and u, where
 * u = (F_o - v_j,o) / (v_l,o - v_j,o) is its position along the edge measured on the other axis o (unsnapped,
 * clamped to [0, 1]; 1/2 for an edge parallel to the pair axis).  Returns 0 when no edge qualifies. */
int orc_crossing_weights(const double* scr, const int64_t* snap, const int32_t* tri, int fx, int fy, int ox,
                         int oy, int axis, int vout[2], double wout[2])
{
    int64_t X[3], Y[3];
    for (int i = 0; i < 3; ++i) { X[i] = snap[2 * tri[i]]; Y[i] = snap[2 * tri[i] + 1]; }
    int64_t a2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
    if (a2 == 0) return 0;
    int64_t sg = a2 > 0 ? 1 : -1;
    int64_t Fx = 256 * (int64_t)fx + 128, Fy = 256 * (int64_t)fy + 128;
    int64_t Ox = 256 * (int64_t)ox + 128, Oy = 256 * (int64_t)oy + 128;
    int best = -1;
    int64_t bnum = 0, bden = 1;
    for (int k = 0; k < 3; ++k) {
        int j = (k + 1) % 3, l = (k + 2) % 3;
        int64_t eF = sg * edge_fn(X[j], Y[j], X[l], Y[l], Fx, Fy);
        int64_t eO = sg * edge_fn(X[j], Y[j], X[l], Y[l], Ox, Oy);
        if (eO > 0 || eF - eO <= 0) continue;
        if (best < 0 || (__int128)eF * bden < (__int128)bnum * (eF - eO)) { best = k; bnum = eF; bden = eF - eO; }
    }
    if (best < 0) return 0;
    int j = (best + 1) % 3, l = (best + 2) % 3;
    int o = 1 - axis;
    double Fo = (o == 0 ? fx : fy) + 0.5;
    double vj = scr[3 * tri[j] + o], vl = scr[3 * tri[l] + o];
    double u = vl != vj ? (Fo - vj) / (vl - vj) : 0.5;
    u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
    vout[0] = tri[j]; vout[1] = tri[l];
    wout[0] = 1.0 - u; wout[1] = u;
    return 1;
}

static void tri_normal(const double* scr, const int32_t* tri, double N[3])
{
    const double* a = scr + 3 * tri[0];
    const double* b = scr + 3 * tri[1];
    const double* c = scr + 3 * tri[2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    N[0] = u[1] * w[2] - u[2] * w[1];
    N[1] = u[2] * w[0] - u[0] * w[2];
    N[2] = u[0] * w[1] - u[1] * w[0];
}

/* Gather a fragment gradient g = dL/dr (3-vector in x_s, y_s, zeta) of triangle t
 * at pixel (x, y) into its vertices: the fragment at the pixel centre is
 * r = sum_i lambda_i v_i, so dL/dv_i = lambda_i dL/dr (the interpolator's
 * backward, Sec. 4.2 last paragraph). */
static void gather(const double* scr, const int32_t* tris, int t, int x, int y, const double g[3],
                   double* grad_scr, const double gmag[3], double* grad_abs)
{
    const int32_t* tri = tris + 3 * (size_t)t;
    double lam[3];
    screen_lambda(scr, tri, x + 0.5, y + 0.5, lam);
    for (int i = 0; i < 3; ++i)
        for (int q = 0; q < 3; ++q) {
            grad_scr[3 * (size_t)tri[i] + q] += lam[i] * g[q];
            if (grad_abs) grad_abs[3 * (size_t)tri[i] + q] += fabs(lam[i]) * gmag[q];
        }
}

/* The part of orc_backward that belongs to rows [y0, y1): the interior term of those rows' pixels, the
 * horizontal pairs in those rows and the vertical pairs (y, y + 1) with y in them.  The sum over a partition
 * of the rows is orc_backward (up to the order of the FP64 additions); callers may run bands of rows on
 * separate threads, each into its own accumulators. */
int orc_backward_rows(const double* scr, const int64_t* snap, const int32_t* flags, int V,
                      const int32_t* tris, const int32_t* index, int H, int W,
                      const double* image /* [H,W,C] */, const float* grad_image /* [H,W,C] */,
                      const float* attr, const float* tex, const orc_shading* sh, int mode,
                      double* grad_scr /* [V,3], accumulated */, double* grad_attr /* [V,C_attr] or NULL */,
                      int64_t* counts /* [6] */, double* grad_abs /* [V,3] or NULL */,
                      double* grad_attr_abs /* [V,C_attr] or NULL */, int y0, int y1)
{
    const int C = sh->C;
    dual I[64];
    if (C > 64) return -1;
    (void)V;
    if (mode & ORC_INTERIOR) {
        /* Omega: derivative of the shaded value of each covered pixel with the
         * index image held fixed (Eq. 5, second term), through the barycentrics
         * and interpolation (and texture) modules. */
        for (int y = y0 < 0 ? 0 : y0; y < (y1 > H ? H : y1); ++y) {
            for (int x = 0; x < W; ++x) {
                size_t p = (size_t)y * W + x;
                int t = index[p];
                if (t < 0) continue;
                const int32_t* tri = tris + 3 * (size_t)t;
                shade_pixel_dual(scr, snap, tri, x + 0.5, y + 0.5, attr, tex, sh, I);
                const float* g = grad_image + p * C;
                for (int m = 0; m < 3; ++m)
                    for (int q = 0; q < 3; ++q) {
                        double acc = 0.0, mag = 0.0;
                        for (int c = 0; c < C; ++c) {
                            acc += (double)g[c] * I[c].d[3 * m + q];
                            mag += fabs((double)g[c]) * I[c].m[3 * m + q];
                        }
                        grad_scr[3 * (size_t)tri[m] + q] += acc;
                        if (grad_abs) grad_abs[3 * (size_t)tri[m] + q] += mag;
                    }
                if (grad_attr) {
                    double lam[3], b[3], s = 0.0;
                    screen_lambda(scr, tri, x + 0.5, y + 0.5, lam);
                    for (int i = 0; i < 3; ++i) s += lam[i] * scr[3 * tri[i] + 2];
                    for (int i = 0; i < 3; ++i) b[i] = lam[i] * scr[3 * tri[i] + 2] / s;
                    if (sh->uv_offset < 0) {
                        for (int i = 0; i < 3; ++i)
                            for (int c = 0; c < sh->n_main; ++c) {
                                grad_attr[(size_t)tri[i] * sh->C_attr + c] += b[i] * g[c];
                                if (grad_attr_abs) grad_attr_abs[(size_t)tri[i] * sh->C_attr + c] += fabs(b[i] * g[c]);
                            }
                    } else {
                        /* d(texture)/d(u, v) at the interpolated uv, via 2 tangents */
                        dual u = dvar(0.0, 0), v = dvar(0.0, 1);
                        u.v = 0.0; v.v = 0.0;
                        for (int i = 0; i < 3; ++i) {
                            u.v += b[i] * attr[(size_t)tri[i] * sh->C_attr + sh->uv_offset];
                            v.v += b[i] * attr[(size_t)tri[i] * sh->C_attr + sh->uv_offset + 1];
                        }
                        dual T[64];
                        tex_bilinear(tex, sh->tex_h, sh->tex_w, sh->n_main, sh->tex_c, u, v, T);
                        double gu = 0.0, gv = 0.0, gum = 0.0, gvm = 0.0;
                        for (int c = 0; c < sh->n_main; ++c) {
                            gu += g[c] * T[c].d[0];
                            gv += g[c] * T[c].d[1];
                            gum += fabs((double)g[c]) * T[c].m[0];
                            gvm += fabs((double)g[c]) * T[c].m[1];
                        }
                        for (int i = 0; i < 3; ++i) {
                            grad_attr[(size_t)tri[i] * sh->C_attr + sh->uv_offset] += b[i] * gu;
                            grad_attr[(size_t)tri[i] * sh->C_attr + sh->uv_offset + 1] += b[i] * gv;
                            if (grad_attr_abs) {
                                grad_attr_abs[(size_t)tri[i] * sh->C_attr + sh->uv_offset] += fabs(b[i]) * gum;
                                grad_attr_abs[(size_t)tri[i] * sh->C_attr + sh->uv_offset + 1] += fabs(b[i]) * gvm;
                            }
                        }
                    }
                }
            }
        }
    }
    if (!(mode & ORC_EDGE)) return 0;
    /* Edge term: every horizontal pair (x,y)-(x+1,y) and vertical pair
     * (x,y)-(x,y+1) inside the image (no pairs across the border). */
    for (int axis = 0; axis < 2; ++axis) {
        int dx = axis == 0 ? 1 : 0, dy = axis == 0 ? 0 : 1;
        for (int y = y0 < 0 ? 0 : y0; y < (y1 > H ? H : y1) && y + dy < H; ++y) {
            for (int x = 0; x + dx < W; ++x) {
                int xa = x, ya = y, xb = x + dx, yb = y + dy;
                size_t pa = (size_t)ya * W + xa, pb = (size_t)yb * W + xb;
                int ta = index[pa], tb = index[pb];
                if (ta == tb) continue; /* same triangle: no edge (Sec. 4.3) */
                counts[0]++;
                /* Eq. 11: dL/dp_AB = 1/2 (dL/dI_A + dL/dI_B)(I_A - I_B), summed over
                 * the channels of the image, with p increasing from A towards B. */
                double dLdp = 0.0, dLdp_mag = 0.0;
                for (int c = 0; c < C; ++c) {
                    double gm = 0.5 * ((double)grad_image[pa * C + c] + (double)grad_image[pb * C + c]);
                    dLdp += gm * (image[pa * C + c] - image[pb * C + c]);
                    /* conditioning w.r.t. the image values: |g| (|I_A| + |I_B|) */
                    dLdp_mag += fabs(gm) * (fabs(image[pa * C + c]) + fabs(image[pb * C + c]));
                }
                /* Edge classification (Sec. 4.3, Supp. A.2). */
                int fg = -1; /* 0: A's fragment overhangs, 1: B's */
                if (ta < 0 || tb < 0) {
                    fg = ta >= 0 ? 0 : 1; /* one valid id: a primitive over the background */
                } else {
                    int b_in_a = orc_covers_pixel(snap, flags, tris, ta, xb, yb);
                    int a_in_b = orc_covers_pixel(snap, flags, tris, tb, xa, ya);
                    if (!b_in_a && !a_in_b) { counts[2]++; continue; } /* adjacent: no scatter */
                    if (b_in_a && a_in_b) {
                        if (!(mode & ORC_INTERSECT)) { counts[5]++; continue; }
                        /* Intersection (Sec. 4.4, Eq. 12, Supp. A.3): for each side v
                         * with the other side f fixed, in the (axis, zeta) slice,
                         * dp/dr = -n^f_z / (n^f^T [[0,1],[-1,0]] n^v), and the
                         * fragment moves along n^v. */
                        double NA[3], NB[3];
                        tri_normal(scr, tris + 3 * (size_t)ta, NA);
                        tri_normal(scr, tris + 3 * (size_t)tb, NB);
                        double nA[2] = {NA[axis], NA[2]}, nB[2] = {NB[axis], NB[2]};
                        double den_a = nB[0] * nA[1] - nB[1] * nA[0]; /* v = A, f = B */
                        double mag = hypot(nA[0], nA[1]) * hypot(nB[0], nB[1]);
                        if (fabs(den_a) <= 1e-12 * mag) { counts[4]++; continue; }
                        counts[3]++;
                        double dpdr_a = -nB[1] / den_a;
                        double den_b = nA[0] * nB[1] - nA[1] * nB[0]; /* v = B, f = A */
                        double dpdr_b = -nA[1] / den_b;
                        double ga[3] = {0, 0, 0}, gb[3] = {0, 0, 0}, ma[3] = {0, 0, 0}, mb[3] = {0, 0, 0};
                        ga[axis] = dLdp * dpdr_a * nA[0];
                        ga[2] = dLdp * dpdr_a * nA[1];
                        gb[axis] = dLdp * dpdr_b * nB[0];
                        gb[2] = dLdp * dpdr_b * nB[1];
                        ma[axis] = dLdp_mag * fabs(dpdr_a * nA[0]);
                        ma[2] = dLdp_mag * fabs(dpdr_a * nA[1]);
                        mb[axis] = dLdp_mag * fabs(dpdr_b * nB[0]);
                        mb[2] = dLdp_mag * fabs(dpdr_b * nB[1]);
                        gather(scr, tris, ta, xa, ya, ga, grad_scr, ma, grad_abs);
                        gather(scr, tris, tb, xb, yb, gb, grad_scr, mb, grad_abs);
                        continue;
                    }
                    /* Overhang: the primitive on top is the one whose pixel centre
                     * lies inside the other pixel's triangle (the other triangle
                     * continues underneath it). */
                    fg = a_in_b ? 0 : 1;
                }
                counts[1]++;
                /* Overhang: dp/dr = 1 on the pair axis for the foreground fragment,
                 * 0 for the covered one (Sec. 4.3). */
                double g[3] = {0, 0, 0}, m[3] = {0, 0, 0};
                g[axis] = dLdp;
                m[axis] = dLdp_mag;
                if (mode & ORC_EXACT_CROSSING) {
                    int vv[2];
                    double ww[2];
                    int ok = fg == 0 ? orc_crossing_weights(scr, snap, tris + 3 * (size_t)ta, xa, ya, xb, yb, axis, vv, ww)
                                     : orc_crossing_weights(scr, snap, tris + 3 * (size_t)tb, xb, yb, xa, ya, axis, vv, ww);
                    if (ok) {
                        for (int e = 0; e < 2; ++e) {
                            grad_scr[3 * (size_t)vv[e] + axis] += ww[e] * dLdp;
                            if (grad_abs) grad_abs[3 * (size_t)vv[e] + axis] += ww[e] * dLdp_mag;
                        }
                        continue;
                    }
                }
                if (fg == 0) gather(scr, tris, ta, xa, ya, g, grad_scr, m, grad_abs);
                else gather(scr, tris, tb, xb, yb, g, grad_scr, m, grad_abs);
            }
        }
    }
    return 0;
}

int orc_backward(const double* scr, const int64_t* snap, const int32_t* flags, int V,
                 const int32_t* tris, const int32_t* index, int H, int W,
                 const double* image, const float* grad_image, const float* attr, const float* tex,
                 const orc_shading* sh, int mode, double* grad_scr, double* grad_attr, int64_t* counts,
                 double* grad_abs, double* grad_attr_abs)
{
    return orc_backward_rows(scr, snap, flags, V, tris, index, H, W, image, grad_image, attr, tex, sh, mode,
                             grad_scr, grad_attr, counts, grad_abs, grad_attr_abs, 0, H);
}

/* ------------------------------------------------------------------------
 * Texel-cell ambiguity (test helper, not part of the method).  The bilinear
 * sampler's derivative jumps where the texel coordinate x = u*TW - 1/2 crosses
 * an integer (or y reaches a clamp edge).  A pixel is flagged when x or y lies
 * within eps of such a point, eps being a bound of the FP32 rounding error of
 * the texel coordinate when it is formed as the exact x_0 = u_0 TW - 1/2 plus the
 * offset sum_i b_i (x_i - x_0):  eps = 32 ulp TW sum_i |b_i||u_i - u_0| + 4 ulp,
 * with ulp the unit roundoff of that evaluation: 2^-24 for FP32; for an FP64
 * evaluation a deliberately generous 2^-40 (the FP64 error of the same steps is
 * ~2^-50 relative).  Either one-sided derivative is correct at such pixels.
 * ------------------------------------------------------------------------ */
static int near_boundary(double x, double eps) { double f = x - floor(x); return f <= eps || 1.0 - f <= eps; }

int orc_texel_ambiguity(const double* scr, const int32_t* tris, const int32_t* index, int H, int W,
                        const float* attr, const orc_shading* sh, double ulp, uint8_t* flags /* [H,W] */)
{
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            flags[p] = 0;
            int t = index[p];
            if (t < 0 || sh->uv_offset < 0) continue;
            const int32_t* tri = tris + 3 * (size_t)t;
            double lam[3], b[3], s = 0.0;
            screen_lambda(scr, tri, x + 0.5, y + 0.5, lam);
            for (int i = 0; i < 3; ++i) s += lam[i] * scr[3 * tri[i] + 2];
            for (int i = 0; i < 3; ++i) b[i] = lam[i] * scr[3 * tri[i] + 2] / s;
            for (int axis = 0; axis < 2; ++axis) {
                double a0 = attr[(size_t)tri[0] * sh->C_attr + sh->uv_offset + axis];
                double u = 0.0, ext = 0.0;
                for (int i = 0; i < 3; ++i) {
                    double ai = attr[(size_t)tri[i] * sh->C_attr + sh->uv_offset + axis];
                    u += b[i] * ai;
                    ext += fabs(b[i]) * fabs(ai - a0);
                }
                int n = axis == 0 ? sh->tex_w : sh->tex_h;
                double xc = u * n - 0.5;
                double eps = n * 32.0 * ulp * ext + 4.0 * ulp * fabs(xc - floor(xc)) + 1e-12;
                int amb = 0;
                if (axis == 0) amb = near_boundary(xc, eps);
                else amb = fabs(xc) <= eps || fabs(xc - (n - 1)) <= eps || (xc > 0 && xc < n - 1 && near_boundary(xc, eps));
                if (amb) flags[p] = 1;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Vertex transform backward (Supp. B: "a straightforward differentiation of
 * the forward pass"): grad_world += R^T J^T grad_scr with J = d(x_s, y_s,
 * zeta)/d(X_c, Y_c, Z_c).
 * ------------------------------------------------------------------------ */
void orc_project_backward(const float* verts, int V, const orc_camera* cam, const double* grad_scr,
                          double* grad_verts /* [V,3], accumulated */)
{
    const double* R = cam->R;
    for (int v = 0; v < V; ++v) {
        double x = verts[3 * v + 0], y = verts[3 * v + 1], z = verts[3 * v + 2];
        double Xc = ((R[0] * x + R[1] * y) + R[2] * z) + cam->t[0];
        double Yc = ((R[3] * x + R[4] * y) + R[5] * z) + cam->t[1];
        double Zc = ((R[6] * x + R[7] * y) + R[8] * z) + cam->t[2];
        if (!(Zc > cam->znear)) continue;
        const double* g = grad_scr + 3 * (size_t)v;
        double iz = 1.0 / Zc;
        double gX = g[0] * cam->fx * iz;
        double gY = g[1] * cam->fy * iz;
        double gZ = -g[0] * cam->fx * Xc * iz * iz - g[1] * cam->fy * Yc * iz * iz - g[2] * iz * iz;
        grad_verts[3 * v + 0] += R[0] * gX + R[3] * gY + R[6] * gZ;
        grad_verts[3 * v + 1] += R[1] * gX + R[4] * gY + R[7] * gZ;
        grad_verts[3 * v + 2] += R[2] * gX + R[5] * gY + R[8] * gZ;
    }
}

/* ------------------------------------------------------------------------
 * Forward gradients (Sec. 5, "forward gradients"): the per-pixel derivative of
 * the shaded image with respect to one scene parameter theta, given the
 * parameter's effect on the projected vertices, tangent[V,3] =
 * d(x_s, y_s, zeta)/d theta.  It is the transpose of orc_backward's linear
 * map: for every cotangent image g, sum_p g_p . out_p = sum_v grad_scr_v . tangent_v.
 *
 * Interior: the 9 vertex derivatives of the pixel's dual-number shading dotted
 * with its vertices' tangents.  Edge: a scattering pair (A, B) (same
 * classification as orc_backward) with micro-edge position p (increasing from
 * A to B) moves by dp/dtheta; Eq. 11 says that changes I_A and I_B each by
 * 1/2 (I_A - I_B) dp/dtheta.  The moving fragment is r = sum_i lambda_i v_i at
 * its pixel centre, so dr/dtheta = sum_i lambda_i tangent_i; overhang:
 * dp/dtheta = the pair-axis component of the foreground fragment's dr;
 * intersection: the sum over both fragments of Eq. 12's dp/dr times the slice
 * normal n^v dotted with that fragment's (axis, zeta) motion.
 * out and out_abs (the sum of the magnitudes of every term, or NULL) are
 * [H,W,C] and accumulated.
 * ------------------------------------------------------------------------ */
static void frag_tangent(const double* scr, const int32_t* tris, int t, int x, int y, const double* tangent,
                         double dr[3], double dr_abs[3])
{
    const int32_t* tri = tris + 3 * (size_t)t;
    double lam[3];
    screen_lambda(scr, tri, x + 0.5, y + 0.5, lam);
    for (int q = 0; q < 3; ++q) {
        dr[q] = 0.0;
        dr_abs[q] = 0.0;
        for (int i = 0; i < 3; ++i) {
            dr[q] += lam[i] * tangent[3 * (size_t)tri[i] + q];
            dr_abs[q] += fabs(lam[i] * tangent[3 * (size_t)tri[i] + q]);
        }
    }
}

int orc_forward_grad(const double* scr, const int64_t* snap, const int32_t* flags, int V,
                     const int32_t* tris, const int32_t* index, int H, int W,
                     const double* image /* [H,W,C] */, const float* attr, const float* tex,
                     const orc_shading* sh, int mode, const double* tangent /* [V,3] */,
                     double* out /* [H,W,C] */, double* out_abs /* [H,W,C] or NULL */)
{
    const int C = sh->C;
    dual I[64];
    if (C > 64) return -1;
    (void)V;
    if (mode & ORC_INTERIOR) {
        for (int y = 0; y < H; ++y) {
            for (int x = 0; x < W; ++x) {
                size_t p = (size_t)y * W + x;
                int t = index[p];
                if (t < 0) continue;
                const int32_t* tri = tris + 3 * (size_t)t;
                shade_pixel_dual(scr, snap, tri, x + 0.5, y + 0.5, attr, tex, sh, I);
                for (int c = 0; c < C; ++c) {
                    double acc = 0.0, mag = 0.0;
                    for (int m = 0; m < 3; ++m)
                        for (int q = 0; q < 3; ++q) {
                            const double tq = tangent[3 * (size_t)tri[m] + q];
                            acc += I[c].d[3 * m + q] * tq;
                            mag += I[c].m[3 * m + q] * fabs(tq);
                        }
                    out[p * C + c] += acc;
                    if (out_abs) out_abs[p * C + c] += mag;
                }
            }
        }
    }
    if (!(mode & ORC_EDGE)) return 0;
    for (int axis = 0; axis < 2; ++axis) {
        int dx = axis == 0 ? 1 : 0, dy = axis == 0 ? 0 : 1;
        for (int y = 0; y + dy < H; ++y) {
            for (int x = 0; x + dx < W; ++x) {
                int xa = x, ya = y, xb = x + dx, yb = y + dy;
                size_t pa = (size_t)ya * W + xa, pb = (size_t)yb * W + xb;
                int ta = index[pa], tb = index[pb];
                if (ta == tb) continue;
                double dpdt = 0.0, dpdt_abs = 0.0;
                int fg = -1;
                if (ta < 0 || tb < 0) {
                    fg = ta >= 0 ? 0 : 1;
                } else {
                    int b_in_a = orc_covers_pixel(snap, flags, tris, ta, xb, yb);
                    int a_in_b = orc_covers_pixel(snap, flags, tris, tb, xa, ya);
                    if (!b_in_a && !a_in_b) continue;
                    if (b_in_a && a_in_b) {
                        if (!(mode & ORC_INTERSECT)) continue;
                        double NA[3], NB[3];
                        tri_normal(scr, tris + 3 * (size_t)ta, NA);
                        tri_normal(scr, tris + 3 * (size_t)tb, NB);
                        double nA[2] = {NA[axis], NA[2]}, nB[2] = {NB[axis], NB[2]};
                        double den_a = nB[0] * nA[1] - nB[1] * nA[0];
                        double mag = hypot(nA[0], nA[1]) * hypot(nB[0], nB[1]);
                        if (fabs(den_a) <= 1e-12 * mag) continue;
                        double dpdr_a = -nB[1] / den_a;
                        double den_b = nA[0] * nB[1] - nA[1] * nB[0];
                        double dpdr_b = -nA[1] / den_b;
                        double dra[3], drb[3], dra_abs[3], drb_abs[3];
                        frag_tangent(scr, tris, ta, xa, ya, tangent, dra, dra_abs);
                        frag_tangent(scr, tris, tb, xb, yb, tangent, drb, drb_abs);
                        dpdt = dpdr_a * (nA[0] * dra[axis] + nA[1] * dra[2]) +
                               dpdr_b * (nB[0] * drb[axis] + nB[1] * drb[2]);
                        dpdt_abs = fabs(dpdr_a) * (fabs(nA[0]) * dra_abs[axis] + fabs(nA[1]) * dra_abs[2]) +
                                   fabs(dpdr_b) * (fabs(nB[0]) * drb_abs[axis] + fabs(nB[1]) * drb_abs[2]);
                    } else {
                        fg = a_in_b ? 0 : 1;
                    }
                }
                if (fg >= 0) {
                    int vv[2];
                    double ww[2];
                    int ok = 0;
                    if (mode & ORC_EXACT_CROSSING)
                        ok = fg == 0 ? orc_crossing_weights(scr, snap, tris + 3 * (size_t)ta, xa, ya, xb, yb, axis, vv, ww)
                                     : orc_crossing_weights(scr, snap, tris + 3 * (size_t)tb, xb, yb, xa, ya, axis, vv, ww);
                    if (ok) {
                        dpdt = ww[0] * tangent[3 * (size_t)vv[0] + axis] + ww[1] * tangent[3 * (size_t)vv[1] + axis];
                        dpdt_abs = fabs(ww[0] * tangent[3 * (size_t)vv[0] + axis]) +
                                   fabs(ww[1] * tangent[3 * (size_t)vv[1] + axis]);
                    } else {
                        double dr[3], dr_abs[3];
                        if (fg == 0) frag_tangent(scr, tris, ta, xa, ya, tangent, dr, dr_abs);
                        else frag_tangent(scr, tris, tb, xb, yb, tangent, dr, dr_abs);
                        dpdt = dr[axis];
                        dpdt_abs = dr_abs[axis];
                    }
                }
                for (int c = 0; c < C; ++c) {
                    const double h = 0.5 * (image[pa * C + c] - image[pb * C + c]);
                    out[pa * C + c] += h * dpdt;
                    out[pb * C + c] += h * dpdt;
                    if (out_abs) {
                        const double hm = 0.5 * (fabs(image[pa * C + c]) + fabs(image[pb * C + c])) * dpdt_abs;
                        out_abs[pa * C + c] += hm;
                        out_abs[pb * C + c] += hm;
                    }
                }
            }
        }
    }
    return 0;
}

/* Tangent of the projected vertices, d(x_s, y_s, zeta) = J(X_c) R d(X_w), for a world-space vertex tangent
 * (the forward counterpart of orc_project_backward); vertices at or before the near plane get 0. */
void orc_project_jvp(const float* verts, int V, const orc_camera* cam, const double* tangent_world,
                     double* tangent_scr /* [V,3] */)
{
    const double* R = cam->R;
    for (int v = 0; v < V; ++v) {
        double x = verts[3 * v + 0], y = verts[3 * v + 1], z = verts[3 * v + 2];
        double Xc = ((R[0] * x + R[1] * y) + R[2] * z) + cam->t[0];
        double Yc = ((R[3] * x + R[4] * y) + R[5] * z) + cam->t[1];
        double Zc = ((R[6] * x + R[7] * y) + R[8] * z) + cam->t[2];
        double* o = tangent_scr + 3 * (size_t)v;
        if (!(Zc > cam->znear)) { o[0] = o[1] = o[2] = 0.0; continue; }
        const double* d = tangent_world + 3 * (size_t)v;
        double dX = R[0] * d[0] + R[1] * d[1] + R[2] * d[2];
        double dY = R[3] * d[0] + R[4] * d[1] + R[5] * d[2];
        double dZ = R[6] * d[0] + R[7] * d[1] + R[8] * d[2];
        double iz = 1.0 / Zc;
        o[0] = cam->fx * (dX * Zc - Xc * dZ) * iz * iz;
        o[1] = cam->fy * (dY * Zc - Yc * dZ) * iz * iz;
        o[2] = -dZ * iz * iz;
    }
}
