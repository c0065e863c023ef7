// abi.cu -- the extern "C" entry points of libmer.so declared in include/mer.h:
// host-side argument validation, then the kernel launches of the other units.
#include <cuda_runtime.h>

#include <cstdint>

#include "mer_device.cuh"

extern "C" int mer_launch_project(const float*, int, const mer_camera*, int, mer_vertex*, cudaStream_t);
extern "C" int mer_launch_project_screen(const double*, int, int, mer_vertex*, cudaStream_t);
extern "C" int mer_launch_project_backward(int, const mer_camera*, int, const mer_vertex*, const double*, float*,
                                           cudaStream_t);
extern "C" size_t mer_raster_workspace_size(int, int, int, int, int, int, long long);
extern "C" int mer_launch_rasterize(const mer_vertex*, int, const int*, int, int, int, int, int, void*, size_t, int*,
                                    float*, float*, unsigned char*, cudaStream_t);
extern "C" int mer_launch_shade(const mer_vertex*, int, const int*, int, int, int, int, const int*, const float*,
                                const float*, const float*, const mer_shading*, float*, void*, cudaStream_t);
extern "C" int mer_launch_backward(const mer_vertex*, int, const int*, int, int, int, int, const int*,
                                   const unsigned char*, const float*, const float*, const float*, const float*,
                                   const mer_shading*, int, double*, float*, void*, cudaStream_t);

extern "C" size_t mer_batch_raster_workspace_size(long long, long long, long long);
extern "C" int mer_launch_batch_rasterize(const mer_vertex*, const int*, const mer_item*, int, long long, long long, int,
                                          void*, size_t, int*, float*, float*, unsigned char*, int, cudaStream_t);
extern "C" int mer_launch_batch_render(const mer_vertex*, const int*, const mer_item*, int, long long, long long,
                                       long long, int, void*, size_t, int*, float*, float*, unsigned char*,
                                       const float*, const float*, const float*, const mer_shading*, float*, int,
                                       cudaStream_t);
extern "C" int mer_launch_forward_grad(const mer_vertex*, int, const int*, int, int, int, int, const int*, const float*,
                                       const float*, const float*, const float*, const mer_shading*, int, float*, void*,
                                       cudaStream_t);
extern "C" int mer_launch_project_jvp(const float*, int, const mer_camera*, int, const mer_vertex*, float*, cudaStream_t);
extern "C" int mer_launch_project_batch(const float*, const mer_camera*, const mer_item*, int, long long, mer_vertex*,
                                        cudaStream_t);
extern "C" int mer_launch_project_backward_batch(const mer_camera*, const mer_item*, int, long long, long long,
                                                 const mer_vertex*, const double*, float*, void*, cudaStream_t);
extern "C" int mer_launch_shade_batch(const mer_vertex*, const int*, const mer_item*, int, long long, const int*,
                                      const float*, const float*, const float*, const mer_shading*, float*, void*,
                                      cudaStream_t);
extern "C" int mer_launch_backward_batch(const mer_vertex*, const int*, const mer_item*, int, long long, const int*,
                                         const unsigned char*, const float*, const float*, const float*,
                                         const float*, const mer_shading*, int, double*, float*, void*, int, double,
                                         cudaStream_t);
extern "C" size_t mer_det_workspace_size(long long, long long, int);
extern "C" int mer_launch_backward_det(const mer_vertex*, int, const int*, int, int, int, int, const int*, const float*,
                                       const float*, const float*, const float*, const mer_shading*, int, double*,
                                       float*, void*, cudaStream_t);
extern "C" int mer_launch_backward_det_batch(const mer_vertex*, const int*, const mer_item*, int, long long, long long,
                                             long long, const int*, const float*, const float*, const float*,
                                             const float*, const mer_shading*, int, double*, float*, void*,
                                             cudaStream_t);

namespace {

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

inline bool dims_ok(int n, int H, int W) {
    if (n < 0 || H < 0 || W < 0) return false;
    if (H > mer::kMaxDim || W > mer::kMaxDim) return false;
    return (long long)n * H * W < (1LL << 31);
}

inline bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

constexpr int kAllTerms = MER_EDGE | MER_INTERIOR | MER_INTERSECT | MER_EXACT_CROSSING | MER_DETERMINISTIC;

// Attribute-gradient channels a backward pass writes: the interpolated channels, or (u, v) in texture mode.
inline int attr_grad_channels(const mer_shading* sh, const float* grad_attr) {
    if (!grad_attr) return 0;
    return sh->uv_offset < 0 ? sh->n_main : 2;
}

bool shading_ok(const mer_shading* sh) {
    if (!sh) return false;
    if (sh->C < 1 || sh->C > mer::kMaxC) return false;
    if (sh->n_main < 0 || sh->n_main > sh->C) return false;
    if (sh->mask_ch >= sh->C || sh->depth_ch >= sh->C) return false;
    if (sh->mask_ch >= 0 && sh->mask_ch < sh->n_main) return false;
    if (sh->depth_ch >= 0 && sh->depth_ch < sh->n_main) return false;
    if (sh->mask_ch >= 0 && sh->mask_ch == sh->depth_ch) return false;
    if (sh->backface_ch >= sh->C || (sh->backface_ch >= 0 && sh->backface_ch < sh->n_main)) return false;
    if (sh->backface_ch >= 0 && (sh->backface_ch == sh->mask_ch || sh->backface_ch == sh->depth_ch)) return false;
    if (sh->tex_c != 0 && sh->tex_c < sh->n_main) return false;
    if (sh->precise != 0 && sh->precise != 1) return false;
    if (sh->uv_offset >= 0) {
        if (sh->uv_offset + 2 > sh->C_attr || sh->tex_h < 1 || sh->tex_w < 1) return false;
    } else if (sh->n_main > sh->C_attr) {
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

const char* mer_strerror(int code) {
    switch (code) {
        case MER_OK: return "ok";
        case MER_EINVAL: return "invalid argument";
        case MER_ECUDA: return "CUDA error";
        case MER_EOVERFLOW: return "bin list overflow: workspace too small";
        case MER_ERANGE: return "triangle or index-image entry out of range";
        case MER_EFIXED: return "a deterministic-mode gradient contribution exceeded the fixed-point range";
        default: return "unknown error";
    }
}

int mer_version(void) { return 1; }

size_t mer_workspace_size(int V, int T, int n, int H, int W, int tile, int64_t bin_capacity) {
    if (V < 0 || T < 0 || !dims_ok(n, H, W) || (tile != 8 && tile != 16 && tile != 32)) return 0;
    return mer_raster_workspace_size(V, T, n, H, W, tile, (long long)bin_capacity);
}

int mer_project(const float* verts, int V, const mer_camera* cams, int n, mer_vertex* vpix, void* stream) {
    if (V < 0 || n < 0) return MER_EINVAL;
    if ((long long)V * n == 0) return MER_OK;
    if (!verts || !cams || !vpix) return MER_EINVAL;
    return mer_launch_project(verts, V, cams, n, vpix, S(stream));
}

int mer_rasterize_world(const float* verts, int V, const int32_t* tris, int T, const mer_camera* cams, int n, int H,
                        int W, int tile, void* workspace, size_t workspace_bytes, int32_t* index, float* depth,
                        float* bary, mer_vertex* vpix, void* stream) {
    if (V < 0 || T < 0 || !dims_ok(n, H, W)) return MER_EINVAL;
    if ((long long)n * H * W == 0) return MER_OK;
    if (V > 0 && (!verts || !cams || !vpix)) return MER_EINVAL;
    const int rc = mer_project(verts, V, cams, n, vpix, stream);
    if (rc != MER_OK) return rc;
    return mer_rasterize(vpix, V, tris, T, n, H, W, tile, workspace, workspace_bytes, index, depth, bary, nullptr,
                         stream);
}

size_t mer_backward_workspace_size(int64_t vertex_rows, int64_t attr_rows, int attr_channels, int terms) {
    if (vertex_rows < 0 || attr_rows < 0 || attr_channels < 0) return 0;
    if (!(terms & MER_DETERMINISTIC)) return 256;
    return mer_det_workspace_size((long long)vertex_rows, (long long)attr_rows, attr_channels);
}

int mer_project_screen(const double* scr, int V, int n, mer_vertex* vpix, void* stream) {
    if (V < 0 || n < 0) return MER_EINVAL;
    if ((long long)V * n == 0) return MER_OK;
    if (!scr || !vpix) return MER_EINVAL;
    return mer_launch_project_screen(scr, V, n, vpix, S(stream));
}

int mer_rasterize(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W, int tile,
                  void* workspace, size_t workspace_bytes, int32_t* index, float* depth, float* bary, uint8_t* cover,
                  void* stream) {
    if (V < 0 || T < 0 || !dims_ok(n, H, W)) return MER_EINVAL;
    if (tile != 8 && tile != 16 && tile != 32) return MER_EINVAL;
    if ((long long)n * H * W == 0) return MER_OK;
    if (!workspace || !aligned256(workspace) || !index) return MER_EINVAL;
    if (T > 0 && (!tris || !vpix)) return MER_EINVAL;
    if (workspace_bytes < mer_raster_workspace_size(V, T, n, H, W, tile, 1)) return MER_EINVAL;
    return mer_launch_rasterize(vpix, V, tris, T, n, H, W, tile, workspace, workspace_bytes, index, depth, bary,
                                cover, S(stream));
}

int mer_shade(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W, const int32_t* index,
              const float* attr, const float* tex, const float* bg_host, const mer_shading* sh, float* image,
              void* status_ws, void* stream) {
    if (V < 0 || T < 0 || !dims_ok(n, H, W) || !shading_ok(sh)) return MER_EINVAL;
    if ((long long)n * H * W == 0) return MER_OK;
    if (!index || !image) return MER_EINVAL;
    if (T > 0 && (!tris || !vpix)) return MER_EINVAL;
    if (sh->n_main > 0 && !attr) return MER_EINVAL;
    if (sh->uv_offset >= 0 && !tex) return MER_EINVAL;
    if (status_ws && !aligned256(status_ws)) return MER_EINVAL;
    return mer_launch_shade(vpix, V, tris, T, n, H, W, index, attr, tex, bg_host, sh, image, status_ws, S(stream));
}

int mer_backward(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W, const int32_t* index,
                 const uint8_t* cover, const float* image, const float* grad_image, const float* attr, const float* tex,
                 const mer_shading* sh, int terms, double* grad_vpix, float* grad_attr, void* workspace,
                 size_t workspace_bytes, void* stream) {
    if (V < 0 || T < 0 || !dims_ok(n, H, W) || !shading_ok(sh)) return MER_EINVAL;
    if (terms & ~kAllTerms) return MER_EINVAL;
    const int base_terms = terms & (MER_EDGE | MER_INTERIOR);
    if ((long long)n * H * W == 0 || base_terms == 0) return MER_OK;
    if (!index || !grad_image || (V > 0 && !grad_vpix)) return MER_EINVAL;
    if (T > 0 && (!tris || !vpix)) return MER_EINVAL;
    if ((terms & MER_EDGE) && !image) return MER_EINVAL;
    if ((terms & MER_INTERIOR) && sh->n_main > 0 && !attr) return MER_EINVAL;
    if ((terms & MER_INTERIOR) && sh->uv_offset >= 0 && !tex) return MER_EINVAL;
    if (grad_attr && sh->uv_offset < 0 && sh->n_main > 4) return MER_EINVAL;  // attribute gradients: <= 4 channels
    if (workspace && (!aligned256(workspace) || workspace_bytes < 256)) return MER_EINVAL;
    if (terms & MER_DETERMINISTIC) {
        const int A = attr_grad_channels(sh, grad_attr);
        if (!workspace || workspace_bytes < mer_backward_workspace_size((int64_t)n * V, V, A, terms)) return MER_EINVAL;
        return mer_launch_backward_det(vpix, V, tris, T, n, H, W, index, image, grad_image, attr, tex, sh, terms,
                                       grad_vpix, grad_attr, workspace, S(stream));
    }
    return mer_launch_backward(vpix, V, tris, T, n, H, W, index, cover, image, grad_image, attr, tex, sh, terms, grad_vpix,
                               grad_attr, workspace, S(stream));
}

int mer_forward_grad(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W,
                     const int32_t* index, const float* image, const float* tangent, const float* attr,
                     const float* tex, const mer_shading* sh, int terms, float* out, void* status_ws, void* stream) {
    if (V < 0 || T < 0 || !dims_ok(n, H, W) || !shading_ok(sh)) return MER_EINVAL;
    if (terms & ~(MER_EDGE | MER_INTERIOR | MER_INTERSECT | MER_EXACT_CROSSING)) return MER_EINVAL;
    if ((long long)n * H * W == 0) return MER_OK;
    if (!index || !out || (V > 0 && !tangent)) return MER_EINVAL;
    if (T > 0 && (!tris || !vpix)) return MER_EINVAL;
    if ((terms & MER_EDGE) && !image) return MER_EINVAL;
    if ((terms & MER_INTERIOR) && sh->n_main > 0 && !attr) return MER_EINVAL;
    if ((terms & MER_INTERIOR) && sh->uv_offset >= 0 && !tex) return MER_EINVAL;
    if (status_ws && !aligned256(status_ws)) return MER_EINVAL;
    return mer_launch_forward_grad(vpix, V, tris, T, n, H, W, index, image, tangent, attr, tex, sh, terms, out,
                                   status_ws, S(stream));
}

int mer_project_jvp(const float* tangent_world, int V, const mer_camera* cams, int n, const mer_vertex* vpix,
                    float* tangent_vpix, void* stream) {
    if (V < 0 || n < 0) return MER_EINVAL;
    if ((long long)V * n == 0) return MER_OK;
    if (!tangent_world || !cams || !vpix || !tangent_vpix) return MER_EINVAL;
    return mer_launch_project_jvp(tangent_world, V, cams, n, vpix, tangent_vpix, S(stream));
}

int mer_edge_grad_backward(const float* image, const float* grad_image, int C, const int32_t* index,
                           const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W,
                           int intersections, double* grad_vpix, void* status_ws, void* stream) {
    mer_shading sh = {0, C, -1, -1, -1, 0, 0, 0, 0, -1, 0};
    return mer_backward(vpix, V, tris, T, n, H, W, index, nullptr, image, grad_image, nullptr, nullptr, &sh,
                        MER_EDGE | (intersections ? MER_INTERSECT : 0), grad_vpix, nullptr, status_ws,
                        status_ws ? 256 : 0, stream);
}

int mer_interpolate_backward(const float* attr, int C_attr, const int32_t* tris, int T, const mer_vertex* vpix, int V,
                             const int32_t* index, int n, int H, int W, const float* grad_out, float* grad_attr,
                             double* grad_vpix, void* status_ws, void* stream) {
    mer_shading sh = {C_attr, C_attr, -1, -1, -1, C_attr, 0, 0, 0, -1, 0};
    return mer_backward(vpix, V, tris, T, n, H, W, index, nullptr, nullptr, grad_out, attr, nullptr, &sh, MER_INTERIOR,
                        grad_vpix, grad_attr, status_ws, status_ws ? 256 : 0, stream);
}

int mer_project_backward(int V, const mer_camera* cams, int n, const mer_vertex* vpix, const double* grad_vpix,
                         float* grad_verts, void* stream) {
    if (V < 0 || n < 0) return MER_EINVAL;
    if ((long long)V * n == 0) return MER_OK;
    if (!cams || !vpix || !grad_vpix || !grad_verts) return MER_EINVAL;
    return mer_launch_project_backward(V, cams, n, vpix, grad_vpix, grad_verts, S(stream));
}

// ---- batched path ----

int mer_batch_plan(mer_item* items, int n_items, int tile, mer_batch_totals* totals) {
    if (!totals || n_items < 0 || (n_items > 0 && !items)) return MER_EINVAL;
    if (tile != 16 && tile != 32 && tile != 64) return MER_EINVAL;
    int64_t vrec = 0, trec = 0, pix = 0, tiles = 0, btiles = 0, mesh_rows = 0;
    double density = 0.0;
    for (int i = 0; i < n_items; ++i) {
        mer_item& m = items[i];
        if (m.V < 0 || m.T < 0 || m.H < 0 || m.W < 0 || m.H > mer::kMaxDim || m.W > mer::kMaxDim || m.cam < 0 ||
            m.vert < 0 || m.tri < 0)
            return MER_EINVAL;
        m.vrec = vrec;
        m.trec = trec;
        m.pix = pix;
        m.tile = tiles;
        m.btile = btiles;
        vrec += m.V;
        trec += m.T;
        pix += (int64_t)m.H * m.W;
        if (m.vert + m.V > mesh_rows) mesh_rows = m.vert + m.V;
        if ((int64_t)m.H * m.W > 0) {
            const double d = (double)m.T / ((double)m.H * (double)m.W);
            if (d > density) density = d;
        }
        tiles += (int64_t)((m.W + tile - 1) / tile) * ((m.H + tile - 1) / tile);
        btiles += (int64_t)((m.W + mer::kBwdTileW - 1) / mer::kBwdTileW) * ((m.H + mer::kBwdTileH - 1) / mer::kBwdTileH);
    }
    const int64_t lim = (int64_t)1 << 31;
    if (vrec >= lim || trec >= lim || pix >= lim || tiles >= lim || btiles >= lim) return MER_EINVAL;
    totals->vrecs = vrec;
    totals->trecs = trec;
    totals->pixels = pix;
    totals->tiles = tiles;
    totals->btiles = btiles;
    totals->n_items = n_items;
    totals->tile = tile;
    totals->mesh_rows = mesh_rows;
    totals->max_tri_density = density;
    return MER_OK;
}

size_t mer_batch_workspace_size(const mer_batch_totals* t, int64_t bin_capacity) {
    if (!t) return 0;
    return mer_batch_raster_workspace_size(t->tiles, t->trecs, (long long)bin_capacity);
}

static bool totals_ok(const mer_batch_totals* t, const mer_item* items) {
    return t && t->n_items >= 0 && (t->n_items == 0 || items) && t->vrecs >= 0 && t->trecs >= 0 && t->pixels >= 0;
}

int mer_batch_project(const float* verts, const mer_camera* cams, const mer_item* items, const mer_batch_totals* t,
                      mer_vertex* vpix, void* stream) {
    if (!totals_ok(t, items)) return MER_EINVAL;
    if (t->vrecs == 0) return MER_OK;
    if (!verts || !cams || !vpix) return MER_EINVAL;
    return mer_launch_project_batch(verts, cams, items, t->n_items, t->vrecs, vpix, S(stream));
}

int mer_batch_rasterize(const mer_vertex* vpix, const int32_t* tris, const mer_item* items, const mer_batch_totals* t,
                        void* workspace, size_t workspace_bytes, int32_t* index, float* depth, float* bary,
                        uint8_t* cover, int persistent_ctas, void* stream) {
    if (!totals_ok(t, items) || (t->tile != 16 && t->tile != 32 && t->tile != 64)) return MER_EINVAL;
    if (t->pixels == 0) return MER_OK;
    if (!workspace || !aligned256(workspace) || !index || persistent_ctas < 0) return MER_EINVAL;
    if (t->trecs > 0 && (!tris || !vpix)) return MER_EINVAL;
    if (workspace_bytes < mer_batch_raster_workspace_size(t->tiles, t->trecs, 1)) return MER_EINVAL;
    return mer_launch_batch_rasterize(vpix, tris, items, t->n_items, t->trecs, t->tiles, t->tile, workspace,
                                      workspace_bytes, index, depth, bary, cover, persistent_ctas, S(stream));
}

int mer_batch_shade(const mer_vertex* vpix, const int32_t* tris, const mer_item* items, const mer_batch_totals* t,
                    const int32_t* index, const float* attr, const float* tex, const float* bg_host,
                    const mer_shading* sh, float* image, void* status_ws, void* stream) {
    if (!totals_ok(t, items) || !shading_ok(sh)) return MER_EINVAL;
    if (t->pixels == 0) return MER_OK;
    if (!index || !image || (t->trecs > 0 && (!tris || !vpix))) return MER_EINVAL;
    if (sh->n_main > 0 && !attr) return MER_EINVAL;
    if (sh->uv_offset >= 0 && !tex) return MER_EINVAL;
    if (status_ws && !aligned256(status_ws)) return MER_EINVAL;
    return mer_launch_shade_batch(vpix, tris, items, t->n_items, t->pixels, index, attr, tex, bg_host, sh, image,
                                  status_ws, S(stream));
}

int mer_batch_render(const mer_vertex* vpix, const int32_t* tris, const mer_item* items, const mer_batch_totals* t,
                     void* workspace, size_t workspace_bytes, int32_t* index, float* depth, float* bary,
                     uint8_t* cover, const float* attr, const float* tex, const float* bg_host, const mer_shading* sh,
                     float* image, int persistent_ctas, void* stream) {
    if (!totals_ok(t, items) || (t->tile != 16 && t->tile != 32 && t->tile != 64) || !shading_ok(sh)) return MER_EINVAL;
    if (t->pixels == 0) return MER_OK;
    if (!workspace || !aligned256(workspace) || !index || !image || persistent_ctas < 0) return MER_EINVAL;
    if (t->trecs > 0 && (!tris || !vpix)) return MER_EINVAL;
    if (sh->n_main > 0 && !attr) return MER_EINVAL;
    if (sh->uv_offset >= 0 && !tex) return MER_EINVAL;
    if (workspace_bytes < mer_batch_raster_workspace_size(t->tiles, t->trecs, 1)) return MER_EINVAL;
    return mer_launch_batch_render(vpix, tris, items, t->n_items, t->trecs, t->tiles, t->pixels, t->tile, workspace,
                                   workspace_bytes, index, depth, bary, cover, attr, tex, bg_host, sh, image, persistent_ctas,
                                   S(stream));
}

int mer_batch_backward(const mer_vertex* vpix, const int32_t* tris, const mer_item* items, const mer_batch_totals* t,
                       const int32_t* index, const uint8_t* cover, const float* image, const float* grad_image,
                       const float* attr, const float* tex, const mer_shading* sh, int terms, double* grad_vpix,
                       float* grad_attr, void* workspace, size_t workspace_bytes, int persistent_ctas, void* stream) {
    if (!totals_ok(t, items) || !shading_ok(sh)) return MER_EINVAL;
    if (terms & ~kAllTerms) return MER_EINVAL;
    if (t->pixels == 0 || (terms & (MER_EDGE | MER_INTERIOR)) == 0) return MER_OK;
    if (!index || !grad_image || (t->vrecs > 0 && !grad_vpix) || (t->trecs > 0 && (!tris || !vpix))) return MER_EINVAL;
    if ((terms & MER_EDGE) && !image) return MER_EINVAL;
    if ((terms & MER_INTERIOR) && sh->n_main > 0 && !attr) return MER_EINVAL;
    if ((terms & MER_INTERIOR) && sh->uv_offset >= 0 && !tex) return MER_EINVAL;
    if (grad_attr && sh->uv_offset < 0 && sh->n_main > 4) return MER_EINVAL;  // attribute gradients: <= 4 channels
    if (!workspace || !aligned256(workspace) || workspace_bytes < 256 || persistent_ctas < 0) return MER_EINVAL;
    if (terms & MER_DETERMINISTIC) {
        const int A = attr_grad_channels(sh, grad_attr);
        if (workspace_bytes < mer_backward_workspace_size(t->vrecs, t->mesh_rows, A, terms)) return MER_EINVAL;
        return mer_launch_backward_det_batch(vpix, tris, items, t->n_items, t->pixels, t->vrecs, t->mesh_rows, index,
                                             image, grad_image, attr, tex, sh, terms, grad_vpix, grad_attr, workspace,
                                             S(stream));
    }
    return mer_launch_backward_batch(vpix, tris, items, t->n_items, t->btiles, index, cover, image, grad_image, attr,
                                     tex, sh, terms, grad_vpix, grad_attr, workspace, persistent_ctas,
                                     t->max_tri_density, S(stream));
}

int mer_batch_project_backward(const mer_camera* cams, const mer_item* items, const mer_batch_totals* t,
                               const mer_vertex* vpix, const double* grad_vpix, float* grad_verts, void* workspace,
                               size_t workspace_bytes, void* stream) {
    if (!totals_ok(t, items)) return MER_EINVAL;
    if (t->vrecs == 0) return MER_OK;
    if (!cams || !vpix || !grad_vpix || !grad_verts) return MER_EINVAL;
    if (workspace && (!aligned256(workspace) ||
                      workspace_bytes < mer_backward_workspace_size(t->mesh_rows, 0, 0, MER_DETERMINISTIC)))
        return MER_EINVAL;
    return mer_launch_project_backward_batch(cams, items, t->n_items, t->vrecs, t->mesh_rows, vpix, grad_vpix,
                                             grad_verts, workspace, S(stream));
}

int mer_sync_status(void* workspace, int64_t* total_bins, void* stream) {
    if (!workspace || !aligned256(workspace)) return MER_EINVAL;
    mer::WsHeader h;
    if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess) return MER_ECUDA;
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return MER_ECUDA;
    if (total_bins) *total_bins = h.total_bins;
    if (h.status != 0) {
        const int zero = 0;
        if (cudaMemcpyAsync(workspace, &zero, sizeof(int), cudaMemcpyHostToDevice, S(stream)) != cudaSuccess)
            return MER_ECUDA;
        if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return MER_ECUDA;
    }
    if (h.status & mer::kStatusOverflow) return MER_EOVERFLOW;
    if (h.status & mer::kStatusRange) return MER_ERANGE;
    if (h.status & mer::kStatusFixed) return MER_EFIXED;
    return MER_OK;
}

}  // extern "C"
