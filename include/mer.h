/*
 * mer.h -- C-ABI of the GB300 micro-edge rasterizer-gradient library (libmer.so).
 *
 * Method: "Rasterized Edge Gradients: Handling Discontinuities Differentiably"
 * (EdgeGrad, arXiv 2405.02508).  Forward: an unmodified z-buffered triangle
 * rasterizer (index, depth, barycentrics) and deferred shading (interpolated
 * attributes, bilinear texture, coverage mask, depth).  Backward: the micro-edge
 * term -- for every horizontally or vertically adjacent pixel pair whose
 * triangle ids differ, dL/dp = 1/2 (dL/dI_A + dL/dI_B)(I_A - I_B) (Eq. 11),
 * scattered to the fragments through dp/dr (Sec. 4.3 overhang rule, Eq. 12 for
 * intersections) and gathered to the vertices (Sec. 4.2) -- on top of the
 * interior (smooth) term Omega (Eq. 5).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every pointer argument except where stated is a DEVICE pointer.  The caller
 *   owns all memory, including the workspace; the library allocates no device
 *   memory at call time (mer_rasterize_noalloc uses a static device array that
 *   exists from load time; the host call mer_laplacian_csr uses host scratch).
 * - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *   NULL = the legacy default stream).  A call returns MER_OK after queueing its
 *   kernels; argument errors found on the host return at once, without launching.
 *   Errors found on the device (bin overflow, triangle index >= V, index image
 *   entry >= T) set bits of the workspace status word, read by mer_sync_status.
 * - Images are row-major [n, H, W] or [n, H, W, C] (NHWC), float32 unless
 *   stated.  Pixel (x, y) has its centre at (x + 1/2, y + 1/2); y points down.
 *   index = -1 marks background.
 * - Gradient outputs ACCUMULATE (+=); zero them first.
 * - Sizes: 1 <= H, W <= 8192; V, T < 2^31; n * H * W < 2^31.
 */
#ifndef MER_H
#define MER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
enum {
    MER_OK = 0,
    MER_EINVAL = 1,    /* bad argument (null pointer, size out of range, bad option) */
    MER_ECUDA = 2,     /* a CUDA launch or runtime call failed */
    MER_EOVERFLOW = 3, /* the bin list did not fit in the workspace (mer_sync_status) */
    MER_ERANGE = 4,    /* a triangle or index-image entry was out of range (mer_sync_status) */
    MER_EFIXED = 5     /* a contribution exceeded the fixed-point range of MER_DETERMINISTIC (mer_sync_status) */
};

/* Pinhole camera, OpenCV convention (+X right, +Y down, +Z forward), 136 bytes.
 * X_c = R X_w + t; x_s = fx X_c / Z_c + cx; y_s = fy Y_c / Z_c + cy; zeta = 1 / Z_c.
 * Triangles with a vertex at Z_c <= znear are not drawn (vertex transform
 * module, Supp. B). */
typedef struct mer_camera {
    double R[9]; /* row-major */
    double t[3];
    double fx, fy, cx, cy;
    double znear;
} mer_camera;

/* Projected vertex record, 32 bytes, one per (view, vertex).  The screen position
 * is x_s = X/256 + rx, y_s = Y/256 + ry: X, Y are the positions snapped to 1/256
 * px (round half to even) that decide coverage; rx, ry are the sub-snap
 * residuals that keep values and derivatives on the unsnapped geometry.
 * zeta = 1/Z_c is split as zeta + zeta_lo (float + float residual).
 * flags: bit 0 = in front of the near plane, bit 1 = inside the guard band
 * |X|, |Y| <= 2^29; a triangle is drawn only if all its vertices have both. */
typedef struct mer_vertex {
    int32_t X, Y;
    float rx, ry;
    float zeta, zeta_lo;
    uint32_t flags;
    float pad;
} mer_vertex;

/* Layout of the shaded image [n,H,W,C] (deferred shading, Supp. B).
 * Channels [0, n_main) hold interpolated attribute channels 0..n_main-1
 * (uv_offset < 0), or the bilinear texture [tex_h, tex_w, tex_c] (channels 0..n_main-1 used; tex_c =
 * floats per texel in memory, 0 meaning n_main; tex_c = 4 with a 16-byte aligned texture reads each texel
 * with one 128-bit load) sampled at the
 * interpolated (u, v) = attribute channels (uv_offset, uv_offset+1) with u
 * wrapping and v clamped, texel centres at ((i+1/2)/tex_w, (j+1/2)/tex_h).
 * mask_ch / depth_ch (or -1) hold the coverage mask (1 on triangles) and the
 * depth Z.  Attributes are interpolated perspective-correctly. */
typedef struct mer_shading {
    int n_main;
    int C;
    int uv_offset;
    int mask_ch;
    int depth_ch;
    int C_attr;  /* channels per vertex of `attr` */
    int tex_h, tex_w;
    int tex_c;   /* floats per texel in memory (>= n_main), 0 = n_main */
    int backface_ch; /* channel of the back-face image (Supp. B): 1 where the visible triangle faces away
                        from the camera (snapped screen area > 0 with y down), 0 elsewhere; or -1.  It is
                        constant per triangle, so only the edge term differentiates it. */
    int precise;     /* 0: FP32 shading arithmetic.  1: every shaded value is evaluated in FP64 from the FP32
                        inputs and rounded once to FP32, so the image is the correctly rounded value up to FP64
                        rounding (bit-reproducible against any FP64 evaluation of the same definition, except
                        where the FP64 value lies within a few FP64 ulps of an FP32 rounding boundary).
                        Meant for MER_DETERMINISTIC backward passes, whose edge term reads the image; slower
                        (GB300's FP64 rate is low). */
} mer_shading;

/* Terms computed by mer_backward (bit mask). */
enum {
    MER_EDGE = 1,      /* micro-edge term (Eq. 11, Sec. 4.3, Eq. 12) */
    MER_INTERIOR = 2,  /* interior term Omega through barycentrics/interpolation/texture */
    MER_INTERSECT = 4, /* scatter at geometry intersections (Eq. 12); off = the paper's ablation */
    MER_EXACT_CROSSING = 8, /* option: an overhang pair's gradient goes to the two endpoints of the edge
                              through which the segment between the pixel centres leaves the foreground
                              triangle, weighted by the crossing's position along it (pair axis only),
                              instead of the foreground fragment's barycentrics */
    MER_DETERMINISTIC = 16 /* option: every per-pixel quantity is computed in FP64 from the FP32 inputs and
                              each pixel's contribution to a gradient component is rounded once to a fixed-point
                              number with 52 fractional bits (two 64-bit words: resolution 2^-52); the sums are
                              exact integer sums, so the result does not depend on the order of the additions:
                              bitwise identical from run to run, for any bin tile, grid or stored / recomputed
                              barycentrics.  A contribution of magnitude >= 2^33 sets MER_EFIXED (it is
                              dropped); sums must stay below 2^42 in magnitude.  Needs a workspace of
                              mer_backward_workspace_size bytes (the fixed-point sums live there during the
                              call) and ignores the cover image.  Slower than the default path (FP64). */
};

/* Bits of the optional cover image [n,H,W] uint8 that the rasterizers write beside the index image.  It
 * records which triangles cover each pixel centre, as far as the backward pass needs it to skip pixel pairs
 * that cannot scatter: an edge pair (p, q) with triangles t_p != t_q scatters into p's fragment only if t_q
 * covers p's centre too (Sec. 4.3: p on top of t_q, or an intersection), so when no second triangle of
 * t_q's facing covers p, the pair's classification is known without loading either triangle.  This is an
 * implementation aid of this library; the paper has no counterpart and the results do not change.
 * Facing: "front" = negative snapped area (y down: counter-clockwise on screen), "back" = positive.
 * The counts of front-facing triangles are exact.  Those of back-facing ones leave out back-facing triangles
 * that lie behind the whole bin tile (the raster skips them); such a triangle wins no pixel of that tile, so
 * the counts are exact for pairs inside one bin tile, and a pair from a pixel across the border of its bin
 * tile whose neighbour's triangle is back-facing is always classified in full (the border bits). */
enum {
    MER_COVER_SAME_2 = 1,       /* another triangle with the visible triangle's facing covers the centre */
    MER_COVER_OTHER_1 = 2,      /* a triangle with the other facing covers the centre */
    MER_COVER_WINNER_BACK = 4,  /* the visible triangle (the index) is back-facing */
    MER_COVER_BORDER_L = 8,     /* first column of its bin tile (the pair to the left crosses the border) */
    MER_COVER_BORDER_R = 16,    /* last column */
    MER_COVER_BORDER_T = 32,    /* first row */
    MER_COVER_BORDER_B = 64     /* last row */
};

const char* mer_strerror(int code);
int mer_version(void);

/* Bytes of workspace mer_rasterize needs for these sizes.  Zero the first 256
 * bytes (the status header) once before the first use.  `tile` is the bin
 * tile edge in pixels (8, 16 or 32); `bin_capacity` is the number of
 * (triangle, tile) entries to reserve, 0 for the default 4*n*T + 2*n*tiles.
 * The workspace must be 256-byte aligned. */
size_t mer_workspace_size(int V, int T, int n, int H, int W, int tile, int64_t bin_capacity);

/* Vertex transform (Supp. B): world vertices [V,3] and cameras [n] (device) ->
 * projected vertex records vpix [n,V].  FP64 with a fixed operation order and
 * correctly rounded operations, so the snapped positions are reproducible. */
int mer_project(const float* verts, int V, const mer_camera* cams, int n, mer_vertex* vpix, void* stream);

/* Screen-space input path: scr [n,V,3] float64 (x_s, y_s, zeta) -> vpix [n,V].
 * A vertex with zeta <= 0 is behind the camera. */
int mer_project_screen(const double* scr, int V, int n, mer_vertex* vpix, void* stream);

/* Rasterization module with z-buffer (Supp. B): tile binning and raster.
 * tris [T,3] int32.  Outputs index [n,H,W] int32 (-1 = background), and
 * optionally depth [n,H,W] (Z, 0 on background) and bary [n,H,W,2]
 * (perspective-correct b1, b2); pass NULL to skip them (the other calls never
 * read bary: they re-derive barycentrics from index + vpix).
 * Fill rule: a pixel centre is covered iff s*E_i > 0 for all three edge
 * functions E_i = cross(v_j - P, v_k - P) of the snapped positions (s = sign of
 * the area; both windings drawn), or E_i == 0 on a top-left edge.  Depth test:
 * largest zeta_test = sum_i E_i zeta_i / sum_i E_i, ties to the lower id.
 * The workspace keeps the bins; its contents are not needed afterwards.
 * cover [n,H,W] uint8 or NULL: the MER_COVER_* bits of every pixel (background pixels: only the border
 * bits), to pass to mer_backward with this index image. */
int mer_rasterize(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W,
                  int tile, void* workspace, size_t workspace_bytes,
                  int32_t* index, float* depth, float* bary, uint8_t* cover, void* stream);
/* mer_project followed by mer_rasterize: world-space vertices [V,3] and n cameras in, index / depth /
 * bary out, the projected records written to vpix [n,V] (the other calls take them).  Arguments, errors and
 * workspace as the two calls. */
int mer_rasterize_world(const float* verts, int V, const int32_t* tris, int T, const mer_camera* cams, int n,
                        int H, int W, int tile, void* workspace, size_t workspace_bytes, int32_t* index,
                        float* depth, float* bary, mer_vertex* vpix, void* stream);

/* mer_rasterize without a workspace argument, for callers that cannot allocate device memory at the
 * time they call -- code running while a stream is being captured into a CUDA graph (cudaMalloc is not
 * allowed there), or a host framework or plugin that hands the library its buffers but exposes no
 * device allocator.  The paper has no counterpart: this is a deployment variant of the rasterization
 * module above, with the same arguments, results and status codes.
 *
 * The workspace is a 64 MiB array in the library's own device memory (a file-scope __device__ array:
 * every GPU that loads the library holds it until the process exits).  The call rejects, with
 * MER_EINVAL, sizes whose fixed workspace part does not fit in it: 256 B of header, 16 B per bin tile
 * (n * ceil(H/tile) * ceil(W/tile) tiles), 64 B per (view, triangle); the rest holds the bin lists.
 * When the bin lists do not fit, the results are not valid and *status (device int, or NULL) receives
 * bit 0 (bit 1: a triangle index >= V).  *status is written on `stream` after the raster; read it once
 * the stream has passed that point.
 *
 * The call allocates nothing.  Its first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call before any stream capture.
 * All calls on a device share the one array and it keeps the last call's contents (each call clears the
 * part that must start at zero): calls that overlap on the GPU -- on different streams, or from
 * different host threads -- race and must be serialised by the caller. */
int mer_rasterize_noalloc(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W, int tile,
                          int32_t* index, float* depth, float* bary, int32_t* status, void* stream);

/* Interpolation module + deferred shading (Supp. B): shaded image [n,H,W,C]
 * per `shading`; background pixels take bg[c] (host array of C floats, copied
 * into the kernel arguments).  attr [V, C_attr]; tex [tex_h, tex_w, tex_c] or
 * NULL when uv_offset < 0. */
int mer_shade(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W,
              const int32_t* index, const float* attr, const float* tex, const float* bg_host,
              const mer_shading* shading_host, float* image, void* status_ws, void* stream);

/* Bytes of workspace a backward pass needs: 256 (the status header) without MER_DETERMINISTIC; with it, plus
 * 16 bytes per vertex-gradient component (vertex_rows * 3: n * V for mer_backward, totals.vrecs for
 * mer_batch_backward) and per attribute-gradient component (attr_rows * attr_channels: V or
 * totals.mesh_rows rows; attr_channels = the channels of grad_attr the pass writes, 0 without grad_attr),
 * rounded up to 256 bytes. */
size_t mer_backward_workspace_size(int64_t vertex_rows, int64_t attr_rows, int attr_channels, int terms);

/* Backward pass.  image / grad_image [n,H,W,C] are the shaded image passed
 * through the edge-gradient step and dL/d(image).  terms = MER_EDGE |
 * MER_INTERIOR | MER_INTERSECT (any subset), optionally | MER_EXACT_CROSSING | MER_DETERMINISTIC.
 *   MER_EDGE: every pair (x,y)-(x+1,y), (x,y)-(x,y+1) with differing ids:
 *     Eq. 11 summed over channels; classification by the exact coverage test of
 *     each pixel centre against the other pixel's triangle (Sec. 4.3): none ->
 *     adjacent (no scatter), one -> overhang (the triangle on top, whose own
 *     pixel centre lies inside the other triangle, gets dp/dr = 1 on the pair
 *     axis), both -> intersection (Eq. 12 in the (axis, zeta) slice for each
 *     side with the other fixed).  Fragment gradients are gathered to vertices
 *     with the screen barycentrics of the fragment's pixel centre.
 *   MER_INTERIOR: derivative of each covered pixel's shaded value with the
 *     index image fixed (Eq. 5 second term).
 * grad_vpix [n,V,3] float64 (+=): dL/d(x_s, y_s, zeta) per view.  The per-pixel
 * arithmetic is FP32; the sums over pixels are accumulated in FP64 because a
 * vertex gradient component can be a strongly cancelling sum of many terms.
 * grad_attr [V,C_attr] (+=) or NULL: dL/d(attr) of the interior term (interpolation mode: at most 4
 * interpolated channels; texture mode: the u, v columns).
 * cover [n,H,W] uint8 or NULL: the cover image the rasterizer wrote with this index image.  With it,
 * pairs whose neighbour triangle cannot cover the pixel centre (see MER_COVER_*) are not classified;
 * the results are the same as without it.  A cover image that does not belong to `index` can drop
 * scattering pairs (no memory fault).
 * workspace: NULL (no device status is recorded; not allowed with MER_DETERMINISTIC), or 256-byte aligned
 * device memory of workspace_bytes >= mer_backward_workspace_size(n * V, V, attribute channels, terms)
 * bytes whose first 256 bytes are a status header (a mer_rasterize workspace qualifies: the backward
 * overwrites only what lies after the header, which the raster no longer needs). */
int mer_backward(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W,
                 const int32_t* index, const uint8_t* cover, const float* image, const float* grad_image,
                 const float* attr, const float* tex, const mer_shading* shading_host, int terms,
                 double* grad_vpix, float* grad_attr, void* workspace, size_t workspace_bytes, void* stream);

/* EdgeGrad module backward alone (Supp. B): mer_backward with terms =
 * MER_EDGE | (intersections ? MER_INTERSECT : 0) for an image of C channels. */
int mer_edge_grad_backward(const float* image, const float* grad_image, int C, const int32_t* index,
                           const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W,
                           int intersections, double* grad_vpix, void* status_ws, void* stream);

/* Interpolation module backward alone (Supp. B): interior term of plain
 * attribute interpolation, grad_out [n,H,W,C_attr] -> grad_attr [V,C_attr] (+=,
 * or NULL) and grad_vpix [n,V,3] float64 (+=). */
int mer_interpolate_backward(const float* attr, int C_attr, const int32_t* tris, int T, const mer_vertex* vpix,
                             int V, const int32_t* index, int n, int H, int W, const float* grad_out,
                             float* grad_attr, double* grad_vpix, void* status_ws, void* stream);

/* Vertex transform backward (Supp. B): grad_verts [V,3] (+=) = sum over views
 * of R^T J^T grad_vpix with J = d(x_s, y_s, zeta)/d(X_c, Y_c, Z_c), in FP64, the views summed in order
 * (deterministic), rounded once to FP32. */
int mer_project_backward(int V, const mer_camera* cams, int n, const mer_vertex* vpix, const double* grad_vpix,
                         float* grad_verts, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Batched path: many items (a mesh seen by one camera) of uneven triangle counts and image sizes in
 * one launch per stage.  The raster and the backward run as persistent kernels whose CTAs (a whole
 * number of waves of the SM count) take bin / backward tiles of all items from a device work queue,
 * so large and small items balance; a caller can capture the whole step in one CUDA graph.
 *
 * Items index concatenated buffers.  The caller fills V, T, H, W, cam, vert and tri (several items may
 * share a mesh: same vert / tri, e.g. the views of one object); mer_batch_plan fills the other offsets
 * (every item gets its own vertex records, raster records, pixels and tiles) and the totals.
 *   verts / attr / grad_verts / grad_attr rows: item.vert + local vertex id
 *   tris: rows item.tri .. item.tri + T - 1, holding item-local vertex ids 0..V-1
 *   vpix / grad_vpix rows: item.vrec + local vertex id
 *   index / depth / image / grad_image / bary pixels: item.pix + y * W + x
 * ------------------------------------------------------------------------------------------------ */
typedef struct mer_item {
    int V, T, H, W;   /* vertices, triangles, image height and width */
    int cam;          /* camera of the item (index into the camera array) */
    int pad;
    int64_t vert;     /* first world vertex / attribute row (set by the caller) */
    int64_t tri;      /* first triangle row (set by the caller) */
    int64_t vrec;     /* first vertex record (mer_batch_plan) */
    int64_t trec;     /* first raster record (mer_batch_plan) */
    int64_t pix;      /* first pixel (mer_batch_plan) */
    int64_t tile;     /* first bin tile (mer_batch_plan) */
    int64_t btile;    /* first backward tile (mer_batch_plan) */
} mer_item;

typedef struct mer_batch_totals {
    int64_t vrecs, trecs, pixels, tiles, btiles;
    int n_items, tile;
    int64_t mesh_rows;      /* 1 + the largest world-vertex row any item uses (rows of verts / attr) */
    double max_tri_density; /* largest T / (H W) over the items with pixels */
} mer_batch_totals;

/* Host-only: fills the offsets of items[0..n) (host array) for bin tile `tile` (16, 32 or 64) and the
 * totals.  Returns MER_EINVAL on bad sizes (H, W > 8192, totals beyond 2^31 pixels or records). */
int mer_batch_plan(mer_item* items, int n_items, int tile, mer_batch_totals* totals);

/* Workspace bytes of mer_batch_rasterize (bin_capacity 0: 4 * trecs + 2 * tiles + 1024). */
size_t mer_batch_workspace_size(const mer_batch_totals* totals, int64_t bin_capacity);

/* Batched counterparts of the calls above; `items` is the planned table in device memory, `totals`
 * a host pointer.  persistent_ctas: CTAs (of 256 threads) of the persistent raster, which keeps 4 per SM
 * resident; the persistent backward, which keeps 6 per SM, launches persistent_ctas * 6 / 4 of its own
 * (0 = as many as fit on the device at once, for either). */
int mer_batch_project(const float* verts, const mer_camera* cams, const mer_item* items,
                      const mer_batch_totals* totals, mer_vertex* vpix, void* stream);
int mer_batch_rasterize(const mer_vertex* vpix, const int32_t* tris, const mer_item* items,
                        const mer_batch_totals* totals, void* workspace, size_t workspace_bytes,
                        int32_t* index, float* depth, float* bary, uint8_t* cover, int persistent_ctas,
                        void* stream);
int mer_batch_shade(const mer_vertex* vpix, const int32_t* tris, const mer_item* items,
                    const mer_batch_totals* totals, const int32_t* index, const float* attr, const float* tex,
                    const float* bg_host, const mer_shading* shading_host, float* image, void* status_ws,
                    void* stream);
/* mer_batch_rasterize followed by mer_batch_shade, in one persistent pass: each bin tile is shaded from
 * its z-buffer winners as soon as it is resolved, so the index image is written but not read back.
 * Results (index, depth, bary, image) are identical to the two calls; arguments are the union of
 * theirs, with the device status going to `workspace`.  Supp. B: rasterization, barycentrics and
 * interpolation modules. */
int mer_batch_render(const mer_vertex* vpix, const int32_t* tris, const mer_item* items,
                     const mer_batch_totals* totals, void* workspace, size_t workspace_bytes,
                     int32_t* index, float* depth, float* bary, uint8_t* cover, const float* attr,
                     const float* tex, const float* bg_host, const mer_shading* shading_host, float* image,
                     int persistent_ctas, void* stream);
/* cover: [pixels] uint8 or NULL, as for mer_backward (written by mer_batch_rasterize / mer_batch_render
 * with the same index image).  workspace: required (its header holds the backward's work queue), at least
 * mer_backward_workspace_size(totals.vrecs, totals.mesh_rows, attribute channels, terms) bytes; the
 * mer_batch_rasterize workspace of the same step qualifies when it is that large (the backward overwrites
 * only what lies after its header). */
int mer_batch_backward(const mer_vertex* vpix, const int32_t* tris, const mer_item* items,
                       const mer_batch_totals* totals, const int32_t* index, const uint8_t* cover,
                       const float* image,
                       const float* grad_image, const float* attr, const float* tex,
                       const mer_shading* shading_host, int terms, double* grad_vpix, float* grad_attr,
                       void* workspace, size_t workspace_bytes, int persistent_ctas, void* stream);
/* grad_verts [rows of all items' meshes, 3] (+=): items sharing a mesh add into the same rows.
 * workspace NULL: FP32 products added with FP32 atomics (the order of the additions across items that share
 * a mesh varies from run to run).  workspace non-NULL (256-byte aligned, at least
 * mer_backward_workspace_size(totals.mesh_rows, 0, 0, MER_DETERMINISTIC) bytes, header first): FP64 products,
 * each rounded once to 64-bit fixed point with 32 fractional bits and summed exactly, so the result is bitwise
 * reproducible (the counterpart of MER_DETERMINISTIC; MER_EFIXED for a term of magnitude >= 2^33). */
int mer_batch_project_backward(const mer_camera* cams, const mer_item* items, const mer_batch_totals* totals,
                               const mer_vertex* vpix, const double* grad_vpix, float* grad_verts,
                               void* workspace, size_t workspace_bytes, void* stream);

/* Forward gradients (Sec. 5): out [n,H,W,C] = the derivative of the shaded image along one scene
 * parameter whose effect on the projected vertices is tangent [n,V,3] = d(x_s, y_s, zeta)/d theta (FP32).
 * The exact transpose of mer_backward with the same terms: interior through the barycentrics,
 * interpolation / texture and depth; edge: every pair classified as in mer_backward moves its micro-edge
 * by dp/dtheta (the pair-axis motion of the foreground fragment, or Eq. 12 summed over both fragments
 * of an intersection) and, by Eq. 11, both of its pixels change by 1/2 (I_A - I_B) dp/dtheta.  out is
 * overwritten.  Errors as mer_backward. */
int mer_forward_grad(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W,
                     const int32_t* index, const float* image, const float* tangent, const float* attr,
                     const float* tex, const mer_shading* shading_host, int terms, float* out, void* status_ws,
                     void* stream);
/* tangent_vpix [n,V,3] = J(X_c) R tangent_world [V,3] for every view (the tangent map of mer_project;
 * vertices behind the near plane get 0). */
int mer_project_jvp(const float* tangent_world, int V, const mer_camera* cams, int n, const mer_vertex* vpix,
                    float* tangent_vpix, void* stream);

/* Area-weighted vertex normals, for optimisation loops that shade with normals recomputed from the
 * current positions (normal supervision, Supp. B): acc [V,3] = sum over the triangles at each vertex of
 * (p1 - p0) x (p2 - p0), normals [V,3] = acc / max(|acc|, 1e-20).  verts [V,3], tris [T,3] (ids in
 * [0, V), else MER_ERANGE in status_ws), device FP32; acc is caller-owned scratch kept for the backward. */
int mer_vertex_normals(const float* verts, int V, const int32_t* tris, int64_t T, float* acc, float* normals,
                       void* status_ws, void* stream);
/* Backward of mer_vertex_normals: grad_verts [V,3] += dL/d(verts) given dL/d(normals) in grad_normals
 * [V,3], which is overwritten (it receives dL/d(acc)).  acc as left by the forward. */
int mer_vertex_normals_backward(const float* verts, int V, const int32_t* tris, int64_t T, const float* acc,
                                float* grad_normals, float* grad_verts, void* status_ws, void* stream);

/* L2 image loss of an inverse-rendering loop and its gradient in one pass over n floats (device):
 * grad = 2 (image - target) and *loss += sum (image - target)^2 (FP64, device scalar the caller zeroes). */
int mer_l2_loss_grad(const float* image, const float* target, int64_t n, float* grad, double* loss, void* stream);

/* ---- Laplacian preconditioning of vertex updates (Nicolet et al. 2021, used by the paper for every mesh
 * optimisation: Sec. 5, Supp. B, lambda = 16) ----
 * Positions x [V,3] are reparameterised as u = M x, M = I + lambda L, with L the combinatorial Laplacian of
 * the edge graph of all meshes (L_ii = number of distinct neighbours of vertex i, L_ij = -1 for every edge;
 * meshes are independent blocks).  An optimiser steps u with the gradient M^-1 dL/dx and maps back with
 * x = M^-1 u. */

/* Host call (host pointers): the edge graph of triangles [T,3] over V vertices in CSR form.  row_ptr
 * [V+1] is always written (row_ptr[V] = number of directed edges); col [row_ptr[V]] (neighbours of each
 * vertex, ascending) only when not NULL, so a first call with col = NULL sizes it.  Degenerate triangle
 * edges (a == b) are skipped.  MER_ERANGE if a vertex id is outside [0, V). */
int mer_laplacian_csr(const int32_t* tris, int64_t T, int64_t V, int64_t* row_ptr, int32_t* col);
/* y = (I + lambda L) x, x and y [V,3] float32 on the device (distinct buffers). */
int mer_precond_apply(const int64_t* row_ptr, const int32_t* col, int64_t V, float lambda, const float* x,
                      float* y, void* stream);
size_t mer_precond_solve_workspace_size(int64_t V);
/* Solve (I + lambda L) x = b by conjugate gradients on the device (FP32 vectors, FP64 dot products), the
 * three columns as one block-diagonal system.  x holds the initial guess (a warm start) and receives the
 * solution.  Runs at most max_iters iterations as a fixed launch sequence; the iterations after the
 * residual norm falls to rel_tol * |b| return immediately.  workspace: 256-byte aligned device memory of
 * mer_precond_solve_workspace_size(V) bytes, owned by the caller. */
int mer_precond_solve(const int64_t* row_ptr, const int32_t* col, int64_t V, float lambda, const float* b,
                      float* x, int max_iters, float rel_tol, void* workspace, size_t workspace_bytes,
                      void* stream);
/* Synchronises `stream` and reports the last solve in `workspace`: iterations run and |r| / |b|. */
int mer_precond_solve_info(const void* workspace, int* iters, double* rel_residual, void* stream);

/* Synchronises `stream`, reads and clears the device status word of a
 * workspace (or of a status buffer of at least 256 bytes passed as status_ws to
 * the other calls).  Returns MER_OK, MER_EOVERFLOW, MER_ERANGE or MER_EFIXED; *total_bins
 * (if not NULL) receives the number of bin entries the last mer_rasterize
 * needed, so an overflowing caller can size the workspace exactly. */
int mer_sync_status(void* workspace, int64_t* total_bins, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MER_H */
