// backward.cu -- EdgeGrad module backward (Sec. 4.2-4.4, Supp. A.2-A.3) fused with
// the interior term Omega (Eq. 5) and the interpolation / barycentrics backward.
//
// One CTA per 32x16 pixel tile of one view (a warp = two rows of 32 pixels); the
// tile's index image plus a one-pixel halo sits in shared memory.  Each covered
// pixel p owns the fragment of its triangle t at its centre and accumulates that
// fragment's gradient dL/dr (a 3-vector in x_s, y_s, zeta):
//   * interior: -grad_P(L) in x, y from the barycentric derivatives, plus the
//     direct zeta derivative of the perspective weights and depth;
//   * edge: for each of its 4 neighbours q with a different id, Eq. 11 for the
//     pair (oriented left->right / top->bottom), then the Sec. 4.3 rule (p on
//     top -> dp/dr = 1 on the pair axis) or Eq. 12 (intersection) for p's side.
// The fragment gradient is gathered to the 3 vertices with p's screen
// barycentrics (dL/dv_i = lambda_i dL/dr).  A warp first classifies the edge
// pairs of both its rows together (they rarely fill more than one 32-lane pass;
// with the rasterizer's cover image, only the pairs it does not rule out), then
// takes its rows one at a time: the 9 per-pixel vertex terms are summed over each
// run of equal triangle id in the row (segmented shuffle scan, FP32), then per
// triangle in a shared-memory table (FP32), and the flush adds each triangle's
// totals to its 3 vertices in grad_vpix with one FP64 atomic per component.
#include <cuda_runtime.h>

#include <cstdint>

#include "mer_device.cuh"

namespace mer {

constexpr int kTW = kBwdTileW, kTH = kBwdTileH;  // tile: 8 warps, two rows each
constexpr int kRows = 2;                          // rows per warp
constexpr int kHW = kTW + 2, kHH = kTH + 2;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 6;                     // resident CTAs per SM: at most 42 registers a thread
static_assert(kTW == 32 && kTH == kRows * kThreads / 32, "a warp spans the tile's width");
// Per-tile triangle table of 2^BITS slots: a 32x16 tile of the head-scale workloads holds ~20-80 triangles.
// 128 slots keep six CTAs resident with most of the SM's on-chip memory left to the L1 cache that serves the
// vertex, texel and image gathers (256 slots measured 2.7 % slower on the multi-view head workload); a tile
// with more triangles sends the excess straight to global memory, so launches in which some item is dense on
// screen (more than 0.1 triangle per pixel) take 256 slots.  Only the variant without attribute gradients and
// without the exact-crossing option has the 256-slot instantiation: launches with either always use 128.
constexpr int kTableBits = 7, kTableBitsDense = 8;
constexpr double kDenseTrianglesPerPixel = 0.1;
// A triangle insert probes at most this many slots before it goes to global memory, so a tile with more
// triangles than slots does not pay a scan of the whole table for every excess triangle.
constexpr int kMaxProbes = 16;
template <int NA, bool EXACT, int BITS>
struct TriTable {
    static constexpr int kBits = BITS;
    static constexpr int kSlots = 1 << kBits;
};

struct BwdArgs {
    // base pointers of the launch's arrays (an item addresses them through its offsets)
    const mer_vertex* vpix;
    const int* tris;
    const int* index;
    const unsigned char* cover;  // or null
    const float* image;
    const float* grad;
    const float* attr;
    double* grad_vpix;
    float* grad_attr;            // or null
    mer_shading sh;
    int terms;
    int n, H, W, V, T;
    int ntx, nty;
    int tex_stride;  // floats per texel
    bool tex_vec4;   // stride 4 and 16-byte aligned: 128-bit texel loads
};

// Vertex ids of triangle t; false if one is out of range.
__device__ __forceinline__ bool tri_ids(const int* __restrict__ tris, int t, int V, int id[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        id[k] = __ldg(tris + 3 * (size_t)t + k);
        if ((unsigned)id[k] >= (unsigned)V) return false;
    }
    return true;
}

// Plane normal (v1 - v0) x (v2 - v0) in (x_s, y_s, zeta) from accurate differences.
__device__ __forceinline__ void tri_normal(const VRec r[3], float N[3]) {
    float e[2][3];
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        e[k - 1][0] = i2f_exact(r[k].X - r[0].X) * (1.0f / 256.0f) + (r[k].rx - r[0].rx);
        e[k - 1][1] = i2f_exact(r[k].Y - r[0].Y) * (1.0f / 256.0f) + (r[k].ry - r[0].ry);
        e[k - 1][2] = (r[k].zeta - r[0].zeta) + (r[k].zeta_lo - r[0].zeta_lo);
    }
    N[0] = diff_of_products(e[0][1], e[1][2], e[0][2], e[1][1]);
    N[1] = diff_of_products(e[0][2], e[1][0], e[0][0], e[1][2]);
    N[2] = diff_of_products(e[0][0], e[1][1], e[0][1], e[1][0]);
}

// Slot of triangle `key` in the tile table of 2^BITS slots, inserting it if needed; -1 if no slot was free
// within kMaxProbes probes.
template <int BITS>
__device__ __forceinline__ int table_slot(int* keys, int key) {
    constexpr int kSlots = 1 << BITS;
    unsigned h = ((unsigned)key * 2654435761u) >> (32 - BITS);
#pragma unroll 1
    for (int probe = 0; probe < kMaxProbes && probe < kSlots; ++probe) {
        // a slot's key only ever changes from -1 to a triangle id within a tile: a key already seen is final
        int k = *reinterpret_cast<volatile int*>(keys + h);
        if (k == key) return (int)h;
        if (k == -1) {
            k = atomicCAS(keys + h, -1, key);
            if (k == -1 || k == key) return (int)h;
        }
        h = (h + 1) & (kSlots - 1);
    }
    return -1;
}

// One item of a backward pass: a mesh seen by one camera, as offsets into the launch's arrays (kept instead of
// nine pointers: fewer registers live across the pixel pass; the bases are kernel parameters).
struct BItem {
    long long vrec;  // first vertex record (and grad_vpix row)
    long long tri;   // first triangle
    long long pix;   // first pixel of the index, cover, image and gradient images
    long long vert;  // first attribute (and grad_attr) row
    int V, T, H, W;
    __device__ __forceinline__ const mer_vertex* vb(const BwdArgs& a) const { return a.vpix + vrec; }
    __device__ __forceinline__ const int* tris(const BwdArgs& a) const { return a.tris + 3 * tri; }
    __device__ __forceinline__ const int* index(const BwdArgs& a) const { return a.index + pix; }
    __device__ __forceinline__ const unsigned char* cover(const BwdArgs& a) const { return a.cover + pix; }
    __device__ __forceinline__ const float* image(const BwdArgs& a) const { return a.image + pix * a.sh.C; }
    __device__ __forceinline__ const float* grad(const BwdArgs& a) const { return a.grad + pix * a.sh.C; }
    __device__ __forceinline__ const float* attr(const BwdArgs& a) const { return a.attr + vert * a.sh.C_attr; }
    __device__ __forceinline__ double* gv(const BwdArgs& a) const { return a.grad_vpix + 3 * vrec; }
    __device__ __forceinline__ float* gattr(const BwdArgs& a) const { return a.grad_attr + vert * a.sh.C_attr; }
};

constexpr int kMaxA = 4;  // most attribute-gradient channels carried through the per-tile aggregation

template <int NA, bool EXACT, int BITS>
struct BwdShared {
    int sidx[kHH][kHW];
    unsigned char scov[kHH][kHW];  // cover image of the tile and halo (when given)
    static constexpr int kSlots = TriTable<NA, EXACT, BITS>::kSlots;
    int skey[kSlots];                 // triangle id, -1 = free
    int svid[kSlots][3];              // its vertex ids
    float sval[kSlots][3][3];         // per vertex of the triangle: dL/d(x_s, y_s, zeta)
    float sattr[NA > 0 ? kSlots : 1][3][NA > 0 ? NA : 1];
    float efrag[kTH][32][3];  // per row: edge-term fragment gradients returned to the pixel's lane
    unsigned char slist[kThreads / 32][4 * kRows * 32];  // per warp: its edge pairs kept by the first test
    float evert[EXACT ? kTH : 1][32][3][2];  // exact-crossing option: per pixel, (x, y) per triangle vertex
};

// Edge term of the warp's rows r0 .. r0 + kRows - 1, before their per-pixel pass (all 32 lanes call it
// together).  The (pixel, neighbour) pairs whose ids differ, with the pixel covered, are compacted into one
// list for the warp's rows (most rows hold far fewer than 32 such pairs, so the rows share passes) and
// classified 32 at a time; a pair whose source fragment scatters adds into that pixel's slot of the per-row
// shared buffer efrag (evert for the exact-crossing option), read back by the pixel's lane in its row pass.
// Returns false when the rows hold no pair (the buffers are then not written).
template <int NA, bool EXACT, int BITS>
__device__ __forceinline__ bool edge_rows(const BItem& it, const BwdArgs& a, BwdShared<NA, EXACT, BITS>& S, void* ws,
                                          int r0, int lane, int x0, int y0) {
    const unsigned full = 0xffffffffu;
    const int C = a.sh.C;
    constexpr int kM = 4 * kRows;
    unsigned m[kM];  // per (row k, direction d): lanes whose pixel is covered and whose neighbour in d differs
    int np[kM + 1];  // prefix counts
    np[0] = 0;
    const bool hinted = a.cover != nullptr;
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int row = r0 + k;
        const int t = S.sidx[row + 1][lane + 1];  // -2 outside the image
        const unsigned hp = hinted ? S.scov[row + 1][lane + 1] : 0u;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int ddx = d == 0 ? -1 : (d == 1 ? 1 : 0);
            const int ddy = d == 2 ? -1 : (d == 3 ? 1 : 0);
            const int tq = S.sidx[row + 1 + ddy][lane + 1 + ddx];
            bool pair = t >= 0 && tq != t && tq != -2;
            if (hinted && tq >= 0) {
                // p's fragment can scatter only if q's triangle covers p's centre too (Sec. 4.3), which needs
                // another triangle of q's facing at p (a second one when p's own triangle has that facing).
                // The counts of front-facing triangles are exact everywhere; those of back-facing ones only for
                // triangles that win a pixel of p's bin tile, so a pair across the border of p's bin tile whose
                // neighbour triangle is back-facing is always classified.
                const unsigned hq = S.scov[row + 1 + ddy][lane + 1 + ddx];
                const bool same = ((hp ^ hq) & MER_COVER_WINNER_BACK) == 0;
                const unsigned need = same ? MER_COVER_SAME_2 : MER_COVER_OTHER_1;
                const unsigned border = d == 0 ? MER_COVER_BORDER_L
                                                : (d == 1 ? MER_COVER_BORDER_R
                                                          : (d == 2 ? MER_COVER_BORDER_T : MER_COVER_BORDER_B));
                pair = pair && ((hp & need) != 0 || ((hp & border) != 0 && (hq & MER_COVER_WINNER_BACK) != 0));
            }
            m[4 * k + d] = __ballot_sync(full, pair);
            np[4 * k + d + 1] = np[4 * k + d] + __popc(m[4 * k + d]);
        }
    }
    const int n = np[kM];
    if (n == 0) return false;
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        float* acc = &S.efrag[r0 + k][lane][0];
        acc[0] = 0.f;
        acc[1] = 0.f;
        acc[2] = 0.f;
        if (EXACT) {
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                S.evert[r0 + k][lane][v][0] = 0.f;
                S.evert[r0 + k][lane][v][1] = 0.f;
            }
        }
    }
    __syncwarp();
    const mer_vertex* vb = it.vb(a);
    // Pass 1 over the list, 32 entries at a time: the test of p's centre against q's triangle (most pairs end
    // there) or, against the background, nothing; the surviving entries (row-direction mask s, source lane)
    // are compacted into the warp's byte list, so that pass 2 runs the rest with its lanes full.
    unsigned char* keep_list = S.slist[threadIdx.x >> 5];
    int nk = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        bool keep = false;
        int code = 0;
        if (i < n) {
            // list entry i -> mask s (the last one whose prefix count is <= i), its row, direction and source
            int s = 0;
#pragma unroll
            for (int j = 1; j < kM; ++j)
                if (i >= np[j]) s = j;
            unsigned md = m[0];
            int start = 0;
#pragma unroll
            for (int j = 1; j < kM; ++j)
                if (s == j) {
                    md = m[j];
                    start = np[j];
                }
            const int row = r0 + (s >> 2), d = s & 3;
            const int src = (int)__fns(md, 0, i - start + 1);
            const int ddx = d == 0 ? -1 : (d == 1 ? 1 : 0);
            const int ddy = d == 2 ? -1 : (d == 3 ? 1 : 0);
            const int tq = S.sidx[row + 1 + ddy][src + 1 + ddx];
            code = (s << 5) | src;
            keep = true;  // a pair against the background needs only Eq. 11 (the row pass checks p's triangle)
            if (tq >= 0) {
                int vq[3];
                if (tq >= it.T || !tri_ids(it.tris(a), tq, it.V, vq)) {
                    set_status(ws, kStatusRange);
                    keep = false;
                } else {
                    int Xq[3], Yq[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {  // snapped position only: one 64-bit load per vertex
                        const int2 xy = __ldg(reinterpret_cast<const int2*>(vb + vq[k]));
                        Xq[k] = xy.x;
                        Yq[k] = xy.y;
                    }
                    // classification (Sec. 4.3): p's fragment scatters only if p's centre lies inside q's
                    // triangle (p on top of it), or both centres lie in each other's triangles (intersection)
                    keep = covers_xy(Xq, Yq, 256 * (x0 + src) + 128, 256 * (y0 + row) + 128);
                }
            }
        }
        const unsigned kb = __ballot_sync(full, keep);
        if (keep) keep_list[nk + __popc(kb & ((1u << lane) - 1u))] = (unsigned char)code;
        nk += __popc(kb);
    }
    __syncwarp();
    // Pass 2 over the kept entries: the intersection test, Eq. 11 and the fragment gradient.
    for (int i = lane; i < nk; i += 32) {
        const int code = keep_list[i];
        const int s = code >> 5, src = code & 31;
        const int row = r0 + (s >> 2), d = s & 3;
        const int ddx = d == 0 ? -1 : (d == 1 ? 1 : 0);
        const int ddy = d == 2 ? -1 : (d == 3 ? 1 : 0);
        const int px = x0 + src, y = y0 + row;
        const int ts = S.sidx[row + 1][src + 1];
        const int tq = S.sidx[row + 1 + ddy][src + 1 + ddx];
        // p's triangle: its vertex ids and snapped positions (the exact-crossing option, or a neighbour
        // triangle that covers p's centre)
        int vs[3] = {0, 0, 0};
        int Xs[3] = {0, 0, 0}, Ys[3] = {0, 0, 0};
        if (EXACT || tq >= 0) {
            if (ts >= it.T || !tri_ids(it.tris(a), ts, it.V, vs)) {
                set_status(ws, kStatusRange);
                continue;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int2 xy = __ldg(reinterpret_cast<const int2*>(vb + vs[k]));
                Xs[k] = xy.x;
                Ys[k] = xy.y;
            }
        }
        const int qx = px + ddx, qy = y + ddy;
        const int axis = ddx != 0 ? 0 : 1;
        bool inter = false;
        if (tq >= 0 && covers_xy(Xs, Ys, 256 * qx + 128, 256 * qy + 128)) {
            if (!(a.terms & MER_INTERSECT)) continue;
            inter = true;
        }
        // Eq. 11 with A = left/top pixel, B = right/bottom pixel
        const size_t p = (size_t)y * it.W + px;
        const size_t q = (size_t)qy * it.W + qx;
        const float *gp = it.grad(a) + p * C, *gq = it.grad(a) + q * C, *ip = it.image(a) + p * C, *iq = it.image(a) + q * C;
        const bool p_is_a = ddx > 0 || ddy > 0;
        float dLdp = 0.f;
        for (int c = 0; c < C; ++c) {
            const float diff = __ldg(ip + c) - __ldg(iq + c);
            dLdp += 0.5f * (__ldg(gp + c) + __ldg(gq + c)) * (p_is_a ? diff : -diff);
        }
        float ex = 0.f, ey = 0.f, ez = 0.f;
        if (!inter) {
            if (EXACT) {
                // exact-crossing option: the crossing moves with the endpoints of p's exit edge
                const int e = exit_edge(Xs, Ys, 256 * px + 128, 256 * y + 128, 256 * qx + 128, 256 * qy + 128);
                if (e >= 0) {
                    const int j = (e + 1) % 3, l = (e + 2) % 3;
                    const float4 rj = __ldg(reinterpret_cast<const float4*>(vb + vs[j]));
                    const float4 rl = __ldg(reinterpret_cast<const float4*>(vb + vs[l]));
                    const float u = axis == 0 ? crossing_u(Ys[j], rj.w, Ys[l], rl.w, 256 * y + 128)
                                              : crossing_u(Xs[j], rj.z, Xs[l], rl.z, 256 * px + 128);
                    atomicAdd(&S.evert[row][src][j][axis], (1.0f - u) * dLdp);
                    atomicAdd(&S.evert[row][src][l][axis], u * dLdp);
                    continue;
                }
            }
            if (axis == 0) ex = dLdp; else ey = dLdp;
        } else {
            // Eq. 12: p's triangle varies (v), q's triangle is fixed (f), slice (axis, zeta); q's ids were
            // checked in pass 1
            int vq[3];
            tri_ids(it.tris(a), tq, it.V, vq);
            const VRec rv[3] = {load_vrec(vb + vs[0]), load_vrec(vb + vs[1]), load_vrec(vb + vs[2])};
            const VRec rq[3] = {load_vrec(vb + vq[0]), load_vrec(vb + vq[1]), load_vrec(vb + vq[2])};
            float Nv[3], Nf[3];
            tri_normal(rv, Nv);
            tri_normal(rq, Nf);
            const float nv0 = axis == 0 ? Nv[0] : Nv[1], nv1 = Nv[2];
            const float nf0 = axis == 0 ? Nf[0] : Nf[1], nf1 = Nf[2];
            const float den = diff_of_products(nf0, nv1, nf1, nv0);
            const float mag = sqrtf((nv0 * nv0 + nv1 * nv1) * (nf0 * nf0 + nf1 * nf1));
            if (!(fabsf(den) > 1e-12f * mag)) continue;
            const float kk = dLdp * (-nf1 / den);
            if (axis == 0) ex = kk * nv0; else ey = kk * nv0;
            ez = kk * nv1;
        }
        float* acc = &S.efrag[row][src][0];
        if (ex != 0.f) atomicAdd(acc, ex);
        if (ey != 0.f) atomicAdd(acc + 1, ey);
        if (ez != 0.f) atomicAdd(acc + 2, ez);
    }
    __syncwarp();
    return true;
}

// A tile's work is split in three phases separated by CTA barriers: tile_halo (index tile + halo into shared
// memory), tile_compute (every pixel's gradients, aggregated into the triangle table) and tile_flush (table to
// global memory, slots cleared for the next tile).  The table starts clear (table_clear once per CTA), and a
// persistent CTA overlaps the flush of one tile with the halo load of the next.

template <int NA, bool EXACT, int BITS>
__device__ __forceinline__ void table_clear(BwdShared<NA, EXACT, BITS>& S) {
    for (int i = threadIdx.x; i < S.kSlots; i += kThreads) {
        S.skey[i] = -1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            S.sval[i][k][0] = 0.f;
            S.sval[i][k][1] = 0.f;
            S.sval[i][k][2] = 0.f;
            if (NA > 0) {
#pragma unroll
                for (int j = 0; j < (NA > 0 ? NA : 1); ++j) S.sattr[i][k][j] = 0.f;
            }
        }
    }
}

// Returns whether this thread loaded a covered pixel of the tile itself (not the halo).  Each thread issues
// all its loads (at most three entries and their cover bytes) before it stores any.
template <int NA, bool EXACT, int BITS>
__device__ __forceinline__ bool tile_halo(const BItem& it, const BwdArgs& a, int tx, int ty,
                                          BwdShared<NA, EXACT, BITS>& S) {
    constexpr int kN = (kHH * kHW + kThreads - 1) / kThreads;
    int v[kN];
    unsigned char c[kN];
    const int* ib = it.index(a);
    const unsigned char* cb = a.cover ? it.cover(a) : nullptr;
#pragma unroll
    for (int q = 0; q < kN; ++q) {
        const int i = threadIdx.x + q * kThreads;
        const int hy = i / kHW, hx = i % kHW;
        const int gx = tx * kTW + hx - 1, gy = ty * kTH + hy - 1;
        const bool in = i < kHH * kHW && gx >= 0 && gx < it.W && gy >= 0 && gy < it.H;
        const size_t o = in ? (size_t)gy * it.W + gx : 0;
        v[q] = in ? __ldg(ib + o) : -2;
        c[q] = (in && cb) ? __ldg(cb + o) : (unsigned char)0;
    }
    bool covered = false;
#pragma unroll
    for (int q = 0; q < kN; ++q) {
        const int i = threadIdx.x + q * kThreads;
        if (i >= kHH * kHW) break;
        const int hy = i / kHW, hx = i % kHW;
        S.sidx[hy][hx] = v[q];
        if (cb) S.scov[hy][hx] = c[q];
        covered |= v[q] >= 0 && hy >= 1 && hy <= kTH && hx >= 1 && hx <= kTW;
    }
    return covered;
}

// Per-pixel pass of row `row` of the tile (tx, ty) of an item, after its edge_rows (pairs: whether that wrote
// the row's edge buffers).
// NA > 0: also produce the attribute gradients (channels [a0, a0 + NA) of each vertex's attribute row, NA <= 4:
// the interpolated channels, or (u, v) in texture mode), aggregated like the vertex gradients.
template <int NA, bool EXACT, int BITS>
__device__ __forceinline__ void row_pass(const BItem& it, int tx, int ty, int row, int lane, bool pairs,
                                         const BwdArgs& a, const float* __restrict__ tex, BwdShared<NA, EXACT, BITS>& S,
                                         void* ws) {
    const int A = a.sh.uv_offset < 0 ? a.sh.n_main : 2;
    const int a0 = a.sh.uv_offset < 0 ? 0 : a.sh.uv_offset;
    const int x = tx * kTW + lane, y = ty * kTH + row;
    const int C = a.sh.C;
    const mer_vertex* vb = it.vb(a);
    const int* tris = it.tris(a);
    const float* grad = it.grad(a);
    const float* attr = it.attr(a);
    float* grad_attr = it.gattr(a);
    int t = (x < it.W && y < it.H) ? S.sidx[row + 1][lane + 1] : -1;
    if (!__any_sync(0xffffffffu, t >= 0)) return;  // background row: no fragment, no pair
    int vid[3] = {0, 0, 0};
    float c0[3] = {0.f, 0.f, 0.f}, c1[3] = {0.f, 0.f, 0.f}, c2[3] = {0.f, 0.f, 0.f};  // per vertex: x, y, zeta
    float ca[3][NA > 0 ? NA : 1];  // per vertex: attribute-gradient channels (NA > 0)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < (NA > 0 ? NA : 1); ++j) ca[k][j] = 0.f;
    if (t >= it.T) {
        set_status(ws, kStatusRange);
        t = -1;
    }
    if (t >= 0 && !tri_ids(tris, t, it.V, vid)) {
        set_status(ws, kStatusRange);
        t = -1;
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float hz[3] = {0.f, 0.f, 0.f}, lam[3] = {0.f, 0.f, 0.f};
    if (t >= 0) {
        const size_t p = (size_t)y * it.W + x;
        const float* gp = grad + p * C;
        const VRec rv[3] = {load_vrec(vb + vid[0]), load_vrec(vb + vid[1]), load_vrec(vb + vid[2])};
        const Bary B = screen_bary(rv, x, y);
#pragma unroll
        for (int k = 0; k < 3; ++k) lam[k] = B.lam[k];

        if (a.terms & MER_INTERIOR) {
            const float z[3] = {rv[0].zeta, rv[1].zeta, rv[2].zeta};
            const float s = B.lam[0] * z[0] + B.lam[1] * z[1] + B.lam[2] * z[2];
            const float is = rcp_nr(s);
            float b[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) b[k] = B.lam[k] * z[k] * is;
            // G_k = dL/db_k.  Only the differences G_k - G_i enter (sum_i b_i = 1), so they are formed from
            // attribute differences: D01 = G_0 - G_1, D02 = G_0 - G_2, D12 = G_1 - G_2.
            float D01 = 0.f, D02 = 0.f, D12 = 0.f;
            const int Ca = a.sh.C_attr;
            if (a.sh.uv_offset < 0) {
                for (int c = 0; c < a.sh.n_main; ++c) {
                    const float gc = __ldg(gp + c);
                    const float a0 = __ldg(attr + (size_t)vid[0] * Ca + c);
                    const float a1 = __ldg(attr + (size_t)vid[1] * Ca + c);
                    const float a2 = __ldg(attr + (size_t)vid[2] * Ca + c);
                    D01 += gc * (a0 - a1);
                    D02 += gc * (a0 - a2);
                    D12 += gc * (a1 - a2);
                    if (NA > 0) {
#pragma unroll
                        for (int j = 0; j < (NA > 0 ? NA : 1); ++j)
                            if (j == c) {
                                ca[0][j] = b[0] * gc;
                                ca[1][j] = b[1] * gc;
                                ca[2][j] = b[2] * gc;
                            }
                    }
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
                float gu, gv;
                tex_grad_uv(tex, a.sh.tex_h, a.sh.tex_w, a.tex_stride, a.tex_vec4, a.sh.n_main, taps, gp, gu, gv);
                D01 = gu * (uk[0] - uk[1]) + gv * (vk[0] - vk[1]);
                D02 = gu * (uk[0] - uk[2]) + gv * (vk[0] - vk[2]);
                D12 = gu * (uk[1] - uk[2]) + gv * (vk[1] - vk[2]);
                if (NA > 0) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        ca[k][0] = b[k] * gu;
                        ca[k][1] = b[k] * gv;
                    }
                }
            }
            // G_k - Gbar = sum_i b_i (G_k - G_i)
            const float GmG[3] = {b[1] * D01 + b[2] * D02, b[2] * D12 - b[0] * D01, -(b[0] * D02 + b[1] * D12)};
            const float gZ = a.sh.depth_ch >= 0 ? __ldg(gp + a.sh.depth_ch) : 0.f;
            // w = sum_k (dL/d lambda_k) grad lambda_k with dL/d lambda_k = zeta_k is (GmG_k - gZ is).  The depth
            // part -gZ is^2 sum_k zeta_k grad lambda_k equals -gZ is^2 sum_k (zeta_k - zeta_0) grad lambda_k
            // (the gradients sum to zero); the zeta differences come from the hi + lo split, so the near
            // cancellation of an almost constant zeta across the triangle costs no accuracy.
            const float dz1 = (z[1] - z[0]) + (rv[1].zeta_lo - rv[0].zeta_lo);
            const float dz2 = (z[2] - z[0]) + (rv[2].zeta_lo - rv[0].zeta_lo);
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

    }

    if (pairs && t >= 0) {  // the edge term of the pixel's fragment, from edge_rows
        fx += S.efrag[row][lane][0];
        fy += S.efrag[row][lane][1];
        fz += S.efrag[row][lane][2];
    }
    if (t >= 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float l = lam[k];
            c0[k] = l * fx;
            c1[k] = l * fy;
            c2[k] = l * (fz + hz[k]);
        }
        if (EXACT && pairs) {  // the exact-crossing parts, already split per vertex
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                c0[k] += S.evert[row][lane][k][0];
                c1[k] += S.evert[row][lane][k][1];
            }
        }
    }

    // --- sum each run of equal triangle id along the warp's row (inclusive segmented scan) ---
    const unsigned full = 0xffffffffu;
    const int tprev = __shfl_up_sync(full, t, 1);
    const bool head = lane == 0 || tprev != t;
    const unsigned heads = __ballot_sync(full, head);
    const int seg = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of this run
    const bool contributes = t >= 0 && (NA > 0 || c0[0] != 0.f || c1[0] != 0.f || c2[0] != 0.f || c0[1] != 0.f ||
                                        c1[1] != 0.f || c2[1] != 0.f || c0[2] != 0.f || c1[2] != 0.f ||
                                        c2[2] != 0.f);
    const unsigned any = __ballot_sync(full, contributes);
    // longest run in the warp decides how many doubling steps the scan needs
    const int runlen = t >= 0 ? lane - seg + 1 : 0;  // runs of background lanes carry nothing
    const int maxrun = (int)__reduce_max_sync(full, (unsigned)runlen);
#pragma unroll
    for (int dlt = 1; dlt < 32; dlt <<= 1) {
        if (!any || dlt >= maxrun) break;
        const bool take = lane - dlt >= seg;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float a0_ = __shfl_up_sync(full, c0[k], dlt);
            const float a1_ = __shfl_up_sync(full, c1[k], dlt);
            const float a2_ = __shfl_up_sync(full, c2[k], dlt);
            if (take) {
                c0[k] += a0_;
                c1[k] += a1_;
                c2[k] += a2_;
            }
            if (NA > 0) {
#pragma unroll
                for (int j = 0; j < (NA > 0 ? NA : 1); ++j) {
                    if (j >= A) break;
                    const float aj = __shfl_up_sync(full, ca[k][j], dlt);
                    if (take) ca[k][j] += aj;
                }
            }
        }
    }
    const int tnext = __shfl_down_sync(full, t, 1);
    const bool tail = lane == 31 || tnext != t;
    double* gvv = it.gv(a);
    if (tail && t >= 0 && any) {
        // one slot per triangle: the runs of one row hold different triangles, so their adds do not contend
        const int sl = table_slot<TriTable<NA, EXACT, BITS>::kBits>(S.skey, t);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (sl >= 0) {
                S.svid[sl][k] = vid[k];  // every writer of the slot writes the same ids
                atomicAdd(&S.sval[sl][k][0], c0[k]);
                atomicAdd(&S.sval[sl][k][1], c1[k]);
                atomicAdd(&S.sval[sl][k][2], c2[k]);
                if (NA > 0) {
#pragma unroll
                    for (int j = 0; j < (NA > 0 ? NA : 1); ++j)
                        if (j < A) atomicAdd(&S.sattr[sl][k][j], ca[k][j]);
                }
            } else {  // table full: straight to global memory
                atomicAdd(gvv + 3 * (size_t)vid[k], (double)c0[k]);
                atomicAdd(gvv + 3 * (size_t)vid[k] + 1, (double)c1[k]);
                atomicAdd(gvv + 3 * (size_t)vid[k] + 2, (double)c2[k]);
                if (NA > 0) {
#pragma unroll
                    for (int j = 0; j < (NA > 0 ? NA : 1); ++j)
                        if (j < A) atomicAdd(grad_attr + (size_t)vid[k] * a.sh.C_attr + a0 + j, ca[k][j]);
                }
            }
        }
    }
}

// The tile (tx, ty) of an item, after tile_halo and a barrier: each warp takes rows kRows * warp ..
// kRows * warp + kRows - 1, first their edge pairs together, then each row's pixels.
template <int NA, bool EXACT, int BITS>
__device__ __forceinline__ void tile_compute(const BItem& it, int tx, int ty, const BwdArgs& a,
                                             const float* __restrict__ tex, BwdShared<NA, EXACT, BITS>& S, void* ws) {
    const int lane = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * kRows;
    const bool pairs = (a.terms & MER_EDGE) && edge_rows<NA, EXACT, BITS>(it, a, S, ws, r0, lane, tx * kTW, ty * kTH);
#pragma unroll 1
    for (int k = 0; k < kRows; ++k) row_pass<NA, EXACT, BITS>(it, tx, ty, r0 + k, lane, pairs, a, tex, S, ws);
}

// After tile_compute and a barrier: add the table to global memory and clear it.
template <int NA, bool EXACT, int BITS>
__device__ __forceinline__ void tile_flush(const BItem& it, const BwdArgs& a, BwdShared<NA, EXACT, BITS>& S) {
    const int A = a.sh.uv_offset < 0 ? a.sh.n_main : 2;
    const int a0 = a.sh.uv_offset < 0 ? 0 : a.sh.uv_offset;
    double* gvv = it.gv(a);
    float* gattr = it.gattr(a);
    for (int i = threadIdx.x; i < S.kSlots; i += kThreads) {
        if (S.skey[i] < 0) continue;
        S.skey[i] = -1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int v = S.svid[i][k];
            const float s0 = S.sval[i][k][0], s1 = S.sval[i][k][1], s2 = S.sval[i][k][2];
            S.sval[i][k][0] = 0.f;
            S.sval[i][k][1] = 0.f;
            S.sval[i][k][2] = 0.f;
            if (s0 != 0.f) atomicAdd(gvv + 3 * (size_t)v, (double)s0);
            if (s1 != 0.f) atomicAdd(gvv + 3 * (size_t)v + 1, (double)s1);
            if (s2 != 0.f) atomicAdd(gvv + 3 * (size_t)v + 2, (double)s2);
            if (NA > 0) {
#pragma unroll
                for (int j = 0; j < (NA > 0 ? NA : 1); ++j) {
                    if (j >= A) break;
                    const float sa = S.sattr[i][k][j];
                    S.sattr[i][k][j] = 0.f;
                    if (sa != 0.f) atomicAdd(gattr + (size_t)v * a.sh.C_attr + a0 + j, sa);
                }
            }
        }
    }
}

template <int NA, bool EXACT, int BITS>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_backward(const mer_vertex* __restrict__ vpix, const int* __restrict__ tris,
                                                       const int* __restrict__ index,
                                                       const unsigned char* __restrict__ cover,
                                                       const float* __restrict__ image,
                                                       const float* __restrict__ grad, const float* __restrict__ attr,
                                                       const float* __restrict__ tex, BwdArgs a,
                                                       double* __restrict__ grad_vpix, float* __restrict__ grad_attr,
                                                       void* ws) {
    __shared__ BwdShared<NA, EXACT, BITS> S;
    const int tiles_per_view = a.ntx * a.nty;
    const int view = blockIdx.x / tiles_per_view;
    const int local = blockIdx.x % tiles_per_view;
    const size_t plane = (size_t)a.H * a.W;
    BItem it;
    it.vrec = (long long)view * a.V;
    it.tri = 0;
    it.pix = (long long)view * (long long)plane;
    it.vert = 0;
    it.V = a.V; it.T = a.T; it.H = a.H; it.W = a.W;
    table_clear(S);
    const bool covered = tile_halo(it, a, local % a.ntx, local / a.ntx, S);
    if (!__syncthreads_or(covered)) return;  // background tile
    tile_compute<NA, EXACT, BITS>(it, local % a.ntx, local / a.ntx, a, tex, S, ws);
    __syncthreads();
    tile_flush(it, a, S);
}

// Persistent: each CTA takes the next backward tile of any item from the work queue.
template <int NA, bool EXACT, int BITS>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_backward_batch(const mer_vertex* __restrict__ vpix,
                                                             const int* __restrict__ tris,
                                                             const mer_item* __restrict__ items, int n_items,
                                                             long long btiles, const int* __restrict__ index,
                                                             const unsigned char* __restrict__ cover,
                                                             const float* __restrict__ image,
                                                             const float* __restrict__ grad,
                                                             const float* __restrict__ attr,
                                                             const float* __restrict__ tex, BwdArgs a,
                                                             double* __restrict__ grad_vpix,
                                                             float* __restrict__ grad_attr, void* ws) {
    __shared__ BwdShared<NA, EXACT, BITS> S;
    __shared__ long long s_tile;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    table_clear(S);
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(&hdr->queue_backward, 1ull);
    __syncthreads();
    // Per tile two barriers: after the halo load (thread 0 then takes the next tile id) and before the flush
    // (the next id is visible after it).  The flush of a tile and the halo load of the next touch disjoint
    // shared memory, and the next tile's table inserts come only after its first barrier.  (A background row
    // leaves tile_compute at once; skipping whole background tiles here instead costs registers.)
    int cur = 0;                       // item of the previous tile and its tile range [lo, hi)
    long long lo = 0, hi = 0;
    while (true) {
        const long long g = s_tile;
        if (g >= btiles) break;
        // consecutive tiles of a CTA mostly belong to the same item: search the table only on a change
        if (!(g >= lo && g < hi)) {
            cur = find_item(items, n_items, g, kFieldBtile);
            const mer_item c = items[cur];
            lo = c.btile;
            hi = lo + (long long)((c.W + kTW - 1) / kTW) * ((c.H + kTH - 1) / kTH);
        }
        const mer_item m = items[cur];
        const int ntx = (m.W + kTW - 1) / kTW;
        const int local = (int)(g - m.btile);
        BItem it;
        it.vrec = m.vrec;
        it.tri = m.tri;
        it.pix = m.pix;
        it.vert = m.vert;
        it.V = m.V; it.T = m.T; it.H = m.H; it.W = m.W;
        const int tx = local % ntx, ty = local / ntx;
        tile_halo(it, a, tx, ty, S);
        __syncthreads();
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(&hdr->queue_backward, 1ull);
        tile_compute<NA, EXACT, BITS>(it, tx, ty, a, tex, S, ws);
        __syncthreads();
        tile_flush(it, a, S);
    }
}

}  // namespace mer

using namespace mer;

namespace {
// Attribute-gradient channels a launch carries (0 without attribute gradients): the interpolated channels,
// or (u, v) in texture mode.
int attr_channels(const mer_shading* sh, const float* grad_attr) {
    if (!grad_attr) return 0;
    const int A = sh->uv_offset < 0 ? sh->n_main : 2;
    return A >= 1 && A <= kMaxA ? A : -1;
}
}  // namespace

// max_tri_density: the largest T / (H W) over the items (the table size follows the densest item).
extern "C" int mer_launch_backward_batch(const mer_vertex* vpix, const int* tris, const mer_item* items, int n_items,
                                         long long btiles, const int* index, const unsigned char* cover,
                                         const float* image, const float* grad_image, const float* attr, const float* tex,
                                         const mer_shading* sh, int terms, double* grad_vpix, float* grad_attr,
                                         void* ws, int persistent_ctas, double max_tri_density, cudaStream_t s) {
    if (btiles == 0) return 0;
    BwdArgs a;
    a.vpix = vpix; a.tris = tris; a.index = index; a.cover = cover; a.image = image; a.grad = grad_image;
    a.attr = attr; a.grad_vpix = grad_vpix; a.grad_attr = grad_attr;
    a.sh = *sh;
    a.terms = terms;
    a.n = 0; a.H = 0; a.W = 0; a.V = 0; a.T = 0; a.ntx = 0; a.nty = 0;
    a.tex_stride = sh->tex_c > 0 ? sh->tex_c : sh->n_main;
    a.tex_vec4 = a.tex_stride == 4 && tex && (reinterpret_cast<uintptr_t>(tex) & 15u) == 0;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    if (cudaMemsetAsync(&hdr->queue_backward, 0, sizeof(unsigned long long), s) != cudaSuccess) return 2;
    // persistent_ctas sizes the raster's grid (4 resident CTAs per SM); the backward keeps as many waves.
    // Without it, the grid is the device's SM count times the resident CTAs of the instantiation launched.
    const unsigned fixed_grid = persistent_ctas > 0 ? (unsigned)((long long)persistent_ctas * kCtasPerSm / 4) : 0u;
    unsigned grid = fixed_grid;
    int sms = 0;
    if (fixed_grid == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 2;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
    }
    const bool exact = (terms & MER_EXACT_CROSSING) != 0;
    // the resident-CTA grid of kernel k (when no grid was given)
    auto grid_of = [&](const void* k) -> unsigned {
        if (fixed_grid > 0) return fixed_grid;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0) != cudaSuccess) return 0u;
        return (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    };
#define MER_BWD_BATCH(A, E)                                                                                        \
    do {                                                                                                           \
        grid = grid_of((const void*)k_backward_batch<A, E, kTableBits>);                                           \
        if (grid == 0) return 2;                                                                                   \
        k_backward_batch<A, E, kTableBits><<<grid, kThreads, 0, s>>>(vpix, tris, items, n_items, btiles, index,   \
                                                                     cover, image, grad_image, attr, tex, a,      \
                                                                     grad_vpix, grad_attr, ws);                   \
    } while (0)
    const bool dense = max_tri_density > kDenseTrianglesPerPixel;
    switch (attr_channels(sh, grad_attr) * 2 + (exact ? 1 : 0)) {
        case 0:
            if (dense) {
                grid = grid_of((const void*)k_backward_batch<0, false, kTableBitsDense>);
                if (grid == 0) return 2;
                k_backward_batch<0, false, kTableBitsDense><<<grid, kThreads, 0, s>>>(
                    vpix, tris, items, n_items, btiles, index, cover, image, grad_image, attr, tex, a, grad_vpix,
                    grad_attr, ws);
            } else {
                MER_BWD_BATCH(0, false);
            }
            break;
        case 1: MER_BWD_BATCH(0, true); break;
        case 2: MER_BWD_BATCH(1, false); break;
        case 3: MER_BWD_BATCH(1, true); break;
        case 4: MER_BWD_BATCH(2, false); break;
        case 5: MER_BWD_BATCH(2, true); break;
        case 6: MER_BWD_BATCH(3, false); break;
        case 7: MER_BWD_BATCH(3, true); break;
        case 8: MER_BWD_BATCH(4, false); break;
        case 9: MER_BWD_BATCH(4, true); break;
        default: return 1;
    }
#undef MER_BWD_BATCH
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int mer_launch_backward(const mer_vertex* vpix, int V, const int* tris, int T, int n, int H, int W,
                                   const int* index, const unsigned char* cover, const float* image, const float* grad_image, const float* attr,
                                   const float* tex, const mer_shading* sh, int terms, double* grad_vpix,
                                   float* grad_attr, void* ws, cudaStream_t s) {
    BwdArgs a;
    a.vpix = vpix; a.tris = tris; a.index = index; a.cover = cover; a.image = image; a.grad = grad_image;
    a.attr = attr; a.grad_vpix = grad_vpix; a.grad_attr = grad_attr;
    a.sh = *sh;
    a.terms = terms;
    a.n = n; a.H = H; a.W = W; a.V = V; a.T = T;
    a.ntx = (W + kTW - 1) / kTW;
    a.nty = (H + kTH - 1) / kTH;
    a.tex_stride = sh->tex_c > 0 ? sh->tex_c : sh->n_main;
    a.tex_vec4 = a.tex_stride == 4 && tex && (reinterpret_cast<uintptr_t>(tex) & 15u) == 0;
    const long long blocks = (long long)a.ntx * a.nty * n;
    if (blocks == 0) return 0;
    const bool exact = (terms & MER_EXACT_CROSSING) != 0;
#define MER_BWD(A, E)                                                                                             \
    k_backward<A, E, kTableBits><<<(unsigned)blocks, kThreads, 0, s>>>(vpix, tris, index, cover, image, grad_image, attr, tex, a, \
                                                           grad_vpix, grad_attr, ws)
    const bool dense = (double)T > kDenseTrianglesPerPixel * (double)H * (double)W;
    switch (attr_channels(sh, grad_attr) * 2 + (exact ? 1 : 0)) {
        case 0:
            if (dense)
                k_backward<0, false, kTableBitsDense><<<(unsigned)blocks, kThreads, 0, s>>>(
                    vpix, tris, index, cover, image, grad_image, attr, tex, a, grad_vpix, grad_attr, ws);
            else
                MER_BWD(0, false);
            break;
        case 1: MER_BWD(0, true); break;
        case 2: MER_BWD(1, false); break;
        case 3: MER_BWD(1, true); break;
        case 4: MER_BWD(2, false); break;
        case 5: MER_BWD(2, true); break;
        case 6: MER_BWD(3, false); break;
        case 7: MER_BWD(3, true); break;
        case 8: MER_BWD(4, false); break;
        case 9: MER_BWD(4, true); break;
        default: return 1;
    }
#undef MER_BWD
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
