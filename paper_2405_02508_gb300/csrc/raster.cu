// raster.cu -- rasterization module with z-buffer (Supp. B): triangle setup and
// tile binning, then a per-tile raster that stages the tile's triangle records in
// shared memory and resolves visibility in a shared-memory z-buffer.
//
// Pipeline per call:
//   setup + count : per (item, triangle): cull, exact setup record, pixel bbox,
//                   count the bin tiles it overlaps
//   scan          : exclusive scan of the per-tile counts -> list offsets
//   fill          : scatter triangle ids into the per-tile lists
//   raster<TS>    : one CTA per tile: coverage + depth test, write index / depth / bary
// The per-item bodies are shared by the multi-view entry point (items = the views of
// one mesh, addressed by strides) and by the batched path (items from a table; the
// raster runs as a persistent kernel pulling tiles from a device work queue).
#include <cuda_runtime.h>

#include <mutex>

#include "shade_device.cuh"

namespace mer {

// One item of a raster pass: a mesh seen by one camera.
struct RItem {
    const mer_vertex* vpix;  // the item's vertex records
    const int* tris;         // the item's triangles (item-local vertex ids)
    TriRaster* recs;         // the item's raster records
    int V, T, H, W;
    int ntx, nty;            // bin tiles across / down
    long long tile0;         // first global bin tile of the item
    long long pix0;          // first global pixel of the item
    long long vert;          // first attribute row of the item's mesh
};

// Fused shading of the resolved tile (mer_batch_render): the deferred shading arguments and buffers.
struct ShadeOut {
    ShadeArgs a;
    const float* attr;  // attribute rows of all meshes
    const float* tex;
    float* image;       // [pixels, C]
};

__device__ __forceinline__ int floordiv256(int a) { return a >> 8; }  // arithmetic shift = floor

// Pixel bbox of the centres (256x+128) inside [mn, mx] (snapped units), clamped to [0, lim-1].
__device__ __forceinline__ void centre_range(int mn, int mx, int lim, int& lo, int& hi) {
    // x >= ceil((mn - 128) / 256), x <= floor((mx - 128) / 256)
    lo = -floordiv256(-(mn - 128));
    hi = floordiv256(mx - 128);
    lo = max(lo, 0);
    hi = min(hi, lim - 1);
}

// Setup record of triangle t of an item; counts the bin tiles it overlaps.
__device__ __forceinline__ void setup_count_one(const RItem& it, int t, int tile, int* __restrict__ counts,
                                                void* ws) {
    TriRaster r;
    r.flags = (int)0x80000000;  // culled unless set up below
    r.bx0 = 1; r.bx1 = 0; r.by0 = 1; r.by1 = 0;
    int vid[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        vid[k] = it.tris[3 * (size_t)t + k];
        if (vid[k] < 0 || vid[k] >= it.V) ok = false;
    }
    if (!ok) {
        set_status(ws, kStatusRange);
        it.recs[t] = r;
        return;
    }
    float zeta[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // the 32-byte vertex record as two 128-bit loads (records are 32-byte aligned)
        const float4 a = __ldg(reinterpret_cast<const float4*>(it.vpix + vid[k]));
        const float4 b = __ldg(reinterpret_cast<const float4*>(it.vpix + vid[k]) + 1);
        if ((__float_as_uint(b.z) & kValid) != kValid) ok = false;  // flags
        r.X[k] = __float_as_int(a.x);
        r.Y[k] = __float_as_int(a.y);
        zeta[k] = b.x;
    }
    if (!ok) { it.recs[t] = r; return; }
    const int64_t a2 = (int64_t)(r.X[1] - r.X[0]) * (r.Y[2] - r.Y[0]) - (int64_t)(r.Y[1] - r.Y[0]) * (r.X[2] - r.X[0]);
    if (a2 == 0) { it.recs[t] = r; return; }
    const int mnx = min(r.X[0], min(r.X[1], r.X[2])), mxx = max(r.X[0], max(r.X[1], r.X[2]));
    const int mny = min(r.Y[0], min(r.Y[1], r.Y[2])), mxy = max(r.Y[0], max(r.Y[1], r.Y[2]));
    int x0, x1, y0, y1;
    centre_range(mnx, mxx, it.W, x0, x1);
    centre_range(mny, mxy, it.H, y0, y1);
    if (x0 > x1 || y0 > y1) { it.recs[t] = r; return; }
    const int s = a2 > 0 ? 1 : -1;
    int fl = a2 > 0 ? 0 : 8;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int j = (e + 1) % 3, k = (e + 2) % 3;
        const int64_t ga = (int64_t)s * (r.Y[j] - r.Y[k]);
        const int64_t gb = (int64_t)s * (r.X[k] - r.X[j]);
        if (ga > 0 || (ga == 0 && gb > 0)) fl |= 1 << e;
    }
    const bool small = mxx - mnx < (1 << 14) && mxy - mny < (1 << 14);
    if (small) fl |= 16;  // small: exact 32-bit coverage from the edge functions
    r.flags = fl;
    const float Df = ll2f_rn(a2 < 0 ? -a2 : a2);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.zd[k] = __fdiv_rn(zeta[k], Df);
    r.zmax = fmaxf(zeta[0], fmaxf(zeta[1], zeta[2]));
    r.bx0 = (short)x0; r.bx1 = (short)x1; r.by0 = (short)y0; r.by1 = (short)y1;
    r.K[0] = r.K[1] = r.K[2] = 0;
    if (small) {
        // s e_i(P) = s (X_j Y_k - Y_j X_k) + s (Y_j - Y_k) P_x + s (X_k - X_j) P_y with P = 256 (x, y) + 128:
        // coefficients of the pixel indices and the constant with tl_i - 1 folded in, all modulo 2^32
        int ex[3], ey[3], ek[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int j = (e + 1) % 3, k = (e + 2) % 3;
            const unsigned A = (unsigned)(s * (r.Y[j] - r.Y[k])), B = (unsigned)(s * (r.X[k] - r.X[j]));
            const unsigned c = (unsigned)r.X[j] * (unsigned)r.Y[k] - (unsigned)r.Y[j] * (unsigned)r.X[k];
            ex[e] = (int)(256u * A);
            ey[e] = (int)(256u * B);
            ek[e] = (int)((s > 0 ? c : 0u - c) + 128u * A + 128u * B + (unsigned)((fl >> e) & 1) - 1u);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            r.X[e] = ex[e];
            r.Y[e] = ey[e];
            r.K[e] = ek[e];
        }
    }
    it.recs[t] = r;
    int* cnt = counts + it.tile0;
    if (y0 / tile == y1 / tile && x0 / tile == x1 / tile) {
        // one bin tile (the common case): lanes of the warp counting into the same tile add once together
        int* c = cnt + (y0 / tile) * it.ntx + x0 / tile;
        const unsigned peers = __match_any_sync(__activemask(), (unsigned long long)c);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(c, __popc(peers));
        return;
    }
    for (int ty = y0 / tile; ty <= y1 / tile; ++ty)
        for (int tx = x0 / tile; tx <= x1 / tile; ++tx) atomicAdd(cnt + ty * it.ntx + tx, 1);
}

// Bin lists are split by facing: triangles with a negative snapped area (facing the camera for an
// outward-oriented mesh) from the start of the tile's list, the others from its end.  The raster draws the
// first part, then culls triangles of the second part that lie wholly behind the tile's depth buffer.
__device__ __forceinline__ void fill_one(const RItem& it, int t, int tile, const int* __restrict__ offs,
                                         const int* __restrict__ counts, int* __restrict__ cursor,
                                         int* __restrict__ cursor_back, int* __restrict__ list, long long capacity) {
    const TriRaster& r = it.recs[t];
    if (r.flags < 0) return;
    const bool front = (r.flags & 8) != 0;
    if (r.by0 / tile == r.by1 / tile && r.bx0 / tile == r.bx1 / tile) {
        // one bin tile: lanes filling the same (tile, part) take consecutive positions with one atomic
        const size_t g = it.tile0 + (size_t)(r.by0 / tile) * it.ntx + r.bx0 / tile;
        int* cur = front ? cursor + g : cursor_back + g;
        const unsigned peers = __match_any_sync(__activemask(), (unsigned long long)cur);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(cur, __popc(peers));
        base = __shfl_sync(peers, base, leader) + __popc(peers & ((1u << lane) - 1u));
        const long long pos = front ? (long long)offs[g] + base : (long long)offs[g] + counts[g] - 1 - base;
        if (pos < capacity) list[pos] = t;
        return;
    }
    for (int ty = r.by0 / tile; ty <= r.by1 / tile; ++ty)
        for (int tx = r.bx0 / tile; tx <= r.bx1 / tile; ++tx) {
            const size_t g = it.tile0 + (size_t)ty * it.ntx + tx;
            const long long pos = front ? (long long)offs[g] + atomicAdd(cursor + g, 1)
                                        : (long long)offs[g] + counts[g] - 1 - atomicAdd(cursor_back + g, 1);
            if (pos < capacity) list[pos] = t;
        }
}

// --- exclusive scan of the tile counts (3 kernels, 1024 elements per block) ---
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const int before = warp > 0 ? sh[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_blocks(const int* __restrict__ in, long long N, int* __restrict__ out, int* __restrict__ sums) {
    __shared__ int sh[32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const int v = i < N ? in[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, sh, total);
    if (i < N) out[i] = ex;
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single CTA: exclusive scan of the block sums (looping), total written to the header.
__global__ void k_scan_sums(int* __restrict__ sums, int nb, void* ws, long long capacity) {
    __shared__ int sh[32];
    int carry = 0;
    for (int base = 0; base < nb; base += kScanBlock) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? sums[i] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sh, total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        WsHeader* h = reinterpret_cast<WsHeader*>(ws);
        h->total_bins = carry;
        h->capacity = capacity;
        h->queue_raster = 0ull;
        if (carry > capacity) atomicOr(&h->status, kStatusOverflow);
    }
}

// Adds the block offsets and clears the front and back fill cursors (cursor[0, 2N)).
__global__ void k_scan_add(int* __restrict__ out, long long N, const int* __restrict__ sums, int* __restrict__ cursor) {
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    if (i < N) {
        out[i] += sums[blockIdx.x];
        cursor[i] = 0;
        cursor[N + i] = 0;
    }
}

// --- raster ---
// One CTA per tile.  The tile's triangle records are staged in shared memory; each warp takes one
// triangle at a time and its lanes test the pixels of the triangle's bounding box inside the tile (32 at a
// time), so the work follows the bounding-box areas and every lane of a warp runs the same triangle.  The
// nearest fragment per pixel is resolved in a shared-memory z-buffer by a 64-bit atomicMax on
// (depth key bits << 32 | ~triangle id): larger depth key wins, equal keys go to the lower id.
constexpr int kStage = 256;  // triangle records staged per round
constexpr int kRasterThreads = 256;
constexpr int kRasterCtasPerSm = 4;  // resident CTAs per SM (the 64 x 64 tile's shared memory allows four): 64 registers

// Per-pixel bits kept in shared memory for the cover image: a front-facing triangle covered the centre
// (taken when the front part is done), two or more did, one / two or more back-facing ones did, and a
// back-facing fragment raised the depth buffer (the winner is then back-facing: the front part is drawn
// first, so every later raise comes from a back-facing fragment).
constexpr unsigned kCovF1 = 1, kCovF2 = 2, kCovB1 = 4, kCovB2 = 8, kCovWB = 16;

template <int TS>
struct RasterShared {
    static constexpr int kStageTS = TS >= 64 ? 160 : kStage;  // keeps the 64 x 64 tile within 48 KB
    TriRaster rec[kStageTS];
    int id[kStageTS];
    unsigned long long zbuf[TS * TS];
    unsigned cov[TS * TS / 4];  // cover-image bits (kCov*), one byte a pixel
    float red[kRasterThreads / 32];
};

// Smallest depth key (zeta_test) over the tile's pixels inside the image, 0 if one of them is still empty.
// All threads call it; it starts and ends with a barrier.
// With `cover`, also records which pixels a front-facing triangle covers (kCovF1).
template <int TS>
__device__ __forceinline__ float tile_min_zeta(RasterShared<TS>& S, int ox, int oy, int W, int H, bool cover) {
    __syncthreads();
    float mn = 3.0e38f;
    for (int i = threadIdx.x; i < TS * TS; i += kRasterThreads) {
        const int px = ox + (i % TS), py = oy + (i / TS);
        if (px >= W || py >= H) continue;
        const unsigned long long key = S.zbuf[i];
        if (cover && key) atomicOr(&S.cov[i >> 2], kCovF1 << ((i & 3) * 8));
        mn = fminf(mn, key ? __uint_as_float((unsigned)(key >> 32)) : 0.0f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = mn;
    __syncthreads();
    float r = S.red[0];
#pragma unroll
    for (int w = 1; w < kRasterThreads / 32; ++w) r = fminf(r, S.red[w]);
    __syncthreads();
    return r;
}

// SHADE: also shade every pixel of the tile from its z-buffer winner (shade_fragment, as the deferred
// shading kernels do from the index image).
// cover (optional): one byte a pixel (MER_COVER_* bits): whether another triangle of the winner's facing,
// or one of the other facing, covers the pixel centre, the facing of the winner and which borders of its bin
// tile the pixel lies on, from the kCov* bits.  The counts leave out the triangles of the second part that
// are skipped as hidden, which win no pixel of this tile, so they are exact for every triangle that wins a
// pixel of the same bin tile.
// The tile's list holds the camera-facing triangles first (nfront of them) and the others after; before
// the second part the tile's smallest depth key is taken, and a triangle of that part whose largest vertex
// zeta (with a margin above the FP32 rounding of the key) is below it cannot win any pixel: it is skipped.
template <int TS, bool SHADE>
__device__ __forceinline__ void raster_tile(const RItem& it, int local_tile, const int* __restrict__ offs,
                                            const int* __restrict__ cnts, const int* __restrict__ nfront,
                                            const int* __restrict__ list, bool overflow, RasterShared<TS>& S,
                                            int* __restrict__ index, float* __restrict__ depth,
                                            float* __restrict__ bary, unsigned char* __restrict__ cover,
                                            const ShadeOut& so, void* ws) {
    constexpr int kSt = RasterShared<TS>::kStageTS;
    const long long tile = it.tile0 + local_tile;
    const int ty = local_tile / it.ntx, tx = local_tile % it.ntx;
    const int ox = tx * TS, oy = ty * TS;
    for (int i = threadIdx.x; i < TS * TS; i += kRasterThreads) S.zbuf[i] = 0ull;
    if (cover)
        for (int i = threadIdx.x; i < TS * TS / 4; i += kRasterThreads) S.cov[i] = 0u;
    const int count = overflow ? 0 : cnts[tile];
    const int off = overflow ? 0 : offs[tile];
    const int nf = overflow ? 0 : min(nfront[tile], count);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kRasterThreads / 32;
    float zcull = 0.0f;
    int m = 0;
    for (int base = 0; base < count; base += m) {
        // stage boundaries fall on the front / back split so each stage is one part
        const int lim = base < nf ? nf : count;
        m = min(kSt, lim - base);
        if (base == nf && base > 0) zcull = tile_min_zeta<TS>(S, ox, oy, it.W, it.H, cover != nullptr);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kRasterThreads) {
            const int t = list[off + base + j];
            S.rec[j] = it.recs[t];
            S.id[j] = t;
        }
        __syncthreads();
        const bool back = base >= nf;
        for (int j = warp; j < m; j += kWarps) {
            const TriRaster r = S.rec[j];  // in registers: the loop's shared-memory atomics would force reloads
            if (back && r.zmax * (1.0f + 0x1p-20f) < zcull) continue;  // hidden behind the whole tile
            const int x0 = max((int)r.bx0, ox), x1 = min((int)r.bx1, ox + TS - 1);
            const int y0 = max((int)r.by0, oy), y1 = min((int)r.by1, oy + TS - 1);
            const int bw = x1 - x0 + 1, bh = y1 - y0 + 1;
            if (bw <= 0 || bh <= 0) continue;
            const int npx = bw * bh;
            const unsigned idkey = 0xFFFFFFFFu - (unsigned)S.id[j];
            // lane -> (dx, dy) in the bbox, then advance by 32 pixels per pass without dividing per pixel.  The
            // quotients q / bw (q <= 32, bw <= TS <= 64) come from an approximate reciprocal: the product is within
            // 2^-16 of q / bw, whose fraction is 0 or at least 1/64, so q / bw + 2^-10 truncates to the quotient.
            const float rb = __fdividef(1.0f, (float)bw);
            int dy = (int)__fmaf_rn((float)lane, rb, 0x1p-10f);
            int dx = lane - dy * bw;
            const int sy = (int)__fmaf_rn(32.0f, rb, 0x1p-10f), sx = 32 - sy * bw;
            for (int i = lane; i < npx; i += 32) {
                const int px = x0 + dx, py = y0 + dy;
                dx += sx;
                dy += sy;
                if (dx >= bw) {
                    dx -= bw;
                    ++dy;
                }
                float z;
                if (r.flags & 16) {
                    int E[3];
                    if (!covers_small(r, px, py, E)) continue;
                    z = depth_key_small(r, E);
                } else {
                    int64_t E[3];
                    if (!covers(r, 256 * px + 128, 256 * py + 128, E)) continue;
                    z = depth_key(r, E);
                }
                const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | idkey;
                const int pi = (py - oy) * TS + (px - ox);
                // the 64-bit maximum runs as a compare-and-swap loop: its old value costs nothing extra
                const unsigned long long old = atomicMax(&S.zbuf[pi], key);
                if (cover) {
                    const unsigned sh = (pi & 3) * 8;
                    if (!back) {
                        if (old) atomicOr(&S.cov[pi >> 2], kCovF2 << sh);  // a front fragment came first
                    } else {
                        if (key > old) atomicOr(&S.cov[pi >> 2], kCovWB << sh);
                        const unsigned o = atomicOr(&S.cov[pi >> 2], kCovB1 << sh);
                        if (o & (kCovB1 << sh)) atomicOr(&S.cov[pi >> 2], kCovB2 << sh);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TS * TS; i += kRasterThreads) {
        const int px = ox + (i % TS), py = oy + (i / TS);
        if (px >= it.W || py >= it.H) continue;
        const unsigned long long key = S.zbuf[i];
        const int t = key ? (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull)) : -1;
        const size_t p = (size_t)it.pix0 + (size_t)py * it.W + px;
        index[p] = t;
        if (cover) {
            const int lx = i % TS, ly = i / TS;
            unsigned c = (lx == 0 ? MER_COVER_BORDER_L : 0u) | (lx == TS - 1 ? MER_COVER_BORDER_R : 0u) |
                         (ly == 0 ? MER_COVER_BORDER_T : 0u) | (ly == TS - 1 ? MER_COVER_BORDER_B : 0u);
            if (t >= 0) {
                const unsigned b = S.cov[i >> 2] >> ((i & 3) * 8);
                if (b & kCovWB) {  // kCovF1 was taken before the back part (none if the tile has no front part)
                    c |= MER_COVER_WINNER_BACK | ((b & kCovB2) ? MER_COVER_SAME_2 : 0u) |
                         ((b & kCovF1) ? MER_COVER_OTHER_1 : 0u);
                } else {
                    c |= ((b & kCovF2) ? MER_COVER_SAME_2 : 0u) | ((b & kCovB1) ? MER_COVER_OTHER_1 : 0u);
                }
            }
            cover[p] = (unsigned char)c;
        }
        if (SHADE)
            shade_fragment(it.vpix, it.V, it.tris, it.T, t, px, py,
                           so.attr ? so.attr + (size_t)it.vert * so.a.sh.C_attr : nullptr, so.tex, so.a,
                           so.image + p * so.a.sh.C, ws);
        if (!depth && !bary) continue;
        float Z = 0.f, b1 = 0.f, b2 = 0.f;
        if (t >= 0) {
            const VRec v[3] = {load_vrec(it.vpix + it.tris[3 * (size_t)t]), load_vrec(it.vpix + it.tris[3 * (size_t)t + 1]),
                               load_vrec(it.vpix + it.tris[3 * (size_t)t + 2])};
            const Bary B = screen_bary(v, px, py);
            const float z0 = v[0].zeta, z1 = v[1].zeta, z2 = v[2].zeta;
            const float s = B.lam[0] * z0 + B.lam[1] * z1 + B.lam[2] * z2;
            const float is = rcp_nr(s);
            Z = is;
            b1 = B.lam[1] * z1 * is;
            b2 = B.lam[2] * z2 * is;
        }
        if (depth) depth[p] = Z;
        if (bary) {
            bary[2 * p] = b1;
            bary[2 * p + 1] = b2;
        }
    }
    __syncthreads();  // the next tile reuses the shared buffers
}

// ---- multi-view entry: items are the views of one mesh, addressed by strides ----
struct BinGeom {
    int n, H, W, T, V, tile, ntx, nty;
    long long tiles_per_view;
};

__device__ __forceinline__ RItem view_item(const BinGeom& g, const mer_vertex* vpix, const int* tris,
                                           TriRaster* recs, int view) {
    RItem it;
    it.vpix = vpix + (size_t)view * g.V;
    it.tris = tris;
    it.recs = recs + (size_t)view * g.T;
    it.V = g.V; it.T = g.T; it.H = g.H; it.W = g.W;
    it.ntx = g.ntx; it.nty = g.nty;
    it.tile0 = (long long)view * g.tiles_per_view;
    it.pix0 = (long long)view * g.H * g.W;
    it.vert = 0;
    return it;
}

__global__ void k_setup_count(const mer_vertex* __restrict__ vpix, const int* __restrict__ tris, BinGeom g,
                              TriRaster* __restrict__ recs, int* __restrict__ counts, void* ws) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)g.T * g.n) return;
    const int view = (int)(i / g.T), t = (int)(i % g.T);
    setup_count_one(view_item(g, vpix, tris, recs, view), t, g.tile, counts, ws);
}

__global__ void k_bin_fill(const mer_vertex* __restrict__ vpix, const int* __restrict__ tris, BinGeom g,
                           TriRaster* __restrict__ recs, const int* __restrict__ offs, const int* __restrict__ counts,
                           int* __restrict__ cursor, int* __restrict__ list, long long capacity) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)g.T * g.n) return;
    const int view = (int)(i / g.T), t = (int)(i % g.T);
    fill_one(view_item(g, vpix, tris, recs, view), t, g.tile, offs, counts, cursor,
             cursor + (long long)g.n * g.tiles_per_view, list, capacity);
}

template <int TS>
__global__ void __launch_bounds__(kRasterThreads, kRasterCtasPerSm) k_raster(TriRaster* __restrict__ recs, BinGeom g,
                                                           const int* __restrict__ offs, const int* __restrict__ cnts,
                                                           const int* __restrict__ nfront,
                                                           const int* __restrict__ list, const mer_vertex* __restrict__ vpix,
                                                           const int* __restrict__ tris, void* ws, long long capacity,
                                                           int* __restrict__ index, float* __restrict__ depth,
                                                           float* __restrict__ bary, unsigned char* __restrict__ cover) {
    __shared__ RasterShared<TS> S;
    const WsHeader* hdr = reinterpret_cast<const WsHeader*>(ws);
    const bool overflow = hdr->total_bins > capacity;
    const long long tile = blockIdx.x;
    const int view = (int)(tile / g.tiles_per_view);
    const int local = (int)(tile % g.tiles_per_view);
    ShadeOut none;
    none.attr = nullptr; none.tex = nullptr; none.image = nullptr;
    raster_tile<TS, false>(view_item(g, vpix, tris, recs, view), local, offs, cnts, nfront, list, overflow, S, index,
                           depth, bary, cover, none, ws);
}

// ---- batched entry: items from a table ----
struct BatchGeom {
    const mer_item* items;
    int n_items, tile;
    long long trecs, tiles;
};

__device__ __forceinline__ RItem batch_item(const mer_item& m, int tile, const mer_vertex* vpix, const int* tris,
                                            TriRaster* recs) {
    RItem it;
    it.vpix = vpix + m.vrec;
    it.tris = tris + 3 * m.tri;
    it.recs = recs + m.trec;
    it.V = m.V; it.T = m.T; it.H = m.H; it.W = m.W;
    it.ntx = (m.W + tile - 1) / tile;
    it.nty = (m.H + tile - 1) / tile;
    it.tile0 = m.tile;
    it.pix0 = m.pix;
    it.vert = m.vert;
    return it;
}

__global__ void k_setup_count_batch(const mer_vertex* __restrict__ vpix, const int* __restrict__ tris, BatchGeom b,
                                    TriRaster* __restrict__ recs, int* __restrict__ counts, void* ws) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = block_find_item(b.items, b.n_items, (long long)blockIdx.x * blockDim.x, i, kFieldTrec);
    if (i >= b.trecs) return;
    const mer_item m = b.items[k];
    setup_count_one(batch_item(m, b.tile, vpix, tris, recs), (int)(i - m.trec), b.tile, counts, ws);
}

__global__ void k_bin_fill_batch(const mer_vertex* __restrict__ vpix, const int* __restrict__ tris, BatchGeom b,
                                 TriRaster* __restrict__ recs, const int* __restrict__ offs,
                                 const int* __restrict__ counts, int* __restrict__ cursor, int* __restrict__ list,
                                 long long capacity) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = block_find_item(b.items, b.n_items, (long long)blockIdx.x * blockDim.x, i, kFieldTrec);
    if (i >= b.trecs) return;
    const mer_item m = b.items[k];
    fill_one(batch_item(m, b.tile, vpix, tris, recs), (int)(i - m.trec), b.tile, offs, counts, cursor,
             cursor + b.tiles, list, capacity);
}

// Persistent: each CTA takes the next global tile from the work queue until none is left.
template <int TS, bool SHADE>
__global__ void __launch_bounds__(kRasterThreads, kRasterCtasPerSm) k_raster_batch(TriRaster* __restrict__ recs, BatchGeom b,
                                                                 const int* __restrict__ offs,
                                                                 const int* __restrict__ cnts,
                                                                 const int* __restrict__ nfront,
                                                                 const int* __restrict__ list,
                                                                 const mer_vertex* __restrict__ vpix,
                                                                 const int* __restrict__ tris, void* ws,
                                                                 long long capacity, int* __restrict__ index,
                                                                 float* __restrict__ depth, float* __restrict__ bary,
                                                                 unsigned char* __restrict__ cover, ShadeOut so) {
    __shared__ RasterShared<TS> S;
    __shared__ long long s_tile;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    const bool overflow = hdr->total_bins > capacity;
    int cur = 0;                       // item of the previous tile and its tile range [lo, hi)
    long long lo = 0, hi = 0;
    while (true) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(&hdr->queue_raster, 1ull);
        __syncthreads();
        const long long g = s_tile;
        if (g >= b.tiles) break;
        // consecutive tiles of a CTA mostly belong to the same item: search the table only on a change
        if (!(g >= lo && g < hi)) {
            cur = find_item(b.items, b.n_items, g, kFieldTile);
            const mer_item c = b.items[cur];
            lo = c.tile;
            hi = lo + (long long)((c.W + TS - 1) / TS) * ((c.H + TS - 1) / TS);
        }
        const mer_item m = b.items[cur];
        raster_tile<TS, SHADE>(batch_item(m, b.tile, vpix, tris, recs), (int)(g - m.tile), offs, cnts, nfront, list,
                               overflow, S, index, depth, bary, cover, so, ws);  // ends with a barrier: s_tile may be overwritten after it
    }
}

}  // namespace mer

using namespace mer;

namespace {
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct RasterLayout {
    size_t hdr, counts, offs, cursor, sums, recs, list, total;
    long long ntiles, nblocks, capacity;
};

RasterLayout layout_for(long long ntiles, long long nrecs, long long capacity) {
    RasterLayout L;
    L.ntiles = ntiles;
    L.nblocks = (ntiles + kScanBlock - 1) / kScanBlock;
    if (capacity <= 0) capacity = 4LL * nrecs + 2LL * ntiles + 1024;
    L.capacity = capacity;
    size_t o = 0;
    L.hdr = o; o += align256(sizeof(WsHeader));
    L.counts = o; o += align256((size_t)ntiles * 4);
    L.offs = o; o += align256((size_t)ntiles * 4);
    L.cursor = o; o += align256((size_t)ntiles * 8);  // front and back fill cursors
    L.sums = o; o += align256((size_t)(L.nblocks + 1) * 4);
    L.recs = o; o += align256((size_t)nrecs * sizeof(TriRaster));
    L.list = o; o += align256((size_t)capacity * 4);
    L.total = o;
    return L;
}

RasterLayout raster_layout(int V, int T, int n, int H, int W, int tile, long long capacity) {
    (void)V;
    const long long ntx = (W + tile - 1) / tile, nty = (H + tile - 1) / tile;
    return layout_for(ntx * nty * (long long)n, (long long)n * T, capacity);
}

// Scan of the per-tile counts and the header totals.
int launch_scan(const RasterLayout& L, char* base, long long capacity, cudaStream_t s) {
    WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
    int* counts = reinterpret_cast<int*>(base + L.counts);
    int* offs = reinterpret_cast<int*>(base + L.offs);
    int* cursor = reinterpret_cast<int*>(base + L.cursor);
    int* sums = reinterpret_cast<int*>(base + L.sums);
    if (L.nblocks > 0) k_scan_blocks<<<(unsigned)L.nblocks, kScanBlock, 0, s>>>(counts, L.ntiles, offs, sums);
    k_scan_sums<<<1, kScanBlock, 0, s>>>(sums, (int)L.nblocks, hdr, capacity);
    if (L.nblocks > 0) k_scan_add<<<(unsigned)L.nblocks, kScanBlock, 0, s>>>(offs, L.ntiles, sums, cursor);
    return 0;
}
}  // namespace

extern "C" size_t mer_raster_workspace_size(int V, int T, int n, int H, int W, int tile, long long capacity) {
    return raster_layout(V, T, n, H, W, tile, capacity).total;
}

extern "C" int mer_launch_rasterize(const mer_vertex* vpix, int V, const int* tris, int T, int n, int H, int W,
                                    int tile, void* ws, size_t ws_bytes, int* index, float* depth, float* bary,
                                    unsigned char* cover, cudaStream_t s) {
    // capacity: whatever the workspace holds beyond the fixed part
    RasterLayout L = raster_layout(V, T, n, H, W, tile, 1);
    if (ws_bytes < L.total) return 1;
    const long long capacity = (long long)((ws_bytes - L.list) / 4);
    L = raster_layout(V, T, n, H, W, tile, capacity);
    char* base = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
    int* counts = reinterpret_cast<int*>(base + L.counts);
    int* offs = reinterpret_cast<int*>(base + L.offs);
    int* cursor = reinterpret_cast<int*>(base + L.cursor);
    TriRaster* recs = reinterpret_cast<TriRaster*>(base + L.recs);
    int* list = reinterpret_cast<int*>(base + L.list);
    BinGeom g;
    g.n = n; g.H = H; g.W = W; g.T = T; g.V = V; g.tile = tile;
    g.ntx = (W + tile - 1) / tile;
    g.nty = (H + tile - 1) / tile;
    g.tiles_per_view = (long long)g.ntx * g.nty;
    // header: the status word is sticky until mer_sync_status; k_scan_sums writes the totals
    if (cudaMemsetAsync(counts, 0, (size_t)L.ntiles * 4, s) != cudaSuccess) return 2;
    const long long NT = (long long)T * n;
    if (NT > 0) k_setup_count<<<(unsigned)((NT + 255) / 256), 256, 0, s>>>(vpix, tris, g, recs, counts, hdr);
    launch_scan(L, base, capacity, s);
    if (NT > 0)
        k_bin_fill<<<(unsigned)((NT + 255) / 256), 256, 0, s>>>(vpix, tris, g, recs, offs, counts, cursor, list,
                                                                capacity);
    const unsigned grid = (unsigned)L.ntiles;
    switch (tile) {
        case 8: k_raster<8><<<grid, kRasterThreads, 0, s>>>(recs, g, offs, counts, cursor, list, vpix, tris, hdr, capacity, index, depth, bary, cover); break;
        case 16: k_raster<16><<<grid, kRasterThreads, 0, s>>>(recs, g, offs, counts, cursor, list, vpix, tris, hdr, capacity, index, depth, bary, cover); break;
        case 32: k_raster<32><<<grid, kRasterThreads, 0, s>>>(recs, g, offs, counts, cursor, list, vpix, tris, hdr, capacity, index, depth, bary, cover); break;
        default: return 1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" size_t mer_batch_raster_workspace_size(long long tiles, long long trecs, long long capacity) {
    return layout_for(tiles, trecs, capacity).total;
}

template <int TS, bool SHADE>
static int launch_raster_batch(unsigned grid, TriRaster* recs, BatchGeom b, const int* offs, const int* counts,
                               const int* nfront, const int* list, const mer_vertex* vpix, const int* tris, void* hdr, long long capacity,
                               int* index, float* depth, float* bary, unsigned char* cover, const ShadeOut& so,
                               cudaStream_t s) {
    if (grid == 0) {
        int per_sm = 0, sms = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 2;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_batch<TS, SHADE>, kRasterThreads, 0) !=
            cudaSuccess)
            return 2;
        grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    }
    k_raster_batch<TS, SHADE><<<grid, kRasterThreads, 0, s>>>(recs, b, offs, counts, nfront, list, vpix, tris, hdr, capacity,
                                                              index, depth, bary, cover, so);
    return 0;
}

template <bool SHADE>
static int launch_raster_batch_tile(int tile, unsigned grid, TriRaster* recs, BatchGeom b, const int* offs,
                                    const int* counts, const int* nfront, const int* list, const mer_vertex* vpix, const int* tris,
                                    void* hdr, long long capacity, int* index, float* depth, float* bary,
                                    unsigned char* cover, const ShadeOut& so, cudaStream_t s) {
    switch (tile) {
        case 16: return launch_raster_batch<16, SHADE>(grid, recs, b, offs, counts, nfront, list, vpix, tris, hdr, capacity, index, depth, bary, cover, so, s);
        case 32: return launch_raster_batch<32, SHADE>(grid, recs, b, offs, counts, nfront, list, vpix, tris, hdr, capacity, index, depth, bary, cover, so, s);
        case 64: return launch_raster_batch<64, SHADE>(grid, recs, b, offs, counts, nfront, list, vpix, tris, hdr, capacity, index, depth, bary, cover, so, s);
        default: return 1;
    }
}

// Binning and the persistent raster of all items; with `so`, each resolved tile is shaded in the same pass.
static int batch_raster(const mer_vertex* vpix, const int* tris, const mer_item* items, int n_items, long long trecs,
                        long long tiles, int tile, void* ws, size_t ws_bytes, int* index, float* depth, float* bary,
                        unsigned char* cover, const ShadeOut* so, int persistent_ctas, cudaStream_t s) {
    RasterLayout L = layout_for(tiles, trecs, 1);
    if (ws_bytes < L.total) return 1;
    const long long capacity = (long long)((ws_bytes - L.list) / 4);
    L = layout_for(tiles, trecs, capacity);
    char* base = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(base + L.hdr);
    int* counts = reinterpret_cast<int*>(base + L.counts);
    int* offs = reinterpret_cast<int*>(base + L.offs);
    int* cursor = reinterpret_cast<int*>(base + L.cursor);
    TriRaster* recs = reinterpret_cast<TriRaster*>(base + L.recs);
    int* list = reinterpret_cast<int*>(base + L.list);
    BatchGeom b;
    b.items = items; b.n_items = n_items; b.tile = tile; b.trecs = trecs; b.tiles = tiles;
    if (tiles > 0 && cudaMemsetAsync(counts, 0, (size_t)tiles * 4, s) != cudaSuccess) return 2;
    if (trecs > 0) k_setup_count_batch<<<(unsigned)((trecs + 255) / 256), 256, 0, s>>>(vpix, tris, b, recs, counts, hdr);
    launch_scan(L, base, capacity, s);  // also resets the raster work queue
    if (trecs > 0)
        k_bin_fill_batch<<<(unsigned)((trecs + 255) / 256), 256, 0, s>>>(vpix, tris, b, recs, offs, counts, cursor, list,
                                                                        capacity);
    if (tiles > 0) {
        const unsigned grid = persistent_ctas > 0 ? (unsigned)persistent_ctas : 0u;
        ShadeOut none;
        none.attr = nullptr; none.tex = nullptr; none.image = nullptr;
        const int rc = so ? launch_raster_batch_tile<true>(tile, grid, recs, b, offs, counts, cursor, list, vpix, tris, hdr,
                                                           capacity, index, depth, bary, cover, *so, s)
                          : launch_raster_batch_tile<false>(tile, grid, recs, b, offs, counts, cursor, list, vpix, tris, hdr,
                                                            capacity, index, depth, bary, cover, none, s);
        if (rc) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int mer_launch_batch_rasterize(const mer_vertex* vpix, const int* tris, const mer_item* items, int n_items,
                                          long long trecs, long long tiles, int tile, void* ws, size_t ws_bytes,
                                          int* index, float* depth, float* bary, unsigned char* cover,
                                          int persistent_ctas, cudaStream_t s) {
    return batch_raster(vpix, tris, items, n_items, trecs, tiles, tile, ws, ws_bytes, index, depth, bary, cover, nullptr,
                        persistent_ctas, s);
}

extern "C" int mer_launch_shade_batch(const mer_vertex*, const int*, const mer_item*, int, long long, const int*,
                                      const float*, const float*, const float*, const mer_shading*, float*, void*,
                                      cudaStream_t);

extern "C" int mer_launch_batch_render(const mer_vertex* vpix, const int* tris, const mer_item* items, int n_items,
                                       long long trecs, long long tiles, long long pixels, int tile, void* ws,
                                       size_t ws_bytes, int* index, float* depth, float* bary, unsigned char* cover,
                                       const float* attr, const float* tex, const float* bg, const mer_shading* sh,
                                       float* image, int persistent_ctas, cudaStream_t s) {
    if (sh->precise) {
        // FP64 shading: the raster pass alone, then the precise shading pass over the index image (the
        // results the fused pass would give with FP64 shading)
        const int rc = batch_raster(vpix, tris, items, n_items, trecs, tiles, tile, ws, ws_bytes, index, depth, bary,
                                    cover, nullptr, persistent_ctas, s);
        if (rc) return rc;
        return mer_launch_shade_batch(vpix, tris, items, n_items, pixels, index, attr, tex, bg, sh, image, ws, s);
    }
    ShadeOut so;
    so.a = make_shade_args(tex, bg, sh);
    so.attr = attr;
    so.tex = tex;
    so.image = image;
    return batch_raster(vpix, tris, items, n_items, trecs, tiles, tile, ws, ws_bytes, index, depth, bary, cover, &so,
                        persistent_ctas, s);
}

// ---------------------------------------------------------------------------------------------------
// mer_rasterize_noalloc: the same binning and raster with the workspace in a fixed device array owned by
// the library, for callers that cannot allocate device memory when they call.
// ---------------------------------------------------------------------------------------------------

namespace {
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB on every GPU that loads the library
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace mer {
__global__ void k_copy_status(const void* ws, int* status_out) {
    *status_out = reinterpret_cast<const WsHeader*>(ws)->status;
}
}  // namespace mer

extern "C" int mer_rasterize_noalloc(const mer_vertex* vpix, int V, const int32_t* tris, int T, int n, int H, int W,
                                     int tile, int32_t* index, float* depth, float* bary, int32_t* status,
                                     void* stream) {
    if (V < 0 || T < 0 || n < 0 || H < 0 || W < 0 || H > kMaxDim || W > kMaxDim) return MER_EINVAL;
    if ((long long)n * H * W >= (1LL << 31)) return MER_EINVAL;
    if (tile != 8 && tile != 16 && tile != 32) return MER_EINVAL;
    if ((long long)n * H * W == 0) return MER_OK;
    if (!index || (T > 0 && (!tris || !vpix))) return MER_EINVAL;
    // the fixed part of the workspace (headers, per-tile counters, one record per view and triangle)
    // must fit; what is left of the array holds the bin lists
    if (raster_layout(V, T, n, H, W, tile, 1).total > kNoAllocScratchBytes) return MER_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MER_ECUDA;
    void* ptr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // host code sees g_noalloc_scratch only as a stand-in symbol: look up its device address once
            // per device, with that device current
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MER_ECUDA;
            g_noalloc_ptr[dev] = p;
        }
        ptr = g_noalloc_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // every call shares the array: clear the status word left by the previous call
    if (cudaMemsetAsync(ptr, 0, sizeof(WsHeader), s) != cudaSuccess) return MER_ECUDA;
    const int rc = mer_launch_rasterize(vpix, V, tris, T, n, H, W, tile, ptr, kNoAllocScratchBytes, index, depth,
                                        bary, nullptr, s);
    if (rc != 0) return rc;
    if (status) {
        k_copy_status<<<1, 1, 0, s>>>(ptr, status);
        if (cudaGetLastError() != cudaSuccess) return MER_ECUDA;
    }
    return MER_OK;
}
