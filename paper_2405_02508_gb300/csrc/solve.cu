// solve.cu -- Laplacian preconditioning of vertex updates (Nicolet et al., "Large Steps in Inverse Rendering
// of Geometry", 2021), which the paper uses for all of its mesh optimisations (Sec. 5 and Supp. B, lambda 16).
//
// The vertex positions x [V, 3] are reparameterised as u = M x with M = I + lambda L, L the combinatorial
// Laplacian of the meshes' edge graph (L_ii = number of neighbours of i, L_ij = -1 for every edge ij).  A
// step then needs M x (once, to start) and two solves M y = b per step: the gradient with respect to u,
// M^-1 dL/dx, and the positions x = M^-1 u after the update.  M is symmetric positive definite (its
// eigenvalues are 1 + lambda * those of L, all >= 1), so the solves are conjugate gradients on the device:
// FP32 vectors, FP64 dot products, all three coordinate columns as one block-diagonal system, the iteration
// scalars kept on the device so a solve is a fixed sequence of launches (graph-capturable) that becomes a
// no-op once the residual is below the tolerance.
//
// The CSR edge graph is built once per mesh on the host (mer_laplacian_csr).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "mer.h"

namespace mer {

constexpr int kSolveThreads = 256;

// Device scalars of one solve, at the start of the solve workspace.
struct CgState {
    double rr;      // r . r of the current residual
    double rr_new;  // r . r after the update of this iteration
    double pAp;     // p . M p
    double rr0;     // b . b (the tolerance is relative to it)
    double tol2;    // (rel_tol)^2 * rr0
    int done;       // 1 once rr <= tol2 (later launches return at once)
    int iters;      // iterations run
    int pad[4];
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

// Row i of y = (I + lambda L) x: x_i + lambda (deg_i x_i - sum of the neighbours' x_j).
__device__ __forceinline__ void apply_row(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                          float lambda, const float* __restrict__ x, int64_t i, float y[3]) {
    const int64_t b = row_ptr[i], e = row_ptr[i + 1];
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int64_t k = b; k < e; ++k) {
        const int64_t j = col[k];
        sx += x[3 * j];
        sy += x[3 * j + 1];
        sz += x[3 * j + 2];
    }
    const float deg = (float)(e - b);
    const float xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    y[0] = xi + lambda * (deg * xi - sx);
    y[1] = yi + lambda * (deg * yi - sy);
    y[2] = zi + lambda * (deg * zi - sz);
}

__global__ void __launch_bounds__(kSolveThreads) k_apply(const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col, int64_t V, float lambda,
                                                         const float* __restrict__ x, float* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    float r[3];
    apply_row(row_ptr, col, lambda, x, i, r);
    y[3 * i] = r[0];
    y[3 * i + 1] = r[1];
    y[3 * i + 2] = r[2];
}

// r = b - M x, p = r; accumulates r . r into st->rr and b . b into st->rr0.
__global__ void __launch_bounds__(kSolveThreads) k_cg_init(const int64_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col, int64_t V, float lambda,
                                                           const float* __restrict__ b, const float* __restrict__ x,
                                                           float* __restrict__ r, float* __restrict__ p,
                                                           CgState* st) {
    __shared__ double sh[kSolveThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0, bb = 0.0;
    if (i < V) {
        float mx[3];
        apply_row(row_ptr, col, lambda, x, i, mx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float bi = b[3 * i + c];
            const float ri = bi - mx[c];
            r[3 * i + c] = ri;
            p[3 * i + c] = ri;
            rr += (double)ri * ri;
            bb += (double)bi * bi;
        }
    }
    const double s1 = block_sum(rr, sh);
    __syncthreads();
    const double s2 = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        atomicAdd(&st->rr, s1);
        atomicAdd(&st->rr0, s2);
    }
}

__global__ void k_cg_start(CgState* st, float rel_tol) {
    st->tol2 = (double)rel_tol * rel_tol * st->rr0;
    st->done = st->rr <= st->tol2 ? 1 : 0;
    st->iters = 0;
    st->pAp = 0.0;
    st->rr_new = 0.0;
}

// Ap = M p, pAp = p . Ap
__global__ void __launch_bounds__(kSolveThreads) k_cg_matvec(const int64_t* __restrict__ row_ptr,
                                                             const int32_t* __restrict__ col, int64_t V,
                                                             float lambda, const float* __restrict__ p,
                                                             float* __restrict__ Ap, CgState* st) {
    __shared__ double sh[kSolveThreads / 32];
    if (st->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (i < V) {
        float y[3];
        apply_row(row_ptr, col, lambda, p, i, y);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Ap[3 * i + c] = y[c];
            d += (double)p[3 * i + c] * y[c];
        }
    }
    const double s = block_sum(d, sh);
    if (threadIdx.x == 0) atomicAdd(&st->pAp, s);
}

// alpha = rr / pAp; x += alpha p; r -= alpha Ap; rr_new = r . r
__global__ void __launch_bounds__(kSolveThreads) k_cg_update(int64_t V, const float* __restrict__ p,
                                                             const float* __restrict__ Ap, float* __restrict__ x,
                                                             float* __restrict__ r, CgState* st) {
    __shared__ double sh[kSolveThreads / 32];
    if (st->done) return;
    const float alpha = st->pAp > 0.0 ? (float)(st->rr / st->pAp) : 0.f;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (i < V) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x[3 * i + c] += alpha * p[3 * i + c];
            const float ri = r[3 * i + c] - alpha * Ap[3 * i + c];
            r[3 * i + c] = ri;
            d += (double)ri * ri;
        }
    }
    const double s = block_sum(d, sh);
    if (threadIdx.x == 0) atomicAdd(&st->rr_new, s);
}

// beta = rr_new / rr; p = r + beta p  (the scalars are advanced by k_cg_next afterwards)
__global__ void __launch_bounds__(kSolveThreads) k_cg_direction(int64_t V, const float* __restrict__ r,
                                                                float* __restrict__ p, const CgState* st) {
    if (st->done) return;
    const float beta = st->rr > 0.0 ? (float)(st->rr_new / st->rr) : 0.f;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[3 * i + c] = r[3 * i + c] + beta * p[3 * i + c];
}

__global__ void k_cg_next(CgState* st) {
    if (st->done) return;
    st->rr = st->rr_new;
    st->rr_new = 0.0;
    st->pAp = 0.0;
    st->iters += 1;
    if (st->rr <= st->tol2) st->done = 1;
}

}  // namespace mer

using namespace mer;

namespace {
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
inline unsigned blocks_for(int64_t V) { return (unsigned)((V + kSolveThreads - 1) / kSolveThreads); }
}  // namespace

extern "C" int mer_laplacian_csr(const int32_t* tris, int64_t T, int64_t V, int64_t* row_ptr, int32_t* col) {
    if (T < 0 || V < 0 || !row_ptr || (T > 0 && !tris) || V >= (int64_t(1) << 31)) return MER_EINVAL;
    for (int64_t t = 0; t < 3 * T; ++t)
        if (tris[t] < 0 || tris[t] >= V) return MER_ERANGE;
    // directed edge list (both directions of every triangle edge), sorted and deduplicated per row
    std::vector<int64_t> deg(V + 1, 0);
    for (int64_t t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) {
            const int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
            if (a == b) continue;
            deg[a] += 1;
            deg[b] += 1;
        }
    std::vector<int64_t> start(V + 1, 0);
    for (int64_t v = 0; v < V; ++v) start[v + 1] = start[v] + deg[v];
    std::vector<int32_t> nb(start[V]);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) {
            const int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
            if (a == b) continue;
            nb[fill[a]++] = b;
            nb[fill[b]++] = a;
        }
    row_ptr[0] = 0;
    for (int64_t v = 0; v < V; ++v) {
        auto first = nb.begin() + start[v], last = nb.begin() + start[v + 1];
        std::sort(first, last);
        const int64_t n = std::unique(first, last) - first;
        if (col) std::copy(first, first + n, col + row_ptr[v]);
        row_ptr[v + 1] = row_ptr[v] + n;
    }
    return MER_OK;
}

extern "C" int mer_precond_apply(const int64_t* row_ptr, const int32_t* col, int64_t V, float lambda,
                                 const float* x, float* y, void* stream) {
    if (V < 0 || !(lambda >= 0.f)) return MER_EINVAL;
    if (V == 0) return MER_OK;
    if (!row_ptr || !col || !x || !y || x == y) return MER_EINVAL;
    k_apply<<<blocks_for(V), kSolveThreads, 0, static_cast<cudaStream_t>(stream)>>>(row_ptr, col, V, lambda, x, y);
    return cudaGetLastError() == cudaSuccess ? MER_OK : MER_ECUDA;
}

extern "C" size_t mer_precond_solve_workspace_size(int64_t V) {
    if (V < 0) return 0;
    return align256(sizeof(CgState)) + 3 * align256((size_t)V * 3 * sizeof(float));
}

extern "C" int mer_precond_solve(const int64_t* row_ptr, const int32_t* col, int64_t V, float lambda,
                                 const float* b, float* x, int max_iters, float rel_tol, void* workspace,
                                 size_t workspace_bytes, void* stream) {
    if (V < 0 || !(lambda >= 0.f) || max_iters < 0 || !(rel_tol >= 0.f)) return MER_EINVAL;
    if (V == 0) return MER_OK;
    if (!row_ptr || !col || !b || !x || b == x || !workspace) return MER_EINVAL;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return MER_EINVAL;
    if (workspace_bytes < mer_precond_solve_workspace_size(V)) return MER_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(workspace);
    CgState* st = reinterpret_cast<CgState*>(base);
    const size_t vec = align256((size_t)V * 3 * sizeof(float));
    float* r = reinterpret_cast<float*>(base + align256(sizeof(CgState)));
    float* p = reinterpret_cast<float*>(base + align256(sizeof(CgState)) + vec);
    float* Ap = reinterpret_cast<float*>(base + align256(sizeof(CgState)) + 2 * vec);
    if (cudaMemsetAsync(st, 0, sizeof(CgState), s) != cudaSuccess) return MER_ECUDA;
    const unsigned g = blocks_for(V);
    k_cg_init<<<g, kSolveThreads, 0, s>>>(row_ptr, col, V, lambda, b, x, r, p, st);
    k_cg_start<<<1, 1, 0, s>>>(st, rel_tol);
    for (int it = 0; it < max_iters; ++it) {
        k_cg_matvec<<<g, kSolveThreads, 0, s>>>(row_ptr, col, V, lambda, p, Ap, st);
        k_cg_update<<<g, kSolveThreads, 0, s>>>(V, p, Ap, x, r, st);
        k_cg_direction<<<g, kSolveThreads, 0, s>>>(V, r, p, st);
        k_cg_next<<<1, 1, 0, s>>>(st);
    }
    return cudaGetLastError() == cudaSuccess ? MER_OK : MER_ECUDA;
}

extern "C" int mer_precond_solve_info(const void* workspace, int* iters, double* rel_residual, void* stream) {
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return MER_EINVAL;
    CgState st;
    if (cudaMemcpyAsync(&st, workspace, sizeof(CgState), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess)
        return MER_ECUDA;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MER_ECUDA;
    if (iters) *iters = st.iters;
    if (rel_residual) *rel_residual = st.rr0 > 0.0 ? std::sqrt(st.rr / st.rr0) : 0.0;
    return MER_OK;
}
