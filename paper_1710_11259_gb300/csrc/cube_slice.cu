// Slice-resident inner level of the FP32 cube ADI (Sec. 5, inner Stein equations in
// the residual-propagating form of cube.cu's stein_res).
//
// The inner level solves A~_a Z A~_b + c Z = R on every slice across the third mode,
// as the Sylvester equation A Z - Z B = C (A = A~_a, B = -c A~_b^{-1}, C = R A~_b^{-1})
// by J ADI iterations in residual form:
//   rho_0 = R A~_b^{-1};  for l:  a1 = rho (B - p)^{-1} = -(A~_b rho)(c + p A~_b)^{-1}
//                                 (l = 0: -R (c + p A~_b)^{-1}),
//                                 Z  += (q - p) (A - q)^{-1} a1,
//                                 rho = (q - p)(A - q)^{-1} w + w,  w = rho + (p - q) a1.
// Slices are independent, so one cluster of 8 CTAs keeps one n x n slice in shared
// memory for all J iterations: CTA r owns rows [r w, r w + w) (w = n/8) in row layout
// for the solves along mb (lane = row, sequential along the row) and columns
// [r w, r w + w) in column layout for the solves along ma (lane = column).  Between
// the two the CTA gathers its columns of a1 and rho from the row owners through
// distributed shared memory, and before the next row solves it pulls its rows of the
// new rho from the column owners; two cluster barriers per iteration (hardware, no
// spin loop) order the phases.  HBM sees R once and Z once
// per inner solve instead of several whole-tensor passes per iteration.
// Every banded solve is the even/odd Thomas sweep of App. B with precomputed
// factors {1/den_t, u_t} of (alpha A~ + beta).
#include <cooperative_groups.h>

#include "cube_slice.cuh"

namespace cg = cooperative_groups;

namespace fps {

namespace {

constexpr int kThreads = 256;
constexpr int kC = 8;  // read-ahead chunk of the sweeps
// rows (of at most w = 32 per CTA) that one of the 8 warps moves per owner in the
// gather and pull phases
constexpr int kRowsPerWarp = 32 / (kThreads / 32);

__host__ __device__ __forceinline__ int slice_w(int n) { return (n + kSliceCluster - 1) / kSliceCluster; }
// Rows keep two zero halo entries on each side (element t at offset 2 + t), so the
// band product A~ rho along a row needs no bounds tests; the pitch is odd so that the
// 32 lanes of a warp (32 rows, same t) hit 32 banks.
__host__ __device__ __forceinline__ int row_pitch(int n) { return (n + 4) | 1; }
__host__ __device__ __forceinline__ int64_t stride_of(int mode, int n)
{
    return mode == 0 ? (int64_t)n * n : (mode == 1 ? (int64_t)n : 1);
}

// Floats of the shared-memory layout: two row arrays [w][P], four column arrays
// [n][w], then (8-byte aligned) two factor sets [n] of float2, d [n] and e with two
// zeros on each side [n + 4].
__host__ __device__ __forceinline__ int slice_floats_before_fac(int n)
{
    const int f = 2 * slice_w(n) * row_pitch(n) + 4 * n * slice_w(n);
    return (f + 1) & ~1;
}

// The sweeps below are the even/odd Thomas recurrences with factors {1/den_t, u_t}:
// forward z_t = in_t - u_{t-2} z_{t-2}, backward x_t = z_t / den_t - u_t x_{t+2}, run in
// chunks of kC steps whose shared-memory operands are read before the dependent
// FMAs.  Two right-hand sides that share a chain run in the same loop (two
// independent dependency chains per thread).

// Rows at the start: rho = (A~)^{-1} IN (set fM) and a1 = -(c + p_0 A~)^{-1} IN (set fA),
// IN in rb; rho to ra, a1 in place.
__device__ __forceinline__ void rows_first(const float2 *__restrict__ fM, const float2 *__restrict__ fA,
                                           float *__restrict__ ra, float *__restrict__ rb, int n, int par)
{
    const int m = (n - par + 1) >> 1;
    float z1 = 0.f, z2 = 0.f, u1 = 0.f, u2 = 0.f;
    for (int i0 = 0; i0 < m; i0 += kC) {
        float v[kC];
        float2 f1[kC], f2[kC];
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            const int t = par + 2 * min(i0 + u, m - 1);
            v[u] = rb[t];
            f1[u] = fM[t];
            f2[u] = fA[t];
        }
#pragma unroll
        for (int u = 0; u < kC; ++u)
            if (i0 + u < m) {
                const int t = par + 2 * (i0 + u);
                z1 = fmaf(-u1, z1, v[u]);
                z2 = fmaf(-u2, z2, -v[u]);
                ra[t] = z1;
                rb[t] = z2;
                u1 = f1[u].y;
                u2 = f2[u].y;
            }
    }
    float x1 = 0.f, x2 = 0.f;
    for (int i0 = m - 1; i0 >= 0; i0 -= kC) {
        float za[kC], zb[kC];
        float2 f1[kC], f2[kC];
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            const int t = par + 2 * max(i0 - u, 0);
            za[u] = ra[t];
            zb[u] = rb[t];
            f1[u] = fM[t];
            f2[u] = fA[t];
        }
#pragma unroll
        for (int u = 0; u < kC; ++u)
            if (i0 - u >= 0) {
                const int t = par + 2 * (i0 - u);
                x1 = fmaf(-f1[u].y, x1, f1[u].x * za[u]);
                x2 = fmaf(-f2[u].y, x2, f2[u].x * zb[u]);
                ra[t] = x1;
                rb[t] = x2;
            }
    }
}

// Rows, l > 0: a1 = -(c + p A~)^{-1} (A~ rho) along the row (set f), rho in ra (with
// halo), a1 to rb.  beH[t + 2] = e_t (zero outside [0, n - 2)).
__device__ __forceinline__ void rows_a1(const float2 *__restrict__ f, const float *__restrict__ bd,
                                        const float *__restrict__ beH, const float *__restrict__ ra,
                                        float *__restrict__ rb, int n, int par)
{
    const int m = (n - par + 1) >> 1;
    float z = 0.f, up = 0.f;
    for (int i0 = 0; i0 < m; i0 += kC) {
        float v[kC], uf[kC];
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            const int t = par + 2 * min(i0 + u, m - 1);
            v[u] = -fmaf(beH[t + 2], ra[t + 2], fmaf(beH[t], ra[t - 2], bd[t] * ra[t]));
            uf[u] = f[t].y;
        }
#pragma unroll
        for (int u = 0; u < kC; ++u)
            if (i0 + u < m) {
                z = fmaf(-up, z, v[u]);
                rb[par + 2 * (i0 + u)] = z;
                up = uf[u];
            }
    }
    float x = 0.f;
    for (int i0 = m - 1; i0 >= 0; i0 -= kC) {
        float zz[kC];
        float2 ff[kC];
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            const int t = par + 2 * max(i0 - u, 0);
            zz[u] = rb[t];
            ff[u] = f[t];
        }
#pragma unroll
        for (int u = 0; u < kC; ++u)
            if (i0 - u >= 0) {
                x = fmaf(-ff[u].y, x, ff[u].x * zz[u]);
                rb[par + 2 * (i0 - u)] = x;
            }
    }
}

// Columns: with w_t = rho_t + (p - q) a1_t, rho <- (q - p)(A - q)^{-1} w + w (when
// `more`) and Z <- Z + (q - p)(A - q)^{-1} a1, both with the set f.  Chain element i of
// column cj, parity par is at (par + 2i) * stride + cj; cR holds rho (then w, then the
// new rho), cT the z of the rho chain, cA a1 (then the z of the Z chain).
__device__ __forceinline__ void cols_update(const float2 *__restrict__ f, float *__restrict__ cR,
                                            float *__restrict__ cA, float *__restrict__ cT, float *__restrict__ cZ,
                                            int n, int par, int stride, float p, float q, bool more)
{
    const int m = (n - par + 1) >> 1;
    const int s2 = 2 * stride;
    const float pq = p - q, qp = q - p;
    float z1 = 0.f, z2 = 0.f, up = 0.f;
    for (int i0 = 0; i0 < m; i0 += kC) {
        float r[kC], a[kC], uf[kC];
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            const int i = min(i0 + u, m - 1);
            r[u] = more ? cR[i * s2] : 0.f;
            a[u] = cA[i * s2];
            uf[u] = f[par + 2 * i].y;
        }
#pragma unroll
        for (int u = 0; u < kC; ++u)
            if (i0 + u < m) {
                const int k = (i0 + u) * s2;
                const float win = fmaf(pq, a[u], r[u]);
                z1 = fmaf(-up, z1, win);
                z2 = fmaf(-up, z2, a[u]);
                if (more) {
                    cR[k] = win;
                    cT[k] = z1;
                }
                cA[k] = z2;
                up = uf[u];
            }
    }
    float x1 = 0.f, x2 = 0.f;
    for (int i0 = m - 1; i0 >= 0; i0 -= kC) {
        float zt[kC], za[kC], rr[kC], zz[kC];
        float2 ff[kC];
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            const int i = max(i0 - u, 0);
            const int k = i * s2;
            zt[u] = more ? cT[k] : 0.f;
            rr[u] = more ? cR[k] : 0.f;
            za[u] = cA[k];
            zz[u] = cZ[k];
            ff[u] = f[par + 2 * i];
        }
#pragma unroll
        for (int u = 0; u < kC; ++u)
            if (i0 - u >= 0) {
                const int k = (i0 - u) * s2;
                x1 = fmaf(-ff[u].y, x1, ff[u].x * zt[u]);
                x2 = fmaf(-ff[u].y, x2, ff[u].x * za[u]);
                if (more) cR[k] = fmaf(qp, x1, rr[u]);
                cZ[k] = fmaf(qp, x2, zz[u]);
            }
    }
}

__global__ void __launch_bounds__(kThreads, 1) stein_slice_kernel(SliceArgs a)
{
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int n = a.n, w = slice_w(n), P = row_pitch(n);
    const int64_t sb = stride_of(a.mb, n), sa = stride_of(a.ma, n);
    const int64_t base = (int64_t)(blockIdx.x / kSliceCluster) * stride_of(3 - a.ma - a.mb, n);
    const int r0 = rank * w;
    const int nr = max(0, min(w, n - r0));  // rows owned, and columns owned (same split)

    extern __shared__ __align__(16) float sm[];
    float *rowA = sm;              // rho, row layout [w][P] (halo of 2)
    float *rowB = rowA + w * P;    // a1 (first the right-hand side), row layout
    float *colR = rowB + w * P;    // rho, column layout [n][w]
    float *colA = colR + n * w;    // a1, column layout
    float *colZ = colA + n * w;    // Z, column layout
    float *colT = colZ + n * w;    // z of the rho column sweeps
    float2 *fM = reinterpret_cast<float2 *>(sm + slice_floats_before_fac(n));  // set of the mb solve
    float2 *fA = fM + n;                                                        // set of the ma solve
    float *bd = reinterpret_cast<float *>(fA + n);
    float *beH = bd + n;           // beH[t + 2] = e_t
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kThreads / 32;

    // ---- load: bands, the first two factor sets, zero rows, rhs rows (warp per row,
    // lanes along the row), Z columns (warp per row of the slice, lanes along columns)
    for (int t = tid; t < n + 4; t += kThreads) {
        beH[t] = (t >= 2 && t < n + 2) ? a.e[t - 2] : 0.f;
        if (t < n) {
            bd[t] = a.d[t];
            fM[t] = a.fac[t];          // set 0: A~
            fA[t] = a.fac[n + t];      // set 1: c + p_0 A~
        }
    }
    for (int k = tid; k < 2 * w * P; k += kThreads) rowA[k] = 0.f;
    __syncthreads();
    for (int li = warp; li < nr; li += kWarps) {
        const int64_t g0 = base + (int64_t)(r0 + li) * sa;
        for (int t = lane; t < n; t += 32) {
            float v = a.r1 * a.R1[g0 + (int64_t)t * sb];
            if (a.R2) v = fmaf(a.r2, a.R2[g0 + (int64_t)t * sb], v);
            rowB[li * P + 2 + t] = v;
        }
    }
    for (int t = warp; t < n; t += kWarps)
        for (int cj = lane; cj < nr; cj += 32)
            colZ[t * w + cj] = a.accumulate ? a.Z[base + (int64_t)t * sa + (int64_t)(r0 + cj) * sb] : 0.f;
    __syncthreads();

    // ---- rho_0 = R A~_b^{-1} and a1 = -R (c + p_0 A~_b)^{-1} along the rows
    if (tid < 2 * nr) {
        const int par = tid / nr, li = tid - par * nr;
        rows_first(fM, fA, rowA + li * P + 2, rowB + li * P + 2, n, par);
    }

    for (int l = 0; l < a.J; ++l) {
        const float p = (float)a.ab[1 + 2 * l].x, q = (float)-a.ab[2 + 2 * l].y;
        const bool more = l + 1 < a.J;
        if (l > 0) {
            // pull this CTA's rows of the new rho from the column owners (their column
            // sweeps ended before the last cluster barrier): warp per row, lanes along
            // the owner's columns
            // (w <= 32: one lane per column; all remote loads of a warp in flight
            // before the local stores)
            float v[kSliceCluster][kRowsPerWarp];
#pragma unroll
            for (int o = 0; o < kSliceCluster; ++o) {
                const int nc = max(0, min(w, n - o * w));
                const float *src = cl.map_shared_rank(colR, o);
#pragma unroll
                for (int j = 0; j < kRowsPerWarp; ++j) {
                    const int li = warp + j * kWarps;
                    v[o][j] = (li < nr && lane < nc) ? src[(r0 + li) * w + lane] : 0.f;
                }
            }
#pragma unroll
            for (int o = 0; o < kSliceCluster; ++o) {
                const int nc = max(0, min(w, n - o * w));
#pragma unroll
                for (int j = 0; j < kRowsPerWarp; ++j) {
                    const int li = warp + j * kWarps;
                    if (li < nr && lane < nc) rowA[li * P + 2 + o * w + lane] = v[o][j];
                }
            }
        }
        if (l == 0) __syncthreads();  // the first two sweeps read fM / fA
        for (int t = tid; t < n; t += kThreads) {  // later: last read before the last cluster barrier
            if (l > 0) fM[t] = a.fac[(int64_t)(1 + 2 * l) * n + t];
            fA[t] = a.fac[(int64_t)(2 + 2 * l) * n + t];
        }
        __syncthreads();
        if (l > 0 && tid < 2 * nr) {  // a1 = -(A~_b rho)(c + p A~_b)^{-1} along the rows
            const int par = tid / nr, li = tid - par * nr;
            rows_a1(fM, bd, beH, rowA + li * P + 2, rowB + li * P + 2, n, par);
        }
        cl.sync();  // a1 rows complete in every CTA (and rho rows, pulled above)
        // gather this CTA's columns of a1 (and rho) from the row owners: warp per row of
        // the slice, lanes along the columns (coalesced on both sides)
        for (int o0 = 0; o0 < kSliceCluster; o0 += 2) {  // two owners' rows in flight at a time
            float va[2][kRowsPerWarp], vr[2][kRowsPerWarp];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int o = o0 + h, nro = max(0, min(w, n - o * w));
                const float *srcB = cl.map_shared_rank(rowB, o);
                const float *srcA = cl.map_shared_rank(rowA, o);
#pragma unroll
                for (int j = 0; j < kRowsPerWarp; ++j) {
                    const int lr = warp + j * kWarps;
                    const bool ok = lr < nro && lane < nr;
                    va[h][j] = ok ? srcB[lr * P + 2 + r0 + lane] : 0.f;
                    vr[h][j] = (ok && more) ? srcA[lr * P + 2 + r0 + lane] : 0.f;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int o = o0 + h, nro = max(0, min(w, n - o * w));
#pragma unroll
                for (int j = 0; j < kRowsPerWarp; ++j) {
                    const int lr = warp + j * kWarps;
                    if (lr < nro && lane < nr) {
                        const int t = o * w + lr;
                        colA[t * w + lane] = va[h][j];
                        colR[t * w + lane] = vr[h][j];
                    }
                }
            }
        }
        __syncthreads();
        if (tid < 2 * nr) {  // along the columns: the rho and Z updates in one sweep
            const int par = tid / nr, cj = tid - par * nr;
            const int o0 = par * w + cj;
            cols_update(fA, colR + o0, colA + o0, colT + o0, colZ + o0, n, par, w, p, q, more);
        }
        // every CTA has gathered this iteration's rows and finished its column sweeps:
        // rows may be rewritten (pull, next a1), the new rho columns may be read, and
        // after the last iteration no CTA leaves while another still reads its memory
        cl.sync();
    }

    // ---- Z out (this CTA's columns of the slice)
    for (int t = warp; t < n; t += kWarps)
        for (int cj = lane; cj < nr; cj += 32)
            a.Z[base + (int64_t)t * sa + (int64_t)(r0 + cj) * sb] = colZ[t * w + cj];
}

}  // namespace

int slice_smem_bytes(int n)
{
    return (int)sizeof(float) * (slice_floats_before_fac(n) + 4 * n + n + (n + 4));
}

cudaError_t slice_setup(int n, bool *usable)
{
    *usable = false;
    if (n < 1 || n > kSliceMaxN) return cudaSuccess;
    const int smem = slice_smem_bytes(n);
    cudaError_t e = cudaFuncSetAttribute(stein_slice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kSliceCluster);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kSliceCluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, stein_slice_kernel, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;  // not usable; the caller keeps the streaming path
    }
    *usable = clusters > 0;
    return cudaSuccess;
}

cudaError_t launch_stein_slice(const SliceArgs &a, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(kSliceCluster * a.n));  // one cluster per slice
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = (size_t)slice_smem_bytes(a.n);
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kSliceCluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, stein_slice_kernel, a);
}

}  // namespace fps
