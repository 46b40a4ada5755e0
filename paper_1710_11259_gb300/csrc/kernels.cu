// sm_103a kernels of the square ADI solve (Algorithm 2 on the symmetrised
// equation (3.9); banded shifted solves by the Thomas algorithm on the even and
// odd index sets, App. B / P3).  The work is HBM/ALU bound streaming with a
// sequential recurrence per system; there is no dense contraction, so no tensor
// cores are involved.
#include "kernels.cuh"
#include "device_info.h"

namespace fps {

namespace {

constexpr int kCols = 32;   // columns per CTA (one warp per row parity)
constexpr int kTR = 32;     // rows per transposed-store tile
constexpr int kRing = 16;   // prefetch depth (rows) of the per-warp rings
constexpr int kGrp = 4;     // rows per ring wait: their independent work (stencil, scaling) overlaps

template <typename T> struct Pair;
template <> struct Pair<double> { using type = double2; };
template <> struct Pair<float> { using type = float2; };

// ---------------------------------------------------------------------------
// Asynchronous global->shared copies (cp.async, per-thread 4/8/16 bytes).  Rows
// are prefetched D-1 steps ahead of the Thomas recurrence so that the load
// latency overlaps the sequential elimination; a copy with valid == false
// zero-fills its destination without reading memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

template <int B>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(B),
                 "r"(valid ? B : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Per-warp prefetch rings.  Forward: G row segment (32), V row segment with a
// two-column halo on each side (36, padded to 40), factors of the row.
// Backward: spill row segment (32) and factors.
template <typename T, int D>
struct FwdRing {
    T g[D][32];
    T v[D][40];
    typename Pair<T>::type f[D];
};
template <typename T, int D>
struct BwdRing {
    T z[D][32];
    typename Pair<T>::type f[D];
};
template <typename T, int D>
union WarpRing {
    FwdRing<T, D> fw;
    BwdRing<T, D> bw;
};

// ---------------------------------------------------------------------------
// Half-step kernel.  CTA = 2 warps over 32 consecutive columns k0..k0+31;
// warp `par` owns the rows i = par, par+2, ... of those columns.
//   forward:  r_i = G[i,k] - (e_{k-2} V[i,k-2] + (d_k+q) V[i,k] + e_k V[i,k+2])
//             z_i = r_i - uf_{i-2} z_{i-2}          (spilled to Z)
//   backward: x_i = ip_i z_i - uf_i x_{i+2}
// The backward results are staged in a shared-memory tile and stored
// transposed (Out[k*n + i]) so that the next half-step reads them row-wise.
// ---------------------------------------------------------------------------
template <typename T, bool ZERO_V, bool TRANS, int D>
__global__ void __launch_bounds__(64) halfstep_kernel(const T *__restrict__ V, const T *__restrict__ G,
                                                      T *__restrict__ Z, T *__restrict__ Out,
                                                      const typename Pair<T>::type *__restrict__ fac,
                                                      const T *__restrict__ dband, const T *__restrict__ eband, T q,
                                                      int64_t n)
{
    using P = typename Pair<T>::type;
    __shared__ __align__(16) WarpRing<T, D> rings[2];
    __shared__ T tile[kCols][kTR + 1];
    const int lane = threadIdx.x & 31;
    const int par = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * kCols;
    const int64_t k = k0 + lane;
    const bool kin = k < n;
    WarpRing<T, D> &R = rings[par];

    T em = 0, c0 = 0, ep = 0;
    if (kin) {
        c0 = dband[k] + q;
        if (k >= 2) em = eband[k - 2];
        ep = eband[k];  // zero-padded: e[k] = 0 when k + 2 >= n
    }
    const int64_t m = (n - par + 1) / 2;  // rows of this parity

    // ---------------- forward elimination ----------------
    auto issue_fwd = [&](int64_t t) {
        if (t < m) {
            const int s = (int)(t % D);
            const int64_t i = par + 2 * t;
            cp_async<sizeof(T)>(&R.fw.g[s][lane], kin ? G + i * n + k : G, kin);
            if (!ZERO_V) {
                const int64_t kk = k0 - 2 + lane;
                const bool ok = kk >= 0 && kk < n;
                cp_async<sizeof(T)>(&R.fw.v[s][lane], ok ? V + i * n + kk : V, ok);
                if (lane < 4) {
                    const int64_t kh = k0 + 30 + lane;
                    const bool okh = kh < n;
                    cp_async<sizeof(T)>(&R.fw.v[s][32 + lane], okh ? V + i * n + kh : V, okh);
                }
            }
            if (lane == 31) cp_async<sizeof(P)>(&R.fw.f[s], fac + i, true);
        }
        cp_commit();
    };
    // Rows are consumed kGrp at a time: the stencils of a group are independent, so
    // only the recurrence z_i = r_i - uf z_{i-2} stays serial.  One commit group per
    // row; D - kGrp rows stay in flight.
    for (int t = 0; t < D - kGrp; ++t) issue_fwd(t);
    T z = 0, uf_prev = 0;
    for (int64_t t0 = 0; t0 < m; t0 += kGrp) {
        __syncwarp();
#pragma unroll
        for (int g = 0; g < kGrp; ++g) issue_fwd(t0 + D - kGrp + g);
        cp_wait<D - kGrp>();
        __syncwarp();
        T r[kGrp], ufs[kGrp];
#pragma unroll
        for (int g = 0; g < kGrp; ++g) {
            const int s = (int)((t0 + g) % D);
            T a = R.fw.g[s][lane];
            if (!ZERO_V) {
                a = fma(-em, R.fw.v[s][lane], a);
                a = fma(-c0, R.fw.v[s][lane + 2], a);
                a = fma(-ep, R.fw.v[s][lane + 4], a);
            }
            r[g] = a;
            ufs[g] = R.fw.f[s].y;
        }
#pragma unroll
        for (int g = 0; g < kGrp; ++g)
            if (t0 + g < m) {
                z = fma(-uf_prev, z, r[g]);
                uf_prev = ufs[g];
                if (kin) Z[(par + 2 * (t0 + g)) * n + k] = z;
            }
    }
    cp_wait<0>();
    __syncwarp();

    // ---------------- backward substitution ----------------
    // u counts rows from the last one: t = m-1-u.
    auto issue_bwd = [&](int64_t u) {
        if (u < m) {
            const int s = (int)(u % D);
            const int64_t i = par + 2 * (m - 1 - u);
            cp_async<sizeof(T)>(&R.bw.z[s][lane], kin ? Z + i * n + k : Z, kin);
            if (lane == 31) cp_async<sizeof(P)>(&R.bw.f[s], fac + i, true);
        }
        cp_commit();
    };
    // Rows again kGrp at a time (each iteration issues as many rows as it consumes,
    // so D - kGrp stay in flight); the products ip z of a group are independent.
    for (int u = 0; u < D - kGrp; ++u) issue_bwd(u);
    T x = 0;
    int64_t u = 0;
    if (!TRANS) {
        for (; u < m; u += kGrp) {
            __syncwarp();
#pragma unroll
            for (int g = 0; g < kGrp; ++g) issue_bwd(u + D - kGrp + g);
            cp_wait<D - kGrp>();
            __syncwarp();
            T w[kGrp], uf[kGrp];
#pragma unroll
            for (int g = 0; g < kGrp; ++g) {
                const int s = (int)((u + g) % D);
                const P f = R.bw.f[s];
                w[g] = f.x * R.bw.z[s][lane];
                uf[g] = f.y;
            }
#pragma unroll
            for (int g = 0; g < kGrp; ++g)
                if (u + g < m) {
                    x = fma(-uf[g], x, w[g]);
                    if (kin) Out[(par + 2 * (m - 1 - (u + g))) * n + k] = x;
                }
        }
        cp_wait<0>();
        return;
    }
    const int64_t ntile = (n + kTR - 1) / kTR;
    for (int64_t b = ntile - 1; b >= 0; --b) {
        const int64_t ilo = b * kTR;
        const int64_t ihi = (ilo + kTR < n) ? ilo + kTR : n;
        int64_t istart = ihi - 1;
        if (((istart - par) & 1) != 0) --istart;
        const int nr = (istart >= ilo) ? (int)((istart - ilo) / 2 + 1) : 0;  // rows of this parity in the tile
        for (int r0 = 0; r0 < nr; r0 += kGrp) {
            const int cnt = (nr - r0 < kGrp) ? nr - r0 : kGrp;
            __syncwarp();
#pragma unroll
            for (int g = 0; g < kGrp; ++g)
                if (g < cnt) issue_bwd(u + D - kGrp + g);
            cp_wait<D - kGrp>();
            __syncwarp();
            T w[kGrp], uf[kGrp];
#pragma unroll
            for (int g = 0; g < kGrp; ++g) {
                const int s = (int)((u + g) % D);
                const P f = R.bw.f[s];
                w[g] = f.x * R.bw.z[s][lane];
                uf[g] = f.y;
            }
#pragma unroll
            for (int g = 0; g < kGrp; ++g)
                if (g < cnt) {
                    x = fma(-uf[g], x, w[g]);
                    tile[lane][istart - 2 * (r0 + g) - ilo] = x;
                }
            u += cnt;
        }
        __syncthreads();
        const int rows = (int)(ihi - ilo);
        for (int idx = threadIdx.x; idx < kCols * kTR; idx += 64) {
            const int c = idx / kTR, rr = idx % kTR;
            if (k0 + c < n && rr < rows) Out[(k0 + c) * n + ilo + rr] = tile[c][rr];
        }
        __syncthreads();
    }
    cp_wait<0>();
}

// Thomas factors of A~ - q_j I for one (shift, parity) per thread.
__global__ void factor_kernel(const double *__restrict__ d, const double *__restrict__ e, const double *__restrict__ q,
                              int J, int64_t n, double2 *__restrict__ fac)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 2 * J) return;
    const int j = tid >> 1, par = tid & 1;
    const double qj = q[j];
    double uf_prev = 0.0;
    for (int64_t i = par; i < n; i += 2) {
        double den = d[i] - qj;
        if (i >= 2) den -= e[i - 2] * uf_prev;
        const double ip = 1.0 / den;
        const double uf = e[i] * ip;
        fac[(int64_t)j * n + i] = make_double2(ip, uf);
        uf_prev = uf;
    }
}

// F~ = D_s F D_s and F~^T through a 32x32 shared tile.
__global__ void scale_in_kernel(const double *__restrict__ F, double *__restrict__ Ft, double *__restrict__ FtT,
                                const double *__restrict__ s, int64_t n)
{
    __shared__ double t[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = by + r, k = bx + threadIdx.x;
        if (i < n && k < n) {
            const double v = F[i * n + k] * s[i] * s[k];
            Ft[i * n + k] = v;
            t[r][threadIdx.x] = v;
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t k = bx + r, i = by + threadIdx.x;
        if (i < n && k < n) FtT[k * n + i] = t[threadIdx.x][r];
    }
}

__global__ void scale_out_kernel(const double *__restrict__ Y, double *__restrict__ X, const double *__restrict__ s,
                                 int64_t n)
{
    const int64_t nn = n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / n, k = t - i * n;
        X[t] = Y[t] * s[i] * s[k];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_halfstep(const HalfStep<T> &h, cudaStream_t st)
{
    const dim3 grid((unsigned)((h.n + kCols - 1) / kCols)), block(64);
    using P = typename Pair<T>::type;
    const P *fac = static_cast<const P *>(h.fac);
    if (h.V == nullptr) {
        if (h.transposed_out)
            halfstep_kernel<T, true, true, kRing><<<grid, block, 0, st>>>(h.V, h.G, h.Z, h.Out, fac, h.d, h.e, h.q, h.n);
        else
            halfstep_kernel<T, true, false, kRing><<<grid, block, 0, st>>>(h.V, h.G, h.Z, h.Out, fac, h.d, h.e, h.q, h.n);
    } else {
        if (h.transposed_out)
            halfstep_kernel<T, false, true, kRing><<<grid, block, 0, st>>>(h.V, h.G, h.Z, h.Out, fac, h.d, h.e, h.q, h.n);
        else
            halfstep_kernel<T, false, false, kRing><<<grid, block, 0, st>>>(h.V, h.G, h.Z, h.Out, fac, h.d, h.e, h.q, h.n);
    }
    return cudaGetLastError();
}

template cudaError_t launch_halfstep<double>(const HalfStep<double> &, cudaStream_t);

cudaError_t launch_factors(const double *d, const double *e, const double *q, int J, int64_t n, double2 *fac,
                           cudaStream_t st)
{
    const int threads = 2 * J;
    factor_kernel<<<(threads + 127) / 128, 128, 0, st>>>(d, e, q, J, n, fac);
    return cudaGetLastError();
}

cudaError_t launch_scale_in(const double *F, double *Ft, double *FtT, const double *s, int64_t n, cudaStream_t st)
{
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
    scale_in_kernel<<<grid, block, 0, st>>>(F, Ft, FtT, s, n);
    return cudaGetLastError();
}

cudaError_t launch_scale_out(const double *Y, double *X, const double *s, int64_t n, cudaStream_t st)
{
    const int64_t nn = n * n;
    int blocks = (int)((nn + 255) / 256);
    const int cap = 16 * current_sm_count();
    if (blocks > cap) blocks = cap;
    scale_out_kernel<<<blocks, 256, 0, st>>>(Y, X, s, n);
    return cudaGetLastError();
}

}  // namespace fps
