// The cube (Sec. 5): nested ADI for (T_01 + T_02 + T_12) Y = G on n x n x n
// tensors (row-major, mode 0 = i, mode 1 = j, mode 2 = k), T_ab applying A~ on
// modes a and b, G = -F / sqrt(E_i E_j E_k), X = Y / sqrt(E_i E_j E_k).
//   outer  (5.3)-(5.4): H = T_01 + T_02, V = T_12,
//          (V + p) Y_h = G - (H - p) Y,   (H - q) Y+ = G - (V + q) Y_h
//   middle (5.5)-(5.6): H + s = (T_01 + s/2) + (T_02 + s/2),
//          (B' + a) W_h = R - (A' - a) W,  (A' + a) W+ = R - (B' - a) W_h
//   inner  (5.7)-(5.9): A~_a Z A~_b + c Z = R per slice, as A~_a Z - Z(-c A~_b^{-1}) = R A~_b^{-1}:
//          Z_h = [R - (A~_a - p) Z A~_b] (c + p A~_b)^{-1}
//          (A~_a - q) Z+ = (R - c Z_h) A~_b^{-1} - q Z_h
// Every operation is a banded product or a banded (even/odd decoupled, App. B)
// solve along one mode of the whole tensor: all slices of a level are solved at
// once.  The solves run one thread per (line, parity) over 32 lines per CTA with
// coalesced global traffic.  The same kernels run in FP64 and in FP32.
//
// FP32 + refinement: the nested ADI (every level in residual-propagating form, see
// run_residual, hsolve_res, stein_res; every level's shifts on the tight
// Sturm-bisection interval of A~, 2.5x fewer inner iterations than on Lemma B.2's
// at n = 256) runs in FP32 at loose level tolerances on
// the normalised residual rho = R / max|R|, R = G - (T_01 + T_02 + T_12) Y computed
// in FP64 (a 27-point product), and Y += max|R| * delta accumulates in FP64, until
// max|R| / max|G| meets the plan's tolerance.  The defect correction only needs
// each round's correction to reduce the residual, so the loose inner levels make a
// round several times cheaper than one solve at the paper's 1e-15 inner levels.
//
// Index arithmetic inside the kernels is 32-bit where it divides: plans cap n at
// 320, so n^3 < 2^31.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/fps.h"
#include "cube.h"
#include "cube_slice.cuh"
#include "device_info.h"
#include "host_math.h"
#include "trace.h"

namespace fps {

namespace {

constexpr int kLines = 32;  // lines per CTA of the solve kernels
constexpr int kLineThreads = 128;  // threads per CTA: all move the tiles, the first 2 kLines sweep
constexpr int kU = 8;       // global loads in flight per thread in the solve output phase

template <typename T>
struct V2;
template <>
struct V2<double> {
    using type = double2;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <>
struct V2<float> {
    using type = float2;
    static __device__ __forceinline__ float2 make(double a, double b) { return make_float2((float)a, (float)b); }
};

// Y = sop * ((alpha A~ + beta) X along `mode`) + sr * R   (R may be null; Y may alias R)
template <typename T>
__global__ void cube_band_kernel(const T *__restrict__ X, const T *R, T *Y, const T *__restrict__ d,
                                 const T *__restrict__ e, int n, int mode, T alpha, T beta, T sop, T sr)
{
    const int N = n * n * n;
    const int st = (mode == 0) ? n * n : ((mode == 1) ? n : 1);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        const int t = (mode == 0) ? idx / (n * n) : ((mode == 1) ? (idx / n) % n : idx % n);
        T v = (alpha * d[t] + beta) * X[idx];
        if (t >= 2) v = fma(alpha * e[t - 2], X[idx - 2 * st], v);
        if (t + 2 < n) v = fma(alpha * e[t], X[idx + 2 * st], v);
        v *= sop;
        if (R) v = fma(sr, R[idx], v);
        Y[idx] = v;
    }
}

// Z = a X + b Y (element-wise; Z may alias X or Y)
template <typename T>
__global__ void cube_axpby_kernel(const T *X, const T *Y, T *Z, int N, T a, T b)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
        Z[idx] = fma(a, X[idx], b * Y[idx]);
}

// V = a X + b Y + c W (element-wise; V may alias any input)
template <typename T>
__global__ void cube_axpy3_kernel(const T *X, const T *Y, const T *W, T *V, int N, T a, T b, T c)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
        V[idx] = fma(a, X[idx], fma(b, Y[idx], c * W[idx]));
}

// Thomas factors of (alpha A~ + beta I) for a list of (alpha, beta) pairs, computed
// in FP64 and stored in T: one thread per (set, parity); fac[set * n + t] =
// {1/den_t, alpha e_t / den_t}.
template <typename T>
__global__ void cube_factor_kernel(const double *__restrict__ d, const double *__restrict__ e, int n,
                                   const double2 *__restrict__ ab, int nsets, typename V2<T>::type *__restrict__ fac)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 2 * nsets) return;
    const int set = tid >> 1, par = tid & 1;
    const double alpha = ab[set].x, beta = ab[set].y;
    double u_prev = 0.0;
    for (int t = par; t < n; t += 2) {
        double den = alpha * d[t] + beta;
        if (t >= 2) den -= alpha * e[t - 2] * u_prev;
        const double ip = 1.0 / den;
        const double u = alpha * e[t] * ip;
        fac[(int64_t)set * n + t] = V2<T>::make(ip, u);
        u_prev = u;
    }
}

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Asynchronous copy of one element (4 or 8 bytes) from global to shared memory.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src)
{
    if constexpr (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// Shared-memory row pitch of a contiguous-mode tile: odd, so that the 32 lanes of a
// warp (one line each, same t) hit distinct banks.
__host__ __device__ __forceinline__ int contig_pitch(int n) { return (n % 2 == 0) ? n + 1 : n + 2; }

// Elements of one shared-memory tile of the line solve.
__host__ __device__ __forceinline__ int line_tile_elems(int n, bool contig)
{
    return contig ? kLines * contig_pitch(n) : kLines * n;
}

// Dynamic shared memory of the line solve: the factor set and one or two tiles.
template <typename T>
int line_smem_bytes(int n, bool contig, int ntiles)
{
    return n * (int)sizeof(typename V2<T>::type) + ntiles * line_tile_elems(n, contig) * (int)sizeof(T);
}

// 16-byte asynchronous copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// Banded solves along one mode for kLines lines per CTA:
//   IN = s1 R1 + s2 R2            (preband: IN = s1 (A~ R1) along the mode, R2 unused)
//   X  = oscale (alpha A~ + beta)^{-1} IN + oin IN + oacc X      (X read only if oacc != 0)
// The whole tile of R1 (and R2) is fetched with asynchronous copies (16-byte ones
// when the rows are aligned), so one CTA has all its bytes in flight at once.  The
// forward sweep forms IN as it goes; both Thomas sweeps (App. B parity decoupling:
// warp = parity, lane = line) run in shared memory in chunks whose operands are
// read ahead of the dependent FMAs, and the output combination is written back
// coalesced.  X may alias R1 or R2.  Tile A holds R1, then z and x; tile B (present
// when R2, oin or preband is used) holds R2, then IN (oin) or z and x (preband, A
// keeping R1 for the stencil).
// CONTIG (mode 2): kLines consecutive lines, tile [line][t].  Otherwise (modes 0,
// 1): kLines lines adjacent in mode 2, one CTA per (index of the other strided mode,
// block of kLines), tile [t][line].
template <typename T, bool CONTIG>
__global__ void __launch_bounds__(kLineThreads) cube_line_kernel(const typename V2<T>::type *__restrict__ fac, const T *R1,
                                                       T s1, const T *R2, T s2, T *X, int n, int mode, T oscale,
                                                       T oin, T oacc, bool preband, const T *__restrict__ d,
                                                       const T *__restrict__ e)
{
    using F2 = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tsz = line_tile_elems(n, CONTIG);
    F2 *fs = reinterpret_cast<F2 *>(smem_raw);  // the factor set, n entries
    T *A = reinterpret_cast<T *>(fs + n);
    T *B = A + tsz;
    for (int t = threadIdx.x; t < n; t += blockDim.x) fs[t] = fac[t];
    const int pitch = CONTIG ? contig_pitch(n) : 0;
    // geometry: element (li, t) of the tile <-> global offset gbase + li * gl + t * gt
    int nl;
    int64_t gbase, gl, gt;
    if (CONTIG) {
        const int L0 = blockIdx.x * kLines;
        nl = min(kLines, n * n - L0);
        gbase = (int64_t)L0 * n;
        gl = n;
        gt = 1;
    } else {
        const int nkb = (n + kLines - 1) / kLines;
        const int other = blockIdx.x / nkb, k0 = (blockIdx.x % nkb) * kLines;
        const int64_t nn = (int64_t)n * n;
        nl = min(kLines, n - k0);
        gbase = ((mode == 0) ? (int64_t)other * n : (int64_t)other * nn) + k0;
        gl = 1;
        gt = (mode == 0) ? nn : (int64_t)n;
    }
    auto sidx = [&](int li, int t) { return CONTIG ? li * pitch + t : t * kLines + li; };
    // element q of the tile in load/store order (consecutive threads -> consecutive addresses)
    auto qmap = [&](int q, int &li, int &t) {
        if (CONTIG) {
            li = q / n;
            t = q - li * n;
        } else {
            t = q >> 5;
            li = q & 31;
        }
    };
    const bool has_r2 = R2 != nullptr && !preband;
    // strided tiles whose rows are whole, 16-byte aligned rows of the tensor move in
    // 16-byte pieces (V elements)
    constexpr int V = 16 / (int)sizeof(T);
    const bool vec = !CONTIG && nl == kLines && ((gt * (int64_t)sizeof(T)) % 16 == 0) &&
                     ((gbase * (int64_t)sizeof(T)) % 16 == 0) && (((uintptr_t)R1 & 15) == 0) &&
                     (!has_r2 || ((uintptr_t)R2 & 15) == 0) && (((uintptr_t)X & 15) == 0) &&
                     ((n * (int)sizeof(F2)) % 16 == 0);
    const int total = kLines * n;
    if (vec) {
        for (int q = threadIdx.x * V; q < total; q += blockDim.x * V) {
            const int t = q >> 5, li = q & 31;
            const int64_t g = gbase + li + t * gt;
            cp_async16(&A[t * kLines + li], R1 + g);
            if (has_r2) cp_async16(&B[t * kLines + li], R2 + g);
        }
    } else {
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            int li, t;
            qmap(q, li, t);
            if (li < nl) {
                const int64_t g = gbase + li * gl + t * gt;
                cp_async_elem(&A[sidx(li, t)], R1 + g);
                if (has_r2) cp_async_elem(&B[sidx(li, t)], R2 + g);
            }
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    T *Z = preband ? B : A;  // z, then x
    const int lane = threadIdx.x & 31, par = threadIdx.x >> 5;
    const int m = (n - par + 1) / 2;  // unknowns of this parity: t = par + 2 i, i < m
    if (threadIdx.x < 2 * kLines && lane < nl) {
        // Both sweeps in chunks of kC steps: the chunk's operands are read from shared
        // memory first, so only the kC dependent FMAs remain on the critical path.
        constexpr int kC = 8;
        T z = 0, u_prev = 0;
        for (int i0 = 0; i0 < m; i0 += kC) {
            T in[kC], uf[kC];
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int t = par + 2 * min(i0 + u, m - 1);
                T v;
                if (preband) {
                    v = d[t] * A[sidx(lane, t)];
                    if (t >= 2) v = fma(e[t - 2], A[sidx(lane, t - 2)], v);
                    if (t + 2 < n) v = fma(e[t], A[sidx(lane, t + 2)], v);
                    v *= s1;
                } else {
                    v = s1 * A[sidx(lane, t)];
                    if (has_r2) v = fma(s2, B[sidx(lane, t)], v);
                }
                in[u] = v;
                uf[u] = fs[t].y;
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (i0 + u < m) {
                    const int k = sidx(lane, par + 2 * (i0 + u));
                    z = fma(-u_prev, z, in[u]);
                    Z[k] = z;
                    if (oin != T(0)) B[k] = in[u];
                    u_prev = uf[u];
                }
        }
        T x = 0;
        for (int i0 = m - 1; i0 >= 0; i0 -= kC) {
            T zz[kC];
            F2 ff[kC];
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int t = par + 2 * max(i0 - u, 0);
                zz[u] = Z[sidx(lane, t)];
                ff[u] = fs[t];
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (i0 - u >= 0) {
                    x = fma(-ff[u].y, x, ff[u].x * zz[u]);
                    Z[sidx(lane, par + 2 * (i0 - u))] = x;
                }
        }
    }
    __syncthreads();
    if (vec) {
        for (int q0 = threadIdx.x * V; q0 < total; q0 += kU * blockDim.x * V) {
            T xo[kU][V];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = q0 + u * blockDim.x * V;
#pragma unroll
                for (int w = 0; w < V; ++w) xo[u][w] = 0;
                if (oacc != T(0) && q < total) {
                    const int t = q >> 5, li = q & 31;
                    const T *src = X + gbase + li + t * gt;
#pragma unroll
                    for (int w = 0; w < V; ++w) xo[u][w] = src[w];
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = q0 + u * blockDim.x * V;
                if (q < total) {
                    const int t = q >> 5, li = q & 31;
                    const int k = t * kLines + li;
                    T v[V];
#pragma unroll
                    for (int w = 0; w < V; ++w) {
                        T val = oscale * Z[k + w];
                        if (oin != T(0)) val = fma(oin, B[k + w], val);
                        if (oacc != T(0)) val = fma(oacc, xo[u][w], val);
                        v[w] = val;
                    }
                    T *dst = X + gbase + li + t * gt;
                    if constexpr (sizeof(T) == 4)
                        *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
                    else
                        *reinterpret_cast<double2 *>(dst) = make_double2(v[0], v[1]);
                }
            }
        }
    } else {
        for (int q0 = threadIdx.x; q0 < total; q0 += kU * blockDim.x) {
            T xo[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = q0 + u * blockDim.x;
                xo[u] = 0;
                if (oacc != T(0) && q < total) {
                    int li, t;
                    qmap(q, li, t);
                    if (li < nl) xo[u] = X[gbase + li * gl + t * gt];
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = q0 + u * blockDim.x;
                if (q < total) {
                    int li, t;
                    qmap(q, li, t);
                    if (li < nl) {
                        const int k = sidx(li, t);
                        T v = oscale * Z[k];
                        if (oin != T(0)) v = fma(oin, B[k], v);
                        if (oacc != T(0)) v = fma(oacc, xo[u], v);
                        X[gbase + li * gl + t * gt] = v;
                    }
                }
            }
        }
    }
}

// The two solves along `ma` of one residual-form inner iteration (stein_res) in one
// launch, both with the set (A~ - q): with w = rho + (p - q) a1,
//   rho <- (q - p) (A~ - q)^{-1} w + w,     Z <- (q - p) (A~ - q)^{-1} a1 + zacc Z.
// Strided modes only (ma is 0 or 1); tiles [t][line]: A holds rho, then the z of the
// w chain, then the new rho; B holds a1, then the z and x of the a1 chain.  The back
// sweep recovers w_t = z_t + u_{t-2} z_{t-2} from the forward values below t (not yet
// overwritten), so no third tile is needed.  Each thread runs both dependency chains.
template <typename T>
__global__ void __launch_bounds__(kLineThreads) cube_dual_kernel(const typename V2<T>::type *__restrict__ fac, T *rho,
                                                                 const T *a1, T *Z, int n, int mode, T pq, T qp,
                                                                 T zacc)
{
    using F2 = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F2 *fs = reinterpret_cast<F2 *>(smem_raw);
    T *A = reinterpret_cast<T *>(fs + n);
    T *B = A + kLines * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) fs[t] = fac[t];
    const int nkb = (n + kLines - 1) / kLines;
    const int other = blockIdx.x / nkb, k0 = (blockIdx.x % nkb) * kLines;
    const int64_t nn = (int64_t)n * n;
    const int nl = min(kLines, n - k0);
    const int64_t gbase = ((mode == 0) ? (int64_t)other * n : (int64_t)other * nn) + k0;
    const int64_t gt = (mode == 0) ? nn : (int64_t)n;
    constexpr int V = 16 / (int)sizeof(T);
    const bool vec = nl == kLines && ((gt * (int64_t)sizeof(T)) % 16 == 0) && ((gbase * (int64_t)sizeof(T)) % 16 == 0) &&
                     (((uintptr_t)rho & 15) == 0) && (((uintptr_t)a1 & 15) == 0) && (((uintptr_t)Z & 15) == 0) &&
                     ((n * (int)sizeof(F2)) % 16 == 0);
    const int total = kLines * n;
    if (vec) {
        for (int q = threadIdx.x * V; q < total; q += blockDim.x * V) {
            const int t = q >> 5, li = q & 31;
            const int64_t g = gbase + li + t * gt;
            cp_async16(&A[t * kLines + li], rho + g);
            cp_async16(&B[t * kLines + li], a1 + g);
        }
    } else {
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            const int t = q >> 5, li = q & 31;
            if (li < nl) {
                const int64_t g = gbase + li + t * gt;
                cp_async_elem(&A[t * kLines + li], rho + g);
                cp_async_elem(&B[t * kLines + li], a1 + g);
            }
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int lane = threadIdx.x & 31, par = threadIdx.x >> 5;
    const int m = (n - par + 1) / 2;
    if (threadIdx.x < 2 * kLines && lane < nl) {
        constexpr int kC = 8;
        T z1 = 0, z2 = 0, up = 0;
        for (int i0 = 0; i0 < m; i0 += kC) {
            T r[kC], a[kC], uf[kC];
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int t = par + 2 * min(i0 + u, m - 1);
                r[u] = A[t * kLines + lane];
                a[u] = B[t * kLines + lane];
                uf[u] = fs[t].y;
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (i0 + u < m) {
                    const int k = (par + 2 * (i0 + u)) * kLines + lane;
                    z1 = fma(-up, z1, fma(pq, a[u], r[u]));
                    z2 = fma(-up, z2, a[u]);
                    A[k] = z1;
                    B[k] = z2;
                    up = uf[u];
                }
        }
        T x1 = 0, x2 = 0;
        for (int i0 = m - 1; i0 >= 0; i0 -= kC) {
            T za[kC + 1], zb[kC], ub[kC];
            F2 ff[kC];
#pragma unroll
            for (int u = 0; u <= kC; ++u) {
                const int i = max(i0 - u, 0);
                za[u] = A[(par + 2 * i) * kLines + lane];
            }
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int i = max(i0 - u, 0);
                zb[u] = B[(par + 2 * i) * kLines + lane];
                ff[u] = fs[par + 2 * i];
                ub[u] = i >= 1 ? fs[par + 2 * i - 2].y : T(0);
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (i0 - u >= 0) {
                    const int k = (par + 2 * (i0 - u)) * kLines + lane;
                    x1 = fma(-ff[u].y, x1, ff[u].x * za[u]);
                    x2 = fma(-ff[u].y, x2, ff[u].x * zb[u]);
                    const T w = (i0 - u >= 1) ? fma(ub[u], za[u + 1], za[u]) : za[u];
                    A[k] = fma(qp, x1, w);
                    B[k] = x2;
                }
        }
    }
    __syncthreads();
    // out: kU groups of V consecutive elements per thread, the old Z of all groups
    // loaded before any store (as in cube_line_kernel)
    const int vw = vec ? V : 1;
    for (int q0 = threadIdx.x * vw; q0 < total; q0 += kU * blockDim.x * vw) {
        T zo[kU][V];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int q = q0 + u * blockDim.x * vw;
#pragma unroll
            for (int w = 0; w < V; ++w) zo[u][w] = 0;
            const int t = q >> 5, li = q & 31;
            if (zacc != T(0) && q < total && (vec || li < nl)) {
                const T *src = Z + gbase + li + t * gt;
                if (vec) {
                    if constexpr (sizeof(T) == 4) {
                        const float4 v4 = *reinterpret_cast<const float4 *>(src);
                        zo[u][0] = v4.x, zo[u][1] = v4.y, zo[u][2] = v4.z, zo[u][3] = v4.w;
                    } else {
                        const double2 v2 = *reinterpret_cast<const double2 *>(src);
                        zo[u][0] = v2.x, zo[u][1] = v2.y;
                    }
                } else {
                    zo[u][0] = src[0];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int q = q0 + u * blockDim.x * vw;
            const int t = q >> 5, li = q & 31;
            if (q < total && (vec || li < nl)) {
                const int k = t * kLines + li;
                const int64_t g = gbase + li + t * gt;
                if (vec) {
                    T zr[V];
#pragma unroll
                    for (int w = 0; w < V; ++w) zr[w] = fma(qp, B[k + w], zacc * zo[u][w]);
                    if constexpr (sizeof(T) == 4) {
                        *reinterpret_cast<float4 *>(rho + g) = make_float4(A[k], A[k + 1], A[k + 2], A[k + 3]);
                        *reinterpret_cast<float4 *>(Z + g) = make_float4(zr[0], zr[1], zr[2], zr[3]);
                    } else {
                        *reinterpret_cast<double2 *>(rho + g) = make_double2(A[k], A[k + 1]);
                        *reinterpret_cast<double2 *>(Z + g) = make_double2(zr[0], zr[1]);
                    }
                } else {
                    rho[g] = A[k];
                    Z[g] = fma(qp, B[k], zacc * zo[u][0]);
                }
            }
        }
    }
}

// G = -F s_i s_j s_k (scale-in) or X = Y s_i s_j s_k (scale-out, sign = +1)
__global__ void cube_scale_kernel(const double *__restrict__ A, double *__restrict__ B, const double *__restrict__ s,
                                  int n, double sign)
{
    const int N = n * n * n;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        const int row = idx / n, k = idx - row * n, i = row / n, j = row - i * n;
        B[idx] = sign * A[idx] * s[i] * s[j] * s[k];
    }
}

// ---- FP64 defect correction ----

// A~[t, t + dt] for dt in {-2, 0, 2} (the caller keeps t + dt inside [0, n))
__device__ __forceinline__ double band_coef(const double *d, const double *e, int t, int dt)
{
    return dt == 0 ? d[t] : (dt > 0 ? e[t] : e[t - 2]);
}

__device__ __forceinline__ void block_max_bits(double local, unsigned long long *out)
{
    for (int off = 16; off > 0; off >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, off));
    __shared__ double wmax[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) wmax[w] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double bm = 0.0;
        for (int t = 0; t < (int)(blockDim.x >> 5); ++t) bm = fmax(bm, wmax[t]);
        atomicMax(out, (unsigned long long)__double_as_longlong(bm));
    }
}

// R = G - (T_01 + T_02 + T_12) Y in FP64 (Y read as zero if y_zero); *rmax = max |R|
// as a bit pattern (must start at 0; NaN and Inf are reported as +Inf).
__global__ void __launch_bounds__(256) cube_residual_kernel(const double *__restrict__ G, const double *__restrict__ Y,
                                                            const double *__restrict__ d, const double *__restrict__ e,
                                                            int n, double *__restrict__ R, bool y_zero,
                                                            unsigned long long *rmax)
{
    const int N = n * n * n;
    const int nn = n * n;
    double local = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        double r = G[idx];
        if (!y_zero) {
            const int row = idx / n, k = idx - row * n, i = row / n, j = row - i * n;
            const int idx3[3] = {i, j, k};
            const int st[3] = {nn, n, 1};
            double acc = 0.0;
            // pairs (0,1), (0,2), (1,2): offsets {0, +-2} on both modes of the pair
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
                const int ma = pr == 2 ? 1 : 0, mb = pr == 0 ? 1 : 2;
                const int ta = idx3[ma], tb = idx3[mb];
#pragma unroll
                for (int da = -2; da <= 2; da += 2) {
                    if (ta + da < 0 || ta + da >= n) continue;
                    const double ca = band_coef(d, e, ta, da);
#pragma unroll
                    for (int db = -2; db <= 2; db += 2) {
                        if (tb + db < 0 || tb + db >= n) continue;
                        acc = fma(ca * band_coef(d, e, tb, db), Y[idx + da * st[ma] + db * st[mb]], acc);
                    }
                }
            }
            r -= acc;
        }
        R[idx] = r;
        const double a = fabs(r);
        local = (a <= 1.7976931348623157e308) ? fmax(local, a) : __longlong_as_double(0x7ff0000000000000LL);
    }
    block_max_bits(local, rmax);
}

// rho = R / max|R| in FP32
__global__ void cube_to32_kernel(const double *__restrict__ R, float *__restrict__ rho, int N,
                                 const unsigned long long *__restrict__ rmax)
{
    const double inv = 1.0 / __longlong_as_double((long long)*rmax);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
        rho[idx] = (float)(R[idx] * inv);
}

// Y = (first ? 0 : Y) + max|R| delta  in FP64
__global__ void cube_update_kernel(double *__restrict__ Y, const float *__restrict__ delta, int N,
                                   const unsigned long long *__restrict__ rmax, bool first)
{
    const double sc = __longlong_as_double((long long)*rmax);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
        Y[idx] = fma(sc, (double)delta[idx], first ? 0.0 : Y[idx]);
}

int grid_for(int64_t N) { return (int)std::min<int64_t>((N + 255) / 256, 16 * (int64_t)current_sm_count()); }

}  // namespace

#define CUBE_CK(call)                                                                                    \
    do {                                                                                                 \
        cudaError_t ce_ = (call);                                                                        \
        if (ce_ != cudaSuccess) {                                                                        \
            err = std::string(#call) + ": " + cudaGetErrorString(ce_);                                   \
            return FPS_ERR_CUDA;                                                                         \
        }                                                                                                \
    } while (0)

// ===========================================================================
// CubeNested<T>
// ===========================================================================

template <typename T>
int CubeNested<T>::add_stein(double c)
{
    // A~_a Z - Z B = C with sigma(A~_a) in [-hi, -lo] and sigma(B) = sigma(-c A~_b^{-1})
    // in [c/hi, c/lo]
    Stein s;
    s.c = c;
    const double a = -hi_, b = -lo_, cl = c / hi_, d = c / lo_;
    s.J = adi_iterations(a, b, cl, d, tol_in_);
    zolotarev_shifts(a, b, cl, d, s.J, s.p, s.q);
    s.ab_off = steins_.empty() ? 0 : steins_.back().ab_off + 2 * steins_.back().J + 1;
    max_sets_ = std::max(max_sets_, 2 * s.J + 1);
    steins_.push_back(std::move(s));
    return (int)steins_.size() - 1;
}

template <typename T>
int CubeNested<T>::create(int64_t n, double tol, double tol_mid, double tol_in, bool residual, bool tight,
                          std::string &err)
{
    residual_ = residual;
    n_ = n;
    tol_ = tol;
    tol_mid_ = tol_mid;
    tol_in_ = tol_in;
    lo_ = square_eps(n);
    hi_ = 1.0;
    if (tight) square_tight_interval(n, lo_, hi_);
    // the schedule of every level, fixed for the plan: T_ab (A~ on two modes) has its
    // spectrum in [lo^2, hi^2], so sigma(H) is in [2 lo^2, 2 hi^2] and sigma(-V) in
    // [-hi^2, -lo^2]
    const double e2 = lo_ * lo_, h2 = hi_ * hi_;
    J_outer = adi_iterations(-h2, -e2, 2 * e2, 2 * h2, tol_);
    std::vector<double> pp, qq;
    zolotarev_shifts(-h2, -e2, 2 * e2, 2 * h2, J_outer, pp, qq);
    inner_per_run = 0;
    for (int j = 0; j < J_outer; ++j) {
        Outer o;
        o.p = qq[j];  // in sigma(H)'s interval [2 lo^2, 2 hi^2]
        o.q = pp[j];  // in sigma(-V)'s interval [-hi^2, -lo^2]
        o.stein_v = add_stein(o.p);
        inner_per_run += (residual_ ? 2 : 1) * steins_[o.stein_v].J;
        const double s = -o.q, lo = e2 + s / 2, hi = h2 + s / 2;
        const int Jm = adi_iterations(-hi, -lo, lo, hi, tol_mid_);
        std::vector<double> am;
        zolotarev_shifts_symmetric(lo, hi, Jm, am);
        for (int m = 0; m < Jm; ++m) {
            Middle mid;
            mid.a = am[m];
            mid.stein = add_stein(s / 2 + am[m]);
            inner_per_run += (residual_ && m + 1 < Jm ? 3 : 2) * steins_[mid.stein].J;
            o.mid.push_back(mid);
        }
        outer_.push_back(std::move(o));
    }
    std::vector<double2> hab;
    for (const Stein &s : steins_) {
        hab.push_back(make_double2(1.0, 0.0));
        for (int l = 0; l < s.J; ++l) {
            hab.push_back(make_double2(s.p[l], s.c));
            hab.push_back(make_double2(1.0, -s.q[l]));
        }
    }
    std::vector<double> d, e;
    square_bands(n, d, e);
    std::vector<T> dT(d.begin(), d.end()), eT(e.begin(), e.end());
    const size_t N = (size_t)n * n * n;
    auto alloc = [&](void **p, size_t b) -> cudaError_t {
        cudaError_t r = cudaMalloc(p, b ? b : 1);
        if (r == cudaSuccess) {
            allocs_.push_back(*p);
            bytes += (int64_t)b;
        }
        return r;
    };
    CUBE_CK(alloc((void **)&bd64_, sizeof(double) * n));
    CUBE_CK(alloc((void **)&be64_, sizeof(double) * n));
    CUBE_CK(alloc((void **)&bd_, sizeof(T) * n));
    CUBE_CK(alloc((void **)&be_, sizeof(T) * n));
    const int nwork = residual_ ? 9 : 8;
    for (int w = 0; w < nwork; ++w) CUBE_CK(alloc((void **)&work_[w], sizeof(T) * N));
    CUBE_CK(alloc(&fac_, sizeof(typename V2<T>::type) * (size_t)max_sets_ * n));
    CUBE_CK(alloc((void **)&ab_, sizeof(double2) * hab.size()));
    CUBE_CK(cudaMemcpy(bd64_, d.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CUBE_CK(cudaMemcpy(be64_, e.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CUBE_CK(cudaMemcpy(bd_, dT.data(), sizeof(T) * n, cudaMemcpyHostToDevice));
    CUBE_CK(cudaMemcpy(be_, eT.data(), sizeof(T) * n, cudaMemcpyHostToDevice));
    CUBE_CK(cudaMemcpy(ab_, hab.data(), sizeof(double2) * hab.size(), cudaMemcpyHostToDevice));
    CUBE_CK(cudaFuncSetAttribute(cube_line_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 line_smem_bytes<T>((int)n, true, 2)));
    CUBE_CK(cudaFuncSetAttribute(cube_line_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 line_smem_bytes<T>((int)n, false, 2)));
    CUBE_CK(cudaFuncSetAttribute(cube_dual_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 line_smem_bytes<T>((int)n, false, 2)));
    fac_entry_ = -1;
    slice_ = false;
    if (std::is_same<T, float>::value && residual_ && std::getenv("FPS_CUBE_SLICE") != nullptr)
        CUBE_CK(slice_setup((int)n, &slice_));
    return FPS_OK;
}

template <typename T>
void CubeNested<T>::release()
{
    for (void *p : allocs_) cudaFree(p);
    allocs_.clear();
}

template <typename T>
cudaError_t CubeNested<T>::band(const T *X, const T *R, T *Y, int mode, double alpha, double beta, double sop,
                                double sr)
{
    const int64_t N = n_ * n_ * n_;
    cube_band_kernel<T><<<grid_for(N), 256, 0, st_>>>(X, R, Y, bd_, be_, (int)n_, mode, (T)alpha, (T)beta, (T)sop,
                                                       (T)sr);
    ++launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t CubeNested<T>::axpby(const T *X, const T *Y, T *Z, double a, double b)
{
    const int64_t N = n_ * n_ * n_;
    cube_axpby_kernel<T><<<grid_for(N), 256, 0, st_>>>(X, Y, Z, (int)N, (T)a, (T)b);
    ++launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t CubeNested<T>::axpy3(const T *X, const T *Y, const T *W, T *V, double a, double b, double c)
{
    const int64_t N = n_ * n_ * n_;
    cube_axpy3_kernel<T><<<grid_for(N), 256, 0, st_>>>(X, Y, W, V, (int)N, (T)a, (T)b, (T)c);
    ++launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t CubeNested<T>::solve(int set, const T *R1, double s1, const T *R2, double s2, T *X, int mode,
                                 double oscale, double oacc, double oin, bool preband)
{
    using F2 = typename V2<T>::type;
    const F2 *fac = reinterpret_cast<const F2 *>(fac_) + (int64_t)set * n_;
    const int n = (int)n_;
    const int ntiles = (R2 != nullptr || oin != 0.0 || preband) ? 2 : 1;
    if (mode == 2) {
        const int blocks = (n * n + kLines - 1) / kLines;
        const int smem = line_smem_bytes<T>(n, true, ntiles);
        cube_line_kernel<T, true><<<blocks, kLineThreads, smem, st_>>>(fac, R1, (T)s1, R2, (T)s2, X, n, mode,
                                                                     (T)oscale, (T)oin, (T)oacc, preband, bd_, be_);
    } else {
        const int nkb = (n + kLines - 1) / kLines;
        const int smem = line_smem_bytes<T>(n, false, ntiles);
        cube_line_kernel<T, false><<<n * nkb, kLineThreads, smem, st_>>>(fac, R1, (T)s1, R2, (T)s2, X, n, mode,
                                                                       (T)oscale, (T)oin, (T)oacc, preband, bd_,
                                                                       be_);
    }
    ++launches;
    return cudaGetLastError();
}

template <typename T>
int CubeNested<T>::load_factors(int entry, std::string &err)
{
    if (fac_entry_ == entry) return FPS_OK;
    const Stein &S = steins_[entry];
    const int nsets = 2 * S.J + 1;
    // factor sets: 0 = A~; 1 + 2l = c + p_l A~; 2 + 2l = A~ - q_l
    cube_factor_kernel<T><<<(2 * nsets + 127) / 128, 128, 0, st_>>>(bd64_, be64_, (int)n_, ab_ + S.ab_off, nsets,
                                                                     reinterpret_cast<typename V2<T>::type *>(fac_));
    ++launches;
    CUBE_CK(cudaGetLastError());
    fac_entry_ = entry;
    return FPS_OK;
}

// Z = (T_ab + c)^{-1} R, the inner level in the paper's form (entry = schedule
// index).  Uses work_[0], work_[1].
template <typename T>
int CubeNested<T>::stein(int ma, int mb, int entry, const T *R, T *Z, std::string &err)
{
    int st = load_factors(entry, err);
    if (st != FPS_OK) return st;
    const Stein &S = steins_[entry];
    T *W1 = work_[0], *W2 = work_[1];
    const double c = S.c;
    for (int l = 0; l < S.J; ++l) {
        const T *U = R;
        if (l > 0) {
            CUBE_CK(band(Z, nullptr, W1, mb, 1.0, 0.0, 1.0, 0.0));                // Z A~_b
            CUBE_CK(band(W1, R, W2, ma, 1.0, -S.p[l], -1.0, 1.0));                // R - (A~_a - p) ( . )
            U = W2;
        }
        CUBE_CK(solve(1 + 2 * l, U, 1.0, nullptr, 0.0, W1, mb, 1.0, 0.0, 0.0, false));  // Z_h = ( . ) (c + p A~_b)^{-1}
        CUBE_CK(solve(0, R, 1.0, W1, -c, W2, mb, 1.0, 0.0, 0.0, false));                 // (R - c Z_h) A~_b^{-1}
        CUBE_CK(solve(2 + 2 * l, W2, 1.0, W1, -S.q[l], Z, ma, 1.0, 0.0, 0.0, false));    // (A~_a - q)^{-1} ( . - q Z_h)
    }
    return FPS_OK;
}

// Y = (T_01 + T_02 + s)^{-1} R with s = -o.q, the middle level in the paper's
// form.  Uses work_[2..4].
template <typename T>
int CubeNested<T>::hsolve(const Outer &o, const T *R, T *Y, std::string &err)
{
    const double s = -o.q;
    T *Wh = work_[2], *T1 = work_[3], *T2 = work_[4];
    for (size_t m = 0; m < o.mid.size(); ++m) {
        const double a = o.mid[m].a;
        const T *U = R;  // R - (T_01 + s/2 - a) Y, with Y = 0 at m = 0
        if (m > 0) {
            CUBE_CK(band(Y, nullptr, T1, 0, 1.0, 0.0, 1.0, 0.0));
            CUBE_CK(band(T1, R, T2, 1, 1.0, 0.0, -1.0, 1.0));
            CUBE_CK(axpby(T2, Y, T1, 1.0, -(s / 2 - a)));
            U = T1;
        }
        int st = stein(0, 2, o.mid[m].stein, U, Wh, err);
        if (st != FPS_OK) return st;
        // T1 = R - (T_02 + s/2 - a) Wh
        CUBE_CK(band(Wh, nullptr, T1, 0, 1.0, 0.0, 1.0, 0.0));
        CUBE_CK(band(T1, R, T2, 2, 1.0, 0.0, -1.0, 1.0));
        CUBE_CK(axpby(T2, Wh, T1, 1.0, -(s / 2 - a)));
        st = stein(0, 1, o.mid[m].stein, T1, Y, err);
        if (st != FPS_OK) return st;
    }
    return FPS_OK;
}

// The inner level with its residual carried.  The slice equation is the Sylvester
// equation A Z - Z B = C with A = A~_a, B = -c A~_b^{-1}, C = R A~_b^{-1}; with
// rho = C - A Z + Z B the two half-steps of Algorithm 2 become
//   rho+ = (A - q)^{-1} (A - p) rho (B - p)^{-1} (B - q),
//   Z+   = Z + (q - p) (A - q)^{-1} rho (B - p)^{-1},
// and rho (B - p)^{-1} = -rho A~_b (c + p A~_b)^{-1}.  Per iteration two launches:
// a1 = rho (B - p)^{-1} along b (the product with A~_b folded in), then one
// cube_dual_kernel along a for rho+ = c1 + (q - p)(A - q)^{-1} c1 with
// c1 = rho + (p - q) a1 (in place) and Z += (q - p)(A - q)^{-1} a1 (the last
// iteration needs only the Z solve).  Solves Z = (T_ab + c)^{-1} (r1 R1 + r2 R2), or
// adds it to Z when accumulate.  Uses work_[0], work_[1].
template <typename T>
int CubeNested<T>::stein_res(int ma, int mb, int entry, const T *R1, double r1, const T *R2, double r2, T *Z,
                             bool accumulate, std::string &err)
{
    int st = load_factors(entry, err);
    if (st != FPS_OK) return st;
    const Stein &S = steins_[entry];
    if constexpr (std::is_same<T, float>::value) {
        if (slice_) {  // all J iterations with every slice on chip (cube_slice.cu)
            SliceArgs sa;
            sa.fac = reinterpret_cast<const float2 *>(fac_);
            sa.ab = ab_ + S.ab_off;
            sa.J = S.J;
            sa.R1 = R1;
            sa.R2 = R2;
            sa.r1 = (float)r1;
            sa.r2 = (float)r2;
            sa.Z = Z;
            sa.accumulate = accumulate;
            sa.d = bd_;
            sa.e = be_;
            sa.n = (int)n_;
            sa.ma = ma;
            sa.mb = mb;
            CUBE_CK(launch_stein_slice(sa, st_));
            ++launches;
            return FPS_OK;
        }
    }
    T *rho = work_[0], *a1 = work_[1];
    CUBE_CK(solve(0, R1, r1, R2, r2, rho, mb, 1.0, 0.0, 0.0, false));                  // rho = R A~_b^{-1}
    for (int l = 0; l < S.J; ++l) {
        const double p = S.p[l], q = S.q[l];
        if (l == 0) CUBE_CK(solve(1, R1, -r1, R2, -r2, a1, mb, 1.0, 0.0, 0.0, false));    // rho A~_b = R
        else CUBE_CK(solve(1 + 2 * l, rho, -1.0, nullptr, 0.0, a1, mb, 1.0, 0.0, 0.0, true));
        const double zacc = (l > 0 || accumulate) ? 1.0 : 0.0;
        if (l + 1 < S.J) {  // both solves along ma in one launch
            using F2 = typename V2<T>::type;
            const int n = (int)n_;
            const int nkb = (n + kLines - 1) / kLines;
            cube_dual_kernel<T><<<n * nkb, kLineThreads, line_smem_bytes<T>(n, false, 2), st_>>>(
                reinterpret_cast<const F2 *>(fac_) + (int64_t)(2 + 2 * l) * n, rho, a1, Z, n, ma, (T)(p - q),
                (T)(q - p), (T)zacc);
            ++launches;
            CUBE_CK(cudaGetLastError());
        } else {
            CUBE_CK(solve(2 + 2 * l, a1, 1.0, nullptr, 0.0, Z, ma, q - p, zacc, 0.0, false));
        }
    }
    return FPS_OK;
}

// The middle level with its residual carried: for A' W + B' W = R (A' = T_01 + s/2,
// B' = T_02 + s/2) and shifts +-a,
//   rho+ = [I - 2a (A' + a)^{-1}] [I - 2a (B' + a)^{-1}] rho,
//   W+   = W + (A' + a)^{-1} 2a (B' + a)^{-1} rho,
// three slice Stein solves per iteration (two in the last).  Uses work_[3..5].
template <typename T>
int CubeNested<T>::hsolve_res(const Outer &o, const T *R, T *W, std::string &err)
{
    T *rho = work_[3], *v = work_[4], *g = work_[5];
    const size_t J = o.mid.size();
    for (size_t m = 0; m < J; ++m) {
        const double a = o.mid[m].a;
        const int entry = o.mid[m].stein;
        const T *r = (m == 0) ? R : rho;
        int st = stein_res(0, 2, entry, r, 1.0, nullptr, 0.0, v, false, err);        // v = (B' + a)^{-1} rho
        if (st != FPS_OK) return st;
        if (m + 1 < J) {
            st = stein_res(0, 1, entry, r, 1.0, v, -2.0 * a, g, false, err);         // g = (A' + a)^{-1} (rho - 2a v)
            if (st != FPS_OK) return st;
            CUBE_CK(axpy3(r, v, g, rho, 1.0, -2.0 * a, -2.0 * a));                  // rho+ = rho - 2a v - 2a g
        }
        st = stein_res(0, 1, entry, v, 2.0 * a, nullptr, 0.0, W, m > 0, err);        // W += (A' + a)^{-1} 2a v
        if (st != FPS_OK) return st;
    }
    return FPS_OK;
}

// The outer level with the residual rho = G - (H + V) Y carried instead of Y's
// right-hand sides.  The two half-steps of (5.3)-(5.4) are Y_h = Y + (V + p)^{-1} rho
// and Y+ = Y_h + (H - q)^{-1} rho_h, so that, the operators commuting,
//   rho+ = [I + (q - p)(V + p)^{-1}] [I + (q - p)(H - q)^{-1}] rho,
//   Y+   = Y + (V + p)^{-1} (p - q) (H - q)^{-1} rho:
// only residuals are solved with and no product with H or V of a growing iterate
// is formed, which keeps FP32 rounding relative to the residual (the paper's form
// loses it to cancellation at small shifts).  Uses work_[6..8].
template <typename T>
int CubeNested<T>::run_residual(const T *G, T *Y, std::string &err)
{
    T *rho = work_[6], *w = work_[7], *u = work_[8];
    for (int j = 0; j < J_outer; ++j) {
        const Outer &o = outer_[j];
        const T *r = (j == 0) ? G : rho;
        int s = hsolve_res(o, r, w, err);                                         // w = (H - q)^{-1} rho
        if (s != FPS_OK) return s;
        s = stein_res(1, 2, o.stein_v, r, 1.0, w, o.q - o.p, u, false, err);      // u = (V + p)^{-1} c,
        if (s != FPS_OK) return s;                                                //   c = rho + (q - p) w
        CUBE_CK(axpy3(r, w, u, rho, 1.0, o.q - o.p, o.q - o.p));                  // rho+ = c + (q - p) u
        // the scalar p - q enters with the right-hand side: w ~ rho / eps^2 and
        // (V + p)^{-1} w ~ rho / eps^4 would leave the FP32 range for n >~ 100
        s = stein_res(1, 2, o.stein_v, w, o.p - o.q, nullptr, 0.0, Y, j > 0, err); // Y += (V + p)^{-1} (p - q) w
        if (s != FPS_OK) return s;
    }
    return FPS_OK;
}

template <typename T>
int CubeNested<T>::run(const T *G, T *Y, cudaStream_t st, std::string &err)
{
    st_ = st;
    launches = 0;
    if (residual_) return run_residual(G, Y, err);
    T *Yh = work_[5], *T1 = work_[6], *T2 = work_[7];
    for (int j = 0; j < J_outer; ++j) {
        const Outer &o = outer_[j];
        const T *U = G;  // G - (H - p) Y, with Y = 0 at j = 0
        if (j > 0) {
            CUBE_CK(band(Y, nullptr, T2, 0, 1.0, 0.0, 1.0, 0.0));      // A~_0 Y
            CUBE_CK(band(T2, G, T1, 1, 1.0, 0.0, -1.0, 1.0));          // G - T_01 Y
            CUBE_CK(band(T2, T1, T1, 2, 1.0, 0.0, -1.0, 1.0));         // ... - T_02 Y (element-wise in place)
            CUBE_CK(axpby(T1, Y, T1, 1.0, o.p));
            U = T1;
        }
        int s = stein(1, 2, o.stein_v, U, Yh, err);
        if (s != FPS_OK) return s;
        // T1 = G - (V + q) Y_h = G - T_12 Y_h - q Y_h
        CUBE_CK(band(Yh, nullptr, T2, 1, 1.0, 0.0, 1.0, 0.0));
        CUBE_CK(band(T2, G, T1, 2, 1.0, 0.0, -1.0, 1.0));
        CUBE_CK(axpby(T1, Yh, T1, 1.0, -o.q));
        s = hsolve(o, T1, Y, err);
        if (s != FPS_OK) return s;
    }
    return FPS_OK;
}

template class CubeNested<double>;
template class CubeNested<float>;

// ===========================================================================
// CubeEngine
// ===========================================================================

// Outer tolerance t of the FP32 rounds.  A round reduces max|R| by about t/2
// (measured 0.52 t at n = 256 with the middle and inner levels at 1e-6 and 1e-7), so
// reaching `tol` takes R(t) = ceil(log(tol) / log(0.55 t)) rounds of J_outer(t) outer
// iterations each; the candidate with the least R(t) J_outer(t) wins.  A round that
// falls short only adds a round: the stopping test is the measured residual.
double refinement_outer_tol(int64_t n, double tol)
{
    double lo = square_eps(n), hi = 1.0;
    square_tight_interval(n, lo, hi);
    const double e2 = lo * lo, h2 = hi * hi;
    double best = CubeEngine::kRefTolOuter[0], best_cost = 1e300;
    for (double t : CubeEngine::kRefTolOuter) {
        const int R = std::max(1, (int)std::ceil(std::log(tol) / std::log(0.55 * t) - 1e-9));
        const double cost = (double)R * adi_iterations(-h2, -e2, 2 * e2, 2 * h2, t);
        if (cost < best_cost) {
            best_cost = cost;
            best = t;
        }
    }
    return best;
}

int CubeEngine::create(int64_t n, double tol, int precision, std::string &err)
{
    n_ = n;
    tol_ = tol;
    precision_ = precision;
    if (const char *mr = std::getenv("FPS_MAX_REFINE_ROUNDS")) {  // cap on refinement rounds (>= 1)
        const int v = std::atoi(mr);
        if (v >= 1) max_rounds = v;
    }
    std::vector<double> d, e, s;
    square_bands(n, d, e);
    inv_sqrt_E(n, s);
    const size_t N = (size_t)n * n * n;
    auto alloc = [&](void **p, size_t b) -> cudaError_t {
        cudaError_t r = cudaMalloc(p, b ? b : 1);
        if (r == cudaSuccess) {
            allocs_.push_back(*p);
            bytes += (int64_t)b;
        }
        return r;
    };
    CUBE_CK(alloc((void **)&bd_, sizeof(double) * n));
    CUBE_CK(alloc((void **)&be_, sizeof(double) * n));
    CUBE_CK(alloc((void **)&bs_, sizeof(double) * n));
    CUBE_CK(alloc((void **)&G_, sizeof(double) * N));
    CUBE_CK(alloc((void **)&Y_, sizeof(double) * N));
    CUBE_CK(cudaMemcpy(bd_, d.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CUBE_CK(cudaMemcpy(be_, e.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CUBE_CK(cudaMemcpy(bs_, s.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    int st;
    if (precision == FPS_FP64) {
        n64_ = new CubeNested<double>();
        st = n64_->create(n, tol, 1e-15, 1e-15, false, false, err);
        if (st != FPS_OK) return st;
        J_outer = n64_->J_outer;
        bytes += n64_->bytes;
    } else {
        CUBE_CK(alloc((void **)&R_, sizeof(double) * N));
        CUBE_CK(alloc((void **)&rho_, sizeof(float) * N));
        CUBE_CK(alloc((void **)&delta_, sizeof(float) * N));
        CUBE_CK(alloc((void **)&d_max_, sizeof(unsigned long long)));
        CUBE_CK(cudaMallocHost((void **)&h_max_, sizeof(unsigned long long)));
        n32_ = new CubeNested<float>();
        ref_tol_outer = refinement_outer_tol(n, tol);
        st = n32_->create(n, ref_tol_outer, kRefTolMid, kRefTolIn, true, true, err);
        if (st != FPS_OK) return st;
        J_outer = J_outer_inner = n32_->J_outer;
        bytes += n32_->bytes;
    }
    return FPS_OK;
}

void CubeEngine::release()
{
    if (n64_) {
        n64_->release();
        delete n64_;
        n64_ = nullptr;
    }
    if (n32_) {
        n32_->release();
        delete n32_;
        n32_ = nullptr;
    }
    for (void *p : allocs_) cudaFree(p);
    allocs_.clear();
    if (h_max_) cudaFreeHost(h_max_);
    h_max_ = nullptr;
}

int CubeEngine::solve_cube(const double *F, double *X, cudaStream_t st, std::string &err)
{
    inner_iters = 0;
    launches_last = 0;
    rounds_last = 0;
    resid_last = 0.0;
    const int64_t N = n_ * n_ * n_;
    cube_scale_kernel<<<grid_for(N), 256, 0, st>>>(F, G_, bs_, (int)n_, -1.0);
    ++launches_last;
    CUBE_CK(cudaGetLastError());
    if (precision_ == FPS_FP64) {
        const int s = n64_->run(G_, Y_, st, err);
        launches_last += n64_->launches;
        if (s != FPS_OK) return s;
        inner_iters = n64_->inner_per_run;
    } else {
        double gmax = 0.0;
        int status = FPS_ERR_NOT_CONVERGED;
        for (int r = 0; r <= max_rounds; ++r) {
            TraceRange tr("fps cube refinement round");
            CUBE_CK(cudaMemsetAsync(d_max_, 0, sizeof(unsigned long long), st));
            cube_residual_kernel<<<grid_for(N), 256, 0, st>>>(G_, Y_, bd_, be_, (int)n_, R_, r == 0, d_max_);
            ++launches_last;
            CUBE_CK(cudaGetLastError());
            CUBE_CK(cudaMemcpyAsync(h_max_, d_max_, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            CUBE_CK(cudaStreamSynchronize(st));
            const unsigned long long bits = *h_max_;
            double rmax;
            std::memcpy(&rmax, &bits, sizeof(double));
            if (!std::isfinite(rmax)) {
                err = "non-finite right-hand side or residual";
                return FPS_ERR_NONFINITE;
            }
            if (r == 0) {
                gmax = rmax;
                if (gmax == 0.0) {
                    CUBE_CK(cudaMemsetAsync(Y_, 0, sizeof(double) * N, st));
                    status = FPS_OK;
                    break;
                }
            }
            resid_last = rmax / gmax;
            if (r > 0 && resid_last <= tol_) {
                status = FPS_OK;
                break;
            }
            if (r == max_rounds) break;
            cube_to32_kernel<<<grid_for(N), 256, 0, st>>>(R_, rho_, (int)N, d_max_);
            ++launches_last;
            CUBE_CK(cudaGetLastError());
            const int s = n32_->run(rho_, delta_, st, err);
            launches_last += n32_->launches;
            if (s != FPS_OK) return s;
            cube_update_kernel<<<grid_for(N), 256, 0, st>>>(Y_, delta_, (int)N, d_max_, r == 0);
            ++launches_last;
            CUBE_CK(cudaGetLastError());
            inner_iters += n32_->inner_per_run;
            rounds_last = r + 1;
        }
        if (status != FPS_OK) {
            cube_scale_kernel<<<grid_for(N), 256, 0, st>>>(Y_, X, bs_, (int)n_, 1.0);
            ++launches_last;
            err = "refinement did not reach the tolerance";
            return status;
        }
    }
    cube_scale_kernel<<<grid_for(N), 256, 0, st>>>(Y_, X, bs_, (int)n_, 1.0);
    ++launches_last;
    CUBE_CK(cudaGetLastError());
    return FPS_OK;
}

}  // namespace fps
