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
// once.  Modes 0 and 1 are solved with one thread per (line, parity), coalesced
// across the contiguous index; mode 2 (contiguous lines) goes through a
// shared-memory tile of 32 lines.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/fps.h"
#include "cube.h"
#include "host_math.h"

namespace fps {

namespace {

constexpr int kLines = 32;  // lines per CTA of the contiguous-mode solve

__device__ __forceinline__ int64_t mode_stride(int n, int mode)
{
    return mode == 0 ? (int64_t)n * n : (mode == 1 ? (int64_t)n : 1);
}

// Y = sop * ((alpha A~ + beta) X along `mode`) + sr * R   (R may be null)
__global__ void cube_band_kernel(const double *__restrict__ X, const double *__restrict__ R, double *__restrict__ Y,
                                 const double *__restrict__ d, const double *__restrict__ e, int n, int mode,
                                 double alpha, double beta, double sop, double sr)
{
    const int64_t N = (int64_t)n * n * n;
    const int64_t st = mode_stride(n, mode);
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)((idx / st) % n);
        double v = (alpha * d[t] + beta) * X[idx];
        if (t >= 2) v = fma(alpha * e[t - 2], X[idx - 2 * st], v);
        if (t + 2 < n) v = fma(alpha * e[t], X[idx + 2 * st], v);
        v *= sop;
        if (R) v = fma(sr, R[idx], v);
        Y[idx] = v;
    }
}

// Z = a X + b Y
__global__ void cube_axpby_kernel(const double *__restrict__ X, const double *__restrict__ Y, double *__restrict__ Z,
                                  int64_t N, double a, double b)
{
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x)
        Z[idx] = fma(a, X[idx], b * Y[idx]);
}

// Thomas factors of (alpha A~ + beta I) for a list of (alpha, beta) pairs: one
// thread per (set, parity); fac[set * n + t] = {1/den_t, alpha e_t / den_t}.
__global__ void cube_factor_kernel(const double *__restrict__ d, const double *__restrict__ e, int n,
                                   const double2 *__restrict__ ab, int nsets, double2 *__restrict__ fac)
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
        fac[(int64_t)set * n + t] = make_double2(ip, u);
        u_prev = u;
    }
}

// X = (alpha A~ + beta)^{-1} (s1 R1 + s2 R2) along mode 0 or 1; X may alias R1/R2
// only element-wise (each thread reads an element before it writes it).
__global__ void cube_solve_strided_kernel(const double2 *__restrict__ fac, const double *R1, double s1,
                                          const double *R2, double s2, double *X, int n, int mode)
{
    const int64_t nn = (int64_t)n * n;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 2 * nn) return;
    const int par = (int)(tid / nn);
    const int64_t line = tid - par * nn;
    const int64_t st = (mode == 0) ? nn : (int64_t)n;
    const int64_t o = (mode == 0) ? line : (line / n) * nn + (line % n);
    double z = 0.0, u_prev = 0.0;
    for (int t = par; t < n; t += 2) {
        const int64_t at = o + (int64_t)t * st;
        double r = s1 * R1[at];
        if (R2) r = fma(s2, R2[at], r);
        z = fma(-u_prev, z, r);
        X[at] = z;
        u_prev = fac[t].y;
    }
    double x = 0.0;
    const int tlast = par + 2 * ((n - 1 - par) / 2);
    for (int t = tlast; t >= 0; t -= 2) {
        const int64_t at = o + (int64_t)t * st;
        const double2 f = fac[t];
        x = fma(-f.y, x, f.x * X[at]);
        X[at] = x;
    }
}

// Same along mode 2 (contiguous lines) through a shared-memory tile of kLines lines.
__global__ void cube_solve_contig_kernel(const double2 *__restrict__ fac, const double *R1, double s1,
                                         const double *R2, double s2, double *X, int n)
{
    extern __shared__ double tile[];  // kLines x (n + 1)
    const int64_t nlines = (int64_t)n * n;
    const int64_t L0 = (int64_t)blockIdx.x * kLines;
    const int pitch = n + 1;
    const int64_t base = L0 * n;
    const int64_t count = ((nlines - L0 < kLines) ? (nlines - L0) : (int64_t)kLines) * n;
    for (int64_t idx = threadIdx.x; idx < count; idx += blockDim.x) {
        double r = s1 * R1[base + idx];
        if (R2) r = fma(s2, R2[base + idx], r);
        tile[(idx / n) * pitch + (idx % n)] = r;
    }
    __syncthreads();
    const int lane_line = threadIdx.x >> 1, par = threadIdx.x & 1;
    if (lane_line < kLines && L0 + lane_line < nlines) {
        double *row = tile + lane_line * pitch;
        double z = 0.0, u_prev = 0.0;
        for (int t = par; t < n; t += 2) {
            z = fma(-u_prev, z, row[t]);
            row[t] = z;
            u_prev = fac[t].y;
        }
        double x = 0.0;
        const int tlast = par + 2 * ((n - 1 - par) / 2);
        for (int t = tlast; t >= 0; t -= 2) {
            const double2 f = fac[t];
            x = fma(-f.y, x, f.x * row[t]);
            row[t] = x;
        }
    }
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < count; idx += blockDim.x) X[base + idx] = tile[(idx / n) * pitch + (idx % n)];
}

// G = -F s_i s_j s_k (scale-in) or X = Y s_i s_j s_k (scale-out, sign = +1)
__global__ void cube_scale_kernel(const double *__restrict__ A, double *__restrict__ B, const double *__restrict__ s,
                                  int n, double sign)
{
    const int64_t N = (int64_t)n * n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx % n), j = (int)((idx / n) % n), i = (int)(idx / ((int64_t)n * n));
        B[idx] = sign * A[idx] * s[i] * s[j] * s[k];
    }
}

}  // namespace

#define CUBE_CK(call)                                                                                    \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                                    \
            return FPS_ERR_CUDA;                                                                         \
        }                                                                                                \
    } while (0)

int CubeEngine::create(int64_t n, double tol, double tol_mid, double tol_in, std::string &err)
{
    n_ = n;
    tol_ = tol;
    tol_mid_ = tol_mid;
    tol_in_ = tol_in;
    eps_ = square_eps(n);
    std::vector<double> d, e, s;
    square_bands(n, d, e);
    inv_sqrt_E(n, s);
    const size_t N = (size_t)n * n * n;
    auto alloc = [&](double **p, size_t cnt) -> cudaError_t {
        cudaError_t r = cudaMalloc((void **)p, sizeof(double) * (cnt ? cnt : 1));
        if (r == cudaSuccess) {
            allocs_.push_back(*p);
            bytes += (int64_t)(sizeof(double) * cnt);
        }
        return r;
    };
    CUBE_CK(alloc(&bd_, n));
    CUBE_CK(alloc(&be_, n));
    CUBE_CK(alloc(&bs_, n));
    for (double *&w : work_) CUBE_CK(alloc(&w, N));
    // factor sets: the constant A~ and two per inner iteration
    max_sets_ = 2 * 512 + 1;
    CUBE_CK(cudaMalloc((void **)&fac_, sizeof(double2) * (size_t)max_sets_ * n));
    CUBE_CK(cudaMalloc((void **)&ab_, sizeof(double2) * (size_t)max_sets_));
    CUBE_CK(cudaMallocHost((void **)&h_ab_, sizeof(double2) * (size_t)max_sets_));
    bytes += (int64_t)(sizeof(double2) * (size_t)max_sets_ * (n + 1));
    CUBE_CK(cudaMemcpy(bd_, d.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CUBE_CK(cudaMemcpy(be_, e.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CUBE_CK(cudaMemcpy(bs_, s.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    const int smem = kLines * (int)(n + 1) * (int)sizeof(double);
    CUBE_CK(cudaFuncSetAttribute(cube_solve_contig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const double e2 = eps_ * eps_;
    J_outer = adi_iterations(-1.0, -e2, 2 * e2, 2.0, tol_);
    return FPS_OK;
}

void CubeEngine::release()
{
    for (double *p : allocs_) cudaFree(p);
    allocs_.clear();
    if (fac_) cudaFree(fac_);
    if (ab_) cudaFree(ab_);
    if (h_ab_) cudaFreeHost(h_ab_);
    fac_ = nullptr;
    ab_ = nullptr;
    h_ab_ = nullptr;
}

// ---- launch helpers (all asynchronous on st_) ----
cudaError_t CubeEngine::band(const double *X, const double *R, double *Y, int mode, double alpha, double beta,
                             double sop, double sr)
{
    const int64_t N = n_ * n_ * n_;
    int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 16);
    cube_band_kernel<<<blocks, 256, 0, st_>>>(X, R, Y, bd_, be_, (int)n_, mode, alpha, beta, sop, sr);
    ++launches_last;
    return cudaGetLastError();
}

cudaError_t CubeEngine::axpby(const double *X, const double *Y, double *Z, double a, double b)
{
    const int64_t N = n_ * n_ * n_;
    int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 16);
    cube_axpby_kernel<<<blocks, 256, 0, st_>>>(X, Y, Z, N, a, b);
    ++launches_last;
    return cudaGetLastError();
}

cudaError_t CubeEngine::solve(int set, const double *R1, double s1, const double *R2, double s2, double *X, int mode)
{
    const double2 *fac = fac_ + (int64_t)set * n_;
    if (mode == 2) {
        const int64_t nlines = n_ * n_;
        const int blocks = (int)((nlines + kLines - 1) / kLines);
        const int smem = kLines * (int)(n_ + 1) * (int)sizeof(double);
        cube_solve_contig_kernel<<<blocks, 2 * kLines, smem, st_>>>(fac, R1, s1, R2, s2, X, (int)n_);
    } else {
        const int64_t threads = 2 * n_ * n_;
        cube_solve_strided_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st_>>>(fac, R1, s1, R2, s2, X, (int)n_,
                                                                                       mode);
    }
    ++launches_last;
    return cudaGetLastError();
}

// Z = (T_ab + c)^{-1} R, the inner level.  Uses work_[6], work_[7].
int CubeEngine::stein(int ma, int mb, double c, const double *R, double *Z, std::string &err)
{
    const double a = -1.0, b = -eps_, cc = c, d = c / eps_;
    const int J = adi_iterations(a, b, cc, d, tol_in_);
    if (2 * J + 1 > max_sets_) {
        err = "inner iteration count exceeds the factor table";
        return FPS_ERR_UNSUPPORTED;
    }
    std::vector<double> p, q;
    zolotarev_shifts(a, b, cc, d, J, p, q);
    // factor sets: 0 = A~ (alpha 1, beta 0); 1 + 2l = c + p_l A~; 2 + 2l = A~ - q_l
    CUBE_CK(cudaStreamSynchronize(st_));  // the pinned staging of the previous call must be consumed
    h_ab_[0] = make_double2(1.0, 0.0);
    for (int l = 0; l < J; ++l) {
        h_ab_[1 + 2 * l] = make_double2(p[l], c);
        h_ab_[2 + 2 * l] = make_double2(1.0, -q[l]);
    }
    const int nsets = 2 * J + 1;
    CUBE_CK(cudaMemcpyAsync(ab_, h_ab_, sizeof(double2) * nsets, cudaMemcpyHostToDevice, st_));
    cube_factor_kernel<<<(2 * nsets + 127) / 128, 128, 0, st_>>>(bd_, be_, (int)n_, ab_, nsets, fac_);
    ++launches_last;
    CUBE_CK(cudaGetLastError());
    double *W1 = work_[6], *W2 = work_[7];
    for (int l = 0; l < J; ++l) {
        const double *U = R;
        if (l > 0) {
            CUBE_CK(band(Z, nullptr, W1, mb, 1.0, 0.0, 1.0, 0.0));         // Z A~_b
            CUBE_CK(band(W1, R, W2, ma, 1.0, -p[l], -1.0, 1.0));           // R - (A~_a - p) ( . )
            U = W2;
        }
        CUBE_CK(solve(1 + 2 * l, U, 1.0, nullptr, 0.0, W1, mb));           // Z_h = ( . ) (c + p A~_b)^{-1}
        CUBE_CK(solve(0, R, 1.0, W1, -c, W2, mb));                          // (R - c Z_h) A~_b^{-1}
        CUBE_CK(solve(2 + 2 * l, W2, 1.0, W1, -q[l], Z, ma));               // (A~_a - q)^{-1} ( . - q Z_h)
    }
    inner_iters += J;
    return FPS_OK;
}

// Y = (T_01 + T_02 + s)^{-1} R, the middle level.  Uses work_[3..5].
int CubeEngine::hsolve(double s, const double *R, double *Y, std::string &err)
{
    const double lo = eps_ * eps_ + s / 2, hi = 1.0 + s / 2;
    const int J = adi_iterations(-hi, -lo, lo, hi, tol_mid_);
    std::vector<double> am;
    zolotarev_shifts_symmetric(lo, hi, J, am);
    double *Wh = work_[3], *T1 = work_[4], *T2 = work_[5];
    CUBE_CK(cudaMemsetAsync(Y, 0, sizeof(double) * n_ * n_ * n_, st_));
    for (int m = 0; m < J; ++m) {
        const double a = am[m];
        // T1 = R - (T_01 + s/2 - a) Y
        CUBE_CK(band(Y, nullptr, T1, 0, 1.0, 0.0, 1.0, 0.0));
        CUBE_CK(band(T1, R, T2, 1, 1.0, 0.0, -1.0, 1.0));
        CUBE_CK(axpby(T2, Y, T1, 1.0, -(s / 2 - a)));
        int st = stein(0, 2, s / 2 + a, T1, Wh, err);
        if (st != FPS_OK) return st;
        // T1 = R - (T_02 + s/2 - a) Wh
        CUBE_CK(band(Wh, nullptr, T1, 0, 1.0, 0.0, 1.0, 0.0));
        CUBE_CK(band(T1, R, T2, 2, 1.0, 0.0, -1.0, 1.0));
        CUBE_CK(axpby(T2, Wh, T1, 1.0, -(s / 2 - a)));
        st = stein(0, 1, s / 2 + a, T1, Y, err);
        if (st != FPS_OK) return st;
    }
    return FPS_OK;
}

int CubeEngine::solve_cube(const double *F, double *X, cudaStream_t st, std::string &err)
{
    st_ = st;
    inner_iters = 0;
    launches_last = 0;
    const int64_t N = n_ * n_ * n_;
    double *G = work_[0], *Y = work_[1], *Yh = work_[2], *T1 = work_[8], *T2 = work_[9];
    {
        int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 16);
        cube_scale_kernel<<<blocks, 256, 0, st_>>>(F, G, bs_, (int)n_, -1.0);
        ++launches_last;
        CUBE_CK(cudaGetLastError());
    }
    const double e2 = eps_ * eps_;
    std::vector<double> pp, qq;
    zolotarev_shifts(-1.0, -e2, 2 * e2, 2.0, J_outer, pp, qq);
    CUBE_CK(cudaMemsetAsync(Y, 0, sizeof(double) * N, st_));
    for (int j = 0; j < J_outer; ++j) {
        const double p = qq[j], q = pp[j];  // p in sigma(H)'s interval, q in sigma(-V)'s
        // T1 = G - (H - p) Y = G - T_01 Y - T_02 Y + p Y
        CUBE_CK(band(Y, nullptr, T2, 0, 1.0, 0.0, 1.0, 0.0));      // A~_0 Y
        CUBE_CK(band(T2, G, T1, 1, 1.0, 0.0, -1.0, 1.0));          // G - T_01 Y
        CUBE_CK(band(T2, T1, T1, 2, 1.0, 0.0, -1.0, 1.0));         // ... - T_02 Y  (T1 read before written, element-wise)
        CUBE_CK(axpby(T1, Y, T1, 1.0, p));
        int s = stein(1, 2, p, T1, Yh, err);
        if (s != FPS_OK) return s;
        // T1 = G - (V + q) Y_h = G - T_12 Y_h - q Y_h
        CUBE_CK(band(Yh, nullptr, T2, 1, 1.0, 0.0, 1.0, 0.0));
        CUBE_CK(band(T2, G, T1, 2, 1.0, 0.0, -1.0, 1.0));
        CUBE_CK(axpby(T1, Yh, T1, 1.0, -q));
        s = hsolve(-q, T1, Y, err);
        if (s != FPS_OK) return s;
    }
    {
        int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 16);
        cube_scale_kernel<<<blocks, 256, 0, st_>>>(Y, X, bs_, (int)n_, 1.0);
        ++launches_last;
        CUBE_CK(cudaGetLastError());
    }
    return FPS_OK;
}

}  // namespace fps
