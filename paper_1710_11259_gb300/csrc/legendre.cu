// Legendre coefficients in and out of the square solve (Sec. 3.4, Table 3.1 steps
// 1 and 4), as two banded 2D maps.  With C~_k = s_k C^(3/2)_k, s_k =
// sqrt((k + 3/2)/((k+1)(k+2))), and the identities
//   (2k+1) P_k = C^(3/2)_k - C^(3/2)_{k-2},
//   (1 - x^2) C^(3/2)_j = (j+1)(j+2)/(2j+3) (P_j - P_{j+2}),
// the input map is F = B G B^T with B[j][j] = 1/((2j+1) s_j), B[j][j+2] =
// -1/((2j+5) s_j), and the output map, the Legendre coefficients of
// u = (1-x^2)(1-y^2) sum X_ij C~_i(y) C~_j(x), is U = L X L^T with L ((n+2) x n)
// L[j][j] = c_j, L[j+2][j] = -c_j, c_j = s_j (j+1)(j+2)/(2j+3): the product
// B^{-1} M of the C~ -> Legendre conversion and the multiplication (3.7) by
// (1 - x^2) collapses to two terms.  Algorithmic traffic is one FP64 read and one
// write per element; at four FP64 operations per element GB300's FP64 rate, not
// its HBM, bounds both maps.
#include "legendre.cuh"

namespace fps {

namespace {

constexpr int kTC = 32;  // output tile: kTC columns (one per lane) ...
constexpr int kTR = 64;  // ... by kTR rows (output map); thread row ty takes parity ty & 1 and 8 rows of it
constexpr int kRows = 8;

__device__ __forceinline__ double snorm(int64_t k)
{
    const double K = (double)k;
    return sqrt((K + 1.5) / ((K + 1.0) * (K + 2.0)));
}

// F[j][k] = sum_{a in {j, j+2}} sum_{b in {k, k+2}} B[j][a] B[k][b] G[a][b]: one thread per
// output element (this kernel runs faster with the extra FP64 products than with
// fewer, longer-running threads that reuse row combinations).
__global__ void __launch_bounds__(256) legendre_to_ctilde_kernel(const double *__restrict__ G,
                                                                 double *__restrict__ F, int64_t n)
{
    __shared__ double rd[kTC], ro[kTC], cd[kTC], co[kTC];  // B entries of the tile's rows and columns
    const int64_t j0 = (int64_t)blockIdx.y * kTC, k0 = (int64_t)blockIdx.x * kTC;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid < kTC) {
        const int64_t j = j0 + tid;
        const double s = snorm(j);
        rd[tid] = 1.0 / ((2.0 * (double)j + 1.0) * s);
        ro[tid] = -1.0 / ((2.0 * (double)j + 5.0) * s);
    } else if (tid < 2 * kTC) {
        const int64_t k = k0 + tid - kTC;
        const double s = snorm(k);
        cd[tid - kTC] = 1.0 / ((2.0 * (double)k + 1.0) * s);
        co[tid - kTC] = -1.0 / ((2.0 * (double)k + 5.0) * s);
    }
    __syncthreads();
    const int64_t k = k0 + threadIdx.x;
    if (k >= n) return;
    const bool k2 = k + 2 < n;
    for (int r = threadIdx.y; r < kTC; r += blockDim.y) {
        const int64_t j = j0 + r;
        if (j >= n) break;
        const double *g0 = G + j * n + k;
        double row0 = cd[threadIdx.x] * g0[0];
        if (k2) row0 = fma(co[threadIdx.x], g0[2], row0);
        double v = rd[r] * row0;
        if (j + 2 < n) {
            const double *g2 = g0 + 2 * n;
            double row2 = cd[threadIdx.x] * g2[0];
            if (k2) row2 = fma(co[threadIdx.x], g2[2], row2);
            v = fma(ro[r], row2, v);
        }
        F[j * n + k] = v;
    }
}

//   U[i] = c_i w_i - c_{i-2} w_{i-2},  w_a = c_k X[a][k] - c_{k-2} X[a][k-2]  (a in [0, n)):
// each thread walks a strip of same-parity rows and forms every w once (FP64
// arithmetic, not HBM, bounds this map on GB300; measured 2.5 ms against 3.1 ms
// for one thread per element at n = 10^4).
__global__ void __launch_bounds__(256) solution_to_legendre_kernel(const double *__restrict__ X,
                                                                   double *__restrict__ U, int64_t n)
{
    __shared__ double rc[kTR + 2];  // c_a for a = i0 - 2 .. i0 + kTR - 1 (0 outside [0, n))
    const int64_t m = n + 2;
    const int64_t i0 = (int64_t)blockIdx.y * kTR, k0 = (int64_t)blockIdx.x * kTC;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    auto cval = [&](int64_t a) {
        if (a < 0 || a >= n) return 0.0;
        const double A = (double)a;
        return snorm(a) * (A + 1.0) * (A + 2.0) / (2.0 * A + 3.0);
    };
    if (tid < kTR + 2) rc[tid] = cval(i0 - 2 + tid);
    __syncthreads();
    const int64_t k = k0 + threadIdx.x;
    if (k >= m) return;
    const bool kin = k < n, km2 = k >= 2;  // columns k and k - 2 present in X (k - 2 < n always)
    const double ck = cval(k), ckm2 = cval(k - 2);
    auto wrow = [&](int64_t a) {  // (X L^T)[a][k], zero outside [0, n)
        if (a < 0 || a >= n) return 0.0;
        const double *x = X + a * n;
        double v = kin ? ck * x[k] : 0.0;
        return km2 ? fma(-ckm2, x[k - 2], v) : v;
    };
    const int par = threadIdx.y & 1, strip = threadIdx.y >> 1;
    const int r_lo = par + 2 * kRows * strip;
    const int r_hi = r_lo + 2 * (kRows - 1);
    double prv = wrow(i0 + r_lo - 2);                   // w_{i-2} for the first row
    for (int r = r_lo; r <= r_hi; r += 2) {
        const int64_t i = i0 + r;
        const double cur = wrow(i);
        if (i < m) U[i * m + k] = fma(-rc[r], prv, rc[r + 2] * cur);
        prv = cur;
    }
}

// Transpose of the input map, Gbar = B^T Fbar B:
//   Gbar[a][b] = sum_{i in {a, a-2}} sum_{j in {b, b-2}} B[i][a] B[j][b] Fbar[i][j],
// with B[a][a] and B[a-2][a] the two entries of column a.  One thread per element.
__global__ void __launch_bounds__(256) legendre_to_ctilde_adjoint_kernel(const double *__restrict__ Fb,
                                                                         double *__restrict__ Gb, int64_t n)
{
    __shared__ double rd[kTC], ro[kTC], cd[kTC], co[kTC];  // column a of B: {B[a][a], B[a-2][a]} (0 if a < 2)
    const int64_t a0 = (int64_t)blockIdx.y * kTC, b0 = (int64_t)blockIdx.x * kTC;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    auto diag = [](int64_t j) { return 1.0 / ((2.0 * (double)j + 1.0) * snorm(j)); };
    auto off = [](int64_t j) { return j < 2 ? 0.0 : -1.0 / ((2.0 * (double)(j - 2) + 5.0) * snorm(j - 2)); };
    if (tid < kTC) {
        rd[tid] = diag(a0 + tid);
        ro[tid] = off(a0 + tid);
    } else if (tid < 2 * kTC) {
        cd[tid - kTC] = diag(b0 + tid - kTC);
        co[tid - kTC] = off(b0 + tid - kTC);
    }
    __syncthreads();
    const int64_t b = b0 + threadIdx.x;
    if (b >= n) return;
    const bool b2 = b >= 2;
    for (int r = threadIdx.y; r < kTC; r += blockDim.y) {
        const int64_t a = a0 + r;
        if (a >= n) break;
        const double *f0 = Fb + a * n + b;
        double row0 = cd[threadIdx.x] * f0[0];
        if (b2) row0 = fma(co[threadIdx.x], f0[-2], row0);
        double v = rd[r] * row0;
        if (a >= 2) {
            const double *f2 = f0 - 2 * n;
            double row2 = cd[threadIdx.x] * f2[0];
            if (b2) row2 = fma(co[threadIdx.x], f2[-2], row2);
            v = fma(ro[r], row2, v);
        }
        Gb[a * n + b] = v;
    }
}

// Transpose of the output map, Xbar = L^T Ubar L with L[a][a] = c_a, L[a+2][a] = -c_a:
//   Xbar[a][k] = c_a c_k (Ubar[a][k] - Ubar[a][k+2] - Ubar[a+2][k] + Ubar[a+2][k+2]).
__global__ void __launch_bounds__(256) solution_to_legendre_adjoint_kernel(const double *__restrict__ Ub,
                                                                           double *__restrict__ Xb, int64_t n)
{
    __shared__ double rc[kTC], cc[kTC];
    const int64_t m = n + 2;
    const int64_t a0 = (int64_t)blockIdx.y * kTC, k0 = (int64_t)blockIdx.x * kTC;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    auto cval = [](int64_t a) {
        const double A = (double)a;
        return snorm(a) * (A + 1.0) * (A + 2.0) / (2.0 * A + 3.0);
    };
    if (tid < kTC) rc[tid] = cval(a0 + tid);
    else if (tid < 2 * kTC) cc[tid - kTC] = cval(k0 + tid - kTC);
    __syncthreads();
    const int64_t k = k0 + threadIdx.x;
    if (k >= n) return;
    for (int r = threadIdx.y; r < kTC; r += blockDim.y) {
        const int64_t a = a0 + r;
        if (a >= n) break;
        const double *u0 = Ub + a * m + k, *u2 = u0 + 2 * m;
        Xb[a * n + k] = rc[r] * cc[threadIdx.x] * ((u0[0] - u0[2]) - (u2[0] - u2[2]));
    }
}

}  // namespace

cudaError_t launch_legendre_to_ctilde(const double *G, double *F, int64_t n, cudaStream_t st)
{
    const dim3 block(kTC, 8), grid((unsigned)((n + kTC - 1) / kTC), (unsigned)((n + kTC - 1) / kTC));
    legendre_to_ctilde_kernel<<<grid, block, 0, st>>>(G, F, n);
    return cudaGetLastError();
}

cudaError_t launch_solution_to_legendre(const double *X, double *U, int64_t n, cudaStream_t st)
{
    const int64_t m = n + 2;
    const dim3 block(kTC, 8), grid((unsigned)((m + kTC - 1) / kTC), (unsigned)((m + kTR - 1) / kTR));
    solution_to_legendre_kernel<<<grid, block, 0, st>>>(X, U, n);
    return cudaGetLastError();
}

cudaError_t launch_legendre_to_ctilde_adjoint(const double *Fbar, double *Gbar, int64_t n, cudaStream_t st)
{
    const dim3 block(kTC, 8), grid((unsigned)((n + kTC - 1) / kTC), (unsigned)((n + kTC - 1) / kTC));
    legendre_to_ctilde_adjoint_kernel<<<grid, block, 0, st>>>(Fbar, Gbar, n);
    return cudaGetLastError();
}

cudaError_t launch_solution_to_legendre_adjoint(const double *Ubar, double *Xbar, int64_t n, cudaStream_t st)
{
    const dim3 block(kTC, 8), grid((unsigned)((n + kTC - 1) / kTC), (unsigned)((n + kTC - 1) / kTC));
    solution_to_legendre_adjoint_kernel<<<grid, block, 0, st>>>(Ubar, Xbar, n);
    return cudaGetLastError();
}

}  // namespace fps
