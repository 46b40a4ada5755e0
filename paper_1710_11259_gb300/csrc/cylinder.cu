// Cylinder Fourier modes |k| >= 2 (Sec. 4.1, Case 1): see cylinder.h for the
// equations.  Host: band entries from closed forms, eigenvalue intervals, shifts and
// factor tables in FP64.  Device: per ADI iteration two launches over every (mode,
// right-hand side) of the plan:
//   z kernel (32 rows per CTA, a row in shared memory per lane):
//       W = solve (M + p_j D) along the row of  -R1 D,   R2 = G - W (M + q_j D) D^{-1}
//   r kernel (32 columns per CTA, a column per lane):
//       X = solve (Q - q_j P) along the column of R2,  then R1 = (Q - p_{j+1} P) X - G
//       (or Y = X after the mode's last iteration)
// with R1 = -G before the first iteration (X_0 = 0).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/fps.h"
#include "cylinder.h"
#include "host_math.h"

namespace fps {

// ---------------------------------------------------------------- band entries
// s_j of C~_j = s_j C_j^(3/2)
static double ct_scale(int64_t j)
{
    const double x = (double)j;
    return std::sqrt((x + 1.5) / ((x + 1.0) * (x + 2.0)));
}

// (3.7) in the normalised basis: M = multiplication by (1 - x^2)
double cyl_M_diag(int64_t j)
{
    const double x = (double)j;
    return 2.0 * (x + 1.0) * (x + 2.0) / ((2.0 * x + 1.0) * (2.0 * x + 5.0));
}
double cyl_M_off(int64_t j)
{
    const double x = (double)j;
    const double prod4 = (x + 1.0) * (x + 2.0) * (x + 3.0) * (x + 4.0);
    return -std::sqrt(prod4 * (2.0 * x + 3.0) / (2.0 * x + 7.0)) / ((2.0 * x + 3.0) * (2.0 * x + 5.0));
}
static double Mentry(int64_t a, int64_t i)
{
    if (a < 0 || i < 0) return 0.0;
    if (a == i) return cyl_M_diag(a);
    if (a == i + 2) return cyl_M_off(i);
    if (i == a + 2) return cyl_M_off(a);
    return 0.0;
}

// x (1 - x^2) d/dx in the C^(3/2) basis, from (1 - x^2) C_m' = al_m C_{m-1} - be_m C_{m+1}
// and x C_j = ga_j C_{j+1} + de_j C_{j-1} (lambda = 3/2), then normalised.
static double X1entry(int64_t a, int64_t m)
{
    if (a < 0 || m < 0) return 0.0;
    const double M_ = (double)m;
    const double al = (M_ + 2.0) * (M_ + 3.0) / (2.0 * M_ + 3.0), be = M_ * (M_ + 1.0) / (2.0 * M_ + 3.0);
    auto ga = [](double j) { return (j + 1.0) / (2.0 * j + 3.0); };
    auto de = [](double j) { return (j + 2.0) / (2.0 * j + 3.0); };
    double v = 0.0;
    if (a == m) v = (m >= 1 ? al * ga(M_ - 1.0) : 0.0) - be * de(M_ + 1.0);
    else if (a == m - 2) v = al * de(M_ - 1.0);
    else if (a == m + 2) v = -be * ga(M_ + 1.0);
    else return 0.0;
    return v * ct_scale(m) / ct_scale(a);
}

// L1 = (I - M) D + 5 [x (1 - x^2) d/dx] + 14 M - 10 I, the matrix of
// r^2(1 - r^2) d^2/dr^2 + (5 - 9 r^2) r d/dr + 4 (1 - 4 r^2)
double cyl_L1(int64_t a, int64_t i)
{
    const double Dii = -((double)i + 1.0) * ((double)i + 2.0);
    return ((a == i ? 1.0 : 0.0) - Mentry(a, i)) * Dii + 5.0 * X1entry(a, i) + 14.0 * Mentry(a, i) -
           (a == i ? 10.0 : 0.0);
}

// Q = M - M^2 (the exact product: the inner index runs past n)
static double Qentry(int64_t a, int64_t i)
{
    double mm = 0.0;
    for (int64_t c = a - 2; c <= a + 2; c += 2) mm += Mentry(a, c) * Mentry(c, i);
    return Mentry(a, i) - mm;
}

namespace {

// Per-parity banded operators of one mode (index s <-> t = par + 2 s).
struct ParityOps {
    int m = 0;
    std::vector<double> pl, pd, pu;      // P[t][t-2], P[t][t], P[t][t+2]
    std::vector<double> q0, q2, q4;      // Q[t][t], Q[t][t+2], Q[t][t+4] (symmetric)
};

ParityOps parity_ops(int64_t n, int64_t k, int par)
{
    ParityOps o;
    o.m = (int)((n - par + 1) / 2);
    const double k2 = (double)k * (double)k;
    for (int s = 0; s < o.m; ++s) {
        const int64_t t = par + 2 * s;
        o.pl.push_back(t >= 2 ? cyl_L1(t, t - 2) - k2 * Mentry(t, t - 2) : 0.0);
        o.pd.push_back(cyl_L1(t, t) - k2 * Mentry(t, t));
        o.pu.push_back(t + 2 < n ? cyl_L1(t, t + 2) - k2 * Mentry(t, t + 2) : 0.0);
        o.q0.push_back(Qentry(t, t));
        o.q2.push_back(t + 2 < n ? Qentry(t, t + 2) : 0.0);
        o.q4.push_back(t + 4 < n ? Qentry(t, t + 4) : 0.0);
    }
    return o;
}

// y = P x, y = Q x (parity blocks)
void apply_P(const ParityOps &o, const std::vector<double> &x, std::vector<double> &y)
{
    for (int s = 0; s < o.m; ++s) {
        double v = o.pd[s] * x[s];
        if (s >= 1) v += o.pl[s] * x[s - 1];
        if (s + 1 < o.m) v += o.pu[s] * x[s + 1];
        y[s] = v;
    }
}
void apply_Q(const ParityOps &o, const std::vector<double> &x, std::vector<double> &y)
{
    for (int s = 0; s < o.m; ++s) {
        double v = o.q0[s] * x[s];
        if (s >= 1) v += o.q2[s - 1] * x[s - 1];
        if (s >= 2) v += o.q4[s - 2] * x[s - 2];
        if (s + 1 < o.m) v += o.q2[s] * x[s + 1];
        if (s + 2 < o.m) v += o.q4[s] * x[s + 2];
        y[s] = v;
    }
}
// x = P^{-1} b (tridiagonal, diagonally dominant: no pivoting)
void solve_P(const ParityOps &o, std::vector<double> b, std::vector<double> &x)
{
    std::vector<double> c(o.m), d(o.m);
    for (int s = 0; s < o.m; ++s) {
        double den = o.pd[s] - (s >= 1 ? o.pl[s] * c[s - 1] : 0.0);
        c[s] = o.pu[s] / den;
        d[s] = (b[s] - (s >= 1 ? o.pl[s] * d[s - 1] : 0.0)) / den;
    }
    for (int s = o.m - 1; s >= 0; --s) x[s] = d[s] - (s + 1 < o.m ? c[s] * x[s + 1] : 0.0);
}
// LU without pivoting of T = Q - q P (pentadiagonal per parity), as used on the device
struct LU5 {
    std::vector<double> l1, l2, iu0, u1, u2;
};
LU5 lu_QminusqP(const ParityOps &o, double q)
{
    LU5 f;
    const int m = o.m;
    f.l1.assign(m, 0.0);
    f.l2.assign(m, 0.0);
    f.iu0.assign(m, 0.0);
    f.u1.assign(m, 0.0);
    f.u2.assign(m, 0.0);
    std::vector<double> u0(m);
    for (int s = 0; s < m; ++s) {
        const double tm2 = s >= 2 ? o.q4[s - 2] : 0.0;                            // T[s][s-2]
        const double tm1 = s >= 1 ? o.q2[s - 1] - q * o.pl[s] : 0.0;              // T[s][s-1]
        const double t0 = o.q0[s] - q * o.pd[s];
        const double tp1 = s + 1 < m ? o.q2[s] - q * o.pu[s] : 0.0;
        const double tp2 = s + 2 < m ? o.q4[s] : 0.0;
        const double l2 = s >= 2 ? tm2 / u0[s - 2] : 0.0;
        const double l1 = s >= 1 ? (tm1 - (s >= 2 ? l2 * f.u1[s - 2] : 0.0)) / u0[s - 1] : 0.0;
        u0[s] = t0 - (s >= 1 ? l1 * f.u1[s - 1] : 0.0) - (s >= 2 ? l2 * f.u2[s - 2] : 0.0);
        f.u1[s] = tp1 - (s >= 1 ? l1 * f.u2[s - 1] : 0.0);
        f.u2[s] = tp2;
        f.l1[s] = l1;
        f.l2[s] = l2;
        f.iu0[s] = 1.0 / u0[s];
    }
    return f;
}
void solve_Q(const ParityOps &o, const std::vector<double> &b, std::vector<double> &x)
{
    const LU5 f = lu_QminusqP(o, 0.0);
    std::vector<double> y(o.m);
    for (int s = 0; s < o.m; ++s)
        y[s] = b[s] - (s >= 1 ? f.l1[s] * y[s - 1] : 0.0) - (s >= 2 ? f.l2[s] * y[s - 2] : 0.0);
    for (int s = o.m - 1; s >= 0; --s)
        x[s] = (y[s] - (s + 1 < o.m ? f.u1[s] * x[s + 1] : 0.0) - (s + 2 < o.m ? f.u2[s] * x[s + 2] : 0.0)) *
               f.iu0[s];
}

// Dominant eigenvalue of x -> op(x) by power iteration with a Rayleigh quotient.
template <class Op>
double power_eig(int m, Op op)
{
    std::vector<double> x(m), y(m);
    for (int s = 0; s < m; ++s) x[s] = 1.0 + 0.25 * std::sin(1.0 + 0.7 * s);
    double lam = 0.0;
    for (int it = 0; it < 3000; ++it) {
        double nx = 0.0;
        for (double v : x) nx += v * v;
        nx = std::sqrt(nx);
        for (double &v : x) v /= nx;
        op(x, y);
        double num = 0.0;
        for (int s = 0; s < m; ++s) num += x[s] * y[s];
        if (it > 20 && std::fabs(num - lam) <= 1e-12 * std::fabs(num)) return num;
        lam = num;
        x.swap(y);
    }
    return lam;
}

}  // namespace

int cyl_mode_interval(int64_t n, int64_t k, double &a, double &b)
{
    double most = 0.0, least = -1e300;
    for (int par = 0; par < 2 && par < n; ++par) {
        const ParityOps o = parity_ops(n, k, par);
        if (o.m == 0) continue;
        std::vector<double> tmp(o.m);
        const double big = power_eig(o.m, [&](const std::vector<double> &x, std::vector<double> &y) {
            apply_Q(o, x, tmp);
            solve_P(o, tmp, y);
        });
        const double inv = power_eig(o.m, [&](const std::vector<double> &x, std::vector<double> &y) {
            apply_P(o, x, tmp);
            solve_Q(o, tmp, y);
        });
        most = std::min(most, big);
        least = std::max(least, 1.0 / inv);
    }
    if (!(most < 0.0) || !(least < 0.0) || !std::isfinite(most) || !std::isfinite(least)) return FPS_ERR_UNSUPPORTED;
    a = 1.03 * most;
    b = 0.97 * least;
    return FPS_OK;
}

// ---------------------------------------------------------------- device side
namespace {

constexpr int kCL = 32;        // lines per CTA
constexpr int kCylThreads = 256;  // threads per CTA: all move the tile, the first 2 kCL sweep

struct CylArgs {
    int n, modes, nrhs, kmin, Jmax, j;
    const double *bands;   // [9][n + 4] (see kBand*)
    const double2 *zfac;   // [sum J][n]
    const double *rfac;    // [sum J][n][6]
    const double *shifts;  // [modes][Jmax][2]
    const int *joff, *jcount;
    const double *G;       // [modes][nrhs][n][n]
    const double *Rin;
    double *Rout, *Y;
    bool first;            // j == 0: the z kernel reads R1 = -G
};
enum { kMd = 0, kMe, kD, kL1d, kL1u, kL1l, kQ0, kQ2, kQ4, kBands };

__host__ __device__ inline int pitch_of(int n) { return (n % 2 == 0) ? n + 1 : n; }

constexpr int kC = 8;  // read-ahead chunk of the sweeps

// z kernel: blockIdx.x = block of 32 rows, blockIdx.y = (mode, rhs).  Shared memory:
// the tile [32][P], then the factor set of (M + p_j D), the bands M_d, M_e, D and -1/D.
__global__ void __launch_bounds__(kCylThreads) cyl_z_kernel(CylArgs A)
{
    const int n = A.n, P = pitch_of(n), st = n + 4;
    const int mode = blockIdx.y / A.nrhs;
    const int J = A.jcount[mode];
    if (A.j >= J) return;
    extern __shared__ double tile[];  // [kCL][P]
    double2 *fz = reinterpret_cast<double2 *>(tile + kCL * P);
    double *md = reinterpret_cast<double *>(fz + n), *me = md + n, *dd = me + n, *nid = dd + n;  // nid = -1/D
    const int64_t pair = blockIdx.y;
    const int i0 = blockIdx.x * kCL, nl = min(kCL, n - i0);
    const double *Rin = A.first ? A.G : A.Rin;
    const double sgn = A.first ? -1.0 : 1.0;
    const int64_t base = pair * (int64_t)n * n + (int64_t)i0 * n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int li = warp; li < nl; li += kCylThreads / 32) {
        const double *src = Rin + base + (int64_t)li * n;
#pragma unroll 4
        for (int t = lane; t < n; t += 32) tile[li * P + t] = sgn * src[t];
    }
    const double2 *fzg = A.zfac + (int64_t)(A.joff[mode] + A.j) * n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        fz[t] = fzg[t];
        md[t] = A.bands[kMd * st + t];
        me[t] = A.bands[kMe * st + t];
        dd[t] = A.bands[kD * st + t];
        nid[t] = -1.0 / dd[t];
    }
    __syncthreads();
    const double qq = A.shifts[((int64_t)mode * A.Jmax + A.j) * 2 + 1];
    const int li = threadIdx.x & (kCL - 1), par = threadIdx.x / kCL;
    if (threadIdx.x < 2 * kCL && li < nl) {
        double *row = tile + li * P;
        const int m = (n - par + 1) / 2;
        // W (M + p D) = -R1 D  (symmetric tridiagonal per parity)
        double z = 0.0, up = 0.0;
        for (int s0 = 0; s0 < m; s0 += kC) {
            double in[kC], uf[kC];
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int t = par + 2 * min(s0 + u, m - 1);
                in[u] = -row[t] * dd[t];
                uf[u] = fz[t].y;
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (s0 + u < m) {
                    z = fma(-up, z, in[u]);
                    row[par + 2 * (s0 + u)] = z;
                    up = uf[u];
                }
        }
        double x = 0.0;
        for (int s0 = m - 1; s0 >= 0; s0 -= kC) {
            double zz[kC];
            double2 ff[kC];
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int t = par + 2 * max(s0 - u, 0);
                zz[u] = row[t];
                ff[u] = fz[t];
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (s0 - u >= 0) {
                    x = fma(-ff[u].y, x, ff[u].x * zz[u]);
                    row[par + 2 * (s0 - u)] = x;
                }
        }
        // -(W (M + q D)) D^{-1} along the row, in place with the previous W in a register
        double prev = 0.0;
        for (int s0 = 0; s0 < m; s0 += kC) {
            double cur[kC + 1];
#pragma unroll
            for (int u = 0; u <= kC; ++u) {
                const int t = par + 2 * (s0 + u);
                cur[u] = t < n ? row[t] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (s0 + u < m) {
                    const int t = par + 2 * (s0 + u);
                    double v = fma(qq, dd[t], md[t]) * cur[u];
                    if (t >= 2) v = fma(me[t - 2], prev, v);
                    v = fma(me[t], cur[u + 1], v);  // me[t] = 0 when t + 2 >= n
                    row[t] = v * nid[t];
                    prev = cur[u];
                }
        }
    }
    __syncthreads();
    for (int l = warp; l < nl; l += kCylThreads / 32) {
        const int64_t g0 = base + (int64_t)l * n;
#pragma unroll 4
        for (int t = lane; t < n; t += 32) A.Rout[g0 + t] = tile[l * P + t] + A.G[g0 + t];
    }
}

// r kernel: blockIdx.x = block of 32 columns, blockIdx.y = (mode, rhs).  Shared memory:
// the tile [n][32], the LU factors of (Q - q_j P) [n][6], and the bands of Q and of
// P = L1 - k^2 M for this mode [6][n].
__global__ void __launch_bounds__(kCylThreads) cyl_r_kernel(CylArgs A)
{
    const int n = A.n, st = n + 4;
    const int mode = blockIdx.y / A.nrhs;
    const int J = A.jcount[mode];
    if (A.j >= J) return;
    const bool last = A.j + 1 == J;
    extern __shared__ double tile[];  // [n][kCL]
    double *fr = tile + (int64_t)n * kCL;   // [n][6]
    double *q0 = fr + 6 * n, *q2 = q0 + n, *q4 = q2 + n, *pl = q4 + n, *pd = pl + n, *pu = pd + n;
    const int64_t pair = blockIdx.y;
    const int c0 = blockIdx.x * kCL, nc = min(kCL, n - c0);
    const int64_t base = pair * (int64_t)n * n + c0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < nc) {
#pragma unroll 4
        for (int t = warp; t < n; t += kCylThreads / 32) tile[t * kCL + lane] = A.Rin[base + (int64_t)t * n + lane];
    }
    const double *frg = A.rfac + (int64_t)(A.joff[mode] + A.j) * n * 6;
    for (int q = threadIdx.x; q < 6 * n; q += blockDim.x) fr[q] = frg[q];
    const double k2 = (double)(A.kmin + mode) * (double)(A.kmin + mode);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const double *bd = A.bands;
        q0[t] = bd[kQ0 * st + t];
        q2[t] = bd[kQ2 * st + t];
        q4[t] = bd[kQ4 * st + t];
        pd[t] = bd[kL1d * st + t] - k2 * bd[kMd * st + t];
        pu[t] = bd[kL1u * st + t] - k2 * bd[kMe * st + t];
        pl[t] = t >= 2 ? bd[kL1l * st + t] - k2 * bd[kMe * st + t - 2] : 0.0;
    }
    __syncthreads();
    const int cj = threadIdx.x & (kCL - 1), par = threadIdx.x / kCL;
    if (threadIdx.x < 2 * kCL && cj < nc) {
        double *col = tile + cj;
        const int m = (n - par + 1) / 2;
        // (Q - q P) X = R2: unit lower then upper sweep of the stored LU
        double y1 = 0.0, y2 = 0.0;  // y at s - 1, s - 2
        for (int s0 = 0; s0 < m; s0 += kC) {
            double bb[kC], l1[kC], l2[kC];
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int t = par + 2 * min(s0 + u, m - 1);
                bb[u] = col[t * kCL];
                l1[u] = fr[t * 6 + 0];
                l2[u] = fr[t * 6 + 1];
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (s0 + u < m) {
                    const double y = fma(-l2[u], y2, fma(-l1[u], y1, bb[u]));
                    col[(par + 2 * (s0 + u)) * kCL] = y;
                    y2 = y1;
                    y1 = y;
                }
        }
        double x1 = 0.0, x2 = 0.0;  // x at s + 1, s + 2
        for (int s0 = m - 1; s0 >= 0; s0 -= kC) {
            double yy[kC], iu[kC], u1[kC], u2[kC];
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int t = par + 2 * max(s0 - u, 0);
                yy[u] = col[t * kCL];
                iu[u] = fr[t * 6 + 2];
                u1[u] = fr[t * 6 + 3];
                u2[u] = fr[t * 6 + 4];
            }
#pragma unroll
            for (int u = 0; u < kC; ++u)
                if (s0 - u >= 0) {
                    const double x = fma(-u2[u], x2, fma(-u1[u], x1, yy[u])) * iu[u];
                    col[(par + 2 * (s0 - u)) * kCL] = x;
                    x2 = x1;
                    x1 = x;
                }
        }
        if (!last) {  // (Q - p' P) X along the column, in place with two previous X in registers
            const double p = A.shifts[((int64_t)mode * A.Jmax + A.j + 1) * 2 + 0];
            double xm2 = 0.0, xm1 = 0.0;  // X at s - 2, s - 1
            for (int s0 = 0; s0 < m; s0 += kC) {
                double xv[kC + 2];
#pragma unroll
                for (int u = 0; u < kC + 2; ++u) {
                    const int t = par + 2 * (s0 + u);
                    xv[u] = t < n ? col[t * kCL] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kC; ++u)
                    if (s0 + u < m) {
                        const int t = par + 2 * (s0 + u);
                        // q2[t], q4[t], pu[t] are zero past the end of the chain
                        double qv = fma(q4[t], xv[u + 2], fma(q2[t], xv[u + 1], q0[t] * xv[u]));
                        double pv = fma(pu[t], xv[u + 1], pd[t] * xv[u]);
                        if (t >= 2) {
                            qv = fma(q2[t - 2], xm1, qv);
                            pv = fma(pl[t], xm1, pv);
                        }
                        if (t >= 4) qv = fma(q4[t - 4], xm2, qv);
                        col[t * kCL] = fma(-p, pv, qv);
                        xm2 = xm1;
                        xm1 = xv[u];
                    }
            }
        }
    }
    __syncthreads();
    if (lane < nc) {
#pragma unroll 4
        for (int t = warp; t < n; t += kCylThreads / 32) {
            const int64_t g = base + (int64_t)t * n + lane;
            if (last) A.Y[g] = tile[t * kCL + lane];
            else A.Rout[g] = tile[t * kCL + lane] - A.G[g];
        }
    }
}

int z_smem(int n) { return (int)sizeof(double) * (kCL * pitch_of(n) + 2 * n + 4 * n); }
int r_smem(int n) { return (int)sizeof(double) * (kCL * n + 6 * n + 6 * n); }

// G = F D^{-1} (column j scaled by 1 / D_jj)
__global__ void cyl_scale_kernel(const double *F, double *G, int n, int64_t total)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q % n);
        G[q] = -F[q] / (((double)j + 1.0) * ((double)j + 2.0));
    }
}

}  // namespace

template <typename U>
cudaError_t CylinderEngine::dalloc(U **p, size_t count)
{
    cudaError_t e = cudaMalloc((void **)p, sizeof(U) * std::max<size_t>(count, 1));
    if (e == cudaSuccess) {
        allocs_.push_back(*p);
        bytes += (int64_t)(sizeof(U) * count);
    }
    return e;
}

#define CYL_CK(call)                                                                                      \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                                     \
            return FPS_ERR_CUDA;                                                                          \
        }                                                                                                 \
    } while (0)

int CylinderEngine::create(int64_t n_, int64_t kmin_, int64_t kmax_, double tol, int nrhs_, std::string &err)
{
    n = n_;
    kmin = kmin_;
    kmax = kmax_;
    nrhs = nrhs_;
    const int modes = (int)(kmax - kmin + 1);
    // Both kernels hold whole lines of 32 (mode, rhs) rows or columns in shared
    // memory: about 352 n bytes per CTA, n <= 660 at 227 KB.
    int dev = 0, optin = 0;
    CYL_CK(cudaGetDevice(&dev));
    CYL_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int need = std::max(z_smem((int)n), r_smem((int)n));
    if (need > optin) {
        err = "n = " + std::to_string(n) + " needs " + std::to_string(need) +
              " bytes of shared memory per CTA (device limit " + std::to_string(optin) + ")";
        return FPS_ERR_UNSUPPORTED;
    }
    // sigma(B) = sigma(-M D^{-1}) = sigma(-A~): the tight interval of A~
    lo = square_eps(n);
    hi = 1.0;
    square_tight_interval(n, lo, hi);
    std::vector<double> bands((size_t)kBands * (n + 4), 0.0);
    for (int64_t t = 0; t < n; ++t) {
        const size_t st = (size_t)(n + 4);
        bands[kMd * st + t] = cyl_M_diag(t);
        bands[kMe * st + t] = t + 2 < n ? cyl_M_off(t) : 0.0;
        bands[kD * st + t] = -((double)t + 1.0) * ((double)t + 2.0);
        bands[kL1d * st + t] = cyl_L1(t, t);
        bands[kL1u * st + t] = t + 2 < n ? cyl_L1(t, t + 2) : 0.0;
        bands[kL1l * st + t] = t >= 2 ? cyl_L1(t, t - 2) : 0.0;
        bands[kQ0 * st + t] = Qentry(t, t);
        bands[kQ2 * st + t] = t + 2 < n ? Qentry(t, t + 2) : 0.0;
        bands[kQ4 * st + t] = t + 4 < n ? Qentry(t, t + 4) : 0.0;
    }
    J.assign(modes, 0);
    a.assign(modes, 0.0);
    b.assign(modes, 0.0);
    std::vector<std::vector<double>> P(modes), Qs(modes);
    Jmax = 0;
    for (int md = 0; md < modes; ++md) {
        const int64_t k = kmin + md;
        if (cyl_mode_interval(n, k, a[md], b[md]) != FPS_OK) {
            err = "mode " + std::to_string(k) + ": eigenvalue interval of A_k not found";
            return FPS_ERR_UNSUPPORTED;
        }
        J[md] = adi_iterations(a[md], b[md], lo, hi, tol);
        zolotarev_shifts(a[md], b[md], lo, hi, J[md], P[md], Qs[md]);
        if (!shifts_valid(Qs[md], lo, hi)) {
            err = "shift list failed validation (a shift is not finite or lies outside the spectral interval)";
            return FPS_ERR_INVALID_ARG;
        }
        for (double &v : P[md]) v = -v;
        const bool ok = shifts_valid(P[md], -b[md], -a[md]);
        for (double &v : P[md]) v = -v;
        if (!ok) {
            err = "shift list failed validation (a shift is not finite or lies outside the spectral interval)";
            return FPS_ERR_INVALID_ARG;
        }
        Jmax = std::max(Jmax, J[md]);
    }
    // tables
    std::vector<int> joff(modes), jc(modes);
    int sumJ = 0;
    for (int md = 0; md < modes; ++md) {
        joff[md] = sumJ;
        jc[md] = J[md];
        sumJ += J[md];
    }
    std::vector<double2> zf((size_t)sumJ * n);
    std::vector<double> rf((size_t)sumJ * n * 6, 0.0), sh((size_t)modes * Jmax * 2, 0.0);
    for (int md = 0; md < modes; ++md) {
        const int64_t k = kmin + md;
        ParityOps ops[2] = {parity_ops(n, k, 0), n > 1 ? parity_ops(n, k, 1) : ParityOps()};
        for (int j = 0; j < J[md]; ++j) {
            const double p = P[md][j], q = Qs[md][j];
            sh[((size_t)md * Jmax + j) * 2 + 0] = p;
            sh[((size_t)md * Jmax + j) * 2 + 1] = q;
            double2 *z = zf.data() + (size_t)(joff[md] + j) * n;
            double *r = rf.data() + (size_t)(joff[md] + j) * n * 6;
            for (int par = 0; par < 2 && par < n; ++par) {
                double u_prev = 0.0;
                for (int64_t t = par; t < n; t += 2) {  // (M + p D), symmetric tridiagonal
                    double den = cyl_M_diag(t) + p * (-((double)t + 1.0) * ((double)t + 2.0));
                    if (t >= 2) den -= cyl_M_off(t - 2) * u_prev;
                    const double u = t + 2 < n ? cyl_M_off(t) / den : 0.0;
                    z[t] = make_double2(1.0 / den, u);
                    u_prev = u;
                }
                const LU5 f = lu_QminusqP(ops[par], q);
                for (int s = 0; s < ops[par].m; ++s) {
                    const int64_t t = par + 2 * s;
                    double *e = r + t * 6;
                    e[0] = f.l1[s];
                    e[1] = f.l2[s];
                    e[2] = f.iu0[s];
                    e[3] = f.u1[s];
                    e[4] = f.u2[s];
                    if (!std::isfinite(e[2]) || !std::isfinite(e[0]) || !std::isfinite(e[1])) {
                        err = "mode " + std::to_string(k) + ": pivot breakdown in the r-direction factors";
                        return FPS_ERR_UNSUPPORTED;
                    }
                }
            }
        }
    }
    const size_t total = (size_t)modes * nrhs * n * n;
    CYL_CK(dalloc(&G_, total));
    CYL_CK(dalloc(&R1_, total));
    CYL_CK(dalloc(&R2_, total));
    CYL_CK(dalloc(&bands_, bands.size()));
    CYL_CK(dalloc(&zfac_, zf.size()));
    CYL_CK(dalloc(&rfac_, rf.size()));
    CYL_CK(dalloc(&shifts_, sh.size()));
    CYL_CK(dalloc(&joff_, (size_t)modes));
    CYL_CK(dalloc(&jcount_, (size_t)modes));
    CYL_CK(cudaMemcpy(bands_, bands.data(), sizeof(double) * bands.size(), cudaMemcpyHostToDevice));
    CYL_CK(cudaMemcpy(zfac_, zf.data(), sizeof(double2) * zf.size(), cudaMemcpyHostToDevice));
    CYL_CK(cudaMemcpy(rfac_, rf.data(), sizeof(double) * rf.size(), cudaMemcpyHostToDevice));
    CYL_CK(cudaMemcpy(shifts_, sh.data(), sizeof(double) * sh.size(), cudaMemcpyHostToDevice));
    CYL_CK(cudaMemcpy(joff_, joff.data(), sizeof(int) * modes, cudaMemcpyHostToDevice));
    CYL_CK(cudaMemcpy(jcount_, jc.data(), sizeof(int) * modes, cudaMemcpyHostToDevice));
    const int zs = z_smem((int)n), rs = r_smem((int)n);
    CYL_CK(cudaFuncSetAttribute(cyl_z_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, zs));
    CYL_CK(cudaFuncSetAttribute(cyl_r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rs));
    return FPS_OK;
}

void CylinderEngine::release()
{
    for (void *p : allocs_) cudaFree(p);
    allocs_.clear();
}

int CylinderEngine::solve(const double *F, double *Y, cudaStream_t st, std::string &err)
{
    const int modes = (int)(kmax - kmin + 1);
    const int64_t total = (int64_t)modes * nrhs * n * n;
    launches_last = 0;
    cyl_scale_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(F, G_, (int)n, total);
    ++launches_last;
    CYL_CK(cudaGetLastError());
    CylArgs A;
    A.n = (int)n;
    A.modes = modes;
    A.nrhs = nrhs;
    A.kmin = (int)kmin;
    A.Jmax = Jmax;
    A.bands = bands_;
    A.zfac = zfac_;
    A.rfac = rfac_;
    A.shifts = shifts_;
    A.joff = joff_;
    A.jcount = jcount_;
    A.G = G_;
    A.Y = Y;
    const dim3 grid((unsigned)((n + kCL - 1) / kCL), (unsigned)(modes * nrhs));
    const int zs = z_smem((int)n), rs = r_smem((int)n);
    for (int j = 0; j < Jmax; ++j) {
        A.j = j;
        A.first = j == 0;
        A.Rin = R1_;
        A.Rout = R2_;
        cyl_z_kernel<<<grid, kCylThreads, zs, st>>>(A);
        A.first = false;
        A.Rin = R2_;
        A.Rout = R1_;
        cyl_r_kernel<<<grid, kCylThreads, rs, st>>>(A);
        launches_last += 2;
        CYL_CK(cudaGetLastError());
    }
    return FPS_OK;
}

}  // namespace fps
