// Small squares (n <= 64) in FP64: the whole of Algorithm 2 in one launch.
//
// For n <= 64 every tridiagonal of the even/odd decoupling (App. B) has at most 32
// unknowns: one warp solves it by parallel cyclic reduction with warp shuffles
// (lane t holds unknown t).  Because A~ - q_j I is the same matrix for every line,
// the reduction coefficients of each shift are computed once on the host and only
// the right-hand side moves through the five reduction steps:
//     r_t <- r_t + alpha_t r_{t-s} + gamma_t r_{t+s},   s = 1, 2, 4, 8, 16,
//     x_t  = r_t / b_t.
// The iterate lives in shared memory.  GB300's FP64 rate is low (about 2 FMA per
// clock per SM), so one right-hand side is spread over a cluster of 8 CTAs: every
// CTA holds a full copy of Y and Y_h, solves the lines it owns and writes its
// results into all 8 copies through distributed shared memory; a cluster barrier
// separates the half-steps.  The iteration is the paper's form, as in the oracle:
//     Y_h (A~ - q I) = F~ - (A~ + q I) Y          (rows)
//     (A~ - q I) Y+  = F~ - Y_h (A~ + q I)        (columns)
// with F~ = D_s F D_s and X = D_s Y_J D_s (3.9).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "small.cuh"

namespace cg = cooperative_groups;

namespace fps {

namespace {

constexpr int kMax = kSmallMaxN;   // largest n
constexpr int kCl = kSmallCluster;  // CTAs per right-hand side
constexpr int kLd = kMax + 1;      // shared row stride (doubles)
constexpr int kThreads = 512;      // 16 warps: one per (owned line, parity)
constexpr size_t kSmem = sizeof(double) * 3 * kMax * kLd;

// One parity system: lane t holds r_t; the coefficients c[] are this lane's
// alpha (steps 0-4), gamma (steps 5-9) and 1/b (10).
__device__ __forceinline__ double pcr_solve(double r, const double (&c)[11], int lane)
{
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int s = 1 << st;
        double up = __shfl_up_sync(0xffffffffu, r, s);
        double dn = __shfl_down_sync(0xffffffffu, r, s);
        if (lane < s) up = 0.0;
        if (lane + s >= 32) dn = 0.0;
        r = fma(c[st], up, fma(c[5 + st], dn, r));
    }
    return r * c[10];
}

__device__ __forceinline__ void load_coefficients(const double *__restrict__ pcr, int j, int p, int lane,
                                                  double (&c)[11])
{
    const double *cf = pcr + ((int64_t)j * 2 + p) * 11 * 32 + lane;
#pragma unroll
    for (int u = 0; u < 11; ++u) c[u] = cf[u * 32];
}

__global__ void __cluster_dims__(kSmallCluster, 1, 1) __launch_bounds__(kThreads)
    small_adi_kernel(SmallArgs a)
{
    extern __shared__ __align__(16) double sm[];
    double *Ft = sm, *A = sm + kMax * kLd, *B = sm + 2 * kMax * kLd;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int rhs = blockIdx.x / kCl;
    const int n = a.n;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const double *F = a.F + (int64_t)rhs * n * n;
    double *X = a.X + (int64_t)rhs * n * n;

    // F~ = D_s F D_s and Y = 0 in every copy
    for (int idx = tid; idx < n * n; idx += kThreads) {
        const int i = idx / n, k = idx - i * n;
        Ft[i * kLd + k] = F[idx] * a.s[i] * a.s[k];
        A[i * kLd + k] = 0.0;
    }
    // lines owned by this CTA: [l0, l0 + L); warp w solves line l0 + w/2, parity w & 1
    const int L = (n + kCl - 1) / kCl;
    const int line = rank * L + (w >> 1), p = w & 1;
    const bool active = (w >> 1) < L && line < n;
    const int pos = 2 * lane + p;  // position along the solved line
    const bool valid = active && pos < n;
    // coefficients of the line's stencil: e_{l-2}, d_l, e_l (rows in step 1, columns in step 2)
    const double el_m = (line >= 2 && line < n) ? a.e[line - 2] : 0.0, el = active ? a.e[line] : 0.0;
    const double dl = active ? a.d[line] : 0.0;
    double c[11], cn[11];
    if (active) load_coefficients(a.pcr, 0, p, lane, c);
    cl.sync();

    for (int j = 0; j < a.J; ++j) {
        const double q = a.q[j];
        if (active && j + 1 < a.J) load_coefficients(a.pcr, j + 1, p, lane, cn);  // next shift, in flight
        // step 1: row `line`, rhs = F~ - (A~ + q) Y along the column index
        if (active) {
            double r = 0.0;
            if (valid) {
                const int i = line, k = pos;
                r = Ft[i * kLd + k];
                if (j > 0) {
                    double v = (dl + q) * A[i * kLd + k];
                    if (i >= 2) v = fma(el_m, A[(i - 2) * kLd + k], v);
                    if (i + 2 < n) v = fma(el, A[(i + 2) * kLd + k], v);
                    r -= v;
                }
            }
            const double x = pcr_solve(r, c, lane);
            if (valid)
#pragma unroll
                for (int rr = 0; rr < kCl; ++rr) *cl.map_shared_rank(B + line * kLd + pos, rr) = x;
        }
        cl.sync();
        // step 2: column `line`, rhs = F~ - Y_h (A~ + q) along the row index
        if (active) {
            double r = 0.0;
            if (valid) {
                const int i = pos, k = line;
                double v = (dl + q) * B[i * kLd + k];
                if (k >= 2) v = fma(el_m, B[i * kLd + k - 2], v);
                if (k + 2 < n) v = fma(el, B[i * kLd + k + 2], v);
                r = Ft[i * kLd + k] - v;
            }
            const double x = pcr_solve(r, c, lane);
            if (valid)
#pragma unroll
                for (int rr = 0; rr < kCl; ++rr) *cl.map_shared_rank(A + pos * kLd + line, rr) = x;
        }
        if (active && j + 1 < a.J)
#pragma unroll
            for (int u = 0; u < 11; ++u) c[u] = cn[u];
        cl.sync();
    }
    // X = D_s Y_J D_s for the rows this CTA owns
    for (int idx = tid; idx < L * n; idx += kThreads) {
        const int i = rank * L + idx / n, k = idx % n;
        if (i < n) X[(int64_t)i * n + k] = A[i * kLd + k] * a.s[i] * a.s[k];
    }
}

}  // namespace

void small_pcr_coefficients(int64_t n, const std::vector<double> &d, const std::vector<double> &e,
                            const std::vector<double> &q, std::vector<double> &out)
{
    const int J = (int)q.size();
    out.assign((size_t)J * 2 * 11 * 32, 0.0);
    for (int j = 0; j < J; ++j)
        for (int p = 0; p < 2; ++p) {
            const int m = (int)((n - p + 1) / 2);
            double *o = out.data() + ((size_t)j * 2 + p) * 11 * 32;
            std::vector<double> sa(32, 0.0), sb(32, 1.0), sc(32, 0.0);
            for (int t = 0; t < m; ++t) {
                const int i = 2 * t + p;
                sa[t] = t >= 1 ? e[i - 2] : 0.0;
                sb[t] = d[i] - q[j];
                sc[t] = t + 1 < m ? e[i] : 0.0;
            }
            for (int st = 0; st < 5; ++st) {
                const int s = 1 << st;
                std::vector<double> na(32, 0.0), nb(sb), nc(32, 0.0);
                for (int t = 0; t < m; ++t) {
                    const double al = t - s >= 0 ? -sa[t] / sb[t - s] : 0.0;
                    const double ga = t + s < m ? -sc[t] / sb[t + s] : 0.0;
                    o[st * 32 + t] = al;
                    o[(5 + st) * 32 + t] = ga;
                    na[t] = t - s >= 0 ? al * sa[t - s] : 0.0;
                    nc[t] = t + s < m ? ga * sc[t + s] : 0.0;
                    nb[t] = sb[t] + (t - s >= 0 ? al * sc[t - s] : 0.0) + (t + s < m ? ga * sa[t + s] : 0.0);
                }
                sa = na;
                sb = nb;
                sc = nc;
            }
            for (int t = 0; t < m; ++t) o[10 * 32 + t] = 1.0 / sb[t];
        }
}

cudaError_t small_setup_kernel()
{
    return cudaFuncSetAttribute(small_adi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

cudaError_t launch_small_adi(const SmallArgs &a, cudaStream_t st)
{
    small_adi_kernel<<<(unsigned)(kCl * a.nrhs), kThreads, kSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fps
