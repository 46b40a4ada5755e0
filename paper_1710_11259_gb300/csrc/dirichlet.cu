// Nonhomogeneous Dirichlet data (Sec. 6.1): the four steps around the homogeneous
// solve, in Legendre coefficients of the mapped variables x, y in [-1, 1].
//   1. u_bc = the transfinite (Coons) interpolant of the traces g_W, g_E, g_S, g_N:
//        u_bc = (1-x)/2 g_W(y) + (1+x)/2 g_E(y) + (1-y)/2 g_S(x) + (1+y)/2 g_N(x)
//               - sum over corners c(sx, sy) (1 + sx x)/2 (1 + sy y)/2,
//      c(sx, sy) the mean of the two traces meeting at the corner.  With
//      (1 -+ t)/2 = P_0/2 -+ P_1/2 its coefficients X_bc live in rows and columns 0, 1.
//   2. lap u_bc = ky [(1-x)/2 g_W'' + (1+x)/2 g_E''] + kx [(1-y)/2 g_S'' + (1+y)/2 g_N'']
//      (the bilinear part is harmonic): again rows and columns 0, 1 only.
//   3. F = B (G - lap u_bc) B^T, and since B is upper triangular with bands 0 and +2,
//      the correction B lap B^T touches rows and columns 0, 1 of F only.
//   4. U = (solution map) + X_bc.
// The second derivative of a Legendre series c has coefficients
//   c''_k = (k + 1/2) sum_{j >= k+2, j - k even} [j(j+1) - k(k+1)] c_j,
// (twice the derivative rule P_j' = sum_{l < j, j - l odd} (2l+1) P_l, with
// sum_{l = k+1, k+3, .., j-1} (2l+1) = [j(j+1) - k(k+1)]/2), so per parity it is two
// suffix sums: of c_j and of j(j+1) c_j.  Its transpose is two prefix sums.  One
// block per (right-hand side, trace, parity) forms them: every thread sums a
// contiguous chunk, one thread scans the 256 chunk totals, and every thread walks
// its chunk again.  All of this is O(n) per right-hand side next to the O(n^2 log^2 n)
// solve; the bulk maps are the Legendre conversions and the solve itself.
#include "dirichlet.cuh"

namespace fps {

namespace {

constexpr int kScanThreads = 256;

// Chunk of the parity sequence idx_r = p + 2 r (r < R) that thread t walks.
struct Chunk {
    int64_t lo, hi;
};
__device__ __forceinline__ Chunk chunk_of(int64_t R, int t)
{
    const int64_t C = (R + kScanThreads - 1) / kScanThreads;
    const int64_t lo = (int64_t)t * C < R ? (int64_t)t * C : R;
    return {lo, lo + C < R ? lo + C : R};
}

// Exclusive scan (ascending = prefix, else suffix) of the per-thread pairs; returns
// this thread's offset and leaves the block total in *total.
__device__ double2 block_scan2(double2 v, bool ascending, double2 *total)
{
    __shared__ double2 part[kScanThreads + 1];
    part[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 run = make_double2(0.0, 0.0);
        for (int i = 0; i < kScanThreads; ++i) {
            const int t = ascending ? i : kScanThreads - 1 - i;
            const double2 x = part[t];
            part[t] = run;
            run.x += x.x;
            run.y += x.y;
        }
        part[kScanThreads] = run;
    }
    __syncthreads();
    const double2 r = part[threadIdx.x];
    *total = part[kScanThreads];
    __syncthreads();
    return r;
}

// blockIdx.x = (r * 4 + side) * 2 + parity
__global__ void __launch_bounds__(kScanThreads) dirichlet_prep_kernel(const double *__restrict__ bc,
                                                                      double *__restrict__ d2,
                                                                      double *__restrict__ tsum, int64_t n)
{
    const int64_t m = n + 2;
    const int p = blockIdx.x & 1;
    const int64_t trace = blockIdx.x >> 1;  // r * 4 + side
    const double *c = bc + trace * m;
    double *out = d2 + trace * n;
    const int64_t R = (m - p + 1) / 2;      // indices p, p+2, .. < m
    const Chunk ch = chunk_of(R, threadIdx.x);
    double2 s = make_double2(0.0, 0.0);     // {sum c_j, sum j(j+1) c_j}
    for (int64_t r = ch.lo; r < ch.hi; ++r) {
        const int64_t j = p + 2 * r;
        const double cj = c[j], J = (double)j;
        s.x += cj;
        s.y = fma(J * (J + 1.0), cj, s.y);
    }
    double2 tot;
    double2 suf = block_scan2(s, false, &tot);  // sums over the chunks above this one
    if (threadIdx.x == 0) tsum[trace * 2 + p] = tot.x;
    for (int64_t r = ch.hi - 1; r >= ch.lo; --r) {
        const int64_t k = p + 2 * r;  // suf holds the sums over j >= k + 2
        if (k < n) {
            const double K = (double)k;
            out[k] = (K + 0.5) * fma(-K * (K + 1.0), suf.x, suf.y);
        }
        const double ck = c[k], K = (double)k;
        suf.x += ck;
        suf.y = fma(K * (K + 1.0), ck, suf.y);
    }
}

// B[j][j] and B[j][j+2] of the Legendre -> C~ map (n x n, truncated at n).
__device__ __forceinline__ double b_diag(int64_t j)
{
    const double J = (double)j;
    return 1.0 / ((2.0 * J + 1.0) * sqrt((J + 1.5) / ((J + 1.0) * (J + 2.0))));
}
__device__ __forceinline__ double b_off(int64_t j)
{
    const double J = (double)j;
    return -1.0 / ((2.0 * J + 5.0) * sqrt((J + 1.5) / ((J + 1.0) * (J + 2.0))));
}

// The four Laplacian vectors of step 2 at index a (< n):
//   col0 = ky (W'' + E'')/2, col1 = ky (E'' - W'')/2   (columns 0, 1 of lap u_bc)
//   row0 = kx (S'' + N'')/2, row1 = kx (N'' - S'')/2   (rows 0, 1)
struct LapVec {
    const double *W, *E, *S, *N;
    double kx, ky;
    __device__ double col(int which, int64_t a) const
    {
        return which == 0 ? 0.5 * ky * (W[a] + E[a]) : 0.5 * ky * (E[a] - W[a]);
    }
    __device__ double row(int which, int64_t b) const
    {
        return which == 0 ? 0.5 * kx * (S[b] + N[b]) : 0.5 * kx * (N[b] - S[b]);
    }
};

// (B v)[i] for one of the Laplacian vectors (n x n B: the +2 band stops at n).
template <typename Fn>
__device__ __forceinline__ double b_apply(Fn v, int64_t i, int64_t n)
{
    double r = b_diag(i) * v(i);
    if (i + 2 < n) r = fma(b_off(i), v(i + 2), r);
    return r;
}

// Thread t (< n) of right-hand side blockIdx.y owns F[t][0], F[t][1] and, for t >= 2,
// F[0][t], F[1][t]:  B lap B^T = B[0][0] (B col0) e_0^T + B[1][1] (B col1) e_1^T
//                             + B[0][0] e_0 (B row0)^T + B[1][1] e_1 (B row1)^T.
__global__ void dirichlet_rhs_kernel(double *__restrict__ F, const double *__restrict__ d2, int64_t n, double kx,
                                     double ky)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t r = blockIdx.y;
    double *Fr = F + r * n * n;
    const double *base = d2 + r * 4 * n;
    const LapVec L{base, base + n, base + 2 * n, base + 3 * n, kx, ky};
    const double b0 = b_diag(0), b1 = b_diag(1);
    for (int c = 0; c < 2 && c < n; ++c) {  // column part at (t, c)
        const double bc_ = c == 0 ? b0 : b1;
        double v = bc_ * b_apply([&](int64_t a) { return L.col(c, a); }, t, n);
        if (t < 2) v = fma(t == 0 ? b0 : b1, b_apply([&](int64_t b) { return L.row((int)t, b); }, c, n), v);
        Fr[t * n + c] -= v;
    }
    if (t >= 2)
        for (int rr = 0; rr < 2 && rr < n; ++rr)  // row part at (rr, t)
            Fr[rr * n + t] -= (rr == 0 ? b0 : b1) * b_apply([&](int64_t b) { return L.row(rr, b); }, t, n);
}

// Corner values c(sx, sy) (index (sx > 0) * 2 + (sy > 0)) from the coefficient sums.
__device__ __forceinline__ void corners(const double *ts, double c[4])
{
    auto val = [&](int side, int s) {
        return s > 0 ? ts[2 * side] + ts[2 * side + 1] : ts[2 * side] - ts[2 * side + 1];
    };
    c[0] = 0.5 * (val(0, -1) + val(2, -1));  // (-1, -1): g_W(-1), g_S(-1)
    c[1] = 0.5 * (val(0, 1) + val(3, -1));   // (-1, +1): g_W(1),  g_N(-1)
    c[2] = 0.5 * (val(1, -1) + val(2, 1));   // (+1, -1): g_E(-1), g_S(1)
    c[3] = 0.5 * (val(1, 1) + val(3, 1));    // (+1, +1): g_E(1),  g_N(1)
}

// Coefficient i (0 or 1) of the linear factor (1 + s t)/2: {1/2, s/2}.
__device__ __forceinline__ double lin(int s, int i) { return i == 0 ? 0.5 : 0.5 * (double)s; }

// Bilinear interpolant of the corner values, coefficient (i, j) (degree i in y, j in x).
__device__ __forceinline__ double bilinear(const double c[4], int i, int j)
{
    double v = 0.0;
    for (int sx = 0; sx < 2; ++sx)
        for (int sy = 0; sy < 2; ++sy) v = fma(c[sx * 2 + sy], lin(sy ? 1 : -1, i) * lin(sx ? 1 : -1, j), v);
    return v;
}

// Thread t (< n + 2) owns U[t][0], U[t][1] and, for t >= 2, U[0][t], U[1][t].
__global__ void dirichlet_lift_kernel(double *__restrict__ U, const double *__restrict__ bc,
                                      const double *__restrict__ tsum, int64_t n)
{
    const int64_t m = n + 2;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int64_t r = blockIdx.y;
    double *Ur = U + r * m * m;
    const double *g = bc + r * 4 * m;
    const double *W = g, *E = g + m, *S = g + 2 * m, *N = g + 3 * m;
    double c[4];
    corners(tsum + r * 8, c);
    Ur[t * m + 0] += 0.5 * (W[t] + E[t]);
    Ur[t * m + 1] += 0.5 * (E[t] - W[t]);
    if (t < 2) {
        for (int j = 0; j < 2; ++j) {
            const double row = t == 0 ? 0.5 * (S[j] + N[j]) : 0.5 * (N[j] - S[j]);
            Ur[t * m + j] += row - bilinear(c, (int)t, j);
        }
    } else {
        Ur[t] += 0.5 * (S[t] + N[t]);
        Ur[m + t] += 0.5 * (N[t] - S[t]);
    }
}

// blockIdx.x = (r * 4 + side) * 2 + parity.  bcbar_side[j] (j = p, p+2, .. < n+2):
//   lift^T:  the linear factors read Ubar's columns (W, E) or rows (S, N) 0 and 1, and
//            every corner value c = (g_a(s_a) + g_b(s_b))/2 passes cbar/2 * s^j on,
//            cbar(sx, sy) = -sum_{i,j < 2} Ubar[i][j] lin(sy, i) lin(sx, j);
//   -lap^T:  v = d<Gbar, lap>/d g'' (length n), and
//            (D2^T v)_j = sum_{k <= j-2, k = j mod 2} (k + 1/2)[j(j+1) - k(k+1)] v_k
//                       = j(j+1) P1 - P2,  P1 = sum (k + 1/2) v_k,  P2 = sum (k + 1/2) k(k+1) v_k.
__global__ void __launch_bounds__(kScanThreads) dirichlet_bc_adjoint_kernel(const double *__restrict__ Ub,
                                                                            const double *__restrict__ Gb,
                                                                            double *__restrict__ bcb, int64_t n,
                                                                            double kx, double ky)
{
    const int64_t m = n + 2;
    const int p = blockIdx.x & 1;
    const int64_t trace = blockIdx.x >> 1;
    const int side = (int)(trace & 3);
    const int64_t r = trace >> 2;
    const double *Ur = Ub + r * m * m, *Gr = Gb + r * n * n;
    double *out = bcb + trace * m;
    double cb[4];  // cbar per corner, same indexing as corners()
    for (int sx = 0; sx < 2; ++sx)
        for (int sy = 0; sy < 2; ++sy) {
            double v = 0.0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j)
                    v = fma(Ur[i * m + j], lin(sy ? 1 : -1, i) * lin(sx ? 1 : -1, j), v);
            cb[sx * 2 + sy] = -v;
        }
    // the corner terms of this trace: {coefficient at s = -1, at s = +1}
    double cm1, cp1;
    switch (side) {
    case 0: cm1 = cb[0]; cp1 = cb[1]; break;   // W: (-1,-1) at y = -1, (-1,+1) at y = +1
    case 1: cm1 = cb[2]; cp1 = cb[3]; break;   // E
    case 2: cm1 = cb[0]; cp1 = cb[2]; break;   // S: (-1,-1) at x = -1, (+1,-1) at x = +1
    default: cm1 = cb[1]; cp1 = cb[3]; break;  // N
    }
    // v_side[k] (k < n)
    auto vk = [&](int64_t k) {
        auto G = [&](int64_t a, int64_t b) { return (a < n && b < n) ? Gr[a * n + b] : 0.0; };
        switch (side) {
        case 0: return 0.5 * ky * (G(k, 0) - G(k, 1));
        case 1: return 0.5 * ky * (G(k, 0) + G(k, 1));
        case 2: return 0.5 * kx * (G(0, k) - G(1, k));
        default: return 0.5 * kx * (G(0, k) + G(1, k));
        }
    };
    const int64_t R = (m - p + 1) / 2;
    const Chunk ch = chunk_of(R, threadIdx.x);
    double2 s = make_double2(0.0, 0.0);
    for (int64_t q = ch.lo; q < ch.hi; ++q) {
        const int64_t k = p + 2 * q;
        if (k >= n) break;
        const double K = (double)k, w = (K + 0.5) * vk(k);
        s.x += w;
        s.y = fma(K * (K + 1.0), w, s.y);
    }
    double2 tot;
    double2 pre = block_scan2(s, true, &tot);  // sums over k in the chunks below
    const double sgn = p ? -1.0 : 1.0;          // (-1)^j
    for (int64_t q = ch.lo; q < ch.hi; ++q) {
        const int64_t j = p + 2 * q;
        const double J = (double)j;
        double lift;
        if (side < 2) {
            const double u0 = Ur[j * m], u1 = Ur[j * m + 1];
            lift = side == 0 ? 0.5 * (u0 - u1) : 0.5 * (u0 + u1);
        } else {
            const double u0 = Ur[j], u1 = Ur[m + j];
            lift = side == 2 ? 0.5 * (u0 - u1) : 0.5 * (u0 + u1);
        }
        lift += 0.5 * (sgn * cm1 + cp1);
        out[j] = lift - fma(J * (J + 1.0), pre.x, -pre.y);  // pre: k <= j - 2
        if (j < n) {
            const double w = (J + 0.5) * vk(j);
            pre.x += w;
            pre.y = fma(J * (J + 1.0), w, pre.y);
        }
    }
}

}  // namespace

cudaError_t launch_dirichlet_prep(const double *bc, double *d2, double *tsum, int64_t n, int nrhs, cudaStream_t st)
{
    dirichlet_prep_kernel<<<nrhs * 8, kScanThreads, 0, st>>>(bc, d2, tsum, n);
    return cudaGetLastError();
}

cudaError_t launch_dirichlet_rhs(double *F, const double *d2, int64_t n, int nrhs, double kx, double ky,
                                 cudaStream_t st)
{
    const dim3 grid((unsigned)((n + 255) / 256), (unsigned)nrhs);
    dirichlet_rhs_kernel<<<grid, 256, 0, st>>>(F, d2, n, kx, ky);
    return cudaGetLastError();
}

cudaError_t launch_dirichlet_lift(double *U, const double *bc, const double *tsum, int64_t n, int nrhs,
                                  cudaStream_t st)
{
    const dim3 grid((unsigned)((n + 2 + 255) / 256), (unsigned)nrhs);
    dirichlet_lift_kernel<<<grid, 256, 0, st>>>(U, bc, tsum, n);
    return cudaGetLastError();
}

cudaError_t launch_dirichlet_bc_adjoint(const double *Ubar, const double *Gbar, double *bcbar, int64_t n, int nrhs,
                                        double kx, double ky, cudaStream_t st)
{
    dirichlet_bc_adjoint_kernel<<<nrhs * 8, kScanThreads, 0, st>>>(Ubar, Gbar, bcbar, n, kx, ky);
    return cudaGetLastError();
}

}  // namespace fps
