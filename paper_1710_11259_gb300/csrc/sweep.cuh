// ADI pass kernels of the square solve, for one problem or a batch (internal header).
//
// Every ADI iteration j of Algorithm 2 (on the symmetric equation (3.9), shifts
// q_j > 0) is run in residual-propagating form,
//     c_j = (L - q_j)^{-1} (R - q_j)^{-1} rho_j,
//     D  <- D - 2 q_j c_j,                  rho_{j+1} = (L + q_j)(R + q_j) c_j,
// with L(Y) = A~ Y (along columns) and R(Y) = Y A~ (along rows); D after J
// iterations is the ADI iterate Y_J of the paper's form started from Y_0 = 0 with
// right-hand side rho_0 (the two forms agree term by term in exact arithmetic).
// On a rectangle the equation is kx A~ Y + ky Y A~ = F~ with shifts p_j (row side)
// and q_j (column side) of App. A's general intervals; the same steps then read
//     c_j = (L - q_j/kx)^{-1} (R + p_j/ky)^{-1} rho_j,
//     D  <- D - (q_j - p_j)/(kx ky) c_j,    rho_{j+1} = (L - p_j/kx)(R + q_j/ky) c_j,
// (the scalars kx, ky of the solves and the stencils cancel), so the kernels only
// see two solve shifts, two stencil shifts and one correction factor per iteration.
//
// Each banded solve is split into the two tridiagonals of App. B (even and odd
// indices) and every tridiagonal into segments of S positions.  A pass solves its
// segments independently ("local" solutions: forward sweep started from zero,
// back substitution ended at zero).  With the pivots of A~ - qI and
//     w_i = ip_i r_i - g_i w_{i-2}        (forward, g_i = e_{i-2} ip_i)
//     x_i = w_i - uf_i x_{i+2}            (back substitution, uf_i = e_i ip_i)
// the true solution in a segment is
//     x_i = xl_i + Bv_i zin + Psi_i xout,
// where zin is the true forward value just before the segment, xout the true
// solution just after it, and Bv, Psi depend only on the shift (tables below).
// zin and xout of every segment follow from a two-sweep recurrence over the
// segment summaries (wl at the segment end, xl at its start): the chain kernels.
// The correction is applied lazily by the NEXT pass when it loads the data, so
// every pass reads its input once and writes its output once:
//   row pass j     reads cl_{j-1} (+ halo), rebuilds c_{j-1}, D -= 2q_{j-1} c_{j-1},
//                  rho_j = (L+q_{j-1})(R+q_{j-1}) c_{j-1}, row-local solve -> al_j
//   row chain j    zin/xout of the row segments
//   column pass j  reads al_j, rebuilds a_j, column-local solve -> cl_j
//   column chain j zin/xout of the column segments
// (j = 0: the row pass reads rho_0 itself).  A finalize kernel adds the last c.
//
// Storage (type T = float or double): every n x n array of a (problem, rhs) is
// padded to N = 64 * ceil(n/64) positions per side plus a halo of 2 rows and 4
// columns on each side, row-major with leading dimension ldp = N + 8; element
// (i, k) sits at (i + 2) * ldp + (k + 4).  Padding is zero and stays zero.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fps {

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// Per-position coefficients of one shift (position i at index i + 2 of a table of
// N + 4 records; the two records on each side and positions >= n are zero).
template <typename T>
struct alignas(16) Fac {
    T ip, g, uf;   // pivot reciprocal, forward multiplier, back-substitution multiplier
    T phi;         // prod of -g from the segment start to i (forward propagation of zin)
    T Bv, Psi;     // coefficients of zin and xout in the true solution at i
    T pad0, pad1;  // 8-word records: the first four words load as 16-byte vectors
};

// One problem at one tolerance level (device table entry).
template <typename T>
struct SwProb {
    int n, S, P, N, ldp, J;
    int64_t off, rhs;      // element offset of rhs 0 / stride between right-hand sides (T arrays)
    int64_t soff, srhs;    // the same for the segment arrays ([P][2][N + 8] entries)
    const Fac<T> *facR;    // [J][N + 4] tables of the row solves (shift -p_j / ky)
    const Fac<T> *facC;    // [J][N + 4] tables of the column solves (shift q_j / kx); == facR on a square
    const T *sh;           // [J][3]: {column-stencil shift -p_j/kx, row-stencil shift q_j/ky,
                           //          correction factor -(q_j - p_j)/(kx ky)}; square: {q, q, -2q}
    const T *d, *e;        // bands of A~ at index i + 2, zero outside [0, n)
};

template <typename T>
struct SwArgs {
    using T2 = typename Vec2<T>::type;
    const SwProb<T> *probs;
    const int4 *items;     // row/column pass: {problem, rhs, block of 64 rows/columns, segment}
                           // chain: {problem, rhs, block of 64 lines, 0}
    int64_t nitems;
    const int *active;     // per problem
    T *rho0, *cl, *al, *D;
    T2 *sumR, *sumC;       // segment summaries {wl_end, xl_start}
    T2 *zxR, *zxC;         // chain results {zin, xout}
    T *zin;                // chain scratch ([P][2][N + 8] per rhs)
    int *err;              // device error word: bit 0 = a bounded wait gave up
    int S;                 // segment length of every problem (sweep_segment_supported)
    int chain_mode;        // chain kernel loads: 0 = by grid size, 1 = short batches, 2 = long batches
};

// Elementwise tile kernels of the solve around the ADI loop.  A tile item is
// {problem * 256 + rhs, tile column, tile row, 0} over the n x n region in 32 x 32 tiles.
struct TileProb {
    int n, ldp;
    int64_t off64;          // FP64 packing of the caller's arrays: offset of rhs 0 (rhs stride n*n)
    int64_t off, rhs;       // padded T arrays (as SwProb)
    const double *d, *e, *s;  // FP64 bands of A~ (d, e zero-padded to length n) and 1/sqrt(E)
    int pair0;              // index of (problem, rhs 0) among all pairs
    double kx, ky;          // scales of the two second derivatives (1, 1 on [-1,1]^2)
};

struct TileArgs {
    const TileProb *probs;
    const int4 *tiles;
    int64_t ntiles;
};

// Shift tables of a list of (problem, shift) jobs, computed in FP64.
template <typename T>
struct FacJob {
    double q;
    int n, N, S;
    const double *d, *e;   // FP64 bands, e zero-padded to length n
    Fac<T> *out;           // N + 4 records
};

cudaError_t sweep_setup_kernels();
// Segment lengths with compiled pass kernels: 64 (FP32, FP64) and 128 (FP32).
bool sweep_segment_supported(bool fp64, int S);

template <typename T>
cudaError_t launch_fac_tables(const FacJob<T> *jobs, int njobs, cudaStream_t st);

// Row pass of iteration j over the items (mode 0: j = 0 reads rho0; mode 1: j = 1,
// D = -2q c; mode 2: D -= 2q c).
template <typename T>
cudaError_t launch_row_pass(const SwArgs<T> &a, int j, int mode, cudaStream_t st);
template <typename T>
cudaError_t launch_col_pass(const SwArgs<T> &a, int j, cudaStream_t st);
// Chains of the row (dir 0) or column (dir 1) segments of iteration j.
template <typename T>
cudaError_t launch_chain(const SwArgs<T> &a, int dir, int j, cudaStream_t st);

// D <- D - 2 q_{J-1} c_{J-1} (or D = -2q c when J = 1) over the n x n region of every
// (problem, rhs) pair with pair_active set.
template <typename T>
cudaError_t launch_finalize(const TileArgs &t, const SwArgs<T> &a, const int *pair_active, cudaStream_t st);
// X = D_s (D - 2 q_{J-1} c_{J-1}) D_s straight into the caller's FP64 X.
cudaError_t launch_finalize_out(const TileArgs &t, const SwArgs<double> &a, double *X, cudaStream_t st);

// Per (problem, rhs): smax = max |D_s F D_s| (bit patterns; must start at 0).
cudaError_t launch_absmax(const TileArgs &t, const double *F, unsigned long long *smax, cudaStream_t st);
// F~ = D_s F D_s (FP64, if Ft != nullptr) and rho0 = F~ / smax (T, padded; smax == nullptr: no scaling).
template <typename T>
cudaError_t launch_scale_in(const TileArgs &t, const double *F, double *Ft, T *rho0, const unsigned long long *smax,
                            cudaStream_t st);
// Yout = Y + smax D (Y read as zero if y_zero), R = F~ - A~ Yout - Yout A~, rho0 = R / smax,
// rmax = max |R| per pair (bit patterns; must start at 0); inactive pairs copy Y.
cudaError_t launch_residual(const TileArgs &t, const double *Y, double *Yout, const float *D, const double *Ft,
                            float *rho0, const unsigned long long *smax, unsigned long long *rmax,
                            const int *pair_active, bool y_zero, cudaStream_t st);
// X = D_s Y D_s.
cudaError_t launch_scale_out(const TileArgs &t, const double *Y, double *X, cudaStream_t st);

}  // namespace fps
