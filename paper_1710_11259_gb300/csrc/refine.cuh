// Kernels of the FP32-sweep / FP64-refinement solve, for one problem or a batch
// (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fps {

// Work decomposition of the FP32 passes for size n: columns in blocks of 32,
// each (column, parity) system cut into P segments of Ls rows.
struct RefineGeometry {
    int64_t ld = 0;      // padded leading dimension (multiple of 32)
    int64_t nblk = 0;    // column blocks
    int64_t nchunk = 0;  // checkpoint chunks per parity system
    int64_t Ls = 0;      // rows per segment (multiple of 32)
    int64_t P = 1;       // segments per system
};
// Geometry aiming at about `target_ctas` CTAs (column blocks x segments) per pass.
RefineGeometry refine_geometry(int64_t n, int target_ctas);
// Scratch per right-hand side: checkpoint floats and summary float2s.
int64_t refine_checkpoint_floats(const RefineGeometry &g);
int64_t refine_summary_float2(const RefineGeometry &g);

// One problem at one inner tolerance level (device-resident table entry).
struct RefProb {
    int n, ld, Ls, P, nchunk, J;
    int64_t off32, rhs32;   // FP32 arrays: element offset of rhs 0, stride between right-hand sides
    int64_t offck, rhsck;   // checkpoint scratch (floats)
    int64_t offsm, rhssm;   // summary scratch (float2)
    const float4 *fac;      // [J][n]      {ip, uf, lf, kappa}
    const float *phick;     // [J][2][nchunk]
    const float4 *segc;     // [J][2][P]   {Phi_end, Psi, B, 0}
    const float *q2;        // [J]         2 q_j
};

// One problem for the FP64 tile kernels (scale-in/out, residual).
struct RefProb64 {
    int n, ld;
    int64_t off64;          // caller/internal FP64 packing: element offset of rhs 0 (rhs stride n*n)
    int64_t off32, rhs32;   // FP32 packing (as RefProb)
    const double *d, *e, *s;  // bands of A~ (e zero-padded to n) and 1/sqrt(E)
    int pair0;              // index of (problem, rhs 0) among all (problem, rhs) pairs
};

// One shift of one problem for factor32 (computed on the device in FP64).
struct FactorJob {
    double q;
    int64_t n, Ls, P, nchunk;
    const double *d, *e;
    float4 *fac;
    float *phick;
    float4 *segc;
};

struct RefPassArgs {
    const RefProb *probs;   // table of one tolerance level
    const int4 *items;      // {problem, rhs, column block, segment}
    int64_t nitems;
    const int *active;      // per problem
    float *Pt, *A, *C, *D;  // rho^T, a, c, correction (FP32, packed)
    float *ck;
    float2 *summ;
};

struct RefTileArgs {
    const RefProb64 *probs;
    const int4 *tiles;      // {problem * 256 + rhs, tile column, tile row, 0}
    int64_t ntiles;
};

// Raise the dynamic shared-memory limits of the pass kernels (once per process).
cudaError_t refine_setup_kernels();

// Row pass of iteration j on rho^T: A = (R - q)^{-1} rho, C = rho + 2q A.
cudaError_t launch_row_pass(const RefPassArgs &a, int j, cudaStream_t st);

// Column pass of iteration j: Pt = (C + 2q (L-q)^{-1} C)^T, D -= 2q (L-q)^{-1} A
// (D = -2q (L-q)^{-1} A when first).  ev0/ev1, if given, are recorded around the
// back-substitution kernel (timing).
cudaError_t launch_col_pass(const RefPassArgs &a, int j, bool first, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                            cudaEvent_t ev1 = nullptr);

// Per (problem, rhs): smax = max |D_s F D_s| (bit patterns; must start at 0).
cudaError_t launch_absmax_tiles(const RefTileArgs &a, const double *F, unsigned long long *smax, cudaStream_t st);
// F~ = D_s F D_s, Pt = (F~ / smax)^T.
cudaError_t launch_scale_in_tiles(const RefTileArgs &a, const double *F, double *Ft, float *Pt,
                                  const unsigned long long *smax, cudaStream_t st);
// Yout = Y + smax D (Y read as zero if y_zero), R = F~ - A~ Yout - Yout A~, Pt = (R/smax)^T,
// rmax = max |R| per pair (bit patterns; must start at 0); pairs with pair_active = 0 skipped.
cudaError_t launch_residual_tiles(const RefTileArgs &a, const double *Y, double *Yout, const float *Dl,
                                  const double *Ft, float *Pt, const unsigned long long *smax,
                                  unsigned long long *rmax, const int *pair_active, bool y_zero, cudaStream_t st);
// X = D_s Y D_s.
cudaError_t launch_scale_out_tiles(const RefTileArgs &a, const double *Y, double *X, cudaStream_t st);
// FP32 factor tables for a list of (problem, shift) jobs.
cudaError_t launch_factors32(const FactorJob *jobs, int njobs, cudaStream_t st);

}  // namespace fps
