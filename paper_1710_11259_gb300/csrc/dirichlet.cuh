// Nonhomogeneous Dirichlet data around the square / rectangle solve (Sec. 6.1),
// internal header.  Layouts (device, FP64, per right-hand side r):
//   bc    [r][4][n+2]  Legendre coefficients of the traces g_W = u(-1, y),
//                      g_E = u(1, y), g_S = u(x, -1), g_N = u(x, 1) (mapped variables)
//   d2    [r][4][n]    Legendre coefficients of g'' for every trace
//   tsum  [r][4][2]    sums of the even- and odd-degree coefficients of each trace
//                      (g(1) = even + odd, g(-1) = even - odd)
//   F     [r][n][n]    C~ coefficients of the right-hand side (row = degree in y)
//   U     [r][n+2][n+2] Legendre coefficients of the solution
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fps {

// Second derivatives and coefficient sums of all traces.
cudaError_t launch_dirichlet_prep(const double *bc, double *d2, double *tsum, int64_t n, int nrhs, cudaStream_t st);
// F <- F - B (kx u_bc,xx + ky u_bc,yy) B^T, after F = B G B^T (rows and columns 0, 1 only).
cudaError_t launch_dirichlet_rhs(double *F, const double *d2, int64_t n, int nrhs, double kx, double ky,
                                 cudaStream_t st);
// U <- U + X_bc, the Coons lifting of the traces (rows and columns 0, 1 only).
cudaError_t launch_dirichlet_lift(double *U, const double *bc, const double *tsum, int64_t n, int nrhs,
                                  cudaStream_t st);
// bcbar = lift^T(Ubar) - lap^T(Gbar): the gradient in the traces, given dL/dU and the
// gradient dL/dG already formed.
cudaError_t launch_dirichlet_bc_adjoint(const double *Ubar, const double *Gbar, double *bcbar, int64_t n, int nrhs,
                                        double kx, double ky, cudaStream_t st);

}  // namespace fps
