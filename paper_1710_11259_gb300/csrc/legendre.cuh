// Legendre coefficients in and out of the square solve (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fps {

// F (n x n) = C~ coefficients of sum G_ab P_a(y) P_b(x) (device pointers).
cudaError_t launch_legendre_to_ctilde(const double *G, double *F, int64_t n, cudaStream_t st);
// U ((n+2) x (n+2)) = Legendre coefficients of (1-x^2)(1-y^2) sum X_ij C~_i(y) C~_j(x).
cudaError_t launch_solution_to_legendre(const double *X, double *U, int64_t n, cudaStream_t st);
// Transposes of the two maps (gradients through them): Gbar = B^T Fbar B (n x n) and
// Xbar (n x n) = L^T Ubar L for Ubar ((n+2) x (n+2)).
cudaError_t launch_legendre_to_ctilde_adjoint(const double *Fbar, double *Gbar, int64_t n, cudaStream_t st);
cudaError_t launch_solution_to_legendre_adjoint(const double *Ubar, double *Xbar, int64_t n, cudaStream_t st);

}  // namespace fps
