// Cylinder Fourier modes |k| >= 2 (Sec. 4.1, Case 1), internal header.
//
// For each mode k the coefficients Y of w_k(r, z) = sum Y_ij C~_i(r) C~_j(z), where
// u_k = r^2 (1 - r^2)(1 - z^2) w_k, satisfy
//     P Y M^T + Q Y D = F,    P = L1 - k^2 M,  Q = M_{r^2} M = M - M^2,
// i.e. A Y - Y B = P^{-1} F D^{-1} with A = P^{-1} Q, B = -M D^{-1}.  The ADI of
// Algorithm 2 on that form, multiplied through by P so that no P^{-1} is applied:
//     W (B - p_j)       = (Q - p_j P) X_j - G,          W = P X_{j+1/2},  G = F D^{-1},
//     (Q - q_j P) X_{j+1} = W (B - q_j) + G,
// with (B - p) = -(M + p D) D^{-1}.  Along z (the second index) every step is a
// symmetric tridiagonal solve or product per parity (M + p D); along r (the first
// index) a pentadiagonal-per-parity solve (Q - q P, non-symmetric, LU without
// pivoting) and product (Q - p P).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace fps {

// Band entries of the operators in the normalised C~ basis (any index j >= 0).
double cyl_M_diag(int64_t j);
double cyl_M_off(int64_t j);      // M[j][j+2] = M[j+2][j]
double cyl_L1(int64_t a, int64_t i);  // L1[a][i] (zero unless |a - i| in {0, 2})
// Interval [a, b] (a < b < 0) containing the eigenvalues of A_k = P^{-1} Q for the
// n x n blocks, by power iteration on A_k and on A_k^{-1} per parity, widened by 3 %.
int cyl_mode_interval(int64_t n, int64_t k, double &a, double &b);

struct CylTables;

class CylinderEngine {
public:
    int create(int64_t n, int64_t kmin, int64_t kmax, double tol, int nrhs, std::string &err);
    void release();
    // F, Y: device, [kmax - kmin + 1][nrhs][n][n] row-major (row index = degree in r).
    int solve(const double *F, double *Y, cudaStream_t st, std::string &err);

    int64_t n = 0, kmin = 0, kmax = 0;
    int nrhs = 1, Jmax = 0;
    std::vector<int> J;             // per mode
    std::vector<double> a, b;       // sigma(A_k) intervals
    double lo = 0, hi = 0;          // sigma(B) interval
    int64_t bytes = 0;
    int64_t launches_last = 0;

private:
    std::vector<void *> allocs_;
    double *G_ = nullptr, *R1_ = nullptr, *R2_ = nullptr;
    double *bands_ = nullptr;       // [7][n + 4]: Md, Me, D, L1d, L1u (a = i - 2), L1l (a = i + 2), Q4
    double2 *zfac_ = nullptr;       // [sum J][n] {1/den, u} of (M + p D)
    double *rfac_ = nullptr;        // [sum J][n][6] LU of (Q - q P): {l1, l2, 1/u0, u1, u2, -}
    double *shifts_ = nullptr;      // [modes][Jmax][2] {p_j, q_j}
    int *joff_ = nullptr;           // [modes] offset of the mode's first iteration in the tables
    int *jcount_ = nullptr;         // [modes] J
    template <typename U>
    cudaError_t dalloc(U **p, size_t count);
};

}  // namespace fps
