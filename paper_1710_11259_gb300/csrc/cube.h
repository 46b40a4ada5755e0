// Nested ADI for the cube (Sec. 5), FP64 (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace fps {

class CubeEngine {
public:
    // tol: outer ADI tolerance of (2.9); tol_mid / tol_in: the middle and inner
    // levels ("to machine precision", 1e-15 by default).
    int create(int64_t n, double tol, double tol_mid, double tol_in, std::string &err);
    void release();
    // X = solution of (5.2) for F (device pointers, n^3 row-major) on stream st.
    int solve_cube(const double *F, double *X, cudaStream_t st, std::string &err);

    int64_t bytes = 0;
    int J_outer = 0;
    int64_t inner_iters = 0;     // inner iterations over full tensors in the last solve
    int64_t launches_last = 0;

private:
    cudaError_t band(const double *X, const double *R, double *Y, int mode, double alpha, double beta, double sop,
                     double sr);
    cudaError_t axpby(const double *X, const double *Y, double *Z, double a, double b);
    cudaError_t solve(int set, const double *R1, double s1, const double *R2, double s2, double *X, int mode);
    int stein(int ma, int mb, double c, const double *R, double *Z, std::string &err);
    int hsolve(double s, const double *R, double *Y, std::string &err);

    int64_t n_ = 0;
    double tol_ = 0, tol_mid_ = 0, tol_in_ = 0, eps_ = 0;
    cudaStream_t st_ = nullptr;
    double *bd_ = nullptr, *be_ = nullptr, *bs_ = nullptr;
    double *work_[10] = {nullptr};
    double2 *fac_ = nullptr, *ab_ = nullptr, *h_ab_ = nullptr;
    int max_sets_ = 0;
    std::vector<double *> allocs_;
};

}  // namespace fps
