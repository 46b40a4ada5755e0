// Nested ADI for the cube (Sec. 5) (internal header).
//
// CubeNested<T> runs the three-level ADI of Sec. 5 in arithmetic T on the
// symmetrised tensor equation (T_01 + T_02 + T_12) Y = G; its schedule (every
// shift of every level) is fixed at plan time.  CubeEngine is the plan object:
// FP64 runs the nested ADI once at the requested tolerance (inner and middle
// levels to 1e-15); FP32 + refinement runs it in FP32 at loose tolerances, every
// level in residual-propagating form, inside an FP64 defect-correction loop on
// the residual G - (T_01 + T_02 + T_12) Y.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

namespace fps {

template <typename T>
class CubeNested {
public:
    // tol: outer tolerance of (2.9); tol_mid / tol_in: middle and inner levels;
    // residual: run every level in residual-propagating form (the FP32 rounds);
    // tight: every level's intervals from the Sturm-bisection interval of A~ instead
    // of Lemma B.2's [-1, -1/(30 n^4)].
    int create(int64_t n, double tol, double tol_mid, double tol_in, bool residual, bool tight, std::string &err);
    void release();
    // Y = the nested-ADI approximation of (T_01 + T_02 + T_12)^{-1} G (device tensors).
    int run(const T *G, T *Y, cudaStream_t st, std::string &err);

    int J_outer = 0;
    int64_t inner_per_run = 0;   // inner (slice Stein) iterations over full tensors per run
    int64_t launches = 0;        // kernel launches of the last run
    int64_t bytes = 0;

private:
    struct Stein {
        double c = 0;
        int J = 0;
        int64_t ab_off = 0;          // first (alpha, beta) set of this entry in the device table
        std::vector<double> p, q;
    };
    struct Middle {
        double a = 0;
        int stein = 0;
    };
    struct Outer {
        double p = 0, q = 0;
        int stein_v = 0;
        std::vector<Middle> mid;
    };
    cudaError_t band(const T *X, const T *R, T *Y, int mode, double alpha, double beta, double sop, double sr);
    cudaError_t axpby(const T *X, const T *Y, T *Z, double a, double b);
    cudaError_t axpy3(const T *X, const T *Y, const T *W, T *V, double a, double b, double c);
    // X = oscale * (alpha A~ + beta)^{-1} IN + oin * IN + oacc * X along `mode`, with
    // IN = s1 R1 + s2 R2, or IN = s1 A~ R1 along `mode` when preband
    cudaError_t solve(int set, const T *R1, double s1, const T *R2, double s2, T *X, int mode, double oscale,
                      double oacc, double oin, bool preband);
    int load_factors(int entry, std::string &err);
    int stein(int ma, int mb, int entry, const T *R, T *Z, std::string &err);
    int hsolve(const Outer &o, const T *R, T *Y, std::string &err);
    int stein_res(int ma, int mb, int entry, const T *R1, double r1, const T *R2, double r2, T *Z, bool accumulate,
                  std::string &err);
    int hsolve_res(const Outer &o, const T *R, T *W, std::string &err);
    int run_residual(const T *G, T *Y, std::string &err);
    int add_stein(double c);

    int64_t n_ = 0;
    double tol_ = 0, tol_mid_ = 0, tol_in_ = 0;
    double lo_ = 0, hi_ = 1;     // sigma(A~) in [-hi_, -lo_]
    bool residual_ = false;
    cudaStream_t st_ = nullptr;
    double *bd64_ = nullptr, *be64_ = nullptr;
    T *bd_ = nullptr, *be_ = nullptr;
    T *work_[9] = {nullptr};
    void *fac_ = nullptr;        // factor sets of the current Stein entry ({1/den, u} in T)
    double2 *ab_ = nullptr;      // (alpha, beta) of every factor set of every Stein entry
    int fac_entry_ = -1;         // entry whose factors fac_ holds (stream order makes reuse safe)
    bool slice_ = false;         // FP32 inner solves by the slice-resident cluster kernel
    int max_sets_ = 0;
    std::vector<Stein> steins_;
    std::vector<Outer> outer_;
    std::vector<void *> allocs_;
};

class CubeEngine {
public:
    // precision: FPS_FP64 or FPS_FP32_REFINE (fps.h).
    int create(int64_t n, double tol, int precision, std::string &err);
    void release();
    // X = solution of (5.2) for F (device pointers, n^3 row-major) on stream st.
    int solve_cube(const double *F, double *X, cudaStream_t st, std::string &err);

    int64_t bytes = 0;
    int J_outer = 0;
    int J_outer_inner = 0;       // FP32 + refinement: J of the outer level inside a round
    int64_t inner_iters = 0;     // inner iterations over full tensors in the last solve
    int64_t launches_last = 0;
    int rounds_last = 0;
    double resid_last = 0.0;     // max|G - T Y| / max|G| after the last solve (FP32 + refinement)
    int max_rounds = 12;

    // Level tolerances of the FP32 rounds: middle and inner fixed; the outer one is
    // picked per plan from kRefTolOuter (refinement_outer_tol).
    static constexpr double kRefTolMid = 1e-6, kRefTolIn = 1e-7;
    static constexpr double kRefTolOuter[] = {1e-3, 7e-4, 5e-4, 3e-4, 2e-4, 1e-4};
    double ref_tol_outer = 1e-3;  // outer tolerance of the FP32 rounds in use

private:
    int64_t n_ = 0;
    double tol_ = 0;
    int precision_ = 0;
    CubeNested<double> *n64_ = nullptr;
    CubeNested<float> *n32_ = nullptr;
    double *bd_ = nullptr, *be_ = nullptr, *bs_ = nullptr;
    double *G_ = nullptr, *Y_ = nullptr, *R_ = nullptr;
    float *rho_ = nullptr, *delta_ = nullptr;
    unsigned long long *d_max_ = nullptr, *h_max_ = nullptr;
    std::vector<void *> allocs_;
};

}  // namespace fps
