// Host side of the square solve on the ADI pass kernels of sweep.cu, for one
// problem or a batch of squares of different sizes (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sweep.cuh"

namespace fps {

// T = float: FP32 sweeps inside an FP64 iterative refinement (tolerance levels,
//            residual R~ = F~ - A~Y - YA~ in FP64, Y += max|R~| D).
// T = double: the plain FP64 method, J iterations of (2.9) at the plan's tolerance.
template <typename T>
class SweepEngine {
public:
    // `ns`: problem sizes (caller packing: problem after problem, each problem's nrhs
    // n x n matrices back to back).  `tight`: shifts from the Sturm-bisection interval
    // of A~ instead of Lemma B.2's.  `seg`: segment length of the partitioned sweeps
    // (64 or 128 for FP32, 64 for FP64); seg <= 0 lets the autotuner pick it (FP32).
    // Returns an fps_status; on error `err` holds a message.
    // kx, ky: scales of the second derivatives along x and y (a kx^{-1/2} x ky^{-1/2}
    // rectangle of half-widths; 1, 1 on [-1,1]^2).
    int create(const std::vector<int64_t> &ns, int nrhs, double tol, bool tight, cudaStream_t setup_stream,
               std::string &err, int seg = 0, double kx = 1.0, double ky = 1.0);
    void release();

    // Solve for device pointers F, X (packed as above) on stream st.  FP32: returns
    // FPS_ERR_NOT_CONVERGED with the last iterate in X when the refinement misses tol.
    int solve(const double *F, double *X, cudaStream_t st, std::string &err);

    int set_instrument(bool on, std::string &err);
    // ADI pass kernels (row and column passes) of the last solve: launches, summed
    // duration, and the bytes they must move (sweep.cuh's residual form: 6 words per
    // element and iteration, 4 in the first two iterations).
    int kernel_times(int *count, double *total_ms, double *alg_bytes, double *row_ms, double *col_ms,
                     std::string &err);

    int64_t bytes = 0;
    int J_first = 0;             // iterations of the finest level for the largest problem
    int rounds_last = 0;
    double resid_last = 0.0;     // largest max|R~|/max|F~| after the last solve (FP32)
    int64_t launches_last = 0;
    int max_rounds = 8;
    std::vector<std::vector<double>> shifts;  // level-0 shifts per problem
    int seg_len = 0;                          // segment length in use
    int chain_mode = 0;                       // chain kernel load batching (SwArgs::chain_mode)
    std::vector<float> tune_ms;               // autotuner timings per candidate (ms), if it ran
    int64_t total_elems() const { return tot64_; }

private:
    using T2 = typename Vec2<T>::type;
    struct Level {
        double tol = 0;
        int Jmax = 0;
        std::vector<int> J;
        SwProb<T> *d_probs = nullptr;
        Fac<T> *fac = nullptr;  // row tables then (rectangle) column tables
        T *sh = nullptr;        // per iteration: stencil shifts and correction factor
        cudaGraphExec_t graph = nullptr;
        std::vector<cudaEvent_t> ev;  // 4 per iteration when instrumented
    };
    int build_graph(Level &L, std::string &err);
    int autotune(const std::vector<int64_t> &ns, int nrhs, double tol, bool tight, std::string &err);
    int time_level(size_t li, int reps, float &ms, std::string &err);
    int time_chain(int mode, float &ms, std::string &err);
    SwArgs<T> args(const Level &L, int which) const;
    int solve_refine(const double *F, double *X, cudaStream_t st, std::string &err);
    int solve_plain(const double *F, double *X, cudaStream_t st, std::string &err);

    std::vector<int64_t> ns_;
    int nrhs_ = 1;
    double tol_ = 0;
    double kx_ = 1.0, ky_ = 1.0;
    cudaStream_t cap_ = nullptr;
    std::vector<int> N_, P_;
    std::vector<int64_t> off64_, offT_, offS_;
    int64_t tot64_ = 0, totT_ = 0, totS_ = 0;
    int npairs_ = 0;
    double *Ft_ = nullptr, *Y0_ = nullptr, *Y1_ = nullptr, *bands64_ = nullptr;
    T *bandsT_ = nullptr, *rho0_ = nullptr, *cl_ = nullptr, *al_ = nullptr, *D_ = nullptr, *zin_ = nullptr;
    T2 *sumR_ = nullptr, *sumC_ = nullptr, *zxR_ = nullptr, *zxC_ = nullptr;
    int *err_ = nullptr;
    TileProb *d_tp_ = nullptr;
    int4 *d_tiles_ = nullptr;
    int64_t ntiles_ = 0;
    int4 *d_items_[3] = {nullptr, nullptr, nullptr};  // row pass, column pass, chains
    int64_t nitems_[3] = {0, 0, 0};
    int *d_active_ = nullptr, *d_pair_active_ = nullptr;
    int *h_active_ = nullptr, *h_pair_active_ = nullptr;
    unsigned long long *d_smax_ = nullptr, *d_rmax_ = nullptr, *h_smax_ = nullptr, *h_rmax_ = nullptr;
    int *h_err_ = nullptr;
    std::vector<Level> levels_;
    std::vector<int> levels_used_;
    bool instrument_ = false;
    std::vector<void *> allocs_;

    template <typename U>
    cudaError_t dalloc(U **p, size_t count);
};

}  // namespace fps
