// Host side of the FP32-sweep / FP64-refinement solve for one problem or a batch
// of squares of different sizes (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "refine.cuh"

namespace fps {

class RefineEngine {
public:
    // Plan `ns.size()` squares with `nrhs` right-hand sides each (caller packing:
    // problem after problem, each problem's nrhs n x n matrices back to back).
    // `target_ctas`: CTAs per pass to aim at for the largest problem (<= 0: default).
    // Returns an fps_status; on error `err` holds a message.
    int create(const std::vector<int64_t> &ns, int nrhs, double tol, cudaStream_t setup_stream, int target_ctas,
               std::string &err);
    void release();

    // Solve for device pointers F, X (packed as above) on stream st.  Returns an
    // fps_status (FPS_ERR_NOT_CONVERGED: X holds the last iterate).
    int solve(const double *F, double *X, cudaStream_t st, std::string &err);

    int set_instrument(bool on, std::string &err);
    int kernel_times(int *count, double *total_ms, double *alg_bytes, std::string &err);

    // facts
    int64_t bytes = 0;
    int J_inner_first = 0;      // J of the finest level for the largest problem
    int rounds_last = 0;
    double resid_last = 0.0;    // largest max|R~|/max|F~| over right-hand sides after the last solve
    int64_t launches_last = 0;
    int max_rounds = 8;
    int64_t total_elems() const { return tot64; }
    int chosen_target_ctas = 0;     // pass size picked by the autotuner (or given)
    std::vector<float> tune_ms;     // autotuner timings of the candidates (ms), if it ran

private:
    struct Level {
        double tol = 0;
        int Jmax = 0;
        std::vector<int> J;     // per problem
        RefProb *d_probs = nullptr;
        float4 *fac = nullptr;
        float *phick = nullptr;
        float4 *segc = nullptr;
        float *q2 = nullptr;
        FactorJob *d_jobs = nullptr;
        cudaGraphExec_t graph = nullptr;
        std::vector<cudaEvent_t> ev;
    };
    int build_graph(Level &L, std::string &err);
    int autotune(const int *cand, int ncand, const std::vector<RefProb64> &p64, int &best, std::string &err);

    std::vector<int64_t> ns_;
    int nrhs_ = 1;
    double tol_ = 0;
    cudaStream_t cap_ = nullptr;
    std::vector<RefineGeometry> geo_;
    std::vector<int64_t> off64_, off32_, offck_, offsm_;
    int64_t tot64 = 0, tot32 = 0, totck = 0, totsm = 0;
    int npairs_ = 0;
    double *Ft_ = nullptr, *Y0_ = nullptr, *Y1_ = nullptr, *bands_ = nullptr;
    float *Pt_ = nullptr, *A_ = nullptr, *C_ = nullptr, *D_ = nullptr, *ck_ = nullptr;
    float2 *summ_ = nullptr;
    RefProb64 *d_p64_ = nullptr;
    int4 *d_tiles_ = nullptr;
    int64_t ntiles_ = 0;
    int4 *d_items_ = nullptr;
    int64_t nitems_ = 0;
    int *d_active_ = nullptr, *d_pair_active_ = nullptr;
    int *h_active_ = nullptr, *h_pair_active_ = nullptr;
    unsigned long long *d_smax_ = nullptr, *d_rmax_ = nullptr, *h_smax_ = nullptr, *h_rmax_ = nullptr;
    std::vector<Level> levels_;
    std::vector<int> levels_used_;
    bool instrument_ = false;
    std::vector<void *> allocs_;

    template <typename T>
    cudaError_t dalloc(T **p, size_t count);
};

}  // namespace fps
