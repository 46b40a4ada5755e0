// Small squares in FP64 (n <= 64): one launch runs all J iterations of Algorithm 2
// with warp-shuffle cyclic reduction on shared-memory-resident iterates, one
// cluster of CTAs per right-hand side (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace fps {

constexpr int kSmallMaxN = 64;   // every parity tridiagonal fits one warp
constexpr int kSmallCluster = 8; // CTAs per right-hand side

struct SmallArgs {
    int n, J, nrhs;
    const double *F;    // nrhs x n x n, row-major (device)
    double *X;          // same layout (device)
    const double *d, *e, *s;  // bands of A~ (e zero-padded to length n) and 1/sqrt(E) (device)
    const double *q;    // [J] shifts (device)
    const double *pcr;  // [J][2][11][32] reduction coefficients: alpha (steps 0-4), gamma (5-9), 1/b (10)
};

// Reduction coefficients of the even (p = 0) and odd (p = 1) tridiagonals of
// A~ - q_j I for every shift, in FP64 on the host.
void small_pcr_coefficients(int64_t n, const std::vector<double> &d, const std::vector<double> &e,
                            const std::vector<double> &q, std::vector<double> &out);

cudaError_t small_setup_kernel();
cudaError_t launch_small_adi(const SmallArgs &a, cudaStream_t st);

}  // namespace fps
