// Launch wrappers of the sm_103a kernels (internal header of the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fps {

// One half-step of Algorithm 2 written as a column solve:
//     W = (A~ - q I)^{-1} ( G - V (A~ + q I) )
// V's stencil runs along its rows (k-2, k, k+2), the solve runs down each column
// (rows i-2, i, i+2: the even/odd decoupling of App. B), one thread per
// (column, row parity).  Step 1 of Algorithm 2 is the transpose of this form
// (A~ symmetric), so storing W transposed makes every half-step the same kernel.
template <typename T>
struct HalfStep {
    const T *V = nullptr;       // previous iterate; nullptr means V = 0 (first half-step)
    const T *G = nullptr;       // F~ or F~^T
    T *Z = nullptr;             // spill of the forward elimination (n x n)
    T *Out = nullptr;           // W^T (transposed) or W (normal)
    const void *fac = nullptr;  // per-row {1/den_i, e_i/den_i} of A~ - q I (T2 of T)
    const T *d = nullptr;       // diagonal of A~
    const T *e = nullptr;       // e[k] = A~[k][k+2], zero-padded to length n
    T q = 0;                    // shift (q_j > 0; p_j = -q_j)
    int64_t n = 0;
    bool transposed_out = true;
};

template <typename T>
cudaError_t launch_halfstep(const HalfStep<T> &h, cudaStream_t st);

// Per-shift Thomas factors of A~ - q_j I (FP64), J shifts, written as
// fac[j*n + i] = {1/den_i, e_i/den_i}.  Optionally also an FP32 copy.
cudaError_t launch_factors(const double *d, const double *e, const double *q, int J, int64_t n, double2 *fac,
                           cudaStream_t st);

// F~ = D_s F D_s and its transpose (D_s = diag(s)).
cudaError_t launch_scale_in(const double *F, double *Ft, double *FtT, const double *s, int64_t n, cudaStream_t st);

// X = D_s Y D_s (elementwise, row-major).
cudaError_t launch_scale_out(const double *Y, double *X, const double *s, int64_t n, cudaStream_t st);

}  // namespace fps
