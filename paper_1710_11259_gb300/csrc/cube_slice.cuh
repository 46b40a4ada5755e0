// Slice-resident inner level of the FP32 cube ADI (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fps {

// One inner (slice Stein) solve of the residual form with every slice on chip:
//   Z (+)= (T_ab + c)^{-1} (r1 R1 + r2 R2)  on every slice across mode 3 - ma - mb,
// all J iterations inside one launch, one 8-CTA cluster per slice.
struct SliceArgs {
    const float2 *fac;   // factor sets of the Stein entry: [2J + 1][n] {1/den, u}
    const double2 *ab;   // (alpha, beta) of every set: set 1 + 2l = (p_l, c), set 2 + 2l = (1, -q_l)
    int J;
    const float *R1, *R2;  // R2 may be null; either may alias Z
    float r1, r2;
    float *Z;
    bool accumulate;       // Z += solution (else Z = solution)
    const float *d, *e;    // bands of A~ (FP32, zero outside [0, n))
    int n, ma, mb;         // slice modes: rows along ma, lines of the first solve along mb
};

// Largest n the slice-resident kernel takes (shared memory of one CTA, FP32).
constexpr int kSliceMaxN = 256;
constexpr int kSliceCluster = 8;

int slice_smem_bytes(int n);
// Sets the kernel's shared-memory limit for n and reports whether a cluster of that
// size fits on the device (false: use the streaming line solves).
cudaError_t slice_setup(int n, bool *usable);
cudaError_t launch_stein_slice(const SliceArgs &a, cudaStream_t st);

}  // namespace fps
