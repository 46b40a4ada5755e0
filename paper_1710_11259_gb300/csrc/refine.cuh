// Kernels of the FP32-sweep / FP64-refinement solve (internal header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fps {

// Work decomposition of the FP32 passes for size n: columns in blocks of 32,
// each (column, parity) system cut into P segments of Ls rows.
struct RefineGeometry {
    int64_t ld = 0;      // padded leading dimension (multiple of 32)
    int64_t nblk = 0;    // column blocks
    int64_t nchunk = 0;  // checkpoint chunks per parity system
    int64_t Ls = 0;      // rows per segment (multiple of 32)
    int64_t P = 1;       // segments per system
};
RefineGeometry refine_geometry(int64_t n, int sms);

// Scratch of the passes (device): checkpoints and per-segment summaries.
struct RefineScratch {
    float *ck = nullptr;
    float2 *summ = nullptr;
};
int64_t refine_checkpoint_floats(const RefineGeometry &g);
int64_t refine_summary_float2(const RefineGeometry &g);

// Raise the dynamic shared-memory limits of the pass kernels (once per process).
cudaError_t refine_setup_kernels();

// Row pass on rho^T: A = (R - q)^{-1} rho, C = rho + 2q A (outputs in rho's orientation).
cudaError_t launch_row_pass(const float *Pt, float *A, float *C, const RefineScratch &w, const float4 *fac,
                            const float *phick, const float4 *segc, float q2, int64_t n, const RefineGeometry &g,
                            cudaStream_t st);

// Column pass: Pt = (C + 2q (L-q)^{-1} C)^T, Dl -= 2q (L-q)^{-1} A (Dl = -2q (L-q)^{-1} A when first).
// If ev0/ev1 are given they are recorded around the back-substitution kernel (timing).
cudaError_t launch_col_pass(const float *C, const float *A, float *Dl, float *Pt, const RefineScratch &w,
                            const float4 *fac, const float *phick, const float4 *segc, float q2, int64_t n,
                            const RefineGeometry &g, bool first, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                            cudaEvent_t ev1 = nullptr);

// Yout = Y + s Dl (if apply_update; Y read as zero if y_zero), R = F~ - A~ Yout - Yout A~,
// Pt = (R/s)^T, rmax = max |R| (bit pattern).  s is read from device memory (bit pattern).
cudaError_t launch_residual(const double *Y, double *Yout, const float *Dl, const double *Ft, float *Pt,
                            const double *d, const double *e, const unsigned long long *s_bits, int64_t n,
                            int64_t ld, unsigned long long *rmax, bool apply_update, bool y_zero, cudaStream_t st);

// F~ = D_s F D_s (FP64), Pt = (F~/s)^T (FP32, ld-strided), s read from device memory.
cudaError_t launch_refine_scale_in(const double *F, double *Ft, float *Pt, const double *sc, int64_t n, int64_t ld,
                                   const unsigned long long *s_bits, cudaStream_t st);

// max |D_s F D_s| into *out (bit pattern of a non-negative double; *out must start at 0).
cudaError_t launch_absmax_scaled(const double *F, const double *sc, int64_t n, unsigned long long *out,
                                 cudaStream_t st);

// FP32 factors of A~ - q_j I for J shifts (fac: J*n, phick: J*2*nchunk, segc: J*2*P).
cudaError_t launch_factors32(const double *d, const double *e, const double *q, int J, int64_t n,
                             const RefineGeometry &g, float4 *fac, float *phick, float4 *segc, cudaStream_t st);

}  // namespace fps
