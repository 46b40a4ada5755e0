// fps_probe_fma_rate: the device's fused multiply-add throughput, measured.  It is
// the denominator of the ALU roofline of the FP64 sweeps, which on GB300 are bound
// by the FP64 FMA rate rather than by HBM.
#include <cuda_runtime.h>

#include "../../include/fps.h"
#include "device_info.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x) * T(1e-3) + T(c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1.25)) out[0] = s;  // never true (x stays near 1): keeps the chains alive
}

template <typename T>
int probe(double *rate)
{
    T *out = nullptr;
    if (cudaMalloc((void **)&out, sizeof(T)) != cudaSuccess) return FPS_ERR_CUDA;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = FPS_ERR_CUDA;
    const int blocks = 16 * fps::current_sm_count(), threads = 256;
    int iters = sizeof(T) == 8 ? 2000 : 40000;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        float ms = 0.f;
        bool ok = true;
        for (int round = 0; round < 2 && ok; ++round) {  // the first round warms up and sizes the second
            fma_probe_kernel<T><<<blocks, threads, 0, st>>>(out, iters, T(0.999999), T(1e-6));
            ok = cudaEventRecord(e0, st) == cudaSuccess;
            fma_probe_kernel<T><<<blocks, threads, 0, st>>>(out, iters, T(0.999999), T(1e-6));
            ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && cudaGetLastError() == cudaSuccess;
            if (ok && round == 0 && ms > 0.f) iters = (int)(iters * (100.0 / ms) + 1);  // about 100 ms
        }
        if (ok && ms > 0.f) {
            *rate = (double)blocks * threads * kChains * (double)iters / (ms * 1e-3);
            status = FPS_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    return status;
}

}  // namespace

extern "C" int fps_probe_fma_rate(int precision, double *fma_per_s)
{
    if (!fma_per_s || (precision != FPS_FP64 && precision != FPS_FP32_REFINE)) return FPS_ERR_INVALID_ARG;
    return precision == FPS_FP64 ? probe<double>(fma_per_s) : probe<float>(fma_per_s);
}
