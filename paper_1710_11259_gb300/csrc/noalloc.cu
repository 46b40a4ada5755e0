// fps_poisson_square_solve_noalloc: the FP64 square solve for small n without
// any memory allocation.
//
// Some callers cannot allocate device memory at solve time: code running under a
// caching allocator that owns all of the device memory, real-time or embedded
// hosts that forbid allocation after start-up, and code that must not trigger the
// implicit synchronisation cudaMalloc/cudaFree can cause.  This entry point keeps
// every work array in one file-scope device array of fixed size (kScratchDoubles
// doubles, 4 MiB) that each GPU loading the library holds until the process exits,
// and uses only stack memory on the host.  The caller still allocates F and X.
// Nothing is copied from host memory: the bands of A~ are computed on the device
// from their closed forms and the shifts reach the device as a kernel argument.
//
// Set-up: the device address of the array is looked up with cudaGetSymbolAddress
// once per device, on the first call made with that device current.  Make that
// first call before any stream capture (the look-up is a runtime call, not an
// enqueued operation).
//
// Sharing: every call on a device uses the same array and leaves its contents
// behind.  Calls whose work overlaps on the GPU (different streams, or different
// host threads without ordering) race on it; order them on one stream.  Every
// value a call reads from the array is written earlier by that same call (the
// zero padding of the band array included), so stale contents never leak into a
// result.
//
// Errors: status codes; fps_last_error() then returns a fixed message naming the
// check that failed (a pointer to a string literal, so reporting allocates nothing).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/fps.h"
#include "host_math.h"
#include "kernels.cuh"
#include "status.h"

namespace {

constexpr int64_t kMaxN = 256;                 // largest n accepted
constexpr int kMaxJ = 256;                     // largest iteration count accepted
constexpr int64_t kScratchDoubles = 524288;    // 4 MiB

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// The message is a string literal: recording it allocates nothing.
int noalloc_fail(int status, const char *why)
{
    fps::set_static_error(why);
    return status;
}

// Shifts q_0..q_{J-1} passed by value (2 KiB of kernel parameters).
struct NoallocShifts {
    double q[kMaxJ];
};

// Bands of A~ from the closed forms of (3.7)/(3.9) (the same formulas as the host
// routine square_bands): d_j = -M_jj / E_j, e_j = -M_{j,j+2} / sqrt(E_j E_{j+2})
// (zero for j + 2 >= n), s_j = 1/sqrt(E_j), E_j = (j+1)(j+2); and the shift table.
__global__ void noalloc_bands_kernel(int64_t n, NoallocShifts sh, int J, double *__restrict__ d,
                                     double *__restrict__ e, double *__restrict__ s, double *__restrict__ q)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < J) q[j] = sh.q[j];
    if (j >= n) return;
    const double x = (double)j;
    const double Ej = (x + 1.0) * (x + 2.0);
    const double Mjj = 2.0 * (x + 1.0) * (x + 2.0) / ((2.0 * x + 1.0) * (2.0 * x + 5.0));
    d[j] = -Mjj / Ej;
    double ej = 0.0;
    if (j + 2 < n) {
        const double Ej2 = (x + 3.0) * (x + 4.0);
        const double prod4 = (x + 1.0) * (x + 2.0) * (x + 3.0) * (x + 4.0);
        const double Mj2 = -sqrt(prod4 * (2.0 * x + 3.0) / (2.0 * x + 7.0)) / ((2.0 * x + 3.0) * (2.0 * x + 5.0));
        ej = -Mj2 / sqrt(Ej * Ej2);
    }
    e[j] = ej;
    s[j] = 1.0 / sqrt(Ej);
}

// Device address of the scratch array on the current device (set up once).
int scratch_for_current_device(double **out, int *device)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(FPS_ERR_CUDA, "no current CUDA device");
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(FPS_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        double *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr)
            return noalloc_fail(FPS_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    *device = dev;
    return FPS_OK;
}

}  // namespace

extern "C" {

int fps_poisson_square_solve_noalloc(int64_t n, double tol, const double *F, double *X, void *stream)
{
    if (n < 1 || n > kMaxN) return noalloc_fail(FPS_ERR_INVALID_ARG, "fps_poisson_square_solve_noalloc: n must be in [1, 256]");
    if (!(tol > 0.0 && tol < 1.0))
        return noalloc_fail(FPS_ERR_INVALID_ARG, "fps_poisson_square_solve_noalloc: tol must lie in (0, 1)");
    if (!F || !X) return noalloc_fail(FPS_ERR_INVALID_ARG, "fps_poisson_square_solve_noalloc: NULL F or X");
    const size_t bytes = sizeof(double) * (size_t)n * (size_t)n;
    const char *f0 = (const char *)F, *x0 = (const char *)X;
    if (f0 < x0 + bytes && x0 < f0 + bytes)
        return noalloc_fail(FPS_ERR_INVALID_ARG, "fps_poisson_square_solve_noalloc: F and X overlap");
    // Lemma B.2 interval, J of (2.9) and the symmetric shifts (2.4) on the host (the
    // same routines as the plan, writing into a stack array); the bands of A~
    // (3.7)/(3.9) are computed on the device below.
    const double eps = fps::square_eps(n);
    const int J = fps::adi_iterations(-1.0, -eps, eps, 1.0, tol);
    if (J < 1 || J > kMaxJ)
        return noalloc_fail(FPS_ERR_INVALID_ARG, "fps_poisson_square_solve_noalloc: tol needs more than 256 iterations");
    NoallocShifts sh;
    fps::zolotarev_shifts_symmetric_into(eps, 1.0, J, sh.q);
    const double *q = sh.q;

    double *base = nullptr;
    int dev = 0;
    int st = scratch_for_current_device(&base, &dev);
    if (st != FPS_OK) return st;
    // F and X must be device memory of the current device (where the kernels and the
    // scratch array run): memory of another GPU would be reached by peer access.
    for (const void *p : {(const void *)F, (const void *)X}) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, p) != cudaSuccess ||
            (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return noalloc_fail(FPS_ERR_INVALID_ARG,
                                "fps_poisson_square_solve_noalloc: F and X must be device memory");
        }
        if (attr.type == cudaMemoryTypeDevice && attr.device != dev)
            return noalloc_fail(FPS_ERR_INVALID_ARG,
                                "fps_poisson_square_solve_noalloc: F and X must be on the current device");
    }
    // Carve the scratch: bands, shifts, factors (J x n double2), then five n x n arrays.
    const int64_t nn = n * n;
    double *d_d = base, *d_e = base + n, *d_s = base + 2 * n, *d_q = base + 3 * n;
    int64_t off = 3 * n + kMaxJ;
    off = (off + 1) & ~int64_t(1);  // 16-byte alignment of the double2 factors
    double2 *fac = reinterpret_cast<double2 *>(base + off);
    off += 2 * (int64_t)J * n;
    double *Ft = base + off, *FtT = Ft + nn, *A = FtT + nn, *B = A + nn, *Z = B + nn;
    if (off + 5 * nn > kScratchDoubles)
        return noalloc_fail(FPS_ERR_INVALID_ARG, "fps_poisson_square_solve_noalloc: problem exceeds the scratch");

    cudaStream_t strm = (cudaStream_t)stream;
#define NA_CK(call)                                                                                      \
    do {                                                                                                 \
        if ((call) != cudaSuccess) return noalloc_fail(FPS_ERR_CUDA, "fps_poisson_square_solve_noalloc: " #call); \
    } while (0)
    {
        const int64_t m = n > J ? n : (int64_t)J;
        noalloc_bands_kernel<<<(unsigned)((m + 127) / 128), 128, 0, strm>>>(n, sh, J, d_d, d_e, d_s, d_q);
        NA_CK(cudaGetLastError());
    }
    NA_CK(fps::launch_factors(d_d, d_e, d_q, J, n, fac, strm));
    NA_CK(fps::launch_scale_in(F, Ft, FtT, d_s, n, strm));
    for (int j = 0; j < J; ++j) {
        fps::HalfStep<double> h;
        h.d = d_d;
        h.e = d_e;
        h.q = q[j];
        h.n = n;
        h.Z = Z;
        h.fac = fac + (int64_t)j * n;
        h.V = (j == 0) ? nullptr : B;
        h.G = FtT;
        h.Out = A;
        h.transposed_out = true;
        NA_CK(fps::launch_halfstep(h, strm));
        h.V = A;
        h.G = Ft;
        h.Out = B;
        h.transposed_out = (j + 1 < J);
        NA_CK(fps::launch_halfstep(h, strm));
    }
    NA_CK(fps::launch_scale_out(B, X, d_s, n, strm));
#undef NA_CK
    (void)dev;
    return FPS_OK;
}

}  // extern "C"
