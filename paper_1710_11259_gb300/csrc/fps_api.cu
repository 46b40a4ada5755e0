// C ABI of the solver (include/fps.h): plans, solves, adjoint, host helpers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <initializer_list>
#include <vector>

#include "../../include/fps.h"
#include "host_math.h"
#include "sweep_engine.h"
#include "small.cuh"
#include "cube.h"
#include "legendre.cuh"
#include "dirichlet.cuh"
#include "cylinder.h"
#include "trace.h"
#include "status.h"

namespace {

thread_local std::string g_last_error;
thread_local const char *g_static_error = nullptr;  // set by allocation-free entry points

int fail(int status, const std::string &msg)
{
    g_last_error = msg;
    g_static_error = nullptr;
    return status;
}

#define FPS_CK(call)                                                                                     \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(FPS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Where a caller's buffer lives, seen from the device `dev` whose kernels will touch it:
// device memory of `dev` or managed memory (kDevice), pageable or pinned host memory
// (kHost, staged through device scratch where an entry point accepts it), or device memory
// of another device (kForeign: rejected everywhere, since the kernels would make peer
// accesses that may not even be enabled).
enum class Mem { kHost, kDevice, kForeign };

Mem memory_kind(const void *p, int dev)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return Mem::kHost;
    }
    if (attr.type == cudaMemoryTypeManaged) return Mem::kDevice;
    if (attr.type == cudaMemoryTypeDevice) return attr.device == dev ? Mem::kDevice : Mem::kForeign;
    return Mem::kHost;
}

int current_device()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    return dev;
}

bool is_device_pointer(const void *p, int dev) { return memory_kind(p, dev) == Mem::kDevice; }

}  // namespace

namespace fps {
void set_static_error(const char *msg) { g_static_error = msg; }
}  // namespace fps

struct fps_plan {
    int64_t n = 0;
    int dim = 2;
    double tol = 0;
    int precision = FPS_FP64;
    int nrhs = 1;
    int device = 0;
    cudaStream_t stream = nullptr;      // user stream
    cudaStream_t cap_stream = nullptr;  // private stream used to capture the graphs

    int J = 0;
    std::vector<double> q;  // shifts q_j > 0 of the FP64 solve (p_j = -q_j)
    int64_t bytes = 0;

    // square: the ADI pass engine (FP32 sweeps + FP64 refinement, or plain FP64)
    fps::SweepEngine<float> *eng32 = nullptr;
    fps::SweepEngine<double> *eng64 = nullptr;
    // FP64 squares with n <= 64: whole ADI in one launch (cluster kernel, warp-shuffle PCR)
    bool small = false;
    double *sm_bands = nullptr, *sm_q = nullptr, *sm_pcr = nullptr;
    // dim = 3: the nested cube ADI
    fps::CubeEngine *cube = nullptr;
    std::vector<int64_t> batch_ns;   // sizes of a batched plan (empty otherwise)
    int64_t total_elems = 0;         // doubles in F (and X) for all right-hand sides / problems
    double *stage_in = nullptr, *stage_out = nullptr;  // lazily allocated for host pointers

    bool instrument = false;
    int64_t launches_last = 0;
    double kx = 1.0, ky = 1.0;  // scales of u_xx and u_yy (rectangle plans)
    // nonhomogeneous Dirichlet solves: C~ right-hand side, C~ solution, trace second
    // derivatives and coefficient sums (allocated by the first such call)
    double *dir_F = nullptr, *dir_X = nullptr, *dir_d2 = nullptr, *dir_ts = nullptr;
    // cylinder Fourier modes |k| >= 2 (Sec. 4.1, Case 1)
    fps::CylinderEngine *cyl = nullptr;
};

namespace {

void release(fps_plan *p)
{
    if (!p) return;
    DeviceGuard g(p->device);
    if (p->stage_in) cudaFree(p->stage_in);
    if (p->stage_out) cudaFree(p->stage_out);
    if (p->sm_bands) cudaFree(p->sm_bands);
    if (p->sm_q) cudaFree(p->sm_q);
    if (p->sm_pcr) cudaFree(p->sm_pcr);
    for (double *b : {p->dir_F, p->dir_X, p->dir_d2, p->dir_ts})
        if (b) cudaFree(b);
    if (p->eng32) {
        p->eng32->release();
        delete p->eng32;
    }
    if (p->eng64) {
        p->eng64->release();
        delete p->eng64;
    }
    if (p->cube) {
        p->cube->release();
        delete p->cube;
    }
    if (p->cyl) {
        p->cyl->release();
        delete p->cyl;
    }
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
}

// The whole packed F at once (every problem and right-hand side of the plan).
template <typename E>
int solve_engine(fps_plan *p, E *eng, const double *F, double *X, bool fdev, bool xdev, const char *what)
{
    const size_t bytes = sizeof(double) * (size_t)p->total_elems;
    const double *Fd = F;
    double *Xd = X;
    if (!fdev) {
        if (!p->stage_in) FPS_CK(cudaMalloc((void **)&p->stage_in, bytes));
        FPS_CK(cudaMemcpyAsync(p->stage_in, F, bytes, cudaMemcpyHostToDevice, p->stream));
        Fd = p->stage_in;
    }
    if (!xdev) {
        if (!p->stage_out) FPS_CK(cudaMalloc((void **)&p->stage_out, bytes));
        Xd = p->stage_out;
    }
    std::string err;
    const int st = eng->solve(Fd, Xd, p->stream, err);
    if (st != FPS_OK && st != FPS_ERR_NOT_CONVERGED) return fail(st, std::string(what) + ": " + err);
    p->launches_last = eng->launches_last;
    if (!xdev) {
        FPS_CK(cudaMemcpyAsync(X, Xd, bytes, cudaMemcpyDeviceToHost, p->stream));
        FPS_CK(cudaStreamSynchronize(p->stream));
    } else if (!fdev) {
        FPS_CK(cudaStreamSynchronize(p->stream));  // host F must stay valid only until copied
    }
    if (st != FPS_OK) return fail(st, std::string(what) + ": " + err);
    FPS_CK(cudaGetLastError());
    return FPS_OK;
}

// FP64, n <= 64: one launch of the cluster kernel for all right-hand sides.
int solve_small(fps_plan *p, const double *F, double *X, bool fdev, bool xdev, const char *what)
{
    const size_t bytes = sizeof(double) * (size_t)p->total_elems;
    const double *Fd = F;
    double *Xd = X;
    if (!fdev) {
        if (!p->stage_in) FPS_CK(cudaMalloc((void **)&p->stage_in, bytes));
        FPS_CK(cudaMemcpyAsync(p->stage_in, F, bytes, cudaMemcpyHostToDevice, p->stream));
        Fd = p->stage_in;
    }
    if (!xdev) {
        if (!p->stage_out) FPS_CK(cudaMalloc((void **)&p->stage_out, bytes));
        Xd = p->stage_out;
    }
    fps::SmallArgs a;
    a.n = (int)p->n;
    a.J = p->J;
    a.nrhs = p->nrhs;
    a.F = Fd;
    a.X = Xd;
    a.d = p->sm_bands;
    a.e = p->sm_bands + p->n;
    a.s = p->sm_bands + 2 * p->n;
    a.q = p->sm_q;
    a.pcr = p->sm_pcr;
    cudaError_t e = fps::launch_small_adi(a, p->stream);
    if (e != cudaSuccess) return fail(FPS_ERR_CUDA, std::string(what) + ": small-n kernel: " + cudaGetErrorString(e));
    p->launches_last = 1;
    if (!xdev) {
        FPS_CK(cudaMemcpyAsync(X, Xd, bytes, cudaMemcpyDeviceToHost, p->stream));
        FPS_CK(cudaStreamSynchronize(p->stream));
    } else if (!fdev) {
        FPS_CK(cudaStreamSynchronize(p->stream));
    }
    return FPS_OK;
}

int solve_square(fps_plan *p, const double *F, double *X, const char *what)
{
    fps::TraceRange tr(what);
    if (!p) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": plan is NULL");
    if (p->dim != 2) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": plan is not two-dimensional");
    if (!F || !X) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": NULL F or X");
    const size_t bytes = sizeof(double) * (size_t)p->total_elems;
    const char *f0 = (const char *)F, *x0 = (const char *)X;
    if (f0 < x0 + bytes && x0 < f0 + bytes) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": F and X overlap");
    DeviceGuard g(p->device);
    const Mem fk = memory_kind(F, p->device), xk = memory_kind(X, p->device);
    if (fk == Mem::kForeign || xk == Mem::kForeign)
        return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": F or X is device memory of another device");
    const bool fdev = fk == Mem::kDevice, xdev = xk == Mem::kDevice;
    p->launches_last = 0;
    if (p->small) return solve_small(p, F, X, fdev, xdev, what);
    if (p->eng32) return solve_engine(p, p->eng32, F, X, fdev, xdev, what);
    return solve_engine(p, p->eng64, F, X, fdev, xdev, what);
}

// A square (kx = ky = 1) or rectangle plan: kx A~ Y + ky Y A~ = F~.
int create_square(fps_plan **out, int64_t n, double tol, int precision, bool tight, int nrhs, void *stream,
                  double kx, double ky, const char *what)
{
    fps_plan *p = new fps_plan();
    p->n = n;
    p->dim = 2;
    p->tol = tol;
    p->precision = precision;
    p->nrhs = nrhs;
    p->kx = kx;
    p->ky = ky;
    p->stream = (cudaStream_t)stream;
    p->total_elems = n * n * nrhs;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(FPS_ERR_CUDA, std::string(what) + ": no CUDA device");
    }
    auto bail = [&](int s) {
        release(p);
        return s;
    };
#define PCK(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return bail(fail(FPS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)));          \
    } while (0)

    // Lemma B.2 interval (or the tight one) of A~, scaled to the intervals of kx A~ and
    // -ky A~; (2.9) J; (2.4) shifts (on a square p_j = -q_j; the q_j are kept for info)
    const bool square = kx == ky;
    double lo = fps::square_eps(n), hi = 1.0;
    if (tight && precision == FPS_FP64) fps::square_tight_interval(n, lo, hi);
    p->J = fps::adi_iterations(-kx * hi, -kx * lo, ky * lo, ky * hi, tol);
    std::vector<double> mp;  // -p_j
    if (square) {
        fps::zolotarev_shifts_symmetric(lo, hi, p->J, p->q);
        for (double &v : p->q) v *= kx;
        mp = p->q;
    } else {
        std::vector<double> pp;
        fps::zolotarev_shifts(-kx * hi, -kx * lo, ky * lo, ky * hi, p->J, pp, p->q);
        for (double v : pp) mp.push_back(-v);
    }
    // validated before anything is launched (every path, including the one-launch small path)
    fps::inject_shift_fault(p->q);
    if (!fps::shifts_valid(p->q, ky * lo, ky * hi) || !fps::shifts_valid(mp, kx * lo, kx * hi))
        return bail(fail(FPS_ERR_INVALID_ARG, std::string(what) +
                                                  ": shift list failed validation (a shift is not finite or lies "
                                                  "outside the spectral interval)"));
    if (n > 40000) return bail(fail(FPS_ERR_UNSUPPORTED, std::string(what) + ": squares support n <= 40000"));
    if (nrhs > 256) return bail(fail(FPS_ERR_UNSUPPORTED, std::string(what) + ": squares support nrhs <= 256"));
    PCK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    std::string err;
    int st;
    if (precision == FPS_FP64 && n <= fps::kSmallMaxN && kx == 1.0 && ky == 1.0) {
        // whole ADI in one launch: bands, shifts and reduction coefficients on the device
        std::vector<double> d, e, s, pcr;
        fps::square_bands(n, d, e);
        fps::inv_sqrt_E(n, s);
        fps::small_pcr_coefficients(n, d, e, p->q, pcr);
        std::vector<double> bands(3 * n);
        std::copy(d.begin(), d.end(), bands.begin());
        std::copy(e.begin(), e.end(), bands.begin() + n);
        std::copy(s.begin(), s.end(), bands.begin() + 2 * n);
        PCK(fps::small_setup_kernel());
        PCK(cudaMalloc((void **)&p->sm_bands, sizeof(double) * 3 * n));
        PCK(cudaMalloc((void **)&p->sm_q, sizeof(double) * p->J));
        PCK(cudaMalloc((void **)&p->sm_pcr, sizeof(double) * pcr.size()));
        PCK(cudaMemcpy(p->sm_bands, bands.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
        PCK(cudaMemcpy(p->sm_q, p->q.data(), sizeof(double) * p->J, cudaMemcpyHostToDevice));
        PCK(cudaMemcpy(p->sm_pcr, pcr.data(), sizeof(double) * pcr.size(), cudaMemcpyHostToDevice));
        p->bytes += (int64_t)sizeof(double) * (3 * n + p->J + (int64_t)pcr.size());
        p->small = true;
        st = FPS_OK;
    } else if (precision == FPS_FP64) {
        p->eng64 = new fps::SweepEngine<double>();
        st = p->eng64->create(std::vector<int64_t>{n}, nrhs, tol, tight, p->cap_stream, err, 0, kx, ky);
        if (st == FPS_OK) p->bytes += p->eng64->bytes;
    } else {
        p->eng32 = new fps::SweepEngine<float>();
        st = p->eng32->create(std::vector<int64_t>{n}, nrhs, tol, true, p->cap_stream, err, 0, kx, ky);
        if (st == FPS_OK) p->bytes += p->eng32->bytes;
    }
    if (st != FPS_OK) return bail(fail(st, std::string(what) + ": " + err));
#undef PCK
    *out = p;
    return FPS_OK;
}

}  // namespace

namespace {

// Arguments shared by the Dirichlet solve and its adjoint: a single (non-batched)
// square or rectangle plan, device buffers, scratch allocated on first use.
int dirichlet_check(fps_plan *p, std::initializer_list<const void *> ptrs, const char *what)
{
    if (!p) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": plan is NULL");
    if (p->dim != 2 || !p->batch_ns.empty())
        return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": needs a single square or rectangle plan");
    for (const void *q : ptrs) {
        if (!q) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": NULL buffer");
        if (!is_device_pointer(q, p->device))
            return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": buffers must be device memory of the plan's device");
    }
    if (!p->dir_F) {
        DeviceGuard g(p->device);
        const size_t nn = (size_t)p->total_elems;
        FPS_CK(cudaMalloc((void **)&p->dir_F, sizeof(double) * nn));
        FPS_CK(cudaMalloc((void **)&p->dir_X, sizeof(double) * nn));
        FPS_CK(cudaMalloc((void **)&p->dir_d2, sizeof(double) * 4 * (size_t)p->n * p->nrhs));
        FPS_CK(cudaMalloc((void **)&p->dir_ts, sizeof(double) * 8 * (size_t)p->nrhs));
        p->bytes += (int64_t)sizeof(double) * (2 * (int64_t)nn + (4 * p->n + 8) * p->nrhs);
    }
    return FPS_OK;
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" {

int fps_plan_create(fps_plan **out, int64_t n, int dim, double tol, int precision, int nrhs, void *stream)
{
    fps::TraceRange tr("fps_plan_create");
    if (!out) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create: out is NULL");
    *out = nullptr;
    if (n < 1) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create: n must be >= 1");
    if (dim != 2 && dim != 3) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create: dim must be 2 or 3");
    if (!(tol > 0.0 && tol < 1.0)) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create: tol must lie in (0, 1)");
    if (nrhs < 1) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create: nrhs must be >= 1");
    const bool tight = (precision & FPS_TIGHT_SPECTRUM) != 0;
    precision &= ~FPS_TIGHT_SPECTRUM;
    if (precision != FPS_FP64 && precision != FPS_FP32_REFINE)
        return fail(FPS_ERR_INVALID_ARG, "fps_plan_create: unknown precision");
    if (tight && dim != 2) return fail(FPS_ERR_UNSUPPORTED, "fps_plan_create: FPS_TIGHT_SPECTRUM is for squares");
    if (dim == 3) {
        if (n > 320) return fail(FPS_ERR_UNSUPPORTED, "fps_plan_create: the cube supports n <= 320");
        fps_plan *p = new fps_plan();
        p->n = n;
        p->dim = 3;
        p->tol = tol;
        p->precision = precision;
        p->nrhs = nrhs;
        p->stream = (cudaStream_t)stream;
        p->total_elems = n * n * n * nrhs;
        if (cudaGetDevice(&p->device) != cudaSuccess) {
            delete p;
            return fail(FPS_ERR_CUDA, "fps_plan_create: no CUDA device");
        }
        p->cube = new fps::CubeEngine();
        std::string err;
        const int st = p->cube->create(n, tol, precision, err);
        if (st != FPS_OK) {
            release(p);
            return fail(st, "fps_plan_create: " + err);
        }
        p->J = p->cube->J_outer;
        p->bytes = p->cube->bytes;
        *out = p;
        return FPS_OK;
    }

    return create_square(out, n, tol, precision, tight, nrhs, stream, 1.0, 1.0, "fps_plan_create");
}

int fps_plan_create_rect(fps_plan **out, int64_t n, double width, double height, double tol, int precision,
                         int nrhs, void *stream)
{
    fps::TraceRange tr("fps_plan_create_rect");
    if (!out) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_rect: out is NULL");
    *out = nullptr;
    if (n < 1) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_rect: n must be >= 1");
    if (!(width > 0.0 && height > 0.0 && std::isfinite(width) && std::isfinite(height)))
        return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_rect: width and height must be positive and finite");
    if (!(tol > 0.0 && tol < 1.0)) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_rect: tol must lie in (0, 1)");
    if (nrhs < 1) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_rect: nrhs must be >= 1");
    const bool tight = (precision & FPS_TIGHT_SPECTRUM) != 0;
    precision &= ~FPS_TIGHT_SPECTRUM;
    if (precision != FPS_FP64 && precision != FPS_FP32_REFINE)
        return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_rect: unknown precision");
    const double kx = (2.0 / width) * (2.0 / width), ky = (2.0 / height) * (2.0 / height);
    return create_square(out, n, tol, precision, tight, nrhs, stream, kx, ky, "fps_plan_create_rect");
}

int fps_plan_create_batched(fps_plan **out, const int64_t *ns, int64_t count, int nrhs, double tol, int precision,
                            void *stream)
{
    fps::TraceRange tr("fps_plan_create_batched");
    if (!out) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_batched: out is NULL");
    *out = nullptr;
    if (!ns || count < 1) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_batched: need count >= 1 sizes");
    if (nrhs < 1 || nrhs > 256) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_batched: nrhs must be in [1, 256]");
    if (!(tol > 0.0 && tol < 1.0)) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_batched: tol must lie in (0, 1)");
    if (precision != FPS_FP32_REFINE)
        return fail(FPS_ERR_UNSUPPORTED, "fps_plan_create_batched: batches run in FPS_FP32_REFINE");
    std::vector<int64_t> v(ns, ns + count);
    int64_t nmax = 0, total = 0;
    for (int64_t n : v) {
        if (n < 1 || n > 40000) return fail(FPS_ERR_INVALID_ARG, "fps_plan_create_batched: every n must be in [1, 40000]");
        nmax = n > nmax ? n : nmax;
        total += n * n * nrhs;
    }
    fps_plan *p = new fps_plan();
    p->n = nmax;
    p->dim = 2;
    p->tol = tol;
    p->precision = precision;
    p->nrhs = nrhs;
    p->stream = (cudaStream_t)stream;
    p->batch_ns = v;
    p->total_elems = total;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(FPS_ERR_CUDA, "fps_plan_create_batched: no CUDA device");
    }
    if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete p;
        return fail(FPS_ERR_CUDA, "fps_plan_create_batched: stream creation failed");
    }
    p->eng32 = new fps::SweepEngine<float>();
    std::string err;
    const int st = p->eng32->create(v, nrhs, tol, true, p->cap_stream, err);
    if (st != FPS_OK) {
        release(p);
        return fail(st, "fps_plan_create_batched: " + err);
    }
    p->bytes += p->eng32->bytes;
    *out = p;
    return FPS_OK;
}

int fps_plan_set_stream(fps_plan *plan, void *stream)
{
    if (!plan) return fail(FPS_ERR_INVALID_ARG, "fps_plan_set_stream: plan is NULL");
    plan->stream = (cudaStream_t)stream;
    return FPS_OK;
}

int fps_poisson_square_solve(fps_plan *plan, const double *F, double *X)
{
    return solve_square(plan, F, X, "fps_poisson_square_solve");
}

int fps_poisson_cube_solve(fps_plan *plan, const double *F, double *X)
{
    fps::TraceRange tr("fps_poisson_cube_solve");
    if (!plan) return fail(FPS_ERR_INVALID_ARG, "fps_poisson_cube_solve: plan is NULL");
    if (plan->dim != 3 || !plan->cube)
        return fail(FPS_ERR_INVALID_ARG, "fps_poisson_cube_solve: plan is not three-dimensional");
    if (!F || !X) return fail(FPS_ERR_INVALID_ARG, "fps_poisson_cube_solve: NULL F or X");
    const int64_t n3 = plan->n * plan->n * plan->n;
    const size_t bytes = sizeof(double) * (size_t)plan->total_elems;
    const char *f0 = (const char *)F, *x0 = (const char *)X;
    if (f0 < x0 + bytes && x0 < f0 + bytes) return fail(FPS_ERR_INVALID_ARG, "fps_poisson_cube_solve: F and X overlap");
    DeviceGuard g(plan->device);
    const Mem fk = memory_kind(F, plan->device), xk = memory_kind(X, plan->device);
    if (fk == Mem::kForeign || xk == Mem::kForeign)
        return fail(FPS_ERR_INVALID_ARG, "fps_poisson_cube_solve: F or X is device memory of another device");
    const bool fdev = fk == Mem::kDevice, xdev = xk == Mem::kDevice;
    if ((!fdev || !xdev) && !plan->stage_in) {
        FPS_CK(cudaMalloc((void **)&plan->stage_in, sizeof(double) * n3));
        FPS_CK(cudaMalloc((void **)&plan->stage_out, sizeof(double) * n3));
    }
    plan->launches_last = 0;
    for (int r = 0; r < plan->nrhs; ++r) {
        const double *Fr = F + (int64_t)r * n3;
        double *Xr = X + (int64_t)r * n3;
        const double *Fd = Fr;
        double *Xd = xdev ? Xr : plan->stage_out;
        if (!fdev) {
            FPS_CK(cudaMemcpyAsync(plan->stage_in, Fr, sizeof(double) * n3, cudaMemcpyHostToDevice, plan->stream));
            Fd = plan->stage_in;
        }
        std::string err;
        const int st = plan->cube->solve_cube(Fd, Xd, plan->stream, err);
        if (st != FPS_OK) return fail(st, "fps_poisson_cube_solve: " + err);
        plan->launches_last += plan->cube->launches_last;
        if (!xdev) {
            FPS_CK(cudaMemcpyAsync(Xr, Xd, sizeof(double) * n3, cudaMemcpyDeviceToHost, plan->stream));
            FPS_CK(cudaStreamSynchronize(plan->stream));
        }
    }
    if (!fdev && xdev) FPS_CK(cudaStreamSynchronize(plan->stream));
    FPS_CK(cudaGetLastError());
    return FPS_OK;
}

int fps_poisson_adjoint(fps_plan *plan, const double *dLdX, double *dLdF)
{
    // The solve map is self-adjoint (see fps.h): same ADI, same shifts.
    if (plan && plan->dim == 3) return fps_poisson_cube_solve(plan, dLdX, dLdF);
    return solve_square(plan, dLdX, dLdF, "fps_poisson_adjoint");
}

int fps_poisson_dirichlet_solve(fps_plan *plan, const double *G, const double *bc, double *U)
{
    const char *what = "fps_poisson_dirichlet_solve";
    fps::TraceRange tr(what);
    if (plan) {
        const size_t n = (size_t)plan->n, m = n + 2, R = (size_t)plan->nrhs;
        if (overlaps(U, 8 * R * m * m, G, 8 * R * n * n) || overlaps(U, 8 * R * m * m, bc, 8 * R * 4 * m))
            return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": U overlaps G or bc");
    }
    int st = dirichlet_check(plan, {G, bc, U}, what);
    if (st != FPS_OK) return st;
    DeviceGuard g(plan->device);
    const int64_t n = plan->n, m = n + 2;
    cudaStream_t s = plan->stream;
    FPS_CK(fps::launch_dirichlet_prep(bc, plan->dir_d2, plan->dir_ts, n, plan->nrhs, s));       // steps 1-2
    for (int r = 0; r < plan->nrhs; ++r)
        FPS_CK(fps::launch_legendre_to_ctilde(G + r * n * n, plan->dir_F + r * n * n, n, s));
    FPS_CK(fps::launch_dirichlet_rhs(plan->dir_F, plan->dir_d2, n, plan->nrhs, plan->kx, plan->ky, s));  // step 3
    st = solve_square(plan, plan->dir_F, plan->dir_X, what);
    if (st != FPS_OK && st != FPS_ERR_NOT_CONVERGED) return st;
    const std::string msg = st == FPS_OK ? std::string() : g_last_error;
    for (int r = 0; r < plan->nrhs; ++r)
        FPS_CK(fps::launch_solution_to_legendre(plan->dir_X + r * n * n, U + r * m * m, n, s));
    FPS_CK(fps::launch_dirichlet_lift(U, bc, plan->dir_ts, n, plan->nrhs, s));                   // step 4
    if (st != FPS_OK) return fail(st, msg);
    return FPS_OK;
}

int fps_poisson_dirichlet_adjoint(fps_plan *plan, const double *dLdU, double *dLdG, double *dLdbc)
{
    const char *what = "fps_poisson_dirichlet_adjoint";
    fps::TraceRange tr(what);
    if (plan) {
        const size_t n = (size_t)plan->n, m = n + 2, R = (size_t)plan->nrhs;
        if (overlaps(dLdU, 8 * R * m * m, dLdG, 8 * R * n * n) || overlaps(dLdU, 8 * R * m * m, dLdbc, 8 * R * 4 * m) ||
            overlaps(dLdG, 8 * R * n * n, dLdbc, 8 * R * 4 * m))
            return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": dLdU, dLdG and dLdbc must not overlap");
    }
    int st = dirichlet_check(plan, {dLdU, dLdG, dLdbc}, what);
    if (st != FPS_OK) return st;
    DeviceGuard g(plan->device);
    const int64_t n = plan->n, m = n + 2;
    cudaStream_t s = plan->stream;
    for (int r = 0; r < plan->nrhs; ++r)
        FPS_CK(fps::launch_solution_to_legendre_adjoint(dLdU + r * m * m, plan->dir_X + r * n * n, n, s));
    st = solve_square(plan, plan->dir_X, plan->dir_F, what);  // the solve map is self-adjoint
    if (st != FPS_OK && st != FPS_ERR_NOT_CONVERGED) return st;
    const std::string msg = st == FPS_OK ? std::string() : g_last_error;
    for (int r = 0; r < plan->nrhs; ++r)
        FPS_CK(fps::launch_legendre_to_ctilde_adjoint(plan->dir_F + r * n * n, dLdG + r * n * n, n, s));
    FPS_CK(fps::launch_dirichlet_bc_adjoint(dLdU, dLdG, dLdbc, n, plan->nrhs, plan->kx, plan->ky, s));
    if (st != FPS_OK) return fail(st, msg);
    return FPS_OK;
}

int fps_plan_create_cylinder(fps_plan **out, int64_t n, int64_t kmin, int64_t kmax, double tol, int nrhs,
                             void *stream)
{
    const char *what = "fps_plan_create_cylinder";
    if (!out) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": out is NULL");
    *out = nullptr;
    if (n < 4) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": n must be >= 4");
    if (n > 4096) return fail(FPS_ERR_UNSUPPORTED, std::string(what) + ": n must be <= 4096");
    if (kmin < 2 || kmax < kmin) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": need 2 <= kmin <= kmax");
    if (kmax - kmin + 1 > 65535 / std::max(nrhs, 1))
        return fail(FPS_ERR_UNSUPPORTED, std::string(what) + ": too many (mode, right-hand side) pairs");
    if (!(tol > 0.0 && tol < 1.0)) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": tol must lie in (0, 1)");
    if (nrhs < 1) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": nrhs must be >= 1");
    fps::TraceRange tr(what);
    fps_plan *p = new fps_plan();
    p->n = n;
    p->dim = 3;
    p->tol = tol;
    p->precision = FPS_FP64;
    p->nrhs = nrhs;
    p->stream = (cudaStream_t)stream;
    p->total_elems = (kmax - kmin + 1) * nrhs * n * n;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(FPS_ERR_CUDA, std::string(what) + ": no CUDA device");
    }
    p->cyl = new fps::CylinderEngine();
    std::string err;
    const int st = p->cyl->create(n, kmin, kmax, tol, nrhs, err);
    if (st != FPS_OK) {
        release(p);
        return fail(st, std::string(what) + ": " + err);
    }
    p->J = p->cyl->Jmax;
    p->bytes = p->cyl->bytes;
    *out = p;
    return FPS_OK;
}

int fps_poisson_cylinder_solve(fps_plan *plan, const double *F, double *Y)
{
    const char *what = "fps_poisson_cylinder_solve";
    fps::TraceRange tr(what);
    if (!plan || !plan->cyl) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": not a cylinder plan");
    if (!F || !Y) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": NULL F or Y");
    const size_t bytes = sizeof(double) * (size_t)plan->total_elems;
    const char *f0 = (const char *)F, *y0 = (const char *)Y;
    if (f0 < y0 + bytes && y0 < f0 + bytes) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": F and Y overlap");
    if (!is_device_pointer(F, plan->device) || !is_device_pointer(Y, plan->device))
        return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": F and Y must be device memory of the plan's device");
    DeviceGuard g(plan->device);
    std::string err;
    const int st = plan->cyl->solve(F, Y, plan->stream, err);
    plan->launches_last = plan->cyl->launches_last;
    if (st != FPS_OK) return fail(st, std::string(what) + ": " + err);
    return FPS_OK;
}

int fps_cylinder_mode_interval(int64_t n, int64_t k, double *a, double *b)
{
    if (n < 4 || n > 4096 || k < 2 || !a || !b)
        return fail(FPS_ERR_INVALID_ARG, "fps_cylinder_mode_interval: need 4 <= n <= 4096, k >= 2");
    if (fps::cyl_mode_interval(n, k, *a, *b) != FPS_OK)
        return fail(FPS_ERR_UNSUPPORTED, "fps_cylinder_mode_interval: power iteration failed");
    return FPS_OK;
}

int fps_cylinder_operators(int64_t n, int64_t k, double *L1, double *Q)
{
    if (n < 1 || n > 4096 || !L1 || !Q) return fail(FPS_ERR_INVALID_ARG, "fps_cylinder_operators: bad arguments");
    (void)k;
    for (int64_t a = 0; a < n; ++a)
        for (int64_t i = 0; i < n; ++i) {
            L1[a * n + i] = (std::llabs(a - i) == 2 || a == i) ? fps::cyl_L1(a, i) : 0.0;
            double mm = 0.0;
            auto Me = [](int64_t x, int64_t y) {
                if (x < 0 || y < 0) return 0.0;
                if (x == y) return fps::cyl_M_diag(x);
                if (x == y + 2) return fps::cyl_M_off(y);
                if (y == x + 2) return fps::cyl_M_off(x);
                return 0.0;
            };
            for (int64_t c = a - 2; c <= a + 2; c += 2) mm += Me(a, c) * Me(c, i);
            Q[a * n + i] = Me(a, i) - mm;
        }
    return FPS_OK;
}

int fps_plan_info(const fps_plan *plan, fps_plan_info_t *info)
{
    if (!plan || !info) return fail(FPS_ERR_INVALID_ARG, "fps_plan_info: NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->n = plan->n;
    info->dim = plan->dim;
    info->precision = plan->precision;
    info->nrhs = plan->nrhs;
    info->batch = plan->batch_ns.empty() ? 1 : (int64_t)plan->batch_ns.size();
    info->J = plan->J;
    info->J_inner = plan->eng32 ? plan->eng32->J_first : 0;
    info->refine_rounds = plan->eng32 ? plan->eng32->rounds_last : 0;
    info->last_residual = plan->eng32 ? plan->eng32->resid_last : 0.0;
    if (plan->cube) {
        info->J_inner = plan->cube->J_outer_inner;
        info->refine_rounds = plan->cube->rounds_last;
        info->last_residual = plan->cube->resid_last;
        info->inner_iterations = plan->cube->inner_iters;
    }
    info->tol = plan->tol;
    info->device_bytes = plan->bytes;
    info->kernel_launches = plan->launches_last;
    info->seg_len = plan->eng32 ? plan->eng32->seg_len : (plan->eng64 ? plan->eng64->seg_len : 0);
    info->chain_mode = plan->eng32 ? plan->eng32->chain_mode : (plan->eng64 ? plan->eng64->chain_mode : 0);
    return FPS_OK;
}

int fps_plan_set_instrument(fps_plan *p, int on)
{
    if (!p) return fail(FPS_ERR_INVALID_ARG, "fps_plan_set_instrument: plan is NULL");
    if (!p->eng32 && !p->eng64)
        return fail(FPS_ERR_UNSUPPORTED, "fps_plan_set_instrument: square plans on the pass kernels only");
    DeviceGuard g(p->device);
    FPS_CK(cudaStreamSynchronize(p->cap_stream));
    if (p->stream) FPS_CK(cudaStreamSynchronize(p->stream));
    else FPS_CK(cudaDeviceSynchronize());
    p->instrument = on != 0;
    std::string err;
    const int st = p->eng32 ? p->eng32->set_instrument(p->instrument, err) : p->eng64->set_instrument(p->instrument, err);
    return st == FPS_OK ? FPS_OK : fail(st, "fps_plan_set_instrument: " + err);
}

namespace {
int pass_times(fps_plan *p, int *count, double *total_ms, double *alg_bytes, double *row_ms, double *col_ms,
               const char *what)
{
    if (!p->instrument) return fail(FPS_ERR_INVALID_ARG, std::string(what) + ": plan is not instrumented");
    DeviceGuard g(p->device);
    if (p->stream) FPS_CK(cudaStreamSynchronize(p->stream));
    else FPS_CK(cudaDeviceSynchronize());
    std::string err;
    const int st = p->eng32 ? p->eng32->kernel_times(count, total_ms, alg_bytes, row_ms, col_ms, err)
                            : p->eng64->kernel_times(count, total_ms, alg_bytes, row_ms, col_ms, err);
    return st == FPS_OK ? FPS_OK : fail(st, std::string(what) + ": " + err);
}
}  // namespace

int fps_plan_kernel_times(fps_plan *p, int *count, double *total_ms, double *alg_bytes)
{
    if (!p || !count || !total_ms || !alg_bytes) return fail(FPS_ERR_INVALID_ARG, "fps_plan_kernel_times: NULL argument");
    return pass_times(p, count, total_ms, alg_bytes, nullptr, nullptr, "fps_plan_kernel_times");
}

int fps_plan_pass_times(fps_plan *p, double *row_ms, double *col_ms)
{
    if (!p || !row_ms || !col_ms) return fail(FPS_ERR_INVALID_ARG, "fps_plan_pass_times: NULL argument");
    int c = 0;
    double t = 0.0, b = 0.0;
    return pass_times(p, &c, &t, &b, row_ms, col_ms, "fps_plan_pass_times");
}

int fps_plan_shifts(const fps_plan *plan, int64_t problem, double *q, int cap)
{
    if (!plan || !q) return fail(FPS_ERR_INVALID_ARG, "fps_plan_shifts: bad argument");
    const std::vector<double> *v = &plan->q;
    const int64_t count = plan->batch_ns.empty() ? 1 : (int64_t)plan->batch_ns.size();
    if (problem < 0 || problem >= count) return fail(FPS_ERR_INVALID_ARG, "fps_plan_shifts: bad problem index");
    if (plan->eng32) v = &plan->eng32->shifts[problem];
    if (cap < (int)v->size()) return fail(FPS_ERR_INVALID_ARG, "fps_plan_shifts: capacity too small");
    std::memcpy(q, v->data(), sizeof(double) * v->size());
    return (int)v->size();
}

void fps_plan_destroy(fps_plan *plan)
{
    if (!plan) return;
    {
        DeviceGuard g(plan->device);
        if (plan->stream) cudaStreamSynchronize(plan->stream);
        else cudaDeviceSynchronize();
    }
    release(plan);
}

const char *fps_status_string(int status)
{
    switch (status) {
    case FPS_OK: return "ok";
    case FPS_ERR_INVALID_ARG: return "invalid argument";
    case FPS_ERR_UNSUPPORTED: return "unsupported";
    case FPS_ERR_CUDA: return "CUDA error";
    case FPS_ERR_NOT_CONVERGED: return "refinement did not converge";
    case FPS_ERR_NONFINITE: return "non-finite input";
    case FPS_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

const char *fps_last_error(void) { return g_static_error ? g_static_error : g_last_error.c_str(); }

int fps_zolotarev_shifts(double a, double b, double c, double d, double tol, int J, int *J_out, double *p, double *q,
                         int cap)
{
    if (!(a < b && b < c && c < d)) return fail(FPS_ERR_INVALID_ARG, "fps_zolotarev_shifts: need a < b < c < d");
    if (!(tol > 0.0 && tol < 1.0)) return fail(FPS_ERR_INVALID_ARG, "fps_zolotarev_shifts: tol must lie in (0,1)");
    if (J <= 0) J = fps::adi_iterations(a, b, c, d, tol);
    if (J_out) *J_out = J;
    if (!p && !q) return FPS_OK;
    if (cap < J) return fail(FPS_ERR_INVALID_ARG, "fps_zolotarev_shifts: capacity too small");
    std::vector<double> pv, qv;
    if (c == -b && d == -a) {
        fps::zolotarev_shifts_symmetric(c, d, J, qv);
        pv.resize(J);
        for (int j = 0; j < J; ++j) pv[j] = -qv[j];
    } else {
        fps::zolotarev_shifts(a, b, c, d, J, pv, qv);
    }
    if (p) std::memcpy(p, pv.data(), sizeof(double) * J);
    if (q) std::memcpy(q, qv.data(), sizeof(double) * J);
    return FPS_OK;
}

int fps_square_bands(int64_t n, double *d, double *e)
{
    if (n < 1 || !d || !e) return fail(FPS_ERR_INVALID_ARG, "fps_square_bands: bad argument");
    std::vector<double> dv, ev;
    fps::square_bands(n, dv, ev);
    std::memcpy(d, dv.data(), sizeof(double) * n);
    if (n > 2) std::memcpy(e, ev.data(), sizeof(double) * (n - 2));
    return FPS_OK;
}

int fps_square_spectral_interval(int64_t n, int tight, double *lo, double *hi)
{
    if (n < 1 || !lo || !hi) return fail(FPS_ERR_INVALID_ARG, "fps_square_spectral_interval: bad argument");
    if (tight) {
        fps::square_tight_interval(n, *lo, *hi);
    } else {
        *lo = fps::square_eps(n);
        *hi = 1.0;
    }
    return FPS_OK;
}

int fps_build_arch(void) { return 103; }

int fps_legendre_to_ctilde(int64_t n, const double *G, double *F, void *stream)
{
    if (n < 1) return fail(FPS_ERR_INVALID_ARG, "fps_legendre_to_ctilde: n must be >= 1");
    if (!G || !F) return fail(FPS_ERR_INVALID_ARG, "fps_legendre_to_ctilde: NULL G or F");
    const size_t bytes = sizeof(double) * (size_t)n * (size_t)n;
    const char *g0 = (const char *)G, *f0 = (const char *)F;
    if (g0 < f0 + bytes && f0 < g0 + bytes) return fail(FPS_ERR_INVALID_ARG, "fps_legendre_to_ctilde: G and F overlap");
    const int dev = current_device();
    if (!is_device_pointer(G, dev) || !is_device_pointer(F, dev))
        return fail(FPS_ERR_INVALID_ARG, "fps_legendre_to_ctilde: G and F must be device memory of the current device");
    FPS_CK(fps::launch_legendre_to_ctilde(G, F, n, (cudaStream_t)stream));
    return FPS_OK;
}

int fps_solution_to_legendre(int64_t n, const double *X, double *U, void *stream)
{
    if (n < 1) return fail(FPS_ERR_INVALID_ARG, "fps_solution_to_legendre: n must be >= 1");
    if (!X || !U) return fail(FPS_ERR_INVALID_ARG, "fps_solution_to_legendre: NULL X or U");
    const size_t xb = sizeof(double) * (size_t)n * (size_t)n;
    const size_t ub = sizeof(double) * (size_t)(n + 2) * (size_t)(n + 2);
    const char *x0 = (const char *)X, *u0 = (const char *)U;
    if (x0 < u0 + ub && u0 < x0 + xb) return fail(FPS_ERR_INVALID_ARG, "fps_solution_to_legendre: X and U overlap");
    const int dev = current_device();
    if (!is_device_pointer(X, dev) || !is_device_pointer(U, dev))
        return fail(FPS_ERR_INVALID_ARG, "fps_solution_to_legendre: X and U must be device memory of the current device");
    FPS_CK(fps::launch_solution_to_legendre(X, U, n, (cudaStream_t)stream));
    return FPS_OK;
}

}  // extern "C"
