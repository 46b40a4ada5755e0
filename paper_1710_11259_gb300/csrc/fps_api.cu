// C ABI of the solver (include/fps.h): plans, solves, adjoint, host helpers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fps.h"
#include "host_math.h"
#include "kernels.cuh"
#include "refine_engine.h"
#include "cube.h"
#include "legendre.cuh"
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

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

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
    cudaStream_t cap_stream = nullptr;  // private stream used to capture the graph

    int J = 0;
    std::vector<double> q;  // shifts q_j > 0 (p_j = -q_j)

    // device data
    double *d_d = nullptr, *d_e = nullptr, *d_s = nullptr, *d_q = nullptr;
    double2 *d_fac = nullptr;
    double *Ft = nullptr, *FtT = nullptr, *A = nullptr, *B = nullptr, *Z = nullptr;
    int64_t bytes = 0;

    cudaGraphExec_t graph = nullptr;
    int refine_rounds = 0;
    double last_residual = 0;

    // FPS_FP32_REFINE (single problem or batch): the refinement engine
    fps::RefineEngine *eng = nullptr;
    // dim = 3: the nested cube ADI
    fps::CubeEngine *cube = nullptr;
    std::vector<int64_t> batch_ns;   // sizes of a batched plan (empty otherwise)
    int64_t total_elems = 0;         // doubles in F (and X) for all right-hand sides / problems
    double *stage_in = nullptr, *stage_out = nullptr;  // lazily allocated for host pointers

    // instrumentation and accounting (FP64 path)
    bool instrument = false;
    std::vector<cudaEvent_t> ev64;          // FP64: 2 per half-step
    int64_t launches_last = 0;
};

namespace {

template <typename T>
cudaError_t dmalloc(fps_plan *p, T **ptr, size_t count)
{
    cudaError_t e = cudaMalloc((void **)ptr, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) p->bytes += (int64_t)(sizeof(T) * count);
    return e;
}

void release(fps_plan *p)
{
    if (!p) return;
    DeviceGuard g(p->device);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    void *bufs[] = {p->d_d, p->d_e, p->d_s, p->d_q, p->d_fac, p->Ft, p->FtT, p->A, p->B, p->Z, p->stage_in,
                    p->stage_out};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (cudaEvent_t e : p->ev64) cudaEventDestroy(e);
    if (p->eng) {
        p->eng->release();
        delete p->eng;
    }
    if (p->cube) {
        p->cube->release();
        delete p->cube;
    }
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
}

// Enqueue the 2J half-steps of Algorithm 2 (FP64) from F~, F~^T to Y_J (normal
// orientation) in p->B.  Buffers: A holds Y_{j+1/2} (normal), B holds Y_j^T.
cudaError_t enqueue_adi_fp64(fps_plan *p, cudaStream_t st)
{
    const int64_t n = p->n;
    for (int j = 0; j < p->J; ++j) {
        fps::HalfStep<double> h;
        h.d = p->d_d;
        h.e = p->d_e;
        h.q = p->q[j];
        h.n = n;
        h.Z = p->Z;
        h.fac = p->d_fac + (int64_t)j * n;
        // step 1 (transposed form): (A~ - q) Y_h^T = F~^T - Y^T (A~ + q); store Y_h
        h.V = (j == 0) ? nullptr : p->B;
        h.G = p->FtT;
        h.Out = p->A;
        h.transposed_out = true;
        const bool ins = p->instrument && (int)p->ev64.size() == 4 * p->J;
        cudaError_t e;
        if (ins && (e = cudaEventRecordWithFlags(p->ev64[4 * j], st, cudaEventRecordExternal)) != cudaSuccess) return e;
        e = fps::launch_halfstep(h, st);
        if (e != cudaSuccess) return e;
        if (ins && (e = cudaEventRecordWithFlags(p->ev64[4 * j + 1], st, cudaEventRecordExternal)) != cudaSuccess)
            return e;
        // step 2: (A~ - q) Y^+ = F~ - Y_h (A~ + q); store (Y^+)^T, or Y_J itself last
        h.V = p->A;
        h.G = p->Ft;
        h.Out = p->B;
        h.transposed_out = (j + 1 < p->J);
        if (ins && (e = cudaEventRecordWithFlags(p->ev64[4 * j + 2], st, cudaEventRecordExternal)) != cudaSuccess)
            return e;
        e = fps::launch_halfstep(h, st);
        if (e != cudaSuccess) return e;
        if (ins && (e = cudaEventRecordWithFlags(p->ev64[4 * j + 3], st, cudaEventRecordExternal)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

int build_graph(fps_plan *p)
{
    FPS_CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_adi_fp64(p, p->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(FPS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    FPS_CK(e2);
    e = cudaGraphInstantiate(&p->graph, g, 0);
    cudaGraphDestroy(g);
    FPS_CK(e);
    return FPS_OK;
}

// One right-hand side, device pointers (FP64 path).
int solve_one(fps_plan *p, const double *F, double *X)
{
    cudaStream_t st = p->stream;
    FPS_CK(fps::launch_scale_in(F, p->Ft, p->FtT, p->d_s, p->n, st));
    FPS_CK(cudaGraphLaunch(p->graph, st));
    FPS_CK(fps::launch_scale_out(p->B, X, p->d_s, p->n, st));
    p->launches_last += 2LL * p->J + 2;
    return FPS_OK;
}

// FP32_REFINE (single or batched): the whole packed F at once.
int solve_engine(fps_plan *p, const double *F, double *X, bool fdev, bool xdev, const char *what)
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
    const int st = p->eng->solve(Fd, Xd, p->stream, err);
    if (st != FPS_OK && st != FPS_ERR_NOT_CONVERGED) return fail(st, std::string(what) + ": " + err);
    p->launches_last = p->eng->launches_last;
    if (!xdev) {
        FPS_CK(cudaMemcpyAsync(X, Xd, bytes, cudaMemcpyDeviceToHost, p->stream));
        FPS_CK(cudaStreamSynchronize(p->stream));
    }
    if (st != FPS_OK) return fail(st, std::string(what) + ": " + err);
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
    const bool fdev = is_device_pointer(F), xdev = is_device_pointer(X);
    p->launches_last = 0;
    if (p->eng) return solve_engine(p, F, X, fdev, xdev, what);
    const int64_t nn = p->n * p->n;
    for (int r = 0; r < p->nrhs; ++r) {
        const double *Fr = F + (int64_t)r * nn;
        double *Xr = X + (int64_t)r * nn;
        const double *Fd = Fr;
        if (!fdev) {
            FPS_CK(cudaMemcpyAsync(p->B, Fr, sizeof(double) * nn, cudaMemcpyHostToDevice, p->stream));
            Fd = p->B;
        }
        double *Xd = xdev ? Xr : p->A;
        int s = solve_one(p, Fd, Xd);
        if (s != FPS_OK) return s;
        if (!xdev) {
            FPS_CK(cudaMemcpyAsync(Xr, p->A, sizeof(double) * nn, cudaMemcpyDeviceToHost, p->stream));
            FPS_CK(cudaStreamSynchronize(p->stream));
        }
    }
    if (!fdev && xdev) FPS_CK(cudaStreamSynchronize(p->stream));  // host F must stay valid only until copied
    FPS_CK(cudaGetLastError());
    return FPS_OK;
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
    if (precision != FPS_FP64 && precision != FPS_FP32_REFINE)
        return fail(FPS_ERR_INVALID_ARG, "fps_plan_create: unknown precision");
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

    fps_plan *p = new fps_plan();
    p->n = n;
    p->dim = dim;
    p->tol = tol;
    p->precision = precision;
    p->nrhs = nrhs;
    p->stream = (cudaStream_t)stream;
    p->total_elems = n * n * nrhs;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(FPS_ERR_CUDA, "fps_plan_create: no CUDA device");
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

    // Lemma B.2 interval, (2.9) J, (2.4) shifts (symmetric intervals: p_j = -q_j).
    const double eps = fps::square_eps(n);
    p->J = fps::adi_iterations(-1.0, -eps, eps, 1.0, tol);
    fps::zolotarev_shifts_symmetric(eps, 1.0, p->J, p->q);
    std::vector<double> d, e, s;
    fps::square_bands(n, d, e);
    fps::inv_sqrt_E(n, s);

    const size_t nn = (size_t)n * (size_t)n;
    PCK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    PCK(dmalloc(p, &p->d_d, n));
    PCK(dmalloc(p, &p->d_e, n));
    PCK(dmalloc(p, &p->d_s, n));
    PCK(dmalloc(p, &p->d_q, p->J));
    if (precision == FPS_FP64) {
        PCK(dmalloc(p, &p->Ft, nn));
        PCK(dmalloc(p, &p->d_fac, (size_t)p->J * n));
        PCK(dmalloc(p, &p->FtT, nn));
        PCK(dmalloc(p, &p->A, nn));
        PCK(dmalloc(p, &p->B, nn));
        PCK(dmalloc(p, &p->Z, nn));
    }
    PCK(cudaMemcpyAsync(p->d_d, d.data(), sizeof(double) * n, cudaMemcpyHostToDevice, p->cap_stream));
    PCK(cudaMemcpyAsync(p->d_e, e.data(), sizeof(double) * n, cudaMemcpyHostToDevice, p->cap_stream));
    PCK(cudaMemcpyAsync(p->d_s, s.data(), sizeof(double) * n, cudaMemcpyHostToDevice, p->cap_stream));
    PCK(cudaMemcpyAsync(p->d_q, p->q.data(), sizeof(double) * p->J, cudaMemcpyHostToDevice, p->cap_stream));
    if (precision == FPS_FP64) {
        PCK(fps::launch_factors(p->d_d, p->d_e, p->d_q, p->J, n, p->d_fac, p->cap_stream));
        PCK(cudaStreamSynchronize(p->cap_stream));
        int st = build_graph(p);
        if (st != FPS_OK) return bail(st);
    } else {
        if (n > 40000) return bail(fail(FPS_ERR_UNSUPPORTED, "fps_plan_create: FP32_REFINE supports n <= 40000"));
        if (nrhs > 256) return bail(fail(FPS_ERR_UNSUPPORTED, "fps_plan_create: FP32_REFINE supports nrhs <= 256"));
        PCK(cudaStreamSynchronize(p->cap_stream));
        p->eng = new fps::RefineEngine();
        std::string err;
        const int st = p->eng->create(std::vector<int64_t>{n}, nrhs, tol, p->cap_stream, 0, err);
        if (st != FPS_OK) return bail(fail(st, "fps_plan_create: " + err));
        p->bytes += p->eng->bytes;
    }
#undef PCK
    *out = p;
    return FPS_OK;
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
    p->eng = new fps::RefineEngine();
    std::string err;
    const int st = p->eng->create(v, nrhs, tol, p->cap_stream, 0, err);
    if (st != FPS_OK) {
        release(p);
        return fail(st, "fps_plan_create_batched: " + err);
    }
    p->bytes += p->eng->bytes;
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
    const bool fdev = is_device_pointer(F), xdev = is_device_pointer(X);
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
    info->J_inner = plan->eng ? plan->eng->J_inner_first : 0;
    info->refine_rounds = plan->eng ? plan->eng->rounds_last : 0;
    info->last_residual = plan->eng ? plan->eng->resid_last : 0.0;
    if (plan->cube) {
        info->J_inner = plan->cube->J_outer_inner;
        info->refine_rounds = plan->cube->rounds_last;
        info->last_residual = plan->cube->resid_last;
        info->inner_iterations = plan->cube->inner_iters;
    }
    info->tol = plan->tol;
    info->device_bytes = plan->bytes;
    info->kernel_launches = plan->launches_last;
    info->pass_ctas = plan->eng ? plan->eng->chosen_target_ctas : 0;
    return FPS_OK;
}

int fps_plan_set_instrument(fps_plan *p, int on)
{
    if (!p) return fail(FPS_ERR_INVALID_ARG, "fps_plan_set_instrument: plan is NULL");
    DeviceGuard g(p->device);
    FPS_CK(cudaStreamSynchronize(p->cap_stream));
    if (p->stream) FPS_CK(cudaStreamSynchronize(p->stream));
    else FPS_CK(cudaDeviceSynchronize());
    p->instrument = on != 0;
    if (p->eng) {
        std::string err;
        const int st = p->eng->set_instrument(p->instrument, err);
        return st == FPS_OK ? FPS_OK : fail(st, "fps_plan_set_instrument: " + err);
    }
    for (cudaEvent_t e : p->ev64) cudaEventDestroy(e);
    p->ev64.clear();
    if (p->instrument) {
        p->ev64.resize(4 * (size_t)p->J);
        for (auto &e : p->ev64) FPS_CK(cudaEventCreate(&e));
    }
    if (p->graph) cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
    return build_graph(p);
}

int fps_plan_kernel_times(fps_plan *p, int *count, double *total_ms, double *alg_bytes)
{
    if (!p || !count || !total_ms || !alg_bytes) return fail(FPS_ERR_INVALID_ARG, "fps_plan_kernel_times: NULL argument");
    if (!p->instrument) return fail(FPS_ERR_INVALID_ARG, "fps_plan_kernel_times: plan is not instrumented");
    DeviceGuard g(p->device);
    if (p->stream) FPS_CK(cudaStreamSynchronize(p->stream));
    else FPS_CK(cudaDeviceSynchronize());
    if (p->eng) {
        std::string err;
        const int st = p->eng->kernel_times(count, total_ms, alg_bytes, err);
        return st == FPS_OK ? FPS_OK : fail(st, "fps_plan_kernel_times: " + err);
    }
    const double nn = (double)p->n * (double)p->n;
    int c = 0;
    double ms = 0.0, bytes = 0.0;
    for (int k = 0; k < 2 * p->J; ++k) {
        float t = 0.f;
        FPS_CK(cudaEventElapsedTime(&t, p->ev64[2 * k], p->ev64[2 * k + 1]));
        ms += t;
        ++c;
        bytes += (k == 0 ? 2.0 : 3.0) * 8.0 * nn;  // V (unless zero), G read; W written
    }
    *count = c;
    *total_ms = ms;
    *alg_bytes = bytes;
    return FPS_OK;
}

int fps_plan_shifts(const fps_plan *plan, int64_t problem, double *q, int cap)
{
    if (!plan || !q || problem != 0) return fail(FPS_ERR_INVALID_ARG, "fps_plan_shifts: bad argument");
    if (cap < plan->J) return fail(FPS_ERR_INVALID_ARG, "fps_plan_shifts: capacity too small");
    std::memcpy(q, plan->q.data(), sizeof(double) * plan->J);
    return plan->J;
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
    if (!is_device_pointer(G) || !is_device_pointer(F))
        return fail(FPS_ERR_INVALID_ARG, "fps_legendre_to_ctilde: G and F must be device memory");
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
    if (!is_device_pointer(X) || !is_device_pointer(U))
        return fail(FPS_ERR_INVALID_ARG, "fps_solution_to_legendre: X and U must be device memory");
    FPS_CK(fps::launch_solution_to_legendre(X, U, n, (cudaStream_t)stream));
    return FPS_OK;
}

}  // extern "C"
