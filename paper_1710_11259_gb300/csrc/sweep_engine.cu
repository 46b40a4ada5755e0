// Host side of the square solve on the ADI pass kernels (sweep.cu), one problem or
// a batch.
//
// FP32 (refinement), per solve:
//   smax = max |F~| per (problem, rhs) pair; F~ = D_s F D_s; rho_0 = F~ / smax
//   round r: inner ADI in FP32 (one CUDA graph per tolerance level: every pass
//            launch covers every problem; a finalize kernel adds the last c) gives
//            the correction D; the FP64 residual kernel applies Y += smax D, forms
//            R~ = F~ - A~Y - YA~ and the next rho_0; pairs with max|R~| <= tol smax
//            stop (their iterate is carried unchanged).
//   X = D_s Y D_s.
// The inner tolerance of a round is the coarsest level that still gains ten times
// what the worst active pair is missing; the first round stops at the coarsest
// level not above sqrt(0.1 tol), so that two rounds of equal gain reach tol (the
// finest level, 1e-7, is about what one FP32 inner solve can deliver).  Inner shifts come from the
// tight spectral interval of A~ (the refinement is judged by the FP64 residual).
// FP64 (plain method): rho_0 = F~, one graph of J iterations of (2.9), then
// X = D_s Y_J D_s fused with the last correction.
#include "sweep_engine.h"
#include "trace.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>

#include <sys/stat.h>

#include "../../include/fps.h"
#include "host_math.h"

namespace fps {

namespace {
double bits_to_double(unsigned long long b)
{
    double d;
    std::memcpy(&d, &b, sizeof(d));
    return d;
}
const double kLevelTols[] = {1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2};
constexpr int kTileW = 64;       // rows of a row-pass tile / columns of a column-pass tile
constexpr int kChainLines = 64;
}  // namespace

template <typename T>
template <typename U>
cudaError_t SweepEngine<T>::dalloc(U **p, size_t count)
{
    cudaError_t e = cudaMalloc((void **)p, sizeof(U) * (count ? count : 1));
    if (e == cudaSuccess) {
        bytes += (int64_t)(sizeof(U) * count);
        allocs_.push_back((void *)*p);
    }
    return e;
}

template <typename T>
void SweepEngine<T>::release()
{
    for (auto &L : levels_) {
        for (cudaEvent_t e : L.ev) cudaEventDestroy(e);
        if (L.graph) cudaGraphExecDestroy(L.graph);
    }
    levels_.clear();
    for (void *p : allocs_) cudaFree(p);
    allocs_.clear();
    void *hp[] = {h_active_, h_pair_active_, h_smax_, h_rmax_, h_err_};
    for (void *p : hp)
        if (p) cudaFreeHost(p);
    h_active_ = h_pair_active_ = nullptr;
    h_smax_ = h_rmax_ = nullptr;
    h_err_ = nullptr;
}

#define ENG_CK(call)                                                                                     \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                                    \
            return FPS_ERR_CUDA;                                                                         \
        }                                                                                                \
    } while (0)

// ---------------------------------------------------------------------------
// Autotuner of the segment length (the tile height of the column pass and width of
// the row pass; it also fixes the number of segments a chain walks).  Every
// candidate gets a complete engine of its own on the same sizes; the graph of the
// coarsest tolerance level is timed with CUDA events and the fastest candidate
// kept.  Results are cached per (GPU name, nrhs, size list) in $FPS_AUTOTUNE_CACHE
// (default ~/.cache/fps_gb300_autotune.txt); FPS_AUTOTUNE=0 skips tuning (128).
// ---------------------------------------------------------------------------
namespace {
std::string tune_key(const std::vector<int64_t> &ns, int nrhs)
{
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    uint64_t h = 1469598103934665603ULL;  // FNV-1a over the sizes
    for (int64_t n : ns) {
        for (int b = 0; b < 8; ++b) {
            h ^= (uint64_t)((n >> (8 * b)) & 0xff);
            h *= 1099511628211ULL;
        }
    }
    std::ostringstream os;
    os << "seg|" << name << "|" << nrhs << "|" << ns.size() << "|" << std::hex << h;
    return os.str();
}

std::string tune_cache_path()
{
    const char *p = std::getenv("FPS_AUTOTUNE_CACHE");
    if (p && *p) return p;
    const char *home = std::getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/fps_gb300_autotune.txt";
}
}  // namespace

template <typename T>
int SweepEngine<T>::time_level(size_t li, int reps, float &ms, std::string &err)
{
    cudaEvent_t e0, e1;
    ENG_CK(cudaEventCreate(&e0));
    ENG_CK(cudaEventCreate(&e1));
    ENG_CK(cudaGraphLaunch(levels_[li].graph, cap_));  // warm-up
    ENG_CK(cudaEventRecord(e0, cap_));
    for (int r = 0; r < reps; ++r) ENG_CK(cudaGraphLaunch(levels_[li].graph, cap_));
    ENG_CK(cudaEventRecord(e1, cap_));
    ENG_CK(cudaEventSynchronize(e1));
    ENG_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ms /= (float)reps;
    return FPS_OK;
}

// Mean time of a chain launch (both directions alternately) with the given load
// batching, on this engine's arrays (the values do not change the time).
template <typename T>
int SweepEngine<T>::time_chain(int mode, float &ms, std::string &err)
{
    SwArgs<T> a = args(levels_.back(), 2);
    a.chain_mode = mode;
    cudaEvent_t e0, e1;
    ENG_CK(cudaEventCreate(&e0));
    ENG_CK(cudaEventCreate(&e1));
    ENG_CK(launch_chain(a, 0, 0, cap_));  // warm-up
    ENG_CK(cudaEventRecord(e0, cap_));
    constexpr int kReps = 20;
    for (int r = 0; r < kReps; ++r) ENG_CK(launch_chain(a, r & 1, 0, cap_));
    ENG_CK(cudaEventRecord(e1, cap_));
    ENG_CK(cudaEventSynchronize(e1));
    ENG_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ms /= (float)kReps;
    return FPS_OK;
}

template <typename T>
int SweepEngine<T>::autotune(const std::vector<int64_t> &ns, int nrhs, double tol, bool tight, std::string &err)
{
    seg_len = 128;
    const char *env = std::getenv("FPS_AUTOTUNE");
    if (env && std::string(env) == "0") return FPS_OK;
    const std::string key = tune_key(ns, nrhs);
    const std::string path = tune_cache_path();
    {
        std::ifstream in(path);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string k;
            int v = 0, cm = 0;
            if (!(ls >> k >> v)) continue;
            if (!(ls >> cm) || cm < 0 || cm > 2) cm = 0;  // entries without a chain mode: by grid size
            if (k == key && sweep_segment_supported(false, v)) {
                seg_len = v;
                chain_mode = cm;
                return FPS_OK;
            }
        }
    }
    // tile shape: the segment length of the passes (a whole graph level timed per
    // candidate); then the chain kernel's load batching, timed on the winner's arrays
    const int cand[] = {64, 128};
    float best = 3.4e38f;
    tune_ms.clear();
    for (int S : cand) {
        SweepEngine<T> t;
        std::string e2;
        int st = t.create(ns, nrhs, tol, tight, cap_, e2, S, kx_, ky_);
        float ms = 0.f, c1 = 0.f, c2 = 0.f;
        if (st == FPS_OK) st = t.time_level(t.levels_.size() - 1, 2, ms, e2);
        if (st == FPS_OK) st = t.time_chain(1, c1, e2);
        if (st == FPS_OK) st = t.time_chain(2, c2, e2);
        t.release();
        if (st != FPS_OK) {
            err = "autotune: " + e2;
            return st;
        }
        tune_ms.push_back(ms);
        if (ms < best) {
            best = ms;
            seg_len = S;
            chain_mode = c2 < c1 ? 2 : 1;
        }
    }
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // may exist
    std::ofstream out(path, std::ios::app);
    if (out) out << key << " " << seg_len << " " << chain_mode << "\n";
    return FPS_OK;
}

template <typename T>
int SweepEngine<T>::create(const std::vector<int64_t> &ns, int nrhs, double tol, bool tight,
                           cudaStream_t setup_stream, std::string &err, int seg, double kx, double ky)
{
    kx_ = kx;
    ky_ = ky;
    constexpr bool kFP64 = sizeof(T) == 8;
    ns_ = ns;
    nrhs_ = nrhs;
    tol_ = tol;
    cap_ = setup_stream;
    const int np = (int)ns.size();
    if (const char *mr = std::getenv("FPS_MAX_REFINE_ROUNDS")) {  // cap on refinement rounds (>= 1)
        const int v = std::atoi(mr);
        if (v >= 1) max_rounds = v;
    }
    if (seg <= 0) {
        if (kFP64) {
            seg_len = 64;
        } else {
            const int st = autotune(ns, nrhs, tol, tight, err);
            if (st != FPS_OK) return st;
        }
    } else {
        if (!sweep_segment_supported(kFP64, seg)) {
            err = "unsupported segment length";
            return FPS_ERR_INVALID_ARG;
        }
        seg_len = seg;
    }
    const int S = seg_len;
    N_.resize(np);
    P_.resize(np);
    off64_.resize(np);
    offT_.resize(np);
    offS_.resize(np);
    tot64_ = totT_ = totS_ = 0;
    int64_t totBT = 0, totB64 = 0;
    for (int p = 0; p < np; ++p) {
        const int64_t n = ns[p];
        const int N = (int)((n + kTileW - 1) / kTileW * kTileW);
        N_[p] = N;
        P_[p] = (N + S - 1) / S;
        off64_[p] = tot64_;
        offT_[p] = totT_;
        offS_[p] = totS_;
        tot64_ += (int64_t)nrhs * n * n;
        totT_ += (int64_t)nrhs * (N + 4) * (N + 8);
        totS_ += (int64_t)nrhs * P_[p] * 2 * (N + 8);
        totBT += 2 * (int64_t)(N + 4);
        totB64 += 3 * n;
    }
    npairs_ = np * nrhs;

    ENG_CK(sweep_setup_kernels());
    if (!kFP64) {
        ENG_CK(dalloc(&Ft_, (size_t)tot64_));
        ENG_CK(dalloc(&Y0_, (size_t)tot64_));
        ENG_CK(dalloc(&Y1_, (size_t)tot64_));
    }
    ENG_CK(dalloc(&bands64_, (size_t)totB64));
    ENG_CK(dalloc(&bandsT_, (size_t)totBT));
    ENG_CK(dalloc(&rho0_, (size_t)totT_));
    ENG_CK(dalloc(&cl_, (size_t)totT_));
    ENG_CK(dalloc(&al_, (size_t)totT_));
    ENG_CK(dalloc(&D_, (size_t)totT_));
    ENG_CK(dalloc(&zin_, (size_t)totS_));
    ENG_CK(dalloc(&sumR_, (size_t)totS_));
    ENG_CK(dalloc(&sumC_, (size_t)totS_));
    ENG_CK(dalloc(&zxR_, (size_t)totS_));
    ENG_CK(dalloc(&zxC_, (size_t)totS_));
    ENG_CK(dalloc(&err_, 1));
    ENG_CK(dalloc(&d_active_, (size_t)np));
    ENG_CK(dalloc(&d_pair_active_, (size_t)npairs_));
    ENG_CK(dalloc(&d_smax_, (size_t)npairs_));
    ENG_CK(dalloc(&d_rmax_, (size_t)npairs_));
    ENG_CK(cudaMallocHost((void **)&h_active_, sizeof(int) * np));
    ENG_CK(cudaMallocHost((void **)&h_pair_active_, sizeof(int) * npairs_));
    ENG_CK(cudaMallocHost((void **)&h_smax_, sizeof(unsigned long long) * npairs_));
    ENG_CK(cudaMallocHost((void **)&h_rmax_, sizeof(unsigned long long) * npairs_));
    ENG_CK(cudaMallocHost((void **)&h_err_, sizeof(int)));
    *h_err_ = 0;
    // padding must be zero and stays zero
    {
        T *tb[] = {rho0_, cl_, al_, D_};
        for (T *b : tb) ENG_CK(cudaMemsetAsync(b, 0, sizeof(T) * (size_t)totT_, cap_));
        ENG_CK(cudaMemsetAsync(zin_, 0, sizeof(T) * (size_t)totS_, cap_));
        T2 *sb[] = {sumR_, sumC_, zxR_, zxC_};
        for (T2 *b : sb) ENG_CK(cudaMemsetAsync(b, 0, sizeof(T2) * (size_t)totS_, cap_));
        ENG_CK(cudaMemsetAsync(err_, 0, sizeof(int), cap_));
    }

    // bands: FP64 (d, e zero-padded, 1/sqrt(E)) and padded T copies (index i + 2)
    std::vector<double> hb64((size_t)totB64);
    std::vector<T> hbT((size_t)totBT, T(0));
    std::vector<TileProb> tp(np);
    std::vector<int4> tiles;
    std::vector<int64_t> ob64(np), obT(np);
    {
        int64_t o64 = 0, oT = 0;
        std::vector<double> d, e, s;
        for (int p = 0; p < np; ++p) {
            const int64_t n = ns[p];
            const int N = N_[p];
            square_bands(n, d, e);
            inv_sqrt_E(n, s);
            std::copy(d.begin(), d.end(), hb64.begin() + o64);
            std::copy(e.begin(), e.end(), hb64.begin() + o64 + n);
            std::copy(s.begin(), s.end(), hb64.begin() + o64 + 2 * n);
            for (int64_t i = 0; i < n; ++i) {
                hbT[oT + i + 2] = (T)d[i];
                hbT[oT + (N + 4) + i + 2] = (T)e[i];
            }
            ob64[p] = o64;
            obT[p] = oT;
            TileProb &t = tp[p];
            t.n = (int)n;
            t.ldp = N + 8;
            t.off64 = off64_[p];
            t.off = offT_[p];
            t.rhs = (int64_t)(N + 4) * (N + 8);
            t.d = bands64_ + o64;
            t.e = bands64_ + o64 + n;
            t.s = bands64_ + o64 + 2 * n;
            t.pair0 = p * nrhs;
            t.kx = kx_;
            t.ky = ky_;
            o64 += 3 * n;
            oT += 2 * (N + 4);
            const int nt = (int)((n + 31) / 32);
            for (int r = 0; r < nrhs; ++r)
                for (int ty = 0; ty < nt; ++ty)
                    for (int tx = 0; tx < nt; ++tx) tiles.push_back(make_int4(p * 256 + r, tx, ty, 0));
        }
    }
    ntiles_ = (int64_t)tiles.size();
    ENG_CK(dalloc(&d_tp_, (size_t)np));
    ENG_CK(dalloc(&d_tiles_, (size_t)ntiles_));
    ENG_CK(cudaMemcpyAsync(bands64_, hb64.data(), sizeof(double) * totB64, cudaMemcpyHostToDevice, cap_));
    ENG_CK(cudaMemcpyAsync(bandsT_, hbT.data(), sizeof(T) * totBT, cudaMemcpyHostToDevice, cap_));
    ENG_CK(cudaMemcpyAsync(d_tp_, tp.data(), sizeof(TileProb) * np, cudaMemcpyHostToDevice, cap_));
    ENG_CK(cudaMemcpyAsync(d_tiles_, tiles.data(), sizeof(int4) * ntiles_, cudaMemcpyHostToDevice, cap_));

    // work items, largest problems first; a row pass sweeps row blocks down each column segment
    {
        std::vector<int> order(np);
        for (int p = 0; p < np; ++p) order[p] = p;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ns[a] > ns[b]; });
        std::vector<int4> it[3];
        for (int p : order) {
            const int nb = N_[p] / kTileW, P = P_[p], nl = (N_[p] + kChainLines - 1) / kChainLines;
            for (int r = 0; r < nrhs; ++r) {
                for (int sg = 0; sg < P; ++sg)
                    for (int b = 0; b < nb; ++b) {
                        it[0].push_back(make_int4(p, r, b, sg));
                        it[1].push_back(make_int4(p, r, b, sg));
                    }
                for (int b = 0; b < nl; ++b) it[2].push_back(make_int4(p, r, b, 0));
            }
        }
        for (int w = 0; w < 3; ++w) {
            nitems_[w] = (int64_t)it[w].size();
            ENG_CK(dalloc(&d_items_[w], (size_t)nitems_[w]));
            ENG_CK(cudaMemcpyAsync(d_items_[w], it[w].data(), sizeof(int4) * nitems_[w], cudaMemcpyHostToDevice, cap_));
        }
    }
    for (int p = 0; p < np; ++p) h_active_[p] = 1;
    for (int k = 0; k < npairs_; ++k) h_pair_active_[k] = 1;
    ENG_CK(cudaMemcpyAsync(d_active_, h_active_, sizeof(int) * np, cudaMemcpyHostToDevice, cap_));
    ENG_CK(cudaMemcpyAsync(d_pair_active_, h_pair_active_, sizeof(int) * npairs_, cudaMemcpyHostToDevice, cap_));

    // tolerance levels: shifts, per-shift tables (FP64 arithmetic on the device)
    std::vector<double> lo(np), hi(np);
    for (int p = 0; p < np; ++p) {
        if (tight) square_tight_interval(ns[p], lo[p], hi[p]);
        else {
            lo[p] = square_eps(ns[p]);
            hi[p] = 1.0;
        }
    }
    std::vector<double> tols;
    if (kFP64) tols.push_back(tol);
    else tols.assign(std::begin(kLevelTols), std::end(kLevelTols));
    shifts.assign(np, {});
    for (size_t li = 0; li < tols.size(); ++li) {
        Level L;
        L.tol = tols[li];
        L.J.resize(np);
        // intervals of kx A~ (row side) and -ky A~ (column side): [a, b] = -kx [hi, lo],
        // [c, d] = ky [lo, hi]; on a square (kx = ky) the symmetric route gives p = -q
        const bool sym = kx_ == ky_;
        const int ntab = sym ? 1 : 2;  // one table serves rows and columns on a square
        int64_t nfac = 0, nq = 0;
        for (int p = 0; p < np; ++p) {
            L.J[p] = adi_iterations(-kx_ * hi[p], -kx_ * lo[p], ky_ * lo[p], ky_ * hi[p], L.tol);
            L.Jmax = std::max(L.Jmax, L.J[p]);
            nfac += (int64_t)ntab * L.J[p] * (N_[p] + 4);
            nq += L.J[p];
        }
        ENG_CK(dalloc(&L.fac, (size_t)nfac));
        ENG_CK(dalloc(&L.sh, (size_t)(3 * nq)));
        ENG_CK(dalloc(&L.d_probs, (size_t)np));
        ENG_CK(cudaMemsetAsync(L.fac, 0, sizeof(Fac<T>) * (size_t)nfac, cap_));
        FacJob<T> *d_jobs = nullptr;
        ENG_CK(cudaMalloc((void **)&d_jobs, sizeof(FacJob<T>) * (size_t)(ntab * nq)));
        std::vector<SwProb<T>> probs(np);
        std::vector<FacJob<T>> jobs;
        std::vector<T> shh;
        jobs.reserve(ntab * nq);
        shh.reserve(3 * nq);
        int64_t of = 0, oq = 0;
        std::vector<double> q, pp;
        for (int p = 0; p < np; ++p) {
            const int64_t n = ns[p];
            const int N = N_[p];
            const double a = -kx_ * hi[p], b = -kx_ * lo[p], c = ky_ * lo[p], d = ky_ * hi[p];
            if (sym) {
                zolotarev_shifts_symmetric(lo[p], hi[p], L.J[p], q);
                pp.resize(q.size());
                for (size_t u = 0; u < q.size(); ++u) {
                    q[u] *= kx_;
                    pp[u] = -q[u];
                }
            } else {
                zolotarev_shifts(a, b, c, d, L.J[p], pp, q);
            }
            inject_shift_fault(q);
            std::vector<double> mp(pp.size());
            for (size_t u = 0; u < pp.size(); ++u) mp[u] = -pp[u];
            if (!shifts_valid(q, c, d) || !shifts_valid(mp, -b, -a)) {
                cudaFree(d_jobs);
                levels_.push_back(std::move(L));
                err = "shift list failed validation (a shift is not finite or lies outside the spectral interval)";
                return FPS_ERR_INVALID_ARG;
            }
            if (li == 0) shifts[p] = q;
            SwProb<T> &sp = probs[p];
            sp.n = (int)n;
            sp.S = S;
            sp.P = P_[p];
            sp.N = N;
            sp.ldp = N + 8;
            sp.J = L.J[p];
            sp.off = offT_[p];
            sp.rhs = (int64_t)(N + 4) * (N + 8);
            sp.soff = offS_[p];
            sp.srhs = (int64_t)P_[p] * 2 * (N + 8);
            sp.facR = L.fac + of;
            sp.facC = L.fac + of + (sym ? 0 : (int64_t)L.J[p] * (N + 4));
            sp.sh = L.sh + 3 * oq;
            sp.d = bandsT_ + obT[p];
            sp.e = bandsT_ + obT[p] + (N + 4);
            for (int t = 0; t < ntab; ++t)
                for (int j = 0; j < L.J[p]; ++j) {
                    FacJob<T> jb;
                    jb.q = t == 0 ? -pp[j] / ky_ : q[j] / kx_;  // row solve, then column solve
                    jb.n = (int)n;
                    jb.N = N;
                    jb.S = S;
                    jb.d = bands64_ + ob64[p];
                    jb.e = bands64_ + ob64[p] + n;
                    jb.out = L.fac + of + ((int64_t)t * L.J[p] + j) * (N + 4);
                    jobs.push_back(jb);
                }
            for (int j = 0; j < L.J[p]; ++j) {
                shh.push_back((T)(-pp[j] / kx_));                    // column-stencil shift
                shh.push_back((T)(q[j] / ky_));                      // row-stencil shift
                shh.push_back((T)(-(q[j] - pp[j]) / (kx_ * ky_)));  // correction factor
            }
            of += (int64_t)ntab * L.J[p] * (N + 4);
            oq += L.J[p];
        }
        cudaError_t e1 = cudaMemcpyAsync(L.d_probs, probs.data(), sizeof(SwProb<T>) * np, cudaMemcpyHostToDevice, cap_);
        if (e1 == cudaSuccess)
            e1 = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(FacJob<T>) * jobs.size(), cudaMemcpyHostToDevice, cap_);
        if (e1 == cudaSuccess)
            e1 = cudaMemcpyAsync(L.sh, shh.data(), sizeof(T) * shh.size(), cudaMemcpyHostToDevice, cap_);
        if (e1 == cudaSuccess) e1 = launch_fac_tables<T>(d_jobs, (int)jobs.size(), cap_);
        // the host vectors and the job table must outlive the asynchronous work
        if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(cap_);
        cudaFree(d_jobs);
        levels_.push_back(std::move(L));
        ENG_CK(e1);
    }
    {
        int big = 0;
        for (int p = 0; p < np; ++p)
            if (ns[p] > ns[big]) big = p;
        J_first = levels_[0].J[big];
    }
    for (auto &L : levels_) {
        int st = build_graph(L, err);
        if (st != FPS_OK) return st;
    }
    return FPS_OK;
}

template <typename T>
SwArgs<T> SweepEngine<T>::args(const Level &L, int which) const
{
    SwArgs<T> a;
    a.probs = L.d_probs;
    a.items = d_items_[which];
    a.nitems = nitems_[which];
    a.active = d_active_;
    a.rho0 = rho0_;
    a.cl = cl_;
    a.al = al_;
    a.D = D_;
    a.sumR = sumR_;
    a.sumC = sumC_;
    a.zxR = zxR_;
    a.zxC = zxC_;
    a.zin = zin_;
    a.err = err_;
    a.S = seg_len;
    a.chain_mode = chain_mode;
    return a;
}

template <typename T>
int SweepEngine<T>::build_graph(Level &L, std::string &err)
{
    if (L.graph) {
        cudaGraphExecDestroy(L.graph);
        L.graph = nullptr;
    }
    const SwArgs<T> ar = args(L, 0), ac = args(L, 1), ach = args(L, 2);
    TileArgs ta;
    ta.probs = d_tp_;
    ta.tiles = d_tiles_;
    ta.ntiles = ntiles_;
    ENG_CK(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const bool ins = instrument_ && (int)L.ev.size() == 4 * L.Jmax;
    auto rec = [&](int k) {
        if (ins && e == cudaSuccess) e = cudaEventRecordWithFlags(L.ev[k], cap_, cudaEventRecordExternal);
    };
    for (int j = 0; j < L.Jmax && e == cudaSuccess; ++j) {
        rec(4 * j);
        if (e == cudaSuccess) e = launch_row_pass<T>(ar, j, j == 0 ? 0 : (j == 1 ? 1 : 2), cap_);
        rec(4 * j + 1);
        if (e == cudaSuccess) e = launch_chain<T>(ach, 0, j, cap_);
        rec(4 * j + 2);
        if (e == cudaSuccess) e = launch_col_pass<T>(ac, j, cap_);
        rec(4 * j + 3);
        if (e == cudaSuccess) e = launch_chain<T>(ach, 1, j, cap_);
    }
    if (e == cudaSuccess && sizeof(T) == 4) e = launch_finalize<T>(ta, ar, d_pair_active_, cap_);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap_, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        err = std::string("sweep graph capture: ") + cudaGetErrorString(e);
        return FPS_ERR_CUDA;
    }
    ENG_CK(e2);
    e = cudaGraphInstantiate(&L.graph, g, 0);
    cudaGraphDestroy(g);
    ENG_CK(e);
    return FPS_OK;
}

template <typename T>
int SweepEngine<T>::solve(const double *F, double *X, cudaStream_t st, std::string &err)
{
    launches_last = 0;
    levels_used_.clear();
    return sizeof(T) == 8 ? solve_plain(F, X, st, err) : solve_refine(F, X, st, err);
}

template <typename T>
int SweepEngine<T>::solve_plain(const double *F, double *X, cudaStream_t st, std::string &err)
{
    if constexpr (sizeof(T) == 8) {
        TileArgs ta;
        ta.probs = d_tp_;
        ta.tiles = d_tiles_;
        ta.ntiles = ntiles_;
        ENG_CK(launch_scale_in<double>(ta, F, nullptr, rho0_, nullptr, st));
        ENG_CK(cudaGraphLaunch(levels_[0].graph, st));
        ENG_CK(launch_finalize_out(ta, args(levels_[0], 0), X, st));
        ENG_CK(cudaMemcpyAsync(h_err_, err_, sizeof(int), cudaMemcpyDeviceToHost, st));
        levels_used_.push_back(0);
        launches_last = 2 + 4LL * levels_[0].Jmax;
        rounds_last = 1;
        return FPS_OK;
    } else {
        (void)F;
        (void)X;
        (void)st;
        err = "plain solve needs FP64 sweeps";
        return FPS_ERR_UNSUPPORTED;
    }
}

template <typename T>
int SweepEngine<T>::solve_refine(const double *F, double *X, cudaStream_t st, std::string &err)
{
    if constexpr (sizeof(T) == 4) {
        const int np = (int)ns_.size();
        TileArgs ta;
        ta.probs = d_tp_;
        ta.tiles = d_tiles_;
        ta.ntiles = ntiles_;

        ENG_CK(cudaMemsetAsync(d_smax_, 0, sizeof(unsigned long long) * npairs_, st));
        ENG_CK(launch_absmax(ta, F, d_smax_, st));
        ENG_CK(cudaMemcpyAsync(h_smax_, d_smax_, sizeof(unsigned long long) * npairs_, cudaMemcpyDeviceToHost, st));
        ENG_CK(cudaStreamSynchronize(st));
        launches_last += 1;
        std::vector<double> sF(npairs_);
        for (int k = 0; k < npairs_; ++k) {
            sF[k] = bits_to_double(h_smax_[k]);
            if (!std::isfinite(sF[k])) {
                err = "F holds NaN or Inf";
                return FPS_ERR_NONFINITE;
            }
            h_pair_active_[k] = sF[k] > 0.0 ? 1 : 0;  // an all-zero right-hand side is already solved (X = 0)
        }
        for (int p = 0; p < np; ++p) {
            h_active_[p] = 0;
            for (int r = 0; r < nrhs_; ++r) h_active_[p] |= h_pair_active_[p * nrhs_ + r];
        }
        ENG_CK(cudaMemcpyAsync(d_active_, h_active_, sizeof(int) * np, cudaMemcpyHostToDevice, st));
        ENG_CK(cudaMemcpyAsync(d_pair_active_, h_pair_active_, sizeof(int) * npairs_, cudaMemcpyHostToDevice, st));
        ENG_CK(launch_scale_in<float>(ta, F, Ft_, rho0_, d_smax_, st));
        launches_last += 1;

        std::vector<double> rel(npairs_, 0.0);
        for (int k = 0; k < npairs_; ++k) rel[k] = h_pair_active_[k] ? 1.0 : 0.0;
        double *Ycur = Y0_, *Ynext = Y1_;
        bool any_active = false;
        for (int k = 0; k < npairs_; ++k) any_active = any_active || h_pair_active_[k];
        int round = 0;
        bool converged = !any_active;
        for (; round < max_rounds && !converged; ++round) {
            TraceRange tr("fps refinement round");
            double worst = 0.0;
            for (int k = 0; k < npairs_; ++k)
                if (h_pair_active_[k]) worst = std::max(worst, rel[k]);
            const double want = 0.1 * tol_ / worst;
            size_t li = 0;
            for (size_t l = 0; l < levels_.size(); ++l)
                if (levels_[l].tol <= want) li = l;
            if (round == 0) {
                // two balanced rounds: the first stops near sqrt(0.1 tol), which leaves the
                // second a gain of the same size (1e-6 then 1e-5 for tol = 1e-10)
                const double first = std::sqrt(0.1 * tol_);
                li = 0;
                for (size_t l = 0; l < levels_.size(); ++l)
                    if (levels_[l].tol <= first) li = l;
            }
            ENG_CK(cudaGraphLaunch(levels_[li].graph, st));
            levels_used_.push_back((int)li);
            launches_last += 4LL * levels_[li].Jmax + 1;
            ENG_CK(cudaMemsetAsync(d_rmax_, 0, sizeof(unsigned long long) * npairs_, st));
            ENG_CK(launch_residual(ta, Ycur, Ynext, D_, Ft_, rho0_, d_smax_, d_rmax_, d_pair_active_, round == 0, st));
            launches_last += 1;
            ENG_CK(cudaMemcpyAsync(h_rmax_, d_rmax_, sizeof(unsigned long long) * npairs_, cudaMemcpyDeviceToHost, st));
            ENG_CK(cudaMemcpyAsync(h_err_, err_, sizeof(int), cudaMemcpyDeviceToHost, st));
            ENG_CK(cudaStreamSynchronize(st));
            if (*h_err_) {
                err = "a bounded device wait gave up (tile copy not completed)";
                return FPS_ERR_TIMEOUT;
            }
            std::swap(Ycur, Ynext);
            converged = true;
            for (int k = 0; k < npairs_; ++k) {
                if (!h_pair_active_[k]) continue;
                const double r = bits_to_double(h_rmax_[k]) / sF[k];
                if (!std::isfinite(r)) {
                    err = "non-finite residual";
                    return FPS_ERR_NONFINITE;
                }
                rel[k] = r;
                if (r <= tol_) h_pair_active_[k] = 0;
                else converged = false;
            }
            for (int p = 0; p < np; ++p) {
                h_active_[p] = 0;
                for (int r = 0; r < nrhs_; ++r) h_active_[p] |= h_pair_active_[p * nrhs_ + r];
            }
            ENG_CK(cudaMemcpyAsync(d_active_, h_active_, sizeof(int) * np, cudaMemcpyHostToDevice, st));
            ENG_CK(cudaMemcpyAsync(d_pair_active_, h_pair_active_, sizeof(int) * npairs_, cudaMemcpyHostToDevice, st));
        }
        rounds_last = round;
        resid_last = 0.0;
        for (int k = 0; k < npairs_; ++k) resid_last = std::max(resid_last, rel[k]);
        if (round == 0) {
            ENG_CK(cudaMemsetAsync(X, 0, sizeof(double) * tot64_, st));  // every right-hand side was zero
            return FPS_OK;
        }
        ENG_CK(launch_scale_out(ta, Ycur, X, st));
        launches_last += 1;
        if (!converged) {
            err = "refinement did not reach tol";
            return FPS_ERR_NOT_CONVERGED;
        }
        return FPS_OK;
    } else {
        (void)F;
        (void)X;
        (void)st;
        err = "refinement needs FP32 sweeps";
        return FPS_ERR_UNSUPPORTED;
    }
}

template <typename T>
int SweepEngine<T>::set_instrument(bool on, std::string &err)
{
    instrument_ = on;
    for (auto &L : levels_) {
        for (cudaEvent_t e : L.ev) cudaEventDestroy(e);
        L.ev.clear();
        if (on) {
            L.ev.resize(4 * (size_t)L.Jmax);
            for (auto &e : L.ev) ENG_CK(cudaEventCreate(&e));
        }
        int st = build_graph(L, err);
        if (st != FPS_OK) return st;
    }
    return FPS_OK;
}

template <typename T>
int SweepEngine<T>::kernel_times(int *count, double *total_ms, double *alg_bytes, double *row_ms, double *col_ms,
                                 std::string &err)
{
    if (h_err_ && *h_err_) {
        err = "a bounded device wait gave up (tile copy not completed)";
        return FPS_ERR_TIMEOUT;
    }
    int c = 0;
    double rms = 0.0, cms = 0.0, by = 0.0;
    std::vector<int> seen;
    for (int li : levels_used_) {
        if (std::find(seen.begin(), seen.end(), li) != seen.end()) continue;
        seen.push_back(li);
        const Level &L = levels_[li];
        if ((int)L.ev.size() != 4 * L.Jmax) continue;
        for (int j = 0; j < L.Jmax; ++j) {
            float t0 = 0.f, t1 = 0.f;
            ENG_CK(cudaEventElapsedTime(&t0, L.ev[4 * j], L.ev[4 * j + 1]));
            ENG_CK(cudaEventElapsedTime(&t1, L.ev[4 * j + 2], L.ev[4 * j + 3]));
            rms += t0;
            cms += t1;
            c += 2;
            double ej = 0.0;
            for (size_t p = 0; p < ns_.size(); ++p)
                if (j < L.J[p]) ej += (double)nrhs_ * (double)ns_[p] * (double)ns_[p];
            // row pass: rho (or c) read, al written, D read and written (j >= 2) or written (j = 1);
            // column pass: al read, cl written
            const double row_words = j == 0 ? 2.0 : (j == 1 ? 3.0 : 4.0);
            by += (row_words + 2.0) * sizeof(T) * ej;
        }
    }
    *count = c;
    *total_ms = rms + cms;
    *alg_bytes = by;
    if (row_ms) *row_ms = rms;
    if (col_ms) *col_ms = cms;
    return FPS_OK;
}

template class SweepEngine<float>;
template class SweepEngine<double>;

}  // namespace fps
