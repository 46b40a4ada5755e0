// ADI pass kernels of the square solve (see sweep.cuh for the scheme and layout).
//
// Tiles travel through shared memory by bulk asynchronous copies (cp.async.bulk,
// one copy per tile row, completion on an mbarrier; results leave by bulk stores),
// so no thread spends registers or issue slots on address streams.  Inside a tile
// every thread owns one line (a row in the row pass, a column in the column pass)
// and keeps the whole segment of that line in registers: two interleaved
// recurrences (even and odd positions, App. B) per thread, no shared-memory
// traffic during the sweeps.
#include <cuda_runtime.h>

#include "bulk.cuh"
#include "device_info.h"
#include "sweep.cuh"

namespace fps {

namespace {

constexpr int kR = 64;    // rows per row-pass tile
constexpr int kC = 64;    // columns per column-pass tile
constexpr int kRT = 128;  // row-pass threads: one per (row, parity of the column index)
constexpr int kCT = 128;  // column-pass threads: one per (column, parity of the row index)
constexpr int kChainLines = 64;

// 16-byte chunks of T
template <typename T>
struct Ch {
    static constexpr int V = 16 / sizeof(T);
};

template <typename T>
__device__ __forceinline__ void ld16(const T *p, T (&v)[16 / sizeof(T)]);
template <>
__device__ __forceinline__ void ld16<float>(const float *p, float (&v)[4])
{
    const float4 f = *reinterpret_cast<const float4 *>(p);
    v[0] = f.x;
    v[1] = f.y;
    v[2] = f.z;
    v[3] = f.w;
}
template <>
__device__ __forceinline__ void ld16<double>(const double *p, double (&v)[2])
{
    const double2 f = *reinterpret_cast<const double2 *>(p);
    v[0] = f.x;
    v[1] = f.y;
}
template <typename T>
__device__ __forceinline__ void st16(T *p, const T (&v)[16 / sizeof(T)]);
template <>
__device__ __forceinline__ void st16<float>(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st16<double>(double *p, const double (&v)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
// four consecutive words (16-byte aligned) as one or two vector loads
__device__ __forceinline__ void ld4(const float *p, float &a, float &b, float &c, float &d)
{
    const float4 f = *reinterpret_cast<const float4 *>(p);
    a = f.x;
    b = f.y;
    c = f.z;
    d = f.w;
}
__device__ __forceinline__ void ld4(const double *p, double &a, double &b, double &c, double &d)
{
    const double2 f = *reinterpret_cast<const double2 *>(p);
    const double2 h = *reinterpret_cast<const double2 *>(p + 2);
    a = f.x;
    b = f.y;
    c = h.x;
    d = h.y;
}

template <typename T>
__device__ __forceinline__ typename Vec2<T>::type mk2(T x, T y);
template <>
__device__ __forceinline__ float2 mk2<float>(float x, float y)
{
    return make_float2(x, y);
}
template <>
__device__ __forceinline__ double2 mk2<double>(double x, double y)
{
    return make_double2(x, y);
}

// Shared-memory row stride of the row-pass tile: S + 8 loaded columns plus padding
// that makes the stride an odd number of 16-byte chunks (conflict-free 16-byte
// accesses by threads that own consecutive rows).
template <typename T, int S>
struct RowGeom {
    static constexpr int V = Ch<T>::V;
    static constexpr int SW = S + 8 + V;
    static_assert((SW * sizeof(T) / 16) % 2 == 1, "row stride must be an odd number of 16-byte chunks");
    static constexpr size_t off_ct = 16;
    static constexpr size_t off_zx = off_ct + sizeof(T) * (kR + 4) * SW;
    static constexpr size_t off_frow = off_zx + sizeof(typename Vec2<T>::type) * 6 * (S + 8);
    static constexpr size_t off_fcol = off_frow + sizeof(Fac<T>) * (kR + 4);
    static constexpr size_t off_cf = off_fcol + sizeof(Fac<T>) * S;  // {cA, cB, cC, g} per column
    static constexpr size_t bytes = off_cf + sizeof(T) * 4 * S;
    static_assert(off_zx % 16 == 0 && off_frow % 16 == 0 && off_fcol % 16 == 0 && off_cf % 16 == 0, "alignment");
};

template <typename T, int S>
struct ColGeom {
    static constexpr int ZS = S + 2;  // padded stride of the two parity rows of zx
    static constexpr size_t off_tile = 16;
    static constexpr size_t off_fac = off_tile + sizeof(T) * S * kC;
    static constexpr size_t off_zx = off_fac + sizeof(Fac<T>) * S;
    static constexpr size_t bytes = off_zx + sizeof(typename Vec2<T>::type) * 2 * ZS;
    static_assert(off_fac % 16 == 0 && off_zx % 16 == 0, "alignment");
};

// ---------------------------------------------------------------------------
// Shift tables: one thread per (job, parity), FP64 arithmetic.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fac_tables_kernel(const FacJob<T> *__restrict__ jobs, int njobs)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 2 * njobs) return;
    const FacJob<T> &jb = jobs[tid >> 1];
    const int p = tid & 1;
    const int n = jb.n, N = jb.N, S = jb.S;
    Fac<T> *out = jb.out + 2;  // position i at out[i]
    // forward: pivots of the parity-p tridiagonal of A~ - qI, and phi within segments
    double piv_prev = 1.0, phi = 1.0;
    for (int i = p; i < N; i += 2) {
        double ip = 0.0, g = 0.0, uf = 0.0;
        if (i < n) {
            const double em2 = (i >= 2) ? jb.e[i - 2] : 0.0;
            double piv = jb.d[i] - jb.q;
            if (i >= 2) piv -= em2 * em2 / piv_prev;
            ip = 1.0 / piv;
            g = em2 * ip;
            uf = jb.e[i] * ip;
            piv_prev = piv;
        }
        if ((i - p) % S == 0) phi = 1.0;  // first parity-p position of a segment
        phi *= -g;
        Fac<T> f;
        f.ip = (T)ip;
        f.g = (T)g;
        f.uf = (T)uf;
        f.phi = (T)phi;
        f.Bv = 0;
        f.Psi = 0;
        out[i] = f;
    }
    // backward within each segment: Bv_i = phi_i - uf_i Bv_{i+2}, Psi_i = -uf_i Psi_{i+2}
    double Bv = 0.0, Psi = 1.0;
    for (int i = N - 2 + p; i >= p; i -= 2) {
        if (i + 2 >= N || ((i + 2 - p) % S) == 0) {  // last parity-p position of its segment
            Bv = 0.0;
            Psi = 1.0;
        }
        const double uf = (double)out[i].uf;
        Bv = (double)out[i].phi - uf * Bv;
        Psi = -uf * Psi;
        out[i].Bv = (T)Bv;
        out[i].Psi = (T)Psi;
    }
}

// Bounded wait on the tile barrier; on a timeout flag the error word and give the
// copies in flight one more bounded wait before the CTA leaves.
__device__ __forceinline__ bool tile_ready(uint64_t *bar, int *err)
{
    if (bulk::mbar_wait_bounded(bar, 0)) return true;
    if (threadIdx.x == 0) atomicOr(err, 1);
    bulk::mbar_wait_bounded(bar, 0);
    return false;
}

// ---------------------------------------------------------------------------
// Row pass.  Item {problem, rhs, row block (64 rows), column segment}.
// MODE 0: j = 0, input rho_0.  MODE 1: j = 1, D = -2 q_0 c_0.  MODE 2: D -= 2 q_{j-1} c_{j-1}.
// W: columns of this tile's segment (S, or 64 for a short last segment).
// ---------------------------------------------------------------------------
template <typename T, int S, int MODE, int W>
__device__ __forceinline__ void row_pass_tile(const SwArgs<T> &a, int j, const int4 it, const SwProb<T> &pr,
                                              unsigned char *smem)
{
    using G = RowGeom<T, S>;
    using T2 = typename Vec2<T>::type;
    constexpr int V = G::V, SW = G::SW;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    T *ct = reinterpret_cast<T *>(smem + G::off_ct);
    T2 *zx = reinterpret_cast<T2 *>(smem + G::off_zx);
    Fac<T> *frow = reinterpret_cast<Fac<T> *>(smem + G::off_frow);
    Fac<T> *fcol = reinterpret_cast<Fac<T> *>(smem + G::off_fcol);
    T *cf = reinterpret_cast<T *>(smem + G::off_cf);

    const int tid = threadIdx.x;
    const int N = pr.N, ldp = pr.ldp;
    const int i0 = it.z * kR, cs = it.w, k0 = cs * S;
    const int64_t base = pr.off + (int64_t)it.y * pr.rhs;
    const T *src = (MODE == 0 ? a.rho0 : a.cl) + base;
    T *Dp = a.D + base;
    T *alp = a.al + base;
    const int64_t sbase = pr.soff + (int64_t)it.y * pr.srhs;
    const Fac<T> *facj = pr.facR + (int64_t)j * (N + 4);                      // this row solve
    const Fac<T> *facp = pr.facC + (int64_t)(MODE > 0 ? j - 1 : 0) * (N + 4);  // previous column solve
    const T sL = MODE > 0 ? pr.sh[3 * (j - 1)] : T(0);      // column-stencil shift of iteration j-1
    const T sR = MODE > 0 ? pr.sh[3 * (j - 1) + 1] : T(0);  // row-stencil shift
    const T fD = MODE > 0 ? pr.sh[3 * (j - 1) + 2] : T(0);  // correction factor

    // column segments of the halo rows (row systems of the previous column pass)
    const int sc = i0 / S, segstart = sc * S, segend = min(segstart + S, N);
    const int s_above = (MODE > 0 && i0 == segstart && i0 > 0) ? sc - 1 : -1;
    const int s_below = (MODE > 0 && i0 + kR == segend && segend < N) ? sc + 1 : -1;
    constexpr int rows_ld = MODE == 0 ? kR : kR + 4;
    constexpr int cw = MODE == 0 ? W : W + 8;  // loaded columns
    const int row0 = MODE == 0 ? i0 : i0 - 2;  // first global row loaded
    constexpr int smr0 = MODE == 0 ? 2 : 0;    // its shared-memory row
    const int kc0 = MODE == 0 ? k0 : k0 - 4;   // first loaded column
    constexpr int scc0 = MODE == 0 ? 4 : 0;    // its shared-memory column

    if (tid == 0) {
        bulk::mbar_init(bar, 1);
        bulk::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        unsigned bytes = (unsigned)(rows_ld * cw * sizeof(T) + W * sizeof(Fac<T>));
        if (MODE > 0)
            bytes += (unsigned)((kR + 4) * sizeof(Fac<T>) +
                                2 * cw * sizeof(T2) * (1 + (s_above >= 0) + (s_below >= 0)));
        bulk::mbar_arrive_expect_tx(bar, bytes);
    }
    __syncthreads();
    for (int r = tid; r < rows_ld; r += kRT)
        bulk::g2s(ct + (smr0 + r) * SW + scc0, src + (int64_t)(row0 + r + 2) * ldp + (kc0 + 4),
                  (unsigned)(cw * sizeof(T)), bar);
    if (tid == kRT - 1) bulk::g2s(fcol, facj + k0 + 2, (unsigned)(W * sizeof(Fac<T>)), bar);
    if (MODE > 0) {
        if (tid == kRT - 2) bulk::g2s(frow, facp + i0, (unsigned)((kR + 4) * sizeof(Fac<T>)), bar);
        if (tid >= kRT - 8 && tid < kRT - 2) {
            const int k = tid - (kRT - 8), slot = k >> 1, par = k & 1;
            const int sg = slot == 0 ? s_above : (slot == 1 ? sc : s_below);
            if (sg >= 0)
                bulk::g2s(zx + (slot * 2 + par) * (S + 8), a.zxC + sbase + ((int64_t)sg * 2 + par) * (N + 8) + k0,
                          (unsigned)(cw * sizeof(T2)), bar);
        }
    }
    // D of the tile's core into registers while the tile is in flight: thread t owns
    // chunk t % CPR of rows t / CPR + m * (kRT / CPR) (coalesced 16-byte loads)
    constexpr int CPR = W / V;
    constexpr int DSTEP = kRT / CPR;
    constexpr int NDC = kR / DSTEP;  // chunks per thread
    const int dr0 = tid / CPR, dc = tid % CPR;
    T dreg[NDC][V];
    if (MODE == 2) {
#pragma unroll
        for (int m = 0; m < NDC; ++m)
            ld16(Dp + (int64_t)(i0 + dr0 + m * DSTEP + 2) * ldp + (k0 + 4 + dc * V), dreg[m]);
    }
    if (!tile_ready(bar, a.err)) return;

    // per-column records {ip e_{k-2}, ip (d_k + q), ip e_k, g} of the ip-scaled row stencil
    for (int c = tid; c < W; c += kRT) {
        const int k = k0 + c;
        const T ipk = fcol[c].ip;
        if (MODE > 0) {
            cf[4 * c + 0] = ipk * pr.e[k];
            cf[4 * c + 1] = ipk * (pr.d[k + 2] + sR);
            cf[4 * c + 2] = ipk * pr.e[k + 2];
        } else {
            cf[4 * c + 0] = T(0);
            cf[4 * c + 1] = ipk;
            cf[4 * c + 2] = T(0);
        }
        cf[4 * c + 3] = fcol[c].g;
    }
    if (MODE > 0) {
        // rebuild c_{j-1} = cl + Bv zin + Psi xout on the whole loaded tile
        constexpr int cpr = cw / V;
        constexpr int total = (kR + 4) * cpr;
        for (int idx = tid; idx < total; idx += kRT) {
            const int r = idx / cpr, cc = (idx - r * cpr) * V;
            const int i = i0 - 2 + r;
            if (i >= 0 && i < N) {
                T *cp = ct + r * SW + cc;
                T v[V];
                ld16(cp, v);
                const int slot = i < segstart ? 0 : (i >= segend ? 2 : 1);
                const T2 *z = zx + (slot * 2 + (i & 1)) * (S + 8) + cc;
                const T bv = frow[r].Bv, ps = frow[r].Psi;
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const T2 zz = z[e];
                    v[e] = fma(bv, zz.x, fma(ps, zz.y, v[e]));
                }
                st16(cp, v);
            }
        }
        __syncthreads();
        // D -= 2 q_{j-1} c_{j-1} on the core (D = -2 q_0 c_0 at j = 1)

#pragma unroll
        for (int m = 0; m < NDC; ++m) {
            const int rr = dr0 + m * DSTEP;
            T v[V], dv[V];
            ld16(ct + (rr + 2) * SW + 4 + dc * V, v);
#pragma unroll
            for (int e = 0; e < V; ++e) dv[e] = MODE == 1 ? fD * v[e] : fma(fD, v[e], dreg[m][e]);
            st16(Dp + (int64_t)(i0 + rr + 2) * ldp + (k0 + 4 + dc * V), dv);
        }
    }
    __syncthreads();

    // one thread per (row, parity of the column index): a warp holds 16 rows x 2 parities
    const int lane = tid & 31;
    const int rr = (tid >> 5) * 16 + (lane & 15), p = lane >> 4;
    const int r = rr + 2, i = i0 + rr;
    T wr[W / 2];
    T we;
    {
        T w = 0;
        if (MODE == 0) {
#pragma unroll
            for (int t = 0; t < W / 2; ++t) {
                const int c = 2 * t + p;
                const T rho = cf[4 * c + 1] * ct[r * SW + 4 + c];
                w = fma(-cf[4 * c + 3], w, rho);
                wr[t] = w;
            }
        } else {
            // rho = ip (R + q)(L + q) c: column stencil u = (L + q) c, then the row stencil
            const T eu = pr.e[i], dq = pr.d[i + 2] + sL, ed = pr.e[i + 2];
            const T *r0 = ct + (r - 2) * SW + 4, *r1 = ct + r * SW + 4, *r2 = ct + (r + 2) * SW + 4;
            auto u = [&](int x) { return fma(eu, r0[x], fma(dq, r1[x], ed * r2[x])); };
            T um = u(p - 2), u0 = u(p);
#pragma unroll
            for (int t = 0; t < W / 2; ++t) {
                const int c = 2 * t + p;
                const T up = u(c + 2);
                T cA, cB, cC, g;
                ld4(cf + 4 * c, cA, cB, cC, g);
                const T rho = fma(cA, um, fma(cB, u0, cC * up));
                w = fma(-g, w, rho);
                wr[t] = w;
                um = u0;
                u0 = up;
            }
        }
        we = w;
    }
    {
        T x = 0;  // local back substitution: zero beyond the segment
#pragma unroll
        for (int t = W / 2 - 1; t >= 0; --t) {
            x = fma(-fcol[2 * t + p].uf, x, wr[t]);
            wr[t] = x;
        }
    }
    const bool live = i < pr.n;
    __syncthreads();  // every thread is done reading the tile
#pragma unroll
    for (int t = 0; t < W / 2; ++t) ct[r * SW + 4 + 2 * t + p] = live ? wr[t] : T(0);
    a.sumR[sbase + ((int64_t)cs * 2 + p) * (N + 8) + i + 4] = mk2<T>(live ? we : T(0), live ? wr[0] : T(0));
    bulk::fence_proxy_async_shared();
    __syncthreads();
    if (tid < kR)
        bulk::s2g(alp + (int64_t)(i0 + tid + 2) * ldp + (k0 + 4), ct + (tid + 2) * SW + 4, (unsigned)(W * sizeof(T)));
    bulk::commit();
    bulk::wait_read_all();
}

template <typename T, int S, int MODE>
__global__ void __launch_bounds__(kRT, 3) row_pass_kernel(SwArgs<T> a, int j)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 it = a.items[blockIdx.x];
    const SwProb<T> &pr = a.probs[it.x];
    if (!a.active[it.x] || j >= pr.J) return;
    // after a timeout anywhere, leave at once (one read, agreed on by the whole CTA)
    if (__syncthreads_or(threadIdx.x == 0 ? *(volatile int *)a.err : 0)) return;
    if (S == kR || pr.N - it.w * S >= S) row_pass_tile<T, S, MODE, S>(a, j, it, pr, smem);
    else row_pass_tile<T, S, MODE, kR>(a, j, it, pr, smem);
}

// ---------------------------------------------------------------------------
// Column pass.  Item {problem, rhs, column block (64 columns), row segment}.
// H: rows of this tile's segment (S, or 64 for a short last segment).
// ---------------------------------------------------------------------------
template <typename T, int S, int H>
__device__ __forceinline__ void col_pass_tile(const SwArgs<T> &a, int j, const int4 it, const SwProb<T> &pr,
                                              unsigned char *smem)
{
    using G = ColGeom<T, S>;
    using T2 = typename Vec2<T>::type;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    T *tile = reinterpret_cast<T *>(smem + G::off_tile);
    Fac<T> *fac = reinterpret_cast<Fac<T> *>(smem + G::off_fac);
    T2 *zx = reinterpret_cast<T2 *>(smem + G::off_zx);

    const int tid = threadIdx.x;
    const int N = pr.N, ldp = pr.ldp;
    const int k0 = it.z * kC, rs = it.w, i0 = rs * S;
    const int cs = k0 / S;  // row-system segment holding these columns
    const int64_t base = pr.off + (int64_t)it.y * pr.rhs;
    const int64_t sbase = pr.soff + (int64_t)it.y * pr.srhs;
    const Fac<T> *facj = pr.facC + (int64_t)j * (N + 4);  // this column solve
    const Fac<T> *facr = pr.facR + (int64_t)j * (N + 4);  // the row solve whose result is rebuilt

    if (tid == 0) {
        bulk::mbar_init(bar, 1);
        bulk::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        bulk::mbar_arrive_expect_tx(bar, (unsigned)(H * kC * sizeof(T) + H * sizeof(Fac<T>) + 2 * H * sizeof(T2)));
    __syncthreads();
    for (int r = tid; r < H; r += kCT)
        bulk::g2s(tile + r * kC, a.al + base + (int64_t)(i0 + r + 2) * ldp + (k0 + 4), (unsigned)(kC * sizeof(T)), bar);
    if (tid == kCT - 1) bulk::g2s(fac, facj + i0 + 2, (unsigned)(H * sizeof(Fac<T>)), bar);
    if (tid == kCT - 2 || tid == kCT - 3) {
        const int par = kCT - 2 - tid;
        bulk::g2s(zx + par * G::ZS, a.zxR + sbase + ((int64_t)cs * 2 + par) * (N + 8) + i0 + 4,
                  (unsigned)(H * sizeof(T2)), bar);
    }
    // one thread per (column, parity of the row index)
    const int kk = tid % kC, p = tid / kC;
    const int k = k0 + kk;
    const T bv = facr[k + 2].Bv, ps = facr[k + 2].Psi;
    const T2 *zp = zx + (k & 1) * G::ZS;
    if (!tile_ready(bar, a.err)) return;

    // forward sweep and back substitution in place in the tile (own column, own parity)
    const bool live = k < pr.n;
    T we, x = 0;
    {
        T w = 0;
#pragma unroll 8
        for (int t = 0; t < H / 2; ++t) {
            const int r = 2 * t + p;
            const T2 z = zp[r];
            const T av = fma(bv, z.x, fma(ps, z.y, tile[r * kC + kk]));
            T ip, g, uf, phi;
            ld4(&fac[r].ip, ip, g, uf, phi);
            w = fma(-g, w, ip * av);
            tile[r * kC + kk] = w;
        }
        we = w;
    }
#pragma unroll 8
    for (int t = H / 2 - 1; t >= 0; --t) {
        const int r = 2 * t + p;
        x = fma(-fac[r].uf, x, tile[r * kC + kk]);
        tile[r * kC + kk] = live ? x : T(0);
    }
    a.sumC[sbase + ((int64_t)rs * 2 + p) * (N + 8) + k + 4] = mk2<T>(live ? we : T(0), live ? x : T(0));
    bulk::fence_proxy_async_shared();
    __syncthreads();
    for (int r = tid; r < H; r += kCT)
        bulk::s2g(a.cl + base + (int64_t)(i0 + r + 2) * ldp + (k0 + 4), tile + r * kC, (unsigned)(kC * sizeof(T)));
    bulk::commit();
    bulk::wait_read_all();
}

template <typename T, int S>
__global__ void __launch_bounds__(kCT) col_pass_kernel(SwArgs<T> a, int j)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 it = a.items[blockIdx.x];
    const SwProb<T> &pr = a.probs[it.x];
    if (!a.active[it.x] || j >= pr.J) return;
    if (__syncthreads_or(threadIdx.x == 0 ? *(volatile int *)a.err : 0)) return;
    if (S == kC || pr.N - it.w * S >= S) col_pass_tile<T, S, S>(a, j, it, pr, smem);
    else col_pass_tile<T, S, kC>(a, j, it, pr, smem);
}

// ---------------------------------------------------------------------------
// Chains: true forward value entering and true solution leaving every segment.
// Item {problem, rhs, block of 64 lines}; thread = (line, parity).
//   W_s = wl_end(s) + phi_end(s) W_{s-1},           zin(s)  = W_{s-1}
//   X_s = xl_start(s) + Bv_start(s) zin(s) + Psi_start(s) X_{s+1},   xout(s) = X_{s+1}
// ---------------------------------------------------------------------------
// BIG: long load batches (fewer dependent round trips to L2, more registers) for
// grids of a few CTAs per SM, where latency is all; short ones keep occupancy when
// the grid fills the GPU (batches of many problems).
template <typename T, bool BIG>
__global__ void __launch_bounds__(2 * kChainLines) chain_kernel(SwArgs<T> a, int dir, int j)
{
    using T2 = typename Vec2<T>::type;
    // segments whose loads are issued together (forward: 2 values, backward: 4 values
    // per segment); each batch is one dependent round trip to L2
    constexpr int B = BIG ? (sizeof(T) == 4 ? 40 : 20) : 16, B2 = BIG ? (sizeof(T) == 4 ? 24 : 12) : 16;
    const int4 it = a.items[blockIdx.x];
    const SwProb<T> &pr = a.probs[it.x];
    if (!a.active[it.x] || j >= pr.J) return;
    const int p = threadIdx.x / kChainLines;
    const int l = it.z * kChainLines + (threadIdx.x % kChainLines);
    const int N = pr.N, S = pr.S, P = pr.P;
    if (l >= N) return;
    const int64_t sbase = pr.soff + (int64_t)it.y * pr.srhs;
    const T2 *__restrict__ sum = (dir == 0 ? a.sumR : a.sumC) + sbase + p * (N + 8) + l + 4;
    T2 *__restrict__ zx = (dir == 0 ? a.zxR : a.zxC) + sbase + p * (N + 8) + l + 4;
    T *__restrict__ zs = a.zin + sbase + p * (N + 8) + l + 4;
    const int64_t step = 2 * (int64_t)(N + 8);  // next segment, same parity and line
    const Fac<T> *__restrict__ facj = (dir == 0 ? pr.facR : pr.facC) + (int64_t)j * (N + 4) + 2;
    T W = 0;
    for (int s0 = 0; s0 < P; s0 += B) {
        T sx[B], ph[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int s = s0 + b;
            if (s < P) {
                sx[b] = sum[s * step].x;
                ph[b] = facj[min(s * S + S, N) - 2 + p].phi;
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int s = s0 + b;
            if (s < P) {
                zs[s * step] = W;
                W = fma(ph[b], W, sx[b]);
            }
        }
    }
    T X = 0;
    for (int s1 = P - 1; s1 >= 0; s1 -= B2) {
        T sy[B2], zi[B2], bv[B2], ps[B2];
#pragma unroll
        for (int b = 0; b < B2; ++b) {
            const int s = s1 - b;
            if (s >= 0) {
                sy[b] = sum[s * step].y;
                zi[b] = zs[s * step];
                bv[b] = facj[s * S + p].Bv;
                ps[b] = facj[s * S + p].Psi;
            }
        }
#pragma unroll
        for (int b = 0; b < B2; ++b) {
            const int s = s1 - b;
            if (s >= 0) {
                zx[s * step] = mk2<T>(zi[b], X);
                X = fma(bv[b], zi[b], fma(ps[b], X, sy[b]));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Elementwise kernels over 32 x 32 tiles of the n x n region.
// ---------------------------------------------------------------------------
struct TileView {
    int n, ldp, prob, rhs, pair;
    int64_t off64, offT;
    const double *d, *e, *s;
    double kx, ky;
    int bx, by;
};
__device__ __forceinline__ TileView tile_view(const TileArgs &t, int64_t idx = -1)
{
    const int4 q = t.tiles[idx < 0 ? (int64_t)blockIdx.x : idx];
    const TileProb &p = t.probs[q.x >> 8];
    TileView v;
    v.prob = q.x >> 8;
    v.rhs = q.x & 255;
    v.n = p.n;
    v.ldp = p.ldp;
    v.off64 = p.off64 + (int64_t)v.rhs * p.n * p.n;
    v.offT = p.off + (int64_t)v.rhs * p.rhs;
    v.d = p.d;
    v.e = p.e;
    v.s = p.s;
    v.pair = p.pair0 + v.rhs;
    v.kx = p.kx;
    v.ky = p.ky;
    v.bx = q.y * 32;
    v.by = q.z * 32;
    return v;
}

// The contiguous run of tiles of this CTA, for the reduction kernels (tiles are
// ordered pair by pair, so a run meets each (problem, rhs) pair once: one atomic per
// pair and CTA instead of one per tile).
__device__ __forceinline__ void tile_run(int64_t ntiles, int64_t &t0, int64_t &t1)
{
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    t0 = (int64_t)blockIdx.x * per;
    t1 = t0 + per < ntiles ? t0 + per : ntiles;
}

// c_{J-1} at (i, k) rebuilt from the column pass's local result and its chain.
template <typename T>
__device__ __forceinline__ T rebuilt_c(const SwArgs<T> &a, const SwProb<T> &pr, int64_t offT, int64_t sbase,
                                       const Fac<T> &fi, int i, int k)
{
    const T cl = a.cl[offT + (int64_t)(i + 2) * pr.ldp + k + 4];
    const typename Vec2<T>::type z = a.zxC[sbase + ((int64_t)(i / pr.S) * 2 + (i & 1)) * (pr.N + 8) + k + 4];
    return fma(fi.Bv, z.x, fma(fi.Psi, z.y, cl));
}

template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(TileArgs t, SwArgs<T> a, const int *__restrict__ pair_active)
{
    const TileView v = tile_view(t);
    if (!pair_active[v.pair]) return;
    const SwProb<T> &pr = a.probs[v.prob];
    const int J = pr.J;
    const T fD = pr.sh[3 * (J - 1) + 2];
    const Fac<T> *fac = pr.facC + (int64_t)(J - 1) * (pr.N + 4) + 2;
    const int64_t sbase = pr.soff + (int64_t)v.rhs * pr.srhs;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = v.by + r, k = v.bx + threadIdx.x;
        if (i < v.n && k < v.n) {
            const T c = rebuilt_c(a, pr, v.offT, sbase, fac[i], i, k);
            T *dp = a.D + v.offT + (int64_t)(i + 2) * pr.ldp + k + 4;
            *dp = (J >= 2) ? fma(fD, c, *dp) : fD * c;
        }
    }
}

__global__ void __launch_bounds__(256) finalize_out_kernel(TileArgs t, SwArgs<double> a, double *__restrict__ X)
{
    const TileView v = tile_view(t);
    const SwProb<double> &pr = a.probs[v.prob];
    if (!a.active[v.prob]) return;
    const int J = pr.J;
    const double fD = pr.sh[3 * (J - 1) + 2];
    const Fac<double> *fac = pr.facC + (int64_t)(J - 1) * (pr.N + 4) + 2;
    const int64_t sbase = pr.soff + (int64_t)v.rhs * pr.srhs;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = v.by + r, k = v.bx + threadIdx.x;
        if (i < v.n && k < v.n) {
            const double c = rebuilt_c(a, pr, v.offT, sbase, fac[i], i, k);
            const double y = (J >= 2) ? fma(fD, c, a.D[v.offT + (int64_t)(i + 2) * pr.ldp + k + 4]) : fD * c;
            X[v.off64 + (int64_t)i * v.n + k] = y * v.s[i] * v.s[k];
        }
    }
}

__device__ __forceinline__ double flag_nonfinite(double x, double local)
{
    // NaN and Inf both become +Inf so that the maximum flags them (fmax drops NaN)
    return (x <= 1.7976931348623157e308) ? fmax(local, x) : __longlong_as_double(0x7ff0000000000000LL);
}

__device__ __forceinline__ void block_max_to(double local, unsigned long long *out)
{
    for (int off = 16; off > 0; off >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, off));
    __shared__ double wmax[8];
    if (threadIdx.x == 0) wmax[threadIdx.y] = local;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double bm = 0.0;
        for (int q = 0; q < (int)blockDim.y; ++q) bm = fmax(bm, wmax[q]);
        atomicMax(out, (unsigned long long)__double_as_longlong(bm));
    }
    __syncthreads();  // wmax is reused by the next reduction
}

__global__ void __launch_bounds__(256) absmax_kernel(TileArgs t, const double *__restrict__ F,
                                                     unsigned long long *__restrict__ smax)
{
    int64_t t0, t1;
    tile_run(t.ntiles, t0, t1);
    double local = 0.0;
    int cur = -1;
    for (int64_t tt = t0; tt < t1; ++tt) {
        const TileView v = tile_view(t, tt);
        if (v.pair != cur) {
            if (cur >= 0) block_max_to(local, smax + cur);
            local = 0.0;
            cur = v.pair;
        }
        for (int r = threadIdx.y; r < 32; r += 8) {
            const int i = v.by + r, k = v.bx + threadIdx.x;
            if (i < v.n && k < v.n)
                local = flag_nonfinite(fabs(F[v.off64 + (int64_t)i * v.n + k] * v.s[i] * v.s[k]), local);
        }
    }
    if (cur >= 0) block_max_to(local, smax + cur);
}

template <typename T>
__global__ void __launch_bounds__(256) scale_in_kernel(TileArgs t, const double *__restrict__ F, double *__restrict__ Ft,
                                                       T *__restrict__ rho0, const unsigned long long *__restrict__ smax)
{
    const TileView v = tile_view(t);
    double inv = 1.0;
    if (smax) {
        const double sF = __longlong_as_double((long long)smax[v.pair]);
        inv = sF > 0.0 ? 1.0 / sF : 0.0;
    }
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = v.by + r, k = v.bx + threadIdx.x;
        if (i < v.n && k < v.n) {
            const double val = F[v.off64 + (int64_t)i * v.n + k] * v.s[i] * v.s[k];
            if (Ft) Ft[v.off64 + (int64_t)i * v.n + k] = val;
            rho0[v.offT + (int64_t)(i + 2) * v.ldp + k + 4] = (T)(val * inv);
        }
    }
}

// Yout = Y + s D; R = F~ - A~ Yout - Yout A~; rho0 = R / s; rmax = max |R|.
// Y and Yout are distinct buffers, so every CTA sees the same not-yet-updated halo.
__global__ void __launch_bounds__(256) residual_kernel(TileArgs t, const double *__restrict__ Y,
                                                       double *__restrict__ Yout, const float *__restrict__ D,
                                                       const double *__restrict__ Ft, float *__restrict__ rho0,
                                                       const unsigned long long *__restrict__ smax,
                                                       unsigned long long *__restrict__ rmax,
                                                       const int *__restrict__ pair_active, int y_zero)
{
    __shared__ double Ys[36][37];
    // stencil coefficients of the tile's rows and columns: -kx d_i, -kx e_{i-2}, -kx e_i
    // and -ky d_k, -ky e_{k-2}, -ky e_k (formed once per tile, not per element)
    __shared__ double cr[3][32], cc[3][32];
    int64_t t0, t1;
    tile_run(t.ntiles, t0, t1);
    double local = 0.0;
    int cur = -1;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int64_t tt = t0; tt < t1; ++tt) {
        const TileView v = tile_view(t, tt);
        const int n = v.n;
        if (v.pair != cur) {
            if (cur >= 0) block_max_to(local, rmax + cur);
            local = 0.0;
            cur = v.pair;
        }
        if (!pair_active[v.pair]) {  // converged pair: carry its iterate over unchanged
            for (int r = ty; r < 32; r += 8) {
                const int i = v.by + r, k = v.bx + tx;
                if (i < n && k < n) Yout[v.off64 + (int64_t)i * n + k] = y_zero ? 0.0 : Y[v.off64 + (int64_t)i * n + k];
            }
            continue;
        }
        const double sF = __longlong_as_double((long long)smax[v.pair]);
        const double inv = sF > 0.0 ? 1.0 / sF : 0.0;
        for (int r = ty; r < 36; r += 8) {
            const int i = v.by - 2 + r;
            for (int cc = tx; cc < 36; cc += 32) {
                const int k = v.bx - 2 + cc;
                double val = 0.0;
                if (i >= 0 && i < n && k >= 0 && k < n) {
                    val = y_zero ? 0.0 : Y[v.off64 + (int64_t)i * n + k];
                    val = fma(sF, (double)D[v.offT + (int64_t)(i + 2) * v.ldp + k + 4], val);
                }
                Ys[r][cc] = val;
            }
        }
        {
            const int q = ty * 32 + tx;  // 192 of the 256 threads form one coefficient each
            if (q < 192) {
                const int which = q >> 5, w = q & 31, set = which % 3;
                const bool row = which < 3;
                const int idx = (row ? v.by : v.bx) + w;
                const double sc = row ? v.kx : v.ky;
                double c = 0.0;
                if (idx < n) {
                    if (set == 0) c = -sc * v.d[idx];
                    else if (set == 1) c = idx >= 2 ? -sc * v.e[idx - 2] : 0.0;
                    else c = -sc * v.e[idx];  // e[idx] = 0 when idx + 2 >= n
                }
                (row ? cr : cc)[set][w] = c;
            }
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int i = v.by + r, k = v.bx + tx;
            if (i < n && k < n) {
                const double y = Ys[r + 2][tx + 2];
                double acc = Ft[v.off64 + (int64_t)i * n + k];
                // halo entries outside [0, n) are zero in Ys, and so are their coefficients
                acc = fma(cr[0][r] + cc[0][tx], y, acc);
                acc = fma(cr[1][r], Ys[r][tx + 2], acc);
                acc = fma(cr[2][r], Ys[r + 4][tx + 2], acc);
                acc = fma(cc[1][tx], Ys[r + 2][tx], acc);
                acc = fma(cc[2][tx], Ys[r + 2][tx + 4], acc);
                Yout[v.off64 + (int64_t)i * n + k] = y;
                local = flag_nonfinite(fabs(acc), local);
                rho0[v.offT + (int64_t)(i + 2) * v.ldp + k + 4] = (float)(acc * inv);
            }
        }
        __syncthreads();  // Ys is refilled by the next tile
    }
    if (cur >= 0) block_max_to(local, rmax + cur);
}

__global__ void __launch_bounds__(256) scale_out_kernel(TileArgs t, const double *__restrict__ Y, double *__restrict__ X)
{
    const TileView v = tile_view(t);
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = v.by + r, k = v.bx + threadIdx.x;
        if (i < v.n && k < v.n)
            X[v.off64 + (int64_t)i * v.n + k] = Y[v.off64 + (int64_t)i * v.n + k] * v.s[i] * v.s[k];
    }
}

template <typename T, int S>
cudaError_t row_pass_S(const SwArgs<T> &a, int j, int mode, cudaStream_t st)
{
    const size_t sm = RowGeom<T, S>::bytes;
    const dim3 grid((unsigned)a.nitems);
    if (mode == 0) row_pass_kernel<T, S, 0><<<grid, kRT, sm, st>>>(a, j);
    else if (mode == 1) row_pass_kernel<T, S, 1><<<grid, kRT, sm, st>>>(a, j);
    else row_pass_kernel<T, S, 2><<<grid, kRT, sm, st>>>(a, j);
    return cudaGetLastError();
}
template <typename T, int S>
cudaError_t col_pass_S(const SwArgs<T> &a, int j, cudaStream_t st)
{
    col_pass_kernel<T, S><<<(unsigned)a.nitems, kCT, ColGeom<T, S>::bytes, st>>>(a, j);
    return cudaGetLastError();
}

// CTAs of a reduction kernel: 8 per SM (all resident), at most one per tile.
unsigned reduction_grid(int64_t ntiles)
{
    const int64_t g = 8 * (int64_t)current_sm_count();
    return (unsigned)(ntiles < g ? (ntiles > 0 ? ntiles : 1) : g);
}

}  // namespace

bool sweep_segment_supported(bool fp64, int S) { return S == 64 || (!fp64 && S == 128); }

cudaError_t sweep_setup_kernels()
{
    cudaError_t e;
#define SETSM(kern, bytes)                                                                                \
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes))) !=    \
        cudaSuccess)                                                                                      \
        return e;
    SETSM((row_pass_kernel<float, 128, 0>), (RowGeom<float, 128>::bytes));
    SETSM((row_pass_kernel<float, 128, 1>), (RowGeom<float, 128>::bytes));
    SETSM((row_pass_kernel<float, 128, 2>), (RowGeom<float, 128>::bytes));
    SETSM((row_pass_kernel<float, 64, 0>), (RowGeom<float, 64>::bytes));
    SETSM((row_pass_kernel<float, 64, 1>), (RowGeom<float, 64>::bytes));
    SETSM((row_pass_kernel<float, 64, 2>), (RowGeom<float, 64>::bytes));
    SETSM((row_pass_kernel<double, 64, 0>), (RowGeom<double, 64>::bytes));
    SETSM((row_pass_kernel<double, 64, 1>), (RowGeom<double, 64>::bytes));
    SETSM((row_pass_kernel<double, 64, 2>), (RowGeom<double, 64>::bytes));
    SETSM((col_pass_kernel<float, 128>), (ColGeom<float, 128>::bytes));
    SETSM((col_pass_kernel<float, 64>), (ColGeom<float, 64>::bytes));
    SETSM((col_pass_kernel<double, 64>), (ColGeom<double, 64>::bytes));
#undef SETSM
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_fac_tables(const FacJob<T> *jobs, int njobs, cudaStream_t st)
{
    const int threads = 2 * njobs;
    fac_tables_kernel<T><<<(threads + 127) / 128, 128, 0, st>>>(jobs, njobs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row_pass(const SwArgs<T> &a, int j, int mode, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        if (a.S == 128) return row_pass_S<T, 128>(a, j, mode, st);
    }
    if (a.S == 64) return row_pass_S<T, 64>(a, j, mode, st);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_col_pass(const SwArgs<T> &a, int j, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        if (a.S == 128) return col_pass_S<T, 128>(a, j, st);
    }
    if (a.S == 64) return col_pass_S<T, 64>(a, j, st);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_chain(const SwArgs<T> &a, int dir, int j, cudaStream_t st)
{
    const bool big = a.chain_mode == 2 || (a.chain_mode == 0 && a.nitems <= 2 * (int64_t)current_sm_count());
    if (big)
        chain_kernel<T, true><<<(unsigned)a.nitems, 2 * kChainLines, 0, st>>>(a, dir, j);
    else
        chain_kernel<T, false><<<(unsigned)a.nitems, 2 * kChainLines, 0, st>>>(a, dir, j);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize(const TileArgs &t, const SwArgs<T> &a, const int *pair_active, cudaStream_t st)
{
    finalize_kernel<T><<<(unsigned)t.ntiles, dim3(32, 8), 0, st>>>(t, a, pair_active);
    return cudaGetLastError();
}

cudaError_t launch_finalize_out(const TileArgs &t, const SwArgs<double> &a, double *X, cudaStream_t st)
{
    finalize_out_kernel<<<(unsigned)t.ntiles, dim3(32, 8), 0, st>>>(t, a, X);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const TileArgs &t, const double *F, unsigned long long *smax, cudaStream_t st)
{
    absmax_kernel<<<reduction_grid(t.ntiles), dim3(32, 8), 0, st>>>(t, F, smax);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_in(const TileArgs &t, const double *F, double *Ft, T *rho0, const unsigned long long *smax,
                            cudaStream_t st)
{
    scale_in_kernel<T><<<(unsigned)t.ntiles, dim3(32, 8), 0, st>>>(t, F, Ft, rho0, smax);
    return cudaGetLastError();
}

cudaError_t launch_residual(const TileArgs &t, const double *Y, double *Yout, const float *D, const double *Ft,
                            float *rho0, const unsigned long long *smax, unsigned long long *rmax,
                            const int *pair_active, bool y_zero, cudaStream_t st)
{
    residual_kernel<<<reduction_grid(t.ntiles), dim3(32, 8), 0, st>>>(t, Y, Yout, D, Ft, rho0, smax, rmax, pair_active,
                                                               y_zero ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_scale_out(const TileArgs &t, const double *Y, double *X, cudaStream_t st)
{
    scale_out_kernel<<<(unsigned)t.ntiles, dim3(32, 8), 0, st>>>(t, Y, X);
    return cudaGetLastError();
}

template cudaError_t launch_fac_tables<float>(const FacJob<float> *, int, cudaStream_t);
template cudaError_t launch_fac_tables<double>(const FacJob<double> *, int, cudaStream_t);
template cudaError_t launch_row_pass<float>(const SwArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_row_pass<double>(const SwArgs<double> &, int, int, cudaStream_t);
template cudaError_t launch_col_pass<float>(const SwArgs<float> &, int, cudaStream_t);
template cudaError_t launch_col_pass<double>(const SwArgs<double> &, int, cudaStream_t);
template cudaError_t launch_chain<float>(const SwArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_chain<double>(const SwArgs<double> &, int, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const TileArgs &, const SwArgs<float> &, const int *, cudaStream_t);
template cudaError_t launch_finalize<double>(const TileArgs &, const SwArgs<double> &, const int *, cudaStream_t);
template cudaError_t launch_scale_in<float>(const TileArgs &, const double *, double *, float *,
                                            const unsigned long long *, cudaStream_t);
template cudaError_t launch_scale_in<double>(const TileArgs &, const double *, double *, double *,
                                             const unsigned long long *, cudaStream_t);

}  // namespace fps
