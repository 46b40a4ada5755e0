// FP32 sweeps inside an FP64 iterative refinement (precision FPS_FP32_REFINE).
//
// The refinement solves A~ D + D A~ = R~ for the correction D of the current
// FP64 iterate Y, with R~ = F~ - A~ Y - Y A~ computed in FP64.  The inner solve
// is Algorithm 2 written in residual-propagating form.  With L(Y) = A~ Y,
// R(Y) = Y A~ and one shift q, the ADI iteration
//     (R - q) Y_h = F - (L + q) Y,   (L - q) Y+ = F - (R + q) Y_h
// is algebraically the same as
//     Y+  = Y - 2q (L - q)^{-1} (R - q)^{-1} rho,      rho = F - (L + R) Y,
//     rho+ = (L + q)(L - q)^{-1} (R + q)(R - q)^{-1} rho.
// The second form never multiplies the (large) iterate by A~: every quantity
// fed back into a solve is the residual, whose propagation factors are bounded
// by one.  In FP32 it keeps the accuracy the first form loses to cancellation
// at small shifts.  One iteration is two kernels:
//   row pass   a = (R - q)^{-1} rho,   c = rho + 2q a            [(R+q)(R-q)^{-1} rho]
//   column pass g = (L - q)^{-1} c,  b = (L - q)^{-1} a,
//               rho+ = c + 2q g,  D <- D - 2q b
// Both are column solves (the row pass runs on rho^T), one thread per (column,
// row parity), Thomas elimination on the even/odd decoupled A~ - q I (App. B).
// Instead of spilling the forward elimination, each thread checkpoints it every
// kChunk rows and recomputes chunk by chunk in reverse, so every matrix is read
// twice and written once (no n x n scratch traffic).
#include <cuda_runtime.h>

#include "refine.cuh"

namespace fps {

namespace {

constexpr int kRC = 32;       // columns per CTA
constexpr int kChunk = 32;    // rows per checkpoint chunk (per parity)
constexpr int kTileRows = 64; // rows of a transposed-store tile (both parities)

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rows move through shared memory in slots of kU consecutive rows of one
// parity; a warp waits once per slot.
constexpr int kU = 4;         // rows per slot
constexpr int kMaxSeg = 32;   // segments per (column, parity) system

// ---------------------------------------------------------------------------
// Partitioned elimination.  Each (column, parity) system of m rows is cut into
// P segments of Ls rows (Ls a multiple of kChunk); one warp owns one segment of
// 32 columns.  With the true forward value z_in entering a segment and the true
// back-substitution value x_out leaving it,
//     z_t = zl_t + Phi_t z_in                 (zl: forward sweep started from 0)
//     x_start = a + B z_in + Psi x_out,        a = sum_t kappa_t zl_t
// where Phi_t = prod(-lf), kappa_t = ip_t prod_{u<t}(-uf_u), Psi = prod(-uf),
// B = sum kappa_t Phi_t depend only on the shift (precomputed per shift).
// Kernel 1 runs the local forward sweeps, checkpoints zl every kChunk rows and
// writes (zl_end, a) per segment; kernel 2 chains the segments (O(P) per warp),
// then recomputes each chunk from its checkpoint (converted to the true z) in
// reverse order and back-substitutes.  Every input is read twice, every output
// written once, and the segments multiply the number of independent warps.
// ---------------------------------------------------------------------------
template <int NR, int DS>
struct FwdSmem {
    float ring[2][DS][NR][kU][32];
    float4 fring[2][DS][kU];
};

template <int NR, int DS>
__global__ void __launch_bounds__(64) fwd_local_kernel(const float *__restrict__ In0, const float *__restrict__ In1,
                                                       float *__restrict__ ck, float2 *__restrict__ summ,
                                                       const float4 *__restrict__ fac, int n, int ld, int Ls)
{
    __shared__ __align__(16) FwdSmem<NR, DS> S;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, par = w;
    const int k0 = blockIdx.x * kRC, seg = blockIdx.y;
    const int m = (n - par + 1) / 2;
    const int tb = seg * Ls;
    const int te = min(tb + Ls, m);
    const int nrows = max(te - tb, 0);
    const int nslot = (nrows + kU - 1) / kU;
    const int rsub = lane >> 3, piece = lane & 7;
    const float *in[2] = {In0, In1};

    auto issue = [&](int v) {
        if (v < nslot) {
            const int b = v % DS;
            const int t = tb + v * kU + rsub;
            if (t < te) {
                const int i = par + 2 * t;
#pragma unroll
                for (int r = 0; r < NR; ++r) cp16(&S.ring[w][b][r][rsub][piece * 4], in[r] + i * ld + k0 + piece * 4);
                if (piece == 0) cp16(&S.fring[w][b][rsub], fac + i);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int v = 0; v < DS - 1; ++v) issue(v);
    float z[NR], a[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) z[r] = a[r] = 0.f;
    for (int v = 0; v < nslot; ++v) {
        __syncwarp();
        issue(v + DS - 1);
        cp_wait<DS - 1>();
        __syncwarp();
        const int b = v % DS;
#pragma unroll
        for (int rr = 0; rr < kU; ++rr) {
            const int t = tb + v * kU + rr;
            if (t < te) {
                const float4 f = S.fring[w][b][rr];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    z[r] = fmaf(-f.z, z[r], S.ring[w][b][r][rr][lane]);
                    a[r] = fmaf(f.w, z[r], a[r]);
                }
                if ((t & (kChunk - 1)) == kChunk - 1) {
                    const int c = t / kChunk;
#pragma unroll
                    for (int r = 0; r < NR; ++r) ck[((c * 2 + par) * NR + r) * ld + k0 + lane] = z[r];
                }
            }
        }
    }
    cp_wait<0>();
#pragma unroll
    for (int r = 0; r < NR; ++r) summ[((seg * 2 + par) * NR + r) * ld + k0 + lane] = make_float2(z[r], a[r]);
}

// Chain the segments of this warp's (column, parity) systems: true z entering
// segment `seg` and true x leaving it, for each of the NR right-hand sides.
template <int NR>
__device__ __forceinline__ void segment_chain(const float2 *__restrict__ summ, const float4 *__restrict__ segc,
                                              int P, int seg, int par, int ld, int kcol, float (*zin_s)[32],
                                              int lane, float *zin, float *xout)
{
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        float zi = 0.f;
        for (int s = 0; s < P; ++s) {
            zin_s[s][lane] = zi;
            const float2 ea = summ[((s * 2 + par) * NR + r) * ld + kcol];
            zi = fmaf(segc[par * P + s].x, zi, ea.x);
        }
        float xs = 0.f;
        for (int s = P - 1; s > seg; --s) {
            const float2 ea = summ[((s * 2 + par) * NR + r) * ld + kcol];
            const float4 sc = segc[par * P + s];
            xs = fmaf(sc.y, xs, fmaf(sc.z, zin_s[s][lane], ea.y));
        }
        zin[r] = zin_s[seg][lane];
        xout[r] = xs;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Row pass, kernel 2.  Input Pt = rho^T (solve down its columns).
// Outputs (stored transposed, i.e. in rho's orientation): A = a, C = c = rho + 2q a.
// ---------------------------------------------------------------------------
template <int DS>
struct RowBwdSmem {
    float ring[2][DS][kU][32];
    float4 fring[2][DS][kU];
    float zb[2][kChunk][32];    // ip * z of the chunk
    float rb[2][kChunk][32];    // rho of the chunk
    float ufb[2][kChunk];
    float zin_s[2][kMaxSeg][32];
    float tileA[kRC][kTileRows + 1];
    float tileC[kRC][kTileRows + 1];
};

template <int DS>
__global__ void __launch_bounds__(64) row_bwd_kernel(const float *__restrict__ Pt, float *__restrict__ Aout,
                                                     float *__restrict__ Cout, const float *__restrict__ ck,
                                                     const float2 *__restrict__ summ, const float4 *__restrict__ fac,
                                                     const float *__restrict__ phick, const float4 *__restrict__ segc,
                                                     float q2, int n, int ld, int Ls, int P, int nchunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowBwdSmem<DS> &S = *reinterpret_cast<RowBwdSmem<DS> *>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, par = w;
    const int k0 = blockIdx.x * kRC, seg = blockIdx.y;
    const int m = (n - par + 1) / 2, m0 = (n + 1) / 2;
    const int tb = seg * Ls;
    const int te = min(tb + Ls, m);
    const int cfirst = tb / kChunk;
    const int cend = (min(tb + Ls, m0) + kChunk - 1) / kChunk;  // same for both warps
    const int rsub = lane >> 3, piece = lane & 7;

    float zin, xout;
    segment_chain<1>(summ, segc, P, seg, par, ld, k0 + lane, S.zin_s[w], lane, &zin, &xout);

    // slots: chunks from last to first, rows ascending in each chunk
    const int last_len = max(min(te, cend * kChunk) - (cend - 1) * kChunk, 0);
    const int last_slots = (last_len + kU - 1) / kU;
    const int nslot = (te > tb) ? last_slots + (cend - 1 - cfirst) * (kChunk / kU) : 0;
    auto issue = [&](int v) {
        if (v < nslot) {
            const int b = v % DS;
            int c, t;
            if (v < last_slots) {
                c = cend - 1;
                t = c * kChunk + v * kU;
            } else {
                const int u = v - last_slots;
                c = cend - 2 - u / (kChunk / kU);
                t = c * kChunk + (u % (kChunk / kU)) * kU;
            }
            const int tr = t + rsub;
            if (tr < min((c + 1) * kChunk, te)) {
                const int i = par + 2 * tr;
                cp16(&S.ring[w][b][rsub][piece * 4], Pt + i * ld + k0 + piece * 4);
                if (piece == 0) cp16(&S.fring[w][b][rsub], fac + i);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int v = 0; v < DS - 1; ++v) issue(v);
    int v = 0;
    float x = xout;
    const float *phi = phick + par * nchunk;
    for (int c = cend - 1; c >= cfirst; --c) {
        const int t0 = c * kChunk;
        const int t1 = min(t0 + kChunk, te);
        float zz = zin;
        if (c > cfirst && t0 < te) zz = fmaf(phi[c - 1], zin, ck[((c - 1) * 2 + par) * ld + k0 + lane]);
        for (int ts = t0; ts < t1; ts += kU, ++v) {
            __syncwarp();
            issue(v + DS - 1);
            cp_wait<DS - 1>();
            __syncwarp();
            const int b = v % DS;
#pragma unroll
            for (int rr = 0; rr < kU; ++rr) {
                const int t = ts + rr;
                if (t < t1) {
                    const float rho = S.ring[w][b][rr][lane];
                    const float4 f = S.fring[w][b][rr];
                    zz = fmaf(-f.z, zz, rho);
                    S.zb[w][t - t0][lane] = zz * f.x;
                    S.rb[w][t - t0][lane] = rho;
                    if (lane == 0) S.ufb[w][t - t0] = f.y;
                }
            }
        }
        __syncwarp();
        for (int t = t1 - 1; t >= t0; --t) {
            const int tt = t - t0;
            x = fmaf(-S.ufb[w][tt], x, S.zb[w][tt][lane]);
            S.tileA[lane][2 * tt + par] = x;
            S.tileC[lane][2 * tt + par] = fmaf(q2, x, S.rb[w][tt][lane]);
        }
        __syncthreads();
        const int ibase = c * kTileRows;
        const int rows = min(kTileRows, n - ibase);
        for (int idx = threadIdx.x; idx < kRC * kTileRows; idx += 64) {
            const int cc = idx / kTileRows, rr = idx % kTileRows;
            if (k0 + cc < n && rr < rows) {
                const int o = (k0 + cc) * ld + ibase + rr;
                Aout[o] = S.tileA[cc][rr];
                Cout[o] = S.tileC[cc][rr];
            }
        }
        __syncthreads();
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// Column pass, kernel 2.  Inputs C = c, A = a (solve down columns), Dl = D.
// Outputs: Pt = (c + 2q g)^T (transposed store), Dl -= 2q b (Dl = -2q b when first).
// ---------------------------------------------------------------------------
template <int DS>
struct ColBwdSmem {
    float ring[2][DS][3][kU][32];
    float4 fring[2][DS][kU];
    float zc[2][kChunk][32];
    float za[2][kChunk][32];
    float cb[2][kChunk][32];
    float db[2][kChunk][32];
    float ufb[2][kChunk];
    float zin_s[2][kMaxSeg][32];
    float tile[kRC][kTileRows + 1];
};

template <int DS, bool FIRST>
__global__ void __launch_bounds__(64) col_bwd_kernel(const float *__restrict__ Cin, const float *__restrict__ Ain,
                                                     float *__restrict__ Dl, float *__restrict__ Pt,
                                                     const float *__restrict__ ck, const float2 *__restrict__ summ,
                                                     const float4 *__restrict__ fac, const float *__restrict__ phick,
                                                     const float4 *__restrict__ segc, float q2, int n, int ld, int Ls,
                                                     int P, int nchunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ColBwdSmem<DS> &S = *reinterpret_cast<ColBwdSmem<DS> *>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, par = w;
    const int k0 = blockIdx.x * kRC, seg = blockIdx.y;
    const int k = k0 + lane;
    const bool kin = k < n;
    const int m = (n - par + 1) / 2, m0 = (n + 1) / 2;
    const int tb = seg * Ls;
    const int te = min(tb + Ls, m);
    const int cfirst = tb / kChunk;
    const int cend = (min(tb + Ls, m0) + kChunk - 1) / kChunk;
    const int rsub = lane >> 3, piece = lane & 7;

    float zin[2], xout[2];
    segment_chain<2>(summ, segc, P, seg, par, ld, k, S.zin_s[w], lane, zin, xout);

    const int last_len = max(min(te, cend * kChunk) - (cend - 1) * kChunk, 0);
    const int last_slots = (last_len + kU - 1) / kU;
    const int nslot = (te > tb) ? last_slots + (cend - 1 - cfirst) * (kChunk / kU) : 0;
    auto issue = [&](int v) {
        if (v < nslot) {
            const int b = v % DS;
            int c, t;
            if (v < last_slots) {
                c = cend - 1;
                t = c * kChunk + v * kU;
            } else {
                const int u = v - last_slots;
                c = cend - 2 - u / (kChunk / kU);
                t = c * kChunk + (u % (kChunk / kU)) * kU;
            }
            const int tr = t + rsub;
            if (tr < min((c + 1) * kChunk, te)) {
                const int i = par + 2 * tr;
                const int o = i * ld + k0 + piece * 4;
                cp16(&S.ring[w][b][0][rsub][piece * 4], Cin + o);
                cp16(&S.ring[w][b][1][rsub][piece * 4], Ain + o);
                if (!FIRST) cp16(&S.ring[w][b][2][rsub][piece * 4], Dl + o);
                if (piece == 0) cp16(&S.fring[w][b][rsub], fac + i);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int v = 0; v < DS - 1; ++v) issue(v);
    int v = 0;
    float g = xout[0], bb = xout[1];
    const float *phi = phick + par * nchunk;
    for (int c = cend - 1; c >= cfirst; --c) {
        const int t0 = c * kChunk;
        const int t1 = min(t0 + kChunk, te);
        float zzc = zin[0], zza = zin[1];
        if (c > cfirst && t0 < te) {
            const float ph = phi[c - 1];
            zzc = fmaf(ph, zin[0], ck[(((c - 1) * 2 + par) * 2 + 0) * ld + k]);
            zza = fmaf(ph, zin[1], ck[(((c - 1) * 2 + par) * 2 + 1) * ld + k]);
        }
        for (int ts = t0; ts < t1; ts += kU, ++v) {
            __syncwarp();
            issue(v + DS - 1);
            cp_wait<DS - 1>();
            __syncwarp();
            const int b = v % DS;
#pragma unroll
            for (int rr = 0; rr < kU; ++rr) {
                const int t = ts + rr;
                if (t < t1) {
                    const int tt = t - t0;
                    const float4 f = S.fring[w][b][rr];
                    const float cv = S.ring[w][b][0][rr][lane];
                    zzc = fmaf(-f.z, zzc, cv);
                    zza = fmaf(-f.z, zza, S.ring[w][b][1][rr][lane]);
                    S.zc[w][tt][lane] = zzc * f.x;
                    S.za[w][tt][lane] = zza * f.x;
                    S.cb[w][tt][lane] = cv;
                    if (!FIRST) S.db[w][tt][lane] = S.ring[w][b][2][rr][lane];
                    if (lane == 0) S.ufb[w][tt] = f.y;
                }
            }
        }
        __syncwarp();
        for (int t = t1 - 1; t >= t0; --t) {
            const int tt = t - t0;
            const float uf = S.ufb[w][tt];
            g = fmaf(-uf, g, S.zc[w][tt][lane]);
            bb = fmaf(-uf, bb, S.za[w][tt][lane]);
            S.tile[lane][2 * tt + par] = fmaf(q2, g, S.cb[w][tt][lane]);
            if (kin) Dl[(par + 2 * t) * ld + k] = FIRST ? -q2 * bb : fmaf(-q2, bb, S.db[w][tt][lane]);
        }
        __syncthreads();
        const int ibase = c * kTileRows;
        const int rows = min(kTileRows, n - ibase);
        for (int idx = threadIdx.x; idx < kRC * kTileRows; idx += 64) {
            const int cc = idx / kTileRows, rr = idx % kTileRows;
            if (k0 + cc < n && rr < rows) Pt[(k0 + cc) * ld + ibase + rr] = S.tile[cc][rr];
        }
        __syncthreads();
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// FP64 residual with the pending correction folded in:
//   Yout = Y + s * D ;  R = F~ - A~ Yout - Yout A~ ;  Pt = (R / s)^T in FP32 ;  rmax = max |R|
// 32x32 output tile per CTA with a halo of two in both directions.  Y and Yout
// are distinct buffers, so every CTA sees the same not-yet-updated halo.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) residual_kernel(const double *__restrict__ Y, double *__restrict__ Yout,
                                                       const float *__restrict__ Dl,
                                                       const double *__restrict__ Ft, float *__restrict__ Pt,
                                                       const double *__restrict__ dband,
                                                       const double *__restrict__ eband,
                                                       const unsigned long long *__restrict__ s_bits, int64_t n,
                                                       int64_t ld, unsigned long long *__restrict__ rmax,
                                                       int apply_update, int y_zero)
{
    const double s = __longlong_as_double((long long)*s_bits);
    const double inv_s = 1.0 / s;
    __shared__ double Ys[36][37];
    __shared__ float Ts[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    // load the 36 x 36 window (rows by-2..by+33, cols bx-2..bx+33) of the updated iterate
    for (int r = ty; r < 36; r += 8) {
        const int64_t i = by - 2 + r;
        for (int cc = tx; cc < 36; cc += 32) {
            const int64_t kk = bx - 2 + cc;
            double v = 0.0;
            if (i >= 0 && i < n && kk >= 0 && kk < n) {
                v = y_zero ? 0.0 : Y[i * n + kk];
                if (apply_update) v = fma(s, (double)Dl[i * ld + kk], v);
            }
            Ys[r][cc] = v;
        }
    }
    __syncthreads();
    double local = 0.0;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = by + r;
        const int64_t kk = bx + tx;
        float out = 0.f;
        if (i < n && kk < n) {
            const double y = Ys[r + 2][tx + 2];
            double acc = Ft[i * n + kk];
            acc = fma(-(dband[i] + dband[kk]), y, acc);
            if (i >= 2) acc = fma(-eband[i - 2], Ys[r][tx + 2], acc);
            acc = fma(-eband[i], Ys[r + 4][tx + 2], acc);  // e[i] = 0 when i + 2 >= n
            if (kk >= 2) acc = fma(-eband[kk - 2], Ys[r + 2][tx], acc);
            acc = fma(-eband[kk], Ys[r + 2][tx + 4], acc);
            if (apply_update) Yout[i * n + kk] = y;
            const double aa = fabs(acc);
            local = (aa <= 1.7976931348623157e308) ? fmax(local, aa) : __longlong_as_double(0x7ff0000000000000LL);
            out = (float)(acc * inv_s);
        }
        Ts[r][tx] = out;
    }
    __syncthreads();
    // transposed FP32 store: Pt[k][i]
    for (int r = ty; r < 32; r += 8) {
        const int64_t kk = bx + r, i = by + tx;
        if (kk < n && i < n) Pt[kk * ld + i] = Ts[tx][r];
    }
    // block max -> global max (non-negative doubles order like their bit patterns)
    for (int off = 16; off > 0; off >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, off));
    __shared__ double wmax[8];
    if (tx == 0) wmax[ty] = local;
    __syncthreads();
    if (tx == 0 && ty == 0) {
        double bm = 0.0;
        for (int t = 0; t < 8; ++t) bm = fmax(bm, wmax[t]);
        atomicMax(rmax, (unsigned long long)__double_as_longlong(bm));
    }
}

// Scale-in for the refinement: F~ = D_s F D_s (FP64, n x n), rho0^T = (F~ / s)^T
// in FP32 (ld-strided), and max |F~|.
__global__ void __launch_bounds__(256) refine_scale_in_kernel(const double *__restrict__ F, double *__restrict__ Ft,
                                                              float *__restrict__ Pt, const double *__restrict__ sc,
                                                              int64_t n, int64_t ld,
                                                              const unsigned long long *__restrict__ s_bits)
{
    const double inv_s = 1.0 / __longlong_as_double((long long)*s_bits);
    __shared__ float t[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = by + r, kk = bx + threadIdx.x;
        float v32 = 0.f;
        if (i < n && kk < n) {
            const double v = F[i * n + kk] * sc[i] * sc[kk];
            Ft[i * n + kk] = v;
            v32 = (float)(v * inv_s);
        }
        t[r][threadIdx.x] = v32;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t kk = bx + r, i = by + threadIdx.x;
        if (i < n && kk < n) Pt[kk * ld + i] = t[threadIdx.x][r];
    }
}

__global__ void absmax_kernel(const double *__restrict__ F, const double *__restrict__ sc, int64_t n,
                              unsigned long long *__restrict__ out)
{
    double local = 0.0;
    const int64_t nn = n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / n, kk = t - i * n;
        const double a = fabs(F[t] * sc[i] * sc[kk]);
        // NaN and Inf both become +Inf so that the maximum flags them (fmax drops NaN)
        local = (a <= 1.7976931348623157e308) ? fmax(local, a) : __longlong_as_double(0x7ff0000000000000LL);
    }
    for (int off = 16; off > 0; off >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(local));
}

// FP32 factors of A~ - q I for the partitioned sweeps, from FP64 arithmetic:
//   fac[i]   = {1/den_i, e_i/den_i, e_{i-2}/den_{i-2}, kappa_i}
//   phick[c] = Phi at the last row of chunk c (relative to its segment start)
//   segc[s]  = {Phi_end, Psi, B, 0} of segment s ({1, 1, 0, 0} when empty)
__global__ void factor32_kernel(const double *__restrict__ d, const double *__restrict__ e,
                                const double *__restrict__ q, int J, int64_t n, int Ls, int P, int nchunk,
                                float4 *__restrict__ fac, float *__restrict__ phick, float4 *__restrict__ segc)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 2 * J) return;
    const int j = tid >> 1, par = tid & 1;
    const double qj = q[j];
    const int64_t m = (n - par + 1) / 2;
    float4 *fj = fac + (int64_t)j * n;
    float *pj = phick + ((int64_t)j * 2 + par) * nchunk;
    float4 *sj = segc + ((int64_t)j * 2 + par) * P;
    double uf_prev = 0.0, Phi = 1.0, prodU = 1.0, B = 0.0;
    for (int64_t t = 0; t < m; ++t) {
        const int64_t i = par + 2 * t;
        if (t % Ls == 0) {
            Phi = 1.0;
            prodU = 1.0;
            B = 0.0;
        }
        double den = d[i] - qj;
        if (i >= 2) den -= e[i - 2] * uf_prev;
        const double ip = 1.0 / den;
        const double uf = e[i] * ip;
        const double lf = uf_prev;
        Phi *= -lf;
        const double kappa = ip * prodU;
        prodU *= -uf;
        B += kappa * Phi;
        fj[i] = make_float4((float)ip, (float)uf, (float)lf, (float)kappa);
        if (t % kChunk == kChunk - 1) pj[t / kChunk] = (float)Phi;
        const int64_t seg = t / Ls;
        const int64_t seg_end = ((seg + 1) * Ls < m) ? (seg + 1) * Ls : m;
        if (t == seg_end - 1) sj[seg] = make_float4((float)Phi, (float)prodU, (float)B, 0.f);
        uf_prev = uf;
    }
    for (int64_t s = (m + Ls - 1) / Ls; s < P; ++s) sj[s] = make_float4(1.f, 1.f, 0.f, 0.f);
}

constexpr int kDF = 12;  // ring depth (slots) of the forward kernels
constexpr int kDB = 8;   // ring depth (slots) of the backward kernels

template <int DS>
size_t rowb_smem() { return sizeof(RowBwdSmem<DS>); }
template <int DS>
size_t colb_smem() { return sizeof(ColBwdSmem<DS>); }

}  // namespace

RefineGeometry refine_geometry(int64_t n, int sms)
{
    RefineGeometry g;
    g.ld = (n + 31) / 32 * 32;
    const int64_t m0 = (n + 1) / 2;
    const int64_t nblk = (n + kRC - 1) / kRC;
    g.nblk = nblk;
    g.nchunk = (m0 + kChunk - 1) / kChunk;
    // enough segments for ~16 warps per SM, at most kMaxSeg, each a whole number of chunks
    int64_t want = (16LL * sms + 2 * nblk - 1) / (2 * nblk);
    if (want < 1) want = 1;
    if (want > kMaxSeg) want = kMaxSeg;
    int64_t Ls = (m0 + want - 1) / want;
    Ls = (Ls + kChunk - 1) / kChunk * kChunk;
    if (Ls < kChunk) Ls = kChunk;
    g.Ls = Ls;
    g.P = (m0 + Ls - 1) / Ls;
    if (g.P < 1) g.P = 1;
    return g;
}

int64_t refine_checkpoint_floats(const RefineGeometry &g) { return g.nchunk * 2 * 2 * g.ld; }
int64_t refine_summary_float2(const RefineGeometry &g) { return g.P * 2 * 2 * g.ld; }

cudaError_t refine_setup_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(row_bwd_kernel<kDB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rowb_smem<kDB>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(col_bwd_kernel<kDB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)colb_smem<kDB>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(col_bwd_kernel<kDB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)colb_smem<kDB>());
}

cudaError_t launch_row_pass(const float *Pt, float *A, float *C, const RefineScratch &w, const float4 *fac,
                            const float *phick, const float4 *segc, float q2, int64_t n, const RefineGeometry &g,
                            cudaStream_t st)
{
    const dim3 grid((unsigned)g.nblk, (unsigned)g.P), block(64);
    fwd_local_kernel<1, kDF><<<grid, block, 0, st>>>(Pt, nullptr, w.ck, w.summ, fac, (int)n, (int)g.ld, (int)g.Ls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    row_bwd_kernel<kDB><<<grid, block, rowb_smem<kDB>(), st>>>(Pt, A, C, w.ck, w.summ, fac, phick, segc, q2, (int)n,
                                                             (int)g.ld, (int)g.Ls, (int)g.P, (int)g.nchunk);
    return cudaGetLastError();
}

cudaError_t launch_col_pass(const float *C, const float *A, float *Dl, float *Pt, const RefineScratch &w,
                            const float4 *fac, const float *phick, const float4 *segc, float q2, int64_t n,
                            const RefineGeometry &g, bool first, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)
{
    const dim3 grid((unsigned)g.nblk, (unsigned)g.P), block(64);
    fwd_local_kernel<2, kDF><<<grid, block, 0, st>>>(C, A, w.ck, w.summ, fac, (int)n, (int)g.ld, (int)g.Ls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev0 && (e = cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (first)
        col_bwd_kernel<kDB, true><<<grid, block, colb_smem<kDB>(), st>>>(C, A, Dl, Pt, w.ck, w.summ, fac, phick, segc,
                                                                        q2, (int)n, (int)g.ld, (int)g.Ls, (int)g.P,
                                                                        (int)g.nchunk);
    else
        col_bwd_kernel<kDB, false><<<grid, block, colb_smem<kDB>(), st>>>(C, A, Dl, Pt, w.ck, w.summ, fac, phick,
                                                                         segc, q2, (int)n, (int)g.ld, (int)g.Ls,
                                                                         (int)g.P, (int)g.nchunk);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev1) e = cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal);
    return e;
}

cudaError_t launch_residual(const double *Y, double *Yout, const float *Dl, const double *Ft, float *Pt, const double *d,
                            const double *e, const unsigned long long *s_bits, int64_t n, int64_t ld,
                            unsigned long long *rmax, bool apply_update, bool y_zero, cudaStream_t st)
{
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
    residual_kernel<<<grid, block, 0, st>>>(Y, Yout, Dl, Ft, Pt, d, e, s_bits, n, ld, rmax, apply_update ? 1 : 0,
                                            y_zero ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_refine_scale_in(const double *F, double *Ft, float *Pt, const double *sc, int64_t n, int64_t ld,
                                   const unsigned long long *s_bits, cudaStream_t st)
{
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
    refine_scale_in_kernel<<<grid, block, 0, st>>>(F, Ft, Pt, sc, n, ld, s_bits);
    return cudaGetLastError();
}

cudaError_t launch_absmax_scaled(const double *F, const double *sc, int64_t n, unsigned long long *out,
                                 cudaStream_t st)
{
    const int64_t nn = n * n;
    int blocks = (int)((nn + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    absmax_kernel<<<blocks, 256, 0, st>>>(F, sc, n, out);
    return cudaGetLastError();
}

cudaError_t launch_factors32(const double *d, const double *e, const double *q, int J, int64_t n,
                             const RefineGeometry &g, float4 *fac, float *phick, float4 *segc, cudaStream_t st)
{
    const int threads = 2 * J;
    factor32_kernel<<<(threads + 127) / 128, 128, 0, st>>>(d, e, q, J, n, (int)g.Ls, (int)g.P, (int)g.nchunk, fac,
                                                          phick, segc);
    return cudaGetLastError();
}

}  // namespace fps
