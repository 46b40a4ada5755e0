// FP32 sweeps inside an FP64 iterative refinement (precision FPS_FP32_REFINE),
// for one problem or a batch of problems of different sizes.
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
// at small shifts.  One iteration is two passes:
//   row pass    a = (R - q)^{-1} rho,   c = rho + 2q a            [(R+q)(R-q)^{-1} rho]
//   column pass g = (L - q)^{-1} c,  b = (L - q)^{-1} a,
//               rho+ = c + 2q g,  D <- D - 2q b
// Both are column solves (the row pass runs on rho^T), one thread per (column,
// row parity), Thomas elimination on the even/odd decoupled A~ - q I (App. B).
//
// Work decomposition.  Each (column, parity) system of m rows is cut into P
// segments of Ls rows; a CTA (two warps, one per parity) owns 32 columns of one
// segment of one right-hand side of one problem.  With the true forward value
// z_in entering a segment and the true back-substitution value x_out leaving it,
//     z_t = zl_t + Phi_t z_in                 (zl: forward sweep started from 0)
//     x_start = a + B z_in + Psi x_out,        a = sum_t kappa_t zl_t
// where Phi_t = prod(-lf), kappa_t = ip_t prod_{u<t}(-uf_u), Psi = prod(-uf),
// B = sum kappa_t Phi_t depend only on the shift (precomputed per shift in FP64).
// Pass kernel 1 runs the local forward sweeps, checkpoints zl every kChunk rows
// and writes (zl_end, a) per segment; pass kernel 2 chains the segments (O(P) per
// warp, in registers), recomputes each chunk from its checkpoint (converted to the
// true z) in reverse order and back-substitutes.  Every input is read twice and
// every output written once; no n x n scratch.  A work-item table lists the CTAs
// of all problems, so one launch sweeps a whole batch; problems that have finished
// their iterations (or are inactive) exit at once.
#include <cuda_runtime.h>

#include "refine.cuh"

namespace fps {

namespace {

constexpr int kRC = 32;        // columns per CTA
constexpr int kChunk = 16;     // rows per checkpoint chunk (per parity)
constexpr int kTileRows = 2 * kChunk;  // rows of a transposed-store tile (both parities)
constexpr int kU = 4;          // rows per shared-memory slot
constexpr int kMaxSeg = 64;    // segments per (column, parity) system

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

// Per-CTA view of one work item.
struct ItemView {
    int n, ld, Ls, P, nchunk, seg, k0;
    const float4 *fac;
    const float *phick;
    const float4 *segc;
    float q2;
    int64_t off;   // FP32 element offset of this problem / right-hand side
    float *ck;     // checkpoints of this problem / right-hand side
    float2 *summ;  // segment summaries of this problem / right-hand side
};

// Returns false when the item's problem is inactive or has no iteration j.
__device__ __forceinline__ bool load_item(const RefProb *__restrict__ probs, const int4 *__restrict__ items,
                                          const int *__restrict__ active, int j, float *ck, float2 *summ,
                                          ItemView &v)
{
    const int4 it = items[blockIdx.x];
    const RefProb &p = probs[it.x];
    if (!active[it.x] || j >= p.J) return false;
    v.n = p.n;
    v.ld = p.ld;
    v.Ls = p.Ls;
    v.P = p.P;
    v.nchunk = p.nchunk;
    v.seg = it.w;
    v.k0 = it.z * kRC;
    v.fac = p.fac + (int64_t)j * p.n;
    v.phick = p.phick + (int64_t)j * 2 * p.nchunk;
    v.segc = p.segc + (int64_t)j * 2 * p.P;
    v.q2 = p.q2[j];
    v.off = p.off32 + (int64_t)it.y * p.rhs32;
    v.ck = ck + p.offck + (int64_t)it.y * p.rhsck;
    v.summ = summ + p.offsm + (int64_t)it.y * p.rhssm;
    return true;
}

// ---------------------------------------------------------------------------
// Pass kernel 1: local forward sweeps of one segment (NR right-hand sides).
// ---------------------------------------------------------------------------
template <int NR, int DS>
struct FwdSmem {
    float ring[2][DS][NR][kU][32];
    float4 fring[2][DS][kU];
};

template <int NR, int DS>
__global__ void __launch_bounds__(64) fwd_local_kernel(const RefProb *__restrict__ probs,
                                                       const int4 *__restrict__ items, const int *__restrict__ active,
                                                       int j, const float *__restrict__ In0,
                                                       const float *__restrict__ In1, float *__restrict__ ckbase,
                                                       float2 *__restrict__ summbase)
{
    __shared__ __align__(16) FwdSmem<NR, DS> S;
    ItemView v;
    if (!load_item(probs, items, active, j, ckbase, summbase, v)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, par = w;
    const int n = v.n, ld = v.ld, k0 = v.k0;
    const int m = (n - par + 1) / 2;
    const int tb = v.seg * v.Ls;
    const int te = min(tb + v.Ls, m);
    const int nrows = max(te - tb, 0);
    const int nslot = (nrows + kU - 1) / kU;
    const int rsub = lane >> 3, piece = lane & 7;
    const float *in[2] = {In0 + v.off, (NR > 1 ? In1 : In0) + v.off};
    const float4 *fac = v.fac;

    auto issue = [&](int s) {
        if (s < nslot) {
            const int b = s % DS;
            const int t = tb + s * kU + rsub;
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
    for (int s = 0; s < DS - 1; ++s) issue(s);
    float z[NR], a[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) z[r] = a[r] = 0.f;
    for (int s = 0; s < nslot; ++s) {
        __syncwarp();
        issue(s + DS - 1);
        cp_wait<DS - 1>();
        __syncwarp();
        const int b = s % DS;
#pragma unroll
        for (int rr = 0; rr < kU; ++rr) {
            const int t = tb + s * kU + rr;
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
                    for (int r = 0; r < NR; ++r) v.ck[((c * 2 + par) * NR + r) * ld + k0 + lane] = z[r];
                }
            }
        }
    }
    cp_wait<0>();
#pragma unroll
    for (int r = 0; r < NR; ++r) v.summ[((v.seg * 2 + par) * NR + r) * ld + k0 + lane] = make_float2(z[r], a[r]);
}

// Chain the segments of this lane's (column, parity) system for right-hand side r:
// the true z entering segment `seg` and the true x leaving it, in one ascending
// pass:  z_in(s+1) = zl_end(s) + Phi_end(s) z_in(s);
//        x_out(seg) = sum_{s > seg} (a_s + B_s z_in(s)) prod_{seg < s' < s} Psi_s'.
template <int NR>
__device__ __forceinline__ void segment_chain(const ItemView &v, int par, int r, int kcol, float &zin, float &xout)
{
    float zi = 0.f, xo = 0.f, prod = 1.f;
    zin = 0.f;
    for (int s = 0; s < v.P; ++s) {
        const float2 ea = v.summ[((s * 2 + par) * NR + r) * v.ld + kcol];
        const float4 sc = v.segc[par * v.P + s];
        if (s == v.seg) zin = zi;
        if (s > v.seg) {
            xo = fmaf(fmaf(sc.z, zi, ea.y), prod, xo);
            prod *= sc.y;
        }
        zi = fmaf(sc.x, zi, ea.x);
    }
    xout = xo;
}

// Chunk slots of pass kernel 2: chunks from last to first, rows ascending inside.
struct SlotMap {
    int cend, cfirst, last_slots, nslot, te;
    __device__ __forceinline__ void at(int s, int &c, int &t) const
    {
        if (s < last_slots) {
            c = cend - 1;
            t = c * kChunk + s * kU;
        } else {
            const int u = s - last_slots;
            c = cend - 2 - u / (kChunk / kU);
            t = c * kChunk + (u % (kChunk / kU)) * kU;
        }
    }
};
__device__ __forceinline__ SlotMap make_slots(int tb, int te, int Ls, int m0)
{
    SlotMap sm;
    sm.cfirst = tb / kChunk;
    sm.cend = (min(tb + Ls, m0) + kChunk - 1) / kChunk;
    const int last_len = max(min(te, sm.cend * kChunk) - (sm.cend - 1) * kChunk, 0);
    sm.last_slots = (last_len + kU - 1) / kU;
    sm.nslot = (te > tb) ? sm.last_slots + (sm.cend - 1 - sm.cfirst) * (kChunk / kU) : 0;
    sm.te = te;
    return sm;
}

// Transposed store of a 32 x kTileRows tile: Out[(k0 + cc) * ld + ibase + rr] for
// cc < 32 (k0 + cc < n), rr < kTileRows (ibase + rr < ld), four rows per 16-byte store.
// Rows beyond n inside the padded leading dimension receive don't-care values.
__device__ __forceinline__ void store_tile(float *__restrict__ out, const float (*tile)[kTileRows + 1], int k0,
                                           int ibase, int n, int ld)
{
    const int lim = min(kTileRows, ld - ibase);
    for (int idx = threadIdx.x; idx < kRC * (kTileRows / 4); idx += 64) {
        const int cc = idx / (kTileRows / 4), r4 = (idx % (kTileRows / 4)) * 4;
        if (k0 + cc < n && r4 < lim) {
            const float4 val = make_float4(tile[cc][r4], tile[cc][r4 + 1], tile[cc][r4 + 2], tile[cc][r4 + 3]);
            *reinterpret_cast<float4 *>(out + (int64_t)(k0 + cc) * ld + ibase + r4) = val;
        }
    }
}

// ---------------------------------------------------------------------------
// Row pass, kernel 2.  Input rho^T (solve down its columns).  Outputs stored
// transposed (in rho's orientation): a and c = rho + 2q a.
// ---------------------------------------------------------------------------
template <int DS>
struct RowBwdSmem {
    float ring[2][DS][kU][32];
    float4 fring[2][DS][kU];
    float zb[2][kChunk][32];  // ip * z of the chunk
    float rb[2][kChunk][32];  // rho of the chunk
    float ufb[2][kChunk];
    float tileA[kRC][kTileRows + 1];
    float tileC[kRC][kTileRows + 1];
};

template <int DS>
__global__ void __launch_bounds__(64) row_bwd_kernel(const RefProb *__restrict__ probs,
                                                     const int4 *__restrict__ items, const int *__restrict__ active,
                                                     int j, const float *__restrict__ Ptb, float *__restrict__ Ab,
                                                     float *__restrict__ Cb, float *__restrict__ ckbase,
                                                     float2 *__restrict__ summbase)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowBwdSmem<DS> &S = *reinterpret_cast<RowBwdSmem<DS> *>(smem_raw);
    ItemView v;
    if (!load_item(probs, items, active, j, ckbase, summbase, v)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, par = w;
    const int n = v.n, ld = v.ld, k0 = v.k0;
    const int m = (n - par + 1) / 2, m0 = (n + 1) / 2;
    const int tb = v.seg * v.Ls;
    const int te = min(tb + v.Ls, m);
    const int rsub = lane >> 3, piece = lane & 7;
    const float *Pt = Ptb + v.off;
    float *Aout = Ab + v.off, *Cout = Cb + v.off;
    const float4 *fac = v.fac;
    const float q2 = v.q2;

    float zin, xout;
    segment_chain<1>(v, par, 0, k0 + lane, zin, xout);

    const SlotMap sm = make_slots(tb, te, v.Ls, m0);
    auto issue = [&](int s) {
        if (s < sm.nslot) {
            const int b = s % DS;
            int c, t;
            sm.at(s, c, t);
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
    for (int s = 0; s < DS - 1; ++s) issue(s);
    int s = 0;
    float x = xout;
    const float *phi = v.phick + par * v.nchunk;
    for (int c = sm.cend - 1; c >= sm.cfirst; --c) {
        const int t0 = c * kChunk;
        const int t1 = min(t0 + kChunk, te);
        float zz = zin;
        if (c > sm.cfirst && t0 < te) zz = fmaf(phi[c - 1], zin, v.ck[((c - 1) * 2 + par) * ld + k0 + lane]);
        for (int ts = t0; ts < t1; ts += kU, ++s) {
            __syncwarp();
            issue(s + DS - 1);
            cp_wait<DS - 1>();
            __syncwarp();
            const int b = s % DS;
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
#pragma unroll 8
        for (int tt = kChunk - 1; tt >= 0; --tt) {
            if (t0 + tt < t1) {
                x = fmaf(-S.ufb[w][tt], x, S.zb[w][tt][lane]);
                S.tileA[lane][2 * tt + par] = x;
                S.tileC[lane][2 * tt + par] = fmaf(q2, x, S.rb[w][tt][lane]);
            }
        }
        __syncthreads();
        store_tile(Aout, S.tileA, k0, c * kTileRows, n, ld);
        store_tile(Cout, S.tileC, k0, c * kTileRows, n, ld);
        __syncthreads();
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// Column pass, kernel 2.  Inputs c, a (solve down columns), D.  Outputs rho+ =
// c + 2q g stored transposed, D -= 2q b in place (D = -2q b when FIRST).  The D
// values of a chunk are loaded into registers while the chunk is recomputed.
// ---------------------------------------------------------------------------
template <int DS>
struct ColBwdSmem {
    float ring[2][DS][2][kU][32];
    float4 fring[2][DS][kU];
    float zc[2][kChunk][32];
    float za[2][kChunk][32];
    float cb[2][kChunk][32];
    float ufb[2][kChunk];
    float tile[kRC][kTileRows + 1];
};

template <int DS, bool FIRST>
__global__ void __launch_bounds__(64) col_bwd_kernel(const RefProb *__restrict__ probs,
                                                     const int4 *__restrict__ items, const int *__restrict__ active,
                                                     int j, const float *__restrict__ Cb, const float *__restrict__ Ab,
                                                     float *__restrict__ Db, float *__restrict__ Ptb,
                                                     float *__restrict__ ckbase, float2 *__restrict__ summbase)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ColBwdSmem<DS> &S = *reinterpret_cast<ColBwdSmem<DS> *>(smem_raw);
    ItemView v;
    if (!load_item(probs, items, active, j, ckbase, summbase, v)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, par = w;
    const int n = v.n, ld = v.ld, k0 = v.k0;
    const int k = k0 + lane;
    const bool kin = k < n;
    const int m = (n - par + 1) / 2, m0 = (n + 1) / 2;
    const int tb = v.seg * v.Ls;
    const int te = min(tb + v.Ls, m);
    const int rsub = lane >> 3, piece = lane & 7;
    const float *Cin = Cb + v.off, *Ain = Ab + v.off;
    float *Dl = Db + v.off, *Pt = Ptb + v.off;
    const float4 *fac = v.fac;
    const float q2 = v.q2;

    float zin0, zin1, g, bb;
    segment_chain<2>(v, par, 0, k, zin0, g);
    segment_chain<2>(v, par, 1, k, zin1, bb);

    const SlotMap sm = make_slots(tb, te, v.Ls, m0);
    auto issue = [&](int s) {
        if (s < sm.nslot) {
            const int b = s % DS;
            int c, t;
            sm.at(s, c, t);
            const int tr = t + rsub;
            if (tr < min((c + 1) * kChunk, te)) {
                const int i = par + 2 * tr;
                const int o = i * ld + k0 + piece * 4;
                cp16(&S.ring[w][b][0][rsub][piece * 4], Cin + o);
                cp16(&S.ring[w][b][1][rsub][piece * 4], Ain + o);
                if (piece == 0) cp16(&S.fring[w][b][rsub], fac + i);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int s = 0; s < DS - 1; ++s) issue(s);
    int s = 0;
    const float *phi = v.phick + par * v.nchunk;
    for (int c = sm.cend - 1; c >= sm.cfirst; --c) {
        const int t0 = c * kChunk;
        const int t1 = min(t0 + kChunk, te);
        float dreg[kChunk];
        if (!FIRST) {
#pragma unroll
            for (int tt = 0; tt < kChunk; ++tt)
                dreg[tt] = (kin && t0 + tt < t1) ? Dl[(par + 2 * (t0 + tt)) * ld + k] : 0.f;
        }
        float zzc = zin0, zza = zin1;
        if (c > sm.cfirst && t0 < te) {
            const float ph = phi[c - 1];
            zzc = fmaf(ph, zin0, v.ck[(((c - 1) * 2 + par) * 2 + 0) * ld + k]);
            zza = fmaf(ph, zin1, v.ck[(((c - 1) * 2 + par) * 2 + 1) * ld + k]);
        }
        for (int ts = t0; ts < t1; ts += kU, ++s) {
            __syncwarp();
            issue(s + DS - 1);
            cp_wait<DS - 1>();
            __syncwarp();
            const int b = s % DS;
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
                    if (lane == 0) S.ufb[w][tt] = f.y;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int tt = kChunk - 1; tt >= 0; --tt) {
            if (t0 + tt < t1) {
                const float uf = S.ufb[w][tt];
                g = fmaf(-uf, g, S.zc[w][tt][lane]);
                bb = fmaf(-uf, bb, S.za[w][tt][lane]);
                S.tile[lane][2 * tt + par] = fmaf(q2, g, S.cb[w][tt][lane]);
                if (kin) Dl[(par + 2 * (t0 + tt)) * ld + k] = FIRST ? -q2 * bb : fmaf(-q2, bb, dreg[tt]);
            }
        }
        __syncthreads();
        store_tile(Pt, S.tile, k0, c * kTileRows, n, ld);
        __syncthreads();
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// FP64 kernels over 32 x 32 tiles of every (problem, right-hand side).
// A tile item is {problem * 256 + rhs, tile column, tile row, 0}.
// ---------------------------------------------------------------------------
struct TileView {
    int n, ld;
    int64_t off64, off32;
    const double *d, *e, *s;
    int idx;  // index of the (problem, rhs) pair for per-pair scalars
    int64_t bx, by;
};
__device__ __forceinline__ TileView load_tile(const RefProb64 *__restrict__ probs, const int4 *__restrict__ tiles)
{
    const int4 t = tiles[blockIdx.x];
    const RefProb64 &p = probs[t.x >> 8];
    const int rhs = t.x & 255;
    TileView v;
    v.n = p.n;
    v.ld = p.ld;
    v.off64 = p.off64 + (int64_t)rhs * p.n * p.n;
    v.off32 = p.off32 + (int64_t)rhs * p.rhs32;
    v.d = p.d;
    v.e = p.e;
    v.s = p.s;
    v.idx = p.pair0 + rhs;
    v.bx = (int64_t)t.y * 32;
    v.by = (int64_t)t.z * 32;
    return v;
}

__device__ __forceinline__ double flag_nonfinite(double a, double local)
{
    // NaN and Inf both become +Inf so that the maximum flags them (fmax drops NaN)
    return (a <= 1.7976931348623157e308) ? fmax(local, a) : __longlong_as_double(0x7ff0000000000000LL);
}

__device__ __forceinline__ void block_max_to(double local, unsigned long long *out)
{
    for (int off = 16; off > 0; off >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, off));
    __shared__ double wmax[8];
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (tx == 0) wmax[ty] = local;
    __syncthreads();
    if (tx == 0 && ty == 0) {
        double bm = 0.0;
        for (int t = 0; t < (int)blockDim.y; ++t) bm = fmax(bm, wmax[t]);
        atomicMax(out, (unsigned long long)__double_as_longlong(bm));
    }
}

// max |D_s F D_s| per (problem, rhs)
__global__ void __launch_bounds__(256) absmax_tiles_kernel(const RefProb64 *__restrict__ probs,
                                                           const int4 *__restrict__ tiles,
                                                           const double *__restrict__ F,
                                                           unsigned long long *__restrict__ smax)
{
    const TileView v = load_tile(probs, tiles);
    double local = 0.0;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t i = v.by + r, kk = v.bx + threadIdx.x;
        if (i < v.n && kk < v.n) local = flag_nonfinite(fabs(F[v.off64 + i * v.n + kk] * v.s[i] * v.s[kk]), local);
    }
    block_max_to(local, smax + v.idx);
}

// F~ = D_s F D_s (FP64) and rho0^T = (F~ / s)^T (FP32, ld-strided)
__global__ void __launch_bounds__(256) scale_in_tiles_kernel(const RefProb64 *__restrict__ probs,
                                                             const int4 *__restrict__ tiles,
                                                             const double *__restrict__ F, double *__restrict__ Ft,
                                                             float *__restrict__ Pt,
                                                             const unsigned long long *__restrict__ smax)
{
    __shared__ float t[32][33];
    const TileView v = load_tile(probs, tiles);
    const double sF = __longlong_as_double((long long)smax[v.idx]);
    const double inv_s = sF > 0.0 ? 1.0 / sF : 0.0;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t i = v.by + r, kk = v.bx + threadIdx.x;
        float v32 = 0.f;
        if (i < v.n && kk < v.n) {
            const double val = F[v.off64 + i * v.n + kk] * v.s[i] * v.s[kk];
            Ft[v.off64 + i * v.n + kk] = val;
            v32 = (float)(val * inv_s);
        }
        t[r][threadIdx.x] = v32;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t kk = v.bx + r, i = v.by + threadIdx.x;
        if (i < v.n && kk < v.n) Pt[v.off32 + kk * v.ld + i] = t[threadIdx.x][r];
    }
}

// Yout = Y + s D ; R = F~ - A~ Yout - Yout A~ ; Pt = (R / s)^T ; rmax = max |R|.
// Y and Yout are distinct buffers, so every CTA sees the same not-yet-updated halo.
// Right-hand sides that have converged only copy Y to Yout.
__global__ void __launch_bounds__(256) residual_tiles_kernel(const RefProb64 *__restrict__ probs,
                                                             const int4 *__restrict__ tiles,
                                                             const double *__restrict__ Y, double *__restrict__ Yout,
                                                             const float *__restrict__ Dl,
                                                             const double *__restrict__ Ft, float *__restrict__ Pt,
                                                             const unsigned long long *__restrict__ smax,
                                                             unsigned long long *__restrict__ rmax,
                                                             const int *__restrict__ pair_active, int y_zero)
{
    __shared__ double Ys[36][37];
    __shared__ float Ts[32][33];
    const TileView v = load_tile(probs, tiles);
    if (!pair_active[v.idx]) {
        // converged right-hand side: carry its iterate over to the other buffer unchanged
        for (int r = threadIdx.y; r < 32; r += 8) {
            const int64_t i = v.by + r, kk = v.bx + threadIdx.x;
            if (i < v.n && kk < v.n) Yout[v.off64 + i * v.n + kk] = y_zero ? 0.0 : Y[v.off64 + i * v.n + kk];
        }
        return;
    }
    const double sF = __longlong_as_double((long long)smax[v.idx]);
    const double inv_s = sF > 0.0 ? 1.0 / sF : 0.0;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t n = v.n;
    for (int r = ty; r < 36; r += 8) {
        const int64_t i = v.by - 2 + r;
        for (int cc = tx; cc < 36; cc += 32) {
            const int64_t kk = v.bx - 2 + cc;
            double val = 0.0;
            if (i >= 0 && i < n && kk >= 0 && kk < n) {
                val = y_zero ? 0.0 : Y[v.off64 + i * n + kk];
                val = fma(sF, (double)Dl[v.off32 + i * v.ld + kk], val);
            }
            Ys[r][cc] = val;
        }
    }
    __syncthreads();
    double local = 0.0;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = v.by + r;
        const int64_t kk = v.bx + tx;
        float out = 0.f;
        if (i < n && kk < n) {
            const double y = Ys[r + 2][tx + 2];
            double acc = Ft[v.off64 + i * n + kk];
            acc = fma(-(v.d[i] + v.d[kk]), y, acc);
            if (i >= 2) acc = fma(-v.e[i - 2], Ys[r][tx + 2], acc);
            acc = fma(-v.e[i], Ys[r + 4][tx + 2], acc);  // e[i] = 0 when i + 2 >= n
            if (kk >= 2) acc = fma(-v.e[kk - 2], Ys[r + 2][tx], acc);
            acc = fma(-v.e[kk], Ys[r + 2][tx + 4], acc);
            Yout[v.off64 + i * n + kk] = y;
            local = flag_nonfinite(fabs(acc), local);
            out = (float)(acc * inv_s);
        }
        Ts[r][tx] = out;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t kk = v.bx + r, i = v.by + tx;
        if (kk < n && i < n) Pt[v.off32 + kk * v.ld + i] = Ts[tx][r];
    }
    block_max_to(local, rmax + v.idx);
}

// X = D_s Y D_s
__global__ void __launch_bounds__(256) scale_out_tiles_kernel(const RefProb64 *__restrict__ probs,
                                                              const int4 *__restrict__ tiles,
                                                              const double *__restrict__ Y, double *__restrict__ X)
{
    const TileView v = load_tile(probs, tiles);
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t i = v.by + r, kk = v.bx + threadIdx.x;
        if (i < v.n && kk < v.n) X[v.off64 + i * v.n + kk] = Y[v.off64 + i * v.n + kk] * v.s[i] * v.s[kk];
    }
}

// FP32 factors of A~ - q I for the partitioned sweeps, from FP64 arithmetic, one
// thread per (problem, shift, parity):
//   fac[i]   = {1/den_i, e_i/den_i, e_{i-2}/den_{i-2}, kappa_i}
//   phick[c] = Phi at the last row of chunk c (relative to its segment start)
//   segc[s]  = {Phi_end, Psi, B, 0} of segment s ({1, 1, 0, 0} when empty)
__global__ void factor32_kernel(const FactorJob *__restrict__ jobs, int njobs)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 2 * njobs) return;
    const FactorJob &jb = jobs[tid >> 1];
    const int par = tid & 1;
    const double qj = jb.q;
    const int64_t n = jb.n, Ls = jb.Ls;
    const int64_t m = (n - par + 1) / 2;
    float *pj = jb.phick + par * jb.nchunk;
    float4 *sj = jb.segc + par * jb.P;
    double uf_prev = 0.0, Phi = 1.0, prodU = 1.0, B = 0.0;
    for (int64_t t = 0; t < m; ++t) {
        const int64_t i = par + 2 * t;
        if (t % Ls == 0) {
            Phi = 1.0;
            prodU = 1.0;
            B = 0.0;
        }
        double den = jb.d[i] - qj;
        if (i >= 2) den -= jb.e[i - 2] * uf_prev;
        const double ip = 1.0 / den;
        const double uf = jb.e[i] * ip;
        const double lf = uf_prev;
        Phi *= -lf;
        const double kappa = ip * prodU;
        prodU *= -uf;
        B += kappa * Phi;
        jb.fac[i] = make_float4((float)ip, (float)uf, (float)lf, (float)kappa);
        if (t % kChunk == kChunk - 1) pj[t / kChunk] = (float)Phi;
        const int64_t seg = t / Ls;
        const int64_t seg_end = ((seg + 1) * Ls < m) ? (seg + 1) * Ls : m;
        if (t == seg_end - 1) sj[seg] = make_float4((float)Phi, (float)prodU, (float)B, 0.f);
        uf_prev = uf;
    }
    for (int64_t s = (m + Ls - 1) / Ls; s < jb.P; ++s) sj[s] = make_float4(1.f, 1.f, 0.f, 0.f);
}

constexpr int kDF = 12;  // ring depth (slots) of the forward kernels
constexpr int kDB = 8;   // ring depth (slots) of the backward kernels

template <int DS>
size_t rowb_smem() { return sizeof(RowBwdSmem<DS>); }
template <int DS>
size_t colb_smem() { return sizeof(ColBwdSmem<DS>); }

}  // namespace

RefineGeometry refine_geometry(int64_t n, int target_ctas)
{
    RefineGeometry g;
    g.ld = (n + 31) / 32 * 32;
    const int64_t m0 = (n + 1) / 2;
    const int64_t nblk = (n + kRC - 1) / kRC;
    g.nblk = nblk;
    g.nchunk = (m0 + kChunk - 1) / kChunk;
    // enough segments for the requested number of CTAs, each a whole number of chunks
    int64_t want = (target_ctas + nblk - 1) / nblk;
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

cudaError_t launch_row_pass(const RefPassArgs &a, int j, cudaStream_t st)
{
    const dim3 grid((unsigned)a.nitems), block(64);
    fwd_local_kernel<1, kDF><<<grid, block, 0, st>>>(a.probs, a.items, a.active, j, a.Pt, nullptr, a.ck, a.summ);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    row_bwd_kernel<kDB><<<grid, block, rowb_smem<kDB>(), st>>>(a.probs, a.items, a.active, j, a.Pt, a.A, a.C, a.ck,
                                                             a.summ);
    return cudaGetLastError();
}

cudaError_t launch_col_pass(const RefPassArgs &a, int j, bool first, cudaStream_t st, cudaEvent_t ev0,
                            cudaEvent_t ev1)
{
    const dim3 grid((unsigned)a.nitems), block(64);
    fwd_local_kernel<2, kDF><<<grid, block, 0, st>>>(a.probs, a.items, a.active, j, a.C, a.A, a.ck, a.summ);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev0 && (e = cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (first)
        col_bwd_kernel<kDB, true><<<grid, block, colb_smem<kDB>(), st>>>(a.probs, a.items, a.active, j, a.C, a.A, a.D,
                                                                        a.Pt, a.ck, a.summ);
    else
        col_bwd_kernel<kDB, false><<<grid, block, colb_smem<kDB>(), st>>>(a.probs, a.items, a.active, j, a.C, a.A,
                                                                         a.D, a.Pt, a.ck, a.summ);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev1) e = cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal);
    return e;
}

cudaError_t launch_absmax_tiles(const RefTileArgs &a, const double *F, unsigned long long *smax, cudaStream_t st)
{
    absmax_tiles_kernel<<<(unsigned)a.ntiles, dim3(32, 8), 0, st>>>(a.probs, a.tiles, F, smax);
    return cudaGetLastError();
}

cudaError_t launch_scale_in_tiles(const RefTileArgs &a, const double *F, double *Ft, float *Pt,
                                  const unsigned long long *smax, cudaStream_t st)
{
    scale_in_tiles_kernel<<<(unsigned)a.ntiles, dim3(32, 8), 0, st>>>(a.probs, a.tiles, F, Ft, Pt, smax);
    return cudaGetLastError();
}

cudaError_t launch_residual_tiles(const RefTileArgs &a, const double *Y, double *Yout, const float *Dl,
                                  const double *Ft, float *Pt, const unsigned long long *smax,
                                  unsigned long long *rmax, const int *pair_active, bool y_zero, cudaStream_t st)
{
    residual_tiles_kernel<<<(unsigned)a.ntiles, dim3(32, 8), 0, st>>>(a.probs, a.tiles, Y, Yout, Dl, Ft, Pt, smax,
                                                                      rmax, pair_active, y_zero ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_scale_out_tiles(const RefTileArgs &a, const double *Y, double *X, cudaStream_t st)
{
    scale_out_tiles_kernel<<<(unsigned)a.ntiles, dim3(32, 8), 0, st>>>(a.probs, a.tiles, Y, X);
    return cudaGetLastError();
}

cudaError_t launch_factors32(const FactorJob *jobs, int njobs, cudaStream_t st)
{
    const int threads = 2 * njobs;
    factor32_kernel<<<(threads + 127) / 128, 128, 0, st>>>(jobs, njobs);
    return cudaGetLastError();
}

}  // namespace fps
