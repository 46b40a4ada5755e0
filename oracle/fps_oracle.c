/*
 * fps_oracle.c -- plain, slow, CPU reference ("oracle") for the spectral Poisson
 * ADI solver of Fortunato & Townsend, "Fast Poisson solvers for spectral methods"
 * (arXiv 1710.11259).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the GPU
 * library: only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA path, and the CUDA path never calls it.
 *
 * Everything is written for clarity: arithmetic in `real` (double, or long double
 * in the rounding-check build), textbook Thomas elimination with divisions, the
 * ADI steps in the order of Algorithm 2.  OpenMP only distributes independent
 * right-hand sides of one banded solve over threads; it does not change the
 * arithmetic of any single system.
 *
 * Readings of the paper taken here (each is argued in the design notes):
 *   R1  Algorithm 2's first half-step is used in the sign-consistent form
 *       X_{j+1/2}(B - p_j I) = (A - p_j I) X_j - F; as printed it produces the
 *       negated half-iterate (the whole iterates are the same either way).
 *   R2  The symmetrised unknown of (3.9) is recovered by X = D_s Y D_s with
 *       D_s = |D|^{-1/2}; that is the reading consistent with the printed
 *       right-hand side D_s^{-1}(D^{-1} F D^{-1})D_s^{-1}.
 *   R3  The number of iterations is (2.9), J = ceil(log(16 gamma) log(4/eps)/pi^2),
 *       with the cross-ratio gamma of the intervals (as in Appendix A); the
 *       simplified count printed for the square in Sec. 3.3 is not used.
 *   R4  The spectral intervals are those of Lemma B.2: sigma(A~) in
 *       [-1, -1/(30 n^4)], sigma(B~) = -sigma(A~).
 */
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

static const real ORC_PI = (real)3.14159265358979323846264338327950288L;

/* ------------------------------------------------------------------------- */
/* Section 3.2, eq. (3.7): multiplication by (1 - x^2) in the normalised       */
/* ultraspherical basis C~^(3/2), and D_jj = -(j(j+3)+2).                      */
/* ------------------------------------------------------------------------- */

/* M_{j,j} = 2(j+1)(j+2) / ((2j+1)(2j+5)) */
static real M_diag(long j)
{
    real J = (real)j;
    return 2 * (J + 1) * (J + 2) / ((2 * J + 1) * (2 * J + 5));
}

/* M_{j,j+2} = -1/((2j+3)(2j+5)) * sqrt( (j+4)!/j! * (2j+3)/(2j+7) ),
 * with (j+4)!/j! = (j+1)(j+2)(j+3)(j+4).  M_{j,j+1} = 0. */
static real M_off2(long j)
{
    real J = (real)j;
    real fact_ratio = (J + 1) * (J + 2) * (J + 3) * (J + 4);
    return -sqrt(fact_ratio * (2 * J + 3) / (2 * J + 7)) / ((2 * J + 3) * (2 * J + 5));
}

/* D_{j,j} = -(j(j+3)+2), eq. (3.6) */
static real D_diag(long j)
{
    real J = (real)j;
    return -(J * (J + 3) + 2);
}

/* Exported for the quadrature pin: the first n diagonal entries of M and the
 * n-2 entries M_{j,j+2}. */
void orc_M_bands(long n, double *diag, double *off2)
{
    for (long j = 0; j < n; ++j) diag[j] = (double)M_diag(j);
    for (long j = 0; j + 2 < n; ++j) off2[j] = (double)M_off2(j);
}

/* ------------------------------------------------------------------------- */
/* Section 3.3, eq. (3.8)-(3.9): A = D^{-1} M, A~ = D_s^{-1} A D_s symmetric.   */
/* A~ is pentadiagonal with zero first off-diagonals, i.e. a "stride-2"        */
/* symmetric tridiagonal: diagonal ad[j], coupling ae[j] between j and j+2.    */
/* ------------------------------------------------------------------------- */

/* D_s such that D_s^{-1} A D_s is symmetric: (D_s)_jj = |D_jj|^{-1/2}. */
static real Ds_diag(long j) { return 1 / sqrt(-D_diag(j)); }

static void square_bands(long n, real *ad, real *ae)
{
    for (long j = 0; j < n; ++j) {
        real A_jj = M_diag(j) / D_diag(j);                 /* (D^{-1} M)_{jj} */
        ad[j] = A_jj;                                       /* similarity keeps the diagonal */
    }
    for (long j = 0; j + 2 < n; ++j) {
        real A_j_j2 = M_off2(j) / D_diag(j);               /* (D^{-1} M)_{j,j+2} */
        ae[j] = A_j_j2 * Ds_diag(j + 2) / Ds_diag(j);       /* (D_s^{-1} A D_s)_{j,j+2} */
    }
}

void orc_square_bands(long n, double *ad, double *ae)
{
    real *d = malloc(sizeof(real) * (size_t)n), *e = malloc(sizeof(real) * (size_t)(n > 2 ? n : 1));
    square_bands(n, d, e);
    for (long j = 0; j < n; ++j) ad[j] = (double)d[j];
    for (long j = 0; j + 2 < n; ++j) ae[j] = (double)e[j];
    free(d);
    free(e);
}

/* ------------------------------------------------------------------------- */
/* Elliptic functions for Theorem 2.1 / Appendix A.                            */
/* Parameter convention: m = kappa^2 (MATLAB's ellipke/ellipj convention).      */
/* ------------------------------------------------------------------------- */

/* Complete elliptic integral of the first kind via the arithmetic-geometric
 * mean, K(m) = pi / (2 AGM(1, sqrt(1-m)))  (DLMF 19.8.5). */
static real ellip_K(real m)
{
    real a = 1, b = sqrt(1 - m);
    for (int it = 0; it < 64 && fabs(a - b) > 4 * (real)1e-19 * a; ++it) {
        real an = (a + b) / 2;
        b = sqrt(a * b);
        a = an;
    }
    return ORC_PI / (2 * a);
}

/* Jacobi dn(u | m) by the descending Landen / AGM scheme (DLMF 22.20(ii)):
 * a_0 = 1, b_0 = sqrt(1-m), c_0 = sqrt(m); a_{k+1} = (a_k+b_k)/2,
 * b_{k+1} = sqrt(a_k b_k), c_{k+1} = (a_k-b_k)/2 until c_N ~ 0;
 * phi_N = 2^N a_N u, phi_{k-1} = (phi_k + asin(c_k sin(phi_k)/a_k))/2;
 * dn = cos(phi_0)/cos(phi_1 - phi_0). */
static real ellip_dn(real u, real m)
{
    real a[80], c[80];
    real b = sqrt(1 - m);
    a[0] = 1;
    c[0] = sqrt(m);
    int N = 0;
    while (N < 70 && fabs(c[N]) > (real)1e-18) {
        a[N + 1] = (a[N] + b) / 2;
        c[N + 1] = (a[N] - b) / 2;
        b = sqrt(a[N] * b);
        ++N;
    }
    if (N == 0) return 1; /* m == 0: dn == 1 */
    real phi = ldexp(a[N] * u, N);
    real phi_prev = phi;
    for (int k = N; k >= 1; --k) {
        phi_prev = phi;
        phi = (phi + asin(c[k] * sin(phi) / a[k])) / 2;
    }
    /* phi now holds phi_0 and phi_prev holds phi_1 */
    return cos(phi) / cos(phi_prev - phi);
}

/* ------------------------------------------------------------------------- */
/* Eq. (2.9) and Appendix A: iteration count and Zolotarev shifts for          */
/* A X - X B = F with sigma(A) in [a,b], sigma(B) in [c,d], a < b < c < d.     */
/* ------------------------------------------------------------------------- */

/* gamma = |c-a||d-b| / (|c-b||d-a|)  (Theorem 2.1) */
static real cross_ratio(real a, real b, real c, real d)
{
    return fabs(c - a) * fabs(d - b) / (fabs(c - b) * fabs(d - a));
}

/* J = ceil( log(16 gamma) log(4/eps) / pi^2 )  (2.9) */
int orc_adi_iterations(double a, double b, double c, double d, double tol)
{
    real gam = cross_ratio(a, b, c, d);
    real J = ceil(log(16 * gam) * log(4 / (real)tol) / (ORC_PI * ORC_PI));
    return (int)J;
}

/* Shifts (2.4): p_j = T(-alpha dn[(2j+1)K/(2J), kappa]), q_j = T(+alpha dn[...]),
 * kappa = sqrt(1 - 1/alpha^2), alpha = -1 + 2 gamma + 2 sqrt(gamma^2 - gamma),
 * T the Moebius map taking (-alpha, -1, 1, alpha) to (a, b, c, d).
 * Writes J values into p and q; returns J. */
int orc_adi_shifts(double a_, double b_, double c_, double d_, double tol, int J, double *p, double *q)
{
    real a = a_, b = b_, c = c_, d = d_;
    real gam = cross_ratio(a, b, c, d);
    real alp = -1 + 2 * gam + 2 * sqrt(gam * gam - gam);

    /* Moebius T(z) = (TA z + TB)/(TC z + TD) with T(1)=c, T(-1)=b, T(-alp)=a.
     * From T(1)=c and T(-1)=b: 2 TA = (c+b) TC + (c-b) TD, 2 TB = (c-b) TC + (c+b) TD;
     * T(-alp)=a then fixes TC : TD up to scale. */
    real TC = (c + b) - alp * (c - b) - 2 * a;
    real TD = alp * (c + b) - (c - b) - 2 * a * alp;
    real TA = ((c + b) * TC + (c - b) * TD) / 2;
    real TB = ((c - b) * TC + (c + b) * TD) / 2;

    for (int j = 0; j < J; ++j) {
        real dn;
        if (alp < (real)1e7) {
            real m = 1 - 1 / (alp * alp);
            real K = ellip_K(m);
            real u = ((real)j + (real)0.5) * K / (real)J;
            dn = ellip_dn(u, m);
        } else {
            /* kappa' = 1/alp is tiny: leading terms of the expansions about m = 1,
             * K = log(4/kappa') + (kappa'^2/4)(log(4/kappa') - 1)   (DLMF 19.12.1),
             * dn(u) = sech u + (kappa'^2/4)(sinh u cosh u + u) tanh u sech u (DLMF 22.10.ii). */
            real m1 = 1 / (alp * alp);
            real L4 = log(4 * alp);
            real K = L4 + m1 * (L4 - 1) / 4;
            real u = ((real)j + (real)0.5) * K / (real)J;
            real sech = 1 / cosh(u);
            dn = sech + m1 / 4 * (sinh(u) * cosh(u) + u) * tanh(u) * sech;
        }
        real zp = -alp * dn, zq = alp * dn;
        p[j] = (double)((TA * zp + TB) / (TC * zp + TD));
        q[j] = (double)((TA * zq + TB) / (TC * zq + TD));
    }
    return J;
}

/* ------------------------------------------------------------------------- */
/* Banded pieces of Algorithm 2.  A "stride-s tridiagonal" symmetric matrix T  */
/* has diagonal td[i] and off-diagonal tu[i] = T[i][i+s] = T[i+s][i]; indices  */
/* of different residue mod s never couple, so a solve splits into s           */
/* independent tridiagonal systems (App. B, P3).  s = 1 for the finite-        */
/* difference matrix K of (1.2), s = 2 for A~ of (3.9).                        */
/* ------------------------------------------------------------------------- */

typedef struct {
    long n;
    int s;
    const real *td, *tu;
} band_t;

/* Thomas elimination of (T - sigma I): for each index i,
 *   den[i] = (t_ii - sigma) - sub_i * cp[i-s],   cp[i] = tu[i] / den[i],
 * with sub_i = tu[i-s] (zero for the first index of each residue class).
 * The factors depend only on the matrix, so they are shared by every
 * right-hand side.  (Thomas algorithm, cited by the paper for P3.) */
static void thomas_factor(const band_t *T, real sigma, real *cp, real *den)
{
    long n = T->n;
    int s = T->s;
    for (long i = 0; i < n; ++i) {
        real diag = T->td[i] - sigma;
        if (i >= s) {
            real sub = T->tu[i - s];
            den[i] = diag - sub * cp[i - s];
        } else {
            den[i] = diag;
        }
        cp[i] = (i + s < n) ? T->tu[i] / den[i] : 0;
    }
}

/* X = (T - sigma I)^{-1} R acting on columns (left multiplication).  R and X
 * are n x ncol row-major; X may alias R.  Forward sweep
 * dp[i] = (r[i] - sub_i dp[i-s]) / den[i], backward x[i] = dp[i] - cp[i] x[i+s]. */
static void solve_left(const band_t *T, real sigma, long ncol, const real *R, real *X, real *cp, real *den)
{
    long n = T->n;
    int s = T->s;
    thomas_factor(T, sigma, cp, den);
    /* Each thread owns a contiguous range of columns and walks the rows in the
     * order of the recurrence, so that memory is read row by row. */
#pragma omp parallel
    {
        long c0 = 0, c1 = ncol;
#ifdef _OPENMP
        int nt = omp_get_num_threads(), id = omp_get_thread_num();
        c0 = ncol * id / nt;
        c1 = ncol * (id + 1) / nt;
#endif
        for (long i = 0; i < n; ++i)
            for (long c = c0; c < c1; ++c) {
                real r = R[i * ncol + c];
                if (i >= s) r -= T->tu[i - s] * X[(i - s) * ncol + c];
                X[i * ncol + c] = r / den[i];
            }
        for (long i = n - 1; i >= 0; --i)
            if (i + s < n)
                for (long c = c0; c < c1; ++c) X[i * ncol + c] -= cp[i] * X[(i + s) * ncol + c];
    }
}

/* X = R (T - sigma I)^{-1} acting on rows (right multiplication; T symmetric so
 * each row x solves (T - sigma I) x^T = r^T).  R, X are nrow x n row-major. */
static void solve_right(const band_t *T, real sigma, long nrow, const real *R, real *X, real *cp, real *den)
{
    long n = T->n;
    int s = T->s;
    thomas_factor(T, sigma, cp, den);
#pragma omp parallel for schedule(static)
    for (long r = 0; r < nrow; ++r) {
        const real *rr = R + r * n;
        real *xr = X + r * n;
        for (long i = 0; i < n; ++i) {
            real v = rr[i];
            if (i >= s) v -= T->tu[i - s] * xr[i - s];
            xr[i] = v / den[i];
        }
        for (long i = n - 1; i >= 0; --i) {
            if (i + s < n) xr[i] -= cp[i] * xr[i + s];
        }
    }
}

/* Y = (T - sigma I) X  (left multiplication, acts along columns). */
static void mul_left(const band_t *T, real sigma, long ncol, const real *X, real *Y)
{
    long n = T->n;
    int s = T->s;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        for (long c = 0; c < ncol; ++c) {
            real v = (T->td[i] - sigma) * X[i * ncol + c];
            if (i >= s) v += T->tu[i - s] * X[(i - s) * ncol + c];
            if (i + s < n) v += T->tu[i] * X[(i + s) * ncol + c];
            Y[i * ncol + c] = v;
        }
    }
}

/* Y = X (T - sigma I)  (right multiplication, acts along rows; T symmetric). */
static void mul_right(const band_t *T, real sigma, long nrow, const real *X, real *Y)
{
    long n = T->n;
    int s = T->s;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < nrow; ++r) {
        const real *xr = X + r * n;
        real *yr = Y + r * n;
        for (long k = 0; k < n; ++k) {
            real v = (T->td[k] - sigma) * xr[k];
            if (k >= s) v += T->tu[k - s] * xr[k - s];
            if (k + s < n) v += T->tu[k] * xr[k + s];
            yr[k] = v;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2: ADI for A X - X B = F (A, B symmetric stride-s tridiagonals,   */
/* both n x n), J iterations with shifts p_j, q_j, X_0 = 0.  Reading R1:        */
/*   X_{j+1/2} (B - p_j I) = (A - p_j I) X_j - F                               */
/*   (A - q_j I) X_{j+1}   = F + X_{j+1/2} (B - q_j I)                          */
/* ------------------------------------------------------------------------- */
static void adi_sylvester(const band_t *A, const band_t *B, const real *F, int J, const real *p, const real *q,
                          real *X)
{
    long n = A->n;
    size_t nn = (size_t)n * (size_t)n;
    real *Xh = malloc(sizeof(real) * nn);
    real *W = malloc(sizeof(real) * nn);
    real *cp = malloc(sizeof(real) * (size_t)n), *den = malloc(sizeof(real) * (size_t)n);
    memset(X, 0, sizeof(real) * nn);
    for (int j = 0; j < J; ++j) {
        /* first half-step: W = (A - p_j I) X_j - F, then X_{j+1/2} = W (B - p_j I)^{-1} */
        mul_left(A, p[j], n, X, W);
#pragma omp parallel for schedule(static)
        for (size_t t = 0; t < nn; ++t) W[t] -= F[t];
        solve_right(B, p[j], n, W, Xh, cp, den);
        /* second half-step: W = F + X_{j+1/2} (B - q_j I), then X_{j+1} = (A - q_j I)^{-1} W */
        mul_right(B, q[j], n, Xh, W);
#pragma omp parallel for schedule(static)
        for (size_t t = 0; t < nn; ++t) W[t] += F[t];
        solve_left(A, q[j], n, W, X, cp, den);
    }
    free(Xh);
    free(W);
    free(cp);
    free(den);
}

/* Exported generic driver (used with the finite-difference matrix K of (1.2)
 * as a closed-form check of the ADI machinery).  Bands in double; J shifts. */
void orc_adi_sylvester(long n, int s, const double *Ad, const double *Ae, const double *Bd, const double *Be,
                       const double *F, int J, const double *p, const double *q, double *X)
{
    size_t nn = (size_t)n * (size_t)n;
    long ne = n > s ? n - s : 1;
    real *ad = malloc(sizeof(real) * (size_t)n), *ae = malloc(sizeof(real) * (size_t)ne);
    real *bd = malloc(sizeof(real) * (size_t)n), *be = malloc(sizeof(real) * (size_t)ne);
    real *pr = malloc(sizeof(real) * (size_t)(J > 0 ? J : 1)), *qr = malloc(sizeof(real) * (size_t)(J > 0 ? J : 1));
    real *Fr = malloc(sizeof(real) * nn), *Xr = malloc(sizeof(real) * nn);
    for (long i = 0; i < n; ++i) { ad[i] = Ad[i]; bd[i] = Bd[i]; }
    for (long i = 0; i + s < n; ++i) { ae[i] = Ae[i]; be[i] = Be[i]; }
    for (int j = 0; j < J; ++j) { pr[j] = p[j]; qr[j] = q[j]; }
    for (size_t t = 0; t < nn; ++t) Fr[t] = F[t];
    band_t A = {n, s, ad, ae}, B = {n, s, bd, be};
    adi_sylvester(&A, &B, Fr, J, pr, qr, Xr);
    for (size_t t = 0; t < nn; ++t) X[t] = (double)Xr[t];
    free(ad); free(ae); free(bd); free(be); free(pr); free(qr); free(Fr); free(Xr);
}

/* ------------------------------------------------------------------------- */
/* A tighter spectral interval than Lemma B.2 (used only when asked for).      */
/* The eigenvalues of A~ are those of its two decoupled tridiagonals (even and  */
/* odd indices, App. B).  By Sylvester's law of inertia the number of           */
/* eigenvalues below x equals the number of negative pivots of the LDL^T        */
/* factorisation of T - x I, whose pivots follow the Sturm recurrence            */
/*     u_0 = t_00 - x,   u_k = (t_kk - x) - t_{k,k-1}^2 / u_{k-1}.               */
/* Bisection on that count brackets the extreme eigenvalues; the returned        */
/* interval is padded (half the smallest magnitude, 1.01 times the largest,      */
/* capped at Lemma B.2's 1) so that it contains the spectrum with margin.        */
/* ------------------------------------------------------------------------- */
static long negative_pivots(long n, const double *ad, const double *ae, double x)
{
    long neg = 0;
    for (int par = 0; par < 2; ++par) {
        double u = 0.0;
        for (long i = par; i < n; i += 2) {
            double next = ad[i] - x;
            if (i >= 2) next -= ae[i - 2] * ae[i - 2] / (u != 0.0 ? u : 1e-300);
            if (next == 0.0) next = -1e-300;
            neg += next < 0.0;
            u = next;
        }
    }
    return neg;
}

void orc_tight_interval(long n, double *lo, double *hi)
{
    double *ad = malloc(sizeof(double) * (size_t)n), *ae = malloc(sizeof(double) * (size_t)(n > 2 ? n : 1));
    orc_square_bands(n, ad, ae);
    /* most negative eigenvalue: count(x) == 0 means no eigenvalue below x */
    double left = -1.0, right = 0.0;
    for (int it = 0; it < 100; ++it) {
        double mid = 0.5 * (left + right);
        if (negative_pivots(n, ad, ae, mid) == 0) left = mid;
        else right = mid;
    }
    /* eigenvalue closest to zero, on a logarithmic scale between eps/8 and 1:
     * count(-exp(t)) == n means every eigenvalue lies below -exp(t) */
    double nd = (double)n;
    double tl = log(1.0 / (240.0 * nd * nd * nd * nd)), tr = 0.0;
    for (int it = 0; it < 100; ++it) {
        double tm = 0.5 * (tl + tr);
        if (negative_pivots(n, ad, ae, -exp(tm)) == n) tl = tm;
        else tr = tm;
    }
    *lo = 0.5 * exp(tl);
    *hi = 1.01 * (-left) < 1.0 ? 1.01 * (-left) : 1.0;
    free(ad);
    free(ae);
}

/* ------------------------------------------------------------------------- */
/* Section 3 end to end (Table 3.1, steps 2-3) for  M X D^T + D X M^T = F.     */
/*   1. A~ = D_s^{-1} D^{-1} M D_s, B~ = -A~                     (3.8)-(3.9)   */
/*   2. F~ = D_s^{-1} (D^{-1} F D^{-1}) D_s^{-1}                 (3.9)         */
/*   3. intervals [a,b] = [-1, -1/(30 n^4)], [c,d] = [1/(30 n^4), 1] (Lemma B.2)*/
/*   4. J from (2.9), shifts from (2.4) / Appendix A                           */
/*   5. Algorithm 2 on A~ Y - Y B~ = F~                                         */
/*   6. X = D_s Y D_s                                            (reading R2)  */
/* F, X: n x n row-major, X_ij pairs C~_i(y) with C~_j(x).  Returns J.         */
/* ------------------------------------------------------------------------- */
static int poisson_square(long n, double tol, const real *F, real *X, double *shifts_q_out, int jmax, int tight,
                          double kx, double ky)
{
    size_t nn = (size_t)n * (size_t)n;
    long ne = n > 2 ? n - 2 : 1;
    real *ad = malloc(sizeof(real) * (size_t)n), *ae = malloc(sizeof(real) * (size_t)ne);
    real *bd = malloc(sizeof(real) * (size_t)n), *be = malloc(sizeof(real) * (size_t)ne);
    square_bands(n, ad, ae);
    /* rectangle (Sec. 3 on [x0,x1] x [y0,y1]): kx A~ Y + ky Y A~ = F~ with k = (2/length)^2;
     * A = kx A~ acts on the row (y) index, B = -ky A~ on the column (x) index */
    for (long j = 0; j < n; ++j) { bd[j] = -ky * ad[j]; ad[j] *= kx; }
    for (long j = 0; j + 2 < n; ++j) { be[j] = -ky * ae[j]; ae[j] *= kx; }

    real *Ft = malloc(sizeof(real) * nn), *Y = malloc(sizeof(real) * nn);
    for (long i = 0; i < n; ++i)
        for (long k = 0; k < n; ++k) {
            real g = F[i * n + k] / (D_diag(i) * D_diag(k)); /* D^{-1} F D^{-1} */
            Ft[i * n + k] = g / (Ds_diag(i) * Ds_diag(k));    /* D_s^{-1} ( . ) D_s^{-1} */
        }

    double nd = (double)n;
    double eps_n = 1.0 / (30.0 * nd * nd * nd * nd);
    double a = -1.0, b = -eps_n, c = eps_n, d = 1.0;
    if (tight) {
        double tlo, thi;
        orc_tight_interval(n, &tlo, &thi);
        a = -thi;
        b = -tlo;
        c = tlo;
        d = thi;
    }
    a *= kx;
    b *= kx;
    c *= ky;
    d *= ky;
    int J = orc_adi_iterations(a, b, c, d, tol);
    double *p = malloc(sizeof(double) * (size_t)J), *q = malloc(sizeof(double) * (size_t)J);
    orc_adi_shifts(a, b, c, d, tol, J, p, q);
    real *pr = malloc(sizeof(real) * (size_t)J), *qr = malloc(sizeof(real) * (size_t)J);
    for (int j = 0; j < J; ++j) { pr[j] = p[j]; qr[j] = q[j]; }
    if (shifts_q_out)
        for (int j = 0; j < J; ++j) shifts_q_out[j] = q[j];

    band_t A = {n, 2, ad, ae}, B = {n, 2, bd, be};
    adi_sylvester(&A, &B, Ft, (jmax > 0 && jmax < J) ? jmax : J, pr, qr, Y);

    for (long i = 0; i < n; ++i)
        for (long k = 0; k < n; ++k) X[i * n + k] = Ds_diag(i) * Y[i * n + k] * Ds_diag(k);

    free(ad); free(ae); free(bd); free(be); free(Ft); free(Y); free(p); free(q); free(pr); free(qr);
    return J;
}

int orc_poisson_square(long n, double tol, const double *F, double *X)
{
    size_t nn = (size_t)n * (size_t)n;
    real *Fr = malloc(sizeof(real) * nn), *Xr = malloc(sizeof(real) * nn);
    for (size_t t = 0; t < nn; ++t) Fr[t] = F[t];
    int J = poisson_square(n, tol, Fr, Xr, NULL, 0, 0, 1.0, 1.0);
    for (size_t t = 0; t < nn; ++t) X[t] = (double)Xr[t];
    free(Fr);
    free(Xr);
    return J;
}

/* Poisson on the rectangle [x0, x1] x [y0, y1] with homogeneous Dirichlet data: the
 * affine map to [-1,1]^2 scales the second derivatives by kx = (2/(x1-x0))^2 and
 * ky = (2/(y1-y0))^2, so (3.6) becomes kx M X D^T + ky D X M^T = F; in the variables
 * of (3.9), kx A~ Y + ky Y A~ = F~, a Sylvester equation whose two spectral intervals
 * differ (non-symmetric shifts from App. A's general Moebius path). */
int orc_poisson_rectangle(long n, double kx, double ky, double tol, int tight, const double *F, double *X)
{
    size_t nn = (size_t)n * (size_t)n;
    real *Fr = malloc(sizeof(real) * nn), *Xr = malloc(sizeof(real) * nn);
    for (size_t t = 0; t < nn; ++t) Fr[t] = F[t];
    int J = poisson_square(n, tol, Fr, Xr, NULL, 0, tight, kx, ky);
    for (size_t t = 0; t < nn; ++t) X[t] = (double)Xr[t];
    free(Fr);
    free(Xr);
    return J;
}

/* The same solve with the shifts of the tight interval (orc_tight_interval). */
int orc_poisson_square_tight(long n, double tol, const double *F, double *X)
{
    size_t nn = (size_t)n * (size_t)n;
    real *Fr = malloc(sizeof(real) * nn), *Xr = malloc(sizeof(real) * nn);
    for (size_t t = 0; t < nn; ++t) Fr[t] = F[t];
    int J = poisson_square(n, tol, Fr, Xr, NULL, 0, 1, 1.0, 1.0);
    for (size_t t = 0; t < nn; ++t) X[t] = (double)Xr[t];
    free(Fr);
    free(Xr);
    return J;
}

/* The same pipeline stopped after at most jmax ADI iterations (a bounded sample
 * of the full solve, used to time the oracle on large problems).  Returns the
 * full J of (2.9). */
int orc_poisson_square_partial(long n, double tol, int jmax, const double *F, double *X)
{
    size_t nn = (size_t)n * (size_t)n;
    real *Fr = malloc(sizeof(real) * nn), *Xr = malloc(sizeof(real) * nn);
    for (size_t t = 0; t < nn; ++t) Fr[t] = F[t];
    int J = poisson_square(n, tol, Fr, Xr, NULL, jmax, 0, 1.0, 1.0);
    for (size_t t = 0; t < nn; ++t) X[t] = (double)Xr[t];
    free(Fr);
    free(Xr);
    return J;
}


/* ------------------------------------------------------------------------- */
/* Section 5: the cube.  (D_xx + D_yy + D_zz) vec(X) = vec(F), eq. (5.2).      */
/* In the symmetrised variables of (3.9) applied on every mode,                 */
/*     (T_01 + T_02 + T_12) Y = G,   G = -F / sqrt(E_i E_j E_k),                */
/*     X = Y / sqrt(E_i E_j E_k),                                               */
/* where T_ab applies A~ on modes a and b of the n x n x n tensor (row-major,   */
/* mode 0 = i, mode 1 = j, mode 2 = k).  The sign of G comes from the three     */
/* factors D^{-1} = -E^{-1} (reading R11).  Nested ADI of Sec. 5 (readings      */
/* R1, R12): outer split (5.3)-(5.4) H = T_01 + T_02 | V = T_12; middle split   */
/* (5.5)-(5.6) of H + s into (T_01 + s/2) | (T_02 + s/2); inner slice Stein     */
/* equations (5.7)-(5.9) (A~ Z A~ + c Z = R on two modes) by ADI on             */
/* (c A~^{-1}) Z - Z (-A~) = A~^{-1} R.                                        */
/* ------------------------------------------------------------------------- */

typedef struct {
    long n;
    const real *d, *e; /* A~ bands (stride 2), e zero-padded to n */
} cube_t;

static long mode_stride(long n, int mode) { return mode == 0 ? n * n : (mode == 1 ? n : 1); }

/* Y = (alpha A~ + beta I) X along `mode` (every line of the tensor in that mode). */
static void t_apply(const cube_t *C, int mode, real alpha, real beta, const real *X, real *Y)
{
    long n = C->n, st = mode_stride(n, mode);
    long nn = n * n;
#pragma omp parallel for schedule(static)
    for (long line = 0; line < nn; ++line) {
        /* the two other indices of this line */
        long o;
        if (mode == 0) o = line;                          /* (j, k) = line */
        else if (mode == 1) o = (line / n) * n * n + (line % n); /* (i, k) */
        else o = line * n;                                /* (i, j) */
        for (long t = 0; t < n; ++t) {
            real v = (alpha * C->d[t] + beta) * X[o + t * st];
            if (t >= 2) v += alpha * C->e[t - 2] * X[o + (t - 2) * st];
            if (t + 2 < n) v += alpha * C->e[t] * X[o + (t + 2) * st];
            Y[o + t * st] = v;
        }
    }
}

/* X = (alpha A~ + beta I)^{-1} R along `mode` (Thomas on the even and odd index
 * sets of every line, App. B).  X may alias R. */
static void t_solve(const cube_t *C, int mode, real alpha, real beta, const real *R, real *X)
{
    long n = C->n, st = mode_stride(n, mode);
    long nn = n * n;
    real *cp = malloc(sizeof(real) * (size_t)n), *den = malloc(sizeof(real) * (size_t)n);
    for (long t = 0; t < n; ++t) {
        real diag = alpha * C->d[t] + beta;
        den[t] = (t >= 2) ? diag - alpha * C->e[t - 2] * cp[t - 2] : diag;
        cp[t] = (t + 2 < n) ? alpha * C->e[t] / den[t] : 0;
    }
#pragma omp parallel for schedule(static)
    for (long line = 0; line < nn; ++line) {
        long o;
        if (mode == 0) o = line;
        else if (mode == 1) o = (line / n) * n * n + (line % n);
        else o = line * n;
        for (long t = 0; t < n; ++t) {
            real v = R[o + t * st];
            if (t >= 2) v -= alpha * C->e[t - 2] * X[o + (t - 2) * st];
            X[o + t * st] = v / den[t];
        }
        for (long t = n - 1; t >= 0; --t)
            if (t + 2 < n) X[o + t * st] -= cp[t] * X[o + (t + 2) * st];
    }
    free(cp);
    free(den);
}

static void t_axpby(long N, real a, const real *X, real b, const real *Y, real *Z)
{
#pragma omp parallel for schedule(static)
    for (long t = 0; t < N; ++t) Z[t] = a * X[t] + b * Y[t];
}

/* Z = (T_ab + c)^{-1} R, c > 0, i.e. the slice Stein equations A~_a Z A~_b + c Z = R
 * of (5.7).  As in (5.8)-(5.9), a Sylvester equation for the slice:
 * A~_a Z - Z (-c A~_b^{-1}) = R A~_b^{-1}, sigma(A~) in [-1, -eps] and
 * sigma(-c A~^{-1}) in [c, c/eps]; Algorithm 2 in the sign-consistent form (R1),
 * the first half-step multiplied through by A~_b on the right:
 *   Z_h = [ R - (A~_a - p) Z A~_b ] (c + p A~_b)^{-1}
 *   (A~_a - q) Z+ = (R - c Z_h) A~_b^{-1} - q Z_h                                */
static int stein_solve(const cube_t *C, int ma, int mb, real c, real eps, double tol, const real *R, real *Z,
                       real *W1, real *W2)
{
    long N = C->n * C->n * C->n;
    double a = -1.0, b = -(double)eps, cc = (double)c, d = (double)(c / eps);
    int J = orc_adi_iterations(a, b, cc, d, tol);
    double *p = malloc(sizeof(double) * (size_t)J), *q = malloc(sizeof(double) * (size_t)J);
    orc_adi_shifts(a, b, cc, d, tol, J, p, q);
    memset(Z, 0, sizeof(real) * (size_t)N);
    for (int l = 0; l < J; ++l) {
        real pl = p[l], ql = q[l];
        t_apply(C, mb, 1, 0, Z, W1);              /* Z A~_b */
        t_apply(C, ma, 1, -pl, W1, W2);           /* (A~_a - p) ( . ) */
        t_axpby(N, 1, R, -1, W2, W1);             /* R - ( . ) */
        t_solve(C, mb, pl, c, W1, W2);            /* ( . ) (c + p A~_b)^{-1}: Z_h in W2 */
        t_axpby(N, 1, R, -c, W2, W1);             /* R - c Z_h */
        t_solve(C, mb, 1, 0, W1, W1);             /* ( . ) A~_b^{-1} */
        t_axpby(N, 1, W1, -ql, W2, W1);           /* ... - q Z_h */
        t_solve(C, ma, 1, -ql, W1, Z);            /* (A~_a - q)^{-1} */
    }
    free(p);
    free(q);
    return J;
}

/* Y = (T_01 + T_02 + s)^{-1} R, s > 0 (middle ADI, (5.5)-(5.6)): A' = T_01 + s/2,
 * B' = T_02 + s/2 with spectra in [eps^2 + s/2, 1 + s/2]; shifts a_m there:
 *   (B' + a) W_h = R - (A' - a) W,     (A' + a) W+ = R - (B' - a) W_h           */
static long h_solve(const cube_t *C, real s, real eps, double tol_mid, double tol_in, const real *R, real *Y,
                    real *Wh, real *T1, real *T2, real *S1, real *S2)
{
    long N = C->n * C->n * C->n;
    double lo = (double)(eps * eps + s / 2), hi = (double)(1 + s / 2);
    int J = orc_adi_iterations(-hi, -lo, lo, hi, tol_mid);
    double *p = malloc(sizeof(double) * (size_t)J), *q = malloc(sizeof(double) * (size_t)J);
    orc_adi_shifts(-hi, -lo, lo, hi, tol_mid, J, p, q);
    long inner = 0;
    memset(Y, 0, sizeof(real) * (size_t)N);
    for (int m = 0; m < J; ++m) {
        real am = q[m]; /* in [lo, hi] */
        /* T1 = R - (T_01 + s/2 - a) Y */
        t_apply(C, 0, 1, 0, Y, T1);
        t_apply(C, 1, 1, 0, T1, T2);
        t_axpby(N, 1, R, -1, T2, T1);
        t_axpby(N, 1, T1, -(s / 2 - am), Y, T1);
        inner += stein_solve(C, 0, 2, s / 2 + am, eps, tol_in, T1, Wh, S1, S2);
        /* T1 = R - (T_02 + s/2 - a) Wh */
        t_apply(C, 0, 1, 0, Wh, T1);
        t_apply(C, 2, 1, 0, T1, T2);
        t_axpby(N, 1, R, -1, T2, T1);
        t_axpby(N, 1, T1, -(s / 2 - am), Wh, T1);
        inner += stein_solve(C, 0, 1, s / 2 + am, eps, tol_in, T1, Y, S1, S2);
    }
    free(p);
    free(q);
    return inner;
}

/* Outer ADI (5.3)-(5.4) on H Y + V Y = G with H = T_01 + T_02 (sigma in [2 eps^2, 2])
 * and V = T_12 (sigma in [eps^2, 1]), as A Y - Y B with A = H, B = -V:
 *   (V + p) Y_h = G - (H - p) Y,     (H - q) Y+ = G - (V + q) Y_h,
 * p in [2 eps^2, 2], q in [-1, -eps^2] (Appendix A with the roles of the two
 * intervals exchanged to keep a < b < c < d). */
static long cube_adi(const cube_t *C, real eps, double tol, double tol_mid, double tol_in, const real *G, real *Y,
                     int *Jout)
{
    long N = C->n * C->n * C->n;
    size_t bytes = sizeof(real) * (size_t)N;
    real *Yh = malloc(bytes), *T1 = malloc(bytes), *T2 = malloc(bytes), *Wh = malloc(bytes);
    real *H1 = malloc(bytes), *H2 = malloc(bytes), *S1 = malloc(bytes), *S2 = malloc(bytes);
    double e2 = (double)(eps * eps);
    int J = orc_adi_iterations(-1.0, -e2, 2 * e2, 2.0, tol);
    double *pp = malloc(sizeof(double) * (size_t)J), *qq = malloc(sizeof(double) * (size_t)J);
    orc_adi_shifts(-1.0, -e2, 2 * e2, 2.0, tol, J, pp, qq);
    long inner = 0;
    memset(Y, 0, bytes);
    for (int j = 0; j < J; ++j) {
        real p = qq[j], q = pp[j]; /* p in sigma(H)'s interval, q in sigma(-V)'s */
        /* T1 = G - (H - p) Y */
        t_apply(C, 0, 1, 0, Y, T1);
        t_apply(C, 1, 1, 0, T1, T2);   /* T_01 Y */
        t_apply(C, 2, 1, 0, T1, H1);   /* T_02 Y */
        t_axpby(N, 1, T2, 1, H1, T2);
        t_axpby(N, 1, G, -1, T2, T1);
        t_axpby(N, 1, T1, p, Y, T1);
        inner += stein_solve(C, 1, 2, p, eps, tol_in, T1, Yh, S1, S2);
        /* T1 = G - (V + q) Y_h */
        t_apply(C, 1, 1, 0, Yh, T1);
        t_apply(C, 2, 1, 0, T1, T2);   /* T_12 Y_h */
        t_axpby(N, 1, G, -1, T2, T1);
        t_axpby(N, 1, T1, -q, Yh, T1);
        inner += h_solve(C, -q, eps, tol_mid, tol_in, T1, Y, Wh, T2, H1, S1, S2);
    }
    free(pp); free(qq);
    free(Yh); free(T1); free(T2); free(Wh); free(H1); free(H2); free(S1); free(S2);
    if (Jout) *Jout = J;
    return inner;
}

/* Cube end to end: F (n^3, row-major, X_ijk pairs C~_i C~_j C~_k) -> X.
 * Returns the number of inner (slice-Stein) ADI iterations over full tensors. */
long orc_poisson_cube(long n, double tol, double tol_mid, double tol_in, const double *F, double *X, int *Jout)
{
    long N = n * n * n;
    real *d = malloc(sizeof(real) * (size_t)n), *e = calloc((size_t)n, sizeof(real));
    square_bands(n, d, e);
    cube_t C = {n, d, e};
    real *G = malloc(sizeof(real) * (size_t)N), *Y = malloc(sizeof(real) * (size_t)N);
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < n; ++j)
            for (long k = 0; k < n; ++k) {
                long t = (i * n + j) * n + k;
                real s = Ds_diag(i) * Ds_diag(j) * Ds_diag(k); /* |D|^{-1/2} on every mode */
                G[t] = -(real)F[t] * s;
            }
    real eps = 1 / ((real)30 * (real)n * (real)n * (real)n * (real)n);
    long inner = cube_adi(&C, eps, tol, tol_mid, tol_in, G, Y, Jout);
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < n; ++j)
            for (long k = 0; k < n; ++k) {
                long t = (i * n + j) * n + k;
                X[t] = (double)(Y[t] * Ds_diag(i) * Ds_diag(j) * Ds_diag(k));
            }
    free(d); free(e); free(G); free(Y);
    return inner;
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.4 / Table 3.1, steps 1 and 4: Legendre coefficients in and out.       */
/* The conversion from Legendre to the C^(3/2) basis is banded:                 */
/*   (2k+1) P_k = C^(3/2)_k - C^(3/2)_{k-2},                                    */
/* so in the normalised basis C~_k = s_k C^(3/2)_k the C~ coefficients of       */
/* sum_k g_k P_k are B g with B upper bidiagonal with stride 2.  On the way in  */
/* F = B G B^T; on the way out the C~ coefficients of u = (1-x^2)(1-y^2) sum     */
/* X_ij C~_i(y) C~_j(x) are W = M X M^T with M of (3.7) taken (n+2) x n, and    */
/* the Legendre coefficients U solve B U B^T = W (back substitution).  This     */
/* follows the reading that B maps Legendre to C~ (the direction is garbled in  */
/* the printed text).                                                           */
/* ------------------------------------------------------------------------- */

/* s_k of C~_k = s_k C^(3/2)_k (footnote of Sec. 3.1) */
static real ct_norm(long k)
{
    real K = (real)k;
    return sqrt((K + (real)1.5) / ((K + 1) * (K + 2)));
}

/* P_k = C~_k / ((2k+1) s_k) - C~_{k-2} / ((2k+1) s_{k-2}):
 * B[j][j] = 1/((2j+1) s_j), B[j][j+2] = -1/((2j+5) s_j). */
static real B_diag(long j) { return 1 / ((2 * (real)j + 1) * ct_norm(j)); }
static real B_off2(long j) { return -1 / ((2 * (real)j + 5) * ct_norm(j)); }

/* F (n x n) = B G B^T for Legendre coefficients G[a*n + b] of sum G_ab P_a(y) P_b(x). */
void orc_legendre_to_ctilde(long n, const double *G, double *F)
{
    real *T = malloc(sizeof(real) * (size_t)(n * n));
    for (long j = 0; j < n; ++j) /* T = B G */
        for (long k = 0; k < n; ++k) {
            real v = B_diag(j) * (real)G[j * n + k];
            if (j + 2 < n) v += B_off2(j) * (real)G[(j + 2) * n + k];
            T[j * n + k] = v;
        }
    for (long j = 0; j < n; ++j) /* F = T B^T */
        for (long k = 0; k < n; ++k) {
            real v = B_diag(k) * T[j * n + k];
            if (k + 2 < n) v += B_off2(k) * T[j * n + k + 2];
            F[j * n + k] = (double)v;
        }
    free(T);
}

/* M[i][a] of (3.7) (symmetric, bands 0 and +-2), for any i, a >= 0 */
static real M_entry(long i, long a)
{
    if (i == a) return M_diag(i);
    if (i == a + 2) return M_off2(a);
    if (a == i + 2) return M_off2(i);
    return 0;
}

/* U ((n+2) x (n+2)): Legendre coefficients of u = (1-x^2)(1-y^2) sum X_ij C~_i(y) C~_j(x). */
void orc_solution_to_legendre(long n, const double *X, double *U)
{
    long m = n + 2;
    real *W1 = calloc((size_t)(m * n), sizeof(real));
    real *W = calloc((size_t)(m * m), sizeof(real));
    for (long i = 0; i < m; ++i) /* W1 = M X, (n+2) x n */
        for (long k = 0; k < n; ++k) {
            real v = 0;
            for (long a = i - 2; a <= i + 2; a += 2)
                if (a >= 0 && a < n) v += M_entry(i, a) * (real)X[a * n + k];
            W1[i * n + k] = v;
        }
    for (long i = 0; i < m; ++i) /* W = W1 M^T, (n+2) x (n+2) */
        for (long j = 0; j < m; ++j) {
            real v = 0;
            for (long b = j - 2; b <= j + 2; b += 2)
                if (b >= 0 && b < n) v += W1[i * n + b] * M_entry(j, b);
            W[i * m + j] = v;
        }
    for (long j = 0; j < m; ++j) /* B V = W, column by column from the bottom (V in W) */
        for (long i = m - 1; i >= 0; --i) {
            real v = W[i * m + j];
            if (i + 2 < m) v -= B_off2(i) * W[(i + 2) * m + j];
            W[i * m + j] = v / B_diag(i);
        }
    for (long i = 0; i < m; ++i) /* U B^T = V, row by row from the right */
        for (long k = m - 1; k >= 0; --k) {
            real v = W[i * m + k];
            if (k + 2 < m) v -= B_off2(k) * W[i * m + k + 2];
            W[i * m + k] = v / B_diag(k);
        }
    for (long t = 0; t < m * m; ++t) U[t] = (double)W[t];
    free(W1);
    free(W);
}

/* ------------------------------------------------------------------------- */
/* Transposes of the two Legendre maps, for gradients through them (the         */
/* chain rule of a loss L(U) back to G): with F = B G B^T the gradient in G is  */
/* B^T Fbar B; with U = B^{-1} (M X M^T) B^{-T} (M taken (n+2) x n) the         */
/* gradient in X is M^T (B^{-T} Ubar B^{-1}) M.                                 */
/* ------------------------------------------------------------------------- */

/* Gbar (n x n) = B^T Fbar B. */
void orc_legendre_to_ctilde_adjoint(long n, const double *Fbar, double *Gbar)
{
    real *T = malloc(sizeof(real) * (size_t)(n * n));
    for (long j = 0; j < n; ++j) /* T = Fbar B: column b takes B[b][b] and B[b-2][b] */
        for (long b = 0; b < n; ++b) {
            real v = B_diag(b) * (real)Fbar[j * n + b];
            if (b >= 2) v += B_off2(b - 2) * (real)Fbar[j * n + b - 2];
            T[j * n + b] = v;
        }
    for (long a = 0; a < n; ++a) /* Gbar = B^T T: row a takes B[a][a] and B[a-2][a] */
        for (long b = 0; b < n; ++b) {
            real v = B_diag(a) * T[a * n + b];
            if (a >= 2) v += B_off2(a - 2) * T[(a - 2) * n + b];
            Gbar[a * n + b] = (double)v;
        }
    free(T);
}

/* Xbar (n x n) = M^T (B^{-T} Ubar B^{-1}) M for Ubar ((n+2) x (n+2)). */
void orc_solution_to_legendre_adjoint(long n, const double *Ubar, double *Xbar)
{
    long m = n + 2;
    real *V = malloc(sizeof(real) * (size_t)(m * m));
    real *W1 = calloc((size_t)(n * m), sizeof(real));
    for (long t = 0; t < m * m; ++t) V[t] = (real)Ubar[t];
    for (long j = 0; j < m; ++j) /* B^T V' = V, column by column from the top (lower triangular) */
        for (long i = 0; i < m; ++i) {
            real v = V[i * m + j];
            if (i >= 2) v -= B_off2(i - 2) * V[(i - 2) * m + j];
            V[i * m + j] = v / B_diag(i);
        }
    for (long i = 0; i < m; ++i) /* V'' B = V', row by row from the left */
        for (long k = 0; k < m; ++k) {
            real v = V[i * m + k];
            if (k >= 2) v -= B_off2(k - 2) * V[i * m + k - 2];
            V[i * m + k] = v / B_diag(k);
        }
    for (long a = 0; a < n; ++a) /* W1 = M^T V, n x (n+2) */
        for (long j = 0; j < m; ++j) {
            real v = 0;
            for (long i = a - 2; i <= a + 2; i += 2)
                if (i >= 0 && i < m) v += M_entry(i, a) * V[i * m + j];
            W1[a * m + j] = v;
        }
    for (long a = 0; a < n; ++a) /* Xbar = W1 M, n x n */
        for (long b = 0; b < n; ++b) {
            real v = 0;
            for (long j = b - 2; j <= b + 2; j += 2)
                if (j >= 0 && j < m) v += W1[a * m + j] * M_entry(j, b);
            Xbar[a * n + b] = (double)v;
        }
    free(V);
    free(W1);
}

/* Threads OpenMP will use (reported beside the CPU-baseline timings). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* sizeof(real): 8 for the double build, 16 (80-bit payload) for long double. */
int orc_real_bytes(void) { return (int)sizeof(real); }
