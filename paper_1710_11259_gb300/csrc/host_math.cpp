// Host FP64 mathematics: A~ of (3.9), Lemma B.2, eq. (2.9), shifts (2.4).
//
// Elliptic functions are parametrised by the complementary modulus k' so that
// the tiny k' = 1/(30 n^4) of the square (down to ~3e-18 at n = 10^4) keeps its
// full relative precision:
//   K(k')  = pi / (2 AGM(1, k'))                                  (DLMF 19.8.5)
//   dn(u)  for u <= K/2:
//          k' < 1e-7 : expansion about k = 1,
//                      dn = sech u + (k'^2/4)(sinh u cosh u + u) tanh u sech u   (DLMF 22.10.ii)
//          otherwise : descending Landen / AGM scheme                  (DLMF 22.20(ii))
//   dn(u)  for u >  K/2: quarter-period reflection dn(u) = k' / dn(K - u)        (DLMF 22.4.3)
// The shift arguments u_j = (2j+1)K/(2J) satisfy K - u_j = u_{J-1-j}, so every
// shift comes from an argument u <= K/2 where dn >= sqrt(k') is well conditioned.
#include "host_math.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>

namespace fps {

namespace {
constexpr double kPi = 3.14159265358979323846;

double agm(double a, double b)
{
    for (int it = 0; it < 80; ++it) {
        double an = 0.5 * (a + b);
        double bn = std::sqrt(a * b);
        if (std::fabs(an - bn) <= 1e-17 * an) return an;
        a = an;
        b = bn;
    }
    return a;
}

double ellip_K_kp(double kp) { return kPi / (2.0 * agm(1.0, kp)); }

// dn(u | k) with k = sqrt(1 - kp^2), valid for 0 <= u <= K/2.
double dn_lower_half(double u, double kp)
{
    if (kp < 1e-7) {
        double ch = std::cosh(u), sh = std::sinh(u);
        double sech = 1.0 / ch;
        return sech + 0.25 * kp * kp * (sh * ch + u) * (sh / ch) * sech;
    }
    // descending Landen: a0 = 1, b0 = k', c0 = k
    double a[64], c[64];
    double b = kp;
    a[0] = 1.0;
    c[0] = std::sqrt((1.0 - kp) * (1.0 + kp));
    int N = 0;
    while (N < 60 && std::fabs(c[N]) > 1e-17 * a[N]) {
        a[N + 1] = 0.5 * (a[N] + b);
        c[N + 1] = 0.5 * (a[N] - b);
        b = std::sqrt(a[N] * b);
        ++N;
    }
    if (N == 0) return 1.0;
    double phi = std::ldexp(a[N] * u, N), phi1 = phi;
    for (int k = N; k >= 1; --k) {
        phi1 = phi;
        phi = 0.5 * (phi + std::asin(c[k] * std::sin(phi) / a[k]));
    }
    return std::cos(phi) / std::cos(phi1 - phi);
}

// dn(u_j) for u_j = (2j+1) K / (2J), j = 0..J-1, complementary modulus kp.
std::vector<double> dn_at_shift_points(int J, double kp)
{
    double K = ellip_K_kp(kp);
    std::vector<double> dn(J);
    for (int j = 0; 2 * j + 1 <= J; ++j) {       // u_j <= K/2
        double u = (2.0 * j + 1.0) * K / (2.0 * J);
        dn[j] = dn_lower_half(u, kp);
    }
    for (int j = 0; j < J; ++j) {
        if (2 * j + 1 > J) dn[j] = kp / dn[J - 1 - j];
    }
    return dn;
}
}  // namespace

void square_bands(int64_t n, std::vector<double> &d, std::vector<double> &e)
{
    d.assign(n, 0.0);
    e.assign(n, 0.0);
    for (int64_t j = 0; j < n; ++j) {
        double x = (double)j;
        double Ej = (x + 1.0) * (x + 2.0);
        double Mjj = 2.0 * (x + 1.0) * (x + 2.0) / ((2.0 * x + 1.0) * (2.0 * x + 5.0));       // (3.7)
        d[j] = -Mjj / Ej;
        if (j + 2 < n) {
            double Ej2 = (x + 3.0) * (x + 4.0);
            double prod4 = (x + 1.0) * (x + 2.0) * (x + 3.0) * (x + 4.0);                        // (j+4)!/j!
            double Mj2 = -std::sqrt(prod4 * (2.0 * x + 3.0) / (2.0 * x + 7.0)) / ((2.0 * x + 3.0) * (2.0 * x + 5.0));
            e[j] = -Mj2 / std::sqrt(Ej * Ej2);
        }
    }
}

void inv_sqrt_E(int64_t n, std::vector<double> &s)
{
    s.resize(n);
    for (int64_t j = 0; j < n; ++j) s[j] = 1.0 / std::sqrt(((double)j + 1.0) * ((double)j + 2.0));
}

double square_eps(int64_t n)
{
    double x = (double)n;
    return 1.0 / (30.0 * x * x * x * x);
}

int adi_iterations(double a, double b, double c, double d, double tol)
{
    double gam = std::fabs(c - a) * std::fabs(d - b) / (std::fabs(c - b) * std::fabs(d - a));
    return (int)std::ceil(std::log(16.0 * gam) * std::log(4.0 / tol) / (kPi * kPi));
}

void zolotarev_shifts_symmetric(double lo, double hi, int J, std::vector<double> &q)
{
    q.resize(J);
    zolotarev_shifts_symmetric_into(lo, hi, J, q.data());
}

void zolotarev_shifts(double a, double b, double c, double d, int J, std::vector<double> &p, std::vector<double> &q)
{
    double gam = std::fabs(c - a) * std::fabs(d - b) / (std::fabs(c - b) * std::fabs(d - a));
    double alp = -1.0 + 2.0 * gam + 2.0 * std::sqrt(gam * gam - gam);
    // T is the Moebius map with T(-alp) = a, T(-1) = b, T(1) = c (and then T(alp) = d,
    // the cross-ratios being equal).  Built as the composition of the map sending
    // (-alp, -1, 1) to (0, 1, inf) with the inverse of the map sending (a, b, c) to
    // (0, 1, inf):  s = (z + alp) * 2 / ((1 - z)(alp - 1)),  then w solves
    // s = (w - a)(b - c) / ((w - c)(b - a)), i.e. w = c + (c - a)(b - c) / (s (b - a) - (b - c)).
    auto T = [&](double z) {
        double s = 2.0 * (z + alp) / ((1.0 - z) * (alp - 1.0));
        return c + (c - a) * (b - c) / (s * (b - a) - (b - c));
    };
    std::vector<double> dn = dn_at_shift_points(J, 1.0 / alp);
    p.resize(J);
    q.resize(J);
    for (int j = 0; j < J; ++j) {
        p[j] = T(-alp * dn[j]);
        q[j] = T(alp * dn[j]);
    }
}

// Number of eigenvalues of A~ (size n) below x: Sturm count, i.e. the negative
// pivots of the LDL^T factorisation of A~ - x I on the even and on the odd index
// set (the two decoupled tridiagonals of App. B).
static int64_t sturm_count_below(const std::vector<double> &d, const std::vector<double> &e, double x)
{
    const int64_t n = (int64_t)d.size();
    int64_t count = 0;
    for (int par = 0; par < 2; ++par) {
        double piv = 0.0;
        for (int64_t i = par; i < n; i += 2) {
            double v = d[i] - x;
            if (i >= 2) {
                const double off = e[i - 2];
                v -= (piv != 0.0) ? off * off / piv : off * off / 1e-300;
            }
            if (v == 0.0) v = -1e-300;
            if (v < 0.0) ++count;
            piv = v;
        }
    }
    return count;
}

void square_tight_interval(int64_t n, double &lo, double &hi)
{
    std::vector<double> d, e;
    square_bands(n, d, e);
    // largest eigenvalue (closest to zero): bisection in log|x| on [-1, -eps/8]
    double a = std::log(square_eps(n) / 8.0), b = 0.0;  // log of |x|: the largest eig has |x| in [e^a, e^b]
    for (int it = 0; it < 80; ++it) {
        const double mid = 0.5 * (a + b);
        // all n eigenvalues below -exp(mid)  <=>  lambda_max < -exp(mid)
        if (sturm_count_below(d, e, -std::exp(mid)) == n) a = mid;
        else b = mid;
    }
    const double lam_max_abs = std::exp(a);  // |lambda_max| >= this
    // smallest eigenvalue: bisection on [-1, 0]
    double l = -1.0, r = 0.0;
    for (int it = 0; it < 80; ++it) {
        const double mid = 0.5 * (l + r);
        if (sturm_count_below(d, e, mid) == 0) l = mid;
        else r = mid;
    }
    // safety margins: a factor of two at the small end, one percent at the large end
    lo = 0.5 * lam_max_abs;
    hi = std::min(1.0, 1.01 * (-l));
}

// Allocation-free form of zolotarev_shifts_symmetric (caller-provided array), for
// the entry point that must not allocate; the vector form calls it.
void zolotarev_shifts_symmetric_into(double lo, double hi, int J, double *q)
{
    const double kp = lo / hi;
    const double K = ellip_K_kp(kp);
    for (int j = 0; 2 * j + 1 <= J; ++j) q[j] = dn_lower_half((2.0 * j + 1.0) * K / (2.0 * J), kp);
    for (int j = 0; j < J; ++j)
        if (2 * j + 1 > J) q[j] = kp / q[J - 1 - j];
    for (int j = 0; j < J; ++j) q[j] = hi * q[j];
}

bool shifts_valid(const std::vector<double> &q, double lo, double hi)
{
    for (double v : q)
        if (!std::isfinite(v) || v < lo * (1.0 - 1e-12) || v > hi * (1.0 + 1e-12)) return false;
    return !q.empty();
}

void inject_shift_fault(std::vector<double> &q)
{
    const char *f = std::getenv("FPS_INJECT_SHIFT_FAULT");
    if (!f || q.empty()) return;
    if (std::string(f) == "nan") q[0] = std::nan("");
    else if (std::string(f) == "neg") q[0] = -q[0];
}

}  // namespace fps
