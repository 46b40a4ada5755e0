// Host-side FP64 mathematics of the solver: the symmetric matrix A~ of (3.9),
// the spectral interval of Lemma B.2, the iteration count (2.9) and the
// Zolotarev shifts (2.4).  Internal header of the library.
#pragma once
#include <cstdint>
#include <vector>

namespace fps {

// A~ = -E^{-1/2} M E^{-1/2}, E = diag((j+1)(j+2)): diag d (n) and e[j] = A~[j][j+2]
// (padded to length n with zeros so that e[j] = 0 for j+2 >= n).
void square_bands(int64_t n, std::vector<double> &d, std::vector<double> &e);

// 1/sqrt(E_j), j < n: the diagonal D_s of (3.9) (D_s = |D|^{-1/2}).
void inv_sqrt_E(int64_t n, std::vector<double> &s);

// Lemma B.2 lower end of |sigma(A~)|: 1/(30 n^4).
double square_eps(int64_t n);

// Tight bounds sigma(A~) in [-hi, -lo] from Sturm-count bisection, with a safety
// factor 1/2 on lo and 1.01 on hi.
void square_tight_interval(int64_t n, double &lo, double &hi);

// J = ceil(log(16 gamma) log(4/tol) / pi^2), gamma the cross-ratio of [a,b], [c,d].
int adi_iterations(double a, double b, double c, double d, double tol);

// Shifts p_j in [a,b] and q_j in [c,d] of (2.4) for J iterations.
void zolotarev_shifts(double a, double b, double c, double d, int J, std::vector<double> &p, std::vector<double> &q);

// Symmetric case [a,b] = [-hi,-lo], [c,d] = [lo,hi]: q_j = hi * dn(u_j; k' = lo/hi), p_j = -q_j.
void zolotarev_shifts_symmetric(double lo, double hi, int J, std::vector<double> &q);

// Allocation-free variant writing into a caller array q of length J (the vector
// form above calls it, so both give the same bits).
void zolotarev_shifts_symmetric_into(double lo, double hi, int J, double *q);

// Every shift must be finite and lie in its interval [lo, hi] (up to rounding): the
// shifted matrices are only guaranteed non-singular there.
bool shifts_valid(const std::vector<double> &q, double lo, double hi);

// Host-side fault injection for the failure-path tests: with FPS_INJECT_SHIFT_FAULT=nan
// or =neg in the environment the first shift of the list is corrupted.
void inject_shift_fault(std::vector<double> &q);

}  // namespace fps
