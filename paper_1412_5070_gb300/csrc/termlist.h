// termlist.h -- host-side term lists of the F12 kernels.
//
// Every kernel k_i(r) of Sec. 2.2 (Eqs. k1-k6) built from the
// range-separated factor of Sec. 3.1 (Eq. rs12, Eq. ttdamp) is a finite sum
// of terms c r^a exp(b r - g r^2).  Expanding the damping function in the
// kernel is the separation of Eq. hj00eps; every integral over one term is
// then a generating integral S(alpha, beta, gamma) of Eq. sila, understood
// as its finite part when alpha <= -1.
//
// The lists are grouped into families: terms with the same (b, g) whose
// powers a differ by integers.  One family shares one S(alpha_0 + N, ...)
// sequence (Sec. 3.1: S is needed only on alpha_0 + N families).
#pragma once

#include <vector>

namespace f12 {

struct Term {
  double c, a, b, g;  // c * x^a * exp(b x - g x^2)
};
using TermList = std::vector<Term>;

struct Factor {
  double c0, rho, B, mu;
  int n;
};

// f(r) of Eq. rs12 with S_n of Eq. ttdamp expanded:
//   (1 + r/2) e^{-mu r^2} + c0 r^rho e^{B r} - c0 sum_k mu^k/k! r^{rho+2k} e^{B r - mu r^2}
TermList factor_terms(const Factor &f);
TermList derivative(const TermList &t);                       // d/dr
TermList product(const TermList &x, const TermList &y);
TermList times_power(const TermList &t, double m);            // r^m * t
void simplify(TermList &t);                                   // merge like terms, drop zeros

// Kernel of class cls (1..6; class 5 uses the I3 kernel f, Eq. I5_), from the
// factor pair as term lists or as parameters of Eq. rs12.
TermList kernel_terms(int cls, const TermList &f, const TermList &fp);
TermList kernel_terms(int cls, const Factor &f, const Factor &fp);

struct Family {
  double b, g;     // common exponential parameters
  double a0;       // lowest power in the family
  std::vector<double> poly;   // coefficient of x^{a0 + j}, j = 0..
};

std::vector<Family> families(const TermList &t);

// The radial operator D_r = r^-1 d/dr applied to one family:
//   D_r [x^a e^{bx - g x^2}] = (a x^{a-2} + b x^{a-1} - 2 g x^a) e^{bx - g x^2}.
// Returns the new family (a0 lowered by 2).
Family radial_derivative(const Family &f);

}  // namespace f12
