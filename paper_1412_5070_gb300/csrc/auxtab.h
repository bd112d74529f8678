// auxtab.h -- host-side construction of the tables that the auxiliary-function
// stage (aux.cuh) reads: quadrature nodes, series coefficient ratios and the
// kernel families of each integral class.  The library fills them before it
// uploads them to the device; the CPU test build of aux.cuh fills them the
// same way.
#pragma once

#include <cmath>
#include <map>
#include <vector>

#include "aux.cuh"
#include "termlist.h"

namespace f12dev {

// Gauss-Hermite nodes and weights (weight e^{-t^2}) from the orthonormal
// Hermite recurrence: sign changes on a fine grid, then Newton.
inline void gauss_hermite(int n, double *x, double *w) {
  auto eval = [n](double t, double &pn, double &pn1) {
    double p0 = 0.0, p1 = std::pow(M_PI, -0.25);
    for (int k = 0; k < n; ++k) {
      double p2 = t * std::sqrt(2.0 / (k + 1)) * p1 - std::sqrt((double)k / (k + 1)) * p0;
      p0 = p1;
      p1 = p2;
    }
    pn = p1;
    pn1 = p0;
  };
  double lim = std::sqrt(2.0 * n + 1.0) + 1.0;
  int found = 0;
  const int grid = 200000;
  double tprev = -lim, pprev, dummy;
  eval(tprev, pprev, dummy);
  for (int i = 1; i <= grid && found < n; ++i) {
    double t = -lim + 2.0 * lim * i / grid, pc;
    eval(t, pc, dummy);
    if ((pc < 0) != (pprev < 0)) {
      double r = 0.5 * (t + tprev);
      for (int it = 0; it < 100; ++it) {
        double pn, pn1;
        eval(r, pn, pn1);
        double dp = std::sqrt(2.0 * n) * pn1;
        double dr = pn / dp;
        r -= dr;
        if (std::fabs(dr) < 1e-15 * (1.0 + std::fabs(r))) break;
      }
      double pn, pn1;
      eval(r, pn, pn1);
      x[found] = r;
      w[found] = 1.0 / (n * pn1 * pn1);
      ++found;
    }
    tprev = t;
    pprev = pc;
  }
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton on P_n from the
// Chebyshev-like first guesses cos(pi (i + 3/4)/(n + 1/2)), with P_n and
// P_n' from the three-term recurrence; w = 2 / ((1 - t^2) P_n'(t)^2).
inline void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
    }
    x[n - 1 - i] = t;
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

struct AuxConst {
  double gh_x[NGH], gh_w[NGH];
  double gl_x[NGL], gl_w[NGL];
  double cratio[LAUX + 1][KTAB];
  double inv_dfact[LAUX + 2];
  double kum_inv[2][NKUM];
  double sm1_ratio[NKUM];
};

inline void fill_aux_const(AuxConst &c) {
  gauss_hermite(NGH, c.gh_x, c.gh_w);
  gauss_legendre(NGL, c.gl_x, c.gl_w);
  for (int l = 0; l <= LAUX; ++l)
    for (int k = 0; k < KTAB; ++k)
      c.cratio[l][k] = (double)(k + l + 1) / ((double)(k + 1) * (2.0 * k + 2.0 * l + 2.0) * (2.0 * k + 2.0 * l + 3.0));
  c.inv_dfact[0] = 1.0;
  for (int l = 1; l < LAUX + 2; ++l) c.inv_dfact[l] = c.inv_dfact[l - 1] / (2.0 * l + 1.0);
  for (int n = 0; n < NKUM; ++n) {
    c.kum_inv[0][n] = 1.0 / ((0.5 + n) * (n + 1.0));
    c.kum_inv[1][n] = 1.0 / ((1.5 + n) * (n + 1.0));
    // Gamma((m+1)/2) / (Gamma(m/2) (m+1)); entry 0 unused
    c.sm1_ratio[n] = n == 0 ? 0.0 : std::exp(std::lgamma(0.5 * (n + 1.0)) - std::lgamma(0.5 * n)) / (n + 1.0);
  }
}

// Families of every class on the host: fams and coef are uploaded as they are;
// nfam/fam0 index them per class (class 5 shares class 3's families, Eq. I5_).
struct ClassTables {
  std::vector<FamDev> fams;
  std::vector<double> coef;
  int nfam[NCLASS] = {};
  int fam0[NCLASS] = {};
  bool supported[NCLASS] = {};
  bool quad[NCLASS] = {};        // the class has a family evaluated by quadrature (FamDev::quad)
};

// kernels[cls] (cls = 1..6; entry 5 unused) are the kernel term lists.  A class
// is left out (supported false) when x^2 k(x) is not integrable at r = 0 (the
// families' coefficients of some power x^p, p <= -1, do not cancel; the
// damping of Eq. rs12 always cancels them), when a family's lowest power is
// below -KSING (= -2), when a family evaluated by quadrature (b < 0 or lowest power
// below -1) has a power that is neither an integer nor a half-integer (the
// end-point forms family_quad handles), or when it has more than MAXFAM
// families.  Returns false if a family polynomial is longer than JMAX.
inline bool build_class_tables(const f12::TermList kernels[NCLASS], ClassTables &ct) {
  ct.fams.clear();
  ct.coef.clear();
  ct.supported[0] = false;
  for (int cls = 1; cls <= 6; ++cls) {
    ct.fam0[cls] = (int)ct.fams.size();
    ct.nfam[cls] = 0;
    ct.supported[cls] = true;
    ct.quad[cls] = false;
    if (cls == 5) {
      ct.fam0[cls] = ct.fam0[3];
      ct.nfam[cls] = ct.nfam[3];
      ct.supported[5] = ct.supported[3];
      ct.quad[5] = ct.quad[3];
      continue;
    }
    std::vector<f12::Family> fl = f12::families(kernels[cls]);
    std::vector<FamDev> mine;
    // integrable at r = 0: for every power p <= -1 of x^2 k(x) near 0, the
    // families' Taylor coefficients of x^alpha0 P(x) e^{bx - gx^2} at x^p
    // (each family taken as a finite part) must cancel between them
    std::map<long, std::pair<double, double>> sing;   // 2p -> (sum, sum of |.|)
    for (const f12::Family &fam0 : fl) {
      const double a = fam0.a0 + 2.0;
      if (a < -(double)KSING - 1e-9) ct.supported[cls] = false;
      if (a > -1.0 + 1e-9 || !ct.supported[cls]) continue;
      const double twice = 2.0 * a;
      if (std::fabs(twice - std::round(twice)) > 1e-9) {   // a general power below -1
        ct.supported[cls] = false;
        continue;
      }
      double h[KSING + 1] = {1.0, fam0.b};                 // Taylor of e^{bx - gx^2}
      for (int j = 2; j <= KSING; ++j) h[j] = (fam0.b * h[j - 1] - 2.0 * fam0.g * h[j - 2]) / j;
      for (int k = 0; a + k <= -1.0 + 1e-9; ++k) {
        double c = 0.0;
        for (int i = 0; i <= k && i < (int)fam0.poly.size(); ++i) c += fam0.poly[(size_t)i] * h[k - i];
        auto &e = sing[std::lround(twice) + 2 * k];
        e.first += c;
        e.second += std::fabs(c);
      }
    }
    for (const auto &e : sing)
      if (std::fabs(e.second.first) > 1e-10 * e.second.second) ct.supported[cls] = false;
    if ((int)fl.size() > MAXFAM) ct.supported[cls] = false;
    if (!ct.supported[cls]) continue;
    std::vector<double> coef;
    for (const f12::Family &fam0 : fl) {
      FamDev d{};
      d.b = fam0.b;
      d.g = fam0.g;
      d.alpha0 = fam0.a0 + 2.0;   // F_l = x^{2l+2} D_r^l k: lowest power a0 + 2 for every l
      d.fp_minus1 = std::fabs(d.alpha0 + 1.0) < 1e-9 ? 1 : 0;
      if (d.fp_minus1) d.alpha0 = -1.0;
      for (int j = 0; j < JMAX; ++j) {   // Gamma((alpha0+1+j)/2); 0 at the poles
        double arg = 0.5 * (d.alpha0 + 1.0 + j);
        const bool pole = arg <= 0.0 && std::fabs(arg - std::round(arg)) < 1e-9;
        d.gam_tab[j] = pole ? 0.0 : std::tgamma(arg);
      }
      {
        double flo = std::floor(d.alpha0 + 1e-9);
        double fr = d.alpha0 - flo;
        d.pow_int = (int)flo;
        d.pow_kind = (std::fabs(fr) < 1e-9) ? 1 : (std::fabs(fr - 0.5) < 1e-9 ? 2 : 0);
      }
      d.nsing = d.alpha0 <= -1.0 + 1e-9 ? (int)std::floor(-d.alpha0 + 1e-9) : 0;
      d.quad = (d.b < 0.0 || d.alpha0 < -1.0 - 1e-9) ? 1 : 0;
      if (d.quad && d.pow_kind == 0) ct.supported[cls] = false;
      double as = d.fp_minus1 ? 0.0 : d.alpha0;
      d.rho_start = std::exp(std::lgamma(0.5 * (as + 2.0)) - std::lgamma(0.5 * (as + 1.0)));
      f12::Family cur = fam0;
      for (int l = 0; l <= LAUX; ++l) {
        if ((int)cur.poly.size() > JMAX) return false;
        d.coff[l] = (int)(ct.coef.size() + coef.size());
        d.span[l] = (int)cur.poly.size();
        coef.insert(coef.end(), cur.poly.begin(), cur.poly.end());
        cur = f12::radial_derivative(cur);
      }
      mine.push_back(d);
    }
    if (!ct.supported[cls]) continue;
    ct.fams.insert(ct.fams.end(), mine.begin(), mine.end());
    ct.coef.insert(ct.coef.end(), coef.begin(), coef.end());
    ct.nfam[cls] = (int)mine.size();
    for (const FamDev &d : mine) ct.quad[cls] = ct.quad[cls] || d.quad;
  }
  return true;
}

}  // namespace f12dev
