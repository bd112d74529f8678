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
  double gh_x[NGH + NGHF], gh_w[NGH + NGHF];   // the NGH-node rule, then the NGHF-node one
  double gl_x[NGL], gl_w[NGL];
  double cratio[LAUX + 1][KTAB];
  double inv_dfact[LAUX + 2];
  double kum_inv[2][NKUM];
  double sm1_ratio[NKUM];
  double cser[LAUX + 1][KMAX];   // d_cser
  double vstep[KMAX];            // d_vstep
  double quarter[NQUARTER];      // d_quarter
};

inline void fill_aux_const(AuxConst &c) {
  gauss_hermite(NGH, c.gh_x, c.gh_w);
  gauss_hermite(NGHF, c.gh_x + NGH, c.gh_w + NGH);
  gauss_legendre(NGL, c.gl_x, c.gl_w);
  for (int l = 0; l <= LAUX; ++l)
    for (int k = 0; k < KTAB; ++k)
      c.cratio[l][k] = (double)(k + l + 1) / ((double)(k + 1) * (2.0 * k + 2.0 * l + 2.0) * (2.0 * k + 2.0 * l + 3.0));
  c.inv_dfact[0] = 1.0;
  for (int l = 1; l < LAUX + 2; ++l) c.inv_dfact[l] = c.inv_dfact[l - 1] / (2.0 * l + 1.0);
  {
    // c_{l,k} as a long double mantissa times 2^ex (frexp after every step)
    int E[KMAX];
    long double m0 = 1.0L;   // c_{0,k} = m0 2^x0
    int x0 = 0;
    for (int k = 0; k < KMAX; ++k) {
      int e = 0;
      const long double f = std::frexp(m0, &e);   // c_{0,k} = f 2^{x0 + e}, f in [1/2, 1)
      E[k] = -(x0 + e - 1);                        // c_{0,k} 2^{E_k} = 2 f in [1, 2)
      m0 = f;
      x0 += e;
      m0 *= (long double)(k + 1) / ((long double)(k + 1) * (2.0L * k + 2.0L) * (2.0L * k + 3.0L));
    }
    for (int l = 0; l <= LAUX; ++l) {
      long double m = 1.0L;   // c_{l,0} = 2^l l!/(2l+1)! = 1/(2l+1)!!
      for (int i = 1; i <= l; ++i) m /= (2.0L * i + 1.0L);
      int x = 0;
      for (int k = 0; k < KMAX; ++k) {
        int e = 0;
        m = std::frexp(m, &e);
        x += e;
        c.cser[l][k] = (double)std::ldexp(m, x + E[k]);
        m *= (long double)(k + l + 1) / ((long double)(k + 1) * (2.0L * k + 2.0L * l + 2.0L) * (2.0L * k + 2.0L * l + 3.0L));
      }
    }
    for (int k = 0; k + 1 < KMAX; ++k) c.vstep[k] = std::ldexp(1.0, E[k] - E[k + 1]);
    c.vstep[KMAX - 1] = 0.0;
    for (int i = 0; i < NQUARTER; ++i) c.quarter[i] = 0.25 * i;
  }
  for (int n = 0; n < NKUM; ++n) {
    c.kum_inv[0][n] = 1.0 / ((0.5 + n) * (n + 1.0));
    c.kum_inv[1][n] = 1.0 / ((1.5 + n) * (n + 1.0));
    // Gamma((m+1)/2) / (Gamma(m/2) (m+1)); entry 0 unused
    c.sm1_ratio[n] = n == 0 ? 0.0 : std::exp(std::lgamma(0.5 * (n + 1.0)) - std::lgamma(0.5 * n)) / (n + 1.0);
  }
}

// Families of every class on the host: fams, coef and groups are uploaded as
// they are; nfam/fam0 index the families per class (class 5 shares class 3's
// families, Eq. I5_).
struct ClassTables {
  std::vector<FamDev> fams;
  std::vector<double> coef;
  std::vector<GroupDev> groups;
  std::vector<double> jtab;      // start-value tables (FamDev::jtab)
  int nfam[NCLASS] = {};
  int fam0[NCLASS] = {};
  bool supported[NCLASS] = {};
  bool quad[NCLASS] = {};        // the class has a family evaluated by quadrature (FamDev::quad)
};

// kernels[cls] (cls = 1..6; entry 5 unused) are the kernel term lists.  A class
// is left out (supported false) when x^2 k(x) is not integrable at r = 0 (the
// families' coefficients of some power x^p, p <= -1, do not cancel; the
// damping of Eq. rs12 always cancels them), when a power below -1 is neither
// an integer nor a half-integer, when it has more than MAXFAM families, or
// when a family evaluated alone by quadrature (b < 0, or a lowest power below
// -1 outside a group) has a general power or a lowest power below -KSING.
// Families with a lowest power below -1 are grouped with the families of the
// same b and power lattice when their singular terms cancel within the group
// (GroupDev).  Returns false if a family polynomial is longer than JMAX.
inline void build_start_tables(ClassTables &ct);

inline bool build_class_tables(const f12::TermList kernels[NCLASS], ClassTables &ct) {
  constexpr int KTAY = 16;    // Taylor terms for the integrability check (lowest power >= -KTAY + 1)
  ct.fams.clear();
  ct.coef.clear();
  ct.groups.clear();
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
    // integrable at r = 0: for every power p <= -1 of x^2 k(x) near 0, the
    // families' Taylor coefficients of x^alpha0 P(x) e^{bx - gx^2} at x^p
    // (each family taken as a finite part) must cancel between them
    std::map<long, std::pair<double, double>> sing;   // 2p -> (sum, sum of |.|)
    for (const f12::Family &fam0 : fl) {
      const double a = fam0.a0 + 2.0;
      if (a > -1.0 + 1e-9) continue;
      const double twice = 2.0 * a;
      if (std::fabs(twice - std::round(twice)) > 1e-9 || a < -(double)(KTAY - 1)) {
        ct.supported[cls] = false;                     // a general power below -1, or too singular
        break;
      }
      double h[KTAY] = {1.0, fam0.b};                    // Taylor of e^{bx - gx^2}
      for (int q = 2; q < KTAY; ++q) h[q] = (fam0.b * h[q - 1] - 2.0 * fam0.g * h[q - 2]) / q;
      for (int k = 0; a + k <= -1.0 + 1e-9; ++k) {
        double c = 0.0;
        for (int q = 0; q <= k && q < (int)fam0.poly.size(); ++q) c += fam0.poly[(size_t)q] * h[k - q];
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
    std::vector<FamDev> mine;
    for (const f12::Family &fam0 : fl) {
      FamDev d{};
      d.b = fam0.b;
      d.g = fam0.g;
      d.alpha0 = fam0.a0 + 2.0;   // F_l = x^{2l+2} D_r^l k: lowest power a0 + 2 for every l
      d.fp_minus1 = std::fabs(d.alpha0 + 1.0) < 1e-9 ? 1 : 0;
      if (d.fp_minus1) d.alpha0 = -1.0;
      for (int q = 0; q < JMAX; ++q) {   // Gamma((alpha0+1+q)/2); 0 at the poles
        double arg = 0.5 * (d.alpha0 + 1.0 + q);
        const bool pole = arg <= 0.0 && std::fabs(arg - std::round(arg)) < 1e-9;
        d.gam_tab[q] = pole ? 0.0 : std::tgamma(arg);
      }
      {
        double flo = std::floor(d.alpha0 + 1e-9);
        double fr = d.alpha0 - flo;
        d.pow_int = (int)flo;
        d.pow_kind = (std::fabs(fr) < 1e-9) ? 1 : (std::fabs(fr - 0.5) < 1e-9 ? 2 : 0);
      }
      d.nsing = d.alpha0 <= -1.0 + 1e-9 ? (int)std::floor(-d.alpha0 + 1e-9) : 0;
      d.quad = (d.b < 0.0 || d.alpha0 < -1.0 - 1e-9) ? 1 : 0;
      d.group = -1;
      d.lead = 0;
      d.jtab = -1;
      d.jrow = 0;
      d.ktab = 0;   // set once the spans are known (mark_kummer_families)
      d.ha_base = (int)std::lround(2.0 * d.alpha0) - 2;
      d.ha_tab = (d.pow_kind != 0 && d.ha_base >= -4 && d.ha_base + 2 * (JMAX + 2 * KMAX) < NQUARTER) ? 1 : 0;
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
    // groups around each family whose lowest power is below -1
    std::vector<GroupDev> gl;
    std::vector<int> gid(mine.size(), -1);
    auto try_group = [&](size_t i0) -> bool {
      std::vector<size_t> mem;
      for (size_t j2 = 0; j2 < mine.size(); ++j2) {
        if (gid[j2] >= 0) continue;
        if (std::fabs(mine[j2].b - mine[i0].b) > 1e-12 * (1.0 + std::fabs(mine[i0].b))) continue;
        const double dd = mine[j2].alpha0 - mine[i0].alpha0;
        if (std::fabs(dd - std::round(dd)) > 1e-9) continue;
        mem.push_back(j2);
      }
      if (mem.size() < 2 || mem.size() > (size_t)MAXMEM) return false;
      GroupDev G{};
      G.b = mine[i0].b;
      G.nmem = (int)mem.size();
      G.abase = mine[mem[0]].alpha0;
      G.gmin = G.gmax = mine[mem[0]].g;
      for (size_t m = 0; m < mem.size(); ++m) {
        G.abase = std::min(G.abase, mine[mem[m]].alpha0);
        G.gmin = std::min(G.gmin, mine[mem[m]].g);
        G.gmax = std::max(G.gmax, mine[mem[m]].g);
      }
      G.xs = G.gmax > 0.0 ? 1.0 / std::sqrt(G.gmax) : 0.0;
      {
        double flo = std::floor(G.abase + 1e-9), fr = G.abase - flo;
        G.pow_int = (int)flo;
        G.pow_kind = (std::fabs(fr) < 1e-9) ? 1 : (std::fabs(fr - 0.5) < 1e-9 ? 2 : 0);
        if (G.pow_kind == 0) return false;
      }
      for (size_t m = 0; m < mem.size(); ++m) {
        const FamDev &F = mine[mem[m]];
        G.dpow[m] = (int)std::lround(F.alpha0 - G.abase);
        if (F.g == 0.0) {
          G.kexp[m] = -1;
        } else {
          int k = 0;
          while (F.alpha0 + 2.0 * k <= -1.0 + 1e-9) ++k;
          if (k >= KEXP) return false;
          G.kexp[m] = k;
        }
      }
      // base polynomial per order: the members' Taylor heads T_k(-g x^2), and
      // the whole of the g = 0 members, in powers x^{abase + j}
      std::vector<double> add;
      for (int l = 0; l <= LAUX; ++l) {
        int len = 0;
        for (size_t m = 0; m < mem.size(); ++m) {
          const int k = G.kexp[m];
          if (k == 0) continue;
          const int ext = G.dpow[m] + mine[mem[m]].span[l] + (k > 0 ? 2 * (k - 1) : 0);
          len = std::max(len, ext);
        }
        std::vector<double> c((size_t)len, 0.0), ab((size_t)len, 0.0);
        for (size_t m = 0; m < mem.size(); ++m) {
          const FamDev &F = mine[mem[m]];
          const double *P = coef.data() + (F.coff[l] - (int)ct.coef.size());
          const int k = G.kexp[m];
          if (k == 0) continue;
          const int nt = k < 0 ? 1 : k;
          double ft = 1.0;                                 // (-g)^t / t!
          for (int t = 0; t < nt; ++t) {
            if (t > 0) ft *= -F.g / t;
            for (int q = 0; q < F.span[l]; ++q) {
              const double v = P[q] * (k < 0 ? 1.0 : ft);
              c[(size_t)(G.dpow[m] + q + 2 * t)] += v;
              ab[(size_t)(G.dpow[m] + q + 2 * t)] += std::fabs(v);
            }
          }
        }
        for (int q = 0; q < len; ++q)
          if (G.abase + q <= -1.0 + 1e-9) {              // singular: must cancel
            if (std::fabs(c[(size_t)q]) > 1e-10 * ab[(size_t)q]) return false;
            c[(size_t)q] = 0.0;
          }
        G.boff[l] = (int)(ct.coef.size() + coef.size() + add.size());
        G.bspan[l] = len;
        add.insert(add.end(), c.begin(), c.end());
      }
      coef.insert(coef.end(), add.begin(), add.end());
      for (size_t m = 0; m < mem.size(); ++m) {
        G.mem[m] = ct.fam0[cls] + (int)mem[m];
        gid[mem[m]] = (int)(ct.groups.size() + gl.size());
      }
      mine[mem[0]].lead = 1;
      gl.push_back(G);
      return true;
    };
    // (the alpha0 = -1 families with b >= 0 stay in the series with their
    // closed-form finite part; those with b < 0 are in the quadrature launch
    // anyway, where a group is the more accurate form)
    for (size_t i0 = 0; i0 < mine.size(); ++i0)
      if ((mine[i0].alpha0 < -1.0 - 1e-9 || (mine[i0].alpha0 < -1.0 + 1e-9 && mine[i0].b < 0.0)) && gid[i0] < 0)
        try_group(i0);
    for (size_t i0 = 0; i0 < mine.size(); ++i0) {
      FamDev &d = mine[i0];
      if (gid[i0] >= 0) {
        d.group = gid[i0];
        d.quad = 1;
        continue;
      }
      if (d.alpha0 < -(double)KSING - 1e-9) ct.supported[cls] = false;
      if (d.quad && d.pow_kind == 0) ct.supported[cls] = false;
    }
    if (!ct.supported[cls]) continue;
    ct.fams.insert(ct.fams.end(), mine.begin(), mine.end());
    ct.coef.insert(ct.coef.end(), coef.begin(), coef.end());
    ct.groups.insert(ct.groups.end(), gl.begin(), gl.end());
    ct.nfam[cls] = (int)mine.size();
    for (const FamDev &d : mine) ct.quad[cls] = ct.quad[cls] || d.quad;
  }
  build_start_tables(ct);
  for (FamDev &d : ct.fams) {
    // the Kummer table serves b = 0 series families with an integer alpha0 >= 0
    // whose a_j = (alpha0 + j + 1)/2 stay on its grid for every order
    int jmax = 0;
    for (int l = 0; l <= LAUX; ++l) jmax = std::max(jmax, d.span[l]);
    d.ktab = (!d.quad && d.b == 0.0 && d.group < 0 && !d.fp_minus1 && d.pow_kind == 1 && d.pow_int >= 0 &&
              d.pow_int + jmax - 1 < MT_NA) ? 1 : 0;
  }
  return true;
}

// Kummer M(a, b, x) e^{-x} for x >= 0, a > 0, b > 0, in long double: the
// series sum_k (a)_k x^k / (k! (b)_k) (every term positive) times e^{-x}.
inline long double kummer_scaled(long double a, long double b, long double x) {
  long double t = 1.0L, s = 1.0L;
  for (int k = 0; k < 5000; ++k) {
    t *= (a + k) * x / ((b + k) * (k + 1));
    s += t;
    if (t <= 1e-21L * s && k > 2) break;
  }
  return s * std::exp(-x);
}

// The table d_mtab: for l <= LAUX, a = (ia + 1)/2 (ia < MT_NA), x_i = i MT_DX,
// the Taylor coefficients (1/m!) d^m T/dx^m of T(a, l, x) = e^{-x} M(a, l + 3/2, x),
//   d^m T/dx^m = (-1)^m (b - a)_m / (b)_m  e^{-x} M(a, b + m, x),  b = l + 3/2.
inline void fill_kummer_table(std::vector<double> &tab) {
  tab.assign((size_t)(LAUX + 1) * MT_NA * MT_NX * MT_NT, 0.0);
  constexpr int NB = LAUX + MT_NT;   // b = 3/2 .. LAUX + MT_NT + 1/2
  std::vector<long double> tb((size_t)NB);
  for (int ia = 0; ia < MT_NA; ++ia) {
    const long double a = 0.5L * (ia + 1);
    for (int ix = 0; ix < MT_NX; ++ix) {
      const long double x = (long double)ix * (long double)MT_DX;
      for (int ib = 0; ib < NB; ++ib) tb[ib] = kummer_scaled(a, 1.5L + ib, x);
      for (int l = 0; l <= LAUX; ++l) {
        const long double b = 1.5L + l;
        long double c = 1.0L;   // (-1)^m (b - a)_m / ((b)_m m!)
        double *row = &tab[(((size_t)l * MT_NA + ia) * MT_NX + ix) * MT_NT];
        for (int m = 0; m < MT_NT; ++m) {
          row[m] = (double)(c * tb[l + m]);
          c *= -(b - a + m) / ((b + m) * (m + 1));
        }
      }
    }
  }
}

// J_a(y) = int_0^inf t^a e^{y t - t^2} dt, a > -1, y >= 0, in long double from
// the Kummer form (Eq. msmallz of App. B, valid for y >= 0; every term
// positive):  J = 1/2 [Gamma((a+1)/2) M((a+1)/2, 1/2, y^2/4)
//                     + y Gamma((a+2)/2) M((a+2)/2, 3/2, y^2/4)].
inline long double kummer_host(long double a, long double b, long double z) {
  long double t = 1.0L, s = 1.0L;
  for (int n = 0; n < 4000; ++n) {
    t *= (a + n) * z / ((b + n) * (n + 1));
    s += t;
    if (t <= 1e-21L * s) break;
  }
  return s;
}

inline long double jstart_host(long double a, long double y) {
  const long double z = 0.25L * y * y;
  return 0.5L * (std::tgamma(0.5L * (a + 1.0L)) * kummer_host(0.5L * (a + 1.0L), 0.5L, z) +
                 y * std::tgamma(0.5L * (a + 2.0L)) * kummer_host(0.5L * (a + 2.0L), 1.5L, z));
}

// Start-value tables of the series families with b > 0 (FamDev::jtab): at
// y_i = i JT_DY, row i holds e_k = J_{as+k}(y_i)/k! for k < JT_NK (as = alpha0,
// or 0 for the finite-part family alpha0 = -1), J_{as+k} from J_{as},
// J_{as+1} by the upward recursion J_{a+1} = (y J_a + a J_{a-1})/2 (positive
// terms).  A finite-part family's rows carry, after the J part, the Taylor
// coefficients of the y-series of S(-1, b, gamma): T(y) = 1/2 sum_{m>=1}
// y^m Gamma(m/2)/m!, whose derivative is J_0(y), so T(y_i + h) = T(y_i) +
// sum_{k>=1} e_{k-1} h^k / k.
inline void build_start_tables(ClassTables &ct) {
  ct.jtab.clear();
  for (FamDev &d : ct.fams) {
    d.jtab = -1;
    d.jrow = 0;
    if (d.quad || !(d.b > 0.0) || d.group >= 0) continue;
    const long double as = d.fp_minus1 ? 0.0L : (long double)d.alpha0;
    d.jrow = d.fp_minus1 ? 2 * JT_NK : JT_NK;
    d.jtab = (int)ct.jtab.size();
    for (int i = 0; i < JT_NY; ++i) {
      const long double y = (long double)i * (long double)JT_DY;
      long double J[JT_NK + 1];
      J[0] = jstart_host(as, y);
      J[1] = jstart_host(as + 1.0L, y);
      for (int k = 2; k <= JT_NK; ++k) J[k] = 0.5L * (y * J[k - 1] + (as + k - 1) * J[k - 2]);
      long double fk = 1.0L;
      long double e[JT_NK];
      for (int k = 0; k < JT_NK; ++k) {
        if (k > 0) fk *= k;
        e[k] = J[k] / fk;
        ct.jtab.push_back((double)e[k]);
      }
      if (d.fp_minus1) {
        // t_m = y^m Gamma(m/2) / (2 m!): t_1 = y sqrt(pi)/2, t_{m+1} = t_m y g_m/(m+1)
        // with g_m = Gamma((m+1)/2)/Gamma(m/2), g_1 = 1/sqrt(pi), g_{m+1} = (m/2)/g_m
        long double T = 0.0L;
        if (y > 0.0L) {
          const long double sqpi = 1.772453850905516027298167483341145182798L;
          long double t = 0.5L * y * sqpi, g = 1.0L / sqpi;
          for (int m = 1; m < 4000; ++m) {
            T += t;
            t *= y * g / (m + 1);
            g = 0.5L * m / g;
            if (m > 2.0L * y * y + 10 && t <= 1e-21L * T) break;
          }
        }
        ct.jtab.push_back((double)T);
        for (int k = 1; k < JT_NK; ++k) ct.jtab.push_back((double)(e[k - 1] / k));
      }
    }
  }
}

}  // namespace f12dev
