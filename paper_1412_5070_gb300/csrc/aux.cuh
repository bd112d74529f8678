// aux.cuh -- device evaluation of the radial derivatives of the basic
// integrals (the auxiliary-function stage).
//
// For a kernel k(r) the quantity needed per primitive quartet is, for
// l = 0..L (Sec. 2.4-2.5, Eq. DQ),
//
//   hat g_l(xi, D) = int_0^inf k(r) r D_Q^l [(e^{-xi(r-D)^2} - e^{-xi(r+D)^2}) / D] dr,
//
// D_Q = D^-1 d/dD, so that g_l = sqrt(pi^5/(p+q))/(pq) hat g_l (Eq. bfinal).
// Moving the l derivatives from the Gaussian onto the kernel (integration
// by parts, Hobson's operator identity in 2l+3 dimensions) gives the form
// evaluated here,
//
//   hat g_l = 4 xi (2 xi)^l e^{-xi D^2} int_0^inf F_l(x) e^{-xi x^2} j_l(2 xi D x) dx,
//   F_l(x)  = x^{2l+2} (D_r^l k)(x),  D_r = x^-1 d/dx,
//   j_l(z)  = (z^-1 d/dz)^l (sinh z / z) = sum_k 2^l (k+l)!/(k!(2k+2l+1)!) z^{2k},
//
// whose integrand carries no cancelling alternating terms.  Each family
// (b, g, alpha_0 + j) of F_l contributes through the generating integrals
// S(alpha, beta, gamma) = int_0^inf x^alpha e^{beta x - gamma x^2} dx of
// Eq. sila with gamma = g + xi:
//
//  * z = (b + 2 xi D)^2 / (4 gamma) below a threshold that grows with l:
//    the small-Q series (Sec. 2.5.1, Eq. bidersmall, here with j_l in place
//    of the alternating D_Q expansion)
//      sum_j P_lj sum_k c_lk (2 xi D)^{2k} S(alpha_0 + j + 2k, b, gamma),
//    S on one alpha_0 + N family from two start values by the recursion of
//    Eq. Srec1 (upward in alpha; every term positive for beta >= 0), the
//    start values from Kummer's M (App. B, Eq. msmallz) in the form valid
//    for beta >= 0, and the finite part S(-1, beta, gamma) for the integer
//    family of the f_r f'_r kernel (Sec. 3.3.2);
//  * above it, Gauss-Hermite quadrature of the same integral about the
//    peak x* = (b + 2 xi D)/(2 gamma) of e^{(b + 2 xi D) x - gamma x^2}
//    (the moderate/large-Q case of Sec. 2.5.2; the r12 -> 0 end contributes
//    below double precision there).
//
// Families with b < 0 (a factor that decays exponentially, B < 0 in Eq. rs12,
// or a Ten-no-type term e^{-w r}): S(alpha, beta, gamma) with beta < 0 is the
// minimal solution of the alpha recursion (the Tricomi-U case of App. B), so
// the upward recursion above loses accuracy; and families whose lowest power
// is below -1 (a singular factor whose damping makes only the kernel as a
// whole integrable; the T_s functions of Sec. 3.3.1 for integer alpha): the
// non-peak orders of both are instead integrated directly by composite
// Gauss-Legendre quadrature of the same integral: singular families together
// with the families of the same b whose singular terms they cancel
// (group_quad), the others each as its Hadamard finite part (family_quad).
// Both run only in a second launch of the evaluation kernel (QUAD).
//
// The header also compiles as plain C++ (without nvcc) so that a CPU test can
// evaluate this stage against the oracle; the library itself only runs it on
// the GPU.
#pragma once

#ifdef __CUDACC__
#include <cuda_runtime.h>
#define F12_DEV __device__
#define F12_CONST __constant__
#define F12_GLOBAL __device__
#else
#include <algorithm>
#include <cmath>
#include <cstring>
#define F12_DEV
#define F12_CONST
#define F12_GLOBAL
#endif

namespace f12dev {

#ifndef __CUDACC__
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
using std::max;
using std::min;
using std::exp;
using std::fabs;
using std::fma;
using std::log;
using std::pow;
using std::sqrt;
#endif

constexpr int LAUX = 14;     // highest radial order (f shells, I5: 3+3+3+3+2)
constexpr int JMAX = 48;     // longest family polynomial
constexpr int WIN = 64;      // circular window over the S sequence (> JMAX + 2)
constexpr int KMAX = 400;    // series length cap (the longest series in use needs about 200 terms)
constexpr int NGH = 16;      // Gauss-Hermite nodes
constexpr int NGHF = 10;     // the shorter Gauss-Hermite rule, far from r = 0 (stored after the first)
constexpr int KTAB = 320;    // tabulated series coefficient ratios
constexpr int MAXFAM = 24;   // families per kernel
constexpr int NCLASS = 7;    // index by class 1..6
constexpr int NGL = 16;      // Gauss-Legendre nodes per panel (b < 0 families)
constexpr int NPMAX = 40;    // panels at most (the rule of family_quad needs about 30)
// Start values of the series: per family a table of J_{as+k}(y_i)/k!, k < JT_NK,
// on the grid y_i = i JT_DY, i < JT_NY (y = b/sqrt(gamma) <= 20 in the series
// region), evaluated by Taylor steps from the nearest point
constexpr int JT_NK = 17;
constexpr int JT_NY = 321;
constexpr double JT_DY = 1.0 / 16.0;

struct FamDev {
  double b, g;
  double alpha0;              // lowest power of F_l (a0 + 2)
  double gam_tab[JMAX];       // Gamma((alpha0 + 1 + j)/2); unused entry for alpha0 + 1 + j == 0
  double rho_start;           // Gamma((as+2)/2) / Gamma((as+1)/2), as = first regular alpha
  int fp_minus1;              // alpha0 == -1: the j = 0 term needs the finite part S(-1,...)
  int pow_kind;               // x^alpha0: 1 integer, 2 half-integer, 0 general
  int pow_int;                // integer part for pow_kind 1 and 2 (floor of alpha0)
  int quad;                   // b < 0 or alpha0 < -1: evaluated by family_quad (second launch)
  int nsing;                  // powers alpha0 + k <= -1 (k < nsing) taken as finite parts
  int group;                  // index of its GroupDev (families evaluated together), -1 none
  int lead;                   // the group's first member, which evaluates the whole group
  int jtab;                   // offset of its start-value table in Tables::jtab, -1 none
  int ktab;                   // 1: b = 0, integer alpha0 >= 0 and every a_j on the Kummer table's grid
  int ha_base;                // 2 alpha0 - 2: index of (alpha0 + m - 1)/2 in d_quarter is ha_base + 2m
  int ha_tab;                 // 1: that index stays inside d_quarter for every m of the series
  int jrow;                   // doubles per table row (JT_NK, or 2 JT_NK for a finite-part family)
  int span[LAUX + 1];
  int coff[LAUX + 1];         // offset of P_l in the coefficient pool
};

// Families with the same b and power lattice whose singular terms at r = 0
// cancel between them (the damped long range of Eq. rs12 with rho <= -1):
// evaluated together by group_quad.  Below xs each member's Gaussian is split
// as e^{-g x^2} = T_k(-g x^2) + R_k(g x^2), T_k its first k Taylor terms; the
// T_k parts of all members form one base polynomial, whose singular
// coefficients cancel exactly (the host builds it and zeroes them), and
// R_k = O(x^{2k}) leaves each member's rest integrable.
constexpr int MAXMEM = 8;
constexpr int KEXP = 6;      // remainder orders below this
struct GroupDev {
  double b, gmin, gmax, xs;   // common b; smallest and largest member g; split point 1/sqrt(gmax)
  double abase;               // lowest power of the group (the base polynomial's x^abase)
  int pow_kind, pow_int;      // of abase, as in FamDev
  int nmem;
  int mem[MAXMEM];            // member families (indices into Tables::fam)
  int kexp[MAXMEM];           // remainder order k of each member; -1: g = 0, wholly in the base
  int dpow[MAXMEM];           // alpha0 of the member minus abase (an integer)
  int bspan[LAUX + 1];        // base polynomial per order in the coefficient pool
  int boff[LAUX + 1];
};

struct Tables {
  int nfam[NCLASS];
  int fam0[NCLASS];
  const FamDev *fam;
  const double *coef;
  const GroupDev *grp;
  const double *jtab;         // start-value tables (FamDev::jtab)
  int kcap;                   // series length cap (KMAX; lowered only to test the status word)
};

F12_CONST double c_gh_x[NGH + NGHF];
F12_CONST double c_gh_w[NGH + NGHF];
F12_CONST double c_gl_x[NGL];   // Gauss-Legendre on [-1, 1]
F12_CONST double c_gl_w[NGL];
// c_{l,k+1}/c_{l,k} = (k+l+1) / ((k+1)(2k+2l+2)(2k+2l+3)),  c_{l,k} = 2^l (k+l)!/(k!(2k+2l+1)!)
// (the same ratios advance the power series of j_l)
F12_CONST double c_cratio[LAUX + 1][KTAB];
F12_CONST double c_inv_dfact[LAUX + 2];        // 1/(2l+1)!! = c_{l,0}
constexpr int NKUM = 512;
F12_GLOBAL double d_kum_inv[2][NKUM];             // 1/((b+n)(n+1)) for b = 1/2, 3/2
F12_GLOBAL double d_sm1_ratio[NKUM];              // Gamma((m+1)/2)/(Gamma(m/2)(m+1))
// The series coefficients c_{l,k} = 2^l (k+l)!/(k!(2k+2l+1)!) with a power of
// two that depends on k alone split off: c_{l,k} = d_cser[l][k] 2^{-E_k},
// E_k = -floor(log2 c_{0,k}) (so d_cser[0][k] lies in [1, 2)), and the step
// d_vstep[k] = 2^{E_k - E_{k+1}}.  Built in long double by the ratio
// recursion c_{l,k+1}/c_{l,k} = (k+l+1)/((k+1)(2k+2l+2)(2k+2l+3)).
F12_GLOBAL double d_cser[LAUX + 1][KMAX];
F12_GLOBAL double d_vstep[KMAX];
// d_quarter[i] = i/4: the coefficients (alpha0 + m - 1)/2 of the S recursion
// for integer and half-integer alpha0, read instead of being accumulated
constexpr int NQUARTER = 2 * (JMAX + 2 * KMAX) + 16;
F12_GLOBAL double d_quarter[NQUARTER];
// Families with b = 0 (Gaussian terms e^{-g r^2} x^alpha): S(alpha, 0, gamma) is
// a Gamma function, and the series of each order sums to a confluent
// hypergeometric (Kummer) function: with a_j = (alpha0 + j + 1)/2,
//   sum_k c_{l,k} v^k Gamma(a_j + k) = Gamma(a_j) c_{l,0} M(a_j, l + 3/2, x),  x = v/4,
// tabulated as T(a, l, x) = e^{-x} M(a, l + 3/2, x) on the grid x_i = i MT_DX,
// a = (ia + 1)/2, with MT_NT Taylor coefficients per point:
//   d^m T/dx^m = (-1)^m (b - a)_m / (b)_m  e^{-x} M(a, b + m, x),  b = l + 3/2.
constexpr int MT_NA = 40;            // a = 1/2 .. 20
constexpr int MT_NX = 201;           // x = 0 .. 100 (the series region: x < 36 + 4.5 l <= 99)
constexpr double MT_DX = 0.5;
constexpr int MT_NT = 14;            // Taylor terms: (DX/2)^14 / 14! < 1e-19
F12_GLOBAL const double *d_mtab;     // [l][ia][ix][m], built on the host (fill_kummer_table)

F12_DEV inline double threshold_z(int l) { return 36.0 + 4.5 * l; }
// The peak quadrature's integrand is x^alpha0 P_l(x) e^{-z} j_l(z) about a
// Gaussian of width 1/sqrt(gamma) centred at x*; relative to that width it
// varies on the scale sqrt(z)/(l + 1), so that the shorter rule suffices for
// orders l < ls once z is past this bound.
#ifndef F12_GHF_A
#define F12_GHF_A 60.0
#define F12_GHF_B 12.0
#endif
F12_DEV inline double few_nodes_z(int l) { return F12_GHF_A + F12_GHF_B * l; }
// ... and only up to this order: at higher orders the family sums cancel
// (k2 at xi = 10, D = 20, order 13), and the shorter rule's different
// rounding was measured to move the result by 1e-9 of itself there
constexpr int FEW_NODES_LMAX = 3;

// High 32 bits of a double (sign, exponent, top of the mantissa): integer
// comparisons of these stand in for floating-point tests that would
// otherwise take FP64 instructions.
F12_DEV inline int hi_word(double x) {
#ifdef __CUDA_ARCH__
  return __double2hiint(x);
#else
  long long b;
  std::memcpy(&b, &x, sizeof b);
  return (int)(b >> 32);
#endif
}
// biased binary exponent of |x| (0 for zero)
F12_DEV inline int exp_bits(double x) { return (hi_word(x) >> 20) & 0x7FF; }

// e^{-z} j_l(z) for l = 0..N (N <= LAUX): power series for the top two orders
// and the stable downward recurrence j_{l-1} = z^2 j_{l+1} + (2l+1) j_l for
// small z; closed forms of j_0, j_1 and the upward recurrence for large z.
F12_DEV inline void jhat_all(double z, int N, double *jh) {
  if (z > 2.0 * N + 30.0) {
    double e2 = z < 40.0 ? exp(-2.0 * z) : 0.0, iz = 1.0 / z;
    jh[0] = 0.5 * (1.0 - e2) * iz;
    if (N >= 1) jh[1] = 0.5 * ((1.0 - iz) + e2 * (1.0 + iz)) * iz * iz;
    for (int m = 1; m < N; ++m) jh[m + 1] = (jh[m - 1] - (2 * m + 1) * jh[m]) * iz * iz;
    return;
  }
  double z2 = z * z, ez = exp(-z);
  int mlo = N > 0 ? N - 1 : 0;
  for (int m = N; m >= mlo; --m) {
    double term = c_inv_dfact[m], s = 0.0;
    for (int k = 0; k < KTAB; ++k) {
      s += term;
      term *= z2 * c_cratio[m][k];
      if (term <= 1e-18 * s && k > 1) break;
    }
    jh[m] = ez * s;
  }
  for (int m = N - 1; m >= 1; --m) jh[m - 1] = z2 * jh[m + 1] + (2 * m + 1) * jh[m];
}

// Kummer M(a, b, z), z >= 0, a > 0, b = 1/2 (ib = 0) or 3/2 (ib = 1) (App. B, Eq. msmallz).
F12_DEV inline double kummer_m(double a, int ib, double z, int *bad) {
  double t = 1.0, s = 1.0;
  if (z == 0.0) return 1.0;
  for (int n = 0; n < NKUM; ++n) {
    t *= (a + n) * z * d_kum_inv[ib][n];
    s += t;
    if (t <= 1e-18 * s) return s;
  }
  *bad = 1;
  return s;
}

// Normalised scaled generating integral
//   Jh_alpha(y) = [int_0^inf t^alpha e^{y t - t^2} dt] / Gamma((alpha+1)/2),  y >= 0,
// from the Kummer form  J = 1/2 [Gamma((a+1)/2) M((a+1)/2, 1/2, y^2/4)
//                               + y Gamma((a+2)/2) M((a+2)/2, 3/2, y^2/4)].
// rho = Gamma((alpha+2)/2)/Gamma((alpha+1)/2).
F12_DEV inline double jhat_start(double alpha, double rho, double y, int *bad) {
  double z = 0.25 * y * y;
  if (y == 0.0) return 0.5;
  return 0.5 * (kummer_m(0.5 * (alpha + 1.0), 0, z, bad) + y * rho * kummer_m(0.5 * (alpha + 2.0), 1, z, bad));
}

// Finite part S(-1, b, gamma) (Sec. 3.3.2, integer alpha; Eq. sila):
//   = -gamma_E/2 - log(gamma)/2 + 1/2 sum_{m>=1} y^m Gamma(m/2)/m!,  y = b/sqrt(gamma) >= 0.
F12_DEV inline double s_minus1(double b, double gam, int *bad) {
  const double euler = 0.57721566490153286061;
  double y = b / sqrt(gam);
  double s = -0.5 * euler - 0.5 * log(gam);
  if (y > 0.0) {
    // t_m = y^m Gamma(m/2) / (2 m!);  t_1 = y sqrt(pi)/2;
    // t_{m+1}/t_m = y Gamma((m+1)/2) / (Gamma(m/2) (m+1))  (tabulated)
    double t = 0.5 * y * 1.77245385090551602730;
    double acc = 0.0;
    for (int m = 1; m < NKUM; ++m) {
      acc += t;
      t *= y * d_sm1_ratio[m];
      if (t <= 1e-18 * acc && m > 2) {
        s += acc;
        return s;
      }
    }
    *bad = 1;
    s += acc;
  }
  return s;
}

// Orders l = l0..L of a family evaluated by quadrature (b < 0, or a lowest
// power alpha0 < -1), added into out[l] times fct[l]:
//   I_l = int_0^inf x^alpha0 u_l(x) dx,
//   u_l(x) = P_l(x) e^{b x - g x^2 - xi (x - D)^2} jhat_l(2 xi D x) = e^{-gamma x^2} v_l(x),
//   v_l(x) = e^{-xi D^2} P_l(x) e^{b x} j_l(2 xi D x),
// the integral of the header written with e^{-xi x^2 - xi D^2} j_l(2 xi D x)
// = e^{-xi (x - D)^2} jhat_l(2 xi D x), by composite Gauss-Legendre quadrature.
// With beta = b + 2 xi D, gamma = g + xi and d the highest power of the
// integrand, the integrand is below e^{-40} of its largest value past
//   beta > 0:  hi = beta/(2 gamma) + (sqrt(d/2) + 6.5)/sqrt(gamma)
//              (about the peak of e^{beta x - gamma x^2}, moved out by x^d);
//   beta <= 0: hi = (sqrt(d/2) + 6.5)/sqrt(gamma), and for beta < 0 at most
//              (d + 9 sqrt(d) + 45)/|beta| (the tail of x^d e^{-|beta| x}).
// A panel starting at a is 1.25/max(sqrt(gamma), |beta|/sqrt(max(1, |beta| a)))
// wide: about two widths of the Gaussian, or of the bump x^m e^{-|beta| x}
// that peaks near a (twice that width left errors up to 1e-8 at l = 5).  On
// the first panel a half-integer power is integrated in u = sqrt(x)
// (x^{n+1/2} dx = 2 u^{2n+2} du).
// End point: the powers alpha0 + k <= -1 (k < K = nsing) are not integrable
// one family at a time.  Their sum over the kernel's families cancels (the
// host refuses a kernel where it does not), so each family's integral is
// taken as its Hadamard finite part (Sec. 3.3.2 for alpha = -1; the integer
// alpha <= -1 cases of Sec. 3.3.1), and the finite parts add up to the
// kernel's integral:
//   FP I_l = int_0^inf x^alpha0 [u_l(x) - e^{-lam x^2} sum_{k<K} t_k x^k] dx
//            + sum_{k<K} t_k M(alpha0 + k),
// t_k the Taylor coefficients of u_l(x) e^{lam x^2} = v_l(x) e^{(lam - gamma) x^2}
// at 0, and M(beta) the finite part of int_0^inf x^beta e^{-lam x^2} dx:
// Gamma((beta+1)/2) / (2 lam^{(beta+1)/2}), or for beta = -1 - 2m (a pole of
// Gamma) (lam^m/2) ((-1)^m/m!) (psi(m+1) - log lam), what is left of
// int_eps^inf after the powers of eps and log eps are dropped (m = 0 is the
// convention of s_minus1).  The regulator e^{-lam x^2} is free; lam =
// max(gamma, (6.5/hi)^2) makes the subtracted terms end with the range too
// (with lam = gamma they would reach past hi where beta < 0 ends it early).
// Singular powers per family at most: alpha0 >= -2.  Below that the per-family
// finite parts cancel too strongly in FP64 (for alpha0 = -2.5 and -3 the
// errors reached 1e-5 against the oracle), and the host refuses the class.
constexpr int KSING = 2;

F12_DEV inline int family_quad(const Tables &T, const FamDev &F, double xi, double D, int l0, int L,
                               const double *fct, double *out, unsigned long long *nfma) {
  const double gam = F.g + xi, sg = sqrt(gam);
  const double beta = F.b + 2.0 * xi * D;
  int spmax = 0;
  for (int l = l0; l <= L; ++l) spmax = F.span[l] > spmax ? F.span[l] : spmax;
  const double d = fmax(0.0, F.alpha0 + (double)(spmax - 1));
  double hi;
  if (beta > 0.0) {
    hi = 0.5 * beta / gam + (sqrt(0.5 * d) + 6.5) / sg;
  } else {
    hi = (sqrt(0.5 * d) + 6.5) / sg;
    if (beta < 0.0) hi = fmin(hi, (d + 9.0 * sqrt(d) + 45.0) / -beta);
  }
  const double edd = exp(-xi * D * D);
  const double twoxd = 2.0 * xi * D;
  const int K = F.nsing < KSING ? F.nsing : KSING;
  const double lam = K > 0 ? fmax(gam, (6.5 / hi) * (6.5 / hi)) : gam;
  // Taylor coefficients t_k (k < K) of P_l e^{b x} e^{(lam - gamma) x^2} j_l(2 xi D x) e^{-xi D^2}
  double tc[LAUX + 1][KSING];
  if (K > 0) {
    double eb[KSING];                        // e^{b x} e^{(lam - gamma) x^2}
    {
      double e1[KSING];
      e1[0] = 1.0;
      for (int k = 1; k < K; ++k) e1[k] = e1[k - 1] * F.b / k;
      const double dl = lam - gam;
      for (int k = 0; k < K; ++k) eb[k] = 0.0;
      double em = 1.0;                       // (lam - gamma)^m / m!
      for (int m = 0; 2 * m < K; ++m) {
        for (int k = 2 * m; k < K; ++k) eb[k] = fma(em, e1[k - 2 * m], eb[k]);
        em *= dl / (m + 1);
      }
    }
    for (int l = l0; l <= L; ++l) {
      double q[KSING];                       // eb times j_l(2 xi D x)
      for (int k = 0; k < K; ++k) q[k] = 0.0;
      double cj = c_inv_dfact[l];            // c_{l,m} (2 xi D)^{2m}
      for (int m = 0; 2 * m < K; ++m) {
        for (int k = 2 * m; k < K; ++k) q[k] = fma(cj, eb[k - 2 * m], q[k]);
        cj *= c_cratio[l][m] * twoxd * twoxd;
      }
      const double *P = T.coef + F.coff[l];
      for (int k = 0; k < K; ++k) {
        double t = 0.0;
        for (int i = 0; i <= k && i < F.span[l]; ++i) t = fma(P[i], q[k - i], t);
        tc[l][k] = edd * t;
      }
    }
  }
  double acc[LAUX + 1], jh[LAUX + 2];
  for (int l = l0; l <= L; ++l) acc[l] = 0.0;
  unsigned long long n = 0;
  double a = 0.0;
  int stretched = 0;
  const double sl = sqrt(lam);
  for (int p = 0; p < NPMAX && a < hi; ++p) {
    double r = 0.0;
    if (beta < 0.0) r = -beta / sqrt(fmax(1.0, -beta * a));
    const double w = 1.25 / fmax(sl, r);
    // the last panel reaches hi (flagged if that makes it wider than the rule)
    if (p == NPMAX - 1 && hi - a > w) stretched = 1;
    const double hw = 0.5 * (p == NPMAX - 1 ? fmax(w, hi - a) : w);
    const bool usq = (p == 0 && F.pow_kind == 2);
    const double su = usq ? sqrt(2.0 * hw) : 0.0;
    for (int i = 0; i < NGL; ++i) {
      double x, wt;
      if (usq) {                       // x = u^2, u in [0, sqrt(2 hw)]
        const double u = 0.5 * su * (c_gl_x[i] + 1.0);
        x = u * u;
        wt = 0.5 * su * c_gl_w[i] * 2.0 * u;
      } else {
        x = a + hw * (c_gl_x[i] + 1.0);
        wt = hw * c_gl_w[i];
      }
      const double ex = exp(F.b * x - F.g * x * x - xi * (x - D) * (x - D));
      jhat_all(twoxd * x, L, jh);
      double xa;                       // x^alpha0
      if (F.pow_kind == 0) {
        xa = pow(x, F.alpha0);
      } else {
        xa = F.pow_kind == 2 ? sqrt(x) : 1.0;
        if (F.pow_int >= 0) {
          for (int k = 0; k < F.pow_int; ++k) xa *= x;
        } else {
          const double ix = 1.0 / x;
          for (int k = 0; k < -F.pow_int; ++k) xa *= ix;
        }
      }
      const double es = K > 0 ? exp(-lam * x * x) : 0.0;
      for (int l = l0; l <= L; ++l) {
        const double *P = T.coef + F.coff[l];
        const int sp = F.span[l];
        double h = 0.0;
        for (int j = sp - 1; j >= 0; --j) h = fma(h, x, P[j]);
        double v = ex * jh[l] * h;
        if (K > 0) {
          double tk = 0.0;
          for (int k = K - 1; k >= 0; --k) tk = fma(tk, x, tc[l][k]);
          v = fma(-es, tk, v);
        }
        acc[l] = fma(wt * xa, v, acc[l]);
        n += sp + K + 1;
      }
    }
    a += 2.0 * hw;
  }
  // finite parts of the subtracted terms
  for (int k = 0; k < K; ++k) {
    const double bk = F.alpha0 + k;
    double M;
    const double mm = -0.5 * (bk + 1.0);
    if (F.pow_kind == 1 && mm >= 0.0 && fabs(mm - floor(mm + 0.5)) < 1e-9) {   // beta = -1 - 2m
      const int m = (int)floor(mm + 0.5);
      double psi = -0.57721566490153286061, fact = 1.0, gm = 1.0;
      for (int i = 1; i <= m; ++i) {
        psi += 1.0 / i;
        fact *= i;
        gm *= lam;
      }
      M = 0.5 * gm * ((m & 1) ? -1.0 : 1.0) / fact * (psi - log(lam));
    } else {
      M = 0.5 * F.gam_tab[k] * pow(lam, -0.5 * (bk + 1.0));
    }
    for (int l = l0; l <= L; ++l) acc[l] = fma(tc[l][k], M, acc[l]);
  }
  for (int l = l0; l <= L; ++l) out[l] += fct[l] * acc[l];
  if (nfma) *nfma += n;
  return stretched;
}

// Orders l < ls of one family by Gauss-Hermite quadrature about the peak
// (see the header), added into out[l] times fct[l].
template <bool QUAD>
F12_DEV inline void family_gh(const Tables &T, const FamDev &F, double xi, double D, int ls, const double *fct,
                              double *out, unsigned long long &nfma) {
  const double gam = F.g + xi;
  const double beta = F.b + 2.0 * xi * D;
  const double sg = sqrt(gam), isg = 1.0 / sg;
  const double xs = beta / (2.0 * gam);
  const double estar = (F.b * F.b + 4.0 * F.b * xi * D - 4.0 * F.g * xi * D * D) / (4.0 * gam);
  const double pre = exp(estar) * isg;
  double acc[LAUX + 1];
  for (int l = 0; l < ls; ++l) acc[l] = 0.0;
  double jh[LAUX + 2];
  const double twoxd = 2.0 * xi * D;
  // (not for the powers below -1 that the quadrature launch also takes here)
  const bool few = !QUAD && ls <= FEW_NODES_LMAX + 1 && beta * beta / (4.0 * gam) >= few_nodes_z(ls - 1);
  const int i0 = few ? NGH : 0, i1 = few ? NGH + NGHF : NGH;
  for (int i = i0; i < i1; ++i) {
    const double x = xs + c_gh_x[i] * isg;
    if (x <= 0.0) continue;
    jhat_all(twoxd * x, ls - 1, jh);
    double xa;
    if constexpr (QUAD) {           // any power (a grouped member's may be below -2)
      if (F.pow_kind == 0) {
        xa = pow(x, F.alpha0);
      } else {
        xa = F.pow_kind == 2 ? sqrt(x) : 1.0;
        if (F.pow_int >= 0) {
          for (int k = 0; k < F.pow_int; ++k) xa *= x;
        } else {
          const double ix = 1.0 / x;
          for (int k = 0; k < -F.pow_int; ++k) xa *= ix;
        }
      }
    } else if (F.pow_kind == 1) {   // alpha0 = integer n0
      xa = 1.0;
      for (int k = 0; k < F.pow_int; ++k) xa *= x;
      if (F.pow_int < 0) xa = 1.0 / x;  // only alpha0 = -1 occurs
    } else if (F.pow_kind == 2) {   // alpha0 = n0 + 1/2
      xa = sqrt(x);
      for (int k = 0; k < F.pow_int; ++k) xa *= x;
      if (F.pow_int < 0) xa /= x;     // alpha0 = -1/2
    } else {
      xa = pow(x, F.alpha0);
    }
    xa *= c_gh_w[i];
    for (int l = 0; l < ls; ++l) {
      const double *P = T.coef + F.coff[l];
      const int sp = F.span[l];
      double h = 0.0;
      for (int j = sp - 1; j >= 0; --j) h = fma(h, x, P[j]);
      acc[l] = fma(xa * jh[l], h, acc[l]);
      nfma += sp + 1;
    }
  }
  for (int l = 0; l < ls; ++l) out[l] += fct[l] * pre * acc[l];
}

// R_k(y) = e^{-y} - sum_{i<k} (-y)^i/i!, 0 <= y: for y < 1 from its own series
// (terms decreasing, no cancellation), else directly.
F12_DEV inline double exp_rem(double y, int k) {
  if (k == 0) return exp(-y);
  if (y < 1.0) {
    double t = 1.0;
    for (int i = 1; i <= k; ++i) t *= -y / i;
    double s = 0.0;
    for (int i = k; i < k + 40; ++i) {
      s += t;
      t *= -y / (i + 1);
      if (fabs(t) <= 1e-17 * fabs(s)) break;
    }
    return s;
  }
  double s = 0.0, t = 1.0;
  for (int i = 0; i < k; ++i) {
    s += t;
    t *= -y / (i + 1);
  }
  return exp(-y) - s;
}

// Orders l0..L of a group of families (GroupDev) by composite Gauss-Legendre
// quadrature of their sum,
//   int_0^inf e^{b x - xi (x - D)^2} jhat_l(2 xi D x) sum_m x^{a_m} P_{m,l}(x) e^{-g_m x^2} dx,
// whose integrand is regular at x = 0 although its members are not.  Below
// xs the sum is evaluated as x^abase B_l(x) + sum_m x^{a_m} P_{m,l}(x) R_{k_m}(g_m x^2)
// (B_l the base polynomial; members with g = 0 are wholly in it), so that the
// singular terms have cancelled in B_l's coefficients on the host; above xs,
// where nothing is singular, member by member.  Range and panels as in
// family_quad, with the widest Gaussian (gmin) setting the range and the
// narrowest (gmax) the panels while it is still significant.
F12_DEV inline int group_quad(const Tables &T, const GroupDev &G, double xi, double D, int l0, int L,
                              const double *fct, double *out, unsigned long long *nfma) {
  const double gam = G.gmin + xi, sg = sqrt(gam), sgx = sqrt(G.gmax + xi);
  const double beta = G.b + 2.0 * xi * D;
  int dmax = 0;
  for (int m = 0; m < G.nmem; ++m) {
    const FamDev &F = T.fam[G.mem[m]];
    for (int l = l0; l <= L; ++l) dmax = G.dpow[m] + F.span[l] - 1 > dmax ? G.dpow[m] + F.span[l] - 1 : dmax;
  }
  const double d = fmax(0.0, G.abase + (double)dmax);
  double hi;
  if (beta > 0.0) {
    hi = 0.5 * beta / gam + (sqrt(0.5 * d) + 6.5) / sg;
  } else {
    hi = (sqrt(0.5 * d) + 6.5) / sg;
    if (beta < 0.0) hi = fmin(hi, (d + 9.0 * sqrt(d) + 45.0) / -beta);
  }
  const double twoxd = 2.0 * xi * D;
  const double narrow = 6.5 / sgx;   // the largest-g members are negligible beyond
  double acc[LAUX + 1], jh[LAUX + 2], xm[MAXMEM], fm[MAXMEM];
  for (int l = l0; l <= L; ++l) acc[l] = 0.0;
  unsigned long long n = 0;
  double a = 0.0;
  int stretched = 0;
  for (int p = 0; p < NPMAX && a < hi; ++p) {
    double r = 0.0;
    if (beta < 0.0) r = -beta / sqrt(fmax(1.0, -beta * a));
    const double w = 1.25 / fmax(a < narrow ? sgx : sg, r);
    if (p == NPMAX - 1 && hi - a > w) stretched = 1;
    const double hw = 0.5 * (p == NPMAX - 1 ? fmax(w, hi - a) : w);
    const bool usq = (p == 0 && G.pow_kind == 2);
    const double su = usq ? sqrt(2.0 * hw) : 0.0;
    for (int i = 0; i < NGL; ++i) {
      double x, wt;
      if (usq) {
        const double u = 0.5 * su * (c_gl_x[i] + 1.0);
        x = u * u;
        wt = 0.5 * su * c_gl_w[i] * 2.0 * u;
      } else {
        x = a + hw * (c_gl_x[i] + 1.0);
        wt = hw * c_gl_w[i];
      }
      const double ex = exp(G.b * x - xi * (x - D) * (x - D));
      jhat_all(twoxd * x, L, jh);
      double xb = G.pow_kind == 2 ? sqrt(x) : 1.0;   // x^abase
      if (G.pow_int >= 0) {
        for (int k = 0; k < G.pow_int; ++k) xb *= x;
      } else {
        const double ix = 1.0 / x;
        for (int k = 0; k < -G.pow_int; ++k) xb *= ix;
      }
      const bool split = x < G.xs;
      for (int m = 0; m < G.nmem; ++m) {
        double xp = xb;
        for (int k = 0; k < G.dpow[m]; ++k) xp *= x;
        xm[m] = xp;
        const double gm = T.fam[G.mem[m]].g;
        fm[m] = split ? (G.kexp[m] < 0 ? 0.0 : exp_rem(gm * x * x, G.kexp[m])) : exp(-gm * x * x);
      }
      const double e = wt * ex;
      for (int l = l0; l <= L; ++l) {
        double v = 0.0;
        if (split) {
          const double *B = T.coef + G.boff[l];
          double h = 0.0;
          for (int j = G.bspan[l] - 1; j >= 0; --j) h = fma(h, x, B[j]);
          v = xb * h;
          n += G.bspan[l];
        }
        for (int m = 0; m < G.nmem; ++m) {
          if (fm[m] == 0.0) continue;
          const FamDev &F = T.fam[G.mem[m]];
          const double *P = T.coef + F.coff[l];
          double h = 0.0;
          for (int j = F.span[l] - 1; j >= 0; --j) h = fma(h, x, P[j]);
          v = fma(xm[m] * fm[m], h, v);
          n += F.span[l] + 1;
        }
        acc[l] = fma(e * jh[l], v, acc[l]);
      }
    }
    a += 2.0 * hw;
  }
  for (int l = l0; l <= L; ++l) out[l] += fct[l] * acc[l];
  if (nfma) *nfma += n;
  return stretched;
}

// A group: orders whose every member has its peak well inside (0, inf) are
// taken member by member about the peak (family_gh; the r -> 0 end is below
// double precision there for each of them), the rest by group_quad.
F12_DEV inline int group_eval(const Tables &T, const GroupDev &G, double xi, double D, int L, const double *fct,
                              double *out, unsigned long long &nfma) {
  const double beta = G.b + 2.0 * xi * D;
  int ls = 0;
  if (beta > 0.0) {
    ls = L + 1;
    for (int m = 0; m < G.nmem; ++m) {
      const double z = beta * beta / (4.0 * (T.fam[G.mem[m]].g + xi));
      int lm = 0;
      while (lm <= L && z >= threshold_z(lm)) ++lm;
      ls = lm < ls ? lm : ls;
    }
  }
  if (ls > 0)
    for (int m = 0; m < G.nmem; ++m) family_gh<true>(T, T.fam[G.mem[m]], xi, D, ls, fct, out, nfma);
  return ls <= L ? group_quad(T, G, xi, D, ls, L, fct, out, &nfma) : 0;
}

// Contribution of one family to hat g_l, l = 0..L, added into out[] with the
// common factor 4 xi (2 xi)^l applied.  Returns nonzero if a series did not
// converge within KMAX terms.  QUAD: a family with b < 0 or alpha0 < -1
// (FamDev::quad), whose non-peak orders go to family_quad (kept out of the
// other instantiation, which the main evaluation kernel uses, so that its
// register budget is unchanged).
template <bool QUAD = false>
F12_DEV inline int family_eval(const Tables &T, const FamDev &F, double xi, double D, int L, double *out,
                               unsigned long long *fma_count = nullptr) {
  int bad = 0;
  unsigned long long nfma = 0;
  const double gam = F.g + xi;
  const double beta = F.b + 2.0 * xi * D;
  const double z = beta * beta / (4.0 * gam);
  if constexpr (QUAD) {
    if (F.group >= 0) {            // the group's first member evaluates the whole group
      if (!F.lead) return 0;
      double fct[LAUX + 1];
      fct[0] = 4.0 * xi;
      for (int l = 1; l <= L; ++l) fct[l] = fct[l - 1] * 2.0 * xi;
      bad = group_eval(T, T.grp[F.group], xi, D, L, fct, out, nfma);
      if (fma_count) *fma_count += nfma;
      return bad;
    }
  }
  // orders l < ls use the quadrature about the peak, l >= ls the series (or,
  // for a family on the Kummer table, the table wherever x = z lies in its
  // range: it is exact there, with no r -> 0 argument to satisfy)
  int ls = 0;
  const bool ktab = !QUAD && F.ktab && z < (MT_NX - 1) * MT_DX;
  if (!ktab && (!QUAD || beta > 0.0))   // beta <= 0 (b < 0): no peak inside (0, inf)
    while (ls <= L && z >= threshold_z(ls)) ++ls;
  double fct[LAUX + 1];
  fct[0] = 4.0 * xi;
  for (int l = 1; l <= L; ++l) fct[l] = fct[l - 1] * 2.0 * xi;

  if (ls > 0) family_gh<QUAD>(T, F, xi, D, ls, fct, out, nfma);

  if constexpr (QUAD) {
    if (ls <= L) bad |= family_quad(T, F, xi, D, ls, L, fct, out, &nfma);
  } else if (ktab) {
    // b = 0: each order from the Kummer table,
    //   sum_l = e^{-xi g D^2 / gamma} gamma^{-(alpha0+1)/2} c_{l,0}/2
    //           sum_j P_lj gamma^{-j/2} Gamma(a_j) T(a_j, l, x),  x = z = xi^2 D^2 / gamma
    const double rgam = rsqrt(gam);
    double gpow0 = 1.0;                    // gamma^{-(alpha0+1)/2}, alpha0 = pow_int >= 0
    for (int k = 0; k < F.pow_int + 1; ++k) gpow0 *= rgam;
    const double E = exp(-xi * F.g * D * D / gam) * gpow0 * 0.5;
    const double xt = z * (1.0 / MT_DX);
    const double ri = rint(xt);
    const double h = (xt - ri) * MT_DX;
    const int ix = (int)ri;
    const int ia0 = F.pow_int;             // a_j = (alpha0 + j + 1)/2 is grid point alpha0 + j
    for (int l = ls; l <= L; ++l) {
      const double *P = T.coef + F.coff[l];
      const double *rowl = d_mtab + ((size_t)l * MT_NA * MT_NX + ix) * MT_NT;
      double s = 0.0, gp = 1.0;
      for (int j = 0; j < F.span[l]; ++j) {
        const double *row = rowl + (size_t)(ia0 + j) * MT_NX * MT_NT;
        double t = row[MT_NT - 1];
        for (int m = MT_NT - 2; m >= 0; --m) t = fma(t, h, row[m]);
        s = fma(P[j] * gp * F.gam_tab[j], t, s);
        gp *= rgam;
      }
      out[l] += fct[l] * E * c_inv_dfact[l] * s;
      nfma += (unsigned long long)F.span[l] * (MT_NT + 1);
    }
  } else if (ls <= L) {
    const double y = F.b * rsqrt(gam);
    const double v = 4.0 * xi * xi * D * D / gam;
    const double eT = exp(-xi * D * D);
    const double rgam = rsqrt(gam);
    const int m0 = F.fp_minus1 ? 1 : 0;      // first regular index of the S family
    const double as = F.alpha0 + m0;
    // unnormalised start values J_{as}, J_{as+1} (J_alpha = int t^alpha e^{yt - t^2} dt)
    double J0, J1, sm1 = 0.0;
    const double yt = y * (1.0 / JT_DY);
    if (F.jtab >= 0 && yt < JT_NY - 0.5) {
      // Taylor steps from the nearest grid point: with e_k = J_{as+k}(y_i)/k!,
      // J_{as}(y_i + h) = sum_k e_k h^k and J_{as+1} = dJ_{as}/dy its derivative
      const double r = rint(yt);
      const double h = (yt - r) * JT_DY;
      const double *row = T.jtab + F.jtab + (int)r * F.jrow;
      double p = row[JT_NK - 1], dp = 0.0;
      for (int kk = JT_NK - 2; kk >= 0; --kk) {
        dp = fma(dp, h, p);
        p = fma(p, h, row[kk]);
      }
      J0 = p;
      J1 = dp;
      if (F.fp_minus1) {
        // the y-series of S(-1, b, gamma) (s_minus1): its Taylor coefficients
        // follow the J row (constant term, then JT_NK - 1 more)
        const double *tr = row + JT_NK;
        double t = tr[JT_NK - 1];
        for (int kk = JT_NK - 2; kk >= 0; --kk) t = fma(t, h, tr[kk]);
        sm1 = -0.5 * 0.57721566490153286061 - 0.5 * log(gam) + t;
      }
    } else {
      const double rho1 = 0.5 * (as + 1.0) / F.rho_start;
      J0 = jhat_start(as, F.rho_start, y, &bad) * F.gam_tab[m0];
      J1 = jhat_start(as + 1.0, rho1, y, &bad) * F.gam_tab[m0 + 1];
      if (F.fp_minus1) sm1 = s_minus1(F.b, gam, &bad);
    }
    // gamma^{-(alpha0+1)/2}: products of rsqrt for integer and half-integer alpha0
    double gpow0;
    if (F.pow_kind == 1) {                 // (alpha0+1)/2 = (n0+1)/2: powers of gamma^{-1/2}
      gpow0 = 1.0;
      for (int k = 0; k < F.pow_int + 1; ++k) gpow0 *= rgam;
      if (F.pow_int + 1 < 0) gpow0 = 1.0;  // alpha0 = -1: gamma^0
    } else if (F.pow_kind == 2) {          // (alpha0+1)/2 = (2 n0 + 3)/4: powers of gamma^{-1/4}
      const double r4 = sqrt(rgam);
      gpow0 = 1.0;
      for (int k = 0; k < 2 * F.pow_int + 3; ++k) gpow0 *= r4;
    } else {
      gpow0 = pow(gam, -0.5 * (F.alpha0 + 1.0));
    }
    const double TWO600 = 4.149515568880993e+180, MTWO600 = 2.409919865102884e-181;
    constexpr int HI_2P600 = (1023 + 600) << 20;   // high word of 2^600

    // all orders l = ls..L advance together over the series index k: the S
    // window is extended once per k, each order adds one FMA per coefficient
    constexpr int QMAX = 512;
    double qv[QMAX];
    int qoff[LAUX + 2];
    double sum[LAUX + 1];
    int tot = 0;
    for (int l = ls; l <= L; ++l) {
      qoff[l] = tot;
      tot += F.span[l];
    }
    qoff[L + 1] = tot;
    if (tot > QMAX) {
      bad = 1;
    } else {
      for (int l = ls; l <= L; ++l) {
        const double *P = T.coef + F.coff[l];
        double gp = gpow0;
        for (int j = 0; j < F.span[l]; ++j) {
          qv[qoff[l] + j] = P[j] * gp;
          gp *= rgam;
        }
        sum[l] = F.fp_minus1 ? qv[qoff[l]] * (c_inv_dfact[l] * eT) * sm1 : 0.0;   // c_{l,0} e^{-xi D^2} S(-1)
      }
      const int spmax = F.span[L];
      double win[WIN];
      win[m0 & (WIN - 1)] = J0;
      win[(m0 + 1) & (WIN - 1)] = J1;
      int mfill = m0 + 2;
      // J_m = (y/2) J_{m-1} + ((alpha0 + m - 1)/2) J_{m-2}: hy and ha, the
      // latter advanced by 1/2 per step (exact for integer and half-integer
      // alpha0, recomputed otherwise)
      const double hy = 0.5 * y;
      // the k-dependence every order shares: Vk = e^{-xi D^2} v^k 2^{-E_k}, so
      // that term_{l,k} = d_cser[l][k] Vk sum_j q_j J_{j+2k}
      double Vk = eT;
      // convergence: the terms of the lowest and highest order fall below
      // 2^-56 of the largest term so far, twice (exponent comparisons)
      int emax_lo = 0, emax_hi = 0;
      int small = 0;
      const int kmin = (int)(0.5 * v) + 2;   // past the largest term (terms ~ z^k/k!)
      int k;
      const int kcap = T.kcap > 0 && T.kcap < KMAX ? T.kcap : KMAX;
      for (k = 0; k < kcap; ++k) {
        const int need = spmax - 1 + 2 * k;
        int hmax = 0;
        while (mfill <= need) {
          // J_m = (y/2) J_{m-1} + ((alpha0 + m - 1)/2) J_{m-2}
          const double ha = F.ha_tab ? d_quarter[F.ha_base + 2 * mfill] : 0.5 * (F.alpha0 + (double)(mfill - 1));
          const double jn = fma(hy, win[(mfill - 1) & (WIN - 1)], ha * win[(mfill - 2) & (WIN - 1)]);
          win[mfill & (WIN - 1)] = jn;
          hmax = max(hmax, hi_word(jn));
          ++mfill;
        }
        if (hmax > HI_2P600) {   // keep the window in range; exact power-of-two rescale
          for (int r = mfill - WIN; r < mfill; ++r)
            if (r >= 0) win[r & (WIN - 1)] *= MTWO600;
          Vk *= TWO600;
        }
        const int jlo = (F.fp_minus1 && k == 0) ? 1 : 0;
        int e_lo = 0, e_hi = 0;
        for (int l = ls; l <= L; ++l) {
          const double *q = qv + qoff[l];
          const int sp = F.span[l];
          double part = 0.0;
          for (int j = jlo; j < sp; ++j) part = fma(q[j], win[(j + 2 * k) & (WIN - 1)], part);
          const double cv = d_cser[l][k] * Vk;
          sum[l] = fma(cv, part, sum[l]);
          // binary exponent of the term cv part (within one), 0 for a zero part
          const int ep = exp_bits(part);
          const int e = ep ? ep + exp_bits(cv) : 0;
          if (l == ls) e_lo = e;
          if (l == L) e_hi = e;
          nfma += sp - jlo + 2;
        }
        Vk *= v * d_vstep[k];
        emax_lo = max(emax_lo, e_lo);
        emax_hi = max(emax_hi, e_hi);
        // (a zero or subnormal term counts as small)
        small = ((e_lo + 57 < emax_lo || e_lo == 0) && (e_hi + 57 < emax_hi || e_hi == 0)) ? small + 1 : 0;
        if (small >= 2 && k >= kmin) break;
      }
      if (k == kcap) bad = 1;
      for (int l = ls; l <= L; ++l) out[l] += fct[l] * sum[l];
    }
  }
  if (fma_count) *fma_count += nfma;
  return bad;
}

// hat g_l for l = 0..L of the kernel of class kcls (sum over its families).
F12_DEV inline int aux_eval(const Tables &T, int kcls, double xi, double D, int L, double *out) {
  for (int l = 0; l <= L; ++l) out[l] = 0.0;
  int bad = 0;
  const int nf = T.nfam[kcls];
  const FamDev *fams = T.fam + T.fam0[kcls];
  for (int f = 0; f < nf; ++f)
    bad |= fams[f].quad ? family_eval<true>(T, fams[f], xi, D, L, out) : family_eval<false>(T, fams[f], xi, D, L, out);
  return bad;
}

// Work-item key used to order (primitive quartet, family) items so that a
// warp runs the same branch with a similar series length: family, total
// order L, and a bin of z (series by z/2, then the quadrature/series split).
F12_DEV inline int item_bin(const FamDev &F, double xi, double D, int L) {
  const double gam = F.g + xi;
  const double beta = F.b + 2.0 * xi * D;
  const double z = beta * beta / (4.0 * gam);
  if (z < threshold_z(0)) return (int)(0.5 * z);            // 0..17
  int ls = 0;
  while (ls <= L && z >= threshold_z(ls)) ++ls;
  return 18 + ls;                                             // 19..33
}
constexpr int NZBIN = 34;

}  // namespace f12dev
