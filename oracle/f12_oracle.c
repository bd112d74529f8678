/*
 * f12_oracle.c -- CPU oracle for the range-separated F12 two-electron integrals.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * What it computes is the plain definition of the integrals of Silkowski,
 * Lesiuk and Moszynski, "Calculation of the molecular integrals with the
 * range-separated correlation factor" (arXiv:1412.5070):
 *
 *   - primitives are unnormalised Cartesian Gaussians (Sec. 2.1, Eq. basis);
 *   - the six classes I1..I6 (Sec. 2.1, Eqs. I1-I6) with the kernels k1..k6
 *     (Sec. 2.2, Eqs. k1-k6); I5 through Green's identity (Eq. I5_) as
 *     I5 = 1/2 [ (lap a, b|f|c d) - (a, lap b|f|c d) ], i.e. the kinetic-energy
 *     transform of I3 applied to the Cartesian functions themselves;
 *     I6 with the commutator reduced to f_r f'_r (Eq. I6_);
 *   - the correlation factor of Eq. rs12 with the Tang-Toennies damping of
 *     Eq. ttdamp, evaluated pointwise, or any factor given as a sum of terms
 *     c r^a exp(b r - g r^2) (the Ten-no factor, Gaussian geminals), from
 *     which the six kernels are formed as Eqs. k1-k6 and I6_ define them;
 *   - the Hermite expansion of Eq. AB / Eq. Lambda, with the E coefficients
 *     obtained by direct binomial expansion about P followed by the
 *     monomial -> Hermite-function conversion (not the recursions
 *     Eqs. Erec0-Erect);
 *   - the basic integral B of Eq. bfinal and its radial derivatives
 *     g_n = (Q^-1 d/dQ)^n B, with the operator applied analytically to the
 *     bracket of Eq. bfinal and the remaining one-dimensional integral over
 *     r12 done by numerical quadrature (tanh-sinh on the piece touching
 *     r12 = 0, adaptive Gauss-Legendre elsewhere);
 *   - R_tuv = d^t/dQx^t d^u/dQy^u d^v/dQz^v B (Eq. ri) by the Cartesian
 *     Hermite recursion for a radial function;
 *   - the contraction of Eq. ii, nested as printed (inner ket sum first).
 *
 * All arithmetic is binary128: __float128 on x86-64 (libquadmath), the native
 * long double on AArch64 Linux.  Results are returned rounded to double.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 real;
#define R_EXP expq
#define R_LOG logq
#define R_POW powq
#define R_SQRT sqrtq
#define R_FABS fabsq
#define R_ACOS acosq
#define R_COS cosq
#define R_TANH tanhq
#define R_COSH coshq
#define R_SINH sinhq
#else
#if LDBL_MANT_DIG != 113
#error "the oracle needs a binary128 long double on this platform"
#endif
typedef long double real;
#define R_EXP expl
#define R_LOG logl
#define R_POW powl
#define R_SQRT sqrtl
#define R_FABS fabsl
#define R_ACOS acosl
#define R_COS cosl
#define R_TANH tanhl
#define R_COSH coshl
#define R_SINH sinhl
#endif

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORK_MAXN 24   /* highest radial derivative order the oracle supports */
#define ORK_MAXL 5    /* highest shell angular momentum (f = 3, plus 2 for I5) */

/* Kernel description.  id = 0 selects the range-separated factor pair (f, f')
 * of Eq. rs12; id = 20 a factor pair given as sums of terms
 * c r^a exp(b r - g r^2) (t[i] = {c, a, b, g}), from which the kernels of the
 * six classes are formed as for id 0 (Eqs. k1-k6, I6_); other ids select
 * plain test kernels used to pin the oracle:
 *   10: k = 1          11: k = exp(-gam r^2)     12: k = r
 *   13: k = 1/r        14: k = exp(-gam r)                                     */
#define ORK_TERMS 20
#define ORK_MAXT 16
typedef struct {
  int id;
  double c0, rho, B, mu;
  int n;
  double c0p, rhop, Bp, mup;
  int np;
  double gam;
  int nt, ntp;
  double t[ORK_MAXT][4], tp[ORK_MAXT][4];
} ork_kernel;

/* ---------------------------------------------------------------- kernels -- */

/* Tang-Toennies damping S_n(x) = 1 - e^{-x} sum_{k<=n} x^k/k!  (Eq. ttdamp).
 * For small x the tail sum e^{-x} sum_{k>n} x^k/k! avoids the cancellation. */
static real tt_damp(real x, int n) {
  if (x < (real)(n + 4)) {
    real term = 1;
    for (int k = 1; k <= n + 1; ++k) term *= x / k;
    real s = 0;
    int k = n + 1;
    for (int it = 0; it < 400; ++it) {
      s += term;
      ++k;
      term *= x / k;
      if (term <= s * (real)1e-40) break;
    }
    return R_EXP(-x) * s;
  }
  real term = 1, s = 1;
  for (int k = 1; k <= n; ++k) {
    term *= x / k;
    s += term;
  }
  return 1 - R_EXP(-x) * s;
}

/* dS_n/dx = e^{-x} x^n / n! */
static real tt_damp_dx(real x, int n) {
  real t = R_EXP(-x);
  for (int k = 1; k <= n; ++k) t *= x / k;
  return t;
}

/* f(r) of Eq. rs12 and its derivative f_r(r) = df/dr. */
static void factor_eval(real r, double c0, double rho, double B, double mu, int n,
                        real *f, real *fr) {
  real m = mu, x = m * r * r;
  real g = R_EXP(-x);
  real sr = (1 + r / 2) * g;
  real sr_r = ((real)0.5 - 2 * m * r * (1 + r / 2)) * g;
  real lr = 0, lr_r = 0;
  if (c0 != 0.0) {
    real S = tt_damp(x, n), Sp = tt_damp_dx(x, n);
    real pw = R_POW(r, (real)rho) * R_EXP((real)B * r);
    lr = (real)c0 * S * pw;
    lr_r = (real)c0 * (Sp * 2 * m * r * pw + S * pw * ((real)rho / r + (real)B));
  }
  *f = sr + lr;
  *fr = sr_r + lr_r;
}

/* f(r) and f_r(r) of a factor given as terms c r^a e^{b r - g r^2}. */
static void terms_eval(const double (*t)[4], int nt, real r, real *f, real *fr) {
  real s = 0, sr = 0;
  for (int i = 0; i < nt; ++i) {
    const real a = t[i][1], b = t[i][2], g = t[i][3];
    const real v = (real)t[i][0] * R_POW(r, a) * R_EXP(b * r - g * r * r);
    s += v;
    sr += v * (a / r + b - 2 * g * r);
  }
  *f = s;
  *fr = sr;
}

/* f (prime = 0) or f' (prime = 1) of the kernel's factor pair, and its derivative. */
static void pair_eval(const ork_kernel *K, int prime, real r, real *f, real *fr) {
  if (K->id == ORK_TERMS) {
    if (prime) terms_eval(K->tp, K->ntp, r, f, fr);
    else terms_eval(K->t, K->nt, r, f, fr);
  } else if (prime) {
    factor_eval(r, K->c0p, K->rhop, K->Bp, K->mup, K->np, f, fr);
  } else {
    factor_eval(r, K->c0, K->rho, K->B, K->mu, K->n, f, fr);
  }
}

/* k_i(r) of Eqs. k1-k6 (class 5 uses the I3 kernel f, see Eq. I5_). */
static real kernel_value(const ork_kernel *K, int cls, real r) {
  if (K->id && K->id != ORK_TERMS) {
    switch (K->id) {
      case 10: return 1;
      case 11: return R_EXP(-(real)K->gam * r * r);
      case 12: return r;
      case 13: return 1 / r;
      case 14: return R_EXP(-(real)K->gam * r);
      default: return 0;
    }
  }
  real f, fr, fp, frp;
  switch (cls) {
    case 1: return 1 / r;
    case 2: pair_eval(K, 0, r, &f, &fr); return f / r;
    case 3:
    case 5: pair_eval(K, 0, r, &f, &fr); return f;
    case 4:
      pair_eval(K, 0, r, &f, &fr);
      pair_eval(K, 1, r, &fp, &frp);
      return f * fp;
    case 6:
      pair_eval(K, 0, r, &f, &fr);
      pair_eval(K, 1, r, &fp, &frp);
      return fr * frp;
    default: return 0;
  }
}

/* ------------------------------------------------------- Taylor jets -- */

/* Truncated Taylor series c[k] = f^(k)(x0) / k!, k < ORK_JET, about a point
 * x0, carried through the kernel's formula by the standard recurrences of
 * automatic differentiation (products by the Cauchy rule; b = e^a from
 * b' = a' b; b = a^e from a b' = e a' b).  Used by the large-T form of the
 * radial integral, which needs d^m/dx^m [x k(x)] up to m = ORK_MAXN. */
#define ORK_JET (ORK_MAXN + 2)
typedef struct {
  int n;              /* coefficients kept: c[0..n-1] */
  real c[ORK_JET];
} jet;

static jet jet_cst(real v, int n) {
  jet r;
  memset(&r, 0, sizeof r);
  r.n = n;
  r.c[0] = v;
  return r;
}

static jet jet_var(real x0, int n) {
  jet r = jet_cst(x0, n);
  if (n > 1) r.c[1] = 1;
  return r;
}

static jet jet_add(jet a, jet b) {
  for (int k = 0; k < a.n; ++k) a.c[k] += b.c[k];
  return a;
}

static jet jet_scale(jet a, real s) {
  for (int k = 0; k < a.n; ++k) a.c[k] *= s;
  return a;
}

static jet jet_mul(jet a, jet b) {
  jet r = jet_cst(0, a.n);
  for (int k = 0; k < a.n; ++k) {
    real s = 0;
    for (int j = 0; j <= k; ++j) s += a.c[j] * b.c[k - j];
    r.c[k] = s;
  }
  return r;
}

static jet jet_exp(jet a) {
  jet r = jet_cst(R_EXP(a.c[0]), a.n);
  for (int k = 1; k < a.n; ++k) {
    real s = 0;
    for (int j = 1; j <= k; ++j) s += (real)j * a.c[j] * r.c[k - j];
    r.c[k] = s / k;
  }
  return r;
}

/* a^e for a.c[0] > 0 */
static jet jet_pow(jet a, real e) {
  jet r = jet_cst(R_POW(a.c[0], e), a.n);
  for (int k = 1; k < a.n; ++k) {
    real s = 0;
    for (int j = 1; j <= k; ++j) s += (e * j - (k - j)) * a.c[j] * r.c[k - j];
    r.c[k] = s / (k * a.c[0]);
  }
  return r;
}

/* d/dx (the top coefficient becomes unknown and is set to zero) */
static jet jet_der(jet a) {
  jet r = jet_cst(0, a.n);
  for (int k = 0; k + 1 < a.n; ++k) r.c[k] = (real)(k + 1) * a.c[k + 1];
  return r;
}

/* antiderivative with value v at x0 */
static jet jet_int(jet a, real v) {
  jet r = jet_cst(v, a.n);
  for (int k = 1; k < a.n; ++k) r.c[k] = a.c[k - 1] / k;
  return r;
}

/* f(r) of Eq. rs12 as a jet in r; the Tang-Toennies factor S_n(mu r^2) is
 * carried through S_n' = e^{-x} x^n / n! (Eq. ttdamp), so that its small-x
 * cancellation never enters the higher coefficients. */
static jet factor_jet(jet r, double c0, double rho, double B, double mu, int n) {
  jet x = jet_scale(jet_mul(r, r), (real)mu);
  jet g = jet_exp(jet_scale(x, -1));
  jet f = jet_mul(jet_add(jet_cst(1, r.n), jet_scale(r, (real)0.5)), g);
  if (c0 != 0.0) {
    jet xn = jet_cst(1, r.n);
    real nf = 1;
    for (int k = 1; k <= n; ++k) {
      xn = jet_mul(xn, x);
      nf *= k;
    }
    jet dS = jet_mul(jet_scale(jet_mul(g, xn), 1 / nf), jet_der(x)); /* dS/dr */
    jet S = jet_int(dS, tt_damp(x.c[0], n));
    jet pw = jet_mul(jet_pow(r, (real)rho), jet_exp(jet_scale(r, (real)B)));
    f = jet_add(f, jet_scale(jet_mul(S, pw), (real)c0));
  }
  return f;
}

/* A factor given as terms c r^a e^{b r - g r^2}, as a jet in r. */
static jet terms_jet(jet r, const double (*t)[4], int nt) {
  jet f = jet_cst(0, r.n);
  for (int i = 0; i < nt; ++i) {
    jet e = jet_exp(jet_add(jet_scale(r, (real)t[i][2]), jet_scale(jet_mul(r, r), -(real)t[i][3])));
    f = jet_add(f, jet_scale(jet_mul(jet_pow(r, (real)t[i][1]), e), (real)t[i][0]));
  }
  return f;
}

static jet pair_jet(const ork_kernel *K, int prime, jet r) {
  if (K->id == ORK_TERMS) return prime ? terms_jet(r, K->tp, K->ntp) : terms_jet(r, K->t, K->nt);
  if (prime) return factor_jet(r, K->c0p, K->rhop, K->Bp, K->mup, K->np);
  return factor_jet(r, K->c0, K->rho, K->B, K->mu, K->n);
}

/* x k_i(x) of Eqs. k1-k6 as a jet about x0 > 0 with coefficients up to order
 * nord (test kernels as in kernel_value); f_r takes one order more. */
static jet phi_jet(const ork_kernel *K, int cls, real x0, int nord) {
  jet r = jet_var(x0, nord + 2), k;
  if (K->id && K->id != ORK_TERMS) {
    switch (K->id) {
      case 10: k = jet_cst(1, r.n); break;
      case 11: k = jet_exp(jet_scale(jet_mul(r, r), -(real)K->gam)); break;
      case 12: k = r; break;
      case 13: k = jet_pow(r, -1); break;
      case 14: k = jet_exp(jet_scale(r, -(real)K->gam)); break;
      default: k = jet_cst(0, r.n);
    }
    return jet_mul(r, k);
  }
  switch (cls) {
    case 1: return jet_cst(1, r.n);
    case 2: return pair_jet(K, 0, r);
    case 3:
    case 5: k = pair_jet(K, 0, r); break;
    case 4: k = jet_mul(pair_jet(K, 0, r), pair_jet(K, 1, r)); break;
    case 6: k = jet_mul(jet_der(pair_jet(K, 0, r)), jet_der(pair_jet(K, 1, r))); break;
    default: k = jet_cst(0, r.n);
  }
  return jet_mul(r, k);
}

/* Largest exponential growth rate of the kernel (the e^{B r} factors). */
static double kernel_growth(const ork_kernel *K, int cls) {
  double b = 0.0, bp = 0.0;
  if (K->id == ORK_TERMS) {
    for (int i = 0; i < K->nt; ++i) b = K->t[i][2] > b ? K->t[i][2] : b;
    for (int i = 0; i < K->ntp; ++i) bp = K->tp[i][2] > bp ? K->tp[i][2] : bp;
  } else if (K->id) {
    return 0.0;
  } else {
    b = K->c0 != 0.0 && K->B > 0 ? K->B : 0.0;
    bp = K->c0p != 0.0 && K->Bp > 0 ? K->Bp : 0.0;
  }
  switch (cls) {
    case 2: case 3: case 5: return b;
    case 4: case 6: return b + bp;
    default: return 0.0;
  }
}

/* -------------------------------------------------- radial derivative kernel */

/* jh[m] = e^{-z} j_m(z),  j_m(z) = (z^-1 d/dz)^m (sinh z / z), m = 0..N.
 * Small z: power series for m = N and N-1 followed by the (always stable)
 * downward recurrence j_{m-1} = z^2 j_{m+1} + (2m+1) j_m.
 * Large z: closed forms of j_0, j_1 and the upward recurrence, which is stable
 * for z above the order. */
static void jhat(real z, int N, real *jh) {
  const real zser = (real)(40 + 2 * N);
  if (z <= zser) {
    real z2 = z * z, ez = R_EXP(-z);
    int mlo = N > 0 ? N - 1 : 0;
    for (int m = N; m >= mlo; --m) {
      real c = 1; /* 2^m m!/(2m+1)! = 1/(2m+1)!! */
      for (int j = 1; j <= m; ++j) c /= (real)(2 * j + 1);
      real term = c, s = 0;
      for (int k = 0; k < 2000; ++k) {
        s += term;
        term *= z2 * (real)(k + m + 1) / ((real)(k + 1) * (real)(2 * k + 2 * m + 2) * (real)(2 * k + 2 * m + 3));
        if (term <= s * (real)1e-40 && k > 2) break;
      }
      jh[m] = ez * s;
    }
    for (int m = N - 1; m >= 1; --m) jh[m - 1] = z2 * jh[m + 1] + (real)(2 * m + 1) * jh[m];
    return;
  }
  real e2 = R_EXP(-2 * z), iz = 1 / z;
  jh[0] = (1 - e2) * iz / 2;
  if (N >= 1) jh[1] = ((1 - iz) + e2 * (1 + iz)) * iz * iz / 2;
  for (int m = 1; m < N; ++m) jh[m + 1] = (jh[m - 1] - (real)(2 * m + 1) * jh[m]) * iz * iz;
}

typedef struct {
  const ork_kernel *K;
  int cls, N;
  int mode;   /* 0: Bessel form (small T), 1: separated exponentials,
                 2: derivatives moved onto x k(x) (very large T) */
  real xi, D;
  real binom[ORK_MAXN + 1][ORK_MAXN + 1];
  real anm[ORK_MAXN + 1][ORK_MAXN + 1];   /* D_Q^n (h/D) = sum_m a_nm h^(m) / D^(2n+1-m) */
} radial_ctx;

/* Large-T form of the same integrand:
 *   D_Q^n [h(D)/D] = sum_m a_nm h^(m)(D) / D^(2n+1-m),
 *   a_00 = 1,  a_{n+1,m} = a_{n,m-1} - (2n+1-m) a_{n,m},
 * applied to h(D) = e^{-xi (x-D)^2} - e^{-xi (x+D)^2}, whose D-derivatives are
 *   d^m/dD^m e^{-xi (x-D)^2} = xi^{m/2} H_m(sqrt(xi)(x-D)) e^{-xi (x-D)^2},
 *   d^m/dD^m e^{-xi (x+D)^2} = (-sqrt(xi))^m H_m(sqrt(xi)(x+D)) e^{-xi (x+D)^2}
 * (H_m the physicists' Hermite polynomials).  The two exponentials are kept
 * apart, which avoids the cancellation of the Bessel form when T = xi D^2 is
 * large. */
static void radial_integrand_sep(const radial_ctx *c, real x, real *out, real *mag) {
  const int N = c->N;
  real xi = c->xi, D = c->D, sx = R_SQRT(xi);
  real kx = kernel_value(c->K, c->cls, x);
  real phi = kx * x;
  real y1 = sx * (x - D), y2 = sx * (x + D);
  real e1 = R_EXP(-y1 * y1), e2 = R_EXP(-y2 * y2);
  real h[ORK_MAXN + 1], H1p = 1, H1 = 2 * y1, H2p = 1, H2 = 2 * y2, sm = 1;
  /* h[m] = d^m/dD^m [e^{-xi(x-D)^2} - e^{-xi(x+D)^2}] */
  h[0] = e1 - e2;
  if (N >= 1) h[1] = sx * (H1 * e1 + H2 * e2);
  real s1 = sx;
  for (int m = 2; m <= N; ++m) {
    real H1n = 2 * y1 * H1 - 2 * (m - 1) * H1p;
    real H2n = 2 * y2 * H2 - 2 * (m - 1) * H2p;
    H1p = H1; H1 = H1n; H2p = H2; H2 = H2n;
    s1 *= sx;
    sm = (m % 2) ? -1 : 1;
    h[m] = s1 * (H1 * e1 - sm * H2 * e2);
  }
  real iD = 1 / D, iD2 = iD * iD;
  real pw[2 * ORK_MAXN + 2];
  pw[0] = 1;
  for (int k = 1; k <= 2 * N + 1; ++k) pw[k] = pw[k - 1] * iD;
  (void)iD2;
  for (int n = 0; n <= N; ++n) {
    real s = 0, sa = 0;
    for (int m = 0; m <= n; ++m) {
      real term = c->anm[n][m] * h[m] * pw[2 * n + 1 - m];
      s += term;
      sa += R_FABS(term);
    }
    out[n] = phi * s;
    mag[n] = R_FABS(phi) * sa;
  }
}

/* Very-large-T form.  With h(D) as above, drop the image term
 * e^{-xi (x+D)^2} (below e^{-T}) and the range x < x_c = D - 16/sqrt(xi)
 * (Gaussian weight below e^{-256}); on the rest, d/dD e^{-xi(x-D)^2} =
 * -d/dx e^{-xi(x-D)^2} and m integrations by parts (boundary terms of the
 * same e^{-256} size) give
 *   h^(m)(D) = int_{x_c}^inf [x k(x)]^(m) e^{-xi (x-D)^2} dx,
 * whose integrand has no cancellation: the Hermite-polynomial form loses
 * about T^{m/2} to it, which exceeds binary128 for T near 1e4 and m = 14. */
static void radial_integrand_ibp(const radial_ctx *c, real x, real *out, real *mag) {
  const int N = c->N;
  real D = c->D, dx = x - D;
  real G = R_EXP(-c->xi * dx * dx);
  jet ph = phi_jet(c->K, c->cls, x, N);
  real hm[ORK_MAXN + 1], fact = 1;
  for (int m = 0; m <= N; ++m) {
    if (m > 0) fact *= m;
    hm[m] = fact * ph.c[m] * G;
  }
  real iD = 1 / D, pw[2 * ORK_MAXN + 2];
  pw[0] = 1;
  for (int k = 1; k <= 2 * N + 1; ++k) pw[k] = pw[k - 1] * iD;
  for (int n = 0; n <= N; ++n) {
    real s = 0, sa = 0;
    for (int m = 0; m <= n; ++m) {
      real term = c->anm[n][m] * hm[m] * pw[2 * n + 1 - m];
      s += term;
      sa += R_FABS(term);
    }
    out[n] = s;
    mag[n] = sa;
  }
}

/* The integrand of hat g_n for n = 0..N at r12 = x:
 *   k(x) x D_Q^n [ (e^{-xi (x-D)^2} - e^{-xi (x+D)^2}) / D ]
 * with D_Q = D^-1 d/dD applied analytically.  Writing the bracket as
 *   4 xi x e^{-xi (x^2 + D^2)} j_0(2 xi x D)
 * and using D_Q j_m(2 xi x D) = (2 xi x)^2 j_{m+1}, Leibniz' rule gives
 *   4 xi x e^{-xi (x-D)^2} sum_m C(n,m) (-2 xi)^{n-m} (2 xi x)^{2m} e^{-z} j_m(z). */
static void radial_integrand(const radial_ctx *c, real x, real *out, real *mag) {
  const int N = c->N;
  real xi = c->xi, D = c->D;
  if (x <= 0) {
    for (int n = 0; n <= N; ++n) out[n] = mag[n] = 0;
    return;
  }
  if (c->mode == 2) {
    radial_integrand_ibp(c, x, out, mag);
    return;
  }
  if (c->mode) {
    radial_integrand_sep(c, x, out, mag);
    return;
  }
  real kx = kernel_value(c->K, c->cls, x);
  real dx = x - D;
  real w = kx * x * 4 * xi * x * R_EXP(-xi * dx * dx);
  real jh[ORK_MAXN + 2];
  jhat(2 * xi * x * D, N, jh);
  real a = 2 * xi * x, a2 = a * a;
  real pa[ORK_MAXN + 1], pm[ORK_MAXN + 1];
  pa[0] = 1;
  pm[0] = 1;
  for (int m = 1; m <= N; ++m) {
    pa[m] = pa[m - 1] * a2;
    pm[m] = pm[m - 1] * (-2 * xi);
  }
  for (int n = 0; n <= N; ++n) {
    real s = 0, sa = 0;
    for (int m = 0; m <= n; ++m) {
      real term = c->binom[n][m] * pm[n - m] * pa[m] * jh[m];
      s += term;
      sa += R_FABS(term);
    }
    out[n] = w * s;
    mag[n] = R_FABS(w) * sa; /* size before cancellation: sets the noise floor */
  }
}

/* Gauss-Legendre rules of 32 and 48 points on [-1, 1], built by Newton
 * iteration in binary128 on first use. */
static real gl_x[2][48], gl_w[2][48];
static const int gl_n[2] = {32, 48};
static int gl_ready = 0;

static void gl_build(void) {
  const real pi = R_ACOS((real)-1);
  for (int r = 0; r < 2; ++r) {
    int n = gl_n[r];
    for (int i = 0; i < n; ++i) {
      real x = R_COS(pi * ((real)i + (real)0.75) / ((real)n + (real)0.5));
      real dp = 0;
      for (int it = 0; it < 100; ++it) {
        real p0 = 1, p1 = x;
        for (int k = 2; k <= n; ++k) {
          real p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1);
        real dx = p1 / dp;
        x -= dx;
        if (R_FABS(dx) < (real)1e-36) break;
      }
      gl_x[r][i] = x;
      gl_w[r][i] = 2 / ((1 - x * x) * dp * dp);
    }
  }
  gl_ready = 1;
}

/* Gauss-Legendre on [a,b] with rule r; also returns the integral of |f_n|. */
static void gl_apply(const radial_ctx *c, int r, real a, real b, real *I, real *A) {
  const int N = c->N;
  real h = (b - a) / 2, m = (a + b) / 2, f[ORK_MAXN + 1], g[ORK_MAXN + 1];
  for (int n = 0; n <= N; ++n) I[n] = A[n] = 0;
  for (int i = 0; i < gl_n[r]; ++i) {
    radial_integrand(c, m + h * gl_x[r][i], f, g);
    for (int n = 0; n <= N; ++n) {
      I[n] += gl_w[r][i] * f[n];
      A[n] += gl_w[r][i] * g[n];
    }
  }
  for (int n = 0; n <= N; ++n) {
    I[n] *= h;
    A[n] *= h;
  }
}

/* Adaptive Gauss-Legendre: accept when the 32- and 48-point rules agree to
 * tol relative to the piece's absolute integral, otherwise bisect. */
static int gl_adapt(const radial_ctx *c, real a, real b, real tol, int depth, real *I, real *A) {
  const int N = c->N;
  real I1[ORK_MAXN + 1], A1[ORK_MAXN + 1], I2[ORK_MAXN + 1], A2[ORK_MAXN + 1];
  gl_apply(c, 0, a, b, I1, A1);
  gl_apply(c, 1, a, b, I2, A2);
  int ok = 1;
  for (int n = 0; n <= N; ++n)
    if (R_FABS(I1[n] - I2[n]) > tol * A2[n] + (real)1e-300) ok = 0;
  if (ok || depth >= 24) {
    for (int n = 0; n <= N; ++n) {
      I[n] += I2[n];
      A[n] += A2[n];
    }
    return ok ? 0 : 1;
  }
  real m = (a + b) / 2;
  int e = gl_adapt(c, a, m, tol, depth + 1, I, A);
  e |= gl_adapt(c, m, b, tol, depth + 1, I, A);
  return e;
}

/* tanh-sinh on [0, b]; nodes placed by their distance to the end points so
 * that the non-analytic behaviour at r12 = 0 is resolved.  The step is halved
 * until two successive levels agree to tol relative to the absolute integral. */
static int tanh_sinh0(const radial_ctx *c, real b, real tol, real *I, real *A) {
  const int N = c->N;
  const real pi2 = R_ACOS((real)-1) / 2;
  const real tmax = (real)4.3;
  real S[ORK_MAXN + 1], Sa[ORK_MAXN + 1], f[ORK_MAXN + 1], g[ORK_MAXN + 1], prev[ORK_MAXN + 1];
  for (int n = 0; n <= N; ++n) S[n] = Sa[n] = prev[n] = 0;
  real h = 1;
  int converged = 0;
  for (int level = 0; level <= 12; ++level) {
    if (level > 0) h /= 2;
    int kmax = (int)(tmax / h) + 1;
    for (int k = -kmax; k <= kmax; ++k) {
      if (level > 0 && (k % 2 == 0)) continue;  /* even nodes were summed before */
      real t = k * h;
      real u = pi2 * R_SINH(t);
      real ch = R_COSH(u);
      real wgt = pi2 * R_COSH(t) / (ch * ch) * b / 2; /* dx/dt */
      real x;
      if (u < 0) {
        real e = R_EXP(2 * u);
        x = b * e / (1 + e);
      } else {
        real e = R_EXP(-2 * u);
        x = b / (1 + e);
      }
      if (!(x > 0) || !(x < b)) continue;
      radial_integrand(c, x, f, g);
      for (int n = 0; n <= N; ++n) {
        S[n] += wgt * f[n];
        Sa[n] += wgt * g[n];
      }
    }
    if (level >= 3) {
      int ok = 1;
      for (int n = 0; n <= N; ++n)
        if (R_FABS(S[n] * h - prev[n]) > tol * Sa[n] * h + (real)1e-300) ok = 0;
      if (ok) converged = 1;
    }
    for (int n = 0; n <= N; ++n) prev[n] = S[n] * h;
    if (converged) break;
  }
  for (int n = 0; n <= N; ++n) {
    I[n] += prev[n];
    A[n] += Sa[n] * h;
  }
  return converged ? 0 : 1;
}

/* hat g_n(xi, D) = int_0^inf k(x) x D_Q^n [(e^{-xi(x-D)^2} - e^{-xi(x+D)^2})/D] dx
 * for n = 0..N.  The basic integral of Eq. bfinal is
 *   g_n = sqrt(pi^5/(p+q)) / (p q) * hat g_n.
 * Returns 0 on success, nonzero when a quadrature piece did not converge. */
#define ORK_T_SWITCH 16
#define ORK_T_SWITCH2 1000
#define ORK_IBP_CUT 16
static int radial_hat(const ork_kernel *K, int cls, real xi, real D, int N, real *out,
                      int mode_override) {
  radial_ctx c;
  c.K = K;
  c.cls = cls;
  c.N = N;
  c.xi = xi;
  c.D = D;
  for (int n = 0; n <= N; ++n) {
    c.binom[n][0] = c.binom[n][n] = 1;
    for (int m = 1; m < n; ++m) c.binom[n][m] = c.binom[n - 1][m - 1] + c.binom[n - 1][m];
  }
  for (int n = 0; n <= N; ++n)
    for (int m = 0; m <= N; ++m) c.anm[n][m] = 0;
  c.anm[0][0] = 1;
  for (int n = 0; n < N; ++n)
    for (int m = 0; m <= n + 1; ++m)
      c.anm[n + 1][m] = (m > 0 ? c.anm[n][m - 1] : 0) - (real)(2 * n + 1 - m) * (m <= n ? c.anm[n][m] : 0);
  real T = xi * D * D;
  c.mode = (mode_override >= 0) ? mode_override : (T >= (real)ORK_T_SWITCH2 ? 2 : T >= (real)ORK_T_SWITCH);
  real I[ORK_MAXN + 1], A[ORK_MAXN + 1];
  for (int n = 0; n <= N; ++n) I[n] = A[n] = 0;
  real w = 1 / R_SQRT(xi);
  real cen = D + (real)kernel_growth(K, cls) / (2 * xi);
  real xend = cen + 18 * w;
  real tol = (real)1e-28;
  int err = 0;
  if (c.mode == 2) {
    real xc = D - ORK_IBP_CUT * w;
    if (!(xc > 0)) return 2;
    for (real a = xc; a < xend; a += w) {
      real b = a + w;
      if (b > xend) b = xend;
      err |= gl_adapt(&c, a, b, tol, 0, I, A);
    }
    for (int n = 0; n <= N; ++n) out[n] = I[n];
    return err;
  }
  /* piece 1: [0, x_ts] by tanh-sinh (end-point behaviour of k(x) x at 0) */
  real x_ts = w / 2;
  if (x_ts > (real)0.5) x_ts = (real)0.5;
  err |= tanh_sinh0(&c, x_ts, tol, I, A);
  /* piece 2: the stretch between x_ts and the Gaussian peak region */
  real x_lo = cen - 11 * w;
  real a0 = x_ts;
  if (x_lo > x_ts) {
    err |= gl_adapt(&c, x_ts, x_lo, tol, 0, I, A);
    a0 = x_lo;
  }
  /* pieces 3..: the peak region in steps of one Gaussian width */
  for (real a = a0; a < xend; a += w) {
    real b = a + w;
    if (b > xend) b = xend;
    err |= gl_adapt(&c, a, b, tol, 0, I, A);
  }
  for (int n = 0; n <= N; ++n) out[n] = I[n];
  return err;
}

/* ---------------------------------------------------- McMurchie-Davidson -- */

static real binom_r(int n, int k) {
  real c = 1;
  for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
  return c;
}

/* 1-D Hermite expansion coefficients by direct expansion (Eq. AB):
 *   x_A^i x_B^j e^{-a x_A^2 - b x_B^2} = sum_t E_t^{ij} Lambda_t(x; p, P)
 * x_A = x_P + X_PA, binomial in x_P, then
 *   x_P^m e^{-p x_P^2} = sum_t m!/(2^m t! ((m-t)/2)!) p^{-(m+t)/2} Lambda_t.
 * E[i][j][t] for i <= imax, j <= jmax, t <= i + j. */
#define EDIM (2 * ORK_MAXL + 1)
static void hermite_E(real a, real b, real Ax, real Bx, int imax, int jmax,
                      real E[ORK_MAXL + 1][ORK_MAXL + 1][EDIM]) {
  real p = a + b, Px = (a * Ax + b * Bx) / p;
  real XPA = Px - Ax, XPB = Px - Bx, XAB = Ax - Bx;
  real K = R_EXP(-a * b / p * XAB * XAB);
  real c[EDIM][EDIM];
  for (int m = 0; m < EDIM; ++m)
    for (int t = 0; t < EDIM; ++t) {
      c[m][t] = 0;
      if (t <= m && ((m - t) % 2 == 0)) {
        int h = (m - t) / 2;
        real v = 1;
        for (int k = 2; k <= m; ++k) v *= k;      /* m! */
        for (int k = 2; k <= t; ++k) v /= k;      /* / t! */
        for (int k = 2; k <= h; ++k) v /= k;      /* / h! */
        for (int k = 0; k < m; ++k) v /= 2;       /* / 2^m */
        v *= R_POW(p, -(real)(m + t) / 2);
        c[m][t] = v;
      }
    }
  for (int i = 0; i <= imax; ++i)
    for (int j = 0; j <= jmax; ++j)
      for (int t = 0; t < EDIM; ++t) {
        real s = 0;
        if (t <= i + j)
          for (int r = 0; r <= i; ++r)
            for (int q = 0; q <= j; ++q) {
              if (t > r + q) continue;
              s += binom_r(i, r) * binom_r(j, q) * R_POW(XPA, i - r) * R_POW(XPB, j - q) * c[r + q][t];
            }
        E[i][j][t] = K * s;
      }
}

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian exponents in lexicographic order xx, xy, xz, yy, yz, zz, ... */
static void cart_list(int l, int (*e)[3]) {
  int k = 0;
  for (int i = l; i >= 0; --i)
    for (int j = l - i; j >= 0; --j) {
      e[k][0] = i;
      e[k][1] = j;
      e[k][2] = l - i - j;
      ++k;
    }
}

#define RDIM (4 * ORK_MAXL + 3)

/* One primitive quartet.  Computes, for the given class, the block
 * out[a][b][c][d] over Cartesian components.  Returns nonzero on a
 * quadrature failure. */
/* Hermite recursion and contraction of Eq. ii for one primitive quartet from
 * its radial derivatives g_n (prefactor included).  absval != 0 evaluates the
 * same expression with every factor replaced by its absolute value (|g_n|,
 * |X_PQ|, |E|, no bra sign, Laplacian coefficients taken positive): the
 * magnitude M of the terms that Eq. ii sums, which bounds to first order how
 * far relative errors in the g_n (and rounding in the recursion and sums)
 * can move each element. */
static int md_contract(int cls, const int l[4], const real ex[4], const real cen[4][3], const real *g,
                       const real Xin[3], int absval, real *out) {
  int la = l[0], lb = l[1], lc = l[2], ld = l[3];
  int ext = cls == 5 ? 2 : 0;
  int lab = la + lb + ext, lcd = lc + ld;
  int L = lab + lcd;
  real a = ex[0], b = ex[1], cc = ex[2], d = ex[3];
  real X[3];
  for (int k = 0; k < 3; ++k) X[k] = absval ? R_FABS(Xin[k]) : Xin[k];

  /* R^{(n)}_{tuv}: R^{(n)}_{000} = g_n; raising t uses
   *   R^{(n)}_{t+1,u,v} = t R^{(n+1)}_{t-1,u,v} + X R^{(n+1)}_{t,u,v},
   * valid for any radial B because d/dQx D_Q^n B = X D_Q^{n+1} B. */
  int S = L + 1;
  real *R = (real *)calloc((size_t)S * S * S * S, sizeof(real));
  if (!R) return 3;
#define RIX(n, t, u, v) R[(((size_t)(n) * S + (t)) * S + (u)) * S + (v)]
  for (int n = 0; n <= L; ++n) RIX(n, 0, 0, 0) = absval ? R_FABS(g[n]) : g[n];
  for (int n = L - 1; n >= 0; --n)
    for (int tot = 1; tot <= L - n; ++tot)
      for (int t = tot; t >= 0; --t)
        for (int u = tot - t; u >= 0; --u) {
          int v = tot - t - u;
          real val;
          if (t > 0) {
            val = X[0] * RIX(n + 1, t - 1, u, v);
            if (t > 1) val += (t - 1) * RIX(n + 1, t - 2, u, v);
          } else if (u > 0) {
            val = X[1] * RIX(n + 1, t, u - 1, v);
            if (u > 1) val += (u - 1) * RIX(n + 1, t, u - 2, v);
          } else {
            val = X[2] * RIX(n + 1, t, u, v - 1);
            if (v > 1) val += (v - 1) * RIX(n + 1, t, u, v - 2);
          }
          RIX(n, t, u, v) = val;
        }

  /* E tables per dimension */
  static __thread real Eab[3][ORK_MAXL + 1][ORK_MAXL + 1][EDIM];
  static __thread real Ecd[3][ORK_MAXL + 1][ORK_MAXL + 1][EDIM];
  for (int k = 0; k < 3; ++k) {
    hermite_E(a, b, cen[0][k], cen[1][k], la + ext, lb + ext, Eab[k]);
    hermite_E(cc, d, cen[2][k], cen[3][k], lc, ld, Ecd[k]);
    if (absval) {
      for (int i = 0; i <= ORK_MAXL; ++i)
        for (int j = 0; j <= ORK_MAXL; ++j)
          for (int t = 0; t < EDIM; ++t) {
            Eab[k][i][j][t] = R_FABS(Eab[k][i][j][t]);
            Ecd[k][i][j][t] = R_FABS(Ecd[k][i][j][t]);
          }
    }
  }
  int ea[64][3], eb[64][3], ec[64][3], ed[64][3];
  cart_list(la, ea);
  cart_list(lb, eb);
  cart_list(lc, ec);
  cart_list(ld, ed);
  int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);

  /* inner (ket) sum of Eq. ii for every bra Hermite index:
   *   W[tuv][cd] = sum_{t'u'v'} E^{cd}_{t'u'v'} R_{t+t',u+u',v+v'} */
  int nt = lab + 1;
  size_t ncd = (size_t)nc * nd;
  real *W = (real *)calloc((size_t)nt * nt * nt * ncd, sizeof(real));
  if (!W) {
    free(R);
    return 3;
  }
#define WIX(t, u, v, j) W[((((size_t)(t) * nt + (u)) * nt + (v)) * ncd) + (j)]
  for (int t = 0; t <= lab; ++t)
    for (int u = 0; u <= lab - t; ++u)
      for (int v = 0; v <= lab - t - u; ++v)
        for (int ic = 0; ic < nc; ++ic)
          for (int id = 0; id < nd; ++id) {
            real s = 0;
            for (int t2 = 0; t2 <= ec[ic][0] + ed[id][0]; ++t2)
              for (int u2 = 0; u2 <= ec[ic][1] + ed[id][1]; ++u2)
                for (int v2 = 0; v2 <= ec[ic][2] + ed[id][2]; ++v2)
                  s += Ecd[0][ec[ic][0]][ed[id][0]][t2] * Ecd[1][ec[ic][1]][ed[id][1]][u2] *
                       Ecd[2][ec[ic][2]][ed[id][2]][v2] * RIX(0, t + t2, u + u2, v + v2);
            WIX(t, u, v, ic * nd + id) = s;
          }

  /* outer (bra) sum for a bra pair given by exponent triples */
#define BRA(A3, B3, j, res)                                                                    \
  do {                                                                                         \
    real s_ = 0;                                                                               \
    for (int t_ = 0; t_ <= (A3)[0] + (B3)[0]; ++t_)                                            \
      for (int u_ = 0; u_ <= (A3)[1] + (B3)[1]; ++u_)                                          \
        for (int v_ = 0; v_ <= (A3)[2] + (B3)[2]; ++v_) {                                      \
          real e_ = Eab[0][(A3)[0]][(B3)[0]][t_] * Eab[1][(A3)[1]][(B3)[1]][u_] *              \
                    Eab[2][(A3)[2]][(B3)[2]][v_];                                              \
          if (((t_ + u_ + v_) & 1) && !absval) e_ = -e_;                                       \
          s_ += e_ * WIX(t_, u_, v_, j);                                                       \
        }                                                                                      \
    (res) = s_;                                                                                \
  } while (0)

  for (int ia = 0; ia < na; ++ia)
    for (int ib = 0; ib < nb; ++ib)
      for (size_t j = 0; j < ncd; ++j) {
        real val;
        if (cls != 5) {
          BRA(ea[ia], eb[ib], j, val);
        } else {
          /* I5 = 1/2 [(lap a, b|f|cd) - (a, lap b|f|cd)] (Eq. I5_), with
           * lap x^i e^{-a x^2} = [i(i-1) x^{i-2} - 2a(2i+1) x^i + 4a^2 x^{i+2}] e^{-a x^2}
           * in each Cartesian direction. */
          real lapa = 0, lapb = 0, tmp;
          for (int k = 0; k < 3; ++k) {
            int A3[3] = {ea[ia][0], ea[ia][1], ea[ia][2]};
            int i0 = A3[k];
            if (i0 >= 2) {
              A3[k] = i0 - 2;
              BRA(A3, eb[ib], j, tmp);
              lapa += (real)(i0 * (i0 - 1)) * tmp;
            }
            A3[k] = i0;
            BRA(A3, eb[ib], j, tmp);
            lapa += (absval ? 1 : -1) * 2 * a * (2 * i0 + 1) * tmp;
            A3[k] = i0 + 2;
            BRA(A3, eb[ib], j, tmp);
            lapa += 4 * a * a * tmp;
            int B3[3] = {eb[ib][0], eb[ib][1], eb[ib][2]};
            int j0 = B3[k];
            if (j0 >= 2) {
              B3[k] = j0 - 2;
              BRA(ea[ia], B3, j, tmp);
              lapb += (real)(j0 * (j0 - 1)) * tmp;
            }
            B3[k] = j0;
            BRA(ea[ia], B3, j, tmp);
            lapb += (absval ? 1 : -1) * 2 * b * (2 * j0 + 1) * tmp;
            B3[k] = j0 + 2;
            BRA(ea[ia], B3, j, tmp);
            lapb += 4 * b * b * tmp;
          }
          val = absval ? (lapa + lapb) / 2 : (lapa - lapb) / 2;
        }
        out[((size_t)ia * nb + ib) * ncd + j] = val;
      }
#undef BRA
#undef WIX
#undef RIX
  free(W);
  free(R);
  return 0;
}

static int prim_block(const ork_kernel *K, int cls, const int l[4], const real ex[4],
                      const real cen[4][3], real *out, real *mag) {
  int la = l[0], lb = l[1], lc = l[2], ld = l[3];
  int ext = cls == 5 ? 2 : 0;             /* kinetic transform raises la or lb by 2 */
  int lab = la + lb + ext, lcd = lc + ld;
  int L = lab + lcd;
  if (L > ORK_MAXN || la + ext > ORK_MAXL || lb + ext > ORK_MAXL) return 2;
  real a = ex[0], b = ex[1], cc = ex[2], d = ex[3];
  real p = a + b, q = cc + d;
  real P[3], Q[3], X[3];
  for (int k = 0; k < 3; ++k) {
    P[k] = (a * cen[0][k] + b * cen[1][k]) / p;
    Q[k] = (cc * cen[2][k] + d * cen[3][k]) / q;
    X[k] = Q[k] - P[k];
  }
  real xi = p * q / (p + q);
  real D = R_SQRT(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
  real gh[ORK_MAXN + 1];
  int kcls = cls == 5 ? 3 : cls;
  int err = radial_hat(K, kcls, xi, D, L, gh, -1);
  const real pi = R_ACOS((real)-1);
  real pref = R_SQRT(pi * pi * pi * pi * pi / (p + q)) / (p * q);
  for (int n = 0; n <= L; ++n) gh[n] *= pref;
  int e = md_contract(cls, l, ex, cen, gh, X, 0, out);
  if (!e && mag) e = md_contract(cls, l, ex, cen, gh, X, 1, mag);
  return e ? e : err;
}


/* ------------------------------------------------------------ public API -- */

int ork_radial_mode(const ork_kernel *K, int cls, double xi, double D, int nmax, int mode,
                    double *out);

/* hat g_n for n = 0..nmax (see radial_hat); returns nonzero on failure. */
int ork_radial(const ork_kernel *K, int cls, double xi, double D, int nmax, double *out) {
  return ork_radial_mode(K, cls, xi, D, nmax, -1, out);
}

/* As ork_radial with the integrand form forced (0: Bessel form, 1: separated
 * exponentials, 2: derivatives moved onto x k(x), needs sqrt(xi) D > 16;
 * -1: by T); lets the tests check that the forms agree. */
int ork_radial_mode(const ork_kernel *K, int cls, double xi, double D, int nmax, int mode,
                    double *out) {
  if (nmax < 0 || nmax > ORK_MAXN || !(xi > 0) || !(D >= 0)) return 2;
  if (mode >= 1 && !(D > 0)) return 2;
  if (!gl_ready) gl_build();
  real g[ORK_MAXN + 1];
  int e = radial_hat(K, cls, (real)xi, (real)D, nmax, g, mode);
  for (int n = 0; n <= nmax; ++n) out[n] = (double)g[n];
  return e;
}

/* Block of one primitive quartet: exps[4], centers[4][3], l[4]. */
int ork_prim_block(const ork_kernel *K, int cls, const int *l, const double *exps,
                   const double *centers, double *out) {
  if (cls < 1 || cls > 6) return 2;
  for (int i = 0; i < 4; ++i)
    if (l[i] < 0 || l[i] > 3) return 2;
  if (!gl_ready) gl_build();
  real ex[4], cen[4][3];
  for (int i = 0; i < 4; ++i) {
    ex[i] = exps[i];
    for (int k = 0; k < 3; ++k) cen[i][k] = centers[3 * i + k];
  }
  size_t nblk = (size_t)ncart(l[0]) * ncart(l[1]) * ncart(l[2]) * ncart(l[3]);
  real *blk = (real *)malloc(nblk * sizeof(real));
  if (!blk) return 3;
  int e = prim_block(K, cls, l, ex, cen, blk, NULL);
  for (size_t i = 0; i < nblk; ++i) out[i] = (double)blk[i];
  free(blk);
  return e;
}

/* Contracted shell-quartet blocks.
 *   shells: centers[nshell][3], l[nshell], nprim[nshell], prim_off[nshell]
 *           indexes exps[] and coefs[] (unnormalised primitives; the
 *           contraction coefficients multiply them as given)
 *   quartets[nq][4] shell indices; out + offsets[q] receives the dense block
 *   [a][b][c][d] in lexicographic Cartesian order.
 * Work is spread over primitive quartets with OpenMP; every shell quartet is
 * summed over its primitive quartets in a fixed order.  Returns the number
 * of primitive quartets whose quadrature reported non-convergence.
 * mag (may be NULL) receives, in the same layout, the magnitude of the terms
 * summed for each element: sum over primitive quartets of |coefficient
 * product| times the absolute-value evaluation of Eq. ii (see md_contract). */
int64_t ork_shell_blocks(const ork_kernel *K, int cls, const double *centers, const int *l,
                         const int *nprim, const int *prim_off, const double *exps,
                         const double *coefs, int64_t nq, const int32_t *quartets,
                         const int64_t *offsets, double *out, double *mag, int nthreads) {
  if (!gl_ready) gl_build();
  int64_t nbad = 0;
  for (int64_t q0 = 0; q0 < nq;) {
    /* gather a chunk of primitive-quartet tasks */
    int64_t q1 = q0, ntask = 0;
    while (q1 < nq && ntask < 4096) {
      const int32_t *s = quartets + 4 * q1;
      ntask += (int64_t)nprim[s[0]] * nprim[s[1]] * nprim[s[2]] * nprim[s[3]];
      ++q1;
    }
    int64_t *task_q = (int64_t *)malloc(sizeof(int64_t) * ntask);
    int64_t *task_p = (int64_t *)malloc(sizeof(int64_t) * ntask);
    size_t *task_off = (size_t *)malloc(sizeof(size_t) * ntask);
    size_t tot = 0;
    int64_t t = 0;
    for (int64_t q = q0; q < q1; ++q) {
      const int32_t *s = quartets + 4 * q;
      size_t nb = (size_t)ncart(l[s[0]]) * ncart(l[s[1]]) * ncart(l[s[2]]) * ncart(l[s[3]]);
      int64_t np = (int64_t)nprim[s[0]] * nprim[s[1]] * nprim[s[2]] * nprim[s[3]];
      for (int64_t i = 0; i < np; ++i) {
        task_q[t] = q;
        task_p[t] = i;
        task_off[t] = tot;
        tot += nb;
        ++t;
      }
    }
    real *buf = (real *)malloc(sizeof(real) * (tot ? tot : 1));
    real *mbuf = mag ? (real *)malloc(sizeof(real) * (tot ? tot : 1)) : NULL;
    int64_t bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t i = 0; i < ntask; ++i) {
      const int32_t *s = quartets + 4 * task_q[i];
      int64_t rem = task_p[i];
      int pi[4];
      for (int k = 3; k >= 0; --k) {
        pi[k] = (int)(rem % nprim[s[k]]);
        rem /= nprim[s[k]];
      }
      int ll[4];
      real ex[4], cen[4][3], coef = 1;
      for (int k = 0; k < 4; ++k) {
        ll[k] = l[s[k]];
        ex[k] = exps[prim_off[s[k]] + pi[k]];
        coef *= coefs[prim_off[s[k]] + pi[k]];
        for (int m = 0; m < 3; ++m) cen[k][m] = centers[3 * s[k] + m];
      }
      real *blk = buf + task_off[i];
      real *mblk = mbuf ? mbuf + task_off[i] : NULL;
      int e = prim_block(K, cls, ll, ex, cen, blk, mblk);
      if (e) ++bad;
      size_t nb = (size_t)ncart(ll[0]) * ncart(ll[1]) * ncart(ll[2]) * ncart(ll[3]);
      for (size_t j = 0; j < nb; ++j) blk[j] *= coef;
      if (mblk)
        for (size_t j = 0; j < nb; ++j) mblk[j] *= R_FABS(coef);
    }
    nbad += bad;
    for (int64_t i = 0; i < ntask;) {
      int64_t q = task_q[i];
      const int32_t *s = quartets + 4 * q;
      size_t nb = (size_t)ncart(l[s[0]]) * ncart(l[s[1]]) * ncart(l[s[2]]) * ncart(l[s[3]]);
      for (size_t j = 0; j < nb; ++j) {
        real acc = 0;
        for (int64_t k = i; k < ntask && task_q[k] == q; ++k) acc += buf[task_off[k] + j];
        out[offsets[q] + j] = (double)acc;
        if (mbuf) {
          real macc = 0;
          for (int64_t k = i; k < ntask && task_q[k] == q; ++k) macc += mbuf[task_off[k] + j];
          mag[offsets[q] + j] = (double)macc;
        }
      }
      while (i < ntask && task_q[i] == q) ++i;
    }
    free(buf);
    free(mbuf);
    free(task_q);
    free(task_p);
    free(task_off);
    q0 = q1;
  }
  return nbad;
}

/* e^{-z} j_m(z) exposed for the tests of the series/recurrence switch. */
int ork_jhat(double z, int N, double *out) {
  if (N < 0 || N > ORK_MAXN) return 2;
  real jh[ORK_MAXN + 2];
  jhat((real)z, N, jh);
  for (int m = 0; m <= N; ++m) out[m] = (double)jh[m];
  return 0;
}

/* Pointwise kernel value, exposed for the tests. */
double ork_kernel_value(const ork_kernel *K, int cls, double r) {
  return (double)kernel_value(K, cls, (real)r);
}

/* Size of the binary128 mantissa this build uses (113 expected). */
int ork_mantissa_bits(void) {
#if defined(__x86_64__) || defined(__i386__)
  return FLT128_MANT_DIG;
#else
  return LDBL_MANT_DIG;
#endif
}
