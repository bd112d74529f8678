// aux_host.cpp -- CPU build of the library's auxiliary-function stage, for tests.
//
// Compiles paper_1412_5070_gb300/csrc/aux.cuh as plain C++ (no nvcc, no GPU)
// with the tables filled by the library's own host code (auxtab.h,
// termlist.cpp), so that tests without a GPU can compare the stage's
// arithmetic, hat g_l(xi, D) for every class, with the oracle.  The library
// never loads this file's build; on the GPU the same functions run inside
// the kernels.
#include <cstdint>
#include <cstring>
#include <vector>

#include "../paper_1412_5070_gb300/csrc/aux.cuh"
#include "../paper_1412_5070_gb300/csrc/auxtab.h"
#include "../paper_1412_5070_gb300/csrc/termlist.h"

using namespace f12dev;

namespace {

void load_constants() {
  static bool done = false;
  if (done) return;
  static AuxConst ac;
  fill_aux_const(ac);
  std::memcpy(c_gh_x, ac.gh_x, sizeof(ac.gh_x));
  std::memcpy(c_gh_w, ac.gh_w, sizeof(ac.gh_w));
  std::memcpy(c_gl_x, ac.gl_x, sizeof(ac.gl_x));
  std::memcpy(c_gl_w, ac.gl_w, sizeof(ac.gl_w));
  std::memcpy(c_cratio, ac.cratio, sizeof(ac.cratio));
  std::memcpy(c_inv_dfact, ac.inv_dfact, sizeof(ac.inv_dfact));
  std::memcpy(d_kum_inv, ac.kum_inv, sizeof(ac.kum_inv));
  std::memcpy(d_sm1_ratio, ac.sm1_ratio, sizeof(ac.sm1_ratio));
  std::memcpy(d_cser, ac.cser, sizeof(ac.cser));
  std::memcpy(d_vstep, ac.vstep, sizeof(ac.vstep));
  std::memcpy(d_quarter, ac.quarter, sizeof(ac.quarter));
  static std::vector<double> kt;
  fill_kummer_table(kt);
  d_mtab = kt.data();
  done = true;
}

int eval(const f12::TermList kt[NCLASS], int cls, int64_t n, const double *xi, const double *D, int nmax,
         double *out) {
  load_constants();
  ClassTables ct;
  if (!build_class_tables(kt, ct)) return -3;
  if (!ct.supported[cls]) return -3;
  Tables T{};
  for (int c = 0; c < NCLASS; ++c) {
    T.nfam[c] = ct.nfam[c];
    T.fam0[c] = ct.fam0[c];
  }
  T.fam = ct.fams.data();
  T.coef = ct.coef.data();
  T.grp = ct.groups.data();
  T.jtab = ct.jtab.data();
  int bad = 0;
  double g[LAUX + 1];
  for (int64_t i = 0; i < n; ++i) {
    bad |= aux_eval(T, cls == 5 ? 3 : cls, xi[i], D[i], nmax, g);
    for (int l = 0; l <= nmax; ++l) out[i * (nmax + 1) + l] = g[l];
  }
  return bad ? 1 : 0;
}

}  // namespace

extern "C" {

// hat g_l, l = 0..nmax, of class cls for the factor pair (f, fp) given as
// {c0, rho, B, mu, n} (Eq. rs12).  Returns 0, 1 if a series or quadrature
// reported a failure, -3 if the class is outside what the stage supports,
// -1 for bad arguments.
int aux_host_eval(const double *f, const double *fp, int cls, int64_t n, const double *xi, const double *D,
                  int nmax, double *out) {
  if (!f || !fp || cls < 1 || cls > 6 || nmax < 0 || nmax > LAUX || n < 0) return -1;
  f12::Factor F1{f[0], f[1], f[2], f[3], (int)f[4]}, F2{fp[0], fp[1], fp[2], fp[3], (int)fp[4]};
  f12::TermList kt[NCLASS];
  for (int c = 1; c <= 6; ++c)
    if (c != 5) kt[c] = f12::kernel_terms(c, F1, F2);
  return eval(kt, cls, n, xi, D, nmax, out);
}

// The same for factors given as terms: t[4 i + (0..3)] = c, a, b, g of
// c r^a exp(b r - g r^2), nt terms in f and ntp in f'.
int aux_host_eval_terms(const double *t, int nt, const double *tp, int ntp, int cls, int64_t n, const double *xi,
                        const double *D, int nmax, double *out) {
  if (!t || !tp || nt < 1 || ntp < 1 || cls < 1 || cls > 6 || nmax < 0 || nmax > LAUX || n < 0) return -1;
  f12::TermList T1, T2;
  for (int i = 0; i < nt; ++i) T1.push_back({t[4 * i], t[4 * i + 1], t[4 * i + 2], t[4 * i + 3]});
  for (int i = 0; i < ntp; ++i) T2.push_back({tp[4 * i], tp[4 * i + 1], tp[4 * i + 2], tp[4 * i + 3]});
  f12::simplify(T1);
  f12::simplify(T2);
  f12::TermList kt[NCLASS];
  for (int c = 1; c <= 6; ++c)
    if (c != 5) kt[c] = f12::kernel_terms(c, T1, T2);
  return eval(kt, cls, n, xi, D, nmax, out);
}

// Single device functions of the stage, for unit tests.
void aux_host_jhat(double z, int N, double *out) {
  load_constants();
  double jh[LAUX + 2];
  jhat_all(z, N, jh);
  for (int m = 0; m <= N; ++m) out[m] = jh[m];
}

double aux_host_kummer(double a, int ib, double z, int *bad) {
  load_constants();
  *bad = 0;
  return kummer_m(a, ib, z, bad);
}

double aux_host_s_minus1(double b, double gam, int *bad) {
  load_constants();
  *bad = 0;
  return s_minus1(b, gam, bad);
}

double aux_host_exp_rem(double y, int k) { return exp_rem(y, k); }

// Jh_alpha(y) = [int_0^inf t^alpha e^{y t - t^2} dt] / Gamma((alpha+1)/2), y >= 0
double aux_host_jhat_start(double alpha, double y, int *bad) {
  load_constants();
  *bad = 0;
  const double rho = std::exp(std::lgamma(0.5 * (alpha + 2.0)) - std::lgamma(0.5 * (alpha + 1.0)));
  return jhat_start(alpha, rho, y, bad);
}

void aux_host_gauss_legendre(double *x, double *w) {
  load_constants();
  for (int i = 0; i < NGL; ++i) {
    x[i] = c_gl_x[i];
    w[i] = c_gl_w[i];
  }
}

}  // extern "C"
