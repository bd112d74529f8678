// termlist.cpp -- host-side term lists of the F12 kernels (see termlist.h).
#include "termlist.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

namespace f12 {

namespace {
const double kTol = 1e-12;

bool same(double x, double y) { return std::fabs(x - y) <= kTol * (1.0 + std::fabs(x) + std::fabs(y)); }
}  // namespace

void simplify(TermList &t) {
  std::sort(t.begin(), t.end(), [](const Term &x, const Term &y) {
    if (!same(x.b, y.b)) return x.b < y.b;
    if (!same(x.g, y.g)) return x.g < y.g;
    if (!same(x.a, y.a)) return x.a < y.a;
    return false;
  });
  TermList out;
  for (const Term &x : t) {
    if (!out.empty() && same(out.back().a, x.a) && same(out.back().b, x.b) && same(out.back().g, x.g)) {
      out.back().c += x.c;
    } else {
      out.push_back(x);
    }
  }
  // drop terms whose coefficient vanished (exact cancellation of like terms)
  double cmax = 0.0;
  for (const Term &x : out) cmax = std::max(cmax, std::fabs(x.c));
  TermList kept;
  for (const Term &x : out)
    if (std::fabs(x.c) > 1e-15 * cmax && x.c != 0.0) kept.push_back(x);
  t.swap(kept);
}

TermList factor_terms(const Factor &f) {
  TermList t;
  t.push_back({1.0, 0.0, 0.0, f.mu});
  t.push_back({0.5, 1.0, 0.0, f.mu});
  if (f.c0 != 0.0) {
    t.push_back({f.c0, f.rho, f.B, 0.0});
    double fac = 1.0;
    for (int k = 0; k <= f.n; ++k) {
      if (k > 0) fac *= f.mu / k;
      t.push_back({-f.c0 * fac, f.rho + 2.0 * k, f.B, f.mu});
    }
  }
  simplify(t);
  return t;
}

TermList derivative(const TermList &t) {
  TermList r;
  for (const Term &x : t) {
    if (x.a != 0.0) r.push_back({x.c * x.a, x.a - 1.0, x.b, x.g});
    if (x.b != 0.0) r.push_back({x.c * x.b, x.a, x.b, x.g});
    if (x.g != 0.0) r.push_back({-2.0 * x.g * x.c, x.a + 1.0, x.b, x.g});
  }
  simplify(r);
  return r;
}

TermList product(const TermList &x, const TermList &y) {
  TermList r;
  for (const Term &u : x)
    for (const Term &v : y) r.push_back({u.c * v.c, u.a + v.a, u.b + v.b, u.g + v.g});
  simplify(r);
  return r;
}

TermList times_power(const TermList &t, double m) {
  TermList r = t;
  for (Term &x : r) x.a += m;
  return r;
}

TermList kernel_terms(int cls, const TermList &f, const TermList &fp) {
  switch (cls) {
    case 1: return TermList{{1.0, -1.0, 0.0, 0.0}};    // Eq. k1: 1/r
    case 2: return times_power(f, -1.0);              // Eq. k2: f/r
    case 3:
    case 5: return f;                                 // Eq. k3: f
    case 4: return product(f, fp);                    // Eq. k4: f f'
    case 6: return product(derivative(f), derivative(fp));   // Eq. I6_
    default: return TermList{};
  }
}

TermList kernel_terms(int cls, const Factor &f, const Factor &fp) {
  return kernel_terms(cls, factor_terms(f), factor_terms(fp));
}

std::vector<Family> families(const TermList &t) {
  std::vector<Family> out;
  for (const Term &x : t) {
    Family *hit = nullptr;
    for (Family &f : out) {
      if (!same(f.b, x.b) || !same(f.g, x.g)) continue;
      double d = x.a - f.a0;
      if (std::fabs(d - std::round(d)) <= 1e-9) {
        hit = &f;
        break;
      }
    }
    if (!hit) {
      out.push_back(Family{x.b, x.g, x.a, {}});
      hit = &out.back();
    }
    int j = (int)std::lround(x.a - hit->a0);
    if (j < 0) {  // new lowest power: shift the polynomial up
      hit->poly.insert(hit->poly.begin(), (size_t)(-j), 0.0);
      hit->a0 = x.a;
      j = 0;
    }
    if ((size_t)j >= hit->poly.size()) hit->poly.resize((size_t)j + 1, 0.0);
    hit->poly[(size_t)j] += x.c;
  }
  return out;
}

Family radial_derivative(const Family &f) {
  Family r{f.b, f.g, f.a0 - 2.0, std::vector<double>(f.poly.size() + 2, 0.0)};
  for (size_t j = 0; j < f.poly.size(); ++j) {
    double c = f.poly[j], a = f.a0 + (double)j;
    r.poly[j] += c * a;
    r.poly[j + 1] += c * f.b;
    r.poly[j + 2] += -2.0 * f.g * c;
  }
  return r;
}

}  // namespace f12
