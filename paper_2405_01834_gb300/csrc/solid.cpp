// Real solid harmonics S_lm as Cartesian polynomials, for the spherical output
// of the engine (the paper works in solid harmonics throughout, Eqs.
// solid2herm-1/2 with the Cartesian-to-solid coefficients it cites).
//
// Built by the standard recurrences in l (starting from S_00 = 1):
//   S_{l+1, l+1}  = sqrt(2^d (2l+1)/(2l+2)) (x S_ll - (1-d) y S_{l,-l})
//   S_{l+1,-l-1}  = sqrt(2^d (2l+1)/(2l+2)) (y S_ll + (1-d) x S_{l,-l})
//   S_{l+1, m}    = ((2l+1) z S_lm - sqrt((l+m)(l-m)) r^2 S_{l-1,m}) / sqrt((l+m+1)(l-m+1)),  |m| <= l
// with d = 1 for l = 0 and 0 otherwise. Every S_lm then has the angular norm
// of z^l, so functions built on x^l-normalised primitives stay normalised.
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include "mdx_internal.h"

namespace mdx {
namespace {

using Poly = std::map<std::tuple<int, int, int>, double>;   // (px, py, pz) -> coefficient

Poly mul_mono(const Poly& p, int dx, int dy, int dz, double f) {
  Poly r;
  for (const auto& kv : p) {
    const auto& k = kv.first;
    r[std::make_tuple(std::get<0>(k) + dx, std::get<1>(k) + dy, std::get<2>(k) + dz)] += f * kv.second;
  }
  return r;
}
void add_to(Poly& a, const Poly& b, double f) {
  for (const auto& kv : b) a[kv.first] += f * kv.second;
}

}  // namespace

std::vector<std::vector<double>> build_solid_tables(int lmax) {
  // S[l][m + l]
  std::vector<std::vector<Poly>> S(lmax + 1);
  S[0] = {Poly{{std::make_tuple(0, 0, 0), 1.0}}};
  for (int l = 0; l < lmax; ++l) {
    std::vector<Poly> nx(2 * l + 3);
    const double dl = l == 0 ? 1.0 : 0.0;
    const double f = std::sqrt(std::pow(2.0, dl) * (2.0 * l + 1.0) / (2.0 * l + 2.0));
    Poly top = mul_mono(S[l][2 * l], 1, 0, 0, f);
    Poly bot = mul_mono(S[l][2 * l], 0, 1, 0, f);
    if (l > 0) {
      add_to(top, mul_mono(S[l][0], 0, 1, 0, f), -1.0);
      add_to(bot, mul_mono(S[l][0], 1, 0, 0, f), 1.0);
    }
    nx[2 * l + 2] = top;
    nx[0] = bot;
    for (int m = -l; m <= l; ++m) {
      Poly p = mul_mono(S[l][m + l], 0, 0, 1, 2.0 * l + 1.0);
      if (l >= 1 && std::abs(m) <= l - 1) {
        const Poly& q = S[l - 1][m + l - 1];
        const double g = -std::sqrt((double)(l + m) * (l - m));
        add_to(p, mul_mono(q, 2, 0, 0, g), 1.0);
        add_to(p, mul_mono(q, 0, 2, 0, g), 1.0);
        add_to(p, mul_mono(q, 0, 0, 2, g), 1.0);
      }
      const double den = std::sqrt((double)(l + m + 1) * (l - m + 1));
      for (auto& kv : p) kv.second /= den;
      nx[m + l + 1] = p;
    }
    S[l + 1] = nx;
  }
  std::vector<std::vector<double>> out(lmax + 1);
  for (int l = 0; l <= lmax; ++l) {
    const int nc = ncart(l);
    out[l].assign((size_t)(2 * l + 1) * nc, 0.0);
    for (int m = -l; m <= l; ++m) {
      int k = 0;
      for (int ax = l; ax >= 0; --ax)
        for (int ay = l - ax; ay >= 0; --ay, ++k) {
          auto it = S[l][m + l].find(std::make_tuple(ax, ay, l - ax - ay));
          if (it != S[l][m + l].end() && std::fabs(it->second) > 1e-15) out[l][(size_t)(m + l) * nc + k] = it->second;
        }
    }
  }
  return out;
}

int solid_nnz(int l) {
  static const std::vector<std::vector<double>> tabs = build_solid_tables(kLmax);
  if (l < 0 || l > kLmax) return 0;
  int n = 0;
  for (double c : tabs[l]) n += c != 0.0;
  return n;
}

}  // namespace mdx
