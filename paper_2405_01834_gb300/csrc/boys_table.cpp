// Boys-function interpolation table for the device (Eq. boys of the paper:
// F_m(T) = int_0^1 y^(2m) exp(-T y^2) dy; the paper names an
// interpolation-based Boys code but gives no grid, Sec. 5).
//
// Grid T0_i = i / 16 for T0 in [0, 100]; row i holds, for m = 0 .. kBoysMmax
// and k = 0 .. 7, the Taylor coefficients F_{m+k}(T0_i) / k!. The device
// evaluates
//   F_m(T0 + d) = sum_{k=0}^{7} F_{m+k}(T0) (-d)^k / k!,   |d| <= 1/32,
// by Horner's rule in -d; the truncation error is below (1/32)^8 / 8! = 2.2e-17
// relative.
//
// Values are computed in long double by downward recursion
//   F_m(T) = (2T F_{m+1}(T) + exp(-T)) / (2m+1)
// started at an order m_top >= 2T + 60 from F_{m_top} = 0. Downward
// recursion never amplifies relative error, and the start error is damped
// by the factor 2T/(2m+1) < 1 at every step above m = T, so after the
// 60 or more steps down to the tabulated orders the start error is far below
// long-double rounding.
#include <cmath>
#include <vector>

#include "mdx_internal.h"

namespace mdx {

std::vector<double> build_boys_table() {
  std::vector<double> tab((size_t)kBoysNgrid * kBoysRow, 0.0);
  for (int i = 0; i < kBoysNgrid; ++i) {
    const long double T = (long double)i / (long double)kBoysInvH;
    const long double ex = expl(-T);
    const int ncol = kBoysOrders + kBoysTerms;   // F_0 .. F_{kBoysMmax + 7}
    int mtop = (int)(2.0L * T) + 60 + ncol;
    long double F = 0.0L;
    std::vector<long double> col(ncol);
    for (int m = mtop; m >= 0; --m) {
      F = (2.0L * T * F + ex) / (long double)(2 * m + 1);
      if (m < ncol) col[m] = F;
    }
    for (int m = 0; m < kBoysOrders; ++m) {
      long double kfac = 1.0L;
      for (int k = 0; k < kBoysTerms; ++k) {
        if (k > 0) kfac *= (long double)k;
        tab[(size_t)i * kBoysRow + (size_t)m * kBoysTerms + k] = (double)(col[m + k] / kfac);
      }
    }
  }
  return tab;
}

}  // namespace mdx
