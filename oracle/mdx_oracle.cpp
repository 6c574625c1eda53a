// Oracle: plain, slow, CPU McMurchie-Davidson electron-repulsion integrals.
//
// TEST INFRASTRUCTURE ONLY. This file is the correctness reference for the
// GPU engine. Only the test-suite, the smoke check and the CPU-baseline leg
// of the benchmark may load it; the product path never does. It shares no
// code, header, table or constant generator with the CUDA engine.
//
// Every routine is written from the formalism of Asadchev & Valeev,
// "3-center and 4-center 2-particle Gaussian AO integrals on modern
// accelerated processors" (arXiv:2405.01834), Sec. 2 "Formalism":
//   - primitive / contracted Cartesian Gaussians ............. Eqs. 1 and 3
//   - 3-/4-center Coulomb integrals (the definitions) ......... Eqs. def-acd, def-abcd
//   - Hermite expansion coefficients E (1- and 2-center) ...... Eqs. E1rr, E2rr1, E2rr2,
//                                                               E1-00, E1-aa, E2-000, E2-abp
//   - Boys function and auxiliary integrals [0]^(m) ........... Eqs. 0m, boys
//   - Hermite auxiliary recursion [r+1_i]^(m) ................ Eq. r
//   - Hermite 2-index integrals [p|q] = (-1)^|q| [p+q]^(0) ..... Eq. pq
//   - ket then bra Hermite->Cartesian transform ............... Eqs. ket-from-hermite,
//                                                               bra-from-hermite
//   - exchange K_bc = sum_ad [ab|cd] D_ad ..................... Sec. 6
// The Hermite sign convention is the one of the E recursions above
// (Hermite Gaussians as derivatives with respect to the product centre),
// which is the convention under which Eq. pq carries (-1)^|q|.
//
// Everything is templated on the scalar type so that the same source built
// with `long double` certifies the `double` build. Plain loops; the only
// parallelism is OpenMP over independent shell quartets.
//
// Cartesian component order inside a shell of angular momentum l:
// a_x runs from l down to 0, then a_y from l-a_x down to 0 (xx,xy,xz,yy,yz,zz).
// A 4-center shellset is stored row-major as [a][b][c][d] (d fastest);
// a 3-center one as [a][c][d].

#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

template <typename T> T t_exp(T x);
template <> double t_exp<double>(double x) { return std::exp(x); }
template <> long double t_exp<long double>(long double x) { return expl(x); }
template <typename T> T t_sqrt(T x);
template <> double t_sqrt<double>(double x) { return std::sqrt(x); }
template <> long double t_sqrt<long double>(long double x) { return sqrtl(x); }
template <typename T> T t_erf(T x);
template <> double t_erf<double>(double x) { return std::erf(x); }
template <> long double t_erf<long double>(long double x) { return erfl(x); }

template <typename T> T pi_v() { return T(3.14159265358979323846264338327950288L); }

// Boys function F_m(x) = int_0^1 y^(2m) exp(-x y^2) dy (Eq. boys), m = 0..mmax.
// For x <= 30 + mmax: the convergent series
//   F_m(x) = exp(-x) sum_k (2x)^k / [(2m+1)(2m+3)...(2m+2k+1)],
// summed until a term is below eps * sum (all terms positive, no cancellation).
// Otherwise: F_0 = (1/2) sqrt(pi/x) erf(sqrt(x)) and the upward recursion
//   F_{m+1} = ((2m+1) F_m - exp(-x)) / (2x),
// which is stable while 2x > 2m+1.
template <typename T>
void boys(int mmax, T x, T* F) {
  const T eps = std::numeric_limits<T>::epsilon() * T(0.01);
  if (x <= T(30) + T(mmax)) {
    const T ex = t_exp<T>(-x);
    for (int m = 0; m <= mmax; ++m) {
      T term = T(1) / T(2 * m + 1);
      T sum = term;
      for (int k = 1; k < 100000; ++k) {
        term *= T(2) * x / T(2 * m + 2 * k + 1);
        sum += term;
        if (term < eps * sum) break;
      }
      F[m] = ex * sum;
    }
  } else {
    const T ex = t_exp<T>(-x);
    F[0] = T(0.5) * t_sqrt<T>(pi_v<T>() / x) * t_erf<T>(t_sqrt<T>(x));
    for (int m = 0; m < mmax; ++m) F[m + 1] = (T(2 * m + 1) * F[m] - ex) / (T(2) * x);
  }
}

// Cartesian components of a shell, in the library order.
struct Cart { int x, y, z; };
std::vector<Cart> cart_list(int l) {
  std::vector<Cart> v;
  for (int ax = l; ax >= 0; --ax)
    for (int ay = l - ax; ay >= 0; --ay) v.push_back({ax, ay, l - ax - ay});
  return v;
}
int ncart(int l) { return (l + 1) * (l + 2) / 2; }

// 2-center Hermite expansion coefficients along one axis, (E)_{ij}^t with
// 0<=i<=la, 0<=j<=lb, 0<=t<=i+j (Eqs. E2rr1, E2rr2, E2-000, E2-abp).
// Stored as E[(i*(lb+1)+j)*(la+lb+1)+t].
template <typename T>
std::vector<T> e_table_2c(int la, int lb, T za, T zb, T A, T B) {
  const int nt = la + lb + 1;
  std::vector<T> E((la + 1) * (lb + 1) * nt, T(0));
  const T p = za + zb;
  const T P = (za * A + zb * B) / p;
  const T XPA = P - A, XPB = P - B, XAB = A - B;
  const T inv2p = T(1) / (T(2) * p);
  auto at = [&](int i, int j, int t) -> T& { return E[(i * (lb + 1) + j) * nt + t]; };
  auto get = [&](int i, int j, int t) -> T {
    if (t < 0 || t > i + j) return T(0);
    return E[(i * (lb + 1) + j) * nt + t];
  };
  at(0, 0, 0) = t_exp<T>(-za * zb * XAB * XAB / p);              // Eq. E2-000
  for (int i = 0; i < la; ++i)                                     // Eq. E2rr1 (raise a)
    for (int t = 0; t <= i + 1; ++t)
      at(i + 1, 0, t) = inv2p * get(i, 0, t - 1) + XPA * get(i, 0, t) + T(t + 1) * get(i, 0, t + 1);
  for (int i = 0; i <= la; ++i)                                    // Eq. E2rr2 (raise b)
    for (int j = 0; j < lb; ++j)
      for (int t = 0; t <= i + j + 1; ++t)
        at(i, j + 1, t) = inv2p * get(i, j, t - 1) + XPB * get(i, j, t) + T(t + 1) * get(i, j, t + 1);
  return E;
}

// 1-center Hermite expansion coefficients along one axis, E_a^t with
// 0<=a<=la, 0<=t<=a (Eqs. E1rr, E1-00, E1-aa). Stored as E[a*(la+1)+t].
template <typename T>
std::vector<T> e_table_1c(int la, T za) {
  const int nt = la + 1;
  std::vector<T> E((la + 1) * nt, T(0));
  const T inv2a = T(1) / (T(2) * za);
  auto get = [&](int a, int t) -> T {
    if (t < 0 || t > a || ((t + a) & 1)) return T(0);              // Eq. E1-aa
    return E[a * nt + t];
  };
  E[0] = T(1);                                                     // Eq. E1-00
  for (int a = 0; a < la; ++a)                                     // Eq. E1rr
    for (int t = 0; t <= a + 1; ++t)
      E[(a + 1) * nt + t] = inv2a * get(a, t - 1) + T(t + 1) * get(a, t + 1);
  return E;
}

// Hermite auxiliary integrals [tuv]^(0) for t+u+v <= L (Eqs. 0m and r),
// built as the table R^(n)_{tuv} for n = L down to 0:
//   R^(n)_{000}   = (-2 rho)^n * pref * F_n(rho |P-Q|^2)
//   R^(n)_{t+1uv} = t R^(n+1)_{t-1uv} + X_PQ R^(n+1)_{tuv}   (and u with Y_PQ, v with Z_PQ)
// Returned as R0[(t*(L+1)+u)*(L+1)+v].
template <typename T>
std::vector<T> r_table(int L, T rho, T pref, const T PQ[3]) {
  const int d = L + 1;
  std::vector<T> F(L + 1);
  boys<T>(L, rho * (PQ[0] * PQ[0] + PQ[1] * PQ[1] + PQ[2] * PQ[2]), F.data());
  std::vector<T> R((size_t)d * d * d * d, T(0));
  auto at = [&](int n, int t, int u, int v) -> T& { return R[(((size_t)n * d + t) * d + u) * d + v]; };
  T fac = T(1);
  for (int n = 0; n <= L; ++n) { at(n, 0, 0, 0) = fac * pref * F[n]; fac *= T(-2) * rho; }
  for (int n = L - 1; n >= 0; --n) {
    for (int N = 1; N <= L - n; ++N)
      for (int t = 0; t <= N; ++t)
        for (int u = 0; u <= N - t; ++u) {
          const int v = N - t - u;
          T val;
          if (v > 0) {
            val = PQ[2] * at(n + 1, t, u, v - 1);
            if (v > 1) val += T(v - 1) * at(n + 1, t, u, v - 2);
          } else if (u > 0) {
            val = PQ[1] * at(n + 1, t, u - 1, v);
            if (u > 1) val += T(u - 1) * at(n + 1, t, u - 2, v);
          } else {
            val = PQ[0] * at(n + 1, t - 1, u, v);
            if (t > 1) val += T(t - 1) * at(n + 1, t - 2, u, v);
          }
          at(n, t, u, v) = val;
        }
  }
  std::vector<T> R0((size_t)d * d * d, T(0));
  for (int t = 0; t <= L; ++t)
    for (int u = 0; u + t <= L; ++u)
      for (int v = 0; v + u + t <= L; ++v) R0[((size_t)t * d + u) * d + v] = at(0, t, u, v);
  return R0;
}

// Basis description shared with the callers (plain arrays, one entry per shell).
struct Basis {
  const int32_t* l;
  const int32_t* nprim;
  const int32_t* prim_off;
  const double* center;   // [n_shells][3]
  const double* exps;
  const double* coefs;
};

// One contracted 4-center shellset [ab|cd] (Eq. def-abcd with Eq. 3),
// accumulated over all primitive quartets. out has ncart(la)*ncart(lb)*ncart(lc)*ncart(ld)
// entries in [a][b][c][d] order.
template <typename T>
void shellset4(const Basis& bs, int sa, int sb, int sc, int sd, T* out) {
  const int la = bs.l[sa], lb = bs.l[sb], lc = bs.l[sc], ld = bs.l[sd];
  const int Lb = la + lb, Lk = lc + ld, L = Lb + Lk, d = L + 1;
  const auto ca = cart_list(la), cb = cart_list(lb), cc = cart_list(lc), cd = cart_list(ld);
  const size_t nk = cc.size() * cd.size();
  const size_t nout = ca.size() * cb.size() * nk;
  for (size_t i = 0; i < nout; ++i) out[i] = T(0);
  const double* A = bs.center + 3 * sa; const double* B = bs.center + 3 * sb;
  const double* C = bs.center + 3 * sc; const double* D = bs.center + 3 * sd;
  const T pi = pi_v<T>();
  // Hermite bra index (t,u,v), t+u+v <= Lb; ket (tau,nu,phi), <= Lk.
  for (int ia = 0; ia < bs.nprim[sa]; ++ia)
  for (int ib = 0; ib < bs.nprim[sb]; ++ib) {
    const T za = bs.exps[bs.prim_off[sa] + ia], zb = bs.exps[bs.prim_off[sb] + ib];
    const T cab = T(bs.coefs[bs.prim_off[sa] + ia]) * T(bs.coefs[bs.prim_off[sb] + ib]);
    const T p = za + zb;
    T P[3];
    std::vector<T> Eab[3];
    for (int k = 0; k < 3; ++k) {
      P[k] = (za * T(A[k]) + zb * T(B[k])) / p;
      Eab[k] = e_table_2c<T>(la, lb, za, zb, T(A[k]), T(B[k]));
    }
    for (int ic = 0; ic < bs.nprim[sc]; ++ic)
    for (int id = 0; id < bs.nprim[sd]; ++id) {
      const T zc = bs.exps[bs.prim_off[sc] + ic], zd = bs.exps[bs.prim_off[sd] + id];
      const T ccd = T(bs.coefs[bs.prim_off[sc] + ic]) * T(bs.coefs[bs.prim_off[sd] + id]);
      const T q = zc + zd;
      T Q[3], PQ[3];
      std::vector<T> Ecd[3];
      for (int k = 0; k < 3; ++k) {
        Q[k] = (zc * T(C[k]) + zd * T(D[k])) / q;
        PQ[k] = P[k] - Q[k];
        Ecd[k] = e_table_2c<T>(lc, ld, zc, zd, T(C[k]), T(D[k]));
      }
      const T rho = p * q / (p + q);
      const T pref = T(2) * pi * pi * t_sqrt<T>(pi) / (p * q * t_sqrt<T>(p + q));   // Eq. 0m
      const std::vector<T> R = r_table<T>(L, rho, pref, PQ);
      auto Rat = [&](int t, int u, int v) { return R[((size_t)t * d + u) * d + v]; };
      const int ntb = Lb + 1, ntk = Lk + 1;
      // [p|cd] = sum_q (-1)^|q| E^{cd}_q [p+q]^(0)       (Eqs. pq, ket-from-hermite)
      std::vector<T> pket((size_t)(Lb + 1) * (Lb + 1) * (Lb + 1) * nk, T(0));
      for (int t = 0; t <= Lb; ++t)
      for (int u = 0; u + t <= Lb; ++u)
      for (int v = 0; v + u + t <= Lb; ++v) {
        T* row = &pket[(((size_t)t * (Lb + 1) + u) * (Lb + 1) + v) * nk];
        size_t kcol = 0;
        for (const Cart& c : cc)
        for (const Cart& dd : cd) {
          T s = T(0);
          for (int tau = 0; tau <= c.x + dd.x; ++tau)
          for (int nu = 0; nu <= c.y + dd.y; ++nu)
          for (int phi = 0; phi <= c.z + dd.z; ++phi) {
            const T e = Ecd[0][(c.x * (ld + 1) + dd.x) * ntk + tau] *
                        Ecd[1][(c.y * (ld + 1) + dd.y) * ntk + nu] *
                        Ecd[2][(c.z * (ld + 1) + dd.z) * ntk + phi];
            const T sgn = ((tau + nu + phi) & 1) ? T(-1) : T(1);
            s += sgn * e * Rat(t + tau, u + nu, v + phi);
          }
          row[kcol++] = s;
        }
      }
      // [ab|cd] += c_a c_b c_c c_d sum_p E^{ab}_p [p|cd]    (Eq. bra-from-hermite)
      const T w = cab * ccd;
      size_t o = 0;
      for (const Cart& a : ca)
      for (const Cart& b : cb) {
        for (size_t kcol = 0; kcol < nk; ++kcol) {
          T s = T(0);
          for (int t = 0; t <= a.x + b.x; ++t)
          for (int u = 0; u <= a.y + b.y; ++u)
          for (int v = 0; v <= a.z + b.z; ++v) {
            const T e = Eab[0][(a.x * (lb + 1) + b.x) * ntb + t] *
                        Eab[1][(a.y * (lb + 1) + b.y) * ntb + u] *
                        Eab[2][(a.z * (lb + 1) + b.z) * ntb + v];
            s += e * pket[(((size_t)t * (Lb + 1) + u) * (Lb + 1) + v) * nk + kcol];
          }
          out[o + kcol] += w * s;
        }
        o += nk;
      }
    }
  }
}

// One contracted 3-center shellset [a|cd] (Eq. def-acd with Eq. 3). The bra is a
// single Gaussian: zeta_p = zeta_a, P = A, 1-center E coefficients (Eq. E1rr).
// out has ncart(la)*ncart(lc)*ncart(ld) entries in [a][c][d] order.
template <typename T>
void shellset3(const Basis& aux, const Basis& orb, int sa, int sc, int sd, T* out) {
  const int la = aux.l[sa], lc = orb.l[sc], ld = orb.l[sd];
  const int Lk = lc + ld, L = la + Lk, d = L + 1;
  const auto ca = cart_list(la), cc = cart_list(lc), cd = cart_list(ld);
  const size_t nk = cc.size() * cd.size();
  const size_t nout = ca.size() * nk;
  for (size_t i = 0; i < nout; ++i) out[i] = T(0);
  const double* A = aux.center + 3 * sa;
  const double* C = orb.center + 3 * sc; const double* D = orb.center + 3 * sd;
  const T pi = pi_v<T>();
  for (int ia = 0; ia < aux.nprim[sa]; ++ia) {
    const T za = aux.exps[aux.prim_off[sa] + ia];
    const T ca_ = aux.coefs[aux.prim_off[sa] + ia];
    const std::vector<T> Ea = e_table_1c<T>(la, za);   // same for all three axes
    const int nta = la + 1;
    for (int ic = 0; ic < orb.nprim[sc]; ++ic)
    for (int id = 0; id < orb.nprim[sd]; ++id) {
      const T zc = orb.exps[orb.prim_off[sc] + ic], zd = orb.exps[orb.prim_off[sd] + id];
      const T ccd = T(orb.coefs[orb.prim_off[sc] + ic]) * T(orb.coefs[orb.prim_off[sd] + id]);
      const T q = zc + zd;
      T PQ[3];
      std::vector<T> Ecd[3];
      for (int k = 0; k < 3; ++k) {
        const T Qk = (zc * T(C[k]) + zd * T(D[k])) / q;
        PQ[k] = T(A[k]) - Qk;
        Ecd[k] = e_table_2c<T>(lc, ld, zc, zd, T(C[k]), T(D[k]));
      }
      const T p = za;
      const T rho = p * q / (p + q);
      const T pref = T(2) * pi * pi * t_sqrt<T>(pi) / (p * q * t_sqrt<T>(p + q));
      const std::vector<T> R = r_table<T>(L, rho, pref, PQ);
      auto Rat = [&](int t, int u, int v) { return R[((size_t)t * d + u) * d + v]; };
      const int ntk = Lk + 1;
      const T w = ca_ * ccd;
      size_t o = 0;
      for (const Cart& a : ca) {
        size_t kcol = 0;
        for (const Cart& c : cc)
        for (const Cart& dd : cd) {
          T s = T(0);
          for (int t = 0; t <= a.x; ++t)
          for (int u = 0; u <= a.y; ++u)
          for (int v = 0; v <= a.z; ++v) {
            const T ea = Ea[a.x * nta + t] * Ea[a.y * nta + u] * Ea[a.z * nta + v];
            if (ea == T(0)) continue;
            T sk = T(0);
            for (int tau = 0; tau <= c.x + dd.x; ++tau)
            for (int nu = 0; nu <= c.y + dd.y; ++nu)
            for (int phi = 0; phi <= c.z + dd.z; ++phi) {
              const T e = Ecd[0][(c.x * (ld + 1) + dd.x) * ntk + tau] *
                          Ecd[1][(c.y * (ld + 1) + dd.y) * ntk + nu] *
                          Ecd[2][(c.z * (ld + 1) + dd.z) * ntk + phi];
              const T sgn = ((tau + nu + phi) & 1) ? T(-1) : T(1);
              sk += sgn * e * Rat(t + tau, u + nu, v + phi);
            }
            s += ea * sk;
          }
          out[o + kcol] += w * s;
          ++kcol;
        }
        o += nk;
      }
    }
  }
}

int nthreads_or_default(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

template <typename T>
void eri4_batch(const Basis& bs, const int32_t* quartets, int64_t n, T* out, const int64_t* offsets, int nthreads) {
  const int nt = nthreads_or_default(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* s = quartets + 4 * q;
    shellset4<T>(bs, s[0], s[1], s[2], s[3], out + offsets[q]);
  }
}

template <typename T>
void eri3_batch(const Basis& aux, const Basis& orb, const int32_t* triplets, int64_t n, T* out,
                const int64_t* offsets, int nthreads) {
  const int nt = nthreads_or_default(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* s = triplets + 3 * q;
    shellset3<T>(aux, orb, s[0], s[1], s[2], out + offsets[q]);
  }
}

}  // namespace

extern "C" {

int orc_version() { return 1; }

// F_m(x), m = 0..mmax (Eq. boys). precision 0: double, 1: long double (result rounded).
void orc_boys(int mmax, double x, double* F, int precision) {
  if (precision == 1) {
    std::vector<long double> Fl(mmax + 1);
    boys<long double>(mmax, (long double)x, Fl.data());
    for (int m = 0; m <= mmax; ++m) F[m] = (double)Fl[m];
  } else {
    boys<double>(mmax, x, F);
  }
}

// Per-axis 2-center E table (Eqs. E2rr1/E2rr2): E[(i*(lb+1)+j)*(la+lb+1)+t].
void orc_e2c(int la, int lb, double za, double zb, double A, double B, double* E) {
  const auto v = e_table_2c<double>(la, lb, za, zb, A, B);
  std::memcpy(E, v.data(), v.size() * sizeof(double));
}

// Per-axis 1-center E table (Eq. E1rr): E[a*(la+1)+t].
void orc_e1c(int la, double za, double* E) {
  const auto v = e_table_1c<double>(la, za);
  std::memcpy(E, v.data(), v.size() * sizeof(double));
}

// Hermite auxiliary integrals [tuv]^(0) (Eqs. 0m, r) with pref = 1, rho, PQ given:
// R[(t*(L+1)+u)*(L+1)+v], zero outside t+u+v <= L.
void orc_rtable(int L, double rho, const double* PQ, double* R) {
  const auto v = r_table<double>(L, rho, 1.0, PQ);
  std::memcpy(R, v.data(), v.size() * sizeof(double));
}

// Real solid harmonics as Cartesian polynomials (the transformation the paper
// applies through its C coefficients, Eqs. solid2herm-1/2): the explicit form
//   S_lm = N_lm sum_t sum_u sum_v C_tuv x^(2t+|m|-2(u+v)) y^(2(u+v)) z^(l-2t-|m|),
//   C_tuv = (-1)^(t+v-v_m) (1/4)^t binom(l,t) binom(l-t,|m|+t) binom(t,u) binom(|m|,2v),
//   N_lm = sqrt(2 (l+|m|)! (l-|m|)! / 2^delta_m0) / (2^|m| l!),
// v_m = 0 (m >= 0) or 1/2 (m < 0), t <= (l-|m|)/2, u <= t, v from v_m in steps of 1
// up to |m|/2. Rows m = -l..l, columns the Cartesian components in library
// order: C[(m+l)*ncart(l) + k]. With this normalisation every S_lm has the
// angular norm of z^l, so functions built on x^l-normalised primitives stay
// normalised.
double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
double fact(int n) { double r = 1.0; for (int i = 2; i <= n; ++i) r *= i; return r; }

std::vector<double> solid_coefs(int l) {
  const auto cl = cart_list(l);
  std::vector<double> C((size_t)(2 * l + 1) * cl.size(), 0.0);
  for (int m = -l; m <= l; ++m) {
    const int am = m < 0 ? -m : m;
    const int vv0 = m < 0 ? 1 : 0;   // 2 v_m
    const double N = std::sqrt(2.0 * fact(l + am) * fact(l - am) / (m == 0 ? 2.0 : 1.0)) / (std::pow(2.0, am) * fact(l));
    for (int t = 0; 2 * t <= l - am; ++t)
      for (int u = 0; u <= t; ++u)
        for (int vv = vv0; vv <= am; vv += 2) {   // vv = 2v
          const int sgn_exp = t + (vv - vv0) / 2;
          const double c = ((sgn_exp & 1) ? -1.0 : 1.0) * std::pow(0.25, t) * binom(l, t) * binom(l - t, am + t) *
                           binom(t, u) * binom(am, vv);
          const int px = 2 * t + am - 2 * u - vv, py = 2 * u + vv, pz = l - 2 * t - am;
          for (size_t k = 0; k < cl.size(); ++k)
            if (cl[k].x == px && cl[k].y == py && cl[k].z == pz) C[(size_t)(m + l) * cl.size() + k] += N * c;
        }
  }
  return C;
}

// Batch of 4-center shellsets. quartets[n][4] are shell indices into the basis;
// shellset q is written at out + offsets[q]. precision 1 runs the long double build.
void orc_eri4(const int32_t* l, const int32_t* nprim, const int32_t* prim_off, const double* center,
              const double* exps, const double* coefs, const int32_t* quartets, int64_t n, double* out,
              const int64_t* offsets, int nthreads, int precision) {
  Basis bs{l, nprim, prim_off, center, exps, coefs};
  if (precision == 1) {
    int64_t total = 0;
    for (int64_t q = 0; q < n; ++q) {
      const int32_t* s = quartets + 4 * q;
      const int64_t sz = (int64_t)ncart(l[s[0]]) * ncart(l[s[1]]) * ncart(l[s[2]]) * ncart(l[s[3]]);
      total = std::max<int64_t>(total, offsets[q] + sz);
    }
    std::vector<long double> tmp(total);
    eri4_batch<long double>(bs, quartets, n, tmp.data(), offsets, nthreads);
    for (int64_t i = 0; i < total; ++i) out[i] = (double)tmp[i];
  } else {
    eri4_batch<double>(bs, quartets, n, out, offsets, nthreads);
  }
}

// Solid-harmonic coefficient matrix of one l (see solid_coefs): C[(2l+1)][ncart(l)].
void orc_solid_coefs(int l, double* C) {
  const auto v = solid_coefs(l);
  std::memcpy(C, v.data(), v.size() * sizeof(double));
}

// Batch of 4-center shellsets over real solid harmonics: the Cartesian shellset of
// shellset4 contracted with solid_coefs on each of its four indices,
//   [a'b'|c'd'] = sum_{abcd} C_{a'a} C_{b'b} C_{c'c} C_{d'd} [ab|cd],
// applied one index at a time (d, then c, b, a: the same sum regrouped), written
// [a][b][c][d] with m = -l..l in every position; shellset q at out + offsets[q].
// precision 1 runs the long double build (Cartesian shellset and transform),
// rounded at the end.
}  // extern "C"

// Cartesian shellset v (index k of extent dim[k] = ncart(L[k]), k < naxes, row-major) to real solid
// harmonics: every index contracted with the solid-harmonic coefficients of its l, one index at a time
// (Eqs. solid2herm-1/2 applied to the finished shellset).
template <typename T>
void to_solid(std::vector<T>& v, int* dim, const int* L, int naxes) {
  for (int axis = naxes - 1; axis >= 0; --axis) {   // contract index `axis`: ncart -> 2l+1
    const std::vector<double> C = solid_coefs(L[axis]);
    const int nc = dim[axis], ns = 2 * L[axis] + 1;
    size_t outer = 1, inner = 1;
    for (int k = 0; k < axis; ++k) outer *= dim[k];
    for (int k = axis + 1; k < naxes; ++k) inner *= dim[k];
    std::vector<T> w(outer * ns * inner, T(0));
    for (size_t o = 0; o < outer; ++o)
      for (int m = 0; m < ns; ++m)
        for (int c = 0; c < nc; ++c) {
          const T f = T(C[(size_t)m * nc + c]);
          for (size_t i = 0; i < inner; ++i) w[(o * ns + m) * inner + i] += f * v[(o * nc + c) * inner + i];
        }
    v.swap(w);
    dim[axis] = ns;
  }
}

template <typename T>
void eri4_sph_batch(const Basis& bs, const int32_t* l, const int32_t* quartets, int64_t n, double* out,
                    const int64_t* offsets, int nthreads) {
  const int nt = nthreads_or_default(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* s4 = quartets + 4 * q;
    const int L[4] = {l[s4[0]], l[s4[1]], l[s4[2]], l[s4[3]]};
    int dim[4] = {ncart(L[0]), ncart(L[1]), ncart(L[2]), ncart(L[3])};
    std::vector<T> v((size_t)dim[0] * dim[1] * dim[2] * dim[3]);
    shellset4<T>(bs, s4[0], s4[1], s4[2], s4[3], v.data());
    to_solid<T>(v, dim, L, 4);
    double* o = out + offsets[q];
    for (size_t i = 0; i < v.size(); ++i) o[i] = (double)v[i];
  }
}

// [a|cd] over real solid harmonics: the 3-center shellset (Eq. def-acd) with a, c and d transformed.
template <typename T>
void eri3_sph_batch(const Basis& aux, const Basis& orb, const int32_t* al, const int32_t* l, const int32_t* triplets,
                    int64_t n, double* out, const int64_t* offsets, int nthreads) {
  const int nt = nthreads_or_default(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* s3 = triplets + 3 * q;
    const int L[3] = {al[s3[0]], l[s3[1]], l[s3[2]]};
    int dim[3] = {ncart(L[0]), ncart(L[1]), ncart(L[2])};
    std::vector<T> v((size_t)dim[0] * dim[1] * dim[2]);
    shellset3<T>(aux, orb, s3[0], s3[1], s3[2], v.data());
    to_solid<T>(v, dim, L, 3);
    double* o = out + offsets[q];
    for (size_t i = 0; i < v.size(); ++i) o[i] = (double)v[i];
  }
}

extern "C" {

void orc_eri4_sph(const int32_t* l, const int32_t* nprim, const int32_t* prim_off, const double* center,
                  const double* exps, const double* coefs, const int32_t* quartets, int64_t n, double* out,
                  const int64_t* offsets, int nthreads, int precision) {
  Basis bs{l, nprim, prim_off, center, exps, coefs};
  if (precision == 1) eri4_sph_batch<long double>(bs, l, quartets, n, out, offsets, nthreads);
  else eri4_sph_batch<double>(bs, l, quartets, n, out, offsets, nthreads);
}

void orc_eri3_sph(const int32_t* al, const int32_t* anprim, const int32_t* aprim_off, const double* acenter,
                  const double* aexps, const double* acoefs, const int32_t* l, const int32_t* nprim,
                  const int32_t* prim_off, const double* center, const double* exps, const double* coefs,
                  const int32_t* triplets, int64_t n, double* out, const int64_t* offsets, int nthreads,
                  int precision) {
  Basis aux{al, anprim, aprim_off, acenter, aexps, acoefs};
  Basis orb{l, nprim, prim_off, center, exps, coefs};
  if (precision == 1) eri3_sph_batch<long double>(aux, orb, al, l, triplets, n, out, offsets, nthreads);
  else eri3_sph_batch<double>(aux, orb, al, l, triplets, n, out, offsets, nthreads);
}

// Batch of 3-center shellsets [a|cd]; triplets[n][3] = (aux shell, orb shell, orb shell).
void orc_eri3(const int32_t* al, const int32_t* anprim, const int32_t* aprim_off, const double* acenter,
              const double* aexps, const double* acoefs, const int32_t* l, const int32_t* nprim,
              const int32_t* prim_off, const double* center, const double* exps, const double* coefs,
              const int32_t* triplets, int64_t n, double* out, const int64_t* offsets, int nthreads,
              int precision) {
  Basis aux{al, anprim, aprim_off, acenter, aexps, acoefs};
  Basis orb{l, nprim, prim_off, center, exps, coefs};
  if (precision == 1) {
    int64_t total = 0;
    for (int64_t q = 0; q < n; ++q) {
      const int32_t* s = triplets + 3 * q;
      const int64_t sz = (int64_t)ncart(al[s[0]]) * ncart(l[s[1]]) * ncart(l[s[2]]);
      total = std::max<int64_t>(total, offsets[q] + sz);
    }
    std::vector<long double> tmp(total);
    eri3_batch<long double>(aux, orb, triplets, n, tmp.data(), offsets, nthreads);
    for (int64_t i = 0; i < total; ++i) out[i] = (double)tmp[i];
  } else {
    eri3_batch<double>(aux, orb, triplets, n, out, offsets, nthreads);
  }
}

// Dense exchange matrix K_ik = sum_jl D_jl (ij|kl) (Sec. 6 with a->j, b->i,
// c->k, d->l). The sum over all ordered shell quartets is regrouped by unique
// quartets {i>=j, k>=l, ij>=kl}: each shellset is evaluated once and every
// DISTINCT index permutation (p1,p2,p3,p4) of it adds D_{p2 p4} (p1 p2|p3 p4)
// to K_{p1 p3}. D and K are [nao][nao] row-major; ao_off[s] is the first AO
// of shell s.
void orc_exchange(const int32_t* l, const int32_t* nprim, const int32_t* prim_off, const double* center,
                  const double* exps, const double* coefs, const int32_t* ao_off, int32_t n_shells,
                  int32_t nao, const double* D, double* K, int nthreads) {
  Basis bs{l, nprim, prim_off, center, exps, coefs};
  for (int64_t i = 0; i < (int64_t)nao * nao; ++i) K[i] = 0.0;
  std::vector<std::array<int32_t, 4>> quarts;
  for (int32_t i = 0; i < n_shells; ++i)
    for (int32_t j = 0; j <= i; ++j)
      for (int32_t k = 0; k <= i; ++k)
        for (int32_t ll = 0; ll <= (k == i ? j : k); ++ll) quarts.push_back({i, j, k, ll});
  const int nt = nthreads_or_default(nthreads);
  std::vector<std::vector<double>> Kt(nt, std::vector<double>((size_t)nao * nao, 0.0));
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t n = 0; n < (int64_t)quarts.size(); ++n) {
#ifdef _OPENMP
    std::vector<double>& Kp = Kt[omp_get_thread_num()];
#else
    std::vector<double>& Kp = Kt[0];
#endif
    const auto& q = quarts[n];
    const int nc[4] = {ncart(l[q[0]]), ncart(l[q[1]]), ncart(l[q[2]]), ncart(l[q[3]])};
    std::vector<double> v((size_t)nc[0] * nc[1] * nc[2] * nc[3]);
    shellset4<double>(bs, q[0], q[1], q[2], q[3], v.data());
    // the 8 index permutations that leave (ij|kl) unchanged, as positions into (0,1,2,3)
    static const int perms[8][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {0, 1, 3, 2}, {1, 0, 3, 2},
                                    {2, 3, 0, 1}, {3, 2, 0, 1}, {2, 3, 1, 0}, {3, 2, 1, 0}};
    std::vector<std::array<int32_t, 4>> done;
    for (const auto& pm : perms) {
      const std::array<int32_t, 4> sh{q[pm[0]], q[pm[1]], q[pm[2]], q[pm[3]]};
      bool dup = false;
      for (const auto& d : done) dup = dup || d == sh;
      if (dup) continue;   // identical shell tuple: the same ordered quartet, counted once
      done.push_back(sh);
      const int n0 = nc[pm[0]], n1 = nc[pm[1]], n2 = nc[pm[2]], n3 = nc[pm[3]];
      int idx[4];
      for (idx[0] = 0; idx[0] < nc[0]; ++idx[0])
        for (idx[1] = 0; idx[1] < nc[1]; ++idx[1])
          for (idx[2] = 0; idx[2] < nc[2]; ++idx[2])
            for (idx[3] = 0; idx[3] < nc[3]; ++idx[3]) {
              const double val = v[(((size_t)idx[0] * nc[1] + idx[1]) * nc[2] + idx[2]) * nc[3] + idx[3]];
              const int a = idx[pm[0]], b = idx[pm[1]], c = idx[pm[2]], d = idx[pm[3]];
              (void)n0; (void)n1; (void)n2; (void)n3;
              Kp[(size_t)(ao_off[sh[0]] + a) * nao + ao_off[sh[2]] + c] +=
                  D[(size_t)(ao_off[sh[1]] + b) * nao + ao_off[sh[3]] + d] * val;
            }
    }
  }
  for (int t = 0; t < nt; ++t)
    for (int64_t i = 0; i < (int64_t)nao * nao; ++i) K[i] += Kt[t][i];
}

// Nuclear gradient of S = sum_{ijkl} D_ik D_jl (ij|kl) (the exchange energy
// E_x = alpha S with D held fixed; the paper lists geometric derivatives as
// future work, Sec. 7). Every ordered shell quartet and every one of its four
// centres is differentiated explicitly with the textbook rule for a primitive
// Cartesian Gaussian (Eq. 1):
//   d/dA_x [x_A^a exp(-z x_A^2)] = 2 z x_A^(a+1) exp(..) - a x_A^(a-1) exp(..),
// i.e. the shell is replaced by a shell of l+1 with coefficients 2 z c and one
// of l-1 with coefficients c. grad[atom][x] receives dS/dR for each centre
// on that atom; atom[s] is the atom of shell s. Plain loops over all
// quartets: small systems only.
void orc_exchange_grad(const int32_t* l, const int32_t* nprim, const int32_t* prim_off, const double* center,
                       const double* exps, const double* coefs, const int32_t* ao_off, const int32_t* atom,
                       int32_t n_shells, int32_t nao, const double* D, int32_t n_atoms, double* grad, int nthreads) {
  // augmented basis: original shells, then s+ (l+1, 2 z c), then s- (l-1, c; only for l >= 1)
  const int32_t n = n_shells;
  std::vector<int32_t> L(3 * n), NP(3 * n), PO(3 * n);
  std::vector<double> CEN(9 * n), EX, CO;
  for (int32_t s = 0; s < n; ++s)
    for (int v = 0; v < 3; ++v) {
      const int32_t t = v * n + s;
      L[t] = v == 0 ? l[s] : (v == 1 ? l[s] + 1 : std::max(l[s] - 1, 0));
      NP[t] = nprim[s];
      PO[t] = (int32_t)EX.size();
      for (int k = 0; k < 3; ++k) CEN[3 * t + k] = center[3 * s + k];
      for (int p = 0; p < nprim[s]; ++p) {
        const double z = exps[prim_off[s] + p], c = coefs[prim_off[s] + p];
        EX.push_back(z);
        CO.push_back(v == 1 ? 2.0 * z * c : c);
      }
    }
  Basis bs{L.data(), NP.data(), PO.data(), CEN.data(), EX.data(), CO.data()};
  for (int64_t i = 0; i < (int64_t)n_atoms * 3; ++i) grad[i] = 0.0;
  const int nt = nthreads_or_default(nthreads);
  std::vector<std::vector<double>> G(nt, std::vector<double>((size_t)n_atoms * 3, 0.0));
  const int64_t nq = (int64_t)n * n * n * n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t qi = 0; qi < nq; ++qi) {
#ifdef _OPENMP
    std::vector<double>& g = G[omp_get_thread_num()];
#else
    std::vector<double>& g = G[0];
#endif
    const int32_t sh[4] = {(int32_t)(qi / ((int64_t)n * n * n)), (int32_t)((qi / ((int64_t)n * n)) % n),
                           (int32_t)((qi / n) % n), (int32_t)(qi % n)};
    const int nc[4] = {ncart(l[sh[0]]), ncart(l[sh[1]]), ncart(l[sh[2]]), ncart(l[sh[3]])};
    for (int pos = 0; pos < 4; ++pos) {
      const int lp = l[sh[pos]];
      const auto cp = cart_list(lp);
      const auto cplus = cart_list(lp + 1);
      const auto cminus = cart_list(lp > 0 ? lp - 1 : 0);
      auto index_of = [](const std::vector<Cart>& cl, int x, int y, int z) {
        for (size_t i = 0; i < cl.size(); ++i)
          if (cl[i].x == x && cl[i].y == y && cl[i].z == z) return (int)i;
        return -1;
      };
      int sp[4] = {sh[0], sh[1], sh[2], sh[3]}, sm[4] = {sh[0], sh[1], sh[2], sh[3]};
      sp[pos] = n + sh[pos];
      sm[pos] = 2 * n + sh[pos];
      int ncp[4] = {nc[0], nc[1], nc[2], nc[3]}, ncm[4] = {nc[0], nc[1], nc[2], nc[3]};
      ncp[pos] = ncart(lp + 1);
      ncm[pos] = ncart(lp > 0 ? lp - 1 : 0);
      std::vector<double> vp((size_t)ncp[0] * ncp[1] * ncp[2] * ncp[3]);
      shellset4<double>(bs, sp[0], sp[1], sp[2], sp[3], vp.data());
      std::vector<double> vm;
      if (lp > 0) {
        vm.resize((size_t)ncm[0] * ncm[1] * ncm[2] * ncm[3]);
        shellset4<double>(bs, sm[0], sm[1], sm[2], sm[3], vm.data());
      }
      double acc[3] = {0.0, 0.0, 0.0};
      int idx[4];
      for (idx[0] = 0; idx[0] < nc[0]; ++idx[0])
        for (idx[1] = 0; idx[1] < nc[1]; ++idx[1])
          for (idx[2] = 0; idx[2] < nc[2]; ++idx[2])
            for (idx[3] = 0; idx[3] < nc[3]; ++idx[3]) {
              const double w = D[(size_t)(ao_off[sh[0]] + idx[0]) * nao + ao_off[sh[2]] + idx[2]] *
                               D[(size_t)(ao_off[sh[1]] + idx[1]) * nao + ao_off[sh[3]] + idx[3]];
              const Cart a = cp[idx[pos]];
              for (int dir = 0; dir < 3; ++dir) {
                const int dx = dir == 0, dy = dir == 1, dz = dir == 2;
                int jp[4] = {idx[0], idx[1], idx[2], idx[3]};
                jp[pos] = index_of(cplus, a.x + dx, a.y + dy, a.z + dz);
                double val = vp[(((size_t)jp[0] * ncp[1] + jp[1]) * ncp[2] + jp[2]) * ncp[3] + jp[3]];
                const int am = dir == 0 ? a.x : (dir == 1 ? a.y : a.z);
                if (am > 0) {
                  int jm[4] = {idx[0], idx[1], idx[2], idx[3]};
                  jm[pos] = index_of(cminus, a.x - dx, a.y - dy, a.z - dz);
                  val -= am * vm[(((size_t)jm[0] * ncm[1] + jm[1]) * ncm[2] + jm[2]) * ncm[3] + jm[3]];
                }
                acc[dir] += w * val;
              }
            }
      for (int dir = 0; dir < 3; ++dir) g[(size_t)atom[sh[pos]] * 3 + dir] += acc[dir];
    }
  }
  for (int t = 0; t < nt; ++t)
    for (int64_t i = 0; i < (int64_t)n_atoms * 3; ++i) grad[i] += G[t][i];
}

// Rows of K_ik = sum_jl D_jl (ij|kl) for the shells in row_shells only,
// summed directly over all (j, k, l) shells; other rows are left zero.
void orc_exchange_rows(const int32_t* l, const int32_t* nprim, const int32_t* prim_off, const double* center,
                       const double* exps, const double* coefs, const int32_t* ao_off, int32_t n_shells,
                       int32_t nao, const double* D, double* K, const int32_t* row_shells, int32_t nrows,
                       int nthreads) {
  Basis bs{l, nprim, prim_off, center, exps, coefs};
  for (int64_t i = 0; i < (int64_t)nao * nao; ++i) K[i] = 0.0;
  const int nt = nthreads_or_default(nthreads);
  const int64_t ntask = (int64_t)nrows * n_shells;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t task = 0; task < ntask; ++task) {
    const int32_t si = row_shells[task / n_shells];
    const int32_t sk = (int32_t)(task % n_shells);
    const int ni = ncart(l[si]), nk = ncart(l[sk]);
    std::vector<double> blk((size_t)ni * nk, 0.0);
    for (int32_t sj = 0; sj < n_shells; ++sj)
      for (int32_t sl = 0; sl < n_shells; ++sl) {
        const int nj = ncart(l[sj]), nl = ncart(l[sl]);
        std::vector<double> v((size_t)ni * nj * nk * nl);
        shellset4<double>(bs, si, sj, sk, sl, v.data());
        for (int a = 0; a < ni; ++a)
          for (int b = 0; b < nj; ++b)
            for (int c = 0; c < nk; ++c)
              for (int d = 0; d < nl; ++d)
                blk[(size_t)a * nk + c] +=
                    D[(size_t)(ao_off[sj] + b) * nao + ao_off[sl] + d] * v[(((size_t)a * nj + b) * nk + c) * nl + d];
      }
    for (int a = 0; a < ni; ++a)
      for (int c = 0; c < nk; ++c) K[(size_t)(ao_off[si] + a) * nao + ao_off[sk] + c] = blk[(size_t)a * nk + c];
  }
}

}  // extern "C"
