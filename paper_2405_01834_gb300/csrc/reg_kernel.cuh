// Register-resident quartet kernel for small classes: one thread per shell
// quartet, every intermediate of Sec. 2 in registers (the paper's smallest
// GPU variant V0, Sec. 3, where a thread owns a whole shellset).
//
// Per thread, for every bra primitive pair and every ket primitive pair:
// Boys seeds [0]^(m) = (-2 rho)^m pref F_m(T) (Eq. 0m), the Hermite integrals
// [tuv] by Eq. r computed in place (orders high to low), and the ket
// transform [p|cd] += sum_q (-1)^|q| E^cd_q [p+q] (Eqs. pq, ket-from-hermite;
// the ket records carry the sign); after the ket primitives, the bra
// transform [ab|cd] += sum_p E^ab_p [p|cd] (Eq. bra-from-hermite). All loop
// bounds and indices are compile-time constants, so the arrays live in
// registers. Only the store and the exchange-digestion epilogues exist here;
// gradient launches use the team kernel.
#pragma once

#include <utility>

#include "kernels.cuh"

namespace mdx {
namespace reg {

constexpr __host__ __device__ int ncart(int l) { return (l + 1) * (l + 2) / 2; }
constexpr __host__ __device__ int tet(int n) { return n < 0 ? 0 : n * (n + 1) * (n + 2) / 6; }
constexpr __host__ __device__ int tri(int n) { return n < 0 ? 0 : n * (n + 1) / 2; }
constexpr __host__ __device__ int nherm(int L) { return tet(L + 1); }
// (t,u,v) -> position in a [t][u][v] simplex of total order N (t+u+v <= N)
constexpr __host__ __device__ int hidx(int N, int t, int u, int v) {
  return tet(N + 1) - tet(N - t + 1) + tri(N - t + 1) - tri(N - t - u + 1) + v;
}
// Cartesian component k of shell l (a_x = l..0, then a_y = l-a_x..0)
constexpr __host__ __device__ int cx(int l, int k) {
  int ax = l;
  while (k > l - ax) { k -= l - ax + 1; --ax; }
  return ax;
}
constexpr __host__ __device__ int cy(int l, int k) {
  int ax = l;
  while (k > l - ax) { k -= l - ax + 1; --ax; }
  return l - ax - k;
}
constexpr __host__ __device__ int cz(int l, int k) { return l - cx(l, k) - cy(l, k); }
// per-axis E table of a record: (a,b) block start, t contiguous (library record layout)
constexpr __host__ __device__ int etab_size(int la, int lb) {
  int s = 0;
  for (int a = 0; a <= la; ++a)
    for (int b = 0; b <= lb; ++b) s += a + b + 1;
  return s;
}
constexpr __host__ __device__ int etab_off(int lb, int a, int b) {
  int s = 0;
  for (int a2 = 0; a2 < a; ++a2)
    for (int b2 = 0; b2 <= lb; ++b2) s += a2 + b2 + 1;
  for (int b2 = 0; b2 < b; ++b2) s += a + b2 + 1;
  return s;
}
constexpr __host__ __device__ int rec_size(int la, int lb) { return (kRecHeader + 3 * etab_size(la, lb) + 1) & ~1; }

// Compile-time loop: f(Ic<I>) for I = 0..N-1 (Ic<I> converts to the constant I).
template <int I>
struct Ic {
  static constexpr int value = I;
  constexpr __host__ __device__ operator int() const { return I; }
};
template <typename F, int... I>
__device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(Ic<I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (N > 0) sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// Per-thread array of N doubles: in registers (SH = false), or one column of a
// block-wide shared-memory table (element i of thread t at p[i * kXsBlock]).
// (Single-warp blocks pack the shared memory more tightly but measured slower
// on [pp|pp] (-5 %) and no faster on the exchange, gradient and 3-center runs.)
constexpr int kXsBlock = 64;
constexpr int kRegMaxDevices = 64;
template <bool SH, int N>
struct TArr {
  double r[N];
  __device__ __forceinline__ double& operator[](int i) { return r[i]; }
};
template <int N>
struct TArr<true, N> {
  double* p;
  __device__ __forceinline__ double& operator[](int i) { return p[i * kXsBlock]; }
};

// XS = false: R, [p|cd] and the shellset in registers (classes with
// reg_eligible). XS = true: R in registers, [p|cd] and the shellset in shared
// memory (classes with reg_xs_eligible, total angular momentum <= 6).
template <int LA, int LB, int LC, int LD, bool DIGEST, bool XS>
__global__ void __launch_bounds__(XS ? kXsBlock : 128) k_reg(const QuartetLaunch a) {
  constexpr int Lb = LA + LB, Lk = LC + LD, L = Lb + Lk;
  constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  constexpr int Nb = NA * NB, Nk = NC * ND;
  constexpr int HB = nherm(Lb), HL = nherm(L);
  constexpr int RB = rec_size(LA, LB), RK = rec_size(LC, LD);
  constexpr int EB = etab_size(LA, LB), EK = etab_size(LC, LD);

  extern __shared__ double xs_smem[];
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.nq) return;
  const int2 qp = a.qpairs[q];
  const double* __restrict__ rb0 = a.recs + a.pair_rec[qp.x + a.bra_var_off];
  const double* __restrict__ rk0 = a.recs_signed + a.pair_rec[qp.y + a.ket_var_off];
  const double* __restrict__ boys = a.boys;
  const int Kb = a.plan.Kb, Kk = a.plan.Kk;

  // shared-memory variant: [p|cd] in shared memory, and the shellset too when the digestion epilogue needs
  // it whole; the store epilogue adds each bra pair's row straight into the output instead (less shared
  // memory per thread, more warps per SM)
  constexpr bool VSH = XS && DIGEST;
  TArr<XS, Nb * Nk> V;
  TArr<XS, HB * Nk> X;
  if constexpr (XS) {
    V.p = xs_smem + threadIdx.x;
    X.p = xs_smem + (VSH ? Nb * Nk : 0) * kXsBlock + threadIdx.x;
  }
  if constexpr (!XS || VSH) sfor<Nb * Nk>([&](auto i) { V[i] = 0.0; });
  double* const outq = DIGEST ? nullptr : a.out + (a.qout ? a.qout[q] : q * (int64_t)(Nb * Nk));

  for (int pb = 0; pb < Kb; ++pb) {
    const double* __restrict__ rb = rb0 + (int64_t)pb * RB;
    const double zp = __ldg(rb), izp = __ldg(rb + 1);
    const double Px = __ldg(rb + 2), Py = __ldg(rb + 3), Pz = __ldg(rb + 4);
    // 2 pi^(5/2) / zp * c_a c_b K_ab (the ket part and 1/sqrt(zp+zq) per ket primitive)
    const double prefb = 34.986836655249725693 * izp * __ldg(rb + 5);
    sfor<HB * Nk>([&](auto i) { X[i] = 0.0; });

    for (int pk = 0; pk < Kk; ++pk) {
      const double* __restrict__ rk = rk0 + (int64_t)pk * RK;
      const double zq = __ldg(rk), izq = __ldg(rk + 1);
      const double PQx = Px - __ldg(rk + 2), PQy = Py - __ldg(rk + 3), PQz = Pz - __ldg(rk + 4);
      const double s = zp + zq;
      const double rs = rsqrt(s);
      const double rho = zp * zq * rs * rs;
      const double Tb = rho * (PQx * PQx + PQy * PQy + PQz * PQz);
      const double pref = prefb * izq * rs * __ldg(rk + 5);
      const double m2r = -2.0 * rho;
      // Boys seeds G[m] = (-2 rho)^m pref F_m(T), m = 0..L (Eq. 0m)
      double G[L + 1];
      if (Tb < kBoysTmax) {
        const int i = __double2int_rn(Tb * kBoysInvH);
        const double nd = (double)i * (1.0 / kBoysInvH) - Tb;
        const double2* row = reinterpret_cast<const double2*>(boys + (size_t)i * kBoysRow);
        double pw = pref;
        sfor<L + 1>([&](auto m) {
          const double2 c01 = __ldg(row + 4 * m), c23 = __ldg(row + 4 * m + 1);
          const double2 c45 = __ldg(row + 4 * m + 2), c67 = __ldg(row + 4 * m + 3);
          double f = fma(c67.y, nd, c67.x);
          f = fma(f, nd, c45.y);
          f = fma(f, nd, c45.x);
          f = fma(f, nd, c23.y);
          f = fma(f, nd, c23.x);
          f = fma(f, nd, c01.y);
          f = fma(f, nd, c01.x);
          G[m] = pw * f;
          pw *= m2r;
        });
      } else {
        // F_m(T) = Gamma(m+1/2) / (2 T^(m+1/2)), Gamma(m+1/2)/2 = sqrt(pi)/2 (2m-1)!!/2^m
        // (exp(-T) terms negligible above the table)
        const double t1 = rsqrt(Tb);
        const double x = m2r * t1 * t1;
        double g = 0.88622692545275801365 * pref * t1;
        sfor<L + 1>([&](auto m) {
          G[m] = g;
          g *= x * ((double)m + 0.5);
        });
      }
      // R^(n)_tuv for n = L..0 in one array indexed in the order-L simplex:
      // level n overwrites orders N = L-n..1 from the top down (an entry reads
      // orders N-1 and N-2 of level n+1, not yet overwritten), then [000]
      double R[HL];
      R[0] = G[L];
      sfor<L>([&](auto k) {
        constexpr int n = L - 1 - k;
        sfor<L - n>([&](auto j) {
          constexpr int N = L - n - j;
          sfor<N + 1>([&](auto t) {
            sfor<N + 1 - t>([&](auto u) {
              constexpr int v = N - t - u;
              double val;
              if constexpr (v > 0) {
                val = PQz * R[hidx(L, t, u, v - 1)];
                if constexpr (v > 1) val = fma((double)(v - 1), R[hidx(L, t, u, v - 2)], val);
              } else if constexpr (u > 0) {
                val = PQy * R[hidx(L, t, u - 1, 0)];
                if constexpr (u > 1) val = fma((double)(u - 1), R[hidx(L, t, u - 2, 0)], val);
              } else {
                val = PQx * R[hidx(L, t - 1, 0, 0)];
                if constexpr (t > 1) val = fma((double)(t - 1), R[hidx(L, t - 2, 0, 0)], val);
              }
              R[hidx(L, t, u, v)] = val;
            });
          });
        });
        R[0] = G[n];
      });
      // ket transform: X[p][cd] += sum_{tau,nu,phi} Ex Ey Ez (signed tables) R[p + q]
      sfor<NC>([&](auto c) {
        sfor<ND>([&](auto d) {
          constexpr int ex = cx(LC, c), ey = cy(LC, c), ez = cz(LC, c);
          constexpr int fx = cx(LD, d), fy = cy(LD, d), fz = cz(LD, d);
          constexpr int nx = ex + fx + 1, ny = ey + fy + 1, nz = ez + fz + 1;
          const double* Ex = rk + kRecHeader + etab_off(LD, ex, fx);
          const double* Ey = rk + kRecHeader + EK + etab_off(LD, ey, fy);
          const double* Ez = rk + kRecHeader + 2 * EK + etab_off(LD, ez, fz);
          double E[nx * ny * nz];
          sfor<nx>([&](auto tau) {
            const double vx = __ldg(Ex + tau);
            sfor<ny>([&](auto nu) {
              const double vxy = vx * __ldg(Ey + nu);
              sfor<nz>([&](auto phi) { E[(tau * ny + nu) * nz + phi] = vxy * __ldg(Ez + phi); });
            });
          });
          sfor<Lb + 1>([&](auto t) {
            sfor<Lb + 1 - t>([&](auto u) {
              sfor<Lb + 1 - t - u>([&](auto v) {
                constexpr int o = hidx(Lb, t, u, v) * Nk + c * ND + d;
                double acc = X[o];
                sfor<nx>([&](auto tau) {
                  sfor<ny>([&](auto nu) {
                    sfor<nz>([&](auto phi) {
                      acc = fma(E[(tau * ny + nu) * nz + phi], R[hidx(L, t + tau, u + nu, v + phi)], acc);
                    });
                  });
                });
                X[o] = acc;
              });
            });
          });
        });
      });
    }
    // bra transform: V[ab][cd] += sum_{t,u,v} Ex Ey Ez X[tuv][cd]
    if constexpr (XS) {
      // [p|cd] and the shellset are in shared memory: runtime loops over ab and
      // (t,u,v), the ket pairs cd unrolled (keeps the unrolled body small)
      for (int ia = 0; ia < NA; ++ia) {
        const int ax = cx(LA, ia), ay = cy(LA, ia), az = LA - ax - ay;
        for (int ib = 0; ib < NB; ++ib) {
          const int bx = cx(LB, ib), by = cy(LB, ib), bz = LB - bx - by;
          const double* Ex = rb + kRecHeader + etab_off(LB, ax, bx);
          const double* Ey = rb + kRecHeader + EB + etab_off(LB, ay, by);
          const double* Ez = rb + kRecHeader + 2 * EB + etab_off(LB, az, bz);
          double acc[Nk];
          sfor<Nk>([&](auto cd) { acc[cd] = 0.0; });
          for (int t = 0; t <= ax + bx; ++t) {
            const double vx = __ldg(Ex + t);
            for (int u = 0; u <= ay + by; ++u) {
              const double vxy = vx * __ldg(Ey + u);
              for (int v = 0; v <= az + bz; ++v) {
                const double e = vxy * __ldg(Ez + v);
                const int h = hidx(Lb, t, u, v) * Nk;
                sfor<Nk>([&](auto cd) { acc[cd] = fma(e, X[h + cd], acc[cd]); });
              }
            }
          }
          const int o = (ia * NB + ib) * Nk;
          if constexpr (VSH) {
            sfor<Nk>([&](auto cd) { V[o + cd] += acc[cd]; });
          } else if (pb == 0) {
            sfor<Nk>([&](auto cd) { outq[o + cd] = acc[cd]; });
          } else {
            sfor<Nk>([&](auto cd) { outq[o + cd] += acc[cd]; });
          }
        }
      }
    } else {
      sfor<NA>([&](auto ia) {
        sfor<NB>([&](auto ib) {
          constexpr int ax = cx(LA, ia), ay = cy(LA, ia), az = cz(LA, ia);
          constexpr int bx = cx(LB, ib), by = cy(LB, ib), bz = cz(LB, ib);
          constexpr int nx = ax + bx + 1, ny = ay + by + 1, nz = az + bz + 1;
          const double* Ex = rb + kRecHeader + etab_off(LB, ax, bx);
          const double* Ey = rb + kRecHeader + EB + etab_off(LB, ay, by);
          const double* Ez = rb + kRecHeader + 2 * EB + etab_off(LB, az, bz);
          double E[nx * ny * nz];
          sfor<nx>([&](auto t) {
            const double vx = __ldg(Ex + t);
            sfor<ny>([&](auto u) {
              const double vxy = vx * __ldg(Ey + u);
              sfor<nz>([&](auto v) { E[(t * ny + u) * nz + v] = vxy * __ldg(Ez + v); });
            });
          });
          sfor<Nk>([&](auto cd) {
            constexpr int o = (ia * NB + ib) * Nk + cd;
            double acc = V[o];
            sfor<nx>([&](auto t) {
              sfor<ny>([&](auto u) {
                sfor<nz>([&](auto v) { acc = fma(E[(t * ny + u) * nz + v], X[hidx(Lb, t, u, v) * Nk + cd], acc); });
              });
            });
            V[o] = acc;
          });
        });
      });
    }
  }

  if constexpr (!DIGEST) {
    // (no offsets: shellsets back to back); the shared-memory variant has written its rows already
    if constexpr (!XS) sfor<Nb * Nk>([&](auto i) { outq[i] = V[i]; });
  } else {
    // Exchange digestion of the unique quartet (ij|kl) with weight w, as in
    // the team kernel: K_ik += w D_jl V, K_il += w D_jk V, K_jk += w D_il V,
    // K_jl += w D_ik V (the host adds K^T afterwards).
    const int2 bp = a.pair_shells[qp.x], kp = a.pair_shells[qp.y];
    const int si = bp.x, sj = bp.y, sk = kp.x, sl = kp.y;
    const double w = (si == sj ? 0.5 : 1.0) * (sk == sl ? 0.5 : 1.0) * (qp.x == qp.y ? 0.5 : 1.0);
    const int mol = a.pair_mol ? a.pair_mol[qp.x] : -1;
    const int64_t nao = mol >= 0 ? a.mol_nao[mol] : a.nao;
    const double* __restrict__ D = mol >= 0 ? a.mol_D[mol] : a.D;
    double* K = mol >= 0 ? a.mol_K[mol] : a.K;
    const int64_t ai = a.ao_off[si], aj = a.ao_off[sj], ak = a.ao_off[sk], al = a.ao_off[sl];
    if constexpr (XS) {
      // the shellset is in shared memory: runtime loops
      auto Vr = [&](int x, int b, int c, int d) -> double { return V[((x * NB + b) * NC + c) * ND + d]; };
      for (int x = 0; x < NA; ++x) {
        for (int c = 0; c < NC; ++c) {   // K_ik
          double s1 = 0.0;
          for (int b = 0; b < NB; ++b)
            for (int d = 0; d < ND; ++d) s1 = fma(__ldg(D + (aj + b) * nao + al + d), Vr(x, b, c, d), s1);
          atomicAdd(K + (ai + x) * nao + ak + c, w * s1);
        }
        for (int d = 0; d < ND; ++d) {   // K_il
          double s2 = 0.0;
          for (int b = 0; b < NB; ++b)
            for (int c = 0; c < NC; ++c) s2 = fma(__ldg(D + (aj + b) * nao + ak + c), Vr(x, b, c, d), s2);
          atomicAdd(K + (ai + x) * nao + al + d, w * s2);
        }
      }
      for (int x = 0; x < NB; ++x) {
        for (int c = 0; c < NC; ++c) {   // K_jk
          double s3 = 0.0;
          for (int y = 0; y < NA; ++y)
            for (int d = 0; d < ND; ++d) s3 = fma(__ldg(D + (ai + y) * nao + al + d), Vr(y, x, c, d), s3);
          atomicAdd(K + (aj + x) * nao + ak + c, w * s3);
        }
        for (int d = 0; d < ND; ++d) {   // K_jl
          double s4 = 0.0;
          for (int y = 0; y < NA; ++y)
            for (int c = 0; c < NC; ++c) s4 = fma(__ldg(D + (ai + y) * nao + ak + c), Vr(y, x, c, d), s4);
          atomicAdd(K + (aj + x) * nao + al + d, w * s4);
        }
      }
    } else {
      auto Vat = [&](auto x, auto b, auto c, auto d) -> double { return V[((x * NB + b) * NC + c) * ND + d]; };
      sfor<NA>([&](auto x) {
        sfor<NC>([&](auto c) {   // K_ik
          double s1 = 0.0;
          sfor<NB>([&](auto b) {
            sfor<ND>([&](auto d) { s1 = fma(__ldg(D + (aj + b) * nao + al + d), Vat(x, b, c, d), s1); });
          });
          atomicAdd(K + (ai + x) * nao + ak + c, w * s1);
        });
        sfor<ND>([&](auto d) {   // K_il
          double s2 = 0.0;
          sfor<NB>([&](auto b) {
            sfor<NC>([&](auto c) { s2 = fma(__ldg(D + (aj + b) * nao + ak + c), Vat(x, b, c, d), s2); });
          });
          atomicAdd(K + (ai + x) * nao + al + d, w * s2);
        });
      });
      sfor<NB>([&](auto x) {
        sfor<NC>([&](auto c) {   // K_jk
          double s3 = 0.0;
          sfor<NA>([&](auto y) {
            sfor<ND>([&](auto d) { s3 = fma(__ldg(D + (ai + y) * nao + al + d), Vat(y, x, c, d), s3); });
          });
          atomicAdd(K + (aj + x) * nao + ak + c, w * s3);
        });
        sfor<ND>([&](auto d) {   // K_jl
          double s4 = 0.0;
          sfor<NA>([&](auto y) {
            sfor<NC>([&](auto c) { s4 = fma(__ldg(D + (ai + y) * nao + ak + c), Vat(y, x, c, d), s4); });
          });
          atomicAdd(K + (aj + x) * nao + al + d, w * s4);
        });
      });
    }
  }
}

template <int LA, int LB, int LC, int LD>
cudaError_t launch_reg_class(const QuartetLaunch& a, cudaStream_t s) {
  constexpr bool XS = !reg_eligible(LA, LB, LC, LD);
  constexpr int bs = XS ? kXsBlock : 128;
  constexpr int Nk = ncart(LC) * ncart(LD);
  // shared memory per block: [p|cd] (and, with the digestion epilogue, the shellset) of every thread
  constexpr size_t shm_x = XS ? (size_t)nherm(LA + LB) * Nk * kXsBlock * sizeof(double) : 0;
  constexpr size_t shm_d = XS ? (size_t)ncart(LA) * ncart(LB) * Nk * kXsBlock * sizeof(double) + shm_x : 0;
  const int64_t grid = (a.nq + bs - 1) / bs;
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  if constexpr (shm_d > 48 * 1024) {
    // opt in to more than 48 KB of dynamic shared memory, once per instance and device
    static bool attr[kRegMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kRegMaxDevices) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
      e = cudaFuncSetAttribute(k_reg<LA, LB, LC, LD, true, XS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)shm_d);
      if (e == cudaSuccess && shm_x > 48 * 1024)
        e = cudaFuncSetAttribute(k_reg<LA, LB, LC, LD, false, XS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shm_x);
      if (e != cudaSuccess) return e;
      attr[dev] = true;
    }
  }
  if (a.D) k_reg<LA, LB, LC, LD, true, XS><<<(unsigned)grid, bs, shm_d, s>>>(a);
  else k_reg<LA, LB, LC, LD, false, XS><<<(unsigned)grid, bs, shm_x, s>>>(a);
  return cudaGetLastError();
}

using RegLaunchFn = cudaError_t (*)(const QuartetLaunch&, cudaStream_t);

// Launcher of class code C = ((la*7 + lb)*7 + lc)*7 + ld, or nullptr when the
// class has no register kernel.
template <int C>
constexpr RegLaunchFn reg_fn() {
  constexpr int la = C / 343, lb = C / 49 % 7, lc = C / 7 % 7, ld = C % 7;
  if constexpr (reg_eligible(la, lb, lc, ld) || reg_xs_eligible(la, lb, lc, ld))
    return &launch_reg_class<la, lb, lc, ld>;
  else return nullptr;
}
template <int BASE, int... I>
__host__ RegLaunchFn reg_pick(int code, std::integer_sequence<int, I...>) {
  constexpr RegLaunchFn table[] = {reg_fn<BASE + I>()...};
  return table[code - BASE];
}

}  // namespace reg
}  // namespace mdx
