// CUDA kernels of the McMurchie-Davidson engine (sm_103a, FP64).
//
// Two kernels carry the method:
//  * k_pair_records: per primitive pair, zeta_p, P, the prefactor
//    c_a c_b exp(-zeta_a zeta_b |A-B|^2 / zeta_p) (Eq. E2-000 folded into one
//    scalar) and the three per-axis Hermite tables (E_i)_{ab}^t from
//    Eqs. E2rr1/E2rr2 (one-centre bra: Eq. E1rr), plain and with the ket sign
//    (-1)^t of Eq. pq folded in.
//  * k_quartets: one team of threads per shell quartet. For every primitive
//    quartet the team forms the Boys seeds [0]^(m) (Eq. 0m), the Hermite
//    integrals [tuv]^(0) (Eq. r) and applies the ket transform
//    (Eq. ket-from-hermite) axis by axis; per bra primitive pair it applies
//    the bra transform (Eq. bra-from-hermite). The transforms run from step
//    programs the host planner emits for the class.
//
// GB300 executes FP64 at 2 FMA/clk/SM (measured: 1.20 TFLOP/s DFMA, 1.05
// TFLOP/s DMMA, 74.8 TFLOP/s FFMA), so the kernels spend integer and
// shared-memory bandwidth freely to save FP64 instructions.
#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace mdx {

// integers 0..63 as doubles, to multiply by small integers without an
// int->double conversion on the FP64 pipe
__constant__ double c_dint[64];
// the same small integers in global memory, for per-lane (divergent) reads through L1
__device__ double g_dint[64];
// sqrt(pi)/2 * (2m-1)!! / 2^m: F_m(T) = c_gh[m] T^(-m-1/2) for large T
__constant__ double c_gh[kBoysOrders];
// Cartesian components of shells l <= 7 in library order, packed x | y << 8 | z << 16
__constant__ uint32_t c_cart[8][36];
// real solid harmonics l <= 6 as Cartesian polynomials: c_sph[c_sph_off[l] + (m+l)*ncart(l) + k]
__constant__ double c_sph[840];
__constant__ int c_sph_off[kLmax + 2];
// the same, sparse: row m' = m + l of shell l has c_spn[l][m'] non-zero terms, Cartesian
// components c_spk[l][m'][j] with coefficients c_spv[l][m'][j]
constexpr int kSphNnzMax = 12;
__constant__ int c_spn[kLmax + 1][2 * kLmax + 1];
__constant__ uint8_t c_spk[kLmax + 1][2 * kLmax + 1][kSphNnzMax];
__constant__ double c_spv[kLmax + 1][2 * kLmax + 1][kSphNnzMax];
// c_top[l][k]: offset, in an X column of bra order L_b = l, of the top Hermite index (a_x, a_y, a_z) of
// Cartesian component k of shell l (X rows (u, v) = (a_y, a_z), t = a_x contiguous)
__constant__ uint16_t c_top[kLmax + 1][(kLmax + 1) * (kLmax + 2) / 2];

cudaError_t kernel_attributes_init();

// ----------------------------------------------------------------- pair records
__global__ void k_pair_records(BasisDev b0, BasisDev b1, const PrimPairJob* __restrict__ jobs, int64_t njobs,
                               double* __restrict__ recs, double* __restrict__ recs_signed, int* err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= njobs) return;
  const PrimPairJob jb = jobs[g];
  const BasisDev& B = jb.which ? b1 : b0;
  const int la = B.l[jb.i];
  const int lb = jb.j >= 0 ? B.l[jb.j] : 0;
  if (la < 0 || la > kLmax || lb < 0 || lb > kLmax) { atomicExch(err, kDevBadInput); return; }
  const double za = B.exps[B.prim_off[jb.i] + jb.ia];
  const double ca = B.coefs[B.prim_off[jb.i] + jb.ia];
  double zb = 0.0, cb = 1.0;
  double A[3], Bc[3];
  for (int k = 0; k < 3; ++k) A[k] = B.center[3 * jb.i + k];
  if (jb.j >= 0) {
    zb = B.exps[B.prim_off[jb.j] + jb.ib];
    cb = B.coefs[B.prim_off[jb.j] + jb.ib];
    for (int k = 0; k < 3; ++k) Bc[k] = B.center[3 * jb.j + k];
  } else {
    for (int k = 0; k < 3; ++k) Bc[k] = A[k];
  }
  const double p = za + zb;
  const double ip = 1.0 / p;
  const double inv2p = 0.5 * ip;
  double P[3], ab2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    P[k] = (za * A[k] + zb * Bc[k]) * ip;
    const double d = A[k] - Bc[k];
    ab2 += d * d;
  }
  double* r = recs + jb.off;
  double* rs = recs_signed + jb.off;
  const double pref = ca * cb * exp(-za * zb * ab2 * ip);
  const double hdr[kRecHeader] = {p, ip, P[0], P[1], P[2], pref, 0.0, 0.0};
  for (int k = 0; k < kRecHeader; ++k) { r[k] = hdr[k]; rs[k] = hdr[k]; }
  // per-axis tables, E_00^0 = 1 (the exponential is in the prefactor)
  int tab = 0;  // etab size
  for (int a = 0; a <= la; ++a)
    for (int b = 0; b <= lb; ++b) tab += a + b + 1;
  const int nt = la + lb + 1;
  for (int ax = 0; ax < 3; ++ax) {
    double* E = r + kRecHeader + ax * tab;
    double* Es = rs + kRecHeader + ax * tab;
    const double XPA = P[ax] - A[ax], XPB = P[ax] - Bc[ax];
    // block offsets: (a,b) at off(a,b); (a,b) block has a+b+1 entries
    // a-major order; off(a,0) = sum_{a'<a} sum_b (a'+b+1)
    auto off = [&](int a, int b) {
      int s = 0;
      for (int a2 = 0; a2 < a; ++a2) s += (lb + 1) * (a2 + 1) + lb * (lb + 1) / 2;
      s += b * (a + 1) + b * (b - 1) / 2;
      return s;
    };
    E[off(0, 0)] = 1.0;
    // raise a with b = 0 (Eq. E2rr1; E1rr when XPA = 0 and zb = 0)
    for (int a = 0; a < la; ++a) {
      const double* s = E + off(a, 0);
      double* d = E + off(a + 1, 0);
      for (int t = 0; t <= a + 1; ++t) {
        double v = 0.0;
        if (t >= 1) v = inv2p * s[t - 1];
        if (t <= a) v = fma(XPA, s[t], v);
        if (t + 1 <= a) v = fma(c_dint[t + 1], s[t + 1], v);
        d[t] = v;
      }
    }
    // raise b (Eq. E2rr2)
    for (int a = 0; a <= la; ++a)
      for (int b = 0; b < lb; ++b) {
        const double* s = E + off(a, b);
        double* d = E + off(a, b + 1);
        for (int t = 0; t <= a + b + 1; ++t) {
          double v = 0.0;
          if (t >= 1) v = inv2p * s[t - 1];
          if (t <= a + b) v = fma(XPB, s[t], v);
          if (t + 1 <= a + b) v = fma(c_dint[t + 1], s[t + 1], v);
          d[t] = v;
        }
      }
    for (int a = 0; a <= la; ++a)
      for (int b = 0; b <= lb; ++b) {
        const int o = off(a, b);
        for (int t = 0; t <= a + b; ++t) Es[o + t] = (t & 1) ? -E[o + t] : E[o + t];
      }
    (void)nt;
  }
}

cudaError_t launch_pair_records(const BasisDev& b0, const BasisDev& b1, const PrimPairJob* jobs, int64_t njobs,
                                double* recs, double* recs_signed, int* err, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  const int bs = 128;
  const int64_t grid = (njobs + bs - 1) / bs;
  k_pair_records<<<(unsigned)grid, bs, 0, s>>>(b0, b1, jobs, njobs, recs, recs_signed, err);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- quartets
// Barrier of one team. CTA = false (k_quartets with T <= 32): `mask` holds
// the lanes of this warp that take part. CTA = true: `mask` is 0 when the team
// is the whole block; all ones for teams that fill whole warps of T <= 32
// threads (warp barrier); else (barrier id << 16) | team threads for a named
// barrier of the team's own (several teams of whole warps in one block).
template <bool CTA>
__device__ __forceinline__ void team_sync(unsigned mask) {
  if (CTA) {
    if (mask == 0) __syncthreads();
    else if (mask == 0xffffffffu) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(mask >> 16), "r"(mask & 0xffffu) : "memory");
  } else {
    __syncwarp(mask);
  }
}

__device__ __forceinline__ int d_tet(int n) { return n < 0 ? 0 : n * (n + 1) * (n + 2) / 6; }
__device__ __forceinline__ int d_tri(int n) { return n < 0 ? 0 : n * (n + 1) / 2; }

__device__ __forceinline__ double ipow(double x, int m) {
  double r = 1.0;
  while (m) {
    if (m & 1) r *= x;
    x *= x;
    m >>= 1;
  }
  return r;
}

// Boys seeds [0]^(m) = (-2 rho)^m pref F_m(T), m = 0..L (Eq. 0m), then the
// Hermite integrals [tuv]^(0) (Eq. r), level by level, into ws[o_R0] with
// the [t][u][v] layout of total order L.
template <bool CTA>
__device__ void compute_R(const QuartetLaunch& a, double* ws, int tl, unsigned mask) {
  const PlanDev& P = a.plan;
  const int T = P.T;
  const int L = P.L;
  double* G = ws + P.o_G;
  const double* rb = ws + P.o_recb;
  const double* rk = ws + P.o_reck;
  // every lane needs P - Q for the R levels; the Boys lanes (m = tl, tl + T,
  // ... <= L) also derive rho, T and the prefactor (no barrier needed)
  const double PQx = rb[2] - rk[2], PQy = rb[3] - rk[3], PQz = rb[4] - rk[4];
  if (tl <= L) {
    const double zp = rb[0], izp = rb[1], zq = rk[0], izq = rk[1];
    const double s = zp + zq;
    const double rs = rsqrt(s);
    const double rho = zp * zq * rs * rs;
    const double Tb = rho * (PQx * PQx + PQy * PQy + PQz * PQz);
    // 2 pi^(5/2) / (zp zq sqrt(zp+zq)) * c_a c_b K_ab * c_c c_d K_cd
    const double pref = 34.986836655249725693 * izp * izq * rs * rb[5] * rk[5];
    const double m2r = -2.0 * rho;
    if (Tb < kBoysTmax) {
      const int i = __double2int_rn(Tb * kBoysInvH);
      const double nd = (double)i * (1.0 / kBoysInvH) - Tb;   // -d
      // (-2 rho)^m pref, stepped by (-2 rho)^T from lane to lane's next m
      double pw = pref * ipow(m2r, tl);
      const double step = T <= L ? ipow(m2r, T) : 1.0;
      const double* row = a.boys + (size_t)i * kBoysRow;
      for (int m = tl; m <= L; m += T) {
        const double2* c = reinterpret_cast<const double2*>(row + m * kBoysTerms);
        const double2 c01 = __ldg(c), c23 = __ldg(c + 1), c45 = __ldg(c + 2), c67 = __ldg(c + 3);
        double f = fma(c67.y, nd, c67.x);
        f = fma(f, nd, c45.y);
        f = fma(f, nd, c45.x);
        f = fma(f, nd, c23.y);
        f = fma(f, nd, c23.x);
        f = fma(f, nd, c01.y);
        f = fma(f, nd, c01.x);
        G[m] = pw * f;
        pw *= step;
      }
    } else {
      // F_m(T) = Gamma(m+1/2) / (2 T^(m+1/2)); neglected exp(-T) terms < 1e-17 relative for m <= 25
      const double t1 = rsqrt(Tb);
      const double x = m2r * t1 * t1;
      double pw = pref * t1 * ipow(x, tl);
      const double step = T <= L ? ipow(x, T) : 1.0;
      for (int m = tl; m <= L; m += T) {
        G[m] = c_gh[m] * pw;
        pw *= step;
      }
    }
  }
  team_sync<CTA>(mask);
  double* R0 = ws + P.o_R0;
  double* R1 = ws + P.o_R1;
  if (L == 0) {
    if (tl == 0) R0[0] = G[0];
    team_sync<CTA>(mask);
    return;
  }
  // level L holds only [000]^(L)
  if (tl == 0) ((L & 1) ? R1 : R0)[0] = G[L];
  team_sync<CTA>(mask);
  for (int n = L - 1; n >= 0; --n) {
    const int N = L - n;
    double* dst = (n & 1) ? R1 : R0;
    const double* src = (n & 1) ? R0 : R1;
    const uint32_t* prog = a.rprog + a.rprog_off[N];
    const int cnt = d_tet(N + 1);
    const double g = G[n];
    // one branch-free program word per entry (build_rlevel_programs): the two
    // sources in the previous level, the axis of X_PQ and the coefficient
    for (int e = tl; e < cnt; e += T) {
      const uint32_t w = __ldg(prog + e);
      const int ax = (w >> 24) & 3;
      const double pq = ax == 0 ? PQx : (ax == 1 ? PQy : PQz);
      double val = pq * src[w & 0xfff];
      val = fma(__ldg(g_dint + (w >> 26)), src[(w >> 12) & 0xfff], val);
      dst[e] = e == 0 ? g : val;
    }
    team_sync<CTA>(mask);
  }
}

// Two dot products side by side, operands loaded one term ahead of the FMAs
// that consume them (shared-memory latency overlaps the FP64 pipe).
__device__ __forceinline__ void dual_dot(const double* __restrict__ c0, const double* __restrict__ x0, int st0, int n0,
                                         const double* __restrict__ c1, const double* __restrict__ x1, int st1, int n1,
                                         double& v0, double& v1) {
  const int nm = min(n0, n1);
  if (nm > 0) {
    double a0 = c0[0], b0 = x0[0], a1 = c1[0], b1 = x1[0];
    for (int k = 1; k < nm; ++k) {
      const double na0 = c0[k * st0], nb0 = x0[k * st0], na1 = c1[k * st1], nb1 = x1[k * st1];
      v0 = fma(a0, b0, v0);
      v1 = fma(a1, b1, v1);
      a0 = na0; b0 = nb0; a1 = na1; b1 = nb1;
    }
    v0 = fma(a0, b0, v0);
    v1 = fma(a1, b1, v1);
  }
  for (int k = nm; k < n0; ++k) v0 = fma(c0[k * st0], x0[k * st0], v0);
  for (int k = nm; k < n1; ++k) v1 = fma(c1[k * st1], x1[k * st1], v1);
}

// out = (acc ? out : 0) + sum_k coef[c + k s] src[x + k s]
// Each lane runs two entries (e, e + T) side by side: two independent FMA
// chains hide the FP64 pipe latency. Entries are sorted by length, so the
// two usually have the same n. The next pair of entries is fetched while the
// current pair is computed.
__device__ __forceinline__ void run_step(const StepEntry* __restrict__ prog, int n, double* ws, int tl, int T,
                                         bool acc) {
  int e = tl;
  StepEntry p0{}, p1{};
  if (e + T < n) { p0 = prog[e]; p1 = prog[e + T]; }
  for (; e + T < n; e += 2 * T) {
    const StepEntry s0 = p0, s1 = p1;
    if (e + 3 * T < n) { p0 = prog[e + 2 * T]; p1 = prog[e + 3 * T]; }
    double v0 = acc ? ws[s0.out] : 0.0;
    double v1 = acc ? ws[s1.out] : 0.0;
    dual_dot(ws + s0.coef, ws + s0.src, s0.stride, s0.n, ws + s1.coef, ws + s1.src, s1.stride, s1.n, v0, v1);
    ws[s0.out] = v0;
    ws[s1.out] = v1;
  }
  if (e < n) {
    const StepEntry s = prog[e];
    const double* c = ws + s.coef;
    const double* x = ws + s.src;
    const int st = s.stride;
    double v = acc ? ws[s.out] : 0.0;
    for (int k = 0; k < s.n; ++k) v = fma(c[k * st], x[k * st], v);
    ws[s.out] = v;
  }
}

__device__ __forceinline__ void load_record(double* dst, const double* __restrict__ src, int n, int tl, int T) {
  for (int i = tl; i < n; i += T) dst[i] = __ldg(src + i);
}

__device__ __forceinline__ int d_ncart(int l) { return (l + 1) * (l + 2) / 2; }

// Exchange digestion of one column group: with V = (ij|kl) (a in i, b in j,
// c in k, d in l) and w the weight of the unique quartet,
//   K[i][k] += w sum_bd D[j][l] V,  K[i][l] += w sum_bc D[j][k] V,
//   K[j][k] += w sum_ad D[i][l] V,  K[j][l] += w sum_ac D[i][k] V.
// Together with K <- K + K^T afterwards this adds all eight index
// permutations of the quartet exactly once.
__device__ void digest_group(const QuartetLaunch& a, const double* ws, const Group& grp, int g, int2 qp, int tl,
                             int T) {
  const PlanDev& P = a.plan;
  const int2 bp = a.pair_shells[qp.x], kp = a.pair_shells[qp.y];
  const int si = bp.x, sj = bp.y, sk = kp.x, sl = kp.y;
  const double w = (si == sj ? 0.5 : 1.0) * (sk == sl ? 0.5 : 1.0) * (qp.x == qp.y ? 0.5 : 1.0);
  const int na = d_ncart(P.la), nb = d_ncart(P.lb), nd = d_ncart(P.ld);
  const int nc = d_ncart(P.lc);
  const int mol = a.pair_mol ? a.pair_mol[qp.x] : -1;
  const int64_t nao = mol >= 0 ? a.mol_nao[mol] : a.nao;
  const int64_t ai = a.ao_off[si], aj = a.ao_off[sj], ak = a.ao_off[sk], al = a.ao_off[sl];
  const int ncols = grp.ncols;
  const uint16_t* inv = P.colinv + (int64_t)g * P.Nk;   // this group's column of ket pair (c, d), or 0xffff
  const double* OUT = ws + P.o_OUT;
  const double* D = mol >= 0 ? a.mol_D[mol] : a.D;
  double* K = mol >= 0 ? a.mol_K[mol] : a.K;
  // u1: (a,c) over b,d ; u2: (a,d) over b,c ; u3: (b,c) over a,d ; u4: (b,d) over a,c
  const int n1 = na * nc, n2 = na * nd, n3 = nb * nc, n4 = nb * nd;
  for (int e = tl; e < n1 + n2 + n3 + n4; e += T) {
    int u, x, y;
    if (e < n1) { u = 0; x = e / nc; y = e - x * nc; }
    else if (e < n1 + n2) { u = 1; const int f = e - n1; x = f / nd; y = f - x * nd; }
    else if (e < n1 + n2 + n3) { u = 2; const int f = e - n1 - n2; x = f / nc; y = f - x * nc; }
    else { u = 3; const int f = e - n1 - n2 - n3; x = f / nd; y = f - x * nd; }
    double s = 0.0;
    bool any = false;
    if (u == 0 || u == 2) {
      // ket component c = y: the group's columns (y, d)
      for (int d = 0; d < nd; ++d) {
        const int col = inv[y * nd + d];
        if (col == 0xffff) continue;
        any = true;
        if (u == 0)        // K[i+x][k+y] += D[j+b][l+d] V[x,b,y,d]
          for (int b = 0; b < nb; ++b) s = fma(__ldg(D + (aj + b) * nao + al + d), OUT[(x * nb + b) * ncols + col], s);
        else               // K[j+x][k+y] += D[i+aa][l+d] V[aa,x,y,d]
          for (int aa = 0; aa < na; ++aa)
            s = fma(__ldg(D + (ai + aa) * nao + al + d), OUT[(aa * nb + x) * ncols + col], s);
      }
    } else {
      // ket component d = y: the group's columns (c, y)
      for (int c = 0; c < nc; ++c) {
        const int col = inv[c * nd + y];
        if (col == 0xffff) continue;
        any = true;
        if (u == 1)        // K[i+x][l+y] += D[j+b][k+c] V[x,b,c,y]
          for (int b = 0; b < nb; ++b) s = fma(__ldg(D + (aj + b) * nao + ak + c), OUT[(x * nb + b) * ncols + col], s);
        else               // K[j+x][l+y] += D[i+aa][k+c] V[aa,x,c,y]
          for (int aa = 0; aa < na; ++aa)
            s = fma(__ldg(D + (ai + aa) * nao + ak + c), OUT[(aa * nb + x) * ncols + col], s);
      }
    }
    if (!any) continue;
    int64_t row, colk;
    if (u == 0) { row = ai + x; colk = ak + y; }
    else if (u == 1) { row = ai + x; colk = al + y; }
    else if (u == 2) { row = aj + x; colk = ak + y; }
    else { row = aj + x; colk = al + y; }
    atomicAdd(K + row * nao + colk, w * s);
  }
}

__device__ __forceinline__ double dens_G(const double* __restrict__ D, int64_t nao, int64_t ri, int64_t rj,
                                         int64_t ck, int64_t cl) {
  // G = D_ik D_jl + D_il D_jk for AO rows ri (of i), rj (of j) and columns ck (of k), cl (of l)
  return __ldg(D + ri * nao + ck) * __ldg(D + rj * nao + cl) + __ldg(D + ri * nao + cl) * __ldg(D + rj * nao + ck);
}

// Exchange-energy gradient of one column group. S = sum_ijkl D_ik D_jl (ij|kl)
// restricted to the unique quartet is 4 w sum_abcd G_abcd (ab|cd) with
// G = D_ik (x) D_jl + D_il (x) D_jk; its derivative with respect to the centre
// of the shell at position gpos uses
//   d/dA_x phi_a = 2 zeta phi_{a+1_x} - a_x phi_{a-1_x},
// i.e. this launch's shifted class: every element of the l+1 shellset feeds
// each direction x whose component is >= 1 (weight +1), every element of the
// l-1 shellset each direction (weight -(a_x + 1)). Three of the four centres
// are differentiated; the fourth (position ginv) follows from translational
// invariance: what centre gpos gains, its atom loses. gpos = -1 accumulates
// the energy alpha S instead.
template <bool CTA>
__device__ void grad_group(const QuartetLaunch& a, const double* ws, const Group& grp, int2 qp, int tl, int T,
                           bool active, unsigned mask) {
  const PlanDev& P = a.plan;
  const int2 bp = a.pair_shells[qp.x], kp = a.pair_shells[qp.y];
  const int si = bp.x, sj = bp.y, sk = kp.x, sl = kp.y;
  const double w = (si == sj ? 0.5 : 1.0) * (sk == sl ? 0.5 : 1.0) * (qp.x == qp.y ? 0.5 : 1.0);
  const int nb_s = d_ncart(P.lb), nd_s = d_ncart(P.ld);
  const int64_t nao = a.nao;
  const int64_t ai = a.ao_off[si], aj = a.ao_off[sj], ak = a.ao_off[sk], al = a.ao_off[sl];
  const int ncols = grp.ncols;
  const uint16_t* cm = P.colmap + grp.col_off;
  const double* OUT = ws + P.o_OUT;
  const int pos = a.gpos, sg = a.gsign;
  const int lsh = pos == 0 ? P.la : (pos == 1 ? P.lb : (pos == 2 ? P.lc : P.ld));
  const int lorg = pos >= 0 ? a.lorig[pos] : 0;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const int tot = P.Nb * ncols;
  for (int e = tl; e < tot; e += T) {
    const int ab = e / ncols, col = e - ab * ncols;
    const double v = OUT[e];
    const int cd = cm[col];
    const int ia = ab / nb_s, ib = ab - ia * nb_s, ic = cd / nd_s, id = cd - ic * nd_s;
    if (pos < 0) {
      s0 = fma(v, dens_G(a.D, nao, ai + ia, aj + ib, ak + ic, al + id), s0);
      continue;
    }
    const int sidx = pos == 0 ? ia : (pos == 1 ? ib : (pos == 2 ? ic : id));
    const uint32_t xyz = c_cart[lsh][sidx];
    const int cmp[3] = {(int)(xyz & 0xff), (int)((xyz >> 8) & 0xff), (int)((xyz >> 16) & 0xff)};
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
      int o[3] = {cmp[0], cmp[1], cmp[2]};
      double wt;
      if (sg > 0) {
        if (o[dir] == 0) continue;
        o[dir] -= 1;
        wt = 1.0;
      } else {
        o[dir] += 1;
        wt = -(double)o[dir];
      }
      const int oidx = d_tri(lorg - o[0]) + o[2];
      const int ja = pos == 0 ? oidx : ia, jb = pos == 1 ? oidx : ib, jc = pos == 2 ? oidx : ic;
      const int jd = pos == 3 ? oidx : id;
      const double t = wt * v * dens_G(a.D, nao, ai + ja, aj + jb, ak + jc, al + jd);
      if (dir == 0) s0 += t; else if (dir == 1) s1 += t; else s2 += t;
    }
  }
  // reduce over the lanes of the team (whole warps for CTA teams, aligned lane groups otherwise)
  const int width = T < 32 ? T : 32;
  const unsigned lanes = CTA ? 0xffffffffu : mask;
  for (int off = width / 2; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(lanes, s0, off);
    s1 += __shfl_xor_sync(lanes, s1, off);
    s2 += __shfl_xor_sync(lanes, s2, off);
  }
  if (!active || (threadIdx.x & (width - 1)) != 0) return;
  const double f = a.alpha * 4.0 * w;
  if (pos < 0) {
    atomicAdd(a.energy, f * s0);
    return;
  }
  const int sh = pos == 0 ? si : (pos == 1 ? sj : (pos == 2 ? sk : sl));
  const int sv = a.ginv == 0 ? si : (a.ginv == 1 ? sj : (a.ginv == 2 ? sk : sl));
  double* gA = a.grad + 3 * (int64_t)a.atom[sh];
  double* gD = a.grad + 3 * (int64_t)a.atom[sv];
  atomicAdd(gA + 0, f * s0); atomicAdd(gA + 1, f * s1); atomicAdd(gA + 2, f * s2);
  atomicAdd(gD + 0, -f * s0); atomicAdd(gD + 1, -f * s1); atomicAdd(gD + 2, -f * s2);
}

// Exchange-gradient contraction of shellsets already written to memory (the
// register-kernel path of mdx_exchange_grad): the same sums as grad_group,
// one warp per quartet, V = the launch's (shifted) shellset of quartet q at
// V + q N_b N_k.
__global__ void k_grad_contract(const QuartetLaunch a, const double* __restrict__ V) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= a.nq) return;
  const PlanDev& P = a.plan;
  const int2 qp = a.qpairs[q];
  const int2 bp = a.pair_shells[qp.x], kp = a.pair_shells[qp.y];
  const int si = bp.x, sj = bp.y, sk = kp.x, sl = kp.y;
  const double w = (si == sj ? 0.5 : 1.0) * (sk == sl ? 0.5 : 1.0) * (qp.x == qp.y ? 0.5 : 1.0);
  const int nb_s = d_ncart(P.lb), nd_s = d_ncart(P.ld);
  const int64_t nao = a.nao;
  const int64_t ai = a.ao_off[si], aj = a.ao_off[sj], ak = a.ao_off[sk], al = a.ao_off[sl];
  const int pos = a.gpos, sg = a.gsign;
  const int lsh = pos == 0 ? P.la : (pos == 1 ? P.lb : (pos == 2 ? P.lc : P.ld));
  const int lorg = pos >= 0 ? a.lorig[pos] : 0;
  const int Nk = P.Nk, tot = P.Nb * P.Nk;
  const double* v0 = V + q * (int64_t)tot;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int e = lane; e < tot; e += 32) {
    const int ab = e / Nk, cd = e - ab * Nk;
    const double v = __ldg(v0 + e);
    const int ia = ab / nb_s, ib = ab - ia * nb_s, ic = cd / nd_s, id = cd - ic * nd_s;
    if (pos < 0) {
      s0 = fma(v, dens_G(a.D, nao, ai + ia, aj + ib, ak + ic, al + id), s0);
      continue;
    }
    const int sidx = pos == 0 ? ia : (pos == 1 ? ib : (pos == 2 ? ic : id));
    const uint32_t xyz = c_cart[lsh][sidx];
    const int cmp[3] = {(int)(xyz & 0xff), (int)((xyz >> 8) & 0xff), (int)((xyz >> 16) & 0xff)};
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
      int o[3] = {cmp[0], cmp[1], cmp[2]};
      double wt;
      if (sg > 0) {
        if (o[dir] == 0) continue;
        o[dir] -= 1;
        wt = 1.0;
      } else {
        o[dir] += 1;
        wt = -(double)o[dir];
      }
      const int oidx = d_tri(lorg - o[0]) + o[2];
      const int ja = pos == 0 ? oidx : ia, jb = pos == 1 ? oidx : ib, jc = pos == 2 ? oidx : ic;
      const int jd = pos == 3 ? oidx : id;
      const double t = wt * v * dens_G(a.D, nao, ai + ja, aj + jb, ak + jc, al + jd);
      if (dir == 0) s0 += t; else if (dir == 1) s1 += t; else s2 += t;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if (lane != 0) return;
  const double f = a.alpha * 4.0 * w;
  if (pos < 0) {
    atomicAdd(a.energy, f * s0);
    return;
  }
  const int sh = pos == 0 ? si : (pos == 1 ? sj : (pos == 2 ? sk : sl));
  const int sv = a.ginv == 0 ? si : (a.ginv == 1 ? sj : (a.ginv == 2 ? sk : sl));
  double* gA = a.grad + 3 * (int64_t)a.atom[sh];
  double* gD = a.grad + 3 * (int64_t)a.atom[sv];
  atomicAdd(gA + 0, f * s0); atomicAdd(gA + 1, f * s1); atomicAdd(gA + 2, f * s2);
  atomicAdd(gD + 0, -f * s0); atomicAdd(gD + 1, -f * s1); atomicAdd(gD + 2, -f * s2);
}

cudaError_t launch_grad_contract(const QuartetLaunch& a, const double* V, cudaStream_t s) {
  if (a.nq <= 0) return cudaSuccess;
  const int64_t threads = a.nq * 32;
  const int bs = 256;
  const int64_t grid = (threads + bs - 1) / bs;
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  k_grad_contract<<<(unsigned)grid, bs, 0, s>>>(a, V);
  return cudaGetLastError();
}

// b1: C1 = Ex (x) X for `ncols` columns (X column stride hb at o_X, C1 column
// stride c1stride at o_C1); two entries per lane (see run_step).
__device__ __forceinline__ void bra_b1(const PlanDev& P, double* ws, int o_X, int o_C1, int c1stride, int ncols, int tl,
                                       int T) {
  const int tot = P.nb1 * ncols;
  for (int e = tl; e < tot; e += 2 * T) {
    const int e1 = e + T < tot ? e + T : e;
    const int ent0 = e / ncols, col0 = e - ent0 * ncols;
    const int ent1 = e1 / ncols, col1 = e1 - ent1 * ncols;
    const StepEntry s0 = P.b1[ent0], s1 = P.b1[ent1];
    const double* c0 = ws + s0.coef;
    const double* x0 = ws + o_X + col0 * P.hb + s0.src;
    const double* c1 = ws + s1.coef;
    const double* x1 = ws + o_X + col1 * P.hb + s1.src;
    double v0 = 0.0, v1 = 0.0;
    dual_dot(c0, x0, s0.stride, s0.n, c1, x1, s1.stride, s1.n, v0, v1);
    ws[o_C1 + col0 * c1stride + s0.out] = v0;
    if (e1 != e) ws[o_C1 + col1 * c1stride + s1.out] = v1;
  }
}

// b23: OUT[ab][col] (+)= Ez (x) Ey (x) C1 for `ncols` columns; two Hermite
// z-indices v in flight per lane (independent inner sums over u). to_global:
// the finished value goes to outq[ab * out_stride + cm[col]] instead of OUT.
__device__ __forceinline__ void bra_b23(const PlanDev& P, double* ws, int o_C1, int c1stride, int o_OUT, int ncols,
                                        bool accumulate, bool to_global, double* outq, const uint16_t* cm,
                                        int out_stride, bool active, int tl, int T) {
  const int tot = P.nb23 * ncols;
  for (int e = tl; e < tot; e += T) {
    const int ent = e / ncols, col = e - ent * ncols;
    const B23Entry s = P.b23[ent];
    const double* c1 = ws + o_C1 + col * c1stride + s.src + s.u0;
    double* o = ws + o_OUT + s.out * ncols + col;
    double acc = accumulate ? *o : 0.0;
    const int r1 = s.r + 1;
    const double* ey = ws + s.ey;
    const double* ez = ws + s.ez;
    const int su = s.su, sv = s.sv, nu = s.nu;
    int iv = 0;
    for (; iv + 1 < s.nv; iv += 2) {
      const int va = s.v0 + iv * sv, vb = va + sv;
      const double* ra = c1 + va * r1 - (va * (va - 1)) / 2;
      const double* rb = c1 + vb * r1 - (vb * (vb - 1)) / 2;
      double ia = 0.0, ib = 0.0;
      double y = ey[0], xa = ra[0], xb = rb[0];
      for (int iu = 1; iu < nu; ++iu) {
        const double ny = ey[iu * su], nxa = ra[iu * su], nxb = rb[iu * su];
        ia = fma(y, xa, ia);
        ib = fma(y, xb, ib);
        y = ny; xa = nxa; xb = nxb;
      }
      ia = fma(y, xa, ia);
      ib = fma(y, xb, ib);
      acc = fma(ez[iv * sv], ia, acc);
      acc = fma(ez[(iv + 1) * sv], ib, acc);
    }
    if (iv < s.nv) {
      const int va = s.v0 + iv * sv;
      const double* ra = c1 + va * r1 - (va * (va - 1)) / 2;
      double ia = 0.0;
      for (int iu = 0; iu < nu; ++iu) ia = fma(ey[iu * su], ra[iu * su], ia);
      acc = fma(ez[iv * sv], ia, acc);
    }
    if (to_global) {
      if (active) outq[(int64_t)s.out * out_stride + cm[col]] = acc;
    } else {
      *o = acc;
    }
  }
}

// R of primitive quartet i from the cache into R0, where the k1 programs read it.
__device__ __forceinline__ void load_cached_R(const PlanDev& P, double* ws, int i, int tl) {
  const int nR = d_tet(P.L + 1);
  const double* src = ws + P.o_Rc + (int64_t)i * P.rstride;
  for (int e = tl; e < nR; e += P.T) ws[P.o_R0 + e] = src[e];
}

// The R tables of the primitive quartets of bra primitives pb0 <= pb < pb1 of
// q, computed once and kept in the workspace region o_Rc, table
// (pb - pb0) Kk + pk (plans with cache_R == 2: every primitive quartet, filled
// once per quartet; cache_R == 3, solid-harmonic plans: those of one bra
// primitive, filled per bra primitive). Contracted classes of several column
// groups would otherwise compute each R once per group.
template <bool CTA>
__device__ __forceinline__ void fill_R_cache(const QuartetLaunch& a, double* ws, int64_t bra0, int64_t ket0, int pb0,
                                             int pb1, int tl, unsigned mask) {
  const PlanDev& P = a.plan;
  const int nR = d_tet(P.L + 1);
  for (int pb = pb0; pb < pb1; ++pb)
    for (int pk = 0; pk < P.Kk; ++pk) {
      load_record(ws + P.o_recb, a.recs + bra0 + (int64_t)pb * P.recb, P.recb, tl, P.T);
      load_record(ws + P.o_reck, a.recs_signed + ket0 + (int64_t)pk * P.reck, P.reck, tl, P.T);
      team_sync<CTA>(mask);   // also orders the previous table's copy before compute_R rewrites R0
      compute_R<CTA>(a, ws, tl, mask);
      double* dst = ws + P.o_Rc + (int64_t)((pb - pb0) * P.Kk + pk) * P.rstride;
      for (int e = tl; e < nR; e += P.T) dst[e] = ws[P.o_R0 + e];
    }
  team_sync<CTA>(mask);
}

// The work of one team on one shell quartet q (all groups, all primitives,
// store / digestion / gradient epilogue). Inactive teams run the same control
// flow on a shadow quartet (so that barriers match) and write nothing global.
template <bool CTA>
__device__ __forceinline__ void quartet_body(const QuartetLaunch& a, double* ws, int64_t q, bool active, int tl,
                                             unsigned mask) {
  const PlanDev& P = a.plan;
  const int T = P.T;
  const int2 qp = a.qpairs[q];
  const int64_t bra0 = a.pair_rec[qp.x + a.bra_var_off];
  const int64_t ket0 = a.pair_rec[qp.y + a.ket_var_off];
  const int Kb = P.Kb, Kk = P.Kk;
  if (P.cache_R == 1) {
    load_record(ws + P.o_recb, a.recs + bra0, P.recb, tl, T);
    load_record(ws + P.o_reck, a.recs_signed + ket0, P.reck, tl, T);
    team_sync<CTA>(mask);
    compute_R<CTA>(a, ws, tl, mask);
  } else if (P.cache_R == 2) {
    fill_R_cache<CTA>(a, ws, bra0, ket0, 0, Kb, tl, mask);
  }
  // qout == nullptr: shellsets back to back, N_b N_k doubles each
  double* outq = a.D ? nullptr : a.out + (a.qout ? a.qout[q] : q * (int64_t)P.Nb * P.Nk);
  // store epilogue: b23 of the last bra primitive writes the shellset to global
  // memory itself (no OUT pass, no barrier after it)
  const bool direct = !a.D && !a.grad;
  for (int g = 0; g < P.ngroups; ++g) {
    const Group grp = P.groups[g];
    const int ncols = grp.ncols;
    for (int pb = 0; pb < Kb; ++pb) {
      if (P.cache_R != 1) load_record(ws + P.o_recb, a.recs + bra0 + (int64_t)pb * P.recb, P.recb, tl, T);
      for (int pk = 0; pk < Kk; ++pk) {
        if (P.cache_R != 1) {
          load_record(ws + P.o_reck, a.recs_signed + ket0 + (int64_t)pk * P.reck, P.reck, tl, T);
          if (P.cache_R == 2) load_cached_R(P, ws, pb * Kk + pk, tl);
          team_sync<CTA>(mask);
          if (P.cache_R == 0) compute_R<CTA>(a, ws, tl, mask);
        }
        if (grp.k1_n > 0) {   // groups after the first of a z-pair reuse its A (uncontracted classes)
          run_step(P.kprog + grp.k1_off, grp.k1_n, ws, tl, T, false);
          team_sync<CTA>(mask);
        }
        run_step(P.kprog + grp.k2_off, grp.k2_n, ws, tl, T, false);
        team_sync<CTA>(mask);
        run_step(P.kprog + grp.k3_off, grp.k3_n, ws, tl, T, pk > 0);
        team_sync<CTA>(mask);
      }
      bra_b1(P, ws, P.o_X, P.o_C1, P.c1size, ncols, tl, T);
      team_sync<CTA>(mask);
      bra_b23(P, ws, P.o_C1, P.c1size, P.o_OUT, ncols, pb > 0, direct && pb == Kb - 1, outq,
              P.colmap + grp.col_off, P.Nk, active, tl, T);
      // Barrier before the next writer of what b23 reads: the bra record (reloaded
      // per bra primitive unless the class has one primitive quartet) or OUT (read
      // by other lanes in the digestion / gradient epilogue). C1 is overwritten by
      // the next b1 only after the k-step barriers.
      if (P.cache_R != 1 || (!direct && pb == Kb - 1)) team_sync<CTA>(mask);
    }
    if (a.grad) {
      grad_group<CTA>(a, ws, grp, qp, tl, T, active, mask);
      team_sync<CTA>(mask);
    } else if (a.D) {
      // exchange digestion of this group's columns (Sec. 6: K_bc = sum_ad [ab|cd] D_ad),
      // unique quartet (ij|kl) with i>=j, k>=l, ij>=kl and weight w; the host adds K^T at the end
      if (active) digest_group(a, ws, grp, g, qp, tl, T);
      team_sync<CTA>(mask);
    }
  }
  // the records of the next quartet (persistent kernel) overwrite what b23 reads
  if (direct) team_sync<CTA>(mask);
}

template <bool CTA>
__global__ void __launch_bounds__(CTA ? 1024 : 128) k_quartets(const QuartetLaunch a) {
  extern __shared__ __align__(16) double smem[];
  const PlanDev& P = a.plan;
  const int T = P.T;
  const int team = threadIdx.x / T;
  const int tl = threadIdx.x - team * T;
  double* ws = smem + (size_t)team * P.team_doubles;
  // lanes of this warp that exist (a partial last warp when the CTA is not a multiple of 32);
  // a CTA team is the whole block
  unsigned mask = CTA ? 0u : 0xffffffffu;
  if (!CTA) {
    const int wbase = threadIdx.x & ~31;
    const int live = blockDim.x - wbase;
    if (live < 32) mask = (1u << live) - 1u;
  }
  int64_t q = (int64_t)blockIdx.x * P.teams_per_cta + team;
  const bool active = q < a.nq;
  if (!active) q = a.nq - 1;   // idle teams shadow the last quartet and store nothing
  quartet_body<CTA>(a, ws, q, active, tl, mask);
}

// One quartet over real solid harmonics (Eqs. solid2herm-1/2: the
// Cartesian-to-solid coefficients are contracted into the transforms, so the
// bra steps and everything after them run on 2l+1 components per shell). For
// every bra primitive pair:
//   1. the ket groups build the Cartesian columns [p|cd] as in the Cartesian
//      kernel and stage them in the team's global area Xg[cd][p];
//   2. ket pass d -> d':  Yg[c][d'][p] = sum_d C^{ld}_{d'd} Xg[c][d][p];
//   3. per group of spherical columns c'd':
//        ket pass c -> c': Xs[c'd'][p] = sum_c C^{lc}_{c'c} Yg[c][d'][p]   (shared memory)
//        bra steps b1/b23 on those columns: OUT[ab][c'd']                  (Eq. bra-from-hermite)
//        bra pass b -> b': T[a][b'][c'd'] = sum_b C^{lb}_{b'b} OUT[ab][c'd']
//        bra pass a -> a': out[a'b'][c'd'] (+)= sum_a C^{la}_{a'a} T[a][b'][c'd']
// Each pass is a sparse product (the solid harmonics of l have few Cartesian
// terms per row); applied one index at a time it costs far less than the
// Cartesian bra steps it removes.
template <bool CTA>
__device__ void quartet_sph(const QuartetLaunch& a, double* ws, double* xg, int64_t q, bool active, int tl,
                            unsigned mask) {
  const PlanDev& P = a.plan;
  const int T = P.T;
  const int2 qp = a.qpairs[q];
  const int64_t bra0 = a.pair_rec[qp.x + a.bra_var_off];
  const int64_t ket0 = a.pair_rec[qp.y + a.ket_var_off];
  const int Kb = P.Kb, Kk = P.Kk;
  const int hbp = P.hbp;
  const int la = P.la, lb = P.lb, lc = P.lc, ld = P.ld;
  const int nb = d_ncart(lb), nd = d_ncart(ld), nc = d_ncart(lc);
  const int nsb = P.nsb, nsd = P.nsd;
  const int nks = P.nsc * nsd;
  double* yg = xg + (int64_t)P.Nk * hbp;
  double* outq = a.out + a.qout[q];
  if (P.cache_R == 1) {
    load_record(ws + P.o_recb, a.recs + bra0, P.recb, tl, T);
    load_record(ws + P.o_reck, a.recs_signed + ket0, P.reck, tl, T);
    team_sync<CTA>(mask);
    compute_R<CTA>(a, ws, tl, mask);
  } else if (P.cache_R == 2) {
    fill_R_cache<CTA>(a, ws, bra0, ket0, 0, Kb, tl, mask);
  }
  for (int pb = 0; pb < Kb; ++pb) {
    if (P.cache_R == 3) fill_R_cache<CTA>(a, ws, bra0, ket0, pb, pb + 1, tl, mask);
    if (P.cache_R != 1) load_record(ws + P.o_recb, a.recs + bra0 + (int64_t)pb * P.recb, P.recb, tl, T);
    // 1. Cartesian ket columns, group by group, staged in Xg
    for (int g = 0; g < P.ngroups; ++g) {
      const Group grp = P.groups[g];
      for (int pk = 0; pk < Kk; ++pk) {
        if (P.cache_R != 1) {
          load_record(ws + P.o_reck, a.recs_signed + ket0 + (int64_t)pk * P.reck, P.reck, tl, T);
          if (P.cache_R >= 2) load_cached_R(P, ws, P.cache_R == 2 ? pb * Kk + pk : pk, tl);
          team_sync<CTA>(mask);
          if (P.cache_R == 0) compute_R<CTA>(a, ws, tl, mask);
        }
        if (grp.k1_n > 0) {
          run_step(P.kprog + grp.k1_off, grp.k1_n, ws, tl, T, false);
          team_sync<CTA>(mask);
        }
        run_step(P.kprog + grp.k2_off, grp.k2_n, ws, tl, T, false);
        team_sync<CTA>(mask);
        run_step(P.kprog + grp.k3_off, grp.k3_n, ws, tl, T, pk > 0);
        team_sync<CTA>(mask);
      }
      const uint16_t* cm = P.colmap + grp.col_off;
      const int tot = grp.ncols * hbp;
      for (int e = tl; e < tot; e += T) {
        const int col = e / hbp, i = e - col * hbp;
        xg[(int64_t)cm[col] * hbp + i] = ws[P.o_X + col * P.hb + i];
      }
      team_sync<CTA>(mask);   // the next group's k3 rewrites X; every lane reads Xg below
    }
    // 2. ket pass d -> d'
    {
      const int tot = nc * nsd * hbp;
      for (int e = tl; e < tot; e += T) {
        const int cdp = e / hbp, i = e - cdp * hbp;
        const int c = cdp / nsd, dp = cdp - c * nsd;
        const int n = c_spn[ld][dp];
        double v = 0.0;
        for (int j = 0; j < n; ++j) v = fma(c_spv[ld][dp][j], xg[((int64_t)c * nd + c_spk[ld][dp][j]) * hbp + i], v);
        yg[(int64_t)cdp * hbp + i] = v;
      }
      team_sync<CTA>(mask);
    }
    // 3. groups of spherical ket columns
    for (int c0 = 0; c0 < nks; c0 += P.ncols_s) {
      const int ncols = min(P.ncols_s, nks - c0);
      // ket pass c -> c' into shared memory (the X layout the bra steps read)
      for (int e = tl; e < ncols * hbp; e += T) {
        const int col = e / hbp, i = e - col * hbp;
        const int gcol = c0 + col, cp = gcol / nsd, dp = gcol - cp * nsd;
        const int n = c_spn[lc][cp];
        double v = 0.0;
        for (int j = 0; j < n; ++j) v = fma(c_spv[lc][cp][j], yg[((int64_t)c_spk[lc][cp][j] * nsd + dp) * hbp + i], v);
        ws[P.o_Xs + col * P.hb + i] = v;
      }
      team_sync<CTA>(mask);
      if (P.top_only) {
        // one-centre bra over solid harmonics: OUT[m][col] = (2 zeta)^-la sum_a C_ma X[top(a)][col]
        const double zeta = ws[P.o_recb];
        double f = 1.0;
        for (int k = 0; k < la; ++k) f *= 0.5 / zeta;
        for (int e = tl; e < P.nsa * ncols; e += T) {
          const int m = e / ncols, col = e - m * ncols;
          const int n = c_spn[la][m];
          const double* x = ws + P.o_Xs + col * P.hb;
          double v = 0.0;
          for (int j = 0; j < n; ++j) v = fma(c_spv[la][m][j], x[c_top[la][c_spk[la][m][j]]], v);
          if (active) {
            double* o = outq + (int64_t)m * nks + c0 + col;
            *o = pb > 0 ? *o + f * v : f * v;
          }
        }
        team_sync<CTA>(mask);
        continue;
      }
      bra_b1(P, ws, P.o_Xs, P.o_C1s, P.c1s, ncols, tl, T);
      team_sync<CTA>(mask);
      bra_b23(P, ws, P.o_C1s, P.c1s, P.o_OUTs, ncols, false, false, nullptr, nullptr, 0, active, tl, T);
      team_sync<CTA>(mask);
      // bra pass b -> b' into the C1 slots: T[col][a][b']
      {
        const int na = d_ncart(la);
        for (int e = tl; e < na * nsb * ncols; e += T) {
          const int ab = e / ncols, col = e - ab * ncols;
          const int aa = ab / nsb, bp = ab - aa * nsb;
          const int n = c_spn[lb][bp];
          double v = 0.0;
          for (int j = 0; j < n; ++j)
            v = fma(c_spv[lb][bp][j], ws[P.o_OUTs + (aa * nb + c_spk[lb][bp][j]) * ncols + col], v);
          ws[P.o_C1s + col * P.c1s + ab] = v;
        }
      }
      team_sync<CTA>(mask);
      // bra pass a -> a' into the output (summed over the bra primitive pairs)
      for (int e = tl; e < P.nsa * nsb * ncols; e += T) {
        const int ab = e / ncols, col = e - ab * ncols;
        const int ap = ab / nsb, bp = ab - ap * nsb;
        const int n = c_spn[la][ap];
        double v = 0.0;
        for (int j = 0; j < n; ++j) v = fma(c_spv[la][ap][j], ws[P.o_C1s + col * P.c1s + c_spk[la][ap][j] * nsb + bp], v);
        if (active) {
          double* o = outq + (int64_t)ab * nks + c0 + col;
          *o = pb > 0 ? *o + v : v;
        }
      }
      team_sync<CTA>(mask);
    }
  }
}

// Solid-harmonic launches: as many CTAs as can be resident (`grid`, chosen
// by the host), each looping over quartets; team `slot` owns global staging
// area slot * xg_doubles of a.sph_scratch.
template <bool CTA>
__global__ void __launch_bounds__(CTA ? 1024 : 128) k_quartets_sph(const QuartetLaunch a) {
  extern __shared__ __align__(16) double smem[];
  const PlanDev& P = a.plan;
  const int T = P.T;
  const int team = threadIdx.x / T;
  const int tl = threadIdx.x - team * T;
  double* ws = smem + (size_t)team * P.team_doubles;
  unsigned mask = CTA ? 0u : 0xffffffffu;
  if (!CTA) {
    const int wbase = threadIdx.x & ~31;
    const int live = blockDim.x - wbase;
    if (live < 32) mask = (1u << live) - 1u;
  }
  const int64_t slot = (int64_t)blockIdx.x * P.teams_per_cta + team;
  double* xg = a.sph_scratch + slot * P.xg_doubles;
  const int64_t stride = (int64_t)gridDim.x * P.teams_per_cta;
  const int64_t rounds = (a.nq + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    int64_t q = r * stride + slot;
    const bool active = q < a.nq;
    if (!active) q = a.nq - 1;   // idle teams shadow the last quartet and store nothing
    quartet_sph<CTA>(a, ws, xg, q, active, tl, mask);
  }
}

cudaError_t sph_grid(const PlanDev& P, int64_t nq, int* grid) {
  const int block = P.teams_per_cta * P.T;
  const size_t shm = (size_t)P.teams_per_cta * P.team_doubles * sizeof(double);
  int bps = 0, dev = 0, sms = 0;
  cudaError_t e = P.T > 32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_quartets_sph<true>, block, shm)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_quartets_sph<false>, block, shm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t need = (nq + P.teams_per_cta - 1) / P.teams_per_cta;
  *grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(1, bps) * sms));
  return cudaSuccess;
}

cudaError_t launch_quartets_sph(const QuartetLaunch& a, int grid, cudaStream_t s) {
  if (a.nq <= 0) return cudaSuccess;
  const PlanDev& P = a.plan;
  if (!P.sph || !a.sph_scratch || !a.qout || grid < 1) return cudaErrorInvalidValue;
  const int block = P.teams_per_cta * P.T;
  const size_t shm = (size_t)P.teams_per_cta * P.team_doubles * sizeof(double);
  if (P.T > 32) k_quartets_sph<true><<<grid, block, shm, s>>>(a);
  else k_quartets_sph<false><<<grid, block, shm, s>>>(a);
  return cudaGetLastError();
}

// Persistent kernel over a queue of work items from many launches (classes,
// molecules): each CTA takes the next item with one atomicAdd (no waiting on
// other CTAs), adopts that item's plan and runs its quartets in teams_per_cta
// teams of T threads (the class's own team size; threads past the last team
// wait for the next item). Warp teams synchronise per warp, teams of whole
// warps on a named barrier of their own, so teams never wait for each other.
__global__ void __launch_bounds__(kPersistBlock) k_persistent(const PersistLaunch pl) {
  extern __shared__ __align__(16) double smem[];
  __shared__ long long s_item;
  __shared__ __align__(16) QuartetLaunch s_launch;   // the item's descriptor, read in every inner loop
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(pl.counter, 1ull);
    __syncthreads();
    const long long it = s_item;
    if (it >= pl.nitems) return;
    const WorkItem w = pl.items[it];
    if (w.launch != cur) {   // uniform across the block
      const int nw = (int)(sizeof(QuartetLaunch) / sizeof(int));
      const int* src = reinterpret_cast<const int*>(pl.launches + w.launch);
      int* dst = reinterpret_cast<int*>(&s_launch);
      for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
      cur = w.launch;
    }
    __syncthreads();
    const QuartetLaunch& a = s_launch;
    const int T = a.plan.T;
    const int tpb = a.plan.teams_per_cta;   // T x tpb <= blockDim.x, whole warps (host-checked)
    const int team = threadIdx.x / T;
    if (team >= tpb) continue;   // idle warps: straight to the next item's barrier
    const int tl = threadIdx.x - team * T;
    double* ws = smem + (size_t)team * a.plan.team_doubles;
    // barriers 1..tpb of T threads each for teams of whole warps; a warp barrier for
    // warps of teams of T <= 32 (one body for both, so that one set of registers serves)
    const unsigned mask = T > 32 ? ((unsigned)(team + 1) << 16) | (unsigned)T : 0xffffffffu;
    for (int64_t sub = 0; sub < w.count; sub += tpb) {   // an item holds a few rounds of teams
      const bool active = team < w.count - sub;
      const int64_t q = w.begin + sub + (active ? team : 0);
      quartet_body<true>(a, ws, q, active, tl, mask);
    }
  }
}

const void* persistent_kernel_ptr() { return (const void*)k_persistent; }

cudaError_t launch_persistent(const PersistLaunch& pl, int64_t smem_bytes, int grid, cudaStream_t s) {
  if (pl.nitems <= 0) return cudaSuccess;
  k_persistent<<<grid, kPersistBlock, (size_t)smem_bytes, s>>>(pl);
  return cudaGetLastError();
}

cudaError_t launch_reg_part00(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part01(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part02(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part03(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part04(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part05(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part06(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part07(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part08(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part09(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part10(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part11(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part12(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part13(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
cudaError_t launch_reg_part14(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled);
using RegPart = cudaError_t (*)(int, const QuartetLaunch&, cudaStream_t, bool*);
static const RegPart kRegParts[] = {launch_reg_part00, launch_reg_part01, launch_reg_part02, launch_reg_part03,
                                    launch_reg_part04, launch_reg_part05, launch_reg_part06, launch_reg_part07,
                                    launch_reg_part08, launch_reg_part09, launch_reg_part10, launch_reg_part11,
                                    launch_reg_part12, launch_reg_part13, launch_reg_part14};

cudaError_t launch_quartets(const QuartetLaunch& a, cudaStream_t s) {
  if (a.nq <= 0) return cudaSuccess;
  const PlanDev& P = a.plan;
  if (!P.has_out && (a.D || a.grad)) return cudaErrorInvalidValue;   // store-only plan in an epilogue launch
  if (P.reg && !a.grad) {
    // one thread per quartet, registers only (store and digestion epilogues)
    const int code = ((P.la * 7 + P.lb) * 7 + P.lc) * 7 + P.ld;
    for (RegPart part : kRegParts) {
      bool handled = false;
      const cudaError_t e = part(code, a, s, &handled);
      if (handled || e != cudaSuccess) return e;
    }
  }
  const int64_t grid = (a.nq + P.teams_per_cta - 1) / P.teams_per_cta;
  const int block = P.teams_per_cta * P.T;
  const size_t shm = (size_t)P.teams_per_cta * P.team_doubles * sizeof(double);
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  if (P.T > 32) k_quartets<true><<<(unsigned)grid, block, shm, s>>>(a);
  else k_quartets<false><<<(unsigned)grid, block, shm, s>>>(a);
  return cudaGetLastError();
}

// Screened-out shellsets: one block per range (grid-strided), threads over its doubles.
__global__ void k_zero_ranges(const int64_t* __restrict__ ranges, int64_t n, double* __restrict__ out) {
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
    const int64_t off = ranges[2 * r], len = ranges[2 * r + 1];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) out[off + i] = 0.0;
  }
}

cudaError_t launch_zero_ranges(const int64_t* ranges, int64_t n, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(n, 65536);
  k_zero_ranges<<<grid, 256, 0, s>>>(ranges, n, out);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- exchange support
__global__ void k_dmax(const double* __restrict__ D, int32_t nao, const int32_t* __restrict__ ao_off,
                       const int32_t* __restrict__ l, int32_t n, double* __restrict__ dmax, int64_t ld) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)n * n) return;
  const int x = (int)(g / n), y = (int)(g - (int64_t)x * n);
  const int64_t r0 = ao_off[x], c0 = ao_off[y];
  const int nr = d_ncart(l[x]), nc = d_ncart(l[y]);
  double m = 0.0;
  for (int r = 0; r < nr; ++r)
    for (int c = 0; c < nc; ++c) m = fmax(m, fabs(D[(r0 + r) * nao + c0 + c]));
  dmax[(int64_t)x * ld + y] = m;
}

cudaError_t launch_dmax(const double* D, int32_t nao, const int32_t* ao_off, const int32_t* l, int32_t n_shells,
                        double* dmax, int64_t ld, cudaStream_t s) {
  const int64_t tot = (int64_t)n_shells * n_shells;
  if (tot <= 0) return cudaSuccess;
  k_dmax<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(D, nao, ao_off, l, n_shells, dmax, ld);
  return cudaGetLastError();
}

__global__ void k_rowmax(const double* __restrict__ dmax, int32_t n, double* __restrict__ rowmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* r = dmax + (int64_t)i * n;
  double m = 0.0;
  for (int k = 0; k < n; ++k) m = fmax(m, r[k]);
  rowmax[i] = m;
}

cudaError_t launch_rowmax(const double* dmax, int32_t n, double* rowmax, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_rowmax<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(dmax, n, rowmax);
  return cudaGetLastError();
}

// One block per bra pair p (see ScreenArgs). Counting pass: per-bucket totals;
// fill pass: (p, q) written into its bucket. One atomic per warp and step:
// the kept lanes of a warp take consecutive slots.
__global__ void __launch_bounds__(256) k_screen(const ScreenArgs a, bool fill) {
  const int64_t p = blockIdx.x;
  if (p >= a.npairs) return;
  const int2 ij = a.pair_shells[p];
  const double qp = a.Q[p];
  const int cp = a.pair_class[p];
  const int m = a.pair_mol ? a.pair_mol[p] : 0;
  const int f = a.shell_first[m], nm = a.shell_first[m + 1] - f;
  const double* dm = a.dmax + a.dmax_off[m];
  const double* di = dm + (int64_t)(ij.x - f) * nm;
  const double* dj = dm + (int64_t)(ij.y - f) * nm;
  const double dr = fmax(a.rowmax[ij.x], a.rowmax[ij.y]);
  const double tau = a.tau;
  const int lane = threadIdx.x & 31;
  const unsigned lower = (1u << lane) - 1u;
  for (int g = a.mol_seg[m]; g < a.mol_seg[m + 1]; ++g) {
    const int cq = a.seg_class[g];
    if (cq > cp) break;
    const int64_t b0 = a.seg_begin[g];
    const int64_t e0 = cq == cp ? a.pos[p] + 1 : a.seg_begin[g + 1];
    // the segment's largest Q first: most pairs of a large molecule meet none of its pairs
    if (b0 >= e0 || qp * a.Q[a.order[b0]] * dr < tau) continue;
    // first position whose Q_p Q_q rowmax falls below tau (Q decreasing along the segment)
    int64_t lo = b0, hi = e0;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (qp * a.Q[a.order[mid]] * dr >= tau) lo = mid + 1; else hi = mid;
    }
    const int64_t cut = lo;
    const int64_t bucket = (int64_t)cp * (cp + 1) / 2 + cq;
    for (int64_t base = b0; base < cut; base += blockDim.x) {
      const int64_t i = base + threadIdx.x;
      bool keep = false;
      int q = 0;
      if (i < cut) {
        q = a.order[i];
        const int2 kl = a.pair_shells[q];
        const double d = fmax(fmax(di[kl.x - f], di[kl.y - f]), fmax(dj[kl.x - f], dj[kl.y - f]));
        keep = qp * a.Q[q] * d >= tau;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, keep);
      if (!mask) continue;
      const int leader = __ffs(mask) - 1;
      unsigned long long slot = 0;
      if (lane == leader) slot = atomicAdd(a.counts + bucket, (unsigned long long)__popc(mask));
      slot = __shfl_sync(0xffffffffu, slot, leader);
      if (fill && keep) a.out[a.bucket_off[bucket] + (int64_t)slot + __popc(mask & lower)] = make_int2((int)p, q);
    }
  }
}

cudaError_t launch_screen(const ScreenArgs& a, bool fill, cudaStream_t s) {
  if (a.npairs <= 0) return cudaSuccess;
  if (a.npairs > 0x7fffffff) return cudaErrorInvalidValue;
  k_screen<<<(unsigned)a.npairs, 256, 0, s>>>(a, fill);
  return cudaGetLastError();
}

__global__ void k_map_pairs(const int2* __restrict__ qp, int64_t n, const int64_t* __restrict__ orig,
                            int32_t* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int2 v = qp[k];
  out[2 * k] = (int32_t)orig[v.x];
  out[2 * k + 1] = (int32_t)orig[v.y];
}

cudaError_t launch_map_pairs(const int2* qp, int64_t n, const int64_t* orig, int32_t* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_map_pairs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(qp, n, orig, out);
  return cudaGetLastError();
}

// energy += alpha sum_i D[i] K[i] over n doubles (block sums, one atomic per block)
__global__ void __launch_bounds__(256) k_dot_energy(const double* __restrict__ D, const double* __restrict__ K,
                                                    int64_t n, double alpha, double* energy) {
  __shared__ double part[8];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(D[i], K[i], acc);
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(energy, alpha * t);
  }
}

cudaError_t launch_dot_energy(const double* D, const double* K, int64_t n, double alpha, double* energy,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 2048);
  k_dot_energy<<<grid, 256, 0, s>>>(D, K, n, alpha, energy);
  return cudaGetLastError();
}

__global__ void k_symmetrize(double* K, int32_t nao) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = nao;
  if (g >= n * n) return;
  const int64_t r = g / n, c = g - r * n;
  if (c < r) return;
  const double t = K[r * n + c] + K[c * n + r];
  K[r * n + c] = t;
  K[c * n + r] = t;
}

cudaError_t launch_symmetrize(double* K, int32_t nao, cudaStream_t s) {
  const int64_t tot = (int64_t)nao * nao;
  if (tot <= 0) return cudaSuccess;
  k_symmetrize<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(K, nao);
  return cudaGetLastError();
}

// K <- K + K^T for several molecules at once: blockIdx.y is the molecule.
__global__ void k_symmetrize_multi(double* const* K, const int32_t* nao) {
  const int m = blockIdx.y;
  const int64_t n = nao[m];
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * n) return;
  const int64_t r = g / n, c = g - r * n;
  if (c < r) return;
  double* k = K[m];
  const double t = k[r * n + c] + k[c * n + r];
  k[r * n + c] = t;
  k[c * n + r] = t;
}

// K = 0 for several molecules at once.
__global__ void k_zero_multi(double* const* K, const int32_t* nao) {
  const int m = blockIdx.y;
  const int64_t n = nao[m];
  double* k = K[m];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n * n; g += (int64_t)gridDim.x * blockDim.x)
    k[g] = 0.0;
}

cudaError_t launch_multi_k(double* const* K, const int32_t* nao, int32_t nmol, int64_t max_nao, bool zero,
                           cudaStream_t s) {
  if (nmol <= 0 || max_nao <= 0) return cudaSuccess;
  const int64_t tot = max_nao * max_nao;
  if (zero) {
    dim3 grid((unsigned)std::min<int64_t>((tot + 255) / 256, 4096), (unsigned)nmol);
    k_zero_multi<<<grid, 256, 0, s>>>(K, nao);
  } else {
    dim3 grid((unsigned)((tot + 255) / 256), (unsigned)nmol);
    k_symmetrize_multi<<<grid, 256, 0, s>>>(K, nao);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------- solid harmonics
// Cartesian -> real-solid-harmonic transform of one class of shellsets, one
// thread per solid-harmonic element:
//   out[a'b'c'd'] = sum C_{a'a} C_{b'b} C_{c'c} C_{d'd} [ab|cd]
// over the non-zero coefficients only (the sparse tables). Used for the small
// classes of the register kernels, whose shellsets hold at most a few hundred
// values.
__global__ void __launch_bounds__(256) k_cart2sph(const SphLaunch a) {
  const int la = a.la, lb = a.lb, lc = a.lc, ld = a.ld;
  const int nsb = 2 * lb + 1, nsc = 2 * lc + 1, nsd = 2 * ld + 1;
  const int ns = (2 * la + 1) * nsb * nsc * nsd;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.nq * ns) return;
  const int64_t q = g / ns;
  int o = (int)(g - q * ns);
  const int dp = o % nsd; o /= nsd;
  const int cp = o % nsc; o /= nsc;
  const int bp = o % nsb;
  const int ap = o / nsb;
  const int ncb = d_ncart(lb), ncc = d_ncart(lc), ncd = d_ncart(ld);
  const double* in = a.cart + a.coff[q];
  double acc = 0.0;
  for (int i = 0; i < c_spn[la][ap]; ++i)
    for (int j = 0; j < c_spn[lb][bp]; ++j) {
      const double cab = c_spv[la][ap][i] * c_spv[lb][bp][j];
      const int rab = c_spk[la][ap][i] * ncb + c_spk[lb][bp][j];
      for (int k = 0; k < c_spn[lc][cp]; ++k) {
        const double cabc = cab * c_spv[lc][cp][k];
        const double* row = in + (int64_t)(rab * ncc + c_spk[lc][cp][k]) * ncd;
        for (int m = 0; m < c_spn[ld][dp]; ++m) acc = fma(cabc * c_spv[ld][dp][m], __ldg(row + c_spk[ld][dp][m]), acc);
      }
    }
  a.out[a.ooff[q] + (((int64_t)ap * nsb + bp) * nsc + cp) * nsd + dp] = acc;
}

cudaError_t launch_cart2sph(const SphLaunch& a, cudaStream_t s) {
  if (a.nq <= 0) return cudaSuccess;
  const int64_t ns = (int64_t)(2 * a.la + 1) * (2 * a.lb + 1) * (2 * a.lc + 1) * (2 * a.ld + 1);
  const int64_t grid = (a.nq * ns + 255) / 256;
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  k_cart2sph<<<(unsigned)grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- Schwarz
__global__ void k_schwarz_reduce(const int64_t* __restrict__ off, const int32_t* __restrict__ nab, int64_t n,
                                 const double* __restrict__ vals, double* __restrict__ Q) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int m = nab[p];
  const double* v = vals + off[p];
  double mx = 0.0;
  for (int i = 0; i < m; ++i) mx = fmax(mx, fabs(v[(int64_t)i * m + i]));
  Q[p] = sqrt(mx);
}

cudaError_t launch_schwarz_reduce(const int64_t* off, const int32_t* nab, int64_t n, const double* vals, double* Q,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int bs = 128;
  k_schwarz_reduce<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(off, nab, n, vals, Q);
  return cudaGetLastError();
}

cudaError_t kernel_attributes_init() {
  double dint[64];
  for (int i = 0; i < 64; ++i) dint[i] = (double)i;
  cudaError_t e = cudaMemcpyToSymbol(c_dint, dint, sizeof(dint));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dint, dint, sizeof(dint));
  if (e != cudaSuccess) return e;
  double gh[kBoysOrders];
  // sqrt(pi)/2 * (2m-1)!! / 2^m
  double v = 0.88622692545275801365;
  for (int m = 0; m < kBoysOrders; ++m) {
    gh[m] = v;
    v *= (2.0 * m + 1.0) * 0.5;
  }
  e = cudaMemcpyToSymbol(c_gh, gh, sizeof(gh));
  if (e != cudaSuccess) return e;
  uint32_t cart[8][36] = {};
  for (int l = 0; l < 8; ++l) {
    int i = 0;
    for (int ax = l; ax >= 0; --ax)
      for (int ay = l - ax; ay >= 0; --ay) cart[l][i++] = (uint32_t)ax | ((uint32_t)ay << 8) | ((uint32_t)(l - ax - ay) << 16);
  }
  e = cudaMemcpyToSymbol(c_cart, cart, sizeof(cart));
  if (e != cudaSuccess) return e;
  {
    const auto tabs = build_solid_tables(kLmax);
    std::vector<double> flat;
    int offs[kLmax + 2];
    for (int l = 0; l <= kLmax; ++l) { offs[l] = (int)flat.size(); flat.insert(flat.end(), tabs[l].begin(), tabs[l].end()); }
    offs[kLmax + 1] = (int)flat.size();
    if (flat.size() > 840) return cudaErrorInvalidValue;
    e = cudaMemcpyToSymbol(c_sph, flat.data(), flat.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sph_off, offs, sizeof(offs));
    if (e != cudaSuccess) return e;
    int spn[kLmax + 1][2 * kLmax + 1] = {};
    uint8_t spk[kLmax + 1][2 * kLmax + 1][kSphNnzMax] = {};
    double spv[kLmax + 1][2 * kLmax + 1][kSphNnzMax] = {};
    for (int l = 0; l <= kLmax; ++l) {
      const int nc = ncart(l);
      for (int m = 0; m < 2 * l + 1; ++m)
        for (int k = 0; k < nc; ++k) {
          const double c = tabs[l][(size_t)m * nc + k];
          if (c == 0.0) continue;
          if (spn[l][m] >= kSphNnzMax) return cudaErrorInvalidValue;
          spk[l][m][spn[l][m]] = (uint8_t)k;
          spv[l][m][spn[l][m]] = c;
          ++spn[l][m];
        }
    }
    e = cudaMemcpyToSymbol(c_spn, spn, sizeof(spn));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_spk, spk, sizeof(spk));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_spv, spv, sizeof(spv));
    if (e != cudaSuccess) return e;
    uint16_t top[kLmax + 1][(kLmax + 1) * (kLmax + 2) / 2] = {};
    for (int l = 0; l <= kLmax; ++l) {
      int k = 0;
      for (int ax = l; ax >= 0; --ax)
        for (int ay = l - ax; ay >= 0; --ay, ++k) {
          const int az = l - ax - ay;
          // offset of row (u, v) = (ay, az) in the [u][v][t] simplex of order l, then t = ax
          const int row = tet(l + 1) - tet(l - ay + 1) + tri(l - ay + 1) - tri(l - ay - az + 1);
          top[l][k] = (uint16_t)(row + ax);
        }
    }
    e = cudaMemcpyToSymbol(c_top, top, sizeof(top));
    if (e != cudaSuccess) return e;
  }
  const int maxshm = 227 * 1024;
  e = cudaFuncSetAttribute(k_quartets<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxshm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_quartets<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxshm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_quartets_sph<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxshm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_quartets_sph<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxshm);
  if (e != cudaSuccess) return e;
  // the persistent kernel also holds ~0.5 KB of static shared memory (item index, launch descriptor)
  e = cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, maxshm - 1024);
  return e;
}

}  // namespace mdx
