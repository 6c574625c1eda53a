// Materialized-Hermite path (the paper's third GPU variant V2, Sec. 3: the
// Hermite integral matrix [p|q] is written to memory and both transforms are
// dense matrix products), kept as an A/B experiment against the
// axis-factored team and register kernels.
//
// Per uncontracted 4-center class, this file builds
//   E^ab  [N_b x Nt(L_b)]  per bra pair   (E^ab_{tuv} = Ex Ey Ez, Eq. E2rr1/2),
//   E^cd  [Nt(L_k) x N_k]  per ket pair,
//   [p|q] [Nt(L_b) x Nt(L_k)] per quartet: (-1)^{|q|} [p+q] (Eqs. pq, r, 0m),
// and the host multiplies [p|cd] = [p|q] E^cd, then [ab|cd] = E^ab [p|cd]
// with batched DGEMMs (cuBLAS, which runs FP64 GEMMs on the DMMA units).
#include "kernels.cuh"

namespace mdx {
namespace {

__device__ __forceinline__ int m_tet(int n) { return n < 0 ? 0 : n * (n + 1) * (n + 2) / 6; }
__device__ __forceinline__ int m_tri(int n) { return n < 0 ? 0 : n * (n + 1) / 2; }
// position of (t,u,v) in the [t][u][v] simplex of total order N
__device__ __forceinline__ int m_hidx(int N, int t, int u, int v) {
  return m_tet(N + 1) - m_tet(N - t + 1) + m_tri(N - t + 1) - m_tri(N - t - u + 1) + v;
}
// Cartesian component k of shell l: a_x = l..0, then a_y = l-a_x..0
__device__ __forceinline__ void m_cart(int l, int k, int& ax, int& ay, int& az) {
  ax = l;
  while (k > l - ax) { k -= l - ax + 1; --ax; }
  ay = l - ax - k;
  az = l - ax - ay;
}
__device__ __forceinline__ int m_etab_size(int la, int lb) {
  int s = 0;
  for (int a = 0; a <= la; ++a)
    for (int b = 0; b <= lb; ++b) s += a + b + 1;
  return s;
}
__device__ __forceinline__ int m_etab_off(int lb, int a, int b) {
  int s = 0;
  for (int a2 = 0; a2 < a; ++a2)
    for (int b2 = 0; b2 <= lb; ++b2) s += a2 + b2 + 1;
  for (int b2 = 0; b2 < b; ++b2) s += a + b2 + 1;
  return s;
}

// E^ab (bra: rows = Cartesian pair ab, cols = Hermite p) or E^cd (ket: rows =
// Hermite q, cols = Cartesian pair cd) of each listed pair, from its record.
__global__ void k_mat_emat(const double* __restrict__ recs, const int64_t* __restrict__ pair_rec,
                           const int32_t* __restrict__ pairs, int64_t npairs, int la, int lb, int bra,
                           double* __restrict__ E) {
  const int L = la + lb;
  const int nc_a = (la + 1) * (la + 2) / 2, nc_b = (lb + 1) * (lb + 2) / 2;
  const int ncart = nc_a * nc_b, nh = m_tet(L + 1);
  const int64_t per = (int64_t)ncart * nh;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npairs * per) return;
  const int64_t u = g / per;
  const int r = (int)(g - u * per);
  int ab, h;
  if (bra) { ab = r / nh; h = r - ab * nh; } else { h = r / ncart; ab = r - h * ncart; }
  // Hermite index h -> (t,u,v) in the simplex of order L
  int t = 0, uu = 0, v = 0;
  {
    int rem = h;
    for (t = 0; t <= L; ++t) {
      const int cnt = m_tri(L - t + 1);
      if (rem < cnt) break;
      rem -= cnt;
    }
    for (uu = 0; uu <= L - t; ++uu) {
      const int cnt = L - t - uu + 1;
      if (rem < cnt) break;
      rem -= cnt;
    }
    v = rem;
  }
  int ax, ay, az, bx, by, bz;
  m_cart(la, ab / nc_b, ax, ay, az);
  m_cart(lb, ab % nc_b, bx, by, bz);
  double val = 0.0;
  if (t <= ax + bx && uu <= ay + by && v <= az + bz) {
    const double* rec = recs + pair_rec[pairs[u]];
    const int tab = m_etab_size(la, lb);
    val = rec[kRecHeader + m_etab_off(lb, ax, bx) + t] * rec[kRecHeader + tab + m_etab_off(lb, ay, by) + uu] *
          rec[kRecHeader + 2 * tab + m_etab_off(lb, az, bz) + v];
  }
  E[g] = val;
}

// [p|q] = (-1)^{|q|} R_{p+q} of each quartet of a chunk: one block per quartet;
// Boys seeds by the library's Taylor table (Horner's rule), R levels in shared
// memory (Eq. r), then the Nt(L_b) x Nt(L_k) matrix, row-major.
__global__ void k_mat_hermite(const double* __restrict__ recs, const int64_t* __restrict__ pair_rec,
                              const int2* __restrict__ qp, int64_t nq, int Lb, int Lk,
                              const double* __restrict__ boys, double* __restrict__ PQ) {
  extern __shared__ double sm[];
  const int L = Lb + Lk;
  const int nR = m_tet(L + 1);
  double* G = sm;                 // L + 1
  double* R0 = sm + 32;           // nR
  double* R1 = R0 + nR;           // nR
  const int64_t q = blockIdx.x;
  if (q >= nq) return;
  const int2 p = qp[q];
  const double* rb = recs + pair_rec[p.x];
  const double* rk = recs + pair_rec[p.y];
  const int tl = threadIdx.x, T = blockDim.x;
  const double PQx = rb[2] - rk[2], PQy = rb[3] - rk[3], PQz = rb[4] - rk[4];
  if (tl <= L) {
    const double zp = rb[0], zq = rk[0];
    const double s = zp + zq;
    const double rs = rsqrt(s);
    const double rho = zp * zq * rs * rs;
    const double Tb = rho * (PQx * PQx + PQy * PQy + PQz * PQz);
    const double pref = 34.986836655249725693 * rb[1] * rk[1] * rs * rb[5] * rk[5];
    double pw = pref;
    for (int m = 0; m < tl; ++m) pw *= -2.0 * rho;
    double f;
    if (Tb < kBoysTmax) {
      const int i = __double2int_rn(Tb * kBoysInvH);
      const double nd = (double)i * (1.0 / kBoysInvH) - Tb;
      const double* c = boys + (size_t)i * kBoysRow + tl * kBoysTerms;
      f = c[kBoysTerms - 1];
      for (int k = kBoysTerms - 2; k >= 0; --k) f = fma(f, nd, c[k]);
    } else {
      // F_m(T) = Gamma(m+1/2) / (2 T^(m+1/2))
      const double t1 = rsqrt(Tb);
      f = 0.88622692545275801365 * t1;
      for (int m = 0; m < tl; ++m) f *= (m + 0.5) * t1 * t1;
    }
    G[tl] = pw * f;
  }
  __syncthreads();
  // level n holds [tuv]^(n) for t+u+v <= L-n in the simplex of order L
  double* cur = (L & 1) ? R1 : R0;
  if (tl == 0) cur[0] = G[L];
  __syncthreads();
  for (int n = L - 1; n >= 0; --n) {
    const double* src = cur;
    double* dst = (n & 1) ? R1 : R0;
    const int N = L - n;
    const int cnt = m_tet(N + 1);
    for (int e = tl; e < cnt; e += T) {
      int rem = e, t, u;
      for (t = 0; t <= N; ++t) { const int c = m_tri(N - t + 1); if (rem < c) break; rem -= c; }
      for (u = 0; u <= N - t; ++u) { const int c = N - t - u + 1; if (rem < c) break; rem -= c; }
      const int v = rem;
      double val;
      if (v > 0) {
        val = PQz * src[m_hidx(L, t, u, v - 1)];
        if (v > 1) val = fma((double)(v - 1), src[m_hidx(L, t, u, v - 2)], val);
      } else if (u > 0) {
        val = PQy * src[m_hidx(L, t, u - 1, 0)];
        if (u > 1) val = fma((double)(u - 1), src[m_hidx(L, t, u - 2, 0)], val);
      } else if (t > 0) {
        val = PQx * src[m_hidx(L, t - 1, 0, 0)];
        if (t > 1) val = fma((double)(t - 1), src[m_hidx(L, t - 2, 0, 0)], val);
      } else {
        val = G[n];
      }
      dst[m_hidx(L, t, u, v)] = val;
    }
    __syncthreads();
    cur = dst;
  }
  // [p|q] with rows p in the order-Lb simplex, columns q in the order-Lk simplex
  const int nb = m_tet(Lb + 1), nk = m_tet(Lk + 1);
  double* out = PQ + (int64_t)q * nb * nk;
  for (int e = tl; e < nb * nk; e += T) {
    const int ip = e / nk, iq = e - ip * nk;
    int rem = ip, t, u;
    for (t = 0; t <= Lb; ++t) { const int c = m_tri(Lb - t + 1); if (rem < c) break; rem -= c; }
    for (u = 0; u <= Lb - t; ++u) { const int c = Lb - t - u + 1; if (rem < c) break; rem -= c; }
    const int v = rem;
    int rq = iq, tq, uq;
    for (tq = 0; tq <= Lk; ++tq) { const int c = m_tri(Lk - tq + 1); if (rq < c) break; rq -= c; }
    for (uq = 0; uq <= Lk - tq; ++uq) { const int c = Lk - tq - uq + 1; if (rq < c) break; rq -= c; }
    const int vq = rq;
    const double r = cur[m_hidx(L, t + tq, u + uq, v + vq)];
    out[e] = ((tq + uq + vq) & 1) ? -r : r;
  }
}

// Pointer arrays of the two batched products of a chunk of quartets.
__global__ void k_mat_ptrs(int64_t nq, const int32_t* __restrict__ ib, const int32_t* __restrict__ ik,
                           const int64_t* __restrict__ qoff, const double* Eab, int64_t sEab, const double* Ecd,
                           int64_t sEcd, const double* PQ, int64_t sPQ, double* Tm, int64_t sT, double* out,
                           const double** a1, const double** b1, double** c1, const double** a2,
                           const double** b2, double** c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  a1[i] = Ecd + (int64_t)ik[i] * sEcd;
  b1[i] = PQ + i * sPQ;
  c1[i] = Tm + i * sT;
  a2[i] = Tm + i * sT;
  b2[i] = Eab + (int64_t)ib[i] * sEab;
  c2[i] = out + qoff[i];
}

}  // namespace

cudaError_t launch_mat_emat(const double* recs, const int64_t* pair_rec, const int32_t* pairs, int64_t npairs,
                            int la, int lb, bool bra, double* E, cudaStream_t s) {
  const int L = la + lb;
  const int64_t per = (int64_t)((la + 1) * (la + 2) / 2) * ((lb + 1) * (lb + 2) / 2) * ((L + 1) * (L + 2) * (L + 3) / 6);
  const int64_t tot = npairs * per;
  if (tot <= 0) return cudaSuccess;
  k_mat_emat<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(recs, pair_rec, pairs, npairs, la, lb, bra ? 1 : 0, E);
  return cudaGetLastError();
}

cudaError_t launch_mat_hermite(const double* recs, const int64_t* pair_rec, const int2* qp, int64_t nq, int Lb,
                               int Lk, const double* boys, double* PQ, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  const int L = Lb + Lk;
  const size_t shm = (32 + 2 * (size_t)((L + 1) * (L + 2) * (L + 3) / 6)) * sizeof(double);
  k_mat_hermite<<<(unsigned)nq, 256, shm, s>>>(recs, pair_rec, qp, nq, Lb, Lk, boys, PQ);
  return cudaGetLastError();
}

cudaError_t launch_mat_ptrs(int64_t nq, const int32_t* ib, const int32_t* ik, const int64_t* qoff,
                            const double* Eab, int64_t sEab, const double* Ecd, int64_t sEcd, const double* PQ,
                            int64_t sPQ, double* Tm, int64_t sT, double* out, const double** a1, const double** b1,
                            double** c1, const double** a2, const double** b2, double** c2, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  k_mat_ptrs<<<(unsigned)((nq + 127) / 128), 128, 0, s>>>(nq, ib, ik, qoff, Eab, sEab, Ecd, sEcd, PQ, sPQ, Tm, sT,
                                                         out, a1, b1, c1, a2, b2, c2);
  return cudaGetLastError();
}

}  // namespace mdx
