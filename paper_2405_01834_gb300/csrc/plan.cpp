// Host planner: turns one integral class into the step programs that the
// generic quartet kernel executes.
//
// The Hermite->Cartesian transforms of the paper (Eqs. ket-from-hermite and
// bra-from-hermite) contract the 2-index Hermite integrals [p|q] (Eq. pq)
// with E^{cd}_q and E^{ab}_p. Those matrices are products of per-axis factors
// (Sec. 2: E_{ab}^p = prod_i (E_i)_{a_i b_i}^{p_i}), so each transform is
// applied here one Cartesian axis at a time instead of as one dense product:
//
//   ket (for every ket column cd = (c, d)):
//     k1  A_z[t',u',v]  = sum_phi (-1)^phi Ez[cz,dz][phi] R[t',u',v+phi]
//     k2  B  [t',u ,v]  = sum_nu  (-1)^nu  Ey[cy,dy][nu]  A_z[t',u+nu,v]
//     k3  X  [t ,u ,v] += sum_tau (-1)^tau Ex[cx,dx][tau] B[t+tau,u,v]       (X = [p|cd])
//   bra (for every column, per bra primitive pair):
//     b1  C1[ax,bx; u,v] = sum_t Ex[ax,bx][t] X[t,u,v]
//     b23 OUT[ab]       += sum_v Ez[az,bz][v] sum_u Ey[ay,by][u] C1[ax,bx; u,v]
//
// (the signs (-1)^|q| of Eq. pq are folded into the ket-side E tables). The
// result is identical to the dense transforms up to rounding order; the FP64
// operation count is several times lower at l >= 2, which is what matters on a
// part whose FP64 rate is 1/64 of its FP32 rate.
//
// Every step is emitted as a list of entries "out = sum_k coef[c+k*s] *
// src[x+k*s]" over offsets in the team's shared-memory workspace; only
// entries some output depends on are emitted.
#include <array>
#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <tuple>

#include "mdx_internal.h"

namespace mdx {
namespace {

struct CartC { int x, y, z; };
std::vector<CartC> carts(int l) {
  std::vector<CartC> v;
  for (int ax = l; ax >= 0; --ax)
    for (int ay = l - ax; ay >= 0; --ay) v.push_back({ax, ay, l - ax - ay});
  return v;
}

// offset of row (t,u) in a [t][u][v] simplex layout of total order N
inline int roff(int N, int t, int u) { return tet(N + 1) - tet(N - t + 1) + tri(N - t + 1) - tri(N - t - u + 1); }

struct Layout {                  // a set of rows, each a contiguous run of doubles from its lowest used index
  std::map<std::pair<int, int>, std::pair<int, int>> rows;   // row key -> [lo, hi] of the used indices
  std::map<std::pair<int, int>, int> rowoff;
  int size = 0;
  void need(int r0, int r1, int lo, int hi) {   // elements lo..hi of row (r0,r1) are used
    auto it = rows.find({r0, r1});
    if (it == rows.end()) {
      rows[{r0, r1}] = {lo, hi};
    } else {
      it->second.first = std::min(it->second.first, lo);
      it->second.second = std::max(it->second.second, hi);
    }
  }
  void finalize() {
    size = 0;
    for (auto& kv : rows) { rowoff[kv.first] = size; size += kv.second.second - kv.second.first + 1; }
  }
  int at(int r0, int r1, int idx) const { return rowoff.at({r0, r1}) + idx - rows.at({r0, r1}).first; }
};

struct ColInfo { CartC c, d; int gcol; };

// Builds the ket programs of one group of columns; returns false on overflow.
// Offsets emitted are absolute in the team workspace. The A blocks (k1
// outputs) are laid out for the columns `a_cols` (default: the group's own),
// so that groups of one z-pair can share one A computed by the first of them
// (emit_k1 = false for the others).
bool build_group_k(const PlanDev& P, const std::vector<ColInfo>& cols, int o_A, int o_B, int o_X,
                   std::vector<StepEntry>& k1, std::vector<StepEntry>& k2, std::vector<StepEntry>& k3,
                   int& a_size, int& b_size, double& fma, const std::vector<ColInfo>* a_cols = nullptr,
                   bool emit_k1 = true) {
  const int Lb = P.Lb, L = P.L;
  const int Tcd = etab_size(P.lc, P.ld);
  // the X rows formed: t from tlo(u,v) (all of them, or the top Hermite shell t + u + v = Lb alone)
  auto tlo = [&](int u, int v) { return P.top_only ? Lb - u - v : 0; };
  // B layout per column: rows (u,v), t' contiguous over what k3 reads
  std::vector<Layout> BL(cols.size());
  for (size_t j = 0; j < cols.size(); ++j) {
    const int xx = cols[j].c.x + cols[j].d.x;
    for (int u = 0; u <= Lb; ++u)
      for (int v = 0; u + v <= Lb; ++v) BL[j].need(u, v, tlo(u, v), Lb - u - v + xx);
    BL[j].finalize();
  }
  std::map<std::pair<int, int>, Layout> AL;    // per z-pair (cz,dz): rows (t',v), u' contiguous over what k2 reads
  for (const ColInfo& ci : a_cols ? *a_cols : cols) {
    const CartC& c = ci.c; const CartC& d = ci.d;
    const int xx = c.x + d.x, yy = c.y + d.y;
    Layout& A = AL[{c.z, d.z}];
    for (int u = 0; u <= Lb; ++u)
      for (int v = 0; u + v <= Lb; ++v)
        for (int tp = tlo(u, v); tp <= Lb - u - v + xx; ++tp) A.need(tp, v, u, u + yy);
  }
  // A blocks back to back
  std::map<std::pair<int, int>, int> abase;
  int asz = 0;
  for (auto& kv : AL) { kv.second.finalize(); abase[kv.first] = asz; asz += kv.second.size; }
  std::vector<int> bbase(cols.size());
  int bsz = 0;
  for (size_t j = 0; j < cols.size(); ++j) { bbase[j] = bsz; bsz += BL[j].size; }
  a_size = asz; b_size = bsz;
  const int reck = P.o_reck + kRecHeader;
  auto push = [&](std::vector<StepEntry>& v, long out, long src, long coef, int n) {
    if (out > 65535 || src > 65535 || coef > 65535 || n > 255) return false;
    v.push_back(StepEntry{(uint16_t)out, (uint16_t)src, (uint16_t)coef, (uint8_t)n, (uint8_t)1});
    fma += n;
    return true;
  };
  // k1: A_z[t',u',v] = sum_phi Ez'[cz,dz][phi] R[t',u',v+phi]
  for (auto& kv : AL) {
    if (!emit_k1) break;
    const int cz = kv.first.first, dz = kv.first.second;
    const int coef = reck + 2 * Tcd + etab_off(P.lc, P.ld, cz, dz);
    for (auto& row : kv.second.rows) {
      const int tp = row.first.first, v = row.first.second;
      for (int up = row.second.first; up <= row.second.second; ++up) {
        if (tp + up + v + cz + dz > L) return false;   // cannot happen (see derivation)
        if (!push(k1, o_A + abase[kv.first] + kv.second.at(tp, v, up), P.o_R0 + roff(L, tp, up) + v, coef, cz + dz + 1))
          return false;
      }
    }
  }
  for (size_t j = 0; j < cols.size(); ++j) {
    const CartC& c = cols[j].c; const CartC& d = cols[j].d;
    const int xx = c.x + d.x, yy = c.y + d.y;
    const Layout& A = AL[{c.z, d.z}];
    const int ab0 = o_A + abase[{c.z, d.z}];
    const int coefy = reck + Tcd + etab_off(P.lc, P.ld, c.y, d.y);
    const int coefx = reck + etab_off(P.lc, P.ld, c.x, d.x);
    // k2: B[t',u,v] = sum_nu Ey'[cy,dy][nu] A[t',u+nu,v]
    for (auto& row : BL[j].rows) {
      const int u = row.first.first, v = row.first.second;
      for (int tp = row.second.first; tp <= row.second.second; ++tp)
        if (!push(k2, o_B + bbase[j] + BL[j].at(u, v, tp), ab0 + A.at(tp, v, u), coefy, yy + 1)) return false;
    }
    // k3: X[t,u,v] += sum_tau Ex'[cx,dx][tau] B[t+tau,u,v]   (top_only: the rows t + u + v = Lb alone)
    for (int u = 0; u <= Lb; ++u)
      for (int v = 0; u + v <= Lb; ++v)
        for (int t = tlo(u, v); t + u + v <= Lb; ++t) {
          const int xo = o_X + (int)j * P.hb + roff(Lb, u, v) + t;   // X rows (u,v), t contiguous
          if (!push(k3, xo, o_B + bbase[j] + BL[j].at(u, v, t), coefx, xx + 1)) return false;
        }
  }
  return true;
}

// Sort a step's entries so that neighbouring lanes run loops of equal length.
void sort_by_n(std::vector<StepEntry>& v) {
  std::stable_sort(v.begin(), v.end(), [](const StepEntry& a, const StepEntry& b) { return a.n > b.n; });
}

// Every shared-memory access the kernel will make from these programs stays
// inside the team's workspace and inside the region it belongs to.
bool validate_plan(const Plan& plan, std::string& err) {
  const PlanDev& P = plan.d;
  const long W = P.team_doubles;
  auto in = [&](long lo, long hi, long a) { return a >= lo && a < hi; };
  const long xr = P.o_X;   // the ket groups' X columns
  // the bra steps' layout: the plan's own, or the bra pass of a solid-harmonic plan
  const long bx = P.sph ? P.o_Xs : P.o_X, cr = P.sph ? P.o_C1s : P.o_C1, orr = P.sph ? P.o_OUTs : P.o_OUT;
  const long c1stride = P.sph ? P.c1s : P.c1size;
  const long out_cols = P.sph ? (long)P.ncols_s * P.Nb : (P.has_out ? (long)P.ncols_max * P.Nb : 0);
  for (const Group& g : plan.groups) {
    if (g.ncols < 1 || g.ncols > P.ncols_max) { err = "bad group width"; return false; }
    const StepEntry* k = plan.kprog.data();
    for (int i = 0; i < g.k1_n + g.k2_n + g.k3_n; ++i) {
      const StepEntry& s = k[g.k1_off + i];
      const long last = (long)(s.n - 1) * s.stride;
      if (s.n < 1 || !in(0, W, s.out) || !in(0, W, s.src + last) || !in(0, W, s.coef + last)) {
        err = "ket program entry out of the workspace";
        return false;
      }
    }
    // k1 reads R0 and writes A; k2 reads A writes B; k3 reads B writes X
    for (int i = 0; i < g.k1_n; ++i) {
      const StepEntry& s = k[g.k1_off + i];
      if (!in(P.o_R0, P.o_R0 + tet(P.L + 1), s.src) || !in(P.o_R0, P.o_R0 + tet(P.L + 1), s.src + s.n - 1) ||
          !in(P.o_A, g.o_B, s.out)) { err = "k1 entry outside R/A"; return false; }
    }
    for (int i = 0; i < g.k2_n; ++i) {
      const StepEntry& s = k[g.k2_off + i];
      if (!in(P.o_A, g.o_B, s.src) || !in(P.o_A, g.o_B, s.src + s.n - 1) || !in(g.o_B, P.o_X, s.out)) {
        err = "k2 entry outside A/B"; return false;
      }
    }
    for (int i = 0; i < g.k3_n; ++i) {
      const StepEntry& s = k[g.k3_off + i];
      if (!in(g.o_B, P.o_X, s.src) || !in(g.o_B, P.o_X, s.src + s.n - 1) ||
          !in(xr, xr + (long)g.ncols * P.hb, s.out)) { err = "k3 entry outside B/X"; return false; }
    }
    for (int i = g.col_off; i < g.col_off + g.ncols; ++i)
      if (plan.colmap[i] >= P.Nk) { err = "column map out of range"; return false; }
  }
  const long ncm = P.sph ? P.ncols_s : P.ncols_max;
  for (const StepEntry& s : plan.b1) {
    const long last = (long)(s.n - 1) * s.stride;
    if (!in(0, P.hb, s.src) || !in(0, P.hb, s.src + last) || !in(0, P.c1size, s.out) ||
        !in(P.o_recb, P.o_recb + P.recb, s.coef) || !in(P.o_recb, P.o_recb + P.recb, s.coef + last) ||
        bx + (ncm - 1) * P.hb + P.hb > cr) { err = "b1 entry out of range"; return false; }
  }
  for (const B23Entry& s : plan.b23) {
    const int vmax = s.v0 + (s.nv - 1) * s.sv;
    const long rowmax = (long)vmax * (s.r + 1) - (long)vmax * (vmax - 1) / 2;
    const long umax = s.u0 + (long)(s.nu - 1) * s.su;
    if (s.out >= P.Nb || !in(0, P.c1size, s.src + rowmax + umax) || umax > s.r - vmax ||
        !in(P.o_recb, P.o_recb + P.recb, s.ey + (long)(s.nu - 1) * s.su) ||
        !in(P.o_recb, P.o_recb + P.recb, s.ez + (long)(s.nv - 1) * s.sv) ||
        cr + ncm * c1stride > orr || orr + out_cols > W) {
      err = "b23 entry out of range";
      return false;
    }
  }
  if (P.o_R1 + tet(P.L) > P.o_X || P.o_R0 + tet(P.L + 1) > P.o_R1 || P.o_G + P.L + 1 > P.o_R0 ||
      P.o_reck + P.reck > P.o_scal) { err = "fixed regions overlap"; return false; }
  if (P.cache_R >= 2) {
    // the cached R tables lie after every other region of the workspace
    const long end_other = P.sph ? std::max<long>(P.o_OUT + (long)P.ncols_max * (P.has_out ? P.Nb : 0),
                                                  P.o_OUTs + (long)P.ncols_s * P.Nb)
                                 : P.o_OUT + (long)P.ncols_max * (P.has_out ? P.Nb : 0);
    if (P.o_Rc < end_other || P.o_Rc < P.o_X + (long)P.ncols_max * P.hb || P.rstride < tet(P.L + 1) ||
        P.o_Rc + (long)(P.cache_R == 2 ? P.Kb : 1) * P.Kk * P.rstride > W || (P.cache_R == 3 && !P.sph)) {
      err = "cached R tables out of range";
      return false;
    }
  }
  if (P.sph) {
    // the bra pass starts where the ket groups' region starts (R at level 0 stays below it), and the
    // [a][b'] pass of each column fits its C1 slot
    if (P.o_Xs < P.o_R0 + tet(P.L + 1) || P.c1size > P.c1s || ncart(P.la) * P.nsb > P.c1s || P.ncols_s < 1 ||
        P.ncols_s > P.nsc * P.nsd || P.o_C1s < P.o_Xs + (long)P.ncols_s * P.hb ||
        P.o_OUTs < P.o_C1s + (long)P.ncols_s * P.c1s || P.hbp > P.hb) {
      err = "solid-harmonic bra pass out of range";
      return false;
    }
  }
  return true;
}

}  // namespace

void build_rlevel_programs(std::vector<uint32_t>& prog, std::vector<int32_t>& off) {
  prog.clear();
  off.clear();
  for (int N = 0; N <= kLtot; ++N) {
    off.push_back((int32_t)prog.size());
    for (int t = 0; t <= N; ++t)
      for (int u = 0; t + u <= N; ++u)
        for (int v = 0; t + u + v <= N; ++v) {
          // [tuv]^(n) = X_PQ [tuv - 1]^(n+1) + (i - 1) [tuv - 2]^(n+1) along the last raised axis
          int axis, i, s1, s2;
          if (v > 0) {
            axis = 2; i = v;
            s1 = roff(N - 1, t, u) + v - 1;
            s2 = v > 1 ? roff(N - 1, t, u) + v - 2 : s1;
          } else if (u > 0) {
            axis = 1; i = u;
            s1 = roff(N - 1, t, u - 1);
            s2 = u > 1 ? roff(N - 1, t, u - 2) : s1;
          } else if (t > 0) {
            axis = 0; i = t;
            s1 = roff(N - 1, t - 1, 0);
            s2 = t > 1 ? roff(N - 1, t - 2, 0) : s1;
          } else {
            axis = 0; i = 1; s1 = 0; s2 = 0;
          }
          prog.push_back((uint32_t)s1 | ((uint32_t)s2 << 12) | ((uint32_t)axis << 24) | ((uint32_t)(i - 1) << 26));
        }
  }
}

bool build_plan(const ClassKey& key, const PlanConfig& cfg, Plan& plan, std::string& err) {
  const int smem_budget_bytes = std::min(cfg.budget, 220 * 1024);
  PlanDev& P = plan.d;
  P = PlanDev{};
  P.la = key.la; P.lb = key.lb; P.lc = key.lc; P.ld = key.ld;
  P.Kb = key.Kb; P.Kk = key.Kk; P.onec = key.onec;
  if (key.onec && key.lb != 0) { err = "one-centre bra needs lb = 0"; return false; }
  P.Lb = key.la + key.lb; P.Lk = key.lc + key.ld; P.L = P.Lb + P.Lk;
  P.Nb = ncart(key.la) * ncart(key.lb); P.Nk = ncart(key.lc) * ncart(key.ld);
  // per-column strides of X and C1 are odd numbers of doubles, so the 16 lanes
  // of a half-warp that read the same entry of consecutive columns hit 16
  // different shared-memory bank pairs
  P.hb = nherm(P.Lb) | 1;
  P.recb = rec_size(key.la, key.lb);
  P.reck = rec_size(key.lc, key.ld);
  const int Tab = etab_size(key.la, key.lb);
  const auto ca = carts(key.la), cb = carts(key.lb), cc = carts(key.lc), cd = carts(key.ld);

  // fixed part of the workspace
  P.o_recb = 0;
  P.o_reck = P.recb;
  P.o_scal = P.o_reck + P.reck;          // end of the records
  P.o_G = P.o_scal;
  P.o_R0 = P.o_G + ((P.L + 2 + 1) & ~1);
  const int r0size = tet(P.L + 1);
  const int r1size = tet(P.L);
  const int o_region = P.o_R0 + ((r0size + 1) & ~1);

  // ---- bra templates (per column) -------------------------------------
  // C1 per column: blocks (ax,bx), rows v = 0..r, row v holds u = 0..r-v
  std::map<std::pair<int, int>, int> c1off;
  int c1 = 0;
  for (int ax = 0; ax <= key.la; ++ax)
    for (int bx = 0; bx <= key.lb; ++bx) {
      c1off[{ax, bx}] = c1;
      c1 += tri(P.Lb - ax - bx + 1);
    }
  P.c1size = c1 | 1;
  const int recb_tab = P.o_recb + kRecHeader;
  plan.b1.clear(); plan.b23.clear();
  double fma_b = 0;
  for (int ax = 0; ax <= key.la; ++ax)
    for (int bx = 0; bx <= key.lb; ++bx) {
      const int r = P.Lb - ax - bx;
      const int t0 = key.onec ? (ax & 1) : 0, st = key.onec ? 2 : 1;
      const int n = key.onec ? (ax - t0) / 2 + 1 : ax + bx + 1;
      for (int v = 0; v <= r; ++v)
        for (int u = 0; u + v <= r; ++u) {
          const int out = c1off[{ax, bx}] + v * (r + 1) - v * (v - 1) / 2 + u;
          const int src = roff(P.Lb, u, v) + t0;
          const int coef = recb_tab + etab_off(key.la, key.lb, ax, bx) + t0;
          plan.b1.push_back(StepEntry{(uint16_t)out, (uint16_t)src, (uint16_t)coef, (uint8_t)n, (uint8_t)st});
          fma_b += n;
        }
    }
  sort_by_n(plan.b1);
  for (size_t ia = 0; ia < ca.size(); ++ia)
    for (size_t ib = 0; ib < cb.size(); ++ib) {
      const CartC a = ca[ia], b = cb[ib];
      const int r = P.Lb - a.x - b.x;
      B23Entry e{};
      e.out = (uint16_t)(ia * cb.size() + ib);
      e.src = (uint16_t)c1off[{a.x, b.x}];
      e.r = (uint8_t)r;
      if (key.onec) {
        e.u0 = (uint8_t)(a.y & 1); e.su = 2; e.nu = (uint8_t)((a.y - e.u0) / 2 + 1);
        e.v0 = (uint8_t)(a.z & 1); e.sv = 2; e.nv = (uint8_t)((a.z - e.v0) / 2 + 1);
      } else {
        e.u0 = 0; e.su = 1; e.nu = (uint8_t)(a.y + b.y + 1);
        e.v0 = 0; e.sv = 1; e.nv = (uint8_t)(a.z + b.z + 1);
      }
      e.ey = (uint16_t)(recb_tab + Tab + etab_off(key.la, key.lb, a.y, b.y) + e.u0);
      e.ez = (uint16_t)(recb_tab + 2 * Tab + etab_off(key.la, key.lb, a.z, b.z) + e.v0);
      plan.b23.push_back(e);
      fma_b += e.nv * (e.nu + 1.0);
    }
  // equal loop shapes next to each other (lanes of a warp run the same trip counts)
  std::stable_sort(plan.b23.begin(), plan.b23.end(), [](const B23Entry& x, const B23Entry& y) {
    return x.nv != y.nv ? x.nv > y.nv : x.nu > y.nu;
  });
  P.nb1 = (int)plan.b1.size();
  P.nb23 = (int)plan.b23.size();

  // ---- columns ----------------------------------------------------------
  std::vector<ColInfo> allcols;
  for (size_t ic = 0; ic < cc.size(); ++ic)
    for (size_t id = 0; id < cd.size(); ++id) allcols.push_back({cc[ic], cd[id], (int)(ic * cd.size() + id)});

  // store-only plans of uncontracted-bra classes need no OUT region: b23 writes the shellset to global memory;
  // the ket groups of a solid-harmonic plan hold only their X columns (the bra pass has its own layout)
  const bool sph = key.store == 2;
  P.sph = sph ? 1 : 0;
  P.top_only = (sph && key.onec) ? 1 : 0;
  P.has_out = sph ? 0 : ((key.store && key.Kb == 1) ? 0 : 1);
  const int out_per_col = P.has_out ? P.Nb : 0;
  const int c1_per_col = sph ? 0 : P.c1size;
  auto region_size = [&](int a_size, int b_size) { return std::max(r1size, a_size + b_size); };
  auto team_doubles = [&](int a_size, int b_size, int ncols) {
    int reg = (region_size(a_size, b_size) + 1) & ~1;
    int tot = o_region + reg + ncols * P.hb + ncols * c1_per_col + ncols * out_per_col;
    return (tot + 1) & ~1;
  };

  // try a single group holding every column
  std::vector<std::vector<ColInfo>> groups;
  // z-pair columns whose shared A a group uses (uncontracted classes: R, and so
  // A, stays valid from one group to the next), and whether it computes that A
  std::vector<const std::vector<ColInfo>*> gz;
  std::vector<char> gfirst;
  const bool share_a = key.Kb * key.Kk == 1;
  auto group_sizes = [&](const std::vector<ColInfo>& g, int& as, int& bs, const std::vector<ColInfo>* zc) {
    std::vector<StepEntry> k1, k2, k3;
    double f = 0;
    return build_group_k(P, g, 0, 0, 0, k1, k2, k3, as, bs, f, zc);
  };
  {
    int as = 0, bs = 0;
    bool ok = group_sizes(allcols, as, bs, nullptr);
    const int td = team_doubles(as, bs, (int)allcols.size());
    if (ok && td * 8 <= std::min(smem_budget_bytes, cfg.single_max)) {
      groups.push_back(allcols);
      gz.push_back(nullptr);
      gfirst.push_back(1);
    }
  }
  int regmax = 0, cmax = 0;
  std::map<std::pair<int, int>, std::vector<ColInfo>> byz;   // columns per z-pair (outlives gz)
  if (groups.empty()) {
    // one group per z-pair, columns split into chunks of at most `cap` so that
    // the largest region plus the widest group fit the budget together
    for (auto& c : allcols) byz[{c.c.z, c.d.z}].push_back(c);
    size_t maxcap = 0;
    for (auto& kv : byz) maxcap = std::max(maxcap, kv.second.size());
    // groups of at most `cap` columns: a z-pair's columns split into chunks of nearly equal size, and
    // z-pairs of at most cap columns packed whole, in order, into shared groups (fewer barrier-separated
    // steps and wider bra steps than one small group per z-pair; each computes its own z-pairs' A)
    auto try_cap = [&](size_t cap) {
      groups.clear(); gz.clear(); gfirst.clear();
      regmax = 0; cmax = 0;
      bool ok = true;
      auto emit = [&](std::vector<ColInfo>&& g, const std::vector<ColInfo>* zc, bool first) {
        groups.push_back(std::move(g));
        gz.push_back(zc);
        gfirst.push_back(first);
        int as = 0, bs = 0;
        if (!group_sizes(groups.back(), as, bs, gz.back())) ok = false;
        regmax = std::max(regmax, region_size(as, bs));
        cmax = std::max(cmax, (int)groups.back().size());
      };
      std::vector<ColInfo> pending;
      for (auto& kv : byz) {
        std::vector<ColInfo>& cs = kv.second;
        if (cfg.pack_zpairs && cs.size() <= cap) {
          if (pending.size() + cs.size() > cap) emit(std::move(pending), nullptr, true), pending.clear();
          pending.insert(pending.end(), cs.begin(), cs.end());
          continue;
        }
        const size_t nchunk = (cs.size() + cap - 1) / cap;
        const size_t len = (cs.size() + nchunk - 1) / nchunk;
        for (size_t s0 = 0; s0 < cs.size(); s0 += len)
          emit(std::vector<ColInfo>(cs.begin() + s0, cs.begin() + std::min(cs.size(), s0 + len)),
               share_a ? &cs : nullptr, s0 == 0 || !share_a);
      }
      if (!pending.empty()) emit(std::move(pending), nullptr, true);
      const int td = o_region + ((regmax + 1) & ~1) + cmax * (P.hb + c1_per_col + out_per_col);
      return ok && td * 8 <= smem_budget_bytes;
    };
    // the largest cap that fits (binary search; the workspace grows with the cap)
    if (!try_cap(maxcap)) {
      size_t lo = 0, hi = maxcap;   // try_cap(hi) fails; lo is the largest known fit (0: none yet)
      while (hi - lo > 1) {
        const size_t mid = (lo + hi) / 2;
        if (try_cap(mid)) lo = mid; else hi = mid;
      }
      if (lo == 0) { err = "class does not fit the shared-memory budget"; return false; }
      try_cap(lo);
    }
  } else {
    int as = 0, bs = 0;
    group_sizes(groups[0], as, bs, nullptr);
    regmax = region_size(as, bs);
    cmax = (int)groups[0].size();
  }
  P.o_R1 = o_region;
  P.o_A = o_region;
  const int reg = (regmax + 1) & ~1;
  P.o_B = o_region;   // per group: o_A + that group's A size (programs carry absolute offsets)
  P.o_X = o_region + reg;
  P.o_C1 = P.o_X + cmax * P.hb;
  P.o_OUT = P.o_C1 + cmax * c1_per_col;
  // odd: the workspaces of the teams of a CTA start on different shared-memory
  // bank pairs, so lanes of different teams at the same offset do not conflict
  P.team_doubles = (P.o_OUT + cmax * out_per_col) | 1;
  P.ncols_max = cmax;
  if (sph) {
    // bra pass: spherical ket columns in groups of ncols_s, each column holding X (hb), C1 or the
    // [a][b'] pass (c1s) and OUT (Nb), laid out from o_region (the ket groups are finished by then)
    P.nsa = 2 * key.la + 1; P.nsb = 2 * key.lb + 1; P.nsc = 2 * key.lc + 1; P.nsd = 2 * key.ld + 1;
    P.c1s = std::max(P.c1size, ncart(key.la) * P.nsb) | 1;
    const int nks = P.nsc * P.nsd;
    const int per = P.hb + P.c1s + P.Nb;
    // as wide as fits in the ket groups' footprint (the workspace, and so the CTAs per SM, stay as the
    // ket part needs them), at least one column within the budget
    const int room = std::max(P.team_doubles - o_region, per);
    int cs = std::min(nks, std::min(room, smem_budget_bytes / 8 - o_region) / per);
    if (cs < 1) { err = "solid-harmonic bra pass does not fit the shared-memory budget"; return false; }
    const int ngs = (nks + cs - 1) / cs;
    cs = (nks + ngs - 1) / ngs;
    P.ncols_s = cs;
    P.o_Xs = o_region;
    P.o_C1s = P.o_Xs + cs * P.hb;
    P.o_OUTs = P.o_C1s + cs * P.c1s;
    P.team_doubles = std::max(P.team_doubles, P.o_OUTs + cs * P.Nb) | 1;
    P.hbp = nherm(P.Lb);
    P.xg_doubles = (int64_t)P.hbp * (P.Nk + (int64_t)ncart(key.lc) * P.nsd);
  }
  if (P.team_doubles >= 65536 || P.team_doubles * 8 > smem_budget_bytes) {
    err = "workspace exceeds the shared-memory budget";
    return false;
  }

  // emit the group programs with final offsets
  plan.groups.clear(); plan.kprog.clear(); plan.colmap.clear();
  double fma_k = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const std::vector<ColInfo>& g = groups[gi];
    std::vector<StepEntry> k1, k2, k3;
    int as = 0, bs = 0; double f = 0;
    group_sizes(g, as, bs, gz[gi]);
    const int oB = P.o_A + as;
    if (!build_group_k(P, g, P.o_A, oB, P.o_X, k1, k2, k3, as, bs, f, gz[gi], gfirst[gi] != 0)) {
      err = "program offsets overflow";
      return false;
    }
    fma_k += f;
    sort_by_n(k1); sort_by_n(k2); sort_by_n(k3);
    Group G{};
    G.k1_off = (int)plan.kprog.size(); G.k1_n = (int)k1.size();
    plan.kprog.insert(plan.kprog.end(), k1.begin(), k1.end());
    G.k2_off = (int)plan.kprog.size(); G.k2_n = (int)k2.size();
    plan.kprog.insert(plan.kprog.end(), k2.begin(), k2.end());
    G.k3_off = (int)plan.kprog.size(); G.k3_n = (int)k3.size();
    plan.kprog.insert(plan.kprog.end(), k3.begin(), k3.end());
    G.ncols = (int)g.size();
    G.o_B = oB;
    G.col_off = (int)plan.colmap.size();
    for (auto& c : g) plan.colmap.push_back((uint16_t)c.gcol);
    plan.groups.push_back(G);
  }
  P.ngroups = (int)plan.groups.size();
  P.cache_R = (key.Kb * key.Kk == 1) ? 1 : 0;
  // Contracted classes of several column groups would compute every primitive quartet's R once per
  // group: keep all Kb Kk tables in a region of their own instead (computed once per quartet, copied
  // into R0 before each group's k1), where it fits and the SM keeps as many teams (or at least two)
  P.rstride = (tet(P.L + 1) + 1) & ~1;
  P.o_Rc = 0;
  // (solid-harmonic plans, whose bra-primitive loop is outermost, fall back to the tables of one bra
  // primitive at a time)
  if (!P.cache_R && P.ngroups > 1 && cfg.rcache != 0) {
    const int o_Rc = (P.team_doubles + 1) & ~1;
    const int tps0 = std::max(1, (220 * 1024) / (P.team_doubles * 8));
    for (int mode = 2; mode <= (sph && key.Kb > 1 ? 3 : 2); ++mode) {
      const long td = ((long)o_Rc + (long)(mode == 2 ? key.Kb : 1) * key.Kk * P.rstride) | 1;
      const int tps1 = (int)((220L * 1024) / (td * 8));
      // (the cache may take the team past its planning budget, up to what one team can have: a smaller
      // budget means more column groups and so more R tables saved)
      if (td * 8 <= 220 * 1024 && td < 65536 && (cfg.rcache > 0 || tps1 >= std::min(tps0, 2))) {
        P.cache_R = mode;
        P.o_Rc = o_Rc;
        P.team_doubles = (int)td;
        break;
      }
    }
  }
  // inverse column maps: the digestion epilogue visits only the columns of its own K block
  plan.colinv.assign((size_t)P.ngroups * P.Nk, 0xffff);
  for (int gi = 0; gi < P.ngroups; ++gi)
    for (int j = 0; j < plan.groups[gi].ncols; ++j)
      plan.colinv[(size_t)gi * P.Nk + plan.colmap[plan.groups[gi].col_off + j]] = (uint16_t)j;

  // R recursion work: every level n < L has tet(L-n+1) - 1 entries of <= 2 ops
  double fma_r = 0;
  for (int n = 0; n < P.L; ++n) fma_r += tet(P.L - n + 1) - 1;
  const double nrec = (P.cache_R || P.ngroups == 1) ? 1.0 : P.ngroups;
  plan.exec_fma = key.Kb * key.Kk * (fma_k + nrec * (fma_r + 8.0 * (P.L + 1))) + key.Kb * fma_b * P.Nk;
  if (sph) {
    // per bra primitive: the two ket passes over the staged columns, the bra steps on the spherical
    // columns, and the two bra passes
    const double nks = (double)P.nsc * P.nsd;
    const double ket_sph = (double)P.hbp * ((double)ncart(key.lc) * solid_nnz(key.ld) + (double)solid_nnz(key.lc) * P.nsd);
    const double bra_sph = nks * ((double)ncart(key.la) * solid_nnz(key.lb) + (double)solid_nnz(key.la) * P.nsb);
    // top_only: one sparse sum over the top Hermite shell per solid-harmonic bra component and column
    const double bra = P.top_only ? nks * (double)solid_nnz(key.la) : fma_b * nks + bra_sph;
    plan.exec_fma = key.Kb * key.Kk * (fma_k + nrec * (fma_r + 8.0 * (P.L + 1))) + key.Kb * (ket_sph + bra);
  }
  const double team_fma_per_prim = plan.exec_fma / ((double)key.Kb * key.Kk);

  // register kernel (one thread per quartet) where the class has one
  const bool has_reg = reg_eligible(key.la, key.lb, key.lc, key.ld) || reg_xs_eligible(key.la, key.lb, key.lc, key.ld);
  if (cfg.variant == 2 && !has_reg && !sph) { err = "class has no register kernel"; return false; }
  // default: the register kernel (either variant) where the class has one; measured 1.6-4.4x faster than
  // the team kernel on contracted and uncontracted classes of total angular momentum <= 6
  P.reg = (has_reg && cfg.variant != 1 && !sph) ? 1 : 0;
  if (P.reg) {
    // its FP64 work: per primitive quartet Boys, R, the ket E products and
    // X += E R; per bra primitive the bra E products and V += E X
    auto comps = [](int l) {
      std::vector<std::array<int, 3>> v;
      for (int ax = l; ax >= 0; --ax)
        for (int ay = l - ax; ay >= 0; --ay) v.push_back({ax, ay, l - ax - ay});
      return v;
    };
    double ket = 0, bra = 0;
    for (auto& c : comps(key.lc))
      for (auto& d : comps(key.ld)) {
        const int nx = c[0] + d[0] + 1, ny = c[1] + d[1] + 1, nz = c[2] + d[2] + 1;
        ket += nx * ny * nz + nx * ny + (double)nherm(P.Lb) * nx * ny * nz;
      }
    for (auto& a : comps(key.la))
      for (auto& b : comps(key.lb)) {
        const int nx = a[0] + b[0] + 1, ny = a[1] + b[1] + 1, nz = a[2] + b[2] + 1;
        bra += nx * ny * nz + nx * ny + (double)P.Nk * nx * ny * nz;
      }
    plan.exec_fma = key.Kb * key.Kk * (fma_r + 8.0 * (P.L + 1) + ket) + key.Kb * bra;
  }

  if (!validate_plan(plan, err)) return false;

  // ---- team shape ------------------------------------------------------
  const int bytes = P.team_doubles * 8;
  const int tps = std::max(1, (220 * 1024) / bytes);   // teams that fit one SM's shared memory
  if (cfg.T > 0) {
    if (cfg.T > 1024 || (cfg.T & (cfg.T - 1))) { err = "team size must be a power of two <= 1024"; return false; }
    P.T = cfg.T;
  } else if (key.Kb * key.Kk > 1) {
    // contracted: the work per primitive quartet (Boys, R, ket steps) sets the
    // team; about 30 FMAs per lane per primitive quartet, at most 128 lanes
    // (GB300 sweeps of team sizes over contracted classes of L = 6..10) ...
    int Twork = 1;
    while (Twork < 512 && 2 * Twork * 30.0 <= team_fma_per_prim) Twork *= 2;
    P.T = std::min(Twork, 128);
    // ... unless shared memory leaves room for so few teams per SM that the SM would hold fewer
    // than 16 warps: then the team grows (up to what its work fills) to keep the FP64 pipe fed
    while (P.T < Twork && (long)tps * P.T < 512) P.T *= 2;
  } else if (P.ngroups > 1) {
    // solid-harmonic plans that hold one team per SM take 1024 lanes: their passes over the global
    // staging areas wait on loads, which 32 warps per SM hide better than 16 (autotuned [ii|ii]: 0.80 of
    // the FP64 peak against 0.74)
    P.T = (sph && tps == 1) ? 1024 : 512;
  } else {
    int Tocc = 1;
    while (Tocc * tps < 512 && Tocc < 512) Tocc *= 2;
    // about 8 output elements per lane, but at least half as many lanes as the largest R level has
    // entries: classes with few Cartesian components and a high total angular momentum ([l0|l0]) are
    // bound by their barrier-separated R levels (GB300 sweeps of the team size: [40|40] 16 -> 64 lanes
    // 1.9x, [50|50] 32 -> 128 lanes 1.9x, solid-harmonic output)
    int work = std::max({1, P.Nb * P.Nk / 8, nherm(P.L) / 2});
    int Twork = 1;
    while (Twork * 2 <= work && Twork < 512) Twork *= 2;
    P.T = std::min(Tocc, Twork);
  }
  if (P.T > 32) {
    P.teams_per_cta = 1;
  } else {
    // warp-sized teams share CTAs of at most 128 threads in whole warps; pick the count that keeps the
    // most teams resident per SM (228 KB of shared memory per SM, 1 KB of it reserved per CTA; at most
    // 32 CTAs and 2048 threads), the fewest teams per CTA among equals
    const int cap = std::min(std::max(1, 128 / P.T), tps);
    int best = cap;
    while (best > 1 && (long)best * bytes > smem_budget_bytes) --best;
    long best_res = -1;
    for (int tpc = 1; tpc <= cap; ++tpc) {
      const long cta = (long)tpc * bytes;
      if (cta > smem_budget_bytes) break;
      if ((tpc * P.T) % 32 != 0) continue;   // a part-filled warp idles FP64 lanes
      const long ctas = std::min({228L * 1024 / (cta + 1024), 2048L / ((long)tpc * P.T), 32L});
      if (ctas * tpc > best_res) { best_res = ctas * tpc; best = tpc; }
    }
    P.teams_per_cta = best;
  }
  if (P.T * P.teams_per_cta > 1024 || (long)P.teams_per_cta * P.team_doubles * 8 > 227 * 1024) {
    err = "team shape exceeds the CTA limits";
    return false;
  }
  // A contracted class of several column groups whose R tables do not fit next to a full-budget workspace:
  // a smaller planning budget (more, narrower groups) with the tables cached computes R once per primitive
  // quartet instead of once per group. The R levels are barrier-bound, so R work is weighted 3x against the
  // step programs' multiply-adds when the two plans are compared (the autotuner, which times both, measured
  // the cached plan 1.45-1.67x faster on contracted solid-harmonic [55|55] and [66|66]).
  if (P.cache_R == 0 && P.ngroups > 1 && key.Kb * key.Kk > 1 && cfg.rcache < 0 && cfg.budget >= 200 * 1024 &&
      cfg.T == 0) {
    PlanConfig alt = cfg;
    alt.budget = 108 * 1024;
    alt.rcache = 1;
    Plan p2;
    std::string e2;
    double r_eval = 8.0 * (P.L + 1);   // one R table: Boys seeds and the levels
    for (int n = 0; n < P.L; ++n) r_eval += tet(P.L - n + 1) - 1;
    const double r_cur = (double)key.Kb * key.Kk * P.ngroups * r_eval;
    const double r_alt = (double)key.Kb * key.Kk * r_eval;
    if (build_plan(key, alt, p2, e2) && p2.d.cache_R >= 2 &&
        p2.exec_fma + 2.0 * r_alt < 0.9 * (plan.exec_fma + 2.0 * r_cur))
      plan = std::move(p2);
  }
  return true;
}

}  // namespace mdx
