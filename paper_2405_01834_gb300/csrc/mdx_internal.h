// Internal definitions shared by the host planner and the CUDA kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace mdx {

constexpr int kLmax = 6;
constexpr int kKmax = 32;
constexpr int kLtot = 4 * kLmax + 1;   // highest Boys order used (gradients need L+1)

// ----------------------------------------------------------------- Boys table
// F_m(T0 + d) = sum_{k<kBoysTerms} F_{m+k}(T0) (-d)^k / k!, grid T0 = i * h,
// evaluated by Horner's rule in -d from coefficients F_{m+k}(T0) / k!.
constexpr int kBoysTerms = 8;
constexpr int kBoysMmax = kLtot;                    // highest m evaluated
constexpr int kBoysOrders = kBoysMmax + 1;          // m = 0 .. kBoysMmax
constexpr int kBoysRow = kBoysOrders * kBoysTerms;  // one grid point: [m][k]
constexpr double kBoysInvH = 16.0;                  // grid spacing h = 1/16
constexpr double kBoysTmax = 100.0;                 // asymptotic form above
constexpr int kBoysNgrid = 1601 + 1;                // T0 = 0 .. 100 (+1 guard row)

// Builds the interpolation table [kBoysNgrid][kBoysOrders][kBoysTerms]
// (row-major) in long double by downward recursion (see boys_table.cpp).
std::vector<double> build_boys_table();

// ----------------------------------------------------------------- records
// Primitive-pair record: header of kRecHeader doubles, then the three per-axis
// E tables (x, y, z). Header: [0] zeta_p, [1] 1/zeta_p, [2..4] P, [5] prefactor
// c_a c_b exp(-zeta_a zeta_b |A-B|^2 / zeta_p), [6], [7] unused.
constexpr int kRecHeader = 8;

inline int etab_size(int la, int lb) {      // sum over a<=la, b<=lb of (a+b+1)
  int s = 0;
  for (int a = 0; a <= la; ++a)
    for (int b = 0; b <= lb; ++b) s += a + b + 1;
  return s;
}
inline int etab_off(int la, int lb, int a, int b) {   // start of (a,b) block; t contiguous
  (void)la;
  int s = 0;
  for (int a2 = 0; a2 < a; ++a2)
    for (int b2 = 0; b2 <= lb; ++b2) s += a2 + b2 + 1;
  for (int b2 = 0; b2 < b; ++b2) s += a + b2 + 1;
  return s;
}
inline int rec_size(int la, int lb) {        // padded to a multiple of 2 doubles (16 bytes)
  int s = kRecHeader + 3 * etab_size(la, lb);
  return (s + 1) & ~1;
}

constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
constexpr int tri(int n) { return n < 0 ? 0 : n * (n + 1) / 2; }
constexpr int tet(int n) { return n < 0 ? 0 : n * (n + 1) * (n + 2) / 6; }
constexpr int nherm(int l) { return tet(l + 1); }

// Register kernel (one thread per quartet, all intermediates in registers):
// classes of total angular momentum <= 4 whose R table, [p|cd] block and
// shellset hold at most 100 doubles together have one.
constexpr int reg_footprint(int la, int lb, int lc, int ld) {
  return nherm(la + lb + lc + ld) + nherm(la + lb) * ncart(lc) * ncart(ld) + ncart(la) * ncart(lb) * ncart(lc) * ncart(ld);
}
constexpr bool reg_eligible(int la, int lb, int lc, int ld) {
  return la + lb + lc + ld <= 4 && reg_footprint(la, lb, lc, ld) <= 100;
}
// Size of the unrolled register-kernel body of a class: the R recursion, the
// ket transform (E products and FMAs per Cartesian ket pair and Hermite bra
// index) and, with_bra, the bra transform (the shared-memory variant runs the
// bra transform and the epilogues as runtime loops).
constexpr int reg_body_size(int la, int lb, int lc, int ld, bool with_bra = true) {
  int c = 2 * nherm(la + lb + lc + ld);
  for (int cx = lc; cx >= 0; --cx)
    for (int cy = lc - cx; cy >= 0; --cy)
      for (int dx = ld; dx >= 0; --dx)
        for (int dy = ld - dx; dy >= 0; --dy) {
          const int n = (cx + dx + 1) * (cy + dy + 1) * (lc - cx - cy + ld - dx - dy + 1);
          c += n + nherm(la + lb) * n;
        }
  if (!with_bra) return c;
  for (int ax = la; ax >= 0; --ax)
    for (int ay = la - ax; ay >= 0; --ay)
      for (int bx = lb; bx >= 0; --bx)
        for (int by = lb - bx; by >= 0; --by) {
          const int n = (ax + bx + 1) * (ay + by + 1) * (la - ax - ay + lb - bx - by + 1);
          c += n + ncart(lc) * ncart(ld) * n;
        }
  return c;
}
// Further classes of total angular momentum <= 6 have a variant with R in
// registers and [p|cd] plus the shellset in shared memory (64 threads x their
// doubles within 200 KB), as long as the unrolled body stays small enough to
// compile quickly.
constexpr bool reg_xs_eligible(int la, int lb, int lc, int ld) {
  return !reg_eligible(la, lb, lc, ld) && la + lb + lc + ld <= 6 &&
         (nherm(la + lb) + ncart(la) * ncart(lb)) * ncart(lc) * ncart(ld) * 64 * 8 <= 200 * 1024 &&
         reg_body_size(la, lb, lc, ld, false) <= 1000;
}

// ----------------------------------------------------------------- programs
// A "step" computes entries out = sum_{k<n} coef[c + k*s] * src[x + k*s]
// (offsets in doubles inside the team's shared-memory workspace).
struct StepEntry {            // 8 bytes
  uint16_t out;
  uint16_t src;
  uint16_t coef;
  uint8_t n;
  uint8_t stride;
};
// Two-level bra entry: out += sum_v Ez[ez + v*sv] * sum_u Ey[ey + u*su] * C1[row(v) + u*su]
// with row(v) = src + v*(r+1) - v*(v-1)/2 (rows of decreasing length r+1-v).
struct B23Entry {             // 16 bytes
  uint16_t out;
  uint16_t src;
  uint16_t ey;
  uint16_t ez;
  uint8_t u0, nu, su, v0;
  uint8_t nv, sv, r, pad;
};

struct Group {
  int32_t k1_off, k1_n;      // k programs are stored back to back in one array
  int32_t k2_off, k2_n;
  int32_t k3_off, k3_n;
  int32_t ncols;             // columns (ket Cartesian pairs cd) of this group
  int32_t col_off;           // into colmap
  int32_t o_B;               // start of this group's B region (after its A region)
  int32_t pad;
};

struct ClassKey {
  int la, lb, lc, ld, Kb, Kk, onec;
  int store = 0;   // 1: plan for the store epilogue only (no OUT region when Kb = 1);
                   // 2: solid-harmonic store (k_quartets_sph; see PlanDev::sph)
  bool operator<(const ClassKey& o) const {
    const int a[8] = {la, lb, lc, ld, Kb, Kk, onec, store}, b[8] = {o.la, o.lb, o.lc, o.ld, o.Kb, o.Kk, o.onec, o.store};
    for (int i = 0; i < 8; ++i) if (a[i] != b[i]) return a[i] < b[i];
    return false;
  }
};

// Everything the quartet kernel needs about one class (device-visible POD).
struct PlanDev {
  int32_t la, lb, lc, ld, Kb, Kk, onec;
  int32_t L, Lb, Lk, Nb, Nk, hb;         // hb = Nt(Lb)
  int32_t T, teams_per_cta, team_doubles;
  int32_t recb, reck;                    // record sizes (doubles)
  int32_t o_recb, o_reck, o_scal, o_G, o_R0, o_R1, o_A, o_B, o_X, o_C1, o_OUT;   // o_scal: end of the records
  int32_t c1size;                        // C1 doubles per column
  int32_t ngroups, ncols_max;
  int32_t nb1, nb23;
  int32_t cache_R;                       // 1: R computed once (single primitive quartet); 2: the R tables of all
                                         // primitive quartets kept at o_Rc (rstride doubles each); 3 (solid-
                                         // harmonic plans): those of the current bra primitive; 0: R per group
  int32_t o_Rc, rstride;
  int32_t reg;                           // launch the register kernel (store / digestion launches)
  int32_t has_out;                       // OUT region present (0: store-only plan, b23 writes global memory)
  // Solid-harmonic output (store = 2). The ket groups write their Cartesian columns [p|cd] to a
  // per-team global staging area Xg; two sparse passes (d -> d', then c -> c') form the spherical
  // ket columns [p|c'd'] in shared memory, group by group of ncols_s columns; the bra steps b1/b23
  // run on those columns, and two sparse passes (b -> b', a -> a') write the spherical shellset.
  int32_t sph;
  int32_t nsa, nsb, nsc, nsd;            // 2l + 1 per shell
  int32_t ncols_s;                       // spherical ket columns per bra-pass group
  int32_t o_Xs, o_C1s, o_OUTs, c1s;      // bra-pass layout (C1 stride c1s also holds the [a][b'] pass)
  int32_t hbp;                           // Hermite entries of the bra: length of one staged column
  // 3-center solid-harmonic plans (one-centre bra): a real solid harmonic times a Gaussian expands in the
  // top Hermite shell alone (S_lm(grad) exp(-zeta r^2) = (-2 zeta)^l S_lm(r) exp(-zeta r^2): every
  // lower Hermite term of its Cartesian expansion cancels), so the ket steps form only the rows |p| = l_a
  // and the bra step is OUT[m] = (2 zeta)^-l_a sum_a C_ma [a|cd] over those rows
  int32_t top_only;
  int64_t xg_doubles;                    // staging per team: Xg [Nk][hbp] then Yg [nc_c * nsd][hbp]
  const Group* groups;
  const StepEntry* kprog;
  const StepEntry* b1;
  const B23Entry* b23;
  const uint16_t* colmap;
  const uint16_t* colinv;   // per group g: colinv[g * Nk + ket column] = its column in g, or 0xffff
};

// Host-side plan with its program arrays.
struct Plan {
  PlanDev d{};
  std::vector<Group> groups;
  std::vector<StepEntry> kprog, b1;
  std::vector<B23Entry> b23;
  std::vector<uint16_t> colmap;
  std::vector<uint16_t> colinv;
  double exec_fma = 0;     // FMAs executed per primitive-quartet pass (for reports)
  void* dev_blob = nullptr;
};

// Tunable shape of a plan (0 = the planner's default).
struct PlanConfig {
  int T = 0;                 // threads per team (1..1024, a power of two)
  int budget = 200 * 1024;   // shared-memory bytes per team
  int single_max = 96 * 1024;  // largest workspace for which all ket columns form one group
  int variant = 0;           // 0: register kernel where the class has one, else team; 1: team; 2: register
  int rcache = -1;           // cached R tables of contracted multi-group classes: -1 where they fit without
                             // costing occupancy, 0 never, 1 wherever they fit
  int pack_zpairs = 1;       // small ket z-pairs share column groups (0: one group or more per z-pair)
  bool operator==(const PlanConfig& o) const {
    return T == o.T && budget == o.budget && single_max == o.single_max && variant == o.variant &&
           rcache == o.rcache && pack_zpairs == o.pack_zpairs;
  }
};

// R-level programs (Eq. r) for the team kernel: for every total order N, one
// word per entry (t,u,v) of the [t][u][v] simplex of order N, in layout order:
// bits 0-11 the offset of [t',u',v'] = [tuv] - 1_axis and bits 12-23 the
// offset of [tuv] - 2_axis in the order N-1 layout of the previous level,
// bits 24-25 the axis (0 x, 1 y, 2 z; entry 0 is [000]), bits 26-31 the
// coefficient (index along the axis - 1; 0 where there is no second term).
// off[N] is the first word of order N.
void build_rlevel_programs(std::vector<uint32_t>& prog, std::vector<int32_t>& off);

// Builds the plan of a class for the given shape.
bool build_plan(const ClassKey& key, const PlanConfig& cfg, Plan& plan, std::string& err);

}  // namespace mdx

namespace mdx {
// Real solid harmonics as Cartesian polynomials, rows m = -l..l, columns the
// Cartesian components in library order: tables[l][(m+l)*ncart(l) + k].
std::vector<std::vector<double>> build_solid_tables(int lmax);
// Non-zero coefficients of the real solid harmonics of angular momentum l (over all m).
int solid_nnz(int l);
}  // namespace mdx
