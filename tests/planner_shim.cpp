// Host-only test shim: builds the engine's host-side table and program
// generators (csrc/plan.cpp, boys_table.cpp, solid.cpp) with the host
// compiler and hands their output to Python, so that the CPU test suite can
// run the planner's programs in an emulator of the team kernel and check the
// tables against the oracle. Test infrastructure: nothing in the library or the
// benchmark links this file.
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "mdx_internal.h"

namespace {
mdx::Plan g_plan;
std::vector<uint32_t> g_rprog;
std::vector<int32_t> g_roff;

template <typename T>
int64_t copy_out(const std::vector<T>& v, void* dst, int64_t cap) {
  const int64_t bytes = (int64_t)(v.size() * sizeof(T));
  if (dst && cap >= bytes && bytes > 0) std::memcpy(dst, v.data(), (size_t)bytes);
  return bytes;
}
}  // namespace

extern "C" {

// Plan one class (team kernel programs). Returns 0 on success, else 1 with a
// message in err.
int shim_build(int la, int lb, int lc, int ld, int Kb, int Kk, int onec, int store, int T, int budget,
               int single_max, int rcache, int pack, char* err, int errcap) {
  mdx::ClassKey key{la, lb, lc, ld, Kb, Kk, onec, store};
  mdx::PlanConfig cfg;
  cfg.T = T;
  cfg.rcache = rcache;
  cfg.pack_zpairs = pack;
  if (budget > 0) cfg.budget = budget;
  if (single_max > 0) cfg.single_max = single_max;
  cfg.variant = 1;
  g_plan = mdx::Plan();
  std::string e;
  if (!mdx::build_plan(key, cfg, g_plan, e)) {
    if (err && errcap > 0) {
      std::strncpy(err, e.c_str(), (size_t)errcap - 1);
      err[errcap - 1] = 0;
    }
    return 1;
  }
  return 0;
}

// The scalar fields of the last plan, in the order the Python side names them.
int shim_scalars(int32_t* out, int cap) {
  const mdx::PlanDev& P = g_plan.d;
  const int32_t v[] = {P.la, P.lb, P.lc, P.ld, P.Kb, P.Kk, P.onec, P.L, P.Lb, P.Lk, P.Nb, P.Nk, P.hb,
                       P.T, P.teams_per_cta, P.team_doubles, P.recb, P.reck, P.o_recb, P.o_reck, P.o_scal,
                       P.o_G, P.o_R0, P.o_R1, P.o_A, P.o_B, P.o_X, P.o_C1, P.o_OUT, P.c1size, P.ngroups,
                       P.ncols_max, P.nb1, P.nb23, P.cache_R, P.has_out, P.sph, P.nsa, P.nsb, P.nsc, P.nsd,
                       P.ncols_s, P.o_Xs, P.o_C1s, P.o_OUTs, P.c1s, P.hbp, (int32_t)P.xg_doubles, P.o_Rc,
                       P.rstride, P.top_only};
  const int n = (int)(sizeof(v) / sizeof(v[0]));
  if (out && cap >= n) std::memcpy(out, v, sizeof(v));
  return n;
}

// FP64 FMAs per shellset the planner reports for the last plan (the count
// behind the executed-FLOP rates).
double shim_exec_fma() { return g_plan.exec_fma; }

// Raw program arrays of the last plan: 0 groups, 1 ket steps, 2 b1, 3 b23,
// 4 column map. Returns the byte size; copies when cap suffices.
int64_t shim_array(int which, void* dst, int64_t cap) {
  switch (which) {
    case 0: return copy_out(g_plan.groups, dst, cap);
    case 1: return copy_out(g_plan.kprog, dst, cap);
    case 2: return copy_out(g_plan.b1, dst, cap);
    case 3: return copy_out(g_plan.b23, dst, cap);
    case 4: return copy_out(g_plan.colmap, dst, cap);
    default: return -1;
  }
}

// R-level programs: which = 0 the words, 1 the start of each total order.
int64_t shim_rprog(int which, void* dst, int64_t cap) {
  if (g_rprog.empty()) mdx::build_rlevel_programs(g_rprog, g_roff);
  return which == 0 ? copy_out(g_rprog, dst, cap) : copy_out(g_roff, dst, cap);
}

// The device's Boys interpolation table ([grid point][m][k], F_{m+k}(T0)/k!)
// and its shape: dims = {grid points, orders, terms}, inv_h = 1/h.
int64_t shim_boys(double* dst, int64_t cap, int32_t* dims, double* inv_h) {
  const std::vector<double> t = mdx::build_boys_table();
  dims[0] = mdx::kBoysNgrid;
  dims[1] = mdx::kBoysOrders;
  dims[2] = mdx::kBoysTerms;
  *inv_h = mdx::kBoysInvH;
  return copy_out(t, dst, cap * (int64_t)sizeof(double)) / (int64_t)sizeof(double);
}

// The library's real-solid-harmonic table of one l: [2l+1][ncart(l)].
int64_t shim_solid(int l, double* dst, int64_t cap) {
  const std::vector<std::vector<double>> t = mdx::build_solid_tables(mdx::kLmax);
  if (l < 0 || l > mdx::kLmax) return -1;
  return copy_out(t[(size_t)l], dst, cap * (int64_t)sizeof(double)) / (int64_t)sizeof(double);
}

int shim_sizes(int32_t* out) {
  out[0] = (int32_t)sizeof(mdx::StepEntry);
  out[1] = (int32_t)sizeof(mdx::B23Entry);
  out[2] = (int32_t)sizeof(mdx::Group);
  out[3] = mdx::kRecHeader;
  return 0;
}

}  // extern "C"
