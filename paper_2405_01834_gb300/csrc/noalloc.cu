// mdx_eri4_noalloc: the 4-center evaluation without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: applications that own
// all device memory through their own pool or budget and forbid allocations
// behind their back, and steady-state loops that cannot afford cudaMalloc's
// implicit device synchronisation and latency. For them this entry point
// keeps every piece of device scratch it needs -- the Boys table, the Hermite
// decode table, the primitive-pair records, the quartet index lists and the
// class step programs -- in one file-scope __device__ array of fixed size,
// kScratchBytes. Every GPU that loads the library holds that array until the
// process exits. Inputs and outputs stay caller memory.
//
// The kernels are the ones mdx_eri4 uses (k_pair_records, k_quartets); only
// the place their scratch lives differs.
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/mdx.h"
#include "kernels.cuh"
#include "mdx_internal.h"

// 32 MiB of scratch per device. Host code must not use this name as a device
// address: on the host it is only a stand-in symbol (a kernel given it would
// fault, or silently use the wrong memory where the GPU can reach host
// memory). The device address comes from cudaGetSymbolAddress in setup().
static __device__ __align__(256) unsigned char g_noalloc_scratch[size_t(32) << 20];

namespace mdx {
namespace {

constexpr size_t kScratchBytes = sizeof(g_noalloc_scratch);
constexpr int kMaxDevices = 64;

struct DevState {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_scratch on this device
  double* boys = nullptr;
  uint32_t* rprog = nullptr;
  int32_t* rprog_off = nullptr;
  int* err = nullptr;
  size_t fixed = 0;                // bytes used by the tables above
};

std::mutex g_mu;
DevState g_dev[kMaxDevices];
std::map<ClassKey, std::unique_ptr<Plan>> g_plans;   // host-side plan cache

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Once per device, with that device current: find the array's device address
// and fill the constant tables. Synchronous (runs before any stream work).
mdx_status setup(int dev, DevState& st) {
  if (st.ready) return MDX_OK;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) { cudaGetLastError(); return MDX_ECUDA; }
  if (kernel_attributes_init() != cudaSuccess) { cudaGetLastError(); return MDX_ECUDA; }
  unsigned char* base = (unsigned char*)p;
  const std::vector<double> tab = build_boys_table();
  // R-level programs of the team kernel (Eq. r), one word per Hermite entry
  std::vector<uint32_t> dec;
  std::vector<int32_t> doff;
  build_rlevel_programs(dec, doff);
  size_t o = 0;
  st.err = (int*)(base + o);
  o += 256;
  st.boys = (double*)(base + o);
  o += align256(tab.size() * sizeof(double));
  st.rprog = (uint32_t*)(base + o);
  o += align256(dec.size() * sizeof(uint32_t));
  st.rprog_off = (int32_t*)(base + o);
  o += align256(doff.size() * sizeof(int32_t));
  if (cudaMemcpy(st.boys, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(st.rprog, dec.data(), dec.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(st.rprog_off, doff.data(), doff.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return MDX_ECUDA;
  }
  st.base = base;
  st.fixed = o;
  st.ready = true;
  (void)dev;
  return MDX_OK;
}

struct Region {            // one host array bound for the scratch
  const void* src;
  size_t bytes;
  size_t off;
};

}  // namespace
}  // namespace mdx

using namespace mdx;

extern "C" mdx_status mdx_eri4_noalloc(const mdx_basis* basis, const int32_t* quartets, int64_t n, double* out,
                                       int64_t out_capacity, int64_t* out_offsets, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || !out_offsets || (n > 0 && (!quartets || !out)) || !basis) return MDX_EINVAL;
  if (basis->n_shells < 0 || (basis->n_shells > 0 && (!basis->l || !basis->nprim || !basis->prim_off ||
                                                       !basis->center || !basis->exps || !basis->coefs)))
    return MDX_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) { cudaGetLastError(); return MDX_ECUDA; }
  std::lock_guard<std::mutex> lock(g_mu);
  DevState& st = g_dev[dev];
  mdx_status rc = setup(dev, st);
  if (rc != MDX_OK) return rc;
  if (n == 0) return cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), s) == cudaSuccess ? MDX_OK : MDX_ECUDA;

  // host copies of the shell table and the quartets
  const int32_t ns = basis->n_shells;
  std::vector<int32_t> hl(ns), hk(ns), hq((size_t)n * 4);
  cudaError_t e = cudaSuccess;
  if (ns > 0) {
    e = cudaMemcpyAsync(hl.data(), basis->l, ns * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hk.data(), basis->nprim, ns * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hq.data(), quartets, hq.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return MDX_ECUDA;
  for (int i = 0; i < ns; ++i) {
    if (hl[i] < 0 || hl[i] > MDX_LMAX) return MDX_EUNSUPPORTED;
    if (hk[i] < 1 || hk[i] > MDX_KMAX) return MDX_EUNSUPPORTED;
  }
  // distinct shell pairs, primitive-pair records, class grouping, offsets
  std::unordered_map<int64_t, int32_t> pid;
  std::vector<int2> pairs;
  std::vector<int2> qp(n);
  std::vector<int64_t> offs((size_t)n + 1);
  offs[0] = 0;
  auto pair_index = [&](int32_t i, int32_t j) {
    const int64_t key = (int64_t)i * ns + j;
    auto it = pid.find(key);
    if (it != pid.end()) return it->second;
    const int32_t id = (int32_t)pairs.size();
    pairs.push_back(make_int2(i, j));
    pid.emplace(key, id);
    return id;
  };
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* s4 = &hq[(size_t)q * 4];
    for (int k = 0; k < 4; ++k)
      if (s4[k] < 0 || s4[k] >= ns) return MDX_EINVAL;
    qp[q] = make_int2(pair_index(s4[0], s4[1]), pair_index(s4[2], s4[3]));
    offs[q + 1] = offs[q] + (int64_t)ncart(hl[s4[0]]) * ncart(hl[s4[1]]) * ncart(hl[s4[2]]) * ncart(hl[s4[3]]);
  }
  if (offs[n] > out_capacity) return MDX_ECAPACITY;
  std::vector<int64_t> pair_rec(pairs.size());
  std::vector<PrimPairJob> jobs;
  int64_t roff = 0;
  for (size_t p = 0; p < pairs.size(); ++p) {
    const int i = pairs[p].x, j = pairs[p].y;
    pair_rec[p] = roff;
    for (int ia = 0; ia < hk[i]; ++ia)
      for (int ib = 0; ib < hk[j]; ++ib) {
        jobs.push_back(PrimPairJob{i, j, ia, ib, 0, 0, roff});
        roff += rec_size(hl[i], hl[j]);
      }
  }
  std::map<ClassKey, std::vector<int64_t>> classes;
  for (int64_t q = 0; q < n; ++q) {
    const int2 b = pairs[qp[q].x], k = pairs[qp[q].y];
    classes[ClassKey{hl[b.x], hl[b.y], hl[k.x], hl[k.y], hk[b.x] * hk[b.y], hk[k.x] * hk[k.y], 0, 1}].push_back(q);
  }
  std::vector<int2> qp_sorted;
  std::vector<int64_t> qoff_sorted;
  std::vector<std::pair<Plan*, std::pair<int64_t, int64_t>>> ranges;
  for (auto& kv : classes) {
    auto it = g_plans.find(kv.first);
    if (it == g_plans.end()) {
      std::unique_ptr<Plan> p(new Plan());
      std::string err;
      if (!build_plan(kv.first, PlanConfig{}, *p, err)) return MDX_EUNSUPPORTED;
      it = g_plans.emplace(kv.first, std::move(p)).first;
    }
    const int64_t b = (int64_t)qp_sorted.size();
    for (int64_t q : kv.second) { qp_sorted.push_back(qp[q]); qoff_sorted.push_back(offs[q]); }
    ranges.push_back({it->second.get(), {b, (int64_t)kv.second.size()}});
  }
  // scratch layout after the fixed tables
  std::vector<Region> regs;
  size_t o = st.fixed;
  auto place = [&](const void* src, size_t bytes) {
    regs.push_back(Region{src, bytes, o});
    o += align256(bytes);
    return regs.back().off;
  };
  const size_t o_jobs = place(jobs.data(), jobs.size() * sizeof(PrimPairJob));
  const size_t o_prec = place(pair_rec.data(), pair_rec.size() * sizeof(int64_t));
  const size_t o_qp = place(qp_sorted.data(), qp_sorted.size() * sizeof(int2));
  const size_t o_qoff = place(qoff_sorted.data(), qoff_sorted.size() * sizeof(int64_t));
  const size_t o_recs = place(nullptr, (size_t)roff * sizeof(double));
  const size_t o_recs_s = place(nullptr, (size_t)roff * sizeof(double));
  std::vector<PlanDev> pdev;
  for (auto& r : ranges) {
    Plan& P = *r.first;
    PlanDev d = P.d;
    d.groups = (const Group*)(st.base + place(P.groups.data(), P.groups.size() * sizeof(Group)));
    d.kprog = (const StepEntry*)(st.base + place(P.kprog.data(), P.kprog.size() * sizeof(StepEntry)));
    d.b1 = (const StepEntry*)(st.base + place(P.b1.data(), P.b1.size() * sizeof(StepEntry)));
    d.b23 = (const B23Entry*)(st.base + place(P.b23.data(), P.b23.size() * sizeof(B23Entry)));
    d.colmap = (const uint16_t*)(st.base + place(P.colmap.data(), P.colmap.size() * sizeof(uint16_t)));
    d.colinv = (const uint16_t*)(st.base + place(P.colinv.data(), P.colinv.size() * sizeof(uint16_t)));
    pdev.push_back(d);
  }
  if (o > kScratchBytes) return MDX_ESCRATCH;   // request larger than the fixed scratch

  // From the first copy into the scratch on, every return waits for the
  // stream: work already queued may still read the shared array (and the host
  // vectors it is copied from), and the next call, on any stream, rewrites it
  // as soon as the lock is released.
  auto drained = [s](mdx_status code) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return code;
  };
  for (const Region& r : regs)
    if (r.src && r.bytes) {
      e = cudaMemcpyAsync(st.base + r.off, r.src, r.bytes, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return drained(MDX_ECUDA);
    }
  // the error word is the only scratch that must start at zero; everything
  // else is fully written before it is read
  e = cudaMemsetAsync(st.err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_offsets, offs.data(), offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return drained(MDX_ECUDA);
  const BasisDev bd{basis->l, basis->nprim, basis->prim_off, basis->center, basis->exps, basis->coefs};
  double* recs = (double*)(st.base + o_recs);
  double* recs_s = (double*)(st.base + o_recs_s);
  e = launch_pair_records(bd, bd, (const PrimPairJob*)(st.base + o_jobs), (int64_t)jobs.size(), recs, recs_s,
                          st.err, s);
  if (e != cudaSuccess) return drained(MDX_ECUDA);
  for (size_t c = 0; c < ranges.size(); ++c) {
    QuartetLaunch a{};
    a.plan = pdev[c];
    a.nq = ranges[c].second.second;
    a.qpairs = (const int2*)(st.base + o_qp) + ranges[c].second.first;
    a.qout = (const int64_t*)(st.base + o_qoff) + ranges[c].second.first;
    a.pair_rec = (const int64_t*)(st.base + o_prec);
    a.recs = recs;
    a.recs_signed = recs_s;
    a.boys = st.boys;
    a.rprog = st.rprog;
    a.rprog_off = st.rprog_off;
    a.out = out;
    a.err = st.err;
    e = launch_quartets(a, s);
    if (e != cudaSuccess) return drained(MDX_ECUDA);
  }
  int h = 0;
  e = cudaMemcpyAsync(&h, st.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host arrays above are released on return
  if (e != cudaSuccess) return drained(MDX_ECUDA);
  if (h == kDevTimeout) return MDX_ETIMEOUT;
  if (h != kDevOk) return MDX_EDEVICE;
  return MDX_OK;
}
