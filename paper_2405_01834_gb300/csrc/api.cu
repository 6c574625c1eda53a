// Host side of the C ABI declared in include/mdx.h: context, argument
// validation, class grouping, workspace, and the kernel launches.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include <cublas_v2.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/mdx.h"
#include "kernels.cuh"
#include "mdx_internal.h"

using namespace mdx;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace

// NVTX range around each entry point that enqueues GPU work, so that
// profilers can select an entry point's kernels (no effect without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct mdx_ctx {
  int device = 0;
  std::string last_error;
  double* d_boys = nullptr;
  uint32_t* d_rprog = nullptr;
  int32_t* d_rprog_off = nullptr;
  int* d_err = nullptr;
  std::map<ClassKey, std::unique_ptr<Plan>> plans;
  std::map<std::string, DevBuf> bufs;
  std::map<ClassKey, PlanConfig> tuned;   // shapes chosen by mdx_batch_autotune
  std::vector<std::unique_ptr<Plan>> retired;   // replaced plans, kept alive for batches that use them
  int64_t last_quartets = 0;
  cublasHandle_t cublas = nullptr;        // materialized-Hermite path only, created on first use
  // auxiliary streams for independent per-class launches (created on first use)
  static constexpr int kAux = 3;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kAux] = {};
};

namespace {

mdx_status fail(mdx_ctx* c, mdx_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

mdx_status cuda_fail(mdx_ctx* c, cudaError_t e, const char* where) {
  return fail(c, MDX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device buffer that grows on demand. Growing synchronises the stream first
// so that no queued kernel still reads the old allocation.
template <typename T>
mdx_status ensure(mdx_ctx* c, const char* name, size_t count, T** out, cudaStream_t s) {
  DevBuf& b = c->bufs[name];
  const size_t bytes = std::max<size_t>(count * sizeof(T), 256);
  if (b.cap < bytes) {
    if (b.p) {
      cudaStreamSynchronize(s);
      cudaFree(b.p);
      b.p = nullptr;
      b.cap = 0;
    }
    size_t want = bytes + bytes / 4;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, MDX_ENOMEM, std::string("workspace allocation failed for ") + name);
    }
    b.cap = want;
  }
  *out = (T*)b.p;
  return MDX_OK;
}

template <typename T>
mdx_status upload(mdx_ctx* c, const char* name, const std::vector<T>& v, T** out, cudaStream_t s) {
  mdx_status st = ensure<T>(c, name, v.size(), out, s);
  if (st != MDX_OK) return st;
  if (!v.empty()) {
    cudaError_t e = cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload");
  }
  return MDX_OK;
}

// Copy a plan's programs to one device blob and point its PlanDev at it.
mdx_status upload_plan(mdx_ctx* c, Plan* p, cudaStream_t s) {
  const size_t sg = p->groups.size() * sizeof(Group), sk = p->kprog.size() * sizeof(StepEntry),
               s1 = p->b1.size() * sizeof(StepEntry), s2 = p->b23.size() * sizeof(B23Entry),
               sc = p->colmap.size() * sizeof(uint16_t), si = p->colinv.size() * sizeof(uint16_t);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t tot = al(sg) + al(sk) + al(s1) + al(s2) + al(sc) + al(si);
  std::vector<char> blob(tot, 0);
  size_t o = 0;
  auto put = [&](const void* src, size_t n) { size_t at = o; if (n) memcpy(blob.data() + o, src, n); o += al(n); return at; };
  const size_t og = put(p->groups.data(), sg), ok = put(p->kprog.data(), sk), o1 = put(p->b1.data(), s1),
               o2 = put(p->b23.data(), s2), oc = put(p->colmap.data(), sc), oi = put(p->colinv.data(), si);
  cudaError_t e = cudaMalloc(&p->dev_blob, tot);
  if (e != cudaSuccess) { cudaGetLastError(); p->dev_blob = nullptr; return fail(c, MDX_ENOMEM, "plan allocation failed"); }
  e = cudaMemcpyAsync(p->dev_blob, blob.data(), tot, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // blob is a local vector
  if (e != cudaSuccess) return cuda_fail(c, e, "plan upload");
  char* base = (char*)p->dev_blob;
  p->d.groups = (const Group*)(base + og);
  p->d.kprog = (const StepEntry*)(base + ok);
  p->d.b1 = (const StepEntry*)(base + o1);
  p->d.b23 = (const B23Entry*)(base + o2);
  p->d.colmap = (const uint16_t*)(base + oc);
  p->d.colinv = (const uint16_t*)(base + oi);
  return MDX_OK;
}

mdx_status get_plan(mdx_ctx* c, const ClassKey& k, Plan** out, cudaStream_t s) {
  auto it = c->plans.find(k);
  if (it != c->plans.end()) { *out = it->second.get(); return MDX_OK; }
  std::unique_ptr<Plan> p(new Plan());
  std::string err;
  auto tc = c->tuned.find(k);
  const PlanConfig cfg = tc != c->tuned.end() ? tc->second : PlanConfig{};
  if (!build_plan(k, cfg, *p, err)) return fail(c, MDX_EUNSUPPORTED, "planner: " + err);
  mdx_status st = upload_plan(c, p.get(), s);
  if (st != MDX_OK) { if (p->dev_blob) cudaFree(p->dev_blob); return st; }
  *out = p.get();
  c->plans[k] = std::move(p);
  return MDX_OK;
}

mdx_status check_device_error(mdx_ctx* c, cudaStream_t s) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "device error check");
  if (h != kDevOk) {
    cudaMemsetAsync(c->d_err, 0, sizeof(int), s);
    if (h == kDevTimeout) return fail(c, MDX_ETIMEOUT, "a bounded device-side wait expired");
    return fail(c, MDX_EDEVICE, "a kernel flagged invalid input");
  }
  return MDX_OK;
}

struct HostBasis {
  std::vector<int32_t> l, nprim;
  int32_t n = 0;
};

mdx_status fetch_basis(mdx_ctx* c, const mdx_basis* b, HostBasis& hb, cudaStream_t s) {
  if (!b || b->n_shells < 0 || (b->n_shells > 0 && (!b->l || !b->nprim || !b->prim_off || !b->center ||
                                                     !b->exps || !b->coefs)))
    return fail(c, MDX_EINVAL, "invalid basis descriptor");
  hb.n = b->n_shells;
  hb.l.resize(hb.n);
  hb.nprim.resize(hb.n);
  if (hb.n) {
    cudaError_t e = cudaMemcpyAsync(hb.l.data(), b->l, hb.n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.nprim.data(), b->nprim, hb.n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "basis download");
  }
  for (int i = 0; i < hb.n; ++i) {
    if (hb.l[i] < 0 || hb.l[i] > MDX_LMAX) return fail(c, MDX_EUNSUPPORTED, "shell angular momentum outside 0..MDX_LMAX");
    if (hb.nprim[i] < 1 || hb.nprim[i] > MDX_KMAX) return fail(c, MDX_EUNSUPPORTED, "contraction degree outside 1..MDX_KMAX");
  }
  return MDX_OK;
}

BasisDev to_dev(const mdx_basis* b) {
  return BasisDev{b->l, b->nprim, b->prim_off, b->center, b->exps, b->coefs};
}

// A shell pair (i, j) of basis `which`; j = -1 is the one-centre unit partner.
struct PairKey {
  int32_t i, j, which;
  bool operator==(const PairKey& o) const { return i == o.i && j == o.j && which == o.which; }
};
struct PairHash {
  size_t operator()(const PairKey& k) const {
    return std::hash<int64_t>()(((int64_t)k.i << 32) ^ ((int64_t)(k.j + 1) << 1) ^ k.which);
  }
};

// Quartets given as (bra pair, ket pair) over a pair list.
struct Batch {
  std::vector<PairKey> pairs;
  std::vector<int2> qp;          // per evaluated quartet (bra pair idx, ket pair idx)
  std::vector<int64_t> qoff;     // output offset per evaluated quartet
  std::vector<int64_t> qcaller;  // caller index per evaluated quartet
  std::vector<int64_t> zero;     // (offset, doubles) of every screened-out quartet, written as zeros
};

}  // namespace

// A prepared batch: everything on the device, ready to launch.
struct mdx_batch {
  mdx_ctx* ctx = nullptr;
  int64_t n = 0;                  // quartets
  int64_t total = 0;              // output doubles
  BasisDev b0{}, b1{};
  PrimPairJob* jobs = nullptr;
  int64_t njobs = 0;
  int64_t* pair_rec = nullptr;
  double* recs = nullptr;
  double* recs_s = nullptr;
  int2* qp = nullptr;
  int64_t* qoff = nullptr;
  int64_t* offsets = nullptr;     // [n+1] in caller order
  int64_t* zero = nullptr;        // [nzero][2] (offset, doubles) of screened-out shellsets
  int64_t nzero = 0;
  // solid-harmonic batches: offsets, total and qoff count solid-harmonic doubles. Classes without a
  // register kernel run the solid-harmonic team kernel (splan, `grid` CTAs, staging in xg); the
  // others evaluate Cartesian shellsets into `cart` (offsets cqoff) and transform them element by
  // element.
  bool sph = false;
  int64_t* cqoff = nullptr;
  double* cart = nullptr;
  double* xg = nullptr;
  int64_t nxg = 0;                // doubles allocated at xg
  struct Range { Plan* plan; int64_t begin, count; ClassKey key; Plan* splan; int grid; };
  std::vector<Range> ranges;
  std::vector<int64_t> qorig;     // caller index of each class-sorted quartet
  double model_flops = 0.0;
  double exec_fma = 0.0;
  bool owned = true;              // device arrays belong to the batch (else: context workspace of one call)
};

// Several molecules' exchange builds prepared together (one super basis, one
// screened quartet list per class bucket across molecules).
struct mdx_xbatch {
  mdx_ctx* ctx = nullptr;
  int32_t nmol = 0;
  int64_t max_nao = 0, nq = 0, nitems = 0, smem = 0;
  int64_t nitems_team = 0, smem_team = 0;   // the queue without the register-kernel classes
  int grid = 0, grid_team = 0;
  double model_flops = 0.0;
  mdx_basis sb{};
  int32_t *l = nullptr, *nprim = nullptr, *prim_off = nullptr, *ao_off = nullptr;
  double *center = nullptr, *exps = nullptr, *coefs = nullptr;
  const double** molD = nullptr;
  double** molK = nullptr;
  int32_t* molnao = nullptr;
  int2* pshell = nullptr;
  int32_t* pmol = nullptr;
  int64_t* prec = nullptr;
  double *recs = nullptr, *recs_s = nullptr;
  int2* quart = nullptr;
  std::vector<QuartetLaunch> launches, plaunches;
  std::vector<ClassKey> lkey;          // class of each per-class launch
  std::vector<double> lflops;          // its Table-1 model FLOPs
  std::vector<int32_t> reg_launches;   // per-class launches that run a register kernel
  QuartetLaunch* d_plaunches = nullptr;
  WorkItem* items = nullptr;
  WorkItem* items_team = nullptr;
  unsigned long long* counter = nullptr;
};

namespace {

void xbatch_free(mdx_xbatch* x) {
  if (!x) return;
  cudaFree(x->l); cudaFree(x->nprim); cudaFree(x->prim_off); cudaFree(x->ao_off);
  cudaFree(x->center); cudaFree(x->exps); cudaFree(x->coefs);
  cudaFree(x->molD); cudaFree(x->molK); cudaFree(x->molnao);
  cudaFree(x->pshell); cudaFree(x->pmol); cudaFree(x->prec); cudaFree(x->recs); cudaFree(x->recs_s);
  cudaFree(x->quart); cudaFree(x->d_plaunches); cudaFree(x->items); cudaFree(x->items_team);
  cudaFree(x->counter);
  delete x;
}

void batch_free(mdx_batch* b) {
  if (!b) return;
  if (b->owned) {
    cudaFree(b->jobs); cudaFree(b->pair_rec); cudaFree(b->recs); cudaFree(b->recs_s);
    cudaFree(b->qp); cudaFree(b->qoff); cudaFree(b->offsets); cudaFree(b->zero);
    cudaFree(b->cqoff); cudaFree(b->cart); cudaFree(b->xg);
  }
  delete b;
}

template <typename T>
mdx_status dev_upload(mdx_ctx* c, const std::vector<T>& v, T** out, cudaStream_t s) {
  *out = nullptr;
  if (v.empty()) return MDX_OK;
  if (cudaMalloc((void**)out, v.size() * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MDX_ENOMEM, "batch allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch upload");
  return MDX_OK;
}

// Independent launches (one per class, each summing into K or the gradient
// with atomics) spread over the caller's stream and the context's auxiliary
// streams, so that launches too small to fill the GPU overlap. fork() makes
// every auxiliary stream wait for the work enqueued on the caller's stream so
// far (plan uploads included); pick() takes the stream with the least work
// assigned; join() makes the caller's stream wait for all of them.
struct Fanout {
  mdx_ctx* c;
  cudaStream_t s;
  double load[mdx_ctx::kAux + 1] = {};
  cudaStream_t stream(int i) const { return i == 0 ? s : c->aux[i - 1]; }
  cudaError_t fork() {
    if (!c->ev_fork) {
      for (int i = 0; i < mdx_ctx::kAux; ++i) {
        cudaError_t e = c->aux[i] ? cudaSuccess : cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking);
        if (e == cudaSuccess && !c->ev_join[i]) e = cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
      }
      const cudaError_t e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaEventRecord(c->ev_fork, s);
    for (int i = 0; i < mdx_ctx::kAux && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->aux[i], c->ev_fork, 0);
    return e;
  }
  int pick(double work) {
    int best = 0;
    for (int i = 1; i <= mdx_ctx::kAux; ++i)
      if (load[i] < load[best]) best = i;
    load[best] += work;
    return best;
  }
  cudaError_t join() {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < mdx_ctx::kAux && e == cudaSuccess; ++i) {
      e = cudaEventRecord(c->ev_join[i], c->aux[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join[i], 0);
    }
    return e;
  }
};

// The paper's Table 1 work model of one contracted shellset; sph: with the
// solid-harmonic component counts 2l+1 (the paper's own basis), else Cartesian.
double model_flops_class(const ClassKey& k, bool sph = false) {
  auto nh = [](int l) { return (double)nherm(l); };
  auto rl = [](int L) { return (2.0 + L) * (7.0 + L) * (12.0 + 5.0 * L + (double)L * L) / 8.0; };
  auto nf = [sph](int l) { return sph ? 2.0 * l + 1.0 : (double)ncart(l); };
  const int Lb = k.la + k.lb, Lk = k.lc + k.ld;
  const double Nb = nf(k.la) * nf(k.lb), Nk = nf(k.lc) * nf(k.ld);
  return k.Kb * (double)k.Kk * (rl(Lb + Lk) + nh(Lb) * nh(Lk) / 2 + 2 * nh(Lb) * nh(Lk) * Nk) +
         k.Kb * 2.0 * Nb * nh(Lb) * Nk;
}

// FP64 multiply-adds of k_cart2sph on one shellset (every product of non-zero coefficients once).
double cart2sph_fma(const ClassKey& k) {
  return (double)solid_nnz(k.la) * solid_nnz(k.lb) * solid_nnz(k.lc) * solid_nnz(k.ld);
}

// Host preparation of a batch: primitive-pair jobs, class grouping, plans,
// uploads. Synchronises `s` before returning (host vectors go out of scope).
// call_ws: the device arrays live in context workspace (one-shot calls: no
// cudaMalloc / cudaFree, whose implicit device-wide synchronisation would
// stall other streams; consecutive calls on one stream reuse it in order).
mdx_status batch_prepare(mdx_ctx* c, const mdx_basis* b0, const mdx_basis* b1, const HostBasis& h0,
                         const HostBasis& h1, const Batch& bt, const std::vector<int64_t>& offs, mdx_batch** out,
                         cudaStream_t s, bool call_ws = false, bool sph = false) {
  std::unique_ptr<mdx_batch, void (*)(mdx_batch*)> B(new mdx_batch(), batch_free);
  if (sph && call_ws) return fail(c, MDX_EINVAL, "solid-harmonic batches own their arrays");
  B->owned = !call_ws;
  B->sph = sph;
  B->ctx = c;
  B->n = (int64_t)offs.size() - 1;
  B->total = offs.back();
  B->nzero = (int64_t)bt.zero.size() / 2;
  B->b0 = to_dev(b0);
  B->b1 = to_dev(b1 ? b1 : b0);
  const HostBasis* hb[2] = {&h0, &h1};
  std::vector<int64_t> pair_rec(bt.pairs.size());
  std::vector<PrimPairJob> jobs;
  int64_t roff = 0;
  for (size_t p = 0; p < bt.pairs.size(); ++p) {
    const PairKey& k = bt.pairs[p];
    const HostBasis& H = *hb[k.which];
    const int li = H.l[k.i], lj = k.j >= 0 ? H.l[k.j] : 0;
    const int Ki = H.nprim[k.i], Kj = k.j >= 0 ? H.nprim[k.j] : 1;
    const int rs = rec_size(li, lj);
    pair_rec[p] = roff;
    for (int ia = 0; ia < Ki; ++ia)
      for (int ib = 0; ib < Kj; ++ib) {
        jobs.push_back(PrimPairJob{k.i, k.j, ia, ib, k.which, 0, roff});
        roff += rs;
      }
  }
  std::map<ClassKey, std::vector<int64_t>> classes;
  for (size_t q = 0; q < bt.qp.size(); ++q) {
    const PairKey& bp = bt.pairs[bt.qp[q].x];
    const PairKey& kp = bt.pairs[bt.qp[q].y];
    const HostBasis& HB = *hb[bp.which];
    const HostBasis& HK = *hb[kp.which];
    ClassKey key{HB.l[bp.i], bp.j >= 0 ? HB.l[bp.j] : 0, HK.l[kp.i], HK.l[kp.j],
                 HB.nprim[bp.i] * (bp.j >= 0 ? HB.nprim[bp.j] : 1), HK.nprim[kp.i] * HK.nprim[kp.j],
                 bp.j < 0 ? 1 : 0};
    key.store = 1;   // batches only store shellsets
    classes[key].push_back((int64_t)q);
  }
  std::vector<int2> qp_sorted;
  std::vector<int64_t> qoff_sorted, cqoff;
  qp_sorted.reserve(bt.qp.size());
  qoff_sorted.reserve(bt.qp.size());
  int64_t cart_total = 0, xg_total = 0;
  mdx_status st;
  for (auto& kv : classes) {
    const int64_t b = (int64_t)qp_sorted.size();
    for (int64_t q : kv.second) {
      qp_sorted.push_back(bt.qp[q]);
      qoff_sorted.push_back(bt.qoff[q]);
      B->qorig.push_back(bt.qcaller.empty() ? q : bt.qcaller[q]);
    }
    const int64_t cnt = (int64_t)kv.second.size();
    Plan* plan;
    if ((st = get_plan(c, kv.first, &plan, s)) != MDX_OK) return st;
    Plan* splan = nullptr;
    int grid = 0;
    double fma = plan->exec_fma;
    ClassKey ks = kv.first;
    ks.store = 2;
    // the solid-harmonic team kernel: every class without a register kernel, and those the autotuner moved
    if (sph && (!plan->d.reg || c->tuned.count(ks))) {
      const ClassKey& k2 = ks;
      if ((st = get_plan(c, k2, &splan, s)) != MDX_OK) return st;
      cudaError_t e = sph_grid(splan->d, cnt, &grid);
      if (e != cudaSuccess) return cuda_fail(c, e, "solid-harmonic launch shape");
      xg_total = std::max<int64_t>(xg_total, (int64_t)grid * splan->d.teams_per_cta * splan->d.xg_doubles);
      fma = splan->exec_fma;
    }
    if (sph) {
      cqoff.resize(qp_sorted.size(), 0);
      if (!splan) {
        const ClassKey& k = kv.first;
        const int64_t nct = (int64_t)ncart(k.la) * ncart(k.lb) * ncart(k.lc) * ncart(k.ld);
        for (int64_t i = b; i < b + cnt; ++i) {
          cqoff[i] = cart_total;
          cart_total += nct;
        }
        fma += cart2sph_fma(k);
      }
    }
    B->ranges.push_back({plan, b, cnt, kv.first, splan, grid});
    B->model_flops += model_flops_class(kv.first, sph) * (double)cnt;
    B->exec_fma += fma * (double)cnt;
  }
  B->njobs = (int64_t)jobs.size();
  if (call_ws) {
    if ((st = upload(c, "call_jobs", jobs, &B->jobs, s)) != MDX_OK) return st;
    if ((st = upload(c, "call_pair_rec", pair_rec, &B->pair_rec, s)) != MDX_OK) return st;
    if ((st = upload(c, "call_qp", qp_sorted, &B->qp, s)) != MDX_OK) return st;
    if ((st = upload(c, "call_qoff", qoff_sorted, &B->qoff, s)) != MDX_OK) return st;
    if ((st = upload(c, "call_offsets", offs, &B->offsets, s)) != MDX_OK) return st;
    if (!bt.zero.empty() && (st = upload(c, "call_zero", bt.zero, &B->zero, s)) != MDX_OK) return st;
    if ((st = ensure(c, "call_recs", (size_t)std::max<int64_t>(roff, 1), &B->recs, s)) != MDX_OK) return st;
    if ((st = ensure(c, "call_recs_s", (size_t)std::max<int64_t>(roff, 1), &B->recs_s, s)) != MDX_OK) return st;
  } else {
  if ((st = dev_upload(c, jobs, &B->jobs, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, pair_rec, &B->pair_rec, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, qp_sorted, &B->qp, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, qoff_sorted, &B->qoff, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, offs, &B->offsets, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, bt.zero, &B->zero, s)) != MDX_OK) return st;
  }
  if (roff > 0 && !call_ws) {
    if (cudaMalloc(&B->recs, roff * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&B->recs_s, roff * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, MDX_ENOMEM, "record allocation failed");
    }
  }
  if (sph) {
    if ((st = dev_upload(c, cqoff, &B->cqoff, s)) != MDX_OK) return st;
    if ((cart_total > 0 && cudaMalloc(&B->cart, cart_total * sizeof(double)) != cudaSuccess) ||
        (xg_total > 0 && (B->nxg = xg_total, cudaMalloc(&B->xg, xg_total * sizeof(double)) != cudaSuccess))) {
      cudaGetLastError();
      return fail(c, MDX_ENOMEM, "solid-harmonic scratch allocation failed");
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch upload");
  *out = B.release();
  return MDX_OK;
}

// Enqueue the whole hot path of a batch: pair records, then one quartet
// kernel per class. No host synchronisation, no allocation.
mdx_status batch_run(mdx_ctx* c, mdx_batch* B, double* out, int32_t* nlaunch, cudaStream_t s) {
  int32_t nl = 0;
  cudaError_t e = launch_pair_records(B->b0, B->b1, B->jobs, B->njobs, B->recs, B->recs_s, c->d_err, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair records");
  if (B->njobs > 0) ++nl;
  if (B->nzero > 0) {
    e = launch_zero_ranges(B->zero, B->nzero, out, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "screened-out shellsets");
    ++nl;
  }
  for (auto& r : B->ranges) {
    QuartetLaunch a{};
    a.plan = r.plan->d;
    a.nq = r.count;
    a.qpairs = B->qp + r.begin;
    a.qout = B->qoff + r.begin;
    a.pair_rec = B->pair_rec;
    a.recs = B->recs;
    a.recs_signed = B->recs_s;
    a.boys = c->d_boys;
    a.rprog = c->d_rprog;
    a.rprog_off = c->d_rprog_off;
    a.out = out;
    a.err = c->d_err;
    if (B->sph && r.splan) {   // solid harmonics folded into the transforms
      a.plan = r.splan->d;
      a.sph_scratch = B->xg;
      e = launch_quartets_sph(a, r.grid, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "solid-harmonic quartet kernel launch");
      if (r.count > 0) ++nl;
      continue;
    }
    if (B->sph) {              // Cartesian shellsets, then the index-by-index transform
      a.qout = B->cqoff + r.begin;
      a.out = B->cart;
    }
    e = launch_quartets(a, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "quartet kernel launch");
    if (r.count > 0) ++nl;
    if (B->sph) {
      SphLaunch t{r.key.la, r.key.lb, r.key.lc, r.key.ld, r.count, B->cart, B->cqoff + r.begin, out,
                  B->qoff + r.begin};
      e = launch_cart2sph(t, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "solid-harmonic transform");
      if (r.count > 0) ++nl;
    }
  }
  if (nlaunch) *nlaunch = nl;
  return MDX_OK;
}

mdx_status read_quartets(mdx_ctx* c, const int32_t* dev, int64_t n, int w, std::vector<int32_t>& h, cudaStream_t s) {
  h.resize((size_t)n * w);
  cudaError_t e = cudaMemcpyAsync(h.data(), dev, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "index download");
  return MDX_OK;
}

struct PairIndex {
  Batch& bt;
  std::unordered_map<PairKey, int32_t, PairHash> pid;
  explicit PairIndex(Batch& b) : bt(b) {}
  int32_t operator()(int32_t i, int32_t j, int32_t which) {
    PairKey k{i, j, which};
    auto it = pid.find(k);
    if (it != pid.end()) return it->second;
    const int32_t id = (int32_t)bt.pairs.size();
    bt.pairs.push_back(k);
    pid.emplace(k, id);
    return id;
  }
};

// Per-quartet screening bounds (NULL: none) downloaded to the host; a quartet
// with bound < tau is not evaluated (its shellset is written as zeros).
mdx_status read_bounds(mdx_ctx* c, const double* bound, int64_t n, std::vector<double>& h, cudaStream_t s) {
  h.clear();
  if (!bound) return MDX_OK;
  h.resize((size_t)n);
  cudaError_t e = cudaMemcpyAsync(h.data(), bound, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "bound download");
  return MDX_OK;
}

// Adds quartet q (output offs[q], `size` doubles) to the batch, or to its
// zero-filled list when its bound is below tau.
void batch_add(Batch& bt, int64_t q, int2 qp, int64_t off, int64_t size, const std::vector<double>& hbound,
               double tau) {
  if (!hbound.empty() && hbound[(size_t)q] < tau) {
    bt.zero.push_back(off);
    bt.zero.push_back(size);
    return;
  }
  bt.qp.push_back(qp);
  bt.qoff.push_back(off);
  bt.qcaller.push_back(q);
}

mdx_status make_batch4(mdx_ctx* c, const mdx_basis* basis, const int32_t* quartets, int64_t n, mdx_batch** out,
                       cudaStream_t s, bool call_ws = false, const double* bound = nullptr, double tau = 0.0,
                       bool sph = false) {
  HostBasis hb;
  mdx_status st = fetch_basis(c, basis, hb, s);
  if (st != MDX_OK) return st;
  std::vector<int32_t> hq;
  if ((st = read_quartets(c, quartets, n, 4, hq, s)) != MDX_OK) return st;
  std::vector<double> hbound;
  if ((st = read_bounds(c, bound, n, hbound, s)) != MDX_OK) return st;
  Batch bt;
  PairIndex pix(bt);
  std::vector<int64_t> offs((size_t)n + 1);
  offs[0] = 0;
  bt.qp.reserve(n);
  bt.qoff.reserve(n);
  bt.qcaller.reserve(n);
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* s4 = &hq[(size_t)q * 4];
    for (int k = 0; k < 4; ++k)
      if (s4[k] < 0 || s4[k] >= hb.n) return fail(c, MDX_EINVAL, "shell index out of range");
    auto nf = [&](int sh) { return (int64_t)(sph ? 2 * hb.l[sh] + 1 : ncart(hb.l[sh])); };
    const int64_t size = nf(s4[0]) * nf(s4[1]) * nf(s4[2]) * nf(s4[3]);
    offs[q + 1] = offs[q] + size;
    const int2 qp = hbound.empty() || hbound[(size_t)q] >= tau
                        ? make_int2(pix(s4[0], s4[1], 0), pix(s4[2], s4[3], 0)) : make_int2(0, 0);
    batch_add(bt, q, qp, offs[q], size, hbound, tau);
  }
  return batch_prepare(c, basis, nullptr, hb, hb, bt, offs, out, s, call_ws, sph);
}

mdx_status make_batch3(mdx_ctx* c, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets, int64_t n,
                       mdx_batch** out, cudaStream_t s, bool call_ws = false, const double* bound = nullptr,
                       double tau = 0.0, bool sph = false) {
  HostBasis ha, ho;
  mdx_status st = fetch_basis(c, aux, ha, s);
  if (st != MDX_OK) return st;
  if ((st = fetch_basis(c, orb, ho, s)) != MDX_OK) return st;
  std::vector<int32_t> ht;
  if ((st = read_quartets(c, triplets, n, 3, ht, s)) != MDX_OK) return st;
  std::vector<double> hbound;
  if ((st = read_bounds(c, bound, n, hbound, s)) != MDX_OK) return st;
  Batch bt;
  PairIndex pix(bt);
  std::vector<int64_t> offs((size_t)n + 1);
  offs[0] = 0;
  bt.qp.reserve(n);
  bt.qoff.reserve(n);
  bt.qcaller.reserve(n);
  for (int64_t q = 0; q < n; ++q) {
    const int32_t* t3 = &ht[(size_t)q * 3];
    if (t3[0] < 0 || t3[0] >= ha.n || t3[1] < 0 || t3[1] >= ho.n || t3[2] < 0 || t3[2] >= ho.n)
      return fail(c, MDX_EINVAL, "shell index out of range");
    auto nf = [sph](int l) { return (int64_t)(sph ? 2 * l + 1 : ncart(l)); };
    const int64_t size = nf(ha.l[t3[0]]) * nf(ho.l[t3[1]]) * nf(ho.l[t3[2]]);
    offs[q + 1] = offs[q] + size;
    const int2 qp = hbound.empty() || hbound[(size_t)q] >= tau
                        ? make_int2(pix(t3[0], -1, 0), pix(t3[1], t3[2], 1)) : make_int2(0, 0);
    batch_add(bt, q, qp, offs[q], size, hbound, tau);
  }
  return batch_prepare(c, aux, orb, ha, ho, bt, offs, out, s, call_ws, sph);
}

// create, run into `out`, copy offsets, destroy (synchronous)
// One-shot evaluation of a batch built in context workspace: reports errors
// that earlier kernels recorded, enqueues the work and returns without
// waiting for it (its own kernel errors surface at the next call or mdx_sync).
mdx_status run_once(mdx_ctx* c, mdx_batch* B, double* out, int64_t cap, int64_t* out_offsets, cudaStream_t s) {
  std::unique_ptr<mdx_batch, void (*)(mdx_batch*)> guard(B, batch_free);
  if (B->total > cap) return fail(c, MDX_ECAPACITY, "output capacity too small");
  mdx_status st = check_device_error(c, s);
  if (st != MDX_OK) return st;
  cudaError_t e = cudaMemcpyAsync(out_offsets, B->offsets, (B->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "offsets");
  return batch_run(c, B, out, nullptr, s);
}

}  // namespace

extern "C" {

mdx_status mdx_create(mdx_ctx** ctx, int device) {
  if (!ctx) return MDX_EINVAL;
  *ctx = nullptr;
  std::unique_ptr<mdx_ctx> c(new mdx_ctx());
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return MDX_ECUDA;
  e = kernel_attributes_init();
  if (e != cudaSuccess) return MDX_ECUDA;
  std::vector<double> tab = build_boys_table();
  if (cudaMalloc(&c->d_boys, tab.size() * sizeof(double)) != cudaSuccess) return MDX_ENOMEM;
  if (cudaMemcpy(c->d_boys, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return MDX_ECUDA;
  // R-level programs of the team kernel (Eq. r), one word per Hermite entry
  std::vector<uint32_t> dec;
  std::vector<int32_t> doff;
  build_rlevel_programs(dec, doff);
  if (cudaMalloc(&c->d_rprog, dec.size() * sizeof(uint32_t)) != cudaSuccess) return MDX_ENOMEM;
  if (cudaMalloc(&c->d_rprog_off, doff.size() * sizeof(int32_t)) != cudaSuccess) return MDX_ENOMEM;
  if (cudaMemcpy(c->d_rprog, dec.data(), dec.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_rprog_off, doff.data(), doff.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return MDX_ECUDA;
  if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess) return MDX_ENOMEM;
  if (cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) return MDX_ECUDA;
  *ctx = c.release();
  return MDX_OK;
}

void mdx_destroy(mdx_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  for (auto& kv : c->plans) if (kv.second->dev_blob) cudaFree(kv.second->dev_blob);
  for (auto& p : c->retired) if (p->dev_blob) cudaFree(p->dev_blob);
  for (auto& kv : c->bufs) if (kv.second.p) cudaFree(kv.second.p);
  cudaFree(c->d_boys);
  cudaFree(c->d_rprog);
  cudaFree(c->d_rprog_off);
  cudaFree(c->d_err);
  if (c->cublas) cublasDestroy(c->cublas);
  for (int i = 0; i < mdx_ctx::kAux; ++i) {
    if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
    if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
}

const char* mdx_last_error(const mdx_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

mdx_status mdx_sync(mdx_ctx* c, void* stream) {
  if (!c) return MDX_EINVAL;
  cudaSetDevice(c->device);
  return check_device_error(c, (cudaStream_t)stream);
}

mdx_status mdx_eri4(mdx_ctx* c, const mdx_basis* basis, const int32_t* quartets, const double* bound, int64_t n,
                    double tau, double* out, int64_t out_capacity, int64_t* out_offsets, void* stream) {
  const NvtxRange nvtx_range("mdx_eri4");
  if (!c) return MDX_EINVAL;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || !out_offsets || (n > 0 && (!quartets || !out))) return fail(c, MDX_EINVAL, "invalid arguments");
  if (bound && !(tau >= 0.0)) return fail(c, MDX_EINVAL, "tau must be >= 0");
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), s);
    return e == cudaSuccess ? MDX_OK : cuda_fail(c, e, "offsets");
  }
  mdx_batch* B = nullptr;
  mdx_status st = make_batch4(c, basis, quartets, n, &B, s, true, bound, tau);
  if (st != MDX_OK) return st;
  return run_once(c, B, out, out_capacity, out_offsets, s);
}

mdx_status mdx_eri4_sph(mdx_ctx* c, const mdx_basis* basis, const int32_t* quartets, int64_t n, double* out,
                        int64_t out_capacity, int64_t* out_offsets, void* stream) {
  const NvtxRange nvtx_range("mdx_eri4_sph");
  if (!c) return MDX_EINVAL;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || !out_offsets || (n > 0 && (!quartets || !out))) return fail(c, MDX_EINVAL, "invalid arguments");
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), s);
    return e == cudaSuccess ? MDX_OK : cuda_fail(c, e, "offsets");
  }
  mdx_batch* B = nullptr;
  mdx_status st = make_batch4(c, basis, quartets, n, &B, s, false, nullptr, 0.0, true);
  if (st != MDX_OK) return st;
  std::unique_ptr<mdx_batch, void (*)(mdx_batch*)> guard(B, batch_free);
  if (B->total > out_capacity) return fail(c, MDX_ECAPACITY, "output capacity too small");
  if ((st = check_device_error(c, s)) != MDX_OK) return st;
  cudaError_t e = cudaMemcpyAsync(out_offsets, B->offsets, (B->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "offsets");
  if ((st = batch_run(c, B, out, nullptr, s)) != MDX_OK) return st;
  e = cudaStreamSynchronize(s);   // the batch's arrays are released on return
  if (e != cudaSuccess) return cuda_fail(c, e, "eri4_sph");
  return check_device_error(c, s);
}

mdx_status mdx_batch_eri4_sph(mdx_ctx* c, const mdx_basis* basis, const int32_t* quartets, int64_t n, mdx_batch** out,
                              void* stream) {
  const NvtxRange nvtx_range("mdx_batch_eri4_sph");
  if (!c || !out) return MDX_EINVAL;
  *out = nullptr;
  c->last_error.clear();
  cudaSetDevice(c->device);
  if (n < 1 || !quartets) return fail(c, MDX_EINVAL, "invalid arguments");
  return make_batch4(c, basis, quartets, n, out, (cudaStream_t)stream, false, nullptr, 0.0, true);
}

mdx_status mdx_eri3(mdx_ctx* c, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets,
                    const double* bound, int64_t n, double tau, double* out, int64_t out_capacity,
                    int64_t* out_offsets, void* stream) {
  const NvtxRange nvtx_range("mdx_eri3");
  if (!c) return MDX_EINVAL;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || !out_offsets || (n > 0 && (!triplets || !out))) return fail(c, MDX_EINVAL, "invalid arguments");
  if (bound && !(tau >= 0.0)) return fail(c, MDX_EINVAL, "tau must be >= 0");
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), s);
    return e == cudaSuccess ? MDX_OK : cuda_fail(c, e, "offsets");
  }
  mdx_batch* B = nullptr;
  mdx_status st = make_batch3(c, aux, orb, triplets, n, &B, s, true, bound, tau);
  if (st != MDX_OK) return st;
  return run_once(c, B, out, out_capacity, out_offsets, s);
}

mdx_status mdx_eri3_sph(mdx_ctx* c, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets, int64_t n,
                        double* out, int64_t out_capacity, int64_t* out_offsets, void* stream) {
  const NvtxRange nvtx_range("mdx_eri3_sph");
  if (!c) return MDX_EINVAL;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || !out_offsets || (n > 0 && (!triplets || !out))) return fail(c, MDX_EINVAL, "invalid arguments");
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), s);
    return e == cudaSuccess ? MDX_OK : cuda_fail(c, e, "offsets");
  }
  mdx_batch* B = nullptr;
  mdx_status st = make_batch3(c, aux, orb, triplets, n, &B, s, false, nullptr, 0.0, true);
  if (st != MDX_OK) return st;
  std::unique_ptr<mdx_batch, void (*)(mdx_batch*)> guard(B, batch_free);
  if (B->total > out_capacity) return fail(c, MDX_ECAPACITY, "output capacity too small");
  if ((st = check_device_error(c, s)) != MDX_OK) return st;
  cudaError_t e = cudaMemcpyAsync(out_offsets, B->offsets, (B->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "offsets");
  if ((st = batch_run(c, B, out, nullptr, s)) != MDX_OK) return st;
  e = cudaStreamSynchronize(s);   // the batch's arrays are released on return
  if (e != cudaSuccess) return cuda_fail(c, e, "eri3_sph");
  return check_device_error(c, s);
}

mdx_status mdx_batch_eri3_sph(mdx_ctx* c, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets,
                              int64_t n, mdx_batch** out, void* stream) {
  const NvtxRange nvtx_range("mdx_batch_eri3_sph");
  if (!c || !out) return MDX_EINVAL;
  *out = nullptr;
  c->last_error.clear();
  cudaSetDevice(c->device);
  if (n < 1 || !triplets) return fail(c, MDX_EINVAL, "invalid arguments");
  return make_batch3(c, aux, orb, triplets, n, out, (cudaStream_t)stream, false, nullptr, 0.0, true);
}

mdx_status mdx_batch_eri4(mdx_ctx* c, const mdx_basis* basis, const int32_t* quartets, int64_t n, mdx_batch** out,
                          void* stream) {
  const NvtxRange nvtx_range("mdx_batch_eri4");
  if (!c || !out) return MDX_EINVAL;
  *out = nullptr;
  c->last_error.clear();
  cudaSetDevice(c->device);
  if (n < 1 || !quartets) return fail(c, MDX_EINVAL, "invalid arguments");
  return make_batch4(c, basis, quartets, n, out, (cudaStream_t)stream);
}

mdx_status mdx_batch_eri3(mdx_ctx* c, const mdx_basis* aux, const mdx_basis* orb, const int32_t* triplets, int64_t n,
                          mdx_batch** out, void* stream) {
  const NvtxRange nvtx_range("mdx_batch_eri3");
  if (!c || !out) return MDX_EINVAL;
  *out = nullptr;
  c->last_error.clear();
  cudaSetDevice(c->device);
  if (n < 1 || !triplets) return fail(c, MDX_EINVAL, "invalid arguments");
  return make_batch3(c, aux, orb, triplets, n, out, (cudaStream_t)stream);
}

mdx_status mdx_batch_info(const mdx_batch* b, int64_t* n, int64_t* total, double* model_flops, double* exec_fma) {
  if (!b) return MDX_EINVAL;
  if (n) *n = b->n;
  if (total) *total = b->total;
  if (model_flops) *model_flops = b->model_flops;
  if (exec_fma) *exec_fma = b->exec_fma;
  return MDX_OK;
}

mdx_status mdx_batch_offsets(mdx_ctx* c, const mdx_batch* b, int64_t* out_offsets, void* stream) {
  if (!c || !b || !out_offsets) return MDX_EINVAL;
  cudaSetDevice(c->device);
  cudaError_t e = cudaMemcpyAsync(out_offsets, b->offsets, (b->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream);
  return e == cudaSuccess ? MDX_OK : cuda_fail(c, e, "offsets");
}

mdx_status mdx_batch_run(mdx_ctx* c, mdx_batch* b, double* out, int64_t out_capacity, int32_t* n_launches,
                         void* stream) {
  const NvtxRange nvtx_range("mdx_batch_run");
  if (!c || !b || !out) return MDX_EINVAL;
  if (b->ctx != c) return fail(c, MDX_EINVAL, "batch belongs to another context");
  if (b->total > out_capacity) return fail(c, MDX_ECAPACITY, "output capacity too small");
  cudaSetDevice(c->device);
  return batch_run(c, b, out, n_launches, (cudaStream_t)stream);
}

mdx_status mdx_batch_run_materialized(mdx_ctx* c, mdx_batch* B, double* out, int64_t out_capacity,
                                      int32_t* n_launches, void* stream) {
  const NvtxRange nvtx_range("mdx_batch_run_materialized");
  if (!c || !B || !out) return MDX_EINVAL;
  if (B->ctx != c) return fail(c, MDX_EINVAL, "batch belongs to another context");
  if (B->total > out_capacity) return fail(c, MDX_ECAPACITY, "output capacity too small");
  if (B->sph) return fail(c, MDX_EUNSUPPORTED, "materialized path: Cartesian batches only");
  for (auto& r : B->ranges)
    if (r.count > 0 && (r.key.Kb != 1 || r.key.Kk != 1 || r.key.onec))
      return fail(c, MDX_EUNSUPPORTED, "materialized path: uncontracted 4-center classes only");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (!c->cublas && cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS) {
    c->cublas = nullptr;
    return fail(c, MDX_ECUDA, "cublasCreate failed");
  }
  if (cublasSetStream(c->cublas, s) != CUBLAS_STATUS_SUCCESS) return fail(c, MDX_ECUDA, "cublasSetStream failed");
  int32_t nl = 0;
  cudaError_t e = launch_pair_records(B->b0, B->b1, B->jobs, B->njobs, B->recs, B->recs_s, c->d_err, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair records");
  if (B->njobs > 0) ++nl;
  mdx_status st;
  for (auto& r : B->ranges) {
    if (r.count == 0) continue;
    const ClassKey& k = r.key;
    const int Lb = k.la + k.lb, Lk = k.lc + k.ld;
    const int64_t Nb = ncart(k.la) * ncart(k.lb), Nk = ncart(k.lc) * ncart(k.ld);
    const int64_t Hb = nherm(Lb), Hk = nherm(Lk);
    // the class's bra and ket pairs, numbered compactly
    std::vector<int2> hq;
    hq.resize((size_t)r.count);
    e = cudaMemcpyAsync(hq.data(), B->qp + r.begin, r.count * sizeof(int2), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "quartet download");
    std::unordered_map<int32_t, int32_t> mb, mk;
    std::vector<int32_t> ub, uk, qib((size_t)r.count), qik((size_t)r.count);
    for (int64_t i = 0; i < r.count; ++i) {
      auto ib = mb.emplace(hq[i].x, (int32_t)ub.size());
      if (ib.second) ub.push_back(hq[i].x);
      auto ik = mk.emplace(hq[i].y, (int32_t)uk.size());
      if (ik.second) uk.push_back(hq[i].y);
      qib[i] = ib.first->second;
      qik[i] = ik.first->second;
    }
    int32_t *d_ub, *d_uk, *d_qib, *d_qik;
    if ((st = upload(c, "mat_ub", ub, &d_ub, s)) != MDX_OK) return st;
    if ((st = upload(c, "mat_uk", uk, &d_uk, s)) != MDX_OK) return st;
    if ((st = upload(c, "mat_qib", qib, &d_qib, s)) != MDX_OK) return st;
    if ((st = upload(c, "mat_qik", qik, &d_qik, s)) != MDX_OK) return st;
    double *Eab, *Ecd;
    if ((st = ensure(c, "mat_eab", (size_t)(ub.size() * Nb * Hb), &Eab, s)) != MDX_OK) return st;
    if ((st = ensure(c, "mat_ecd", (size_t)(uk.size() * Hk * Nk), &Ecd, s)) != MDX_OK) return st;
    e = launch_mat_emat(B->recs, B->pair_rec, d_ub, (int64_t)ub.size(), k.la, k.lb, true, Eab, s);
    if (e == cudaSuccess) e = launch_mat_emat(B->recs, B->pair_rec, d_uk, (int64_t)uk.size(), k.lc, k.ld, false, Ecd, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "E matrices");
    nl += 2;
    // chunks whose [p|q] and [p|cd] matrices fit a 2 GB workspace
    const int64_t per_q = (Hb * Hk + Hb * Nk) * (int64_t)sizeof(double);
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(r.count, (int64_t(2) << 30) / per_q));
    double *PQ, *Tm;
    const double** ptrs;
    if ((st = ensure(c, "mat_pq", (size_t)(chunk * Hb * Hk), &PQ, s)) != MDX_OK) return st;
    if ((st = ensure(c, "mat_t", (size_t)(chunk * Hb * Nk), &Tm, s)) != MDX_OK) return st;
    if ((st = ensure(c, "mat_ptrs", (size_t)(6 * chunk), &ptrs, s)) != MDX_OK) return st;
    const double** a1 = ptrs;
    const double** b1 = ptrs + chunk;
    double** c1 = (double**)(ptrs + 2 * chunk);
    const double** a2 = ptrs + 3 * chunk;
    const double** b2 = ptrs + 4 * chunk;
    double** c2 = (double**)(ptrs + 5 * chunk);
    const double one = 1.0, zero = 0.0;
    for (int64_t q0 = 0; q0 < r.count; q0 += chunk) {
      const int64_t nq = std::min(chunk, r.count - q0);
      e = launch_mat_hermite(B->recs, B->pair_rec, B->qp + r.begin + q0, nq, Lb, Lk, c->d_boys, PQ, s);
      if (e == cudaSuccess)
        e = launch_mat_ptrs(nq, d_qib + q0, d_qik + q0, B->qoff + r.begin + q0, Eab, Nb * Hb, Ecd, Hk * Nk, PQ,
                            Hb * Hk, Tm, Hb * Nk, out, a1, b1, c1, a2, b2, c2, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "materialized Hermite matrices");
      nl += 2;
      // row-major X[r x c] is column-major X^T: [p|cd]^T = (E^cd)^T [p|q]^T, then
      // [ab|cd]^T = [p|cd]^T (E^ab)^T, both with the Cartesian ket index fastest
      cublasStatus_t cs = cublasDgemmBatched(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, (int)Nk, (int)Hb, (int)Hk, &one,
                                             a1, (int)Nk, b1, (int)Hk, &zero, c1, (int)Nk, (int)nq);
      if (cs == CUBLAS_STATUS_SUCCESS)
        cs = cublasDgemmBatched(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, (int)Nk, (int)Nb, (int)Hb, &one, a2, (int)Nk,
                                b2, (int)Hb, &zero, c2, (int)Nk, (int)nq);
      if (cs != CUBLAS_STATUS_SUCCESS) return fail(c, MDX_ECUDA, "cublasDgemmBatched failed");
      nl += 2;
    }
  }
  if (n_launches) *n_launches = nl;
  return MDX_OK;
}

void mdx_batch_destroy(mdx_batch* b) { batch_free(b); }

// Autotuner of a solid-harmonic batch: for every class that runs the solid-harmonic team kernel, the team
// size (and, for classes of several column groups, the shared-memory budget and the cached R tables) that
// times fastest on the first max_trial quartets of the class. The staging area grows if the chosen shape
// needs more.
mdx_status autotune_sph(mdx_ctx* c, mdx_batch* b, double* out, int64_t max_trial, cudaStream_t s) {
  cudaError_t e = launch_pair_records(b->b0, b->b1, b->jobs, b->njobs, b->recs, b->recs_s, c->d_err, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair records");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto done = [&](mdx_status st) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  };
  for (auto& r : b->ranges) {
    if (r.count == 0) continue;
    ClassKey k2 = r.key;
    k2.store = 2;
    const int64_t nq = std::min(r.count, max_trial);
    // classes on the register-kernel route (Cartesian shellsets, then the transform) also try the
    // solid-harmonic team kernel, and move to it when it is faster
    float reg_ms = 1e30f;
    if (!r.splan) {
      QuartetLaunch a{};
      a.plan = r.plan->d;
      a.nq = nq;
      a.qpairs = b->qp + r.begin;
      a.qout = b->cqoff + r.begin;
      a.pair_rec = b->pair_rec;
      a.recs = b->recs;
      a.recs_signed = b->recs_s;
      a.boys = c->d_boys;
      a.rprog = c->d_rprog;
      a.rprog_off = c->d_rprog_off;
      a.out = b->cart;
      a.err = c->d_err;
      const SphLaunch t{r.key.la, r.key.lb, r.key.lc, r.key.ld, nq, b->cart, b->cqoff + r.begin, out,
                        b->qoff + r.begin};
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        e = launch_quartets(a, s);
        if (e == cudaSuccess) e = launch_cart2sph(t, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return done(cuda_fail(c, e, "autotune"));
        float tm = 0;
        cudaEventElapsedTime(&tm, e0, e1);
        reg_ms = std::min(reg_ms, tm);
      }
    }
    std::vector<PlanConfig> cands;
    Plan* dflt = r.splan;
    std::unique_ptr<Plan> dflt_own;
    if (!dflt) {   // the team plan's default shape decides which candidate family applies
      dflt_own.reset(new Plan());
      std::string err;
      if (!build_plan(k2, PlanConfig{}, *dflt_own, err)) continue;
      dflt = dflt_own.get();
    }
    if (dflt->d.ngroups > 1) {
      for (int budget : {200 * 1024, 108 * 1024})
        for (int T : {128, 256, 512, 1024})
          for (int rc : {-1, 0, 1}) cands.push_back(PlanConfig{T, budget, 96 * 1024, 1, rc});
    } else {
      for (int T : {0, 4, 8, 16, 32, 64, 128, 256, 512}) cands.push_back(PlanConfig{T, 200 * 1024, 96 * 1024, 1, -1});
    }
    float best_ms = reg_ms;   // a register-kernel class keeps its route unless a team shape beats it
    PlanConfig best{};
    std::unique_ptr<Plan> best_plan;
    std::vector<std::array<int, 5>> seen;   // shapes already timed
    for (const PlanConfig& cfg : cands) {
      std::unique_ptr<Plan> p(new Plan());
      std::string err;
      if (!build_plan(k2, cfg, *p, err)) continue;
      const std::array<int, 5> sig{p->d.T, p->d.teams_per_cta, p->d.team_doubles, p->d.ngroups, p->d.cache_R};
      if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
      seen.push_back(sig);
      int grid = 0;
      if ((e = sph_grid(p->d, nq, &grid)) != cudaSuccess) return done(cuda_fail(c, e, "solid-harmonic launch shape"));
      const int64_t need = (int64_t)grid * p->d.teams_per_cta * p->d.xg_doubles;
      if (need > b->nxg) {   // a larger staging area for this shape (all launches so far have completed)
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return done(cuda_fail(c, e, "autotune"));
        cudaFree(b->xg);
        b->xg = nullptr;
        b->nxg = 0;
        if (cudaMalloc(&b->xg, need * sizeof(double)) != cudaSuccess) {
          cudaGetLastError();
          continue;   // this shape's staging does not fit the device: not a candidate
        }
        b->nxg = need;
      }
      mdx_status st = upload_plan(c, p.get(), s);
      if (st != MDX_OK) { if (p->dev_blob) cudaFree(p->dev_blob); return done(st); }
      QuartetLaunch a{};
      a.plan = p->d;
      a.nq = nq;
      a.qpairs = b->qp + r.begin;
      a.qout = b->qoff + r.begin;
      a.pair_rec = b->pair_rec;
      a.recs = b->recs;
      a.recs_signed = b->recs_s;
      a.boys = c->d_boys;
      a.rprog = c->d_rprog;
      a.rprog_off = c->d_rprog_off;
      a.out = out;
      a.err = c->d_err;
      a.sph_scratch = b->xg;
      float ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        e = launch_quartets_sph(a, grid, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { cudaFree(p->dev_blob); return done(cuda_fail(c, e, "autotune")); }
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = cfg;
        if (best_plan && best_plan->dev_blob) cudaFree(best_plan->dev_blob);
        best_plan = std::move(p);
      } else {
        cudaFree(p->dev_blob);
      }
    }
    if (!best_plan) continue;
    int grid = 0;
    if ((e = sph_grid(best_plan->d, r.count, &grid)) != cudaSuccess) return done(cuda_fail(c, e, "solid-harmonic launch shape"));
    const int64_t need = (int64_t)grid * best_plan->d.teams_per_cta * best_plan->d.xg_doubles;
    if (need > b->nxg) {
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return done(cuda_fail(c, e, "autotune"));
      cudaFree(b->xg);
      b->xg = nullptr;
      b->nxg = 0;
      if (cudaMalloc(&b->xg, need * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return done(fail(c, MDX_ENOMEM, "solid-harmonic staging area"));
      }
      b->nxg = need;
    }
    c->tuned[k2] = best;
    // the batch's executed-FMA count follows the route and shape the class runs now
    const double old_fma = r.splan ? r.splan->exec_fma : r.plan->exec_fma + cart2sph_fma(r.key);
    b->exec_fma += (best_plan->exec_fma - old_fma) * (double)r.count;
    auto it = c->plans.find(k2);
    if (it != c->plans.end()) c->retired.push_back(std::move(it->second));
    r.splan = best_plan.get();
    r.grid = grid;
    c->plans[k2] = std::move(best_plan);
  }
  // the staging area must serve every class of the batch
  for (auto& r : b->ranges)
    if (r.splan && (int64_t)r.grid * r.splan->d.teams_per_cta * r.splan->d.xg_doubles > b->nxg)
      return done(fail(c, MDX_EINVAL, "solid-harmonic staging area smaller than a class needs"));
  done(MDX_OK);
  return check_device_error(c, s);
}

mdx_status mdx_batch_autotune(mdx_ctx* c, mdx_batch* b, double* out, int64_t out_capacity, int64_t max_trial,
                              void* stream) {
  const NvtxRange nvtx_range("mdx_batch_autotune");
  if (!c || !b || !out || max_trial < 1) return MDX_EINVAL;
  if (b->ctx != c) return fail(c, MDX_EINVAL, "batch belongs to another context");
  if (b->total > out_capacity) return fail(c, MDX_ECAPACITY, "output capacity too small");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (b->sph) return autotune_sph(c, b, out, max_trial, s);
  cudaError_t e = launch_pair_records(b->b0, b->b1, b->jobs, b->njobs, b->recs, b->recs_s, c->d_err, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair records");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (auto& r : b->ranges) {
    if (r.count == 0) continue;
    // candidate shapes: team sizes x shared-memory budgets (teams per SM)
    // (classes whose default plan splits the ket columns into groups only vary
    // the team size and budget: their plans are expensive to build)
    // plus the register kernel (one thread per quartet) where the class has one
    std::vector<PlanConfig> cands;
    if (r.plan->d.ngroups > 1) {
      for (int pack : {1, 0})
        for (int budget : {200 * 1024, 108 * 1024, 72 * 1024})
          for (int T : {256, 512, 1024}) cands.push_back(PlanConfig{T, budget, 96 * 1024, 1, -1, pack});
    } else {
      for (int single : {96 * 1024, 40 * 1024})
        for (int T : {0, 1, 4, 16, 32, 64, 128, 256, 512}) cands.push_back(PlanConfig{T, 200 * 1024, single, 1});
    }
    const ClassKey& rk = r.key;
    if (reg_eligible(rk.la, rk.lb, rk.lc, rk.ld) || reg_xs_eligible(rk.la, rk.lb, rk.lc, rk.ld))
      cands.push_back(PlanConfig{0, 200 * 1024, 96 * 1024, 2});
    float best_ms = 1e30f;
    PlanConfig best{};
    std::unique_ptr<Plan> best_plan;
    std::vector<std::pair<int, int>> seen;   // (T, team_doubles, ngroups) signature of built plans
    for (const PlanConfig& cfg : cands) {
      std::unique_ptr<Plan> p(new Plan());
      std::string err;
      if (!build_plan(r.key, cfg, *p, err)) continue;
      const std::pair<int, int> sig{p->d.reg ? -1 : p->d.T * 100000 + p->d.ngroups,
                                    p->d.reg ? 0 : p->d.team_doubles * 64 + p->d.teams_per_cta};
      if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;   // same shape as one already timed
      seen.push_back(sig);
      mdx_status st = upload_plan(c, p.get(), s);
      if (st != MDX_OK) { if (p->dev_blob) cudaFree(p->dev_blob); return st; }
      QuartetLaunch a{};
      a.plan = p->d;
      a.nq = std::min(r.count, max_trial);
      a.qpairs = b->qp + r.begin;
      a.qout = b->qoff + r.begin;
      a.pair_rec = b->pair_rec;
      a.recs = b->recs;
      a.recs_signed = b->recs_s;
      a.boys = c->d_boys;
      a.rprog = c->d_rprog;
      a.rprog_off = c->d_rprog_off;
      a.out = out;
      a.err = c->d_err;
      float ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        e = launch_quartets(a, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { cudaFree(p->dev_blob); cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_fail(c, e, "autotune"); }
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = cfg;
        if (best_plan && best_plan->dev_blob) cudaFree(best_plan->dev_blob);
        best_plan = std::move(p);
      } else {
        cudaFree(p->dev_blob);
      }
    }
    if (!best_plan) continue;
    c->tuned[r.key] = best;
    b->exec_fma += (best_plan->exec_fma - r.plan->exec_fma) * (double)r.count;   // the shape it runs now
    auto it = c->plans.find(r.key);
    if (it != c->plans.end()) c->retired.push_back(std::move(it->second));
    r.plan = best_plan.get();
    c->plans[r.key] = std::move(best_plan);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return check_device_error(c, s);
}

mdx_status mdx_schwarz(mdx_ctx* c, const mdx_basis* basis, const int32_t* pairs, int64_t n, double* Q_out,
                       void* stream) {
  const NvtxRange nvtx_range("mdx_schwarz");
  if (!c) return MDX_EINVAL;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || (n > 0 && (!pairs || !Q_out))) return fail(c, MDX_EINVAL, "invalid arguments");
  if (n == 0) return MDX_OK;
  HostBasis hb;
  mdx_status st = fetch_basis(c, basis, hb, s);
  if (st != MDX_OK) return st;
  std::vector<int32_t> hp;
  if ((st = read_quartets(c, pairs, n, 2, hp, s)) != MDX_OK) return st;
  for (int64_t p = 0; p < n; ++p) {
    const int32_t i = hp[2 * p], j = hp[2 * p + 1];
    if (i < 0 || i >= hb.n || j < 0 || j >= hb.n) return fail(c, MDX_EINVAL, "shell index out of range");
  }
  // chunks of pairs whose diagonal shellsets (ab|ab) hold at most kChunk doubles together
  constexpr int64_t kChunk = int64_t(1) << 27;
  for (int64_t p0 = 0; p0 < n;) {
    Batch bt;
    std::vector<int64_t> offs(1, 0);
    std::vector<int32_t> nab;
    int64_t tot = 0, p1 = p0;
    for (; p1 < n; ++p1) {
      const int32_t i = hp[2 * p1], j = hp[2 * p1 + 1];
      const int32_t m = ncart(hb.l[i]) * ncart(hb.l[j]);
      if (p1 > p0 && tot + (int64_t)m * m > kChunk) break;
      const int32_t k = (int32_t)(p1 - p0);
      bt.pairs.push_back(PairKey{i, j, 0});
      bt.qp.push_back(make_int2(k, k));
      bt.qoff.push_back(tot);
      nab.push_back(m);
      tot += (int64_t)m * m;
      offs.push_back(tot);
    }
    const int64_t cnt = p1 - p0;
    double* d_vals; int32_t* d_nab;
    if ((st = ensure(c, "schwarz_vals", (size_t)tot, &d_vals, s)) != MDX_OK) return st;
    if ((st = upload(c, "schwarz_nab", nab, &d_nab, s)) != MDX_OK) return st;
    mdx_batch* B = nullptr;
    if ((st = batch_prepare(c, basis, nullptr, hb, hb, bt, offs, &B, s)) != MDX_OK) return st;
    std::unique_ptr<mdx_batch, void (*)(mdx_batch*)> guard(B, batch_free);
    if ((st = batch_run(c, B, d_vals, nullptr, s)) != MDX_OK) return st;
    cudaError_t e = launch_schwarz_reduce(B->offsets, d_nab, cnt, d_vals, Q_out + p0, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "schwarz reduce");
    e = cudaStreamSynchronize(s);   // the chunk's host vectors and batch are released next
    if (e != cudaSuccess) return cuda_fail(c, e, "schwarz");
    p0 = p1;
  }
  return check_device_error(c, s);
}

}  // extern "C"

namespace {

// Shared front end of the exchange build and its gradient: canonical distinct
// pairs sorted by pair class and, within a class, by decreasing Schwarz
// factor; density-block maxima; Schwarz x density screening of the unique
// quartets into (bra class, ket class) buckets on the GPU (FP64 throughout).
struct XPrep {
  HostBasis hb;
  std::vector<int32_t> ao;
  int64_t nao = 0, np = 0, nq = 0;
  struct P4 { int32_t i, j; double q; int li, lj, K; int64_t orig; };
  std::vector<P4> pl;
  std::vector<std::array<int, 3>> classes;
  std::vector<unsigned long long> counts;
  std::vector<int64_t> boff;
  int2* d_pshell = nullptr;
  int2* d_quart = nullptr;
  int64_t* d_orig = nullptr;   // caller index of each sorted pair
};

// fill = false: counts only (X.d_quart stays unset).
mdx_status exchange_screen(mdx_ctx* c, const mdx_basis* basis, const int32_t* pairs, const double* Q, int64_t n_pairs,
                           double tau, const double* D, XPrep& X, cudaStream_t s, bool fill = true) {
  if (!basis || !basis->ao_off) return fail(c, MDX_EINVAL, "basis needs ao_off");
  mdx_status st = fetch_basis(c, basis, X.hb, s);
  if (st != MDX_OK) return st;
  const HostBasis& hb = X.hb;
  X.ao.resize(hb.n);
  cudaError_t e = cudaSuccess;
  if (hb.n) e = cudaMemcpyAsync(X.ao.data(), basis->ao_off, hb.n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "ao_off download");
  X.nao = 0;
  for (int i = 0; i < hb.n; ++i) X.nao = std::max<int64_t>(X.nao, (int64_t)X.ao[i] + ncart(hb.l[i]));
  if (X.nao > 2000000000 / 2) return fail(c, MDX_EUNSUPPORTED, "too many AOs");
  if (n_pairs > 0x7fffffff) return fail(c, MDX_EUNSUPPORTED, "too many shell pairs");
  X.np = n_pairs;
  if (n_pairs == 0 || hb.n == 0) return MDX_OK;
  std::vector<int32_t> hp;
  if ((st = read_quartets(c, pairs, n_pairs, 2, hp, s)) != MDX_OK) return st;
  std::vector<double> hq(n_pairs);
  e = cudaMemcpyAsync(hq.data(), Q, n_pairs * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Q download");
  X.pl.resize(n_pairs);
  std::unordered_map<int64_t, int> seen;
  for (int64_t p = 0; p < n_pairs; ++p) {
    int32_t i = hp[2 * p], j = hp[2 * p + 1];
    if (i < 0 || i >= hb.n || j < 0 || j >= hb.n) return fail(c, MDX_EINVAL, "shell index out of range");
    if (!(hq[p] >= 0.0)) return fail(c, MDX_EINVAL, "Schwarz factors must be >= 0");
    if (i < j) std::swap(i, j);
    if (!seen.emplace((int64_t)i * hb.n + j, 1).second) return fail(c, MDX_EINVAL, "shell pair listed twice");
    X.pl[p] = XPrep::P4{i, j, hq[p], hb.l[i], hb.l[j], hb.nprim[i] * hb.nprim[j], p};
  }
  std::stable_sort(X.pl.begin(), X.pl.end(), [](const XPrep::P4& a, const XPrep::P4& b) {
    if (a.li != b.li) return a.li < b.li;
    if (a.lj != b.lj) return a.lj < b.lj;
    if (a.K != b.K) return a.K < b.K;
    return a.q > b.q;
  });
  // one molecule: each class is one segment, listed in pair order (already Q-descending)
  std::vector<int2> pshell(n_pairs);
  std::vector<int32_t> pclass(n_pairs), order(n_pairs), seg_class, mol_seg{0, 0}, shell_first{0, hb.n};
  std::vector<int64_t> pos(n_pairs), seg_begin, orig(n_pairs), dmax_off{0};
  std::vector<double> qd(n_pairs);
  for (int64_t p = 0; p < n_pairs; ++p) {
    std::array<int, 3> k{X.pl[p].li, X.pl[p].lj, X.pl[p].K};
    if (X.classes.empty() || X.classes.back() != k) {
      X.classes.push_back(k);
      seg_begin.push_back(p);
      seg_class.push_back((int32_t)X.classes.size() - 1);
    }
    pclass[p] = (int32_t)X.classes.size() - 1;
    pshell[p] = make_int2(X.pl[p].i, X.pl[p].j);
    qd[p] = X.pl[p].q;
    order[p] = (int32_t)p;
    pos[p] = p;
    orig[p] = X.pl[p].orig;
  }
  seg_begin.push_back(n_pairs);
  mol_seg[1] = (int32_t)seg_class.size();
  const int nclass = (int)X.classes.size();
  const int64_t nbucket = (int64_t)nclass * (nclass + 1) / 2;
  int32_t *d_pclass, *d_order, *d_segc, *d_molseg, *d_sfirst;
  int64_t *d_pos, *d_segb, *d_doff, *d_boff;
  double *d_q, *d_dmax, *d_rowmax;
  unsigned long long* d_counts;
  if ((st = upload(c, "x_pshell", pshell, &X.d_pshell, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_pclass", pclass, &d_pclass, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_q", qd, &d_q, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_order", order, &d_order, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_pos", pos, &d_pos, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_orig", orig, &X.d_orig, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_segb", seg_begin, &d_segb, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_segc", seg_class, &d_segc, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_molseg", mol_seg, &d_molseg, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_sfirst", shell_first, &d_sfirst, s)) != MDX_OK) return st;
  if ((st = upload(c, "x_doff", dmax_off, &d_doff, s)) != MDX_OK) return st;
  // the N_shells x N_shells table of density-block maxima (8 bytes per shell pair)
  if ((st = ensure(c, "x_dmax", (size_t)hb.n * hb.n, &d_dmax, s)) != MDX_OK) return st;
  if ((st = ensure(c, "x_rowmax", (size_t)hb.n, &d_rowmax, s)) != MDX_OK) return st;
  if ((st = ensure(c, "x_counts", (size_t)nbucket, &d_counts, s)) != MDX_OK) return st;
  e = launch_dmax(D, (int32_t)X.nao, basis->ao_off, basis->l, hb.n, d_dmax, hb.n, s);
  if (e == cudaSuccess) e = launch_rowmax(d_dmax, hb.n, d_rowmax, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_counts, 0, nbucket * sizeof(unsigned long long), s);
  ScreenArgs sa{};
  sa.npairs = n_pairs;
  sa.pair_shells = X.d_pshell;
  sa.Q = d_q;
  sa.pair_class = d_pclass;
  sa.pos = d_pos;
  sa.order = d_order;
  sa.seg_begin = d_segb;
  sa.seg_class = d_segc;
  sa.mol_seg = d_molseg;
  sa.pair_mol = nullptr;
  sa.shell_first = d_sfirst;
  sa.dmax_off = d_doff;
  sa.dmax = d_dmax;
  sa.rowmax = d_rowmax;
  sa.nclass = nclass;
  sa.tau = tau;
  sa.counts = d_counts;
  if (e == cudaSuccess) e = launch_screen(sa, false, s);
  X.counts.assign(nbucket, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(X.counts.data(), d_counts, nbucket * sizeof(unsigned long long),
                                            cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "exchange screening");
  X.boff.assign(nbucket + 1, 0);
  for (int64_t b = 0; b < nbucket; ++b) X.boff[b + 1] = X.boff[b] + (int64_t)X.counts[b];
  X.nq = X.boff[nbucket];
  c->last_quartets = X.nq;
  if (X.nq > 0 && fill) {
    if ((st = upload(c, "x_boff", X.boff, &d_boff, s)) != MDX_OK) return st;
    if ((st = ensure(c, "x_quart", (size_t)X.nq, &X.d_quart, s)) != MDX_OK) return st;
    e = cudaMemsetAsync(d_counts, 0, nbucket * sizeof(unsigned long long), s);
    sa.bucket_off = d_boff;
    sa.out = X.d_quart;
    if (e == cudaSuccess) e = launch_screen(sa, true, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "exchange screening");
  }
  return MDX_OK;
}

QuartetLaunch base_launch(mdx_ctx* c, Plan* plan, const int2* qp, int64_t nq, const int64_t* prec, const double* recs,
                          const double* recs_s) {
  QuartetLaunch a{};
  a.plan = plan->d;
  a.nq = nq;
  a.qpairs = qp;
  a.pair_rec = prec;
  a.recs = recs;
  a.recs_signed = recs_s;
  a.boys = c->d_boys;
  a.rprog = c->d_rprog;
  a.rprog_off = c->d_rprog_off;
  a.err = c->d_err;
  return a;
}

}  // namespace

extern "C" {

mdx_status mdx_exchange(mdx_ctx* c, const mdx_basis* basis, const int32_t* pairs, const double* Q, int64_t n_pairs,
                        double tau, const double* D, double* K, double alpha, double* energy, void* stream) {
  const NvtxRange nvtx_range("mdx_exchange");
  if (!c) return MDX_EINVAL;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n_pairs < 0 || !D || !K || (n_pairs > 0 && (!pairs || !Q)) || !(tau >= 0.0))
    return fail(c, MDX_EINVAL, "invalid arguments");
  XPrep X;
  mdx_status st = exchange_screen(c, basis, pairs, Q, n_pairs, tau, D, X, s);
  if (st != MDX_OK) return st;
  cudaError_t e = cudaMemsetAsync(K, 0, (size_t)X.nao * X.nao * sizeof(double), s);
  if (e == cudaSuccess && energy) e = cudaMemsetAsync(energy, 0, sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "K clear");
  if (X.nq > 0) {
    const HostBasis& hb = X.hb;
    std::vector<int64_t> pair_rec(X.np);
    std::vector<PrimPairJob> jobs;
    int64_t roff = 0;
    for (int64_t p = 0; p < X.np; ++p) {
      pair_rec[p] = roff;
      for (int ia = 0; ia < hb.nprim[X.pl[p].i]; ++ia)
        for (int ib = 0; ib < hb.nprim[X.pl[p].j]; ++ib) {
          jobs.push_back(PrimPairJob{X.pl[p].i, X.pl[p].j, ia, ib, 0, 0, roff});
          roff += rec_size(X.pl[p].li, X.pl[p].lj);
        }
    }
    PrimPairJob* d_jobs; int64_t* d_prec; double *d_recs, *d_recs_s;
    if ((st = upload(c, "x_jobs", jobs, &d_jobs, s)) != MDX_OK) return st;
    if ((st = upload(c, "x_prec", pair_rec, &d_prec, s)) != MDX_OK) return st;
    if ((st = ensure(c, "x_recs", (size_t)roff, &d_recs, s)) != MDX_OK) return st;
    if ((st = ensure(c, "x_recs_s", (size_t)roff, &d_recs_s, s)) != MDX_OK) return st;
    e = launch_pair_records(to_dev(basis), to_dev(basis), d_jobs, (int64_t)jobs.size(), d_recs, d_recs_s, c->d_err, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "pair records");
    // all plans first (their uploads go to s before the fork), heaviest launch first
    std::vector<std::pair<double, QuartetLaunch>> jobs_k;
    const int nclass = (int)X.classes.size();
    for (int cp = 0; cp < nclass; ++cp)
      for (int cq = 0; cq <= cp; ++cq) {
        const int64_t b = (int64_t)cp * (cp + 1) / 2 + cq;
        if (X.counts[b] == 0) continue;
        const ClassKey key{X.classes[cp][0], X.classes[cp][1], X.classes[cq][0], X.classes[cq][1],
                           X.classes[cp][2], X.classes[cq][2], 0};
        Plan* plan;
        if ((st = get_plan(c, key, &plan, s)) != MDX_OK) return st;
        QuartetLaunch a = base_launch(c, plan, X.d_quart + X.boff[b], (int64_t)X.counts[b], d_prec, d_recs, d_recs_s);
        a.D = D;
        a.K = K;
        a.nao = (int32_t)X.nao;
        a.ao_off = basis->ao_off;
        a.pair_shells = X.d_pshell;
        jobs_k.emplace_back(model_flops_class(key) * (double)X.counts[b], a);
      }
    std::stable_sort(jobs_k.begin(), jobs_k.end(),
                     [](const std::pair<double, QuartetLaunch>& x, const std::pair<double, QuartetLaunch>& y) {
                       return x.first > y.first;
                     });
    Fanout fan{c, s};
    e = fan.fork();
    for (size_t i = 0; i < jobs_k.size() && e == cudaSuccess; ++i)
      e = launch_quartets(jobs_k[i].second, fan.stream(fan.pick(jobs_k[i].first)));
    const cudaError_t ej = fan.join();
    if (e == cudaSuccess) e = ej;
    if (e != cudaSuccess) return cuda_fail(c, e, "exchange quartet launch");
  }
  e = launch_symmetrize(K, (int32_t)X.nao, s);
  // E_x = alpha sum_ik D_ik K_ik = alpha sum_ijkl D_ik D_jl (ij|kl)
  if (e == cudaSuccess && energy) e = launch_dot_energy(D, K, X.nao * X.nao, alpha, energy, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "exchange");
  return check_device_error(c, s);
}

mdx_status mdx_exchange_screen(mdx_ctx* c, const mdx_basis* basis, const int32_t* pairs, const double* Q,
                               int64_t n_pairs, double tau, const double* D, int32_t* kept, int64_t kept_capacity,
                               int64_t* n_kept, double* model_flops, void* stream) {
  const NvtxRange nvtx_range("mdx_exchange_screen");
  if (!c) return MDX_EINVAL;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n_pairs < 0 || !D || !n_kept || (n_pairs > 0 && (!pairs || !Q)) || !(tau >= 0.0) || kept_capacity < 0 ||
      (kept_capacity > 0 && !kept))
    return fail(c, MDX_EINVAL, "invalid arguments");
  *n_kept = 0;
  if (model_flops) *model_flops = 0.0;
  XPrep X;
  // count first; list only when the caller asked for it and it fits
  mdx_status st = exchange_screen(c, basis, pairs, Q, n_pairs, tau, D, X, s, false);
  if (st != MDX_OK) return st;
  *n_kept = X.nq;
  if (model_flops) {
    double f = 0.0;
    const int nclass = (int)X.classes.size();
    for (int cp = 0; cp < nclass; ++cp)
      for (int cq = 0; cq <= cp; ++cq) {
        const int64_t b = (int64_t)cp * (cp + 1) / 2 + cq;
        const ClassKey key{X.classes[cp][0], X.classes[cp][1], X.classes[cq][0], X.classes[cq][1], X.classes[cp][2],
                           X.classes[cq][2], 0};
        f += model_flops_class(key) * (double)X.counts[b];
      }
    *model_flops = f;
  }
  if (!kept || X.nq == 0) return check_device_error(c, s);
  if (X.nq > kept_capacity) return fail(c, MDX_ECAPACITY, "kept-quartet capacity too small");
  XPrep X2;
  if ((st = exchange_screen(c, basis, pairs, Q, n_pairs, tau, D, X2, s, true)) != MDX_OK) return st;
  if (X2.nq != X.nq) return fail(c, MDX_EDEVICE, "screening counts differ between passes");
  cudaError_t e = launch_map_pairs(X2.d_quart, X2.nq, X2.d_orig, kept, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "exchange screening");
  return check_device_error(c, s);
}

mdx_status mdx_exchange_grad(mdx_ctx* c, const mdx_basis* basis, const int32_t* pairs, const double* Q,
                             int64_t n_pairs, double tau, const double* D, double alpha, int32_t n_atoms,
                             double* grad, double* energy, void* stream) {
  const NvtxRange nvtx_range("mdx_exchange_grad");
  if (!c) return MDX_EINVAL;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n_pairs < 0 || !D || !grad || n_atoms < 1 || (n_pairs > 0 && (!pairs || !Q)) || !(tau >= 0.0))
    return fail(c, MDX_EINVAL, "invalid arguments");
  if (!basis || !basis->atom) return fail(c, MDX_EINVAL, "basis needs atom");
  XPrep X;
  mdx_status st = exchange_screen(c, basis, pairs, Q, n_pairs, tau, D, X, s);
  if (st != MDX_OK) return st;
  const HostBasis& hb = X.hb;
  const int32_t n = hb.n;
  // the derivative raises a shell's l by one, and the planner and kernels stop at MDX_LMAX
  for (int i = 0; i < n; ++i)
    if (hb.l[i] >= MDX_LMAX)
      return fail(c, MDX_EUNSUPPORTED, "exchange gradient: shell angular momentum above MDX_LMAX - 1");
  cudaError_t e = cudaMemsetAsync(grad, 0, (size_t)n_atoms * 3 * sizeof(double), s);
  if (e == cudaSuccess && energy) e = cudaMemsetAsync(energy, 0, sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "gradient clear");
  std::vector<int32_t> atom(n);
  if (n) e = cudaMemcpyAsync(atom.data(), basis->atom, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "atom download");
  for (int i = 0; i < n; ++i)
    if (atom[i] < 0 || atom[i] >= n_atoms) return fail(c, MDX_EINVAL, "atom index out of range");
  if (X.nq == 0) return MDX_OK;
  // extended basis: shell s, s+ = n+s (l+1, coefficients 2 zeta c), s- = 2n+s (l-1, coefficients c):
  // d/dA_x of a primitive x_A^a e^(-zeta x_A^2) is 2 zeta x_A^(a+1) e - a x_A^(a-1) e
  const int32_t npr = basis->n_prims;
  std::vector<int32_t> po(n);
  std::vector<double> cen(3 * (size_t)n), ex(npr), co(npr);
  if (n) e = cudaMemcpyAsync(po.data(), basis->prim_off, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(cen.data(), basis->center, cen.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && npr) e = cudaMemcpyAsync(ex.data(), basis->exps, npr * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && npr) e = cudaMemcpyAsync(co.data(), basis->coefs, npr * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "basis download");
  std::vector<int32_t> L3(3 * (size_t)n), K3(3 * (size_t)n), PO3(3 * (size_t)n);
  std::vector<double> C3(9 * (size_t)n), E3, W3;
  for (int v = 0; v < 3; ++v)
    for (int32_t sh = 0; sh < n; ++sh) {
      const size_t t = (size_t)v * n + sh;
      L3[t] = v == 0 ? hb.l[sh] : (v == 1 ? hb.l[sh] + 1 : std::max(hb.l[sh] - 1, 0));
      K3[t] = hb.nprim[sh];
      PO3[t] = (int32_t)E3.size();
      for (int k = 0; k < 3; ++k) C3[3 * t + k] = cen[3 * (size_t)sh + k];
      for (int q = 0; q < hb.nprim[sh]; ++q) {
        const int32_t g = po[sh] + q;
        if (g < 0 || g >= npr) return fail(c, MDX_EINVAL, "primitive index out of range");
        E3.push_back(ex[g]);
        W3.push_back(v == 1 ? 2.0 * ex[g] * co[g] : co[g]);
      }
    }
  int32_t *dL3, *dK3, *dPO3, *datom; double *dC3, *dE3, *dW3;
  if ((st = upload(c, "g_l", L3, &dL3, s)) != MDX_OK) return st;
  if ((st = upload(c, "g_k", K3, &dK3, s)) != MDX_OK) return st;
  if ((st = upload(c, "g_po", PO3, &dPO3, s)) != MDX_OK) return st;
  if ((st = upload(c, "g_c", C3, &dC3, s)) != MDX_OK) return st;
  if ((st = upload(c, "g_e", E3, &dE3, s)) != MDX_OK) return st;
  if ((st = upload(c, "g_w", W3, &dW3, s)) != MDX_OK) return st;
  if ((st = upload(c, "g_atom", atom, &datom, s)) != MDX_OK) return st;
  const BasisDev b3{dL3, dK3, dPO3, dC3, dE3, dW3};
  // five record variants per pair: (i,j), (i+,j), (i-,j), (i,j+), (i,j-)
  std::vector<int64_t> prec(5 * X.np);
  std::vector<PrimPairJob> jobs;
  int64_t roff = 0;
  for (int v = 0; v < 5; ++v)
    for (int64_t p = 0; p < X.np; ++p) {
      int32_t i = X.pl[p].i, j = X.pl[p].j;
      if (v == 1) i += n; else if (v == 2) i += 2 * n; else if (v == 3) j += n; else if (v == 4) j += 2 * n;
      prec[v * X.np + p] = roff;
      for (int ia = 0; ia < K3[i]; ++ia)
        for (int ib = 0; ib < K3[j]; ++ib) {
          jobs.push_back(PrimPairJob{i, j, ia, ib, 0, 0, roff});
          roff += rec_size(L3[i], L3[j]);
        }
    }
  PrimPairJob* d_jobs; int64_t* d_prec; double *d_recs, *d_recs_s;
  if ((st = upload(c, "g_jobs", jobs, &d_jobs, s)) != MDX_OK) return st;
  if ((st = upload(c, "g_prec", prec, &d_prec, s)) != MDX_OK) return st;
  if ((st = ensure(c, "g_recs", (size_t)roff, &d_recs, s)) != MDX_OK) return st;
  if ((st = ensure(c, "g_recs_s", (size_t)roff, &d_recs_s, s)) != MDX_OK) return st;
  e = launch_pair_records(b3, b3, d_jobs, (int64_t)jobs.size(), d_recs, d_recs_s, c->d_err, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair records");
  // per bucket: three of the centres i, j, k, l raised (+) and lowered (-), and, if asked, the energy;
  // the fourth centre follows from translational invariance. A position's raised and lowered shells
  // are record variants 1/2 (first shell of the pair) or 3/4 (second shell) of its pair.
  struct Var { int bra, ket, pos, sign; };
  const Var all_vars[9] = {{1, 0, 0, 1}, {2, 0, 0, -1}, {3, 0, 1, 1}, {4, 0, 1, -1}, {0, 1, 2, 1},
                           {0, 2, 2, -1}, {0, 3, 3, 1}, {0, 4, 3, -1}, {0, 0, -1, 0}};
  // all plans first (their uploads go to s before the fork), then the launches
  // spread over the streams, heaviest first
  struct GradJob {
    QuartetLaunch a;
    double work;
    int64_t per, chunk;   // register path: doubles per shellset, shellsets per chunk (0: team kernel)
  };
  std::vector<GradJob> gjobs;
  int64_t ws_doubles = 0;
  const int nclass = (int)X.classes.size();
  for (int cp = 0; cp < nclass; ++cp)
    for (int cq = 0; cq <= cp; ++cq) {
      const int64_t b = (int64_t)cp * (cp + 1) / 2 + cq;
      if (X.counts[b] == 0) continue;
      const int l0[4] = {X.classes[cp][0], X.classes[cp][1], X.classes[cq][0], X.classes[cq][1]};
      // the centre left to translational invariance: the one whose shifted classes cost most (an s shell
      // has no lowered class, so a class with s shells drops a whole evaluation)
      int ginv = 0;
      double worst = -1.0;
      for (int pos = 0; pos < 4; ++pos) {
        double cost = 0.0;
        for (int sg = 1; sg >= -1; sg -= 2) {
          if (sg < 0 && l0[pos] == 0) continue;
          int ls[4] = {l0[0], l0[1], l0[2], l0[3]};
          ls[pos] += sg;
          cost += model_flops_class(ClassKey{ls[0], ls[1], ls[2], ls[3], X.classes[cp][2], X.classes[cq][2], 0});
        }
        if (cost > worst) { worst = cost; ginv = pos; }
      }
      for (const Var& v : all_vars) {
        if (v.pos < 0 && !energy) continue;
        if (v.pos == ginv) continue;
        if (v.sign < 0 && l0[v.pos] == 0) continue;   // no l-1 term for s shells
        int ls[4] = {l0[0], l0[1], l0[2], l0[3]};
        if (v.pos >= 0) ls[v.pos] += v.sign;
        const ClassKey key{ls[0], ls[1], ls[2], ls[3], X.classes[cp][2], X.classes[cq][2], 0};
        Plan* plan;
        if ((st = get_plan(c, key, &plan, s)) != MDX_OK) return st;
        QuartetLaunch a = base_launch(c, plan, X.d_quart + X.boff[b], (int64_t)X.counts[b], d_prec, d_recs, d_recs_s);
        a.bra_var_off = (int64_t)v.bra * X.np;
        a.ket_var_off = (int64_t)v.ket * X.np;
        a.D = D;
        a.nao = (int32_t)X.nao;
        a.ao_off = basis->ao_off;
        a.pair_shells = X.d_pshell;
        a.grad = grad;
        a.energy = energy;
        a.atom = datom;
        a.alpha = alpha;
        a.gpos = v.pos;
        a.gsign = v.sign;
        a.ginv = ginv;
        for (int k = 0; k < 4; ++k) a.lorig[k] = l0[k];
        GradJob g{a, model_flops_class(key) * (double)a.nq, 0, 0};
        if (plan->d.reg) {
          // register kernel: shifted shellsets to workspace (back to back), then the
          // gradient contraction, in chunks of at most 1 GiB of shellsets
          g.per = (int64_t)plan->d.Nb * plan->d.Nk;
          g.chunk = std::max<int64_t>(1, std::min<int64_t>(a.nq, (int64_t(1) << 27) / g.per));
          ws_doubles = std::max(ws_doubles, g.chunk * g.per);
        }
        gjobs.push_back(g);
      }
    }
  // one shellset workspace per stream
  static const char* const kWsName[mdx_ctx::kAux + 1] = {"g_shellsets0", "g_shellsets1", "g_shellsets2",
                                                          "g_shellsets3"};
  double* ws[mdx_ctx::kAux + 1] = {};
  if (ws_doubles > 0)
    for (int i = 0; i <= mdx_ctx::kAux; ++i)
      if ((st = ensure(c, kWsName[i], (size_t)ws_doubles, &ws[i], s)) != MDX_OK) return st;
  std::stable_sort(gjobs.begin(), gjobs.end(), [](const GradJob& x, const GradJob& y) { return x.work > y.work; });
  Fanout fan{c, s};
  e = fan.fork();
  for (size_t j = 0; j < gjobs.size() && e == cudaSuccess; ++j) {
    const GradJob& g = gjobs[j];
    const int si = fan.pick(g.work);
    const cudaStream_t gs = fan.stream(si);
    if (g.chunk == 0) {
      e = launch_quartets(g.a, gs);
      continue;
    }
    for (int64_t q0 = 0; q0 < g.a.nq && e == cudaSuccess; q0 += g.chunk) {
      QuartetLaunch part = g.a;
      part.qpairs = g.a.qpairs + q0;
      part.nq = std::min(g.chunk, g.a.nq - q0);
      QuartetLaunch st_part = part;
      st_part.D = nullptr;
      st_part.grad = nullptr;
      st_part.energy = nullptr;
      st_part.out = ws[si];
      st_part.qout = nullptr;
      e = launch_quartets(st_part, gs);
      if (e == cudaSuccess) e = launch_grad_contract(part, ws[si], gs);
    }
  }
  const cudaError_t ej = fan.join();
  if (e == cudaSuccess) e = ej;
  if (e != cudaSuccess) return cuda_fail(c, e, "gradient quartet launch");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "exchange gradient");
  return check_device_error(c, s);
}

int64_t mdx_last_quartet_count(const mdx_ctx* c) { return c ? c->last_quartets : -1; }

mdx_status mdx_plan_info(mdx_ctx* c, int la, int lb, int lc, int ld, int Kb, int Kk, int one_centre,
                         mdx_plan_stats* out) {
  if (!out) return MDX_EINVAL;
  if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > MDX_LMAX || lb > MDX_LMAX || lc > MDX_LMAX || ld > MDX_LMAX ||
      Kb < 1 || Kk < 1 || Kb > MDX_KMAX * MDX_KMAX || Kk > MDX_KMAX * MDX_KMAX)
    return fail(c, MDX_EUNSUPPORTED, "class outside the supported range");
  Plan p;
  std::string err;
  const ClassKey key{la, lb, lc, ld, Kb, Kk, one_centre ? 1 : 0};
  PlanConfig cfg{};
  if (c) {
    auto tc = c->tuned.find(key);
    if (tc != c->tuned.end()) cfg = tc->second;
  }
  if (!build_plan(key, cfg, p, err))
    return fail(c, MDX_EUNSUPPORTED, "planner: " + err);
  out->team_threads = p.d.T;
  out->teams_per_cta = p.d.teams_per_cta;
  out->smem_bytes_per_team = p.d.team_doubles * 8;
  out->n_groups = p.d.ngroups;
  out->exec_fma = p.exec_fma;
  out->register_kernel = p.d.reg;
  out->pad = 0;
  return MDX_OK;
}

mdx_status mdx_set_class_shape(mdx_ctx* c, int la, int lb, int lc, int ld, int Kb, int Kk, int one_centre,
                               int team_threads, int smem_budget, int variant) {
  if (!c) return MDX_EINVAL;
  if (la < 0 || lb < 0 || lc < 0 || ld < 0 || la > MDX_LMAX || lb > MDX_LMAX || lc > MDX_LMAX || ld > MDX_LMAX ||
      Kb < 1 || Kk < 1 || Kb > MDX_KMAX * MDX_KMAX || Kk > MDX_KMAX * MDX_KMAX)
    return fail(c, MDX_EUNSUPPORTED, "class outside the supported range");
  if (team_threads < 0 || smem_budget < 0 || smem_budget > 227 * 1024 || variant < 0 || variant > 2)
    return fail(c, MDX_EINVAL, "invalid shape");
  const ClassKey key{la, lb, lc, ld, Kb, Kk, one_centre ? 1 : 0};
  PlanConfig cfg{};
  cfg.T = team_threads;
  if (smem_budget > 0) cfg.budget = smem_budget;
  cfg.variant = variant;
  Plan p;
  std::string err;
  if (!build_plan(key, cfg, p, err)) return fail(c, MDX_EUNSUPPORTED, "planner: " + err);
  for (int store = 0; store <= 2; ++store) {   // the general, the store-only and the solid-harmonic plan
    ClassKey k2 = key;
    k2.store = store;
    c->tuned[k2] = cfg;
    auto it = c->plans.find(k2);
    if (it != c->plans.end()) {
      c->retired.push_back(std::move(it->second));
      c->plans.erase(it);
    }
  }
  return MDX_OK;
}


// ---------------------------------------------------------------- batched exchange
mdx_status mdx_xbatch_create(mdx_ctx* c, int32_t n_mol, const mdx_basis* bases, const double* const* D,
                             double* const* K, double tau, mdx_xbatch** out, void* stream) {
  const NvtxRange nvtx_range("mdx_xbatch_create");
  if (!c || !out) return MDX_EINVAL;
  *out = nullptr;
  c->last_error.clear();
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n_mol < 1 || !bases || !D || !K || !(tau >= 0.0)) return fail(c, MDX_EINVAL, "invalid arguments");
  std::unique_ptr<mdx_xbatch, void (*)(mdx_xbatch*)> X(new mdx_xbatch(), xbatch_free);
  X->ctx = c;
  X->nmol = n_mol;
  // super basis: every molecule's shells back to back; AO offsets stay local to the molecule
  std::vector<int32_t> L, NP, PO, AO, MOLSH, mol_nao(n_mol);
  std::vector<double> CEN, EX, CO;
  std::vector<int32_t> shell_first(n_mol + 1, 0);
  for (int m = 0; m < n_mol; ++m) {
    const mdx_basis& b = bases[m];
    if (!b.ao_off || b.n_shells < 1) return fail(c, MDX_EINVAL, "every molecule needs shells and ao_off");
    HostBasis hb;
    mdx_status st = fetch_basis(c, &b, hb, s);
    if (st != MDX_OK) return st;
    const int n = hb.n;
    std::vector<int32_t> po(n), ao(n);
    std::vector<double> cen(3 * (size_t)n), ex(b.n_prims), co(b.n_prims);
    cudaError_t e = cudaMemcpyAsync(po.data(), b.prim_off, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ao.data(), b.ao_off, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cen.data(), b.center, cen.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && b.n_prims) e = cudaMemcpyAsync(ex.data(), b.exps, ex.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && b.n_prims) e = cudaMemcpyAsync(co.data(), b.coefs, co.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "basis download");
    int64_t nao = 0;
    for (int i = 0; i < n; ++i) {
      nao = std::max<int64_t>(nao, (int64_t)ao[i] + ncart(hb.l[i]));
      L.push_back(hb.l[i]);
      NP.push_back(hb.nprim[i]);
      PO.push_back((int32_t)EX.size());
      AO.push_back(ao[i]);
      MOLSH.push_back(m);
      for (int k = 0; k < 3; ++k) CEN.push_back(cen[3 * (size_t)i + k]);
      for (int q = 0; q < hb.nprim[i]; ++q) {
        if (po[i] + q < 0 || po[i] + q >= b.n_prims) return fail(c, MDX_EINVAL, "primitive index out of range");
        EX.push_back(ex[po[i] + q]);
        CO.push_back(co[po[i] + q]);
      }
    }
    mol_nao[m] = (int32_t)nao;
    shell_first[m + 1] = shell_first[m] + n;
  }
  const int32_t ntot = shell_first[n_mol];
  mdx_status st;
  if ((st = dev_upload(c, L, &X->l, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, NP, &X->nprim, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, PO, &X->prim_off, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, AO, &X->ao_off, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, CEN, &X->center, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, EX, &X->exps, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, CO, &X->coefs, s)) != MDX_OK) return st;
  std::vector<const double*> hD(D, D + n_mol);
  std::vector<double*> hK(K, K + n_mol);
  if ((st = dev_upload(c, hD, &X->molD, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, hK, &X->molK, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, mol_nao, &X->molnao, s)) != MDX_OK) return st;
  X->max_nao = *std::max_element(mol_nao.begin(), mol_nao.end());
  const mdx_basis sb{ntot, (int32_t)EX.size(), X->l, X->nprim, X->prim_off, X->ao_off, nullptr, X->center, X->exps,
                     X->coefs};
  X->sb = sb;
  // all shell pairs i >= j of every molecule, sorted by (molecule, class)
  struct PP { int32_t i, j, m, li, lj, K; };
  std::vector<PP> pl;
  for (int m = 0; m < n_mol; ++m)
    for (int32_t i = shell_first[m]; i < shell_first[m + 1]; ++i)
      for (int32_t j = shell_first[m]; j <= i; ++j) pl.push_back(PP{i, j, m, L[i], L[j], NP[i] * NP[j]});
  std::stable_sort(pl.begin(), pl.end(), [](const PP& a, const PP& b) {
    if (a.m != b.m) return a.m < b.m;
    if (a.li != b.li) return a.li < b.li;
    if (a.lj != b.lj) return a.lj < b.lj;
    return a.K < b.K;
  });
  const int64_t np = (int64_t)pl.size();
  std::map<std::array<int, 3>, int> cid;
  std::vector<std::array<int, 3>> classes;
  std::vector<int2> pshell(np);
  std::vector<int32_t> pclass_raw(np), pmol(np);
  for (int64_t p = 0; p < np; ++p) {
    std::array<int, 3> k{pl[p].li, pl[p].lj, pl[p].K};
    auto it = cid.find(k);
    if (it == cid.end()) it = cid.emplace(k, 0).first;
    pshell[p] = make_int2(pl[p].i, pl[p].j);
    pmol[p] = pl[p].m;
  }
  // class ids ordered like the in-molecule sort, so class(q) <= class(p) for q <= p in a molecule
  { int k = 0; for (auto& kv : cid) { kv.second = k++; classes.push_back(kv.first); } }
  for (int64_t p = 0; p < np; ++p) pclass_raw[p] = cid[{pl[p].li, pl[p].lj, pl[p].K}];
  const int nclass = (int)classes.size();
  const int64_t nbucket = (int64_t)nclass * (nclass + 1) / 2;
  if ((st = dev_upload(c, pshell, &X->pshell, s)) != MDX_OK) return st;
  if ((st = dev_upload(c, pmol, &X->pmol, s)) != MDX_OK) return st;
  int32_t* d_pclass;
  if ((st = upload(c, "xb_pclass", pclass_raw, &d_pclass, s)) != MDX_OK) return st;
  if (np > 0x7fffffff) return fail(c, MDX_EUNSUPPORTED, "too many shell pairs");
  // Schwarz factors and primitive-pair records of every pair (records stay with the batch)
  std::vector<int64_t> prec(np);
  std::vector<PrimPairJob> jobs;
  int64_t roff = 0;
  std::vector<int32_t> nab(np);
  std::vector<int64_t> doffs(np + 1, 0);
  for (int64_t p = 0; p < np; ++p) {
    prec[p] = roff;
    for (int ia = 0; ia < NP[pl[p].i]; ++ia)
      for (int ib = 0; ib < NP[pl[p].j]; ++ib) {
        jobs.push_back(PrimPairJob{pl[p].i, pl[p].j, ia, ib, 0, 0, roff});
        roff += rec_size(pl[p].li, pl[p].lj);
      }
    nab[p] = ncart(pl[p].li) * ncart(pl[p].lj);
    doffs[p + 1] = doffs[p] + (int64_t)nab[p] * nab[p];
  }
  PrimPairJob* d_jobs;
  if ((st = dev_upload(c, prec, &X->prec, s)) != MDX_OK) return st;
  if ((st = upload(c, "xb_jobs", jobs, &d_jobs, s)) != MDX_OK) return st;
  if (cudaMalloc(&X->recs, roff * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&X->recs_s, roff * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MDX_ENOMEM, "record allocation failed");
  }
  const BasisDev bd{X->l, X->nprim, X->prim_off, X->center, X->exps, X->coefs};
  cudaError_t e = launch_pair_records(bd, bd, d_jobs, (int64_t)jobs.size(), X->recs, X->recs_s, c->d_err, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair records");
  {
    // diagonal quartets (ij|ij) for Q_ij, per class
    std::map<ClassKey, std::vector<int64_t>> dcls;
    for (int64_t p = 0; p < np; ++p)
      dcls[ClassKey{pl[p].li, pl[p].lj, pl[p].li, pl[p].lj, pl[p].K, pl[p].K, 0}].push_back(p);
    double* d_vals; int64_t* d_doff; int32_t* d_nab; int2* d_dq; int64_t* d_dqo;
    std::vector<int2> dq;
    std::vector<int64_t> dqo;
    for (auto& kv : dcls) for (int64_t p : kv.second) { dq.push_back(make_int2((int)p, (int)p)); dqo.push_back(doffs[p]); }
    if ((st = ensure(c, "xb_dvals", (size_t)doffs[np], &d_vals, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_doff", doffs, &d_doff, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_nab", nab, &d_nab, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_dq", dq, &d_dq, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_dqo", dqo, &d_dqo, s)) != MDX_OK) return st;
    int64_t at = 0;
    for (auto& kv : dcls) {
      Plan* plan;
      if ((st = get_plan(c, kv.first, &plan, s)) != MDX_OK) return st;
      QuartetLaunch a = base_launch(c, plan, d_dq + at, (int64_t)kv.second.size(), X->prec, X->recs, X->recs_s);
      a.qout = d_dqo + at;
      a.out = d_vals;
      e = launch_quartets(a, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "Schwarz quartets");
      at += (int64_t)kv.second.size();
    }
    double* d_Q;
    if ((st = ensure(c, "xb_Q", (size_t)np, &d_Q, s)) != MDX_OK) return st;
    e = launch_schwarz_reduce(d_doff, d_nab, np, d_vals, d_Q, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Schwarz reduce");
    std::vector<double> hQ(np);
    e = cudaMemcpyAsync(hQ.data(), d_Q, np * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Schwarz");
    // segments of one molecule and one class (contiguous in pair order), each listed by decreasing Q
    std::vector<int32_t> order(np), seg_class, mol_seg(n_mol + 1, 0);
    std::vector<int64_t> pos(np), seg_begin;
    for (int64_t p = 0; p < np; ++p) {
      if (p == 0 || pl[p].m != pl[p - 1].m || pclass_raw[p] != pclass_raw[p - 1]) {
        seg_begin.push_back(p);
        seg_class.push_back(pclass_raw[p]);
        for (int m = pl[p].m + 1; m <= n_mol; ++m) mol_seg[m] = (int32_t)seg_class.size();
      }
      order[p] = (int32_t)p;
    }
    seg_begin.push_back(np);
    for (size_t g = 0; g + 1 < seg_begin.size(); ++g)
      std::stable_sort(order.begin() + seg_begin[g], order.begin() + seg_begin[g + 1],
                       [&](int32_t x, int32_t y) { return hQ[x] > hQ[y]; });
    for (int64_t i = 0; i < np; ++i) pos[order[i]] = i;
    // density-block maxima: one [n_m][n_m] table per molecule, back to back
    std::vector<int64_t> dmax_off(n_mol + 1, 0);
    for (int m = 0; m < n_mol; ++m) {
      const int64_t nm = shell_first[m + 1] - shell_first[m];
      dmax_off[m + 1] = dmax_off[m] + nm * nm;
    }
    int32_t *d_order, *d_segc, *d_molseg, *d_sfirst;
    int64_t *d_pos, *d_segb, *d_dmoff;
    double *d_dmax, *d_rowmax;
    if ((st = upload(c, "xb_order", order, &d_order, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_pos", pos, &d_pos, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_segb", seg_begin, &d_segb, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_segc", seg_class, &d_segc, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_molseg", mol_seg, &d_molseg, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_sfirst", shell_first, &d_sfirst, s)) != MDX_OK) return st;
    if ((st = upload(c, "xb_dmoff", dmax_off, &d_dmoff, s)) != MDX_OK) return st;
    if ((st = ensure(c, "xb_dmax", (size_t)std::max<int64_t>(dmax_off[n_mol], 1), &d_dmax, s)) != MDX_OK) return st;
    if ((st = ensure(c, "xb_rowmax", (size_t)std::max<int32_t>(ntot, 1), &d_rowmax, s)) != MDX_OK) return st;
    for (int m = 0; m < n_mol; ++m) {
      const int32_t f = shell_first[m], nm = shell_first[m + 1] - f;
      e = launch_dmax(D[m], mol_nao[m], X->ao_off + f, X->l + f, nm, d_dmax + dmax_off[m], nm, s);
      if (e == cudaSuccess) e = launch_rowmax(d_dmax + dmax_off[m], nm, d_rowmax + f, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "density maxima");
    }
    unsigned long long* d_counts;
    if ((st = ensure(c, "xb_counts", (size_t)nbucket, &d_counts, s)) != MDX_OK) return st;
    e = cudaMemsetAsync(d_counts, 0, nbucket * sizeof(unsigned long long), s);
    ScreenArgs sa{};
    sa.npairs = np;
    sa.pair_shells = X->pshell;
    sa.Q = d_Q;
    sa.pair_class = d_pclass;
    sa.pos = d_pos;
    sa.order = d_order;
    sa.seg_begin = d_segb;
    sa.seg_class = d_segc;
    sa.mol_seg = d_molseg;
    sa.pair_mol = X->pmol;
    sa.shell_first = d_sfirst;
    sa.dmax_off = d_dmoff;
    sa.dmax = d_dmax;
    sa.rowmax = d_rowmax;
    sa.nclass = nclass;
    sa.tau = tau;
    sa.counts = d_counts;
    if (e == cudaSuccess) e = launch_screen(sa, false, s);
    std::vector<unsigned long long> counts(nbucket);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts.data(), d_counts, nbucket * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "screening");
    std::vector<int64_t> boff(nbucket + 1, 0);
    for (int64_t b = 0; b < nbucket; ++b) boff[b + 1] = boff[b] + (int64_t)counts[b];
    X->nq = boff[nbucket];
    if (X->nq > 0) {
      int64_t* d_boff;
      if ((st = upload(c, "xb_boff", boff, &d_boff, s)) != MDX_OK) return st;
      if (cudaMalloc(&X->quart, X->nq * sizeof(int2)) != cudaSuccess) { cudaGetLastError(); return fail(c, MDX_ENOMEM, "quartet list"); }
      e = cudaMemsetAsync(d_counts, 0, nbucket * sizeof(unsigned long long), s);
      sa.bucket_off = d_boff;
      sa.out = X->quart;
      if (e == cudaSuccess) e = launch_screen(sa, true, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "screening");
    }
    // one launch descriptor per non-empty bucket, plus the persistent work items
    std::vector<WorkItem> items;
    std::vector<double> cost;
    std::vector<char> item_reg;   // the item's class has a register kernel
    int64_t smem = 0, smem_team = 0;
    for (int cp = 0; cp < nclass; ++cp)
      for (int cq = 0; cq <= cp; ++cq) {
        const int64_t b = (int64_t)cp * (cp + 1) / 2 + cq;
        if (counts[b] == 0) continue;
        const ClassKey key{classes[cp][0], classes[cp][1], classes[cq][0], classes[cq][1], classes[cp][2],
                           classes[cq][2], 0};
        Plan* plan;
        if ((st = get_plan(c, key, &plan, s)) != MDX_OK) return st;
        QuartetLaunch a = base_launch(c, plan, X->quart + boff[b], (int64_t)counts[b], X->prec, X->recs, X->recs_s);
        a.D = D[0];                     // any non-null D selects the digestion epilogue
        a.ao_off = X->ao_off;
        a.pair_shells = X->pshell;
        a.pair_mol = X->pmol;
        a.mol_D = X->molD;
        a.mol_K = X->molK;
        a.mol_nao = X->molnao;
        X->launches.push_back(a);
        X->lkey.push_back(key);
        X->lflops.push_back(model_flops_class(key) * (double)counts[b]);
        X->model_flops += X->lflops.back();
        // persistent shape: the class's own team size T, as many teams as fit the block's
        // threads and kPersistSmem of shared memory (two blocks per SM), in whole warps (the
        // kernel's barriers are warp-uniform); a plan whose teams do not fill one warp is
        // rebuilt with at least 32 threads per team and a smaller budget
        Plan* pp = plan;
        auto shape = [](const PlanDev& d) {
          if (d.T > kPersistBlock) return 0;
          int tpb = (int)std::min<int64_t>(kPersistBlock / d.T, kPersistSmem / ((int64_t)d.team_doubles * 8));
          if (d.T < 32) tpb -= tpb % (32 / d.T);
          return tpb;
        };
        int tpb = shape(plan->d);
        if (tpb < 1) {
          std::unique_ptr<Plan> np2(new Plan());
          std::string err;
          PlanConfig cfg{};
          auto tc = c->tuned.find(key);
          if (tc != c->tuned.end()) cfg = tc->second;
          cfg.T = std::min(std::max(plan->d.T, 32), kPersistBlock);
          cfg.budget = std::min<int>(cfg.budget, (int)kPersistSmem);
          cfg.single_max = std::min(cfg.single_max, cfg.budget);
          cfg.variant = 1;
          bool ok = build_plan(key, cfg, *np2, err) && shape(np2->d) >= 1;
          if (!ok && cfg.T != kPersistBlock) {   // one block-wide team
            cfg.T = kPersistBlock;
            ok = build_plan(key, cfg, *np2, err) && shape(np2->d) >= 1;
          }
          if (!ok) return fail(c, MDX_EUNSUPPORTED, "persistent planner: " + err);
          if ((st = upload_plan(c, np2.get(), s)) != MDX_OK) return st;
          pp = np2.get();
          tpb = shape(pp->d);
          c->retired.push_back(std::move(np2));
        }
        QuartetLaunch ap = a;
        ap.plan = pp->d;
        ap.plan.teams_per_cta = tpb;
        X->plaunches.push_back(ap);
        const bool reg_class = plan->d.reg != 0;
        const int64_t need = (int64_t)pp->d.team_doubles * 8 * tpb;
        smem = std::max(smem, need);
        if (!reg_class) smem_team = std::max(smem_team, need);
        const int per_item = tpb * kPersistRounds;
        for (int64_t q0 = 0; q0 < (int64_t)counts[b]; q0 += per_item) {
          const int cnt = (int)std::min<int64_t>(per_item, (int64_t)counts[b] - q0);
          items.push_back(WorkItem{(int32_t)(X->plaunches.size() - 1), cnt, q0});
          cost.push_back(pp->exec_fma * cnt);
          item_reg.push_back(reg_class);
        }
        if (reg_class) X->reg_launches.push_back((int32_t)(X->launches.size() - 1));
      }
    // heaviest items first (the queue hands them out in order)
    std::vector<size_t> iorder(items.size());
    for (size_t i = 0; i < iorder.size(); ++i) iorder[i] = i;
    std::stable_sort(iorder.begin(), iorder.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    // all items (mode 1), and the items of the classes without a register kernel (mode 2)
    std::vector<WorkItem> sorted, sorted_team;
    for (size_t i : iorder) {
      sorted.push_back(items[i]);
      if (!item_reg[i]) sorted_team.push_back(items[i]);
    }
    X->nitems = (int64_t)sorted.size();
    X->nitems_team = (int64_t)sorted_team.size();
    X->smem = smem;
    X->smem_team = smem_team;
    if ((st = dev_upload(c, X->plaunches, &X->d_plaunches, s)) != MDX_OK) return st;
    if ((st = dev_upload(c, sorted, &X->items, s)) != MDX_OK) return st;
    if (!sorted_team.empty() && (st = dev_upload(c, sorted_team, &X->items_team, s)) != MDX_OK) return st;
    if (cudaMalloc(&X->counter, sizeof(unsigned long long)) != cudaSuccess) { cudaGetLastError(); return fail(c, MDX_ENOMEM, "counter"); }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    auto grid_for = [&](int64_t shm) {
      int bps = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, persistent_kernel_ptr(), kPersistBlock, (size_t)std::max<int64_t>(shm, 1));
      return std::max(1, bps) * std::max(1, sms);
    };
    X->grid = grid_for(smem);
    X->grid_team = grid_for(smem_team);
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "batched exchange set-up");
  st = check_device_error(c, s);
  if (st != MDX_OK) return st;
  *out = X.release();
  return MDX_OK;
}

mdx_status mdx_xbatch_info(const mdx_xbatch* xb, int64_t* n_quartets, int64_t* n_items, int32_t* n_class_launches,
                           double* model_flops) {
  if (!xb) return MDX_EINVAL;
  if (model_flops) *model_flops = xb->model_flops;
  if (n_quartets) *n_quartets = xb->nq;
  if (n_items) *n_items = xb->nitems;
  if (n_class_launches) *n_class_launches = (int32_t)xb->launches.size();
  return MDX_OK;
}

mdx_status mdx_xbatch_run(mdx_ctx* c, mdx_xbatch* xb, int32_t persistent, int32_t* n_launches, void* stream) {
  const NvtxRange nvtx_range("mdx_xbatch_run");
  if (!c || !xb || xb->ctx != c || persistent < 0 || persistent > 2) return MDX_EINVAL;
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  int32_t nl = 0;
  cudaError_t e = launch_multi_k(xb->molK, xb->molnao, xb->nmol, xb->max_nao, true, s);
  ++nl;
  if (e == cudaSuccess && xb->nq > 0) {
    if (persistent == 1) {
      e = cudaMemsetAsync(xb->counter, 0, sizeof(unsigned long long), s);
      PersistLaunch pl{xb->d_plaunches, xb->items, xb->nitems, xb->counter};
      if (e == cudaSuccess) e = launch_persistent(pl, xb->smem, xb->grid, s);
      ++nl;
    } else if (persistent == 2) {
      // register-kernel classes one launch each, then one persistent launch for the rest
      for (int32_t i : xb->reg_launches) {
        e = launch_quartets(xb->launches[i], s);
        if (e != cudaSuccess) break;
        ++nl;
      }
      if (e == cudaSuccess && xb->nitems_team > 0) {
        e = cudaMemsetAsync(xb->counter, 0, sizeof(unsigned long long), s);
        PersistLaunch pl{xb->d_plaunches, xb->items_team, xb->nitems_team, xb->counter};
        if (e == cudaSuccess) e = launch_persistent(pl, xb->smem_team, xb->grid_team, s);
        ++nl;
      }
    } else {
      for (const QuartetLaunch& a : xb->launches) {
        e = launch_quartets(a, s);
        if (e != cudaSuccess) break;
        ++nl;
      }
    }
  }
  if (e == cudaSuccess) e = launch_multi_k(xb->molK, xb->molnao, xb->nmol, xb->max_nao, false, s);
  ++nl;
  if (e != cudaSuccess) return cuda_fail(c, e, "batched exchange launch");
  if (n_launches) *n_launches = nl;
  return MDX_OK;
}

mdx_status mdx_xbatch_autotune(mdx_ctx* c, mdx_xbatch* xb, int64_t max_trial, void* stream) {
  const NvtxRange nvtx_range("mdx_xbatch_autotune");
  if (!c || !xb || xb->ctx != c || max_trial < 1) return MDX_EINVAL;
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto done = [&](mdx_status st) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  };
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < xb->launches.size(); ++i) {
    QuartetLaunch& a0 = xb->launches[i];
    if (a0.nq == 0) continue;
    const ClassKey& key = xb->lkey[i];
    // the digestion launch's shapes: register kernel where the class has one, team sizes (with budgets
    // and the cached R tables for classes of several column groups)
    std::vector<PlanConfig> cands;
    if (reg_eligible(key.la, key.lb, key.lc, key.ld) || reg_xs_eligible(key.la, key.lb, key.lc, key.ld))
      cands.push_back(PlanConfig{0, 200 * 1024, 96 * 1024, 2, -1});
    if (a0.plan.ngroups > 1) {
      for (int budget : {200 * 1024, 108 * 1024})
        for (int T : {128, 256, 512})
          for (int rc : {-1, 0, 1}) cands.push_back(PlanConfig{T, budget, 96 * 1024, 1, rc});
    } else {
      for (int T : {0, 4, 8, 16, 32, 64, 128, 256}) cands.push_back(PlanConfig{T, 200 * 1024, 96 * 1024, 1, -1});
    }
    float best_ms = 1e30f;
    PlanConfig best{};
    std::unique_ptr<Plan> best_plan;
    std::vector<std::array<int, 6>> seen;
    for (const PlanConfig& cfg : cands) {
      std::unique_ptr<Plan> p(new Plan());
      std::string err;
      if (!build_plan(key, cfg, *p, err)) continue;
      if (!p->d.reg && !p->d.has_out) continue;   // the digestion epilogue reads OUT
      const std::array<int, 6> sig{p->d.reg, p->d.T, p->d.teams_per_cta, p->d.team_doubles, p->d.ngroups,
                                   p->d.cache_R};
      if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
      seen.push_back(sig);
      mdx_status st = upload_plan(c, p.get(), s);
      if (st != MDX_OK) { if (p->dev_blob) cudaFree(p->dev_blob); return done(st); }
      QuartetLaunch a = a0;
      a.plan = p->d;
      a.nq = std::min(a0.nq, max_trial);
      float ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        e = launch_quartets(a, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { cudaFree(p->dev_blob); return done(cuda_fail(c, e, "autotune")); }
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = cfg;
        if (best_plan && best_plan->dev_blob) cudaFree(best_plan->dev_blob);
        best_plan = std::move(p);
      } else {
        cudaFree(p->dev_blob);
      }
    }
    if (!best_plan) continue;
    c->tuned[key] = best;
    auto it = c->plans.find(key);
    if (it != c->plans.end()) c->retired.push_back(std::move(it->second));
    a0.plan = best_plan->d;
    c->plans[key] = std::move(best_plan);
  }
  // the trial launches added into K: the next mdx_xbatch_run zeroes it first
  done(MDX_OK);
  return check_device_error(c, s);
}

mdx_status mdx_xbatch_launch_info(const mdx_xbatch* xb, int32_t i, int32_t* lk, int64_t* n_quartets,
                                  double* model_flops) {
  if (!xb || i < 0 || i >= (int32_t)xb->launches.size()) return MDX_EINVAL;
  const ClassKey& k = xb->lkey[i];
  if (lk) {
    lk[0] = k.la; lk[1] = k.lb; lk[2] = k.lc; lk[3] = k.ld; lk[4] = k.Kb; lk[5] = k.Kk;
  }
  if (n_quartets) *n_quartets = xb->launches[i].nq;
  if (model_flops) *model_flops = xb->lflops[i];
  return MDX_OK;
}

mdx_status mdx_xbatch_run_class(mdx_ctx* c, mdx_xbatch* xb, int32_t i, void* stream) {
  const NvtxRange nvtx_range("mdx_xbatch_run_class");
  if (!c || !xb || xb->ctx != c || i < 0 || i >= (int32_t)xb->launches.size()) return MDX_EINVAL;
  cudaSetDevice(c->device);
  const cudaError_t e = launch_quartets(xb->launches[i], (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "batched exchange class launch");
  return MDX_OK;
}

void mdx_xbatch_destroy(mdx_xbatch* xb) { xbatch_free(xb); }

}  // extern "C"
