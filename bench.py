"""Benchmark: McMurchie-Davidson 4-center ERI class sweep on one GB300.

Workload (one "step"): the per-class microbenchmark of Asadchev & Valeev
(arXiv:2405.01834, Sec. 5) in Cartesian form -- for each class [pp|pp],
[dd|dd], [ff|ff], [gg|gg], [hh|hh], [ii|ii], a 224 x 224 grid (50,176
quartets) of random uncontracted bra and ket shell pairs (centres uniform in
a 10-bohr box, exponents log-uniform in [0.05, 50]); outputs are written to a
reused device buffer in chunks (the [ii|ii] class alone is 247 GB).

Metric: FP64 GFLOP/s and shell quartets per second, per class and for the
whole sweep, with the fraction of the GB300 FP64 peak. `value` counts the work
in the paper's Table 1 FLOP model (contracted Cartesian shellsets), the unit
both arms share; the kernels execute several times fewer FP64 operations
(axis-factored transforms), so the roofline fraction is taken on the FP64
multiply-adds they do execute, against the FP64 peak measured in the same run
(scalar DFMA and the FP64 tensor instruction, the larger of the two).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2405_01834_gb300 import flops, inputs  # noqa: E402

CLASS_NAMES = {1: "[pp|pp]", 2: "[dd|dd]", 3: "[ff|ff]", 4: "[gg|gg]", 5: "[hh|hh]", 6: "[ii|ii]"}
METRIC = "FP64 GFLOP/s and shell-quartets/s per (la,lb,lc,ld) class; % of GB300 FP64 peak"
UNIT = "GFLOP/s (Table-1 model FLOPs)"
# GB300 FP64 pipe: 2 FP64 multiply-adds per clock per SM, 152 SMs; used only for the derived
# peak that is reported beside the measured one
FP64_FLOP_PER_CLK_SM = 4.0
CHUNK_BYTES = 2 << 30
# DRAM bytes (read + write) per [ii|ii] quartet of one k_quartets launch of the benchmark (456 quartets,
# autotuned plan): ncu --nvtx --nvtx-include "mdx_batch_run/" -k regex:k_quartets -c 1 --metrics
# dram__bytes_read.sum,dram__bytes_write.sum on `bench.py --classes 6 --n-bra 24 --n-ket 19 --steps 1
# --warmup 3 --no-cpu --no-e2e`: 5,659,966,464 B read + 7,211,322,368 B written
NCU_DRAM_BYTES_PER_II_QUARTET = (5659966464 + 7211322368) / 456


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mdx", choices=["mdx", "reference"])
    ap.add_argument("--classes", default="1,2,3,4,5,6")
    ap.add_argument("--n-bra", type=int, default=224)
    ap.add_argument("--n-ket", type=int, default=224)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the per-class team-shape autotuner")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=float, default=0.01, help="fraction of each class the oracle times")
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "xbatch", "df", "grad", "ab", "peak", "sph", "sph3", "counts", "xchain"],
                    help="sweep: the 4-center class sweep (default); xbatch: batched exchange of many molecules; "
                         "df: per-class 3-center rates on the density-fitting cluster; grad: exchange energy "
                         "and its nuclear gradient against the exchange build alone; ab: the default kernels "
                         "against the materialized-Hermite variant (dense [p|q], batched DGEMMs); "
                         "peak: measured FP64 throughput, scalar DFMA vs the FP64 tensor instruction; sph: "
                         "solid-harmonic rates per class of the paper's Tab. nps4; sph3: the same for 3-center [a|cd] "
                         "(Tab. nps3); counts: screened quartets and "
                         "projected time of the full-size exchange workloads; xchain: the exchange build on a long "
                         "chain molecule whose D and K are far larger than L2")
    ap.add_argument("--ab-grid", type=int, default=32, help="ab: bra x ket grid per class")
    ap.add_argument("--df-sample", type=int, default=65536, help="df: triplets timed per team-kernel class")
    ap.add_argument("--df-sample-reg", type=int, default=262144,
                    help="df: triplets timed per register-kernel class (one thread per triplet)")
    ap.add_argument("--df-sph", action="store_true", help="df: solid-harmonic functions (mdx_batch_eri3_sph)")
    ap.add_argument("--grad-atoms", type=int, default=8, help="grad: atoms of the cluster molecule")
    ap.add_argument("--n-mol", type=int, default=64)
    ap.add_argument("--atoms", default="2,5", help="xbatch: atoms per molecule, uniform in [lo,hi]")
    ap.add_argument("--tau", type=float, default=1e-11)
    ap.add_argument("--chain-atoms", type=int, default=500, help="xchain: atoms of the chain")
    ap.add_argument("--chain-k", type=int, default=1, help="xchain: contraction of every shell")
    ap.add_argument("--sph-classes", default="", help="sph: only these classes, e.g. 6666,4040")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    ls = [int(x) for x in args.classes.split(",") if x]
    out = []
    for l in ls:
        b, q = inputs.class_sweep((l, l, l, l), n_bra=args.n_bra, n_ket=args.n_ket)
        out.append((l, b, q))
    return out


def chunk_quartets(l: int, n: int, sms: int) -> int:
    """Quartets per launch: output within CHUNK_BYTES, and a whole number of waves of one team per SM
    (the large classes run one CTA per SM, so a launch of k*SMs quartets has no partial last wave)."""
    per_q = inputs.ncart(l) ** 4 * 8
    cq = max(1, min(n, CHUNK_BYTES // per_q))
    if n > cq >= 2 * sms:
        down = cq - cq % sms
        up = down + sms   # the nearer whole number of waves, up to 12.5 % over the byte budget
        cq = up if (up - cq < cq - down and up * per_q <= CHUNK_BYTES * 1.125) else down
    return min(cq, n)


def model_flops(l, n):
    return flops.eri4_flops(l, l, l, l) * n


def autotune_trial(l: int, n: int) -> int:
    """Quartets the autotuner times per candidate shape: enough to fill the GPU with one-thread-per-
    quartet candidates at low l."""
    return max(304, min(n, 65536 // max(1, l) ** 3))


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """Slowest rank's step time (every rank runs its own replica of the workload)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_step: float) -> float:
    """Weak scaling: all ranks' units divided by the slowest rank's time (units/s)."""
    return world * units_per_rank / (ms_step * 1e-3)


# ------------------------------------------------------------------ oracle arm
def run_oracle(work, frac, seed=2024, nthreads=0, keep=None):
    """Time the oracle on a seeded sample of each class (nthreads = 0: all host cores); returns
    (model flops, seconds, quartets, per-class results). keep: dict that receives, per class l, the
    sampled quartet indices and the oracle's shellsets and offsets."""
    import oracle
    oracle.build()
    rng = np.random.Generator(np.random.PCG64(seed))
    tot_f = tot_t = 0.0
    tot_q = 0
    per = {}
    for l, b, q in work:
        m = max(1, int(round(frac * len(q))))
        idx = np.sort(rng.choice(len(q), m, replace=False))
        t0 = time.perf_counter()
        vals, off = oracle.eri4(b, q[idx], nthreads=nthreads)
        dt = time.perf_counter() - t0
        if keep is not None:
            keep[l] = (idx, vals, off)
        f = model_flops(l, m)
        tot_f += f; tot_t += dt; tot_q += m
        per[CLASS_NAMES[l]] = {"quartets": m, "s": round(dt, 4), "model_gflops": round(f / dt * 1e-9, 4)}
    return tot_f, tot_t, tot_q, per


def omp_threads():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def sweep_config(args, world: int) -> dict:
    """The class-sweep workload as both arms name it in their line."""
    return {"workload": "4-center class sweep [pp|pp]..[ii|ii], %dx%d random uncontracted quartets per class, "
                        "Cartesian, FP64" % (args.n_bra, args.n_ket),
            "classes": args.classes, "parallelism": "replicas" if world > 1 else "1 GPU"}


def reference_main(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    work = workload(args)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        run_oracle(work, min(args.cpu_sample, 0.002), seed=1)
    t_f = t_t = 0.0
    nq = 0
    # the per-step sample shrinks beyond 4 steps so that the whole run stays within about 4 steps' work
    frac = args.cpu_sample * min(1.0, 4.0 / max(1, args.steps))
    for s in range(args.steps):
        f, t, q, _ = run_oracle(work, frac, seed=100 + s)
        t_f += f; t_t += t; nq += q
    v = t_f / t_t * 1e-9
    sample = "seeded %.3f%% of each class's %d quartets per step (%d quartets over %d steps)" % (
        100 * frac, args.n_bra * args.n_ket, nq, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_t / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": sweep_config(args, world),
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0])); mx = max(mx, float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
def xbatch_main(args):
    """Exchange builds of n_mol uneven molecules (heavy 5s4p3d2f1g / light 4s3p2d1f shells, K = 6 s shells,
    D = C C^T): per-molecule mdx_exchange calls vs one launch per class vs one persistent launch vs the
    register-kernel classes per class plus one persistent launch for the rest, the last two also
    replayed from a CUDA graph; then the per-class launches after the batched-exchange autotuner."""
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    eng = mdx.Engine(0)
    lo, hi = (int(x) for x in args.atoms.split(","))
    rng = np.random.Generator(np.random.PCG64(1004))
    sizes = rng.integers(lo, hi + 1, args.n_mol)
    mols = [inputs.molecule(1004 * 1000 + i, int(n)) for i, n in enumerate(sizes)]
    bases = [mdx.DeviceBasis(b) for b in mols]
    Ds = [torch.from_numpy(inputs.density(b.nao, 7 + i)) for i, b in enumerate(mols)]
    pairs = [torch.tensor([(i, j) for i in range(b.n_shells) for j in range(i + 1)], dtype=torch.int32,
                          device="cuda") for b in mols]
    res = {}
    # (a) one mdx_exchange call per molecule (Schwarz factors computed once, outside the timing)
    Qs = [eng.schwarz(db, p) for db, p in zip(bases, pairs)]
    Dd = [D.cuda() for D in Ds]
    for _ in range(max(1, args.warmup)):
        for db, p, Q, D in zip(bases, pairs, Qs, Dd):
            eng.exchange(db, p, Q, D, args.tau)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for db, p, Q, D in zip(bases, pairs, Qs, Dd):
            eng.exchange(db, p, Q, D, args.tau)
    torch.cuda.synchronize()
    res["per_molecule_calls_ms"] = round(1e3 * (time.perf_counter() - t0) / args.steps, 3)
    xb = eng.xbatch(bases, Ds, tau=args.tau)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    launches = {name: xb.run(persistent=mode) for mode, name in ((0, "per_class"), (1, "persistent"), (2, "hybrid"))}
    res["per_class_launches_ms"] = round(timed(lambda: xb.run(persistent=0)), 3)
    res["persistent_ms"] = round(timed(lambda: xb.run(persistent=1)), 3)
    res["hybrid_ms"] = round(timed(lambda: xb.run(persistent=2)), 3)
    for mode, name in ((0, "per_class_graph_ms"), (1, "persistent_graph_ms"), (2, "hybrid_graph_ms")):
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                xb.run(persistent=mode)
        torch.cuda.synchronize()
        res[name] = round(timed(g.replay), 3)
    # the per-class launches again after the autotuner (register kernel or team shape per class, digestion
    # epilogue, timed on up to 65,536 quartets of each class)
    tune_s = None
    if not args.no_tune:
        t0 = time.perf_counter()
        xb.autotune(max_trial=65536)
        torch.cuda.synchronize()
        tune_s = round(time.perf_counter() - t0, 2)
        res["per_class_launches_autotuned_ms"] = round(timed(lambda: xb.run(persistent=0)), 3)
        res["hybrid_autotuned_ms"] = round(timed(lambda: xb.run(persistent=2)), 3)
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                xb.run(persistent=0)
        torch.cuda.synchronize()
        res["per_class_autotuned_graph_ms"] = round(timed(g.replay), 3)
    # per-class breakdown: every class launch alone, bracketed by events (one pass after the runs above)
    n_l = xb.n_class_launches
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(n_l + 1)]
    evs[0].record(stream)
    for i in range(n_l):
        xb.run_class(i)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    by_class = {}
    for i in range(n_l):
        lk, nq, mf = xb.launch_info(i)
        key = "[%d%d|%d%d]" % lk[:4]
        r = by_class.setdefault(key, [0.0, 0, 0.0])
        r[0] += evs[i].elapsed_time(evs[i + 1])
        r[1] += nq
        r[2] += mf
    tot_ms = sum(r[0] for r in by_class.values())
    per_class = [{"class": k, "ms": round(r[0], 3), "share": round(r[0] / tot_ms, 4), "quartets": r[1],
                  "quartets_per_s": round(r[1] / (r[0] * 1e-3), 1),
                  "model_gflops": round(r[2] / (r[0] * 1e-3) * 1e-9, 2)}
                 for k, r in sorted(by_class.items(), key=lambda kv: -kv[1][0])]
    eng.sync()
    best = min(v for k, v in res.items() if k != "per_molecule_calls_ms")
    line = {"metric": "batched exchange build: model FP64 GFLOP/s and shell quartets/s", "unit": UNIT,
            "value": round(xb.model_flops / (best * 1e-3) * 1e-9, 3), "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "exchange K_m of %d molecules of %d-%d atoms (heavy 5s4p3d2f1g / light 4s3p2d1f, "
                                   "K = 6 s shells), tau = %g" % (args.n_mol, lo, hi, args.tau),
                       "n_ao_total": int(sum(b.nao for b in mols))},
            "quartets": xb.n_quartets, "model_flops": xb.model_flops, "work_items": xb.n_items,
            "class_launches": xb.n_class_launches, "kernel_launches_per_build": launches, "modes_ms": res,
            "autotune_s": tune_s,
            "quartets_per_s": {k.replace("_ms", ""): round(xb.n_quartets / (v * 1e-3), 1) for k, v in res.items()},
            "per_class": per_class}
    print(json.dumps(line), flush=True)
    xb.close()
    eng.close()


def _event_ms(torch, stream, fn, steps, warmup):
    for _ in range(max(1, warmup)):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def df_grid(n_aux: int, n_pairs: int, target: int):
    """Auxiliary shells x kept pairs of one class's timing grid: up to 64 auxiliary shells and as many pairs
    as make about `target` triplets; a class with few kept pairs takes more auxiliary shells instead."""
    na = min(n_aux, 64)
    npr = max(1, min(n_pairs, target // na))
    na = min(n_aux, max(na, -(-target // npr)))
    return na, npr


def df_main(args):
    """3-center [a|cd] rates per class on the density-fitting cluster (100 atoms, orbital 4s3p2d1f at
    K 6/3/1/1, auxiliary s..i): orbital pairs Schwarz-screened at 1e-12, then for every (l_a | l_c l_d)
    class a seeded grid of auxiliary shells x kept pairs of the class is timed alone; the full tensor's
    time is extrapolated from the per-class rates. The grid holds up to --df-sample triplets for classes of
    the team kernel (a team per triplet) and up to --df-sample-reg for classes of the register kernel (a
    thread per triplet), so that either launch fills every SM several times over."""
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    eng = mdx.Engine(0)
    aux, orb = inputs.df_cluster()
    dorb, daux = mdx.DeviceBasis(orb), mdx.DeviceBasis(aux)
    ii, jj = np.tril_indices(orb.n_shells)
    pairs = np.stack([ii, jj], axis=1).astype(np.int32)
    Q = eng.schwarz(dorb, pairs).cpu().numpy()
    kept = pairs[Q >= 1e-12]
    lo = np.asarray(orb.l); la_aux = np.asarray(aux.l)
    rng = np.random.Generator(np.random.PCG64(1003))
    stream = torch.cuda.current_stream()
    peak = max(mdx.fp64_peak(0, 3), mdx.fp64_peak(1, 3)) * 1e9   # FP64 FLOP/s, measured
    rows, tot_ms, tot_flops, full_s, full_trip = [], 0.0, 0.0, 0.0, 0
    for la in range(int(la_aux.max()) + 1):
        a_sh = np.where(la_aux == la)[0]
        for lc in range(int(lo.max()) + 1):
            for ld in range(int(lo.max()) + 1):
                pc = kept[(lo[kept[:, 0]] == lc) & (lo[kept[:, 1]] == ld)]
                if len(pc) == 0 or len(a_sh) == 0:
                    continue
                Kcd = int(orb.nprim[pc[0, 0]]) * int(orb.nprim[pc[0, 1]])
                reg = eng.plan_info(la, 0, lc, ld, 1, Kcd, True).register_kernel != 0
                target = args.df_sample_reg if reg else args.df_sample
                na, npr = df_grid(len(a_sh), len(pc), target)
                A = rng.choice(a_sh, na, replace=False)
                Pp = pc[rng.choice(len(pc), npr, replace=False)]
                trip = np.stack([np.repeat(A, npr), np.tile(Pp[:, 0], na), np.tile(Pp[:, 1], na)],
                                axis=1).astype(np.int32)
                bt = (eng.batch_eri3_sph if args.df_sph else eng.batch_eri3)(daux, dorb, trip)
                out = torch.empty(max(bt.total, 1), dtype=torch.float64, device="cuda")
                ms = _event_ms(torch, stream, lambda: bt.run(out), args.steps, args.warmup)
                Kc, Kd = int(orb.nprim[Pp[0, 0]]), int(orb.nprim[Pp[0, 1]])
                n = len(trip)
                f = bt.model_flops
                full = len(a_sh) * len(pc)
                rows.append({"class": "[%d|%d%d]" % (la, lc, ld), "K_cd": Kc * Kd, "triplets": n,
                             "kernel": "register" if reg else "team",
                             "ms": round(ms, 4), "triplets_per_s": round(n / (ms * 1e-3), 1),
                             "model_gflops": round(f / (ms * 1e-3) * 1e-9, 2),
                             "executed_frac": round(2 * bt.exec_fma / (ms * 1e-3) / peak, 4),
                             "full_tensor_triplets": full})
                tot_ms += ms; tot_flops += f
                full_s += full / (n / (ms * 1e-3)); full_trip += full
                bt.close()
    eng.sync()
    line = {"metric": "3-center [a|cd] integrals: model FP64 GFLOP/s and triplets/s per class", "unit": UNIT,
            "value": round(tot_flops / (tot_ms * 1e-3) * 1e-9, 3), "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "density-fitting cluster: 100 atoms (>= 2.8 bohr apart), orbital 4s3p2d1f "
                                   "(K 6/3/1/1), auxiliary s..i (K 1, even-tempered ratio 2.5); orbital pairs "
                                   "kept at Q >= 1e-12; per class a grid of auxiliary shells x kept pairs (<= %d "
                                   "triplets for team-kernel classes, <= %d for register-kernel classes); "
                                   % (args.df_sample, args.df_sample_reg)
                                   + ("solid-harmonic" if args.df_sph else "Cartesian") + " functions",
                       "orbital_pairs": int(len(pairs)), "kept_pairs": int(len(kept)),
                       "aux_shells": int(aux.n_shells)},
            "full_tensor": {"triplets": int(full_trip), "estimated_s": round(full_s, 3)},
            "fp64_peak_gflops": round(peak * 1e-9, 1),
            "per_class": rows}
    print(json.dumps(line), flush=True)
    eng.close()


def grad_main(args):
    """Exchange energy and its nuclear gradient (shifted-class derivative integrals contracted with D (x) D
    in the kernel) on one cluster molecule (heavy 5s4p3d2f1g / light 4s3p2d1f, K = 6 s shells, D = C C^T,
    tau): the gradient call against the exchange build alone on the same quartets (whole calls, host
    screening included)."""
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    eng = mdx.Engine(0)
    mol = inputs.molecule(1005, args.grad_atoms)
    db = mdx.DeviceBasis(mol)
    D = torch.from_numpy(inputs.density(mol.nao, 1005)).cuda()
    pairs = torch.tensor([(i, j) for i in range(mol.n_shells) for j in range(i + 1)], dtype=torch.int32,
                         device="cuda")
    Q = eng.schwarz(db, pairs)
    stream = torch.cuda.current_stream()
    ms_k = _event_ms(torch, stream, lambda: eng.exchange(db, pairs, Q, D, args.tau), args.steps, args.warmup)
    nq = eng.last_quartet_count()
    res = {}
    ms_g = _event_ms(torch, stream, lambda: res.__setitem__("g", eng.exchange_grad(db, pairs, Q, D, args.tau)),
                     args.steps, args.warmup)
    eng.sync()
    g = res["g"][0] if isinstance(res["g"], tuple) else res["g"]
    line = {"metric": "exchange energy nuclear gradient (shifted-class derivative integrals) vs exchange build: ms and shell quartets/s",
            "unit": "ms", "value": round(ms_g, 3), "higher_is_better": False, "dtype": "f64",
            "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "cluster molecule of %d atoms (heavy 5s4p3d2f1g / light 4s3p2d1f, K = 6 s "
                                   "shells), D = C C^T, tau = %g" % (args.grad_atoms, args.tau),
                       "n_ao": int(mol.nao), "n_shells": int(mol.n_shells)},
            "quartets": nq, "exchange_ms": round(ms_k, 3), "gradient_ms": round(ms_g, 3),
            "gradient_over_exchange": round(ms_g / ms_k, 3),
            "quartets_per_s": {"exchange": round(nq / (ms_k * 1e-3), 1), "gradient": round(nq / (ms_g * 1e-3), 1)},
            "translational_residual": float(torch.as_tensor(g).sum(0).abs().max())}
    print(json.dumps(line), flush=True)
    eng.close()


def xchain_main(args):
    """The exchange build where D and K are far larger than the GPU's L2: a chain of --chain-atoms atoms
    (s,p,d shells of contraction --chain-k, 10 AOs per atom), D = C C^T, tau. Reports the build time, its quartet and model
    FLOP rates, the size of D and K, and the algorithmic bytes of the digestion (the four D blocks read and
    the four K blocks updated per unique quartet); the DRAM bytes it really moves come from ncu."""
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    eng = mdx.Engine(0)
    stream = torch.cuda.current_stream()
    b = inputs.chain(1006, args.chain_atoms, K=args.chain_k)
    db = mdx.DeviceBasis(b)
    i, j = np.tril_indices(b.n_shells)
    pairs = torch.from_numpy(np.stack([i, j], axis=1).astype(np.int32)).cuda()
    Q = eng.schwarz(db, pairs)
    D = torch.from_numpy(inputs.density(b.nao, 1006)).cuda()
    kept, n, f = eng.exchange_screen(db, pairs, Q, D, args.tau)
    # algorithmic digestion bytes: per kept quartet (ij|kl), D blocks ik, il, jk, jl read once and the
    # same K blocks read and written once (8 bytes per element)
    nc = torch.tensor([inputs.ncart(int(l)) for l in b.l], dtype=torch.float64, device="cuda")
    nbytes = 0.0
    for c0 in range(0, n, 1 << 24):
        kq = kept[c0:c0 + (1 << 24)].long()
        pi, pj = pairs[kq[:, 0]].long(), pairs[kq[:, 1]].long()
        ni, nj, nk, nl = nc[pi[:, 0]], nc[pi[:, 1]], nc[pj[:, 0]], nc[pj[:, 1]]
        nbytes += float(((ni * nk + ni * nl + nj * nk + nj * nl) * 8 * 3).sum())
    del kept
    clk = ClockSampler(0)
    clk.start()
    ms = _event_ms(torch, stream, lambda: eng.exchange(db, pairs, Q, D, args.tau), args.steps, args.warmup)
    clocks = clk.stop()
    assert eng.last_quartet_count() == n
    eng.sync()
    line = {"metric": "exchange build with D and K beyond L2: ms, shell quartets/s, model FP64 GFLOP/s",
            "unit": "ms", "value": round(ms, 3), "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "chain of %d atoms at 3.0 bohr (jitter 0.5), s,p,d shells K = %d, exponents "
                                   "log-uniform [0.1, 10], D = C C^T, tau = %g" % (args.chain_atoms, args.chain_k,
                                                                                   args.tau),
                       "n_ao": int(b.nao), "n_shells": int(b.n_shells), "shell_pairs": int(len(pairs))},
            "d_and_k_bytes": 2 * 8 * int(b.nao) ** 2, "l2_bytes": 129 * 2 ** 20,
            "quartets": n, "model_flops": f, "quartets_per_s": round(n / (ms * 1e-3), 1),
            "model_gflops": round(f / (ms * 1e-3) * 1e-9, 2),
            "digestion_algorithmic_bytes": nbytes,
            "digestion_algorithmic_gbs": round(nbytes / (ms * 1e-3) * 1e-9, 2),
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    eng.close()


def ab_main(args):
    """A/B of the two designs on the class sweep: the axis-factored kernels (mdx_batch_run) against the
    materialized-Hermite variant of the paper (mdx_batch_run_materialized: [p|q] matrices in HBM, both
    transforms as batched DGEMMs on the FP64 tensor units), same prepared batch, grid --ab-grid^2 per class."""
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    eng = mdx.Engine(0)
    stream = torch.cuda.current_stream()
    rows, ta, tb = [], 0.0, 0.0
    for l in [int(x) for x in args.classes.split(",") if x]:
        b, q = inputs.class_sweep((l, l, l, l), n_bra=args.ab_grid, n_ket=args.ab_grid)
        bt = eng.batch_eri4(mdx.DeviceBasis(b), q)
        out_a = torch.empty(bt.total, dtype=torch.float64, device="cuda")
        out_b = torch.empty(bt.total, dtype=torch.float64, device="cuda")
        ms_a = _event_ms(torch, stream, lambda: bt.run(out_a), args.steps, args.warmup)
        ms_b = _event_ms(torch, stream, lambda: bt.run_materialized(out_b), args.steps, args.warmup)
        diff = float((out_a - out_b).abs().max() / out_a.abs().max())
        f = model_flops(l, len(q))
        rows.append({"class": CLASS_NAMES[l], "quartets": len(q),
                     "axis_factored": {"ms": round(ms_a, 3), "quartets_per_s": round(len(q) / (ms_a * 1e-3), 1),
                                       "model_gflops": round(f / (ms_a * 1e-3) * 1e-9, 1)},
                     "materialized": {"ms": round(ms_b, 3), "quartets_per_s": round(len(q) / (ms_b * 1e-3), 1),
                                      "model_gflops": round(f / (ms_b * 1e-3) * 1e-9, 1)},
                     "speedup_of_axis_factored": round(ms_b / ms_a, 2), "max_rel_diff": diff})
        ta += ms_a; tb += ms_b
        bt.close()
    eng.sync()
    line = {"metric": "materialized-Hermite variant time / axis-factored time on the class sweep", "unit": "x",
            "value": round(tb / ta, 3), "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "class sweep [ll|ll], %dx%d random uncontracted quartets per class" %
                                   (args.ab_grid, args.ab_grid)},
            "per_class": rows}
    print(json.dumps(line), flush=True)
    eng.close()


# The paper's solid-harmonic 4-center rates on one V100 (shellsets/s, Tab. nps4), class [l1 l2|l3 l4] by its
# four angular momenta, columns {K_bra, K_ket} = {1,1}, {1,5}, {5,5}: context for the solid-harmonic workload
PAPER_NPS4_V100 = {
    (0, 0, 0, 0): (4.53e9, 2.98e9, 9.11e8), (1, 0, 1, 0): (2.10e9, 1.23e9, 3.31e8),
    (2, 0, 2, 0): (1.01e9, 5.17e8, 1.27e8), (3, 0, 3, 0): (1.28e8, 8.19e7, 1.75e7),
    (4, 0, 4, 0): (8.31e7, 3.62e7, 7.52e6), (5, 0, 5, 0): (1.80e7, 7.19e6, 1.56e6),
    (6, 0, 6, 0): (6.71e6, 2.47e6, 5.43e5), (1, 1, 1, 1): (2.59e8, 2.05e8, 5.27e7),
    (2, 2, 2, 2): (2.25e7, 1.04e7, 2.12e6), (3, 3, 3, 3): (2.47e6, 8.00e5, 1.69e5),
    (4, 4, 4, 4): (3.25e5, 9.59e4, 2.05e4), (5, 5, 5, 5): (1.11e5, 3.14e4, 6.73e3),
    (6, 6, 6, 6): (3.47e4, 9.74e3, 1.99e3)}


# The paper's Tab. nps3 (one V100, solid harmonics): shellsets/s for {K_bra, K_ket} = {1,1}, {1,5}, {5,5}
PAPER_NPS3_V100 = {
    (1, 0, 0): (5.18e9, 3.29e9, 1.09e9), (2, 0, 0): (3.30e9, 2.10e9, 7.20e8), (3, 0, 0): (2.52e9, 1.44e9, 5.61e8),
    (4, 0, 0): (1.72e9, 1.13e9, 3.70e8), (5, 0, 0): (1.34e9, 8.15e8, 2.64e8), (6, 0, 0): (9.37e8, 5.17e8, 1.46e8),
    (0, 1, 1): (2.17e9, 1.72e9, 5.47e8), (0, 2, 2): (7.81e8, 4.48e8, 1.17e8), (0, 3, 3): (2.04e8, 1.27e8, 2.90e7),
    (0, 4, 4): (7.05e7, 1.57e7, 3.23e6), (0, 5, 5): (2.69e7, 5.77e6, 1.29e6), (0, 6, 6): (1.97e7, 4.67e6, 2.20e6),
    (0, 0, 0): (9.63e9, 5.15e9, 1.64e9), (1, 1, 1): (7.25e8, 8.88e8, 2.59e8), (2, 2, 2): (1.75e8, 5.43e7, 1.18e7),
    (3, 3, 3): (3.34e7, 7.48e6, 2.67e6), (4, 4, 4): (8.88e6, 1.90e6, 8.57e5), (5, 5, 5): (4.17e6, 8.91e5, 3.98e5),
    (6, 6, 6): (1.18e6, 2.63e5, 1.02e5)}


def sph3_main(args):
    """Solid-harmonic 3-center integrals [a|cd] per class of the paper's Tab. nps3: [l|00], [0|ll], [l|ll],
    {K_bra, K_ket} = {1,1}, {1,5}, {5,5} (the auxiliary shell has K_bra; one orbital shell of the pair has
    K = 5). Random shells (class_sweep3); each class on a seeded grid sized to about 0.1 TFLOP of executed
    work; autotuned per class unless --no-tune. The paper's V100 rates are quoted beside ours as context."""
    import math
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    eng = mdx.Engine(0)
    stream = torch.cuda.current_stream()
    peak = max(mdx.fp64_peak(0, 3), mdx.fp64_peak(1, 3)) * 1e9
    kcols = (("{1,1}", (1, 1, 1)), ("{1,5}", (1, 5, 1)), ("{5,5}", (5, 5, 1)))
    only = {tuple(int(ch) for ch in c) for c in args.sph_classes.split(",") if c} if args.sph_classes else None
    rows = []
    for lt in sorted(PAPER_NPS3_V100, key=lambda x: (sum(x), x)):
        if only and lt not in only:
            continue
        for ki, (kname, K) in enumerate(kcols):
            est = mdx.plan_info(lt[0], 0, lt[1], lt[2], K[0], K[1] * K[2], one_centre=True).exec_fma
            n = int(min(2048 * 2048, max(1024, 0.1e12 / max(est, 1.0))))
            side = int(math.ceil(math.sqrt(n)))
            aux, orb, t = inputs.class_sweep3(lt, n_aux=side, n_ket=side, K=K)
            da, do = mdx.DeviceBasis(aux), mdx.DeviceBasis(orb)
            bt = eng.batch_eri3_sph(da, do, t)
            out = torch.empty(bt.total, dtype=torch.float64, device="cuda")
            if not args.no_tune:
                bt.autotune(out, max_trial=int(min(len(t), max(152, 2e9 / max(est, 1.0)))))
            ms = _event_ms(torch, stream, lambda: bt.run(out), args.steps, args.warmup)
            rows.append({"class": "[%d|%d%d]" % lt, "K": kname, "shellsets": len(t), "ms": round(ms, 4),
                         "shellsets_per_s": round(len(t) / (ms * 1e-3), 1),
                         "exec_gflops": round(2 * bt.exec_fma / (ms * 1e-3) * 1e-9, 2),
                         "exec_frac_of_peak": round(2 * bt.exec_fma / (ms * 1e-3) / peak, 4),
                         "paper_v100_shellsets_per_s": PAPER_NPS3_V100[lt][ki]})
            bt.close()
    eng.sync()
    line = {"metric": "solid-harmonic [a|cd]: shellsets/s and FP64 GFLOP/s per class of the paper's Tab. nps3",
            "unit": "shellsets/s", "value": next((r["shellsets_per_s"] for r in rows if r["class"] == "[6|66]" and
                                                 r["K"] == "{1,1}"), None),
            "higher_is_better": True, "dtype": "f64", "data": "synthetic", "steps": args.steps,
            "warmup": args.warmup, "fp64_peak_gflops": round(peak * 1e-9, 1),
            "config": {"workload": "solid-harmonic 3-center class sweep: random shells (centres in a 10-bohr box, "
                                   "exponents log-uniform [0.05, 50]), [l|00], [0|ll], [l|ll], {K_bra, K_ket} = "
                                   "{1,1}, {1,5}, {5,5}; value: [6|66] {1,1}"},
            "paper_context": "Tab. nps3 of the paper: one V100 (FP64 7 TFLOP/s), solid harmonics",
            "per_class": rows}
    print(json.dumps(line), flush=True)
    eng.close()


def sph_main(args):
    """Solid-harmonic 4-center integrals (the paper's basis) per class of the paper's Tab. nps4: [ll|ll] and
    [l0|l0], contraction columns {K_bra, K_ket} = {1,1}, {1,5}, {5,5} (one shell of a contracted pair has
    K = 5). Random shells as in the class sweep; each class on a seeded grid sized to about 0.15 TFLOP of
    executed work (1,024 to 4,194,304 shellsets: the paper's runs are sized by output, up to 500 MB). Classes of the team kernel contract the solid-harmonic coefficients into the transforms
    (mdx_batch_eri4_sph; autotuned per class unless --no-tune); [ll|ll] with l >= 4 is also timed through
    the Cartesian kernel on the same quartets. The paper's V100 rates are quoted beside ours as context
    (another machine)."""
    import math
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    eng = mdx.Engine(0)
    stream = torch.cuda.current_stream()
    peak = max(mdx.fp64_peak(0, 3), mdx.fp64_peak(1, 3)) * 1e9
    kcols = (("{1,1}", (1, 1, 1, 1)), ("{1,5}", (1, 1, 5, 1)), ("{5,5}", (5, 1, 5, 1)))
    rows = []
    only = {tuple(int(ch) for ch in c) for c in args.sph_classes.split(",") if c} if args.sph_classes else None
    for lq in sorted(PAPER_NPS4_V100, key=lambda x: (sum(x), x)):
        if only and lq not in only:
            continue
        for ki, (kname, K) in enumerate(kcols):
            est = mdx.plan_info(*lq, K[0] * K[1], K[2] * K[3]).exec_fma
            n = int(min(2048 * 2048, max(1024, 0.15e12 / max(est, 1.0))))
            side = int(math.ceil(math.sqrt(n)))
            b, q = inputs.class_sweep(lq, n_bra=side, n_ket=side, seed=1002, K=K)
            db = mdx.DeviceBasis(b)
            bt = eng.batch_eri4_sph(db, q)
            out = torch.empty(bt.total, dtype=torch.float64, device="cuda")
            if not args.no_tune:   # team size, budget and cached R tables per class, on about 2 GFMA of work
                bt.autotune(out, max_trial=int(min(len(q), max(152, 2e9 / max(est, 1.0)))))
            ms = _event_ms(torch, stream, lambda: bt.run(out), args.steps, args.warmup)
            row = {"class": "[%d%d|%d%d]" % lq, "K": kname, "shellsets": len(q), "ms": round(ms, 4),
                   "shellsets_per_s": round(len(q) / (ms * 1e-3), 1),
                   "exec_gflops": round(2 * bt.exec_fma / (ms * 1e-3) * 1e-9, 2),
                   "exec_frac_of_peak": round(2 * bt.exec_fma / (ms * 1e-3) / peak, 4),
                   "exec_fma_per_shellset": round(bt.exec_fma / len(q), 1),
                   "model_gflops": round(bt.model_flops / (ms * 1e-3) * 1e-9, 2),
                   "paper_v100_shellsets_per_s": PAPER_NPS4_V100[lq][ki]}
            bt.close()
            if lq[0] == lq[2] and lq[0] == lq[1] and lq[0] >= 4:
                bc = eng.batch_eri4(db, q)
                oc = torch.empty(bc.total, dtype=torch.float64, device="cuda")
                msc = _event_ms(torch, stream, lambda: bc.run(oc), args.steps, args.warmup)
                row["cartesian_ms"] = round(msc, 4)
                row["cartesian_exec_fma_per_shellset"] = round(bc.exec_fma / len(q), 1)
                bc.close()
            rows.append(row)
    eng.sync()
    line = {"metric": "solid-harmonic [ab|cd]: shellsets/s and FP64 GFLOP/s per class of the paper's Tab. nps4",
            "unit": "shellsets/s", "value": next((r["shellsets_per_s"] for r in rows if r["class"] == "[66|66]" and
                                                 r["K"] == "{1,1}"), None),
            "higher_is_better": True, "dtype": "f64", "data": "synthetic", "steps": args.steps,
            "warmup": args.warmup, "fp64_peak_gflops": round(peak * 1e-9, 1),
            "config": {"workload": "solid-harmonic class sweep: random shells (centres in a 10-bohr box, exponents "
                                   "log-uniform [0.05, 50]), [ll|ll] and [l0|l0], {K_bra, K_ket} = {1,1}, {1,5}, "
                                   "{5,5}; value: [66|66] {1,1}"},
            "paper_context": "Tab. nps4 of the paper: one V100 (FP64 7 TFLOP/s), solid harmonics",
            "per_class": rows}
    print(json.dumps(line), flush=True)
    eng.close()


def _density_on_device(torch, nao: int, seed: int, occ_fraction: float = 0.2):
    """inputs.density's recipe (D = C C^T, C an orthonormal basis of a seeded Gaussian nao x nao/5 matrix)
    with the QR and the product done on the GPU: the same projector, for matrices too large for the host."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nocc = max(1, int(nao * occ_fraction))
    G = torch.from_numpy(rng.standard_normal((nao, nocc))).cuda()
    C, _ = torch.linalg.qr(G)
    return C @ C.T


def counts_main(args):
    """Screened unique quartets of the full-size exchange workloads, counted on the GPU with the screening
    of mdx_exchange alone (mdx_exchange_screen, count only): the 400-atom cluster (> 20,000 AOs) and the 64
    uneven molecules of 10-120 atoms, Schwarz x density screening at tau. Their Table-1 model FLOPs are turned
    into a projected time with the exchange build's model rate measured here on an 8-atom cluster."""
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    eng = mdx.Engine(0)
    stream = torch.cuda.current_stream()

    def all_pairs(b):
        i, j = np.tril_indices(b.n_shells)
        return torch.from_numpy(np.stack([i, j], axis=1).astype(np.int32)).cuda()

    # the exchange build's rate on the gradient workload's 8-atom cluster
    m8 = inputs.molecule(1005, 8)
    d8 = mdx.DeviceBasis(m8)
    p8 = all_pairs(m8)
    Q8 = eng.schwarz(d8, p8)
    D8 = torch.from_numpy(inputs.density(m8.nao, 1005)).cuda()
    _, n8, f8 = eng.exchange_screen(d8, p8, Q8, D8, args.tau, list_quartets=False)
    ms8 = _event_ms(torch, stream, lambda: eng.exchange(d8, p8, Q8, D8, args.tau), args.steps, args.warmup)
    rate = f8 / (ms8 * 1e-3)
    res = {"rate_basis": {"workload": "8-atom cluster exchange build", "quartets": n8, "model_flops": f8,
                          "ms": round(ms8, 2), "model_gflops": round(rate * 1e-9, 2)}}
    t0 = time.perf_counter()
    b5 = inputs.molecule(1005, 400)
    db5 = mdx.DeviceBasis(b5)
    p5 = all_pairs(b5)
    Q5 = eng.schwarz(db5, p5)
    D5 = _density_on_device(torch, b5.nao, 1005)
    t1 = time.perf_counter()
    _, n5, f5 = eng.exchange_screen(db5, p5, Q5, D5, args.tau, list_quartets=False)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    res["cluster_400"] = {"atoms": 400, "n_ao": int(b5.nao), "shells": int(b5.n_shells), "shell_pairs": int(len(p5)),
                          "pairs_q_above_tau": int((Q5 >= args.tau).sum()), "kept_quartets": n5,
                          "unique_quartets": int(len(p5)) * (int(len(p5)) + 1) // 2, "model_flops": f5,
                          "projected_exchange_s": round(f5 / rate, 1), "setup_s": round(t1 - t0, 1),
                          "screen_s": round(t2 - t1, 2)}
    del D5, Q5, p5, db5
    mols = inputs.molecule_batch(1004, 64, 10, 120)
    tot_n = tot_f = 0.0
    tot_pairs = 0
    t0 = time.perf_counter()
    for i, b in enumerate(mols):
        db = mdx.DeviceBasis(b)
        p = all_pairs(b)
        Q = eng.schwarz(db, p)
        D = _density_on_device(torch, b.nao, 7 + i)
        _, n, f = eng.exchange_screen(db, p, Q, D, args.tau, list_quartets=False)
        tot_n += n; tot_f += f; tot_pairs += len(p)
    res["batch_64"] = {"molecules": 64, "atoms": [int(b.n_atoms) for b in mols],
                       "n_ao_total": int(sum(b.nao for b in mols)), "shell_pairs": tot_pairs,
                       "kept_quartets": int(tot_n), "model_flops": tot_f,
                       "projected_exchange_s": round(tot_f / rate, 1), "s": round(time.perf_counter() - t0, 1)}
    eng.sync()
    line = {"metric": "screened unique quartets and projected exchange time of the full-size workloads",
            "unit": "s", "value": res["cluster_400"]["projected_exchange_s"], "higher_is_better": False,
            "dtype": "f64", "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "400-atom cluster (seed 1005) and 64 molecules of 10-120 atoms (seed 1004), "
                                   "heavy 5s4p3d2f1g / light 4s3p2d1f, D = C C^T, tau = %g" % args.tau},
            **res}
    print(json.dumps(line), flush=True)
    eng.close()


def peak_main(args):
    """FP64 throughput of this GPU: scalar DFMA against the FP64 tensor instruction (DMMA) in its three
    shapes (mdx_fp64_peak), with the SM clocks sampled meanwhile. The engine's transforms use DFMA
    because DMMA retires FP64 multiply-adds at about the same rate on this part (and needs dense tiles)."""
    import torch
    from paper_2405_01834_gb300 import mdx
    torch.cuda.set_device(0)
    mdx.fp64_peak(0, 1)   # warm-up
    clk = ClockSampler(0)
    clk.start()
    names = {0: "dfma", 1: "dmma_m8n8k4", 2: "dmma_m16n8k4", 3: "dmma_m16n8k16"}
    res = {names[k]: round(max(mdx.fp64_peak(k, 5) for _ in range(max(1, args.steps))), 1) for k in range(4)}
    clocks = clk.stop()
    props = torch.cuda.get_device_properties(0)
    mhz = (clocks or {}).get("sm_mhz") or 0.0
    line = {"metric": "FP64 throughput: scalar DFMA vs the FP64 tensor instruction", "unit": "GFLOP/s",
            "value": max(res.values()), "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "steps": args.steps, "config": {"workload": "register-resident FP64 multiply-add loops, 8 x 256 threads "
                                                        "per SM, %d SMs" % props.multi_processor_count},
            "per_kind": res,
            "per_sm_per_clock": ({k: round(v * 1e9 / (props.multi_processor_count * mhz * 1e6), 3)
                                  for k, v in res.items()} if mhz else None),
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return reference_main(args)
    if args.workload == "xbatch":
        return xbatch_main(args)
    if args.workload == "df":
        return df_main(args)
    if args.workload == "grad":
        return grad_main(args)
    if args.workload == "ab":
        return ab_main(args)
    if args.workload == "peak":
        return peak_main(args)
    if args.workload == "sph":
        return sph_main(args)
    if args.workload == "xchain":
        return xchain_main(args)
    if args.workload == "sph3":
        return sph3_main(args)
    if args.workload == "counts":
        return counts_main(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2405_01834_gb300 import mdx
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    eng = mdx.Engine(dev)
    work = workload(args)

    # prepare: inputs resident on the device, quartet lists split into chunks
    prepared = []
    max_chunk = 0
    sms = props.multi_processor_count
    for l, b, q in work:
        db = mdx.DeviceBasis(b)
        cq = chunk_quartets(l, len(q), sms)
        batches = [eng.batch_eri4(db, q[s:s + cq]) for s in range(0, len(q), cq)]
        max_chunk = max(max_chunk, max(bt.total for bt in batches))
        prepared.append((l, db, q, batches))
    out = torch.empty(max_chunk, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    tuned = {}
    if not args.no_tune:
        # choose each class's team shape on its first chunk (untimed set-up, like a library's autotuning);
        # later chunks of the class use the choice when they are re-planned
        for l, db, q, batches in prepared:
            t0 = time.perf_counter()
            # trials large enough to fill the GPU with one-thread-per-quartet candidates at low l
            batches[0].autotune(out, max_trial=autotune_trial(l, len(q)))
            tuned[CLASS_NAMES[l]] = round(time.perf_counter() - t0, 2)
        # re-prepare so every chunk picks up the tuned plans
        for i, (l, db, q, batches) in enumerate(prepared):
            for bt in batches:
                bt.close()
            cq = chunk_quartets(l, len(q), sms)
            prepared[i] = (l, db, q, [eng.batch_eri4(db, q[s:s + cq]) for s in range(0, len(q), cq)])
    stream = torch.cuda.current_stream()

    def step(record):
        times = []
        nl = 0
        for l, db, q, batches in prepared:
            ev = []
            for bt in batches:
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                nl += bt.run(out)
                e1.record(stream)
                ev.append((e0, e1))
            times.append(ev)
        return times, nl

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False)
        flush.zero_()
    eng.sync()
    barrier()
    clk = ClockSampler(dev)
    clk.start()
    # the FP64 peak of this GPU, measured now (clocks sampled with the timed region): scalar DFMA and
    # the FP64 tensor instruction (m8n8k4); the roofline takes the larger
    probe = {"dfma": mdx.fp64_peak(0, 3), "dmma_m8n8k4": mdx.fp64_peak(1, 3)}
    barrier()
    per_class_ms = {l: [] for l, *_ in prepared}
    per_launch_ms = {l: [] for l, *_ in prepared}
    step_ms = []
    launches = 0
    for s in range(args.steps):
        flush.zero_()
        barrier()
        times, nl = step(True)
        barrier()
        launches += nl
        tot = 0.0
        for (l, *_), ev in zip(prepared, times):
            ms = [a.elapsed_time(b) for a, b in ev]
            per_class_ms[l].append(sum(ms))
            per_launch_ms[l].extend(ms)
            tot += sum(ms)
        step_ms.append(tot)
    clocks = clk.stop()
    eng.sync()
    ms_step = max_over_ranks(sum(step_ms) / len(step_ms), world, "cuda")

    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    derived_gflops = FP64_FLOP_PER_CLK_SM * props.multi_processor_count * sm_max * 1e-3
    peak_gflops = max(probe.values())
    total_flops = sum(model_flops(l, len(q)) for l, _, q, _ in prepared)
    total_exec = sum(2.0 * bt.exec_fma for *_, batches in prepared for bt in batches)
    value = whole_job_rate(total_flops, world, ms_step) * 1e-9
    per_class = {}
    dom_l, dom_ms = None, -1.0
    for l, db, q, batches in prepared:
        ms = sum(per_class_ms[l]) / len(per_class_ms[l])
        f = model_flops(l, len(q))
        ex = sum(2.0 * bt.exec_fma for bt in batches)
        per_class[CLASS_NAMES[l]] = {
            "quartets": len(q), "ms": round(ms, 3), "quartets_per_s": round(len(q) / (ms * 1e-3), 1),
            "exec_gflops": round(ex / (ms * 1e-3) * 1e-9, 2),
            "exec_frac_of_peak": round(ex / (ms * 1e-3) * 1e-9 / peak_gflops, 4),
            "model_gflops": round(f / (ms * 1e-3) * 1e-9, 2),
            "model_over_executed_flops": round(f / ex, 2),
            "launches_per_step": 2 * len(batches)}
        if ms > dom_ms:
            dom_ms, dom_l = ms, l
    # roofline of the dominant class's launches (pair records + quartet kernel per chunk): the FP64
    # multiply-adds its planner counts (x2) per launch over the launch's CUDA-event time
    l = dom_l
    _, _, q, batches = next(p for p in prepared if p[0] == l)
    lm = per_launch_ms[l]
    avg_launch_ms = sum(lm) / len(lm)
    per_launch_exec = sum(2.0 * bt.exec_fma for bt in batches) / len(batches)
    per_launch_model = model_flops(l, len(q)) / len(batches)
    achieved = per_launch_exec / (avg_launch_ms * 1e-3) * 1e-12
    traffic = None
    if NCU_DRAM_BYTES_PER_II_QUARTET is not None and l == 6:
        traffic = round(NCU_DRAM_BYTES_PER_II_QUARTET * len(q) / len(batches))
    roofline = {"bound": "alu", "kernel": "k_quartets %s" % CLASS_NAMES[l], "achieved": round(achieved, 4),
                "peak": round(peak_gflops * 1e-3, 4), "unit": "TFLOP/s", "frac": round(achieved / (peak_gflops * 1e-3), 4),
                "traffic": traffic, "traffic_unit": "DRAM bytes read + written per launch (ncu)",
                "algorithmic_flops_per_launch": per_launch_exec,
                "peak_basis": "FP64, measured in this run: max of scalar DFMA %.1f and DMMA m8n8k4 %.1f GFLOP/s "
                              "(mdx_fp64_peak); derived 2 FMA/clk/SM x %d SMs x %.0f MHz = %.1f GFLOP/s" % (
                                  probe["dfma"], probe["dmma_m8n8k4"], props.multi_processor_count, sm_max,
                                  derived_gflops),
                "model_tflops": round(per_launch_model / (avg_launch_ms * 1e-3) * 1e-12, 4),
                "model_flops_per_launch": per_launch_model}

    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(sweep_config(args, world), l2="256 MB buffer written between timed steps"),
            "quartets_per_s": round(whole_job_rate(sum(len(q) for _, _, q, _ in prepared), world, ms_step), 1),
            "exec_gflops": round(world * total_exec / (ms_step * 1e-3) * 1e-9, 3),
            "exec_frac_of_peak": round(total_exec / (ms_step * 1e-3) * 1e-9 / peak_gflops, 4),
            "fp64_peak_gflops": {k: round(v, 1) for k, v in probe.items()},
            "per_class": per_class, "roofline": roofline, "autotune_s": tuned or None, "gpu_launches": launches,
            "gpu_launches_per_step": launches // args.steps if args.steps else 0,
            "clocks": clocks}

    # ---- end to end through the public call with host buffers (rank 0 timing only)
    if not args.no_e2e:
        line["e2e"] = e2e(eng, work, args, torch)
    if rank == 0 and not args.no_cpu:
        kept = {}
        f, t, nq, per = run_oracle(work, args.cpu_sample, keep=kept)
        line["cpu_baseline"] = {"value": round(f / t * 1e-9, 4), "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
                                "sample": "seeded %.2f%% of each class (%d quartets), oracle as committed" % (
                                    100 * args.cpu_sample, nq), "per_class": per}
        line["parity"] = sample_parity(prepared, kept, out, torch)
        f1, t1, nq1, _ = run_oracle(work, args.cpu_sample / 10, seed=7, nthreads=1)
        line["cpu_baseline"]["one_core"] = {"value": round(f1 / t1 * 1e-9, 4), "unit": UNIT, "cores": 1,
                                            "sample": "seeded %.3f%% of each class (%d quartets)" % (
                                                10 * args.cpu_sample, nq1)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    eng.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def sample_parity(prepared, kept, out, torch):
    """The oracle's CPU-baseline sample of each class against the GPU shellsets of the same quartets, from
    the timed launch configuration (the class's prepared batches, run once more): the parity record of the
    benchmark (rule: oracle/parity.py)."""
    from oracle import parity
    rec, worst_abs, worst_rel, n_cancel, n_el = {}, 0.0, 0.0, 0, 0
    for l, db, q, batches in prepared:
        if l not in kept:
            continue
        idx, ref, off = kept[l]
        per_q = inputs.ncart(l) ** 4
        got = np.zeros(len(idx) * per_q)
        lo = 0
        for bt in batches:
            bt.run(out)
            torch.cuda.synchronize()
            hi = lo + bt.n
            sel = np.where((idx >= lo) & (idx < hi))[0]
            if len(sel):
                rows = torch.as_tensor(idx[sel] - lo, device="cuda")
                vals = out[: bt.n * per_q].view(bt.n, per_q).index_select(0, rows).cpu().numpy()
                for k, n in enumerate(sel):
                    got[n * per_q:(n + 1) * per_q] = vals[k]
            lo = hi
        r = parity.check(got, ref, off, "bench sample %s" % CLASS_NAMES[l], parity.Eri4Evaluator(db.host, q[idx]))
        rec[CLASS_NAMES[l]] = {k: r[k] for k in ("elements", "max_abs_over_scale", "max_rel", "n_cancel")}
        worst_abs = max(worst_abs, r["max_abs_over_scale"])
        worst_rel = max(worst_rel, r["max_rel"])
        n_cancel += r["n_cancel"]
        n_el += r["elements"]
    return {"rule": "abs <= 1e-12 max|shellset|, rel <= 1e-10 above 1e-10, cancellation exception counted "
                    "(oracle/parity.py)", "elements": n_el, "max_abs_over_scale": worst_abs, "max_rel": worst_rel,
            "n_cancel": n_cancel, "per_class": rec}


def e2e(eng, work, args, torch):
    """One step through mdx_eri4 with host buffers: pinned quartet arrays copied in, integrals copied back to
    pinned host memory, chunk by chunk. Two device output buffers; the host copy of chunk i-1 is enqueued (on a
    second stream) right after chunk i's kernels, so it runs while they compute. (Enqueued earlier, it would
    sit in the copy engine ahead of mdx_eri4's small index downloads for chunk i and serialise the two.)"""
    from paper_2405_01834_gb300 import mdx
    host = []
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for l, b, q in work:
        host.append((l, b, torch.from_numpy(q).pin_memory(), chunk_quartets(l, len(q), sms)))
    max_out = max(min(len(q), cq) * inputs.ncart(l) ** 4 for l, b, q, cq in host)
    out_dev = [torch.empty(max_out, dtype=torch.float64, device="cuda") for _ in range(2)]
    out_host = [torch.empty(max_out, dtype=torch.float64).pin_memory() for _ in range(2)]
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    copied = [None, None]   # event: the host copy out of buffer k has finished
    pending = None          # (buffer, doubles) computed but not yet copied out
    h2d = d2h = 0
    tot_f = 0.0
    k = 0

    def copy_out(buf, n, ready):
        with torch.cuda.stream(copy):
            copy.wait_event(ready)
            out_host[buf][:n].copy_(out_dev[buf][:n], non_blocking=True)
            copied[buf] = torch.cuda.Event()
            copied[buf].record(copy)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for l, b, qh, cq in host:
        db = mdx.DeviceBasis(b)   # basis arrays: host -> device
        h2d += sum(t.numel() * t.element_size() for t in (db.l, db.nprim, db.prim_off, db.ao_off, db.atom,
                                                          db.center, db.exps, db.coefs))
        for s in range(0, qh.shape[0], cq):
            if copied[k] is not None:
                comp.wait_event(copied[k])
            qd = qh[s:s + cq].to("cuda", non_blocking=True)
            h2d += qd.numel() * 4
            eng.eri4(db, qd, out=out_dev[k])
            done = torch.cuda.Event()   # this chunk's kernels, for its copy one iteration later
            done.record(comp)
            n = qd.shape[0] * inputs.ncart(l) ** 4
            if pending is not None:
                copy_out(*pending)
            pending = (k, n, done)
            d2h += n * 8
            k ^= 1
        tot_f += model_flops(l, qh.shape[0])
    if pending is not None:
        copy_out(*pending)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": round(tot_f / dt * 1e-9, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": 1, "s": round(dt, 3)}


if __name__ == "__main__":
    main()
