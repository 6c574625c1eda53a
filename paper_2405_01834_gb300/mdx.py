"""Python binding of the C ABI in include/mdx.h (argument marshalling only).

Every integral is computed by the CUDA kernels of libmdx.so; this module only
moves torch tensors' device pointers and sizes across the ABI. There is no
CPU fallback: if the library is missing or no CUDA device is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

_lib = None


class MdxError(RuntimeError):
    pass


class _Basis(ctypes.Structure):
    _fields_ = [("n_shells", ctypes.c_int32), ("n_prims", ctypes.c_int32),
                ("l", ctypes.c_void_p), ("nprim", ctypes.c_void_p), ("prim_off", ctypes.c_void_p),
                ("ao_off", ctypes.c_void_p), ("atom", ctypes.c_void_p), ("center", ctypes.c_void_p),
                ("exps", ctypes.c_void_p), ("coefs", ctypes.c_void_p)]


class PlanStats(ctypes.Structure):
    _fields_ = [("team_threads", ctypes.c_int32), ("teams_per_cta", ctypes.c_int32),
                ("smem_bytes_per_team", ctypes.c_int32), ("n_groups", ctypes.c_int32), ("exec_fma", ctypes.c_double),
                ("register_kernel", ctypes.c_int32), ("pad", ctypes.c_int32)]


def plan_info(la, lb, lc, ld, Kb=1, Kk=1, one_centre=False) -> PlanStats:
    """Team shape and executed FP64 FMA count per shellset of a class (host planner, no GPU)."""
    lib = load()
    st = PlanStats()
    rc = lib.mdx_plan_info(None, la, lb, lc, ld, Kb, Kk, int(one_centre), ctypes.byref(st))
    if rc != 0:
        raise MdxError("mdx_plan_info(%d,%d,%d,%d): %s" % (la, lb, lc, ld, STATUS.get(rc, rc)))
    return st


def _check_out(out: torch.Tensor, what: str):
    """Output buffers cross the ABI as a pointer and a capacity in doubles: only a contiguous
    float64 CUDA tensor has that meaning (anything else would be written past its end)."""
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.float64 or not out.is_contiguous():
        raise MdxError("%s: out must be a contiguous float64 CUDA tensor" % what)


def _opt_ptr(t):
    return None if t is None else t.data_ptr()


def eri4_noalloc(basis: "DeviceBasis", quartets, out: torch.Tensor):
    """mdx_eri4_noalloc on the current device: [ab|cd] into the caller's `out`
    with no device allocation by the library (for callers whose device memory
    is owned by their own pool). Returns (status, offsets[n+1])."""
    lib = load()
    _check_out(out, "mdx_eri4_noalloc")
    q = torch.as_tensor(quartets, dtype=torch.int32, device="cuda").contiguous()
    offs = torch.empty(q.shape[0] + 1, dtype=torch.int64, device="cuda")
    st = lib.mdx_eri4_noalloc(ctypes.byref(basis.desc), q.data_ptr(), q.shape[0], out.data_ptr(), out.numel(),
                              offs.data_ptr(), _stream())
    return st, offs


def fp64_peak(kind: int = 0, reps: int = 3) -> float:
    """Measured FP64 throughput (GFLOP/s) of the current device: kind 0 DFMA,
    1/2/3 the f64 mma.sync shapes m8n8k4 / m16n8k4 / m16n8k16 (mdx_fp64_peak)."""
    lib = load()
    g = ctypes.c_double()
    st = lib.mdx_fp64_peak(int(kind), int(reps), ctypes.byref(g), _stream())
    if st != 0:
        raise MdxError("mdx_fp64_peak(%d): %s" % (kind, STATUS.get(st, st)))
    return g.value


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmdx.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise MdxError("libmdx.so is not built (run paper_2405_01834_gb300.build)")
        _build.build()
    lib = ctypes.CDLL(path)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.mdx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), I32]
    lib.mdx_create.restype = I32
    lib.mdx_destroy.argtypes = [P]
    lib.mdx_destroy.restype = None
    lib.mdx_last_error.argtypes = [P]
    lib.mdx_last_error.restype = ctypes.c_char_p
    lib.mdx_sync.argtypes = [P, P]
    lib.mdx_sync.restype = I32
    lib.mdx_eri4.argtypes = [P, ctypes.POINTER(_Basis), P, P, I64, ctypes.c_double, P, I64, P, P]
    lib.mdx_eri4.restype = I32
    lib.mdx_eri4_sph.argtypes = [P, ctypes.POINTER(_Basis), P, I64, P, I64, P, P]
    lib.mdx_eri4_sph.restype = I32
    lib.mdx_eri3.argtypes = [P, ctypes.POINTER(_Basis), ctypes.POINTER(_Basis), P, P, I64, ctypes.c_double, P, I64,
                             P, P]
    lib.mdx_eri3.restype = I32
    lib.mdx_schwarz.argtypes = [P, ctypes.POINTER(_Basis), P, I64, P, P]
    lib.mdx_schwarz.restype = I32
    lib.mdx_batch_eri4.argtypes = [P, ctypes.POINTER(_Basis), P, I64, ctypes.POINTER(ctypes.c_void_p), P]
    lib.mdx_batch_eri4.restype = I32
    lib.mdx_batch_eri3.argtypes = [P, ctypes.POINTER(_Basis), ctypes.POINTER(_Basis), P, I64,
                                   ctypes.POINTER(ctypes.c_void_p), P]
    lib.mdx_batch_eri3.restype = I32
    lib.mdx_batch_eri4_sph.argtypes = [P, ctypes.POINTER(_Basis), P, I64, ctypes.POINTER(ctypes.c_void_p), P]
    lib.mdx_batch_eri4_sph.restype = I32
    lib.mdx_eri3_sph.argtypes = [P, ctypes.POINTER(_Basis), ctypes.POINTER(_Basis), P, I64, P, I64, P, P]
    lib.mdx_eri3_sph.restype = I32
    lib.mdx_batch_eri3_sph.argtypes = [P, ctypes.POINTER(_Basis), ctypes.POINTER(_Basis), P, I64,
                                       ctypes.POINTER(ctypes.c_void_p), P]
    lib.mdx_batch_eri3_sph.restype = I32
    lib.mdx_batch_info.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.mdx_batch_info.restype = I32
    lib.mdx_batch_offsets.argtypes = [P, P, P, P]
    lib.mdx_batch_offsets.restype = I32
    lib.mdx_batch_run.argtypes = [P, P, P, I64, ctypes.POINTER(ctypes.c_int32), P]
    lib.mdx_batch_run.restype = I32
    lib.mdx_batch_autotune.argtypes = [P, P, P, I64, I64, P]
    lib.mdx_batch_autotune.restype = I32
    lib.mdx_batch_destroy.argtypes = [P]
    lib.mdx_batch_destroy.restype = None
    lib.mdx_exchange.argtypes = [P, ctypes.POINTER(_Basis), P, P, I64, ctypes.c_double, P, P, ctypes.c_double, P,
                                 P]
    lib.mdx_exchange.restype = I32
    lib.mdx_exchange_grad.argtypes = [P, ctypes.POINTER(_Basis), P, P, I64, ctypes.c_double, P, ctypes.c_double,
                                      ctypes.c_int32, P, P, P]
    lib.mdx_exchange_grad.restype = I32
    lib.mdx_exchange_screen.argtypes = [P, ctypes.POINTER(_Basis), P, P, I64, ctypes.c_double, P, P, I64,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double), P]
    lib.mdx_exchange_screen.restype = I32
    lib.mdx_last_quartet_count.argtypes = [P]
    lib.mdx_last_quartet_count.restype = I64
    lib.mdx_eri4_noalloc.argtypes = [ctypes.POINTER(_Basis), P, I64, P, I64, P, P]
    lib.mdx_eri4_noalloc.restype = I32
    lib.mdx_xbatch_create.argtypes = [P, I32, P, P, P, ctypes.c_double, ctypes.POINTER(ctypes.c_void_p), P]
    lib.mdx_xbatch_create.restype = I32
    lib.mdx_xbatch_info.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    lib.mdx_xbatch_info.restype = I32
    lib.mdx_xbatch_run.argtypes = [P, P, I32, ctypes.POINTER(ctypes.c_int32), P]
    lib.mdx_xbatch_run.restype = I32
    lib.mdx_xbatch_launch_info.argtypes = [P, I32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double)]
    lib.mdx_xbatch_launch_info.restype = I32
    lib.mdx_xbatch_run_class.argtypes = [P, P, I32, P]
    lib.mdx_xbatch_run_class.restype = I32
    lib.mdx_xbatch_autotune.argtypes = [P, P, I64, P]
    lib.mdx_xbatch_autotune.restype = I32
    lib.mdx_xbatch_destroy.argtypes = [P]
    lib.mdx_xbatch_destroy.restype = None
    lib.mdx_plan_info.argtypes = [P, I32, I32, I32, I32, I32, I32, I32, ctypes.POINTER(PlanStats)]
    lib.mdx_plan_info.restype = I32
    lib.mdx_batch_run_materialized.argtypes = [P, P, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), P]
    lib.mdx_batch_run_materialized.restype = I32
    lib.mdx_set_class_shape.argtypes = [P] + [I32] * 10
    lib.mdx_set_class_shape.restype = I32
    lib.mdx_fp64_peak.argtypes = [I32, I32, ctypes.POINTER(ctypes.c_double), P]
    lib.mdx_fp64_peak.restype = I32
    _lib = lib
    return lib


STATUS = {0: "MDX_OK", 1: "MDX_EINVAL", 2: "MDX_ENOMEM", 3: "MDX_ECUDA", 4: "MDX_EUNSUPPORTED",
          5: "MDX_ECAPACITY", 6: "MDX_ETIMEOUT", 7: "MDX_EDEVICE", 8: "MDX_ESCRATCH"}


class DeviceBasis:
    """A seeded `inputs.Basis` copied to the device, with its ABI descriptor."""

    def __init__(self, basis, device="cuda"):
        self.host = basis
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        self.l = t(basis.l, torch.int32)
        self.nprim = t(basis.nprim, torch.int32)
        self.prim_off = t(basis.prim_off, torch.int32)
        self.ao_off = t(basis.ao_off, torch.int32)
        self.atom = t(basis.atom, torch.int32)
        self.center = t(basis.center, torch.float64)
        self.exps = t(basis.exps, torch.float64)
        self.coefs = t(basis.coefs, torch.float64)
        self.desc = _Basis(int(basis.n_shells), int(len(basis.exps)), self.l.data_ptr(), self.nprim.data_ptr(),
                           self.prim_off.data_ptr(), self.ao_off.data_ptr(), self.atom.data_ptr(),
                           self.center.data_ptr(), self.exps.data_ptr(), self.coefs.data_ptr())
        self.nc = (basis.l.astype(np.int64) + 1) * (basis.l.astype(np.int64) + 2) // 2


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Engine:
    """One mdx context on one CUDA device."""

    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise MdxError("no CUDA device: the mdx engine has no CPU path")
        self.lib = load()
        self.device = device
        torch.cuda.set_device(device)
        h = ctypes.c_void_p()
        st = self.lib.mdx_create(ctypes.byref(h), device)
        if st != 0:
            raise MdxError("mdx_create failed: %s" % STATUS.get(st, st))
        self.ctx = h

    def close(self):
        if getattr(self, "ctx", None):
            torch.cuda.synchronize()
            self.lib.mdx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.mdx_last_error(self.ctx).decode()
            raise MdxError("%s: %s (%s)" % (what, STATUS.get(st, st), msg))

    def sync(self):
        self._check(self.lib.mdx_sync(self.ctx, _stream()), "mdx_sync")

    # ----------------------------------------------------------------
    def eri4(self, basis: DeviceBasis, quartets, out: torch.Tensor = None, bound=None, tau: float = 0.0):
        """[ab|cd] for quartets [n,4] (device int32). Returns (values, offsets[n+1]).
        bound: optional [n] upper bounds on |(ab|cd)| (e.g. Q_ab Q_cd); quartets with bound < tau are
        written as zeros without being evaluated."""
        q = torch.as_tensor(quartets, dtype=torch.int32, device="cuda").contiguous()
        n = q.shape[0]
        if bound is not None:
            bound = torch.as_tensor(bound, dtype=torch.float64, device="cuda").contiguous()
            if bound.numel() != n:
                raise MdxError("mdx_eri4: bound needs one value per quartet")
        if out is None:
            qn = np.clip(q.cpu().numpy().astype(np.int64), 0, len(basis.nc) - 1)   # the ABI validates indices
            nc = basis.nc
            tot = int(np.sum(nc[qn[:, 0]] * nc[qn[:, 1]] * nc[qn[:, 2]] * nc[qn[:, 3]])) if n else 0
            out = torch.empty(max(tot, 1), dtype=torch.float64, device="cuda")
        _check_out(out, "mdx_eri4")
        offs = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        st = self.lib.mdx_eri4(self.ctx, ctypes.byref(basis.desc), q.data_ptr(), _opt_ptr(bound), n, float(tau),
                               out.data_ptr(), out.numel(), offs.data_ptr(), _stream())
        self._check(st, "mdx_eri4")
        return out, offs

    def eri4_sph(self, basis: DeviceBasis, quartets, out: torch.Tensor = None):
        """[ab|cd] over real solid harmonics (m = -l..l per shell). Returns (values, offsets)."""
        q = torch.as_tensor(quartets, dtype=torch.int32, device="cuda").contiguous()
        n = q.shape[0]
        if out is None:
            qn = np.clip(q.cpu().numpy().astype(np.int64), 0, len(basis.nc) - 1)
            ns = 2 * basis.host.l.astype(np.int64) + 1
            tot = int(np.sum(ns[qn[:, 0]] * ns[qn[:, 1]] * ns[qn[:, 2]] * ns[qn[:, 3]])) if n else 0
            out = torch.empty(max(tot, 1), dtype=torch.float64, device="cuda")
        _check_out(out, "mdx_eri4_sph")
        offs = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        st = self.lib.mdx_eri4_sph(self.ctx, ctypes.byref(basis.desc), q.data_ptr(), n, out.data_ptr(), out.numel(),
                                   offs.data_ptr(), _stream())
        self._check(st, "mdx_eri4_sph")
        return out, offs

    def eri3(self, aux: DeviceBasis, orb: DeviceBasis, triplets, out: torch.Tensor = None, bound=None,
             tau: float = 0.0):
        """[a|cd] for triplets [n,3] = (aux shell, orb shell, orb shell). Returns (values, offsets).
        bound / tau: optional per-triplet bounds and threshold, as in eri4."""
        t = torch.as_tensor(triplets, dtype=torch.int32, device="cuda").contiguous()
        n = t.shape[0]
        if bound is not None:
            bound = torch.as_tensor(bound, dtype=torch.float64, device="cuda").contiguous()
            if bound.numel() != n:
                raise MdxError("mdx_eri3: bound needs one value per triplet")
        if out is None:
            tn = t.cpu().numpy().astype(np.int64)
            tn[:, 0] = np.clip(tn[:, 0], 0, len(aux.nc) - 1)
            tn[:, 1:] = np.clip(tn[:, 1:], 0, len(orb.nc) - 1)
            tot = int(np.sum(aux.nc[tn[:, 0]] * orb.nc[tn[:, 1]] * orb.nc[tn[:, 2]])) if n else 0
            out = torch.empty(max(tot, 1), dtype=torch.float64, device="cuda")
        _check_out(out, "mdx_eri3")
        offs = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        st = self.lib.mdx_eri3(self.ctx, ctypes.byref(aux.desc), ctypes.byref(orb.desc), t.data_ptr(), _opt_ptr(bound),
                               n, float(tau), out.data_ptr(), out.numel(), offs.data_ptr(), _stream())
        self._check(st, "mdx_eri3")
        return out, offs

    def exchange(self, basis: DeviceBasis, pairs, Q, D: torch.Tensor, tau: float = 0.0, alpha: float = None):
        """K_ik = sum_jl D_jl (ij|kl) over the screened unique quartets of the pair list. With alpha given,
        returns (K, E_x) with E_x = alpha sum_ik D_ik K_ik computed by the library (device scalar)."""
        p = torch.as_tensor(pairs, dtype=torch.int32, device="cuda").contiguous()
        q = torch.as_tensor(Q, dtype=torch.float64, device="cuda").contiguous()
        D = D.to(device="cuda", dtype=torch.float64).contiguous()
        K = torch.empty_like(D)
        e = torch.zeros(1, dtype=torch.float64, device="cuda") if alpha is not None else None
        st = self.lib.mdx_exchange(self.ctx, ctypes.byref(basis.desc), p.data_ptr(), q.data_ptr(), p.shape[0],
                                   float(tau), D.data_ptr(), K.data_ptr(), float(alpha or 0.0), _opt_ptr(e),
                                   _stream())
        self._check(st, "mdx_exchange")
        return K if alpha is None else (K, e[0])

    def exchange_screen(self, basis: DeviceBasis, pairs, Q, D: torch.Tensor, tau: float = 0.0,
                        list_quartets: bool = True):
        """The screening of mdx_exchange alone: (kept [n,2] indices into `pairs` or None, n_kept,
        Table-1 model FLOPs of the kept shellsets)."""
        p = torch.as_tensor(pairs, dtype=torch.int32, device="cuda").contiguous()
        q = torch.as_tensor(Q, dtype=torch.float64, device="cuda").contiguous()
        D = D.to(device="cuda", dtype=torch.float64).contiguous()
        n, mf = ctypes.c_int64(), ctypes.c_double()
        st = self.lib.mdx_exchange_screen(self.ctx, ctypes.byref(basis.desc), p.data_ptr(), q.data_ptr(),
                                          p.shape[0], float(tau), D.data_ptr(), None, 0, ctypes.byref(n),
                                          ctypes.byref(mf), _stream())
        self._check(st, "mdx_exchange_screen")
        if not list_quartets:
            return None, n.value, mf.value
        kept = torch.empty((max(n.value, 1), 2), dtype=torch.int32, device="cuda")
        st = self.lib.mdx_exchange_screen(self.ctx, ctypes.byref(basis.desc), p.data_ptr(), q.data_ptr(),
                                          p.shape[0], float(tau), D.data_ptr(), kept.data_ptr(), kept.shape[0],
                                          ctypes.byref(n), ctypes.byref(mf), _stream())
        self._check(st, "mdx_exchange_screen")
        return kept[: n.value], n.value, mf.value

    def exchange_grad(self, basis: DeviceBasis, pairs, Q, D: torch.Tensor, tau: float = 0.0, alpha: float = -1.0,
                      n_atoms: int = None, with_energy: bool = True):
        """(dE_x/dR [n_atoms, 3], E_x) for E_x = alpha sum_ijkl D_ik D_jl (ij|kl), D fixed."""
        p = torch.as_tensor(pairs, dtype=torch.int32, device="cuda").contiguous()
        q = torch.as_tensor(Q, dtype=torch.float64, device="cuda").contiguous()
        D = D.to(device="cuda", dtype=torch.float64).contiguous()
        if n_atoms is None:
            n_atoms = int(basis.host.atom.max()) + 1
        g = torch.empty((n_atoms, 3), dtype=torch.float64, device="cuda")
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = self.lib.mdx_exchange_grad(self.ctx, ctypes.byref(basis.desc), p.data_ptr(), q.data_ptr(), p.shape[0],
                                        float(tau), D.data_ptr(), float(alpha), int(n_atoms), g.data_ptr(),
                                        e.data_ptr() if with_energy else None, _stream())
        self._check(st, "mdx_exchange_grad")
        return g, (e[0] if with_energy else None)

    def plan_info(self, la, lb, lc, ld, Kb=1, Kk=1, one_centre=False) -> PlanStats:
        """The shape this engine uses for a class (tuned or fixed shapes included)."""
        st = PlanStats()
        self._check(self.lib.mdx_plan_info(self.ctx, la, lb, lc, ld, Kb, Kk, int(one_centre), ctypes.byref(st)),
                    "mdx_plan_info")
        return st

    def set_class_shape(self, la, lb, lc, ld, Kb=1, Kk=1, one_centre=False, team_threads=0, smem_budget=0,
                        variant=0):
        """Fix a class's shape (variant 0: default, 1: team kernel, 2: register kernel)."""
        self._check(self.lib.mdx_set_class_shape(self.ctx, la, lb, lc, ld, Kb, Kk, int(one_centre), team_threads,
                                                 smem_budget, variant), "mdx_set_class_shape")

    def last_quartet_count(self) -> int:
        return int(self.lib.mdx_last_quartet_count(self.ctx))

    def xbatch(self, bases, Ds, tau: float = 0.0) -> "ExchangeBatch":
        """Prepare the exchange builds of several molecules (see mdx_xbatch_create)."""
        return ExchangeBatch(self, bases, Ds, tau)

    def batch_eri4(self, basis: DeviceBasis, quartets) -> "Batch":
        """Prepare quartets [n,4] once; run them many times with Batch.run."""
        q = torch.as_tensor(quartets, dtype=torch.int32, device="cuda").contiguous()
        h = ctypes.c_void_p()
        self._check(self.lib.mdx_batch_eri4(self.ctx, ctypes.byref(basis.desc), q.data_ptr(), q.shape[0],
                                            ctypes.byref(h), _stream()), "mdx_batch_eri4")
        return Batch(self, h, (basis,))

    def batch_eri4_sph(self, basis: DeviceBasis, quartets) -> "Batch":
        """Prepare quartets [n,4] for solid-harmonic output (see mdx_batch_eri4_sph)."""
        q = torch.as_tensor(quartets, dtype=torch.int32, device="cuda").contiguous()
        h = ctypes.c_void_p()
        self._check(self.lib.mdx_batch_eri4_sph(self.ctx, ctypes.byref(basis.desc), q.data_ptr(), q.shape[0],
                                                ctypes.byref(h), _stream()), "mdx_batch_eri4_sph")
        return Batch(self, h, (basis,))

    def eri3_sph(self, aux: DeviceBasis, orb: DeviceBasis, triplets, out: torch.Tensor = None):
        """[a|cd] over real solid harmonics (a, c and d: m = -l..l). Returns (values, offsets)."""
        t = torch.as_tensor(triplets, dtype=torch.int32, device="cuda").contiguous()
        n = t.shape[0]
        if out is None:
            tn = t.cpu().numpy().astype(np.int64)
            tn[:, 0] = np.clip(tn[:, 0], 0, len(aux.nc) - 1)
            tn[:, 1:] = np.clip(tn[:, 1:], 0, len(orb.nc) - 1)
            na = 2 * aux.host.l.astype(np.int64) + 1
            no = 2 * orb.host.l.astype(np.int64) + 1
            tot = int(np.sum(na[tn[:, 0]] * no[tn[:, 1]] * no[tn[:, 2]])) if n else 0
            out = torch.empty(max(tot, 1), dtype=torch.float64, device="cuda")
        _check_out(out, "mdx_eri3_sph")
        offs = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        st = self.lib.mdx_eri3_sph(self.ctx, ctypes.byref(aux.desc), ctypes.byref(orb.desc), t.data_ptr(), n,
                                   out.data_ptr(), out.numel(), offs.data_ptr(), _stream())
        self._check(st, "mdx_eri3_sph")
        return out, offs

    def batch_eri3_sph(self, aux: DeviceBasis, orb: DeviceBasis, triplets) -> "Batch":
        """Prepare triplets [n,3] for solid-harmonic output (see mdx_batch_eri3_sph)."""
        t = torch.as_tensor(triplets, dtype=torch.int32, device="cuda").contiguous()
        h = ctypes.c_void_p()
        self._check(self.lib.mdx_batch_eri3_sph(self.ctx, ctypes.byref(aux.desc), ctypes.byref(orb.desc),
                                                t.data_ptr(), t.shape[0], ctypes.byref(h), _stream()),
                    "mdx_batch_eri3_sph")
        return Batch(self, h, (aux, orb))

    def batch_eri3(self, aux: DeviceBasis, orb: DeviceBasis, triplets) -> "Batch":
        t = torch.as_tensor(triplets, dtype=torch.int32, device="cuda").contiguous()
        h = ctypes.c_void_p()
        self._check(self.lib.mdx_batch_eri3(self.ctx, ctypes.byref(aux.desc), ctypes.byref(orb.desc), t.data_ptr(),
                                            t.shape[0], ctypes.byref(h), _stream()), "mdx_batch_eri3")
        return Batch(self, h, (aux, orb))

    def schwarz(self, basis: DeviceBasis, pairs):
        """Q_ij = sqrt(max |(ij|ij)|) for pairs [n,2]."""
        p = torch.as_tensor(pairs, dtype=torch.int32, device="cuda").contiguous()
        Q = torch.empty(max(p.shape[0], 1), dtype=torch.float64, device="cuda")
        st = self.lib.mdx_schwarz(self.ctx, ctypes.byref(basis.desc), p.data_ptr(), p.shape[0], Q.data_ptr(),
                                  _stream())
        self._check(st, "mdx_schwarz")
        return Q[: p.shape[0]]


class Batch:
    """A prepared quartet (or triplet) list; `run` enqueues the whole hot path."""

    def __init__(self, eng: Engine, handle, keep):
        self.eng, self.h, self._keep = eng, handle, keep
        self._read_info()

    def _read_info(self):
        n, tot = ctypes.c_int64(), ctypes.c_int64()
        mf, ef = ctypes.c_double(), ctypes.c_double()
        self.eng._check(self.eng.lib.mdx_batch_info(self.h, ctypes.byref(n), ctypes.byref(tot), ctypes.byref(mf),
                                                    ctypes.byref(ef)), "mdx_batch_info")
        self.n, self.total, self.model_flops, self.exec_fma = n.value, tot.value, mf.value, ef.value

    def offsets(self) -> torch.Tensor:
        o = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        self.eng._check(self.eng.lib.mdx_batch_offsets(self.eng.ctx, self.h, o.data_ptr(), _stream()),
                        "mdx_batch_offsets")
        return o

    def run(self, out: torch.Tensor) -> int:
        """Enqueue on the current stream; returns the number of kernels launched."""
        _check_out(out, "mdx_batch_run")
        nl = ctypes.c_int32()
        self.eng._check(self.eng.lib.mdx_batch_run(self.eng.ctx, self.h, out.data_ptr(), out.numel(),
                                                   ctypes.byref(nl), _stream()), "mdx_batch_run")
        return nl.value

    def run_materialized(self, out: torch.Tensor) -> int:
        """The materialized-Hermite variant (dense [p|q] matrices, batched DGEMMs); uncontracted classes only."""
        _check_out(out, "mdx_batch_run_materialized")
        nl = ctypes.c_int32()
        self.eng._check(self.eng.lib.mdx_batch_run_materialized(self.eng.ctx, self.h, out.data_ptr(), out.numel(),
                                                                ctypes.byref(nl), _stream()),
                        "mdx_batch_run_materialized")
        return nl.value

    def autotune(self, out: torch.Tensor, max_trial: int = 256):
        """Pick the fastest team shape per class on this GPU (kept by the engine); exec_fma then counts
        the shapes the batch runs."""
        _check_out(out, "mdx_batch_autotune")
        self.eng._check(self.eng.lib.mdx_batch_autotune(self.eng.ctx, self.h, out.data_ptr(), out.numel(), max_trial,
                                                        _stream()), "mdx_batch_autotune")
        self._read_info()

    def close(self):
        if self.h:
            self.eng.lib.mdx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def basis_with_centers(basis: DeviceBasis, coords: torch.Tensor) -> DeviceBasis:
    """A copy of `basis` whose shell centres are coords[atom of shell] (coords: [n_atoms, 3], any device
    and floating dtype; the centres are copied to the basis's device in float64)."""
    nb = DeviceBasis.__new__(DeviceBasis)
    nb.__dict__.update(basis.__dict__)
    c = coords.detach().to(device=basis.center.device, dtype=torch.float64)
    nb.center = c[basis.atom.long()].contiguous()
    nb.desc = _Basis(basis.desc.n_shells, basis.desc.n_prims, basis.l.data_ptr(), basis.nprim.data_ptr(),
                     basis.prim_off.data_ptr(), basis.ao_off.data_ptr(), basis.atom.data_ptr(), nb.center.data_ptr(),
                     basis.exps.data_ptr(), basis.coefs.data_ptr())
    return nb


class ExchangeEnergy(torch.autograd.Function):
    """E_x = alpha sum_ijkl D_ik D_jl (ij|kl) as a differentiable function of the
    atom coordinates and of a symmetric D. Forward: mdx_exchange, which returns
    K and E_x = alpha sum D o K. Backward: mdx_exchange_grad for the coordinates
    (derivative integrals contracted with D (x) D inside the kernel) and
    2 alpha K for D (the derivative for symmetric D; a D that is not symmetric
    is rejected in forward, since the library's K assumes symmetry)."""

    @staticmethod
    def forward(ctx, coords, D, eng, basis, pairs, tau, alpha):
        db = basis_with_centers(basis, coords)
        Q = eng.schwarz(db, pairs)
        Dd = D.detach().to(device="cuda", dtype=torch.float64).contiguous()
        if Dd.dim() != 2 or Dd.shape[0] != Dd.shape[1] or not torch.equal(Dd, Dd.T):
            raise MdxError("ExchangeEnergy: D must be a symmetric square matrix")
        K, E = eng.exchange(db, pairs, Q, Dd, tau, alpha=alpha)
        ctx.eng, ctx.db, ctx.pairs, ctx.tau, ctx.alpha = eng, db, pairs, tau, alpha
        ctx.n_atoms = coords.shape[0]
        ctx.coords_like = (coords.device, coords.dtype)
        ctx.D_like = (D.device, D.dtype)
        ctx.save_for_backward(Dd, K, Q)
        return E.to(device=D.device, dtype=D.dtype)

    @staticmethod
    def backward(ctx, gE):
        Dd, K, Q = ctx.saved_tensors
        gcoords = gD = None
        if ctx.needs_input_grad[0]:
            g, _ = ctx.eng.exchange_grad(ctx.db, ctx.pairs, Q, Dd, tau=ctx.tau, alpha=ctx.alpha, n_atoms=ctx.n_atoms,
                                         with_energy=False)
            dev, dt = ctx.coords_like
            gcoords = (gE.to(device=g.device, dtype=g.dtype) * g).to(device=dev, dtype=dt)
        if ctx.needs_input_grad[1]:
            dev, dt = ctx.D_like
            gD = (gE.to(device=K.device, dtype=K.dtype) * 2.0 * ctx.alpha * K).to(device=dev, dtype=dt)
        return gcoords, gD, None, None, None, None, None


def exchange_energy(eng: Engine, basis: DeviceBasis, coords: torch.Tensor, D: torch.Tensor, pairs=None,
                    tau: float = 0.0, alpha: float = -1.0) -> torch.Tensor:
    """Differentiable exchange energy (see ExchangeEnergy); pairs default to all shell pairs."""
    if pairs is None:
        n = basis.desc.n_shells
        pairs = torch.tensor([(i, j) for i in range(n) for j in range(i + 1)], dtype=torch.int32, device="cuda")
    return ExchangeEnergy.apply(coords, D, eng, basis, pairs, tau, alpha)


class ExchangeBatch:
    """Exchange matrices of several molecules: one launch per class, one persistent launch,
    or the register-kernel classes per class plus one persistent launch for the rest."""

    def __init__(self, eng: Engine, bases, Ds, tau: float):
        self.eng = eng
        self.bases = list(bases)
        self.Ds = [D.to(device="cuda", dtype=torch.float64).contiguous() for D in Ds]
        self.Ks = [torch.empty_like(D) for D in self.Ds]
        n = len(self.bases)
        arr = (_Basis * n)(*[b.desc for b in self.bases])
        dp = (ctypes.c_void_p * n)(*[D.data_ptr() for D in self.Ds])
        kp = (ctypes.c_void_p * n)(*[K.data_ptr() for K in self.Ks])
        h = ctypes.c_void_p()
        eng._check(eng.lib.mdx_xbatch_create(eng.ctx, n, arr, dp, kp, float(tau), ctypes.byref(h), _stream()),
                   "mdx_xbatch_create")
        self.h = h
        nq, ni, nl, mf = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
        eng._check(eng.lib.mdx_xbatch_info(h, ctypes.byref(nq), ctypes.byref(ni), ctypes.byref(nl), ctypes.byref(mf)),
                   "mdx_xbatch_info")
        self.n_quartets, self.n_items, self.n_class_launches = nq.value, ni.value, nl.value
        self.model_flops = mf.value

    def run(self, persistent: int = 1) -> int:
        """Enqueue on the current stream (capturable); returns kernels launched. Results in self.Ks.
        persistent: 0 one launch per class, 1 one persistent launch, 2 register-kernel classes
        per class and one persistent launch for the others (True/False mean 1/0)."""
        nl = ctypes.c_int32()
        self.eng._check(self.eng.lib.mdx_xbatch_run(self.eng.ctx, self.h, int(persistent), ctypes.byref(nl),
                                                    _stream()), "mdx_xbatch_run")
        return nl.value

    def launch_info(self, i: int):
        """(la, lb, lc, ld, K_ab, K_cd), kept quartets and model FLOPs of per-class launch i."""
        lk = (ctypes.c_int32 * 6)()
        nq, mf = ctypes.c_int64(), ctypes.c_double()
        self.eng._check(self.eng.lib.mdx_xbatch_launch_info(self.h, int(i), lk, ctypes.byref(nq), ctypes.byref(mf)),
                        "mdx_xbatch_launch_info")
        return tuple(lk), nq.value, mf.value

    def autotune(self, max_trial: int = 65536):
        """Pick the fastest shape (register kernel or team shape) of every per-class launch on this GPU
        (kept by the engine for later calls). Leaves partial sums in self.Ks: run() again before reading them."""
        self.eng._check(self.eng.lib.mdx_xbatch_autotune(self.eng.ctx, self.h, int(max_trial), _stream()),
                        "mdx_xbatch_autotune")

    def run_class(self, i: int):
        """Enqueue the integral kernel of per-class launch i alone (no K zeroing / symmetrisation)."""
        self.eng._check(self.eng.lib.mdx_xbatch_run_class(self.eng.ctx, self.h, int(i), _stream()),
                        "mdx_xbatch_run_class")

    def close(self):
        if self.h:
            self.eng.lib.mdx_xbatch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
