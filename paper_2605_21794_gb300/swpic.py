"""Thin Python binding of the C ABI in include/swpic.h.

Functions carry the C names and only marshal arguments; every step of the
decorated-particle path runs in the CUDA kernels of ``libswpic.so``.  PyTorch
supplies device memory (the particle tensors) and the stream.  There is no
CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libswpic.so")

SWPIC_OK, SWPIC_EINVAL, SWPIC_ENOMEM, SWPIC_ECUDA = 0, 1, 2, 3
SWPIC_ETIMEOUT, SWPIC_ENUMERIC, SWPIC_EUNSUPPORTED, SWPIC_ESTATE, SWPIC_EIO = 4, 5, 6, 7, 8
SWPIC_F32, SWPIC_F64 = 32, 64
SWPIC_DEPOSIT_ATOMIC, SWPIC_DEPOSIT_DETERMINISTIC = 0, 1
SWPIC_D2_LUMPED, SWPIC_D2_NODAL, SWPIC_D2_P2 = 0, 2, 3
SWPIC_NX_MAX = 4096
SWPIC_STATIC_NX_MAX = 4096
SWPIC_FIELD_SOLVE_AUTO, SWPIC_FIELD_SOLVE_LAST_CTA, SWPIC_FIELD_SOLVE_AT_START = 0, 1, 2


class swpic_config(C.Structure):
    _fields_ = [("L", C.c_double), ("dt", C.c_double), ("nx", C.c_int32),
                ("precision", C.c_int32), ("decorated", C.c_int32),
                ("deposit_mode", C.c_int32), ("d2_mode", C.c_int32),
                ("resort_every", C.c_int32), ("threads_per_block", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("use_graphs", C.c_int32),
                ("diag_capacity", C.c_int32)]


class swpic_diag(C.Structure):
    _fields_ = [("t", C.c_double), ("mass", C.c_double), ("momentum", C.c_double),
                ("kinetic", C.c_double), ("field_energy", C.c_double),
                ("hamiltonian", C.c_double), ("e_amp", C.c_double), ("step", C.c_int64)]


class swpic_lattice(C.Structure):
    _fields_ = [("nq", C.c_int32), ("nv", C.c_int32), ("vmin", C.c_double),
                ("vmax", C.c_double), ("alpha", C.c_double), ("kx", C.c_double),
                ("n_terms", C.c_int32), ("quad_order", C.c_int32),
                ("amp", C.c_double * 4), ("c0", C.c_double * 4), ("c2", C.c_double * 4),
                ("beta", C.c_double * 4), ("u", C.c_double * 4),
                ("decorate", C.c_int32), ("reserved", C.c_int32)]


class swpic2d_config(C.Structure):
    _fields_ = [("Lx", C.c_double), ("Ly", C.c_double), ("dt", C.c_double), ("nx", C.c_int32),
                ("ny", C.c_int32), ("precision", C.c_int32), ("decorated", C.c_int32),
                ("threads_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("diag_capacity", C.c_int32), ("reserved", C.c_int32)]


class swpic2d_lattice(C.Structure):
    _fields_ = [("nqx", C.c_int32), ("nqy", C.c_int32), ("nvx", C.c_int32), ("nvy", C.c_int32),
                ("vmin", C.c_double), ("vmax", C.c_double), ("alpha", C.c_double), ("kx", C.c_double),
                ("ky", C.c_double), ("vth", C.c_double), ("quad_order", C.c_int32), ("decorate", C.c_int32)]


class swpic2d_diag(C.Structure):
    _fields_ = [("t", C.c_double), ("mass", C.c_double), ("momentum_x", C.c_double),
                ("momentum_y", C.c_double), ("kinetic", C.c_double), ("field_energy", C.c_double),
                ("hamiltonian", C.c_double), ("e_amp", C.c_double), ("step", C.c_int64)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_CTX = C.c_void_p

# name -> (restype, argtypes); the full exported surface of include/swpic.h
SIGNATURES = {
    "swpic_abi_version": (C.c_int32, []),
    "swpic_status_string": (C.c_char_p, [C.c_int]),
    "swpic_last_error": (C.c_char_p, [_CTX]),
    "swpic_create": (C.c_int, [C.POINTER(swpic_config), C.c_int64, C.POINTER(_CTX)]),
    "swpic_create_batch": (C.c_int, [C.POINTER(swpic_config), C.c_int32,
                                     C.POINTER(C.c_int64), C.POINTER(_CTX)]),
    "swpic_destroy": (None, [_CTX]),
    "swpic_scratch_bytes": (C.c_int, [_CTX, C.POINTER(C.c_int64)]),
    "swpic_bind_state": (C.c_int, [_CTX, _P, _P, _P, _P, _P, _P, C.c_int64, _P]),
    "swpic_init_particles": (C.c_int, [_CTX, _D, _D, _D, _D, _D, C.c_int64]),
    "swpic_init_lattice": (C.c_int, [_CTX, C.c_int32, C.POINTER(swpic_lattice), _D, _D]),
    "swpic_refresh": (C.c_int, [_CTX]),
    "swpic_deposit": (C.c_int, [_CTX]),
    "swpic_solve_field": (C.c_int, [_CTX]),
    "swpic_gather_push": (C.c_int, [_CTX, C.c_double, C.c_double]),
    "swpic_sort": (C.c_int, [_CTX]),
    "swpic_step": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "swpic_diagnostics": (C.c_int, [_CTX, C.c_int32, C.POINTER(swpic_diag), C.c_int32,
                                    C.POINTER(C.c_int32)]),
    "swpic_get_mesh": (C.c_int, [_CTX, C.c_int32, _D, _D, _D, _D, _D]),
    "swpic_get_keys": (C.c_int, [_CTX, C.POINTER(C.c_int32), C.c_int64]),
    "swpic_synchronize": (C.c_int, [_CTX]),
    "swpic_run_status": (C.c_int, [_CTX, C.POINTER(C.c_int32), C.c_int32]),
    "swpic_step_host": (C.c_int, [_CTX, _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_int64,
                                  C.c_int32, C.c_int32]),
    "swpic_deposit_static": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, C.c_double, C.c_int32,
                                       _P, _P]),
    "swpic_kmeans_lump": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, C.c_int32, C.c_double, C.c_int32,
                                    _P, _P, _P, _P, _P, _P, C.POINTER(C.c_int64), _P]),
    "swpic_save": (C.c_int, [_CTX, C.c_char_p]),
    "swpic_load": (C.c_int, [_CTX, C.c_char_p]),
    "swpic_set_launch": (C.c_int, [_CTX, C.c_int32, C.c_int32, C.c_int32]),
    "swpic_get_launch": (C.c_int, [_CTX, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)]),
    "swpic_autotune": (C.c_int, [_CTX, C.c_int32, C.c_char_p]),
    "swpic_set_pipeline": (C.c_int, [_CTX, C.c_int32]),
    "swpic_get_pipeline": (C.c_int, [_CTX, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "swpic_set_wait_test": (C.c_int, [_CTX, C.c_int32, C.c_int64]),
    "swpic_set_field_solve": (C.c_int, [_CTX, C.c_int32]),
    "swpic_get_field_solve": (C.c_int, [_CTX, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "swpic_set_timing": (C.c_int, [_CTX, C.c_int32]),
    "swpic_pass_times": (C.c_int, [_CTX, C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_int32)]),
    "swpic_launch_count": (C.c_int, [_CTX, C.POINTER(C.c_int64)]),
    # include/swpic2d.h
    "swpic2d_create": (C.c_int, [C.POINTER(swpic2d_config), C.c_int64, C.POINTER(_CTX)]),
    "swpic2d_destroy": (None, [_CTX]),
    "swpic2d_last_error": (C.c_char_p, [_CTX]),
    "swpic2d_bind_state": (C.c_int, [_CTX, C.POINTER(_P), _P]),
    "swpic2d_refresh": (C.c_int, [_CTX]),
    "swpic2d_init_lattice": (C.c_int, [_CTX, C.POINTER(swpic2d_lattice)]),
    "swpic2d_step": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "swpic2d_diagnostics": (C.c_int, [_CTX, C.POINTER(swpic2d_diag), C.c_int32, C.POINTER(C.c_int32)]),
    "swpic2d_get_field": (C.c_int, [_CTX, _D, _D, _D, _D]),
    "swpic2d_synchronize": (C.c_int, [_CTX]),
    "swpic2d_step_host": (C.c_int, [_CTX, C.POINTER(_P), C.POINTER(_P), C.c_int32, C.c_int32]),
    "swpic2d_save": (C.c_int, [_CTX, C.c_char_p]),
    "swpic2d_load": (C.c_int, [_CTX, C.c_char_p]),
    "swpic2d_set_timing": (C.c_int, [_CTX, C.c_int32]),
    "swpic2d_pass_times": (C.c_int, [_CTX, C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_int32)]),
    "swpic2d_launch_count": (C.c_int, [_CTX, C.POINTER(C.c_int64)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libswpic.so (build it with ``python -m paper_2605_21794_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libswpic.so not found at %s: the CUDA extension must be built "
                           "(python -c 'import __graft_entry__ as g; g.build()'); "
                           "there is no CPU fallback" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SwpicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


def _check(st, ctx=None, last_error="swpic_last_error"):
    if st != SWPIC_OK:
        lib = load_library()
        msg = getattr(lib, last_error)(ctx).decode() if ctx else ""
        raise SwpicError(st, "%s: %s" % (lib.swpic_status_string(st).decode(), msg))


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_D)


# ---------------------------------------------------------------------------
# same-name wrappers (argument marshalling only)
# ---------------------------------------------------------------------------
def make_config(L, dt, nx, precision=32, decorated=True, deposit_mode=0, d2_mode=0,
                resort_every=0, threads_per_block=0, blocks_per_sm=0, use_graphs=True,
                diag_capacity=0):
    return swpic_config(float(L), float(dt), int(nx), int(precision), int(bool(decorated)),
                        int(deposit_mode), int(d2_mode), int(resort_every),
                        int(threads_per_block), int(blocks_per_sm), int(bool(use_graphs)),
                        int(diag_capacity))


def swpic_create(cfg: swpic_config, n_particles: int):
    lib = load_library()
    ctx = _CTX()
    _check(lib.swpic_create(C.byref(cfg), int(n_particles), C.byref(ctx)))
    return ctx


def swpic_create_batch(cfgs: Sequence[swpic_config], offsets: Sequence[int]):
    lib = load_library()
    arr = (swpic_config * len(cfgs))(*cfgs)
    off = (C.c_int64 * len(offsets))(*[int(x) for x in offsets])
    ctx = _CTX()
    _check(lib.swpic_create_batch(arr, len(cfgs), off, C.byref(ctx)))
    return ctx


def swpic_destroy(ctx):
    load_library().swpic_destroy(ctx)


def swpic_scratch_bytes(ctx):
    n = C.c_int64(0)
    _check(load_library().swpic_scratch_bytes(ctx, C.byref(n)), ctx)
    return n.value


def swpic_bind_state(ctx, Q, P, qs, ps, psi, scratch, scratch_bytes, stream):
    _check(load_library().swpic_bind_state(ctx, Q, P, qs, ps, psi, scratch, int(scratch_bytes),
                                           stream), ctx)


def swpic_init_particles(ctx, Q, P, qs, ps, psi):
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64)
            for a in (Q, P, qs, ps, psi)]
    _check(load_library().swpic_init_particles(ctx, *[_dptr(a) for a in arrs], len(arrs[0])), ctx)


def lattice_struct(spec) -> swpic_lattice:
    """swpic_lattice from a workloads.LatticeSpec."""
    s = swpic_lattice()
    s.nq, s.nv = spec.nq, spec.nv
    s.vmin, s.vmax, s.alpha, s.kx = spec.vmin, spec.vmax, spec.alpha, spec.kx
    s.n_terms = len(spec.terms)
    s.quad_order = spec.quad_order
    for m, (amp, c0, c2, beta, u) in enumerate(spec.terms):
        s.amp[m], s.c0[m], s.c2[m], s.beta[m], s.u[m] = amp, c0, c2, beta, u
    s.decorate = int(bool(spec.decorate))
    return s


def swpic_init_lattice(ctx, run, spec: swpic_lattice, jitter_x=None, jitter_v=None):
    jx = None if jitter_x is None else np.ascontiguousarray(jitter_x, dtype=np.float64)
    jv = None if jitter_v is None else np.ascontiguousarray(jitter_v, dtype=np.float64)
    _check(load_library().swpic_init_lattice(ctx, int(run), C.byref(spec), _dptr(jx), _dptr(jv)), ctx)


def swpic_refresh(ctx):
    _check(load_library().swpic_refresh(ctx), ctx)


def swpic_deposit(ctx):
    _check(load_library().swpic_deposit(ctx), ctx)


def swpic_solve_field(ctx):
    _check(load_library().swpic_solve_field(ctx), ctx)


def swpic_gather_push(ctx, kick_fraction, drift_fraction):
    _check(load_library().swpic_gather_push(ctx, float(kick_fraction), float(drift_fraction)), ctx)


def swpic_sort(ctx):
    _check(load_library().swpic_sort(ctx), ctx)


def swpic_step(ctx, n_steps, diag_every=0):
    _check(load_library().swpic_step(ctx, int(n_steps), int(diag_every)), ctx)


DIAG_FIELDS = ["t", "mass", "momentum", "kinetic", "field_energy", "hamiltonian", "e_amp", "step"]


def swpic_diagnostics(ctx, run=0, max_records=100000):
    buf = (swpic_diag * max_records)()
    n = C.c_int32(0)
    _check(load_library().swpic_diagnostics(ctx, int(run), buf, int(max_records), C.byref(n)), ctx)
    out = np.zeros((n.value, 8))
    for k in range(n.value):
        d = buf[k]
        out[k] = [d.t, d.mass, d.momentum, d.kinetic, d.field_energy, d.hamiltonian, d.e_amp,
                  d.step]
    return out


def swpic_get_mesh(ctx, run, nx):
    arrs = {k: np.zeros(nx) for k in ("b", "btilde", "Phi", "E", "d2")}
    _check(load_library().swpic_get_mesh(ctx, int(run), *[_dptr(arrs[k]) for k in
                                                           ("b", "btilde", "Phi", "E", "d2")]), ctx)
    return arrs


def swpic_get_keys(ctx, n):
    keys = np.zeros(n, dtype=np.int32)
    _check(load_library().swpic_get_keys(ctx, keys.ctypes.data_as(C.POINTER(C.c_int32)), int(n)),
           ctx)
    return keys


def swpic_synchronize(ctx):
    _check(load_library().swpic_synchronize(ctx), ctx)


def swpic_run_status(ctx, n_runs):
    flags = np.zeros(n_runs, dtype=np.int32)
    _check(load_library().swpic_run_status(ctx, flags.ctypes.data_as(C.POINTER(C.c_int32)),
                                           int(n_runs)), ctx)
    return flags


def swpic_step_host(ctx, Q, P, qs, ps, psi, Q_out, P_out, qs_out, ps_out, n, n_steps,
                    diag_every=0):
    _check(load_library().swpic_step_host(ctx, Q, P, qs, ps, psi, Q_out, P_out, qs_out, ps_out,
                                          int(n), int(n_steps), int(diag_every)), ctx)


def swpic_deposit_static(Q, ps, psi, n, precision, L, nx, b, stream):
    """Device pointers in/out (see include/swpic.h); allocates nothing."""
    _check(load_library().swpic_deposit_static(Q, ps, psi, int(n), int(precision), float(L),
                                               int(nx), b, stream))


def swpic_kmeans_lump(Qm, Pm, wm, M, cq, cp, K, L, n_iter, assign, Q, P, qs, ps, psi, stream):
    """Device pointers in/out (see include/swpic.h); returns the number of
    decorated particles written."""
    n = C.c_int64(0)
    _check(load_library().swpic_kmeans_lump(Qm, Pm, wm, int(M), cq, cp, int(K), float(L), int(n_iter),
                                            assign, Q, P, qs, ps, psi, C.byref(n), stream))
    return n.value


def swpic_save(ctx, path):
    _check(load_library().swpic_save(ctx, path.encode()), ctx)


def swpic_load(ctx, path):
    _check(load_library().swpic_load(ctx, path.encode()), ctx)


def swpic_set_launch(ctx, threads_per_block=0, blocks_per_sm=0, resort_every=0):
    _check(load_library().swpic_set_launch(ctx, int(threads_per_block), int(blocks_per_sm),
                                           int(resort_every)), ctx)


def swpic_get_launch(ctx):
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load_library().swpic_get_launch(ctx, C.byref(a), C.byref(b), C.byref(c)), ctx)
    return a.value, b.value, c.value


def swpic_autotune(ctx, steps_per_trial=5, cache_path=None):
    _check(load_library().swpic_autotune(ctx, int(steps_per_trial),
                                         None if cache_path is None else cache_path.encode()), ctx)


def swpic_set_pipeline(ctx, stages):
    _check(load_library().swpic_set_pipeline(ctx, int(stages)), ctx)


def swpic_get_pipeline(ctx):
    """(requested, effective) bulk-copy stage counts; 0 = register loads."""
    a, b = C.c_int32(), C.c_int32()
    _check(load_library().swpic_get_pipeline(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def swpic_set_field_solve(ctx, mode):
    _check(load_library().swpic_set_field_solve(ctx, int(mode)), ctx)


def swpic_get_field_solve(ctx):
    """(requested, effective) field-solve placement (SWPIC_FIELD_SOLVE_*)."""
    a, b = C.c_int32(), C.c_int32()
    _check(load_library().swpic_get_field_solve(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def swpic_set_wait_test(ctx, stall_warp=-1, wait_limit_ns=0):
    _check(load_library().swpic_set_wait_test(ctx, int(stall_warp), int(wait_limit_ns)), ctx)


def swpic_set_timing(ctx, enable):
    _check(load_library().swpic_set_timing(ctx, int(bool(enable))), ctx)


def swpic_pass_times(ctx, max_passes=100000):
    buf = (C.c_float * max_passes)()
    n = C.c_int32(0)
    _check(load_library().swpic_pass_times(ctx, buf, int(max_passes), C.byref(n)), ctx)
    return np.array(buf[: n.value], dtype=np.float64)


def swpic_launch_count(ctx):
    n = C.c_int64(0)
    _check(load_library().swpic_launch_count(ctx, C.byref(n)), ctx)
    return n.value


# ---------------------------------------------------------------------------
# Convenience owner of torch device memory for one context (tests, bench)
# ---------------------------------------------------------------------------
class Simulation:
    """Owns the particle tensors (torch, cuda) and a context bound to them.

    runs: list of (L, dt, nx, n_particles); all runs share precision etc.
    """

    def __init__(self, runs, precision=32, decorated=True, deposit_mode=0, d2_mode=0,
                 resort_every=0, threads_per_block=0, blocks_per_sm=0, use_graphs=True,
                 diag_capacity=0, with_scratch=True, stream=None, device="cuda",
                 pipeline_stages=None):
        import torch
        self.torch = torch
        self.precision = precision
        self.decorated = decorated
        self.dtype = torch.float64 if precision == 64 else torch.float32
        self.runs = list(runs)
        self.offsets = [0]
        for (_, _, _, n) in self.runs:
            self.offsets.append(self.offsets[-1] + int(n))
        self.n = self.offsets[-1]
        cfgs = [make_config(L, dt, nx, precision, decorated, deposit_mode, d2_mode, resort_every,
                            threads_per_block, blocks_per_sm, use_graphs, diag_capacity)
                for (L, dt, nx, _) in self.runs]
        self.ctx = swpic_create_batch(cfgs, self.offsets)
        if pipeline_stages is not None:
            swpic_set_pipeline(self.ctx, pipeline_stages)
        n = max(self.n, 1)
        mk = lambda: torch.zeros(n, dtype=self.dtype, device=device)
        self.Q, self.P, self.psi = mk(), mk(), mk()
        self.qs = mk() if decorated else None
        self.ps = mk() if decorated else None
        self.scratch = None
        sb = swpic_scratch_bytes(self.ctx)
        if with_scratch and sb > 0:
            self.scratch = torch.empty(sb + 256, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        ptr = lambda t: None if t is None else t.data_ptr()
        sp = self.scratch.data_ptr() if self.scratch is not None else None
        if sp is not None and sp % 256:
            sp += 256 - sp % 256
        swpic_bind_state(self.ctx, ptr(self.Q), ptr(self.P), ptr(self.qs), ptr(self.ps),
                         ptr(self.psi), sp, sb if sp else 0, self.stream.cuda_stream)

    def close(self):
        if self.ctx:
            swpic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_particles(self, state: Dict[str, np.ndarray]):
        swpic_init_particles(self.ctx, state["Q"], state["P"], state.get("qs"), state.get("ps"),
                             state["psi"])

    def init_lattice(self, run, spec, jitter_x=None, jitter_v=None):
        swpic_init_lattice(self.ctx, run, lattice_struct(spec), jitter_x, jitter_v)

    def state(self):
        """Host FP64 copies of the state (synchronises)."""
        swpic_synchronize(self.ctx)
        get = lambda t: None if t is None else t[: self.n].double().cpu().numpy()
        return {"Q": get(self.Q), "P": get(self.P), "qs": get(self.qs), "ps": get(self.ps),
                "psi": get(self.psi)}

    def step(self, n, diag_every=0):
        swpic_step(self.ctx, n, diag_every)

    def diagnostics(self, run=0):
        return swpic_diagnostics(self.ctx, run)

    def mesh(self, run=0):
        return swpic_get_mesh(self.ctx, run, self.runs[run][2])


# ---------------------------------------------------------------------------
# 2D2V (include/swpic2d.h): same-name wrappers
# ---------------------------------------------------------------------------
STATE2D = ("Qx", "Qy", "Px", "Py", "qx", "qy", "px", "py", "psi")


def _check2(st, ctx=None):
    _check(st, ctx, "swpic2d_last_error")


def swpic2d_create(cfg: swpic2d_config, n_particles: int):
    ctx = _CTX()
    _check2(load_library().swpic2d_create(C.byref(cfg), int(n_particles), C.byref(ctx)))
    return ctx


def swpic2d_destroy(ctx):
    load_library().swpic2d_destroy(ctx)


def swpic2d_last_error(ctx):
    return load_library().swpic2d_last_error(ctx).decode()


def swpic2d_bind_state(ctx, ptrs, stream):
    arr = (_P * 9)(*[None if p is None else int(p) for p in ptrs])
    _check2(load_library().swpic2d_bind_state(ctx, arr, stream), ctx)


def swpic2d_refresh(ctx):
    _check2(load_library().swpic2d_refresh(ctx), ctx)


def lattice2d_struct(spec) -> swpic2d_lattice:
    """swpic2d_lattice from a workloads.Lattice2DSpec."""
    return swpic2d_lattice(int(spec.nqx), int(spec.nqy), int(spec.nvx), int(spec.nvy), float(spec.vmin),
                           float(spec.vmax), float(spec.alpha), float(spec.kx), float(spec.ky), float(spec.vth),
                           int(spec.quad_order), int(bool(spec.decorate)))


def swpic2d_init_lattice(ctx, spec: swpic2d_lattice):
    _check2(load_library().swpic2d_init_lattice(ctx, C.byref(spec)), ctx)


def swpic2d_step(ctx, n_steps, diag_every=0):
    _check2(load_library().swpic2d_step(ctx, int(n_steps), int(diag_every)), ctx)


def swpic2d_diagnostics(ctx, max_records=100000):
    """(n, 9) array: t, mass, momentum_x, momentum_y, kinetic, field_energy,
    hamiltonian, e_amp, step."""
    buf = (swpic2d_diag * max_records)()
    n = C.c_int32(0)
    _check2(load_library().swpic2d_diagnostics(ctx, buf, int(max_records), C.byref(n)), ctx)
    out = np.zeros((n.value, 9))
    for k in range(n.value):
        d = buf[k]
        out[k] = [d.t, d.mass, d.momentum_x, d.momentum_y, d.kinetic, d.field_energy, d.hamiltonian,
                  d.e_amp, d.step]
    return out


def swpic2d_get_field(ctx, nx, ny):
    arrs = {k: np.zeros((ny, nx)) for k in ("b", "Phi", "gx", "gy")}
    _check2(load_library().swpic2d_get_field(ctx, *[_dptr(arrs[k]) for k in ("b", "Phi", "gx", "gy")]), ctx)
    return arrs


def swpic2d_synchronize(ctx):
    _check2(load_library().swpic2d_synchronize(ctx), ctx)


def swpic2d_step_host(ctx, in_ptrs, out_ptrs, n_steps, diag_every=0):
    """Host pointers: in_ptrs[9] (STATE2D order), out_ptrs[8] (None entries skipped)."""
    a = (_P * 9)(*[None if p is None else int(p) for p in in_ptrs])
    b = (_P * 8)(*[None if p is None else int(p) for p in out_ptrs])
    _check2(load_library().swpic2d_step_host(ctx, a, b, int(n_steps), int(diag_every)), ctx)


def swpic2d_save(ctx, path):
    _check2(load_library().swpic2d_save(ctx, path.encode()), ctx)


def swpic2d_load(ctx, path):
    _check2(load_library().swpic2d_load(ctx, path.encode()), ctx)


def swpic2d_set_timing(ctx, enable):
    _check2(load_library().swpic2d_set_timing(ctx, int(bool(enable))), ctx)


def swpic2d_pass_times(ctx, max_passes=100000):
    buf = (C.c_float * max_passes)()
    n = C.c_int32(0)
    _check2(load_library().swpic2d_pass_times(ctx, buf, int(max_passes), C.byref(n)), ctx)
    return np.array(buf[: n.value], dtype=np.float64)


def swpic2d_launch_count(ctx):
    n = C.c_int64(0)
    _check2(load_library().swpic2d_launch_count(ctx, C.byref(n)), ctx)
    return n.value


class Simulation2D:
    """Owns the nine particle tensors (torch, cuda) of one 2D2V run and a
    context bound to them."""

    def __init__(self, Lx, Ly, nx, ny, dt, n, precision=32, decorated=True, threads_per_block=0,
                 blocks_per_sm=0, diag_capacity=0, stream=None, device="cuda"):
        import torch
        self.torch = torch
        self.nx, self.ny, self.n = int(nx), int(ny), int(n)
        self.decorated = decorated
        self.dtype = torch.float64 if precision == 64 else torch.float32
        cfg = swpic2d_config(float(Lx), float(Ly), float(dt), int(nx), int(ny), int(precision),
                             int(bool(decorated)), int(threads_per_block), int(blocks_per_sm),
                             int(diag_capacity), 0)
        self.ctx = swpic2d_create(cfg, self.n)
        m = max(self.n, 1)
        self.t = {k: (torch.zeros(m, dtype=self.dtype, device=device)
                      if decorated or k not in ("qx", "qy", "px", "py") else None) for k in STATE2D}
        self.stream = stream if stream is not None else torch.cuda.Stream()
        swpic2d_bind_state(self.ctx, [None if v is None else v.data_ptr() for v in self.t.values()],
                           self.stream.cuda_stream)

    def close(self):
        if self.ctx:
            swpic2d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_particles(self, state):
        """Copy a host state (dict of FP64 arrays with the STATE2D keys) into the
        device tensors and take its field (swpic2d_refresh)."""
        torch = self.torch
        torch.cuda.synchronize()
        for k, v in self.t.items():
            if v is None:
                continue
            src = state.get(k)
            src = np.zeros(self.n) if src is None else np.asarray(src, dtype=np.float64)
            v[: self.n].copy_(torch.from_numpy(np.ascontiguousarray(src)).to(self.dtype))
        torch.cuda.synchronize()
        swpic2d_refresh(self.ctx)

    def init_lattice(self, spec):
        """Lattice state of a workloads.Lattice2DSpec, built on the device
        (swpic2d_init_lattice), and its field."""
        swpic2d_init_lattice(self.ctx, lattice2d_struct(spec))

    def state(self):
        swpic2d_synchronize(self.ctx)
        return {k: (None if v is None else v[: self.n].double().cpu().numpy()) for k, v in self.t.items()}

    def step(self, n, diag_every=0):
        swpic2d_step(self.ctx, n, diag_every)

    def diagnostics(self):
        return swpic2d_diagnostics(self.ctx)

    def field(self):
        return swpic2d_get_field(self.ctx, self.nx, self.ny)
