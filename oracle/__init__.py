"""FP64 CPU oracle for the decorated-particle (Scovel-Weinstein, k = 2) step.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA path: the arithmetic lives in ``swpic_oracle.c``
(plain loops, FP64), and this module only marshals numpy arrays into it.

Notation follows the paper: state (Q, P, q*, p*, psi*) of Sec. 3.2 / Sec. 5,
periodic P1 mesh of ``nx`` elements on [0, L).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_wrap.restype = C.c_double
        L.or_wrap.argtypes = [C.c_double, C.c_double]
        L.or_element.restype = C.c_int32
        L.or_element.argtypes = [C.c_double, C.c_double, C.c_int32]
        L.or_element_f32.restype = C.c_int32
        L.or_element_f32.argtypes = [C.c_double, C.c_double, C.c_int32]
        L.or_deposit.restype = None
        L.or_deposit.argtypes = [C.c_int64, _D, _D, _D, _I32, C.c_double, C.c_int32, _D]
        L.or_deposit_bruteforce.restype = None
        L.or_deposit_bruteforce.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_int32, _D]
        L.or_stiffness.restype = None
        L.or_stiffness.argtypes = [C.c_int32, C.c_double, _D]
        L.or_solve.restype = C.c_int
        L.or_solve.argtypes = [C.c_int32, C.c_double, _D, _D, _D]
        L.or_field_tables.restype = C.c_int
        L.or_field_tables.argtypes = [C.c_int32, C.c_double, _D, _D, C.c_int32, _D, _D]
        L.or_gather.restype = None
        L.or_gather.argtypes = [C.c_int64, _D, _I32, C.c_double, C.c_int32, _D, _D,
                                C.c_int32, _D, _D]
        L.or_kick_values.restype = None
        L.or_kick_values.argtypes = [C.c_int64, _D, _D, _D, _D, _D, C.c_double]
        L.or_drift.restype = None
        L.or_drift.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_double, C.c_double]
        L.or_diagnostics.restype = None
        L.or_diagnostics.argtypes = [C.c_int64, _D, _D, _D, C.c_int32, C.c_double, _D, _D]
        L.or_run.restype = C.c_int
        L.or_run.argtypes = [C.c_int64, _D, _D, _D, _D, _D, C.c_int32, C.c_double,
                             C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                             _D, _I32, _D, C.c_int32]
        L.or_field_of_state.restype = C.c_int
        L.or_field_of_state.argtypes = [C.c_int64, _D, _D, _D, C.c_int32, C.c_double,
                                        C.c_int32, C.c_int32, _D, _D, _D, _D, _D]
        L.or_gauss_legendre.restype = C.c_int
        L.or_gauss_legendre.argtypes = [C.c_int32, _D, _D]
        L.or_set_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or_init_lattice.restype = C.c_int
        L.or_kmeans_assign.argtypes = [C.c_int64, _D, _D, C.c_int32, _D, _D, C.c_double, _I32]
        L.or_kmeans_assign.restype = None
        L.or_kmeans_means.argtypes = [C.c_int64, _D, _D, _D, _I32, C.c_int32, C.c_double, _D, _D, _D, _D, _D]
        L.or_kmeans_means.restype = None
        L.or_kmeans.argtypes = [C.c_int64, _D, _D, _D, C.c_int32, C.c_double, C.c_int32, _D, _D, _I32]
        L.or_kmeans.restype = None
        L.or_lump.argtypes = [C.c_int64, _D, _D, _D, _I32, C.c_int32, C.c_double, _D, _D, _D, _D, _D, _D, _D]
        L.or_lump.restype = C.c_int64
        L.or_p2_field.argtypes = [C.c_int64, _D, _D, _D, _I32, C.c_double, C.c_int32, _D, _D, _D]
        L.or_p2_field.restype = C.c_int
        L.or_p2_gather.argtypes = [C.c_int64, _D, _I32, C.c_double, C.c_int32, _D, _D, _D, _D]
        L.or_p2_gather.restype = None
        L.or_p2_energy.argtypes = [C.c_int32, C.c_double, _D, _D, _D, _D]
        L.or_p2_energy.restype = None
        L.or_init_lattice.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, C.c_int32,
                                      _D, _D, _D, _D, _D, C.c_int32, C.c_int32, _D, _D,
                                      _D, _D, _D, _D, _D]
        # 2D2V (swpic2d_oracle.c)
        L.or2d_cell.restype = C.c_int32
        L.or2d_cell.argtypes = [C.c_double, C.c_double, C.c_int32]
        L.or2d_cell_f32.restype = C.c_int32
        L.or2d_cell_f32.argtypes = [C.c_double, C.c_double, C.c_int32]
        L.or2d_deposit.restype = None
        L.or2d_deposit.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _I32, _I32, C.c_double, C.c_double,
                                   C.c_int32, C.c_int32, _D]
        L.or2d_stiffness.restype = None
        L.or2d_stiffness.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, _D]
        L.or2d_solve.restype = C.c_int
        L.or2d_solve.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, _D, _D, _D]
        L.or2d_project.restype = None
        L.or2d_project.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, _D, _D, _D]
        L.or2d_gather.restype = None
        L.or2d_gather.argtypes = [C.c_int64, _D, _D, _I32, _I32, C.c_double, C.c_double, C.c_int32,
                                  C.c_int32, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.or2d_field_energy.restype = C.c_double
        L.or2d_field_energy.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, _D]
        L.or2d_init_lattice.restype = C.c_int
        L.or2d_init_lattice.argtypes = [C.c_int32] * 4 + [C.c_double] * 8 + [C.c_int32, C.c_int32] + [_D] * 9
        L.or2d_run.restype = C.c_int
        L.or2d_run.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _D, _D, _D, _D, C.c_int32, C.c_int32,
                               C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_int32,
                               _D, _I32, _D, C.c_int32]
        _lib = L
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _i(a):
    if a is None:
        return None
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_I32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


D2_LUMPED, D2_CONSISTENT, D2_NODAL, D2_P2 = 0, 1, 2, 3


def wrap(Q, L):
    """Periodic wrap into [0, L) (Sec. 2; reading A5 for the round-up case)."""
    f = lib().or_wrap
    return np.array([f(float(q), float(L)) for q in np.atleast_1d(Q)])


def element(Q, L, nx):
    """Element index floor(Q/h), decided in FP64."""
    f = lib().or_element
    return np.array([f(float(q), float(L), int(nx)) for q in np.atleast_1d(Q)], dtype=np.int32)


def element_f32(Q, L, nx):
    """Element index decided in FP32 from FP32 positions:
    floor(fl32(Q) * fl32(nx / L)), clamped to [0, nx-1].  Used where an FP32
    kernel takes the decision, so both sides decide in the same precision."""
    q = np.asarray(Q, dtype=np.float32)
    inv_h = np.float32(nx / L)
    k = np.floor(q * inv_h).astype(np.int64)
    return np.clip(k, 0, nx - 1).astype(np.int32)


def element_key(Q, L, nx, dtype):
    """Element index decided in the given precision from values of that
    precision: floor(Q * dtype(nx / L)), clamped to [0, nx-1].  Where a kernel
    takes this integer decision in FP32 or FP64, the oracle takes it the same
    way, so keys can be compared bit for bit."""
    q = np.asarray(Q).astype(dtype)
    inv_h = dtype(np.float64(nx) / np.float64(L))
    k = np.floor(q * inv_h)
    k = np.where(np.isfinite(k), k, 0).astype(np.int64)
    return np.clip(k, 0, nx - 1).astype(np.int32)


def deposit(Q, p_star, psi_star, L, nx, elem=None):
    """b_j = sum_a psi*_a phi_j(Q_a) - p*_a phi_j'(Q_a)  (Eq. rhs-assembly)."""
    Q = _f64(Q); ps = _f64(p_star); psi = _f64(psi_star)
    e = None if elem is None else np.ascontiguousarray(elem, dtype=np.int32)
    b = np.zeros(nx)
    lib().or_deposit(len(Q), _d(Q), _d(ps), _d(psi), _i(e), float(L), int(nx), _d(b))
    return b


def deposit_bruteforce(Q, p_star, psi_star, L, nx):
    """Same assembly by evaluating every hat at every particle; tiny inputs."""
    Q = _f64(Q); ps = _f64(p_star); psi = _f64(psi_star)
    b = np.zeros(nx)
    lib().or_deposit_bruteforce(len(Q), _d(Q), _d(ps), _d(psi), float(L), int(nx), _d(b))
    return b


def stiffness(nx, L):
    A = np.zeros((nx, nx))
    lib().or_stiffness(int(nx), float(L), _d(A))
    return A


def solve(b, L):
    """Galerkin Poisson solve (Eq. lin-sys) with the zero-mean gauge.
    Returns (Phi, lambda); lambda = mean(b) is the removed background."""
    b = _f64(b)
    nx = len(b)
    Phi = np.zeros(nx)
    lam = C.c_double(0.0)
    rc = lib().or_solve(int(nx), float(L), _d(b), _d(Phi), C.byref(lam))
    if rc != 0:
        raise RuntimeError("oracle solve failed")
    return Phi, lam.value


def field_tables(Phi, L, d2_mode=D2_LUMPED, btilde=None):
    """(dphi per element, d2 per element (modes 0/1) or per node (mode 2))."""
    Phi = _f64(Phi)
    nx = len(Phi)
    dphi = np.zeros(nx); d2 = np.zeros(nx)
    rc = lib().or_field_tables(int(nx), float(L), _d(Phi), _d(_f64(btilde)), int(d2_mode),
                               _d(dphi), _d(d2))
    if rc != 0:
        raise RuntimeError("oracle field_tables failed")
    return dphi, d2


def gather(Q, L, dphi, d2, d2_mode=D2_LUMPED, elem=None):
    Q = _f64(Q); dphi = _f64(dphi); d2 = _f64(d2)
    e = None if elem is None else np.ascontiguousarray(elem, dtype=np.int32)
    n = len(Q)
    dV = np.zeros(n); d2V = np.zeros(n)
    lib().or_gather(n, _d(Q), _i(e), float(L), len(dphi), _d(dphi), _d(d2), int(d2_mode),
                    _d(dV), _d(d2V))
    return dV, d2V


def kick_values(p_star, P, q_star, dV, d2V, c):
    """In place: P -= c dV; q* += c p* d2V."""
    lib().or_kick_values(len(P), _d(p_star), _d(P), _d(q_star), _d(_f64(dV)), _d(_f64(d2V)),
                         float(c))


def drift(Q, P, q_star, p_star, L, c):
    """In place: Q = wrap(Q + c P); p* -= c q*."""
    lib().or_drift(len(Q), _d(Q), _d(P), _d(q_star), _d(p_star), float(L), float(c))


def diagnostics(P, q_star, psi_star, Phi, L):
    """{mass, momentum, kinetic, field, H, E_amp} (Eqs. Hh, Eamp)."""
    P = _f64(P); qs = _f64(q_star); psi = _f64(psi_star); Phi = _f64(Phi)
    out = np.zeros(6)
    lib().or_diagnostics(len(P), _d(P), _d(qs), _d(psi), len(Phi), float(L), _d(Phi), _d(out))
    return dict(zip(["mass", "momentum", "kinetic", "field", "H", "E_amp"], out))


DIAG_KEYS = ["t", "mass", "momentum", "kinetic", "field", "H", "E_amp"]


def field_of_state(Q, p_star, psi_star, L, nx, d2_mode=D2_LUMPED, decorated=True):
    """Deposit -> solve -> tables for one state.  Returns a dict of FP64 arrays."""
    Q = _f64(Q); psi = _f64(psi_star)
    ps = _f64(p_star) if p_star is not None else np.zeros_like(Q)
    out = {k: np.zeros(nx) for k in ("b", "btilde", "Phi", "dphi", "d2")}
    rc = lib().or_field_of_state(len(Q), _d(Q), _d(ps), _d(psi), int(nx), float(L),
                                 int(d2_mode), int(bool(decorated)),
                                 *[_d(out[k]) for k in ("b", "btilde", "Phi", "dphi", "d2")])
    if rc != 0:
        raise RuntimeError("oracle field_of_state failed")
    return out


def set_threads(n):
    """Host threads of or_run's particle loops (1 = the serial loops every
    test uses; more splits the particles into blocks whose deposit and
    diagnostic partials are added in block order).  Returns the count in
    effect (1 when the oracle was built without OpenMP)."""
    return int(lib().or_set_threads(int(n)))


def run(state, nx, L, dt, n_steps, diag_every=1, d2_mode=D2_LUMPED, decorated=True,
        store_f32=False):
    """KDK leapfrog run (Sec. 5).  ``state`` is a dict with Q, P, qs, ps, psi
    (FP64 copies are made; the returned dict holds the final state, the
    diagnostics history as an (n, 7) array and the final Phi).  store_f32:
    keep the state in FP32 storage (values rounded to FP32 after every update,
    element decisions in FP32), arithmetic in FP64."""
    Q = np.array(state["Q"], dtype=np.float64)
    P = np.array(state["P"], dtype=np.float64)
    psi = np.array(state["psi"], dtype=np.float64)
    n = len(Q)
    qs = np.array(state["qs"], dtype=np.float64) if state.get("qs") is not None else np.zeros(n)
    ps = np.array(state["ps"], dtype=np.float64) if state.get("ps") is not None else np.zeros(n)
    n_rec = (n_steps // diag_every + 1) if diag_every > 0 else 0
    diag = np.zeros((max(n_rec, 1), 7))
    nd = C.c_int32(0)
    Phi = np.zeros(nx)
    rc = lib().or_run(n, _d(Q), _d(P), _d(qs), _d(ps), _d(psi), int(nx), float(L), float(dt),
                      int(d2_mode), int(bool(decorated)), int(n_steps), int(diag_every),
                      _d(diag), C.byref(nd), _d(Phi), int(bool(store_f32)))
    if rc != 0:
        raise RuntimeError("oracle run failed")
    return {"Q": Q, "P": P, "qs": qs, "ps": ps, "psi": psi,
            "diag": diag[: nd.value], "Phi": Phi}


def gauss_legendre(n):
    x = np.zeros(n); w = np.zeros(n)
    if lib().or_gauss_legendre(int(n), _d(x), _d(w)) != 0:
        raise ValueError(n)
    return x, w


def init_lattice(spec, jitter_x=None, jitter_v=None):
    """Decorated lattice particles (reading A6 of Sec. 4.2 / Alg. 1 with the
    lattice cell as the cluster).  ``spec`` is a workloads.LatticeSpec."""
    nq, nv = spec.nq, spec.nv
    n = nq * nv
    out = {k: np.zeros(n) for k in ("Q", "P", "qs", "ps", "psi")}
    t = spec.terms
    m = len(t)
    amp = np.array([x[0] for x in t] + [0.0] * (4 - m))
    c0 = np.array([x[1] for x in t] + [0.0] * (4 - m))
    c2 = np.array([x[2] for x in t] + [0.0] * (4 - m))
    beta = np.array([x[3] for x in t] + [0.0] * (4 - m))
    u = np.array([x[4] for x in t] + [0.0] * (4 - m))
    rc = lib().or_init_lattice(int(nq), int(nv), float(spec.L), float(spec.vmin),
                               float(spec.vmax), float(spec.alpha), float(spec.kx), int(m),
                               _d(amp), _d(c0), _d(c2), _d(beta), _d(u),
                               int(spec.quad_order), int(bool(spec.decorate)),
                               _d(_f64(jitter_x)), _d(_f64(jitter_v)),
                               *[_d(out[k]) for k in ("Q", "P", "qs", "ps", "psi")])
    if rc != 0:
        raise RuntimeError("oracle init_lattice failed")
    return out


def stable_sort_order(keys):
    """Stable ordering by integer key: the permutation that sorts by
    (key, original index).  Definition of a stable counting sort."""
    keys = np.asarray(keys)
    return np.lexsort((np.arange(len(keys)), keys))


# --- decorated-particle initialization from marker particles (Alg. lumping_procedure) ---
def kmeans_assign(Qm, Pm, cq, cp, L):
    """Nearest center of every marker (FP32 decision, ties to the smaller index)."""
    Qm, Pm, cq, cp = _f64(Qm), _f64(Pm), _f64(cq), _f64(cp)
    out = np.zeros(len(Qm), dtype=np.int32)
    lib().or_kmeans_assign(len(Qm), _d(Qm), _d(Pm), len(cq), _d(cq), _d(cp), L, _i(out))
    return out


def kmeans_means(Qm, Pm, wm, assign, cq, cp, L):
    """psi-weighted member means about the centers; (mq, mp, w_sum)."""
    Qm, Pm, wm, cq, cp = _f64(Qm), _f64(Pm), _f64(wm), _f64(cq), _f64(cp)
    assign = np.ascontiguousarray(assign, dtype=np.int32)
    K = len(cq)
    mq, mp, ws = np.zeros(K), np.zeros(K), np.zeros(K)
    lib().or_kmeans_means(len(Qm), _d(Qm), _d(Pm), _d(wm), _i(assign), K, L, _d(cq), _d(cp),
                          _d(mq), _d(mp), _d(ws))
    return mq, mp, ws


def kmeans(Qm, Pm, wm, cq0, cp0, L, n_iter):
    """n_iter Lloyd iterations from (cq0, cp0); returns (cq, cp, assign)."""
    Qm, Pm, wm = _f64(Qm), _f64(Pm), _f64(wm)
    cq, cp = np.array(cq0, dtype=np.float64), np.array(cp0, dtype=np.float64)
    assign = np.zeros(len(Qm), dtype=np.int32)
    lib().or_kmeans(len(Qm), _d(Qm), _d(Pm), _d(wm), len(cq), L, int(n_iter), _d(cq), _d(cp), _i(assign))
    return cq, cp, assign


def lump(Qm, Pm, wm, assign, cq, cp, L):
    """Alg. lumping_procedure: decorated particles of the non-empty clusters."""
    Qm, Pm, wm, cq, cp = _f64(Qm), _f64(Pm), _f64(wm), _f64(cq), _f64(cp)
    assign = np.ascontiguousarray(assign, dtype=np.int32)
    K = len(cq)
    out = [np.zeros(K) for _ in range(5)]
    n = lib().or_lump(len(Qm), _d(Qm), _d(Pm), _d(wm), _i(assign), K, L, _d(cq), _d(cp),
                      *[_d(a) for a in out])
    Q, P, qs, ps, psi = [a[:n].copy() for a in out]
    return {"Q": Q, "P": P, "qs": qs, "ps": ps, "psi": psi}


# --- P2 (quadratic Lagrange) elements ---
def p2_field(Q, p_star, psi_star, L, nx, elem=None):
    """P2 Galerkin field: (Phi2 [2 nx], a [nx], beta [nx]) with
    phi_h'(xi) = a + beta (1 - 2 xi) and phi_h'' = -2 beta / h on each element."""
    Q, ps, psi = _f64(Q), _f64(p_star), _f64(psi_star)
    e = None if elem is None else np.ascontiguousarray(elem, dtype=np.int32)
    Phi2, a, beta = np.zeros(2 * nx), np.zeros(nx), np.zeros(nx)
    rc = lib().or_p2_field(len(Q), _d(Q), _d(ps), _d(psi), _i(e), L, nx, _d(Phi2), _d(a), _d(beta))
    if rc != 0:
        raise RuntimeError("P2 solve failed")
    return Phi2, a, beta


def p2_gather(Q, a, beta, L, nx):
    Q = _f64(Q)
    dV, d2V = np.zeros(len(Q)), np.zeros(len(Q))
    lib().or_p2_gather(len(Q), _d(Q), None, L, nx, _d(_f64(a)), _d(_f64(beta)), _d(dV), _d(d2V))
    return dV, d2V


def p2_energy(a, beta, L):
    W, E = C.c_double(), C.c_double()
    lib().or_p2_energy(len(a), L, _d(_f64(a)), _d(_f64(beta)), C.byref(W), C.byref(E))
    return W.value, E.value


# ---------------------------------------------------------------------------
# 2D2V: periodic bilinear (Q1) mesh of nx x ny cells on [0, Lx) x [0, Ly);
# mesh arrays are (ny, nx), node (i, j) at (i hx, j hy).
# ---------------------------------------------------------------------------
STATE2D = ("Qx", "Qy", "Px", "Py", "qx", "qy", "px", "py", "psi")


def cell2d(Q, L, n, f32=False):
    """Cell index along one axis: floor(Q / h) clamped to [0, n-1], decided in
    FP64, or with f32 as or2d_cell_f32 does, floor(fl32(fl32(Q) fl32(n/L)))
    (elementwise numpy arithmetic; the C routines take the same decisions)."""
    Q = np.atleast_1d(np.asarray(Q, dtype=np.float64))
    if f32:
        k = np.floor(Q.astype(np.float32) * np.float32(n / L)).astype(np.float64)
    else:
        k = np.floor(Q / (L / n))
    k = np.where(np.isfinite(k), k, 0.0)
    return np.clip(k, 0, n - 1).astype(np.int32)


def deposit2d(Qx, Qy, psx, psy, psi, Lx, Ly, nx, ny, cx=None, cy=None):
    """b_j = sum_a psi*_a N_j(Q_a) - p*_a . grad N_j(Q_a)  (Eq. swpic_poisson, S_h = delta)."""
    Qx, Qy, psi = _f64(Qx), _f64(Qy), _f64(psi)
    psx, psy = _f64(psx), _f64(psy)
    cx = None if cx is None else np.ascontiguousarray(cx, dtype=np.int32)
    cy = None if cy is None else np.ascontiguousarray(cy, dtype=np.int32)
    b = np.zeros((ny, nx))
    lib().or2d_deposit(len(Qx), _d(Qx), _d(Qy), _d(psx), _d(psy), _d(psi), _i(cx), _i(cy),
                       float(Lx), float(Ly), int(nx), int(ny), _d(b))
    return b


def stiffness2d(nx, ny, Lx, Ly):
    K = np.zeros((nx * ny, nx * ny))
    lib().or2d_stiffness(int(nx), int(ny), float(Lx), float(Ly), _d(K))
    return K


def solve2d(b, Lx, Ly):
    """Zero-mean Q1 Galerkin solve of K Phi + lambda m = b; returns (Phi, lambda)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    ny, nx = b.shape
    Phi = np.zeros_like(b)
    lam = C.c_double(0.0)
    if lib().or2d_solve(int(nx), int(ny), float(Lx), float(Ly), _d(b), _d(Phi), C.byref(lam)) != 0:
        raise RuntimeError("singular 2D system")
    return Phi, lam.value


def project2d(Phi, Lx, Ly):
    """Lumped-mass projection g of grad phi_h onto Q1 (each component)."""
    Phi = np.ascontiguousarray(Phi, dtype=np.float64)
    ny, nx = Phi.shape
    gx, gy = np.zeros_like(Phi), np.zeros_like(Phi)
    lib().or2d_project(int(nx), int(ny), float(Lx), float(Ly), _d(Phi), _d(gx), _d(gy))
    return gx, gy


def gather2d(Qx, Qy, Phi, gx, gy, Lx, Ly, cx=None, cy=None):
    """grad phi_h and H_ik = d_k g_i at the particles: dict Ex, Ey, Hxx, Hxy, Hyx, Hyy."""
    Qx, Qy = _f64(Qx), _f64(Qy)
    Phi, gx, gy = (np.ascontiguousarray(a, dtype=np.float64) for a in (Phi, gx, gy))
    ny, nx = Phi.shape
    n = len(Qx)
    out = {k: np.zeros(n) for k in ("Ex", "Ey", "Hxx", "Hxy", "Hyx", "Hyy")}
    cx = None if cx is None else np.ascontiguousarray(cx, dtype=np.int32)
    cy = None if cy is None else np.ascontiguousarray(cy, dtype=np.int32)
    lib().or2d_gather(n, _d(Qx), _d(Qy), _i(cx), _i(cy), float(Lx), float(Ly), int(nx), int(ny),
                      _d(Phi), _d(gx), _d(gy), *[_d(out[k]) for k in ("Ex", "Ey", "Hxx", "Hxy", "Hyx", "Hyy")])
    return out


def field_energy2d(Phi, Lx, Ly):
    Phi = np.ascontiguousarray(Phi, dtype=np.float64)
    ny, nx = Phi.shape
    return lib().or2d_field_energy(int(nx), int(ny), float(Lx), float(Ly), _d(Phi))


def run2d(state, nx, ny, Lx, Ly, dt, n_steps, diag_every=1, decorated=True, store_f32=False):
    """KDK run of the 2D2V model.  ``state``: dict with the keys of STATE2D
    (qx, qy, px, py may be None).  Returns the final state, the diagnostics
    history as (n, 8) [t, mass, mom_x, mom_y, kinetic, W, H, E_amp] and Phi."""
    st = {k: (np.zeros(len(state["Qx"])) if state.get(k) is None else np.array(state[k], dtype=np.float64))
          for k in STATE2D}
    n = len(st["Qx"])
    n_rec = (n_steps // diag_every + 1) if diag_every > 0 else 0
    diag = np.zeros((max(n_rec, 1), 8))
    nd = C.c_int32(0)
    Phi = np.zeros((ny, nx))
    rc = lib().or2d_run(n, *[_d(st[k]) for k in STATE2D], int(nx), int(ny), float(Lx), float(Ly),
                        float(dt), int(bool(decorated)), int(n_steps), int(diag_every), _d(diag),
                        C.byref(nd), _d(Phi), int(bool(store_f32)))
    if rc != 0:
        raise RuntimeError("2D oracle run failed")
    st["diag"] = diag[: nd.value]
    st["Phi"] = Phi
    return st


def init_lattice2d(spec):
    """2D2V lattice state of a workloads.Lattice2DSpec (cluster reading of
    Sec. 4.2 in 2D2V; see or2d_init_lattice)."""
    n = spec.n
    st = {k: np.zeros(n) for k in STATE2D}
    rc = lib().or2d_init_lattice(int(spec.nqx), int(spec.nqy), int(spec.nvx), int(spec.nvy), float(spec.Lx),
                                 float(spec.Ly), float(spec.vmin), float(spec.vmax), float(spec.alpha),
                                 float(spec.kx), float(spec.ky), float(spec.vth), int(spec.quad_order),
                                 int(bool(spec.decorate)), *[_d(st[k]) for k in STATE2D])
    if rc != 0:
        raise ValueError("bad 2D lattice")
    return st
