"""Seeded synthetic workloads for the decorated-particle step.

This module holds no arithmetic of the method: it describes the five 1D1V
periodic problems (domain, velocity range, initial distribution f0, lattice
size, mesh, time step), generates seeded jitter and seeded random particle
states with the shapes and magnitudes of those problems, and nothing else.
It is the only code shared by the CUDA path's tests/benchmark and the oracle.

Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), used as a
counter-based generator: draw i of stream s under seed k is the SplitMix64
output mix(k ^ (s * 0xD1B54A32D192ED03) + (i + 1) * 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n consecutive 64-bit outputs (counter start .. start+n-1) of stream ``stream``."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream) * _STREAM)
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = base + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, stream, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# Problem descriptions
# ---------------------------------------------------------------------------
SQRT2PI = math.sqrt(2.0 * math.pi)


@dataclass(frozen=True)
class LatticeSpec:
    """Phase-space lattice of nq x nv decorated particles on [0, L) x [vmin, vmax).

    f0(x, v) = (1 + alpha cos(kx x)) * sum_m amp_m (c0_m + c2_m v^2) exp(-beta_m (v - u_m)^2)
    ``terms`` = ((amp, c0, c2, beta, u), ...), at most 4.
    Jitter is uniform in [-jitter, jitter) lattice cells on both axes (seeded).
    """
    nq: int
    nv: int
    L: float
    vmin: float
    vmax: float
    alpha: float
    kx: float
    terms: Tuple[Tuple[float, float, float, float, float], ...]
    jitter: float = 0.0
    seed: int = 0
    quad_order: int = 4
    decorate: bool = True

    @property
    def n(self) -> int:
        return self.nq * self.nv


@dataclass(frozen=True)
class RunSpec:
    name: str
    lattice: LatticeSpec
    nx: int
    dt: float
    steps: int
    precision: int = 32           # particle-state precision: 32 or 64
    decorated: bool = True


MAXWELL = ((1.0 / SQRT2PI, 1.0, 0.0, 0.5, 0.0),)


def landau_linear(jitter: float = 0.0) -> RunSpec:
    """Linear Landau damping: x in [0, 4pi), v in [-6, 6], alpha 0.01, k 0.5,
    64 x 64 lattice, nx 64, dt 0.1, 500 steps, FP64; seed 0 for +-1e-3 cell jitter."""
    lat = LatticeSpec(64, 64, 4 * math.pi, -6.0, 6.0, 0.01, 0.5, MAXWELL, jitter=jitter, seed=0)
    return RunSpec("landau_linear_64x64", lat, 64, 0.1, 500, precision=64)


def two_stream(precision: int = 32) -> RunSpec:
    """Two-stream instability: f0 = (1 + 0.05 cos 0.5x) v^2 exp(-v^2/2)/sqrt(2pi),
    x in [0, 4pi), v in [-8, 8], 256 x 256 lattice, nx 128, dt 0.05, 1000 steps."""
    terms = ((1.0 / SQRT2PI, 0.0, 1.0, 0.5, 0.0),)
    lat = LatticeSpec(256, 256, 4 * math.pi, -8.0, 8.0, 0.05, 0.5, terms)
    return RunSpec("two_stream_256x256", lat, 128, 0.05, 1000, precision=precision)


def landau_strong(precision: int = 32, scale: int = 1, decorated: bool = True) -> RunSpec:
    """Strong Landau damping: alpha 0.5, k 0.5, x in [0, 4pi), v in [-6, 6],
    2048 x 2048 lattice (scale 4 gives the 8192 x 8192 point-particle case),
    +-0.25 cell jitter seed 0, nx 512, dt 0.05, 1000 steps."""
    side = 2048 * scale
    lat = LatticeSpec(side, side, 4 * math.pi, -6.0, 6.0, 0.5, 0.5, MAXWELL, jitter=0.25,
                      seed=0, decorate=decorated)
    name = "landau_strong_%dx%d%s" % (side, side, "" if decorated else "_pic")
    return RunSpec(name, lat, 512, 0.05, 1000, precision=precision, decorated=decorated)


def bump_on_tail(precision: int = 32, side: int = 4096) -> RunSpec:
    """Bump-on-tail at bandwidth-roofline scale: f0 = (1 + 0.04 cos 0.3x)
    [0.9 exp(-v^2/2) + 0.2 exp(-4 (v - 4.5)^2)]/sqrt(2pi), x in [0, 20pi/3),
    v in [-8, 10], 4096 x 4096 lattice, nx 1024, dt 0.05, 2000 steps."""
    terms = ((0.9 / SQRT2PI, 1.0, 0.0, 0.5, 0.0), (0.2 / SQRT2PI, 1.0, 0.0, 4.0, 4.5))
    lat = LatticeSpec(side, side, 20 * math.pi / 3, -8.0, 10.0, 0.04, 0.3, terms)
    return RunSpec("bump_on_tail_%dx%d" % (side, side), lat, 1024, 0.05, 2000,
                   precision=precision)


ENSEMBLE_JSON = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                             "landau_ensemble_256.json")


def make_ensemble_table(n_runs: int = 256, seed: int = 1) -> List[dict]:
    """Draw the ensemble of independent Landau runs from one SplitMix64 stream:
    per run k ~ U[0.3, 0.6], alpha ~ logU[0.01, 0.5], lattice side ~ U{64, 128,
    256, 512}, nx = side / 2, L = 2 pi / k, v in [-6, 6], dt 0.1, 800 steps."""
    u = uniform01(seed, 0, 3 * n_runs).reshape(n_runs, 3)
    sides = (64, 128, 256, 512)
    rows = []
    for r in range(n_runs):
        k = 0.3 + 0.3 * u[r, 0]
        alpha = math.exp(math.log(0.01) + (math.log(0.5) - math.log(0.01)) * u[r, 1])
        side = sides[min(int(u[r, 2] * 4), 3)]
        rows.append({"run": r, "k": k, "alpha": alpha, "side": side, "nx": side // 2,
                     "L": 2 * math.pi / k, "vmin": -6.0, "vmax": 6.0, "dt": 0.1,
                     "steps": 800})
    return rows


def ensemble_table() -> List[dict]:
    """The committed 256-run table (written by ``python -m workloads``)."""
    with open(ENSEMBLE_JSON) as f:
        return json.load(f)["runs"]


def ensemble(n_runs: Optional[int] = None, precision: int = 32) -> List[RunSpec]:
    rows = ensemble_table()
    if n_runs is not None:
        rows = rows[:n_runs]
    out = []
    for row in rows:
        lat = LatticeSpec(row["side"], row["side"], row["L"], row["vmin"], row["vmax"],
                          row["alpha"], row["k"], MAXWELL)
        out.append(RunSpec("landau_ensemble_run%03d" % row["run"], lat, row["nx"], row["dt"],
                           row["steps"], precision=precision))
    return out


# ---------------------------------------------------------------------------
# Seeded inputs
# ---------------------------------------------------------------------------
def jitter(spec: LatticeSpec) -> Tuple[Optional[np.ndarray], Optional[np.ndarray]]:
    """Per-particle jitter in lattice cells on x (stream 1) and v (stream 2),
    uniform in [-spec.jitter, spec.jitter); (None, None) when jitter is 0."""
    if spec.jitter == 0.0:
        return None, None
    n = spec.n
    jx = spec.jitter * (2.0 * uniform01(spec.seed, 1, n) - 1.0)
    jv = spec.jitter * (2.0 * uniform01(spec.seed, 2, n) - 1.0)
    return jx, jv


def random_state(n: int, L: float, seed: int = 0, vth: float = 1.0, decorated: bool = True,
                 dipole_scale: float = 0.25, nx: int = 64) -> dict:
    """A seeded random particle state with the magnitudes of the lattice
    problems: Q ~ U[0, L), P ~ vth * (sum of 3 uniforms - 1.5) * 2,
    psi* > 0 of order L/n, and decorations |p*| ~ dipole_scale * psi* * h,
    |q*| ~ dipole_scale * psi* * vth * 0.1 with random signs.  FP64 arrays."""
    u = uniform01(seed, 10, 7 * n).reshape(7, n) if n > 0 else np.zeros((7, 0))
    Q = L * u[0]
    P = vth * 2.0 * (u[1] + u[2] + u[3] - 1.5)
    psi = (L / max(n, 1)) * (0.5 + u[4])
    h = L / nx
    if decorated:
        ps = dipole_scale * psi * h * (2.0 * u[5] - 1.0)
        qs = dipole_scale * psi * vth * 0.1 * (2.0 * u[6] - 1.0)
    else:
        ps = np.zeros(n)
        qs = np.zeros(n)
    return {"Q": Q, "P": P, "qs": qs, "ps": ps, "psi": psi}


def random_state_2d(n: int, Lx: float, Ly: float, seed: int = 0, vth: float = 1.0,
                    decorated: bool = True, dipole_scale: float = 0.25, nx: int = 16, ny: int = 16,
                    alpha: float = 0.0) -> dict:
    """A seeded random 2D2V state (keys Qx, Qy, Px, Py, qx, qy, px, py, psi):
    Q ~ U([0, Lx) x [0, Ly)), each P component ~ vth * (sum of 3 uniforms -
    1.5) * 2, psi* = (Lx Ly / n)(0.5 + U) (1 + alpha cos(2 pi x/Lx) cos(2 pi y/Ly)),
    p*_x ~ dipole_scale psi* hx U(-1, 1) (and y with hy), q* ~ dipole_scale
    psi* vth 0.1 U(-1, 1).  FP64 arrays."""
    u = uniform01(seed, 30, 13 * n).reshape(13, n) if n > 0 else np.zeros((13, 0))
    Qx, Qy = Lx * u[0], Ly * u[1]
    Px = vth * 2.0 * (u[2] + u[3] + u[4] - 1.5)
    Py = vth * 2.0 * (u[5] + u[6] + u[7] - 1.5)
    psi = (Lx * Ly / max(n, 1)) * (0.5 + u[8]) * (1.0 + alpha * np.cos(2 * np.pi * Qx / Lx) *
                                                   np.cos(2 * np.pi * Qy / Ly))
    z = np.zeros(n)
    if decorated:
        px = dipole_scale * psi * (Lx / nx) * (2.0 * u[9] - 1.0)
        py = dipole_scale * psi * (Ly / ny) * (2.0 * u[10] - 1.0)
        qx = dipole_scale * psi * vth * 0.1 * (2.0 * u[11] - 1.0)
        qy = dipole_scale * psi * vth * 0.1 * (2.0 * u[12] - 1.0)
    else:
        px = py = qx = qy = z
    return {"Qx": Qx, "Qy": Qy, "Px": Px, "Py": Py, "qx": qx, "qy": qy, "px": px, "py": py, "psi": psi}


@dataclass(frozen=True)
class Lattice2DSpec:
    """A 4D phase-space lattice for 2D2V runs: nqx x nqy positions times
    nvx x nvy velocities on [0, Lx) x [0, Ly) x [vmin, vmax]^2, of
    f0 = (1 + alpha cos(kx x + ky y)) exp(-|v|^2 / (2 vth^2)) / (2 pi vth^2)."""
    nqx: int
    nqy: int
    nvx: int
    nvy: int
    Lx: float
    Ly: float
    vmin: float = -6.0
    vmax: float = 6.0
    alpha: float = 0.05
    kx: float = 0.5
    ky: float = 0.5
    vth: float = 1.0
    quad_order: int = 2
    decorate: bool = True

    @property
    def n(self) -> int:
        return self.nqx * self.nqy * self.nvx * self.nvy


def landau_2d(side: int = 64, quad_order: int = 2) -> Lattice2DSpec:
    """Oblique 2D Landau damping: k = (1/2, 1/2) on [0, 4 pi)^2, alpha 0.05,
    side^4 decorated particles (64^4 = 16,777,216)."""
    L = 4 * np.pi
    return Lattice2DSpec(side, side, side, side, L, L, -6.0, 6.0, 0.05, 2 * np.pi / L, 2 * np.pi / L, 1.0,
                         quad_order, True)


def two_stream_markers(M: int, seed: int = 0, alpha: float = 0.01, L: float = 2 * np.pi,
                       v0: float = 1.0, vth: float = 0.3) -> dict:
    """A seeded random sample of M marker particles of the two-stream f0 of the
    paper's initialization experiments: f0 ~ (1 + alpha cos(2 pi x / L)) x
    (N(+v0, vth^2) + N(-v0, vth^2)) / 2 on [0, L).  x by rejection from
    uniform proposals, v by Box-Muller; weights L / M.  FP64 arrays
    (Q, P, psi)."""
    n_prop = 2 * M + 64
    u = uniform01(seed, 20, 5 * n_prop).reshape(5, n_prop)
    xs = L * u[0]
    keep = u[1] * (1.0 + abs(alpha)) <= 1.0 + alpha * np.cos(2 * np.pi * xs / L)
    x = xs[keep][:M]
    if len(x) < M:                                        # practically never: top up without rejection
        x = np.concatenate([x, xs[~keep][:M - len(x)]])
    r = np.sqrt(-2.0 * np.log(np.maximum(u[2][:M], 1e-300)))
    g = r * np.cos(2 * np.pi * u[3][:M])
    sign = np.where(u[4][:M] < 0.5, -1.0, 1.0)
    return {"Q": x, "P": sign * v0 + vth * g, "psi": np.full(M, L / M)}


def lattice_points(spec: LatticeSpec) -> Tuple[np.ndarray, np.ndarray]:
    """Cell centres (x_i, v_j) flattened x-major (index i * nv + j)."""
    dx = spec.L / spec.nq
    dv = (spec.vmax - spec.vmin) / spec.nv
    x = (np.arange(spec.nq) + 0.5) * dx
    v = spec.vmin + (np.arange(spec.nv) + 0.5) * dv
    return np.repeat(x, spec.nv), np.tile(v, spec.nq)


def write_ensemble_json(path: str = ENSEMBLE_JSON) -> None:
    rows = make_ensemble_table()
    with open(path, "w") as f:
        json.dump({"generator": "workloads.make_ensemble_table(n_runs=256, seed=1)",
                   "runs": rows}, f, indent=1)
        f.write("\n")
