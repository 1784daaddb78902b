"""Parity at the benchmark configurations' full sizes, in the launch
configuration the benchmark uses (defaults: 256 threads x 4 CTAs per SM).

Each side initialises from the same lattice description (the device with
its own kernel, the oracle with its own code), takes one step, and the
mesh charge and sampled particles are compared.  The FP32 comparisons use
the oracle's FP32-storage mode (element decisions from FP32-stored
positions, FP64 arithmetic); the bump-on-tail step is also compared with the
plain FP64 oracle.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import cast_state, need_gpu, periodic_diff, rel_max

pytestmark = pytest.mark.gpu

SAMPLE = 4096


def _sim(runs, precision, **kw):
    from paper_2605_21794_gb300 import swpic
    return swpic.Simulation(runs, precision=precision, **kw)


def _sampled(state, idx):
    return {k: (None if v is None else v[idx]) for k, v in state.items()}


def _check_sample(got, ref, idx, L, tol):
    assert np.abs(periodic_diff(got["Q"][idx], ref["Q"][idx], L)).max() <= tol * L
    for k in ("P", "qs", "ps"):
        if ref.get(k) is None or got.get(k) is None:
            continue
        assert rel_max(got[k][idx], ref[k][idx]) <= tol * 4, k


def test_bump_on_tail_full_size_one_fp32_step():
    """16,777,216 decorated particles, nx 1024, dt 0.05 (the benchmark workload)."""
    need_gpu()
    spec = W.bump_on_tail()
    lat = spec.lattice
    sim = _sim([(lat.L, spec.dt, spec.nx, lat.n)], 32)
    try:
        sim.init_lattice(0, lat)
        init = sim.state()
        sim.step(1)
        got = sim.state()
        m = sim.mesh(0)
    finally:
        sim.close()
    st = cast_state(O.init_lattice(lat), 32)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(lat.n, SAMPLE, replace=False))
    for k in ("Q", "P", "psi", "qs", "ps"):
        assert rel_max(init[k][idx], st[k][idx]) <= 1e-6, k
    ref = O.run(st, spec.nx, lat.L, spec.dt, 1, diag_every=0, store_f32=True)
    b = O.deposit(ref["Q"], ref["ps"], ref["psi"], lat.L, spec.nx,
                  elem=O.element_key(ref["Q"], lat.L, spec.nx, np.float32))
    assert rel_max(m["b"], b) <= 1e-5
    _check_sample(got, ref, idx, lat.L, 1e-6)
    # the same step against the plain FP64 oracle (FP64 state and element
    # decisions from the same initial values): mesh charge within 1e-5
    ref64 = O.run(st, spec.nx, lat.L, spec.dt, 1, diag_every=0)
    f64 = O.field_of_state(ref64["Q"], ref64["ps"], ref64["psi"], lat.L, spec.nx)
    assert rel_max(m["b"], f64["b"]) <= 1e-5


def test_strong_landau_full_size_one_fp64_step():
    """4,194,304 decorated particles, +-0.25 cell jitter, nx 512, FP64: <= 1e-12."""
    need_gpu()
    spec = W.landau_strong(precision=64)
    lat = spec.lattice
    jx, jv = W.jitter(lat)
    sim = _sim([(lat.L, spec.dt, spec.nx, lat.n)], 64)
    try:
        sim.init_lattice(0, lat, jx, jv)
        sim.step(1)
        got = sim.state()
        m = sim.mesh(0)
    finally:
        sim.close()
    st = O.init_lattice(lat, jx, jv)
    ref = O.run(st, spec.nx, lat.L, spec.dt, 1, diag_every=0)
    f = O.field_of_state(ref["Q"], ref["ps"], ref["psi"], lat.L, spec.nx)
    assert rel_max(m["b"], f["b"]) <= 1e-12
    assert np.abs(periodic_diff(got["Q"], ref["Q"], lat.L)).max() <= 1e-12 * lat.L
    for k in ("P", "qs", "ps"):
        assert rel_max(got[k], ref[k]) <= 1e-12, k


def test_strong_landau_pic_16x_full_size_one_fp32_step():
    """Point-particle PIC at 16x the particles: 67,108,864 markers, decoration off."""
    need_gpu()
    spec = W.landau_strong(precision=32, scale=4, decorated=False)
    lat = spec.lattice
    jx, jv = W.jitter(lat)
    sim = _sim([(lat.L, spec.dt, spec.nx, lat.n)], 32, decorated=False)
    try:
        sim.init_lattice(0, lat, jx, jv)
        sim.step(1)
        got = sim.state()
        m = sim.mesh(0)
    finally:
        sim.close()
    st = cast_state(O.init_lattice(lat, jx, jv), 32)
    ref = O.run(st, spec.nx, lat.L, spec.dt, 1, diag_every=0, decorated=False, store_f32=True)
    b = O.deposit(ref["Q"], None, ref["psi"], lat.L, spec.nx,
                  elem=O.element_key(ref["Q"], lat.L, spec.nx, np.float32))
    assert rel_max(m["b"], b) <= 1e-5
    rng = np.random.default_rng(6)
    idx = np.sort(rng.choice(lat.n, SAMPLE, replace=False))
    _check_sample(got, ref, idx, lat.L, 1e-6)


def test_ensemble_full_size_one_batched_step():
    """256 runs, 20,537,344 particles, uneven lattices and meshes, one launch per
    step; 8 sampled runs compared with the oracle run alone."""
    need_gpu()
    runs = W.ensemble(precision=32)
    sim = _sim([(r.lattice.L, r.dt, r.nx, r.lattice.n) for r in runs], 32)
    try:
        for i, r in enumerate(runs):
            sim.init_lattice(i, r.lattice)
        sim.step(1)
        got = sim.state()
        meshes = {i: sim.mesh(i) for i in (0, 1, 37, 100, 128, 200, 254, 255)}
    finally:
        sim.close()
    off = np.cumsum([0] + [r.lattice.n for r in runs])
    for i, m in meshes.items():
        r = runs[i]
        lat = r.lattice
        st = cast_state(O.init_lattice(lat), 32)
        ref = O.run(st, r.nx, lat.L, r.dt, 1, diag_every=0, store_f32=True)
        b = O.deposit(ref["Q"], ref["ps"], ref["psi"], lat.L, r.nx,
                      elem=O.element_key(ref["Q"], lat.L, r.nx, np.float32))
        assert rel_max(m["b"], b) <= 1e-5, i
        sl = slice(off[i], off[i + 1])
        g = {k: v[sl] for k, v in got.items()}
        _check_sample(g, ref, np.arange(lat.n), lat.L, 1e-6)


def test_bump_on_tail_full_size_one_fp32_step_p2_field():
    """The benchmark workload with the P2 field (its own bench leg): 16.7M
    decorated FP32 particles, nx 1024, in the launch shape that leg tunes to
    (256 x 3, bulk copy), one step against the oracle's dense P2 solve."""
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    spec = W.bump_on_tail()
    lat = spec.lattice
    sim = _sim([(lat.L, spec.dt, spec.nx, lat.n)], 32, d2_mode=swpic.SWPIC_D2_P2, threads_per_block=256,
               blocks_per_sm=3, pipeline_stages=3)
    try:
        sim.init_lattice(0, lat)
        sim.step(1, diag_every=1)
        got = sim.state()
        d = sim.diagnostics()
    finally:
        sim.close()
    st = cast_state(O.init_lattice(lat), 32)
    ref = O.run(st, spec.nx, lat.L, spec.dt, 1, diag_every=1, d2_mode=swpic.SWPIC_D2_P2, store_f32=True)
    rng = np.random.default_rng(6)
    idx = np.sort(rng.choice(lat.n, SAMPLE, replace=False))
    _check_sample(got, ref, idx, lat.L, 1e-6)
    for col in (4, 6):            # P2 field energy and E_amp, both records
        assert rel_max(d[:, col], ref["diag"][:, col]) < 1e-5, col
