"""GPU parity of the P2 (quadratic Lagrange) field of Sec. 5 against the
oracle's dense P2 Galerkin solve, through the C ABI.

The kernels never assemble the 2 nx + 1 system: the element-midpoint unknowns
are eliminated (static condensation), so the vertex values come from the P1
solve of the same load and each element adds one curvature coefficient from
its exact integer midpoint load.  One FP64 step: every state array within
1e-12 and the diagnostics (with the P2 field energy and E_amp) within 1e-11.
FP32: the oracle keeps FP32 storage and FP32 element decisions.  Also: the
step in pieces equals the fused step (the stand-alone solve reads the same
midpoint accumulator), ragged batched runs with non-power-of-two meshes equal
the oracle run by run, the bulk-copy stream equals the register stream bit
for bit, and a long run tracks the oracle's energy history.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import cast_state, need_gpu, periodic_diff, rel_max

pytestmark = pytest.mark.gpu
P2 = 3


def _compare_state(got, ref, L, tol, keys=("Q", "P", "qs", "ps")):
    for k in keys:
        if ref.get(k) is None:
            continue
        if k == "Q":
            err = np.abs(periodic_diff(got[k], ref[k], L)).max() / L
        else:
            err = rel_max(got[k], ref[k])
        assert err <= tol, (k, err)


def _sim(runs, precision, **kw):
    from paper_2605_21794_gb300 import swpic
    return swpic.Simulation(runs, precision=precision, d2_mode=P2, **kw)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("decorated", [True, False])
def test_one_fp64_step_matches_oracle(mode, decorated):
    need_gpu()
    spec = W.landau_linear()
    L = spec.lattice.L
    st = W.random_state(4096, L, seed=21, nx=spec.nx)
    if not decorated:
        st["qs"] = None
        st["ps"] = None
    sim = _sim([(L, spec.dt, spec.nx, 4096)], 64, deposit_mode=mode, decorated=decorated)
    try:
        sim.init_particles(st)
        sim.step(1, diag_every=1)
        got = sim.state()
        diag = sim.diagnostics()
    finally:
        sim.close()
    ref = O.run(st, spec.nx, L, spec.dt, 1, diag_every=1, d2_mode=P2, decorated=decorated)
    _compare_state(got, ref, L, 1e-12, keys=("Q", "P", "qs", "ps") if decorated else ("Q", "P"))
    assert diag.shape[0] == 2
    for col in (1, 3, 4, 5, 6):
        assert rel_max(diag[:, col], ref["diag"][:, col]) < 1e-11, col


def test_p2_field_energy_exceeds_p1_by_the_curvature_term():
    """Same state, P1 lumped and P2: the element slopes agree (static
    condensation), so the P2 field energy is the P1 one plus (h/6) sum beta^2,
    with beta from the oracle's dense solve."""
    need_gpu()
    L, nx, n = 4 * np.pi, 48, 3000
    st = W.random_state(n, L, seed=5, nx=nx)
    W_ = {}
    for d2 in (0, P2):
        from paper_2605_21794_gb300 import swpic
        sim = swpic.Simulation([(L, 0.1, nx, n)], precision=64, d2_mode=d2)
        try:
            sim.init_particles(st)
            sim.step(1, diag_every=1)
            W_[d2] = sim.diagnostics()[0, 4]           # the t = 0 record: the initial field
        finally:
            sim.close()
    _, a, beta = O.p2_field(st["Q"], st["ps"], st["psi"], L, nx)
    h = L / nx
    assert W_[P2] - W_[0] == pytest.approx(h / 6 * np.sum(beta * beta), rel=1e-10)


def test_one_fp32_step_matches_fp32_oracle():
    need_gpu()
    lat = W.LatticeSpec(512, 256, 4 * np.pi, -6.0, 6.0, 0.5, 0.5, W.MAXWELL, jitter=0.25, seed=0)
    jx, jv = W.jitter(lat)
    st = cast_state(O.init_lattice(lat, jx, jv), 32)
    nx, dt = 128, 0.05
    sim = _sim([(lat.L, dt, nx, lat.n)], 32, deposit_mode=0)
    try:
        sim.init_lattice(0, lat, jx, jv)
        sim.step(1, diag_every=1)
        got = sim.state()
        diag = sim.diagnostics()
    finally:
        sim.close()
    ref = O.run(st, nx, lat.L, dt, 1, diag_every=1, d2_mode=P2, store_f32=True)
    _compare_state(got, ref, lat.L, 1e-6)
    for col in (4, 6):
        assert rel_max(diag[:, col], ref["diag"][:, col]) < 1e-5, col


def test_step_in_pieces_equals_fused_step():
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    spec = W.landau_linear(jitter=1e-3)
    jx, jv = W.jitter(spec.lattice)
    L = spec.lattice.L
    out = []
    for pieces in (False, True):
        sim = _sim([(L, spec.dt, spec.nx, spec.lattice.n)], 64, deposit_mode=1)
        try:
            sim.init_lattice(0, spec.lattice, jx, jv)
            for _ in range(3):
                if pieces:
                    swpic.swpic_gather_push(sim.ctx, 0.5, 1.0)
                    swpic.swpic_deposit(sim.ctx)
                    swpic.swpic_solve_field(sim.ctx)
                    swpic.swpic_gather_push(sim.ctx, 0.5, 0.0)
                else:
                    sim.step(1)
            out.append(sim.state())
        finally:
            sim.close()
    for k in ("Q", "P", "qs", "ps"):
        assert np.array_equal(out[0][k], out[1][k]), k


RUNS = [(4 * np.pi, 0.1, 64, 4097), (2 * np.pi / 0.45, 0.1, 30, 3), (9.0, 0.05, 128, 0),
        (9.0, 0.05, 100, 70001), (6.0, 0.02, 48, 1031)]


@pytest.mark.parametrize("mode", [0, 1])
def test_ragged_batch_matches_oracle_run_by_run(mode):
    """Run sizes not multiples of the vector width, an empty run, a run split
    over many CTAs, non-power-of-two meshes: three FP64 steps per run."""
    need_gpu()
    parts = [W.random_state(n, L, seed=40 + r, nx=nx) for r, (L, dt, nx, n) in enumerate(RUNS)]
    st = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    sim = _sim(RUNS, 64, deposit_mode=mode)
    try:
        sim.init_particles(st)
        sim.step(3, diag_every=1)
        got = sim.state()
        diags = [sim.diagnostics(r) for r in range(len(RUNS))]
    finally:
        sim.close()
    o = 0
    for r, (L, dt, nx, n) in enumerate(RUNS):
        g = {k: v[o:o + n] for k, v in got.items()}
        o += n
        if n == 0:
            continue
        ref = O.run(parts[r], nx, L, dt, 3, diag_every=1, d2_mode=P2)
        _compare_state(g, ref, L, 1e-11)
        for col in (4, 6):
            assert rel_max(diags[r][:, col], ref["diag"][:, col]) < 1e-10, (r, col)


@pytest.mark.parametrize("precision", [32, 64])
def test_bulk_stream_equals_register_stream_bitwise(precision):
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    out = []
    for stages in (0, 4):
        parts = [W.random_state(n, L, seed=80 + r, nx=nx) for r, (L, dt, nx, n) in enumerate(RUNS)]
        st = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
        sim = _sim(RUNS, precision, deposit_mode=1, resort_every=3, threads_per_block=256,
                   blocks_per_sm=2, pipeline_stages=stages)
        try:
            assert swpic.swpic_get_pipeline(sim.ctx)[1] == stages
            sim.init_particles(st)
            sim.step(7)
            out.append(sim.state())
        finally:
            sim.close()
    for k in ("Q", "P", "qs", "ps", "psi"):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_fifty_fp64_steps_track_the_oracle():
    need_gpu()
    spec = W.landau_linear(jitter=1e-3)
    jx, jv = W.jitter(spec.lattice)
    st = O.init_lattice(spec.lattice, jx, jv)
    L = spec.lattice.L
    sim = _sim([(L, spec.dt, spec.nx, spec.lattice.n)], 64)
    try:
        sim.init_lattice(0, spec.lattice, jx, jv)
        sim.step(50, diag_every=5)
        got = sim.state()
        diag = sim.diagnostics()
    finally:
        sim.close()
    ref = O.run(st, spec.nx, L, spec.dt, 50, diag_every=5, d2_mode=P2)
    _compare_state(got, ref, L, 1e-9, keys=("Q", "P"))
    assert diag.shape[0] == ref["diag"].shape[0]
    assert rel_max(diag[:, 6], ref["diag"][:, 6]) < 1e-8
    assert rel_max(diag[:, 5], ref["diag"][:, 5]) < 1e-11
