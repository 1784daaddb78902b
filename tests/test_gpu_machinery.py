"""The machinery around the step, through the C ABI: the bounded device
wait (failure detection without a GPU fault), the autotuner, CUDA-graph
replay against direct launches, the 1D fixed-point overflow report, a
checkpoint loaded into a context that has already stepped, and the two
placements of the field solve."""
import json
import os

import numpy as np
import pytest

import workloads as W
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

L, NX, DT = 4 * np.pi, 64, 0.1


def _sim(n, **kw):
    from paper_2605_21794_gb300 import swpic
    return swpic.Simulation([(L, DT, NX, n)], precision=32, **kw)


def _states_equal(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("Q", "P", "qs", "ps", "psi"))


def test_bounded_wait_runs_out_reports_timeout_and_a_refresh_recovers():
    """A warp whose first stage is never armed waits 2 ms, flags the run, waits
    (bounded) for its other copies and its CTA leaves the pass; the next
    synchronous call reports SWPIC_ETIMEOUT and bit 4 of the run's status.
    Restoring the state and refreshing recovers: the next steps equal those of
    a fresh context bit for bit (deterministic deposit)."""
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    n = 100003
    st = W.random_state(n, L, seed=31, nx=NX)
    sim = _sim(n, deposit_mode=1, threads_per_block=256, blocks_per_sm=2, pipeline_stages=3)
    ref = _sim(n, deposit_mode=1, threads_per_block=256, blocks_per_sm=2, pipeline_stages=3)
    try:
        assert swpic.swpic_get_pipeline(sim.ctx)[1] == 3
        sim.init_particles(st)
        swpic.swpic_set_wait_test(sim.ctx, 0, 2_000_000)
        sim.step(1, 1)
        with pytest.raises(swpic.SwpicError) as e:
            swpic.swpic_synchronize(sim.ctx)
        assert e.value.status == swpic.SWPIC_ETIMEOUT
        assert swpic.swpic_run_status(sim.ctx, 1)[0] & 4
        # the context is still usable: restore, refresh (init_particles), step
        swpic.swpic_set_wait_test(sim.ctx, -1, 0)
        sim.init_particles(st)
        assert swpic.swpic_run_status(sim.ctx, 1)[0] == 0
        sim.step(3, 1)
        swpic.swpic_synchronize(sim.ctx)
        ref.init_particles(st)
        ref.step(3, 1)
        assert _states_equal(sim.state(), ref.state())
        with pytest.raises(swpic.SwpicError):
            swpic.swpic_set_wait_test(sim.ctx, -2, 0)
    finally:
        sim.close()
        ref.close()


def test_autotune_restores_state_and_picks_a_valid_shape(tmp_path):
    """The autotuner times its trials on the bound state and restores it bit
    for bit (state, step counter, records); the field is re-derived from it
    with the chosen launch shape (the deterministic deposit is exact for a
    fixed shape, so b agrees to the rounding of the per-segment FP32 sums);
    the chosen shape and stage count are valid ones and go into the JSON
    cache, from which a second context with the same configuration takes
    them."""
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    n = 200000
    st = W.random_state(n, L, seed=32, nx=NX)
    cache = str(tmp_path / "tune.json")
    sim = _sim(n, deposit_mode=1)
    try:
        sim.init_particles(st)
        sim.step(5, 1)
        before, mesh0 = sim.state(), sim.mesh(0)
        nrec0 = sim.diagnostics().shape[0]
        swpic.swpic_autotune(sim.ctx, 3, cache)
        after, mesh1 = sim.state(), sim.mesh(0)
        assert _states_equal(before, after)
        assert np.abs(mesh1["b"] - mesh0["b"]).max() <= 1e-6 * np.abs(mesh0["b"]).max()
        assert sim.diagnostics().shape[0] == nrec0
        tpb, bpsm, resort = swpic.swpic_get_launch(sim.ctx)
        req, eff = swpic.swpic_get_pipeline(sim.ctx)
        assert tpb in (128, 192, 256, 384, 512, 768) and bpsm in (1, 2, 3, 4, 6, 8)
        assert tpb * bpsm <= 2048 and resort in (0, 5, 20, 50)
        assert eff == 0 or 2 <= eff <= req
        with open(cache) as f:
            entries = json.load(f)
        assert entries, "the cache holds the tuned shape"
        # the step continues from where it was: 2 more steps are finite
        sim.step(2, 1)
        assert np.all(np.isfinite(sim.diagnostics()))
    finally:
        sim.close()
    sim2 = _sim(n, deposit_mode=1)
    try:
        sim2.init_particles(st)
        swpic.swpic_autotune(sim2.ctx, 3, cache)
        assert swpic.swpic_get_launch(sim2.ctx) == (tpb, bpsm, resort)
        assert swpic.swpic_get_pipeline(sim2.ctx)[0] == req
    finally:
        sim2.close()


def test_graph_replay_equals_direct_launches():
    """200 steps (graphs of >= 64 passes engage) with and without CUDA-graph
    capture, deterministic deposit: the states and mesh charges are equal bit
    for bit; the diagnostic records agree up to the order of the FP64 atomics
    that combine CTA partials."""
    need_gpu()
    n = 70001
    st = W.random_state(n, L, seed=33, nx=NX)
    out = []
    for graphs in (True, False):
        sim = _sim(n, deposit_mode=1, use_graphs=graphs, resort_every=20, diag_capacity=64)
        try:
            sim.init_particles(st)
            sim.step(200, 5)
            out.append((sim.state(), sim.mesh(0), sim.diagnostics()))
        finally:
            sim.close()
    (a, ma, da), (b, mb, db) = out
    assert _states_equal(a, b)
    assert np.array_equal(ma["b"], mb["b"]) and np.array_equal(ma["E"], mb["E"])
    assert da.shape == db.shape
    scale = np.abs(db).max(axis=0) + 1e-300
    assert (np.abs(da - db) <= 1e-12 * scale).all()


@pytest.mark.parametrize("precision", [32, 64])
def test_accumulator_overflow_is_reported_and_a_refresh_recovers(precision):
    """Weights scaled far beyond the fixed-point unit taken at set-up: the
    deposit flags the overflow (no wrap-around), the next synchronous call
    reports SWPIC_ENUMERIC with bit 1 of the run's status, and a refresh takes
    a new unit from which the steps are finite again."""
    need_gpu()
    import torch
    from paper_2605_21794_gb300 import swpic
    n = 5000
    st = W.random_state(n, L, seed=34, nx=NX)
    sim = swpic.Simulation([(L, DT, NX, n)], precision=precision)
    try:
        sim.init_particles(st)
        torch.cuda.synchronize()
        sim.psi.mul_(1e6)
        torch.cuda.synchronize()
        sim.step(1)
        with pytest.raises(swpic.SwpicError) as e:
            swpic.swpic_synchronize(sim.ctx)
        assert e.value.status == swpic.SWPIC_ENUMERIC
        assert swpic.swpic_run_status(sim.ctx, 1)[0] & 1
        swpic.swpic_refresh(sim.ctx)
        sim.step(2, 1)
        swpic.swpic_synchronize(sim.ctx)
        d = sim.diagnostics()
        assert np.all(np.isfinite(d[-3:, 1:7]))
    finally:
        sim.close()


def test_load_into_a_context_that_has_stepped(tmp_path):
    """A checkpoint loaded into a context that has already run: the state,
    the step count and the following steps are those of the saved run (to
    FP64 rounding: the loading context takes its fixed-point charge unit from
    the loaded state, the saving context took it at its start), and the
    context's earlier diagnostic records are discarded (its records restart at
    the checkpoint)."""
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    n = 30011
    st = W.random_state(n, L, seed=35, nx=NX)
    path = str(tmp_path / "ck.bin")
    a = swpic.Simulation([(L, DT, NX, n)], precision=64, deposit_mode=1)
    try:
        a.init_particles(st)
        a.step(4, 1)
        swpic.swpic_save(a.ctx, path)
        a.step(3, 1)
        ref, dref = a.state(), a.diagnostics()
    finally:
        a.close()
    b = swpic.Simulation([(L, DT, NX, n)], precision=64, deposit_mode=1)
    try:
        b.init_particles(W.random_state(n, L, seed=36, nx=NX))
        b.step(9, 1)
        swpic.swpic_load(b.ctx, path)
        b.step(3, 1)
        got, dgot = b.state(), b.diagnostics()
    finally:
        b.close()
    for k in ("Q", "P", "qs", "ps"):
        assert np.abs(got[k] - ref[k]).max() <= 1e-12 * np.abs(ref[k]).max(), k
    assert np.array_equal(got["psi"], ref["psi"])
    assert dgot.shape[0] <= 4
    np.testing.assert_array_equal(dgot[-3:, 0], dref[-3:, 0])
    np.testing.assert_allclose(dgot[-3:, 6], dref[-3:, 6], rtol=1e-13)


@pytest.mark.parametrize("precision,d2_mode,runs", [(32, 0, 1), (64, 0, 1), (32, 3, 3), (64, 2, 3), (32, 0, 6)])
def test_field_solved_at_pass_start_equals_last_cta_solve(precision, d2_mode, runs):
    """The two placements of the field solve (swpic_set_field_solve): each
    depositing pass ending in a one-CTA solve, or every CTA of the next pass
    solving the finished deposit at its start.  Deterministic deposit, a call
    of 60 steps (direct launches) and one of 200 (a graph of 195 passes),
    several runs and phi'' readings, weak decorations (a noisy random plasma
    with the default ones grows them past the fixed-point headroom within a
    few hundred steps): states, mesh charges and fields are equal bit for
    bit, records up to the order of the FP64 atomics that combine CTA
    partials."""
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    sizes = [70001, 33333, 50002, 20000, 41111, 9999][:runs]
    cfg = [(L * (1 + 0.25 * r), DT, NX, n) for r, n in enumerate(sizes)]
    parts = [W.random_state(n, Lr, seed=40 + r, nx=NX, dipole_scale=0.02) for r, (Lr, _, _, n) in enumerate(cfg)]
    st = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    out = []
    for mode in (swpic.SWPIC_FIELD_SOLVE_LAST_CTA, swpic.SWPIC_FIELD_SOLVE_AT_START):
        sim = swpic.Simulation(cfg, precision=precision, deposit_mode=1, d2_mode=d2_mode, resort_every=7,
                               diag_capacity=512)
        try:
            swpic.swpic_set_field_solve(sim.ctx, mode)
            assert swpic.swpic_get_field_solve(sim.ctx) == (mode, mode)
            sim.init_particles(st)
            sim.step(60, 3)
            sim.step(200, 5)
            out.append((sim.state(), [sim.mesh(r) for r in range(runs)],
                        [sim.diagnostics(r) for r in range(runs)]))
        finally:
            sim.close()
    (a, ma, da), (b, mb, db) = out
    assert _states_equal(a, b)
    for r in range(runs):
        for k in ("b", "E"):
            assert np.array_equal(ma[r][k], mb[r][k]), (r, k)
    for r in range(runs):
        assert da[r].shape == db[r].shape
        scale = np.abs(db[r]).max(axis=0) + 1e-300
        assert (np.abs(da[r] - db[r]) <= 1e-12 * scale).all(), r


def test_field_solve_placement_default_follows_the_run_count():
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    for runs, eff in ((1, swpic.SWPIC_FIELD_SOLVE_AT_START), (4, swpic.SWPIC_FIELD_SOLVE_AT_START),
                      (5, swpic.SWPIC_FIELD_SOLVE_LAST_CTA)):
        sim = swpic.Simulation([(L, DT, NX, 1000)] * runs, precision=32)
        try:
            assert swpic.swpic_get_field_solve(sim.ctx) == (swpic.SWPIC_FIELD_SOLVE_AUTO, eff)
            with pytest.raises(swpic.SwpicError):
                swpic.swpic_set_field_solve(sim.ctx, 3)
        finally:
            sim.close()
