"""The bulk-copy (TMA) particle stream against the register-load stream.

Both streams push each particle with the same arithmetic and give every thread
the same vectors in the same order, so in the deterministic deposit mode (exact
integer accumulation) the whole state, the mesh charge and the field must agree
bit for bit, whatever the stage count; the diagnostic records agree up to the
order of the FP64 atomics that combine CTA partials.  The batch mixes ragged run sizes (run
starts that are not multiples of the vector width, a run shorter than one
vector, an empty run, partial last tiles) and re-sorts, which sends psi* through
the stream as well.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

RUNS = [(4 * np.pi, 0.1, 64, 4097), (2 * np.pi / 0.45, 0.1, 32, 3), (9.0, 0.05, 128, 0),
        (9.0, 0.05, 100, 70001), (6.0, 0.02, 48, 1031)]


def _batch_state(runs, seed):
    parts = [W.random_state(n, L, seed=seed + r, nx=nx) for r, (L, dt, nx, n) in enumerate(runs)]
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def _run(stages, precision, decorated, tpb, bpsm, resort, steps=7):
    from paper_2605_21794_gb300 import swpic
    st = _batch_state(RUNS, 70)
    if not decorated:
        st["qs"] = None
        st["ps"] = None
    sim = swpic.Simulation(RUNS, precision=precision, decorated=decorated, deposit_mode=1,
                           resort_every=resort, threads_per_block=tpb, blocks_per_sm=bpsm,
                           pipeline_stages=stages)
    try:
        req, eff = swpic.swpic_get_pipeline(sim.ctx)
        sim.init_particles(st)
        sim.step(steps, diag_every=2)
        out = sim.state()
        diags = [sim.diagnostics(r) for r in range(len(RUNS))]
        meshes = [sim.mesh(r) for r in range(len(RUNS))]
    finally:
        sim.close()
    return eff, out, diags, meshes


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("decorated", [True, False])
@pytest.mark.parametrize("stages,tpb,bpsm", [(2, 256, 2), (3, 128, 1), (4, 256, 2), (8, 128, 1)])
def test_bulk_stream_equals_register_stream_bitwise(precision, decorated, stages, tpb, bpsm):
    need_gpu()
    eff0, ref, dref, mref = _run(0, precision, decorated, tpb, bpsm, resort=3)
    eff, got, dgot, mgot = _run(stages, precision, decorated, tpb, bpsm, resort=3)
    assert eff0 == 0
    assert eff == stages, "the requested stages must fit this launch shape"
    for k in ("Q", "P", "qs", "ps", "psi"):
        if ref.get(k) is None:
            continue
        assert np.array_equal(got[k], ref[k]), k
    for r in range(len(RUNS)):
        # diagnostic partials meet in FP64 atomics across CTAs, whose order is
        # not fixed: equal to the rounding of that sum
        assert dgot[r].shape == dref[r].shape, r
        if dref[r].size:                 # an empty run keeps no records
            scale = np.abs(dref[r]).max(axis=0) + 1e-300
            assert (np.abs(dgot[r] - dref[r]) <= 1e-13 * scale).all(), r
        for k in ("b", "E"):
            assert np.array_equal(mgot[r][k], mref[r][k]), (r, k)


def test_stage_count_is_reduced_to_what_fits():
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    sim = swpic.Simulation([(9.0, 0.05, 4096, 100000)], precision=64, threads_per_block=512,
                           blocks_per_sm=4, pipeline_stages=8)
    try:
        req, eff = swpic.swpic_get_pipeline(sim.ctx)
        assert req == 8
        assert eff == 0        # 4 CTAs of 512 threads: not even two 40 KB stages fit beside a 4096 mesh
        swpic.swpic_set_launch(sim.ctx, 256, 1, 0)
        req, eff = swpic.swpic_get_pipeline(sim.ctx)
        assert 2 <= eff <= 8
        for bad in (-1, 1, 9):
            with pytest.raises(swpic.SwpicError):
                swpic.swpic_set_pipeline(sim.ctx, bad)
        assert swpic.swpic_get_pipeline(sim.ctx)[0] == 8
    finally:
        sim.close()
