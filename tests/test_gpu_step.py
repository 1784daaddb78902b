"""GPU parity of whole steps and runs against the FP64 oracle, through the C ABI.

One FP64 step: every state array within 1e-12 relative.  One FP32 step: the
mesh charge within 1e-5 relative (the FP32 path takes its element decisions
in FP32; both sides start from the same FP32 values).  Long runs, where
trajectories may diverge: field-energy / E_amp histories and fitted rates.
Also: batched runs equal the same runs alone, the deterministic mode is
bitwise reproducible, checkpoints resume bit for bit, the host-memory entry
point equals the device path, the step in pieces equals the fused step.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle as O
from workloads import physics as ph
import workloads as W
from gpu_util import cast_state, need_gpu, periodic_diff, rel_max

pytestmark = pytest.mark.gpu


def _sim(runs, precision, **kw):
    from paper_2605_21794_gb300 import swpic
    return swpic.Simulation(runs, precision=precision, **kw)


def _lattice_state(spec):
    jx, jv = W.jitter(spec.lattice)
    return O.init_lattice(spec.lattice, jx, jv), jx, jv


def _compare_state(got, ref, L, tol, keys=("Q", "P", "qs", "ps")):
    for k in keys:
        if ref.get(k) is None:
            continue
        if k == "Q":
            err = np.abs(periodic_diff(got[k], ref[k], L)).max() / L
        else:
            err = rel_max(got[k], ref[k])
        assert err <= tol, (k, err)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("d2_mode", [0, 2])
def test_one_fp64_step_matches_oracle(mode, d2_mode):
    """Identical seeded inputs on both sides (linear-Landau geometry: L = 4pi,
    nx 64, dt 0.1, 4096 particles): every array within 1e-12 after one step."""
    need_gpu()
    spec = W.landau_linear()
    L = spec.lattice.L
    st = W.random_state(4096, L, seed=11, nx=spec.nx)
    sim = _sim([(L, spec.dt, spec.nx, 4096)], 64, deposit_mode=mode, d2_mode=d2_mode)
    try:
        sim.init_particles(st)
        sim.step(1, diag_every=1)
        got = sim.state()
        diag = sim.diagnostics()
    finally:
        sim.close()
    ref = O.run(st, spec.nx, L, spec.dt, 1, diag_every=1, d2_mode=d2_mode)
    _compare_state(got, ref, L, 1e-12)
    assert diag.shape[0] == 2 and np.allclose(diag[:, 0], [0.0, spec.dt])
    for col, rc in ((1, 1), (3, 3), (4, 4), (5, 5), (6, 6)):
        assert rel_max(diag[:, col], ref["diag"][:, rc]) < 1e-11, col


def test_one_fp64_step_from_each_sides_lattice_init():
    """Each side initialises the jittered linear-Landau lattice itself.  With
    jitter 1e-3 cell, p* is a small remainder of the cell integral; the oracle
    forms sin(2pi (Q - q)/L) from Q - q directly and loses ~1e-12 of p* to
    cancellation (the kernel forms the angle from the offsets), so p*, q* are
    compared to 1e-10 and Q, P to 1e-12."""
    need_gpu()
    spec = W.landau_linear(jitter=1e-3)
    st, jx, jv = _lattice_state(spec)
    L = spec.lattice.L
    sim = _sim([(L, spec.dt, spec.nx, spec.lattice.n)], 64)
    try:
        sim.init_lattice(0, spec.lattice, jx, jv)
        sim.step(1, diag_every=1)
        got = sim.state()
    finally:
        sim.close()
    ref = O.run(st, spec.nx, L, spec.dt, 1, diag_every=1)
    _compare_state(got, ref, L, 1e-12, keys=("Q", "P"))
    _compare_state(got, ref, L, 1e-10, keys=("qs", "ps"))


@pytest.mark.parametrize("mode", [0, 1])
def test_one_fp32_step_mesh_charge_within_1e5(mode):
    """Strong-Landau lattice (jitter 0.25 cell, alpha 0.5) at a reduced size.
    The oracle keeps the state in FP32 storage and takes its element decisions
    in FP32 from the stored positions, as the FP32 path does; its arithmetic
    stays FP64."""
    need_gpu()
    lat = W.LatticeSpec(512, 256, 4 * np.pi, -6.0, 6.0, 0.5, 0.5, W.MAXWELL, jitter=0.25, seed=0)
    jx, jv = W.jitter(lat)
    st = cast_state(O.init_lattice(lat, jx, jv), 32)
    nx, dt = 128, 0.05
    sim = _sim([(lat.L, dt, nx, lat.n)], 32, deposit_mode=mode)
    try:
        sim.init_lattice(0, lat, jx, jv)
        sim.step(1)
        got = sim.state()
        m = sim.mesh(0)
    finally:
        sim.close()
    ref = O.run(st, nx, lat.L, dt, 1, diag_every=0, store_f32=True)
    b = O.deposit(ref["Q"], ref["ps"], ref["psi"], lat.L, nx,
                  elem=O.element_key(ref["Q"], lat.L, nx, np.float32))
    assert rel_max(m["b"], b) <= 1e-5
    _compare_state(got, ref, lat.L, 1e-6)


def _node_dipole_allowance(Q, ps, L, nx):
    """Sum of 2|p*|/h over the particles within 4 FP32 ulps of a node: the
    element decision of such a particle may differ between an FP32 state and
    an FP64 state, and the dipole term -p* phi_j'(Q) of Eq. rhs-assembly
    jumps by 2 p*/h across a node (the monopole term is continuous)."""
    x = np.asarray(Q, dtype=np.float64) * (nx / L)
    d = np.abs(x - np.round(x))
    ulp = np.spacing(np.float32(L)).astype(np.float64) * (nx / L)
    near = d <= 4 * ulp
    return float(np.sum(2 * np.abs(ps[near])) * nx / L)


@pytest.mark.parametrize("mode", [0, 1])
def test_one_fp32_step_mesh_charge_vs_plain_fp64_oracle(mode):
    """The same FP32 step against the plain FP64 oracle (FP64 state, FP64
    element decisions), from the same FP32-representable initial values: the
    mesh charge agrees within 1e-5 relative, plus the dipole jump of the
    particles that sit within FP32 rounding of a node (their element may be
    decided differently; one such particle of this jittered lattice moves
    ~1e-4 of max |b|)."""
    need_gpu()
    lat = W.LatticeSpec(512, 256, 4 * np.pi, -6.0, 6.0, 0.5, 0.5, W.MAXWELL, jitter=0.25, seed=0)
    jx, jv = W.jitter(lat)
    st = cast_state(O.init_lattice(lat, jx, jv), 32)
    nx, dt = 128, 0.05
    sim = _sim([(lat.L, dt, nx, lat.n)], 32, deposit_mode=mode)
    try:
        sim.init_particles(st)
        sim.step(1)
        m = sim.mesh(0)
    finally:
        sim.close()
    ref = O.run(st, nx, lat.L, dt, 1, diag_every=0)
    f = O.field_of_state(ref["Q"], ref["ps"], ref["psi"], lat.L, nx)
    scale = np.abs(f["b"]).max()
    allow = _node_dipole_allowance(ref["Q"], ref["ps"], lat.L, nx)
    assert np.abs(m["b"] - f["b"]).max() <= 1e-5 * scale + allow, (rel_max(m["b"], f["b"]), allow / scale)


def test_step_in_pieces_equals_fused_step():
    """KDK = gather_push(1/2, 1); deposit; solve_field; gather_push(1/2, 0)."""
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


def test_fifty_fp64_steps_track_the_oracle():
    need_gpu()
    spec = W.landau_linear(jitter=1e-3)
    st, jx, jv = _lattice_state(spec)
    L = spec.lattice.L
    sim = _sim([(L, spec.dt, spec.nx, spec.lattice.n)], 64)
    try:
        sim.init_lattice(0, spec.lattice, jx, jv)
        sim.step(20, diag_every=5)
        sim.step(30, diag_every=5)
        got = sim.state()
        diag = sim.diagnostics()
    finally:
        sim.close()
    ref = O.run(st, spec.nx, L, spec.dt, 50, diag_every=5)
    _compare_state(got, ref, L, 1e-10)
    assert diag.shape[0] == ref["diag"].shape[0]
    assert rel_max(diag[:, 6], ref["diag"][:, 6]) < 1e-9
    assert rel_max(diag[:, 5], ref["diag"][:, 5]) < 1e-12


def test_linear_landau_full_run_rates_match_oracle():
    """Linear Landau (64 x 64 lattice, nx 64, dt 0.1, 500 steps, FP64): the
    E_amp history and the fitted rate over t in [2, 10] agree with the oracle."""
    need_gpu()
    spec = W.landau_linear()
    st, _, _ = _lattice_state(spec)
    L = spec.lattice.L
    sim = _sim([(L, spec.dt, spec.nx, spec.lattice.n)], 64)
    try:
        sim.init_lattice(0, spec.lattice)
        sim.step(spec.steps, diag_every=1)
        diag = sim.diagnostics()
    finally:
        sim.close()
    ref = O.run(st, spec.nx, L, spec.dt, spec.steps, diag_every=1)
    g1, o1, _ = ph.rate_fit(diag[:, 0], diag[:, 6], 2.0, 10.0, min_sep=1.5)
    g2, o2, _ = ph.rate_fit(ref["diag"][:, 0], ref["diag"][:, 6], 2.0, 10.0, min_sep=1.5)
    assert abs(g1 / g2 - 1) < 0.01 and abs(o1 / o2 - 1) < 0.01
    assert rel_max(diag[:, 6], ref["diag"][:, 6]) < 1e-6
    assert rel_max(diag[:, 5], ref["diag"][:, 5]) < 1e-9


@pytest.mark.parametrize("prec", [32, 64])
def test_two_stream_growth_matches_oracle(prec):
    """Two-stream (256 x 256 lattice, nx 128, dt 0.05): the growth phase of
    E_amp and its fitted rate agree with the FP64 oracle within 1%."""
    need_gpu()
    spec = W.two_stream(precision=prec)
    st, _, _ = _lattice_state(spec)
    st = cast_state(st, prec)
    L = spec.lattice.L
    n_steps = 600                         # t = 30, before the decorations blow up
    sim = _sim([(L, spec.dt, spec.nx, spec.lattice.n)], prec)
    try:
        sim.init_lattice(0, spec.lattice)
        sim.step(n_steps, diag_every=1)
        diag = sim.diagnostics()
    finally:
        sim.close()
    ref = O.run(st, spec.nx, L, spec.dt, n_steps, diag_every=1)
    t, E, Er = diag[:, 0], diag[:, 6], ref["diag"][:, 6]
    sel = (t >= 6.0) & (t <= 13.0)
    g1 = np.polyfit(t[sel], np.log(E[sel]), 1)[0]
    g2 = np.polyfit(t[sel], np.log(Er[sel]), 1)[0]
    assert abs(g1 / g2 - 1) < 0.01
    assert np.abs(E[t <= 20] / Er[t <= 20] - 1).max() < 0.01
    assert rel_max(diag[:, 5], ref["diag"][:, 5]) < (1e-4 if prec == 32 else 1e-9)


def test_batched_runs_equal_runs_alone():
    need_gpu()
    specs = [(4 * np.pi, 0.1, 64, 4096), (2 * np.pi / 0.45, 0.1, 32, 1031), (9.0, 0.05, 128, 20000)]
    states = [W.random_state(n, L, seed=40 + r, nx=nx) for r, (L, dt, nx, n) in enumerate(specs)]
    cat = {k: np.concatenate([s[k] for s in states]) for k in states[0]}
    sim = _sim(specs, 64)
    try:
        sim.init_particles(cat)
        sim.step(10, diag_every=2)
        got = sim.state()
        dg = [sim.diagnostics(r) for r in range(3)]
    finally:
        sim.close()
    off = 0
    for r, (L, dt, nx, n) in enumerate(specs):
        one = _sim([specs[r]], 64)
        try:
            one.init_particles(states[r])
            one.step(10, diag_every=2)
            alone = one.state()
            da = one.diagnostics()
        finally:
            one.close()
        sl = slice(off, off + n)
        _compare_state({k: (v[sl] if v is not None else None) for k, v in got.items()}, alone, L, 1e-12)
        assert rel_max(dg[r][:, 6], da[:, 6]) < 1e-11
        off += n


def test_deterministic_mode_is_bitwise_reproducible_fp32():
    need_gpu()
    lat = W.LatticeSpec(512, 512, 4 * np.pi, -6.0, 6.0, 0.5, 0.5, W.MAXWELL, jitter=0.25, seed=0)
    jx, jv = W.jitter(lat)
    outs = []
    for rep in range(2):
        sim = _sim([(lat.L, 0.05, 128, lat.n)], 32, deposit_mode=1, resort_every=4)
        try:
            sim.init_lattice(0, lat, jx, jv)
            sim.step(20, diag_every=5)
            outs.append(sim.state())
        finally:
            sim.close()
    for k in ("Q", "P", "qs", "ps", "psi"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_checkpoint_resume_is_bitwise():
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    lat = W.LatticeSpec(256, 256, 4 * np.pi, -6.0, 6.0, 0.5, 0.5, W.MAXWELL, jitter=0.25, seed=0)
    jx, jv = W.jitter(lat)
    path = os.path.join(tempfile.mkdtemp(), "ck.bin")
    sim = _sim([(lat.L, 0.05, 128, lat.n)], 32, deposit_mode=1)
    try:
        sim.init_lattice(0, lat, jx, jv)
        sim.step(10, diag_every=5)
        swpic.swpic_save(sim.ctx, path)
        sim.step(10, diag_every=5)
        a = sim.state()
        da = sim.diagnostics()
        swpic.swpic_load(sim.ctx, path)
        sim.step(10, diag_every=5)
        b = sim.state()
        db = sim.diagnostics()
    finally:
        sim.close()
    for k in ("Q", "P", "qs", "ps", "psi"):
        assert np.array_equal(a[k], b[k]), k
    assert da[-1, 7] == 20 and db[-1, 7] == 20 and da[-1, 6] == db[-1, 6]


def test_host_entry_point_equals_device_path():
    need_gpu()
    import torch
    from paper_2605_21794_gb300 import swpic
    lat = W.LatticeSpec(256, 128, 4 * np.pi, -6.0, 6.0, 0.5, 0.5, W.MAXWELL, jitter=0.25, seed=3)
    jx, jv = W.jitter(lat)
    n = lat.n
    sim = _sim([(lat.L, 0.05, 128, n)], 32, deposit_mode=1)
    try:
        sim.init_lattice(0, lat, jx, jv)
        st = sim.state()
        sim.step(7)
        dev = sim.state()
        host_in = {k: torch.from_numpy(st[k].astype(np.float32)).pin_memory() for k in st}
        host_out = {k: torch.empty(n, dtype=torch.float32).pin_memory() for k in ("Q", "P", "qs", "ps")}
        p = lambda t: t.data_ptr()
        swpic.swpic_step_host(sim.ctx, p(host_in["Q"]), p(host_in["P"]), p(host_in["qs"]),
                              p(host_in["ps"]), p(host_in["psi"]), p(host_out["Q"]),
                              p(host_out["P"]), p(host_out["qs"]), p(host_out["ps"]), n, 7)
    finally:
        sim.close()
    for k in ("Q", "P", "qs", "ps"):
        assert np.array_equal(host_out[k].numpy().astype(np.float64), dev[k]), k


def test_resorting_changes_order_not_physics():
    need_gpu()
    lat = W.LatticeSpec(256, 256, 4 * np.pi, -6.0, 6.0, 0.5, 0.5, W.MAXWELL, jitter=0.25, seed=0)
    jx, jv = W.jitter(lat)
    res = []
    for rs in (0, 3):
        sim = _sim([(lat.L, 0.05, 128, lat.n)], 64, resort_every=rs)
        try:
            sim.init_lattice(0, lat, jx, jv)
            sim.step(12, diag_every=3)
            res.append((sim.state(), sim.diagnostics()))
        finally:
            sim.close()
    (a, da), (b, db) = res
    assert rel_max(db[:, 6], da[:, 6]) < 1e-11
    # same multiset of particles: order by (Q, P)
    oa = np.lexsort((a["P"], a["Q"]))
    ob = np.lexsort((b["P"], b["Q"]))
    for k in ("Q", "P", "qs", "ps", "psi"):
        assert rel_max(b[k][ob], a[k][oa]) < 1e-11, k
    # and the re-sorted state is ordered by element
    keys = O.element_key(b["Q"], lat.L, 128, np.float64)
    assert np.all(np.diff(keys[:1000]) >= -128)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_empty_run_and_empty_batch_member():
    need_gpu()
    sim = _sim([(1.0, 0.1, 8, 0)], 32)
    try:
        sim.step(3)
        assert sim.state()["Q"].size == 0
    finally:
        sim.close()
    specs = [(4.0, 0.1, 16, 1000), (3.0, 0.1, 8, 0), (5.0, 0.1, 32, 513)]
    st = [W.random_state(n, L, seed=60 + r, nx=nx) for r, (L, dt, nx, n) in enumerate(specs)]
    cat = {k: np.concatenate([s[k] for s in st]) for k in st[0]}
    sim = _sim(specs, 64)
    try:
        sim.init_particles(cat)
        sim.step(4, diag_every=1)
        got = sim.state()
        d2 = sim.diagnostics(2)
    finally:
        sim.close()
    ref = O.run(st[2], 32, 5.0, 0.1, 4, diag_every=1)
    _compare_state({k: v[1000:] for k, v in got.items()}, ref, 5.0, 1e-12)
    assert rel_max(d2[:, 6], ref["diag"][:, 6]) < 1e-11


def test_nodes_domain_edge_and_fast_particles():
    """Particles exactly on nodes, at the last representable point below L, and
    moving more than one period per step."""
    need_gpu()
    L, nx, dt = 8.0, 16, 0.5
    h = L / nx
    Q = np.array([0.0, h, 3 * h, L - h, np.nextafter(L, 0.0), 2.5, 7.75, 1e-300])
    P = np.array([0.0, 1.0, -3.0, 40.0, -37.3, 0.5, 100.0, -0.1])
    n = len(Q)
    st = {"Q": Q, "P": P, "qs": np.full(n, 0.01), "ps": np.full(n, 0.02), "psi": np.full(n, 0.125)}
    sim = _sim([(L, dt, nx, n)], 64)
    try:
        sim.init_particles(st)
        sim.step(3)
        got = sim.state()
    finally:
        sim.close()
    ref = O.run(st, nx, L, dt, 3, diag_every=0)
    assert np.all((got["Q"] >= 0) & (got["Q"] < L))
    _compare_state(got, ref, L, 1e-12)


def test_invalid_calls_are_rejected():
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    lib = swpic.load_library()
    sim = _sim([(4.0, 0.1, 16, 100)], 32, with_scratch=False)
    try:
        assert lib.swpic_step(sim.ctx, -1, 0) == swpic.SWPIC_EINVAL
        assert lib.swpic_sort(sim.ctx) == swpic.SWPIC_ESTATE          # no scratch bound
        assert lib.swpic_get_keys(sim.ctx, None, 99) == swpic.SWPIC_EINVAL
        assert lib.swpic_diagnostics(sim.ctx, 5, None, 0, None) == swpic.SWPIC_EINVAL
        assert lib.swpic_set_launch(sim.ctx, 100, 0, 0) == swpic.SWPIC_EINVAL
    finally:
        sim.close()
