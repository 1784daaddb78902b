"""GPU parity of the 2D2V decorated-particle step (general-d model of Sec. 3.3
on the torus, bilinear elements) against the 2D oracle, through the C ABI
of include/swpic2d.h.

The kernels solve the Q1 system by the discrete Fourier transform (the
stiffness is diagonal in Fourier modes) and take the projected gradient from
its closed form; the oracle assembles the stiffness by quadrature, solves
the bordered system by LU and projects by quadrature.  FP64: the field
(b, Phi, g) within 1e-12 of the oracle's, every state array within 1e-12
after one step, diagnostics within 1e-11, several steps within 1e-10.  FP32:
the oracle keeps FP32 storage and FP32 cell decisions; 1e-5.  Also: a call
of n steps equals n calls of one step (the closing and opening half-kicks of
the fused pass are the same two operations) up to the order of the deposit's
shared-memory sums, an empty run, invalid calls, and the workload size at
the property level.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import need_gpu, periodic_diff, rel_max

pytestmark = pytest.mark.gpu
KEYS = ("Qx", "Qy", "Px", "Py", "qx", "qy", "px", "py")


def _sim(Lx, Ly, nx, ny, dt, n, precision, **kw):
    from paper_2605_21794_gb300 import swpic
    return swpic.Simulation2D(Lx, Ly, nx, ny, dt, n, precision=precision, **kw)


def _cast(st, precision):
    dt = np.float32 if precision == 32 else np.float64
    return {k: (None if v is None else np.asarray(v).astype(dt).astype(np.float64)) for k, v in st.items()}


def _compare(got, ref, Lx, Ly, tol, keys=KEYS):
    for k in keys:
        if ref.get(k) is None or got.get(k) is None:
            continue
        if k in ("Qx", "Qy"):
            L = Lx if k == "Qx" else Ly
            err = np.abs(periodic_diff(got[k], ref[k], L)).max() / L
        else:
            err = rel_max(got[k], ref[k])
        assert err <= tol, (k, err)


def _run(precision, st, Lx, Ly, nx, ny, dt, steps, diag_every=1, decorated=True, calls=None):
    sim = _sim(Lx, Ly, nx, ny, dt, len(st["Qx"]), precision, decorated=decorated)
    try:
        sim.init_particles(st)
        for k in (calls or [steps]):
            sim.step(k, diag_every)
        return sim.state(), sim.diagnostics(), sim.field()
    finally:
        sim.close()


@pytest.mark.parametrize("decorated", [True, False])
def test_field_of_a_state_matches_oracle_fp64(decorated):
    need_gpu()
    Lx, Ly, nx, ny = 4 * np.pi, 2 * np.pi, 32, 16
    st = W.random_state_2d(6000, Lx, Ly, seed=3, nx=nx, ny=ny, decorated=decorated)
    sim = _sim(Lx, Ly, nx, ny, 0.1, 6000, 64, decorated=decorated)
    try:
        sim.init_particles(st)
        f = sim.field()
    finally:
        sim.close()
    b = O.deposit2d(st["Qx"], st["Qy"], st["px"] if decorated else None, st["py"], st["psi"], Lx, Ly, nx, ny)
    Phi, _ = O.solve2d(b, Lx, Ly)
    gx, gy = O.project2d(Phi, Lx, Ly)
    assert rel_max(f["b"], b) < 1e-12
    assert rel_max(f["Phi"], Phi) < 1e-12
    assert rel_max(f["gx"], gx) < 1e-12
    assert rel_max(f["gy"], gy) < 1e-12


@pytest.mark.parametrize("decorated", [True, False])
def test_one_fp64_step_matches_oracle(decorated):
    need_gpu()
    Lx, Ly, nx, ny, dt = 4 * np.pi, 4 * np.pi, 16, 16, 0.1
    st = W.random_state_2d(4096, Lx, Ly, seed=11, nx=nx, ny=ny, decorated=decorated)
    got, diag, _ = _run(64, st, Lx, Ly, nx, ny, dt, 1, decorated=decorated)
    ref = O.run2d(st, nx, ny, Lx, Ly, dt, 1, diag_every=1, decorated=decorated)
    _compare(got, ref, Lx, Ly, 1e-12, KEYS if decorated else KEYS[:4])
    assert diag.shape == (2, 9)
    np.testing.assert_allclose(diag[:, 0], [0.0, dt])
    np.testing.assert_array_equal(diag[:, 8], [0, 1])
    for c in range(1, 8):
        assert rel_max(diag[:, c], ref["diag"][:, c]) < 1e-11, c


def test_several_fp64_steps_non_square_mesh_ragged_count():
    need_gpu()
    Lx, Ly, nx, ny, dt = 6.0, 2.5, 32, 8, 0.05
    st = W.random_state_2d(1031, Lx, Ly, seed=12, nx=nx, ny=ny, alpha=0.3)
    got, diag, _ = _run(64, st, Lx, Ly, nx, ny, dt, 6, diag_every=2)
    ref = O.run2d(st, nx, ny, Lx, Ly, dt, 6, diag_every=2)
    _compare(got, ref, Lx, Ly, 1e-10)
    assert diag.shape[0] == ref["diag"].shape[0] == 4
    for c in range(1, 8):
        assert rel_max(diag[:, c], ref["diag"][:, c]) < 1e-10, c


def test_one_fp32_step_matches_fp32_oracle():
    need_gpu()
    Lx, Ly, nx, ny, dt = 4 * np.pi, 2 * np.pi, 32, 16, 0.1
    st = _cast(W.random_state_2d(20000, Lx, Ly, seed=13, nx=nx, ny=ny, alpha=0.2), 32)
    got, diag, _ = _run(32, st, Lx, Ly, nx, ny, dt, 1)
    ref = O.run2d(st, nx, ny, Lx, Ly, dt, 1, diag_every=1, store_f32=True)
    _compare(got, ref, Lx, Ly, 1e-5)
    for c in (1, 2, 3, 4, 5, 7):
        assert rel_max(diag[:, c], ref["diag"][:, c]) < 1e-5, c


@pytest.mark.parametrize("precision", [32, 64])
def test_n_steps_in_one_call_equal_n_calls(precision):
    """Same operations either way; the per-CTA shared-memory sums of the
    deposit meet in an order the hardware picks, so the two agree to the
    rounding of those sums, not bit for bit."""
    need_gpu()
    Lx, Ly, nx, ny, dt = 5.0, 5.0, 16, 32, 0.08
    st = _cast(W.random_state_2d(3000, Lx, Ly, seed=14, nx=nx, ny=ny), precision)
    a, da, fa = _run(precision, st, Lx, Ly, nx, ny, dt, 4, diag_every=1)
    b, db, fb = _run(precision, st, Lx, Ly, nx, ny, dt, 4, diag_every=1, calls=[1, 1, 2])
    tol = 1e-5 if precision == 32 else 1e-12
    _compare(a, b, Lx, Ly, tol)
    np.testing.assert_array_equal(da[:, 8], np.arange(5))
    np.testing.assert_array_equal(db[:, 8], np.arange(5))
    assert rel_max(fa["Phi"], fb["Phi"]) < tol


def test_empty_run_and_invalid_calls():
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    sim = _sim(1.0, 1.0, 8, 8, 0.1, 0, 32)
    try:
        sim.init_particles({k: np.zeros(0) for k in swpic.STATE2D})
        sim.step(3, 1)
        d = sim.diagnostics()
        assert d.shape == (4, 9) and np.all(d[:, 1:8] == 0.0)
        with pytest.raises(swpic.SwpicError):
            swpic.swpic2d_step(sim.ctx, -1, 0)
    finally:
        sim.close()
    sim = _sim(1.0, 1.0, 8, 8, 0.1, 10, 32)
    try:
        with pytest.raises(swpic.SwpicError) as e:        # no refresh after binding
            swpic.swpic2d_step(sim.ctx, 1, 0)
        assert e.value.status == swpic.SWPIC_ESTATE
    finally:
        sim.close()


def test_workload_size_properties():
    """16,777,216 FP32 particles on a 32 x 32 mesh (the 2D benchmark's size):
    the field of the state against the oracle's (FP32 cell decisions), mass
    and charge conservation over steps, the diagnostics finite."""
    need_gpu()
    n, Lx, Ly, nx, ny, dt = 1 << 24, 4 * np.pi, 4 * np.pi, 32, 32, 0.1
    st = _cast(W.random_state_2d(n, Lx, Ly, seed=15, nx=nx, ny=ny, alpha=0.1), 32)
    sim = _sim(Lx, Ly, nx, ny, dt, n, 32)
    try:
        sim.init_particles(st)
        f0 = sim.field()
        sim.step(5, 1)
        f1 = sim.field()
        d = sim.diagnostics()
    finally:
        sim.close()
    cx = O.cell2d(st["Qx"], Lx, nx, f32=True)
    cy = O.cell2d(st["Qy"], Ly, ny, f32=True)
    b = O.deposit2d(st["Qx"], st["Qy"], st["px"], st["py"], st["psi"], Lx, Ly, nx, ny, cx=cx, cy=cy)
    assert rel_max(f0["b"], b) < 1e-5
    Phi, _ = O.solve2d(b, Lx, Ly)
    assert rel_max(f0["Phi"], Phi) < 1e-4
    total = st["psi"].sum()
    assert f1["b"].sum() == pytest.approx(total, rel=1e-6)
    assert np.all(np.isfinite(d)) and d.shape[0] == 6
    np.testing.assert_allclose(d[:, 1], total, rtol=1e-6)


@pytest.mark.parametrize("nx,ny", [(4, 256), (256, 4)])
def test_extreme_aspect_meshes_fp64(nx, ny):
    """The smallest axis (4 cells) against the longest (256): one FP64 step."""
    need_gpu()
    Lx, Ly, dt = 2.0 * nx / 16, 2.0 * ny / 16, 0.05
    st = W.random_state_2d(3000, Lx, Ly, seed=16, nx=nx, ny=ny, alpha=0.2)
    got, diag, _ = _run(64, st, Lx, Ly, nx, ny, dt, 2, diag_every=1)
    ref = O.run2d(st, nx, ny, Lx, Ly, dt, 2, diag_every=1)
    _compare(got, ref, Lx, Ly, 1e-11)
    for c in range(1, 8):
        assert rel_max(diag[:, c], ref["diag"][:, c]) < 1e-10, c


def test_fp32_point_particles_and_largest_fp32_mesh():
    """Undecorated FP32 particles on the largest FP32 mesh (128 x 64 = 8192
    nodes: the table and mesh fill 160 KB of shared memory) against the
    FP32-storage oracle, whose dense solve is the slow part here."""
    need_gpu()
    Lx, Ly, nx, ny, dt = 8.0, 4.0, 128, 64, 0.05
    st = _cast(W.random_state_2d(30000, Lx, Ly, seed=17, nx=nx, ny=ny, decorated=False, alpha=0.3), 32)
    got, diag, _ = _run(32, st, Lx, Ly, nx, ny, dt, 1, decorated=False)
    ref = O.run2d(st, nx, ny, Lx, Ly, dt, 1, diag_every=1, decorated=False, store_f32=True)
    _compare(got, ref, Lx, Ly, 1e-5, KEYS[:4])
    for c in (1, 2, 3, 4, 5, 7):
        assert rel_max(diag[:, c], ref["diag"][:, c]) < 1e-4, c


@pytest.mark.parametrize("precision", [64, 32])
def test_lattice_init_matches_oracle(precision):
    """The device builds the lattice state itself (n^4 Gauss rule in FP64)."""
    need_gpu()
    sp = W.Lattice2DSpec(8, 4, 12, 10, 4 * np.pi, 2 * np.pi, -6.0, 6.0, 0.2, 0.5, 1.0, 1.0, 3, True)
    sim = _sim(sp.Lx, sp.Ly, 16, 8, 0.1, sp.n, precision)
    try:
        sim.init_lattice(sp)
        got = sim.state()
    finally:
        sim.close()
    ref = _cast(O.init_lattice2d(sp), precision)
    tol = 1e-13 if precision == 64 else 0.0
    for k in ("Qx", "Qy", "Px", "Py", "psi", "qx", "qy", "px", "py"):
        s = np.abs(ref[k]).max()
        assert np.abs(got[k] - ref[k]).max() <= max(tol * s, 0.0 if precision == 64 else 2e-7 * s), k


def test_axis_mode_reproduces_the_1d_step():
    """A y-uniform f0 on a lattice whose y spacing is the mesh spacing keeps
    the field y-independent (rows of particles deposit uniformly, and their
    y-dipoles cancel along each row), so every particle's x-motion is that of
    a 1D particle: the 2D step must reproduce the 1D step run on the rows
    merged into 1D particles (weights summed over y and vy, divided by Ly).
    Both GPU paths (each pinned to its own oracle) advance 100 FP64 steps of
    linear Landau damping from the oracle's lattice; E_amp agrees."""
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    L, Ly, nqx, nqy, nvx, nvy = 4 * np.pi, 3.0, 32, 4, 48, 6
    sp = W.Lattice2DSpec(nqx, nqy, nvx, nvy, L, Ly, -6.0, 6.0, 0.01, 0.5, 0.0, 1.0, 2, True)
    st2 = O.init_lattice2d(sp)
    sim = _sim(L, Ly, 32, nqy, 0.05, sp.n, 64)
    try:
        sim.init_particles(st2)
        sim.step(100, 1)
        d2 = sim.diagnostics()
    finally:
        sim.close()
    shape = (nvx, nvy, nqy, nqx)                   # particle index ((k nvy + l) nqy + j) nqx + i
    merged = lambda k: st2[k].reshape(shape).sum(axis=(1, 2)).ravel() / Ly
    st1 = {"Q": st2["Qx"].reshape(shape)[:, 0, 0, :].ravel(), "P": st2["Px"].reshape(shape)[:, 0, 0, :].ravel(),
           "psi": merged("psi"), "qs": merged("qx"), "ps": merged("px")}
    s1 = swpic.Simulation([(L, 0.05, 32, len(st1["Q"]))], precision=64)
    try:
        s1.init_particles(st1)
        s1.step(100, 1)
        d1 = s1.diagnostics()
    finally:
        s1.close()
    assert d1.shape[0] == d2.shape[0] == 101
    assert rel_max(d2[:, 7], d1[:, 6]) < 1e-8
    assert rel_max(d2[:, 5], Ly * d1[:, 4]) < 1e-8          # W_2D = Ly W_1D


def test_oblique_landau_damping_rate():
    """Linear Landau damping of an oblique mode, k = (1, 1) 2 pi / L with
    |k| = 1/2, from the decorated lattice start: the decay rate of E_amp fitted
    over t in [1, 8] is the kinetic dispersion root of a Maxwellian at |k|
    (an isotropic plasma damps an oblique mode as a 1D one of the same |k|)
    within 10%, the accuracy the 1D step has at this resolution."""
    need_gpu()
    from workloads import physics as ph
    kq = 0.5 / np.sqrt(2)
    L = 2 * np.pi / kq
    sp = W.Lattice2DSpec(32, 32, 48, 48, L, L, -6.0, 6.0, 0.01, kq, kq, 1.0, 2, True)
    sim = _sim(L, L, 32, 32, 0.05, sp.n, 64)
    try:
        sim.init_lattice(sp)
        sim.step(180, 1)
        d = sim.diagnostics()
    finally:
        sim.close()
    root = ph.landau_root(0.5, 1.4 - 0.15j)
    g, _, _ = ph.rate_fit(d[:, 0], d[:, 7], 1.0, 8.0, min_sep=1.0)
    assert g == pytest.approx(root.imag, rel=0.10), (g, root)


def test_largest_fp64_mesh_one_step():
    """The largest FP64 mesh (64 x 64 = 4096 nodes; table and padded mesh fill
    166 KB of shared memory): one decorated FP64 step against the oracle."""
    need_gpu()
    Lx, Ly, nx, ny, dt = 4 * np.pi, 4 * np.pi, 64, 64, 0.05
    st = W.random_state_2d(20000, Lx, Ly, seed=18, nx=nx, ny=ny, alpha=0.2)
    got, diag, _ = _run(64, st, Lx, Ly, nx, ny, dt, 1, diag_every=1)
    ref = O.run2d(st, nx, ny, Lx, Ly, dt, 1, diag_every=1)
    _compare(got, ref, Lx, Ly, 1e-12)
    for c in range(1, 8):
        assert rel_max(diag[:, c], ref["diag"][:, c]) < 1e-11, c


@pytest.mark.parametrize("precision", [32, 64])
def test_accumulator_overflow_is_reported_and_a_refresh_recovers(precision):
    """Weights scaled far beyond the fixed-point unit taken at refresh: the
    deposit flags the overflow (no wrap-around), the next synchronous call
    reports SWPIC_ENUMERIC, and a refresh takes a new unit."""
    need_gpu()
    import torch
    from paper_2605_21794_gb300 import swpic
    L, nx = 4.0, 16
    st = W.random_state_2d(1000, L, L, seed=19, nx=nx, ny=nx)
    sim = _sim(L, L, nx, nx, 0.05, 1000, precision)
    try:
        sim.init_particles(st)
        torch.cuda.synchronize()
        sim.t["psi"].mul_(1e6)
        torch.cuda.synchronize()
        sim.step(1)
        with pytest.raises(swpic.SwpicError) as e:
            swpic.swpic2d_synchronize(sim.ctx)
        assert e.value.status == swpic.SWPIC_ENUMERIC
        swpic.swpic2d_refresh(sim.ctx)
        sim.step(2, 1)
        d = sim.diagnostics()
        assert np.all(np.isfinite(d[-3:, 1:8]))
    finally:
        sim.close()


def test_checkpoint_resume(tmp_path):
    """Save after 3 FP64 steps, run 4 more; a fresh context loading the file
    and running the same 4 steps reaches the same state (up to the order of
    the deposit's shared-memory sums) with the same step numbering; a
    mismatched context and a missing file are refused."""
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    Lx, Ly, nx, ny, dt = 5.0, 4.0, 16, 16, 0.05
    st = W.random_state_2d(2500, Lx, Ly, seed=20, nx=nx, ny=ny, alpha=0.2)
    path = str(tmp_path / "ck.bin")
    a = _sim(Lx, Ly, nx, ny, dt, 2500, 64)
    try:
        a.init_particles(st)
        a.step(3, 1)
        swpic.swpic2d_save(a.ctx, path)
        a.step(4, 1)
        ref, dref = a.state(), a.diagnostics()
    finally:
        a.close()
    b = _sim(Lx, Ly, nx, ny, dt, 2500, 64)
    try:
        swpic.swpic2d_load(b.ctx, path)
        b.step(4, 1)
        got, dgot = b.state(), b.diagnostics()
    finally:
        b.close()
    _compare(got, ref, Lx, Ly, 1e-12)
    np.testing.assert_array_equal(dgot[:, 8], np.arange(4, 8))
    assert rel_max(dgot[:, 6], dref[-4:, 6]) < 1e-12
    # a context that has already stepped loads the same file: its earlier
    # records are discarded and the records restart at the checkpoint
    d = _sim(Lx, Ly, nx, ny, dt, 2500, 64)
    try:
        d.init_particles(st)
        d.step(6, 1)
        swpic.swpic2d_load(d.ctx, path)
        d.step(4, 1)
        got2, dgot2 = d.state(), d.diagnostics()
    finally:
        d.close()
    _compare(got2, ref, Lx, Ly, 1e-12)
    np.testing.assert_array_equal(dgot2[:, 8], np.arange(4, 8))
    c = _sim(Lx, Ly, nx, ny, dt, 2500, 32)
    try:
        with pytest.raises(swpic.SwpicError) as e:
            swpic.swpic2d_load(c.ctx, path)
        assert e.value.status == swpic.SWPIC_EINVAL
        with pytest.raises(swpic.SwpicError) as e:
            swpic.swpic2d_load(c.ctx, str(tmp_path / "missing.bin"))
        assert e.value.status == swpic.SWPIC_EIO
    finally:
        c.close()


def test_host_entry_point_equals_device_path():
    """swpic2d_step_host from host arrays (copies, refresh, steps, copies
    back) reaches the device path's state (FP64, up to the order of the
    deposit's shared-memory sums)."""
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    Lx, Ly, nx, ny, dt = 5.0, 4.0, 16, 16, 0.05
    st = W.random_state_2d(2100, Lx, Ly, seed=21, nx=nx, ny=ny, alpha=0.2)
    ref, _, _ = _run(64, st, Lx, Ly, nx, ny, dt, 5, diag_every=0)
    sim = _sim(Lx, Ly, nx, ny, dt, 2100, 64)
    try:
        hin = [np.ascontiguousarray(st[k], dtype=np.float64) for k in swpic.STATE2D]
        hout = [np.zeros(2100) for _ in swpic.STATE2D[:8]]
        swpic.swpic2d_step_host(sim.ctx, [a.ctypes.data for a in hin], [a.ctypes.data for a in hout], 5, 0)
    finally:
        sim.close()
    got = dict(zip(swpic.STATE2D[:8], hout))
    _compare(got, ref, Lx, Ly, 1e-12)
