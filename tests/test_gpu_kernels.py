"""GPU parity of each piece of the step against the FP64 oracle, through the C ABI.

Sizes span several CTA chunks, vector widths and ragged tails; every input is
seeded and synthetic (workloads), identical on both sides.  Tolerances: keys
and the sort are bit-exact; FP64 values within 1e-12 relative (max-norm
relative to the largest oracle value); FP32 values within 1e-5 relative
(mesh charge) or the FP32 rounding of the quantity.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import cast_state, need_gpu, periodic_diff, rel_max

pytestmark = pytest.mark.gpu

PRECS = [32, 64]


def _sim(runs, precision, **kw):
    from paper_2605_21794_gb300 import swpic
    return swpic.Simulation(runs, precision=precision, **kw)


def _rand_runs(specs, seed=0, decorated=True):
    """specs: list of (L, dt, nx, n). Returns per-run FP64 states and the concatenation."""
    states = [W.random_state(n, L, seed=seed + 17 * r, decorated=decorated, nx=nx)
              for r, (L, dt, nx, n) in enumerate(specs)]
    cat = {k: np.concatenate([s[k] for s in states]) for k in states[0]}
    return states, cat


RAGGED = [(2.0 * np.pi, 0.1, 16, 1), (4 * np.pi, 0.05, 64, 4099), (7.3, 0.1, 33, 40001),
          (3.0, 0.2, 128, 3)]


# ---------------------------------------------------------------------------
# a1 keys and a2 stable sort: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PRECS)
def test_keys_bit_exact(prec):
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    states, cat = _rand_runs(RAGGED, seed=1)
    sim = _sim(RAGGED, prec)
    try:
        sim.init_particles(cat)
        keys = swpic.swpic_get_keys(sim.ctx, sim.n)
        st = sim.state()
    finally:
        sim.close()
    dt = np.float32 if prec == 32 else np.float64
    off = 0
    for (L, _, nx, n) in RAGGED:
        ref = O.element_key(st["Q"][off:off + n], L, nx, dt)
        assert np.array_equal(keys[off:off + n], ref)
        off += n


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("decorated", [True, False])
def test_stable_sort_bit_exact(prec, decorated):
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    runs = RAGGED + [(5.0, 0.1, 8, 70000)]          # a run spanning several sort chunks
    states, cat = _rand_runs(runs, seed=2, decorated=decorated)
    # a nearly sorted run with long equal-key stretches
    L, _, nx, n = runs[-1]
    q = np.sort(cat["Q"][-n:]) % L
    cat["Q"][-n:] = q
    sim = _sim(runs, prec, decorated=decorated)
    try:
        sim.init_particles(cat)
        before = sim.state()
        swpic.swpic_sort(sim.ctx)
        after = sim.state()
    finally:
        sim.close()
    dt = np.float32 if prec == 32 else np.float64
    off = 0
    for (L, _, nx, n) in runs:
        sl = slice(off, off + n)
        keys = O.element_key(before["Q"][sl], L, nx, dt)
        order = O.stable_sort_order(keys)
        for k in ("Q", "P", "qs", "ps", "psi"):
            if before[k] is None:
                continue
            assert np.array_equal(after[k][sl], before[k][sl][order]), k
        off += n


# ---------------------------------------------------------------------------
# a3 + a4 deposit and neutralisation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("decorated", [True, False])
def test_deposit_matches_oracle(prec, mode, decorated):
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    states, cat = _rand_runs(RAGGED, seed=3, decorated=decorated)
    sim = _sim(RAGGED, prec, deposit_mode=mode, decorated=decorated)
    try:
        sim.init_particles(cat)
        st = sim.state()
        swpic.swpic_deposit(sim.ctx)
        meshes = [sim.mesh(r) for r in range(len(RAGGED))]
    finally:
        sim.close()
    dt = np.float32 if prec == 32 else np.float64
    tol = 1e-5 if prec == 32 else 1e-12
    off = 0
    for r, (L, _, nx, n) in enumerate(RAGGED):
        sl = slice(off, off + n)
        elem = O.element_key(st["Q"][sl], L, nx, dt)
        ps = st["ps"][sl] if decorated else None
        ref = O.deposit(st["Q"][sl], ps, st["psi"][sl], L, nx, elem=elem)
        assert rel_max(meshes[r]["b"], ref) <= tol, r
        bt = ref - ref.mean()
        assert np.abs(meshes[r]["btilde"] - bt).max() <= tol * np.abs(ref).max()
        assert abs(meshes[r]["btilde"].sum()) <= 1e-12 * np.abs(ref).sum() * nx
        off += n


def test_deterministic_deposit_is_bitwise_reproducible():
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    specs = [(4 * np.pi, 0.05, 512, 300001)]
    _, cat = _rand_runs(specs, seed=4)
    out = []
    for rep in range(2):
        sim = _sim(specs, 32, deposit_mode=1)
        try:
            sim.init_particles(cat)
            swpic.swpic_deposit(sim.ctx)
            out.append(sim.mesh(0)["b"])
        finally:
            sim.close()
    assert np.array_equal(out[0], out[1])


# ---------------------------------------------------------------------------
# a5 solve and field tables
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("d2_mode", [0, 2])
def test_solve_and_tables_match_oracle_fp64(d2_mode):
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    specs = [(4 * np.pi, 0.1, 64, 5000), (7.3, 0.1, 1024, 20001), (2.0, 0.1, 4096, 9000)]
    _, cat = _rand_runs(specs, seed=5)
    sim = _sim(specs, 64, d2_mode=d2_mode)
    try:
        sim.init_particles(cat)
        st = sim.state()
        swpic.swpic_deposit(sim.ctx)
        swpic.swpic_solve_field(sim.ctx)
        meshes = [sim.mesh(r) for r in range(len(specs))]
    finally:
        sim.close()
    off = 0
    for r, (L, _, nx, n) in enumerate(specs):
        sl = slice(off, off + n)
        f = O.field_of_state(st["Q"][sl], st["ps"][sl], st["psi"][sl], L, nx, d2_mode=d2_mode)
        m = meshes[r]
        assert rel_max(m["Phi"], f["Phi"]) < 1e-12
        assert rel_max(-m["E"], f["dphi"]) < 1e-12
        assert rel_max(m["d2"], f["d2"]) < 1e-11
        off += n


def test_solve_matches_thm1_single_particle():
    """One decorated source: the device potential equals the nodal values of
    the closed form (Eq. solution) for the monopole and the explicit P1
    dipole solution (proof of Thm 2), up to the gauge constant."""
    need_gpu()
    from workloads import physics as ph
    from paper_2605_21794_gb300 import swpic
    L, nx, Q, psi, ps = 5.0, 40, 1.2345, 0.8, 0.0
    sim = _sim([(L, 0.1, nx, 1)], 64)
    try:
        sim.init_particles({"Q": np.array([Q]), "P": np.zeros(1), "qs": np.zeros(1),
                            "ps": np.array([ps]), "psi": np.array([psi])})
        swpic.swpic_deposit(sim.ctx)
        swpic.swpic_solve_field(sim.ctx)
        Phi = sim.mesh(0)["Phi"]
    finally:
        sim.close()
    ref = ph.thm1_phi(np.arange(nx) * L / nx, Q, psi, 0.0, L)
    ref -= ref.mean()
    assert np.abs(Phi - ref).max() < 1e-12 * np.abs(ref).max()
    sim = _sim([(L, 0.1, nx, 1)], 64)
    try:
        sim.init_particles({"Q": np.array([Q]), "P": np.zeros(1), "qs": np.zeros(1),
                            "ps": np.array([-0.6]), "psi": np.array([1e-300])})
        swpic.swpic_deposit(sim.ctx)
        swpic.swpic_solve_field(sim.ctx)
        Phi = sim.mesh(0)["Phi"]
    finally:
        sim.close()
    assert np.abs(Phi - ph.dipole_galerkin_nodes(Q, -0.6, L, nx)).max() < 1e-12


# ---------------------------------------------------------------------------
# a6 gather + kick + drift
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d2_mode", [0, 2])
def test_gather_push_matches_oracle(prec, d2_mode):
    need_gpu()
    from paper_2605_21794_gb300 import swpic
    specs = [(4 * np.pi, 0.1, 64, 4099), (7.3, 0.05, 256, 30001)]
    _, cat = _rand_runs(specs, seed=6)
    sim = _sim(specs, prec, d2_mode=d2_mode)
    try:
        sim.init_particles(cat)
        st0 = sim.state()
        meshes = [sim.mesh(r) for r in range(len(specs))]
        swpic.swpic_gather_push(sim.ctx, 0.5, 1.0)
        st1 = sim.state()
    finally:
        sim.close()
    dt_ = np.float32 if prec == 32 else np.float64
    tol = 2e-6 if prec == 32 else 1e-13
    off = 0
    for r, (L, dt, nx, n) in enumerate(specs):
        sl = slice(off, off + n)
        s = {k: st0[k][sl].copy() for k in st0}
        elem = O.element_key(s["Q"], L, nx, dt_)
        # the oracle's own field of the same stored state (Eq. rhs-assembly with
        # the elements decided in the state's precision, the Galerkin solve, the
        # tables), rounded to the storage precision of the step's tables
        b = O.deposit(s["Q"], s["ps"], s["psi"], L, nx, elem=elem)
        Phi, lam = O.solve(b, L)
        dphi, d2 = O.field_tables(Phi, L, d2_mode, btilde=b - lam)
        dphi = dphi.astype(dt_).astype(np.float64)
        d2 = d2.astype(dt_).astype(np.float64)
        # the FP32 deposit forms its node weights in FP32 (the deposit tolerance)
        assert rel_max(-meshes[r]["E"], dphi) <= (1e-5 if prec == 32 else 1e-12)
        dV, d2V = O.gather(s["Q"], L, dphi, d2, d2_mode=d2_mode, elem=elem)
        O.kick_values(s["ps"], s["P"], s["qs"], dV, d2V, 0.5 * dt)
        O.drift(s["Q"], s["P"], s["qs"], s["ps"], L, dt)
        assert np.abs(periodic_diff(st1["Q"][sl], s["Q"], L)).max() <= tol * L
        for k in ("P", "qs", "ps"):
            assert rel_max(st1[k][sl], s[k]) <= tol * 4, k
        off += n


# ---------------------------------------------------------------------------
# initialisation on the lattice (reading A6) and diagnostics
# ---------------------------------------------------------------------------
LATTICES = [
    W.landau_linear(jitter=1e-3).lattice,
    W.two_stream().lattice,
    W.LatticeSpec(96, 80, 4 * np.pi, -6.0, 6.0, 0.5, 0.5, W.MAXWELL, jitter=0.25, seed=0),
    W.LatticeSpec(64, 128, 20 * np.pi / 3, -8.0, 10.0, 0.04, 0.3,
                  W.bump_on_tail().lattice.terms),
]


@pytest.mark.parametrize("idx", range(len(LATTICES)))
def test_init_lattice_matches_oracle_fp64(idx):
    need_gpu()
    lat = LATTICES[idx]
    jx, jv = W.jitter(lat)
    ref = O.init_lattice(lat, jx, jv)
    sim = _sim([(lat.L, 0.1, 64, lat.n)], 64)
    try:
        sim.init_lattice(0, lat, jx, jv)
        st = sim.state()
    finally:
        sim.close()
    assert np.abs(periodic_diff(st["Q"], ref["Q"], lat.L)).max() < 1e-14 * lat.L
    assert rel_max(st["P"], ref["P"]) < 1e-15
    assert rel_max(st["psi"], ref["psi"]) < 1e-14
    assert rel_max(st["ps"], ref["ps"]) < 1e-10
    assert rel_max(st["qs"], ref["qs"]) < 1e-10


@pytest.mark.parametrize("prec", PRECS)
def test_initial_diagnostics_match_oracle(prec):
    need_gpu()
    specs = [(4 * np.pi, 0.1, 64, 5003), (5.0, 0.1, 32, 777)]
    _, cat = _rand_runs(specs, seed=8)
    sim = _sim(specs, prec)
    try:
        sim.init_particles(cat)
        st = sim.state()
        d = [sim.diagnostics(r) for r in range(len(specs))]
    finally:
        sim.close()
    tol = 1e-12 if prec == 64 else 2e-6
    off = 0
    for r, (L, dt, nx, n) in enumerate(specs):
        sl = slice(off, off + n)
        f = O.field_of_state(st["Q"][sl], st["ps"][sl], st["psi"][sl], L, nx)
        ref = O.diagnostics(st["P"][sl], st["qs"][sl], st["psi"][sl], f["Phi"], L)
        rec = d[r][0]
        assert rec[0] == 0.0 and rec[7] == 0
        assert abs(rec[1] - ref["mass"]) <= 1e-14 * ref["mass"]
        assert abs(rec[2] - ref["momentum"]) <= tol * ref["mass"] * 3
        assert abs(rec[3] - ref["kinetic"]) <= tol * abs(ref["kinetic"])
        assert abs(rec[4] - ref["field"]) <= (1e-11 if prec == 64 else 2e-5) * ref["field"]
        assert abs(rec[6] - ref["E_amp"]) <= (1e-11 if prec == 64 else 2e-5) * ref["E_amp"]
        off += n
