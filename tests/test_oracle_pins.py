"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form printed in the paper (Thm 1, the explicit P1 dipole solution in the proof
of Thm 2), an independent computation (brute-force hat evaluation, a DFT
eigen-solve, numpy's Gauss-Legendre rule, numerical differentiation of the
discrete Hamiltonian), an exact discrete map (leapfrog on a quadratic
potential), an invariant (charge, time reversibility, mass), or a physical
root (kinetic dispersion relation).  A plausible slip in the oracle (a sign
of the dipole term, an index shift in the stiffness matrix, a transposed
kick/drift) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from workloads import physics as ph
import workloads as W


def rng_state(n, L, nx, seed, decorated=True):
    return W.random_state(n, L, seed=seed, decorated=decorated, nx=nx)


# ---------------------------------------------------------------------------
# generators
# ---------------------------------------------------------------------------
def test_splitmix64_published_vectors():
    # SplitMix64 reference outputs (Steele-Lea-Flood / Vigna) for seeds 0 and 1234567
    assert [int(x) for x in W.splitmix64(0, 0, 5)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
        0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [int(x) for x in W.splitmix64(1234567, 0, 3)] == [
        0x599ED017FB08FC85, 0x2C73F08458540FA5, 0x883EBCE5A3F27C77]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, rtol=0, atol=1e-14)
    assert np.allclose(w, wr, rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# deposit (Eq. rhs-assembly)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,nx,seed", [(1, 4, 1), (7, 5, 2), (33, 16, 3), (64, 9, 4), (0, 8, 5)])
@pytest.mark.parametrize("decorated", [True, False])
def test_deposit_matches_bruteforce(n, nx, seed, decorated):
    L = 2.0 + seed
    s = rng_state(n, L, nx, seed, decorated)
    b = O.deposit(s["Q"], s["ps"], s["psi"], L, nx)
    bb = O.deposit_bruteforce(s["Q"], s["ps"], s["psi"], L, nx)
    scale = max(np.abs(bb).max(), 1e-300) if n else 1.0
    assert np.abs(b - bb).max() <= 1e-14 * scale
    assert np.allclose(b.sum(), s["psi"].sum(), rtol=1e-13, atol=1e-300)   # dipoles carry no net charge


def test_deposit_dipole_is_derivative_of_monopole():
    """p* delta'(q - Q) is the limit of two opposite charges (Eq. rho): the
    dipole part of the deposit equals -p* d/dQ of a unit monopole deposit."""
    L, nx = 3.0, 12
    Q0 = np.array([0.7312, 2.2501, 1.1234])
    ps = np.array([0.3, -0.7, 1.1])
    zero = np.zeros(3)
    b_dip = O.deposit(Q0, ps, zero, L, nx)
    eps = 1e-6
    fd = np.zeros(nx)
    for a in range(3):
        one = np.zeros(3); one[a] = 1.0
        bp = O.deposit(Q0 + eps * one, zero, one, L, nx)
        bm = O.deposit(Q0 - eps * one, zero, one, L, nx)
        fd += -ps[a] * (bp - bm) / (2 * eps)
    assert np.allclose(b_dip, fd, rtol=0, atol=1e-8)


def test_deposit_shift_by_one_element_rolls_mesh():
    L, nx = 8.0, 16          # h = 0.5 so Q + h is exact
    s = rng_state(50, L, nx, 7)
    h = L / nx
    b0 = O.deposit(s["Q"], s["ps"], s["psi"], L, nx)
    Q1 = np.mod(s["Q"] + h, L)
    b1 = O.deposit(Q1, s["ps"], s["psi"], L, nx)
    assert np.allclose(b1, np.roll(b0, 1), rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------
# Galerkin Poisson solve (Eq. lin-sys) and Thm 1 / Thm 2
# ---------------------------------------------------------------------------
def test_stiffness_is_circulant_laplacian():
    nx, L = 10, 5.0
    A = O.stiffness(nx, L)
    h = L / nx
    ref = (2 * np.eye(nx) - np.roll(np.eye(nx), 1, 1) - np.roll(np.eye(nx), -1, 1)) / h
    assert np.allclose(A, ref, atol=1e-14)
    assert np.allclose(A @ np.ones(nx), 0, atol=1e-13)        # kernel = constants


@pytest.mark.parametrize("nx", [4, 17, 64, 256])
def test_solve_matches_dft_eigensolve(nx):
    L = 7.3
    h = L / nx
    rng = W.uniform01(11, 0, nx)
    b = rng - 0.2
    Phi, lam = O.solve(b, L)
    assert abs(lam - b.mean()) < 1e-13
    bt = b - b.mean()
    m = np.arange(nx)
    eig = 4.0 * np.sin(np.pi * m / nx) ** 2 / h
    bh = np.fft.fft(bt)
    ph_ = np.zeros(nx, dtype=complex)
    ph_[1:] = bh[1:] / eig[1:]
    ref = np.fft.ifft(ph_).real
    assert np.abs(Phi - ref).max() <= 1e-11 * np.abs(ref).max()
    assert abs(Phi.sum()) < 1e-11 * np.abs(ref).max() * nx


@pytest.mark.parametrize("Q,nx", [(1.234, 16), (0.01, 8), (4.9, 32), (2.5 + 1e-7, 10)])
def test_monopole_galerkin_is_nodally_exact_thm1(Q, nx):
    """1D P1 Galerkin is nodally exact for the continuous monopole solution of
    Eq. (solution): Phi_j = phi(q_j) up to the constant fixed by the gauge."""
    L, psi = 5.0, 0.8
    b = O.deposit(np.array([Q]), np.array([0.0]), np.array([psi]), L, nx)
    Phi, _ = O.solve(b, L)
    q = np.arange(nx) * L / nx
    ref = ph.thm1_phi(q, Q, psi, 0.0, L)
    ref -= ref.mean()
    assert np.abs(Phi - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("Q,nx", [(1.234, 16), (0.37, 8), (4.9, 32), (2.6, 10)])
def test_dipole_galerkin_matches_thm2_explicit_solution(Q, nx):
    L, ps = 5.0, -0.6
    h = L / nx
    b = O.deposit(np.array([Q]), np.array([ps]), np.array([0.0]), L, nx)
    Phi, _ = O.solve(b, L)
    ref = ph.dipole_galerkin_nodes(Q, ps, L, nx)
    assert np.abs(Phi - ref).max() <= 1e-12 * abs(ps)
    # eta = phi_D - phi_h^D is the constant C0 = p*(b - a)/(2L) at every node
    iQ = int(Q // h)
    a_, b_ = Q - iQ * h, (iQ + 1) * h - Q
    C0 = ps * (b_ - a_) / (2 * L)
    q = np.arange(nx) * h
    assert np.abs(ph.thm1_phi(q, Q, 0.0, ps, L) - Phi - C0).max() <= 1e-12


def test_thm1_closed_form_jumps_and_equation():
    L, Q, psi, ps = 6.0, 2.2, 0.9, -0.4
    e = 1e-7
    f = lambda q: ph.thm1_phi(np.array([q]), Q, psi, ps, L)[0]
    assert abs((f(Q + e) - f(Q - e)) - (-ps)) < 1e-6                       # [phi]_Q = -p*
    d = lambda q: (f(q + 1e-5) - f(q - 1e-5)) / 2e-5
    assert abs((d(Q + 1e-3) - d(Q - 1e-3)) - (-psi)) < 1e-3                 # [phi']_Q = -psi*
    q0, hh = 4.1, 1e-3                                                       # -phi'' = -n0 away from Q
    sec = (f(q0 + hh) - 2 * f(q0) + f(q0 - hh)) / hh ** 2
    assert abs(sec - psi / L) < 1e-5
    qq = np.linspace(0, L, 200001)[:-1]
    assert abs(ph.thm1_phi(qq, Q, psi, ps, L).mean()) < 1e-5                # zero mean


def test_thm2_dipole_l2_rate_is_half():
    """||phi_D - phi_h^D||_L2 = O(h^{1/2}) (Thm 2), with Q at a fixed relative
    position in its element so the constant is the same at every level."""
    L, ps = 4.0, 1.0
    errs, hs = [], []
    for nx in (16, 32, 64, 128, 256, 512):
        h = L / nx
        Q = (nx // 3 + 0.3) * h
        b = O.deposit(np.array([Q]), np.array([ps]), np.array([0.0]), L, nx)
        Phi, _ = O.solve(b, L)
        # integrate (phi - phi_h)^2 with many sub-points per element
        sub = 64
        qq = (np.arange(nx * sub) + 0.5) * (h / sub)
        ph_h = np.interp(qq, np.arange(nx + 1) * h, np.append(Phi, Phi[0]))
        err = np.sqrt(np.sum((ph.thm1_phi(qq, Q, 0.0, ps, L) - ph_h) ** 2) * h / sub)
        errs.append(err); hs.append(h)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 0.45 < slope < 0.55


# ---------------------------------------------------------------------------
# field tables (phi_h' from the basis, phi_h'' by projection; reading A1)
# ---------------------------------------------------------------------------
def test_dphi_is_element_slope():
    L, nx = 3.0, 12
    Phi = W.uniform01(3, 0, nx)
    dphi, _ = O.field_tables(Phi, L)
    h = L / nx
    assert np.allclose(dphi, (np.roll(Phi, -1) - Phi) / h, atol=1e-13)


@pytest.mark.parametrize("mode", [O.D2_LUMPED, O.D2_CONSISTENT])
def test_d2_projection_converges_second_order(mode):
    L = 2 * np.pi
    errs = []
    for nx in (32, 64, 128):
        h = L / nx
        q = np.arange(nx) * h
        _, d2 = O.field_tables(np.cos(q), L, mode)
        mid = (np.arange(nx) + 0.5) * h
        errs.append(np.abs(d2 + np.cos(mid)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_d2_lumped_exact_for_quadratic_interior():
    L, nx = 10.0, 20
    h = L / nx
    q = np.arange(nx) * h
    _, d2 = O.field_tables(3.0 * q ** 2, L, O.D2_LUMPED)
    assert np.allclose(d2[1:nx - 2], 6.0, atol=1e-10)


def test_d2_nodal_converges_second_order_to_phi_second_derivative():
    """NODAL (reading A1): the nodal phi'' is the lumped projection -btilde/h of
    the distributional phi_h'' of the P1 field.  For Phi_j = cos(q_j) and the
    charge that produces it, btilde = A Phi (the stiffness matrix), the nodal
    values converge at second order to phi'' = -cos at the nodes."""
    L = 2 * np.pi
    errs = []
    for nx in (32, 64, 128):
        h = L / nx
        q = np.arange(nx) * h
        Phi = np.cos(q)
        bt = O.stiffness(nx, L) @ Phi
        _, d2 = O.field_tables(Phi, L, O.D2_NODAL, btilde=bt)
        errs.append(np.abs(d2 + np.cos(q)).max())
    assert errs[2] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_nodal_gather_is_periodic_linear_interpolation():
    """The nodal branch of the gather interpolates the nodal phi'' linearly
    inside each element, periodically across x = L (checked against numpy's
    periodic interpolation), and reads phi_h' as the element slope."""
    L, nx = 7.0, 11
    h = L / nx
    s = W.uniform01(21, 0, nx) - 0.5
    dphi = W.uniform01(21, 1, nx)
    Q = np.concatenate([W.uniform01(21, 2, 400) * L, np.arange(nx) * h, [L - 1e-12]])
    dV, d2V = O.gather(Q, L, dphi, s, d2_mode=O.D2_NODAL)
    ref = np.interp(Q, np.arange(nx) * h, s, period=L)
    assert np.abs(d2V - ref).max() < 1e-12
    assert np.array_equal(dV, dphi[O.element(Q, L, nx)])


def test_nodal_gather_of_a_smooth_field_is_second_order_at_particles():
    """Whole NODAL chain at arbitrary particle positions: Phi = cos sampled on
    the nodes, btilde = A Phi, table, gather -> phi''(Q) = -cos Q + O(h^2)."""
    L = 2 * np.pi
    Q = W.uniform01(5, 0, 1000) * L
    errs = []
    for nx in (32, 64, 128):
        h = L / nx
        Phi = np.cos(np.arange(nx) * h)
        bt = O.stiffness(nx, L) @ Phi
        dphi, d2 = O.field_tables(Phi, L, O.D2_NODAL, btilde=bt)
        _, d2V = O.gather(Q, L, dphi, d2, d2_mode=O.D2_NODAL)
        errs.append(np.abs(d2V + np.cos(Q)).max())
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7


def test_d2_nodal_is_minus_neutral_charge_density():
    L, nx = 4.0, 8
    h = L / nx
    bt = W.uniform01(9, 0, nx) - 0.5
    bt -= bt.mean()
    _, d2 = O.field_tables(np.zeros(nx), L, O.D2_NODAL, btilde=bt)
    assert np.allclose(d2, -bt / h, atol=1e-15)


# ---------------------------------------------------------------------------
# Hamilton's equations from H_h and the bracket (Eq. lp1d, App. B)
# ---------------------------------------------------------------------------
def _H(st, L, nx):
    f = O.field_of_state(st["Q"], st["ps"], st["psi"], L, nx)
    kin = np.sum(0.5 * st["psi"] * st["P"] ** 2 + st["qs"] * st["P"])
    A = O.stiffness(nx, L)
    return kin + 0.5 * f["Phi"] @ A @ f["Phi"], f


def test_hamilton_equations_by_numerical_differentiation():
    """Q' = dH/dq*, P' = dH/dp*, p*' = -dH/dP + psi* dH/dq*; for P1 inside
    an element dH/dQ + psi* dH/dp* = 0 (exact phi_h'' vanishes there)."""
    L, nx, n = 5.0, 16, 24
    st = rng_state(n, L, nx, 21)
    H0, f = _H(st, L, nx)
    dV, _ = O.gather(st["Q"], L, f["dphi"], f["d2"])
    for a in range(0, n, 5):
        grads = {}
        for key, eps in (("Q", 1e-7), ("P", 1e-6), ("qs", 1e-6), ("ps", 1e-6)):
            sp = {k: v.copy() for k, v in st.items()}
            sm = {k: v.copy() for k, v in st.items()}
            sp[key][a] += eps
            sm[key][a] -= eps
            grads[key] = (_H(sp, L, nx)[0] - _H(sm, L, nx)[0]) / (2 * eps)
        psi = st["psi"][a]
        assert abs(grads["qs"] - st["P"][a]) < 1e-7                         # Q' = P
        assert abs(grads["ps"] - (-dV[a])) < 1e-6 * max(1, abs(dV[a]))     # P' = -phi_h'(Q)
        pdot = -grads["P"] + psi * grads["qs"]
        assert abs(pdot - (-st["qs"][a])) < 1e-7                            # p*' = -q*
        assert abs(grads["Q"] - psi * dV[a]) < 1e-6 * max(1, abs(dV[a]))    # dW/dQ = psi* phi_h'


# ---------------------------------------------------------------------------
# integrator (leapfrog) on prescribed potentials (Sec. 3.3 / Sec. 7.1)
# ---------------------------------------------------------------------------
def _kdk_prescribed(st, dVf, d2Vf, L, dt, n):
    for _ in range(n):
        O.kick_values(st["ps"], st["P"], st["qs"], dVf(st["Q"]), d2Vf(st["Q"]), 0.5 * dt)
        O.drift(st["Q"], st["P"], st["qs"], st["ps"], L, dt)
        O.kick_values(st["ps"], st["P"], st["qs"], dVf(st["Q"]), d2Vf(st["Q"]), 0.5 * dt)
    return st


def test_leapfrog_harmonic_matches_exact_discrete_map():
    L, q0, om, dt, n = 1000.0, 500.0, 1.3, 0.07, 400
    st = {"Q": np.array([500.3, 499.1]), "P": np.array([0.2, -0.5]),
          "qs": np.array([0.01, -0.02]), "ps": np.array([0.03, 0.05]), "psi": np.ones(2)}
    x0 = st["Q"] - q0; v0 = st["P"].copy(); ps0 = st["ps"].copy(); qs0 = st["qs"].copy()
    _kdk_prescribed(st, lambda Q: om ** 2 * (Q - q0), lambda Q: om ** 2 * np.ones_like(Q),
                    L, dt, n)
    c = om ** 2 * dt
    M = np.array([[1 - c * dt / 2, dt], [-c * (1 - c * dt / 4), 1 - c * dt / 2]])
    Mn = np.linalg.matrix_power(M, n)
    x, v = Mn @ np.vstack([x0, v0])
    assert np.allclose(st["Q"] - q0, x, atol=1e-12) and np.allclose(st["P"], v, atol=1e-12)
    # (p*, -q*) obeys the same linear map: p* plays x, -q* plays v
    y, w = Mn @ np.vstack([ps0, -qs0])
    assert np.allclose(st["ps"], y, atol=1e-13) and np.allclose(-st["qs"], w, atol=1e-13)


def test_decoration_converges_to_continuous_closed_form():
    """V'' = w^2: p*(t) = p*0 cos wt - (q*0/w) sin wt, q*(t) = q*0 cos wt + w p*0 sin wt
    (Eq. sw_prescribed_potential); leapfrog error is O(dt^2)."""
    om, T = 0.9, 5.0
    ps0, qs0 = 0.4, -0.3
    errs = []
    for dt in (0.05, 0.025, 0.0125):
        st = {"Q": np.array([1.0]), "P": np.array([0.0]), "qs": np.array([qs0]),
              "ps": np.array([ps0]), "psi": np.ones(1)}
        _kdk_prescribed(st, lambda Q: np.zeros_like(Q), lambda Q: om ** 2 * np.ones_like(Q),
                        1e9, dt, int(round(T / dt)))
        pe = ps0 * np.cos(om * T) - qs0 / om * np.sin(om * T)
        qe = qs0 * np.cos(om * T) + om * ps0 * np.sin(om * T)
        errs.append(max(abs(st["ps"][0] - pe), abs(st["qs"][0] - qe)))
    assert 3.7 < errs[0] / errs[1] < 4.3 and 3.7 < errs[1] / errs[2] < 4.3


def test_uniform_field_decoration_is_exact():
    st = {"Q": np.array([0.5]), "P": np.array([0.1]), "qs": np.array([0.25]),
          "ps": np.array([-0.125]), "psi": np.ones(1)}
    dt, n = 0.125, 64
    _kdk_prescribed(st, lambda Q: 0.5 * np.ones_like(Q), lambda Q: np.zeros_like(Q), 1e6, dt, n)
    assert st["qs"][0] == 0.25
    assert abs(st["ps"][0] - (-0.125 - 0.25 * dt * n)) < 1e-14
    assert abs(st["P"][0] - (0.1 - 0.5 * dt * n)) < 1e-13


def test_test_particle_energy_bounded_second_order():
    """Sec. 7.1: V = 1 - cos(kappa q), L = 10; H_SWPIC per particle has a
    bounded O(dt^2) error and no drift over long times."""
    L = 10.0
    kap = 2 * np.pi / L
    dV = lambda Q: kap * np.sin(kap * Q)
    d2V = lambda Q: kap ** 2 * np.cos(kap * Q)

    def H(s):
        return (0.5 * s["psi"] * s["P"] ** 2 + s["P"] * s["qs"] + s["psi"] * (1 - np.cos(kap * s["Q"]))
                - s["ps"] * kap * np.sin(kap * s["Q"]))
    devs = []
    for dt in (0.1, 0.05):
        # two trapped orbits and one passing orbit, away from the separatrix
        st = {"Q": np.array([1.0, 9.5, 2.0]), "P": np.array([0.3, -0.2, 2.2]),
              "qs": np.array([0.02, -0.05, 0.01]), "ps": np.array([0.05, 0.02, -0.03]),
              "psi": np.array([1.0, 0.7, 1.3])}
        H0 = H(st)
        dev = np.zeros(3)
        n_out = 50
        for _ in range(n_out):
            _kdk_prescribed(st, dV, d2V, L, dt, int(round(2.0 / dt)))
            dev = np.maximum(dev, np.abs(H(st) - H0))
        devs.append(dev.max())
    assert devs[0] < 5e-3
    assert 3.7 < devs[0] / devs[1] < 4.3


# ---------------------------------------------------------------------------
# whole runs: invariants, reversibility, physics
# ---------------------------------------------------------------------------
def test_reversibility_of_the_step():
    spec = W.landau_linear(jitter=1e-3)
    jx, jv = W.jitter(spec.lattice)
    st = O.init_lattice(spec.lattice, jx, jv)
    L = spec.lattice.L
    r1 = O.run(st, spec.nx, L, spec.dt, 50, diag_every=0)
    back = dict(r1, P=-r1["P"], qs=-r1["qs"])
    r2 = O.run(back, spec.nx, L, spec.dt, 50, diag_every=0)
    dQ = np.abs(np.mod(r2["Q"] - st["Q"] + L / 2, L) - L / 2)
    assert dQ.max() < 1e-11 * L
    assert np.abs(-r2["P"] - st["P"]).max() < 1e-11 * np.abs(st["P"]).max()
    assert np.abs(-r2["qs"] - st["qs"]).max() < 1e-10 * np.abs(st["qs"]).max()
    assert np.abs(r2["ps"] - st["ps"]).max() < 1e-10 * np.abs(st["ps"]).max()


def test_mass_is_bit_constant_and_neutral_mesh():
    spec = W.landau_linear(jitter=1e-3)
    jx, jv = W.jitter(spec.lattice)
    st = O.init_lattice(spec.lattice, jx, jv)
    r = O.run(st, spec.nx, spec.lattice.L, spec.dt, 40, diag_every=10)
    assert np.array_equal(r["psi"], st["psi"])
    assert np.all(r["diag"][:, 1] == r["diag"][0, 1])
    f = O.field_of_state(r["Q"], r["ps"], r["psi"], spec.lattice.L, spec.nx)
    assert abs(f["btilde"].sum()) < 1e-13 * np.abs(f["b"]).sum()


def test_landau_rate_and_frequency_resolved_lattice():
    """k = 0.5 Maxwellian (alpha 0.01): the E_amp history fitted over t in
    [2, 20] on a resolved 256 x 256 lattice (nx 64, dt 0.1) gives gamma and
    omega within 1% of the dispersion root (omega 1.41566, gamma -0.15336)."""
    import dataclasses
    base = W.landau_linear()
    lat = dataclasses.replace(base.lattice, nq=256, nv=256)
    st = O.init_lattice(lat)
    r = O.run(st, 64, lat.L, 0.1, 200, diag_every=1)
    root = ph.landau_root(0.5)
    g, om, tm = ph.rate_fit(r["diag"][:, 0], r["diag"][:, 6], 2.0, 20.0, min_sep=1.5)
    assert abs(g / root.imag - 1) < 0.01
    assert abs(om / root.real - 1) < 0.01


@pytest.mark.parametrize("k", [0.35, 0.45, 0.55])
def test_landau_rates_across_k_resolved_lattice(k):
    """Linear Landau damping (alpha 0.01) at the wavenumbers of the ensemble,
    L = 2 pi/k, 256^2 lattice on v in [-6, 6], nx 128, dt 0.1: the damping
    rate fitted over the maxima in t in [2, t1], t1 = min(0.8 T_R, 2/|gamma|,
    40) (T_R = 2 pi/(k dv) the lattice recurrence), is within 1% of the kinetic
    dispersion root, and the frequency within 0.5%."""
    L = 2 * math.pi / k
    root = ph.landau_root(k, 1.0 + 0.5 * k - 0.1j)
    lat = W.LatticeSpec(256, 256, L, -6.0, 6.0, 0.01, k, W.MAXWELL)
    t_rec = 2 * math.pi / (k * 12.0 / 256)
    t1 = max(12.0, min(0.8 * t_rec, 2 / abs(root.imag), 40.0))
    r = O.run(O.init_lattice(lat), 128, L, 0.1, int(round((t1 + 2) / 0.1)), diag_every=1)
    g, om, _ = ph.rate_fit(r["diag"][:, 0], r["diag"][:, 6], 2.0, t1, min_sep=1.2)
    assert abs(g / root.imag - 1) < 0.01, (g, root)
    assert abs(om / root.real - 1) < 0.005, (om, root)


def test_energy_error_shrinks_with_lattice_resolution():
    """H_h (Eq. Hh) drifts only through the projected phi'' (reading A1),
    whose effect scales with the decoration size ~ (cell size)^2."""
    import dataclasses
    base = W.landau_linear()
    drifts = []
    for side in (128, 256):
        lat = dataclasses.replace(base.lattice, nq=side, nv=side)
        r = O.run(O.init_lattice(lat), 64, lat.L, 0.1, 300, diag_every=5)
        H = r["diag"][:, 5]
        drifts.append(np.abs(H - H[0]).max() / abs(H[0]))
    assert drifts[1] < 1e-4
    assert drifts[0] / drifts[1] > 4.0


# ---------------------------------------------------------------------------
# initialisation on the lattice (reading A6 of Sec. 4.2 / Alg. 1)
# ---------------------------------------------------------------------------
def test_init_lattice_moments_closed_form_uniform_in_x():
    """alpha = 0: f0 = M(v). Then p* = [int M over the v-cell] * int_cell c(Q,q) dq
    and q* = int_cell dq * int M(p)(p - P) dp, both with closed forms."""
    from scipy.special import erf
    lat = W.LatticeSpec(8, 24, 5.0, -3.0, 3.0, 0.0, 1.0, W.MAXWELL, jitter=0.3, seed=4)
    jx, jv = W.jitter(lat)
    st = O.init_lattice(lat, jx, jv)
    dx, dv = lat.L / lat.nq, (lat.vmax - lat.vmin) / lat.nv
    x, v = W.lattice_points(lat)
    L = lat.L
    Q = st["Q"]; P = st["P"]
    Phi = lambda z: 0.5 * (1 + erf(z / np.sqrt(2)))
    Mv = Phi(v + dv / 2) - Phi(v - dv / 2)
    kk = 2 * np.pi / L
    # int_{x-dx/2}^{x+dx/2} (L/2pi) sin(kk (Q - q)) dq = (1/kk^2)[cos(kk(Q - q))]
    cint = (np.cos(kk * (Q - (x + dx / 2))) - np.cos(kk * (Q - (x - dx / 2)))) / kk ** 2
    assert np.abs(st["ps"] - Mv * cint).max() <= 1e-9 * np.abs(Mv * cint).max()
    Mp = lambda z: np.exp(-z * z / 2) / np.sqrt(2 * np.pi)
    first = -(Mp(v + dv / 2) - Mp(v - dv / 2))          # int M(p) p dp
    qref = dx * (first - P * Mv)
    assert np.abs(st["qs"] - qref).max() <= 1e-9 * np.abs(qref).max()
    assert np.allclose(st["psi"], Mp(v) * dx * dv, rtol=1e-15)
    # on a fine lattice a particle jittered by delta cells in x carries
    # p* ~ psi* delta dx (consequence of reading A6), to O(cell^2)
    fine = W.LatticeSpec(40, 60, 5.0, -3.0, 3.0, 0.0, 1.0, W.MAXWELL, jitter=0.3, seed=4)
    fx, fv = W.jitter(fine)
    sf = O.init_lattice(fine, fx, fv)
    approx = sf["psi"] * fx * (fine.L / fine.nq)
    assert np.abs(sf["ps"] - approx).max() < 2e-2 * np.abs(approx).max()


def test_init_lattice_order_and_wrap():
    lat = W.LatticeSpec(4, 3, 2.0, -1.0, 2.0, 0.1, np.pi, W.MAXWELL, jitter=0.5, seed=9)
    jx, jv = W.jitter(lat)
    st = O.init_lattice(lat, jx, jv)
    x, v = W.lattice_points(lat)
    dx, dv = 0.5, 1.0
    assert np.all((st["Q"] >= 0) & (st["Q"] < lat.L))
    assert np.allclose(np.mod(x + jx * dx, lat.L), st["Q"], atol=1e-15)
    assert np.allclose(v + jv * dv, st["P"], atol=1e-15)


def test_field_energy_equals_half_integral_of_E_squared():
    """W = (1/2) Phi^T A Phi (Eq. Hh) equals (1/2) int E^2 = (L/2) E_amp^2
    (Eq. Eamp) for the piecewise-constant P1 field."""
    L, nx = 6.0, 24
    s = rng_state(300, L, nx, 31)
    f = O.field_of_state(s["Q"], s["ps"], s["psi"], L, nx)
    d = O.diagnostics(s["P"], s["qs"], s["psi"], f["Phi"], L)
    assert abs(d["field"] - 0.5 * L * d["E_amp"] ** 2) < 1e-13 * d["field"]
    assert abs(d["H"] - d["kinetic"] - d["field"]) < 1e-14 * abs(d["H"])


def test_two_stream_growth_rate():
    """f0 = (1 + alpha cos 0.5x) v^2 exp(-v^2/2)/sqrt(2pi) on the 256 x 256
    lattice (nx 128, dt 0.05) with alpha = 1e-4 so the mode stays linear:
    E_amp grows at the purely growing dispersion root (gamma ~ 0.2592).
    (With the benchmark's alpha = 0.05 the mode saturates by t ~ 16.)"""
    import dataclasses
    spec = W.two_stream()
    lat = dataclasses.replace(spec.lattice, alpha=1e-4)
    r = O.run(O.init_lattice(lat), spec.nx, lat.L, spec.dt, 620, diag_every=1)
    t, E = r["diag"][:, 0], r["diag"][:, 6]
    root = ph.vsquared_maxwell_root(0.5)
    assert abs(root.real) < 1e-8
    sel = (t >= 10.0) & (t <= 30.0)
    g = np.polyfit(t[sel], np.log(E[sel]), 1)[0]
    assert abs(g / root.imag - 1) < 0.01


def test_strong_landau_paper_setup_damping_rate():
    """Sec. 7.3 (strong Landau damping): L = 12, A = 0.5, k = 2 pi/L, a 100-element
    CG mesh, dt = 0.2.  The paper prints gamma = -0.236 for its E_amp history
    (fit method not stated, reading A10).  With the lattice start (reading A6)
    on 128^2 and 256^2 lattices, the least-squares fit of log E_amp over the
    maxima in t in [0, 15] is within 7% of the printed rate for the decorated
    run (reading A1, LUMPED) and the decorated and point-particle runs agree
    to 1%; the 7% covers the maxima that enter or leave the window as the
    lattice changes (fits of -0.224 ... -0.251 between 128^2 and 256^2).  The
    decorated run stays finite over the fitted time (the decorations' growth
    at later times is described with the findings of the oracle)."""
    L = 12.0
    for side in (128, 256):
        lat = W.LatticeSpec(side, side, L, -6.0, 6.0, 0.5, 2 * math.pi / L, W.MAXWELL)
        st = O.init_lattice(lat)
        rates = []
        for dec in (True, False):
            r = O.run(st, 100, L, 0.2, 250, diag_every=1, decorated=dec)
            t, E = r["diag"][:, 0], r["diag"][:, 6]
            assert np.all(np.isfinite(E))
            g, _, peaks = ph.rate_fit(t, E, 0.0, 15.0, min_sep=1.0)
            assert len(peaks) >= 5
            rates.append(g)
        assert abs(rates[0] / -0.236 - 1) < 0.07, (side, rates)
        assert abs(rates[0] / rates[1] - 1) < 0.01, (side, rates)


def test_two_beam_root_cold_limit_and_the_printed_rate():
    """The warm two-beam dispersion relation used to read Sec. 7.2: as T -> 0
    it tends to the cold symmetric-beam relation (w^2 - x^2)^2 = w^2 + x^2
    (x = k u, n0 = 1), whose growing root is
    gamma^2 = [sqrt(8 x^2 + 1) - (2 x^2 + 1)]/2; at the printed setup (u = 1,
    T = 0.09, L = 2 pi so k = 1, n0 = 1) the root is about 0.21, far from the
    printed 0.7863, which needs n0 of about 20 (gamma 0.78 there)."""
    for x in (0.4, 0.6, 0.8):
        cold = math.sqrt((math.sqrt(8 * x * x + 1) - (2 * x * x + 1)) / 2)
        warm = ph.two_beam_root(x, T=1e-5)
        assert abs(warm / cold - 1) < 0.01, (x, warm, cold)
    g1 = ph.two_beam_root(1.0, n0=1.0)
    assert 0.19 < g1 < 0.22
    assert abs(ph.two_beam_root(1.0, n0=20.0) / 0.7863 - 1) < 0.02


def test_wrap_maps_round_up_into_domain():
    """Reading A5: a position that rounds up to exactly L wraps to 0."""
    L = 4 * math.pi
    w = O.wrap(np.array([-1e-20, -L, 2 * L - 1e-17, L, 0.0, 3.5]), L)
    assert np.all((w >= 0.0) & (w < L))
    assert w[0] == 0.0 and w[3] == 0.0 and w[4] == 0.0 and w[5] == 3.5


def test_momentum_and_kinetic_are_pairings_with_the_ansatz():
    """momentum = <Gamma_2, p> and kinetic = <Gamma_2, p^2/2> (pairing Eq.
    pairing with the ansatz Eq. sw_f_ansatz), computed here by quadrature with
    the deltas replaced by narrow Gaussians of width s: the momentum is exact
    for any s, the kinetic carries an extra psi* s^2/2."""
    L, nx = 5.0, 8
    st = rng_state(3, L, nx, 41)
    st["qs"] *= 50.0          # make the decoration terms visible
    f = O.field_of_state(st["Q"], st["ps"], st["psi"], L, nx)
    d = O.diagnostics(st["P"], st["qs"], st["psi"], f["Phi"], L)
    s = 0.05
    p = np.linspace(-6, 6, 24001)
    dp = p[1] - p[0]
    g = lambda z: np.exp(-z * z / (2 * s * s)) / (math.sqrt(2 * math.pi) * s)
    dg = lambda z: -z / (s * s) * g(z)
    mom = kin = 0.0
    for a in range(3):
        # q-integrals of g and g' are 1 and 0, so only the p-parts remain
        fp = st["psi"][a] * g(p - st["P"][a]) - st["qs"][a] * dg(p - st["P"][a])
        mom += np.sum(p * fp) * dp
        kin += np.sum(0.5 * p * p * fp) * dp - 0.5 * st["psi"][a] * s * s
    assert abs(d["momentum"] - mom) < 1e-10 * max(1.0, abs(mom))
    assert abs(d["kinetic"] - kin) < 1e-9 * max(1.0, abs(kin))


def test_fp32_storage_mode_rounds_state_and_decides_in_fp32():
    """store_f32 keeps every updated value representable in FP32 and takes the
    element decision from the stored FP32 position; it stays within FP32
    rounding of the FP64 run."""
    spec = W.landau_linear(jitter=1e-3)
    jx, jv = W.jitter(spec.lattice)
    st = O.init_lattice(spec.lattice, jx, jv)
    st = {k: v.astype(np.float32).astype(np.float64) for k, v in st.items()}
    L = spec.lattice.L
    a = O.run(st, spec.nx, L, spec.dt, 10, diag_every=0, store_f32=True)
    b = O.run(st, spec.nx, L, spec.dt, 10, diag_every=0)
    for k in ("Q", "P", "qs", "ps"):
        assert np.array_equal(a[k].astype(np.float32).astype(np.float64), a[k]), k
        assert np.abs(a[k] - b[k]).max() <= 1e-5 * max(np.abs(b[k]).max(), 1e-30), k
    assert np.all((a["Q"] >= 0) & (a["Q"] < L))
