"""Pins of the oracle's P2 (quadratic Lagrange) field, V_h^(2) of Sec. 5.

- Charges on mesh vertices: the exact periodic solution phi' = n0 (q - Q0) -
  psi/2 (sawtooth about each charge, n0 = sum psi / L, zero mean) is piecewise
  linear with jumps at vertices, so it lies in the P2 derivative space and
  Galerkin must reproduce it exactly.
- For any monopole + dipole load the P2 vertex values (hence the element
  slopes) equal the P1 ones: eliminating the element midpoints (static
  condensation) turns the P2 system into the P1 system with the same load.
- An element with no particles carries phi'' = n0 (Eq. poisson with rho = 0).
- The field energy (1/2) int phi'^2 of the quadratic matches a fine
  quadrature of the gathered phi'.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

L = 2 * np.pi


def test_vertex_charges_give_the_exact_sawtooth():
    nx = 32
    h = L / nx
    Q = np.array([3 * h, 17 * h, 17 * h, 29 * h])
    psi = np.array([1.0, 0.25, 0.5, 2.0])
    Phi2, a, beta = O.p2_field(Q, np.zeros(4), psi, L, nx)
    n0 = psi.sum() / L
    xm = (np.arange(nx) + 0.5) * h

    def dphi_exact(q):
        return sum(w * (((q - Q0) % L) / L - 0.5) for Q0, w in zip(Q, psi))
    np.testing.assert_allclose(a, dphi_exact(xm), atol=1e-13)
    np.testing.assert_allclose(-2 * beta / h, n0, rtol=1e-12)
    # the gathered phi' at arbitrary points inside elements
    q = np.random.default_rng(0).uniform(0, L, 200)
    dV, d2V = O.p2_gather(q, a, beta, L, nx)
    np.testing.assert_allclose(dV, dphi_exact(q), atol=1e-12)


def test_vertex_values_equal_p1():
    nx = 24
    st = W.random_state(500, L, seed=3, nx=nx)
    Phi2, a, beta = O.p2_field(st["Q"], st["ps"], st["psi"], L, nx)
    f1 = O.field_of_state(st["Q"], st["ps"], st["psi"], L, nx)
    Phi, dphi = f1["Phi"], f1["dphi"]
    np.testing.assert_allclose(a, dphi, atol=1e-12 * np.abs(dphi).max())
    # same potential up to the gauge constant at the vertices
    d = Phi2[0::2] - Phi
    assert np.ptp(d) < 1e-12 * np.abs(Phi).max()


def test_empty_element_curvature_is_n0():
    nx = 16
    h = L / nx
    Q = np.array([2.3 * h, 2.7 * h, 9.4 * h])
    psi = np.array([0.7, 0.2, 1.1])
    ps = np.array([0.01, -0.02, 0.005])
    Phi2, a, beta = O.p2_field(Q, ps, psi, L, nx)
    empty = [e for e in range(nx) if e not in (2, 9)]
    np.testing.assert_allclose(-2 * beta[empty] / h, psi.sum() / L, rtol=1e-11)


def test_field_energy_matches_quadrature():
    nx = 20
    st = W.random_state(300, L, seed=4, nx=nx)
    Phi2, a, beta = O.p2_field(st["Q"], st["ps"], st["psi"], L, nx)
    Wf, Ea = O.p2_energy(a, beta, L)
    q = (np.arange(20 * nx * 64) + 0.5) * (L / (20 * nx * 64))
    dV, _ = O.p2_gather(q, a, beta, L, nx)
    w_quad = 0.5 * np.sum(dV ** 2) * (L / len(q))
    assert Wf == pytest.approx(w_quad, rel=1e-6)
    assert Ea == pytest.approx(np.sqrt(2 * Wf / L), rel=1e-14)
