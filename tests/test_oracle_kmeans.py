"""Pins of the oracle's decorated-particle initialization (Sec. 4.1-4.2,
Alg. lumping_procedure, Eqs. psi-star and moment-def with the periodic c).

Each check is fixed by the paper or by the mathematics, not by the oracle's
own formulas:
- the defining moment requirements of the torus subsection: for every cluster
  the decorated particle reproduces the markers' sin(2 pi (q - Q)/L) moment and
  the p moment exactly;
- a worked two-marker cluster with the numbers written out by hand;
- single-marker clusters carry no dipole; psi* conserves the total weight;
- the nearest-center assignment is valid against an FP64 brute force, the
  Lloyd cost never increases, and well separated blobs are recovered exactly,
  across the periodic boundary too.
"""
import numpy as np
import pytest

import oracle as O

L = 2 * np.pi


def _per_d(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def _cost(Qm, Pm, wm, cq, cp, assign, L):
    dq = _per_d(Qm, cq[assign], L)
    dp = Pm - cp[assign]
    return float(np.sum(wm * (dq * dq + dp * dp)))


def _markers(M, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, L, M), rng.normal(0, 1, M), rng.uniform(0.5, 1.5, M) / M


def test_worked_two_marker_cluster():
    # markers (Q, P, psi): (1.0, 0.5, 2.0) and (1.2, -0.5, 1.0); weighted mean
    # (16/15, 1/6): marker 0 is nearer (d^2 0.1156 vs 0.4622)
    Qm, Pm, wm = np.array([1.0, 1.2]), np.array([0.5, -0.5]), np.array([2.0, 1.0])
    out = O.lump(Qm, Pm, wm, np.array([0, 0], np.int32), np.array([1.0]), np.array([0.0]), L)
    assert out["Q"][0] == 1.0 and out["P"][0] == 0.5
    assert out["psi"][0] == 3.0
    assert out["ps"][0] == pytest.approx(np.sin(-0.2), rel=1e-15)      # 1.0 * (L/2pi) sin(2pi(1.0-1.2)/L)
    assert out["qs"][0] == pytest.approx(-1.0, rel=1e-15)               # -(1.0)(0.5 - (-0.5))


def test_moment_requirements_hold_per_cluster():
    Qm, Pm, wm = _markers(600, 1)
    K = 40
    cq, cp, a = O.kmeans(Qm, Pm, wm, Qm[:K], Pm[:K], L, 8)
    out = O.lump(Qm, Pm, wm, a, cq, cp, L)
    ks = [k for k in range(K) if np.any(a == k)]
    assert len(out["Q"]) == len(ks)
    for s, k in enumerate(ks):
        m = a == k
        Qa, Pa = out["Q"][s], out["P"][s]
        # int sin(2pi(q - Qa)/L) f dq dp: markers vs psi* delta + p* d/dq delta - q* d/dp delta
        lhs = np.sum(wm[m] * np.sin(2 * np.pi * (Qm[m] - Qa) / L))
        rhs = -out["ps"][s] * (2 * np.pi / L)
        assert lhs == pytest.approx(rhs, abs=1e-15 * max(1.0, np.sum(wm[m])))
        # int p f dq dp
        assert np.sum(wm[m] * Pm[m]) == pytest.approx(out["psi"][s] * Pa + out["qs"][s], abs=1e-14)
        # the center is a member
        assert np.any((Qm[m] == Qa) & (Pm[m] == Pa))
    assert out["psi"].sum() == pytest.approx(wm.sum(), rel=1e-14)


def test_single_marker_clusters_carry_no_dipole():
    Qm, Pm, wm = _markers(50, 2)
    out = O.lump(Qm, Pm, wm, np.arange(50, dtype=np.int32), Qm, Pm, L)
    assert np.array_equal(out["Q"], Qm) and np.array_equal(out["P"], Pm)
    assert np.array_equal(out["psi"], wm)
    assert np.all(out["qs"] == 0.0) and np.all(out["ps"] == 0.0)


def test_empty_clusters_are_skipped_in_order():
    Qm, Pm, wm = np.array([1.0, 2.0, 3.0]), np.array([0.0, 0.0, 0.0]), np.ones(3)
    a = np.array([3, 0, 3], np.int32)
    out = O.lump(Qm, Pm, wm, a, np.array([2.0, 0.0, 0.0, 2.0]), np.zeros(4), L)
    assert len(out["Q"]) == 2
    assert out["Q"][0] == 2.0 and out["psi"][1] == 2.0


def test_assignment_is_a_nearest_center():
    Qm, Pm, wm = _markers(3000, 3)
    cq, cp = _markers(97, 4)[:2]
    a = O.kmeans_assign(Qm, Pm, cq, cp, L)
    dq = _per_d(Qm[:, None], cq[None, :], L)
    d2 = dq * dq + (Pm[:, None] - cp[None, :]) ** 2
    best = d2.min(axis=1)
    got = d2[np.arange(len(Qm)), a]
    assert np.all(got <= best * (1 + 1e-6) + 1e-12)     # FP32 decision: within its rounding


def test_lloyd_cost_never_increases():
    Qm, Pm, wm = _markers(2000, 5)
    K = 64
    cq, cp = Qm[:K].copy(), Pm[:K].copy()
    costs = []
    for it in range(10):
        cq, cp, a = O.kmeans(Qm, Pm, wm, cq, cp, L, 1)
        costs.append(_cost(Qm, Pm, wm, cq, cp, a, L))
    assert all(c1 <= c0 * (1 + 1e-6) for c0, c1 in zip(costs, costs[1:]))


def test_separated_blobs_are_recovered_across_the_boundary():
    rng = np.random.default_rng(6)
    centers = np.array([[0.02, 0.0], [2.0, 3.0], [4.0, -3.0], [6.2, 6.0]])   # blob 0 and 3 straddle q = 0
    Qm, Pm, lab = [], [], []
    for k, (q, p) in enumerate(centers):
        Qm.append(np.mod(q + 0.05 * rng.standard_normal(100), L))
        Pm.append(p + 0.05 * rng.standard_normal(100))
        lab.append(np.full(100, k))
    Qm, Pm, lab = np.concatenate(Qm), np.concatenate(Pm), np.concatenate(lab)
    wm = np.full(len(Qm), 0.01)
    init_q = centers[:, 0] + 0.3
    cq, cp, a = O.kmeans(Qm, Pm, wm, np.mod(init_q, L), centers[:, 1] - 0.4, L, 10)
    assert np.array_equal(a, lab)
    # the q mean of the straddling blobs sits near their centers, not near L/2
    assert abs(_per_d(cq[0], 0.02, L)) < 0.02 and abs(_per_d(cq[3], 6.2, L)) < 0.02
