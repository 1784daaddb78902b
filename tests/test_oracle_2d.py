"""Pins of the 2D2V oracle (general-d model of Sec. 3.3 on the torus, bilinear
elements) against what mathematics and the pinned 1D oracle fix.

- Stiffness: the Q1 stiffness of a periodic uniform mesh is the tensor sum
  Kx (x) My + Mx (x) Ky of the 1D P1 stiffness and consistent mass, so a
  Fourier mode is an eigenvector with the closed-form symbol; the solve of a
  mode returns the mode divided by the symbol, and the background
  multiplier is the mean load.
- Deposit: brute force over all nodes with periodic hat products and their
  analytic derivatives; the dipole part carries no net charge.
- Projection: for a Fourier mode the lumped projection of grad phi_h is the
  central difference smoothed by (1/6, 2/3, 1/6) across, in closed form.
- Energy: (1/2) int |grad phi_h|^2 = (1/2) Phi^T K Phi = (1/2) Phi^T btilde.
- Reduction to 1D: a state replicated on every mesh row (on the row nodes,
  no y motion, weights times hy) evolves exactly like the 1D oracle with the
  lumped phi'' (and the same with x and y exchanged).
- Free streaming: one particle on every node with equal weight has no field.
- Gather: grad phi_h and the projected Hessian converge to the exact ones at
  first order in h for a smooth potential.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _mode(nx, ny, mx, my):
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    tx, ty = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
    return tx, ty, tx * i + ty * j


def _symbol(tx, ty, hx, hy):
    return ((2 - 2 * np.cos(tx)) * (4 + 2 * np.cos(ty)) * hy / (6 * hx)
            + (2 - 2 * np.cos(ty)) * (4 + 2 * np.cos(tx)) * hx / (6 * hy))


@pytest.mark.parametrize("nx,ny,mx,my", [(8, 6, 1, 0), (8, 6, 0, 2), (8, 6, 3, 1), (16, 8, 5, 3)])
def test_fourier_mode_is_an_eigenvector_with_the_closed_form_symbol(nx, ny, mx, my):
    Lx, Ly = 2.0, 3.5
    hx, hy = Lx / nx, Ly / ny
    tx, ty, a = _mode(nx, ny, mx, my)
    v = np.cos(a)
    K = O.stiffness2d(nx, ny, Lx, Ly)
    lam = _symbol(tx, ty, hx, hy)
    np.testing.assert_allclose(K @ v.ravel(), lam * v.ravel(), atol=1e-12 * max(lam, 1))
    # solve: load = lam v + a constant; Phi = v, background = constant / (hx hy)
    Phi, bg = O.solve2d(lam * v + 0.7, Lx, Ly)
    np.testing.assert_allclose(Phi, v, atol=1e-11)
    assert bg == pytest.approx(0.7 / (hx * hy), rel=1e-12)


def _hat(d, h):
    return np.maximum(0.0, 1.0 - np.abs(d) / h)


def _dhat(d, h):
    # one-sided at the node itself: a particle on a mesh line belongs to the
    # cell on its right, where its own node's hat falls
    return np.where((d >= 0) & (d < h), -1.0 / h, np.where((d < 0) & (d >= -h), 1.0 / h, 0.0))


def test_deposit_matches_brute_force_over_all_nodes():
    rng = np.random.default_rng(3)
    nx, ny, Lx, Ly = 7, 5, 3.5, 2.5          # hx = hy = 1/2: mesh-line positions are exact
    hx, hy = Lx / nx, Ly / ny
    n = 60
    Qx = rng.uniform(0, Lx, n)
    Qy = rng.uniform(0, Ly, n)
    Qx[:4] = [0.0, 2 * hx, Lx - 1e-13, 5 * hx]          # on mesh lines and at the edge
    Qy[:4] = [3 * hy, 0.0, hy, Ly - 1e-13]
    psi = rng.uniform(0.5, 1.5, n)
    psx, psy = rng.normal(0, 0.05, n), rng.normal(0, 0.05, n)
    b = O.deposit2d(Qx, Qy, psx, psy, psi, Lx, Ly, nx, ny)
    ref = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            dx = Qx - i * hx
            dx = dx - Lx * np.round(dx / Lx)
            dy = Qy - j * hy
            dy = dy - Ly * np.round(dy / Ly)
            Nx, Ny = _hat(dx, hx), _hat(dy, hy)
            ref[j, i] = np.sum(psi * Nx * Ny - psx * _dhat(dx, hx) * Ny - psy * Nx * _dhat(dy, hy))
    np.testing.assert_allclose(b, ref, atol=1e-12)
    assert b.sum() == pytest.approx(psi.sum(), rel=1e-13)


@pytest.mark.parametrize("mx,my", [(1, 0), (2, 1), (3, 3)])
def test_projection_of_a_mode_is_the_smoothed_central_difference(mx, my):
    nx, ny, Lx, Ly = 12, 8, 4.0, 2.5
    hx, hy = Lx / nx, Ly / ny
    tx, ty, a = _mode(nx, ny, mx, my)
    gx, gy = O.project2d(np.cos(a), Lx, Ly)
    np.testing.assert_allclose(gx, -np.sin(tx) / hx * (2 / 3 + np.cos(ty) / 3) * np.sin(a), atol=1e-12)
    np.testing.assert_allclose(gy, -np.sin(ty) / hy * (2 / 3 + np.cos(tx) / 3) * np.sin(a), atol=1e-12)


def test_field_energy_identities():
    st = W.random_state_2d(500, 3.0, 2.0, seed=5)
    nx, ny, Lx, Ly = 9, 6, 3.0, 2.0
    b = O.deposit2d(st["Qx"], st["Qy"], st["px"], st["py"], st["psi"], Lx, Ly, nx, ny)
    Phi, lam = O.solve2d(b, Lx, Ly)
    K = O.stiffness2d(nx, ny, Lx, Ly)
    Wq = O.field_energy2d(Phi, Lx, Ly)
    bt = b - lam * (Lx / nx) * (Ly / ny)
    assert Wq == pytest.approx(0.5 * Phi.ravel() @ K @ Phi.ravel(), rel=1e-12)
    assert Wq == pytest.approx(0.5 * Phi.ravel() @ bt.ravel(), rel=1e-11)
    assert abs(Phi.sum()) < 1e-12 * np.abs(Phi).max() * Phi.size


def _replicate(st1, L, ny, Ly, axis):
    """1D state -> 2D state on every mesh row (axis 0: rows along y) at the row
    nodes, no motion across; weights psi*, q*, p* times the row spacing."""
    hy = Ly / ny
    n = len(st1["Q"])
    rows = np.repeat(np.arange(ny) * hy, n)
    tile = lambda a: np.tile(a, ny)
    z = np.zeros(n * ny)
    along = {"Q": tile(st1["Q"]), "P": tile(st1["P"]), "q": tile(st1["qs"]) * hy, "p": tile(st1["ps"]) * hy}
    if axis == 0:
        return {"Qx": along["Q"], "Qy": rows, "Px": along["P"], "Py": z, "qx": along["q"], "qy": z,
                "px": along["p"], "py": z, "psi": tile(st1["psi"]) * hy}
    return {"Qx": rows, "Qy": along["Q"], "Px": z, "Py": along["P"], "qx": z, "qy": along["q"],
            "px": z, "py": along["p"], "psi": tile(st1["psi"]) * hy}


@pytest.mark.parametrize("axis", [0, 1])
def test_row_replicated_state_evolves_like_the_1d_oracle(axis):
    L, nx1, dt, steps = 4 * np.pi, 16, 0.1, 6
    ny, Lc = 5, 3.0
    st1 = W.random_state(300, L, seed=9, nx=nx1)
    ref = O.run(st1, nx1, L, dt, steps, diag_every=2)
    st2 = _replicate(st1, L, ny, Lc, axis)
    if axis == 0:
        got = O.run2d(st2, nx1, ny, L, Lc, dt, steps, diag_every=2)
        Q, P, qs, ps, tr = got["Qx"], got["Px"], got["qx"], got["px"], got["Qy"]
    else:
        got = O.run2d(st2, ny, nx1, Lc, L, dt, steps, diag_every=2)
        Q, P, qs, ps, tr = got["Qy"], got["Py"], got["qy"], got["py"], got["Qx"]
    hy = Lc / ny
    n = len(st1["Q"])
    for r in range(ny):
        sl = slice(r * n, (r + 1) * n)
        np.testing.assert_allclose(Q[sl], ref["Q"], atol=1e-12)
        np.testing.assert_allclose(P[sl], ref["P"], atol=1e-12)
        np.testing.assert_allclose(qs[sl] / hy, ref["qs"], atol=1e-12)
        np.testing.assert_allclose(ps[sl] / hy, ref["ps"], atol=1e-12)
    # no motion across (the solve's rounding leaves a field of ~1e-16 across)
    np.testing.assert_allclose(tr, st2["Qy"] if axis == 0 else st2["Qx"], atol=1e-13)
    d2, d1 = got["diag"], ref["diag"]
    assert d2.shape[0] == d1.shape[0]
    # 1D record: t, mass, momentum, kinetic, W, H, E_amp (column 2 unused here)
    np.testing.assert_allclose(d2[:, 0], d1[:, 0])
    np.testing.assert_allclose(d2[:, 1], Lc * d1[:, 1], rtol=1e-12)
    np.testing.assert_allclose(d2[:, 2 + axis], Lc * d1[:, 2], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(d2[:, 4], Lc * d1[:, 3], rtol=1e-11)
    np.testing.assert_allclose(d2[:, 5], Lc * d1[:, 4], rtol=1e-10)
    np.testing.assert_allclose(d2[:, 7], d1[:, 6], rtol=1e-10)


def test_one_particle_per_node_has_no_field_and_streams_freely():
    nx, ny, Lx, Ly, dt = 6, 4, 3.0, 2.0, 0.05
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    n = nx * ny
    rng = np.random.default_rng(0)
    st = {"Qx": (i.ravel() * Lx / nx).astype(float), "Qy": (j.ravel() * Ly / ny).astype(float),
          "Px": np.full(n, 0.0), "Py": np.full(n, 0.0), "psi": np.full(n, 0.3)}
    b = O.deposit2d(st["Qx"], st["Qy"], None, None, st["psi"], Lx, Ly, nx, ny)
    Phi, _ = O.solve2d(b, Lx, Ly)
    assert np.abs(Phi).max() < 1e-14
    st["Px"] = rng.normal(size=n) * 1e-3      # moves, but stays off no node long enough to matter here
    got = O.run2d(st, nx, ny, Lx, Ly, dt, 1, diag_every=1, decorated=False)
    np.testing.assert_allclose(got["Qx"], (st["Qx"] + dt * st["Px"]) % Lx, atol=1e-12)


def test_gather_converges_at_first_order():
    Lx, Ly = 2.0, 3.0
    rng = np.random.default_rng(1)
    q = (rng.uniform(0, Lx, 4000), rng.uniform(0, Ly, 4000))
    kx, ky = 2 * np.pi / Lx, 2 * np.pi / Ly
    phi = lambda x, y: np.sin(kx * x) * np.cos(2 * ky * y)
    exact = {"Ex": kx * np.cos(kx * q[0]) * np.cos(2 * ky * q[1]),
             "Ey": -2 * ky * np.sin(kx * q[0]) * np.sin(2 * ky * q[1]),
             "Hxx": -kx * kx * phi(*q), "Hyy": -4 * ky * ky * phi(*q),
             "Hxy": -2 * kx * ky * np.cos(kx * q[0]) * np.sin(2 * ky * q[1])}
    exact["Hyx"] = exact["Hxy"]
    ns = np.array([16, 32, 64, 128])
    errs = {k: [] for k in exact}
    for n in ns:
        x = np.arange(n) * Lx / n
        y = np.arange(n) * Ly / n
        Phi = phi(x[None, :], y[:, None])
        gx, gy = O.project2d(Phi, Lx, Ly)
        g = O.gather2d(q[0], q[1], Phi, gx, gy, Lx, Ly)
        for k in exact:
            errs[k].append(np.mean(np.abs(g[k] - exact[k])) / np.mean(np.abs(exact[k])))
    for k in exact:
        order = -np.polyfit(np.log(ns), np.log(errs[k]), 1)[0]
        assert 0.85 < order < 2.3, (k, order, errs[k])
        assert errs[k][-1] < 0.05, (k, errs[k])


def test_fp32_cell_decision():
    L, n = 2 * np.pi, 64
    h = L / n
    Q = np.array([0.0, h, 3 * h, L - 1e-7, np.nextafter(np.float32(L), 0)], dtype=np.float64)
    got = O.cell2d(Q, L, n, f32=True)
    assert [O.lib().or2d_cell_f32(float(x), L, n) for x in Q] == list(got)
    assert [O.lib().or2d_cell(float(x), L, n) for x in Q] == list(O.cell2d(Q, L, n))
    q = Q.astype(np.float32)
    ref = np.clip(np.floor(q * np.float32(n / L)), 0, n - 1).astype(np.int32)
    np.testing.assert_array_equal(got, ref)


def test_lattice_init_with_ky_zero_factors_into_the_1d_init():
    """ky = 0: f0 = (1 + alpha cos kx x) M(vx) M(vy), so every 2D decoration
    is the pinned 1D one (same x-vx lattice, Maxwellian term) times the
    y-vy cell integral of M(vy) by the same Gauss rule; p*_y vanishes (odd
    integrand over a centred cell) and q*_y is the vy cell moment."""
    nq, nv, n, L, Ly = 8, 12, 3, 4 * np.pi, 3.0
    sp2 = W.Lattice2DSpec(nq, 2, nv, 6, L, Ly, -6.0, 6.0, 0.3, 0.5, 0.0, 1.0, n, True)
    st2 = O.init_lattice2d(sp2)
    lat1 = W.LatticeSpec(nq, nv, L, -6.0, 6.0, 0.3, 0.5, W.MAXWELL, quad_order=n)
    st1 = O.init_lattice(lat1)
    g, gw = O.gauss_legendre(n)
    dy, dvy = Ly / 2, 12.0 / 6
    M = lambda v: np.exp(-v * v / 2) / np.sqrt(2 * np.pi)
    a = np.arange(sp2.n)
    i, j, l, k = a % nq, (a // nq) % 2, (a // (2 * nq)) % 6, a // (2 * nq * 6)    # positions fastest
    one = i * nv + k                                        # the 1D particle of (i, k)
    wc = -6.0 + (l + 0.5) * dvy
    vy = wc[:, None] + 0.5 * dvy * g[None, :]
    Imy = (gw[None, :] * 0.5 * dvy * M(vy)).sum(1) * dy          # int_cell dy dvy M(vy)
    Imy1 = (gw[None, :] * 0.5 * dvy * M(vy) * (wc[:, None] - vy)).sum(1) * dy
    np.testing.assert_allclose(st2["psi"], st1["psi"][one] * M(wc) * dy * dvy, rtol=1e-13)
    np.testing.assert_allclose(st2["px"], st1["ps"][one] * Imy, atol=1e-16, rtol=1e-11)
    np.testing.assert_allclose(st2["qx"], st1["qs"][one] * Imy, atol=1e-16, rtol=1e-11)
    assert np.abs(st2["py"]).max() < 1e-14 * np.abs(st2["px"]).max()
    # q*_y: the x-vx cell integral of f0 times -(int M(vy)(wc - vy)) over the vy cell
    x = (i + 0.5)[:, None] * (L / nq) + 0.5 * (L / nq) * g[None, :]
    vx = (-6.0 + (k + 0.5) * (12.0 / nv))[:, None] + 0.5 * (12.0 / nv) * g[None, :]
    Ix = (gw[None, :] * 0.5 * (L / nq) * (1 + 0.3 * np.cos(0.5 * x))).sum(1)
    Ivx = (gw[None, :] * 0.5 * (12.0 / nv) * M(vx)).sum(1)
    np.testing.assert_allclose(st2["qy"], -Ix * Ivx * Imy1, atol=1e-16, rtol=1e-11)


def test_lattice_init_mass_and_symmetry():
    sp = W.Lattice2DSpec(8, 6, 16, 16, 4 * np.pi, 2 * np.pi, alpha=0.0, quad_order=2)
    st = O.init_lattice2d(sp)
    assert st["psi"].sum() == pytest.approx(sp.Lx * sp.Ly, rel=2e-3)
    assert np.abs(st["px"]).max() < 1e-15 and np.abs(st["py"]).max() < 1e-15     # uniform in space
    assert np.all(st["Qx"] < sp.Lx) and np.all(st["Qy"] < sp.Ly)
