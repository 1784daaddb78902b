"""Closed-form physics used to pin the oracle and to assess long runs.

* Kinetic dispersion relations of the 1D Vlasov-Poisson system (e = m =
  eps0 = 1) in terms of the plasma dispersion function Z, evaluated with
  scipy's Faddeeva function: Z(z) = i sqrt(pi) w(z).
* Thm 1 (single decorated source on the torus): closed-form potential and the
  explicit P1 dipole Galerkin solution used in the proof of Thm 2.
* A rate fit of log E_amp at its local maxima (the paper fits rates to the
  E_amp history, Sec. 7.2/7.3, without stating a method; this least-squares
  fit over de-duplicated maxima is the reading used here).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import fsolve
from scipy.special import wofz


def Zfun(z):
    return 1j * math.sqrt(math.pi) * wofz(z)


def _solve(eps, guess):
    def f(x):
        v = eps(x[0] + 1j * x[1])
        return [v.real, v.imag]
    s = fsolve(f, [guess.real, guess.imag], xtol=1e-14, full_output=True)
    x = s[0]
    return complex(x[0], x[1])


def landau_root(k, guess=1.4 - 0.15j):
    """Least-damped root of 1 + (1 + zeta Z(zeta))/k^2 = 0, zeta = w/(sqrt2 k),
    for the Maxwellian f0 = exp(-v^2/2)/sqrt(2 pi)."""
    def eps(w):
        z = w / (math.sqrt(2) * k)
        return 1 + (1 + z * Zfun(z)) / k ** 2
    return _solve(eps, guess)


def vsquared_maxwell_root(k, guess=0.0 + 0.25j):
    """Root for f0 = v^2 exp(-v^2/2)/sqrt(2 pi):
    eps = 1 - [(2 - u^2)(1 + zeta Z(zeta)) - 1]/k^2, u = w/k, zeta = u/sqrt2
    (from int f0'(v)/(v - u) dv with the moments of the Maxwellian)."""
    def eps(w):
        u = w / k
        z = u / math.sqrt(2)
        return 1 - ((2 - u * u) * (1 + z * Zfun(z)) - 1) / k ** 2
    return _solve(eps, guess)


def bump_on_tail_root(k, guess=1.0 + 0.2j):
    """Root for f0 = [0.9 exp(-v^2/2) + 0.2 exp(-4 (v - 4.5)^2)]/sqrt(2 pi):
    each Gaussian n exp(-(v-u)^2/(2 s^2))/(sqrt(2 pi) s) adds
    (n/s^2)(1 + zeta Z(zeta))/k^2, zeta = (w/k - u)/(sqrt2 s)."""
    # component m: n_m * exp(-(v-u_m)^2/(2 s_m^2))/(sqrt(2pi) s_m) with n_m = amp * s_m
    comps = [(0.9 * 1.0, 0.0, 1.0), (0.2 * (1.0 / math.sqrt(8.0)), 4.5, 1.0 / math.sqrt(8.0))]

    def eps(w):
        tot = 0
        for n_m, u_m, s_m in comps:
            z = (w / k - u_m) / (math.sqrt(2) * s_m)
            tot += n_m / (s_m ** 2) * (1 + z * Zfun(z))
        return 1 + tot / k ** 2
    return _solve(eps, guess)


def two_beam_root(k, n0=1.0, u=1.0, T=0.09, guesses=(0.1, 0.3, 0.6, 0.9, 1.2, 1.5)):
    """Fastest purely growing root of two Maxwellian beams at +-u, temperature
    T, each of density n0/2 (the warm two-stream setup of Sec. 7.2):
    eps = 1 + sum_b (n0/2)(1 + zeta_b Z(zeta_b))/(T k^2), zeta_b = (w/k -+ u)/sqrt(2T).
    Returns the growth rate (0 when no growing root is found)."""
    def eps(w):
        tot = 0
        for ub in (u, -u):
            z = (w / k - ub) / math.sqrt(2 * T)
            tot += 0.5 * n0 / T * (1 + z * Zfun(z))
        return 1 + tot / k ** 2
    best = 0.0
    for g0 in guesses:
        try:
            with np.errstate(all="ignore"):
                r = _solve(eps, complex(0.0, g0))
        except Exception:
            continue
        if abs(eps(r)) < 1e-8 and abs(r.real) < 1e-6 and r.imag > best:
            best = r.imag
    return best


def rate_fit(t, E, t0, t1, min_sep=None):
    """Least-squares slope of log E at local maxima inside [t0, t1].
    Maxima closer than ``min_sep`` are merged (the larger kept).  The
    frequency is pi / (mean spacing of the kept maxima), since |E| peaks twice
    per period.  Returns (gamma, omega, kept peak times)."""
    t = np.asarray(t); E = np.asarray(E)
    idx = [i for i in range(1, len(E) - 1) if E[i] > E[i - 1] and E[i] >= E[i + 1]
           and t0 <= t[i] <= t1]
    if min_sep is not None:
        kept = []
        for i in idx:
            if kept and t[i] - t[kept[-1]] < min_sep:
                if E[i] > E[kept[-1]]:
                    kept[-1] = i
            else:
                kept.append(i)
        idx = kept
    tm, Em = t[idx], E[idx]
    if len(tm) < 2:
        raise ValueError("not enough maxima in window")
    g = np.polyfit(tm, np.log(Em), 1)[0]
    om = math.pi / np.mean(np.diff(tm))
    return g, om, tm


# --- Thm 1 / Thm 2 closed forms -------------------------------------------
def r_of(q, Q, L):
    """Unique r in (-L/2, L/2] with r = q - Q (mod L)."""
    r = np.mod(np.asarray(q, dtype=float) - Q + L / 2, L) - L / 2
    r = np.where(r == -L / 2, L / 2, r)
    return r


def thm1_phi(q, Q, psi, ps, L):
    """Eq. (solution): the zero-mean periodic solution of
    -phi'' = psi delta(q - Q) + p* delta'(q - Q) - n0 with n0 L = psi."""
    r = r_of(q, Q, L)
    return psi * (r * r / (2 * L) - np.abs(r) / 2 + L / 12) + ps * (r / L - 0.5 * np.sign(r))


def dipole_galerkin_nodes(Q, ps, L, nx):
    """Explicit P1 Galerkin dipole solution from the proof of Thm 2: slope
    p*/L off the element e_Q, p*/L - p*/h on it, zero mean; nodal values."""
    h = L / nx
    iQ = int(math.floor(Q / h))
    phi = np.zeros(nx)
    phi[iQ] = ps * (L - h) / (2 * L)
    # walk from node iQ+1 (value -p*(L-h)/(2L)) around the torus with slope p*/L
    v = -ps * (L - h) / (2 * L)
    for m in range(nx - 1):
        j = (iQ + 1 + m) % nx
        phi[j] = v + m * h * ps / L
    return phi
