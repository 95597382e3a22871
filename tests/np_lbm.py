"""Independent whole-array numpy evaluation of one step of the method.

Used only to pin the C oracle (brute-force comparison on tiny periodic
lattices).  It is written in a different style from the oracle: whole-field
array expressions, ``np.roll`` for every shift, the fugacity taken from the
printed form of Eq. (12) (which needs p > 0), and no shared tables.

Array layout: ``g[i, a, z, y, x]`` post-streaming populations (Eq. 1a),
fields ``[z, y, x]``.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


def d2q9():
    e = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0],
                  [1, 1, 0], [-1, 1, 0], [-1, -1, 0], [1, -1, 0]])
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return 2, e, w


def d3q19():
    e = [[0, 0, 0]]
    w = [1 / 3]
    for v in ([1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]):
        e.append(v)
        w.append(1 / 18)
    for sx in (1, -1):
        for sy in (1, -1):
            e += [[sx, sy, 0], [sx, 0, sy], [0, sx, sy]]
            w += [1 / 36] * 3
    return 3, np.array(e), np.array(w)


def shifted(X, e):
    """X(r + e) on the periodic box (X indexed [z, y, x])."""
    return np.roll(X, shift=(-e[2], -e[1], -e[0]), axis=(-3, -2, -1))


def grad(X, e, w):
    return np.stack([sum(w[a] * e[a, d] * shifted(X, e[a]) for a in range(len(w))) / CS2
                     for d in range(3)])


def lap(X, e, w):
    return 2.0 / CS2 * sum(w[a] * (shifted(X, e[a]) - X) for a in range(len(w)))


def alpha(a, b, omega, T, R):
    Tc = 0.077796074 / 0.457235529 * a / (R * b)
    m = np.where(omega <= 0.49,
                 0.374640 + 1.54226 * omega - 0.26992 * omega ** 2,
                 0.379642 + 1.48503 * omega - 0.164423 * omega ** 2 + 0.016666 * omega ** 3)
    return (1.0 + m * (1.0 - np.sqrt(T / Tc))) ** 2


def pr_fields(rhom, a, b, omega, kij, T, R):
    """Pressure and ln f_i on whole fields from Eqs. (9)-(12) as printed."""
    nc = rhom.shape[0]
    rho = rhom.sum(axis=0)
    x = rhom / rho
    aa = a * alpha(a, b, omega, T, R)
    Aij = np.sqrt(np.outer(aa, aa)) * (1.0 - kij)
    aam = np.einsum("i...,ij,j...->...", x, Aij, x)
    bm = np.einsum("i,i...->...", b, x)
    v = 1.0 / rho
    RT = R * T
    p = RT / (v - bm) - aam / (v * v + 2 * bm * v - bm * bm)
    if np.any(p <= 0):
        raise ValueError("printed Eq. (12) needs p > 0")
    s2 = np.sqrt(2.0)
    logr = np.log((v + (1 + s2) * bm) / (v + (1 - s2) * bm))
    lnf = np.empty_like(rhom)
    for i in range(nc):
        sumj = np.einsum("j,j...->...", Aij[i], x)
        lnphi = (b[i] / bm) * (p * v / RT - 1) - np.log((v - bm) * p / RT) \
            + aam / (2 * s2 * bm * RT) * (b[i] / bm - 2.0 / aam * sumj) * logr
        lnf[i] = lnphi + np.log(x[i] * p)
    return p, lnf


def step(g, lattice, a, b, omega, kij, M, T, tau, R=1.0, kappa_ref=0.02, kappa_ref_index=0):
    """One step g(t) -> g(t+1) (post-streaming states)."""
    D, e, w = d2q9() if lattice == 0 else d3q19()
    nc, Q = g.shape[:2]
    rho = g.sum(axis=1)                               # mass densities rho_i
    rhom = rho / M[:, None, None, None]               # molar densities
    _, lnf = pr_fields(rhom, a, b, omega, kij, T, R)
    kappa = kappa_ref * a / a[kappa_ref_index]        # Eq. (6)
    laps = np.stack([lap(rhom[j], e, w) for j in range(nc)])
    F = np.empty((nc, 3) + rho.shape[1:])
    for i in range(nc):
        inter = sum(np.sqrt(kappa[i] * kappa[j]) * laps[j] for j in range(nc))
        F[i] = -rhom[i] * R * T * grad(lnf[i], e, w) + rhom[i] * grad(inter, e, w)   # Eq. (5)
    gradrho = np.stack([grad(rho[i], e, w) for i in range(nc)])
    mom = np.einsum("iaxyz,ad->dxyz", g.reshape((nc, Q) + rho.shape[1:]), e.astype(float))
    u = (mom + 0.5 * F.sum(axis=0)) / rho.sum(axis=0)
    uu = (u * u).sum(axis=0)
    out = np.empty_like(g)
    for a_ in range(Q):
        ea = e[a_].astype(float)[:, None, None, None]
        ue = (u * ea).sum(axis=0)
        e2 = float((e[a_] ** 2).sum())
        B = ue / CS2 + ue ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2)
        for i in range(nc):
            geq = w[a_] * rho[i] * B + (rho[i] if a_ == 0 else 0.0)
            vF = (ea - u) / CS2 + ue * ea / CS2 ** 2
            vG = -u + ue * ea / CS2 + 0.5 * (e2 / CS2 - D) * u
            Fa = w[a_] * ((F[i] * vF).sum(axis=0) + (gradrho[i] * vG).sum(axis=0))
            post = g[i, a_] - (g[i, a_] - geq) / tau + (1 - 0.5 / tau) * Fa
            out[i, a_] = np.roll(post, shift=(e[a_][2], e[a_][1], e[a_][0]), axis=(-3, -2, -1))
    return out
