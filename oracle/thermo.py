"""Peng-Robinson phase-equilibrium tools of the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``lattice_units``: the paper's conversion to lattice units, fixing R = 1,
  a_C1 = 2/49, b_C1 = 2/21 and M_C1 = 1 (Sec. 3.1, Sec. 3.2).
* ``maxwell``: single-component coexistence from equal pressure and equal
  fugacity (Eq. 9 and Eq. 12 with N = 1).
* ``flash``: two-phase PT flash, the "theoretical prediction" the paper
  compares against (Sec. 3.2): Wilson start, Rachford-Rice for the vapour
  fraction, the PR cubic for each phase's compressibility and successive
  substitution K_i <- phi_i^L / phi_i^V until the fugacities are equal.
* ``hessian_lnf``: d ln f_i / d rho~_j, whose smallest eigenvalue going
  negative marks the spinodal region used by the spinodal-decomposition runs
  (Sec. 3.5).

All of it evaluates the EOS through the C oracle (``OracleProblem.eos``); the
cubic in Z is solved here and its roots are checked against the C pressure.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq

from .orc import OracleProblem

R_SI = 8.314462618  # J/(mol K); the paper does not print the value it used
OMEGA_A = 0.457235529
OMEGA_B = 0.077796074


# ---------------------------------------------------------------------------
# unit conversion (Sec. 3.1: R = 1, a_C1 = 2/49, b_C1 = 2/21, M_C1 = 1)
# ---------------------------------------------------------------------------
class LatticeUnits:
    """Maps physical PR components to lattice units.

    Physical a_i = 0.457235529 R^2 Tc^2/pc, b_i = 0.077796074 R Tc/pc
    (Sec. 2.3).  With a reference component fixed to (a_ref, b_ref, M_ref) in
    lattice units and R = 1, the molar-volume scale is V* = b_phys/b_lat, the
    molar-energy scale E* = a_phys/(a_lat V*), temperatures map as
    T_lat = R T / E* and pressures as p_lat = p V* / E*.
    """

    def __init__(self, Tc, pc_bar, omega, M, ref=0, a_ref=2.0 / 49.0, b_ref=2.0 / 21.0):
        self.Tc = np.asarray(Tc, float)
        self.pc = np.asarray(pc_bar, float) * 1e5
        self.omega = np.asarray(omega, float)
        self.Mphys = np.asarray(M, float)  # g/mol
        a_phys = OMEGA_A * R_SI ** 2 * self.Tc ** 2 / self.pc
        b_phys = OMEGA_B * R_SI * self.Tc / self.pc
        self.V = b_phys[ref] / b_ref
        self.E = a_phys[ref] / (a_ref * self.V)
        self.a = a_phys / (self.E * self.V)
        self.b = b_phys / self.V
        self.M = self.Mphys / self.Mphys[ref]
        self.ref = ref

    def T(self, T_kelvin):
        return R_SI * T_kelvin / self.E

    def p(self, p_bar):
        return p_bar * 1e5 * self.V / self.E

    def p_to_bar(self, p_lat):
        return p_lat * self.E / self.V / 1e5

    def mass_density_kg_m3(self, rho_molar_lat_i):
        """kg/m^3 of a phase from lattice molar densities rho~_i (per component)."""
        rho = np.asarray(rho_molar_lat_i, float)
        return float(np.sum(rho / self.V * self.Mphys / 1000.0))

    def problem(self, T_kelvin, kij=None, lattice=0, nx=1, ny=1, nz=1, tau=1.0, kappa_ref=0.02):
        return OracleProblem(lattice, nx, ny, nz, self.a, self.b, self.omega, kij, self.T(T_kelvin),
                             tau, M=self.M, R=1.0, kappa_ref=kappa_ref, kappa_ref_index=self.ref)


# ---------------------------------------------------------------------------
# PR cubic in Z at given (T, p, x)
# ---------------------------------------------------------------------------
def _mix(P: OracleProblem, x):
    aal = P.a * P.alpha()
    A = np.sqrt(np.outer(aal, aal)) * (1.0 - P.kij)
    return float(x @ A @ x), float(x @ P.b)


def z_roots(P: OracleProblem, p, x):
    """Real roots Z > B of the PR cubic at (T, p, x), ascending."""
    RT = P.R * P.T
    aam, bm = _mix(P, x)
    A = aam * p / RT ** 2
    B = bm * p / RT
    coeffs = [1.0, -(1.0 - B), A - 3.0 * B * B - 2.0 * B, -(A * B - B * B - B ** 3)]
    r = np.roots(coeffs)
    real = np.sort(r[np.abs(r.imag) < 1e-10].real)
    real = real[real > B]
    # polish with Newton on the cubic
    out = []
    for z in real:
        for _ in range(4):
            f = ((z + coeffs[1]) * z + coeffs[2]) * z + coeffs[3]
            df = (3 * z + 2 * coeffs[1]) * z + coeffs[2]
            if df == 0:
                break
            z -= f / df
        out.append(z)
    return np.array(out), B


def phase_state(P: OracleProblem, p, x, phase):
    """(rho~ total, ln phi_i) of the liquid ('L': smallest Z) or vapour ('V': largest Z) root."""
    Z, B = z_roots(P, p, x)
    if Z.size == 0:
        raise ValueError("no physical PR root")
    z = Z[0] if phase == "L" else Z[-1]
    rho = p / (z * P.R * P.T)
    pc, lnf = P.eos(x * rho)
    if abs(pc - p) > 1e-9 * max(abs(p), 1e-300):
        raise AssertionError(f"cubic root inconsistent with Eq. (9): {pc} vs {p}")
    lnphi = lnf - np.log(x * p)
    return rho, lnphi


# ---------------------------------------------------------------------------
# Maxwell construction (N = 1)
# ---------------------------------------------------------------------------
def spinodal_densities(P: OracleProblem):
    """Densities where dp/drho~ = 0 for a single component (None if supercritical)."""
    assert P.nc == 1
    bmax = 1.0 / P.b[0]
    grid = np.linspace(1e-6 * bmax, 0.999 * bmax, 20001)
    ps = np.array([P.eos([r])[0] for r in grid])
    dp = np.diff(ps)
    idx = np.where(np.sign(dp[1:]) != np.sign(dp[:-1]))[0]
    if len(idx) < 2:
        return None
    def dpdr(r):
        h = 1e-7 * r
        return (P.eos([r + h])[0] - P.eos([r - h])[0]) / (2 * h)
    r1 = brentq(dpdr, grid[idx[0]], grid[idx[0] + 2])
    r2 = brentq(dpdr, grid[idx[1]], grid[idx[1] + 2])
    return r1, r2


def maxwell(P: OracleProblem):
    """(p_sat, rho~_V, rho~_L) of a pure component: equal p (Eq. 9) and equal ln f (Eq. 12)."""
    sp = spinodal_densities(P)
    if sp is None:
        raise ValueError("no two-phase region at this temperature")
    r1, r2 = sp
    p_hi = P.eos([r1])[0]
    p_lo = max(P.eos([r2])[0], 1e-12 * p_hi)
    x = np.ones(1)

    def dlnf(p):
        Z, _ = z_roots(P, p, x)
        rV = p / (Z[-1] * P.R * P.T)
        rL = p / (Z[0] * P.R * P.T)
        return P.eos([rL])[1][0] - P.eos([rV])[1][0]

    lo, hi = p_lo * (1 + 1e-9), p_hi * (1 - 1e-9)
    psat = brentq(dlnf, lo, hi, xtol=1e-15 * p_hi, rtol=1e-15, maxiter=500)
    Z, _ = z_roots(P, psat, x)
    return psat, psat / (Z[-1] * P.R * P.T), psat / (Z[0] * P.R * P.T)


# ---------------------------------------------------------------------------
# Two-phase PT flash
# ---------------------------------------------------------------------------
def wilson_k(P: OracleProblem, p):
    Tc = P.critical_temperatures()
    pc = OMEGA_B * P.R * Tc / P.b
    return pc / p * np.exp(5.373 * (1.0 + P.omega) * (1.0 - Tc / P.T))


def rachford_rice(z, K):
    """Vapour mole fraction beta of sum_i z_i (K_i - 1)/(1 + beta (K_i - 1)) = 0."""
    def f(beta):
        return float(np.sum(z * (K - 1.0) / (1.0 + beta * (K - 1.0))))
    kmax, kmin = K.max(), K.min()
    if kmax <= 1.0 or kmin >= 1.0:
        return None
    lo = 1.0 / (1.0 - kmax)
    hi = 1.0 / (1.0 - kmin)
    eps = 1e-14 * (hi - lo)
    try:
        return brentq(f, lo + eps, hi - eps, xtol=1e-16, rtol=1e-15, maxiter=500)
    except ValueError:
        return None  # no sign change resolvable between the asymptotes


class FlashResult(dict):
    __getattr__ = dict.__getitem__


def flash(P: OracleProblem, p, z, tol=1e-12, maxit=10000, K0=None):
    """Two-phase split of overall composition z at (T, p).

    Returns a FlashResult with beta (vapour mole fraction), x (liquid), y
    (vapour), rho_L, rho_V (total molar densities), rhoi_L, rhoi_V (per
    component), S_V (vapour volume fraction), iterations and the final
    max |ln f_i^L - ln f_i^V|; or None if no two-phase split is found.
    """
    z = np.asarray(z, float)
    z = z / z.sum()
    K = wilson_k(P, p) if K0 is None else np.asarray(K0, float)
    beta = None
    for it in range(1, maxit + 1):
        beta = rachford_rice(z, K)
        if beta is None:
            return None
        # beta may leave (0, 1) during the iteration (negative flash); only
        # the converged value decides whether z splits at this (T, p)
        x = z / (1.0 + beta * (K - 1.0))
        y = K * x
        x /= x.sum()
        y /= y.sum()
        rL, lnphiL = phase_state(P, p, x, "L")
        rV, lnphiV = phase_state(P, p, y, "V")
        lnfL = lnphiL + np.log(x * p)
        lnfV = lnphiV + np.log(y * p)
        err = float(np.max(np.abs(lnfL - lnfV)))
        K = np.exp(lnphiL - lnphiV)
        if err < tol:
            break
        if np.max(np.abs(np.log(K))) < 1e-6:
            return None  # trivial solution
    else:
        return None
    if not (0.0 < beta < 1.0):
        return None
    vV = beta / rV
    vL = (1.0 - beta) / rL
    return FlashResult(beta=beta, x=x, y=y, rho_L=rL, rho_V=rV, rhoi_L=x * rL, rhoi_V=y * rV,
                       S_V=vV / (vV + vL), iterations=it, residual=err, K=K)


# ---------------------------------------------------------------------------
# Multiphase PT flash (three-phase case of Sec. 3.4), textbook successive
# substitution: K-values of every phase against a reference phase, phase
# fractions from the multiphase Rachford-Rice equations, ln phi of each phase
# from its own cubic root.
# ---------------------------------------------------------------------------
def rachford_rice_multi(z, K, beta0):
    """Phase fractions beta[k] of the non-reference phases, K[k, i] = x_{k,i} / x_{ref,i}:
    the roots of g_k = sum_i z_i (K_{k,i} - 1) / t_i, t_i = 1 + sum_m beta_m (K_{m,i} - 1)
    (the reference phase takes 1 - sum beta).  Newton's method with step halving that
    keeps every t_i positive; None if it does not converge."""
    beta = np.array(beta0, float)
    D = K - 1.0
    for _ in range(200):
        t = 1.0 + beta @ D
        g = D @ (z / t)
        H = -(D * (z / t ** 2)) @ D.T
        try:
            step = np.linalg.solve(H, g)
        except np.linalg.LinAlgError:
            return None
        lam = 1.0
        feasible = False
        while lam > 1e-12:
            nb = beta - lam * step
            if np.all(1.0 + nb @ D > 0.0):
                feasible = True
                break
            lam *= 0.5
        if not feasible:  # no step keeps every t_i > 0: the split is not found
            return None
        beta = nb
        if np.max(np.abs(lam * step)) < 1e-15:
            break
    t = 1.0 + beta @ D
    if np.max(np.abs(D @ (z / t))) > 1e-12:
        return None
    return beta


def flash3(P: OracleProblem, p, z, guesses, phases, tol=1e-12, maxit=20000):
    """Multiphase split of overall composition z at (T, p) by successive
    substitution.  guesses: starting compositions of the phases; phases: their
    cubic roots ('V' largest Z, 'L' smallest Z).  The last phase is the
    reference.  Returns a FlashResult with beta (mole fraction of each phase),
    x (compositions), rho (total molar densities), rhoi (per component), S
    (volume fractions), iterations and the final max |ln f_{k,i} - ln f_{ref,i}|;
    None if a phase vanishes or the iteration does not converge."""
    z = np.asarray(z, float)
    z = z / z.sum()
    n = len(phases)
    x = [np.asarray(g, float) / np.sum(g) for g in guesses]
    beta = np.full(n - 1, 1.0 / n)
    for it in range(1, maxit + 1):
        st = [phase_state(P, p, x[k], phases[k]) for k in range(n)]
        lnphi = np.array([s[1] for s in st])
        lnf = lnphi + np.log(np.array(x) * p)
        err = float(np.max(np.abs(lnf[:-1] - lnf[-1])))
        if err < tol:
            break
        K = np.exp(lnphi[-1] - lnphi[:-1])  # x_k / x_ref
        beta = rachford_rice_multi(z, K, beta)
        if beta is None:
            return None
        xr = z / (1.0 + beta @ (K - 1.0))
        x = [K[k] * xr for k in range(n - 1)] + [xr]
        x = [xi / xi.sum() for xi in x]
    else:
        return None
    b = np.append(beta, 1.0 - beta.sum())
    if np.any(b <= 0.0):
        return None
    rho = np.array([s[0] for s in st])
    v = b / rho
    return FlashResult(beta=b, x=np.array(x), rho=rho, rhoi=np.array(x) * rho[:, None], S=v / v.sum(),
                       iterations=it, residual=err)


# ---------------------------------------------------------------------------
# spinodal test: d ln f_i / d rho~_j
# ---------------------------------------------------------------------------
def hessian_lnf(P: OracleProblem, rho_molar, rel_step=1e-6):
    """Central-difference Jacobian J_ij = d ln f_i / d rho~_j at rho~ (symmetrised)."""
    r = np.asarray(rho_molar, float)
    n = r.size
    J = np.zeros((n, n))
    for j in range(n):
        h = rel_step * max(r[j], 1e-12)
        rp = r.copy(); rp[j] += h
        rm = r.copy(); rm[j] -= h
        J[:, j] = (P.eos(rp)[1] - P.eos(rm)[1]) / (2 * h)
    return 0.5 * (J + J.T)


def min_stability_eigenvalue(P: OracleProblem, rho_molar):
    """Smallest eigenvalue of diag(rho~) J, i.e. of the Helmholtz Hessian scaled by
    rho~_i; negative inside the spinodal region."""
    r = np.asarray(rho_molar, float)
    J = hessian_lnf(P, r)
    s = np.sqrt(r)
    return float(np.linalg.eigvalsh(s[:, None] * J * s[None, :]).min())
