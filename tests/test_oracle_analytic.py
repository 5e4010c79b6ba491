"""Analytic pins of the oracle: closed-form solutions of Eqs. 1-5.

* Semi-infinite solid with a convective (Robin) surface, Eq. 4: the
  classical erfc solution; the error must be small and fall ~4x when the
  element size halves (dt scales with h^2).
* The same solid with a fixed surface temperature, Eq. 3: erf solution.
* Neumann's two-phase Stefan problem with isothermal freezing (Eq. 5 in the
  isothermal limit): front position 2 lambda sqrt(alpha t).
* Explicit stability (Eq. 13): the Gershgorin step is below 2/lambda_max of
  C^{-1}(K + H), 0.95 x 2/lambda_max stays bounded, 1.05 x diverges.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from paper_1005_3158_gb300 import meshgen as mg

RHO, CP, K = 2700.0, 900.0, 150.0
ALPHA = K / (RHO * CP)


def _bar_problem(n, length, mats, robin_h=None, t_inf=300.0, dirichlet_T=None, T0=973.0):
    xyz, tets, flags, _ = mg.bar(n, length)
    faces = np.zeros((0, 3), np.int32)
    h = t_inf_a = q = np.zeros(0)
    if robin_h is not None:
        faces = mg.box_boundary_faces(tets, flags, plane_mask=1)
        h = np.full(len(faces), robin_h)
        t_inf_a = np.full(len(faces), t_inf)
        q = np.zeros(len(faces))
    p = mg.Problem(xyz=xyz, tets=tets, mat=np.zeros(len(tets), np.int32),
                   materials=np.asarray(mats, float).reshape(1, 6), faces=faces, h=h,
                   t_inf=t_inf_a, q=q, T0=np.full(len(xyz), T0))
    if dirichlet_T is not None:
        d = np.nonzero(xyz[:, 0] < 1e-12)[0].astype(np.int32)
        p.dir_nodes = d
        p.dir_T = np.full(len(d), dirichlet_T)
    return p


def _run_to(o, t_end, frac=0.5):
    dt_max = frac * o.stable_dt()
    n = int(math.ceil(t_end / dt_max))
    o.step(n, t_end / n)
    return n


def _robin_exact(x, t, h, Ti, Tinf):
    s = math.sqrt(ALPHA * t)
    eta = x / (2 * s)
    b = h * s / K
    # exp(hx/k + b^2) erfc(eta + b) = erfcx(eta + b) exp(hx/k + b^2 - (eta+b)^2)
    term = special.erfcx(eta + b) * np.exp(h * x / K + b * b - (eta + b) ** 2)
    theta = special.erfc(eta) - term
    return Ti + (Tinf - Ti) * theta


def test_erfc_robin_slab_convergence():
    length, t_end, h, Ti, Tinf = 0.6, 150.0, 1000.0, 973.0, 300.0
    errs = []
    for n in (24, 48):
        p = _bar_problem(n, length, (RHO, CP, K, 0.0, 0.0, 0.0), robin_h=h, t_inf=Tinf, T0=Ti)
        o = oracle.OracleProblem(p)
        o.set_temperature(p.T0)
        _run_to(o, t_end)
        T = o.temperature()
        ex = _robin_exact(p.xyz[:, 0], o.time, h, Ti, Tinf)
        errs.append(np.abs(T - ex).max() / (Ti - Tinf))
    assert errs[0] < 5e-3
    assert 3.0 < errs[0] / errs[1] < 5.5


def test_erf_dirichlet_slab_convergence():
    length, t_end, Tw, Ti = 0.6, 150.0, 300.0, 973.0
    errs = []
    for n in (24, 48):
        p = _bar_problem(n, length, (RHO, CP, K, 0.0, 0.0, 0.0), dirichlet_T=Tw, T0=Ti)
        o = oracle.OracleProblem(p)
        o.set_temperature(p.T0)
        _run_to(o, t_end)
        T = o.temperature()
        eta = p.xyz[:, 0] / (2 * math.sqrt(ALPHA * o.time))
        ex = Tw + (Ti - Tw) * special.erf(eta)
        errs.append(np.abs(T - ex).max() / (Ti - Tw))
    assert errs[0] < 2e-2
    assert errs[1] < errs[0] / 2.5


def _neumann_lambda(Ti, Tm, Tw, L, c):
    st = c * (Tm - Tw) / L
    r = (Ti - Tm) / (Tm - Tw)

    def g(lam):
        e = math.exp(-lam * lam)
        return e / math.erf(lam) - r * e / math.erfc(lam) - lam * math.sqrt(math.pi) / st

    lo, hi = 1e-6, 5.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_neumann_stefan_front():
    Tm, Ti, Tw, L = 933.0, 973.0, 300.0, 3.9e5
    lam = _neumann_lambda(Ti, Tm, Tw, L, CP)
    length, t_end = 0.6, 180.0
    front_err = []
    for n in (30, 60):
        p = _bar_problem(n, length, (RHO, CP, K, L, Tm, Tm), dirichlet_T=Tw, T0=Ti)
        o = oracle.OracleProblem(p)
        o.set_temperature(p.T0)
        _run_to(o, t_end)
        C, _, Lc = o.lumped()
        E = o.enthalpy()
        fl = np.clip((E - C * Tm) / Lc, 0.0, 1.0)
        x = p.xyz[:, 0]
        xs = np.unique(np.round(x, 12))
        fs = np.array([fl[np.abs(x - xv) < 1e-9].mean() for xv in xs])
        k = int(np.nonzero(fs >= 0.5)[0][0])
        xf = xs[k - 1] + (0.5 - fs[k - 1]) / (fs[k] - fs[k - 1]) * (xs[k] - xs[k - 1])
        X = 2 * lam * math.sqrt(ALPHA * o.time)
        front_err.append(abs(xf - X))
        hsz = length / n
        assert abs(xf - X) < hsz
        # solid region temperature against the analytic profile
        solid = x < 0.8 * X
        Ts_ex = Tw + (Tm - Tw) * special.erf(x[solid] / (2 * math.sqrt(ALPHA * o.time))) / math.erf(lam)
        assert np.abs(o.temperature()[solid] - Ts_ex).max() < 0.03 * (Tm - Tw)
    assert front_err[1] < front_err[0]


def _dense_A(p, o):
    C, _, _ = o.lumped()
    n = p.n_nodes
    M = np.zeros((n, n))
    # columns of F - (K+H) T as a linear map: R(T) - R(0)
    R0, _ = o.residual(np.zeros(n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Rj, _ = o.residual(e)
        M[:, j] = -(Rj - R0)
    return M, C, R0


def test_stability_limit():
    p = mg.random_small(12, nx=4, ny=3, nz=3)
    mats = p.materials.copy()
    mats[:, 3] = 0.0          # linear (sensible-only) problem
    p.materials = mats
    o = oracle.OracleProblem(p)
    M, C, R0 = _dense_A(p, o)
    s = 1.0 / np.sqrt(C)
    lam_max = np.linalg.eigvalsh(s[:, None] * M * s[None, :]).max()
    dt_eig = 2.0 / lam_max
    dt_g = o.stable_dt()
    assert dt_g <= dt_eig * (1 + 1e-12)
    assert dt_g > 0.2 * dt_eig
    # steady state of the linear problem
    T_ss = np.linalg.solve(M, R0)
    growth = {}
    for fac in (0.95, 1.05):
        o.set_temperature(p.T0)
        o.step(600, fac * dt_eig)
        growth[fac] = np.abs(o.temperature() - T_ss).max() / np.abs(p.T0 - T_ss).max()
    assert growth[0.95] < 1.0
    assert growth[1.05] > 1e6
