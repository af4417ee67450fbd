"""Pins of the oracle's neutral-fraction updates (Sec. 2.3, Appendix) against numerical
integration of Eq. e:xn (scipy, tight tolerances) and the numbers the paper prints."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _ode(x0, gamma, nH, alpha, t, ne_fixed=None):
    def f(_, x):
        ne = ne_fixed if ne_fixed is not None else nH * (1 - x[0])
        return [alpha * ne * (1 - x[0]) - x[0] * gamma]
    sol = solve_ivp(f, (0, t), [x0], rtol=1e-12, atol=1e-15, method="LSODA")
    return sol.y[0, -1]


CASES = [(0.9, 3e-3, 2.0, 1e-3, 50.0), (1e-3, 0.0, 100.0, 2e-4, 20.0),
         (0.3, 0.5, 10.0, 0.02, 3.0), (1.0, 1e-2, 1.0, 1e-2, 400.0)]


@pytest.mark.parametrize("x0,gamma,nH,alpha,t", CASES)
def test_method_b_is_exact_for_fixed_electron_density(x0, gamma, nH, alpha, t):
    ne = nH * (1 - x0)
    want = _ode(x0, gamma, nH, alpha, t, ne_fixed=ne)
    assert O.xn_method_b(np.array([x0]), gamma, nH, alpha, t)[0] == pytest.approx(want, rel=1e-8, abs=1e-13)


@pytest.mark.parametrize("x0,gamma,nH,alpha,t", CASES)
def test_method_a_is_exact(x0, gamma, nH, alpha, t):
    want = _ode(x0, gamma, nH, alpha, t)
    got = O.xn_method_a(np.array([x0]), np.array([gamma]), nH, alpha, t)[0]
    assert got == pytest.approx(want, rel=1e-7, abs=1e-12)


def test_gamma_zero_solution():
    for x0, a, t in [(0.0, 1.0, 0.5), (0.2, 3.0, 2.0), (1e-4, 1e-2, 10.0)]:
        want = _ode(x0, 0.0, a, 1.0, t)
        assert O.xn_gamma_zero(x0, a, t) == pytest.approx(want, rel=1e-9)


def test_method_b_bounded_between_start_and_equilibrium():
    rng = np.random.default_rng(1)
    x0 = rng.random(1000)
    g = rng.random(1000) * 2
    x1 = O.xn_method_b(x0, g, 1.0, 0.3, 0.7)
    ne = 1.0 * (1 - x0)
    xeq = 0.3 * ne / (g + 0.3 * ne)
    assert np.all((x1 - x0) * (x1 - xeq) <= 1e-15)


def _one_cell_gamma(x, g):
    pc = GOLD["constants"]["pc_cm"]
    dx = g["dx_pc"] * pc
    tau = g["n_H"] * x * g["sigma_H"] * dx
    return g["Q_i"] / (dx**3) * (-math.expm1(-tau)) / (g["n_H"] * x)


def test_one_cell_numbers():
    g = GOLD["one_cell"]
    pc = GOLD["constants"]["pc_cm"]
    dx = g["dx_pc"] * pc
    tau0 = g["n_H"] * g["sigma_H"] * dx
    assert tau0 == pytest.approx(g["tau0"], rel=0.01)
    gamma0 = _one_cell_gamma(1.0, g)
    assert gamma0 / (g["alpha_B"] * g["n_H"]) == pytest.approx(g["gamma0_over_alpha_nH"], rel=0.02)
    # the printed 1.7e-6 is the optically thin rate sigma_H Q / dx^2
    assert g["sigma_H"] * g["Q_i"] / dx**2 == pytest.approx(g["printed_gamma0"], rel=0.05)
    # equilibrium of Eq. e:xn with the cell's self-shielded rate
    a = g["alpha_B"] * g["n_H"]
    # the paper's estimate alpha_B n_H / (Gamma0 tau0)
    assert a / (gamma0 * tau0) == pytest.approx(g["x_eq"], rel=0.03)
    # the exact equilibrium sits where the cell is already thin (tau ~ 0.07), a few per cent
    # above that estimate
    xeq = brentq(lambda x: a * (1 - x) ** 2 - x * _one_cell_gamma(x, g), 1e-9, 0.5, xtol=1e-16)
    assert xeq == pytest.approx(g["x_eq"], rel=0.08)


def test_one_cell_methods_a_b_agree_with_ode():
    """Appendix: with C = 0.001, methods A and B both follow the true solution."""
    g = GOLD["one_cell"]
    a = g["alpha_B"] * g["n_H"]
    nH, alpha = g["n_H"], g["alpha_B"]
    t_end = 3.0 / _one_cell_gamma(1.0, g)

    def rhs(_, x):
        return [a * (1 - x[0]) ** 2 - x[0] * _one_cell_gamma(max(x[0], 1e-12), g)]
    ref = solve_ivp(rhs, (0, t_end), [1.0], rtol=1e-10, atol=1e-14, method="LSODA",
                    dense_output=True)
    for method in (O.xn_method_a, O.xn_method_b):
        x, t = np.array([1.0]), 0.0
        while t < t_end:
            gam = _one_cell_gamma(x[0], g)
            dt = min(O.dt_substep(x, np.array([gam]), nH, alpha, C=1e-3), t_end - t)
            x = method(x, np.array([gam]), nH, alpha, dt)
            t += dt
        assert x[0] == pytest.approx(ref.sol(t_end)[0], rel=0.02)


def test_dt_substep_definition():
    xn = np.array([0.5, 0.9, 1e-3])
    gam = np.array([1.0, 0.0, 2.0])
    nH, alpha = 10.0, 0.1
    I = xn * nH * gam
    ne = nH * (1 - xn)
    R = alpha * ne * ne
    assert O.dt_substep(xn, gam, nH, alpha, C=0.1) == pytest.approx(0.1 * np.min(nH / np.abs(I - R)))


def test_stromgren_radius_numbers():
    g = GOLD["rtype_front"]
    pc = GOLD["constants"]["pc_cm"]
    R = (3 * g["Q_i"] / (4 * math.pi * g["alpha_B"] * g["n_H"] ** 2)) ** (1 / 3)
    assert g["box_pc"] / (R / pc) == pytest.approx(g["box_over_R_St"], rel=0.01)
    dtau = g["n_H"] * g["sigma_H"] * g["box_pc"] * pc / 128
    assert dtau == pytest.approx(g["dtau_cell_128"], rel=0.01)


def test_stromgren_sphere_equilibrium():
    """Trace + Eq. e:xn3 iterated to equilibrium around one source in a uniform medium
    (Sec. 3.3.1 set-up in code units: R_St = 1, t_rec = 1, box 2.4 R_St, dtau per neutral cell
    109 (128/N)): the ionized volume matches (3Q/(4 pi alpha n^2))^(1/3) and recombinations
    balance the source (the dust-free photon budget of Eq. e:xn at equilibrium)."""
    g = GOLD["rtype_front"]
    N, side, nH, alpha = 32, g["box_over_R_St"], 1.0, 1.0
    Q = 4 * math.pi / 3  # R_St = 1
    dx = side / N
    sigma = g["dtau_cell_128"] * (128 / N) / (nH * dx)
    pos = np.array([[(N // 2 + 0.5) * dx] * 3])
    xn = np.ones((N, N, N))
    for _ in range(80):
        prob = O.Problem(nH0=(xn * nH).astype(np.float32), pos=pos, L=[Q], dx=dx,
                         sigma_H=sigma, level0=4, tau_max=30.0)
        r = O.trace(prob, nthreads=4)
        xn = O.xn_method_b(xn, r.gamma, nH, alpha, 0.5)
    R = (3 * (xn < 0.5).sum() * dx**3 / (4 * math.pi)) ** (1 / 3)
    rec = (alpha * (nH * (1 - xn)) ** 2).sum() * dx**3
    assert R == pytest.approx(1.0, rel=0.02)
    assert rec / Q == pytest.approx(1.0, rel=1e-3)
