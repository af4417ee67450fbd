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


# ---------------------------------------------------------------------------------------
# Eq. e:dtss: the substep bounds the change of x_n (Sec. 2.3: "C = 0.1 restricts the change
# of x_n per substep to below 0.1")
# ---------------------------------------------------------------------------------------

def _rate_of_change(xn, gamma, nH, alpha):
    """|dx_n/dt| at the start of a substep, the right-hand side of Eq. e:xn with
    n_e = n_H (1 - x_n): alpha n_e (1 - x_n) - x_n Gamma."""
    ne = nH * (1.0 - xn)
    return np.abs(alpha * ne * (1.0 - xn) - xn * gamma)


def _transition_fields(n, seed):
    """Cells of a transition layer (0.1 < x_n < 1 with x_eq near 0, where the paper says the
    minimum substep usually comes from) mixed with ionized, neutral and shielded cells."""
    rng = np.random.default_rng(seed)
    nH = 10.0 ** rng.uniform(-1, 3, n)
    xn = rng.uniform(0.1, 1.0, n)
    gamma = 10.0 ** rng.uniform(-2, 3, n)
    k = n // 4
    xn[:k] = 10.0 ** rng.uniform(-6, -2, k)         # ionized
    gamma[k:2 * k] = 0.0                             # shielded
    xn[2 * k:2 * k + 8] = 1.0                        # fully neutral
    return xn, gamma, nH


@pytest.mark.parametrize("C", [0.1, 0.3])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dtss_bounds_method_b_change(C, seed):
    """Over one substep of Eq. e:dtss, Method B (Eq. e:xn3) moves x_n by at most C in every
    cell: it relaxes exponentially, so |dx| = |x0 - x_eq0| (1 - e^{-y}) <= |dx/dt(0)| dt. The
    limiting cell of a transition layer moves by C (1 - e^{-y})/y >= C/2 (y <= 1)."""
    alpha = 2e-3
    xn, gamma, nH = _transition_fields(20_000, seed)
    dt = O.dt_substep(xn, gamma, nH, alpha, C=C)
    x1 = O.xn_method_b(xn, gamma, nH, alpha, dt)
    change = np.abs(x1 - xn)
    assert change.max() <= C * (1 + 1e-12)
    rate = _rate_of_change(xn, gamma, nH, alpha)
    # the substep is the time in which the fastest-changing cell moves by C at its
    # initial rate
    assert rate.max() * dt == pytest.approx(C, rel=1e-12)
    lim = int(np.argmax(rate))
    assert 0.1 <= xn[lim] <= 1.0
    ne = nH[lim] * (1.0 - xn[lim])
    t_ir = 1.0 / (gamma[lim] + alpha * ne)
    y = dt / t_ir
    assert change[lim] == pytest.approx(C * -np.expm1(-y) / y, rel=1e-9)
    assert change[lim] >= 0.5 * C


def test_dtss_misreadings_fail_the_bound():
    """Plausible misreadings of Eq. e:dtss (n_HI for n_H in the numerator, I = n_H Gamma
    without x_n) give substeps whose fastest cell does not move by C at its initial rate."""
    alpha, C = 2e-3, 0.1
    xn, gamma, nH = _transition_fields(5000, 7)
    rate = _rate_of_change(xn, gamma, nH, alpha)
    ne = nH * (1 - xn)
    R = alpha * ne * ne
    wrong_num = C * np.min(xn * nH / np.abs(xn * nH * gamma - R))
    wrong_I = C * np.min(nH / np.abs(nH * gamma - R))
    for dt in (wrong_num, wrong_I):
        assert abs(rate.max() * dt - C) > 1e-3 * C
    assert rate.max() * O.dt_substep(xn, gamma, nH, alpha, C=C) == pytest.approx(C, rel=1e-12)


def test_dtss_infinite_at_equilibrium():
    """Cells already in ionization balance (I = R) do not limit the substep; with every cell
    balanced the substep is unbounded."""
    nH = np.array([1.0, 30.0, 0.2])
    xn = np.array([0.5, 0.1, 0.9])
    alpha = 0.7
    gamma = alpha * (nH * (1 - xn)) ** 2 / (xn * nH)
    assert O.dt_substep(xn, gamma, nH, alpha, C=0.1) == np.inf


# ---------------------------------------------------------------------------------------
# Eq. e:bdf1 (Appendix, Method C)
# ---------------------------------------------------------------------------------------

def test_method_c_solves_its_difference_equation():
    """Eq. e:bdf1 is the solution of the Appendix's semi-implicit difference equation
    (x1 - x0)/dt = alpha n_H (1 - x0)^2 - x1 Gamma."""
    rng = np.random.default_rng(4)
    x0 = rng.random(500)
    gamma = 10.0 ** rng.uniform(-3, 2, 500)
    nH = 10.0 ** rng.uniform(-1, 2, 500)
    alpha, dt = 0.03, 10.0 ** rng.uniform(-3, 1, 500)
    x1 = O.xn_method_c(x0, gamma, nH, alpha, dt)
    lhs = (x1 - x0) / dt
    rhs = alpha * nH * (1 - x0) ** 2 - x1 * gamma
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-12 * np.abs(x0 / dt).max())


def test_method_c_fixed_point_is_the_equilibrium():
    """The fixed point of Eq. e:bdf1 is the equilibrium of Eq. e:xn for any substep."""
    gamma = np.array([1e-3, 0.5, 20.0])
    nH, alpha = 3.0, 0.2
    xeq = O.xn_equilibrium(gamma, nH, alpha)
    # the equilibrium zeroes the right-hand side of Eq. e:xn
    np.testing.assert_allclose(alpha * nH * (1 - xeq) ** 2, xeq * gamma, rtol=1e-12)
    for dt in (1e-4, 0.3, 50.0):
        np.testing.assert_allclose(O.xn_method_c(xeq, gamma, nH, alpha, dt), xeq, rtol=1e-12)


def _one_cell_run(method, C, g, t_end, sample_t):
    nH, alpha = g["n_H"], g["alpha_B"]
    x, t, out = np.array([1.0]), 0.0, {}
    targets = list(sample_t)
    while targets:
        gam = _one_cell_gamma(x[0], g)
        dt = min(O.dt_substep(x, np.array([gam]), nH, alpha, C=C), targets[0] - t)
        x = method(x, np.array([gam]), nH, alpha, dt)
        t += dt
        if abs(t - targets[0]) <= 1e-12 * targets[0]:
            out[targets.pop(0)] = x[0]
    return out


def test_one_cell_method_c_first_order_and_less_accurate():
    """Appendix one-cell test: Method C (Eq. e:bdf1) converges to the solution of Eq. e:xn
    at first order in C, and at the same C it is less accurate than Methods A and B."""
    g = GOLD["one_cell"]
    a = g["alpha_B"] * g["n_H"]
    t_scale = 1.0 / _one_cell_gamma(1.0, g)
    sample_t = [k * 0.25 * t_scale for k in range(1, 13)]

    def rhs(_, x):
        return [a * (1 - x[0]) ** 2 - x[0] * _one_cell_gamma(max(x[0], 1e-12), g)]
    ref = solve_ivp(rhs, (0, sample_t[-1]), [1.0], rtol=1e-11, atol=1e-15, method="LSODA",
                    dense_output=True)

    def err(method, C):
        out = _one_cell_run(method, C, g, sample_t[-1], sample_t)
        return max(abs(out[t] - ref.sol(t)[0]) for t in sample_t)

    # Gamma is held at its start-of-substep value in every method, so all three are first
    # order in the substep; in the asymptotic range halving C halves Method C's error
    e_c = {C: err(O.xn_method_c, C) for C in (0.01, 0.005, 0.0025)}
    assert 1.6 < e_c[0.01] / e_c[0.005] < 2.4
    assert 1.6 < e_c[0.005] / e_c[0.0025] < 2.4
    # the Appendix: Methods A and B are more accurate than Method C at the same C
    for C in (1.0, 0.1, 0.01):
        ec = err(O.xn_method_c, C)
        assert err(O.xn_method_a, C) < 0.8 * ec
        assert err(O.xn_method_b, C) < 0.8 * ec
