"""Pins of the oracle's traversal, attenuation, splitting and whole-field results (Sec. 2.1).

Each test compares against something other than the oracle's own formulas: brute-force
dense sampling of the ray, hand-computed visit sequences, exact geometric exit lengths,
exact photon bookkeeping, the paper's split radius and ray counts, the r^-2 vacuum law
with the accuracy the paper reports, and FP64 quadrature of the exact cell averages in a
uniform medium.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _prob(n, nH0=None, pos=((0.5, 0.5, 0.5),), L=(1.0,), **kw):
    if nH0 is None:
        nH0 = np.zeros((n, n, n))
    return O.Problem(nH0=nH0, pos=np.asarray(pos, float), L=np.asarray(L, float), dx=1.0 / n, **kw)


def _exit_length(u, v, n):
    """Distance (cell units) from u along unit v to the box [0, n]^3."""
    t = math.inf
    for a in range(3):
        if v[a] > 0:
            t = min(t, (n - u[a]) / v[a])
        elif v[a] < 0:
            t = min(t, -u[a] / v[a])
    return t


def _brute(u, v, n, tmax, samples):
    """Per-cell path lengths by dense midpoint sampling of x = u + t v, t in [0, tmax]."""
    dt = tmax / samples
    t = (np.arange(samples) + 0.5) * dt
    p = u[None, :] + t[:, None] * v[None, :]
    c = np.floor(p).astype(np.int64)
    inside = np.all((c >= 0) & (c < n), axis=1)
    idx = c[inside, 0] + n * (c[inside, 1] + n * c[inside, 2])
    cells, counts = np.unique(idx, return_counts=True)
    return dict(zip(cells.tolist(), (counts * dt).tolist()))


def test_brute_force_path_lengths():
    rng = np.random.default_rng(11)
    n = 8
    for trial in range(12):
        u = rng.uniform(0.5, n - 0.5, 3)
        R = np.linalg.qr(rng.standard_normal((3, 3)))[0]
        if np.linalg.det(R) < 0:
            R[:, 0] *= -1
        level = 2
        pix = int(rng.integers(0, 12 * 4**level))
        prob = _prob(n, pos=[u / n], level0=level, level_cap=level, rot=R)
        cells, ds, end = O.ray_segments(prob, level, pix)
        assert end == 0
        v = R @ O.pix2vec(level, pix)
        texit = _exit_length(u, v, n)
        got = {}
        for c, d in zip(cells.tolist(), ds.tolist()):
            got[c] = got.get(c, 0.0) + d * n
        assert sum(got.values()) == pytest.approx(texit, abs=1e-12)
        ref = _brute(u, v, n, texit, 2_000_000)
        assert set(ref) <= set(got)
        for c, d in got.items():
            assert abs(d - ref.get(c, 0.0)) < 1.5e-5, (trial, c)


def test_axis_ray_visit_sequence():
    n = 8
    prob = _prob(n, pos=[[3.5 / n] * 3], level0=0, level_cap=0)
    cells, ds, end = O.ray_segments(prob, 0, 4)  # level-0 pixel 4 is +x
    exp_cells = [i + n * (3 + n * 3) for i in range(3, 8)]
    assert cells.tolist() == exp_cells
    assert np.allclose(ds * n, [0.5, 1, 1, 1, 1], atol=1e-15)
    assert end == 0


def test_diagonal_ray_steps_both_axes():
    n = 8
    c = s = math.sqrt(0.5)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])  # +x -> (1,1,0)/sqrt2
    prob = _prob(n, pos=[[3.5 / n] * 3], level0=0, level_cap=0, rot=R)
    cells, ds, end = O.ray_segments(prob, 0, 4)
    exp_cells = [k + n * (k + n * 3) for k in range(3, 8)]
    assert cells.tolist() == exp_cells
    assert np.allclose(ds * n, np.array([0.5, 1, 1, 1, 1]) * math.sqrt(2), atol=1e-14)


def test_corner_source_face_rules():
    n = 8
    prob = _prob(n, pos=[[4.0 / n] * 3], level0=0, level_cap=0)
    cells, ds, _ = O.ray_segments(prob, 0, 4)   # +x along an edge: upper cells in y and z
    assert cells.tolist() == [i + n * (4 + n * 4) for i in range(4, 8)]
    cells, ds, _ = O.ray_segments(prob, 0, 6)   # -x: the lower cell in x
    assert cells.tolist() == [i + n * (4 + n * 4) for i in range(3, -1, -1)]
    assert np.allclose(ds * n, 1.0)


def test_split_radius_matches_paper():
    g = GOLD["split_radius"]
    n = 64
    prob = _prob(n, pos=[[0.5 + 0.3 / n, 0.5 + 0.1 / n, 0.5 - 0.2 / n]], level0=4, m_ray=g["m_ray"])
    for pix in (0, 777, 3071):
        cells, ds, end = O.ray_segments(prob, 4, pix)
        assert end == 2
        assert ds.sum() * n == pytest.approx(g["r_max_over_dx_level4"], rel=1e-9)


def test_uniform_medium_absorption_closed_form():
    n = 8
    chi = 5.5  # per unit length (0.6875 per cell), exact in float32
    rng = np.random.default_rng(3)
    u = rng.uniform(1.0, 7.0, 3)
    prob = _prob(n, nH0=np.full((n, n, n), chi), pos=[u / n], L=[2.0], level0=1, level_cap=1,
                 sigma_H=1.0)
    r = O.trace(prob)
    want = 0.0
    path = 0.0
    for p in range(48):
        s = _exit_length(u, O.pix2vec(1, p), n) / n
        want += 2.0 / 48 * (1 - math.exp(-chi * s))
        path += s
    assert r.absorbed == pytest.approx(want, rel=1e-12)
    assert float((chi * r.G).sum()) == pytest.approx(want, rel=1e-12)
    assert r.escaped == pytest.approx(2.0 - want, rel=1e-12)
    assert r.dropped == 0.0


def test_vacuum_path_sum_rule():
    n = 12
    rng = np.random.default_rng(5)
    u = rng.uniform(1.0, 11.0, 3)
    prob = _prob(n, pos=[u / n], L=[3.0], level0=2, level_cap=2)
    r = O.trace(prob)
    path = sum(_exit_length(u, O.pix2vec(2, p), n) / n for p in range(192))
    assert float(r.G.sum()) == pytest.approx(3.0 / 192 * path, rel=1e-12)
    assert r.absorbed == 0.0 and r.escaped == pytest.approx(3.0, rel=1e-15)


def test_photon_conservation_and_destroy_counter():
    from paper_1711_06277_gb300 import synth
    n = 24
    rho = synth.lognormal_field(n, 1.5, seed=2).astype(np.float32).astype(np.float64)
    pos = synth.uniform_positions(5, seed=4)
    L = synth.power_law_luminosities(5, seed=4)
    prob = _prob(n, nH0=rho, pos=pos, L=L, sigma_H=12.0, level0=2, tau_max=8.0)
    r = O.trace(prob)
    assert r.absorbed + r.escaped + r.dropped == pytest.approx(r.L_in, rel=1e-12)
    assert float((12.0 * rho * r.G).sum()) == pytest.approx(r.absorbed, rel=1e-10)
    assert r.destroy == r.destroy_expected == 5 * 12 * 4**r.level_max
    assert r.dropped <= math.exp(-8.0) * r.L_in
    assert r.dropped > 0


def test_rays_per_level_exact_in_vacuum():
    n = 64
    prob = _prob(n, pos=[[0.5, 0.5, 0.5]], level0=4)
    r = O.trace(prob)
    # r_max(4), r_max(5), r_max(6) = 7.8, 15.6, 31.3 cells are all inside the 32-cell
    # half-width, so every ray splits at those levels; level 7 (r_max 62.5) reaches the
    # farthest corner (55.4) and never splits.
    assert r.level_max == 7
    assert r.rays_per_level[4:9].tolist() == [3072, 12288, 49152, 196608, 0]
    assert r.destroy == 12 * 4**7


def test_level_max_rule():
    n = 32
    r = O.trace(_prob(n, nH0=np.ones((n, n, n)), sigma_H=5.0))
    assert r.level_max == 6            # r_max(6) = 31.3 >= sqrt(3) * 16 = 27.7 > r_max(5)
    assert r.rays_per_level[4:8].tolist() == [3072, 12288, 49152, 0]
    assert r.near_tie_rays == 0


@pytest.mark.slow
def test_vacuum_inverse_square_accuracy():
    g = GOLD["vacuum"]
    n = 128
    prob = _prob(n, pos=[[0.5, 0.5, 0.5]], level0=4, m_ray=4.0)
    r = O.trace(prob, nthreads=4)
    c = np.arange(n) + 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rr = np.sqrt((x - 64) ** 2 + (y - 64) ** 2 + (z - 64) ** 2)
    sel = (rr > 4) & (rr < 60)
    exact = 1.0 / (4 * np.pi * (rr[sel] / n) ** 2)
    err4 = np.abs(r.energy[sel] / exact - 1)
    lo, hi = g["median_rel_err_m4_l4_range"]
    assert lo <= np.median(err4) <= hi
    r16 = O.trace(_prob(n, pos=[[0.5, 0.5, 0.5]], level0=4, m_ray=16.0), nthreads=4)
    err16 = np.abs(r16.energy[sel] / exact - 1)
    assert np.median(err16) < 0.5 * np.median(err4)


def _cell_average_uniform(n, chi, c):
    """(1/dV) * integral over each cell of e^{-chi r} / (4 pi r^2) for a unit source at
    cell coordinates (c, c, c): composite Gauss-Legendre, 2 sub-intervals x 6 nodes per
    axis in FP64 (accurate to 1e-9 in every cell but the source's own)."""
    x, w = np.polynomial.legendre.leggauss(6)
    nodes = np.concatenate([(s + (x + 1) / 2) / 2 for s in range(2)])
    wts = np.concatenate([w / 4, w / 4])
    q = nodes.size
    d = ((np.arange(n)[:, None] + nodes[None, :]).reshape(-1) - c) / n
    W = np.tile(wts, n)
    out = np.zeros((n, n, n))
    for kz in range(n):
        dz, wz = d[kz * q:(kz + 1) * q], W[kz * q:(kz + 1) * q]
        r2 = dz[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2
        f = np.exp(-chi * np.sqrt(r2)) / (4 * np.pi * r2)
        f *= wz[:, None, None] * W[None, :, None] * W[None, None, :]
        out[kz] = f.reshape(q, n, q, n, q).sum(axis=(0, 2, 4))
    return out


def test_uniform_medium_converges_to_exact_cell_average():
    """In a uniform medium the energy density of every cell (Eq. e:Erad with the segment
    average of Eq. e:photrate2) tends to the exact cell average of L e^{-chi r}/(4 pi r^2)
    as the rays per cell m_ray grow (Sec. 2.1), with the error falling about as 1/m_ray."""
    n, chi, c = 16, 4.0, 8.5                  # 0.25 optical depth per cell, source at a centre
    exact = _cell_average_uniform(n, chi, c)
    cc = np.arange(n) + 0.5
    z, y, x = np.meshgrid(cc, cc, cc, indexing="ij")
    sel = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) > 0.5   # all but the source cell
    med = []
    for m in (4.0, 16.0, 64.0, 256.0, 1000.0):
        r = O.trace(_prob(n, nH0=np.full((n, n, n), chi), pos=[[c / n] * 3], level0=4,
                          m_ray=m), nthreads=4)
        med.append(float(np.median(np.abs(r.energy[sel] / exact[sel] - 1))))
    assert med[0] < 0.1
    for a, b in zip(med, med[1:]):
        assert b < 0.5 * a
    assert med[-1] < 1e-3


def test_two_bin_closed_forms():
    """A second, non-ionizing bin (Sec. 2.3: chi_n = n_H sigma_d) on the same rays: its
    absorption follows the exact exit lengths, and the force sums both bins' momentum
    (Eq. e:radforce)."""
    n = 8
    rng = np.random.default_rng(12)
    u = rng.uniform(1.0, 7.0, 3)
    nH = np.full((n, n, n), 2.0)
    nH0 = np.full((n, n, n), 0.5)
    sH, sd = 3.0, 1.5          # chi_i = 0.5*3 + 2*1.5 = 4.5, chi_n = 3 (per unit length)
    prob = _prob(n, nH0=nH0, pos=[u / n], L=[2.0], level0=1, level_cap=1, sigma_H=sH,
                 sigma_d=sd, nH=nH)
    prob.Ln = np.array([5.0])
    r = O.trace(prob)
    chi_i, chi_n = 0.5 * sH + 2.0 * sd, 2.0 * sd
    want_i = want_n = 0.0
    mom = np.zeros(3)
    for p in range(48):
        v = O.pix2vec(1, p)
        s = _exit_length(u, v, n) / n
        ai = 2.0 / 48 * (1 - math.exp(-chi_i * s))
        an = 5.0 / 48 * (1 - math.exp(-chi_n * s))
        want_i += ai
        want_n += an
        mom += (ai + an) * v
    assert r.absorbed == pytest.approx(want_i, rel=1e-12)
    assert r.absorbed_n == pytest.approx(want_n, rel=1e-12)
    assert r.absorbed_n + r.escaped_n + r.dropped_n == pytest.approx(5.0, rel=1e-13)
    assert r.Ln_in == 5.0
    np.testing.assert_allclose(r.F.reshape(3, -1).sum(axis=1), mom, rtol=1e-12, atol=1e-15)
    # the ionizing bin and Gamma do not see the second bin
    one = O.trace(_prob(n, nH0=nH0, pos=[u / n], L=[2.0], level0=1, level_cap=1, sigma_H=sH,
                        sigma_d=sd, nH=nH))
    np.testing.assert_array_equal(r.G, one.G)


def test_two_bin_drop_uses_the_dust_depth():
    n = 24
    nH = np.ones((n, n, n))
    prob = _prob(n, nH0=nH, pos=[[0.41, 0.52, 0.47]], L=[1.0], level0=2, sigma_H=40.0,
                 sigma_d=4.0, nH=nH, tau_max=3.0)
    one = O.trace(prob)
    prob.Ln = np.array([1.0])
    two = O.trace(prob)
    # per cell length: tau_i = 44/24 ~ 1.8, tau_n = 4/24: the ionizing bin alone is dropped
    # within two cells; with a second bin the rays run until the dust depth passes 3
    assert 0 < one.dropped <= math.exp(-3.0) * one.L_in
    assert two.crossings > 5 * one.crossings
    assert two.dropped <= math.exp(-3.0 * 44.0 / 4.0) * two.L_in
    assert two.absorbed + two.escaped + two.dropped == pytest.approx(1.0, rel=1e-12)
    assert two.absorbed_n + two.escaped_n + two.dropped_n == pytest.approx(1.0, rel=1e-12)


# --- the d_max cutoff (rays terminated at a distance from their source, Sec. 3.1) ----------

def test_dmax_beyond_the_box_changes_nothing():
    from paper_1711_06277_gb300 import synth
    n = 16
    rho = synth.lognormal_field(n, 1.5, seed=7).astype(np.float32).astype(np.float64)
    pos = synth.uniform_positions(3, seed=7)
    base = dict(nH0=rho, pos=pos, L=[1.0, 0.5, 0.25], sigma_H=6.0, level0=2)
    r0 = O.trace(_prob(n, **base))
    r1 = O.trace(_prob(n, **base, d_max=2.0))  # farther than any box corner (sqrt 3)
    assert np.array_equal(r0.G, r1.G) and np.array_equal(r0.F, r1.F)
    assert (r0.escaped, r0.dropped, r0.crossings) == (r1.escaped, r1.dropped, r1.crossings)


def test_dmax_uniform_medium_closed_form():
    """Every path from the source is cut at d_max inside the box, whatever its splits: the
    absorbed share is 1 - e^{-chi d_max}, the rest leaves as cut (counted as escaped)."""
    n = 24
    chi = 3.0
    dmax = 7.3 / n
    prob = _prob(n, nH0=np.full((n, n, n), chi), pos=[[0.5 + 0.1 / n, 0.5 - 0.2 / n, 0.5]],
                 L=[2.0], level0=1, sigma_H=1.0, d_max=dmax)
    r = O.trace(prob)
    want = 2.0 * -math.expm1(-chi * dmax)
    assert r.absorbed == pytest.approx(want, rel=1e-12)
    assert r.escaped == pytest.approx(2.0 - want, rel=1e-12)
    assert r.dropped == 0.0
    # every split radius below d_max is used: levels 1-3 split (r_max 0.98, 1.95, 3.9 cells),
    # level 4 (r_max 7.8 > 7.3) is cut at d_max, so no level-5 rays
    assert r.rays_per_level[1:6].tolist() == [48, 192, 768, 3072, 0]
    assert r.destroy == r.destroy_expected


def test_dmax_leaves_far_cells_empty_and_cuts_paths_exactly():
    n = 20
    u = np.array([9.3, 10.6, 8.2])
    dmax_cells = 5.25
    prob = _prob(n, pos=[u / n], level0=2, level_cap=2, d_max=dmax_cells / n)
    r = O.trace(prob)
    k, j, i = np.indices((n, n, n))
    # nearest point of each cell to the source
    near = np.sqrt(sum(np.maximum(0.0, np.maximum(c - x, x - c - 1.0)) ** 2
                       for c, x in ((i, u[0]), (j, u[1]), (k, u[2]))))
    assert np.all(r.G[near > dmax_cells + 1e-9] == 0.0)
    # vacuum: the path sum rule with every ray cut at d_max
    assert float(r.G.sum()) == pytest.approx(dmax_cells / n, rel=1e-12)
    cells, ds, end = O.ray_segments(prob, 2, 77)
    assert end == 0 and ds.sum() * n == pytest.approx(dmax_cells, rel=1e-12)


def test_dmax_equal_to_a_split_radius_cuts():
    """d_max exactly at r_max(l): the cut wins and level l + 1 gets no rays."""
    n = 32
    m_ray = 4.0
    r3 = math.sqrt(3.0 / (math.pi * m_ray)) * 2**3   # r_max(3) in cells
    prob = _prob(n, pos=[[0.5 + 0.2 / n, 0.5 + 0.3 / n, 0.5 - 0.1 / n]], level0=2,
                 d_max=r3 / n, m_ray=m_ray)
    r = O.trace(prob)
    assert r.rays_per_level[2:5].tolist() == [192, 768, 0]
    assert r.escaped == pytest.approx(1.0, rel=1e-13)
