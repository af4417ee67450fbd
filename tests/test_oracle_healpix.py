"""Pins of the oracle's HEALPix nested directions (Sec. 2.1; Gorski et al. 2005).

pix2vec is pinned by the N_side = 1 closed form, exact ring heights, the nesting of
children inside their parent, the round trip through an independently written vec2pix,
and the equal-area property of vec2pix on uniform random directions.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_nside1_closed_form():
    g = GOLD["healpix_nside1"]
    for p in range(12):
        v = O.pix2vec(0, p)
        phi = math.atan2(v[1], v[0]) % (2 * math.pi)
        assert v[2] == pytest.approx(g["z"][p], abs=1e-15)
        assert phi / math.pi == pytest.approx(g["phi_over_pi"][p], abs=1e-15)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_unit_norm_and_zero_sum(level):
    npix = 12 * 4**level
    V = np.array([O.pix2vec(level, p) for p in range(npix)])
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-14)
    assert np.abs(V.sum(axis=0)).max() < 1e-11


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_ring_heights(level):
    ns = 2**level
    rings = []
    for jr in range(1, 4 * ns):
        if jr < ns:
            rings.append(1 - jr * jr / (3 * ns * ns))
        elif jr > 3 * ns:
            rings.append(-(1 - (4 * ns - jr) ** 2 / (3 * ns * ns)))
        else:
            rings.append(2 * (2 * ns - jr) / (3 * ns))
    rings = np.array(rings)
    zs = np.array([O.pix2vec(level, p)[2] for p in range(12 * 4**level)])
    d = np.abs(zs[:, None] - rings[None, :]).min(axis=1)
    assert d.max() < 1e-15
    # each ring holds 4 * min(jr, ns, 4ns - jr) pixels
    for jr, z in enumerate(rings, start=1):
        count = int(np.sum(np.abs(zs - z) < 1e-15))
        assert count == 4 * min(jr, ns, 4 * ns - jr)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_round_trip(level):
    for p in range(12 * 4**level):
        assert O.vec2pix(level, O.pix2vec(level, p)) == p


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_children_inside_parent(level):
    for p in range(12 * 4**level):
        for k in range(4):
            assert O.vec2pix(level, O.pix2vec(level + 1, 4 * p + k)) == p


def test_equal_area_vec2pix():
    rng = np.random.default_rng(7)
    v = rng.standard_normal((200_000, 3))
    counts = np.zeros(48, dtype=np.int64)
    for row in v:
        counts[O.vec2pix(1, row)] += 1
    expect = len(v) / 48
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 100.0  # 47 dof: mean 47, sd ~ 9.7


def test_exact_axis_components():
    # Level 0: the equatorial pixels are exactly the four +-x, +-y axes.
    V0 = np.array([O.pix2vec(0, p) for p in range(12)])
    assert sorted(map(tuple, V0[4:8].tolist())) == sorted(
        [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (-1.0, 0.0, 0.0), (0.0, -1.0, 0.0)])
    # Level 4: the z = 0 ring (4 N_side pixels) is exact; rings with odd (jr - N_side)
    # carry phi = k pi / 2 pixels, whose other horizontal component is exactly zero;
    # phi = pi/4 pixels have exactly equal |x| and |y|.
    V = np.array([O.pix2vec(4, p) for p in range(12 * 4**4)])
    assert int(np.sum(V[:, 2] == 0.0)) == 4 * 16
    zero_x, zero_y = V[:, 0] == 0.0, V[:, 1] == 0.0
    assert zero_x.sum() > 0 and zero_y.sum() == zero_x.sum()
    phi = np.arctan2(V[:, 1], V[:, 0])
    near_axis = np.abs(np.sin(2 * phi)) < 1e-9
    assert np.array_equal(near_axis, zero_x | zero_y)
    diag = np.abs(np.cos(2 * phi)) < 1e-9
    assert diag.sum() > 0 and np.all(np.abs(V[diag, 0]) == np.abs(V[diag, 1]))
