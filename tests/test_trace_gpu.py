"""GPU forward trace vs the FP64 oracle (per-cell gamma and force, tallies, conservation),
both schedules, on the synthetic workloads and edge cases."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1711_06277_gb300 import synth
from tests import parity as PA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def art():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1711_06277_gb300 import art as A
    return A


def _run(A, nH0, pos, L, dx, params, nH=None, lo=(0.0, 0.0, 0.0)):
    dev = torch.device("cuda")
    t0 = torch.as_tensor(np.ascontiguousarray(nH0, dtype=np.float32), device=dev)
    t1 = None if nH is None else torch.as_tensor(np.ascontiguousarray(nH, dtype=np.float32), device=dev)
    g = A.Grid(t0, dx, lo=lo, nH=t1)
    g.add_sources(pos, L)
    out = g.trace(params, force=True, energy=True)
    res = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    g.close()
    return res


def _oracle(nH0, pos, L, dx, p, nH=None, threads=8):
    prob = O.Problem(nH0=nH0, pos=pos, L=L, dx=dx, nH=nH, sigma_H=p.sigma_H,
                     sigma_d=p.sigma_d, level0=p.level0, level_cap=p.level_max, m_ray=p.m_ray,
                     tau_max=p.tau_max, rot=p.rot, d_max=p.d_max)
    return O.trace(prob, nthreads=threads, count_hits=True)


def _check(res, ref, nH0, p, nH=None, exact_counts=True, net_force=False):
    """GPU trace vs oracle. Per-cell values are checked at the parity bar, or at the
    derived FP32-sum bound of the cell's deposit count where that is larger (tests/parity.py
    sum_tol); with net_force also relative to |f| where little cancels."""
    st = res["stats"]
    assert st["status"] == 0
    PA.compare_field(res["gamma"], ref.gamma, what="gamma", hits=ref.hits)
    PA.compare_field(res["energy"], ref.energy, what="energy", hits=ref.hits)
    chi = nH0.astype(np.float32).astype(np.float64) * p.sigma_H
    if nH is not None:
        chi = chi + nH.astype(np.float32).astype(np.float64) * p.sigma_d
    PA.compare_force(res["force"], ref.force, chi * ref.energy, hits=ref.hits)
    if net_force:
        PA.compare_force_net(res["force"], ref.force, chi * ref.energy)
    if exact_counts:
        assert st["crossings"] == ref.crossings
        assert st["rays_per_level"] == ref.rays_per_level.tolist()
    else:
        assert abs(st["crossings"] - ref.crossings) <= 1e-5 * ref.crossings
    assert st["destroy"] == st["destroy_expected"] == ref.destroy_expected
    assert st["level_max"] == ref.level_max
    L_in = ref.L_in
    assert abs(st["L_escaped"] - ref.escaped) <= PA.CONS * L_in
    assert abs(st["L_dropped"] - ref.dropped) <= PA.CONS * L_in
    assert abs(st["L_absorbed"] - ref.absorbed) <= PA.CONS * L_in
    G_phys = res["energy"] * ref.dV
    assert PA.conservation(chi, G_phys, st) <= PA.CONS


@pytest.mark.parametrize("schedule", ["persistent", "plain"])
def test_config1_uniform_32(art, schedule):
    n = 32
    nH0 = np.ones((n, n, n))
    p = art.Params(level0=4, m_ray=4.0, tau_max=30.0, sigma_H=5.0, schedule=schedule)
    pos, L = np.array([[0.5, 0.5, 0.5]]), np.array([1.0])
    res = _run(art, nH0, pos, L, 1.0 / n, p)
    ref = _oracle(nH0, pos, L, 1.0 / n, p)
    assert ref.near_tie_rays == 0
    _check(res, ref, nH0, p, net_force=True)


@pytest.mark.parametrize("schedule", ["persistent", "plain"])
def test_config2_lognormal_128(art, schedule):
    n = 128
    rho = synth.lognormal_field(n, 1.5, seed=1)
    p = art.Params(level0=4, m_ray=4.0, tau_max=30.0, sigma_H=10.0, schedule=schedule)
    pos = synth.cell_centre_position(n, seed=1)
    L = np.array([1.0])
    res = _run(art, rho, pos, L, 1.0 / n, p)
    ref = _oracle(rho, pos, L, 1.0 / n, p)
    _check(res, ref, rho, p, exact_counts=ref.near_tie_rays == 0, net_force=True)


def test_config4_forward_128_16src(art):
    """The forward trace of the adjoint workload: 128^3 lognormal (sigma_ln = 1.5,
    tau_box = 10), 16 power-law sources."""
    n = 128
    rho = synth.lognormal_field(n, 1.5, seed=4).astype(np.float32)
    pos = synth.uniform_positions(16, seed=4)
    L = synth.power_law_luminosities(16, seed=4)
    p = art.Params(level0=4, m_ray=4.0, tau_max=30.0, sigma_H=10.0)
    res = _run(art, rho, pos, L, 1.0 / n, p)
    ref = _oracle(rho, pos, L, 1.0 / n, p, threads=16)
    _check(res, ref, rho, p, exact_counts=ref.near_tie_rays == 0, net_force=True)


def test_config2_vacuum_128(art):
    n = 128
    p = art.Params(level0=4, m_ray=4.0, tau_max=30.0, sigma_H=10.0)
    pos = synth.cell_centre_position(n, seed=1)
    res = _run(art, np.zeros((n, n, n)), pos, np.array([1.0]), 1.0 / n, p)
    ref = _oracle(np.zeros((n, n, n)), pos, np.array([1.0]), 1.0 / n, p)
    PA.compare_field(res["energy"], ref.energy, what="vacuum energy")
    assert res["stats"]["crossings"] == ref.crossings
    # inverse-square law, paper's accuracy band (Sec. 3.2)
    c = np.arange(n) + 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    u = pos[0] * n
    rr = np.sqrt((x - u[0]) ** 2 + (y - u[1]) ** 2 + (z - u[2]) ** 2)
    sel = (rr > 4) & (rr < 40)
    err = np.abs(res["energy"][sel] * 4 * np.pi * (rr[sel] / n) ** 2 - 1)
    assert 0.005 < np.median(err) < 0.04


@pytest.mark.parametrize("schedule", ["persistent", "plain"])
def test_multisource_dust_rotation_64(art, schedule):
    n = 64
    rho = synth.lognormal_field(n, 1.5, seed=7)
    pos = synth.uniform_positions(8, seed=7)
    L = synth.power_law_luminosities(8, seed=7)
    R = synth.random_rotation(7)
    p = art.Params(level0=3, m_ray=4.0, tau_max=30.0, sigma_H=6.0, sigma_d=2.0, rot=R,
                   schedule=schedule)
    nH = 1.7 * rho
    res = _run(art, 0.5 * rho, pos, L, 1.0 / n, p, nH=nH)
    ref = _oracle(0.5 * rho, pos, L, 1.0 / n, p, nH=nH)
    _check(res, ref, 0.5 * rho, p, nH=nH, exact_counts=ref.near_tie_rays == 0, net_force=True)


def test_small_queue_persistent_matches(art):
    # a front capacity far below the ray count forces many depth-first phases
    n = 48
    rho = synth.lognormal_field(n, 1.0, seed=3)
    pos = synth.uniform_positions(3, seed=3)
    L = synth.power_law_luminosities(3, seed=3)
    p = art.Params(level0=2, tau_max=30.0, sigma_H=4.0, queue_capacity=1000, chunk=32)
    res = _run(art, rho, pos, L, 1.0 / n, p)
    ref = _oracle(rho, pos, L, 1.0 / n, p)
    _check(res, ref, rho, p, exact_counts=ref.near_tie_rays == 0)


@pytest.mark.parametrize("shape,level0,lmax", [((1, 1, 1), 0, -1), ((5, 9, 3), 1, -1),
                                               ((17, 16, 33), 8, -1), ((20, 20, 20), 2, 2)])
def test_odd_shapes_and_levels(art, shape, level0, lmax):
    nz, ny, nx = shape
    rng = np.random.default_rng(sum(shape) + level0)
    rho = rng.random(shape) * 3
    dx = 0.1
    lo = (-0.3, 0.2, 1.0)
    box = np.array([nx, ny, nz]) * dx
    pos = np.asarray(lo) + box * rng.uniform(0.05, 0.95, size=(2, 3))
    L = np.array([0.3, 2.0])
    p = art.Params(level0=level0, level_max=lmax, tau_max=30.0, sigma_H=1.5)
    res = _run(art, rho, pos, L, dx, p, lo=lo)
    prob = O.Problem(nH0=rho, pos=pos, L=L, dx=dx, lo=lo, sigma_H=1.5, level0=level0,
                     level_cap=lmax, tau_max=30.0)
    ref = O.trace(prob, nthreads=8, count_hits=True)
    # At l0 = 8 cells near a source receive 10^4-10^6 deposits: their bar is the FP32-sum
    # bound of their deposit count (parity.sum_tol), the parity bar elsewhere.
    _check(res, ref, rho, p, exact_counts=ref.near_tie_rays == 0)


def test_source_near_faces_and_small_tau_max(art):
    n = 24
    rho = np.ones((n, n, n))
    eps = 1e-7
    pos = np.array([[eps, 0.5, 0.5], [1 - eps, 1 - eps, eps], [0.3, 0.6, 0.9]])
    L = np.array([1.0, 1.0, 2.0])
    p = art.Params(level0=2, tau_max=0.31, sigma_H=8.0)  # 0.3 makes exact ties (ring z=-2/3)
    res = _run(art, rho, pos, L, 1.0 / n, p)
    ref = _oracle(rho, pos, L, 1.0 / n, p)
    assert ref.dropped > 0
    _check(res, ref, rho, p, exact_counts=ref.near_tie_rays == 0)


def test_integer_tallies_deterministic(art):
    n = 64
    rho = synth.lognormal_field(n, 2.0, seed=9)
    pos = synth.uniform_positions(16, seed=9)
    L = synth.power_law_luminosities(16, seed=9)
    p = art.Params(level0=4, tau_max=30.0, sigma_H=10.0)
    a = _run(art, rho, pos, L, 1.0 / n, p)
    b = _run(art, rho, pos, L, 1.0 / n, p)
    for k in ("crossings", "rays_total", "rays_per_level", "destroy"):
        assert a["stats"][k] == b["stats"][k]
    np.testing.assert_allclose(a["gamma"], b["gamma"], rtol=1e-5, atol=1e-6 * a["gamma"].max())


@pytest.mark.parametrize("schedule,d_max", [("persistent", 0.0), ("plain", 0.0),
                                             ("persistent", 0.28)])
def test_two_bin_dust_radiation_pressure(art, schedule, d_max):
    """Second, non-ionizing bin (Sec. 2.3): dust-only attenuation, force of both bins; also
    with the d_max cutoff (both bins end there)."""
    n = 48
    rho = synth.lognormal_field(n, 1.5, seed=11)
    pos = synth.uniform_positions(4, seed=11)
    L = synth.power_law_luminosities(4, seed=11)
    Ln = 3.0 * synth.power_law_luminosities(4, seed=12)
    nH0, nH = 0.3 * rho, rho
    p = art.Params(level0=3, tau_max=30.0, sigma_H=20.0, sigma_d=6.0, schedule=schedule,
                   d_max=d_max)
    dev = torch.device("cuda")
    g = art.Grid(torch.as_tensor(nH0.astype(np.float32), device=dev), 1.0 / n,
                 nH=torch.as_tensor(nH.astype(np.float32), device=dev))
    g.add_sources(pos, L)
    g.set_nonionizing(Ln)
    out = g.trace(p, force=True, energy=True)
    res = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    prob = O.Problem(nH0=nH0, pos=pos, L=L, dx=1.0 / n, nH=nH, sigma_H=20.0, sigma_d=6.0,
                     level0=3, tau_max=30.0, Ln=Ln, d_max=d_max)
    ref = O.trace(prob, nthreads=8)
    st = res["stats"]
    assert st["status"] == 0 and st["destroy"] == st["destroy_expected"]
    PA.compare_field(res["gamma"], ref.gamma, what="gamma")
    chi = nH0.astype(np.float32).astype(np.float64) * 20.0 + nH.astype(np.float32).astype(np.float64) * 6.0
    chin = nH.astype(np.float32).astype(np.float64) * 6.0
    # bound of the two-bin force: chi_i E_i + the non-ionizing absorption in the cell
    Fn_bound = np.abs(ref.force).sum(axis=0) + chi * ref.energy
    PA.compare_force(res["force"], ref.force, np.maximum(Fn_bound, chi * ref.energy))
    if ref.near_tie_rays == 0:
        assert st["crossings"] == ref.crossings
    assert abs(st["Ln_escaped"] - ref.escaped_n) <= PA.CONS * ref.Ln_in
    assert abs(st["Ln_dropped"] - ref.dropped_n) <= PA.CONS * ref.Ln_in
    assert st["Ln_in"] == pytest.approx(ref.Ln_in, rel=1e-12)
    g.close()


def test_two_bin_matches_one_bin_without_second_luminosity(art):
    n = 32
    rho = synth.lognormal_field(n, 1.0, seed=13).astype(np.float32)
    pos = synth.uniform_positions(2, seed=13)
    # tau_max beyond any ray's depth: both traces retire rays only at the grid boundary
    p = art.Params(level0=2, tau_max=1e4, sigma_H=8.0, sigma_d=1.0)
    dev = torch.device("cuda")
    g = art.Grid(torch.as_tensor(rho, device=dev), 1.0 / n, nH=torch.as_tensor(rho, device=dev))
    g.add_sources(pos, [1.0, 0.5])
    one = g.trace(p, force=True)
    g.set_nonionizing([0.0, 0.0])
    two = g.trace(p, force=True)
    # the sums differ only by FP32 summation order
    assert one["stats"]["crossings"] == two["stats"]["crossings"]
    torch.testing.assert_close(one["gamma"], two["gamma"], rtol=1e-5, atol=1e-6 * float(one["gamma"].max()))
    torch.testing.assert_close(one["force"], two["force"], rtol=1e-5, atol=1e-6 * float(one["force"].abs().max()))
    from paper_1711_06277_gb300 import _lib as C
    with pytest.raises(C.ArtError) as e:
        g.trace_backward(p, torch.ones_like(one["gamma"]))
    assert e.value.status == C.ART_EINVAL
    g.close()


def test_zero_luminosity_and_thin_slab(art):
    """A source with L = 0 deposits nothing; a one-cell-thick slab (nz = 1) still matches."""
    shape = (1, 40, 33)
    rng = np.random.default_rng(5)
    rho = rng.random(shape) * 2
    dx = 0.05
    pos = np.array([[0.7, 1.1, 0.025], [0.3, 0.4, 0.02]])
    L = np.array([0.0, 1.5])
    p = art.Params(level0=3, tau_max=30.0, sigma_H=3.0)
    res = _run(art, rho, pos, L, dx, p)
    ref = O.trace(O.Problem(nH0=rho, pos=pos, L=L, dx=dx, sigma_H=3.0, level0=3, tau_max=30.0),
                  nthreads=8, count_hits=True)
    _check(res, ref, rho, p, exact_counts=ref.near_tie_rays == 0)
    only0 = _run(art, rho, pos[:1], L[:1], dx, p)
    assert np.all(only0["gamma"] == 0) and np.all(only0["force"] == 0)


def test_sources_added_and_fields_updated_between_traces(art):
    n = 40
    rng = np.random.default_rng(8)
    rho = rng.random((n, n, n)).astype(np.float32) + 0.1
    dev = torch.device("cuda")
    t = torch.from_numpy(rho.copy()).to(dev)
    g = art.Grid(t, 1.0 / n)
    p = art.Params(level0=2, tau_max=30.0, sigma_H=4.0)
    pos = synth.uniform_positions(3, seed=8)
    g.add_sources(pos[:2], [1.0, 2.0])
    g.trace(p)
    g.add_sources(pos[2:], [0.5])           # a third source after a trace
    t.mul_(0.5)                             # fields are read again by every trace
    out = g.trace(p, force=True, energy=True)
    res = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    ref = O.trace(O.Problem(nH0=0.5 * rho, pos=pos, L=[1.0, 2.0, 0.5], dx=1.0 / n, sigma_H=4.0,
                            level0=2, tau_max=30.0), nthreads=8, count_hits=True)
    _check(res, ref, 0.5 * rho, p, exact_counts=ref.near_tie_rays == 0)
    g.close()


@pytest.mark.parametrize("schedule", ["persistent", "plain"])
def test_dmax_cutoff_64(art, schedule):
    """Rays terminated at d_max from their source (Sec. 3.1), lognormal field with dust."""
    n = 64
    rho = synth.lognormal_field(n, 1.5, seed=17).astype(np.float32)
    nH = (1.4 * rho).astype(np.float32)
    pos = synth.uniform_positions(4, seed=17)
    L = synth.power_law_luminosities(4, seed=17)
    p = art.Params(level0=3, tau_max=30.0, sigma_H=6.0, sigma_d=1.0, schedule=schedule,
                   d_max=0.31)
    res = _run(art, rho, pos, L, 1.0 / n, p, nH=nH)
    ref = _oracle(rho, pos, L, 1.0 / n, p, nH=nH)
    _check(res, ref, rho, p, nH=nH)
    assert res["stats"]["L_escaped"] == pytest.approx(ref.escaped, rel=1e-5)
    # cells beyond d_max (plus a cell diagonal) of every source stay empty
    k, j, i = np.indices((n, n, n))
    c = (np.stack([i, j, k], -1) + 0.5) / n
    far = np.all([np.linalg.norm(c - q, axis=-1) > 0.31 + math.sqrt(3) / n for q in pos], axis=0)
    assert far.any() and np.all(res["gamma"][far] == 0.0)


def test_dmax_at_a_split_radius_and_without_effect(art):
    """d_max exactly at r_max(l) cuts (no level l+1 rays); d_max beyond the box is a no-op."""
    n = 32
    pos = [[0.5 + 0.2 / n, 0.5 + 0.3 / n, 0.5 - 0.1 / n]]
    rho = np.full((n, n, n), 0.5, dtype=np.float32)
    r3 = math.sqrt(3.0 / (math.pi * 4.0)) * 2**3 / n
    p = art.Params(level0=2, tau_max=30.0, sigma_H=2.0, d_max=r3)
    res = _run(art, rho, pos, [1.0], 1.0 / n, p)
    ref = _oracle(rho, pos, [1.0], 1.0 / n, p)
    assert res["stats"]["rays_per_level"][2:5] == [192, 768, 0] == ref.rays_per_level[2:5].tolist()
    _check(res, ref, rho, p)
    p_far = art.Params(level0=2, tau_max=30.0, sigma_H=2.0, d_max=5.0)
    p_none = art.Params(level0=2, tau_max=30.0, sigma_H=2.0)
    a = _run(art, rho, pos, [1.0], 1.0 / n, p_far)
    b = _run(art, rho, pos, [1.0], 1.0 / n, p_none)
    assert a["stats"]["crossings"] == b["stats"]["crossings"]
    PA.compare_field(a["gamma"], b["gamma"], rel=1e-6, what="gamma, d_max beyond the box")
