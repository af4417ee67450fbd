"""GPU adjoint (art_trace_backward / ARTFunction) vs the oracle's reverse sweep, which the
CPU suite pins to FP64 finite differences."""
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


def _case(A, n, nsrc, seed, sigma_ln=1.5, tau_box=10.0, level0=4, nH_scale=None,
          schedule="persistent", signed=False):
    rho = synth.lognormal_field(n, sigma_ln, seed=seed).astype(np.float32)
    pos = synth.uniform_positions(nsrc, seed=seed)
    L = synth.power_law_luminosities(nsrc, seed=seed)
    w = synth.uniform_weights(n, seed=seed).astype(np.float32)
    if signed:
        w = (2.0 * w - 1.0).astype(np.float32)
    p = A.Params(level0=level0, tau_max=30.0, sigma_H=tau_box, schedule=schedule)
    nH = None if nH_scale is None else (nH_scale * rho).astype(np.float32)
    if nH is not None:
        p.sigma_d = 3.0
    dev = torch.device("cuda")
    g = A.Grid(torch.from_numpy(rho).to(dev), 1.0 / n,
               nH=None if nH is None else torch.from_numpy(nH).to(dev))
    g.add_sources(pos, L)
    fwd = g.trace(p, force=False)
    grad, dL, st = g.trace_backward(p, torch.from_numpy(w).to(dev))
    loss = float((w.astype(np.float64) * fwd["gamma"].cpu().numpy()).sum())
    out = dict(grad=grad.cpu().numpy(), dL=dL.cpu().numpy(), stats=st, loss=loss,
               fstats=fwd["stats"])
    g.close()
    prob = O.Problem(nH0=rho, pos=pos, L=L, dx=1.0 / n, nH=nH, sigma_H=p.sigma_H,
                     sigma_d=p.sigma_d, level0=level0, tau_max=30.0)
    rg, rdL, rloss = O.trace_adjoint(prob, w, nthreads=8)
    return out, (rg, rdL, rloss), L


def _check(out, ref, L):
    rg, rdL, rloss = ref
    assert out["stats"]["status"] == 0
    assert out["stats"]["destroy"] == out["stats"]["destroy_expected"]
    assert out["stats"]["crossings"] == out["fstats"]["crossings"]
    PA.compare_field(out["grad"], rg, what="dloss/dlog nH0")
    np.testing.assert_allclose(out["dL"], rdL, rtol=PA.REL)
    # the loss is linear in every L_s: sum_s L_s dloss/dL_s = loss
    assert float((L * out["dL"]).sum()) == pytest.approx(rloss, rel=PA.REL)
    assert out["loss"] == pytest.approx(rloss, rel=PA.REL)


def test_adjoint_32_fd_subcase(art):
    out, ref, L = _case(art, 32, 4, seed=4)
    _check(out, ref, L)


def test_adjoint_config4_128_16src(art):
    out, ref, L = _case(art, 128, 16, seed=4)
    _check(out, ref, L)


def test_adjoint_with_dust_and_deep_levels(art):
    out, ref, L = _case(art, 48, 3, seed=8, level0=1, nH_scale=1.3)
    _check(out, ref, L)


def test_adjoint_signed_weights(art):
    """w of both signs (a general upstream gradient): per-cell sums cancel, so the gradient
    is compared in the max norm (1e-5 of its peak) and dL per source relatively."""
    out, ref, L = _case(art, 64, 5, seed=11, signed=True)
    rg, rdL, rloss = ref
    assert out["stats"]["status"] == 0
    err = np.abs(out["grad"].astype(np.float64) - rg).max() / np.abs(rg).max()
    assert err <= PA.REL, f"signed-weight gradient: max-norm rel err {err:.3e}"
    scale = np.abs(rdL).max()
    assert np.abs(out["dL"] - rdL).max() <= PA.REL * scale


def test_autograd_function_matches_backward(art):
    n = 32
    rho = synth.lognormal_field(n, 1.5, seed=2).astype(np.float32)
    pos = synth.uniform_positions(3, seed=2)
    L = synth.power_law_luminosities(3, seed=2)
    w = torch.from_numpy(synth.uniform_weights(n, seed=2).astype(np.float32)).cuda()
    p = art.Params(level0=3, tau_max=30.0, sigma_H=8.0)
    logn = torch.log(torch.from_numpy(rho).cuda()).requires_grad_(True)
    Lt = torch.tensor(L, dtype=torch.float64, requires_grad=True)
    g = art.Grid(torch.from_numpy(rho).cuda(), 1.0 / n)
    gamma = art.ARTFunction.apply(logn, Lt, g, p, pos)
    loss = (gamma.double() * w.double()).sum()
    loss.backward()
    prob = O.Problem(nH0=np.exp(np.log(rho)), pos=pos, L=L, dx=1.0 / n, sigma_H=8.0, level0=3,
                     tau_max=30.0)
    rg, rdL, rloss = O.trace_adjoint(prob, w.cpu().numpy(), nthreads=8)
    PA.compare_field(logn.grad.cpu().numpy(), rg, rel=3e-5, what="autograd grad")
    np.testing.assert_allclose(Lt.grad.numpy(), rdL, rtol=PA.REL)
    g.close()


def _force_case(A, n, nsrc, seed, with_w=True):
    rho = synth.lognormal_field(n, 1.5, seed=seed).astype(np.float32)
    pos = synth.uniform_positions(nsrc, seed=seed)
    L = synth.power_law_luminosities(nsrc, seed=seed)
    w = (0.5 * synth.uniform_weights(n, seed=seed)).astype(np.float32) if with_w else None
    v = synth.force_weights(n, seed=seed).astype(np.float32)
    p = A.Params(level0=3, tau_max=30.0, sigma_H=10.0)
    dev = torch.device("cuda")
    g = A.Grid(torch.from_numpy(rho).to(dev), 1.0 / n)
    g.add_sources(pos, L)
    fwd = g.trace(p, force=True)
    grad, dL, st = g.trace_backward(p, None if w is None else torch.from_numpy(w).to(dev),
                                    v=torch.from_numpy(v).to(dev))
    out = dict(grad=grad.cpu().numpy(), dL=dL.cpu().numpy(), stats=st,
               gamma=fwd["gamma"].cpu().numpy(), force=fwd["force"].cpu().numpy())
    g.close()
    prob = O.Problem(nH0=rho, pos=pos, L=L, dx=1.0 / n, sigma_H=10.0, level0=3, tau_max=30.0)
    ref = O.trace_adjoint(prob, np.zeros_like(rho) if w is None else w, v=v, nthreads=8)
    return out, ref, w, v


@pytest.mark.parametrize("with_w", [True, False], ids=["gamma_and_force", "force_only"])
def test_adjoint_force_term(art, with_w):
    """loss = sum w gamma + sum v . force with v of both signs (32-byte cell records)."""
    out, (rg, rdL, rloss), w, v = _force_case(art, 48, 3, seed=13, with_w=with_w)
    assert out["stats"]["status"] == 0
    err = np.abs(out["grad"].astype(np.float64) - rg).max() / np.abs(rg).max()
    assert err <= PA.REL, f"gradient with a force term: max-norm rel err {err:.3e}"
    assert np.abs(out["dL"] - rdL).max() <= PA.REL * np.abs(rdL).max()
    terms = (v.astype(np.float64) * out["force"].astype(np.float64))
    gpu_loss = terms.sum()
    scale = np.abs(terms).sum()
    if w is not None:
        gt = w.astype(np.float64) * out["gamma"].astype(np.float64)
        gpu_loss += gt.sum()
        scale += np.abs(gt).sum()
    assert abs(gpu_loss - rloss) <= PA.REL * scale


def test_autograd_function_with_force(art):
    n = 32
    rho = synth.lognormal_field(n, 1.5, seed=6).astype(np.float32)
    pos = synth.uniform_positions(2, seed=6)
    L = synth.power_law_luminosities(2, seed=6)
    w = synth.uniform_weights(n, seed=6).astype(np.float32)
    v = synth.force_weights(n, seed=6).astype(np.float32)
    p = art.Params(level0=3, tau_max=30.0, sigma_H=8.0)
    logn = torch.log(torch.from_numpy(rho).cuda()).requires_grad_(True)
    Lt = torch.tensor(L, dtype=torch.float64, requires_grad=True)
    g = art.Grid(torch.from_numpy(rho).cuda(), 1.0 / n)
    gamma, force = art.ARTFunction.apply(logn, Lt, g, p, pos, True)
    loss = (gamma.double() * torch.from_numpy(w).cuda().double()).sum() + \
        (force.double() * torch.from_numpy(v).cuda().double()).sum()
    loss.backward()
    prob = O.Problem(nH0=rho, pos=pos, L=L, dx=1.0 / n, sigma_H=8.0, level0=3, tau_max=30.0)
    rg, rdL, _ = O.trace_adjoint(prob, w, v=v, nthreads=8)
    err = np.abs(logn.grad.cpu().numpy().astype(np.float64) - rg).max() / np.abs(rg).max()
    assert err <= PA.REL
    assert np.abs(Lt.grad.numpy() - rdL).max() <= PA.REL * np.abs(rdL).max()
    g.close()


def test_adjoint_with_dmax_cutoff(art):
    n = 48
    rho = synth.lognormal_field(n, 1.5, seed=19).astype(np.float32)
    pos = synth.uniform_positions(3, seed=19)
    L = synth.power_law_luminosities(3, seed=19)
    w = synth.uniform_weights(n, seed=19).astype(np.float32)
    p = art.Params(level0=3, tau_max=30.0, sigma_H=10.0, d_max=0.37)
    dev = torch.device("cuda")
    g = art.Grid(torch.from_numpy(rho).to(dev), 1.0 / n)
    g.add_sources(pos, L)
    fwd = g.trace(p, force=False)
    grad, dL, st = g.trace_backward(p, torch.from_numpy(w).to(dev))
    assert st["status"] == 0 and st["crossings"] == fwd["stats"]["crossings"]
    prob = O.Problem(nH0=rho, pos=pos, L=L, dx=1.0 / n, sigma_H=10.0, level0=3, tau_max=30.0,
                     d_max=0.37)
    rg, rdL, rloss = O.trace_adjoint(prob, w, nthreads=8)
    PA.compare_field(grad.cpu().numpy(), rg, what="dloss/dlog nH0 with d_max")
    np.testing.assert_allclose(dL.cpu().numpy(), rdL, rtol=PA.REL)
    g.close()


def test_adjoint_with_rotation_and_plain_schedule_request(art):
    """Rotated ray directions (the same tables as the forward trace) and a plain-schedule
    request: the reverse sweep always runs its persistent schedule and must give the same
    result."""
    n = 40
    rho = synth.lognormal_field(n, 1.5, seed=23).astype(np.float32)
    pos = synth.uniform_positions(3, seed=23)
    L = synth.power_law_luminosities(3, seed=23)
    w = synth.uniform_weights(n, seed=23).astype(np.float32)
    R = synth.random_rotation(23)
    dev = torch.device("cuda")
    g = art.Grid(torch.from_numpy(rho).to(dev), 1.0 / n)
    g.add_sources(pos, L)
    outs = []
    for schedule in ("persistent", "plain"):
        p = art.Params(level0=3, tau_max=30.0, sigma_H=9.0, rot=R, schedule=schedule)
        g.trace(p, force=False)
        grad, dL, st = g.trace_backward(p, torch.from_numpy(w).to(dev))
        assert st["status"] == 0
        outs.append((grad.cpu().numpy(), dL.cpu().numpy()))
    g.close()
    prob = O.Problem(nH0=rho, pos=pos, L=L, dx=1.0 / n, sigma_H=9.0, level0=3, tau_max=30.0,
                     rot=R)
    rg, rdL, _ = O.trace_adjoint(prob, w, nthreads=8)
    for grad, dL in outs:
        PA.compare_field(grad, rg, what="dloss/dlog nH0, rotated")
        np.testing.assert_allclose(dL, rdL, rtol=PA.REL)


def test_autograd_two_forwards_then_backward(art):
    """Two ARTFunction calls with different sources on one shared Grid, then the backward of
    the first: the reverse sweep must trace the first call's sources and field."""
    n = 32
    rho = synth.lognormal_field(n, 1.5, seed=31).astype(np.float32)
    pos_a = synth.uniform_positions(3, seed=31)
    pos_b = synth.uniform_positions(2, seed=32)
    L_a = synth.power_law_luminosities(3, seed=31)
    L_b = synth.power_law_luminosities(2, seed=32)
    w = synth.uniform_weights(n, seed=31).astype(np.float32)
    p = art.Params(level0=3, tau_max=30.0, sigma_H=8.0)
    g = art.Grid(torch.from_numpy(rho).cuda(), 1.0 / n)
    logn = torch.log(torch.from_numpy(rho).cuda()).requires_grad_(True)
    La = torch.tensor(L_a, dtype=torch.float64, requires_grad=True)
    gamma_a = art.ARTFunction.apply(logn, La, g, p, pos_a)
    # a second forward on the same grid with other sources and a denser field
    logn_b = (logn.detach() + 0.7).requires_grad_(True)
    Lb = torch.tensor(L_b, dtype=torch.float64, requires_grad=True)
    art.ARTFunction.apply(logn_b, Lb, g, p, pos_b)
    (gamma_a.double() * torch.from_numpy(w).cuda().double()).sum().backward()
    prob = O.Problem(nH0=rho, pos=pos_a, L=L_a, dx=1.0 / n, sigma_H=8.0, level0=3, tau_max=30.0)
    rg, rdL, _ = O.trace_adjoint(prob, w, nthreads=8)
    PA.compare_field(logn.grad.cpu().numpy(), rg, rel=3e-5, what="grad after a second forward")
    np.testing.assert_allclose(La.grad.numpy(), rdL, rtol=PA.REL)
    g.close()


def test_autograd_with_dust(art):
    """A grid with a total-density field: ARTFunction keeps the dust term of the opacity
    (chi = n_H0 sigma_H + n_H sigma_d, Sec. 2.3) in both the forward and the reverse sweep."""
    n = 32
    rho = synth.lognormal_field(n, 1.5, seed=33).astype(np.float32)
    nH = (1.6 * rho).astype(np.float32)
    pos = synth.uniform_positions(3, seed=33)
    L = synth.power_law_luminosities(3, seed=33)
    w = synth.uniform_weights(n, seed=33).astype(np.float32)
    p = art.Params(level0=3, tau_max=30.0, sigma_H=8.0, sigma_d=3.0)
    g = art.Grid(torch.from_numpy(rho).cuda(), 1.0 / n, nH=torch.from_numpy(nH).cuda())
    logn = torch.log(torch.from_numpy(rho).cuda()).requires_grad_(True)
    Lt = torch.tensor(L, dtype=torch.float64, requires_grad=True)
    gamma = art.ARTFunction.apply(logn, Lt, g, p, pos)
    prob = O.Problem(nH0=rho, pos=pos, L=L, dx=1.0 / n, nH=nH, sigma_H=8.0, sigma_d=3.0,
                     level0=3, tau_max=30.0)
    ref = O.trace(prob, nthreads=8)
    PA.compare_field(gamma.detach().cpu().numpy(), ref.gamma, what="gamma with dust")
    (gamma.double() * torch.from_numpy(w).cuda().double()).sum().backward()
    rg, rdL, _ = O.trace_adjoint(prob, w, nthreads=8)
    PA.compare_field(logn.grad.cpu().numpy(), rg, rel=3e-5, what="autograd grad with dust")
    np.testing.assert_allclose(Lt.grad.numpy(), rdL, rtol=PA.REL)
    # a plain trace of the grid afterwards still sees the dust field
    out = g.trace(p, force=False)
    PA.compare_field(out["gamma"].cpu().numpy(), ref.gamma, what="gamma after backward")
    g.close()


def test_adjoint_config5_512_8src(art):
    """The reverse sweep at full size: the 512^3 workload the bench times the adjoint on
    (lognormal sigma_ln = 2, n_H = 100 rho, x_n = 1e-3, sigma_H = 0.1, loss = sum w gamma, all
    8 of its sources), in the launch configuration the bench uses, against the oracle's
    reverse sweep."""
    import os
    n = 512
    rho = synth.lognormal_field(n, 2.0, seed=5)
    nH0 = (1e-3 * (100.0 * rho).astype(np.float32)).astype(np.float32)
    pos = synth.uniform_positions(8, seed=5)
    L = synth.power_law_luminosities(8, seed=5)
    w = synth.uniform_weights(n, seed=5).astype(np.float32)
    p = art.Params(level0=4, m_ray=4.0, tau_max=30.0, sigma_H=0.1)
    dev = torch.device("cuda")
    g = art.Grid(torch.from_numpy(nH0).to(dev), 1.0 / n)
    g.add_sources(pos, L)
    fwd = g.trace(p, force=False)
    grad, dL, st = g.trace_backward(p, torch.from_numpy(w).to(dev))
    out = dict(grad=grad.cpu().numpy(), dL=dL.cpu().numpy(), stats=st, fstats=fwd["stats"],
               loss=float((w.astype(np.float64) * fwd["gamma"].cpu().numpy()).sum()))
    g.close()
    prob = O.Problem(nH0=nH0, pos=pos, L=L, dx=1.0 / n, sigma_H=0.1, level0=4, tau_max=30.0)
    ref = O.trace_adjoint(prob, w, nthreads=os.cpu_count() or 8)
    _check(out, ref, L)
