"""GPU neutral-fraction update (Eqs. e:xn3, e:xn2) and substep size (Eq. e:dtss) vs the
oracle's closed forms."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def art():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1711_06277_gb300 import art as A
    return A


def _fields(n, seed):
    rng = np.random.default_rng(seed)
    nH = (10.0 ** rng.uniform(-1, 3, n)).astype(np.float32)
    xn = rng.random(n).astype(np.float32)
    special = [0.0, 1.0, 1e-6, 0.5, 0.999][:n]
    xn[:len(special)] = special
    gam = (10.0 ** rng.uniform(-4, 2, n)).astype(np.float32)
    gam[::7] = 0.0
    return nH, xn, gam


@pytest.mark.parametrize("method", ["b", "a"])
@pytest.mark.parametrize("n", [1, 1000, 1 << 20])
def test_xn_update_matches_oracle(art, method, n):
    nH, xn, gam = _fields(n, seed=n)
    alpha, dt = 0.02, 3.0
    t = {k: torch.from_numpy(v.copy()).cuda() for k, v in dict(nH=nH, xn=xn, gam=gam).items()}
    nH0 = torch.empty_like(t["nH"])
    art.xn_update(t["gam"], t["nH"], t["xn"], alpha, dt, nH0_out=nH0, method=method)
    got = t["xn"].cpu().numpy().astype(np.float64)
    f = O.xn_method_b if method == "b" else O.xn_method_a
    want = f(xn.astype(np.float64), gam.astype(np.float64), nH.astype(np.float64), alpha, dt)
    assert np.all((got >= 0) & (got <= 1))
    np.testing.assert_allclose(got, want, rtol=2e-5, atol=2e-7)
    np.testing.assert_allclose(nH0.cpu().numpy(), got * nH, rtol=1e-6, atol=1e-30)


def test_xn_update_empty_and_bad(art):
    from paper_1711_06277_gb300 import _lib as C
    z = torch.zeros(0, device="cuda")
    art.xn_update(z, z, z, 1.0, 1.0)
    x = torch.zeros(4, device="cuda")
    with pytest.raises(C.ArtError):
        art.xn_update(x, x, x, -1.0, 1.0)


@pytest.mark.parametrize("n", [1, 999, 300_000, 1 << 22])
def test_dt_substep_matches_oracle(art, n):
    nH, xn, gam = _fields(n, seed=n + 1)
    alpha = 0.05
    t = {k: torch.from_numpy(v).cuda() for k, v in dict(nH=nH, xn=xn, gam=gam).items()}
    got = float(art.dt_substep(t["gam"], t["nH"], t["xn"], alpha, 0.1).cpu())
    want = O.dt_substep(xn.astype(np.float64), gam.astype(np.float64), nH.astype(np.float64),
                        alpha, 0.1)
    assert got == pytest.approx(want, rel=1e-5)


def test_dt_substep_equilibrium_is_infinite(art):
    # I = R in every cell (x n Gamma = alpha n_e^2): no cell limits the step
    nH = torch.full((64,), 2.0, device="cuda")
    xn = torch.full((64,), 0.5, device="cuda")
    alpha = 0.25
    gam = torch.full((64,), alpha * 2.0 * 0.5 * 0.5 / 0.5, device="cuda")  # x n G = a (n(1-x))^2
    got = float(art.dt_substep(gam, nH, xn, alpha, 0.1).cpu())
    assert got == float("inf")
