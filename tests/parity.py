"""Helpers of the GPU-vs-oracle parity tests (comparison rules in one place)."""
import numpy as np

# Tolerances of the parity bar: per-cell gamma and force within 1e-5 relative where the
# deposit exceeds 1e-6 of the peak; photon conservation within 1e-6 relative.
REL = 1e-5
FLOOR = 1e-6
CONS = 1e-6


U32 = 2.0 ** -24  # unit roundoff of FP32


def sum_tol(hits, cells_checked, rel=REL, p_fail=1e-6):
    """Per-cell tolerance of an FP32 sum of ``hits`` deposits added in an unknown order.

    A cell's value is the sum of n = hits FP32 terms, reduced by atomics in an order that
    changes from run to run. By the probabilistic bound of Higham & Mary (2019, SIAM J. Sci.
    Comput. 41, A2815) for recursive summation, |s_fp32 - s| <= lambda sqrt(n) u sum|x_i|
    with probability at least 1 - 2 n exp(-lambda^2 / 2); lambda is chosen so that the
    probability of any failure over the checked cells stays below p_fail. For positive
    terms sum|x_i| = s, so this bounds the relative error; for the force components the sum
    of |dL n_a| is at most chi E dV, the normalisation of compare_force. Where that bound is
    below ``rel`` the parity bar ``rel`` applies unchanged."""
    n = np.maximum(np.asarray(hits, dtype=np.float64), 1.0)
    lam = np.sqrt(2.0 * np.log(2.0 * n.max() * max(cells_checked, 1) / p_fail))
    return np.maximum(rel, lam * np.sqrt(n) * U32)


def compare_field(gpu, ref, rel=REL, floor=FLOOR, what="field", hits=None):
    """Max relative error over cells whose |ref| exceeds floor * max|ref|; returns it. With
    ``hits`` (deposits per cell, from the oracle) the bar of a cell is sum_tol(hits)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    peak = np.abs(ref).max()
    sel = np.abs(ref) > floor * peak
    err = np.abs(gpu[sel] - ref[sel]) / np.abs(ref[sel])
    if hits is not None:
        tol = sum_tol(np.asarray(hits)[sel], int(sel.sum()), rel)
        worst = float((err / tol).max()) if err.size else 0.0
        assert worst <= 1.0, (f"{what}: error {worst:.3f} x its FP32-sum bound "
                              f"(max rel err {err.max():.3e}) over {sel.sum()} cells")
        return float(err.max()) if err.size else 0.0
    worst = float(err.max()) if err.size else 0.0
    assert worst <= rel, f"{what}: max rel err {worst:.3e} over {sel.sum()} cells (> {rel})"
    # cells below the floor must still be small in absolute terms
    small = np.abs(gpu[~sel] - ref[~sel]).max() if (~sel).any() else 0.0
    assert small <= 10 * floor * peak, f"{what}: sub-floor cells off by {small:.3e}"
    return worst


def compare_force(gpu_f, ref_f, scale, rel=REL, floor=FLOOR, hits=None):
    """Force vectors. The error of each component is measured against the cell's
    flux-limited bound chi E (|f_rad| = chi |F| / c <= chi E, Sec. 2.1): where many rays of
    opposite directions cross a cell the net force is a near-total cancellation, which an
    FP32 sum cannot resolve relative to the net itself (the summation bound scales with the
    sum of |dL n_a| <= chi E dV, not with the net). Cells whose chi E exceeds floor of the
    peak are checked; with ``hits`` the bar of a cell is sum_tol(hits)."""
    g = np.asarray(gpu_f, dtype=np.float64).reshape(3, -1)
    r = np.asarray(ref_f, dtype=np.float64).reshape(3, -1)
    sc = np.asarray(scale, dtype=np.float64).reshape(-1)
    assert np.all(np.sqrt((r**2).sum(axis=0)) <= sc * (1 + 1e-9) + 1e-300)
    sel = sc > floor * sc.max()
    err = np.abs(g[:, sel] - r[:, sel]).max(axis=0) / sc[sel]
    if hits is not None:
        tol = sum_tol(np.asarray(hits).reshape(-1)[sel], int(sel.sum()), rel)
        ratio = float((err / tol).max()) if err.size else 0.0
        assert ratio <= 1.0, f"force: error {ratio:.3f} x its FP32-sum bound over {sel.sum()} cells"
        return float(err.max()) if err.size else 0.0
    worst = float(err.max()) if err.size else 0.0
    assert worst <= rel, f"force: max rel err {worst:.3e} over {sel.sum()} cells"
    return worst


def compare_force_net(gpu_f, ref_f, scale, rel=REL, floor=FLOOR, share=0.1, what="force"):
    """Force relative to the net force itself, |f_gpu - f| / |f| <= rel, on the cells where
    little cancels (|f| >= share * chi E) and chi E exceeds floor of the peak. Returns the
    worst error and the number of cells checked."""
    g = np.asarray(gpu_f, dtype=np.float64).reshape(3, -1)
    r = np.asarray(ref_f, dtype=np.float64).reshape(3, -1)
    sc = np.asarray(scale, dtype=np.float64).reshape(-1)
    net = np.sqrt((r**2).sum(axis=0))
    sel = (sc > floor * sc.max()) & (net >= share * sc)
    err = np.sqrt(((g[:, sel] - r[:, sel]) ** 2).sum(axis=0)) / net[sel]
    worst = float(err.max()) if err.size else 0.0
    print(f"{what}: worst |f|-relative error {worst:.3e} over {int(sel.sum())} cells "
          f"with |f| >= {share} chi E")
    assert worst <= rel, f"{what}: |f|-relative error {worst:.3e} over {sel.sum()} cells (> {rel})"
    return worst, int(sel.sum())


def conservation(chi_cell, G_phys, stats):
    """|sum chi G + escaped + dropped - L_in| / L_in from GPU outputs (FP64 on the host)."""
    absorbed = float((np.asarray(chi_cell, np.float64) * np.asarray(G_phys, np.float64)).sum())
    return abs(absorbed + stats["L_escaped"] + stats["L_dropped"] - stats["L_in"]) / stats["L_in"]
