"""Helpers of the GPU-vs-oracle parity tests (comparison rules in one place)."""
import numpy as np

# Tolerances of the parity bar: per-cell gamma and force within 1e-5 relative where the
# deposit exceeds 1e-6 of the peak; photon conservation within 1e-6 relative.
REL = 1e-5
FLOOR = 1e-6
CONS = 1e-6


def compare_field(gpu, ref, rel=REL, floor=FLOOR, what="field"):
    """Max relative error over cells whose |ref| exceeds floor * max|ref|; returns it."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    peak = np.abs(ref).max()
    sel = np.abs(ref) > floor * peak
    err = np.abs(gpu[sel] - ref[sel]) / np.abs(ref[sel])
    worst = float(err.max()) if err.size else 0.0
    assert worst <= rel, f"{what}: max rel err {worst:.3e} over {sel.sum()} cells (> {rel})"
    # cells below the floor must still be small in absolute terms
    small = np.abs(gpu[~sel] - ref[~sel]).max() if (~sel).any() else 0.0
    assert small <= 10 * floor * peak, f"{what}: sub-floor cells off by {small:.3e}"
    return worst


def compare_force(gpu_f, ref_f, scale, rel=REL, floor=FLOOR):
    """Force vectors. The error of each component is measured against the cell's
    flux-limited bound chi E (|f_rad| = chi |F| / c <= chi E, Sec. 2.1): where many rays of
    opposite directions cross a cell the net force is a near-total cancellation, which an
    FP32 sum cannot resolve relative to the net itself. Cells whose chi E exceeds floor of
    the peak are checked."""
    g = np.asarray(gpu_f, dtype=np.float64).reshape(3, -1)
    r = np.asarray(ref_f, dtype=np.float64).reshape(3, -1)
    sc = np.asarray(scale, dtype=np.float64).reshape(-1)
    assert np.all(np.sqrt((r**2).sum(axis=0)) <= sc * (1 + 1e-9) + 1e-300)
    sel = sc > floor * sc.max()
    err = np.abs(g[:, sel] - r[:, sel]).max(axis=0) / sc[sel]
    worst = float(err.max()) if err.size else 0.0
    assert worst <= rel, f"force: max rel err {worst:.3e} over {sel.sum()} cells"
    return worst


def conservation(chi_cell, G_phys, stats):
    """|sum chi G + escaped + dropped - L_in| / L_in from GPU outputs (FP64 on the host)."""
    absorbed = float((np.asarray(chi_cell, np.float64) * np.asarray(G_phys, np.float64)).sum())
    return abs(absorbed + stats["L_escaped"] + stats["L_dropped"] - stats["L_in"]) / stats["L_in"]
