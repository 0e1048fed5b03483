"""Pixel tolerance of the FP32 path against the FP32-mode oracle, shared by the GPU
tests.

The FP32 path follows the oracle's sample positions and compositing order, so pixels
agree within 1e-5.  A ray whose transmittance passes within 0.1 % of the termination
threshold t_term may stop one sample earlier or later on one side (both are correct
roundings of the same product); one sample's weight is then at most t_term = 1e-4, so
those rays are held to 2e-4.  Every check reports how many rays were near the threshold
and how many of them actually needed the looser bound."""
import numpy as np

PIX_TOL = 1e-5
ERT_TOL = 2e-4


def check_pixels(pairs, ert_margin, label="", tol=PIX_TOL):
    """pairs: (got, expected) arrays of shape (n,) or (n, c).  Asserts the bounds and
    prints the near-threshold counts; returns (rays near the threshold, of them beyond
    tol)."""
    amb = np.asarray(ert_margin) < 1e-3
    worst = np.zeros(len(amb))
    for got, exp in pairs:
        g = np.asarray(got, np.float64).reshape(len(amb), -1)
        e = np.asarray(exp, np.float64).reshape(len(amb), -1)
        worst = np.maximum(worst, np.abs(g - e).max(axis=1))
    assert worst[~amb].max(initial=0.0) <= tol, (label, worst[~amb].max())
    assert worst[amb].max(initial=0.0) <= ERT_TOL, (label, worst[amb].max())
    n_amb, n_loose = int(amb.sum()), int((worst[amb] > tol).sum())
    print(f"[pixel tolerance] {label}: {n_amb} of {len(amb)} rays within 0.1 % of t_term, "
          f"{n_loose} of them beyond {tol:g} (max {worst[amb].max(initial=0.0):.2e})")
    return n_amb, n_loose
