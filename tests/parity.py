"""Shared helpers of the parity tests (the oracle against the CUDA path)."""
import numpy as np

# FP32 sweep against the FP64 oracle: max relative error on every value above
# 1e-6 of its group's maximum.
REL_TOL = 1e-4
FLOOR = 1e-6


def max_rel(gpu, ref, floor=FLOOR):
    """Max over groups (rows) of max |gpu - ref| / |ref| on |ref| > floor * max|ref|."""
    gpu = np.atleast_2d(np.asarray(gpu, np.float64))
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    worst = 0.0
    for a, b in zip(gpu, ref):
        m = np.abs(b).max()
        if m == 0.0:
            worst = max(worst, float(np.abs(a).max()))
            continue
        sel = np.abs(b) > floor * m
        worst = max(worst, float((np.abs(a[sel] - b[sel]) / np.abs(b[sel])).max()))
    return worst
