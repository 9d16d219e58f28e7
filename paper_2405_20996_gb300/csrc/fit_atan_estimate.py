"""Fit of the cell-estimate polynomial used by x_est in kb_mixed.cuh:
(2/pi) atan(u) ~ u (c0 + c1 u^2 + c2 u^4 + c3 u^6) on u in [0, 1], by iteratively
reweighted least squares toward the minimax fit.  Prints the coefficients (as FP32) and
the maximum error; the kernel only needs the estimate to fall within one grid cell."""
import numpy as np


def fit(nterm=4, iters=60):
    u = np.concatenate([np.cos(np.linspace(0, np.pi / 2, 20001)), np.linspace(0, 1, 20001)])
    f = (2 / np.pi) * np.arctan(u)
    M = np.stack([u ** (2 * i + 1) for i in range(nterm)], 1)
    w = np.ones_like(u)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(M * w[:, None], f * w, rcond=None)
        e = M @ c - f
        w = w * np.sqrt(np.abs(e) / np.abs(e).max() + 1e-3)
        w /= w.max()
    c32 = c.astype(np.float32)
    err = np.abs(M @ c32.astype(np.float64) - f).max()
    return c32, err


if __name__ == "__main__":
    c, err = fit()
    print("coefficients", [float(x) for x in c], "max error", err)
