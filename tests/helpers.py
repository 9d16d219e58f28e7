"""Shared test helpers: build matching oracle and GPU inputs from the seeded generator."""

import numpy as np

import seeded as S
from oracle import oracle as O

CLS = ("K1", "K2", "K2p", "K3")

CFG0 = dict(grids=dict(n1=101, n2w=21, n2v=21, n3w=15, n3v=15), nq=1001, U=1.0, Delta=1.0, T=0.1)
CFG1 = dict(grids=dict(n1=401, n2w=101, n2v=101, n3w=51, n3v=51), nq=4001, U=2.0, Delta=1.0, T=0.05)
# ragged sizes that span several 32-wide tiles in every GEMM dimension
RAGGED = dict(grids=dict(n1=37, n2w=13, n2v=11, n3w=9, n3v=11), nq=201, U=1.5, Delta=1.0, T=0.2)


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def seeded_inputs(cfg, seed=0, channels=(0, 1, 2)):
    return S.seeded_vertex(cfg["grids"], cfg["U"], seed=seed, channels=channels)


def oracle_vertex(cfg, ch, has_R=True):
    return O.Vertex(cfg["grids"], U=cfg["U"], has_R=has_R, channels=ch)
