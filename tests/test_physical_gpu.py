"""Physical-only Keldysh structure on the GPU (kb_keldysh_check, kb_vertex_pack/unpack):

- on the oracle's converged parquet solution the parity-structure residual of every class
  is exactly 0 (complex128 and complex64), and the K1 equilibrium residuals (causality,
  conjugation, FDR) equal a host computation on the same arrays; on a seeded vertex the
  structure residuals are of order one;
- the second-order K1 (a bubble of bare vertices, channels a and p) satisfies the bosonic
  FDR and K1^A = (K1^R)* to the quadrature's accuracy;
- packing keeps exactly the representatives, unpacking restores a physical class exactly,
  and unpacking a non-physical class gives its projection (every component replaced by its
  representative)."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS
from oracle import oracle as O

pytestmark = pytest.mark.gpu

G = dict(n1=13, n2w=7, n2v=6, n3w=5, n3v=4)
PAIRS = {0: ((0, 3), (2, 1)), 1: ((0, 1), (2, 3)), 2: ((0, 2), (1, 3))}


def _key(r, k, c):
    b = ((c >> 3) & 1, (c >> 2) & 1, (c >> 1) & 1, c & 1)
    (l0, l1), (r0, r1) = PAIRS[r]
    x, y, xp, yp = b[l0], b[l1], b[r0], b[r1]
    return [2 * (x ^ y) + (xp ^ yp), 4 * x + 2 * y + (xp ^ yp), 4 * (x ^ y) + 2 * xp + yp, c][k]


def _rep(r, k):
    rep = {}
    for c in range(16):
        rep.setdefault(_key(r, k, c), c)
    return [rep[d] for d in sorted(rep)]


def _parquet(g, nq, U, P, iters=25):
    gam = {c: [np.zeros(O.class_shape(g, k), dtype=np.complex128) for k in CLS] for c in range(3)}
    for _ in range(iters):
        Gam = O.Vertex(g, U=U, has_R=True, channels=gam)
        new = {r: O.bubble_all(O.Vertex(g, U=U, has_R=True, channels=gam, include=[c for c in range(3) if c != r]),
                               Gam, P, r, nq) for r in range(3)}
        gam = {c: [0.5 * gam[c][k] + 0.5 * new[c][CLS[k]] for k in range(4)] for c in range(3)}
    return gam


def _host_k1(K1, r, T):
    w = O.grid(K1.shape[0])
    cR = 8 if r == 1 else 1
    dR = _key(r, 0, cR)
    dA = 2 * (dR & 1) + (dR >> 1)
    rep = _rep(r, 0)
    R, A, K, Z = K1[:, cR], K1[:, rep[dA]], K1[:, rep[3]], K1[:, rep[0]]
    m = np.abs(K1).max()
    th = np.tanh(w / (2 * T))
    return (np.abs(Z).max() / m, np.abs(A - np.conj(R)).max() / m, np.abs(th * K - (R - A)).max() / m)


@pytest.fixture(scope="module")
def parquet():
    return _parquet(G, 41, 1.0, O.Prop(Delta=1.0, T=0.2))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_parquet_solution_is_physical(parquet, dtype):
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(G, 41)
    e.set_model(1.0, 0.2)
    e.set_vertex(0, U=1.0, has_R=True, channels={c: tuple(parquet[c]) for c in range(3)}, dtype=dtype)
    e.set_vertex(1, U=1.0, has_R=True, channels=S.seeded_vertex(G, 1.0, seed=3), dtype=dtype)
    for r in range(3):
        res = e.keldysh_check(0, r, 0.2)
        assert [res[n] for n in CLS] == [0.0, 0.0, 0.0, 0.0], (r, res)
        K1 = e.tensors[0][(r, 0)].cpu().numpy().astype(np.complex128)
        host = _host_k1(K1, r, 0.2)
        for name, h in zip(("causality", "conjugation", "fdr"), host):
            assert abs(res[name] - h) <= 1e-6 * max(h, 1e-300) + 1e-15, (r, name, res[name], h)
        assert max(host) < 0.05                  # equilibrium relations to the coarse grids' accuracy
        rs = e.keldysh_check(1, r, 0.2)
        assert min(rs["K1"], rs["K2"], rs["K2p"]) > 0.1 and rs["K3"] == 0.0, (r, rs)
    e.close()


@pytest.mark.parametrize("r", [0, 1])
def test_second_order_k1_fdr(r):
    from paper_2405_20996_gb300.engine import Engine
    g = dict(n1=31, n2w=9, n2v=9, n3w=7, n3v=7)
    T = 0.1
    V = O.Vertex(g, U=1.0, has_R=True)
    K1 = O.bubble_class(V, V, O.Prop(Delta=1.0, T=T), r, "K1", 1001)
    e = Engine(g, 1001)
    e.set_model(1.0, T)
    e.set_vertex(0, channels={r: (K1, None, None, None)}, include=(r,))
    res = e.keldysh_check(0, r, T)
    host = _host_k1(K1, r, T)
    for name, h in zip(("causality", "conjugation", "fdr"), host):
        assert abs(res[name] - h) <= 1e-6 * max(h, 1e-300) + 1e-15, (name, res[name], h)
    assert res["K1"] <= 1e-14 and res["conjugation"] <= 1e-13, res
    # causality and the FDR to the quadrature's accuracy (6.8e-6 here, from the outermost
    # frequencies of the K1 grid)
    assert res["fdr"] <= 2e-5 and res["causality"] <= 2e-5, res
    e.close()


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_pack_unpack(parquet, dtype):
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(G, 41)
    e.set_model(1.0, 0.2)
    e.set_vertex(0, U=1.0, has_R=True, channels={c: tuple(parquet[c]) for c in range(3)}, dtype=dtype)
    seeded = S.seeded_vertex(G, 1.0, seed=4)
    e.set_vertex(1, U=1.0, has_R=True, channels=seeded, dtype=dtype)
    for r in range(3):
        for k in range(4):
            X = e.tensors[0][(r, k)].clone()
            p = e.pack_physical(0, r, k)
            assert p.shape == (X.numel() // 16, (4, 8, 8, 16)[k])
            assert torch.equal(p, X.reshape(-1, 16)[:, _rep(r, k)])
            e.tensors[0][(r, k)].zero_()
            e.unpack_physical(0, r, k, p)
            assert torch.equal(e.tensors[0][(r, k)], X)
            # a non-physical class comes back as its projection
            Y = e.tensors[1][(r, k)].clone().reshape(-1, 16)
            e.unpack_physical(1, r, k, e.pack_physical(1, r, k))
            proj = Y[:, [_rep(r, k)[_key(r, k, c)] for c in range(16)]]
            assert torch.equal(e.tensors[1][(r, k)].reshape(-1, 16), proj)
    e.close()
