"""Checkpoint layers (state_io): a state round-trips exactly, partial writes never appear,
the latest complete layer is found, and a solver interrupted after a checkpoint resumes to
the same result (parquet fixed point on the CPU stand-in map)."""

import numpy as np
import torch

from paper_2405_20996_gb300 import state_io
from test_parquet_host import _Toy


def test_round_trip_and_latest_layer(tmp_path):
    rng = np.random.default_rng(0)
    grids = dict(n1=5, n2w=3, n2v=4, n3w=3, n3v=2)
    ch = {c: (rng.standard_normal((5, 16)) + 1j, rng.standard_normal((3, 4, 16)) + 0j, None,
              torch.from_numpy(rng.standard_normal((3, 2, 2, 16)) * 1j)) for c in range(3)}
    sig = rng.standard_normal((7, 2))
    stem = str(tmp_path / "run")
    assert state_io.latest_layer(stem) is None
    for layer in (0, 1, 2):
        state_io.save_state(stem, layer, ch, grids, {"nq": 41, "U": 1.0}, label=0.1 * layer,
                            extra={"sigR": sig + layer})
    (tmp_path / "run.layer0003.npz.tmp").write_bytes(b"partial")       # an interrupted write
    path = state_io.latest_layer(stem)
    assert path.endswith("layer0002.npz")
    st = state_io.load_state(path)
    assert st["grids"] == grids and st["params"]["U"] == 1.0 and abs(st["label"] - 0.2) < 1e-15
    for c in range(3):
        a = ch[c]
        assert np.array_equal(st["channels"][c][0], a[0]) and np.array_equal(st["channels"][c][1], a[1])
        assert st["channels"][c][2] is None
        assert np.array_equal(st["channels"][c][3], a[3].numpy())
    assert np.array_equal(st["extra"]["sigR"], sig + 2) and set(st["extra"]) == {"sigR"}


def test_resume_from_checkpoint(tmp_path):
    stem = str(tmp_path / "pq")
    grids = dict(n1=12, n2w=1, n2v=1, n3w=1, n3v=1)
    saved = {}

    def ckpt(it, g, r):
        state_io.save_state(stem, it, {0: (g.numpy().reshape(12, 1), None, None, None)}, grids, {"mix": 0.5})
        saved["it"] = it

    full, h_full = _Toy().fixed_point(mix=0.5, tol=1e-13, maxit=2000)
    _Toy().fixed_point(mix=0.5, tol=1e-13, maxit=7, callback=ckpt)          # interrupted after 7 iterations
    st = state_io.load_state(state_io.latest_layer(stem))
    g0 = torch.from_numpy(st["channels"][0][0].reshape(12))
    resumed, h_res = _Toy().fixed_point(mix=0.5, tol=1e-13, maxit=2000, gamma0=g0)
    assert saved["it"] == 6
    assert torch.abs(resumed - full).max() <= 1e-12 * torch.abs(full).max()
    assert len(h_res) == len(h_full) - 7
