"""Checkpoints of a calculation's state (the paper's layered output: one state per flow step
or parquet iteration, from which an interrupted run resumes, Sec. II.F).

A state is the vertex's reducible parts — per channel the classes K1, K2, K2', K3 in the
library's layout — plus the grids, the model parameters, a layer label (the flow parameter
Λ or the iteration) and optional extra arrays (e.g. the self-energy tables Σ^R, Σ^K).  Each layer is one compressed `.npz` file
`<stem>.layer<NNNN>.npz`; `latest_layer` finds the last complete one.  No HDF5 library is
needed.
"""

import glob
import json
import os
import re

import numpy as np

CLASS_NAMES = ("K1", "K2", "K2p", "K3")


def _np(a):
    return a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)


def save_state(stem, layer, channels, grids, params, label=None, extra=None):
    """Write layer `layer` of `stem`: channels {c: (K1, K2, K2p, K3)} (arrays or tensors),
    grids {n1, n2w, n2v, n3w, n3v}, params (JSON-serialisable, e.g. nq, U, Delta, T), extra
    {name: array} (e.g. Σ tables).
    Written to a temporary file and renamed, so a crash never leaves a partial layer."""
    arrays = {}
    for c, classes in channels.items():
        for k, a in zip(CLASS_NAMES, classes):
            if a is None:
                continue
            arrays["ch%d_%s" % (int(c), k)] = _np(a)
    for name, a in (extra or {}).items():
        arrays["x_" + name] = _np(a)
    meta = {"grids": dict(grids), "params": params, "label": label, "layer": int(layer)}
    path = "%s.layer%04d.npz" % (stem, int(layer))
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez_compressed(f, __meta__=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8), **arrays)
    os.replace(tmp, path)
    return path


def load_state(path):
    """{"channels": {c: (K1, K2, K2p, K3)}, "grids", "params", "label", "layer", "extra"} of
    a layer."""
    with np.load(path) as z:
        meta = json.loads(bytes(z["__meta__"]).decode())
        channels, extra = {}, {}
        for key in z.files:
            m = re.fullmatch(r"ch(\d)_(K1|K2|K2p|K3)", key)
            if m:
                channels.setdefault(int(m.group(1)), [None] * 4)[CLASS_NAMES.index(m.group(2))] = z[key]
            elif key.startswith("x_"):
                extra[key[2:]] = z[key]
    meta["channels"] = {c: tuple(v) for c, v in channels.items()}
    meta["extra"] = extra
    return meta


def latest_layer(stem):
    """Path of the highest complete layer of `stem`, or None."""
    paths = sorted(glob.glob(glob.escape(stem) + ".layer*.npz"))
    return paths[-1] if paths else None
