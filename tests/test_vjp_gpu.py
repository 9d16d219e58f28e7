"""Adjoint of the bubble on the GPU (kb_bubble_vjp through the C ABI): element-wise parity
with the oracle's VJP (vertex gradients of both sides and the G^R gradient table) for the
plain FP64 form (1e-10) and the mixed form (complex64 vertex, FP32 records, tiles and GEMMs,
FP64 accumulation of the scatter; 1e-6 of the largest gradient, the forward's bar), the
torch.autograd front end against central finite differences on 64 seeded directions (step
1e-4), and the refused combinations."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS, RAGGED, rel_err
from oracle import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _engine(cfg):
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(cfg["grids"], cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"], cfg.get("eps", 0.0))
    return e


def _cgauss(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def _grad_slot(e, slot):
    import paper_2405_20996_gb300.kb as kb
    kb.kb_set_vertex(e.ctx, slot, False, 0.0)
    e.tensors[slot] = {}
    sh = e.class_shapes()
    for c in range(3):
        for k in range(4):
            e.attach(slot, c, k, torch.zeros(sh[CLS[k]], dtype=torch.complex128, device=e.device))


def _slot_numpy(e, slot):
    return {c: [e.tensors[slot][(c, k)].cpu().numpy() for k in range(4)] for c in range(3)}


def _max_rel(got, ref):
    scale = max(np.abs(ref[c][k]).max() for c in range(3) for k in range(4))
    return max(np.abs(got[c][k] - ref[c][k]).max() for c in range(3) for k in range(4)) / max(scale, 1e-300)


TOL_MIXED = 1e-6


def _c64(ch):
    return {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("r", [0, 1, 2])
def test_vjp_matches_oracle_ragged(r, precision):
    cfg = dict(RAGGED, eps=0.05)
    g = cfg["grids"]
    chL = S.seeded_vertex(g, cfg["U"], seed=31)
    chR = S.seeded_vertex(g, cfg["U"], seed=32)
    e = _engine(cfg)
    dt = torch.complex64 if precision == "mixed" else torch.complex128
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=chL, dtype=dt)
    e.set_vertex(1, U=cfg["U"], has_R=True, channels=chR, dtype=dt)
    if precision == "mixed":
        chL, chR = _c64(chL), _c64(chR)
    VL = O.Vertex(g, U=cfg["U"], has_R=True, channels=chL)
    VR = O.Vertex(g, U=cfg["U"], has_R=True, channels=chR)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], eps=cfg["eps"])
    rng = np.random.default_rng(40 + r)
    e.alloc_out(2, channels=(r,))
    gbar = {}
    for k, name in enumerate(CLS):
        gbar[name] = _cgauss(rng, e.class_shapes()[name])
        e.tensors[2][(r, k)].copy_(torch.from_numpy(gbar[name]))
    _grad_slot(e, 3)
    _grad_slot(e, 4)
    tabs = e.gr_tables()
    alpha = 0.75
    e.bubble_vjp(r, 0, 1, 2, alpha=alpha, grad_left=3, grad_right=4, grad_gr=tabs, precision=precision)
    torch.cuda.synchronize()
    gl_ref, gr_ref = O.zero_grads(g), O.zero_grads(g)
    tab_ref = {"K1": 0, "K2": 0, "K3": 0}
    for name in CLS:
        a, b, t = O.bubble_vjp(VL, VR, P, r, name, cfg["nq"], alpha * gbar[name], want_gr=True)
        for c in range(3):
            for k in range(4):
                gl_ref[c][k] += a[c][k]
                gr_ref[c][k] += b[c][k]
        tab_ref["K2" if name == "K2p" else name] = tab_ref["K2" if name == "K2p" else name] + t
    tol = TOL if precision == "fp64" else TOL_MIXED
    errs = [_max_rel(_slot_numpy(e, 3), gl_ref), _max_rel(_slot_numpy(e, 4), gr_ref)]
    errs += [rel_err(tabs[name].cpu().numpy(), tab_ref[name]) for name in ("K1", "K2", "K3")]
    print("vjp %s r=%d: left %.2e right %.2e G^R K1 %.2e K2 %.2e K3 %.2e" % ((precision, r) + tuple(errs)))
    assert max(errs) <= tol, errs


def test_autograd_vs_central_differences():
    """B(Γ, Γ) summed over all classes of the t channel (the up-up spin terms included):
    64 seeded directions, central differences with step 1e-4."""
    from paper_2405_20996_gb300.autograd import bubble
    cfg = dict(grids=dict(n1=21, n2w=9, n2v=7, n3w=5, n3v=7), nq=41, U=1.2, Delta=1.0, T=0.1)
    g = cfg["grids"]
    e = _engine(cfg)
    ch = S.seeded_vertex(g, cfg["U"], seed=50)
    dev = e.device
    gam = {c: tuple(torch.tensor(a, dtype=torch.complex128, device=dev, requires_grad=True) for a in v)
           for c, v in ch.items()}
    rng = np.random.default_rng(51)
    gbar = {n: torch.tensor(_cgauss(rng, e.class_shapes()[n]), device=dev) for n in CLS}
    kw = dict(U_left=cfg["U"], has_R_left=True, U_right=cfg["U"], has_R_right=True)

    def loss(v):
        out = bubble(e, 2, v, v, **kw)
        return sum(torch.real(torch.vdot(gbar[n].flatten(), out[n].flatten())) for n in CLS)

    L = loss(gam)
    L.backward()
    grads = {c: [t.grad.clone() for t in gam[c]] for c in range(3)}
    h = 1e-4
    worst = 0.0
    with torch.no_grad():
        for i in range(64):
            rd = np.random.default_rng(1000 + i)
            d = {c: tuple(torch.tensor(_cgauss(rd, tuple(t.shape)), device=dev) for t in gam[c]) for c in range(3)}
            plus = {c: tuple(t + h * dt for t, dt in zip(gam[c], d[c])) for c in range(3)}
            minus = {c: tuple(t - h * dt for t, dt in zip(gam[c], d[c])) for c in range(3)}
            fd = (loss(plus) - loss(minus)).item() / (2 * h)
            ad = sum(torch.real(torch.vdot(grads[c][k].flatten(), d[c][k].flatten())).item()
                     for c in range(3) for k in range(4))
            worst = max(worst, abs(fd - ad) / max(abs(fd), 1e-12))
    assert worst <= 1e-7, worst


def test_autograd_complex64_matches_complex128():
    """The autograd front end on complex64 vertices (mixed forward and adjoint) against the
    same values in complex128 (plain FP64): outputs and both-side gradients of B(Γ, Γ) in
    the t channel, to 1e-6 of the largest entry."""
    from paper_2405_20996_gb300.autograd import bubble
    cfg = dict(grids=dict(n1=21, n2w=9, n2v=7, n3w=5, n3v=7), nq=41, U=1.2, Delta=1.0, T=0.1)
    g = cfg["grids"]
    e = _engine(cfg)
    ch = _c64(S.seeded_vertex(g, cfg["U"], seed=52))
    rng = np.random.default_rng(53)
    gbar = {n: _cgauss(rng, e.class_shapes()[n]) for n in CLS}
    kw = dict(U_left=cfg["U"], has_R_left=True, U_right=cfg["U"], has_R_right=True)
    res = {}
    for dt in (torch.complex128, torch.complex64):
        gam = {c: tuple(torch.tensor(a, dtype=dt, device=e.device, requires_grad=True) for a in v)
               for c, v in ch.items()}
        out = bubble(e, 2, gam, gam, **kw)
        L = sum(torch.real(torch.vdot(torch.tensor(gbar[n], dtype=dt, device=e.device).flatten(),
                                      out[n].flatten())) for n in CLS)
        L.backward()
        assert all(t.grad.dtype == dt for c in range(3) for t in gam[c])
        res[dt] = ({n: out[n].detach().cpu().numpy() for n in CLS},
                   {c: [t.grad.cpu().numpy() for t in gam[c]] for c in range(3)})
    o64, g64 = res[torch.complex64]
    o128, g128 = res[torch.complex128]
    for n in CLS:
        assert rel_err(o64[n], o128[n]) <= 1e-6, n
    assert _max_rel(g64, g128) <= 1e-6, _max_rel(g64, g128)


def test_vjp_refusals():
    import paper_2405_20996_gb300.kb as kb
    cfg = dict(RAGGED)
    g = cfg["grids"]
    e = _engine(cfg)
    ch = S.seeded_vertex(g, cfg["U"], seed=60)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch)
    e.alloc_out(2, channels=(0,))
    _grad_slot(e, 3)
    with pytest.raises(kb.KBError) as ex:                 # the mixed form reads complex64 vertices
        e.bubble_vjp(0, 0, 0, 2, grad_left=3, precision="mixed")
    assert ex.value.status == kb.KB_ERR_ARG
    e.set_self_energy(S.seeded_sigma(17, seed=1), np.zeros(17, dtype=np.complex128))
    with pytest.raises(kb.KBError) as ex:
        e.bubble_vjp(0, 0, 0, 2, grad_gr=e.gr_tables())
    assert ex.value.status == kb.KB_ERR_UNSUPPORTED
    e.set_self_energy(None)
    e.attach(3, 0, 0, torch.zeros((g["n1"], 16), dtype=torch.complex64, device=e.device))
    with pytest.raises(kb.KBError) as ex:
        e.bubble_vjp(0, 0, 0, 2, grad_left=3)
    assert ex.value.status == kb.KB_ERR_ARG


CFG3 = dict(grids=dict(n1=201, n2w=81, n2v=81, n3w=41, n3v=41), nq=4001, U=1.0, Delta=1.0, T=0.1)


@pytest.mark.parametrize("r", [0, 2])
def test_mixed_vjp_full_size_vs_fp64(r):
    """K1 201, K2 81², K3 41³, Nq 4001 (the parquet-solve workload): the mixed adjoint of all
    four classes against the plain FP64 adjoint (itself pinned to the oracle above), every
    element of both vertex gradients and of the G^R tables; prints the two times."""
    cfg = CFG3
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=70 + r)
    rng = np.random.default_rng(80 + r)
    e = _engine(cfg)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=torch.complex64)
    e.set_vertex(1, U=cfg["U"], has_R=True, channels=_c64(ch))       # the same values in complex128
    e.alloc_out(2, channels=(r,))
    for k, name in enumerate(CLS):
        e.tensors[2][(r, k)].copy_(torch.from_numpy(_cgauss(rng, e.class_shapes()[name])))
    res, ms = {}, {}
    for prec, src, gs in (("fp64", 1, (3, 4)), ("mixed", 0, (5, 6))):
        _grad_slot(e, gs[0])
        _grad_slot(e, gs[1])
        tabs = e.gr_tables()
        e.bubble_vjp(r, src, src, 2, alpha=0.5, grad_left=gs[0], grad_right=gs[1], grad_gr=tabs, precision=prec)
        torch.cuda.synchronize()
        for s in gs:                                      # time a second call on zeroed slots
            for t in e.tensors[s].values():
                t.zero_()
        for t in tabs.values():
            t.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        e.bubble_vjp(r, src, src, 2, alpha=0.5, grad_left=gs[0], grad_right=gs[1], grad_gr=tabs, precision=prec)
        b.record()
        torch.cuda.synchronize()
        ms[prec] = a.elapsed_time(b)
        res[prec] = (_slot_numpy(e, gs[0]), _slot_numpy(e, gs[1]), {n: t.cpu().numpy() for n, t in tabs.items()})
    errs = [_max_rel(res["mixed"][0], res["fp64"][0]), _max_rel(res["mixed"][1], res["fp64"][1])]
    errs += [rel_err(res["mixed"][2][n], res["fp64"][2][n]) for n in ("K1", "K2", "K3")]
    print("vjp full size r=%d: fp64 %.1f ms, mixed %.1f ms; errors %s" % (r, ms["fp64"], ms["mixed"],
                                                                          ["%.2e" % x for x in errs]))
    assert max(errs) <= TOL_MIXED, errs
