"""torch.autograd front end of the bubble: B_r(Γ_left, Γ_right) as a differentiable
function of the vertices' stored classes, with the backward pass computed by the library's
adjoint kernels (kb_bubble_vjp).  Gradients follow PyTorch's convention for complex tensors
(dL/dRe + i dL/dIm of a real loss L).

A vertex is a dict {channel: (K1, K2, K2p, K3)} of CUDA tensors (None = absent), all
complex128 (the plain FP64 bubble and adjoint) or all complex64 (the mixed-precision forms;
the adjoint accumulates in complex128 and the gradients are returned as complex64).
Passing the same tensors for both sides gives B(Γ, Γ); autograd then adds the left and
right contributions.  The bare part (U, has_R) is a fixed parameter.
"""

import torch

from . import kb
from .engine import CLASS_NAMES

# slots reserved on the engine for the autograd front end
S_LEFT, S_RIGHT, S_OUT, S_GLEFT, S_GRIGHT = 11, 12, 13, 14, 15


def _flatten(vertices, eng):
    present = [t for v in vertices for c in range(3) for t in (v or {}).get(c, (None,) * 4) if t is not None]
    dtype = present[0].dtype if present else torch.complex128
    if dtype not in (torch.complex128, torch.complex64):
        raise TypeError("bubble autograd needs complex128 or complex64 CUDA tensors")
    sh = eng.class_shapes()
    out = []
    for vertex in vertices:
        for c in range(3):
            cls = (vertex or {}).get(c, (None,) * 4)
            for k in range(4):
                t = cls[k]
                if t is None:
                    t = torch.zeros(sh[CLASS_NAMES[k]], dtype=dtype, device=eng.device)
                if t.dtype != dtype or not t.is_cuda:
                    raise TypeError("bubble autograd needs CUDA tensors of one dtype (complex128 or complex64)")
                out.append(t)
    return out


def _attach(eng, slot, flat, U, has_R, include):
    kb.kb_set_vertex(eng.ctx, slot, has_R, U)
    kb.kb_set_vertex_channels(eng.ctx, slot, sum(1 << c for c in include))
    kb.kb_set_vertex_symmetric(eng.ctx, slot, False)
    eng.tensors[slot] = {}
    for i, t in enumerate(flat):
        eng.attach(slot, i // 4, i % 4, t.contiguous())


class _Bubble(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eng, spec, *flat):
        channel, pi_kind, mask, UL, RL, incL, UR, RR, incR = spec
        left, right = flat[:12], flat[12:]
        _attach(eng, S_LEFT, left, UL, RL, incL)
        _attach(eng, S_RIGHT, right, UR, RR, incR)
        dt = flat[0].dtype
        eng.alloc_out(S_OUT, channels=(channel,), dtype=dt)
        eng.bubble(channel, S_LEFT, S_RIGHT, S_OUT, pi_kind=pi_kind, class_mask=mask,
                   precision="fp64" if dt == torch.complex128 else "mixed")
        outs = eng.out(S_OUT, channel)
        ctx.eng, ctx.spec = eng, spec
        ctx.save_for_backward(*flat)
        return tuple(outs[n].clone() for n in CLASS_NAMES)

    @staticmethod
    def backward(ctx, *gouts):
        eng, spec = ctx.eng, ctx.spec
        channel, pi_kind, mask, UL, RL, incL, UR, RR, incR = spec
        flat = ctx.saved_tensors
        left, right = flat[:12], flat[12:]
        dt = flat[0].dtype
        need = ctx.needs_input_grad[2:]
        want_l, want_r = any(need[:12]), any(need[12:])
        _attach(eng, S_LEFT, left, UL, RL, incL)
        _attach(eng, S_RIGHT, right, UR, RR, incR)
        sh = eng.class_shapes()
        kb.kb_set_vertex(eng.ctx, S_OUT, False, 0.0)
        eng.tensors[S_OUT] = {}
        for k, g in enumerate(gouts):
            if g is None:
                g = torch.zeros(sh[CLASS_NAMES[k]], dtype=dt, device=eng.device)
            eng.attach(S_OUT, channel, k, g.to(dt).contiguous())
        grads = []
        for slot, want in ((S_GLEFT, want_l), (S_GRIGHT, want_r)):
            gl = ([torch.zeros(t.shape, dtype=torch.complex128, device=t.device)
                   for t in (left if slot == S_GLEFT else right)] if want else None)
            if want:
                kb.kb_set_vertex(eng.ctx, slot, False, 0.0)
                eng.tensors[slot] = {}
                for i, t in enumerate(gl):
                    eng.attach(slot, i // 4, i % 4, t)
            grads.append(gl)
        eng.bubble_vjp(channel, S_LEFT, S_RIGHT, S_OUT, pi_kind=pi_kind, class_mask=mask,
                       grad_left=S_GLEFT if want_l else -1, grad_right=S_GRIGHT if want_r else -1,
                       precision="fp64" if dt == torch.complex128 else "mixed")
        gl = [t.to(dt) for t in grads[0]] if grads[0] else [None] * 12
        gr = [t.to(dt) for t in grads[1]] if grads[1] else [None] * 12
        return (None, None, *gl, *gr)


def bubble(eng, channel, left, right, U_left=0.0, has_R_left=False, include_left=(0, 1, 2), U_right=0.0,
           has_R_right=False, include_right=(0, 1, 2), pi_kind=kb.KB_PI_GG, class_mask=kb.KB_MASK_ALL):
    """Differentiable bubble B_r(Γ_left, Γ_right), plain FP64 for complex128 vertices and
    mixed precision for complex64 ones; returns {"K1", "K2", "K2p", "K3"} tensors of
    channel r (classes outside class_mask are zero)."""
    spec = (channel, pi_kind, class_mask, float(U_left), bool(has_R_left), tuple(include_left), float(U_right),
            bool(has_R_right), tuple(include_right))
    outs = _Bubble.apply(eng, spec, *_flatten((left, right), eng))
    return dict(zip(CLASS_NAMES, outs))
