"""torch.autograd front end of the bubble: B_r(Γ_left, Γ_right) as a differentiable
function of the vertices' stored classes (complex128), with the backward pass computed by
the library's adjoint kernels (kb_bubble_vjp).  Gradients follow PyTorch's convention for
complex tensors (dL/dRe + i dL/dIm of a real loss L).

A vertex is a dict {channel: (K1, K2, K2p, K3)} of complex128 CUDA tensors (None = absent).
Passing the same tensors for both sides gives B(Γ, Γ); autograd then adds the left and
right contributions.  The bare part (U, has_R) is a fixed parameter.
"""

import torch

from . import kb
from .engine import CLASS_NAMES

# slots reserved on the engine for the autograd front end
S_LEFT, S_RIGHT, S_OUT, S_GLEFT, S_GRIGHT = 11, 12, 13, 14, 15


def _flatten(vertex, eng):
    sh = eng.class_shapes()
    out = []
    for c in range(3):
        cls = (vertex or {}).get(c, (None,) * 4)
        for k in range(4):
            t = cls[k]
            if t is None:
                t = torch.zeros(sh[CLASS_NAMES[k]], dtype=torch.complex128, device=eng.device)
            if t.dtype != torch.complex128 or not t.is_cuda:
                raise TypeError("bubble autograd needs complex128 CUDA tensors")
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
        eng.alloc_out(S_OUT, channels=(channel,), dtype=torch.complex128)
        eng.bubble(channel, S_LEFT, S_RIGHT, S_OUT, pi_kind=pi_kind, class_mask=mask, precision="fp64")
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
        need = ctx.needs_input_grad[2:]
        want_l, want_r = any(need[:12]), any(need[12:])
        _attach(eng, S_LEFT, left, UL, RL, incL)
        _attach(eng, S_RIGHT, right, UR, RR, incR)
        sh = eng.class_shapes()
        kb.kb_set_vertex(eng.ctx, S_OUT, False, 0.0)
        eng.tensors[S_OUT] = {}
        for k, g in enumerate(gouts):
            if g is None:
                g = torch.zeros(sh[CLASS_NAMES[k]], dtype=torch.complex128, device=eng.device)
            eng.attach(S_OUT, channel, k, g.to(torch.complex128).contiguous())
        grads = []
        for slot, want in ((S_GLEFT, want_l), (S_GRIGHT, want_r)):
            gl = [torch.zeros_like(t) for t in (left if slot == S_GLEFT else right)] if want else None
            if want:
                kb.kb_set_vertex(eng.ctx, slot, False, 0.0)
                eng.tensors[slot] = {}
                for i, t in enumerate(gl):
                    eng.attach(slot, i // 4, i % 4, t)
            grads.append(gl)
        eng.bubble_vjp(channel, S_LEFT, S_RIGHT, S_OUT, pi_kind=pi_kind, class_mask=mask,
                       grad_left=S_GLEFT if want_l else -1, grad_right=S_GRIGHT if want_r else -1)
        gl = grads[0] or [None] * 12
        gr = grads[1] or [None] * 12
        return (None, None, *gl, *gr)


def bubble(eng, channel, left, right, U_left=0.0, has_R_left=False, include_left=(0, 1, 2), U_right=0.0,
           has_R_right=False, include_right=(0, 1, 2), pi_kind=kb.KB_PI_GG, class_mask=kb.KB_MASK_ALL):
    """Differentiable FP64 bubble B_r(Γ_left, Γ_right); returns {"K1", "K2", "K2p", "K3"}
    tensors of channel r (classes outside class_mask are zero)."""
    spec = (channel, pi_kind, class_mask, float(U_left), bool(has_R_left), tuple(include_left), float(U_right),
            bool(has_R_right), tuple(include_right))
    outs = _Bubble.apply(eng, spec, *_flatten(left, eng), *_flatten(right, eng))
    return dict(zip(CLASS_NAMES, outs))
