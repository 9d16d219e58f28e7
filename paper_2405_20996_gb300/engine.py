"""PyTorch-facing helper around the C ABI: owns the device tensors of the vertex slots
(PyTorch is used for device memory and streams only) and calls kb_bubble."""

import torch

from . import kb

CLASS_NAMES = ("K1", "K2", "K2p", "K3")
DT = {torch.complex128: kb.KB_DT_C128, torch.complex64: kb.KB_DT_C64}
PREC = {"fp64": kb.KB_PREC_FP64, "mixed": kb.KB_PREC_MIXED}


class Engine:
    def __init__(self, grids, nq, A=5.0, device=0):
        self.device = torch.device("cuda", device)
        self.grids = dict(grids)
        self.nq, self.A = nq, A
        self.ctx = kb.kb_create(device)
        g = self.grids
        kb.kb_set_grids(self.ctx, g["n1"], g["n2w"], g["n2v"], g["n3w"], g["n3v"], nq, A)
        self.tensors = {}

    def close(self):
        if self.ctx is not None:
            kb.kb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def class_shapes(self):
        g = self.grids
        return {"K1": (g["n1"], 16), "K2": (g["n2w"], g["n2v"], 16), "K2p": (g["n2w"], g["n2v"], 16),
                "K3": (g["n3w"], g["n3v"], g["n3v"], 16)}

    def set_model(self, Delta, T, eps=0.0):
        kb.kb_set_model(self.ctx, Delta, T, eps)

    def set_regulator(self, kind, lam=1.0):
        """Flow scheme of the single-scale propagator (kb.KB_REG_DELTA / _U / _T)."""
        kb.kb_set_regulator(self.ctx, kind, lam)

    def set_self_energy_derivative(self, dsigR=None, dsigK=None, A_dsig=5.0):
        """dΣ/dΛ tables: the Katanin substitution S -> S + G dΣ G in Π-dot."""
        kb.kb_set_self_energy_derivative(self.ctx, dsigR, dsigK, A_dsig)

    def set_self_energy(self, sigR=None, sigK=None, A_sig=5.0):
        kb.kb_set_self_energy(self.ctx, sigR, sigK, A_sig)

    def set_propagator_table(self, which, tabR=None, tabK=None, A_tab=5.0):
        """Tabulated line (which: "G" or "S"): retarded and Keldysh parts on the tan grid of
        scale A_tab; tabR None removes it (kb_set_propagator_table)."""
        w = {"G": kb.KB_PROP_G, "S": kb.KB_PROP_S}[which]
        kb.kb_set_propagator_table(self.ctx, w, tabR, tabK, A_tab)

    def set_vertex(self, slot, U=0.0, has_R=False, channels=None, dtype=torch.complex128, include=(0, 1, 2),
                   symmetric=False):
        """channels: {channel: (K1, K2, K2p, K3)} arrays (numpy or torch; None = absent);
        include: channels that are part of the vertex (others: crossing partners only);
        symmetric: the caller vouches for conjugation + crossing symmetry."""
        kb.kb_set_vertex(self.ctx, slot, has_R, U)
        kb.kb_set_vertex_channels(self.ctx, slot, sum(1 << c for c in include))
        kb.kb_set_vertex_symmetric(self.ctx, slot, symmetric)
        self.tensors[slot] = {}
        for ch, classes in (channels or {}).items():
            for k, arr in enumerate(classes):
                if arr is None:
                    continue
                t = torch.as_tensor(arr).to(device=self.device, dtype=dtype).contiguous()
                self.attach(slot, ch, k, t)

    def attach(self, slot, ch, k, t):
        assert t.is_cuda and t.is_contiguous() and t.dtype in DT
        self.tensors.setdefault(slot, {})[(ch, k)] = t
        kb.kb_set_vertex_class(self.ctx, slot, ch, k, t.data_ptr(), DT[t.dtype])

    def alloc_out(self, slot, channels=(0, 1, 2), dtype=torch.complex128, classes=(0, 1, 2, 3)):
        kb.kb_set_vertex(self.ctx, slot, False, 0.0)
        self.tensors[slot] = {}
        sh = self.class_shapes()
        for ch in channels:
            for k in classes:
                self.attach(slot, ch, k, torch.zeros(sh[CLASS_NAMES[k]], dtype=dtype, device=self.device))

    def out(self, slot, ch):
        return {CLASS_NAMES[k]: t for (c, k), t in self.tensors[slot].items() if c == ch}

    def bubble(self, channel, left, right, out, pi_kind=kb.KB_PI_GG, class_mask=kb.KB_MASK_ALL, alpha=1.0,
               beta=0.0, precision="fp64", stream=None):
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        kb.kb_bubble(self.ctx, channel, left, right, out, pi_kind, class_mask, alpha, beta, PREC[precision], st)

    def bubble_vjp(self, channel, left, right, gout, pi_kind=kb.KB_PI_GG, class_mask=kb.KB_MASK_ALL, alpha=1.0,
                   grad_left=-1, grad_right=-1, grad_gr=None, precision="fp64", stream=None):
        """Accumulate the vector-jacobian product of bubble(...) into the gradient slots
        grad_left / grad_right (-1 = not wanted) and, if grad_gr is a dict
        {"K1", "K2", "K3"} -> complex128 device tensors [nw][nq][2], the G^R gradient."""
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        tabs = [None, None, None]
        for i, name in enumerate(("K1", "K2", "K3")):
            t = (grad_gr or {}).get(name)
            if t is not None:
                assert t.is_cuda and t.is_contiguous() and t.dtype == torch.complex128
                tabs[i] = t.data_ptr()
        kb.kb_bubble_vjp(self.ctx, channel, left, right, gout, pi_kind, class_mask, alpha, grad_left, grad_right,
                         *tabs, PREC[precision], st)

    def gr_tables(self):
        """Zeroed G^R gradient tables [nw][nq][2] for the K1, K2 and K3 bosonic grids."""
        g = self.grids
        return {name: torch.zeros((nw, self.nq, 2), dtype=torch.complex128, device=self.device)
                for name, nw in (("K1", g["n1"]), ("K2", g["n2w"]), ("K3", g["n3w"]))}

    def desc(self, channel, left, right, out, pi_kind=kb.KB_PI_GG, class_mask=kb.KB_MASK_ALL, alpha=1.0, beta=0.0,
             precision="fp64"):
        """Descriptor of one bubble of this engine for a StepGraph."""
        return kb.kb_bubble_desc(self.ctx, channel, left, right, out, pi_kind, class_mask, alpha, beta,
                                 PREC[precision])

    def bubble_t_su2(self, slot, out, pi_kind=kb.KB_PI_GG, class_mask=kb.KB_MASK_ALL, alpha=1.0, stream=None):
        """The t bubble of a symmetric slot with itself in its SU(2) form (kb_bubble_t_su2);
        its K3 class is complete after t_su2_finish with the a bubble's K3."""
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        kb.kb_bubble_t_su2(self.ctx, slot, out, pi_kind, class_mask, alpha, st)

    def t_su2_finish(self, out, a_k3, alpha=1.0, stream=None):
        """kb_t_su2_finish: a_k3 the K3 class (device tensor) of B_a of the same vertex."""
        assert a_k3.is_cuda and a_k3.is_contiguous() and a_k3.dtype in DT
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        kb.kb_t_su2_finish(self.ctx, out, a_k3.data_ptr(), DT[a_k3.dtype], alpha, st)

    def desc_t_su2(self, slot, out, pi_kind=kb.KB_PI_GG, class_mask=kb.KB_MASK_ALL, alpha=1.0):
        """Step-graph entry of bubble_t_su2."""
        return kb.kb_t_su2_desc(self.ctx, slot, out, pi_kind, class_mask, alpha)

    def desc_t_su2_finish(self, out, a_engine, a_slot, alpha=1.0):
        """Step-graph entry of t_su2_finish with the K3 class of channel a of slot a_slot of
        the engine a_engine (which has earlier entries in the same graph)."""
        return kb.kb_t_su2_finish_desc(self.ctx, out, a_engine.ctx, a_slot, alpha)

    def share_slot(self, slot, other, other_slot, U=0.0, has_R=False, include=(0, 1, 2), symmetric=False):
        """Attach the device tensors of another engine's slot to a slot of this engine
        (no copy), e.g. one vertex read by several contexts."""
        kb.kb_set_vertex(self.ctx, slot, has_R, U)
        kb.kb_set_vertex_channels(self.ctx, slot, sum(1 << c for c in include))
        kb.kb_set_vertex_symmetric(self.ctx, slot, symmetric)
        self.tensors[slot] = {}
        for (ch, k), t in other.tensors[other_slot].items():
            self.attach(slot, ch, k, t)

    def vertex_eval(self, slot, channel, freqs, spin_uu=False, stream=None):
        """The full vertex of a slot at points (w, v, v') in the variables of `channel`
        (array-like [n][3]); returns a complex128 device tensor [n][16].  For the t-channel
        slice at zero transfer frequency pass channel 2 and points (0, v, v')."""
        f = torch.as_tensor(freqs, dtype=torch.float64).reshape(-1, 3).to(self.device).contiguous()
        out = torch.empty((f.shape[0], 16), dtype=torch.complex128, device=self.device)
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        kb.kb_vertex_eval(self.ctx, slot, channel, spin_uu, f.shape[0], f.data_ptr(), out.data_ptr(), st)
        return out

    def loop(self, slot, nus, single_scale=False, stream=None, line=None, ud_only=False):
        """Self-energy loop of a slot's vertex (kb_loop) with the model's G, or with the flow
        scheme's single-scale propagator S when single_scale (line: 0 G, 1 S, 2 G dΣ G with the
        self-energy-derivative tables, overriding single_scale; ud_only: the up-down vertex
        alone), at frequencies nus;
        returns a complex128 device tensor [n][2][2] indexed [a1'][a1] (0 classical,
        1 quantum): [:, 1, 0] = Sigma^R, [:, 0, 1] = Sigma^A, [:, 1, 1] = Sigma^K."""
        v = torch.as_tensor(nus, dtype=torch.float64).reshape(-1).to(self.device).contiguous()
        out = torch.empty((v.shape[0], 2, 2), dtype=torch.complex128, device=self.device)
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        which = int(bool(single_scale)) if line is None else int(line)
        if ud_only:
            which |= kb.KB_LOOP_UD_ONLY
        kb.kb_loop(self.ctx, slot, which, v.shape[0], v.data_ptr(), out.data_ptr(), st)
        return out

    def susceptibility(self, channel, slot, U, stream=None):
        """χ^R(ω), χ^K(ω) on the K1 grid from the K1 class of a slot (kb_susceptibility_k1):
        a transverse spin, p pairing, t charge; complex128 device tensor [n1][2]."""
        out = torch.empty((self.grids["n1"], 2), dtype=torch.complex128, device=self.device)
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        kb.kb_susceptibility_k1(self.ctx, channel, slot, U, out.data_ptr(), st)
        return out

    def susceptibility_legs(self, channel, slot, precision="fp64", scratch=(13, 14, 15), stream=None):
        """χ^R(ω), χ^K(ω) from the full vertex of a slot by contracting pairs of external legs
        (Sec. II.E.5, channels a and p): the K1 of the chain R̂ Π R̂ + R̂ Π Γ Π R̂ closed by a unit
        bare vertex R̂, from three bubbles — X = B_r(Γ, R̂) (only K1, K2 survive), then
        B_r(R̂, R̂) + B_r(R̂, X) in K1 — read out like the vertex's own K1 at U = 1.  Uses the
        three scratch slots for R̂, X and the chain."""
        if channel not in (0, 1):
            raise ValueError("the leg contraction is built for the a and p channels")
        s_r, s_x, s_y = scratch
        dt = torch.complex64 if precision == "mixed" else torch.complex128
        kb.kb_set_vertex(self.ctx, s_r, True, 1.0)
        kb.kb_set_vertex_symmetric(self.ctx, s_r, False)
        self.tensors[s_r] = {}
        self.alloc_out(s_x, channels=(channel,), dtype=dt, classes=(0, 1))
        kb.kb_set_vertex_channels(self.ctx, s_x, 1 << channel)
        self.alloc_out(s_y, channels=(channel,), dtype=dt, classes=(0,))
        k1, k2 = 1 << kb.KB_K1, 1 << kb.KB_K2
        self.bubble(channel, slot, s_r, s_x, class_mask=k1 | k2, precision=precision, stream=stream)
        self.bubble(channel, s_r, s_r, s_y, class_mask=k1, precision=precision, stream=stream)
        self.bubble(channel, s_r, s_x, s_y, class_mask=k1, beta=1.0, precision=precision, stream=stream)
        return self.susceptibility(channel, s_y, 1.0, stream=stream)

    def keldysh_check(self, slot, channel, T, stream=None):
        """Residuals of the physical Keldysh structure of a slot's channel (kb_keldysh_check):
        {"K1", "K2", "K2p", "K3": parity-structure residual, "causality", "conjugation",
        "fdr": the K1 equilibrium relations at temperature T}, each relative to the class max."""
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        r = kb.kb_keldysh_check(self.ctx, slot, channel, T, st)
        return dict(zip(("K1", "K2", "K2p", "K3", "causality", "conjugation", "fdr"), r[:7]))

    def pack_physical(self, slot, channel, k, stream=None):
        """The distinct Keldysh components of class k (kb_vertex_pack): a device tensor
        [records][4 | 8 | 8 | 16] of the class's dtype."""
        t = self.tensors[slot][(channel, k)]
        nd = (4, 8, 8, 16)[k]
        out = torch.empty((t.numel() // 16, nd), dtype=t.dtype, device=self.device)
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        kb.kb_vertex_pack(self.ctx, slot, channel, k, out.data_ptr(), st)
        return out

    def unpack_physical(self, slot, channel, k, packed, stream=None):
        """Overwrite class k of a slot from its distinct components (kb_vertex_unpack)."""
        t = self.tensors[slot][(channel, k)]
        assert packed.is_cuda and packed.is_contiguous() and packed.dtype == t.dtype
        assert packed.numel() == t.numel() // 16 * (4, 8, 8, 16)[k]
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        kb.kb_vertex_unpack(self.ctx, slot, channel, k, packed.data_ptr(), st)

    def set_autotune(self, on=True):
        """Time the tensor-core contraction's split-K candidates per shape (kb_set_autotune)."""
        kb.kb_set_autotune(self.ctx, on)

    def set_workspace_limit(self, nbytes):
        kb.kb_set_workspace_limit(self.ctx, nbytes)

    def launches(self):
        return kb.kb_launch_count(self.ctx)


class StepGraph:
    """Bubbles of one or several engines captured into one CUDA graph (kb_graph_create);
    launch() replays them as one step.  Bubbles of different engines may overlap."""

    def __init__(self, descs, device=None):
        self.descs = list(descs)
        self.device = device
        self.g = kb.kb_graph_create(self.descs)

    def launch(self, stream=None):
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        kb.kb_graph_launch(self.g, st)

    def kernels(self):
        return kb.kb_graph_kernel_count(self.g)

    def close(self):
        if self.g is not None:
            kb.kb_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
