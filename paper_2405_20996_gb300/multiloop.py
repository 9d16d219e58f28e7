"""Right-hand side of the multiloop flow for the vertex (Sec. III.C), as one step graph.

At fixed vertex Γ and self-energy, the l-loop contributions to the derivative of the
reducible vertex of channel r are

    l = 1:   γ̇_r^(1) = B_r(Γ, Γ; Π̇),  Π̇ = G S + S G (the single-scale pair),
    l = 2:   γ̇_r^(2) = L_r^(2) + R_r^(2),
    l >= 3:  γ̇_r^(l) = L_r^(l) + C_r^(l) + R_r^(l),

with L_r^(l) = B_r(γ̇_r̄^(l-1), Γ), R_r^(l) = B_r(Γ, γ̇_r̄^(l-1)), C_r^(l) = B_r(Γ, L_r^(l-1))
(Π = G G; γ̇_r̄ = the sum over the channels other than r), and Γ̇ = Σ_l Σ_r γ̇_r^(l).  Per
channel that is 1 + 2 + 3 (n_loops - 2) bubbles: 15 per channel, 45 per step, at six loops.

Each channel has its own context (workspace), and the three run as parallel branches of
one CUDA graph; a join entry separates the loop orders, because order l of channel r reads
order l - 1 of all channels.  The slot γ̇^(l) serves as the output of order l (each branch
writes its channel) and, with its channel mask excluding r, as the vertex γ̇_r̄^(l-1) of
the next order.  L_r^(l) is computed once into its own slot (it is the right vertex of the
next order's central part, a channel-r-only vertex without bare part) and added to γ̇_r^(l)
by the library's slot addition.  Γ is the same in all 45 bubbles, so its records for the
K2 and K2' contractions of channel r (the other channels at the converted frequencies, per
(w, v, node)) are gathered once per step into a record cache that the later bubbles of that
channel stream from HBM.
"""

import torch

from . import kb
from .engine import CLASS_NAMES, Engine, StepGraph

S_GAMMA = 0
S_TOTAL = 1                    # Γ̇ = Σ_l γ̇^(l)


def _s_order(l):               # γ̇^(l), l = 1 .. n_loops
    return 1 + l


def _s_left(l, n_loops):       # L^(l), l = 2 .. n_loops - 1
    return 1 + n_loops + (l - 1)


def s_central(n_loops):        # Σ_{l >= 3} C^(l), all channels (keep_central)
    return max(2 * n_loops, n_loops + 2)


def step_entries(channels, n_loops, cached=None, image_r2=False, keep_central=False):
    """The entries of one step, as plain tuples (host logic, no device):
    ("cache", r, slot, sides), ("bubble", r, left, right, out, pi_kind, beta),
    ("image", r, src, dst), ("add", r, src, dst), ("join",).  Per channel r: order 1 into
    γ̇^(1); order l the left part (into its own slot, or straight into γ̇^(l) at the last
    order), the central part from the previous order's left part (l >= 3), the right part,
    and the left part added; finally every order added into Γ̇.  image_r2: Γ is conjugation-
    and crossing-symmetric, so γ̇^(1) (from the symmetric one-loop bubble) is too, and the
    second order's right part is the symmetry image of its left part (kb_vertex_image).
    keep_central: every central part C_r^(l) is also added into the slot s_central(n_loops)
    (the multiloop self-energy flow's γ̇^C; zero it before the step); at the last order the
    central part is then computed before the left part, so that it is alone in γ̇^(l) when
    copied."""
    L, G, ent = n_loops, S_GAMMA, []
    SC = s_central(L)
    cached = cached or {}
    for r in channels:
        if r in cached:
            ent.append(("cache", r, G, cached[r]))       # Γ's records
        ent.append(("bubble", r, G, G, _s_order(1), kb.KB_PI_GS_SG, 0.0))
    for l in range(2, L + 1):
        ent.append(("join",))
        prev, out = _s_order(l - 1), _s_order(l)
        last = l == L
        for r in channels:
            lslot = out if last else _s_left(l, L)
            if keep_central and last and l >= 3:
                ent.append(("bubble", r, G, _s_left(l - 1, L), out, kb.KB_PI_GG, 0.0))               # C
                ent.append(("add", r, out, SC))
                ent.append(("bubble", r, prev, G, out, kb.KB_PI_GG, 1.0))                            # L
            else:
                ent.append(("bubble", r, prev, G, lslot, kb.KB_PI_GG, 0.0))                               # L
                if l >= 3:
                    ent.append(("bubble", r, G, _s_left(l - 1, L), out, kb.KB_PI_GG, 1.0 if last else 0.0))   # C
                    if keep_central:
                        ent.append(("add", r, out, SC))
            if image_r2 and l == 2 and not last:
                ent.append(("image", r, lslot, out))                                                 # R = I_r[L]
            else:
                ent.append(("bubble", r, G, prev, out, kb.KB_PI_GG, 1.0 if (last or l >= 3) else 0.0))    # R
            if not last:
                ent.append(("add", r, lslot, out))
    for r in channels:
        for l in range(1, L + 1):
            ent.append(("add", r, _s_order(l), S_TOTAL))
    return ent


class MultiloopStep:
    def __init__(self, grids, nq, U, Delta, T, vertex, n_loops=6, precision="mixed", A=5.0, device=0,
                 symmetric=True, channels=(0, 1, 2), cache="auto", reserve_bytes=40 << 30, keep_central=False):
        """vertex: {channel: (K1, K2, K2p, K3)} arrays of the reducible vertices γ_r (the bare
        part −U/2 is added by the library).  precision "mixed" keeps every vertex in complex64,
        "fp64" in complex128.  cache (mixed only): rebuild the record cache of Γ once per
        step — "auto": its K3 tiles and its K2 records as left vertex (the right parts' K2 and
        the left parts' K2' are zero classes, not computed), as far as they fit in the free
        device memory less reserve_bytes; True: every side; False: none."""
        assert n_loops >= 1
        assert _s_left(n_loops - 1, n_loops) < kb.KB_MAX_SLOTS
        assert not keep_central or s_central(n_loops) < kb.KB_MAX_SLOTS
        self.keep_central = bool(keep_central)
        self.n_loops, self.precision = n_loops, precision
        self.channels = tuple(channels)
        dt = torch.complex64 if precision == "mixed" else torch.complex128
        self.dtype = dt
        self.e = {}
        for r in self.channels:
            e = Engine(grids, nq, A=A, device=device)
            e.set_model(Delta, T)
            self.e[r] = e
        e0 = self.e[self.channels[0]]
        e0.set_vertex(S_GAMMA, U=U, has_R=True, channels=vertex, dtype=dt, symmetric=symmetric)
        for r in self.channels[1:]:
            self.e[r].share_slot(S_GAMMA, e0, S_GAMMA, U=U, has_R=True, symmetric=symmetric)
        sh = e0.class_shapes()
        dev = e0.device
        z = lambda: {(c, k): torch.zeros(sh[CLASS_NAMES[k]], dtype=dt, device=dev) for c in range(3) for k in range(4)}
        self.total = z()
        self.orders = [z() for _ in range(n_loops)]
        self.lefts = {l: {r: {k: torch.zeros(sh[CLASS_NAMES[k]], dtype=dt, device=dev) for k in range(4)}
                          for r in self.channels} for l in range(2, n_loops)}
        # Σ_{l >= 3} C^(l) of all channels: read by the self-energy loop as γ̇^C_t̄ (channels a and
        # p; the t data enters only as the up-up crossing partner)
        self.central = z() if self.keep_central else None
        for r, e in self.e.items():
            others = 7 & ~(1 << r)
            self._attach(e, S_TOTAL, self.total, 7)
            if self.keep_central:
                self._attach(e, s_central(n_loops), self.central, (1 << 0) | (1 << 1))
            for l in range(1, n_loops + 1):
                self._attach(e, _s_order(l), self.orders[l - 1], others)
            for l in range(2, n_loops):
                kb.kb_set_vertex(e.ctx, _s_left(l, n_loops), False, 0.0)
                kb.kb_set_vertex_channels(e.ctx, _s_left(l, n_loops), 1 << r)
                kb.kb_set_vertex_symmetric(e.ctx, _s_left(l, n_loops), False)
                e.tensors[_s_left(l, n_loops)] = {}
                for k in range(4):
                    e.attach(_s_left(l, n_loops), r, k, self.lefts[l][r][k])
        # record cache of Γ (mixed only): channel -> sides (bit 0: K2 records as left vertex,
        # 1: K2' records as right vertex, 2: K3 left tile, 3: K3 right tile with Π = G G)
        self.image_r2 = bool(symmetric)
        self.cached = {}
        if cache and precision == "mixed":
            ns = lambda r: 2 if r == 2 else 1
            nbytes = {0: lambda r: grids["n2w"] * grids["n2v"] * ((nq - 2 + 31) // 32 * 32) * ns(r) * 128,
                      2: lambda r: grids["n3w"] * 4 * 4 * grids["n3v"] * 4 * ns(r) * nq * 4}
            nbytes[1], nbytes[3] = nbytes[0], nbytes[2]
            if cache == "auto":
                # the sides that serve nonzero classes, in order of time saved per byte: the K3
                # tiles (left: 9 bubbles per channel, right: 5), then the K2 records of the
                # first order and the central parts
                order = [(r, sd) for sd in (2, 3, 0) for r in self.channels]
                budget = torch.cuda.mem_get_info(dev)[0] - reserve_bytes
            else:
                order = [(r, sd) for sd in (0, 1, 2, 3) for r in self.channels]
                budget = float("inf")
            used = 0
            for r, sd in order:
                if used + nbytes[sd](r) <= budget:
                    self.cached[r] = self.cached.get(r, 0) | (1 << sd)
                    used += nbytes[sd](r)
        self.descs = self._descs()
        self.graph = None

    @staticmethod
    def _attach(e, slot, tensors, mask):
        kb.kb_set_vertex(e.ctx, slot, False, 0.0)
        kb.kb_set_vertex_channels(e.ctx, slot, mask)
        kb.kb_set_vertex_symmetric(e.ctx, slot, False)
        e.tensors[slot] = {}
        for (c, k), t in tensors.items():
            e.attach(slot, c, k, t)

    def _descs(self):
        """The step as a list of graph entries (bubbles, slot additions, joins)."""
        d = []
        for x in step_entries(self.channels, self.n_loops, self.cached, image_r2=self.image_r2,
                              keep_central=self.keep_central):
            if x[0] == "join":
                d.append(kb.kb_join_desc())
                continue
            kind, r = x[0], x[1]
            e = self.e[r]
            if kind == "cache":
                d.append(kb.kb_cache_desc(e.ctx, r, x[2], x[3]))
            elif kind == "add":
                d.append(kb.kb_add_desc(e.ctx, r, x[2], x[3]))
            elif kind == "image":
                d.append(kb.kb_image_desc(e.ctx, r, x[2], x[3]))
            else:
                _, _, left, right, out, pi, beta = x
                d.append(e.desc(r, left, right, out, pi_kind=pi, beta=beta, precision=self.precision))
        return d

    def bubbles_per_step(self):
        return sum(1 for x in self.descs if x.op == kb.KB_OP_BUBBLE)

    def parts_per_step(self):
        """Bubble parts delivered per step: the bubbles and the right parts made as images."""
        return sum(1 for x in self.descs if x.op in (kb.KB_OP_BUBBLE, kb.KB_OP_IMAGE))

    def zero(self):
        for t in self.total.values():
            t.zero_()
        if self.central is not None:
            for t in self.central.values():
                t.zero_()

    def build(self):
        self.graph = StepGraph(self.descs)
        return self.graph

    def run(self, stream=None):
        """One step: Γ̇ accumulates into `total` (zero it first for a fresh derivative)."""
        if self.graph is None:
            self.build()
        self.graph.launch(stream)

    def run_eager(self, stream=None):
        """The same entries launched one by one on one stream (reference for the graph)."""
        st = (stream or torch.cuda.current_stream(self.e[self.channels[0]].device)).cuda_stream
        for x in self.descs:
            if x.op == kb.KB_OP_JOIN:
                continue
            if x.op == kb.KB_OP_CACHE:
                kb.kb_vertex_cache(x.ctx, x.slot_left, x.channel, x.class_mask, st)
            elif x.op == kb.KB_OP_IMAGE:
                kb.kb_vertex_image(x.ctx, x.channel, x.slot_left, x.out_slot, x.class_mask, st)
            elif x.op == kb.KB_OP_ADD:
                kb.kb_vertex_add(x.ctx, x.channel, x.slot_left, x.out_slot, x.class_mask, x.alpha, st)
            else:
                kb.kb_bubble(x.ctx, x.channel, x.slot_left, x.slot_right, x.out_slot, x.pi_kind, x.class_mask,
                             x.alpha, x.beta, x.precision, st)

    def order(self, l, ch):
        return {CLASS_NAMES[k]: self.orders[l - 1][(ch, k)] for k in range(4)}

    def derivative(self, ch):
        return {CLASS_NAMES[k]: self.total[(ch, k)] for k in range(4)}

    def close(self):
        if self.graph is not None:
            self.graph.close()
            self.graph = None
        for e in self.e.values():
            e.close()
