"""Host logic of the multiloop step (no device): the graph entries, replayed on symbolic slot
contents, build exactly the loop-order recursion of the multiloop flow (Sec. III.C) —

    γ̇_r^(1) = B_r(Γ, Γ; Π-dot),
    γ̇_r^(l) = B_r(γ̇_r̄^(l-1), Γ) + [l >= 3] B_r(Γ, B_r(γ̇_r̄^(l-2), Γ)) + B_r(Γ, γ̇_r̄^(l-1)),

with γ̇_r̄ the channels other than r (the slot's channel mask), Γ̇ = Σ_l γ̇^(l); every slot is
written before it is read within a branch, and no branch reads another channel's result of
the same order before the join.  With keep_central the central parts C_r^(l) (l >= 3)
are also collected, alone, in their own slot (the multiloop self-energy flow's γ̇^C)."""

import collections

import pytest

from paper_2405_20996_gb300 import kb
from paper_2405_20996_gb300.multiloop import S_GAMMA, S_TOTAL, s_central, step_entries


def _expected(channels, n_loops):
    """The recursion as strings: a term is 'B_r(left|right;pi)', a vertex a sorted tuple."""
    order = {}
    for r in channels:
        order[(1, r)] = ("B%d(G|G;dot)" % r,)
    left = {}
    for l in range(2, n_loops + 1):
        for r in channels:
            bar = "o%d!%d" % (l - 1, r)              # γ̇^(l-1) without channel r
            terms = ["B%d(%s|G;GG)" % (r, bar), "B%d(G|%s;GG)" % (r, bar)]
            if l >= 3:
                terms.append("B%d(G|%s;GG)" % (r, left[(l - 1, r)]))
            left[(l, r)] = "B%d(%s|G;GG)" % (r, bar)
            order[(l, r)] = tuple(sorted(terms))
    return order


def _replay(channels, n_loops, image_r2=False, keep_central=False):
    """Apply the entries to slots holding sums of symbolic terms; the vertex a bubble reads
    from an order slot is named by its order and the channel left out (the mask)."""
    slots = collections.defaultdict(list)      # (slot, channel) -> list of terms
    name_of_order = {1 + l: l for l in range(1, n_loops + 1)}
    joined_upto = 1                            # orders complete in all channels
    written = set()
    for x in step_entries(channels, n_loops, image_r2=image_r2, keep_central=keep_central):
        if x[0] == "join":
            joined_upto += 1
            continue
        if x[0] == "add":
            _, r, src, dst = x
            assert (src, r) in written
            slots[(dst, r)] = slots[(dst, r)] + slots[(src, r)]
            written.add((dst, r))
            continue
        if x[0] == "image":
            # the symmetry image of a left part B_r(X|G) is the right part B_r(G|X)
            _, r, src, dst = x
            (term,) = slots[(src, r)]
            head, body = term.split("(", 1)
            lr, pi = body[:-1].rsplit(";", 1)
            depth, cut = 0, None
            for i, ch in enumerate(lr):
                depth += ch == "("
                depth -= ch == ")"
                if ch == "|" and depth == 0:
                    cut = i
            slots[(dst, r)] = ["%s(%s|%s;%s)" % (head, lr[cut + 1:], lr[:cut], pi)]
            written.add((dst, r))
            continue
        if x[0] != "bubble":
            continue
        _, r, lft, rgt, out, pi, beta = x

        def vname(s):
            if s == S_GAMMA:
                return "G"
            if s in name_of_order:             # an order slot read as γ̇_r̄ (mask without r)
                l = name_of_order[s]
                assert l <= joined_upto, ("read before join", s, l, joined_upto)
                return "o%d!%d" % (l, r)
            assert (s, r) in written, ("left-part slot read before written", s)
            (term,) = slots[(s, r)]            # a left part: a single bubble term
            return term

        term = "B%d(%s|%s;%s)" % (r, vname(lft), vname(rgt), "dot" if pi == kb.KB_PI_GS_SG else "GG")
        slots[(out, r)] = ([] if beta == 0.0 else slots[(out, r)]) + [term]
        written.add((out, r))
    return slots


@pytest.mark.parametrize("image_r2", [False, True])
@pytest.mark.parametrize("n_loops", [1, 2, 3, 4, 6])
def test_entries_build_the_loop_order_recursion(n_loops, image_r2):
    ch = (0, 1, 2)
    slots = _replay(ch, n_loops, image_r2)
    exp = _expected(ch, n_loops)
    for l in range(1, n_loops + 1):
        for r in ch:
            assert tuple(sorted(slots[(1 + l, r)])) == exp[(l, r)], (l, r)
    for r in ch:
        total = sorted(t for l in range(1, n_loops + 1) for t in exp[(l, r)])
        assert sorted(slots[(S_TOTAL, r)]) == total
    bubbles = sum(1 for x in step_entries(ch, n_loops, image_r2=image_r2) if x[0] == "bubble")
    saved = 3 if (image_r2 and n_loops >= 3) else 0
    assert bubbles == 3 * (1 + (2 if n_loops >= 2 else 0) + 3 * max(0, n_loops - 2)) - saved


def test_slot_budget_and_cache_entries():
    ent = step_entries((0, 1, 2), 6, cached={0: 13, 2: 4})
    slots = {s for x in ent if x[0] == "bubble" for s in x[2:5]} | {x[3] for x in ent if x[0] == "add"}
    assert max(slots) < kb.KB_MAX_SLOTS
    caches = [x for x in ent if x[0] == "cache"]
    assert [(c[1], c[3]) for c in caches] == [(0, 13), (2, 4)]
    # a cache entry precedes every bubble of its channel
    for r in (0, 2):
        first_bubble = next(i for i, x in enumerate(ent) if x[0] == "bubble" and x[1] == r)
        assert next(i for i, x in enumerate(ent) if x[0] == "cache" and x[1] == r) < first_bubble


@pytest.mark.parametrize("image_r2", [False, True])
@pytest.mark.parametrize("n_loops", [2, 3, 4, 6])
def test_entries_keep_the_central_parts(n_loops, image_r2):
    ch = (0, 1, 2)
    slots = _replay(ch, n_loops, image_r2, keep_central=True)
    exp = _expected(ch, n_loops)
    for l in range(1, n_loops + 1):
        for r in ch:
            assert tuple(sorted(slots[(1 + l, r)])) == exp[(l, r)], (l, r)
    left = {}
    for l in range(2, n_loops + 1):
        for r in ch:
            left[(l, r)] = "B%d(o%d!%d|G;GG)" % (r, l - 1, r)
    sc = s_central(n_loops)
    assert sc < kb.KB_MAX_SLOTS
    for r in ch:
        central = sorted("B%d(G|%s;GG)" % (r, left[(l - 1, r)]) for l in range(3, n_loops + 1))
        assert sorted(slots[(sc, r)]) == central, r
    used = {s for x in step_entries(ch, n_loops, image_r2=image_r2) if x[0] == "bubble" for s in x[2:5]}
    assert sc not in used
