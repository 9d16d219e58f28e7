"""Susceptibilities from the K1 class (the paper's post-processing, Sec. II.E.5: for a
converged parquet solution they follow directly from K1).

K1 of channel r is the ω-only part of the vertex: the bare vertex, the r-channel
susceptibility and the bare vertex, K1_r = R χ_r R with R = −U/2 on the Keldysh components
with an odd number of quantum indices.  In the 4×4 form of a channel (a: rows (a1', a2),
columns (a2', a1); p: rows (a1', a2'), columns (a1, a2)) the components of one parity block
(row pair parity, column pair parity) carry one number: (odd, even) the retarded, (even,
odd) the advanced, (odd, odd) the Keldysh part; (even, even) vanishes.  Normalised so that
at second order in U (K1_r = (U/2)² Π_r, Π the bubble of the dv/(2πi) measure) they are the
static-limit-positive bare susceptibilities:

    transverse spin (a channel, up-down):  χ_±(ω)    = −2 K1_a(ω) / U²   (χ0 = −Π_ph/2),
    pairing (p channel, up-down):          χ_pair(ω) = +2 K1_p(ω) / U²   (χ0 = +Π_pp/2),

so that their third order is the ladder χ = χ0 + U χ0² (spin, enhanced by a repulsive U) and
χ = χ0 − U χ0² (pairing, suppressed).

Charge (t channel): the density response sums both spins of the t-channel pair,
χ_c(ω) = 2 [K1_t^↑↓(ω) + K1_t^↑↑(ω)] / U², with the up-up part from crossing,
K1_t^↑↑(ω) = K1_t^↑↓(ω) − K1_a^↑↓(−ω) (Keldysh indices a1 <-> a2), in the t channel's 4×4 form
(rows (a1', a1), columns (a2', a2)) whose (even, odd) block is the retarded one; at second
order χ_c = χ0 = −Π_ph/2, at third order the ladder χ0 − U χ0² (suppressed).  (The
longitudinal spin combination K1_t^↑↑ − K1_t^↑↓ is the a channel's by that same crossing.)
"""

import numpy as np

# a representative component (index 8 a1' + 4 a2' + 2 a1 + a2, 0 classical, 1 quantum) of the
# retarded and Keldysh blocks of each channel's 4x4 form
_COMP = {0: {"R": 1, "K": 3}, 1: {"R": 8, "K": 9}}
_SCALE = {0: -2.0, 1: 2.0}


def susceptibility_from_K1(K1, channel, U):
    """χ^R(ω), χ^K(ω) of channel a (0, transverse spin) or p (1, pairing) from its K1 array
    [n1][16] (numpy or torch, any complex dtype) at coupling U."""
    if channel not in _COMP:
        raise ValueError("susceptibilities from K1 are defined for the a and p channels")
    if U == 0:
        raise ValueError("U = 0: K1 vanishes")
    c = _COMP[channel]
    f = _SCALE[channel] / (U * U)
    return f * K1[:, c["R"]], f * K1[:, c["K"]]


_T_COMP = {"R": 1, "K": 3}
_SWAP12 = [(c & 12) | ((c & 1) << 1) | ((c >> 1) & 1) for c in range(16)]


def charge_susceptibility_from_K1(K1_t, K1_a, U):
    """χ_c^R(ω), χ_c^K(ω) from the t and a channels' K1 arrays [n1][16] on the same
    (symmetric) bosonic grid, at coupling U."""
    if U == 0:
        raise ValueError("U = 0: K1 vanishes")
    upup = K1_t - K1_a.flip(0)[:, _SWAP12] if hasattr(K1_a, "flip") else K1_t - K1_a[::-1][:, _SWAP12]
    tot = K1_t + upup
    f = 2.0 / (U * U)
    return f * tot[:, _T_COMP["R"]], f * tot[:, _T_COMP["K"]]
