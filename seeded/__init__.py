"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random numbers and arranges them into the vertex layout;
it computes nothing of the bubble itself.  Both the CPU oracle and the CUDA path
receive the arrays it returns as inputs.

Layout of one channel's reducible vertex (the up-down spin component), complex:

    K1  [n1][16]            K1(w)
    K2  [n2w][n2v][16]      K2(w, v)
    K2p [n2w][n2v][16]      K2'(w, v')
    K3  [n3w][n3v][n3v][16] K3(w, v, v')

The 16 Keldysh components are ordered lexicographically over (a1', a2', a1, a2),
each a in {1 (classical), 2 (quantum)}; component index c = 8b1' + 4b2' + 2b1 + b2
with b = a - 1.

Recipe (the seeded SIAM-shaped vertex of the paper's workloads, Sec. II.C, III.A):
  1. draw complex Gaussians (Re, Im ~ N(0, 1/2)) from a counter-based generator
     (SplitMix64 of (seed, channel, class, counter) -> two uniforms -> Box-Muller);
  2. scale by 0.1 U / ((1 + w^2)(1 + v^2)(1 + v'^2)) at the grid frequencies
     (arguments a class does not have are dropped);
  3. average over the four-element group generated by complex conjugation C and
     crossing X of the vertex, so that both relations hold exactly;
  4. set every 1111 (all-classical) component to zero (causality).
The grid frequencies for the envelope are w_i = A tan(pi x_i / 2) with
x_i = -1 + 2 (i + 1) / (N + 1); this is the input recipe's envelope only.
"""

import numpy as np

MASK64 = (1 << 64) - 1

CH_A, CH_P, CH_T = 0, 1, 2
CLASS_NAMES = ("K1", "K2", "K2p", "K3")


def _splitmix64(z):
    """SplitMix64 finaliser applied to a uint64 numpy array (Steele, Lea, Flood 2014)."""
    z = (z + np.uint64(0x9E3779B97F4A7C15))
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def complex_normals(seed, stream, n):
    """n complex normals with E|z|^2 = 1, from counters (seed, stream, 0..n-1)."""
    with np.errstate(over="ignore"):
        base = np.uint64((seed * 0x100000001B3 + stream * 0x9E3779B1) & MASK64)
        ctr = np.arange(2 * n, dtype=np.uint64)
        bits = _splitmix64(base ^ _splitmix64(ctr + np.uint64(stream << 40 & MASK64)))
    u = ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-np.log(u1))          # Box-Muller with variance 1/2 per part
    return rad * np.cos(2 * np.pi * u2) + 1j * rad * np.sin(2 * np.pi * u2)


def grid_freqs(n, A=5.0):
    x = -1.0 + 2.0 * (np.arange(n) + 1) / (n + 1)
    return A * np.tan(np.pi * x / 2)


# --- Keldysh index permutations used by the symmetrisation -------------------
def _bits(c):
    return (c >> 3) & 1, (c >> 2) & 1, (c >> 1) & 1, c & 1


def _comp(b1p, b2p, b1, b2):
    return 8 * b1p + 4 * b2p + 2 * b1 + b2


# conjugation: (a1' a2' | a1 a2) -> (a1 a2 | a1' a2'), sign (-1)^(1 + sum of a)
PERM_C = np.array([_comp(b1, b2, b1p, b2p) for (b1p, b2p, b1, b2) in map(_bits, range(16))])
SIGN_C = np.array([(-1.0) ** (1 + sum(_bits(c))) for c in range(16)])
# crossing: (a1' a2' | a1 a2) -> (a2' a1' | a2 a1), no sign for the up-down component
PERM_X = np.array([_comp(b2p, b1p, b2, b1) for (b1p, b2p, b1, b2) in map(_bits, range(16))])


def conj_image(ch, V):
    """Image of one channel's classes under complex conjugation (one reading of the
    conjugation symmetry; a,p: (w,v,v') -> (w,v',v); t: (w,v,v') -> (-w,v,v'))."""
    K1, K2, K2p, K3 = V
    f = lambda X: SIGN_C * np.conj(X[..., PERM_C])
    if ch in (CH_A, CH_P):
        return (f(K1), f(K2p), f(K2), f(np.swapaxes(K3, 1, 2)))
    return (f(K1[::-1]), f(K2[::-1]), f(K2p[::-1]), f(K3[::-1]))


def cross_image(ch, V):
    """Image under crossing of both leg pairs (a,t: (w,v,v') -> (-w,v',v);
    p: (w,v,v') -> (w,-v,-v'))."""
    K1, K2, K2p, K3 = V
    f = lambda X: X[..., PERM_X]
    if ch in (CH_A, CH_T):
        return (f(K1[::-1]), f(K2p[::-1]), f(K2[::-1]), f(np.swapaxes(K3[::-1], 1, 2)))
    return (f(K1), f(K2[:, ::-1]), f(K2p[:, ::-1]), f(K3[:, ::-1, ::-1]))


def symmetrise(ch, V):
    C = conj_image(ch, V)
    X = cross_image(ch, V)
    CX = conj_image(ch, X)
    out = tuple((a + b + c + d) / 4 for a, b, c, d in zip(V, C, X, CX))
    for arr in out:
        arr[..., 0] = 0.0          # 1111 component (causality of the input vertex)
    return out


def seeded_channel(ch, grids, U, seed, A=5.0, symmetric=True):
    """Return (K1, K2, K2p, K3) complex128 arrays for channel ch.

    grids = dict(n1, n2w, n2v, n3w, n3v)."""
    n1, n2w, n2v, n3w, n3v = (grids[k] for k in ("n1", "n2w", "n2v", "n3w", "n3v"))
    w1, w2, v2, w3, v3 = (grid_freqs(n, A) for n in (n1, n2w, n2v, n3w, n3v))
    def env(*fs):
        e = np.ones([len(f) for f in fs])
        for ax, f in enumerate(fs):
            shp = [1] * len(fs)
            shp[ax] = len(f)
            e = e * (1.0 / (1.0 + f * f)).reshape(shp)
        return e

    shapes = [((n1, 16), env(w1)), ((n2w, n2v, 16), env(w2, v2)),
              ((n2w, n2v, 16), env(w2, v2)), ((n3w, n3v, n3v, 16), env(w3, v3, v3))]
    out = []
    for k, (shape, e) in enumerate(shapes):
        z = complex_normals(seed, 16 * ch + k + 1, int(np.prod(shape))).reshape(shape)
        out.append(0.1 * U * z * e[..., None])
    out = tuple(out)
    return symmetrise(ch, out) if symmetric else out


def seeded_vertex(grids, U, seed, A=5.0, channels=(0, 1, 2), symmetric=True):
    """dict channel -> (K1, K2, K2p, K3) for the requested channels."""
    return {ch: seeded_channel(ch, grids, U, seed, A, symmetric) for ch in channels}


def seeded_sigma(n, seed, scale=0.1, A=5.0):
    """A causal, FDR-free synthetic dynamic self-energy table on a tan-map grid:
    Sigma^R = scale * (z - i|z'|) / (1 + v^2) with Im Sigma^R <= 0, and Sigma^K = 0
    replaced by the equilibrium form by the caller if wanted."""
    v = grid_freqs(n, A)
    z = complex_normals(seed, 999, n)
    sigR = scale * (z.real - 1j * np.abs(z.imag)) / (1.0 + v * v)
    return sigR
