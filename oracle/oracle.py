"""Python front end of the FP64 CPU oracle (kb_oracle.c).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and the CPU-baseline leg of
bench.py use this module.  It shares no code with the CUDA library.

Everything here follows the paper's definitions directly (see the header of
kb_oracle.c for the formulas and the readings taken where the paper defers to its
companion paper).
"""

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

CH_A, CH_P, CH_T = 0, 1, 2
SEL_ZERO, SEL_NU, SEL_FULL = 0, 1, 2
PI_GG, PI_GS = 0, 1
# (left selection, right selection) of each output class (Sec. II.C.1)
CLASS_SEL = {"K1": (SEL_ZERO, SEL_ZERO), "K2": (SEL_NU, SEL_ZERO),
             "K2p": (SEL_ZERO, SEL_NU), "K3": (SEL_NU, SEL_NU)}

_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc (plain C99, OpenMP)."""
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(HERE, "kb_oracle.c")
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(src):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, src, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            L.og_bubble_points.restype = C.c_int
            L.og_bubble_points_adaptive.restype = C.c_int
            L.og_loop.restype = C.c_int
            L.og_loop_spin.restype = C.c_int
            _lib = L
    return _lib


class _OVtx(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2w", C.c_int), ("n2v", C.c_int), ("n3w", C.c_int), ("n3v", C.c_int),
                ("A", C.c_double), ("U", C.c_double), ("has_R", C.c_int), ("mask", C.c_int),
                ("K1", C.c_void_p * 3), ("K2", C.c_void_p * 3), ("K2p", C.c_void_p * 3), ("K3", C.c_void_p * 3)]


class _OProp(C.Structure):
    _fields_ = [("Delta", C.c_double), ("T", C.c_double), ("eps", C.c_double), ("A_sig", C.c_double),
                ("n_sig", C.c_int), ("sigR", C.c_void_p), ("sigK", C.c_void_p), ("reg", C.c_int),
                ("lam", C.c_double), ("n_dsig", C.c_int), ("A_dsig", C.c_double), ("dsigR", C.c_void_p),
                ("dsigK", C.c_void_p), ("n_gt", C.c_int), ("A_gt", C.c_double), ("gtR", C.c_void_p),
                ("gtK", C.c_void_p), ("n_st", C.c_int), ("A_st", C.c_double), ("stR", C.c_void_p),
                ("stK", C.c_void_p)]


REG_DELTA, REG_U, REG_T, REG_NONE = 0, 1, 2, 3


def grid(n, A=5.0):
    """Frequency grid of Sec. II.G.4 read as N interior points of a uniform x-grid."""
    x = -1.0 + 2.0 * (np.arange(n) + 1) / (n + 1)
    return A * np.tan(np.pi * x / 2)


class Vertex:
    """Bare part (U, on/off) plus per-channel classes (K1, K2, K2p, K3) as complex128.
    include: channels that are part of the vertex (default all three); data of an
    excluded channel is used only as the crossing partner of the up-up component."""

    def __init__(self, grids, U=0.0, has_R=False, channels=None, A=5.0, include=(0, 1, 2)):
        self.grids = dict(grids)
        self.A, self.U, self.has_R = A, float(U), bool(has_R)
        self.ch = {}
        for c, classes in (channels or {}).items():
            self.ch[c] = tuple(None if a is None else np.ascontiguousarray(a, dtype=np.complex128) for a in classes)
        s = _OVtx()
        g = self.grids
        s.n1, s.n2w, s.n2v, s.n3w, s.n3v = g["n1"], g["n2w"], g["n2v"], g["n3w"], g["n3v"]
        s.A, s.U, s.has_R = A, self.U, int(self.has_R)
        s.mask = sum(1 << c for c in include)
        for c in range(3):
            cl = self.ch.get(c, (None,) * 4)
            for k, name in enumerate(("K1", "K2", "K2p", "K3")):
                arr = cl[k]
                getattr(s, name)[c] = None if arr is None else arr.ctypes.data
        self._s = s

    def ptr(self):
        return C.byref(self._s)


class Prop:
    """G^R = 1/(v - eps + i Delta - Sigma^R(v)) with optional Sigma tables on a tan grid, and
    the single-scale propagator of the flow scheme reg (REG_DELTA, REG_U with parameter lam:
    G^R = lam / (v - eps + i Delta - lam Sigma^R), REG_T, or REG_NONE: S = 0), with the
    Katanin substitution S + G dSigma G when dSigma/dLambda tables are given (with REG_NONE
    the change of G along dSigma).  Tabulated lines: gtR, gtK (G) and stR, stK (S) on tan
    grids of scales A_gt, A_st replace the computed G and S (the Keldysh parts default to 0;
    a tabulated G needs a tabulated S wherever S is used)."""

    def __init__(self, Delta=1.0, T=0.1, eps=0.0, sigR=None, sigK=None, A_sig=5.0, reg=REG_DELTA, lam=1.0,
                 dsigR=None, dsigK=None, A_dsig=5.0, gtR=None, gtK=None, A_gt=5.0, stR=None, stK=None,
                 A_st=5.0):
        self.sigR = None if sigR is None else np.ascontiguousarray(sigR, dtype=np.complex128)
        self.sigK = None if sigK is None else np.ascontiguousarray(sigK, dtype=np.complex128)
        self.dsigR = None if dsigR is None else np.ascontiguousarray(dsigR, dtype=np.complex128)
        self.dsigK = None if dsigK is None else np.ascontiguousarray(dsigK, dtype=np.complex128)
        s = _OProp()
        s.Delta, s.T, s.eps, s.A_sig = Delta, T, eps, A_sig
        s.reg, s.lam = int(reg), float(lam)
        s.n_dsig = 0 if self.dsigR is None else len(self.dsigR)
        s.A_dsig = A_dsig
        s.dsigR = None if self.dsigR is None else self.dsigR.ctypes.data
        s.dsigK = None if self.dsigK is None else self.dsigK.ctypes.data
        s.n_sig = 0 if self.sigR is None else len(self.sigR)
        s.sigR = None if self.sigR is None else self.sigR.ctypes.data
        s.sigK = None if self.sigK is None else self.sigK.ctypes.data
        self.tabs = {}
        for name, R, K, A in (("g", gtR, gtK, A_gt), ("s", stR, stK, A_st)):
            n = 0
            if R is not None:
                R = np.ascontiguousarray(R, dtype=np.complex128)
                K = np.zeros_like(R) if K is None else np.ascontiguousarray(K, dtype=np.complex128)
                assert K.shape == R.shape
                self.tabs[name] = (R, K)
                n = len(R)
            setattr(s, "n_%st" % name, n)
            setattr(s, "A_%st" % name, float(A))
            setattr(s, "%stR" % name, None if n == 0 else R.ctypes.data)
            setattr(s, "%stK" % name, None if n == 0 else K.ctypes.data)
        self.has_g_table, self.has_s_table = "g" in self.tabs, "s" in self.tabs
        self._s = s
        self.Delta, self.T, self.eps = Delta, T, eps

    def ptr(self):
        return C.byref(self._s)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def gl5_rule(Nq):
    x = np.zeros(Nq)
    w = np.zeros(Nq)
    if lib().og_gl5_rule(C.c_int(Nq), _dptr(x), _dptr(w)) != 0:
        raise ValueError("Nq must be 4P+1")
    return x, w


def bubble_points(V1, V2, P, r, lsel, rsel, Nq, freqs, pi_kind=PI_GG, nthreads=0):
    """Bubble B_r at arbitrary (w, v, v') rows of freqs; returns (n, 16) complex128."""
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64).reshape(-1, 3))
    out = np.zeros((len(f), 16), dtype=np.complex128)
    rc = lib().og_bubble_points(V1.ptr(), V2.ptr(), P.ptr(), C.c_int(pi_kind), C.c_int(r), C.c_int(lsel),
                                C.c_int(rsel), C.c_int(Nq), C.c_int(len(f)), _dptr(f),
                                out.ctypes.data_as(C.c_void_p), C.c_int(nthreads))
    if rc != 0:
        raise RuntimeError("og_bubble_points failed: %d" % rc)
    return out


def class_freqs(grids, cls, A=5.0, idx=None):
    """(w, v, v') rows of the output grid points of one class; idx selects a subset
    (list of index tuples of the class array without the Keldysh axis)."""
    g = grids
    if cls == "K1":
        w = grid(g["n1"], A)
        pts = [(w[i], 0.0, 0.0) for (i,) in (idx if idx is not None else [(i,) for i in range(g["n1"])])]
    elif cls in ("K2", "K2p"):
        w, v = grid(g["n2w"], A), grid(g["n2v"], A)
        ids = idx if idx is not None else [(i, j) for i in range(g["n2w"]) for j in range(g["n2v"])]
        pts = [(w[i], v[j], 0.0) if cls == "K2" else (w[i], 0.0, v[j]) for (i, j) in ids]
    else:
        w, v = grid(g["n3w"], A), grid(g["n3v"], A)
        ids = idx if idx is not None else [(i, j, k) for i in range(g["n3w"]) for j in range(g["n3v"])
                                           for k in range(g["n3v"])]
        pts = [(w[i], v[j], v[k]) for (i, j, k) in ids]
    return np.array(pts, dtype=np.float64).reshape(-1, 3)


def class_shape(grids, cls):
    g = grids
    return {"K1": (g["n1"],), "K2": (g["n2w"], g["n2v"]), "K2p": (g["n2w"], g["n2v"]),
            "K3": (g["n3w"], g["n3v"], g["n3v"])}[cls] + (16,)


def bubble_class(V1, V2, P, r, cls, Nq, pi_kind=PI_GG, idx=None, nthreads=0):
    """One output class of B_r on its grid (or at the index tuples idx)."""
    ls, rs = CLASS_SEL[cls]
    f = class_freqs(V1.grids, cls, V1.A, idx)
    out = bubble_points(V1, V2, P, r, ls, rs, Nq, f, pi_kind, nthreads)
    if idx is None:
        return out.reshape(class_shape(V1.grids, cls))
    return out


def bubble_all(V1, V2, P, r, Nq, pi_kind=PI_GG, classes=("K1", "K2", "K2p", "K3"), nthreads=0):
    return {c: bubble_class(V1, V2, P, r, c, Nq, pi_kind, nthreads=nthreads) for c in classes}


class _OGrad(C.Structure):
    _fields_ = [("K1", C.c_void_p * 3), ("K2", C.c_void_p * 3), ("K2p", C.c_void_p * 3), ("K3", C.c_void_p * 3)]


CLASSES = ("K1", "K2", "K2p", "K3")


def zero_grads(grids):
    """Gradient arrays of every class of every channel (complex128, zeros)."""
    return {c: [np.zeros(class_shape(grids, k), dtype=np.complex128) for k in CLASSES] for c in range(3)}


def _ograd(gr):
    s = _OGrad()
    for c in range(3):
        for k, name in enumerate(CLASSES):
            getattr(s, name)[c] = gr[c][k].ctypes.data
    return s


def class_omega_index(grids, cls, idx=None):
    """Bosonic index (on the class's own w grid) of each output point of a class."""
    shp = class_shape(grids, cls)[:-1]
    if idx is None:
        return np.repeat(np.arange(shp[0]), int(np.prod(shp[1:])) if len(shp) > 1 else 1).astype(np.int32)
    return np.array([t[0] for t in idx], dtype=np.int32)


def bubble_vjp(V1, V2, P, r, cls, Nq, gbar, pi_kind=PI_GG, want_left=True, want_right=True, want_gr=False,
               idx=None, nthreads=0):
    """Vector-Jacobian product of one output class of B_r (real-embedding convention:
    bar(z) = dL/dRe z + i dL/dIm z for a real loss L).  gbar has the class's shape (or
    (len(idx), 16)).  Returns (grad_left, grad_right, grad_GR): gradient dicts
    channel -> [K1, K2, K2p, K3] with the vertex's shapes (None if not wanted), and the
    gradient with respect to G^R at the samples [w index][node][side] (side 0: the
    propagator at v''+w/2 (a, t) or w/2+v'' (p); side 1: at v''-w/2 or w/2-v'')."""
    ls, rs = CLASS_SEL[cls]
    f = class_freqs(V1.grids, cls, V1.A, idx)
    gb = np.ascontiguousarray(np.asarray(gbar, dtype=np.complex128).reshape(-1, 16))
    if len(gb) != len(f):
        raise ValueError("gbar does not match the class's points")
    iw = np.ascontiguousarray(class_omega_index(V1.grids, cls, idx))
    gl = zero_grads(V1.grids) if want_left else None
    gr = zero_grads(V2.grids) if want_right else None
    ggr = None
    n_gr = 0
    if want_gr:
        nw = class_shape(V1.grids, cls)[0]
        ggr = np.zeros((nw, Nq, 2), dtype=np.complex128)
        n_gr = ggr.size
    sl = _ograd(gl) if gl is not None else None
    sr = _ograd(gr) if gr is not None else None
    rc = lib().og_bubble_vjp_points(V1.ptr(), V2.ptr(), P.ptr(), C.c_int(pi_kind), C.c_int(r), C.c_int(ls),
                                    C.c_int(rs), C.c_int(Nq), C.c_int(len(f)), _dptr(f),
                                    gb.ctypes.data_as(C.c_void_p), iw.ctypes.data_as(C.c_void_p),
                                    C.byref(sl) if sl is not None else None,
                                    C.byref(sr) if sr is not None else None,
                                    ggr.ctypes.data_as(C.c_void_p) if ggr is not None else None, C.c_int(n_gr),
                                    C.c_int(nthreads))
    if rc != 0:
        raise RuntimeError("og_bubble_vjp_points failed: %d" % rc)
    return gl, gr, ggr


def integrand(V1, V2, P, r, lsel, rsel, w, v, vp, xs, pi_kind=PI_GG):
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    out = np.zeros((len(xs), 16), dtype=np.complex128)
    lib().og_integrand(V1.ptr(), V2.ptr(), P.ptr(), C.c_int(pi_kind), C.c_int(r), C.c_int(lsel), C.c_int(rsel),
                       C.c_double(w), C.c_double(v), C.c_double(vp), C.c_int(len(xs)), _dptr(xs),
                       out.ctypes.data_as(C.c_void_p))
    return out


def vertex_eval(V, r, spin_uu, side_right, sel, freqs):
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64).reshape(-1, 3))
    out = np.zeros((len(f), 16), dtype=np.complex128)
    lib().og_vertex_eval(V.ptr(), C.c_int(r), C.c_int(spin_uu), C.c_int(side_right), C.c_int(sel),
                         C.c_int(len(f)), _dptr(f), out.ctypes.data_as(C.c_void_p))
    return out


def prop_eval(P, which, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros((len(v), 2, 2), dtype=np.complex128)
    lib().og_prop_eval(P.ptr(), C.c_int(which), C.c_int(len(v)), _dptr(v), out.ctypes.data_as(C.c_void_p))
    return out


def loop(V, P, Nq, nus, nthreads=0, which=0, ud_only=False):
    """Self-energy loop Sigma^{a1'|a1}(v) = -int dv'/(2 pi i) sum Gamma_s^{a1' a2'|a1 a2}(v, v'|v, v')
    P^{a2|a2'}(v') with Gamma_s = Gamma_ud + Gamma_uu (Sec. II.D.2; readings in kb_oracle.c),
    P = G (which 0), the flow scheme's single-scale propagator S (which 1), or the line with one
    insertion of the dSigma tables, G dSigma G (which 2); ud_only: the up-down vertex alone.
    Returns (n, 2, 2) complex: [a1'][a1], 0 = classical, 1 = quantum."""
    nus = np.ascontiguousarray(nus, dtype=np.float64)
    out = np.zeros((len(nus), 2, 2), dtype=np.complex128)
    rc = lib().og_loop_spin(V.ptr(), P.ptr(), C.c_int(which), C.c_int(int(bool(ud_only))), C.c_int(Nq),
                            C.c_int(len(nus)), _dptr(nus),
                       out.ctypes.data_as(C.c_void_p), C.c_int(nthreads))
    if rc != 0:
        raise RuntimeError("og_loop failed: %d" % rc)
    return out


def loop_pieces(V, P, nu, x, which=0):
    """(J (P - M v'/(v'^2+A^2)) [2x2], (pi/2A) v' D(v, v') [16], v' P [2x2]) at one x in (-1, 1)."""
    out = np.zeros(24, dtype=np.complex128)
    lib().og_loop_pieces(V.ptr(), P.ptr(), C.c_int(which), C.c_double(nu), C.c_double(x),
                         out.ctypes.data_as(C.c_void_p))
    return out[:4].reshape(2, 2), out[4:20], out[20:].reshape(2, 2)


def loop_limits(V, P, nu, side, which=0):
    """The loop rule's values at x = side (+-1): ((pi/2A) N [2x2], D_edge [16])."""
    out = np.zeros(20, dtype=np.complex128)
    lib().og_loop_limits(V.ptr(), P.ptr(), C.c_int(which), C.c_double(nu), C.c_int(side),
                         out.ctypes.data_as(C.c_void_p))
    return out[:4].reshape(2, 2), out[4:]


# ----------------------------------------------------------------------------------
# Adaptive Gauss-Lobatto-Kronrod rules (Sec. II.G.5).  The paper prints the nodes:
# GL4 at +-1, +-1/sqrt5; the 7-point extension adds 0, +-sqrt(2/3); the 13-point
# extension adds +-0.942882, +-0.641853, +-0.236383 (six digits).  The weights follow
# from exactness on polynomials; the three extra 13-point nodes are refined to full
# precision by Newton's method on the moment equations (exact to degree 19).
# ----------------------------------------------------------------------------------
def _moments(deg):
    return np.array([2.0 / (k + 1) if k % 2 == 0 else 0.0 for k in range(deg + 1)])


def _sym_weights(half_nodes, degs):
    """Weights of a symmetric rule with nodes +-h (h in half_nodes, 0 allowed once)."""
    M = np.array([[(2.0 if h != 0 else 1.0) * h ** d for h in half_nodes] for d in degs])
    return np.linalg.solve(M, _moments(max(degs))[degs])


def lobatto_kronrod_rules():
    s5, s23 = 1 / np.sqrt(5.0), np.sqrt(2.0 / 3.0)
    # GL4: nodes (1, 1/sqrt5), degrees 0, 2
    w_gl4 = _sym_weights([1.0, s5], [0, 2])
    # GLK7: nodes (1, sqrt(2/3), 1/sqrt5, 0), degrees 0..6 even
    w_k7 = _sym_weights([1.0, s23, s5, 0.0], [0, 2, 4, 6])
    # GLK13: Newton on (x1, x2, x3, 7 weights) for even degrees 0..18
    fixed = [1.0, s23, s5, 0.0]
    z = np.array([0.942882, 0.641853, 0.236383])

    def resid(z):
        nodes = [1.0, z[0], s23, z[1], s5, z[2], 0.0]
        w = _sym_weights(nodes, [0, 2, 4, 6, 8, 10, 12])
        r = []
        for d in (14, 16, 18):
            r.append(sum((2.0 if h != 0 else 1.0) * wi * h ** d for h, wi in zip(nodes, w)) - 2.0 / (d + 1))
        return np.array(r), nodes, w

    for _ in range(50):
        r0, _, _ = resid(z)
        Jm = np.zeros((3, 3))
        for k in range(3):
            dz = np.zeros(3)
            dz[k] = 1e-7
            Jm[:, k] = (resid(z + dz)[0] - resid(z - dz)[0]) / 2e-7
        step = np.linalg.solve(Jm, r0)
        z = z - step
        if np.max(np.abs(step)) < 1e-15:
            break
    r0, nodes13, w13 = resid(z)
    x7 = np.array([-1.0, -s23, -s5, 0.0, s5, s23, 1.0])
    w4_7 = np.array([w_gl4[0], 0.0, w_gl4[1], 0.0, w_gl4[1], 0.0, w_gl4[0]])
    w7_7 = np.array([w_k7[0], w_k7[1], w_k7[2], w_k7[3], w_k7[2], w_k7[1], w_k7[0]])
    half = nodes13[:-1]
    x13 = np.concatenate([-np.array(half), [0.0], np.array(half[::-1])])
    w13h = list(w13[:-1])
    w13a = np.concatenate([np.array(w13h), [w13[-1]], np.array(w13h[::-1])])
    order = np.argsort(x13)
    return dict(x7=x7, w4=w4_7, w7=w7_7, x13=x13[order], w13=w13a[order], kronrod_nodes=z, resid=r0)


def bubble_points_adaptive(V1, V2, P, r, lsel, rsel, freqs, eps=1e-10, depth_max=40, pi_kind=PI_GG,
                           nthreads=0):
    R = lobatto_kronrod_rules()
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64).reshape(-1, 3))
    out = np.zeros((len(f), 16), dtype=np.complex128)
    arrs = [np.ascontiguousarray(R[k]) for k in ("x7", "w4", "w7", "x13", "w13")]
    n = lib().og_bubble_points_adaptive(V1.ptr(), V2.ptr(), P.ptr(), C.c_int(pi_kind), C.c_int(r),
                                        C.c_int(lsel), C.c_int(rsel), C.c_int(len(f)), _dptr(f),
                                        *[_dptr(a) for a in arrs], C.c_double(eps), C.c_int(depth_max),
                                        out.ctypes.data_as(C.c_void_p), C.c_int(nthreads))
    return out, n
