"""Thin ctypes binding of libkb (include/kb.h): the same entry points, argument
marshalling only.  Every step of the bubble runs in the library's CUDA kernels; there is
no CPU fallback — if libkb.so cannot be built or loaded, importing the functions fails.
"""

import ctypes as C
import os
import re

from . import build as _build

KB_OK, KB_ERR_ARG, KB_ERR_STATE, KB_ERR_CUDA, KB_ERR_OOM, KB_ERR_TIMEOUT, KB_ERR_UNSUPPORTED = range(7)
KB_CH_A, KB_CH_P, KB_CH_T = 0, 1, 2
KB_K1, KB_K2, KB_K2P, KB_K3 = 0, 1, 2, 3
KB_MASK_ALL = 0xF
KB_PI_GG, KB_PI_GS_SG = 0, 1
KB_DT_C128, KB_DT_C64 = 0, 1
KB_PREC_FP64, KB_PREC_MIXED = 0, 1
KB_MAX_SLOTS = 16

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kb.h")


class kb_grid_desc(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2w", C.c_int), ("n2v", C.c_int), ("n3w", C.c_int), ("n3v", C.c_int),
                ("nq", C.c_int), ("A", C.c_double)]


class KBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("kb status %d: %s" % (status, msg))
        self.status = status


class kb_vertex_desc(C.Structure):
    _fields_ = [("has_R", C.c_int), ("U", C.c_double), ("channels", C.c_uint),
                ("cls", (C.c_void_p * 4) * 3), ("dtype", (C.c_int * 4) * 3)]


class kb_bubble_desc(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("channel", C.c_int), ("slot_left", C.c_int), ("slot_right", C.c_int),
                ("out_slot", C.c_int), ("pi_kind", C.c_int), ("class_mask", C.c_uint), ("alpha", C.c_double),
                ("beta", C.c_double), ("precision", C.c_int), ("op", C.c_int), ("ctx2", C.c_void_p),
                ("slot2", C.c_int)]


KB_OP_BUBBLE, KB_OP_ADD, KB_OP_JOIN, KB_OP_CACHE, KB_OP_IMAGE, KB_OP_T_SU2, KB_OP_T_SU2_FINISH = 0, 1, 2, 3, 4, 5, 6
KB_ERR_TOO_LARGE = 7
KB_NOALLOC_SCRATCH_BYTES = 32 << 20

_lib = None
_SIGS = {
    "kb_create": [C.POINTER(C.c_void_p), C.c_int],
    "kb_destroy": [C.c_void_p],
    "kb_set_grids": [C.c_void_p, C.POINTER(kb_grid_desc)],
    "kb_set_model": [C.c_void_p, C.c_double, C.c_double, C.c_double],
    "kb_set_self_energy": [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p],
    "kb_set_regulator": [C.c_void_p, C.c_int, C.c_double],
    "kb_set_self_energy_derivative": [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p],
    "kb_set_propagator_table": [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p],
    "kb_set_vertex": [C.c_void_p, C.c_int, C.c_int, C.c_double],
    "kb_set_vertex_channels": [C.c_void_p, C.c_int, C.c_uint],
    "kb_set_vertex_symmetric": [C.c_void_p, C.c_int, C.c_int],
    "kb_set_vertex_class": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int],
    "kb_bubble": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint, C.c_double, C.c_double,
                  C.c_int, C.c_void_p],
    "kb_bubble_t_su2": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint, C.c_double, C.c_void_p],
    "kb_t_su2_finish": [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_void_p],
    "kb_bubble_vjp": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint, C.c_double, C.c_int,
                      C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p],
    "kb_vertex_add": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint, C.c_double, C.c_void_p],
    "kb_vertex_eval": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "kb_loop": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p],
    "kb_vertex_cache": [C.c_void_p, C.c_int, C.c_int, C.c_uint, C.c_void_p],
    "kb_vertex_image": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint, C.c_void_p],
    "kb_vertex_uncache": [C.c_void_p, C.c_int],
    "kb_graph_create": [C.POINTER(C.c_void_p), C.POINTER(kb_bubble_desc), C.c_int],
    "kb_graph_launch": [C.c_void_p, C.c_void_p],
    "kb_graph_kernel_count": [C.c_void_p, C.POINTER(C.c_ulonglong)],
    "kb_graph_destroy": [C.c_void_p],
    "kb_set_workspace_limit": [C.c_void_p, C.c_ulonglong],
    "kb_set_autotune": [C.c_void_p, C.c_int],
    "kb_workspace_bytes": [C.c_void_p, C.POINTER(C.c_ulonglong)],
    "kb_check_device": [C.c_void_p],
    "kb_inject_alloc_failures": [C.c_void_p, C.c_int],
    "kb_set_wait_budget": [C.c_void_p, C.c_longlong],
    "kb_check_wait": [C.c_void_p, C.c_void_p],
    "kb_susceptibility_k1": [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p],
    "kb_keldysh_check": [C.c_void_p, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double), C.c_void_p],
    "kb_vertex_pack": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "kb_vertex_unpack": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "kb_launch_count": [C.c_void_p, C.POINTER(C.c_ulonglong)],
    "kb_bubble_fp64_noalloc": [C.POINTER(kb_grid_desc), C.c_double, C.c_double, C.c_double,
                               C.POINTER(kb_vertex_desc), C.POINTER(kb_vertex_desc), C.c_int, C.c_int, C.c_int,
                               C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p],
    "kb_profile_enable": [C.c_void_p, C.c_int],
    "kb_profile_read": [C.c_void_p, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                        C.POINTER(C.c_ulonglong), C.POINTER(C.c_int)],
}


def lib(path=None):
    """Load libkb.so (building it in-tree first if it is missing or stale); with the
    environment variable KB_CHECKED=1 the bounds-checked variant instead."""
    global _lib
    if _lib is None:
        p = path or _build.build(checked=os.environ.get("KB_CHECKED") == "1")
        L = C.CDLL(p)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.kb_last_error.argtypes = [C.c_void_p]
        L.kb_last_error.restype = C.c_char_p
        L.kb_build_checked.argtypes = []
        L.kb_build_checked.restype = C.c_int
        _lib = L
    return _lib


def declared_symbols():
    """Entry points declared in include/kb.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:kb_status|const char \*)\s*(kb_\w+)\s*\(", txt, re.M)))


def _check(ctx, st):
    if st != KB_OK:
        msg = lib().kb_last_error(ctx).decode() if ctx else ""
        raise KBError(st, msg)


# ---- same-name wrappers --------------------------------------------------------------
def kb_create(device=0):
    ctx = C.c_void_p()
    st = lib().kb_create(C.byref(ctx), device)
    if st != KB_OK:
        raise KBError(st, "kb_create failed (no CUDA device %d?)" % device)
    return ctx


def kb_destroy(ctx):
    _check(None, lib().kb_destroy(ctx))


def kb_set_grids(ctx, n1, n2w, n2v, n3w, n3v, nq, A=5.0):
    g = kb_grid_desc(n1, n2w, n2v, n3w, n3v, nq, A)
    _check(ctx, lib().kb_set_grids(ctx, C.byref(g)))


def kb_set_model(ctx, Delta, T, eps=0.0):
    _check(ctx, lib().kb_set_model(ctx, Delta, T, eps))


KB_REG_DELTA, KB_REG_U, KB_REG_T, KB_REG_NONE = 0, 1, 2, 3
KB_LOOP_UD_ONLY = 4                  # or-ed into kb_loop's line: the up-down vertex alone


def kb_set_regulator(ctx, kind, lam=1.0):
    _check(ctx, lib().kb_set_regulator(ctx, kind, lam))


def kb_set_self_energy_derivative(ctx, dsigR=None, dsigK=None, A_dsig=5.0):
    import numpy as np
    if dsigR is None:
        _check(ctx, lib().kb_set_self_energy_derivative(ctx, 0, A_dsig, None, None))
        return
    r = np.ascontiguousarray(np.asarray(dsigR, dtype=np.complex128))
    k = None if dsigK is None else np.ascontiguousarray(np.asarray(dsigK, dtype=np.complex128))
    _check(ctx, lib().kb_set_self_energy_derivative(ctx, len(r), A_dsig, r.ctypes.data,
                                                    None if k is None else k.ctypes.data))


KB_PROP_G, KB_PROP_S = 0, 1


def kb_set_propagator_table(ctx, which, tabR=None, tabK=None, A_tab=5.0):
    import numpy as np
    if tabR is None:
        _check(ctx, lib().kb_set_propagator_table(ctx, which, 0, A_tab, None, None))
        return
    r = np.ascontiguousarray(np.asarray(tabR, dtype=np.complex128))
    k = None if tabK is None else np.ascontiguousarray(np.asarray(tabK, dtype=np.complex128))
    _check(ctx, lib().kb_set_propagator_table(ctx, which, len(r), A_tab, r.ctypes.data,
                                              None if k is None else k.ctypes.data))


def kb_set_self_energy(ctx, sigR=None, sigK=None, A_sig=5.0):
    import numpy as np
    if sigR is None:
        _check(ctx, lib().kb_set_self_energy(ctx, 0, A_sig, None, None))
        return
    r = np.ascontiguousarray(np.asarray(sigR, dtype=np.complex128))
    k = None if sigK is None else np.ascontiguousarray(np.asarray(sigK, dtype=np.complex128))
    _check(ctx, lib().kb_set_self_energy(ctx, len(r), A_sig, r.ctypes.data, None if k is None else k.ctypes.data))


def kb_set_vertex(ctx, slot, has_R, U=0.0):
    _check(ctx, lib().kb_set_vertex(ctx, slot, int(bool(has_R)), float(U)))


def kb_set_vertex_channels(ctx, slot, mask):
    _check(ctx, lib().kb_set_vertex_channels(ctx, slot, mask))


def kb_set_vertex_symmetric(ctx, slot, symmetric=True):
    _check(ctx, lib().kb_set_vertex_symmetric(ctx, slot, int(bool(symmetric))))


def kb_set_vertex_class(ctx, slot, channel, cls, dev_ptr, dtype):
    _check(ctx, lib().kb_set_vertex_class(ctx, slot, channel, cls, dev_ptr, dtype))


def kb_bubble(ctx, channel, slot_left, slot_right, out_slot, pi_kind=KB_PI_GG, class_mask=KB_MASK_ALL,
              alpha=1.0, beta=0.0, precision=KB_PREC_FP64, stream=0):
    _check(ctx, lib().kb_bubble(ctx, channel, slot_left, slot_right, out_slot, pi_kind, class_mask, alpha, beta,
                                precision, stream))


def kb_bubble_t_su2(ctx, slot, out_slot, pi_kind=KB_PI_GG, class_mask=KB_MASK_ALL, alpha=1.0, stream=0):
    _check(ctx, lib().kb_bubble_t_su2(ctx, slot, out_slot, pi_kind, class_mask, alpha, stream))


def kb_t_su2_finish(ctx, out_slot, a_k3_ptr, a_dtype, alpha=1.0, stream=0):
    _check(ctx, lib().kb_t_su2_finish(ctx, out_slot, a_k3_ptr, a_dtype, alpha, stream))


def kb_t_su2_desc(ctx, slot, out_slot, pi_kind=KB_PI_GG, class_mask=KB_MASK_ALL, alpha=1.0):
    """Step-graph entry: kb_bubble_t_su2."""
    return kb_bubble_desc(ctx, KB_CH_T, slot, slot, out_slot, pi_kind, class_mask, alpha, 0.0, KB_PREC_MIXED,
                          KB_OP_T_SU2)


def kb_t_su2_finish_desc(ctx, out_slot, ctx_a, slot_a, alpha=1.0):
    """Step-graph entry: kb_t_su2_finish with the K3 class of channel a of slot slot_a of
    context ctx_a, after ctx_a's earlier entries."""
    return kb_bubble_desc(ctx, KB_CH_T, -1, -1, out_slot, 0, KB_MASK_ALL, alpha, 0.0, 0, KB_OP_T_SU2_FINISH, ctx_a,
                          slot_a)


def kb_bubble_vjp(ctx, channel, slot_left, slot_right, gout_slot, pi_kind=KB_PI_GG, class_mask=KB_MASK_ALL,
                  alpha=1.0, grad_left_slot=-1, grad_right_slot=-1, grad_GR_K1=None, grad_GR_K2=None,
                  grad_GR_K3=None, precision=KB_PREC_FP64, stream=0):
    _check(ctx, lib().kb_bubble_vjp(ctx, channel, slot_left, slot_right, gout_slot, pi_kind, class_mask, alpha,
                                    grad_left_slot, grad_right_slot, grad_GR_K1, grad_GR_K2, grad_GR_K3,
                                    precision, stream))


def kb_vertex_add(ctx, channel, slot_src, slot_dst, class_mask=KB_MASK_ALL, alpha=1.0, stream=0):
    _check(ctx, lib().kb_vertex_add(ctx, channel, slot_src, slot_dst, class_mask, alpha, stream))


def kb_vertex_eval(ctx, slot, channel, spin_uu, n, freqs_ptr, out_ptr, stream=0):
    _check(ctx, lib().kb_vertex_eval(ctx, slot, channel, int(bool(spin_uu)), n, freqs_ptr, out_ptr, stream))


def kb_loop(ctx, slot, which, n, nus_ptr, out_ptr, stream=0):
    _check(ctx, lib().kb_loop(ctx, slot, which, n, nus_ptr, out_ptr, stream))


def kb_add_desc(ctx, channel, slot_src, slot_dst, class_mask=KB_MASK_ALL, alpha=1.0):
    """Step-graph entry: slot_dst += alpha * slot_src (classes of one channel)."""
    return kb_bubble_desc(ctx, channel, slot_src, -1, slot_dst, 0, class_mask, alpha, 0.0, 0, KB_OP_ADD)


def kb_vertex_cache(ctx, slot, channel, sides=3, stream=0):
    _check(ctx, lib().kb_vertex_cache(ctx, slot, channel, sides, stream))


def kb_vertex_uncache(ctx, slot):
    _check(ctx, lib().kb_vertex_uncache(ctx, slot))


def kb_cache_desc(ctx, channel, slot, sides=3):
    """Step-graph entry: rebuild the record cache of `slot` for `channel` (sides bit 0 left,
    bit 1 right) at every replay."""
    return kb_bubble_desc(ctx, channel, slot, -1, -1, 0, sides, 0.0, 0.0, 0, KB_OP_CACHE)


def kb_vertex_image(ctx, channel, slot_src, slot_dst, class_mask=KB_MASK_ALL, stream=0):
    _check(ctx, lib().kb_vertex_image(ctx, channel, slot_src, slot_dst, class_mask, stream))


def kb_image_desc(ctx, channel, slot_src, slot_dst, class_mask=KB_MASK_ALL):
    """Step-graph entry: slot_dst = the symmetry image of slot_src (one channel)."""
    return kb_bubble_desc(ctx, channel, slot_src, -1, slot_dst, 0, class_mask, 0.0, 0.0, 0, KB_OP_IMAGE)


def kb_join_desc():
    """Step-graph entry: every later entry waits for all earlier ones (all branches)."""
    return kb_bubble_desc(None, 0, -1, -1, -1, 0, 0, 0.0, 0.0, 0, KB_OP_JOIN)


def kb_graph_create(descs):
    """descs: sequence of kb_bubble_desc; returns the graph handle."""
    arr = (kb_bubble_desc * len(descs))(*descs)
    g = C.c_void_p()
    st = lib().kb_graph_create(C.byref(g), arr, len(descs))
    if st != KB_OK:
        ctx = next((d.ctx for d in descs if d.ctx), None)
        raise KBError(st, lib().kb_last_error(ctx).decode() if ctx else "")
    return g


def kb_graph_launch(graph, stream=0):
    _check(None, lib().kb_graph_launch(graph, stream))


def kb_graph_kernel_count(graph):
    v = C.c_ulonglong()
    _check(None, lib().kb_graph_kernel_count(graph, C.byref(v)))
    return v.value


def kb_graph_destroy(graph):
    _check(None, lib().kb_graph_destroy(graph))


def kb_set_autotune(ctx, on=True):
    _check(ctx, lib().kb_set_autotune(ctx, int(bool(on))))


def kb_set_workspace_limit(ctx, nbytes):
    _check(ctx, lib().kb_set_workspace_limit(ctx, int(nbytes)))


def kb_check_device(ctx):
    _check(ctx, lib().kb_check_device(ctx))


def kb_workspace_bytes(ctx):
    v = C.c_ulonglong()
    _check(ctx, lib().kb_workspace_bytes(ctx, C.byref(v)))
    return v.value


def kb_launch_count(ctx):
    v = C.c_ulonglong()
    _check(ctx, lib().kb_launch_count(ctx, C.byref(v)))
    return v.value


def kb_last_error(ctx):
    return lib().kb_last_error(ctx).decode()


def kb_profile_enable(ctx, on=True):
    _check(ctx, lib().kb_profile_enable(ctx, int(bool(on))))


def kb_profile_read(ctx):
    """{kernel name: (total ms, launches)} of the records since profiling was enabled."""
    n = C.c_int()
    _check(ctx, lib().kb_profile_read(ctx, 0, None, None, None, C.byref(n)))
    out = {}
    for i in range(n.value):
        nm, ms, cnt = C.c_char_p(), C.c_double(), C.c_ulonglong()
        _check(ctx, lib().kb_profile_read(ctx, i, C.byref(nm), C.byref(ms), C.byref(cnt), None))
        out[nm.value.decode()] = (ms.value, cnt.value)
    return out


def kb_bubble_fp64_noalloc(grid, Delta, T, eps, left, right, channel, pi_kind, cls, out_ptr, out_dtype, alpha=1.0,
                           beta=0.0, stream=0):
    """Allocation-free FP64 bubble of one class (see include/kb.h); returns the status."""
    return lib().kb_bubble_fp64_noalloc(C.byref(grid), Delta, T, eps, C.byref(left), C.byref(right), channel,
                                        pi_kind, cls, out_ptr, out_dtype, alpha, beta, stream)


def kb_inject_alloc_failures(ctx, n):
    _check(ctx, lib().kb_inject_alloc_failures(ctx, int(n)))


def kb_set_wait_budget(ctx, cycles):
    _check(ctx, lib().kb_set_wait_budget(ctx, int(cycles)))


def kb_check_wait(ctx, stream=None):
    _check(ctx, lib().kb_check_wait(ctx, stream))


def kb_susceptibility_k1(ctx, channel, slot, U, out_ptr, stream=None):
    _check(ctx, lib().kb_susceptibility_k1(ctx, channel, slot, U, out_ptr, stream))


def kb_keldysh_check(ctx, slot, channel, T, stream=None):
    """Residuals of the physical Keldysh structure (8 floats, see include/kb.h)."""
    out = (C.c_double * 8)()
    _check(ctx, lib().kb_keldysh_check(ctx, slot, channel, T, out, stream))
    return list(out)


def kb_vertex_pack(ctx, slot, channel, cls, dst_ptr, stream=None):
    _check(ctx, lib().kb_vertex_pack(ctx, slot, channel, cls, dst_ptr, stream))


def kb_vertex_unpack(ctx, slot, channel, cls, src_ptr, stream=None):
    _check(ctx, lib().kb_vertex_unpack(ctx, slot, channel, cls, src_ptr, stream))


def kb_build_checked():
    """1 if the loaded library is the bounds-checked variant (KB_CHECKED=1 at load)."""
    return lib().kb_build_checked()
