"""The C-ABI library builds, loads and exports every entry point include/kb.h declares
(no compute call: runs without a GPU)."""

import ctypes

from paper_2405_20996_gb300 import kb


def test_library_exports_declared_symbols():
    names = kb.declared_symbols()
    assert "kb_bubble" in names and "kb_create" in names and len(names) >= 10
    L = kb.lib()
    for n in names:
        assert hasattr(L, n), n


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    ctx = ctypes.c_void_p()
    st = kb.lib().kb_create(ctypes.byref(ctx), 0)
    assert st == kb.KB_ERR_CUDA and not ctx.value


def test_null_context_arguments_rejected():
    L = kb.lib()
    assert L.kb_bubble(None, 0, 0, 0, 0, 0, 15, 1.0, 0.0, 0, None) == kb.KB_ERR_ARG
    assert L.kb_set_model(None, 1.0, 0.1, 0.0) == kb.KB_ERR_ARG
    assert L.kb_last_error(None) == b"null context"


def test_null_arguments_of_vjp_and_graph_rejected():
    L = kb.lib()
    assert L.kb_bubble_vjp(None, 0, 0, 0, 0, 0, 15, 1.0, -1, -1, None, None, None, 0, None) == kb.KB_ERR_ARG
    g = ctypes.c_void_p()
    assert L.kb_graph_create(ctypes.byref(g), None, 0) == kb.KB_ERR_ARG and not g.value
    d = (kb.kb_bubble_desc * 1)()
    assert L.kb_graph_create(ctypes.byref(g), d, 1) == kb.KB_ERR_ARG      # null context
    assert L.kb_graph_launch(None, None) == kb.KB_ERR_ARG
    assert L.kb_graph_destroy(None) == kb.KB_ERR_ARG
    assert L.kb_set_workspace_limit(None, 1 << 30) == kb.KB_ERR_ARG
