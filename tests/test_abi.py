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


def test_slot_add_and_graph_entry_kinds_rejected_without_context():
    L = kb.lib()
    assert L.kb_vertex_add(None, 0, 0, 1, 15, 1.0, None) == kb.KB_ERR_ARG
    g = ctypes.c_void_p()
    d = (kb.kb_bubble_desc * 2)(kb.kb_join_desc(), kb.kb_join_desc())     # joins only: no context
    assert L.kb_graph_create(ctypes.byref(g), d, 2) == kb.KB_ERR_ARG and not g.value


def test_graph_descriptor_layout_matches_header(tmp_path):
    """sizeof and field offsets of kb_bubble_desc as the C compiler lays it out."""
    import os
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "kb.h"\nint main(void) {\n'
                   '  printf("%zu %zu %zu %zu\\n", sizeof(kb_bubble_desc), offsetof(kb_bubble_desc, alpha),\n'
                   '         offsetof(kb_bubble_desc, precision), offsetof(kb_bubble_desc, op));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    D = kb.kb_bubble_desc
    assert got == [ctypes.sizeof(D), D.alpha.offset, D.precision.offset, D.op.offset]


def test_record_cache_calls_rejected_without_context():
    L = kb.lib()
    assert L.kb_vertex_cache(None, 0, 0, 3, None) == kb.KB_ERR_ARG
    assert L.kb_vertex_uncache(None, 0) == kb.KB_ERR_ARG


def test_regulator_call_rejected_without_context():
    assert kb.lib().kb_set_regulator(None, 0, 1.0) == kb.KB_ERR_ARG


def test_self_energy_derivative_call_rejected_without_context():
    assert kb.lib().kb_set_self_energy_derivative(None, 0, 5.0, None, None) == kb.KB_ERR_ARG


def test_propagator_table_call_rejected_without_context():
    assert kb.lib().kb_set_propagator_table(None, kb.KB_PROP_G, 0, 5.0, None, None) == kb.KB_ERR_ARG


def test_vertex_eval_rejected_without_context():
    assert kb.lib().kb_vertex_eval(None, 0, 0, 0, 1, None, None, None) == kb.KB_ERR_ARG


def test_loop_rejected_without_context():
    assert kb.lib().kb_loop(None, 0, 0, 1, None, None, None) == kb.KB_ERR_ARG


def test_vertex_image_rejected_without_context():
    assert kb.lib().kb_vertex_image(None, 0, 0, 1, 15, None) == kb.KB_ERR_ARG


def test_failure_hooks_reject_null_context():
    L = kb.lib()
    assert L.kb_inject_alloc_failures(None, 1) == kb.KB_ERR_ARG
    assert L.kb_set_wait_budget(None, 0) == kb.KB_ERR_ARG
    assert L.kb_check_wait(None, None) == kb.KB_ERR_ARG
