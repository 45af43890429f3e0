"""The C-ABI library builds, loads and exports what include/gamma.h declares;
the Python binding's structures match the C layout.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "gamma.h")


def _declared():
    src = open(HDR).read()
    return sorted(set(re.findall(r"GAMMA_API[^;(]*?\b(gamma_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["gamma_create", "gamma_destroy", "gamma_load_graph", "gamma_register_query",
              "gamma_apply_batch", "gamma_fetch_matches", "gamma_commit", "gamma_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2401_17018_gb300 import build
    lib_path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gamma_\w+)", out))
    assert set(_declared()) <= exported
    lib = ctypes.CDLL(lib_path)
    for n in _declared():
        assert getattr(lib, n) is not None


def test_binding_has_the_c_names():
    from paper_2401_17018_gb300 import gamma
    for n in _declared():
        assert callable(getattr(gamma, n)), n


def test_struct_layouts_match_header(tmp_path):
    from paper_2401_17018_gb300 import gamma
    c = tmp_path / "sz.c"
    c.write_text('#include "gamma.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                 'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(gamma_options), sizeof(gamma_matches),'
                 ' sizeof(gamma_stats), offsetof(gamma_matches, written), offsetof(gamma_stats, expansions));'
                 'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(gamma.gamma_options), ctypes.sizeof(gamma.gamma_matches), ctypes.sizeof(gamma.gamma_stats),
            gamma.gamma_matches.written.offset, gamma.gamma_stats.expansions.offset]
    assert got == want


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2401_17018_gb300 import gamma
    with pytest.raises(gamma.GammaError) as e:
        gamma.Context()
    assert e.value.code == gamma.GAMMA_ECUDA


def test_null_handles_are_rejected_without_a_gpu():
    """Every entry point refuses a null context or server with GAMMA_EINVAL
    (no device work is attempted, nothing crashes)."""
    from paper_2401_17018_gb300 import gamma
    lib = gamma.load_library()
    E = gamma.GAMMA_EINVAL
    i64 = ctypes.c_int64(0)
    i32 = ctypes.c_int32(0)
    calls = {
        "gamma_load_graph": (None, 1, None, 0, None, None),
        "gamma_register_query": (None, 2, None, 1, None, None, ctypes.byref(i32)),
        "gamma_apply_batch": (None, 0, None, None, None, 0, None, None, None, None),
        "gamma_apply_batches": (None, 1, None, None, None, None, 0, None, None, None),
        "gamma_load_graph_el": (None, 1, None, 0, None, None, None),
        "gamma_register_query_el": (None, 2, None, 1, None, None, None, ctypes.byref(i32)),
        "gamma_apply_batch_el": (None, 0, None, None, None, None, 0, None, None, None, None),
        "gamma_fetch_matches": (None, None),
        "gamma_commit": (None,),
        "gamma_update_counts": (None, 0, None),
        "gamma_recount_noalloc": (None, 1, None, None),
        "gamma_autotune": (None, 0, None, 1, None),
        "gamma_export_adjacency": (None, None, None, None, 0),
        "gamma_get_stats": (None, None),
        "gamma_set_options": (None, None),
        "gamma_reserve_vertices": (None, 4),
        "gamma_add_vertices": (None, 1, None, ctypes.byref(i32)),
        "gamma_vertex_neighbors": (None, 0, None, 0, ctypes.byref(i64)),
        "gamma_checkpoint": (None, None, 0, ctypes.byref(i64)),
        "gamma_restore": (None, None, 0),
        "gamma_server_stats_get": (None, None),
        "gamma_server_stop": (None,),
    }
    for name, args in calls.items():
        if name not in gamma._SIGS:
            continue
        assert getattr(lib, name)(*args) == E, name
    assert lib.gamma_last_error(None) == b"null context"
    lib.gamma_destroy(None)
