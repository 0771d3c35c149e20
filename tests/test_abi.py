"""CPU checks of the C-ABI library: it builds, loads and exports every
entry point that include/*.h declares; host-side argument checks behave."""
import ctypes
import glob
import os
import re

import pytest

from paper_2502_00317_gb300 import kclique as kc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(kc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("kc_create", "kc_destroy", "kc_upload", "kc_free_graph", "kc_count", "kc_list", "kc_list_range",
                 "kc_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = kc.load()
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(_declared()) <= set(kc.EXPORTS)
    for n in kc.EXPORTS:
        assert callable(getattr(kc, n))


def test_status_names():
    for code, name in [(0, "KC_OK"), (1, "KC_E_INVALID_ARG"), (2, "KC_E_INVALID_GRAPH"), (4, "KC_E_CAPACITY"),
                       (5, "KC_E_DEVICE_TIMEOUT"), (8, "KC_E_UNSUPPORTED"), (9, "KC_E_NOT_FOUND")]:
        assert kc.kc_strerror(code) == name
    assert kc.kc_strerror(12345) == "KC_E_UNKNOWN"


def test_null_arguments_rejected_without_a_device():
    lib = kc.load()
    assert lib.kc_create(None, 0, None) == kc.KC_E_INVALID_ARG
    assert lib.kc_destroy(None) == kc.KC_E_INVALID_ARG
    assert lib.kc_count(None, 1, 3, None, None) == kc.KC_E_INVALID_ARG
    assert lib.kc_list(None, 1, 3, None, 0, None, None, None, None) == kc.KC_E_INVALID_ARG
    assert lib.kc_last_stats(None, None) == kc.KC_E_INVALID_ARG
    assert lib.kc_serve_start(None, None) == kc.KC_E_INVALID_ARG
    assert lib.kc_serve_submit(None, 1, 3, 0, None) == kc.KC_E_INVALID_ARG
    assert lib.kc_serve_poll(None, 1, None) == kc.KC_E_INVALID_ARG
    assert lib.kc_serve_stop(None) == kc.KC_E_INVALID_ARG
    assert lib.kc_count_batched(None, None, None, 0, None, None) == kc.KC_E_INVALID_ARG


def test_create_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = kc.load().kc_create(ctypes.byref(h), 0, None)
    assert st in (kc.KC_E_CUDA, kc.KC_E_OOM)
    assert not h.value


def test_struct_sizes_match_header(tmp_path):
    """The ctypes mirrors have the layout the C compiler gives the header's structs."""
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    names = ["kc_opts", "kc_graph_info", "kc_stats", "kc_upload_stats", "kc_serve_opts", "kc_serve_result",
             "kc_serve_stats"]
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "kclique.h"\nint main(void) {\n' +
                   "".join(f'  printf("%zu\\n", sizeof({n}));\n' for n in names) + "  return 0;\n}\n")
    exe = tmp_path / "sizes"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    for n, size in zip(names, got):
        assert ctypes.sizeof(getattr(kc, n)) == size, n
