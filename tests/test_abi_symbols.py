"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/mlc.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mlc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mlc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_call_list():
    names = declared_functions()
    for required in ["mlc_plan_create", "mlc_solve", "mlc_batch_solve", "mlc_server_enqueue"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1702_08111_gb300 import build, mlc
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(mlc.EXPORTED) <= set(declared_functions())


def test_status_strings_without_gpu():
    from paper_1702_08111_gb300 import mlc
    lib = mlc.load_library()
    assert lib.mlc_status_string(0) == b"ok"
    assert lib.mlc_status_string(5).startswith(b"request exceeds")
