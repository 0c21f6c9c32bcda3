"""Host-side checks of the C ABI without a GPU: the library builds, loads and exports
every entry point that include/msh.h declares, and the Python binding names them all."""
import re
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "msh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(msh_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1210_5246_gb300 import build, msh
    build.build()
    lib = msh.load()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(msh.SIGNATURES), set(names) ^ set(msh.SIGNATURES)


def test_no_device_means_loud_failure():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1210_5246_gb300 import msh
    with pytest.raises(msh.MshError) as ei:
        msh.Grid((8,), (0.0,), (1.0,), ((1, 1),), 0.5)
    assert ei.value.status == msh.MSH_E_CUDA


def test_header_declares_status_codes():
    src = open(os.path.join(ROOT, "include", "msh.h")).read()
    for name, val in (("MSH_OK", 0), ("MSH_E_INVALID_ARG", 1), ("MSH_E_CUDA", 2), ("MSH_E_NOMEM", 3),
                      ("MSH_E_REALIZABILITY", 4), ("MSH_E_TIMEOUT", 5), ("MSH_E_STATE", 6)):
        assert re.search(rf"#define {name} {val}\b", src), name
