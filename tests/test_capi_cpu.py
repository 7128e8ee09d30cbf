"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol the header declares, its host-only collocation table agrees with
the oracle, and set-up calls fail with an error code instead of crashing when
no device is usable."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "pbad.h")).read()
    return sorted(set(re.findall(r"PBAD_API\s+[\w\s\*]+?\b(pbad_\w+)\s*\(", text)))


def test_library_exports_every_header_symbol():
    from paper_1709_04145_b300 import _native
    lib = _native.lib()
    syms = _header_symbols()
    assert len(syms) >= 13
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(_native.SYMBOLS) == syms


def test_version_and_last_error():
    from paper_1709_04145_b300 import _native
    lib = _native.lib()
    assert lib.pbad_version() >= 100
    assert isinstance(lib.pbad_last_error(), bytes)


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5])
def test_library_colloc_matches_oracle(S):
    import paper_1709_04145_b300 as P
    n1, W1 = P.colloc(S)
    n2, W2 = O.colloc(S)
    assert np.max(np.abs(n1 - n2)) < 1e-15
    assert np.max(np.abs(W1 - W2)) < 1e-12 * np.max(np.abs(W2))


def test_colloc_rejects_bad_stage_count():
    from paper_1709_04145_b300 import _native
    lib = _native.lib()
    nodes = (C.c_double * 16)()
    W = (C.c_double * 64)()
    assert lib.pbad_colloc(0, nodes, W) == -1
    assert lib.pbad_colloc(6, nodes, W) == -1
    assert b"stages" in lib.pbad_last_error()


def test_model_create_rejects_malformed_tree():
    from paper_1709_04145_b300 import _native
    lib = _native.lib()
    parent = (C.c_int32 * 2)(-1, 1)  # parent[1] == 1 is not < 1
    jt = (C.c_int32 * 2)(0, 0)
    ax = (C.c_double * 6)(0, 1, 0, 0, 1, 0)
    mm = (C.c_double * 20)()
    rest = (C.c_double * 24)()
    g = (C.c_double * 3)(0, 0, -9.81)
    out = C.c_void_p()
    rc = lib.pbad_model_create(2, parent, jt, ax, 1, mm, rest, g, 0, C.byref(out))
    assert rc == -1 and not out.value


def test_model_create_without_usable_device_returns_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300 import inputs as I
    with pytest.raises(P.PBADError):
        P.Model.from_spec(I.rod_chain(1, 3))


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1709_04145_b300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _native.lib()


def test_header_constants_match_binding():
    """Solver, joint-type and status codes of include/pbad.h are the ones the
    Python binding passes."""
    import re
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300 import inputs as I
    text = open(os.path.join(ROOT, "include", "pbad.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define (PBAD_\w+) \(?(-?\d+)\)?", text)}
    assert defs["PBAD_LBFGS"] == P.LBFGS
    assert defs["PBAD_NEWTON"] == P.NEWTON
    assert defs["PBAD_LBFGS_F32"] == P.LBFGS_F32
    assert (defs["PBAD_HINGE"], defs["PBAD_BALL"], defs["PBAD_TRANSLATION"]) == \
        (I.HINGE, I.BALL, I.TRANSLATION)
    for code, name in P.STATUS.items():
        assert defs["PBAD_" + name] == code


def test_queue_setter_rejects_null_batch():
    from paper_1709_04145_b300._native import lib
    assert lib().pbad_batch_set_queue(None, 0) != 0


def test_build_tracks_every_cuda_source():
    """The in-tree build compiles every .cu file and rebuilds when any .cu or
    .cuh file changes (a header left out of its dependency list would leave
    a stale library)."""
    import os

    from paper_1709_04145_b300 import _build
    files = os.listdir(_build.CSRC)
    assert sorted(f for f in files if f.endswith(".cu")) == sorted(_build.SOURCES)
    assert sorted(f for f in files if f.endswith(".cuh")) == sorted(_build.HEADERS)
