"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point include/lbm.h declares, rejects bad arguments before
touching the device, and stays separate from the CPU oracle."""
import ctypes
import os
import re

import pytest

import __graft_entry__
from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    import paper_2112_08926_gb300 as P
    return P.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    import paper_2112_08926_gb300 as P
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(P.EXPORTS) == names


def _params(P, **kw):
    d = dict(nx=8, ny=8, nz=8, velset=1, collision=0, storage=1, arith=0, scheme=0, tau=0.8,
             trt_lambda=0.1875)
    d.update(kw)
    p = P.lbm.lbm_params(d["nx"], d["ny"], d["nz"], d["velset"], d["collision"], d["storage"], d["arith"],
                         d["scheme"], d["tau"], d["trt_lambda"], (ctypes.c_double * 3)(0, 0, 0))
    return p


@pytest.mark.parametrize("kw,status", [
    (dict(tau=0.5), 1), (dict(tau=float("nan")), 1), (dict(nx=0), 1), (dict(velset=3), 1),
    (dict(velset=0, nz=2), 1), (dict(collision=3), 1), (dict(collision=2, velset=0, nz=1), 4), (dict(storage=10), 1), (dict(arith=2), 1),
    (dict(scheme=3), 1), (dict(collision=1, trt_lambda=0.0), 1),
    (dict(arith=1, storage=3), 4),                       # FP64 arithmetic with 16-bit storage
    (dict(nx=1300, ny=1300, nz=1300), 4),                # more than 2^31 cells
])
def test_create_rejects_bad_parameters(lib, kw, status):
    import paper_2112_08926_gb300 as P
    h = ctypes.c_void_p()
    assert lib.lbm_create(ctypes.byref(_params(P, **kw)), None, None, ctypes.byref(h)) == status
    assert not h.value


def test_allocator_failure_is_reported_as_oom(lib):
    import paper_2112_08926_gb300 as P
    calls = []

    def alloc(nbytes, ctx):
        calls.append(nbytes)
        return None

    def release(ptr, ctx):
        pass

    a = P.lbm.lbm_allocator(P.lbm._ALLOC_FN(alloc), P.lbm._RELEASE_FN(release), None)
    h = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(_params(P)), ctypes.byref(a), None, ctypes.byref(h))
    assert st == 2 and not h.value
    assert calls and calls[0] == 19 * 8 * 8 * 8 * 4     # one population copy in FP32


def test_codec_entry_points_validate_without_gpu(lib):
    assert lib.lbm_codec_encode(1, None, None, 10, None) == 1        # FP32 is not a 16-bit codec
    assert lib.lbm_codec_encode(3, None, None, 10, None) == 1        # NULL pointers
    assert lib.lbm_codec_encode(3, None, None, 0, None) == 0         # nothing to do
    assert lib.lbm_codec_encode_bits(3, 0, (1 << 32) + 1, None, None) == 1


def test_null_handles_are_rejected(lib):
    assert lib.lbm_step(None, 1) == 1
    assert lib.lbm_destroy(None) == 0
    assert lib.lbm_ensemble_step(None, 1) == 1
    assert lib.lbm_status_string(4) == b"unsupported combination"


def _imports(path):
    out = set()
    for dirpath, _, files in os.walk(path):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                out |= set(re.findall(r"^\s*(?:from|import)\s+([\w.]+)", src, flags=re.M))
    return out


def test_product_and_oracle_are_separate():
    prod = _imports(os.path.join(ROOT, "paper_2112_08926_gb300"))
    orc = _imports(os.path.join(ROOT, "oracle"))
    assert not any(m.startswith("oracle") for m in prod)
    assert not any(m.startswith("paper_2112_08926_gb300") for m in orc)
    csrc = os.path.join(ROOT, "paper_2112_08926_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower(), f
    for f in ("codecs.cpp", "lattice.cpp", "oracle.h"):
        src = open(os.path.join(ROOT, "oracle", f)).read()
        assert "lbm_device" not in src and "lbm_kernels" not in src and '#include "lbm.h"' not in src


def test_missing_library_fails_loudly(monkeypatch):
    import paper_2112_08926_gb300.lbm as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", "/nonexistent/liblbm.so")
    with pytest.raises(ImportError):
        L.load()
