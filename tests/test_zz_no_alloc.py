"""The allocation-free field readback, lbm_get_rho_u_static, against
lbm_get_rho_u (which stages through memory from the lattice's allocator).

It serves callers that cannot allocate device memory while they read out a
simulation (a lattice that fills the GPU, or a process whose memory pool
belongs to another framework).  Called through the C ABI twice in a row, with
a step in between so that the shared static array holds the previous call's
results when the second call starts; both calls must return exactly what
lbm_get_rho_u returns.  Lattices whose xy-plane does not fit the static array
are refused with LBM_ERR_UNSUPPORTED.  A fresh process checks that the first
call takes no device memory (the array is placed when the lattice is
created), and a lattice whose bounded wait gave up reports it here as in
lbm_get_rho_u.  This file is collected last."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import __graft_entry__
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _read(lib, g, fn):
    out = [np.empty(g.N, dtype=np.float64) for _ in range(4)]
    st = getattr(lib, fn)(g.handle, *[ctypes.c_void_p(a.ctypes.data) for a in out])
    return st, [a.reshape(g.shape) for a in out]


@pytest.mark.parametrize("storage,scheme,shape", [
    ("FP16S", "AB", (150, 64, 64)),     # three chunks of the static array; chunked layout
    ("FP32", "AA", (9, 23, 37)),        # flags, in-place streaming
    ("FP64", "AB", (5, 6, 7)),
])
def test_static_readback_matches_allocating_readback(storage, scheme, shape):
    import paper_2112_08926_gb300 as P
    lib = P.load()
    nz, ny, nx = shape
    arith = "FP64" if storage == "FP64" else "FP32"
    g = P.Lattice(nx, ny, nz, "D3Q19", "SRT", storage, arith, scheme, tau=0.7, force=(1e-5, 0.0, 0.0))
    if storage != "FP16S":
        g.set_geometry(*W.random_geometry(shape, 3, outflow=0.0, freeslip_frac=0.0))
    g.set_rho_u(*W.random_fields(shape, 4))
    for _ in range(2):
        g.step(3)
        st_ref, ref = _read(lib, g, "lbm_get_rho_u")
        st, got = _read(lib, g, "lbm_get_rho_u_static")
        assert st_ref == 0 and st == 0
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
    g.close()


def test_static_readback_refuses_planes_beyond_the_buffer():
    import paper_2112_08926_gb300 as P
    lib = P.load()
    g = P.Lattice(1024, 257, 1, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=0.7)
    g.set_rho_u()
    st, _ = _read(lib, g, "lbm_get_rho_u_static")
    assert st == P.lbm.LBM_ERR_UNSUPPORTED
    assert b"262144" in lib.lbm_last_error(g.handle)
    g.close()


def test_static_readback_reports_a_wait_that_gave_up():
    """After a kernel's bounded wait ran out, the readback must not hand out
    the fields of an unfinished update as if nothing happened."""
    import paper_2112_08926_gb300 as P
    lib = P.load()
    g = P.Lattice(16, 8, 4, "D3Q19", "SRT", "FP32", "FP32", "AB", tau=0.7)
    g.set_rho_u()
    assert lib.lbm_selftest_wait_timeout(g.handle) == P.lbm.LBM_ERR_TIMEOUT
    st, _ = _read(lib, g, "lbm_get_rho_u_static")
    assert st in (P.lbm.LBM_ERR_TIMEOUT, P.lbm.LBM_ERR_STATE)
    g.close()


_FRESH = r"""
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2112_08926_gb300 as P
lib = P.load()
nz, ny, nx = 40, 48, 64
g = P.Lattice(nx, ny, nz, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=0.7)
g.set_rho_u(np.full((nz, ny, nx), 1.001), np.full((nz, ny, nx), 0.01))
g.step(2)
ref = g.rho_u()                      # loads the probe kernel, like any first readback
torch.cuda.synchronize()
torch.cuda.reset_peak_memory_stats()
free0 = torch.cuda.mem_get_info()[0]
alloc0 = torch.cuda.memory_allocated()
bytes0 = g.info().device_bytes
out = [np.empty(g.N, dtype=np.float64) for _ in range(4)]
st = lib.lbm_get_rho_u_static(g.handle, *[ctypes.c_void_p(a.ctypes.data) for a in out])
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
print(st, free0 - free1, torch.cuda.max_memory_allocated() - alloc0, g.info().device_bytes - bytes0,
      int(all(np.array_equal(a.reshape(g.shape), b) for a, b in zip(out, ref))))
"""


def test_first_static_call_in_a_fresh_process_takes_no_device_memory():
    """The first call in a process takes no device memory: not through the
    lattice's allocator (torch's caching allocator here), and not through the
    CUDA runtime placing the static array (done when the lattice was
    created)."""
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    st, free_drop, torch_peak, lattice_bytes, same = (int(v) for v in r.stdout.split()[-5:])
    assert st == 0
    assert free_drop == 0, f"device free memory fell by {free_drop} bytes"
    assert torch_peak == 0 and lattice_bytes == 0
    assert same == 1
