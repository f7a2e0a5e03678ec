"""Failure detection without a GPU fault.

Every device-side wait of the library is bounded: the wait gives up after
about a second, the kernel records it in the handle's status word, and the
host reports LBM_ERR_TIMEOUT.  The self-test entry point makes such a wait
run out on purpose (an mbarrier that nothing arrives on); the handle is then
poisoned while the CUDA context stays usable for other lattices.
"""
import ctypes
import time

import numpy as np
import pytest

import __graft_entry__
import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LBM_ERR_TIMEOUT, LBM_ERR_STATE = 6, 7


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def test_bounded_wait_runs_out_and_is_reported():
    import paper_2112_08926_gb300 as P
    L = P.load()
    g = P.Lattice(8, 8, 8, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=0.8)
    t0 = time.perf_counter()
    st = L.lbm_selftest_wait_timeout(g.handle)
    dt = time.perf_counter() - t0
    assert st == LBM_ERR_TIMEOUT
    assert 0.5 < dt < 30.0
    assert b"gave up" in L.lbm_last_error(g.handle)
    # the handle is poisoned ...
    with pytest.raises(P.LBMError) as e:
        g.step(1)
    assert e.value.status == LBM_ERR_STATE
    g.close()
    # ... the context is not: a new lattice still matches the oracle bit for bit
    shape = (6, 7, 9)
    fields = W.random_fields(shape, seed=21)
    h = P.Lattice(9, 7, 6, "D3Q19", "SRT", "FP16S", "FP32", "AB", tau=0.8)
    h.set_rho_u(*fields)
    h.step(5)
    o = oracle.Lattice(9, 7, 6, "D3Q19", "SRT", "ORD32", "FP16S", tau=0.8)
    o.set_rho_u(*fields)
    o.step(5)
    assert np.array_equal(h.f(), o.f())
    h.close()


def test_null_handle_is_rejected():
    import paper_2112_08926_gb300 as P
    assert P.load().lbm_selftest_wait_timeout(ctypes.c_void_p(0)) == 1
