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


LBM_ERR_DIVERGED = 5


@pytest.mark.parametrize("storage,arith,shape", [("FP32", "FP32", (6, 7, 9)), ("FP16S", "FP32", (8, 8, 64)),
                                                 ("FP64", "FP64", (5, 6, 7))])
def test_divergence_check_in_step_finds_an_injected_nan(storage, arith, shape):
    """The failure is made on the host: one population of one cell is set to
    NaN through lbm_set_f.  With the check on every 10 steps, lbm_step stops
    at the first check after the NaN has entered (step 10) with
    LBM_ERR_DIVERGED; the handle stays usable.  A run with the check on and no
    fault gives bit for bit the populations of a run without it."""
    import paper_2112_08926_gb300 as P
    nz, ny, nx = shape
    fields = W.random_fields(shape, seed=5)
    ref = P.Lattice(nx, ny, nz, "D3Q19", "SRT", storage, arith, "AB", tau=0.7)
    ref.set_rho_u(*fields)
    ref.step(40)
    chk = P.Lattice(nx, ny, nz, "D3Q19", "SRT", storage, arith, "AB", tau=0.7)
    chk.set_rho_u(*fields)
    chk.set_divergence_check(10, 1e-6)
    chk.step(17)
    chk.step(23)
    assert np.array_equal(chk.f(), ref.f())
    ref.close()
    f = chk.f()
    f[3, nz // 2, ny // 2, nx // 2] = np.nan
    chk.set_f(f)                       # resets the step counter to 0
    with pytest.raises(P.LBMError) as e:
        chk.step(25)
    assert e.value.status == LBM_ERR_DIVERGED
    assert b"step 10" in chk._L.lbm_last_error(chk.handle)
    assert chk.info().step == 10
    chk.set_divergence_check(0)        # off: the handle still steps
    chk.step(1)
    chk.close()


def test_divergence_check_finds_a_mass_jump():
    """Mass drift beyond the tolerance counts as divergence: the populations
    of one cell get a large positive offset (injected through lbm_set_f
    after the check was set)."""
    import paper_2112_08926_gb300 as P
    shape = (6, 7, 9)
    g = P.Lattice(9, 7, 6, "D3Q19", "SRT", "FP32", "FP32", "AB", tau=0.7)
    g.set_rho_u(*W.random_fields(shape, seed=6))
    g.set_divergence_check(4, 1e-6)
    g.step(8)
    f = g.f()
    f[:, 2, 3, 4] += 0.01
    g.set_f(f)
    with pytest.raises(P.LBMError) as e:
        g.step(8)
    assert e.value.status == LBM_ERR_DIVERGED
    g.set_divergence_check(4, 0.0)     # finiteness only: passes
    g.step(8)
    g.close()
