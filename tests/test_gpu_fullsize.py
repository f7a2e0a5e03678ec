"""Parity at the benchmark's full size and launch configuration: D3Q19 SRT
Taylor-Green vortex, periodic 256^3, FP32 arithmetic with FP16S (and FP32)
storage, A-B streaming through the kernel variant bench.py times (the
default); and a 640^3 TRT lid-driven cavity whose populations need 64-bit
offsets.  The oracle recomputes sampled cells one by one (a 1x1x1 periodic
lattice collides exactly the populations it is given); every kernel variant
must equal the generic kernel bit for bit; the FP64 mass sum must stay
constant."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 256


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


@pytest.fixture(scope="module")
def fields():
    return W.taylor_green_3d(N, 0.05)


def lattice(fields, storage="FP16S", variant="auto"):
    import paper_2112_08926_gb300 as P
    g = P.Lattice(N, N, N, "D3Q19", "SRT", storage, "FP32", "AB", tau=0.53)
    g.set_variant(variant)
    g.set_rho_u(*fields)
    return g


@pytest.mark.parametrize("storage", ["FP16S", "FP32"])
def test_sampled_cells_against_oracle(fields, storage):
    g = lattice(fields, storage)
    g.step(3)
    f0 = g.f()
    g.step(1)
    f1 = g.f()
    g.close()
    c, _ = oracle.velset("D3Q19")
    rng = np.random.default_rng(5)
    cells = rng.integers(0, N, (150, 3))
    cells[:4] = [[0, 0, 0], [N - 1, N - 1, N - 1], [0, N - 1, 7], [N - 1, 0, 0]]   # wrap corners
    o = oracle.Lattice(1, 1, 1, "D3Q19", "SRT", "ORD32", storage, tau=0.53)
    for z, y, x in cells:
        o.set_f(f0[:, z, y, x].reshape(19, 1, 1, 1))
        o.step(1)
        post = o.f().reshape(19)
        got = np.array([f1[i, (z + c[i, 2]) % N, (y + c[i, 1]) % N, (x + c[i, 0]) % N] for i in range(19)])
        assert np.array_equal(got, post), (z, y, x)


def test_kernel_variants_agree_at_full_size(fields):
    ref = lattice(fields, variant="generic")
    assert ref.variant() == "generic"
    ref.step(10)
    fr = ref.f()
    ref.close()
    for v in ("paired", "staged"):
        g = lattice(fields, variant=v)
        assert g.variant() == v
        g.step(10)
        assert np.array_equal(g.f(), fr), v
        g.close()


def test_mass_is_conserved_at_full_size(fields):
    g = lattice(fields)
    m0, e0 = g.reduce()
    g.step(200)
    m1, e1 = g.reduce()
    assert abs(m1 / m0 - 1) < 1e-6
    assert 0 < e1 < e0


def _cavity_640(scheme, n=640, u_lid=0.1, re=1000.0):
    import paper_2112_08926_gb300 as P
    tau = 0.5 + 3 * u_lid * (n - 2) / re
    g = P.Lattice(n, n, n, "D3Q19", "TRT", "FP16S", "FP32", scheme, tau=tau)
    g.set_geometry(W.cavity_flags(n))
    g.set_nodes(*W.cavity_lid(n, u_lid))
    g.set_rho_u()
    return g, tau


def test_cavity_with_64bit_offsets_against_oracle():
    """D3Q19 TRT lid-driven cavity, 640^3, FP16S: 19 N > 2^32, so populations
    are addressed with 64-bit offsets.  Sampled cells (near the lid, where
    the flow has started, and deep inside) are recomputed by the oracle from
    the streamed populations; in-place A-A must equal A-B bit for bit."""
    n = 640
    c, _ = oracle.velset("D3Q19")
    rng = np.random.default_rng(9)
    near_lid = np.stack([rng.integers(n - 6, n - 2, 80), rng.integers(2, n - 2, 80), rng.integers(2, n - 2, 80)], 1)
    inside = rng.integers(2, n - 2, (40, 3))
    sample = np.concatenate([near_lid, inside, [[n - 3, n - 3, n - 3], [n - 3, 2, n - 3], [2, 2, 2]]])
    flat = lambda zyx: zyx[:, 2] + n * (zyx[:, 1] + n * zyx[:, 0])
    dest = np.stack([flat(sample + c[i][::-1]) for i in range(19)])       # (19, samples)
    runs = {}
    for scheme in ("AB", "AA"):
        g, tau = _cavity_640(scheme)
        g.step(6)
        f0 = g.f_cells(flat(sample))
        g.step(1)
        f1 = g.f_cells(dest.reshape(-1)).reshape(19, 19, -1)
        runs[scheme] = (f0, f1, g.rho_u_cells(flat(sample)))
        g.close()
    f0, f1, _ = runs["AB"]
    assert np.abs(f0[:, :80]).max() > 0      # the lid has set the top layers moving
    o = oracle.Lattice(1, 1, 1, "D3Q19", "TRT", "ORD32", "FP16S", tau=tau)
    for k in range(sample.shape[0]):
        o.set_f(f0[:, k].reshape(19, 1, 1, 1))
        o.step(1)
        post = o.f().reshape(19)
        got = np.array([f1[i, i, k] for i in range(19)])
        assert np.array_equal(got, post), sample[k]
    (a0, a1, a_fields), (b0, b1, b_fields) = runs["AB"], runs["AA"]
    assert np.array_equal(a0, b0) and np.array_equal(a1, b1)
    for x, y in zip(a_fields, b_fields):
        assert np.array_equal(x, y)
