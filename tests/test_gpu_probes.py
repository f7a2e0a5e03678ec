"""Point probes and sparse boundary-node data through the C ABI.

lbm_get_f_cells / lbm_get_rho_u_cells must return exactly the values of the
full readbacks at the listed cells, in every memory layout and precision;
lbm_set_nodes must give bit for bit the lattice that full node arrays give.
"""
import numpy as np
import pytest

import __graft_entry__
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _P():
    import paper_2112_08926_gb300 as P
    return P


CASES = [  # (shape (nz, ny, nx), storage, arith, scheme, flags?, variant)
    ((6, 5, 128), "FP16S", "FP32", "AB", False, "auto"),       # chunked layout
    ((6, 5, 64), "FP16C", "FP32", "AB", False, "generic"),     # SoA
    ((7, 9, 11), "FP32", "FP32", "AB", True, "auto"),
    ((7, 9, 11), "P16_1S", "FP32", "AA", True, "auto"),
    ((5, 6, 7), "FP64", "FP64", "AA", False, "auto"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[1]}-{c[3]}-{'flags' if c[4] else 'free'}-{c[5]}")
def test_point_probes_equal_full_readback(case):
    shape, storage, arith, scheme, with_flags, variant = case
    nz, ny, nx = shape
    g = _P().Lattice(nx, ny, nz, "D3Q19", "TRT", storage, arith, scheme, tau=0.7)
    g.set_variant(variant)
    if with_flags:
        extra = {"outflow": 0.0, "freeslip_frac": 0.0} if scheme == "AA" else {}
        flags, node_u, node_rho = W.random_geometry(shape, seed=3, **extra)
        g.set_geometry(flags, node_u, node_rho)
    g.set_rho_u(*W.random_fields(shape, seed=4))
    g.step(3)
    full_f = g.f().reshape(19, -1)
    full = [a.reshape(-1) for a in g.rho_u()]
    rng = np.random.default_rng(1)
    cells = np.concatenate([[0, nx * ny * nz - 1, 5, 5], rng.integers(0, nx * ny * nz, 60)]).astype(np.int64)
    fc = g.f_cells(cells)
    assert np.array_equal(fc, full_f[:, cells])
    pts = g.rho_u_cells(cells)
    for a, b in zip(pts, full):
        assert np.array_equal(a, b[cells])
    # (z, y, x) triples name the same cells
    zyx = np.stack([cells // (nx * ny), (cells // nx) % ny, cells % nx], axis=1)
    assert np.array_equal(g.f_cells(zyx), fc)
    # empty list
    assert g.f_cells(np.zeros(0, dtype=np.int64)).shape == (19, 0)
    g.close()


def test_point_probe_rejects_bad_indices():
    P = _P()
    g = P.Lattice(4, 4, 4, "D3Q19", "SRT", "FP32", "FP32", "AB", tau=0.8)
    for bad in ([64], [-1], [3, 70]):
        with pytest.raises(P.LBMError) as e:
            g.f_cells(np.array(bad, dtype=np.int64))
        assert e.value.status == 1
    g.step(1)   # the handle stays usable
    g.close()


@pytest.mark.parametrize("scheme", ["AB", "AA"])
def test_sparse_nodes_equal_full_node_arrays(scheme):
    P = _P()
    n, u_lid = 20, 0.08
    flags, node_u = W.cavity(n, u_lid)
    a = P.Lattice(n, n, n, "D3Q19", "TRT", "FP16S", "FP32", scheme, tau=0.6)
    a.set_geometry(flags, node_u)
    a.set_rho_u()
    b = P.Lattice(n, n, n, "D3Q19", "TRT", "FP16S", "FP32", scheme, tau=0.6)
    b.set_geometry(W.cavity_flags(n))
    cells, u = W.cavity_lid(n, u_lid)
    b.set_nodes(cells, u)
    b.set_rho_u()
    a.step(25)
    b.step(25)
    assert np.array_equal(a.f(), b.f())
    a.close()
    b.close()


def test_sparse_nodes_set_equilibrium_states():
    P = _P()
    shape = (8, 9, 10)
    flags, node_u, node_rho = W.random_geometry(shape, seed=11)
    a = P.Lattice(10, 9, 8, "D3Q19", "SRT", "FP32", "FP32", "AB", tau=0.9)
    a.set_geometry(flags, node_u, node_rho)
    a.set_rho_u()
    b = P.Lattice(10, 9, 8, "D3Q19", "SRT", "FP32", "FP32", "AB", tau=0.9)
    b.set_geometry(flags)
    cells = np.flatnonzero((flags.reshape(-1) & (W.MOVING | W.EQ)) != 0).astype(np.int64)
    b.set_nodes(cells, node_u.reshape(3, -1)[:, cells], node_rho.reshape(-1)[cells])
    b.set_rho_u()
    a.step(10)
    b.step(10)
    assert np.array_equal(a.f(), b.f())
    a.close()
    b.close()


def test_sparse_nodes_validation():
    P = _P()
    g = P.Lattice(4, 4, 4, "D3Q19", "SRT", "FP32", "FP32", "AB", tau=0.8)
    u = np.zeros((3, 2), dtype=np.float32)
    with pytest.raises(P.LBMError):            # no flags yet
        g.set_nodes(np.array([1, 2]), u)
    g.set_geometry(np.zeros((4, 4, 4), dtype=np.uint8))
    with pytest.raises(P.LBMError):            # listed twice
        g.set_nodes(np.array([2, 2]), u)
    with pytest.raises(P.LBMError):            # out of range
        g.set_nodes(np.array([1, 64]), u)
    g.set_nodes(np.array([1, 2]), u)
    g.close()
