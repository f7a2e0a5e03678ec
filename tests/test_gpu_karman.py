"""Karman channel (Sec. 4.3 in its 3-D channel form), downscaled to
256 x 64 x 16: equilibrium inflow, zero-gradient outflow, free-slip side
walls, a solid cylinder along z.  The GPU FP64 tier must stay within 1e-12
of the FP64 definition and equal the ordered FP64 oracle bit for bit over
2000 steps; FP16C and FP32 storage must equal the ordered FP32 oracle bit
for bit."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NX, NY, NZ, R, TAU = 256, 64, 16, 6, 0.5288


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


@pytest.fixture(scope="module")
def channel():
    flags, node_u, node_rho = W.karman_channel(NX, NY, NZ, radius=R, cx=64, cy=32)
    fields = W.karman_initial_fields(NX, NY, NZ, x_perturb=64)
    return flags, node_u, node_rho, fields


def _gpu(channel, storage, arith, steps):
    import paper_2112_08926_gb300 as P
    flags, node_u, node_rho, fields = channel
    g = P.Lattice(NX, NY, NZ, "D3Q19", "SRT", storage, arith, "AB", tau=TAU)
    g.set_geometry(flags, node_u, node_rho)
    g.set_rho_u(*fields)
    g.step(steps)
    out = g.f(), g.rho_u()
    g.close()
    return out


def _oracle(channel, arith, storage, steps):
    flags, node_u, node_rho, fields = channel
    o = oracle.Lattice(NX, NY, NZ, "D3Q19", "SRT", arith, storage, tau=TAU)
    o.set_geometry(flags, node_u, node_rho)
    o.set_rho_u(*fields)
    o.step(steps)
    return o.f(), o.rho_u()


def test_fp64_tier_on_channel(channel):
    f, (rho, ux, uy, uz) = _gpu(channel, "FP64", "FP64", 2000)
    fd, (rd, uxd, uyd, uzd) = _oracle(channel, "DEF64", "FP64", 2000)
    u, ud = np.stack([ux, uy, uz]), np.stack([uxd, uyd, uzd])
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-12
    assert np.linalg.norm(f - fd) / np.linalg.norm(fd) < 1e-12
    fo, _ = _oracle(channel, "ORD64", "FP64", 2000)
    assert np.array_equal(f, fo)


@pytest.mark.parametrize("storage", ["FP16C", "FP32"])
def test_fp32_arithmetic_tiers_on_channel(channel, storage):
    f, _ = _gpu(channel, storage, "FP32", 300)
    fo, _ = _oracle(channel, "ORD32", storage, 300)
    assert np.array_equal(f, fo)
