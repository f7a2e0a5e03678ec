"""Pins of the oracle's lattice Boltzmann step against closed forms, invariants
and values printed in the paper.

A plausible mistake in the oracle (a dropped term, a wrong sign or index, a
transposed weight, a wrong relaxation factor) changes at least one of:
equilibrium moments, Table 1's bound, conservation, the Guo momentum input,
the exact TRT / magic-tau Poiseuille parabola, the Poiseuille start-up series,
the Taylor-Green decay rate (which fixes nu = (tau - 1/2)/3), Couette flow, or
the uniform open channel.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from conftest import golden

VELSETS = ["D2Q9", "D3Q19", "D3Q27"]


@pytest.mark.parametrize("vs", VELSETS)
@pytest.mark.parametrize("arith,tol", [("DEF64", 2e-15), ("ORD64", 2e-15), ("ORD32", 2e-6)])
def test_equilibrium_moments(vs, arith, tol):
    """Sec. 2.2: sum_i f^eq-s = rho - 1, sum_i c_i f^eq-s = rho u and
    sum_i c_i c_i f^eq-s = rho u u + (rho - 1) c^2 I (weights moved out by the shift)."""
    c, w = oracle.velset(vs)
    d = 2 if vs == "D2Q9" else 3
    rng = np.random.default_rng(5)
    for _ in range(20):
        rho = 1 + 0.2 * rng.uniform(-1, 1)
        u = 0.1 * rng.uniform(-1, 1, 3)
        if d == 2:
            u[2] = 0
        f = oracle.equilibrium(vs, arith, rho, u)
        assert abs(f.sum() - (rho - 1)) <= tol
        assert np.allclose(c.T @ f, rho * u, rtol=0, atol=tol)
        P = (c[:, :, None] * c[:, None, :] * f[:, None, None]).sum(0)
        expect = rho * np.outer(u, u) + (rho - 1) / 3 * np.eye(3)
        if d == 2:
            expect[2, 2] = 0
        assert np.allclose(P, expect, rtol=0, atol=5 * tol)


def test_weights_sum_and_isotropy():
    for vs in VELSETS:
        c, w = oracle.velset(vs)
        assert abs(w.sum() - 1) < 1e-15
        d = 2 if vs == "D2Q9" else 3
        M2 = (w[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0)
        assert np.allclose(M2[:d, :d], np.eye(d) / 3, atol=1e-15)
        for i in range(1, len(w), 2):        # 2k-1 and 2k are opposite
            assert np.array_equal(c[i], -c[i + 1])


@pytest.mark.parametrize("row", golden("delta_table1.txt"), ids=lambda r: r[0])
def test_table1_delta(row):
    """Table 1: the maxima of |f^eq| / rho and |f^eq-s| / rho over the rest
    state and u_j = c c_j/|c_j| (c = 1/sqrt(3)) round up to the printed
    values (the oracle's equilibrium is the shifted one; f^eq = f^eq-s + w)."""
    vs, printed, printed_s = row[0], float(row[1]), float(row[2])
    c, w = oracle.velset(vs)
    best = best_s = 0.0
    us = [np.zeros(3)] + [c[j] / np.linalg.norm(c[j]) / math.sqrt(3) for j in range(1, len(w))]
    for u in us:
        feq_s = oracle.equilibrium(vs, "DEF64", 1.0, u)
        best_s = max(best_s, np.abs(feq_s).max())
        best = max(best, np.abs(feq_s + w).max())
    for exact, shown in ((best, printed), (best_s, printed_s)):
        assert shown - 0.01 < exact <= shown
        assert math.ceil(exact * 100 - 1e-9) / 100 == pytest.approx(shown)
    # the unshifted bound comes from the rest state: the rest population w_0
    assert best == pytest.approx(w[0], abs=1e-15)


@pytest.mark.parametrize("vs", VELSETS)
@pytest.mark.parametrize("coll", ["SRT", "TRT"])
@pytest.mark.parametrize("arith", ["DEF64", "ORD64"])
def test_collision_conserves_mass_and_momentum(vs, coll, arith):
    c, w = oracle.velset(vs)
    q = len(w)
    rng = np.random.default_rng(2)
    L = oracle.Lattice(1, 1, 1, vs, coll, arith, "FP64", tau=0.63, trt_lambda=0.25)
    for _ in range(5):
        f = rng.uniform(-0.02, 0.02, (q, 1, 1, 1))
        L.set_f(f)
        L.step(1)
        g = L.f().reshape(q)
        assert abs(g.sum() - f.sum()) < 1e-15
        assert np.allclose(c.T @ g, c.T @ f.reshape(q), rtol=0, atol=1e-16)
        assert not np.allclose(g, f.reshape(q))     # something did relax


@pytest.mark.parametrize("coll", ["SRT", "TRT"])
def test_guo_force_adds_F_per_step(coll):
    F = (1e-5, -2e-5, 3e-5)
    L = oracle.Lattice(6, 5, 4, "D3Q19", coll, "DEF64", "FP64", tau=0.7, force=F)
    L.set_rho_u(*W.random_fields((4, 5, 6), 3))
    L.step(1)

    def momentum():
        r, ux, uy, uz = L.rho_u()
        return np.array([(r * ux).sum(), (r * uy).sum(), (r * uz).sum()])

    p0 = momentum()
    L.step(10)
    assert np.allclose((momentum() - p0) / (6 * 5 * 4 * 10), F, rtol=1e-10, atol=0)


@pytest.mark.parametrize("vs,shape", [("D2Q9", (1, 12, 14)), ("D3Q19", (6, 7, 9)), ("D3Q27", (5, 6, 7))])
def test_periodic_and_bounce_back_mass_conservation(vs, shape):
    nz, ny, nx = shape
    rng = np.random.default_rng(9)
    flags = np.where(rng.uniform(size=shape) < 0.1, W.WALL, 0).astype(np.uint8)
    L = oracle.Lattice(nx, ny, nz, vs, "SRT", "DEF64", "FP64", tau=0.6)
    L.set_geometry(flags)
    L.set_rho_u(*W.random_fields(shape, 4))
    m0, _ = L.reduce()
    L.step(300)
    m1, _ = L.reduce()
    assert abs(m1 / m0 - 1) < 1e-13


def _startup_series(F, nu, H, eta, t, terms=400):
    u = F / (2 * nu) * eta * (H - eta)
    for n in range(1, 2 * terms, 2):
        u -= 4 * F * H * H / (nu * math.pi ** 3 * n ** 3) * np.sin(n * math.pi * eta / H) * \
            math.exp(-nu * n * n * math.pi ** 2 * t / (H * H))
    return u


def test_poiseuille_plate_startup_series():
    """Plane Poiseuille flow from rest, walls half-way at y = 0.5 and ny - 1.5:
    u(eta, t) = F eta (H - eta)/(2 nu) - sum_odd 4 F H^2/(nu pi^3 n^3) sin(n pi eta/H) e^{-nu n^2 pi^2 t/H^2}.
    The 64-cell plate of the 8x64x8 workload (x and z periodic, so one column
    carries the same flow); BGK bounce-back slip keeps the error near 1e-4."""
    tau, F, ny, T = 0.8, 1e-6, 64, 10000
    L = oracle.Lattice(1, ny, 1, "D3Q19", "SRT", "DEF64", "FP64", tau=tau, force=(F, 0, 0))
    L.set_geometry(W.poiseuille_plate(1, ny, 1))
    L.set_rho_u()
    L.step(T)
    _, ux, _, _ = L.rho_u()
    nu, H = (tau - 0.5) / 3, ny - 2
    eta = np.arange(1, ny - 1) - 0.5
    ref = _startup_series(F, nu, H, eta, T)
    err = np.sqrt(((ux[0, 1:-1, 0] - ref) ** 2).sum() / (ref ** 2).sum())
    assert err < 3e-4


@pytest.mark.parametrize("coll,tau", [("TRT", 0.8), ("SRT", 0.5 + math.sqrt(3) / 4)])
def test_poiseuille_exact_at_magic_parameter(coll, tau):
    """With Lambda = (tau+ - 1/2)(tau- - 1/2) = 3/16, half-way bounce-back sits
    exactly mid-grid and the steady force-driven profile is the exact parabola."""
    F, ny = 1e-6, 34
    L = oracle.Lattice(1, ny, 1, "D3Q19", coll, "DEF64", "FP64", tau=tau, trt_lambda=3 / 16, force=(F, 0, 0))
    L.set_geometry(W.poiseuille_plate(1, ny, 1))
    L.set_rho_u()
    L.step(60000)
    _, ux, _, _ = L.rho_u()
    nu, H = (tau - 0.5) / 3, ny - 2
    eta = np.arange(1, ny - 1) - 0.5
    ref = F / (2 * nu) * eta * (H - eta)
    assert np.abs(ux[0, 1:-1, 0] - ref).max() / ref.max() < 1e-11


def test_couette_linear_profile():
    """Moving bounce-back (Ladd, rho_w = 1): steady shear flow is linear."""
    U, ny = 0.01, 18
    flags, node_u = W.couette_plate(1, ny, 1, U)
    for tau in (0.6, 1.0, 1.7):
        L = oracle.Lattice(1, ny, 1, "D3Q19", "SRT", "DEF64", "FP64", tau=tau)
        L.set_geometry(flags, node_u)
        L.set_rho_u()
        L.step(40000)
        _, ux, _, _ = L.rho_u()
        eta = np.arange(1, ny - 1) - 0.5
        assert np.abs(ux[0, 1:-1, 0] - U * eta / (ny - 2)).max() / U < 1e-6


@pytest.mark.parametrize("vs,nz", [("D2Q9", 1), ("D3Q19", 2), ("D3Q27", 2)])
def test_taylor_green_decay_rate(vs, nz):
    """Sec. 4.2: E(t) = E0 exp(-4 nu k^2 t) with nu = (tau - 1/2)/3."""
    n, tau, u0, T = 64, 0.8, 0.01, 400
    L = oracle.Lattice(n, n, nz, vs, "SRT", "DEF64", "FP64", tau=tau)
    L.set_rho_u(*W.taylor_green_extruded(n, u0, nz=nz))
    _, E0 = L.reduce()
    L.step(T)
    _, E1 = L.reduce()
    nu, k = (tau - 0.5) / 3, 2 * math.pi / n
    rate = -math.log(E1 / E0) / T
    assert abs(rate / (4 * nu * k * k) - 1) < 2e-3


def test_open_channel_stays_uniform():
    """Equilibrium inflow, zero-gradient outflow and free-slip walls leave a
    uniform stream uniform."""
    nx, ny, nz = 20, 8, 3
    u = float(np.float32(0.05))
    flags, node_u, node_rho = W.karman_channel(nx, ny, nz, radius=0, cx=-100, cy=-100, u_in=u)
    L = oracle.Lattice(nx, ny, nz, "D3Q19", "SRT", "DEF64", "FP64", tau=0.6)
    L.set_geometry(flags, node_u, node_rho)
    L.set_rho_u(np.ones((nz, ny, nx)), np.full((nz, ny, nx), u), None, None)
    L.step(200)
    r, ux, uy, uz = L.rho_u()
    fl = flags == 0
    assert np.abs(ux[fl] - u).max() < 1e-14
    assert np.abs(r[fl] - 1).max() < 1e-14
    assert np.abs(uy[fl]).max() < 1e-14


def test_freeslip_is_mirror_and_bounce_back_is_reversal():
    """One streaming step next to a free-slip wall (normal y) returns the
    mirrored population of the neighbouring column; next to a plain wall the
    cell's own opposite population."""
    nx, ny, nz = 4, 3, 1
    c, w = oracle.velset("D2Q9")
    for kind in ("freeslip", "wall"):
        flags = np.zeros((nz, ny, nx), np.uint8)
        flags[:, 0, :] = W.freeslip(1) if kind == "freeslip" else W.WALL
        L = oracle.Lattice(nx, ny, nz, "D2Q9", "SRT", "DEF64", "FP64", tau=1.0)
        L.set_geometry(flags)
        rng = np.random.default_rng(1)
        f = rng.uniform(-0.01, 0.01, (9, nz, ny, nx))
        f[:, flags != 0] = 0
        L.set_f(f)
        g = L.f()
        x, y = 1, 1
        for i in range(9):
            if c[i][1] != 1:          # only populations coming out of the y = 0 wall
                continue
            if kind == "freeslip":
                j = [k for k in range(9) if c[k][0] == c[i][0] and c[k][1] == -c[i][1]][0]
                assert g[i, 0, y, x] == f[j, 0, y, x - c[i][0]]
            else:
                j = [k for k in range(9) if np.array_equal(c[k], -c[i])][0]
                assert g[i, 0, y, x] == f[j, 0, y, x]


@pytest.mark.parametrize("vs", VELSETS)
@pytest.mark.parametrize("coll", ["SRT", "TRT"])
def test_ordered_modes_track_definition(vs, coll):
    """The paper's operation order changes results only by rounding."""
    shape = (1, 9, 11) if vs == "D2Q9" else (5, 6, 7)
    flags, node_u, node_rho = W.random_geometry(shape, 12)
    out = {}
    for arith, storage in (("DEF64", "FP64"), ("ORD64", "FP64"), ("ORD32", "FP32")):
        L = oracle.Lattice(shape[2], shape[1], shape[0], vs, coll, arith, storage, tau=0.7,
                           force=(1e-5, 2e-5, 0 if vs == "D2Q9" else -1e-5))
        L.set_geometry(flags, node_u, node_rho)
        L.set_rho_u(*W.random_fields(shape, 13))
        L.step(40)
        out[arith] = L.f()
    ref = out["DEF64"]
    scale = np.abs(ref).max()
    assert np.abs(out["ORD64"] - ref).max() / scale < 1e-13
    assert np.abs(out["ORD32"] - ref).max() / scale < 2e-5


@pytest.mark.parametrize("fmt", oracle.CODEC_FORMATS)
def test_sixteen_bit_storage_holds_codec_values(fmt):
    """In ORD32 mode every stored population is a decoded code of the format."""
    shape = (3, 4, 5)
    L = oracle.Lattice(5, 4, 3, "D3Q19", "SRT", "ORD32", fmt, tau=0.8)
    L.set_rho_u(*W.random_fields(shape, 1))
    L.step(3)
    f = L.f().astype(np.float32).reshape(-1)
    assert np.array_equal(oracle.decode(fmt, oracle.encode(fmt, f)), f)


# ---------------------------------------------------------------- no DDF shifting
@pytest.mark.parametrize("vs,coll", [("D2Q9", "SRT"), ("D3Q19", "TRT"), ("D3Q27", "SRT")])
def test_unshifted_lattice_is_shifted_lattice_plus_weights(vs, coll):
    """Appendix, with and without DDF-shifting: the two formulations are the
    same LBM, so in FP64 the unshifted populations equal the shifted ones plus
    w_i (up to rounding), on every boundary kind, with forcing."""
    shape = (1, 9, 11) if vs == "D2Q9" else (5, 6, 7)
    flags, node_u, node_rho = W.random_geometry(shape, 31)
    c, w = oracle.velset(vs)
    res = {}
    for shifting in (True, False):
        L = oracle.Lattice(shape[2], shape[1], shape[0], vs, coll, "DEF64", "FP64", tau=0.7,
                           force=(1e-5, -2e-5, 0 if vs == "D2Q9" else 1e-5), shifting=shifting)
        L.set_geometry(flags, node_u, node_rho)
        L.set_rho_u(*W.random_fields(shape, 32))
        L.step(30)
        res[shifting] = (L.f(), L.rho_u())
    fs, fu = res[True][0], res[False][0]
    fluid = (flags & W.WALL) == 0
    diff = (fu - w.reshape(-1, 1, 1, 1) - fs)[:, fluid]
    assert np.abs(diff).max() < 1e-13
    for a, b in zip(res[True][1], res[False][1]):
        assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("vs", ["D2Q9", "D3Q19", "D3Q27"])
def test_unshifted_equilibrium_moments(vs):
    """Plain equilibrium (appendix, without shifting): sum f = rho, sum c f = rho u."""
    c, w = oracle.velset(vs)
    rng = np.random.default_rng(8)
    for _ in range(5):
        rho = 1 + 0.1 * rng.uniform(-1, 1)
        u = 0.1 * rng.uniform(-1, 1, 3)
        if vs == "D2Q9":
            u[2] = 0.0
        L = oracle.Lattice(1, 1, 1, vs, "SRT", "DEF64", "FP64", tau=0.8, shifting=False)
        L.set_rho_u(np.array([rho]), np.array([u[0]]), np.array([u[1]]), np.array([u[2]]))
        f = L.f().reshape(-1)
        assert abs(f.sum() - rho) < 1e-14
        assert np.abs(c.T @ f - rho * u).max() < 1e-14
        r, ux, uy, uz = L.rho_u()
        assert abs(r.item() - rho) < 1e-14


def test_unshifted_lattice_starts_at_rest():
    L = oracle.Lattice(3, 4, 5, "D3Q19", "SRT", "DEF64", "FP64", tau=0.8, shifting=False)
    r, ux, uy, uz = L.rho_u()
    assert np.abs(r - 1.0).max() < 1e-15 and not ux.any() and not uy.any() and not uz.any()
    # unshifted 16-bit storage cannot even hold rest exactly (w_i are not FP16S values)
    L = oracle.Lattice(3, 4, 5, "D3Q19", "SRT", "ORD32", "FP16S", tau=0.8, shifting=False)
    r = L.rho_u()[0]
    assert 0 < np.abs(r - 1.0).max() < 1e-3


def test_outflow_needs_a_fluid_upstream_cell():
    flags = np.zeros((2, 3, 4), dtype=np.uint8)
    flags[1, 1, 2] = W.OUTFLOW
    flags[1, 1, 1] = W.WALL
    L = oracle.Lattice(4, 3, 2, "D3Q19", "SRT", "DEF64", "FP64")
    with pytest.raises(ValueError):
        L.set_geometry(flags)
    flags[1, 1, 1] = 0
    L.set_geometry(flags)


def test_shifting_wins_back_sixteen_bit_accuracy():
    """Sec. 2.2 / 4.2: with FP16 storage the unshifted populations (f near w)
    lose the small deviations that carry the flow; the shifted ones keep
    them.  2-D Taylor-Green vortex, velocity error against FP64 after 200 steps."""
    n, u0, tau = 32, 0.01, 0.8
    fields = W.taylor_green_extruded(n, u0, nz=1)
    ref = oracle.Lattice(n, n, 1, "D2Q9", "SRT", "DEF64", "FP64", tau=tau)
    ref.set_rho_u(*fields)
    ref.step(200)
    uref = np.stack(ref.rho_u()[1:3])
    err = {}
    for shifting in (True, False):
        L = oracle.Lattice(n, n, 1, "D2Q9", "SRT", "ORD32", "FP16", tau=tau, shifting=shifting)
        L.set_rho_u(*fields)
        L.step(200)
        u = np.stack(L.rho_u()[1:3])
        err[shifting] = np.linalg.norm(u - uref) / np.linalg.norm(uref)
    assert err[True] < 0.05
    assert err[False] > 5 * err[True]


# ---------------------------------------------------------------- MRT (D3Q19)
def test_mrt_basis_is_the_orthogonal_polynomial_basis():
    """d'Humieres et al. (2002) D3Q19 moments: rows are the stated velocity
    polynomials, mutually orthogonal; density and momentum rows are exact."""
    M = oracle.mrt_basis()
    c, w = oracle.velset("D3Q19")
    c2 = (c * c).sum(1)
    assert np.array_equal(M[0], np.ones(19))
    assert np.array_equal(M[1], 19 * c2 - 30)
    assert np.array_equal(M[3], c[:, 0]) and np.array_equal(M[5], c[:, 1]) and np.array_equal(M[7], c[:, 2])
    assert np.array_equal(M[13], c[:, 0] * c[:, 1])
    G = M @ M.T
    assert np.array_equal(G, np.diag(np.diag(G)))
    # equilibrium energy moment: e_eq = rho (-11 + 19 u.u) for the second-order equilibrium
    rho, u = 1.03, np.array([0.05, -0.02, 0.03])
    feq = oracle.equilibrium("D3Q19", "DEF64", rho, u) + w
    assert abs(M[1] @ feq - rho * (-11 + 19 * u @ u)) < 1e-13


def _mrt_lattice(arith, storage, shape, seed, force=(0.0, 0.0, 0.0), tau=0.8):
    geo = W.random_geometry(shape, seed)
    o = oracle.Lattice(shape[2], shape[1], shape[0], "D3Q19", "MRT", arith, storage, tau=tau, force=force)
    o.set_geometry(*geo)
    o.set_rho_u(*W.random_fields(shape, seed + 1))
    return o


def test_mrt_ordered_modes_track_matrix_definition():
    """DEF64 applies M^-1 from a general matrix inverse; ORD64/ORD32 use the
    orthogonal form sum_k M_ki x_k / |M_k|^2 in a fixed order."""
    shape = (5, 6, 7)
    out = {}
    for arith, storage in (("DEF64", "FP64"), ("ORD64", "FP64"), ("ORD32", "FP32")):
        o = _mrt_lattice(arith, storage, shape, 71, force=(1e-5, -2e-5, 1e-5))
        o.step(30)
        out[arith] = o.f()
    scale = np.abs(out["DEF64"]).max()
    assert np.abs(out["ORD64"] - out["DEF64"]).max() / scale < 1e-13
    assert np.abs(out["ORD32"] - out["DEF64"]).max() / scale < 2e-5


def test_mrt_conserves_mass_and_momentum():
    n = 6
    o = oracle.Lattice(n, n, n, "D3Q19", "MRT", "DEF64", "FP64", tau=0.7)
    o.set_rho_u(*W.random_fields((n, n, n), 73))
    r0, ux0, uy0, uz0 = o.rho_u()
    j0 = [(r0 * u).sum() for u in (ux0, uy0, uz0)]
    o.step(50)
    r1, ux1, uy1, uz1 = o.rho_u()
    assert abs(r1.sum() / r0.sum() - 1) < 1e-13
    for a, u in zip(j0, (ux1, uy1, uz1)):
        assert abs((r1 * u).sum() - a) < 1e-12


def test_mrt_viscosity_from_taylor_green_decay():
    """The shear moments relax with omega = 1/tau, so the vortex decays with
    nu = (tau - 1/2)/3 as with SRT (Sec. 4.2 closed form)."""
    n, u0, tau, T = 32, 0.01, 0.9, 400
    o = oracle.Lattice(n, n, 1, "D3Q19", "MRT", "DEF64", "FP64", tau=tau)
    o.set_rho_u(*W.taylor_green_extruded(n, u0, nz=1))
    e0 = o.reduce()[1]
    o.step(T)
    e1 = o.reduce()[1]
    nu, k = (tau - 0.5) / 3, 2 * math.pi / n
    # within the discretisation error at n = 32 (SRT itself: 2e-3)
    assert abs(np.log(e1 / e0) / (-4 * nu * k * k * T) - 1) < 1e-2


def test_mrt_poiseuille_curvature():
    """Steady plane Poiseuille under MRT: the profile's curvature is -F/nu."""
    nx, ny, nz, tau, F = 1, 34, 1, 0.8, 1e-6
    o = oracle.Lattice(nx, ny, nz, "D3Q19", "MRT", "DEF64", "FP64", tau=tau, force=(F, 0, 0))
    o.set_geometry(W.poiseuille_plate(nx, ny, nz))
    o.set_rho_u()
    o.step(40000)
    ux = o.rho_u()[1][0, 1:-1, 0]
    y = np.arange(1, ny - 1, dtype=float)
    a = np.polyfit(y, ux, 2)[0]
    nu = (tau - 0.5) / 3
    assert abs(2 * a / (-F / nu) - 1) < 1e-6


def test_oracle_result_does_not_depend_on_thread_count():
    """The parallel loops are over independent cells: one thread and all
    threads give the same populations bit for bit (the timing legs of the
    benchmark change the thread count)."""
    shape = (4, 5, 6)
    fields = W.random_fields(shape, 91)
    geo = W.random_geometry(shape, 92)
    out = []
    n0 = oracle.threads()
    try:
        for t in (1, n0):
            oracle.set_threads(t)
            o = oracle.Lattice(6, 5, 4, "D3Q19", "TRT", "ORD32", "FP16S", tau=0.7)
            o.set_geometry(*geo)
            o.set_rho_u(*fields)
            o.step(7)
            out.append(o.f())
    finally:
        oracle.set_threads(n0)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("arith", ["ORD32", "ORD64"])
@pytest.mark.parametrize("with_force", [False, True])
def test_ordered_velocity_is_the_correctly_rounded_quotient(arith, with_force):
    """Sec. 2.2 writes each velocity component as the momentum sum divided by
    rho (u_x = (f1 - f2 + ...)/rho); the ordered modes take one IEEE division
    per component.  A one-cell periodic lattice streams onto itself, so
    rho and j are the sums of the populations set here.  They are chosen on a
    coarse dyadic grid, which makes rho = sum f + 1 and j (+ F/2) exact in
    either precision; IEEE division is then the exactly rounded quotient
    (for FP32 operands the FP64 quotient rounded once more to FP32 is that
    same value).  A reciprocal multiplied into j differs from it in many of
    these cells, which the test also checks, so it tells the two apart."""
    rng = np.random.default_rng(20211216)
    dt = np.float32 if arith == "ORD32" else np.float64
    n_recip_differs = 0
    for _ in range(200):
        F = (rng.integers(-64, 65) * 2.0 ** -14, 0.0, 0.0) if with_force else (0.0, 0.0, 0.0)
        L = oracle.Lattice(1, 1, 1, "D3Q19", "SRT", arith, "FP32" if arith == "ORD32" else "FP64",
                           tau=0.8, force=F)
        f = np.zeros(19)
        f[1:] = rng.integers(-2048, 2049, 18) * 2.0 ** -16
        L.set_f(f)
        rho, ux, uy, uz = (float(a.ravel()[0]) for a in L.rho_u())
        c, _ = oracle.velset("D3Q19")
        assert rho == 1.0 + f.sum()                       # exact on this grid
        for a, got in enumerate((ux, uy, uz)):
            j = float(c[:, a] @ f) + 0.5 * F[a]           # exact on this grid
            quotient = float(dt(np.float64(j) / np.float64(rho)))
            assert got == quotient
            if float(dt(dt(j) * (dt(1) / dt(rho)))) != quotient:
                n_recip_differs += 1
    assert n_recip_differs > 10
