"""Accuracy of every storage tier on the paper's test systems.

Each tier's velocity error is stated as a number (the bounds below are the
measured values rounded up):
  - plane Poiseuille 8x64x8 (tau 0.8, body force 1e-6, 10,000 steps):
    relative L2 of u_x against the FP64 CPU oracle and against the analytic
    start-up series (Sec. 4.1 error norm);
  - 2-D Taylor-Green vortex extruded along z, 256^3 (u0 0.05, tau 0.53,
    2000 steps): E/E0 against the closed form exp(-4 nu k^2 t) (Sec. 4.2) and
    the velocity L2 against the GPU FP64 tier (itself within 1e-12 of the
    FP64 oracle on smaller lattices);
  - D2Q9 Taylor-Green, L = 256, u0 = 0.25, tau = 1 (Sec. 4.2): the kinetic
    energy stops decaying at a plateau within a few decades of the square of
    the storage format's truncation error (Table 2 epsilon).
"""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle
import workloads as W
from conftest import golden

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TIERS = [("FP64", "FP64"), ("FP64", "FP32"), ("FP32", "FP64"), ("FP32", "FP32"), ("FP32", "FP16"),
         ("FP32", "FP16S"), ("FP32", "FP16C"), ("FP32", "P16_0S"), ("FP32", "P16_1S"), ("FP32", "P16_2C"),
         ("FP32", "P16_0"), ("FP32", "P16_1")]

# relative L2 bounds, about 1.5x the measured values: (vs FP64 reference, vs
# analytic solution).  The tiers whose populations cannot resolve the force
# increment near rest do not move at all: their error is the whole profile,
# held to [0.95, 1.001] instead.
POISEUILLE_BOUND = {
    "FP64/FP64": (1e-12, 2.3e-4), "FP64/FP32": (2e-6, 2.3e-4), "FP32/FP64": (2.1e-5, 2.5e-4),
    "FP32/FP32": (2.1e-5, 2.5e-4), "FP32/FP16": (0.37, 0.37), "FP32/FP16S": (0.37, 0.37),
    "FP32/FP16C": (0.19, 0.19), "FP32/P16_1S": (0.11, 0.11), "FP32/P16_2C": (0.55, 0.55),
}
POISEUILLE_STUCK = ("FP32/P16_0S", "FP32/P16_0", "FP32/P16_1")
TG_BOUND = {   # (|E/E0 / closed form - 1|, L2 of u vs FP64 tier), about 1.5x the measured values
    "FP64/FP64": (4e-4, 1e-14), "FP64/FP32": (4e-4, 1.1e-7), "FP32/FP64": (4.8e-4, 4.2e-5),
    "FP32/FP32": (4.8e-4, 4.2e-5), "FP32/FP16": (2.7e-4, 8.8e-4), "FP32/FP16S": (1.1e-4, 6.8e-4),
    "FP32/FP16C": (6.6e-4, 4.8e-4), "FP32/P16_0S": (7.7e-4, 2.5e-4), "FP32/P16_1S": (7.1e-4, 2.7e-4),
    "FP32/P16_2C": (3.1e-4, 6.6e-4), "FP32/P16_0": (2.1e-3, 2.2e-2), "FP32/P16_1": (1.5e-4, 2.4e-3),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _pkg():
    import paper_2112_08926_gb300 as P
    return P


def _startup_series(F, nu, H, eta, t, terms=400):
    u = F / (2 * nu) * eta * (H - eta)
    for n in range(1, 2 * terms, 2):
        u -= 4 * F * H * H / (nu * math.pi ** 3 * n ** 3) * np.sin(n * math.pi * eta / H) * \
            math.exp(-nu * n * n * math.pi ** 2 * t / (H * H))
    return u


def test_poiseuille_error_per_tier():
    P = _pkg()
    nx, ny, nz, tau, F, T = 8, 64, 8, 0.8, 1e-6, 10000
    flags = W.poiseuille_plate(nx, ny, nz)
    o = oracle.Lattice(nx, ny, nz, "D3Q19", "SRT", "DEF64", "FP64", tau=tau, force=(F, 0, 0))
    o.set_geometry(flags)
    o.set_rho_u()
    o.step(T)
    ref = o.rho_u()[1][:, 1:-1, :]
    nu, H = (tau - 0.5) / 3, ny - 2
    eta = np.arange(1, ny - 1) - 0.5
    ana = _startup_series(F, nu, H, eta, T)[None, :, None] * np.ones_like(ref)
    lines, errs = [], {}
    for arith, storage in TIERS:
        g = P.Lattice(nx, ny, nz, "D3Q19", "SRT", storage, arith, "AB", tau=tau, force=(F, 0, 0))
        g.set_geometry(flags)
        g.set_rho_u()
        g.step(T)
        ux = g.rho_u()[1][:, 1:-1, :]
        g.close()
        e_ref = np.linalg.norm(ux - ref) / np.linalg.norm(ref)
        e_ana = np.linalg.norm(ux - ana) / np.linalg.norm(ana)
        name = f"{arith}/{storage}"
        lines.append(f"{name:12s} L2 vs FP64 oracle {e_ref:.3e}   vs analytic {e_ana:.3e}")
        errs[name] = (e_ref, e_ana)
    print("\nPoiseuille 8x64x8, 10000 steps\n" + "\n".join(lines))
    for name, (e_ref, e_ana) in errs.items():
        if name in POISEUILLE_STUCK:
            assert 0.95 <= e_ref <= 1.001 and 0.95 <= e_ana <= 1.001, (name, e_ref, e_ana)
            continue
        b_ref, b_ana = POISEUILLE_BOUND[name]
        assert e_ref <= b_ref and e_ana <= b_ana, (name, e_ref, e_ana)


def test_taylor_green_error_per_tier():
    P = _pkg()
    n, u0, tau, T = 256, 0.05, 0.53, 2000
    fields = W.taylor_green_extruded(n, u0)
    nu, k = (tau - 0.5) / 3, 2 * math.pi / n
    closed = math.exp(-4 * nu * k * k * T)
    ref_u = None
    lines, errs = [], {}
    for arith, storage in TIERS:
        g = P.Lattice(n, n, n, "D3Q19", "SRT", storage, arith, "AB", tau=tau)
        g.set_rho_u(*fields)
        _, e0 = g.reduce()
        g.step(T)
        _, e1 = g.reduce()
        _, ux, uy, _ = g.rho_u()
        g.close()
        u = np.stack([ux, uy])
        if ref_u is None:
            ref_u = u
        e_E = abs(e1 / e0 / closed - 1)
        e_u = np.linalg.norm(u - ref_u) / np.linalg.norm(ref_u)
        name = f"{arith}/{storage}"
        lines.append(f"{name:12s} |E/E0 / closed form - 1| {e_E:.3e}   L2 of u vs FP64 tier {e_u:.3e}")
        errs[name] = (e_E, e_u)
    print(f"\nTaylor-Green 256^3 extruded, {T} steps, closed-form E/E0 = {closed:.6f}\n" + "\n".join(lines))
    for name, (e_E, e_u) in errs.items():
        b_E, b_u = TG_BOUND[name]
        assert e_E <= b_E and e_u <= b_u, (name, e_E, e_u)


def _table2_eps():
    eps = {"FP32": 2.0 ** -23, "FP64": 2.0 ** -52}
    for row in golden("format_table2.txt"):
        eps[row[0]] = float(row[1])
    return eps


def test_taylor_green_2d_energy_plateau():
    """Sec. 4.2: E/E0 follows exp(-4 nu k^2 t) until it stalls at a plateau;
    for the IEEE-like formats the plateau sits near the square of the storage
    format's truncation error (Table 2)."""
    P = _pkg()
    eps = _table2_eps()
    L, u0, tau = 256, 0.25, 1.0
    nu, k = (tau - 0.5) / 3, 2 * math.pi / L
    rate = 4 * nu * k * k
    fields = W.taylor_green_extruded(L, u0, nz=1)
    lines, plateaus, firsts = [], {}, {}
    for arith, storage in TIERS:
        g = P.Lattice(L, L, 1, "D2Q9", "SRT", storage, arith, "AB", tau=tau)
        g.set_rho_u(*fields)
        _, e0 = g.reduce()
        hist, prev = [], e0
        for _ in range(250):
            g.step(1000)
            _, e = g.reduce()
            hist.append(e / e0)
            if e > 0.9 * prev:      # decay has stopped
                break
            prev = e
        g.close()
        name = f"{arith}/{storage}"
        plateaus[name] = hist[-1]
        first = abs(hist[0] / math.exp(-rate * 1000) - 1)
        lines.append(f"{name:12s} plateau E/E0 {hist[-1]:.3e} at {1000 * len(hist):6d} steps   "
                     f"eps^2 {eps.get(storage, math.nan) ** 2:.2e}   first-1000-step decay vs closed form {first:.1e}")
        firsts[name] = first
    print("\nD2Q9 Taylor-Green L=256 u0=0.25 tau=1\n" + "\n".join(lines))
    for name, first in firsts.items():
        assert first < 0.05, (name, first)
    # the plateau sits within a few decades of eps^2: about 1e-2 eps^2 for
    # formats whose range fits the shifted populations (FP64, FP32, FP16S),
    # about eps^2 for FP16, FP16C and the scaled posits
    for name in ("FP64/FP64", "FP32/FP32", "FP32/FP16", "FP32/FP16S", "FP32/FP16C", "FP32/P16_1S", "FP32/P16_2C"):
        e2 = eps[name.split("/")[1]] ** 2
        assert 1e-3 * e2 < plateaus[name] < 1e1 * e2, name
    # Sec. 4.2: P16_0S holds the populations outside its accurate interval
    assert plateaus["FP32/P16_0S"] > 1e2 * eps["P16_0S"] ** 2
    # Sec. 4.2: FP64 arithmetic with FP32 storage plateaus far below FP32 / FP32
    assert plateaus["FP64/FP32"] < 1e-2 * plateaus["FP32/FP32"]


def _energy_history(P, arith, storage, shifting, L=256, u0=0.25, tau=1.0):
    """E/E0 every 1000 steps until the decay stops (or E reaches 0)."""
    g = P.Lattice(L, L, 1, "D2Q9", "SRT", storage, arith, "AB", tau=tau, shifting=shifting)
    g.set_rho_u(*W.taylor_green_extruded(L, u0, nz=1))
    _, e0 = g.reduce()
    prev, hist = e0, []
    for _ in range(250):
        g.step(1000)
        _, e = g.reduce()
        hist.append(e / e0)
        if e > 0.9 * prev or e == 0.0:
            break
        prev = e
    g.close()
    return hist


def _tracked_depth(hist, L=256, tau=1.0, factor=1.5):
    """The lowest closed-form E/E0 = exp(-4 nu k^2 t) the run reproduces
    within a factor `factor` before it departs for good (plateau above, or
    decay to zero below): the smaller, the more accurate the run."""
    nu, k = (tau - 0.5) / 3, 2 * math.pi / L
    depth = 1.0
    for j, v in enumerate(hist):
        closed = math.exp(-4 * nu * k * k * 1000 * (j + 1))
        if not closed / factor < v < factor * closed:
            break
        depth = closed
    return depth


def test_taylor_green_2d_plateau_without_shifting():
    """Sec. 4.2 (dashed curves): without DDF shifting accuracy is lost in
    every format.  Accuracy here is how far the run follows the closed-form
    decay exp(-4 nu k^2 t): the lowest E/E0 reproduced within a factor 1.5.
    Unshifted runs depart earlier, either stalling higher or, where the small
    velocities are quantised away, decaying to rest; both count as the loss
    the paper describes.  The margins below are set under the measured ones."""
    P = _pkg()
    lines, res = [], {}
    for arith, storage in [("FP32", "FP32"), ("FP32", "FP16"), ("FP32", "FP16S"), ("FP32", "FP16C"),
                           ("FP32", "P16_1S"), ("FP32", "P16_2C")]:
        hs, hu = _energy_history(P, arith, storage, True), _energy_history(P, arith, storage, False)
        ds, du = _tracked_depth(hs), _tracked_depth(hu)
        res[storage] = (ds, du)
        lines.append(f"{arith}/{storage:7s} shifted: tracks down to {ds:.2e}, plateau {hs[-1]:.3e} "
                     f"({1000 * len(hs)} steps)   unshifted: tracks down to {du:.2e}, plateau {hu[-1]:.3e} "
                     f"({1000 * len(hu)} steps)")
    print("\nD2Q9 Taylor-Green L=256 u0=0.25 tau=1, with and without DDF shifting\n" + "\n".join(lines))
    for storage, margin in [("FP32", 1e5), ("FP16", 3e3), ("FP16S", 1e4), ("FP16C", 1e4), ("P16_1S", 2e3),
                            ("P16_2C", 80.0)]:
        ds, du = res[storage]
        assert du > margin * ds, (storage, ds, du)


def cylinder_poiseuille_error(P, arith, storage, R, u_max=0.1, re=10.0, shifting=True, diffusion_times=12,
                              block=None):
    """Sec. 4.1: D3Q19 SRT flow through a cylinder of radius R driven by the
    Guo force f = 4 rho nu u_max / R^2, nu = 2 R u_max / Re; relative L2 error
    of u_x over the fluid cells against u_theo(r) = f (R^2 - r^2) / (4 rho nu)
    once the flow has settled (diffusion_times * R^2 / nu steps)."""
    flags, r = W.cylinder_channel(R)
    nu = 2 * R * u_max / re
    tau = 3 * nu + 0.5
    f = 4 * nu * u_max / R ** 2
    L = flags.shape[0]
    g = P.Lattice(1, L, L, "D3Q19", "SRT", storage, arith, "AB", tau=tau, force=(f, 0, 0), shifting=shifting)
    if block is not None:
        g.set_block(*block)
    g.set_geometry(flags)
    g.set_rho_u()
    g.step(int(diffusion_times * R * R / nu))
    ux = g.rho_u()[1]
    g.close()
    fluid = flags == 0
    theo = f * (R * R - r * r) / (4 * nu)
    return float(np.sqrt(np.sum((ux - theo)[fluid] ** 2) / np.sum(theo[fluid] ** 2)))


def test_cylinder_poiseuille_radius_sweep():
    """Sec. 4.1 radius sweep at Re = 10, u_max = 0.1 (with and without DDF
    shifting): every tier matches FP64 where the staircase of the wall
    dominates (small R); FP32 stays with FP64 at every R; FP16 and FP16S
    fall behind at large R, FP16C later, the scaled posits hold up best;
    without shifting the 16-bit tiers fail."""
    P = _pkg()
    radii = [7, 15, 31, 63]
    tiers = [("FP64", "FP64"), ("FP32", "FP32"), ("FP32", "FP16"), ("FP32", "FP16S"), ("FP32", "FP16C"),
             ("FP32", "P16_1S"), ("FP32", "P16_2C")]
    err, err_ns = {}, {}
    for arith, storage in tiers:
        for R in radii:
            err[(storage, R)] = cylinder_poiseuille_error(P, arith, storage, R)
            if storage != "FP64":
                err_ns[(storage, R)] = cylinder_poiseuille_error(P, arith, storage, R, shifting=False)
    lines = ["tier          " + "".join(f"R={R:<4d}     " for R in radii)]
    for arith, storage in tiers:
        lines.append(f"{arith}/{storage:7s}" + "".join(f"{err[(storage, R)]:.3e}  " for R in radii))
        if storage != "FP64":
            lines.append(f"  unshifted   " + "".join(f"{err_ns[(storage, R)]:.3e}  " for R in radii))
    print("\nCylinder Poiseuille, D3Q19 SRT, Re=10, u_max=0.1: relative L2 error of u_x\n" + "\n".join(lines))
    for R in radii:
        assert abs(err[("FP32", R)] / err[("FP64", R)] - 1) < 0.1
    for storage in ("FP16", "FP16S", "FP16C", "P16_1S", "P16_2C"):
        assert err[(storage, 7)] < 1.5 * err[("FP64", 7)], storage
    assert err[("FP16", 63)] > 2 * err[("FP64", 63)] and err[("FP16S", 63)] > 2 * err[("FP64", 63)]
    # the posits hold up best at large R (their accurate interval fits the populations)
    assert err[("P16_1S", 63)] < 1.5 * err[("FP64", 63)]
    for storage in ("FP16", "FP16S", "FP16C", "P16_1S", "P16_2C"):
        assert err_ns[(storage, 63)] > 5 * err[(storage, 63)], storage


# Sec. 4.1 u_max sweeps: multiples of u_max at tau = 1, u_tau1 = Re / (12 R),
# per (R, Re); at Re = 100 the multiples stop near u_max = 0.2 (R = 63) and
# 0.13 (R = 31, where u_tau1 itself is 0.27)
UMAX_MULTIPLES = {
    (31, 1.0): (0.5, 1.0, 2.0, 4.0), (31, 10.0): (0.5, 1.0, 2.0, 4.0), (31, 100.0): (0.25, 0.5),
    (63, 1.0): (0.5, 1.0, 2.0, 4.0), (63, 10.0): (0.5, 1.0, 2.0, 4.0), (63, 100.0): (0.5, 1.0, 1.5),
}


def test_cylinder_poiseuille_umax_sweeps():
    """Sec. 4.1, u_max sweeps at constant R in {31, 63} and Re in {1, 10, 100}
    (nu = 2 R u_max / Re, so tau = 1 at u_max = Re / (12 R)), from rest for
    12 R^2 / nu steps, with and without DDF shifting.  The paper's findings
    asserted here: FP32 agrees with FP64; from u_max at tau = 1 upwards FP16C
    is almost always more accurate than FP16S (at Re 10 and 100); the error
    of the FP64 run is smaller at tau = 1 than at tau = 2.5 (the minimum lies
    near tau = 1); without shifting the 16-bit formats become very
    inaccurate, while FP64 does not notice."""
    P = _pkg()
    tiers = [("FP64", "FP64"), ("FP32", "FP32"), ("FP32", "FP16"), ("FP32", "FP16S"), ("FP32", "FP16C"),
             ("FP32", "P16_1S"), ("FP32", "P16_2C")]
    unshifted = ("FP64", "FP16", "FP16S", "FP16C", "P16_1S")
    err, err_ns, lines = {}, {}, []
    for (R, re), mults in UMAX_MULTIPLES.items():
        u_tau1 = re / (12 * R)
        for m in mults:
            u = m * u_tau1
            row = []
            for arith, storage in tiers:
                e = cylinder_poiseuille_error(P, arith, storage, R, u_max=u, re=re, block=(1, 32))
                err[(R, re, m, storage)] = e
                row.append(f"{e:.2e}")
                if storage in unshifted:
                    err_ns[(R, re, m, storage)] = cylinder_poiseuille_error(
                        P, arith, storage, R, u_max=u, re=re, shifting=False, block=(1, 32))
            lines.append(f"R={R:2d} Re={re:5.1f} u_max={u:.3e} ({m:4.2f} u_tau1)  " + "  ".join(row))
            lines.append("              unshifted                    " + "  ".join(
                f"{err_ns[(R, re, m, s)]:.2e}" if s in unshifted else "   -    " for _, s in tiers))
    print("\nCylinder Poiseuille u_max sweeps, D3Q19 SRT: relative L2 error of u_x\n"
          "tiers: " + ", ".join(f"{a}/{s}" for a, s in tiers) + "\n" + "\n".join(lines))
    keys = sorted({k[:3] for k in err})
    for R, re, m in keys:
        assert abs(err[(R, re, m, "FP32")] / err[(R, re, m, "FP64")] - 1) < 0.2, (R, re, m)
        assert abs(err_ns[(R, re, m, "FP64")] / err[(R, re, m, "FP64")] - 1) < 0.05, (R, re, m)
    # without shifting the 16-bit runs lose (most fail outright, error ~1);
    # only at the highest velocities, where the populations are large, does
    # an unshifted run come close
    for s in ("FP16", "FP16S", "FP16C", "P16_1S"):
        lost = sum(err_ns[k + (s,)] > 3 * err[k + (s,)] for k in keys)
        assert lost >= 0.8 * len(keys), (s, lost, len(keys))
    above = [k for k in keys if k[1] >= 10 and k[2] >= 1.0]
    wins = sum(err[k + ("FP16C",)] < err[k + ("FP16S",)] for k in above)
    assert wins >= len(above) - 1, (wins, len(above))
    for R in (31, 63):
        for re in (1.0, 10.0):
            assert err[(R, re, 1.0, "FP64")] < err[(R, re, 4.0, "FP64")], (R, re)
    # the format that resolves the smallest numbers (FP16S) still works at the
    # lowest velocity, where FP16 and FP16C fail
    low = (63, 1.0, 0.5)
    assert err[low + ("FP16S",)] < 0.5 * min(err[low + ("FP16",)], err[low + ("FP16C",)])
