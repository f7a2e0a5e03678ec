"""Seeded synthetic inputs shaped like the paper's test systems.

This module builds only INPUTS: cell flags, boundary-node velocities and
densities, initial density / velocity fields and ensemble descriptors.  It
holds none of the lattice Boltzmann arithmetic, so the CUDA path, the CPU
oracle, the tests and the benchmark can all draw the same inputs from it.

Arrays are numpy, shaped (nz, ny, nx) (x fastest), matching the cell index
n = x + nx*(y + ny*z).  node_u is shaped (3, nz, ny, nx).

Flag bits (one byte per cell):
  WALL 0x01 solid (half-way bounce-back), MOVING 0x02 (with WALL: moving wall,
  velocity in node_u), EQ 0x04 (equilibrium node with node_rho / node_u),
  OUTFLOW 0x08 (zero-gradient outflow, -x neighbour), FREESLIP 0x10 (with
  WALL: specular wall) with its normal axis in bits 5-6.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

WALL, MOVING, EQ, OUTFLOW, FREESLIP = 0x01, 0x02, 0x04, 0x08, 0x10


def freeslip(axis: int) -> int:
    """Flag byte of a free-slip wall whose normal is along `axis` (0=x, 1=y, 2=z)."""
    return WALL | FREESLIP | (axis << 5)


# ----------------------------------------------------------------- geometry
def poiseuille_plate(nx=8, ny=64, nz=8):
    """Plane channel: walls at y = 0 and y = ny-1, periodic in x and z."""
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    flags[:, 0, :] = WALL
    flags[:, ny - 1, :] = WALL
    return flags


def couette_plate(nx, ny, nz, u_wall):
    """Plane channel with a moving wall at y = ny-1 (velocity u_wall along x)."""
    flags = poiseuille_plate(nx, ny, nz)
    flags[:, ny - 1, :] = WALL | MOVING
    node_u = np.zeros((3, nz, ny, nx), dtype=np.float32)
    node_u[0, :, ny - 1, :] = u_wall
    return flags, node_u


def cavity(n, u_lid, ny=None, nz=None):
    """Lid-driven cavity: solid shell one cell thick, the whole z = nz-1 plane
    is a lid moving along +y with speed u_lid."""
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    flags[0, :, :] = WALL
    flags[:, 0, :] = WALL
    flags[:, ny - 1, :] = WALL
    flags[:, :, 0] = WALL
    flags[:, :, nx - 1] = WALL
    flags[nz - 1, :, :] = WALL | MOVING
    node_u = np.zeros((3, nz, ny, nx), dtype=np.float32)
    node_u[1, nz - 1, :, :] = u_lid
    return flags, node_u


def cavity_flags(n):
    """Flags of the n^3 lid-driven cavity of `cavity` alone (one byte per
    cell), for lattices too large for full-size node arrays."""
    flags = np.full((n, n, n), WALL, dtype=np.uint8)
    flags[1:n - 1, 1:n - 1, 1:n - 1] = 0
    flags[n - 1, :, :] = WALL | MOVING
    return flags


def cavity_lid(n, u_lid):
    """The lid of the n^3 cavity as a sparse node list: (cell indices of the
    z = n-1 plane, node velocities shaped (3, n*n) with u_y = u_lid)."""
    cells = (n - 1) * n * n + np.arange(n * n, dtype=np.int64)
    u = np.zeros((3, n * n), dtype=np.float32)
    u[1] = u_lid
    return cells, u


def karman_channel(nx=1024, ny=256, nz=64, radius=24, cx=256, cy=128, u_in=0.05):
    """Channel along x: equilibrium inflow plane x = 0 (rho=1, u=(u_in,0,0)),
    zero-gradient outflow plane x = nx-1, free-slip walls at y = 0 and
    y = ny-1, periodic in z, solid cylinder of `radius` along z."""
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    node_u = np.zeros((3, nz, ny, nx), dtype=np.float32)
    node_rho = np.ones((nz, ny, nx), dtype=np.float32)
    flags[:, :, 0] = EQ
    node_u[0, :, :, 0] = u_in
    flags[:, :, nx - 1] = OUTFLOW
    flags[:, 0, :] = freeslip(1)
    flags[:, ny - 1, :] = freeslip(1)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    inside = (xx - cx) ** 2 + (yy - cy) ** 2 <= radius * radius
    flags[:, inside] = WALL
    return flags, node_u, node_rho


def karman_initial_fields(nx, ny, nz, u_in=0.05, x_perturb=256, amp=0.005):
    """Uniform inflow velocity with a deterministic transverse perturbation
    u_y = amp*sin(2 pi z / nz + 1) upstream of x_perturb (breaks symmetry)."""
    rho = np.ones((nz, ny, nx))
    ux = np.full((nz, ny, nx), u_in)
    uy = np.zeros((nz, ny, nx))
    uz = np.zeros((nz, ny, nx))
    z = np.arange(nz)[:, None, None]
    pert = amp * np.sin(2 * math.pi * z / nz + 1.0) * np.ones((1, ny, nx))
    mask = np.arange(nx)[None, None, :] < x_perturb
    uy = np.where(mask, pert, 0.0)
    return rho, ux, uy, uz


# ----------------------------------------------------------------- fields
def taylor_green_extruded(n, u0, nz=None, ny=None):
    """2-D Taylor-Green vortex (Sec. 4.2 closed form at t = 0) extruded along z:
    u_x = u0 cos(kx) sin(ky), u_y = -u0 sin(kx) cos(ky), u_z = 0,
    rho = 1 - 3 u0^2 / 4 (cos 2kx + cos 2ky), k = 2 pi / n."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    k = 2.0 * math.pi / n
    ky = 2.0 * math.pi / ny
    x = np.arange(n)[None, None, :]
    y = np.arange(ny)[None, :, None]
    ux = u0 * np.cos(k * x) * np.sin(ky * y) * np.ones((nz, 1, 1))
    uy = -u0 * np.sin(k * x) * np.cos(ky * y) * np.ones((nz, 1, 1))
    uz = np.zeros((nz, ny, n))
    rho = 1.0 - 0.75 * u0 * u0 * (np.cos(2 * k * x) + np.cos(2 * ky * y)) * np.ones((nz, 1, 1))
    return rho, ux, uy, uz


def taylor_green_3d(n, u0):
    """Classic 3-D Taylor-Green vortex initial velocity (sin, cos, cos form),
    unit density."""
    k = 2.0 * math.pi / n
    c = np.arange(n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    ux = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    uy = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    uz = np.zeros_like(ux)
    rho = np.ones_like(ux)
    return rho, ux, uy, uz


def random_fields(shape, seed, u_amp=0.05, rho_amp=0.01):
    """Seeded random density around 1 and velocity of amplitude u_amp."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1, 1, shape)
    ux = u_amp * rng.uniform(-1, 1, shape)
    uy = u_amp * rng.uniform(-1, 1, shape)
    uz = u_amp * rng.uniform(-1, 1, shape)
    return rho, ux, uy, uz


def random_geometry(shape, seed, wall=0.08, moving=0.03, eq=0.02, outflow=0.02,
                    freeslip_frac=0.03, u_amp=0.05):
    """Seeded random mix of every cell kind (for parity tests), with wall
    velocities and equilibrium-node states."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(0, 1, shape)
    flags = np.zeros(shape, dtype=np.uint8)
    t = 0.0
    for frac, val in ((wall, WALL), (moving, WALL | MOVING), (eq, EQ), (outflow, OUTFLOW)):
        flags[(r >= t) & (r < t + frac)] = val
        t += frac
    fs = (r >= t) & (r < t + freeslip_frac)
    axes = rng.integers(0, 4, shape).astype(np.uint8)   # axis code 3: plain bounce-back
    flags[fs] = (WALL | FREESLIP | (axes << 5))[fs]
    # an outflow cell pulls as if one cell upstream in x: keep that cell fluid
    upstream_solid = (np.roll(flags, 1, axis=-1) & WALL) != 0
    flags[((flags & OUTFLOW) != 0) & upstream_solid] = 0
    node_u = (u_amp * rng.uniform(-1, 1, (3,) + tuple(shape))).astype(np.float32)
    node_rho = (1.0 + 0.01 * rng.uniform(-1, 1, shape)).astype(np.float32)
    return flags, node_u, node_rho


# ----------------------------------------------------------------- ensemble
def splitmix64(state: int):
    """splitmix64 (Steele, Lea, Flood 2014): returns (next_state, output)."""
    mask = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & mask
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    return state, z ^ (z >> 31)


@dataclass
class CavitySpec:
    n: int
    tau: float
    u_lid: float


def ensemble_cavities(count=512, seed=20211216, n_min=16, n_max=128,
                      tau_range=(0.51, 0.9), u_range=(0.02, 0.1)):
    """Lid-driven cavities with edges uniform in [n_min, n_max], tau and lid
    speed uniform in the given ranges, drawn from splitmix64(seed)."""
    st = seed
    out = []
    for _ in range(count):
        st, a = splitmix64(st)
        st, b = splitmix64(st)
        st, c = splitmix64(st)
        n = n_min + a % (n_max - n_min + 1)
        tau = tau_range[0] + (b >> 11) * (1.0 / (1 << 53)) * (tau_range[1] - tau_range[0])
        u = u_range[0] + (c >> 11) * (1.0 / (1 << 53)) * (u_range[1] - u_range[0])
        out.append(CavitySpec(int(n), float(tau), float(u)))
    return out


def cylinder_channel(R):
    """Sec. 4.1 channel: L_x = 1, L_y = L_z = 2 (R + 1), axis along x through
    the box centre; a cell is solid when its centre lies outside radius R.
    Returns (flags (nz, ny, 1), r of every cell centre (nz, ny, 1))."""
    L = 2 * (R + 1)
    c = np.arange(L) + 0.5 - L / 2.0
    z, y = np.meshgrid(c, c, indexing="ij")
    r = np.sqrt(y * y + z * z)[:, :, None]
    flags = np.where(r > R, WALL, 0).astype(np.uint8)
    return flags, r
