"""Thin Python binding of the C ABI in include/lbm.h (ctypes).

Only argument marshalling lives here: every step of the lattice Boltzmann
path runs in the CUDA kernels of ``_build/liblbm.so``.  Device memory comes
from PyTorch's caching allocator through the library's allocator hook, and
launches go to PyTorch's current CUDA stream.  Importing this module does
not need a GPU; creating a lattice does, and fails loudly if the compiled
library is missing.

Function names mirror the C entry points (``lbm_create`` ...); the classes
``Lattice`` and ``Ensemble`` bundle them with numpy conversion.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

# ---------------------------------------------------------------- constants
LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_UNSUPPORTED = 0, 1, 2, 3, 4
LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, LBM_ERR_STATE = 5, 6, 7
VELSETS = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2}
COLLISIONS = {"SRT": 0, "TRT": 1, "MRT": 2}
STORAGES = {"FP64": 0, "FP32": 1, "FP16": 2, "FP16S": 3, "FP16C": 4,
            "P16_0S": 5, "P16_1S": 6, "P16_2C": 7, "P16_0": 8, "P16_1": 9}
ARITHS = {"FP32": 0, "FP64": 1}
SCHEMES = {"AB": 0, "AA": 1, "AUTO": 2}
VARIANTS = {"auto": 0, "generic": 1, "staged": 2, "paired": 3}
Q = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}
WALL, MOVING, EQ, OUTFLOW, FREESLIP = 0x01, 0x02, 0x04, 0x08, 0x10
EXPORTS = [
    "lbm_create", "lbm_destroy", "lbm_set_geometry", "lbm_set_rho_u", "lbm_step",
    "lbm_get_rho_u", "lbm_get_f", "lbm_set_f", "lbm_reduce", "lbm_get_info",
    "lbm_set_block", "lbm_autotune", "lbm_last_error", "lbm_status_string",
    "lbm_codec_encode", "lbm_codec_decode", "lbm_codec_encode_bits",
    "lbm_ensemble_create", "lbm_ensemble_step", "lbm_ensemble_step_each",
    "lbm_ensemble_set_block", "lbm_ensemble_autotune", "lbm_ensemble_destroy",
    "lbm_ensemble_last_error", "lbm_set_variant", "lbm_get_variant", "lbm_get_rho_u_static",
    "lbm_set_nodes", "lbm_get_f_cells", "lbm_get_rho_u_cells", "lbm_selftest_wait_timeout",
    "lbm_set_scheme", "lbm_ensemble_scheme", "lbm_set_divergence_check", "lbm_codec_encode_bits_table",
    "lbm_ensemble_set_variant", "lbm_ensemble_get_variant", "lbm_ensemble_set_layout", "lbm_ensemble_get_layout",
]


class LBMError(RuntimeError):
    def __init__(self, status, message=""):
        super().__init__(f"lbm status {status}: {message}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("velset", ctypes.c_int), ("collision", ctypes.c_int), ("storage", ctypes.c_int),
        ("arith", ctypes.c_int), ("scheme", ctypes.c_int),
        ("tau", ctypes.c_double), ("trt_lambda", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("no_ddf_shifting", ctypes.c_int),
    ]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lbm_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _RELEASE_FN), ("ctx", ctypes.c_void_p)]


class lbm_info(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int), ("cells", ctypes.c_int64), ("step", ctypes.c_int64),
        ("bytes_per_population", ctypes.c_int), ("has_flags", ctypes.c_int),
        ("device_bytes", ctypes.c_size_t), ("ddf", ctypes.c_void_p * 2), ("layout", ctypes.c_int),
        ("scheme", ctypes.c_int),
    ]


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """The compiled library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"CUDA library {LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        pI = ctypes.POINTER(ctypes.c_int)
        pD = ctypes.POINTER(ctypes.c_double)
        sig = {
            "lbm_create": [ctypes.POINTER(lbm_params), ctypes.POINTER(lbm_allocator), P, ctypes.POINTER(P)],
            "lbm_destroy": [P],
            "lbm_set_geometry": [P, P, P, P],
            "lbm_set_rho_u": [P, P, P, P, P],
            "lbm_step": [P, I64],
            "lbm_set_divergence_check": [P, I64, D],
            "lbm_get_rho_u": [P, P, P, P, P],
            "lbm_get_rho_u_static": [P, P, P, P, P],
            "lbm_get_f": [P, P],
            "lbm_set_nodes": [P, I64, P, P, P],
            "lbm_selftest_wait_timeout": [P],
            "lbm_set_scheme": [P, I],
            "lbm_ensemble_scheme": [P],
            "lbm_get_f_cells": [P, I64, P, P],
            "lbm_get_rho_u_cells": [P, I64, P, P, P, P, P],
            "lbm_set_f": [P, P],
            "lbm_reduce": [P, pD, pD],
            "lbm_get_info": [P, ctypes.POINTER(lbm_info)],
            "lbm_set_block": [P, I, I],
            "lbm_autotune": [P, I, pI, pI],
            "lbm_codec_encode": [I, P, P, I64, P],
            "lbm_codec_decode": [I, P, P, I64, P],
            "lbm_codec_encode_bits": [I, ctypes.c_uint32, I64, P, P],
            "lbm_codec_encode_bits_table": [I, ctypes.c_uint32, I64, P, P],
            "lbm_ensemble_create": [ctypes.POINTER(P), I, ctypes.POINTER(P)],
            "lbm_ensemble_step": [P, I64],
            "lbm_ensemble_step_each": [P, I64],
            "lbm_ensemble_set_block": [P, I, I],
            "lbm_ensemble_set_variant": [P, I, I],
            "lbm_ensemble_get_variant": [P],
            "lbm_ensemble_set_layout": [P, I],
            "lbm_ensemble_get_layout": [P],
            "lbm_ensemble_autotune": [P, I, pI, pI],
            "lbm_ensemble_destroy": [P],
            "lbm_set_variant": [P, I],
            "lbm_get_variant": [P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        for name in ("lbm_last_error", "lbm_ensemble_last_error"):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = ctypes.c_char_p
        L.lbm_status_string.argtypes = [I]
        L.lbm_status_string.restype = ctypes.c_char_p
        _ = D
        _lib = L
        return L


def _check(status, handle=None, ensemble=False):
    if status == LBM_OK:
        return
    L = load()
    msg = L.lbm_status_string(status).decode()
    if handle:
        detail = (L.lbm_ensemble_last_error if ensemble else L.lbm_last_error)(handle).decode()
        if detail:
            msg += f" ({detail})"
    raise LBMError(status, msg)


# ---------------------------------------------------------------- torch glue
def _torch():
    import torch
    return torch


class TorchAllocator:
    """lbm_allocator backed by torch.empty on one CUDA device."""

    def __init__(self, device):
        self.device = device
        self.live = {}

        def alloc(nbytes, ctx):
            torch = _torch()
            try:
                t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=self.device)
            except RuntimeError:
                return None
            p = t.data_ptr()
            self.live[p] = t
            return p

        def release(ptr, ctx):
            self.live.pop(ptr, None)

        self._alloc = _ALLOC_FN(alloc)
        self._release = _RELEASE_FN(release)
        self.struct = lbm_allocator(self._alloc, self._release, None)


_allocators = {}


def torch_allocator(device=None):
    torch = _torch()
    index = torch.device(device).index if device is not None else None
    dev = torch.device("cuda", torch.cuda.current_device() if index is None else index)
    key = dev.index
    if key not in _allocators:
        _allocators[key] = TorchAllocator(dev)
    return _allocators[key]


def current_stream_ptr():
    return _torch().cuda.current_stream().cuda_stream


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------- C names
def lbm_create(params: lbm_params, allocator=None, stream=None):
    L = load()
    h = ctypes.c_void_p()
    al = ctypes.byref(allocator.struct) if allocator is not None else None
    _check(L.lbm_create(ctypes.byref(params), al, ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def lbm_status_string(status):
    return load().lbm_status_string(status).decode()


# ---------------------------------------------------------------- lattice
class Lattice:
    """One lattice on the current CUDA device; arrays are (nz, ny, nx) numpy."""

    def __init__(self, nx, ny, nz, velset="D3Q19", collision="SRT", storage="FP32",
                 arith="FP32", scheme="AB", tau=0.8, trt_lambda=3.0 / 16.0,
                 force=(0.0, 0.0, 0.0), stream=None, allocator=None, shifting=True):
        self._L = load()
        self.params = lbm_params(nx, ny, nz, VELSETS[velset], COLLISIONS[collision], STORAGES[storage],
                                 ARITHS[arith], SCHEMES[scheme], float(tau), float(trt_lambda),
                                 (ctypes.c_double * 3)(*[float(v) for v in force]), 0 if shifting else 1)
        self.allocator = allocator if allocator is not None else torch_allocator()
        self.stream = current_stream_ptr() if stream is None else stream
        self._h = None
        self._h = lbm_create(self.params, self.allocator, self.stream)
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.q = Q[velset]
        self.velset, self.storage = velset, storage
        self.scheme = {0: "AB", 1: "AA"}[self.info().scheme]   # AUTO resolved at creation

    def close(self):
        """Release the lattice's device memory (lbm_destroy); idempotent."""
        if self._h:
            self._L.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        """The lbm_handle* of the C ABI."""
        return self._h

    def _c(self, status):
        _check(status, self._h)

    def set_geometry(self, flags=None, node_u=None, node_rho=None):
        """Cell flags (N bytes, x fastest; None: fully periodic fluid), wall/EQ
        velocities (3 x N floats) and EQ densities (N floats) (lbm_set_geometry)."""
        fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        nu = None if node_u is None else np.ascontiguousarray(node_u, dtype=np.float32).reshape(-1)
        nr = None if node_rho is None else np.ascontiguousarray(node_rho, dtype=np.float32).reshape(-1)
        self._c(self._L.lbm_set_geometry(self._h, _ptr(fl), _ptr(nu), _ptr(nr)))

    def set_nodes(self, cells, node_u=None, node_rho=None):
        """Boundary-node data of the listed cells only: node_u shaped (3, count),
        node_rho (count,); either may be None (unchanged)."""
        c = np.ascontiguousarray(cells, dtype=np.int64).reshape(-1)
        nu = None if node_u is None else np.ascontiguousarray(node_u, dtype=np.float32).reshape(3, c.size)
        nr = None if node_rho is None else np.ascontiguousarray(node_rho, dtype=np.float32).reshape(c.size)
        self._c(self._L.lbm_set_nodes(self._h, c.size, _ptr(c), _ptr(nu), _ptr(nr)))

    def _cells(self, cells):
        c = np.asarray(cells, dtype=np.int64)
        if c.ndim == 2 and c.shape[1] == 3:      # (z, y, x) triples
            nz, ny, nx = self.shape
            c = c[:, 2] + nx * (c[:, 1] + ny * c[:, 0])
        return np.ascontiguousarray(c.reshape(-1))

    def f_cells(self, cells):
        """Streamed populations of listed cells (flat indices or (z, y, x)
        triples), shaped (q, count)."""
        c = self._cells(cells)
        out = np.empty((self.q, c.size), dtype=np.float64)
        self._c(self._L.lbm_get_f_cells(self._h, c.size, _ptr(c), _ptr(out)))
        return out

    def rho_u_cells(self, cells):
        """(rho, ux, uy, uz) of listed cells, each shaped (count,)."""
        c = self._cells(cells)
        out = [np.empty(c.size, dtype=np.float64) for _ in range(4)]
        self._c(self._L.lbm_get_rho_u_cells(self._h, c.size, _ptr(c), *[_ptr(a) for a in out]))
        return tuple(out)

    def set_rho_u(self, rho=None, ux=None, uy=None, uz=None):
        """Equilibrium populations from host fields of N values each; None: rho
        1, u 0 (lbm_set_rho_u)."""
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
                for a in (rho, ux, uy, uz)]
        self._c(self._L.lbm_set_rho_u(self._h, *[_ptr(a) for a in arrs]))

    def set_rho_u_ptr(self, rho, ux, uy, uz):
        """Host pointers (e.g. pinned torch tensors' data_ptr()) or None."""
        cv = lambda p: None if p is None else ctypes.c_void_p(p)
        self._c(self._L.lbm_set_rho_u(self._h, cv(rho), cv(ux), cv(uy), cv(uz)))

    def set_f(self, f):
        """Populations f_i (not shifted), q x N doubles, slot-major (lbm_set_f)."""
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert a.size == self.q * self.N
        self._c(self._L.lbm_set_f(self._h, _ptr(a)))

    def step(self, n=1):
        """Advance n stream-collide steps (lbm_step)."""
        self._c(self._L.lbm_step(self._h, int(n)))

    def set_divergence_check(self, every, mass_tol=0.0):
        """FP64 check inside step() every `every` steps (0: off): raises
        LBMError(LBM_ERR_DIVERGED) on a non-finite state or a relative mass
        drift above mass_tol (lbm_set_divergence_check)."""
        self._c(self._L.lbm_set_divergence_check(self._h, int(every), float(mass_tol)))

    def rho_u(self):
        """(rho, ux, uy, uz) of every cell, each shaped (nz, ny, nx) (lbm_get_rho_u)."""
        out = [np.empty(self.N, dtype=np.float64) for _ in range(4)]
        self._c(self._L.lbm_get_rho_u(self._h, *[_ptr(a) for a in out]))
        return tuple(a.reshape(self.shape) for a in out)

    def get_rho_u_ptr(self, rho, ux, uy, uz):
        """lbm_get_rho_u into host pointers (e.g. pinned tensors' data_ptr()) or None."""
        cv = lambda p: None if p is None else ctypes.c_void_p(p)
        self._c(self._L.lbm_get_rho_u(self._h, cv(rho), cv(ux), cv(uy), cv(uz)))

    def f(self):
        """Streamed populations f_i (not shifted), shaped (q, nz, ny, nx) (lbm_get_f)."""
        out = np.empty(self.q * self.N, dtype=np.float64)
        self._c(self._L.lbm_get_f(self._h, _ptr(out)))
        return out.reshape((self.q,) + self.shape)

    def reduce(self):
        """(mass, kinetic energy) as FP64 sums over the lattice (lbm_reduce)."""
        m, e = ctypes.c_double(), ctypes.c_double()
        self._c(self._L.lbm_reduce(self._h, ctypes.byref(m), ctypes.byref(e)))
        return m.value, e.value

    def info(self) -> lbm_info:
        """Layout, variant, scheme, step count and device bytes (lbm_get_info)."""
        inf = lbm_info()
        self._c(self._L.lbm_get_info(self._h, ctypes.byref(inf)))
        return inf

    def set_block(self, bx, by):
        """Thread-block shape of the kernels that take one (lbm_set_block)."""
        self._c(self._L.lbm_set_block(self._h, int(bx), int(by)))

    def autotune(self, trial_steps=20):
        """Picks the kernel variant (and with it the layout) and then the block
        shape by timing (lbm_autotune); returns (bx, by)."""
        bx, by = ctypes.c_int(), ctypes.c_int()
        self._c(self._L.lbm_autotune(self._h, int(trial_steps), ctypes.byref(bx), ctypes.byref(by)))
        self.scheme = {0: "AB", 1: "AA"}[self.info().scheme]
        return bx.value, by.value

    def set_scheme(self, scheme: str):
        """Switch between A-B and in-place A-A streaming (after an even step count)."""
        self._c(self._L.lbm_set_scheme(self._h, SCHEMES[scheme]))
        self.scheme = scheme

    def set_variant(self, variant: str):
        """'auto', 'generic', 'staged' or 'paired' (see lbm_set_variant)."""
        self._c(self._L.lbm_set_variant(self._h, VARIANTS[variant]))

    def variant(self) -> str:
        """The kernel variant in use (lbm_get_variant)."""
        return {v: k for k, v in VARIANTS.items()}[self._L.lbm_get_variant(self._h)]


class Ensemble:
    """Many lattices advanced by one launch per step (members must share
    velocity set, collision, storage, arithmetic and scheme, and have flags)."""

    def __init__(self, members):
        self._L = load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.handle for m in self.members])
        self._e = ctypes.c_void_p()
        _check(self._L.lbm_ensemble_create(arr, len(self.members), ctypes.byref(self._e)))

    def close(self):
        """Free the ensemble's tables and return chunked members to their own
        layout (lbm_ensemble_destroy); idempotent."""
        if self._e:
            self._L.lbm_ensemble_destroy(self._e)
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        """Advance every member n steps, one launch per step for all (lbm_ensemble_step)."""
        _check(self._L.lbm_ensemble_step(self._e, int(n)), self._e, ensemble=True)

    def step_each(self, n=1):
        """The same steps as launches member by member (lbm_ensemble_step_each)."""
        _check(self._L.lbm_ensemble_step_each(self._e, int(n)), self._e, ensemble=True)

    def set_block(self, bx, by):
        """Cells per tile of the per-cell kernel (by = 1; lbm_ensemble_set_block)."""
        _check(self._L.lbm_ensemble_set_block(self._e, int(bx), int(by)), self._e, ensemble=True)

    def set_variant(self, variant, warps=4):
        """'per_cell' or 'paired' (two cells per thread, `warps` runs of 64
        cells per tile); see lbm_ensemble_set_variant."""
        code = {"per_cell": 0, "paired": 1}[variant]
        _check(self._L.lbm_ensemble_set_variant(self._e, code, int(warps)), self._e, ensemble=True)

    def variant(self) -> str:
        """The ensemble kernel in use: 'per_cell' or 'paired'."""
        return {0: "per_cell", 1: "paired"}[self._L.lbm_ensemble_get_variant(self._e)]

    def set_layout(self, layout):
        """'soa' or 'chunked' (the members' population layout; see
        lbm_ensemble_set_layout)."""
        _check(self._L.lbm_ensemble_set_layout(self._e, {"soa": 0, "chunked": 1}[layout]), self._e, ensemble=True)

    def layout(self) -> str:
        """The members' population layout: 'soa' or 'chunked'."""
        return {0: "soa", 1: "chunked"}[self._L.lbm_ensemble_get_layout(self._e)]

    def autotune(self, trial_steps=5):
        """Picks the member layout, the kernel, the tile and the streaming
        scheme by timing (lbm_ensemble_autotune); returns (cells per tile, 1
        for the per-cell kernel or warps per tile of the paired one)."""
        bx, by = ctypes.c_int(), ctypes.c_int()
        _check(self._L.lbm_ensemble_autotune(self._e, int(trial_steps), ctypes.byref(bx), ctypes.byref(by)),
               self._e, ensemble=True)
        return bx.value, by.value

    def scheme(self) -> str:
        """The members' streaming scheme: 'AB' or 'AA' (lbm_ensemble_scheme)."""
        return {v: k for k, v in SCHEMES.items()}[self._L.lbm_ensemble_scheme(self._e)]


# ---------------------------------------------------------------- codecs
def codec_encode(storage, x, out=None, stream=None):
    """x: float32 CUDA tensor -> uint16 codes (returned as an int16 tensor view)."""
    torch = _torch()
    x = x.contiguous()
    if out is None:
        out = torch.empty(x.shape, dtype=torch.int16, device=x.device)
    st = load().lbm_codec_encode(STORAGES[storage], ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), x.numel(),
                                 ctypes.c_void_p(stream or current_stream_ptr()))
    _check(st)
    return out


def codec_decode(storage, codes, out=None, stream=None):
    torch = _torch()
    codes = codes.contiguous()
    if out is None:
        out = torch.empty(codes.shape, dtype=torch.float32, device=codes.device)
    st = load().lbm_codec_decode(STORAGES[storage], ctypes.c_void_p(codes.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), codes.numel(),
                                 ctypes.c_void_p(stream or current_stream_ptr()))
    _check(st)
    return out


def codec_encode_bits(storage, first, n, out=None, stream=None, device=None, table=False):
    """Codes of the floats with bit patterns first .. first+n-1; table=True
    uses the paired kernel's table-driven posit encoder."""
    torch = _torch()
    if out is None:
        out = torch.empty(n, dtype=torch.int16, device=device or "cuda")
    fn = load().lbm_codec_encode_bits_table if table else load().lbm_codec_encode_bits
    st = fn(STORAGES[storage], ctypes.c_uint32(first), int(n), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(stream or current_stream_ptr()))
    _check(st)
    return out
