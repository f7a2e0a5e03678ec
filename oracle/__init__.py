"""CPU oracle for the mixed-precision lattice Boltzmann step (arXiv 2112.08926).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
``paper_2112_08926_gb300`` never imports this module, and this module never
imports the product package.

The C++ sources next to this file (``codecs.cpp``, ``lattice.cpp``) are built
into ``_build/liboracle.so`` with floating-point contraction disabled, so the
ordered FP32/FP64 modes fuse exactly the operations written as ``fma`` there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, n) for n in ("codecs.cpp", "lattice.cpp", "oracle.h")]

FORMATS = {
    "FP64": 0, "FP32": 1, "FP16": 2, "FP16S": 3, "FP16C": 4,
    "P16_0S": 5, "P16_1S": 6, "P16_2C": 7, "P16_0": 8, "P16_1": 9,
}
CODEC_FORMATS = ["FP16", "FP16S", "FP16C", "P16_0S", "P16_1S", "P16_2C", "P16_0", "P16_1"]
VELSETS = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2}
COLLISIONS = {"SRT": 0, "TRT": 1, "MRT": 2}
ARITH = {"DEF64": 0, "ORD32": 1, "ORD64": 2}

WALL, MOVING, EQ, OUTFLOW, FREESLIP = 0x01, 0x02, 0x04, 0x08, 0x10

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (C++17, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in _SOURCES):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = [
        "g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
        "-ffp-contract=off", "-fno-fast-math", "-Wall",
        "-o", tmp, os.path.join(_HERE, "codecs.cpp"), os.path.join(_HERE, "lattice.cpp"),
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("velset", ctypes.c_int), ("collision", ctypes.c_int), ("arith", ctypes.c_int),
        ("storage", ctypes.c_int), ("tau", ctypes.c_double), ("trt_lambda", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("no_shift", ctypes.c_int),
    ]


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            L.orc_encode.restype = ctypes.c_uint16
            L.orc_encode.argtypes = [ctypes.c_int, ctypes.c_float]
            L.orc_decode.restype = ctypes.c_float
            L.orc_decode.argtypes = [ctypes.c_int, ctypes.c_uint16]
            L.orc_encode_array.argtypes = [ctypes.c_int, P, P, i64]
            L.orc_decode_array.argtypes = [ctypes.c_int, P, P, i64]
            L.orc_encode_bits_range.argtypes = [ctypes.c_int, ctypes.c_uint32, i64, P]
            L.orc_velset_q.argtypes = [ctypes.c_int]
            L.orc_velset_table.argtypes = [ctypes.c_int, P, P]
            L.orc_mrt_basis.argtypes = [P]
            L.orc_mrt_rates.argtypes = [ctypes.c_double, P]
            L.orc_create.restype = P
            L.orc_create.argtypes = [ctypes.POINTER(_Params)]
            L.orc_destroy.argtypes = [P]
            L.orc_set_geometry.argtypes = [P, P, P, P]
            L.orc_set_geometry.restype = ctypes.c_int
            L.orc_set_rho_u.argtypes = [P, P, P, P, P]
            L.orc_set_f.argtypes = [P, P]
            L.orc_step.argtypes = [P, i64]
            L.orc_get_rho_u.argtypes = [P, P, P, P, P]
            L.orc_get_f.argtypes = [P, P]
            L.orc_reduce.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, P]
            L.orc_threads.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------- codecs
def encode(fmt: str, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib().orc_encode_array(FORMATS[fmt], _ptr(x), _ptr(out), x.size)
    return out


def decode(fmt: str, codes) -> np.ndarray:
    c = np.ascontiguousarray(codes, dtype=np.uint16)
    out = np.empty(c.shape, dtype=np.float32)
    lib().orc_decode_array(FORMATS[fmt], _ptr(c), _ptr(out), c.size)
    return out


def encode_bits_range(fmt: str, first: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint16)
    lib().orc_encode_bits_range(FORMATS[fmt], first, n, _ptr(out))
    return out


def velset(name: str):
    q = lib().orc_velset_q(VELSETS[name])
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    lib().orc_velset_table(VELSETS[name], _ptr(c), _ptr(w))
    return c, w


def equilibrium(vs: str, arith: str, rho: float, u) -> np.ndarray:
    q = lib().orc_velset_q(VELSETS[vs])
    out = np.zeros(q, dtype=np.float64)
    lib().orc_equilibrium(VELSETS[vs], ARITH[arith], float(rho), float(u[0]), float(u[1]),
                          float(u[2]) if len(u) > 2 else 0.0, _ptr(out))
    return out


def mrt_basis() -> np.ndarray:
    """The D3Q19 MRT moment basis (19 x 19) the oracle uses."""
    out = np.zeros((19, 19), dtype=np.float64)
    lib().orc_mrt_basis(_ptr(out))
    return out


def mrt_rates(tau: float) -> np.ndarray:
    out = np.zeros(19, dtype=np.float64)
    lib().orc_mrt_rates(ctypes.c_double(tau), _ptr(out))
    return out


def threads() -> int:
    return lib().orc_threads()


def set_threads(n: int) -> None:
    """Threads of the following oracle calls (for timing; results do not
    depend on the thread count)."""
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------- lattice
class Lattice:
    """A-B pull lattice on the CPU; arrays are shaped (nz, ny, nx)."""

    def __init__(self, nx, ny, nz, velset="D3Q19", collision="SRT", arith="DEF64",
                 storage="FP64", tau=0.8, trt_lambda=3.0 / 16.0, force=(0.0, 0.0, 0.0), shifting=True):
        p = _Params(nx, ny, nz, VELSETS[velset], COLLISIONS[collision], ARITH[arith],
                    FORMATS[storage], float(tau), float(trt_lambda),
                    (ctypes.c_double * 3)(*[float(v) for v in force]), 0 if shifting else 1)
        self._h = lib().orc_create(ctypes.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the lattice parameters")
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.q = lib().orc_velset_q(VELSETS[velset])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_geometry(self, flags=None, node_u=None, node_rho=None):
        fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        nu = None if node_u is None else np.ascontiguousarray(node_u, dtype=np.float32).reshape(-1)
        nr = None if node_rho is None else np.ascontiguousarray(node_rho, dtype=np.float32).reshape(-1)
        if lib().orc_set_geometry(self._h, None if fl is None else _ptr(fl),
                                  None if nu is None else _ptr(nu), None if nr is None else _ptr(nr)):
            raise ValueError("an OUTFLOW cell's -x neighbour is solid")

    def set_rho_u(self, rho=None, ux=None, uy=None, uz=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
                for a in (rho, ux, uy, uz)]
        lib().orc_set_rho_u(self._h, *[None if a is None else _ptr(a) for a in arrs])

    def set_f(self, f):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert a.size == self.q * self.N
        lib().orc_set_f(self._h, _ptr(a))

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def rho_u(self):
        out = [np.empty(self.N, dtype=np.float64) for _ in range(4)]
        lib().orc_get_rho_u(self._h, *[_ptr(a) for a in out])
        return tuple(a.reshape(self.shape) for a in out)

    def f(self):
        out = np.empty(self.q * self.N, dtype=np.float64)
        lib().orc_get_f(self._h, _ptr(out))
        return out.reshape((self.q,) + self.shape)

    def reduce(self):
        m, e = ctypes.c_double(), ctypes.c_double()
        lib().orc_reduce(self._h, ctypes.byref(m), ctypes.byref(e))
        return m.value, e.value
