"""FP64 CPU oracle for the qTask state-vector hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library: the amplitude arithmetic is the plain C file
``qt_oracle.c`` (textbook pair / quad loops in FP64, qTask Section II-A), and
``paper_partition.py`` restates the paper's own block-partition and
range-intersection rules (Sections III-C to III-E) for the worked example.

Gates are passed as objects (or tuples) with ``name``, ``targets``,
``controls`` and ``params`` -- the OpenQASM-style names of the paper's gate
table (Table 1) plus the composites cz, ccx, swap, cp and u3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qt_oracle.c")
_SO = os.path.join(_HERE, "libqt_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP for the timed all-core variant)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", _SO + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # QT_ORACLE_LIB lets the mutation test load a deliberately broken
            # copy of the oracle; it is never set otherwise.
            lib = ctypes.CDLL(os.environ.get("QT_ORACLE_LIB") or build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.orc_base_matrix.argtypes = [ctypes.c_char_p, dp, dp]
            lib.orc_base_matrix.restype = ctypes.c_int
            lib.orc_apply_gate.argtypes = [ctypes.c_int, dp, ctypes.c_char_p, ctypes.c_int, ip,
                                           ctypes.c_int, ip, dp, ctypes.c_int]
            lib.orc_apply_gate.restype = ctypes.c_int
            lib.orc_simulate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ip, ip,
                                         ip, ip, dp, dp, ctypes.c_int]
            lib.orc_simulate.restype = ctypes.c_int
            lib.orc_norm.argtypes = [ctypes.c_int, dp]
            lib.orc_norm.restype = ctypes.c_double
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _fields(g):
    if isinstance(g, tuple):
        name, targets, controls, params = g
    else:
        name, targets, controls, params = g.name, g.targets, g.controls, g.params
    p = list(params) + [0.0] * (3 - len(params))
    return str(name), list(targets), list(controls), p[:3]


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def base_matrix(name: str, params=(0.0, 0.0, 0.0)) -> np.ndarray:
    """The gate's base matrix (2x2, or 4x4 for swap) as complex128."""
    lib = _load()
    p = np.zeros(3, dtype=np.float64)
    p[: len(params)] = params
    out = np.zeros(32, dtype=np.float64)
    dim = lib.orc_base_matrix(name.encode(), _dp(p), _dp(out))
    if dim == 0:
        raise ValueError(f"unknown gate {name!r}")
    return (out[0: 2 * dim * dim: 2] + 1j * out[1: 2 * dim * dim: 2]).reshape(dim, dim)


def apply_gate(psi: np.ndarray, gate, nthreads: int = 1) -> np.ndarray:
    """Apply one gate in place to a complex128 state of length 2^n."""
    lib = _load()
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    n = int(psi.size).bit_length() - 1
    name, t, c, p = _fields(gate)
    ta = np.array(t + [0, 0], dtype=np.int32)
    ca = np.array(c + [0, 0], dtype=np.int32)
    pa = np.array(p, dtype=np.float64)
    rc = lib.orc_apply_gate(n, _dp(psi.view(np.float64)), name.encode(), len(t), _ip(ta), len(c), _ip(ca),
                            _dp(pa), nthreads)
    if rc:
        raise ValueError(f"oracle rejected gate {gate!r}")
    return psi


def simulate(n: int, gates, nthreads: int = 1) -> np.ndarray:
    """Output state of the flat gate list (application order) from |0...0>."""
    lib = _load()
    gl = [_fields(g) for g in gates]
    m = len(gl)
    names = (ctypes.c_char_p * max(m, 1))(*[g[0].encode() for g in gl])
    nt = np.array([len(g[1]) for g in gl] or [0], dtype=np.int32)
    nc = np.array([len(g[2]) for g in gl] or [0], dtype=np.int32)
    tg = np.zeros(2 * max(m, 1), dtype=np.int32)
    cg = np.zeros(2 * max(m, 1), dtype=np.int32)
    pr = np.zeros(3 * max(m, 1), dtype=np.float64)
    for k, (_, t, c, p) in enumerate(gl):
        tg[2 * k: 2 * k + len(t)] = t
        cg[2 * k: 2 * k + len(c)] = c
        pr[3 * k: 3 * k + 3] = p
    psi = np.zeros(1 << n, dtype=np.complex128)
    rc = lib.orc_simulate(n, m, names, _ip(nt), _ip(tg), _ip(nc), _ip(cg), _dp(pr), _dp(psi.view(np.float64)),
                          nthreads)
    if rc:
        raise ValueError(f"oracle rejected gate #{-rc - 2}" if rc < -1 else "oracle rejected the circuit")
    return psi


def norm(psi: np.ndarray) -> float:
    lib = _load()
    n = int(psi.size).bit_length() - 1
    return float(lib.orc_norm(n, _dp(np.ascontiguousarray(psi).view(np.float64))))


def max_threads() -> int:
    return int(_load().orc_max_threads())
