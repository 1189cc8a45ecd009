"""ctypes binding of libqtask.so (C ABI declared in include/qtask.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels.  Module-level functions carry the ABI's names; ``Circuit`` is a
thin object wrapper over them.  The library must have been built
(``paper_2210_01076_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqtask.so")

QT_OK, QT_ERR_ARG, QT_ERR_CONFLICT, QT_ERR_RANGE, QT_ERR_NOT_FOUND, QT_ERR_OOM, QT_ERR_CUDA, QT_ERR_STALE, \
    QT_ERR_TIMEOUT = range(9)
STATUS_NAMES = ["QT_OK", "QT_ERR_ARG", "QT_ERR_CONFLICT", "QT_ERR_RANGE", "QT_ERR_NOT_FOUND", "QT_ERR_OOM",
                "QT_ERR_CUDA", "QT_ERR_STALE", "QT_ERR_TIMEOUT"]
QT_C128, QT_C64, QT_C128_DF = 0, 1, 2
DTYPES = {"c128": QT_C128, "c64": QT_C64, "c128df": QT_C128_DF}
KINDS = {name: i for i, name in enumerate(
    ["h", "x", "y", "z", "s", "sdg", "t", "tdg", "rx", "ry", "rz", "u3", "cnot", "cz", "swap", "ccx", "cp"])}


class qt_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("ntarget", ctypes.c_int32), ("target", ctypes.c_int32 * 2),
                ("ncontrol", ctypes.c_int32), ("control", ctypes.c_int32 * 2), ("theta", ctypes.c_double * 3)]


class qt_update_stats(ctypes.Structure):
    _fields_ = [("segments_total", ctypes.c_int32), ("segments_run", ctypes.c_int32),
                ("passes_total", ctypes.c_int32), ("passes_run", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("gates_total", ctypes.c_int32), ("partition_passes_total", ctypes.c_int64),
                ("partition_passes_run", ctypes.c_int64), ("clean_fraction", ctypes.c_double),
                ("amp_updates", ctypes.c_uint64), ("hbm_bytes", ctypes.c_uint64), ("host_ms", ctypes.c_double),
                ("gpu_ms", ctypes.c_double), ("pass_kernel_ms", ctypes.c_double),
                ("pass_kernel_launches", ctypes.c_int32), ("tensor_blocks", ctypes.c_int32),
                ("pass_kernel_bytes", ctypes.c_uint64), ("h2d_bytes", ctypes.c_uint64),
                ("pass_kernel_alu_ops", ctypes.c_uint64)]


EXPORTED = ["qt_create", "qt_destroy", "qt_num_levels", "qt_num_gates", "qt_insert_level", "qt_remove_level",
            "qt_insert_gate", "qt_remove_gate", "qt_replace_gate", "qt_update_state", "qt_read_amplitudes",
            "qt_read_amplitudes_device", "qt_read_amplitudes_async", "qt_read_wait", "qt_norm", "qt_norm_static", "qt_fidelity", "qt_max_abs_diff", "qt_probabilities",
            "qt_set_option", "qt_set_stream", "qt_num_segments", "qt_segment_info", "qt_segment_touched", "qt_last_error",
            "qt_batch_create", "qt_batch_run", "qt_batch_read_amplitudes", "qt_batch_destroy",
            "qt_batch_last_error",
            "qt_release_device", "qt_device_bytes", "qt_server_create", "qt_server_destroy",
            "qt_server_add_circuit", "qt_server_submit", "qt_server_wait", "qt_server_info"]

QT_EDIT_INSERT_LEVEL, QT_EDIT_INSERT_GATE, QT_EDIT_REMOVE_GATE, QT_EDIT_REPLACE_GATE, QT_EDIT_REMOVE_LEVEL = range(5)


class qt_edit(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("id", ctypes.c_uint64), ("gate", qt_gate)]


class qt_batch_stats(ctypes.Structure):
    _fields_ = [("gpu_ms", ctypes.c_double), ("circuits", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("tiles", ctypes.c_int32), ("graph_replayed", ctypes.c_int32), ("amp_updates", ctypes.c_uint64)]


class Batch:
    """Many small circuits re-simulated together in one persistent launch
    (qt_batch_*); the second and later runs of an unchanged structure replay
    a CUDA graph."""

    def __init__(self, circuits):
        self.circuits = list(circuits)
        arr = (ctypes.c_void_p * len(self.circuits))(*[c.h.value for c in self.circuits])
        h = ctypes.c_void_p()
        st = load().qt_batch_create(arr, len(self.circuits), ctypes.byref(h))
        _check(None, st)
        self.h = h

    def _check(self, status):
        if status != QT_OK:
            raise QtError(status, (load().qt_batch_last_error(self.h) or b"").decode())

    def run(self) -> dict:
        s = qt_batch_stats()
        self._check(load().qt_batch_run(self.h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in qt_batch_stats._fields_}

    def read_amplitudes(self, index: int) -> np.ndarray:
        c = self.circuits[index]
        out = np.empty(1 << c.n, np.complex64 if c.dtype == "c64" else np.complex128)
        self._check(load().qt_batch_read_amplitudes(self.h, index, 0, 1 << c.n, out.ctypes.data))
        return out

    def close(self):
        if self.h:
            load().qt_batch_destroy(self.h)
            self.h = None


class qt_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("circuit", ctypes.c_int32), ("queue_ms", ctypes.c_double),
                ("service_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("stats", qt_update_stats),
                ("n_new_ids", ctypes.c_int32), ("reserved", ctypes.c_int32), ("new_ids", ctypes.c_uint64 * 8)]


class QtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


_lib = None


def load(path: str = LIB_PATH):
    """Load libqtask.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2210_01076_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "qt_create": [i32, i32, i32, ctypes.POINTER(P)],
        "qt_destroy": [P],
        "qt_num_levels": [P, ctypes.POINTER(i32)],
        "qt_num_gates": [P, ctypes.POINTER(i64)],
        "qt_insert_level": [P, i32],
        "qt_remove_level": [P, i32],
        "qt_insert_gate": [P, i32, ctypes.POINTER(qt_gate), ctypes.POINTER(u64)],
        "qt_remove_gate": [P, i32, u64],
        "qt_replace_gate": [P, i32, u64, ctypes.POINTER(qt_gate), ctypes.POINTER(u64)],
        "qt_update_state": [P, i32, ctypes.POINTER(qt_update_stats)],
        "qt_read_amplitudes": [P, u64, u64, P],
        "qt_read_amplitudes_device": [P, u64, u64, P],
        "qt_read_amplitudes_async": [P, u64, u64, P],
        "qt_read_wait": [P],
        "qt_norm": [P, ctypes.POINTER(ctypes.c_double)],
        "qt_norm_static": [P, u64, i32, P, P],
        "qt_fidelity": [P, P, ctypes.POINTER(ctypes.c_double)],
        "qt_max_abs_diff": [P, P, ctypes.POINTER(ctypes.c_double)],
        "qt_probabilities": [P, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)],
        "qt_set_option": [P, ctypes.c_char_p, i64],
        "qt_set_stream": [P, P],
        "qt_num_segments": [P, ctypes.POINTER(i32)],
        "qt_segment_info": [P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32), P, P],
        "qt_segment_touched": [P, i32, P],
        "qt_release_device": [P],
        "qt_device_bytes": [P, ctypes.POINTER(i64)],
        "qt_server_create": [i32, i64, ctypes.POINTER(P)],
        "qt_server_destroy": [P],
        "qt_server_add_circuit": [P, P, ctypes.POINTER(i32)],
        "qt_server_submit": [P, i32, i32, ctypes.POINTER(qt_edit), ctypes.POINTER(u64)],
        "qt_server_wait": [P, u64, ctypes.POINTER(qt_request_result)],
        "qt_server_info": [P, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "qt_batch_create": [ctypes.POINTER(P), i32, ctypes.POINTER(P)],
        "qt_batch_run": [P, ctypes.POINTER(qt_batch_stats)],
        "qt_batch_read_amplitudes": [P, i32, u64, u64, P],
        "qt_batch_destroy": [P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.qt_last_error.argtypes = [P]
    lib.qt_last_error.restype = ctypes.c_char_p
    lib.qt_batch_last_error.argtypes = [P]
    lib.qt_batch_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(handle, status: int):
    if status != QT_OK:
        msg = load().qt_last_error(handle)
        raise QtError(status, msg.decode() if msg else "")


def make_qt_gate(g) -> qt_gate:
    """Marshal a gate (name, targets, controls, params) into the ABI struct."""
    if isinstance(g, tuple) and not hasattr(g, "name"):
        name, targets, controls, params = g
    else:
        name, targets, controls, params = g.name, g.targets, g.controls, g.params
    s = qt_gate()
    s.kind = KINDS[name]
    s.ntarget = len(targets)
    for k, q in enumerate(targets):
        s.target[k] = int(q)
    s.ncontrol = len(controls)
    for k, q in enumerate(controls):
        s.control[k] = int(q)
    for k, a in enumerate(params):
        s.theta[k] = float(a)
    return s


# ------------------------------------------------------ ABI-named functions

def qt_create(n_qubits: int, dtype: int, log2_partition: int):
    h = ctypes.c_void_p()
    _check(None, load().qt_create(n_qubits, dtype, log2_partition, ctypes.byref(h)))
    return h


def qt_destroy(h):
    load().qt_destroy(h)


def qt_num_levels(h) -> int:
    v = ctypes.c_int32()
    _check(h, load().qt_num_levels(h, ctypes.byref(v)))
    return v.value


def qt_num_gates(h) -> int:
    v = ctypes.c_int64()
    _check(h, load().qt_num_gates(h, ctypes.byref(v)))
    return v.value


def qt_insert_level(h, pos: int):
    _check(h, load().qt_insert_level(h, pos))


def qt_remove_level(h, pos: int):
    _check(h, load().qt_remove_level(h, pos))


def qt_insert_gate(h, level: int, gate) -> int:
    out = ctypes.c_uint64()
    g = make_qt_gate(gate)
    _check(h, load().qt_insert_gate(h, level, ctypes.byref(g), ctypes.byref(out)))
    return out.value


def qt_remove_gate(h, level: int, gid: int):
    _check(h, load().qt_remove_gate(h, level, gid))


def qt_replace_gate(h, level: int, gid: int, gate) -> int:
    out = ctypes.c_uint64()
    g = make_qt_gate(gate)
    _check(h, load().qt_replace_gate(h, level, gid, ctypes.byref(g), ctypes.byref(out)))
    return out.value


def stats_dict(s: qt_update_stats) -> Dict[str, float]:
    return {name: getattr(s, name) for name, _ in qt_update_stats._fields_ if name != "reserved"}


def qt_update_state(h, force_full: bool = False) -> Dict[str, float]:
    s = qt_update_stats()
    _check(h, load().qt_update_state(h, 1 if force_full else 0, ctypes.byref(s)))
    return stats_dict(s)


def qt_read_amplitudes(h, first: int, count: int, out: np.ndarray):
    assert out.flags.c_contiguous
    _check(h, load().qt_read_amplitudes(h, first, count, out.ctypes.data))
    return out


def qt_read_amplitudes_device(h, first: int, count: int, device_ptr: int):
    _check(h, load().qt_read_amplitudes_device(h, first, count, ctypes.c_void_p(device_ptr)))


def qt_read_amplitudes_async(h, first: int, count: int, out: np.ndarray):
    assert out.flags.c_contiguous
    _check(h, load().qt_read_amplitudes_async(h, first, count, out.ctypes.data))
    return out


def qt_read_wait(h):
    _check(h, load().qt_read_wait(h))


def qt_norm(h) -> float:
    v = ctypes.c_double()
    _check(h, load().qt_norm(h, ctypes.byref(v)))
    return v.value


def qt_fidelity(ha, hb) -> float:
    v = ctypes.c_double()
    _check(ha, load().qt_fidelity(ha, hb, ctypes.byref(v)))
    return v.value


def qt_max_abs_diff(ha, hb) -> float:
    v = ctypes.c_double()
    _check(ha, load().qt_max_abs_diff(ha, hb, ctypes.byref(v)))
    return v.value


def qt_probabilities(h, qubits) -> np.ndarray:
    k = len(qubits)
    q = (ctypes.c_int32 * max(k, 1))(*[int(x) for x in qubits])
    out = np.zeros(1 << k, np.float64)
    _check(h, load().qt_probabilities(h, k, q, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def qt_norm_static(amps_device_ptr: int, count: int, dtype: int, out_device_ptr: int, stream_ptr: int = 0):
    """Norm of caller-held device amplitudes into a caller-held device double;
    allocates nothing (see include/qtask.h)."""
    _check(None, load().qt_norm_static(ctypes.c_void_p(amps_device_ptr), count, dtype,
                                       ctypes.c_void_p(out_device_ptr), ctypes.c_void_p(stream_ptr or 0)))


def qt_set_option(h, key: str, value: int):
    _check(h, load().qt_set_option(h, key.encode(), int(value)))


def qt_set_stream(h, stream_ptr: Optional[int]):
    _check(h, load().qt_set_stream(h, ctypes.c_void_p(stream_ptr or 0)))


def qt_num_segments(h) -> int:
    v = ctypes.c_int32()
    _check(h, load().qt_num_segments(h, ctypes.byref(v)))
    return v.value


def qt_segment_info(h, seg: int, nparts: int):
    fl, nl, npass = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    F = np.zeros(nparts, np.uint8)
    Wk = np.zeros(nparts, np.uint8)
    _check(h, load().qt_segment_info(h, seg, ctypes.byref(fl), ctypes.byref(nl), ctypes.byref(npass),
                                     F.ctypes.data, Wk.ctypes.data))
    return {"first_level": fl.value, "nlevels": nl.value, "npasses": npass.value, "dirty": F.astype(bool),
            "worklist": Wk.astype(bool)}


def qt_segment_touched(h, seg: int, nparts: int) -> np.ndarray:
    T = np.zeros(nparts, np.uint8)
    _check(h, load().qt_segment_touched(h, seg, T.ctypes.data))
    return T.astype(bool)


def qt_last_error(h) -> str:
    m = load().qt_last_error(h)
    return m.decode() if m else ""


# ------------------------------------------------------------ convenience

class Circuit:
    """Owning wrapper: ``Circuit(n, 'c128df', log2_partition)``."""

    def __init__(self, n: int, dtype: str = "c128", log2_partition: Optional[int] = None):
        self.n = n
        self.dtype = dtype
        self.p = min(n, 16) if log2_partition is None else log2_partition
        self.h = qt_create(n, DTYPES[dtype], self.p)

    @property
    def nparts(self) -> int:
        return 1 << (self.n - self.p)

    def close(self):
        if self.h:
            qt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def num_levels(self):
        return qt_num_levels(self.h)

    def num_gates(self):
        return qt_num_gates(self.h)

    def insert_level(self, pos: int):
        qt_insert_level(self.h, pos)

    def remove_level(self, pos: int):
        qt_remove_level(self.h, pos)

    def insert_gate(self, level: int, gate) -> int:
        return qt_insert_gate(self.h, level, gate)

    def remove_gate(self, level: int, gid: int):
        qt_remove_gate(self.h, level, gid)

    def replace_gate(self, level: int, gid: int, gate) -> int:
        return qt_replace_gate(self.h, level, gid, gate)

    def update_state(self, force_full: bool = False):
        return qt_update_state(self.h, force_full)

    def set_option(self, key: str, value: int):
        qt_set_option(self.h, key, value)

    def set_stream(self, stream_ptr: Optional[int]):
        qt_set_stream(self.h, stream_ptr)

    def read_amplitudes(self, first: int = 0, count: Optional[int] = None, out: Optional[np.ndarray] = None):
        if count is None:
            count = (1 << self.n) - first
        dt = np.complex64 if self.dtype == "c64" else np.complex128
        if out is None:
            out = np.empty(count, dt)
        return qt_read_amplitudes(self.h, first, count, out)

    def read_amplitudes_device(self, first: int, count: int, device_ptr: int):
        qt_read_amplitudes_device(self.h, first, count, device_ptr)

    def read_amplitudes_async(self, out: np.ndarray, first: int = 0, count: Optional[int] = None):
        """Start copying amplitudes into `out` (kept referenced until read_wait)."""
        if count is None:
            count = (1 << self.n) - first
        assert out.size >= count
        self._async_out = out
        return qt_read_amplitudes_async(self.h, first, count, out)

    def read_wait(self):
        qt_read_wait(self.h)
        self._async_out = None

    def norm(self) -> float:
        return qt_norm(self.h)

    def release_device(self):
        """Free the device state and checkpoints; the next update re-simulates."""
        qt_release_device(self.h)

    def device_bytes(self) -> int:
        return qt_device_bytes(self.h)

    def fidelity(self, other: "Circuit") -> float:
        return qt_fidelity(self.h, other.h)

    def max_abs_diff(self, other: "Circuit") -> float:
        return qt_max_abs_diff(self.h, other.h)

    def probabilities(self, qubits) -> np.ndarray:
        return qt_probabilities(self.h, qubits)

    def num_segments(self) -> int:
        return qt_num_segments(self.h)

    def segment_info(self, seg: int):
        return qt_segment_info(self.h, seg, self.nparts)

    def segment_touched(self, seg: int) -> np.ndarray:
        return qt_segment_touched(self.h, seg, self.nparts)

    def load_levels(self, levels):
        """Append levels of gates; returns the gate ids level by level."""
        ids = []
        base = self.num_levels()
        for k, lv in enumerate(levels):
            self.insert_level(base + k)
            ids.append([self.insert_gate(base + k, g) for g in lv])
        return ids


def apply_edit_ops(circ: Circuit, ops, handle_to_id: dict):
    """Replay edit ops produced by workloads.edit_round on a library circuit."""
    for op in ops:
        kind = op[0]
        if kind == "insert_level":
            circ.insert_level(op[1])
        elif kind == "insert":
            _, lvl, h, g = op
            handle_to_id[h] = circ.insert_gate(lvl, g)
        elif kind == "remove":
            _, lvl, h = op
            circ.remove_gate(lvl, handle_to_id.pop(h))
        elif kind == "replace":
            _, lvl, h, nh, g = op
            handle_to_id[nh] = circ.replace_gate(lvl, handle_to_id.pop(h), g)
        else:
            raise ValueError(kind)


# ---------------------------------------------------------------- serving

def qt_release_device(h):
    _check(h, load().qt_release_device(h))


def qt_device_bytes(h) -> int:
    v = ctypes.c_int64()
    _check(h, load().qt_device_bytes(h, ctypes.byref(v)))
    return v.value


def make_edit(op) -> qt_edit:
    """('insert_level', level) | ('insert', level, gate) | ('remove', level, id)
    | ('replace', level, id, gate) | ('remove_level', level)."""
    e = qt_edit()
    kind = op[0]
    e.level = int(op[1])
    if kind == "insert_level":
        e.kind = QT_EDIT_INSERT_LEVEL
    elif kind == "remove_level":
        e.kind = QT_EDIT_REMOVE_LEVEL
    elif kind == "insert":
        e.kind = QT_EDIT_INSERT_GATE
        e.gate = make_qt_gate(op[2])
    elif kind == "remove":
        e.kind = QT_EDIT_REMOVE_GATE
        e.id = int(op[2])
    elif kind == "replace":
        e.kind = QT_EDIT_REPLACE_GATE
        e.id = int(op[2])
        e.gate = make_qt_gate(op[3])
    else:
        raise ValueError(kind)
    return e


class Server:
    """Thin wrapper of qt_server_*: requests are lists of edit tuples (see
    make_edit) followed by an incremental update of one circuit."""

    def __init__(self, workers: int = 8, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(None, load().qt_server_create(workers, hbm_budget_bytes, ctypes.byref(h)))
        self.h = h

    def add_circuit(self, circ: "Circuit") -> int:
        slot = ctypes.c_int32()
        _check(None, load().qt_server_add_circuit(self.h, circ.h, ctypes.byref(slot)))
        return slot.value

    def submit(self, slot: int, ops) -> int:
        arr = (qt_edit * max(len(ops), 1))(*[make_edit(o) for o in ops])
        t = ctypes.c_uint64()
        _check(None, load().qt_server_submit(self.h, slot, len(ops), arr, ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int) -> dict:
        r = qt_request_result()
        _check(None, load().qt_server_wait(self.h, ticket, ctypes.byref(r)))
        return {"status": r.status, "circuit": r.circuit, "queue_ms": r.queue_ms, "service_ms": r.service_ms,
                "latency_ms": r.latency_ms, "stats": stats_dict(r.stats),
                "new_ids": [r.new_ids[k] for k in range(r.n_new_ids)]}

    def info(self) -> dict:
        rb, ev, q = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(None, load().qt_server_info(self.h, ctypes.byref(rb), ctypes.byref(ev), ctypes.byref(q)))
        return {"resident_bytes": rb.value, "evictions": ev.value, "queued": q.value}

    def close(self):
        if self.h:
            load().qt_server_destroy(self.h)
            self.h = None
