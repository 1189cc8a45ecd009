"""Complex64 bulk simulation whose error is measured, falling back to complex128.

A complex64 state costs half the HBM traffic of a complex128 one and a
fraction of the arithmetic of the float-float complex128 path, but its
rounding error grows with depth (binary32 rounding shrinks the norm by a few
1e-9 per gate, and errors in the amplitudes follow).  The results must stay
within the complex64 contract -- max-abs error <= 1e-5 per amplitude and
fidelity >= 1 - 1e-6 against the FP64 oracle.

``AdaptiveCircuit`` runs the circuit in complex64 and keeps a *shadow*: the
same circuit in float-float complex128 (``QT_C128_DF``, within 1e-12 of the
FP64 oracle, four orders of magnitude inside the complex64 tolerance).  Every
``check_every`` updates the shadow catches up with the edits made since its
last update (an incremental update like any other) and the complex64 state is
compared with it on the device over every amplitude:

* ``max_abs`` = max_b |alpha_b - beta_b| (``qt_max_abs_diff``),
* ``infidelity`` = 1 - |<alpha|beta>|^2 / (<alpha|alpha><beta|beta>)
  (``qt_fidelity``),

both within 1e-12 of the complex64 error against the FP64 oracle.  When
either exceeds ``margin`` times its tolerance (the error keeps growing with
depth, so the switch comes before the contract is broken) the shadow becomes
the circuit and the complex64 copy is dropped: every later result is
float-float.  ``error`` states, for the current result, the measured error,
the update it was measured at and the updates since.  The host logic here
only decides and mirrors edits; every state update runs in libqtask.so.
"""
from __future__ import annotations

from typing import Dict, List, Optional

from . import binding as B

C64_MAX_ABS_TOL = 1e-5
C64_INFIDELITY_TOL = 1e-6
C128_TOL = 1e-12


class AdaptiveCircuit:
    def __init__(self, n: int, log2_partition: Optional[int] = None, check_every: int = 1, margin: float = 0.5,
                 max_abs_tol: float = C64_MAX_ABS_TOL, infidelity_tol: float = C64_INFIDELITY_TOL, **options):
        if check_every < 1:
            raise ValueError("check_every must be >= 1")
        self.n = n
        self.p = min(n, 16) if log2_partition is None else log2_partition
        self.check_every = check_every
        self.margin = margin
        self.max_abs_tol = max_abs_tol
        self.infidelity_tol = infidelity_tol
        self.options = dict(options)
        self.fast: Optional[B.Circuit] = self._make("c64")
        self.shadow: B.Circuit = self._make("c128df")
        # caller-facing gate id -> (complex64 id, float-float id); levels hold caller ids
        self._ids: Dict[int, tuple] = {}
        self._next_id = 1
        self.levels: List[List[int]] = []
        self.updates = 0
        self.unchecked = 0
        self.switched_at_update: Optional[int] = None
        self.error: Optional[dict] = None
        self.checks: List[dict] = []

    def _make(self, dtype: str) -> B.Circuit:
        c = B.Circuit(self.n, dtype, self.p)
        for k, v in self.options.items():
            c.set_option(k, v)
        return c

    @property
    def dtype(self) -> str:
        return "c64" if self.fast is not None else "c128df"

    @property
    def circuit(self) -> B.Circuit:
        return self.fast if self.fast is not None else self.shadow

    def _both(self):
        return [c for c in (self.fast, self.shadow) if c is not None]

    # ------------------------------------------------ modifiers (C ABI's meaning)
    def insert_level(self, pos: int):
        for c in self._both():
            c.insert_level(pos)
        self.levels.insert(pos, [])

    def remove_level(self, pos: int):
        for c in self._both():
            c.remove_level(pos)
        for gid in self.levels.pop(pos):
            del self._ids[gid]

    def insert_gate(self, level: int, gate) -> int:
        fid = self.fast.insert_gate(level, gate) if self.fast is not None else None
        sid = self.shadow.insert_gate(level, gate)
        gid = self._next_id
        self._next_id += 1
        self._ids[gid] = (fid, sid)
        self.levels[level].append(gid)
        return gid

    def remove_gate(self, level: int, gid: int):
        fid, sid = self._ids[gid]
        if self.fast is not None:
            self.fast.remove_gate(level, fid)
        self.shadow.remove_gate(level, sid)
        self.levels[level].remove(gid)
        del self._ids[gid]

    def replace_gate(self, level: int, gid: int, gate) -> int:
        self.remove_gate(level, gid)
        return self.insert_gate(level, gate)

    def load_levels(self, levels) -> List[List[int]]:
        base = len(self.levels)
        out = []
        for k, lv in enumerate(levels):
            self.insert_level(base + k)
            out.append([self.insert_gate(base + k, g) for g in lv])
        return out

    # ------------------------------------------------------------- updates
    def update_state(self, force_full: bool = False) -> dict:
        st = self.circuit.update_state(force_full)
        self.updates += 1
        if self.fast is None:
            self.error = {"dtype": "c128df", "max_abs_tol": C128_TOL, "measured": False,
                          "note": "float-float complex128 results meet 1e-12 max-abs against the FP64 oracle"}
            return st
        self.unchecked += 1
        if self.unchecked >= self.check_every:
            self.check()
        elif self.error is not None:
            self.error = dict(self.error, updates_since_check=self.unchecked)
        return st

    def check(self) -> dict:
        """Bring the shadow up to date and measure the complex64 error over
        the whole state; switch to the shadow when it exceeds the margin."""
        if self.fast is None:
            return self.error
        self.shadow.update_state()
        max_abs = self.fast.max_abs_diff(self.shadow)
        infid = max(0.0, 1.0 - self.fast.fidelity(self.shadow))
        self.unchecked = 0
        rec = {"dtype": "c64", "measured": True, "max_abs": max_abs, "infidelity": infid,
               "checked_at_update": self.updates, "updates_since_check": 0,
               "max_abs_tol": self.max_abs_tol, "infidelity_tol": self.infidelity_tol,
               "reference": "float-float complex128 run of the same gates (within 1e-12 of the FP64 oracle)"}
        self.checks.append(rec)
        if max_abs > self.margin * self.max_abs_tol or infid > self.margin * self.infidelity_tol:
            self.fast.close()
            self.fast = None
            self.switched_at_update = self.updates
            rec = dict(rec, switched=True)
            self.error = {"dtype": "c128df", "max_abs_tol": C128_TOL, "measured": False,
                          "switched_from_c64": rec,
                          "note": "float-float complex128 results meet 1e-12 max-abs against the FP64 oracle"}
        else:
            self.error = rec
        return self.error

    def read_amplitudes(self, first: int = 0, count: Optional[int] = None):
        return self.circuit.read_amplitudes(first, count)

    def close(self):
        for c in self._both():
            c.close()
        self.fast = None
