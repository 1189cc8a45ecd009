"""Complex64 bulk simulation with a drift check that falls back to complex128.

A complex64 state costs half the HBM traffic and a quarter of the arithmetic
of a float-float complex128 one, but its rounding error grows with depth.
``AdaptiveCircuit`` runs a circuit in complex64 and, after every update,
measures the drift of the state's norm from 1 (an FP64-class reduction on the
device; a unitary circuit keeps the norm at exactly 1, so the deviation is
pure rounding).  When the drift exceeds ``drift_tol`` it rebuilds the same
circuit in complex128 (float-float) and stays there.  Edits go through the
wrapper, which keeps the level list so the rebuild needs no replay log.
The host logic here only decides; every state update runs in libqtask.so.
"""
from __future__ import annotations

from typing import List, Optional

from . import binding as B


class AdaptiveCircuit:
    def __init__(self, n: int, log2_partition: Optional[int] = None, drift_tol: float = 1e-6, **options):
        self.n = n
        self.p = min(n, 16) if log2_partition is None else log2_partition
        self.drift_tol = drift_tol
        self.options = dict(options)
        self.levels: List[list] = []   # (gate id, gate) per level, mirrored
        self.dtype = "c64"
        self.circuit = self._make("c64")
        self.drift: Optional[float] = None
        self.switched_at_update: Optional[int] = None
        self.updates = 0

    def _make(self, dtype: str) -> B.Circuit:
        c = B.Circuit(self.n, dtype, self.p)
        for k, v in self.options.items():
            c.set_option(k, v)
        return c

    # modifiers (same meaning as the C ABI's)
    def insert_level(self, pos: int):
        self.circuit.insert_level(pos)
        self.levels.insert(pos, [])

    def insert_gate(self, level: int, gate) -> int:
        gid = self.circuit.insert_gate(level, gate)
        self.levels[level].append((gid, gate))
        return gid

    def remove_gate(self, level: int, gid: int):
        self.circuit.remove_gate(level, gid)
        self.levels[level] = [(i, g) for i, g in self.levels[level] if i != gid]

    def load_levels(self, levels):
        base = len(self.levels)
        for k, lv in enumerate(levels):
            self.insert_level(base + k)
            for g in lv:
                self.insert_gate(base + k, g)

    def update_state(self, force_full: bool = False):
        st = self.circuit.update_state(force_full)
        self.updates += 1
        if self.dtype == "c64":
            self.drift = abs(self.circuit.norm() - 1.0)
            if self.drift > self.drift_tol:
                self._switch()
                st = self.circuit.update_state()
        return st

    def _switch(self):
        old = self.circuit
        self.circuit = self._make("c128df")
        remap = []
        for k, lv in enumerate(self.levels):
            self.circuit.insert_level(k)
            remap.append([(self.circuit.insert_gate(k, g), g) for _, g in lv])
        self.levels = remap
        old.close()
        self.dtype = "c128df"
        self.switched_at_update = self.updates

    def read_amplitudes(self, first: int = 0, count: Optional[int] = None):
        return self.circuit.read_amplitudes(first, count)

    def close(self):
        self.circuit.close()
