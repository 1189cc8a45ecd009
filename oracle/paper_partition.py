"""The paper's own block-partition and range-intersection rules, restated.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Pure Python, meant for
the small worked example of the paper (5 qubits, block size 4).

* ``paper_partitions`` -- Section III-C (task decomposition).  A
  non-superposition gate (swaps and scalings: X/CNOT/CCX/Y, SWAP, the phase
  gates, RZ) touches a fixed bit pattern; its B-sized tasks are formed by
  filling the free bits with consecutive values starting at multiples of B.
  Each task covers the memory region [lowest, highest] of the states it
  reads or writes; consecutive tasks whose regions overlap merge into one
  partition.  A superposition gate (H, RX, RY, U3) instead splits the vector
  into equal one-block partitions behind a sync task.
* ``PaperGraph`` -- Sections III-D and III-E.  Rows of partitions in circuit
  order; a partition's successors (predecessors) are found by walking forward
  (backward) row by row, taking every partition whose block range intersects
  the blocks still uncovered, until none remain.  Removing a gate puts the
  successors of its partitions on the frontier; inserting one puts its own
  partitions there; the update re-simulates everything reachable from the
  frontier.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

SWAP_KINDS = {"x", "cnot", "ccx", "y"}
SCALE_KINDS = {"z", "s", "sdg", "t", "tdg", "cz", "cp", "rz"}
MXV_KINDS = {"h", "rx", "ry", "u3"}


def _gate_fields(g):
    if isinstance(g, tuple) and not hasattr(g, "name"):
        name, targets, controls = g[0], g[1], g[2]
    else:
        name, targets, controls = g.name, g.targets, g.controls
    return name, list(targets), list(controls)


def gate_mode(g) -> str:
    name, _, _ = _gate_fields(g)
    if name in MXV_KINDS:
        return "mxv"
    if name in SWAP_KINDS or name == "swap":
        return "swap"
    if name in SCALE_KINDS:
        return "scale"
    raise ValueError(name)


def _compose(n: int, fixed: Dict[int, int], free: Sequence[int], v: int) -> int:
    s = 0
    for q, b in fixed.items():
        s |= b << q
    for k, q in enumerate(free):
        s |= ((v >> k) & 1) << q
    return s


def paper_task_regions(n: int, B: int, g) -> List[Tuple[int, int]]:
    """Memory region [lowest, highest state] of each B-sized task of a
    non-superposition gate, in task order (Section III-C)."""
    name, targets, controls = _gate_fields(g)
    if gate_mode(g) == "mxv":
        raise ValueError("superposition gates have no swap/scale tasks")
    mode = gate_mode(g)
    fixed: Dict[int, int] = {}
    if mode == "swap":
        for c in controls:
            fixed[c] = 1
        if name == "swap":
            a, b = targets
            fixed[a], fixed[b] = 0, 1
            flip = (1 << a) | (1 << b)
        else:
            fixed[targets[0]] = 0
            flip = 1 << targets[0]
    else:
        # scaling acts where the gate's non-identity diagonal entries sit: the
        # phase gates scale the states whose named qubits are all 1; RZ
        # scales every state.
        if name != "rz":
            for q in targets + controls:
                fixed[q] = 1
        flip = 0
    free = [q for q in range(n) if q not in fixed]  # ascending = low bits first
    nfree = 1 << len(free)
    regions = []
    for start in range(0, nfree, B):
        states = [_compose(n, fixed, free, v) for v in range(start, min(start + B, nfree))]
        touched = states + [s ^ flip for s in states] if flip else states
        regions.append((min(touched), max(touched)))
    return regions


def paper_partitions(n: int, B: int, g) -> List[Tuple[int, int]]:
    """Block ranges [first, last] of the gate's partitions (Section III-C)."""
    if gate_mode(g) == "mxv":
        return [(b, b) for b in range((1 << n) // B)]
    parts: List[List[int]] = []
    regions = paper_task_regions(n, B, g)
    for lo, hi in regions:
        if parts and lo <= parts[-1][1]:
            parts[-1][1] = max(parts[-1][1], hi)
        else:
            parts.append([lo, hi])
    return [(lo // B, hi // B) for lo, hi in parts]


class PaperGraph:
    """Rows of partitions (one row per gate; a net's superposition gates share
    one row of one-block partitions) and the range-intersection edges."""

    def __init__(self, n: int, B: int):
        self.n, self.B = n, B
        self.rows: List[Tuple[str, List[Tuple[int, int]]]] = []

    def append_row(self, label: str, parts: List[Tuple[int, int]]):
        self.rows.append((label, list(parts)))

    def row_index(self, label: str) -> int:
        return [r[0] for r in self.rows].index(label)

    @staticmethod
    def _blocks(rng: Tuple[int, int]) -> set:
        return set(range(rng[0], rng[1] + 1))

    def _walk(self, row: int, part: Tuple[int, int], step: int):
        """Neighbours of one partition walking in direction ``step``; returns a
        list of (row distance, row label, partition)."""
        remaining = self._blocks(part)
        found = []
        r = row + step
        while remaining and 0 <= r < len(self.rows):
            label, parts = self.rows[r]
            for p in parts:
                hit = remaining & self._blocks(p)
                if hit:
                    found.append((abs(r - row), label, p))
            for p in parts:
                remaining -= self._blocks(p)
            r += step
        return found

    def successors(self, label: str, part):
        return self._walk(self.row_index(label), tuple(part), +1)

    def predecessors(self, label: str, part):
        return self._walk(self.row_index(label), tuple(part), -1)

    def reachable(self, frontier: List[Tuple[str, Tuple[int, int]]]):
        """DFS from the frontier partitions along successor edges (Section III-E)."""
        seen = set()
        stack = [(lab, tuple(p)) for lab, p in frontier]
        while stack:
            lab, p = stack.pop()
            if (lab, p) in seen:
                continue
            seen.add((lab, p))
            for _, slab, sp in self.successors(lab, p):
                stack.append((slab, tuple(sp)))
        return seen
