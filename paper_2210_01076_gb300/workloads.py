"""Seeded synthetic circuits and edit streams (inputs only, no simulation math).

This module is the single input generator shared by the tests, the benchmark
and the oracle side; it draws gate kinds, qubits and angles and mirrors the
circuit's level structure so that edit streams can be replayed on both sides.
It contains none of the simulation arithmetic.

Workload shapes (the paper's QASMBench circuits are stood in for by synthetic
circuits of the sizes in its Table 3 and the configurations below):

* random circuits: gates drawn by seed from {h,x,y,z,s,t,rx,ry,rz,u3,cnot,cz,
  swap,ccx} on uniformly random distinct qubits, angles ~ U[0, 2 pi).  With
  ``p_multi=None`` the 14 kinds are uniform; with ``p_multi`` a gate is first
  drawn multi-qubit with that probability, then uniform inside its group.
* levels are formed ASAP (a gate's level is one past the last level that used
  any of its qubits), matching the paper's "one net per level" convention
  (Section IV, incremental experiments).
* QFT-like layers: H on q_j followed by controlled phases CP(pi / 2^k) from
  q_{j+k} to q_j, interleaved with layers of U3 on every qubit and CZ on random
  disjoint pairs.
* edit streams: rounds of 1-5 edits drawn from {insert, remove, replace} at
  uniformly random levels; an insert that conflicts with its level goes into a
  fresh level right after it (the paper's insert_net, Table 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, NamedTuple, Optional, Tuple

import numpy as np

SINGLE = ("h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "u3")
MULTI = ("cnot", "cz", "swap", "ccx")
ALL_KINDS = SINGLE + MULTI
# name -> (targets, controls, angles)
ARITY = {
    "h": (1, 0, 0), "x": (1, 0, 0), "y": (1, 0, 0), "z": (1, 0, 0), "s": (1, 0, 0), "sdg": (1, 0, 0),
    "t": (1, 0, 0), "tdg": (1, 0, 0), "rx": (1, 0, 1), "ry": (1, 0, 1), "rz": (1, 0, 1), "u3": (1, 0, 3),
    "cnot": (1, 1, 0), "cz": (1, 1, 0), "swap": (2, 0, 0), "ccx": (1, 2, 0), "cp": (1, 1, 1),
}


class Gate(NamedTuple):
    name: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    params: Tuple[float, ...] = ()

    @property
    def qubits(self) -> Tuple[int, ...]:
        return tuple(self.targets) + tuple(self.controls)


def make_gate(name: str, qubits, params=()) -> Gate:
    nt, nc, npar = ARITY[name]
    q = tuple(int(x) for x in qubits)
    assert len(q) == nt + nc and len(set(q)) == len(q)
    p = tuple(float(x) for x in params)
    assert len(p) == npar
    return Gate(name, q[:nt], q[nt:], p)


def random_gate(rng: np.random.Generator, n: int, p_multi: Optional[float] = None, kinds=None) -> Gate:
    if kinds is None:
        if p_multi is None:
            pool = [k for k in ALL_KINDS if ARITY[k][0] + ARITY[k][1] <= n]
            name = pool[rng.integers(len(pool))]
        else:
            multi = [k for k in MULTI if ARITY[k][0] + ARITY[k][1] <= n]
            if multi and rng.random() < p_multi:
                name = multi[rng.integers(len(multi))]
            else:
                name = SINGLE[rng.integers(len(SINGLE))]
    else:
        name = kinds[rng.integers(len(kinds))]
    nt, nc, npar = ARITY[name]
    q = rng.choice(n, size=nt + nc, replace=False)
    params = tuple(float(x) for x in rng.uniform(0.0, 2.0 * math.pi, size=npar))
    return make_gate(name, q, params)


def asap_levels(n: int, gates: List[Gate]) -> List[List[Gate]]:
    """Group a gate sequence into ASAP levels (disjoint qubits per level)."""
    last = [-1] * n
    levels: List[List[Gate]] = []
    for g in gates:
        lv = 1 + max(last[q] for q in g.qubits)
        while len(levels) <= lv:
            levels.append([])
        levels[lv].append(g)
        for q in g.qubits:
            last[q] = lv
    return levels


def random_circuit(n: int, ngates: int, seed: int, p_multi: Optional[float] = None) -> List[List[Gate]]:
    rng = np.random.default_rng(seed)
    return asap_levels(n, [random_gate(rng, n, p_multi) for _ in range(ngates)])


def batch_circuits(count: int, rng: np.random.Generator, p_multi: float = 0.4) -> List[Tuple[int, List[List[Gate]]]]:
    """The batched-synthesis shape: `count` circuits, qubit counts uniform in
    [10, 20], ASAP depths uniform in [50, 400]; gates are drawn until the
    next one would reach the drawn depth.  Returns (n, levels) pairs."""
    out = []
    for _ in range(count):
        n = int(rng.integers(10, 21))
        depth = int(rng.integers(50, 401))
        gates, last = [], [-1] * n
        while True:
            g = random_gate(rng, n, p_multi)
            lv = 1 + max(last[q] for q in g.qubits)
            if lv >= depth:
                break
            for q in g.qubits:
                last[q] = lv
            gates.append(g)
        out.append((n, asap_levels(n, gates)))
    return out


_INVERSE_NAME = {"s": "sdg", "sdg": "s", "t": "tdg", "tdg": "t"}


def inverse_gate(g: Gate) -> Gate:
    """The gate's inverse under the rotation conventions of the gate table:
    rotations and CP negate their angle, U3(theta, phi, lam) becomes
    U3(-theta, -lam, -phi), S/T become their daggers, the rest are
    self-inverse."""
    if g.name in ("rx", "ry", "rz", "cp"):
        return g._replace(params=(-g.params[0],))
    if g.name == "u3":
        th, ph, la = g.params
        return g._replace(params=(-th, -la, -ph))
    return g._replace(name=_INVERSE_NAME.get(g.name, g.name))


def inverse_levels(levels: List[List[Gate]]) -> List[List[Gate]]:
    """Levels of the inverse circuit: levels in reverse order, each gate
    inverted (gates within a level act on disjoint qubits and commute)."""
    return [[inverse_gate(g) for g in lv] for lv in reversed(levels)]


def qft_like_circuit(n: int, ngates: int, seed: int) -> List[List[Gate]]:
    """QFT-style H + controlled-phase ladders interleaved with random U3/CZ layers."""
    rng = np.random.default_rng(seed)
    seq: List[Gate] = []
    j = 0
    while len(seq) < ngates:
        # one QFT column on qubit j
        seq.append(make_gate("h", [j]))
        for k in range(1, n - j):
            if len(seq) >= ngates:
                break
            seq.append(make_gate("cp", [j, j + k], [math.pi / (1 << k)]))
        j = (j + 1) % n
        if j % 4 == 0 and len(seq) < ngates:
            # a random layer: U3 on every qubit, then CZ on random disjoint pairs
            for q in range(n):
                if len(seq) >= ngates:
                    break
                seq.append(make_gate("u3", [q], rng.uniform(0.0, 2.0 * math.pi, size=3)))
            perm = rng.permutation(n)
            for a in range(0, n - 1, 2):
                if len(seq) >= ngates:
                    break
                seq.append(make_gate("cz", [perm[a], perm[a + 1]]))
    return asap_levels(n, seq[:ngates])


def flatten(levels) -> List[Gate]:
    return [g for lv in levels for g in lv]


# --------------------------------------------------------------- edit streams


@dataclass
class CircuitModel:
    """Mirror of a circuit's levels holding (handle, Gate) pairs.

    Handles are logical integers assigned here; the library's own gate ids are
    mapped to them by whoever replays the stream."""
    n: int
    levels: List[List[Tuple[int, Gate]]] = field(default_factory=list)
    next_handle: int = 0

    @classmethod
    def from_levels(cls, n: int, levels) -> "CircuitModel":
        m = cls(n)
        for lv in levels:
            m.levels.append([])
            for g in lv:
                m.levels[-1].append((m.next_handle, g))
                m.next_handle += 1
        return m

    def conflicts(self, level: int, gate: Gate, ignore: Optional[int] = None) -> bool:
        used = set()
        for h, g in self.levels[level]:
            if h != ignore:
                used.update(g.qubits)
        return bool(used.intersection(gate.qubits))

    def gates(self) -> List[Gate]:
        return [g for lv in self.levels for _, g in lv]

    def num_gates(self) -> int:
        return sum(len(lv) for lv in self.levels)


def _replacement(rng: np.random.Generator, g: Gate) -> Gate:
    """Same qubits, a kind of the same arity (rotations may keep their kind with new angles)."""
    q = list(g.qubits)
    same = [k for k in ARITY if k in ALL_KINDS and ARITY[k][0] + ARITY[k][1] == len(q)]
    name = same[rng.integers(len(same))]
    rng.shuffle(q)
    nt, nc, npar = ARITY[name]
    return make_gate(name, q, rng.uniform(0.0, 2.0 * math.pi, size=npar))


def edit_round(rng: np.random.Generator, model: CircuitModel, p_multi: Optional[float], nedits: int):
    """Draw ``nedits`` edits, apply them to ``model`` and return them as ops:
    ('insert_level', pos) | ('insert', level, handle, Gate) | ('remove', level, handle)
    | ('replace', level, handle, new_handle, Gate)."""
    ops = []
    for _ in range(nedits):
        kind = ("insert", "remove", "replace")[rng.integers(3)]
        nonempty = [i for i, lv in enumerate(model.levels) if lv]
        if kind != "insert" and not nonempty:
            kind = "insert"
        if kind == "insert":
            if not model.levels:
                model.levels.append([])
                ops.append(("insert_level", 0))
            lvl = int(rng.integers(len(model.levels)))
            g = random_gate(rng, model.n, p_multi)
            if model.conflicts(lvl, g):
                lvl += 1
                model.levels.insert(lvl, [])
                ops.append(("insert_level", lvl))
            h = model.next_handle
            model.next_handle += 1
            model.levels[lvl].append((h, g))
            ops.append(("insert", lvl, h, g))
        elif kind == "remove":
            lvl = nonempty[int(rng.integers(len(nonempty)))]
            k = int(rng.integers(len(model.levels[lvl])))
            h, _ = model.levels[lvl].pop(k)
            ops.append(("remove", lvl, h))
        else:
            lvl = nonempty[int(rng.integers(len(nonempty)))]
            k = int(rng.integers(len(model.levels[lvl])))
            h, g = model.levels[lvl][k]
            ng = _replacement(rng, g)
            nh = model.next_handle
            model.next_handle += 1
            model.levels[lvl][k] = (nh, ng)
            ops.append(("replace", lvl, h, nh, ng))
    return ops


def edit_stream(model: CircuitModel, rounds: int, seed: int, p_multi: Optional[float] = 0.4,
                min_edits: int = 1, max_edits: int = 5):
    """Yield ``rounds`` lists of edit ops, mutating ``model`` as it goes."""
    rng = np.random.default_rng(seed)
    for _ in range(rounds):
        k = int(rng.integers(min_edits, max_edits + 1))
        yield edit_round(rng, model, p_multi, k)


def rotation_edit(rng: np.random.Generator, levels: List[List[Gate]]):
    """The batched loop's parameter edit: a uniformly chosen RZ or RY gate
    has its angle moved by N(0, 0.1).  Returns (level, index, new gate), or
    None when the circuit has no such gate."""
    cand = [(l, j) for l, lv in enumerate(levels) for j, g in enumerate(lv) if g.name in ("rz", "ry")]
    if not cand:
        return None
    l, j = cand[int(rng.integers(len(cand)))]
    g = levels[l][j]
    return l, j, g._replace(params=(g.params[0] + float(rng.normal(0.0, 0.1)),))


def tail_edit(rng: np.random.Generator, levels: List[List[Gate]], tail: float = 0.1):
    """The deep circuit's single-gate edit in the last `tail` of the levels:
    a one-qubit gate becomes a small RZ, a two-qubit phase a controlled phase
    of a nearby angle (CZ counts as CP(pi)).  Returns (level, index, new
    gate), or None when the drawn level is empty."""
    L = len(levels)
    lvl = int(rng.integers(int((1.0 - tail) * L), L))
    if not levels[lvl]:
        return None
    k = int(rng.integers(len(levels[lvl])))
    g = levels[lvl][k]
    delta = float(rng.normal(0.0, 0.1))
    if len(g.qubits) == 1:
        return lvl, k, make_gate("rz", [g.qubits[0]], [delta])
    theta = g.params[0] if g.name == "cp" else math.pi
    return lvl, k, make_gate("cp", list(g.targets) + list(g.controls), [theta + delta])


def random_state(n: int, seed: int, dtype=np.complex128) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return (v / np.linalg.norm(v)).astype(dtype)
