"""GPU parity for the register kernel's layout bookkeeping and the IREAL op:
circuits built to stress relabeled X and SWAP gates (their flip and bit
exchange seen by later conditioned ops, diagonals and dense ops on the same
qubits), commuting-op reordering across layout changes, and RX products,
against the FP64 oracle on every dtype and several tile widths."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W
from gpu_helpers import DTYPES, TOL, build_circuit, max_err, prep_levels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


def _stress_levels(n, seed, ngates):
    """Random gates on a few hot qubits: X and SWAP interleaved with CNOT,
    CZ, CP, CCX, diagonals and dense gates that share their qubits."""
    rng = np.random.default_rng(seed)
    hot = list(rng.choice(n, size=min(n, 6), replace=False))
    kinds = ["x", "x", "swap", "swap", "cnot", "cz", "cp", "ccx", "rz", "t", "s", "h", "rx", "ry", "u3", "y"]
    gates = []
    for _ in range(ngates):
        name = kinds[int(rng.integers(len(kinds)))]
        nq = sum(W.ARITY[name][:2])
        pool = hot if rng.random() < 0.8 else list(range(n))
        qs = [int(q) for q in rng.choice(pool, size=nq, replace=False)]
        gates.append(W.make_gate(name, qs, rng.uniform(0, 2 * math.pi, W.ARITY[name][2])))
    return W.asap_levels(n, gates)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("tile_high", [3, 5])
def test_relabels_flips_and_conditions(dtype, tile_high):
    n, p = 13, 9
    for seed in range(4):
        levels = prep_levels(n, seed=seed) + _stress_levels(n, 100 + seed, 160)
        for merge in (0, 1):
            c, _ = build_circuit(n, levels, dtype, p, tile_high=tile_high, merge=merge)
            c.update_state()
            want = oracle.simulate(n, W.flatten(levels))
            assert max_err(c.read_amplitudes(), want) <= TOL[dtype], (seed, merge)
            c.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_rx_products_as_one_op(dtype):
    """RX chains and RX with Z/X/Y neighbours on every qubit role (products
    stay real-diagonal / imaginary-off-diagonal or become dense)."""
    n, p = 11, 8
    rng = np.random.default_rng(17)
    prep = prep_levels(n, seed=7)
    gates = []
    for q in [0, 2, 4, 5, 7, 9, 10]:
        for name in ["rx", "rx", "z", "rx", "x", "rx", "y", "rx"]:
            gates.append(W.make_gate(name, [q], rng.uniform(0, 2 * math.pi, W.ARITY[name][2])))
    levels = prep + W.asap_levels(n, gates)
    for merge in (0, 1):
        c, _ = build_circuit(n, levels, dtype, p, merge=merge)
        c.update_state()
        assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(levels))) <= TOL[dtype], merge
        c.close()


@pytest.mark.parametrize("dtype", ["c128df", "c64"])
def test_incremental_edits_on_relabeled_circuits_are_bit_identical(dtype):
    """Edits that add and remove X / SWAP gates change the relabeling of a
    pass; the incremental result equals a full re-simulation bit for bit."""
    n, p = 13, 9
    levels = prep_levels(n, seed=2) + _stress_levels(n, 77, 200)
    c, ids = build_circuit(n, levels, dtype, p)
    c.update_state()
    rng = np.random.default_rng(3)
    for _ in range(6):
        l = int(rng.integers(len(levels)))
        if ids[l] and rng.random() < 0.5:
            k = int(rng.integers(len(ids[l])))
            c.remove_gate(l, ids[l][k])
            del ids[l][k]
            del levels[l][k]
        else:
            q = [int(x) for x in rng.choice(n, size=2, replace=False)]
            g = W.make_gate("swap", q) if rng.random() < 0.5 else W.make_gate("x", q[:1])
            c.insert_level(l)
            gid = c.insert_gate(l, g)
            ids.insert(l, [gid])
            levels.insert(l, [g])
        c.update_state()
        inc = c.read_amplitudes()
        c.update_state(force_full=True)
        assert np.array_equal(inc, c.read_amplitudes())
    assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(levels))) <= TOL[dtype]
    c.close()


def _qft_with_swaps(n):
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(W.make_gate("h", [j]))
        for m in range(j - 1, -1, -1):
            gates.append(W.make_gate("cp", [j, m], [math.pi / (1 << (j - m))]))
    return gates + [W.make_gate("swap", [i, n - 1 - i]) for i in range(n // 2)]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,p", [(16, 10), (22, 14)])
def test_passes_of_relabels_only(dtype, n, p):
    """A QFT's closing swap network plans into passes that hold nothing but
    relabels (no op runs; the final layout alone moves the amplitudes, in
    place).  Against the oracle, and a re-run gives the same bits."""
    levels = prep_levels(n, seed=1) + W.asap_levels(n, _qft_with_swaps(n))
    c, _ = build_circuit(n, levels, dtype, p)
    c.update_state()
    a = c.read_amplitudes()
    assert max_err(a, oracle.simulate(n, W.flatten(levels), nthreads=oracle.max_threads())) <= TOL[dtype]
    for _ in range(2):
        c.update_state(force_full=True)
        assert np.array_equal(a, c.read_amplitudes())
    c.close()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("opts", [{}, {"tile_high": 3}, {"tma": 1}])
def test_merged_phase_groups(dtype, opts):
    """Runs of phases (controlled-phase ladders with CZ, S, T, Z and phases
    on qubits outside the tile, some behind relabeled X gates) merge into
    one op per run; against the oracle, with incremental edits of a merged
    phase bit-identical to a full re-simulation."""
    n, p = 14, 9
    rng = np.random.default_rng(41)
    gates = []
    for j in range(n):
        gates.append(W.make_gate("h", [j]))
        if j % 3 == 0:
            gates.append(W.make_gate("x", [(j + 5) % n]))
        for k in range(1, n):
            m = (j + k) % n
            name = ["cp", "cp", "cz", "cp"][k % 4]
            par = [float(rng.uniform(0, 2 * math.pi))] if name == "cp" else []
            gates.append(W.make_gate(name, [j, m], par))
        for name in ("s", "t", "z"):
            gates.append(W.make_gate(name, [int(rng.integers(n))]))
    levels = prep_levels(n, seed=4) + W.asap_levels(n, gates)
    c, ids = build_circuit(n, levels, dtype, p, **opts)
    c.update_state()
    want = oracle.simulate(n, W.flatten(levels))
    assert max_err(c.read_amplitudes(), want) <= TOL[dtype]
    for _ in range(3):
        cand = [(l, k) for l, lv in enumerate(levels) for k, g in enumerate(lv) if g.name == "cp"]
        l, k = cand[int(rng.integers(len(cand)))]
        g = levels[l][k]
        ng = g._replace(params=(g.params[0] + 0.3,))
        ids[l][k] = c.replace_gate(l, ids[l][k], ng)
        levels[l][k] = ng
        c.update_state()
        inc = c.read_amplitudes()
        c.update_state(force_full=True)
        assert np.array_equal(inc, c.read_amplitudes())
    assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(levels))) <= TOL[dtype]
    c.close()
