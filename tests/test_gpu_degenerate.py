"""GPU edge cases of the update semantics: circuits with no gates, levels
with no gates, updates with nothing pending, edits that cancel before the
update, and a circuit whose every gate is removed.

With no gate to apply the state is |0...0> exactly (amplitude 0 is 1, every
other amplitude 0, in every dtype), and an update with no pending edit
launches nothing and leaves the state's bits as they were.  An edit stream
that ends with an empty circuit must bring the incremental state back to
|0...0> bit for bit, like a full re-simulation."""
import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W
from gpu_helpers import DTYPES, TOL, build_circuit, max_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


def basis_zero(n):
    z = np.zeros(1 << n, np.complex128)
    z[0] = 1.0
    return z


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,p", [(1, 0), (7, 3), (14, 8)])
def test_circuit_without_gates_is_the_zero_state(dtype, n, p):
    c = B.Circuit(n, dtype, p)
    st = c.update_state()
    assert st["passes_total"] == 0
    assert np.array_equal(c.read_amplitudes().astype(np.complex128), basis_zero(n))
    # levels that hold no gate change nothing either
    for _ in range(3):
        c.insert_level(0)
    c.update_state()
    assert c.num_levels() == 3
    assert np.array_equal(c.read_amplitudes().astype(np.complex128), basis_zero(n))
    assert abs(c.norm() - 1.0) <= 1e-15
    c.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_update_with_nothing_pending_launches_nothing(dtype):
    n, p = 12, 6
    levels = W.random_circuit(n, 150, seed=31, p_multi=0.4)
    c, ids = build_circuit(n, levels, dtype, p, ckpt_interval=3)
    c.update_state()
    before = c.read_amplitudes()
    st = c.update_state()
    assert st["launches"] == 0 and st["passes_run"] == 0
    assert np.array_equal(c.read_amplitudes(), before)
    # an insert and its removal before the update cancel: no work, same bits
    lv = next(l for l in range(len(levels)) if len(levels[l]) < n // 3)
    free = [q for q in range(n) if all(q not in g.qubits for g in levels[lv])]
    c.remove_gate(lv, c.insert_gate(lv, W.make_gate("x", [free[0]])))
    st = c.update_state()
    assert st["launches"] == 0
    assert np.array_equal(c.read_amplitudes(), before)
    assert max_err(before, oracle.simulate(n, W.flatten(levels))) <= TOL[dtype]
    c.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_removing_every_gate_returns_to_the_zero_state(dtype):
    n, p = 11, 5
    levels = W.random_circuit(n, 120, seed=32, p_multi=0.4)
    c, ids = build_circuit(n, levels, dtype, p, ckpt_interval=2)
    c.update_state()
    rng = np.random.default_rng(5)
    remaining = [(lv, gid) for lv, row in enumerate(ids) for gid in row]
    rng.shuffle(remaining)
    # remove the gates in a few incremental rounds, checking each against
    # the oracle and against a full re-simulation
    model = [list(lv) for lv in levels]
    chunks = np.array_split(np.arange(len(remaining)), 4)
    for ch in chunks:
        for k in ch:
            lv, gid = remaining[k]
            pos = ids[lv].index(gid)
            c.remove_gate(lv, gid)
            del ids[lv][pos]
            del model[lv][pos]
        c.update_state()
        inc = c.read_amplitudes()
        assert max_err(inc, oracle.simulate(n, W.flatten(model))) <= TOL[dtype]
        c.update_state(force_full=True)
        assert np.array_equal(inc, c.read_amplitudes())
    assert c.num_gates() == 0
    assert np.array_equal(c.read_amplitudes().astype(np.complex128), basis_zero(n))
    # and with the levels gone as well
    for _ in range(c.num_levels()):
        c.remove_level(0)
    c.update_state()
    assert np.array_equal(c.read_amplitudes().astype(np.complex128), basis_zero(n))
    c.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_passes_whose_gates_cancel_copy_the_state(dtype):
    """Segments holding only a gate and its inverse on one qubit: merged into
    an exact identity and dropped, the fused pass has no ops and copies its
    partitions from one checkpoint to the next.  Edits that make such a pass
    non-empty and empty again stay bit-identical to a full re-simulation."""
    n, p = 12, 8
    levels = [list(lv) for lv in W.random_circuit(n, 40, seed=41, p_multi=0.4)]
    if len(levels) % 2:
        levels.append([W.make_gate("rz", [0], [0.3])])
    first_pair = len(levels)
    for a, b in [("h", "h"), ("z", "z"), ("s", "sdg"), ("t", "tdg"), ("x", "x")]:
        levels += [[W.make_gate(a, [3])], [W.make_gate(b, [3])]]
    levels += [list(lv) for lv in W.random_circuit(n, 40, seed=42, p_multi=0.4)]
    c, ids = build_circuit(n, levels, dtype, p, ckpt_interval=2)  # one pair per segment
    c.update_state()
    assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(levels))) <= TOL[dtype]
    model = [list(lv) for lv in levels]
    for g in (W.make_gate("rx", [3], [0.7]), W.make_gate("h", [3])):
        ids[first_pair][0] = c.replace_gate(first_pair, ids[first_pair][0], g)
        model[first_pair][0] = g
        c.update_state()
        inc = c.read_amplitudes()
        assert max_err(inc, oracle.simulate(n, W.flatten(model))) <= TOL[dtype]
        c.update_state(force_full=True)
        assert np.array_equal(inc, c.read_amplitudes())
    c.close()
