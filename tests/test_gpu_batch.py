"""Batched runs (qt_batch_*): many small circuits of uneven qubit counts in
one persistent launch, then CUDA-graph replays after parameter edits."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W
from gpu_helpers import TOL, max_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


def rotation_handles(levels, ids):
    return [(l, k) for l, lv in enumerate(levels) for k, g in enumerate(lv) if g.name in ("rz", "ry")]


@pytest.mark.parametrize("dtype", ["c128df", "c64", "c128"])
def test_batch_matches_oracle_and_replays_after_parameter_edits(dtype):
    rng = np.random.default_rng(7)
    circs, levels, ids = [], [], []
    for k in range(9):
        n = int(rng.integers(10, 15))
        lv = W.random_circuit(n, int(rng.integers(40, 160)), seed=300 + k, p_multi=0.4)
        c = B.Circuit(n, dtype, min(n, 10))
        ids.append(c.load_levels(lv))
        levels.append([list(x) for x in lv])
        circs.append(c)
    batch = B.Batch(circs)
    for rnd in range(4):
        st = batch.run()
        assert st["circuits"] == 9 and st["tiles"] > 0
        if rnd >= 2:
            assert st["graph_replayed"] == 1
        for k, c in enumerate(circs):
            want = oracle.simulate(c.n, W.flatten(levels[k]))
            assert max_err(batch.read_amplitudes(k), want) <= TOL[dtype], (rnd, k)
        # a parameter edit per circuit: a rotation angle moves by N(0, 0.1)
        for k, c in enumerate(circs):
            cand = rotation_handles(levels[k], ids[k])
            if not cand:
                continue
            l, j = cand[int(rng.integers(len(cand)))]
            g = levels[k][l][j]
            ng = g._replace(params=(g.params[0] + float(rng.normal(0.0, 0.1)),))
            ids[k][l][j] = c.replace_gate(l, ids[k][l][j], ng)
            levels[k][l][j] = ng
    # a structural edit: a new gate and level in one circuit -> a new graph
    circs[0].insert_level(0)
    g = W.make_gate("h", [0])
    circs[0].insert_gate(0, g)
    levels[0].insert(0, [g])
    st = batch.run()
    assert st["graph_replayed"] == 0
    assert max_err(batch.read_amplitudes(0), oracle.simulate(circs[0].n, W.flatten(levels[0]))) <= TOL[dtype]
    batch.close()


def test_batch_rejects_mixed_dtypes_and_tiny_circuits():
    a = B.Circuit(10, "c64", 10)
    b = B.Circuit(10, "c128df", 10)
    a.load_levels([[W.make_gate("h", [0])]])
    b.load_levels([[W.make_gate("h", [0])]])
    batch = B.Batch([a, b])
    with pytest.raises(B.QtError):
        batch.run()
    batch.close()
    t = B.Circuit(6, "c64", 6)
    t.load_levels([[W.make_gate("h", [0])]])
    batch = B.Batch([t])
    with pytest.raises(B.QtError):
        batch.run()
    batch.close()


def test_autotuners_pick_a_measured_setting():
    from paper_2210_01076_gb300 import tuning
    n = 14
    levels = W.random_circuit(n, 200, seed=12, p_multi=0.4)
    res = tuning.tune_circuit(n, "c128df", levels, 8, tile_high=(3, 5), merge=(0, 1), repeats=1)
    assert res["best"] is not None and len(res["table"]) == 4
    c = B.Circuit(n, "c128df", 8)
    for k, v in res["best"]["options"].items():
        c.set_option(k, v)
    c.load_levels(levels)
    c.update_state()
    assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(levels))) <= 1e-12
    circs = []
    for k in range(4):
        cc = B.Circuit(11 + k, "c64", 11 + k)
        cc.load_levels(W.random_circuit(11 + k, 80, seed=k))
        circs.append(cc)
    bt = tuning.tune_batch(circs, tile_high=(3, 5), repeats=1)
    assert bt["best"] is not None and len(bt["table"]) == 2


@pytest.mark.parametrize("dtype", ["c128df", "c64"])
def test_batch_passes_of_relabels_only(dtype):
    """Circuits closing with a swap network (passes that hold only relabels)
    in one batched launch, against the oracle."""
    circs, levels = [], []
    for k, n in enumerate([12, 13, 14, 15, 16]):
        rng = np.random.default_rng(k)
        gates = [W.make_gate("u3", [q], rng.uniform(0, 2 * math.pi, 3)) for q in range(n)]
        gates += [W.make_gate("cnot", [q + 1, q]) for q in range(n - 1)]
        for j in range(n - 1, -1, -1):
            gates.append(W.make_gate("h", [j]))
            for m in range(j - 1, -1, -1):
                gates.append(W.make_gate("cp", [j, m], [math.pi / (1 << (j - m))]))
        gates += [W.make_gate("swap", [i, n - 1 - i]) for i in range(n // 2)]
        lv = W.asap_levels(n, gates)
        c = B.Circuit(n, dtype, min(n, 10))
        c.load_levels(lv)
        circs.append(c)
        levels.append(lv)
    batch = B.Batch(circs)
    for _ in range(2):
        batch.run()
        for k, c in enumerate(circs):
            assert max_err(batch.read_amplitudes(k), oracle.simulate(c.n, W.flatten(levels[k]))) <= TOL[dtype], k
    batch.close()
    for c in circs:
        c.close()


@pytest.mark.parametrize("dtype", ["c128df", "c128", "c64"])
def test_batch_tile_of_2_12_amplitudes(dtype):
    """Tiles of 2^12 amplitudes (tile_high 6 above the 2^6 low run of
    16-byte amplitudes, 5 above the 2^7 run of complex64).  The batch kernel
    holds them only for 8-byte amplitudes: for 16-byte ones the run must fail
    with QT_ERR_ARG (not return a state with tiles left undone), and
    complex64 must match the oracle."""
    circs, levels = [], []
    for k, n in enumerate((12, 13)):
        lv = W.random_circuit(n, 90, seed=700 + k, p_multi=0.4)
        c = B.Circuit(n, dtype, min(n, 10))
        c.set_option("tile_high", 5 if dtype == "c64" else 6)
        c.load_levels(lv)
        levels.append(lv)
        circs.append(c)
    batch = B.Batch(circs)
    if dtype == "c64":
        batch.run()
        for k, c in enumerate(circs):
            want = oracle.simulate(c.n, W.flatten(levels[k]))
            assert max_err(batch.read_amplitudes(k), want) <= TOL[dtype], k
    else:
        with pytest.raises(B.QtError) as e:
            batch.run()
        assert e.value.status == B.QT_ERR_ARG
        assert "2^11" in str(e.value) or "tile" in str(e.value)
    batch.close()
    for c in circs:
        c.close()
