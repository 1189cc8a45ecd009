"""CPU-side tests of libqtask.so: exported symbols, circuit store and modifier
errors (Section III-B, Table 2), and the dirty-partition tracker (Section
III-E) run in dry-run mode (planning and tracking only, no GPU), pinned to the
paper's worked example and to brute force through the oracle."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "qtask.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qt_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = B.load()
    syms = header_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(B.EXPORTED) == syms


def dry(n, p, dtype="c128df", G=1):
    c = B.Circuit(n, dtype, p)
    c.set_option("dry_run", 1)
    c.set_option("ckpt_interval", G)
    return c


def test_conflict_leaves_circuit_unchanged():
    c = dry(5, 2)
    c.insert_level(0)
    c.insert_gate(0, W.make_gate("cnot", [3, 4]))
    with pytest.raises(B.QtError) as e:
        c.insert_gate(0, W.make_gate("h", [4]))
    assert e.value.status == B.QT_ERR_CONFLICT
    assert c.num_gates() == 1
    gid = c.insert_gate(0, W.make_gate("h", [0]))
    with pytest.raises(B.QtError) as e:
        c.replace_gate(0, gid, W.make_gate("x", [3]))
    assert e.value.status == B.QT_ERR_CONFLICT
    assert c.num_gates() == 2
    new = c.replace_gate(0, gid, W.make_gate("x", [1]))
    assert new != gid and c.num_gates() == 2


def test_argument_errors():
    c = dry(4, 2)
    c.insert_level(0)
    cases = [
        (lambda: c.insert_gate(0, W.Gate("h", (4,), (), ())), B.QT_ERR_ARG),
        (lambda: c.insert_gate(0, W.Gate("cnot", (1,), (1,), ())), B.QT_ERR_ARG),
        (lambda: c.insert_gate(0, W.Gate("cnot", (1,), (), ())), B.QT_ERR_ARG),
        (lambda: c.insert_gate(1, W.make_gate("h", [0])), B.QT_ERR_RANGE),
        (lambda: c.insert_level(5), B.QT_ERR_RANGE),
        (lambda: c.remove_gate(0, 12345), B.QT_ERR_NOT_FOUND),
        (lambda: c.remove_level(3), B.QT_ERR_RANGE),
        (lambda: c.set_option("no_such_option", 1), B.QT_ERR_ARG),
        (lambda: c.set_option("tile_high", 9), B.QT_ERR_ARG),
        (lambda: c.set_option("ckpt_interval", 0), B.QT_ERR_ARG),
        (lambda: c.insert_gate(0, W.Gate("rx", (0,), (), (float("nan"),))), B.QT_ERR_ARG),
    ]
    for fn, status in cases:
        with pytest.raises(B.QtError) as e:
            fn()
        assert e.value.status == status
    with pytest.raises(B.QtError) as e:
        B.qt_create(0, B.QT_C128, 0)
    assert e.value.status == B.QT_ERR_ARG
    with pytest.raises(B.QtError):
        B.qt_create(5, 7, 2)
    with pytest.raises(B.QtError):
        B.qt_create(5, B.QT_C64, 6)


def test_read_while_pending_is_stale():
    c = dry(4, 2)
    c.insert_level(0)
    c.insert_gate(0, W.make_gate("h", [0]))
    with pytest.raises(B.QtError) as e:
        c.read_amplitudes()
    assert e.value.status == B.QT_ERR_STALE


def test_remove_level_and_counts():
    c = dry(6, 3)
    ids = c.load_levels([[W.make_gate("h", [q]) for q in range(6)], [W.make_gate("cnot", [0, 1])]])
    assert c.num_levels() == 2 and c.num_gates() == 7
    c.remove_level(0)
    assert c.num_levels() == 1 and c.num_gates() == 1
    with pytest.raises(B.QtError):
        c.remove_gate(0, ids[0][0])


def fig2(c):
    """Listing 1's circuit: H on q4..q0, then CNOT(t,c) G6..G9 on nets 2..5."""
    ids = c.load_levels([[W.make_gate("h", [q]) for q in (4, 3, 2, 1, 0)],
                         [W.make_gate("cnot", [3, 4])], [W.make_gate("cnot", [1, 4])],
                         [W.make_gate("cnot", [2, 3])], [W.make_gate("cnot", [0, 2])]])
    return ids


def test_fig2_dirty_partitions_are_the_papers_24_amplitudes():
    c = dry(5, 2)  # block size 4 = partitions of 2^2 amplitudes; one net per segment
    ids = fig2(c)
    st = c.update_state()
    assert st["clean_fraction"] == 0.0
    c.remove_gate(3, ids[3][0])                       # remove G8
    c.insert_gate(3, W.make_gate("cnot", [1, 2]))     # insert G10 into net4
    st = c.update_state()
    info = [c.segment_info(s) for s in range(c.num_segments())]
    for s in range(3):
        assert not info[s]["dirty"].any() and not info[s]["worklist"].any()
    want = np.zeros(8, bool)
    want[[1, 2, 3, 5, 6, 7]] = True                   # amplitudes [4,15] u [20,31]
    assert np.array_equal(info[3]["dirty"], want)
    assert np.array_equal(info[3]["worklist"], want)
    assert np.array_equal(info[4]["dirty"], want)     # G9 stays inside those partitions
    amps = sorted(a for q in np.flatnonzero(info[4]["dirty"]) for a in range(4 * q, 4 * q + 4))
    assert amps == list(range(4, 16)) + list(range(20, 32))
    assert st["segments_run"] == 2


def boundary_states(n, model_levels, G):
    """Oracle states after every segment boundary (levels [0, (s+1)G))."""
    out = []
    for s in range((len(model_levels) + G - 1) // G):
        gates = [g for lv in model_levels[: (s + 1) * G] for g in lv]
        out.append(oracle.simulate(n, gates))
    return out


@pytest.mark.parametrize("seed,G,p_multi,fusion", [(1, 1, 0.4, 1), (2, 2, 0.4, 1), (3, 3, None, 1),
                                                    (4, 1, 0.6, 0), (5, 4, 0.4, 1)])
def test_tracker_covers_every_changed_partition(seed, G, p_multi, fusion):
    n, p = 8, 4
    levels = W.random_circuit(n, 40, seed=seed, p_multi=p_multi)
    model = W.CircuitModel.from_levels(n, levels)
    c = dry(n, p, G=G)
    c.set_option("fusion", fusion)
    c.set_option("tile_high", 2)
    ids = c.load_levels(levels)
    handle_to_id = {}
    k = 0
    for lv in ids:
        for gid in lv:
            handle_to_id[k] = gid
            k += 1
    c.update_state()
    before = boundary_states(n, [[g for _, g in lv] for lv in model.levels], G)
    rng = np.random.default_rng(seed)
    for r in range(6):
        ops = W.edit_round(rng, model, p_multi, int(rng.integers(1, 4)))
        B.apply_edit_ops(c, ops, handle_to_id)
        st = c.update_state()
        after = boundary_states(n, [[g for _, g in lv] for lv in model.levels], G)
        assert c.num_segments() == len(after)
        for s in range(len(after)):
            info = c.segment_info(s)
            assert np.all(info["worklist"] >= info["dirty"])
            if s >= len(before):
                assert info["dirty"].all()
                continue
            diff = np.abs(after[s] - before[s]).reshape(1 << (n - p), 1 << p).max(axis=1) > 1e-12
            missing = diff & ~info["dirty"]
            assert not missing.any(), (r, s, np.flatnonzero(missing))
        before = after


def test_segment_touched_closed_forms():
    """Section III-D: a gate changes only the partitions where its controls
    (and a phase's own qubit) above the partition bits can be 1."""
    n, p = 10, 6  # 16 partitions; qubits 6..9 are partition bits 0..3
    c = dry(n, p, G=1)
    c.load_levels([[W.make_gate("cz", [8, 0])], [W.make_gate("ccx", [1, 7, 9])], [W.make_gate("h", [0])],
                   [W.make_gate("cp", [9, 6], [0.3])]])
    c.update_state()
    q = np.arange(16)
    want = [(q >> 2) & 1 == 1, ((q >> 1) & 1 == 1) & ((q >> 3) & 1 == 1), np.ones(16, bool),
            ((q >> 3) & 1 == 1) & (q & 1 == 1)]
    assert c.num_segments() == 4
    for s in range(4):
        assert np.array_equal(c.segment_touched(s), want[s]), s
    with pytest.raises(B.QtError):
        c.segment_touched(4)


@pytest.mark.parametrize("seed,G", [(1, 1), (2, 2), (3, 1)])
def test_untouched_partitions_are_unchanged_by_the_segment(seed, G):
    """What a copy-on-write checkpoint store would share (Section III-F): on
    every partition outside qt_segment_touched the oracle's state after the
    segment equals its state before, bit for bit."""
    n, p = 9, 4
    levels = W.random_circuit(n, 60, seed=seed, p_multi=0.7)
    c = dry(n, p, G=G)
    c.load_levels(levels)
    c.update_state()
    states = [oracle.simulate(n, [])] + boundary_states(n, levels, G)
    shared = 0
    for s in range(c.num_segments()):
        t = c.segment_touched(s)
        same = np.all(states[s + 1].reshape(1 << (n - p), 1 << p) == states[s].reshape(1 << (n - p), 1 << p), axis=1)
        assert np.all(same[~t]), (s, np.flatnonzero(~t & ~same))
        shared += int((~t).sum())
    assert shared > 0


def test_incremental_skips_segments_before_the_edit():
    n, p = 10, 5
    levels = W.random_circuit(n, 120, seed=9, p_multi=0.4)
    c = dry(n, p, G=2)
    ids = c.load_levels(levels)
    full = c.update_state()
    last = len(ids) - 1
    c.remove_gate(last, ids[last][0])
    st = c.update_state()
    assert st["segments_run"] == 1
    assert 0.0 < st["passes_run"] < full["passes_run"]
    assert st["clean_fraction"] > 0.8
    st2 = c.update_state(force_full=True)
    assert st2["clean_fraction"] == 0.0 and st2["amp_updates"] == st2["gates_total"] * (1 << n)


def test_full_amp_update_count():
    n = 9
    c = dry(n, 4, G=3)
    c.load_levels(W.random_circuit(n, 77, seed=2))
    st = c.update_state()
    assert st["amp_updates"] == 77 * (1 << n)
    assert st["hbm_bytes"] == st["partition_passes_run"] * (1 << 4) * 32


def test_no_gpu_update_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c = B.Circuit(4, "c128df", 2)
    c.insert_level(0)
    c.insert_gate(0, W.make_gate("h", [0]))
    with pytest.raises(B.QtError) as e:
        c.update_state()
    assert e.value.status == B.QT_ERR_CUDA


@pytest.mark.timeout(60)
@pytest.mark.parametrize("tile_high", [0, 1, 2])
def test_planner_makes_progress_when_a_gate_exceeds_the_tile(tile_high):
    """A SWAP on two qubits above the tile's low run needs two tile qubits;
    with tile_high < 2 it still gets a pass of its own."""
    n, p = 12, 8
    c = dry(n, p, G=2)
    c.set_option("tile_high", tile_high)
    levels = [[W.make_gate("swap", [9, 11]), W.make_gate("h", [0])], [W.make_gate("ccx", [10, 7, 8])],
              [W.make_gate("swap", [6, 10])]]
    c.load_levels(levels)
    st = c.update_state()
    assert st["passes_total"] >= 3 and st["amp_updates"] == 4 * (1 << n)


def test_checkpoint_budget_sets_the_interval():
    """ckpt_budget: the interval is the smallest whose checkpoints (one state
    vector per segment, plus the initial state) fit the budget, and it stays
    while it still fits (dry runs: planning only)."""
    n = 16
    state = (1 << n) * 8  # complex64
    c = B.Circuit(n, "c64", 10)
    c.set_option("dry_run", 1)
    c.set_option("ckpt_budget", 11 * state)  # 11 state vectors: at most 10 segments

    def seg_sizes():
        return [c.segment_info(s)["nlevels"] for s in range(c.num_segments())]

    c.load_levels([[W.make_gate("h", [l % n])] for l in range(85)])
    c.update_state()
    assert max(seg_sizes()) == 9 and len(seg_sizes()) == 10 and sum(seg_sizes()) == 85
    c.load_levels([[W.make_gate("x", [l % n])] for l in range(5)])
    c.update_state()  # 90 levels still fit at 9 per segment: kept
    assert max(seg_sizes()) == 9 and len(seg_sizes()) == 10 and sum(seg_sizes()) == 90
    c.load_levels([[W.make_gate("x", [0])]])
    c.update_state()  # 91 levels at 9 would need 12 vectors: 10 per segment
    assert max(seg_sizes()) == 10 and len(seg_sizes()) == 10 and sum(seg_sizes()) == 91
    c.set_option("ckpt_budget", 0)
    c.set_option("ckpt_interval", 5)
    c.update_state()
    assert len(seg_sizes()) == 19
    with pytest.raises(B.QtError):
        c.set_option("ckpt_budget", -1)
    c.close()
