"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (max-abs per amplitude): QT_C128 and QT_C128_DF 1e-12, QT_C64
1e-5 with fidelity >= 1 - 1e-6.  Incremental updates must be bit-identical
to a full re-simulation of the edited circuit."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W
from gpu_helpers import DTYPES, TOL, build_circuit, fidelity, handles_for, max_err, prep_levels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


ALL = list(W.ALL_KINDS) + ["sdg", "tdg", "cp"]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", ALL)
def test_each_gate_every_position(dtype, name):
    """Every gate kind on every ordered qubit tuple of a 6-qubit generic state,
    with partitions of 2^2 (targets inside and across partitions) and a tile
    of 2 low + up to 2 high qubits (targets inside and outside the tile)."""
    n, p = 6, 2
    nq = sum(W.ARITY[name][:2])
    rng = np.random.default_rng(abs(hash((name, dtype))) % 2**32)
    prep = prep_levels(n, seed=3)
    for qs in itertools.permutations(range(n), nq):
        g = W.make_gate(name, qs, rng.uniform(0, 2 * math.pi, W.ARITY[name][2]))
        levels = prep + [[g]]
        c, _ = build_circuit(n, levels, dtype, p, tile_high=2)
        c.update_state()
        got = c.read_amplitudes()
        want = oracle.simulate(n, W.flatten(levels))
        assert max_err(got, want) <= TOL[dtype], (name, qs)
        c.close()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("name", ALL)
def test_each_gate_register_kernel_roles(dtype, name):
    """Every gate kind on ordered tuples of qubits that land on every role of
    the register kernel: lane bits (q < 5), register and warp bits (tile
    qubits >= 5, layouts changed by OP_PERM), and qubits outside the tile
    (controls and diagonals uniform over a tile), with partitions of 2^7 so
    that tiles also couple partitions."""
    n, p = 10, 7
    qubits = [0, 3, 5, 6, 8, 9]
    nq = sum(W.ARITY[name][:2])
    rng = np.random.default_rng(abs(hash((name, dtype, "reg"))) % 2**32)
    prep = prep_levels(n, seed=4)
    for qs in itertools.permutations(qubits, nq):
        g = W.make_gate(name, qs, rng.uniform(0, 2 * math.pi, W.ARITY[name][2]))
        # a few neighbours in the same pass so that layouts change around it
        extra = [W.make_gate("h", [q]) for q in range(n) if q not in qs][:3]
        levels = prep + [[g] + extra, [W.make_gate("rx", [qs[0]], [0.4])]]
        want = oracle.simulate(n, W.flatten(levels))
        for tile_high in (2, 4):
            c, _ = build_circuit(n, levels, dtype, p, tile_high=tile_high)
            c.update_state()
            assert max_err(c.read_amplitudes(), want) <= TOL[dtype], (name, qs, tile_high)
            c.close()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("fusion,tile_high,reg", [(0, 6, 1), (1, 1, 1), (1, 3, 1), (1, 6, 1), (1, 6, 0),
                                                   (1, 2, 0)])
def test_random_circuit_config1_shape(dtype, fusion, tile_high, reg):
    """n = 12, 200 gates uniform over the 14 kinds, partitions of 2^8."""
    n, p = 12, 8
    levels = W.random_circuit(n, 200, seed=11)
    c, _ = build_circuit(n, levels, dtype, p, fusion=fusion, tile_high=tile_high, reg_kernel=reg)
    st = c.update_state()
    assert st["amp_updates"] == 200 * (1 << n)
    got = c.read_amplitudes()
    want = oracle.simulate(n, W.flatten(levels))
    assert max_err(got, want) <= TOL[dtype]
    if dtype == "c64":
        assert fidelity(got, want) >= 1 - 1e-6
    assert abs(c.norm() - 1.0) <= (1e-12 if dtype != "c64" else 1e-5)


@pytest.mark.parametrize("dtype", DTYPES)
def test_tma_staged_kernel_parity_and_bit_identity(dtype):
    """The persistent kernel that stages tiles with bulk copies (option tma)
    against the oracle, and incremental against full on it."""
    n, p = 14, 7
    levels = W.random_circuit(n, 250, seed=17, p_multi=0.4)
    c, ids = build_circuit(n, levels, dtype, p, tma=1, ckpt_interval=2)
    c.update_state()
    want = oracle.simulate(n, W.flatten(levels))
    assert max_err(c.read_amplitudes(), want) <= TOL[dtype]
    last = len(ids) - 3
    c.remove_gate(last, ids[last][0])
    c.update_state()
    inc = c.read_amplitudes()
    c.update_state(force_full=True)
    assert np.array_equal(inc.view(np.uint8), c.read_amplitudes().view(np.uint8))


def test_fidelity_and_probabilities():
    n = 14
    levels = W.random_circuit(n, 300, seed=23, p_multi=0.4)
    want = oracle.simulate(n, W.flatten(levels))
    cs = {dt: build_circuit(n, levels, dt, 8)[0] for dt in DTYPES}
    for c in cs.values():
        c.update_state()
    got64 = cs["c64"].read_amplitudes().astype(np.complex128)
    f = cs["c64"].fidelity(cs["c128df"])
    assert abs(f - fidelity(got64, want)) <= 1e-9 and f >= 1 - 1e-6
    assert abs(cs["c128df"].fidelity(cs["c128"]) - 1.0) <= 1e-12
    assert abs(cs["c128"].fidelity(cs["c128df"]) - 1.0) <= 1e-12
    probs = np.abs(want) ** 2
    idx = np.arange(1 << n)
    for qs in ([], [3], [0, 5, 13], [13, 2], list(range(10))):
        ref = np.zeros(1 << len(qs))
        v = np.zeros(1 << n, dtype=np.int64)
        for j, q in enumerate(qs):
            v |= ((idx >> q) & 1) << j
        np.add.at(ref, v, probs)
        for dt, c in cs.items():
            tol = 1e-12 if dt != "c64" else 1e-6
            assert np.max(np.abs(c.probabilities(qs) - ref)) <= tol, (dt, qs)
    with pytest.raises(B.QtError):
        cs["c64"].probabilities([1, 1])


def test_bounded_wait_expiry_reports_timeout():
    """Failure detection without a fault: the staging copies are withheld, the
    kernel's bounded wait expires (1 s), the update reports QT_ERR_TIMEOUT, and
    the context stays usable for the next update."""
    n, p = 12, 8
    levels = W.random_circuit(n, 60, seed=3)
    c, _ = build_circuit(n, levels, "c128df", p, tma=1, test_stall_staging=1)
    with pytest.raises(B.QtError) as e:
        c.update_state()
    assert e.value.status == B.QT_ERR_TIMEOUT
    c.set_option("test_stall_staging", 0)
    c.update_state()
    assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(levels))) <= 1e-12


@pytest.mark.parametrize("dtype", DTYPES)
def test_qft_like_circuit(dtype):
    n, p = 13, 6
    levels = W.qft_like_circuit(n, 400, seed=5)
    c, _ = build_circuit(n, levels, dtype, p)
    c.update_state()
    got = c.read_amplitudes()
    want = oracle.simulate(n, W.flatten(levels))
    assert max_err(got, want) <= TOL[dtype]


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_tiny_states(n):
    for p in range(0, n + 1):
        levels = W.random_circuit(n, 30, seed=n * 10 + p)
        for dtype in DTYPES:
            c, _ = build_circuit(n, levels, dtype, p)
            c.update_state()
            assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(levels))) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_ghz_and_qft_closed_forms(dtype):
    n = 18
    levels = W.asap_levels(n, [W.make_gate("h", [0])] + [W.make_gate("cnot", [q + 1, q]) for q in range(n - 1)])
    c, _ = build_circuit(n, levels, dtype, 10)
    c.update_state()
    a = c.read_amplitudes()
    want = np.zeros(1 << n)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert max_err(a, want) <= TOL[dtype]
    # QFT of a basis state: uniform magnitude, phase 2 pi x y / 2^n
    n, x = 14, 9013
    gates = [W.make_gate("x", [q]) for q in range(n) if x >> q & 1]
    for j in range(n - 1, -1, -1):
        gates.append(W.make_gate("h", [j]))
        for m in range(j - 1, -1, -1):
            gates.append(W.make_gate("cp", [j, m], [math.pi / (1 << (j - m))]))
    for i in range(n // 2):
        gates.append(W.make_gate("swap", [i, n - 1 - i]))
    c, _ = build_circuit(n, W.asap_levels(n, gates), dtype, 7)
    c.update_state()
    y = np.arange(1 << n)
    want = np.exp(2j * math.pi * x * y / (1 << n)) / math.sqrt(1 << n)
    assert max_err(c.read_amplitudes(), want) <= (1e-12 if dtype != "c64" else 1e-5)


def test_fig2_uniform_state_before_and_after_edit():
    c = B.Circuit(5, "c128df", 2)
    c.set_option("ckpt_interval", 1)
    ids = c.load_levels([[W.make_gate("h", [q]) for q in (4, 3, 2, 1, 0)], [W.make_gate("cnot", [3, 4])],
                         [W.make_gate("cnot", [1, 4])], [W.make_gate("cnot", [2, 3])],
                         [W.make_gate("cnot", [0, 2])]])
    c.update_state()
    assert max_err(c.read_amplitudes(), np.full(32, 1 / math.sqrt(32))) <= 1e-15
    c.remove_gate(3, ids[3][0])
    c.insert_gate(3, W.make_gate("cnot", [1, 2]))
    st = c.update_state()
    assert st["segments_run"] == 2 and st["partition_passes_run"] == 12
    assert max_err(c.read_amplitudes(), np.full(32, 1 / math.sqrt(32))) <= 1e-15


def run_edit_stream(n, p, dtype, ngates, rounds, seed, G, p_multi=0.4, check_oracle_every=1, **opts):
    levels = W.random_circuit(n, ngates, seed=seed, p_multi=p_multi)
    model = W.CircuitModel.from_levels(n, levels)
    c, ids = build_circuit(n, levels, dtype, p, ckpt_interval=G, **opts)
    h2id = handles_for(ids)
    c.update_state()
    rng = np.random.default_rng(seed + 1)
    cleans = []
    for r in range(rounds):
        ops = W.edit_round(rng, model, p_multi, int(rng.integers(1, 6)))
        B.apply_edit_ops(c, ops, h2id)
        st = c.update_state()
        cleans.append(st["clean_fraction"])
        inc = c.read_amplitudes()
        c.update_state(force_full=True)
        full = c.read_amplitudes()
        assert np.array_equal(inc.view(np.uint8), full.view(np.uint8)), f"round {r}: incremental != full bits"
        if r % check_oracle_every == 0:
            want = oracle.simulate(n, model.gates(), nthreads=oracle.max_threads())
            assert max_err(inc, want) <= TOL[dtype], r
    # a freshly built circuit with the same levels gives the same bits
    fresh, _ = build_circuit(n, [[g for _, g in lv] for lv in model.levels], dtype, p, ckpt_interval=G, **opts)
    fresh.update_state()
    assert np.array_equal(fresh.read_amplitudes().view(np.uint8), inc.view(np.uint8))
    return cleans


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("G", [1, 3])
def test_incremental_bit_identical_to_full(dtype, G):
    cleans = run_edit_stream(12, 6, dtype, 300, rounds=8, seed=21, G=G)
    assert max(cleans) > 0.0


def test_incremental_bit_identical_unfused():
    run_edit_stream(11, 5, "c128df", 200, rounds=6, seed=4, G=2, fusion=0)


@pytest.mark.parametrize("dtype", DTYPES)
def test_option_changes_between_updates_match_a_fresh_circuit(dtype):
    """The host keeps each segment's plan and each pass's encoded ops for the
    next update; changing a planning option in between must plan anew: after
    edits and an option change the state equals, bit for bit, a circuit built
    fresh with the final gates and options, and the oracle."""
    n, p = 13, 8
    levels = W.random_circuit(n, 260, seed=31, p_multi=0.4)
    model_levels = [list(lv) for lv in levels]
    c, ids = build_circuit(n, levels, dtype, p, ckpt_interval=3)
    c.update_state()
    rng = np.random.default_rng(5)
    opts = {"ckpt_interval": 3}
    for key, val in (("tile_high", 3), ("merge", 0), ("fusion", 0), ("reg_kernel", 0), ("reg_kernel", 1),
                     ("fusion", 1), ("tile_high", 5), ("merge", 1)):
        lvl = int(rng.integers(len(model_levels) + 1))
        g = W.random_gate(rng, n, 0.4)
        c.insert_level(lvl)
        c.insert_gate(lvl, g)
        model_levels.insert(lvl, [g])
        c.update_state()                      # an edit under the old options
        c.set_option(key, val)
        opts[key] = val
        c.update_state()                      # the option change alone
        fresh, _ = build_circuit(n, model_levels, dtype, p, **opts)
        fresh.update_state()
        assert np.array_equal(c.read_amplitudes().view(np.uint8), fresh.read_amplitudes().view(np.uint8)), (key, val)
        fresh.close()
    assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(model_levels))) <= TOL[dtype]
    c.close()


def test_remove_and_insert_levels_incremental():
    n, p = 10, 4
    levels = W.random_circuit(n, 150, seed=2, p_multi=0.4)
    model_levels = [list(lv) for lv in levels]
    c, ids = build_circuit(n, levels, "c128df", p, ckpt_interval=2)
    c.update_state()
    c.remove_level(5)
    del model_levels[5]
    c.insert_level(9)
    c.insert_gate(9, W.make_gate("rx", [3], [0.7]))
    model_levels.insert(9, [W.make_gate("rx", [3], [0.7])])
    c.update_state()
    inc = c.read_amplitudes()
    c.update_state(force_full=True)
    assert np.array_equal(inc, c.read_amplitudes())
    assert max_err(inc, oracle.simulate(n, W.flatten(model_levels))) <= 1e-12


def test_norm_and_device_readout():
    import torch
    n = 16
    levels = W.random_circuit(n, 300, seed=8, p_multi=0.4)
    for dtype in DTYPES:
        c, _ = build_circuit(n, levels, dtype, 10)
        c.update_state()
        want = oracle.simulate(n, W.flatten(levels), nthreads=oracle.max_threads())
        assert abs(c.norm() - oracle.norm(want)) <= (1e-12 if dtype != "c64" else 1e-5)
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        t = torch.empty(1 << n, dtype=tdt, device="cuda")
        c.read_amplitudes_device(0, 1 << n, t.data_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy(), c.read_amplitudes())
        part = c.read_amplitudes(1000, 77)
        assert np.array_equal(part, c.read_amplitudes()[1000:1077])


def test_mem_limit_oom_keeps_state():
    """An update refused for memory (QT_ERR_OOM, before any device work)
    keeps the device state and checkpoints of the last successful update:
    the edits stay pending (reads are stale); undoing them gives the old
    state back bit for bit with no segment recomputed; with more memory the
    same edit then updates incrementally, equal to a full re-simulation."""
    n = 14
    levels = W.random_circuit(n, 100, seed=1)
    c, ids = build_circuit(n, levels, "c128df", 8, ckpt_interval=1)
    c.update_state()
    before = c.read_amplitudes()
    held = c.device_bytes()
    c.set_option("mem_limit", held)  # exactly the state and checkpoints held now
    c.insert_level(0)
    gid = c.insert_gate(0, W.make_gate("h", [0]))  # one more level: one more checkpoint
    with pytest.raises(B.QtError) as e:
        c.update_state()
    assert e.value.status == B.QT_ERR_OOM
    with pytest.raises(B.QtError) as e:
        c.read_amplitudes()
    assert e.value.status == B.QT_ERR_STALE
    # undo: the circuit is the last updated one again
    c.remove_gate(0, gid)
    c.remove_level(0)
    st = c.update_state()
    assert st["segments_run"] == 0 and st["launches"] == 0
    assert np.array_equal(c.read_amplitudes(), before)
    # redo with room for the new checkpoint: incremental from the kept checkpoints
    c.set_option("mem_limit", 0)
    c.insert_level(0)
    c.insert_gate(0, W.make_gate("h", [0]))
    st = c.update_state()
    assert st["passes_run"] <= st["passes_total"]
    after = c.read_amplitudes()
    c.update_state(force_full=True)
    assert np.array_equal(after, c.read_amplitudes())
    want = oracle.simulate(n, [W.make_gate("h", [0])] + W.flatten(levels))
    assert max_err(after, want) <= 1e-12 and max_err(before, want) > 1e-3


def test_timeout_mid_update_forces_a_full_resimulation():
    """An update that fails during its device work (here the bounded wait of
    the bulk-copy staged kernel expires: QT_ERR_TIMEOUT) has rewritten part of
    its checkpoints: reads are stale, and the next update re-runs every pass
    and gives the edited circuit's state."""
    n, p = 12, 8
    levels = W.random_circuit(n, 80, seed=9)
    c, ids = build_circuit(n, levels, "c128df", p, ckpt_interval=2)
    c.update_state()
    c.set_option("tma", 1)
    c.set_option("test_stall_staging", 1)
    c.insert_level(len(levels))
    c.insert_gate(len(levels), W.make_gate("rx", [3], [0.7]))
    with pytest.raises(B.QtError) as e:
        c.update_state()
    assert e.value.status == B.QT_ERR_TIMEOUT
    with pytest.raises(B.QtError) as e:
        c.read_amplitudes()
    assert e.value.status == B.QT_ERR_STALE
    c.set_option("test_stall_staging", 0)
    c.set_option("tma", 0)
    st = c.update_state()
    assert st["passes_run"] == st["passes_total"] and st["segments_run"] == st["segments_total"]
    want = oracle.simulate(n, W.flatten(levels) + [W.make_gate("rx", [3], [0.7])])
    assert max_err(c.read_amplitudes(), want) <= 1e-12


def test_config2_full_size_parity_and_bit_identity():
    """n = 24, 1000 gates (~40 % multi-qubit), partitions of 2^16, complex128
    (float-float) with the benchmark's options: the whole state against the
    multi-threaded oracle, then three edit rounds, each incremental result
    bit-identical to a full re-simulation."""
    n, p = 24, 16
    cleans = run_edit_stream(n, p, "c128df", 1000, rounds=3, seed=2210, G=8, check_oracle_every=3)
    assert len(cleans) == 3
