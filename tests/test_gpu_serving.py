"""The serving loop (qt_server_*): many resident circuits, requests of a few
edits plus an incremental update, run by worker threads on per-circuit
streams under a device-memory budget.  Each circuit's result must be the
same alone and in the mix (bit for bit), and must match the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


def state_bytes(circ):
    return (1 << circ.n) * (8 if circ.dtype == "c64" else 16)


def budget_shares(states, budget):
    """The server's checkpoint budget per circuit (qtask.h, qt_server): the
    budget less one spare state per circuit, split by state size, at least
    two states each."""
    tot = float(sum(states))
    pool = budget - tot
    return [int(max(pool * s / tot if pool > 0 else 0.0, 2.0 * s)) for s in states]


def mixed_dtype(c):
    return "c64" if c % 2 else "c128df"


def run_scenario(ncirc, nreq, workers, budget, seed, qubits=(9, 14), gates=(60, 160), log2_part=lambda n: min(n, 7),
                 dtype_of=mixed_dtype, ckpt=lambda levels: 2):
    """Requests are inserts into a fresh level, or replaces of a gate present
    from the start (each at most once), so their ids are known up front."""
    rng = np.random.default_rng(seed)
    ns = [int(rng.integers(*qubits)) for _ in range(ncirc)]
    circuits, mirrors, server_c, ids = [], [], [], []
    for c in range(ncirc):
        levels = W.random_circuit(ns[c], int(rng.integers(*gates)), seed=seed * 100 + c, p_multi=0.4)
        mirrors.append([list(lv) for lv in levels])
        circ = B.Circuit(ns[c], dtype_of(c), log2_part(ns[c]))
        circ.set_option("ckpt_interval", ckpt(levels))
        ids.append(circ.load_levels(levels))
        circ.update_state()
        server_c.append(circ)
    # the same circuits again, edited through the direct ABI one request at a time ("alone")
    alone = []
    for c in range(ncirc):
        circ = B.Circuit(ns[c], dtype_of(c), log2_part(ns[c]))
        circ.set_option("ckpt_interval", ckpt(mirrors[c]))
        circ.load_levels([list(lv) for lv in mirrors[c]])
        circ.update_state()
        alone.append((circ, [list(x) for x in ids[c]]))
    if callable(budget):
        budget = budget(None, server_c)
    if budget > 0:
        # the server gives each circuit this checkpoint budget; the copies
        # edited alone get the same, and both are brought to its segments
        # first, so that both plan the same segments (the segment boundaries
        # decide which gates fuse, and so the rounding)
        shares = budget_shares([state_bytes(c) for c in server_c], budget)
        for circ, (acirc, _), share in zip(server_c, alone, shares):
            for x in (circ, acirc):
                x.set_option("ckpt_budget", share)
                x.update_state()
    srv = B.Server(workers=workers, hbm_budget_bytes=budget)
    slots = [srv.add_circuit(circ) for circ in server_c]
    replaced = [set() for _ in range(ncirc)]
    plan = []
    for _ in range(nreq):
        c = int(rng.integers(ncirc))
        n = ns[c]
        ops = []
        for _ in range(int(rng.integers(1, 4))):
            if rng.random() < 0.5:
                lvl = int(rng.integers(len(mirrors[c]) + 1))
                g = W.random_gate(rng, n, 0.4)
                ops.append(("insert_level", lvl))
                ops.append(("insert", lvl, g))
                mirrors[c].insert(lvl, [g])
                ids[c].insert(lvl, [None])
            else:
                cand = [(l, k) for l, lv in enumerate(ids[c]) for k, gid in enumerate(lv)
                        if gid is not None and gid not in replaced[c]]
                l, k = cand[int(rng.integers(len(cand)))]
                old = mirrors[c][l][k]
                q = list(old.qubits)
                same = [nm for nm in W.ALL_KINDS if sum(W.ARITY[nm][:2]) == len(q)]
                nm = same[int(rng.integers(len(same)))]
                ng = W.make_gate(nm, q, rng.uniform(0, 2 * math.pi, W.ARITY[nm][2]))
                ops.append(("replace", l, ids[c][l][k], ng))
                replaced[c].add(ids[c][l][k])
                mirrors[c][l][k] = ng
                ids[c][l][k] = None
        plan.append((c, ops))
    tickets = [srv.submit(slots[c], ops) for c, ops in plan]
    results = [srv.wait(t) for t in tickets]
    info = srv.info()
    srv.close()
    # alone: replay each request with the direct ABI (same ids: both copies
    # assigned ids in the same order)
    for c, ops in plan:
        circ = alone[c][0]
        for op in ops:
            if op[0] == "insert_level":
                circ.insert_level(op[1])
            elif op[0] == "insert":
                circ.insert_gate(op[1], op[2])
            else:
                circ.replace_gate(op[1], op[2], op[3])
        circ.update_state()
    return ns, server_c, alone, mirrors, results, info


def test_server_results_match_alone_and_oracle():
    ns, server_c, alone, mirrors, results, info = run_scenario(ncirc=6, nreq=40, workers=3, budget=0, seed=5)
    assert all(r["status"] == B.QT_OK for r in results)
    assert all(r["latency_ms"] >= r["service_ms"] >= 0 for r in results)
    for c, circ in enumerate(server_c):
        got = circ.read_amplitudes()
        assert np.array_equal(got.view(np.uint8), alone[c][0].read_amplitudes().view(np.uint8)), c
        want = oracle.simulate(ns[c], W.flatten(mirrors[c]))
        tol = 1e-5 if c % 2 else 1e-12
        assert np.max(np.abs(got.astype(np.complex128) - want)) <= tol, c


def test_server_at_served_sizes_against_the_oracle():
    """The served stream's shapes: complex64 circuits of 20-22 qubits and
    about 1000 random gates with checkpoints every ~1/8 of the levels and
    partitions of 2^16, a mix of edit requests on four workers.  Every
    circuit ends bit-identical to the same requests made alone and within the
    complex64 contract of the FP64 oracle over the whole state."""
    ns, server_c, alone, mirrors, results, info = run_scenario(
        ncirc=4, nreq=24, workers=4, budget=0, seed=21, qubits=(20, 23), gates=(900, 1101),
        log2_part=lambda n: 16, dtype_of=lambda c: "c64", ckpt=lambda levels: max(4, -(-len(levels) // 8)))
    assert all(r["status"] == B.QT_OK for r in results)
    assert max(ns) >= 21
    for c, circ in enumerate(server_c):
        got = circ.read_amplitudes()
        assert np.array_equal(got.view(np.uint8), alone[c][0].read_amplitudes().view(np.uint8)), c
        want = oracle.simulate(ns[c], W.flatten(mirrors[c]), nthreads=oracle.max_threads())
        a = got.astype(np.complex128)
        assert np.max(np.abs(a - want)) <= 1e-5, c
        fid = abs(np.vdot(want, a)) ** 2 / (np.vdot(a, a).real * np.vdot(want, want).real)
        assert 1 - fid <= 1e-6, c
    for circ in server_c:
        circ.close()
    for circ, _ in alone:
        circ.close()


def test_server_budget_evicts_and_stays_correct():
    # a budget that admits the largest circuit with its state, one checkpoint
    # and a spare state, but not the seven circuits' states and checkpoints
    # together (they start resident): the first request already evicts, and
    # evicted circuits are re-simulated in full when their turn comes
    def budget_for(_, circs):
        sizes = sorted((state_bytes(c) for c in circs), reverse=True)
        assert 2 * sum(sizes) > 4 * sizes[0]
        return 4 * sizes[0]
    ns, server_c, alone, mirrors, results, info = run_scenario(ncirc=7, nreq=30, workers=2, budget=budget_for,
                                                               seed=8)
    budget = budget_for(None, server_c)
    assert all(r["status"] == B.QT_OK for r in results)
    assert info["evictions"] > 0
    assert info["resident_bytes"] <= budget
    for c, circ in enumerate(server_c):
        # an evicted circuit holds no state on the device: an update with no
        # pending edits re-simulates it in full (a no-op for resident ones)
        circ.update_state()
        assert np.array_equal(circ.read_amplitudes().view(np.uint8), alone[c][0].read_amplitudes().view(np.uint8))


def test_server_budget_shares_keep_every_circuit_resident():
    """A budget that holds every state with a few checkpoints each: the
    server divides it into checkpoint shares, nothing is evicted, the device
    bytes stay within the budget, and each circuit's result is bit-identical
    to the same requests made alone with the same checkpoint share."""
    def budget_for(_, circs):
        return 6 * sum(state_bytes(c) for c in circs)
    ns, server_c, alone, mirrors, results, info = run_scenario(ncirc=7, nreq=40, workers=3, budget=budget_for,
                                                               seed=12)
    assert all(r["status"] == B.QT_OK for r in results)
    assert info["evictions"] == 0
    assert info["resident_bytes"] <= budget_for(None, server_c)
    for c, circ in enumerate(server_c):
        assert np.array_equal(circ.read_amplitudes().view(np.uint8), alone[c][0].read_amplitudes().view(np.uint8)), c
        want = oracle.simulate(ns[c], W.flatten(mirrors[c]))
        tol = 1e-5 if circ.dtype == "c64" else 1e-12
        assert np.max(np.abs(circ.read_amplitudes().astype(np.complex128) - want)) <= tol, c


def test_server_rejects_a_circuit_larger_than_the_budget():
    circ = B.Circuit(14, "c128df", 8)
    circ.load_levels(W.random_circuit(14, 60, seed=1))
    srv = B.Server(workers=1, hbm_budget_bytes=(1 << 14) * 16)  # one state, fewer than its checkpoints
    slot = srv.add_circuit(circ)
    r = srv.wait(srv.submit(slot, []))
    srv.close()
    assert r["status"] == B.QT_ERR_OOM
