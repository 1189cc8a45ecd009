"""Pins of the paper's partition rules (oracle/paper_partition.py) to the
worked example of Figs. 2-11: the printed task regions and partition block
ranges (Section III-C), the predecessor/successor search for inserting G10
and the range intersection after removing G8 (Section III-D), and the
frontiers and the 24 re-simulated amplitudes (Section III-E)."""
import json
import os

import pytest

from oracle.paper_partition import PaperGraph, paper_partitions, paper_task_regions


@pytest.fixture(scope="module")
def ex(golden_dir):
    return json.load(open(os.path.join(golden_dir, "fig2_example.json")))


def cnot(ex, k):
    gd = ex["gates"][k]
    return ("cnot", [gd["target"]], [gd["control"]])


def test_task_regions(ex):
    n, B = ex["n"], ex["block_size"]
    assert [list(r) for r in paper_task_regions(n, B, cnot(ex, "G6"))] == ex["g6_task_regions"]
    assert [list(r) for r in paper_task_regions(n, B, cnot(ex, "G7"))] == ex["g7_regions"]


@pytest.mark.parametrize("k", ["G6", "G7", "G8", "G9", "G10"])
def test_partition_block_ranges(ex, k):
    n, B = ex["n"], ex["block_size"]
    assert [list(r) for r in paper_partitions(n, B, cnot(ex, k))] == ex["partitions"][k]


def test_h_net_partitions(ex):
    n, B = ex["n"], ex["block_size"]
    parts = paper_partitions(n, B, ("h", [0], []))
    assert len(parts) == ex["h_net_partitions"] and all(a == b for a, b in parts)


def graph(ex, order):
    n, B = ex["n"], ex["block_size"]
    g = PaperGraph(n, B)
    g.append_row("net1", paper_partitions(n, B, ("h", [0], [])))
    for k in order:
        g.append_row(k, paper_partitions(n, B, cnot(ex, k)))
    return g


def test_remove_g8_frontier(ex):
    g = graph(ex, ["G6", "G7", "G8", "G9"])
    p0, q0 = ex["g8_first_partition_meets_successor"]
    assert any(tuple(sp) == tuple(q0) for _, _, sp in g.successors("G8", p0))
    frontier = set()
    for part in g.rows[g.row_index("G8")][1]:
        for _, lab, sp in g.successors("G8", part):
            frontier.add((lab, tuple(sp)))
    want = {(lab, tuple(p)) for lab, ps in ex["remove_g8_frontier"].items() for p in ps}
    assert frontier == want


def test_insert_g10_neighbour_search(ex):
    g = graph(ex, ["G6", "G7", "G10", "G9"])
    succ, pred = [], []
    for part in g.rows[g.row_index("G10")][1]:
        succ += g.successors("G10", part)
        pred += g.predecessors("G10", part)
    assert sum(1 for _, lab, _ in succ if lab == "G9") == ex["insert_g10_successors_from_G9"]
    assert sum(1 for d, lab, _ in pred if lab == "G7" and d == 1) == ex["insert_g10_predecessors_from_G7"]
    assert sum(1 for d, lab, _ in pred if lab == "net1" and d == 3) == ex["insert_g10_predecessors_from_net1"]


def test_incremental_update_touches_24_amplitudes(ex):
    B = ex["block_size"]
    g = graph(ex, ["G6", "G7", "G10", "G9"])
    frontier = [(lab, tuple(p)) for lab, ps in ex["remove_g8_frontier"].items() for p in ps]
    frontier += [("G10", p) for p in g.rows[g.row_index("G10")][1]]
    reached = g.reachable(frontier)
    assert len(reached) == ex["updated_partitions"]
    amps = set()
    for _, (lo, hi) in reached:
        amps.update(range(lo * B, (hi + 1) * B))
    want = set()
    for lo, hi in ex["updated_amplitudes"]:
        want.update(range(lo, hi + 1))
    assert amps == want and len(amps) == ex["updated_amplitude_count"]
