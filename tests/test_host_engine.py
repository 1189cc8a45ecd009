"""Host engine checks that need no GPU (dry runs: the planner, the tracker
and the scheduler run, nothing is launched or allocated).

- A fused pass whose ops all cancel (H then H, Z then Z, S then SDG on one
  qubit, merged into exact identities and dropped) leaves a pass with no ops;
  the register-kernel layout planner must plan it as a plain copy.  Each
  scenario runs in a child process, so that a crash in the library fails the
  test instead of ending the test run.
- The serving loop runs requests of different circuits concurrently on its
  worker threads, but each circuit's requests in submission order, and fails
  a request whose circuit can never fit the memory budget.
- Random edit streams (every edit kind, gate-and-inverse pairs, option
  changes, forced full updates) over random qubit counts, partition sizes
  and dtypes plan without error and keep the circuit's gate count."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_child(body: str):
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        import numpy as np
        from paper_2210_01076_gb300 import binding as B, build as qbuild, workloads as W
        qbuild.build()
        B.load()
    """) + textwrap.dedent(body) + "\nprint('ok')\n"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=240, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), (r.returncode, r.stdout[-2000:], r.stderr[-2000:])


@pytest.mark.parametrize("dtype", ["c128df", "c64", "c128"])
def test_passes_whose_ops_cancel_plan_as_copies(dtype):
    run_child(f"""
        n, p = 12, 8  # tiles of 2^11 / 2^12 amplitudes: the register kernel's planner
        pairs = [("h", "h"), ("z", "z"), ("s", "sdg"), ("t", "tdg"), ("x", "x")]
        levels = []
        for a, b in pairs:
            levels += [[W.make_gate(a, [3])], [W.make_gate(b, [3])]]
        levels += W.random_circuit(n, 60, seed=5, p_multi=0.4)
        c = B.Circuit(n, {dtype!r}, p)
        c.set_option("dry_run", 1)
        c.set_option("ckpt_interval", 2)  # every cancelling pair is a segment of its own
        c.load_levels(levels)
        st = c.update_state(force_full=True)
        assert st["segments_total"] >= len(pairs) and st["passes_total"] >= len(pairs), st
        # the same through edits: a fresh level 0 holding one gate, then its
        # inverse in front of it, one incremental plan after each
        rng = np.random.default_rng(1)
        for k in range(40):
            g = W.make_gate(["h", "x", "z", "s", "t"][k % 5], [int(rng.integers(n))])
            c.insert_level(0)
            c.insert_gate(0, g)
            c.update_state()
            c.insert_level(0)
            c.insert_gate(0, W.inverse_gate(g))
            c.update_state()
        c.close()
    """)


def test_server_runs_each_circuits_requests_in_order():
    run_child("""
        rng = np.random.default_rng(3)
        ns = [int(rng.integers(9, 14)) for _ in range(6)]
        circs, counts = [], []
        for k, n in enumerate(ns):
            lv = W.random_circuit(n, int(rng.integers(60, 160)), seed=100 + k, p_multi=0.4)
            c = B.Circuit(n, "c128df", min(n, 7))
            c.set_option("dry_run", 1)
            c.set_option("ckpt_interval", 2)
            c.load_levels(lv)
            c.update_state()
            circs.append(c)
            counts.append(sum(len(l) for l in lv))
        srv = B.Server(workers=4)
        slots = [srv.add_circuit(c) for c in circs]
        expect, tickets = [], []
        for _ in range(150):
            k = int(rng.integers(len(ns)))
            g = W.random_gate(rng, ns[k], 0.4)
            tickets.append(srv.submit(slots[k], [("insert_level", 0), ("insert", 0, g)]))
            counts[k] += 1
            expect.append((k, counts[k]))
        for t, (k, want) in zip(tickets, expect):
            r = srv.wait(t)
            assert r["status"] == 0 and r["circuit"] == slots[k], r
            # the gates the circuit held when this request's update ran: the
            # requests of one circuit ran in submission order
            assert r["stats"]["gates_total"] == want, (r["stats"]["gates_total"], want)
            assert len(r["new_ids"]) == 1
        srv.close()
        # a budget below one state vector: every request fails, none hangs
        srv = B.Server(workers=2, hbm_budget_bytes=1000)
        slot = srv.add_circuit(circs[0])
        r = srv.wait(srv.submit(slot, [("insert_level", 0), ("insert", 0, W.make_gate("h", [0]))]))
        assert r["status"] == B.QT_ERR_OOM, r
        srv.close()
        for c in circs:
            c.close()
    """)


def test_random_edit_streams_plan_without_errors():
    run_child("""
        def scenario(sc):
            rng = np.random.default_rng(sc)
            n = int(rng.integers(1, 17))
            p = int(rng.integers(0, n + 1))
            c = B.Circuit(n, ["c128", "c64", "c128df"][sc % 3], p)

            def opt(k, v):
                try:
                    c.set_option(k, v)
                except B.QtError:  # e.g. a tile too large for the dtype
                    pass
            opt("dry_run", 1)
            opt("ckpt_interval", int(rng.integers(1, 6)))
            for k, hi in (("fusion", 2), ("merge", 2), ("tile_high", 8), ("reg_kernel", 2)):
                if rng.random() < 0.3:
                    opt(k, int(rng.integers(0, hi)))
            if rng.random() < 0.3:  # checkpoints sized from a budget of state vectors
                opt("ckpt_budget", int(rng.integers(0, 40)) * (1 << n) * 16)
            pm = None if n < 3 else 0.4
            levels = W.random_circuit(n, int(rng.integers(0, 120)), seed=sc, p_multi=pm) if n >= 3 else []
            ids = c.load_levels(levels)
            model = [list(lv) for lv in levels]
            c.update_state()
            for _ in range(int(rng.integers(1, 12))):
                for _ in range(int(rng.integers(1, 6))):
                    L, r = c.num_levels(), rng.random()
                    if r < 0.3 or L == 0:
                        lv = int(rng.integers(L + 1))
                        g = W.random_gate(rng, n, pm) if n >= 3 else W.make_gate("h", [0])
                        c.insert_level(lv)
                        ids.insert(lv, [c.insert_gate(lv, g)])
                        model.insert(lv, [g])
                    elif r < 0.55:
                        lv = int(rng.integers(L))
                        if ids[lv]:
                            k = int(rng.integers(len(ids[lv])))
                            c.remove_gate(lv, ids[lv][k])
                            del ids[lv][k], model[lv][k]
                    elif r < 0.75:
                        lv = int(rng.integers(L))
                        if ids[lv]:
                            k = int(rng.integers(len(ids[lv])))
                            q = list(model[lv][k].qubits)
                            same = [nm for nm in W.ALL_KINDS if sum(W.ARITY[nm][:2]) == len(q)]
                            nm = same[int(rng.integers(len(same)))]
                            ng = W.make_gate(nm, q, rng.uniform(0, 6.28, W.ARITY[nm][2]))
                            ids[lv][k] = c.replace_gate(lv, ids[lv][k], ng)
                            model[lv][k] = ng
                    elif r < 0.85:
                        lv = int(rng.integers(L))
                        c.remove_level(lv)
                        del ids[lv], model[lv]
                    else:  # a gate and its inverse in two fresh levels
                        lv = int(rng.integers(L + 1))
                        g = W.random_gate(rng, n, pm) if n >= 3 else W.make_gate("x", [0])
                        c.insert_level(lv)
                        c.insert_level(lv)
                        ids[lv:lv] = [[c.insert_gate(lv, g)], [c.insert_gate(lv + 1, W.inverse_gate(g))]]
                        model[lv:lv] = [[g], [W.inverse_gate(g)]]
                if rng.random() < 0.1:
                    opt("ckpt_interval", int(rng.integers(1, 6)))
                st = c.update_state(force_full=bool(rng.random() < 0.1))
                assert st["gates_total"] == sum(len(lv) for lv in model), sc
                assert c.num_levels() == len(model), sc
                segs = [c.segment_info(s) for s in range(c.num_segments())]
                assert sum(si["nlevels"] for si in segs) == len(model), sc
            c.close()

        for sc in range(120):
            scenario(sc)
    """)
