"""The complex64 tensor-core path: runs of gates on at most five tile qubits
folded into one 32x32 block and applied with tcgen05 MMAs (3xTF32, fp32
accuracy) inside the register kernel.  Checked against the FP64 oracle at
the complex64 tolerances (max-abs 1e-5, fidelity 1 - 1e-6), against the
register-only path, and for incremental == full bit identity over edit
streams (the blocks are planned per segment like every other op)."""
import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W
from gpu_helpers import build_circuit, fidelity, handles_for, max_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


def local_circuit(n, ngates, seed, window=6):
    """Random gates whose qubits mostly come from a sliding window of six, so
    that runs on five qubits (blocks) form; a quarter of the qubits anywhere."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(ngates):
        g = W.random_gate(rng, window, p_multi=0.4)
        lo = int(rng.integers(0, n - window + 1))
        q = [lo + x if rng.random() > 0.25 else None for x in g.qubits]
        used = set(x for x in q if x is not None)
        for i, x in enumerate(q):
            if x is None:
                c = int(rng.integers(n))
                while c in used:
                    c = int(rng.integers(n))
                q[i] = c
                used.add(c)
        gates.append(W.make_gate(g.name, q, g.params))
    return W.asap_levels(n, gates)


@pytest.mark.parametrize("n,p,threshold", [(12, 12, 0), (13, 10, 0), (14, 9, 40), (16, 12, 20)])
def test_blocks_match_oracle_and_register_path(n, p, threshold):
    levels = local_circuit(n, 300, seed=n * 7 + threshold)
    want = oracle.simulate(n, W.flatten(levels))
    tc, _ = build_circuit(n, levels, "c64", p, tc_blocks=1, tc_threshold=threshold, ckpt_interval=1 << 20)
    st = tc.update_state()
    got = tc.read_amplitudes()
    assert max_err(got, want) <= 1e-5 and 1 - fidelity(got, want) <= 1e-6
    reg, _ = build_circuit(n, levels, "c64", p, ckpt_interval=1 << 20)
    reg.update_state()
    assert tc.max_abs_diff(reg) <= 2e-6
    tc.close()
    reg.close()


def test_blocks_on_the_qft_like_circuit():
    n, p = 16, 12
    levels = W.qft_like_circuit(n, 600, seed=3)
    want = oracle.simulate(n, W.flatten(levels))
    for thr in (0, 40):
        c, _ = build_circuit(n, levels, "c64", p, tc_blocks=1, tc_threshold=thr, ckpt_interval=8)
        c.update_state()
        got = c.read_amplitudes()
        assert max_err(got, want) <= 1e-5 and 1 - fidelity(got, want) <= 1e-6, thr
        c.close()


def test_blocks_incremental_bit_identical_to_full():
    n, p = 13, 9
    levels = local_circuit(n, 250, seed=5)
    model = W.CircuitModel.from_levels(n, levels)
    c, ids = build_circuit(n, levels, "c64", p, tc_blocks=1, tc_threshold=0, ckpt_interval=3)
    h2id = handles_for(ids)
    c.update_state()
    rng = np.random.default_rng(6)
    for r in range(6):
        ops = W.edit_round(rng, model, 0.4, int(rng.integers(1, 6)))
        B.apply_edit_ops(c, ops, h2id)
        st = c.update_state()
        inc = c.read_amplitudes()
        c.update_state(force_full=True)
        full = c.read_amplitudes()
        assert np.array_equal(inc.view(np.uint8), full.view(np.uint8)), r
        assert max_err(inc, oracle.simulate(n, model.gates())) <= 1e-5, r
    c.close()
