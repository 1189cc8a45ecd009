"""Precision policy: complex64 results with their error measured against a
float-float complex128 shadow of the same circuit, and the switch to
complex128 when the error approaches the complex64 contract (max-abs 1e-5,
fidelity 1 - 1e-6 against the FP64 oracle).

Binary32 rounding shrinks the norm by a few 1e-9 per gate, so the max-abs
error of a complex64 state grows with depth times the amplitudes' size:
tiny for a 20-qubit circuit of 2000 gates (amplitudes ~1e-3), past the
contract for a 5-qubit circuit of 50 000 gates (amplitudes ~0.2).  Each
decision of the policy is checked against the oracle: where it keeps
complex64, a plain complex64 run of the same gates is within the contract;
where it switches, the plain complex64 run breaks it or is within a factor
two of breaking it (the margin)."""
import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W
from paper_2210_01076_gb300.precision import AdaptiveCircuit
from gpu_helpers import fidelity, max_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


def plain(n, levels, dtype, p, **opts):
    c = B.Circuit(n, dtype, p)
    for k, v in opts.items():
        c.set_option(k, v)
    c.load_levels(levels)
    c.update_state()
    return c


@pytest.mark.parametrize("pair", [("c64", "c128"), ("c64", "c128df"), ("c128df", "c128"), ("c128", "c128")])
def test_max_abs_diff_is_the_largest_amplitude_difference(pair):
    n = 11
    levels = W.random_circuit(n, 150, seed=41, p_multi=0.4)
    a = plain(n, levels, pair[0], 7)
    b = plain(n, levels, pair[1], 7)
    want = float(np.max(np.abs(a.read_amplitudes().astype(np.complex128) - b.read_amplitudes())))
    got = a.max_abs_diff(b)
    assert abs(got - want) <= 1e-12 * max(want, 1e-300) + 1e-300, (got, want)
    if pair[0] == pair[1]:
        assert got == 0.0
    # a state against a different one: the difference of one edited amplitude region
    c = plain(n, levels + [[W.make_gate("x", [0])]], pair[1], 7)
    want = float(np.max(np.abs(a.read_amplitudes().astype(np.complex128) - c.read_amplitudes())))
    assert abs(a.max_abs_diff(c) - want) <= 1e-12
    for x in (a, b, c):
        x.close()


def test_policy_keeps_complex64_where_the_contract_holds():
    """A 20-qubit QFT-like circuit of 2000 gates and a shallow 5-qubit one:
    the measured error stays far inside the contract, the result is the
    complex64 one, and the measured error is the error against the oracle."""
    for n, levels in ((20, W.qft_like_circuit(20, 2000, seed=7)),
                      (5, W.random_circuit(5, 300, seed=5, p_multi=0.4))):
        ac = AdaptiveCircuit(n, min(n, 16), ckpt_interval=1 << 20)
        ac.load_levels(levels)
        ac.update_state()
        assert ac.dtype == "c64" and ac.switched_at_update is None
        e = ac.error
        assert e["measured"] and e["checked_at_update"] == 1 and e["updates_since_check"] == 0
        want = oracle.simulate(n, W.flatten(levels), nthreads=oracle.max_threads())
        got = ac.read_amplitudes()
        err = max_err(got, want)
        assert err <= 1e-5 and 1 - fidelity(got, want) <= 1e-6
        # the shadow is within 1e-12 of the oracle, so the measured error is the oracle's
        assert abs(e["max_abs"] - err) <= 1e-11, (e["max_abs"], err)
        assert e["max_abs"] <= 0.5e-5 and e["infidelity"] <= 0.5e-6
        ac.close()


def test_policy_switches_before_the_contract_breaks():
    """5 qubits, 50 000 random gates: the complex64 error passes half the
    max-abs tolerance, the policy switches to complex128 at the first check,
    and the result then matches the oracle to 1e-12.  A plain complex64 run
    of the same gates confirms the decision against the oracle."""
    n = 5
    levels = W.random_circuit(n, 50000, seed=5, p_multi=0.4)
    want = oracle.simulate(n, W.flatten(levels))
    ref = plain(n, levels, "c64", n, ckpt_interval=1 << 20)
    c64_err = max_err(ref.read_amplitudes(), want)
    ref.close()
    assert c64_err > 0.5e-5, c64_err  # the plain complex64 result is at or past the margin
    ac = AdaptiveCircuit(n, n, ckpt_interval=1 << 20)
    ac.load_levels(levels)
    ac.update_state()
    assert ac.dtype == "c128df" and ac.switched_at_update == 1
    rec = ac.error["switched_from_c64"]
    assert abs(rec["max_abs"] - c64_err) <= 1e-11
    assert max_err(ac.read_amplitudes(), want) <= 1e-12
    # edits after the switch stay complex128 and incremental
    gid = ac.levels[-1][0]
    g = W.make_gate("h", [1])
    ac.insert_level(len(ac.levels))
    ac.insert_gate(len(ac.levels) - 1, g)
    ac.update_state()
    assert ac.dtype == "c128df"
    want = oracle.simulate(n, W.flatten(levels) + [g])
    assert max_err(ac.read_amplitudes(), want) <= 1e-12
    assert gid in ac.levels[-2]
    ac.close()


def test_policy_checks_every_k_updates_through_edits():
    """check_every = 3 over an edit stream: the error record says how many
    updates ago it was measured, each check measures the current state, and
    every complex64 result stays within the contract."""
    n = 12
    levels = W.random_circuit(n, 300, seed=77, p_multi=0.4)
    model = W.CircuitModel.from_levels(n, [list(lv) for lv in levels])
    ac = AdaptiveCircuit(n, 8, check_every=3, ckpt_interval=2)
    ids = ac.load_levels(levels)
    h2id, k = {}, 0
    for lv in ids:
        for gid in lv:
            h2id[k] = gid
            k += 1
    ac.update_state()
    assert ac.error is None  # no check yet
    for rnd, edits in enumerate(W.edit_stream(model, 7, seed=78, p_multi=0.4)):
        B.apply_edit_ops(ac, edits, h2id)
        ac.update_state()
        since = ac.updates % 3
        if ac.updates < 3:
            assert ac.error is None
        else:
            assert ac.error["updates_since_check"] == since
        want = oracle.simulate(n, model.gates())
        got = ac.read_amplitudes()
        assert max_err(got, want) <= 1e-5
        if since == 0:
            assert abs(ac.error["max_abs"] - max_err(got, want)) <= 1e-11
    assert ac.dtype == "c64" and len(ac.checks) == ac.updates // 3
    ac.close()
