"""qt_read_amplitudes_async / qt_read_wait: the copy of a state overlaps the
next edits and update, and delivers the state as it was when the read was
started (a device snapshot), for every dtype."""
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


@pytest.mark.parametrize("dtype", ["c128df", "c64", "c128"])
def test_async_read_is_a_snapshot_and_matches_the_sync_read(dtype):
    n = 14
    levels = W.random_circuit(n, 300, seed=31, p_multi=0.4)
    c = B.Circuit(n, dtype, 10)
    ids = c.load_levels(levels)
    c.update_state()
    dt = np.complex64 if dtype == "c64" else np.complex128
    bufs = [np.empty(1 << n, dt) for _ in range(2)]
    rng = np.random.default_rng(5)
    for k in range(4):
        want = c.read_amplitudes()
        c.read_amplitudes_async(bufs[k % 2])
        # change the state while the copy may still be in flight
        l = int(rng.integers(len(levels)))
        g = W.make_gate("rz", [int(rng.integers(n))], [float(rng.normal(0.0, 0.5))])
        try:
            c.insert_gate(l, g)
            levels[l] = list(levels[l]) + [g]
        except B.QtError:
            c.insert_level(l + 1)
            c.insert_gate(l + 1, g)
            levels.insert(l + 1, [g])
        c.update_state()
        c.read_wait()
        assert np.array_equal(bufs[k % 2], want), k
    assert max_err(c.read_amplitudes(), oracle.simulate(n, W.flatten(levels))) <= TOL[dtype]
    # a partial range, and a wait with nothing in flight
    part = np.empty(100, dt)
    c.read_amplitudes_async(part, 7, 100)
    c.read_wait()
    c.read_wait()
    assert np.array_equal(part, c.read_amplitudes(7, 100))
    c.close()


def test_async_read_rejects_stale_and_range():
    c = B.Circuit(8, "c64", 8)
    c.load_levels([[W.make_gate("h", [0])]])
    c.update_state()
    buf = np.empty(1 << 8, np.complex64)
    with pytest.raises(B.QtError):
        c.read_amplitudes_async(buf, 200, 100)
    c.insert_level(1)
    c.insert_gate(1, W.make_gate("x", [1]))
    with pytest.raises(B.QtError):
        c.read_amplitudes_async(buf)
    c.close()
