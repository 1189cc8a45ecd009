"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times, on outputs checked one at a time or through properties that
hold at any size.

* The deep configuration: n = 30, partitions of 2^18, checkpoints every 48
  levels, complex64 and float-float complex128.
  - The QFT of a basis state (H + controlled-phase ladders: the circuit's
    QFT layers in full) against its closed form at sampled indices.
  - A U3 layer on every qubit followed by diagonal gates only (CZ on
    disjoint pairs, controlled-phase ladders, T and RZ) against the product
    formula, one amplitude at a time, from the oracle's gate matrices.
  - The 2000-gate QFT-like circuit followed by its inverse gives |0...0>.
  - Single-gate edits near the tail: each incremental result is bit
    identical to a full re-simulation (compared on the device).
* The batched configuration: 256 circuits of 10-20 qubits in one persistent
  launch, then a round of parameter edits replayed from the CUDA graph; a
  sample of circuits (the largest and smallest included) against the FP64
  oracle after each run.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import build as qbuild
from paper_2210_01076_gb300 import workloads as W
from gpu_helpers import TOL, max_err

pytestmark = pytest.mark.gpu

N, P, CKPT = 30, 18, 48
BLOCK = 1 << 12


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    B.load()


def deep_circuit(dtype, levels, ckpt=CKPT):
    c = B.Circuit(N, dtype, P)
    c.set_option("ckpt_interval", ckpt)
    ids = c.load_levels(levels)
    return c, ids


def sample_blocks(seed, count=12):
    """Starts of amplitude blocks: the first, the last and `count` drawn by seed."""
    rng = np.random.default_rng(seed)
    nblk = (1 << N) // BLOCK
    starts = [0, (nblk - 1) * BLOCK] + [int(b) * BLOCK for b in rng.choice(nblk, size=count, replace=False)]
    return starts


def rel_tol(dtype):
    # error bound relative to an amplitude's magnitude, stricter than TOL
    return 1e-4 if dtype == "c64" else 1e-9


@pytest.mark.parametrize("dtype", ["c64", "c128df"])
def test_qft_of_a_basis_state_n30_sampled_closed_form(dtype):
    """QFT|x> = 2^(-n/2) sum_y exp(2 pi i x y / 2^n) |y> (swap network at the
    end so that the output is in natural order)."""
    x = 0x2A5F3C71 & ((1 << N) - 1)
    gates = [W.make_gate("x", [q]) for q in range(N) if x >> q & 1]
    for j in range(N - 1, -1, -1):
        gates.append(W.make_gate("h", [j]))
        for m in range(j - 1, -1, -1):
            gates.append(W.make_gate("cp", [j, m], [math.pi / (1 << (j - m))]))
    for i in range(N // 2):
        gates.append(W.make_gate("swap", [i, N - 1 - i]))
    c, _ = deep_circuit(dtype, W.asap_levels(N, gates))
    c.update_state()
    mag = 2.0 ** (-N / 2)
    for s in sample_blocks(1):
        y = np.arange(s, s + BLOCK, dtype=np.uint64)
        ph = (np.uint64(x) * y) & np.uint64((1 << N) - 1)  # x*y < 2^60: exact in uint64
        want = mag * np.exp(2j * math.pi * ph.astype(np.float64) / (1 << N))
        got = c.read_amplitudes(s, BLOCK)
        err = max_err(got, want)
        assert err <= TOL[dtype] and err <= rel_tol(dtype) * mag, (s, err)
    assert abs(c.norm() - 1.0) <= (1e-5 if dtype == "c64" else 1e-12)
    c.close()


@pytest.mark.parametrize("dtype", ["c64", "c128df"])
def test_product_layer_and_diagonals_n30_sampled(dtype):
    """A U3 on every qubit makes a product state; every later gate is
    diagonal, so each amplitude is the product of the U3 columns times the
    diagonal entries its bits select."""
    rng = np.random.default_rng(23)
    u3 = [rng.uniform(0, 2 * math.pi, 3) for _ in range(N)]
    gates = [W.make_gate("u3", [q], u3[q]) for q in range(N)]
    perm = rng.permutation(N)
    cz = [(int(perm[a]), int(perm[a + 1])) for a in range(0, N - 1, 2)]
    gates += [W.make_gate("cz", list(pq)) for pq in cz]
    cps = []
    for j in (0, 7, 13, 21, 29):
        for k in range(1, N):
            m = (j + k) % N
            lam = math.pi / (1 << min(k, 20))
            cps.append((j, m, lam))
            gates.append(W.make_gate("cp", [j, m], [lam]))
    singles = []
    for q in range(0, N, 3):
        name = "t" if q % 2 else "rz"
        par = [] if name == "t" else [float(rng.uniform(0, 2 * math.pi))]
        singles.append((q, name, par))
        gates.append(W.make_gate(name, [q], par))
    c, _ = deep_circuit(dtype, W.asap_levels(N, gates))
    c.update_state()
    col = [oracle.base_matrix("u3", u3[q])[:, 0] for q in range(N)]
    cp_phase = {lam: oracle.base_matrix("cp", [lam])[1, 1] for _, _, lam in cps}
    for s in sample_blocks(2):
        y = np.arange(s, s + BLOCK, dtype=np.int64)
        bits = [(y >> q) & 1 for q in range(N)]
        want = np.ones(BLOCK, dtype=np.complex128)
        for q in range(N):
            want *= np.where(bits[q] == 1, col[q][1], col[q][0])
        for a, b in cz:
            want *= np.where((bits[a] & bits[b]) == 1, -1.0, 1.0)
        for j, m, lam in cps:
            want *= np.where((bits[j] & bits[m]) == 1, cp_phase[lam], 1.0)
        for q, name, par in singles:
            d = np.diag(oracle.base_matrix(name, par))
            want *= np.where(bits[q] == 1, d[1], d[0])
        got = c.read_amplitudes(s, BLOCK)
        err = max_err(got, want)
        assert err <= TOL[dtype] and err <= rel_tol(dtype) * float(np.max(np.abs(want))), (s, err)
    c.close()


@pytest.mark.parametrize("dtype", ["c64", "c128df"])
def test_deep30_then_inverse_returns_to_zero(dtype):
    """The benchmark's QFT-like circuit (2000 gates) then its inverse: every
    amplitude but the first returns to 0 and the first to 1."""
    levels = W.qft_like_circuit(N, 2000, seed=7)
    c, _ = deep_circuit(dtype, levels)
    c.update_state()
    assert abs(c.norm() - 1.0) <= (1e-5 if dtype == "c64" else 1e-12)
    c.close()
    # forward + inverse: twice the levels, checkpoints half as often (memory)
    c, _ = deep_circuit(dtype, levels + W.inverse_levels(levels), ckpt=2 * CKPT)
    c.update_state()
    tol = TOL[dtype] if dtype != "c64" else 1e-4  # 4000 binary32 gates
    for s in sample_blocks(3):
        want = np.zeros(BLOCK, dtype=np.complex128)
        if s == 0:
            want[0] = 1.0
        assert max_err(c.read_amplitudes(s, BLOCK), want) <= tol, s
    assert abs(c.norm() - 1.0) <= (1e-4 if dtype == "c64" else 1e-12)
    c.close()


@pytest.mark.parametrize("dtype", ["c64", "c128df"])
def test_deep30_tail_edits_incremental_bit_identical(dtype):
    """The benchmark's deep configuration and edit rule: each incremental
    update equals a full re-simulation bit for bit (device compare)."""
    torch = pytest.importorskip("torch")
    levels = W.qft_like_circuit(N, 2000, seed=7)
    c, ids = deep_circuit(dtype, levels)
    c.update_state()
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    inc = torch.empty(1 << N, dtype=tdt, device="cuda")
    full = torch.empty(1 << N, dtype=tdt, device="cuda")
    rng = np.random.default_rng(11)
    done = 0
    while done < 3:
        e = W.tail_edit(rng, levels)
        if e is None:
            continue
        lvl, k, ng = e
        ids[lvl][k] = c.replace_gate(lvl, ids[lvl][k], ng)
        levels[lvl][k] = ng
        st = c.update_state()
        assert st["clean_fraction"] > 0.0
        c.read_amplitudes_device(0, 1 << N, inc.data_ptr())
        c.update_state(force_full=True)
        c.read_amplitudes_device(0, 1 << N, full.data_ptr())
        torch.cuda.synchronize()
        bits = torch.int32 if dtype == "c64" else torch.int64
        assert torch.equal(torch.view_as_real(inc).view(bits), torch.view_as_real(full).view(bits)), done
        done += 1
    del inc, full
    torch.cuda.empty_cache()
    c.close()


def test_batch256_full_size_sampled_circuits_against_oracle():
    """The batched configuration as the benchmark builds it (seed 404):
    a sample of circuits against the oracle after the first run and after a
    round of parameter edits (a CUDA-graph replay)."""
    rng = np.random.default_rng(404)
    circs, levels, ids = [], [], []
    for n, lv in W.batch_circuits(256, rng):
        c = B.Circuit(n, "c64", min(n, 16))
        ids.append(c.load_levels(lv))
        levels.append([list(x) for x in lv])
        circs.append(c)
    ns = [c.n for c in circs]
    order = sorted(range(len(circs)), key=lambda k: (ns[k], sum(len(l) for l in levels[k])))
    pick = sorted({order[0], order[-1]} | {int(k) for k in np.random.default_rng(1).choice(256, 8, replace=False)})
    batch = B.Batch(circs)
    nth = oracle.max_threads()
    for rnd in range(3):
        st = batch.run()
        assert st["circuits"] == 256
        if rnd == 2:
            assert st["graph_replayed"] == 1
        if rnd != 1:
            for k in pick:
                want = oracle.simulate(ns[k], W.flatten(levels[k]), nthreads=nth)
                got = batch.read_amplitudes(k)
                assert max_err(got, want) <= TOL["c64"], (rnd, k)
        if rnd == 1:
            for k, c in enumerate(circs):
                e = W.rotation_edit(rng, levels[k])
                if e is None:
                    continue
                l, j, ng = e
                ids[k][l][j] = c.replace_gate(l, ids[k][l][j], ng)
                levels[k][l][j] = ng
    batch.close()
    for c in circs:
        c.close()


@pytest.mark.parametrize("n,dtype", [(33, "c64"), (32, "c128df")])
def test_largest_states_indices_past_2_to_32(n, dtype):
    """The largest states that fit the device with one segment (64 GiB per
    buffer): GHZ and the QFT of a basis state, checked at sampled blocks on
    both sides of amplitude 2^32 (2^31 at n = 32; byte offsets pass 2^32
    there) and at the ends; FP64 norm."""
    N = 1 << n
    mid = min(1 << 32, N // 2)
    starts = [0, mid - BLOCK, mid, N - BLOCK] + [
        int(b) * BLOCK for b in np.random.default_rng(n).choice(N // BLOCK, size=6, replace=False)]
    ghz = [W.make_gate("h", [0])] + [W.make_gate("cnot", [q + 1, q]) for q in range(n - 1)]
    c = B.Circuit(n, dtype, 20)
    c.set_option("ckpt_interval", 1 << 20)
    c.load_levels(W.asap_levels(n, ghz))
    c.update_state()
    for s in starts:
        want = np.zeros(BLOCK)
        if s == 0:
            want[0] = 1 / math.sqrt(2)
        if s == N - BLOCK:
            want[-1] = 1 / math.sqrt(2)
        assert max_err(c.read_amplitudes(s, BLOCK), want) <= TOL[dtype], s
    assert abs(c.norm() - 1.0) <= TOL[dtype]
    c.close()
    x = 0x15A5F3C71 & (N - 1)
    gates = [W.make_gate("x", [q]) for q in range(n) if x >> q & 1]
    for j in range(n - 1, -1, -1):
        gates.append(W.make_gate("h", [j]))
        for m in range(j - 1, -1, -1):
            gates.append(W.make_gate("cp", [j, m], [math.pi / (1 << (j - m))]))
    gates += [W.make_gate("swap", [i, n - 1 - i]) for i in range(n // 2)]
    c = B.Circuit(n, dtype, 20)
    c.set_option("ckpt_interval", 1 << 20)
    c.load_levels(W.asap_levels(n, gates))
    c.update_state()
    mag = 2.0 ** (-n / 2)
    for s in starts:
        y = np.arange(s, s + BLOCK, dtype=np.uint64)
        ph = (np.uint64(x) * y) & np.uint64(N - 1)  # the product wraps mod 2^64, a multiple of 2^n
        want = mag * np.exp(2j * math.pi * ph.astype(np.float64) / N)
        err = max_err(c.read_amplitudes(s, BLOCK), want)
        assert err <= TOL[dtype] and err <= rel_tol(dtype) * mag, (s, err)
    c.close()
