"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-types the oracle's own formulas: gate matrices are
pinned by the matrices printed in the paper (Section II-A) and by algebraic
identities (Pauli relations, rotations as matrix exponentials, the U3 Euler
decomposition); the amplitude loops are pinned by the paper's brute-force
definition (Kronecker product per level, multiplied in order, Section II-A)
and by closed forms (GHZ, the quantum Fourier transform of a basis state,
norm preservation, a gate followed by its inverse, the Fig. 2 circuit).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2210_01076_gb300 import workloads as W

TOL = 1e-13


def read_golden_matrices(path):
    mats, lines = {}, [l.split("#")[0].strip() for l in open(path)]
    lines = [l for l in lines if l]
    i = 0
    while i < len(lines):
        head = lines[i].split()
        name, dim = head[0], int(head[1])
        scale = 1.0 / math.sqrt(2.0) if len(head) > 2 and head[2] == "1/sqrt2" else 1.0
        rows = [[float(x) for x in lines[i + 1 + r].split()] for r in range(dim)]
        mats[name] = scale * np.array(rows, dtype=np.complex128)
        i += 1 + dim
    return mats


@pytest.fixture(scope="module")
def printed(golden_dir):
    return read_golden_matrices(os.path.join(golden_dir, "paper_matrices.txt"))


# ---------------------------------------------------------------- test-side
# definitions built only from the printed X, H and from identities.

def defs(printed):
    X, H = printed["X"], printed["H"]
    Z = H @ X @ H                      # Hadamard conjugates X into Z
    Y = 1j * X @ Z                     # XZ = -iY
    return X, Y, Z, H


def test_printed_x_h_cx(printed):
    assert np.allclose(oracle.base_matrix("x"), printed["X"], atol=0, rtol=0)
    assert np.allclose(oracle.base_matrix("h"), printed["H"], atol=1e-16)
    # CX: columns are the images of |00>,|01>,|10>,|11> with the MSB as control
    cols = []
    for b in range(4):
        psi = np.zeros(4, np.complex128)
        psi[b] = 1
        oracle.apply_gate(psi, ("cnot", [0], [1], []))
        cols.append(psi)
    assert np.array_equal(np.array(cols).T, printed["CX"])


def test_pauli_and_phase_identities(printed):
    X, Y, Z, H = defs(printed)
    I2 = np.eye(2)
    assert np.allclose(oracle.base_matrix("z"), Z, atol=1e-15)
    assert np.allclose(oracle.base_matrix("y"), Y, atol=1e-15)
    S, T = oracle.base_matrix("s"), oracle.base_matrix("t")
    for M in (S, T):   # diagonal, first entry 1, principal (upper half-plane) root
        assert M[0, 1] == 0 and M[1, 0] == 0 and M[0, 0] == 1 and M[1, 1].imag > 0
    assert np.allclose(S @ S, Z, atol=1e-15)
    assert np.allclose(T @ T, S, atol=1e-15)
    assert np.allclose(oracle.base_matrix("sdg"), S.conj().T, atol=1e-15)
    assert np.allclose(oracle.base_matrix("tdg"), T.conj().T, atol=1e-15)
    for name in ("x", "y", "z", "h"):
        M = oracle.base_matrix(name)
        assert np.allclose(M @ M, I2, atol=1e-15)


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.0, math.pi / 2, math.pi, 4.0, 2 * math.pi - 0.1])
def test_rotations_are_exponentials(printed, theta):
    X, Y, Z, H = defs(printed)
    assert np.allclose(oracle.base_matrix("rx", (theta,)), scipy.linalg.expm(-0.5j * theta * X), atol=1e-14)
    assert np.allclose(oracle.base_matrix("ry", (theta,)), scipy.linalg.expm(-0.5j * theta * Y), atol=1e-14)
    RZ = lambda a: scipy.linalg.expm(-0.5j * a * Z)
    assert np.allclose(oracle.base_matrix("rz", (theta,)), RZ(theta), atol=1e-14)
    # controlled-phase target: P(l) = e^{il/2} RZ(l)
    assert np.allclose(oracle.base_matrix("cp", (theta,)), np.exp(0.5j * theta) * RZ(theta), atol=1e-14)
    rng = np.random.default_rng(int(theta * 1000))
    phi, lam = rng.uniform(0, 2 * math.pi, 2)
    RY = scipy.linalg.expm(-0.5j * theta * Y)
    U3 = np.exp(0.5j * (phi + lam)) * RZ(phi) @ RY @ RZ(lam)
    assert np.allclose(oracle.base_matrix("u3", (theta, phi, lam)), U3, atol=1e-14)


# ------------------------------------------------------- brute-force product

def ref_base(printed, g):
    X, Y, Z, H = defs(printed)
    S = np.diag([1, 1j])
    T = np.diag([1, np.exp(0.25j * math.pi)])
    th = g.params[0] if g.params else 0.0
    RZ = lambda a: scipy.linalg.expm(-0.5j * a * Z)
    RY = lambda a: scipy.linalg.expm(-0.5j * a * Y)
    table = {
        "x": X, "cnot": X, "ccx": X, "y": Y, "z": Z, "cz": Z, "h": H, "s": S, "sdg": S.conj().T,
        "t": T, "tdg": T.conj().T,
        "rx": lambda: scipy.linalg.expm(-0.5j * th * X), "ry": lambda: RY(th), "rz": lambda: RZ(th),
        "cp": lambda: np.exp(0.5j * th) * RZ(th),
        "u3": lambda: np.exp(0.5j * (g.params[1] + g.params[2])) * RZ(g.params[1]) @ RY(th) @ RZ(g.params[2]),
    }
    m = table[g.name]
    return m() if callable(m) else m


def kron_op(n, ops):
    """Kronecker product over qubits q_{n-1} (leftmost) ... q_0 (Section II-A)."""
    M = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        M = np.kron(M, ops.get(q, np.eye(2)))
    return M


def full_operator(n, g, printed):
    P1 = np.diag([0.0, 1.0]).astype(np.complex128)
    if g.name == "swap":
        a, b = g.targets
        X = printed["X"]

        def cx(t, c):
            P = kron_op(n, {c: P1})
            return np.eye(1 << n) - P + P @ kron_op(n, {t: X})
        core = cx(a, b) @ cx(b, a) @ cx(a, b)
    else:
        core = kron_op(n, {g.targets[0]: ref_base(printed, g)})
    if not g.controls:
        return core
    P = kron_op(n, {c: P1 for c in g.controls})
    return np.eye(1 << n) - P + P @ core


def level_unitary(n, level, printed):
    U = np.eye(1 << n, dtype=np.complex128)
    for g in level:
        U = full_operator(n, g, printed) @ U
    return U


ALL_TEST_KINDS = list(W.ALL_KINDS) + ["sdg", "tdg", "cp"]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_brute_force_product_random_circuits(printed, n):
    rng = np.random.default_rng(100 + n)
    kinds = [k for k in ALL_TEST_KINDS if sum(W.ARITY[k][:2]) <= n]
    gates = [W.random_gate(rng, n, kinds=kinds) for _ in range(12 * n)]
    levels = W.asap_levels(n, gates)
    U = np.eye(1 << n, dtype=np.complex128)
    for lv in levels:
        U = level_unitary(n, lv, printed) @ U
    psi = oracle.simulate(n, W.flatten(levels))
    assert np.max(np.abs(psi - U[:, 0])) <= TOL
    # the same gates on a random input state, one gate at a time
    phi = W.random_state(n, seed=7 + n)
    want = U @ phi
    for g in W.flatten(levels):
        oracle.apply_gate(phi, g)
    assert np.max(np.abs(phi - want)) <= TOL


@pytest.mark.parametrize("name", ALL_TEST_KINDS)
def test_each_gate_every_position_brute_force(printed, name):
    n = 4
    rng = np.random.default_rng(hash(name) % 1000)
    nq = sum(W.ARITY[name][:2])
    import itertools
    for qs in itertools.permutations(range(n), nq):
        g = W.make_gate(name, qs, rng.uniform(0, 2 * math.pi, W.ARITY[name][2]))
        phi = W.random_state(n, seed=len(qs) + qs[0])
        want = full_operator(n, g, printed) @ phi
        oracle.apply_gate(phi, g)
        assert np.max(np.abs(phi - want)) <= TOL, (name, qs)


# ----------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [2, 5, 10, 14])
def test_ghz(n):
    gates = [("h", [0], [], [])] + [("cnot", [q + 1], [q], []) for q in range(n - 1)]
    psi = oracle.simulate(n, gates)
    want = np.zeros(1 << n)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - want)) <= TOL


def qft_gates(n):
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(("h", [j], [], []))
        for m in range(j - 1, -1, -1):
            gates.append(("cp", [j], [m], [math.pi / (1 << (j - m))]))
    for i in range(n // 2):
        gates.append(("swap", [i, n - 1 - i], [], []))
    return gates


@pytest.mark.parametrize("n,x", [(3, 5), (6, 0), (6, 37), (8, 201), (10, 777)])
def test_qft_of_basis_state(n, x):
    prep = [("x", [q], [], []) for q in range(n) if x >> q & 1]
    psi = oracle.simulate(n, prep + qft_gates(n))
    y = np.arange(1 << n)
    want = np.exp(2j * math.pi * x * y / (1 << n)) / math.sqrt(1 << n)
    assert np.max(np.abs(psi - want)) <= 1e-13


def test_norm_preserved_over_2000_gates():
    n = 10
    rng = np.random.default_rng(5)
    gates = [W.random_gate(rng, n, kinds=ALL_TEST_KINDS) for _ in range(2000)]
    psi = oracle.simulate(n, gates)
    assert abs(oracle.norm(psi) - 1.0) <= 1e-13


INVERSE = {"s": "sdg", "sdg": "s", "t": "tdg", "tdg": "t"}


def inverse_gate(g):
    if g.name in INVERSE:
        return g._replace(name=INVERSE[g.name])
    if g.name in ("rx", "ry", "rz", "cp"):
        return g._replace(params=(-g.params[0],))
    if g.name == "u3":
        th, ph, la = g.params
        return g._replace(params=(-th, -la, -ph))
    return g  # self-inverse: x y z h cnot cz swap ccx


@pytest.mark.parametrize("name", ALL_TEST_KINDS)
def test_gate_then_inverse_is_identity(name):
    n = 7
    rng = np.random.default_rng(3)
    for _ in range(5):
        g = W.random_gate(rng, n, kinds=[name])
        phi = W.random_state(n, seed=11)
        ref = phi.copy()
        oracle.apply_gate(phi, g)
        if name not in ("z", "cz") and g.name not in ("rz",):
            assert np.max(np.abs(phi - ref)) > 1e-6 or name in ("cp", "ccx")
        oracle.apply_gate(phi, inverse_gate(g))
        assert np.max(np.abs(phi - ref)) <= TOL


def test_multithreaded_matches_single_thread():
    n = 12
    gates = W.flatten(W.random_circuit(n, 100, seed=1, p_multi=0.4))
    a = oracle.simulate(n, gates, nthreads=1)
    b = oracle.simulate(n, gates, nthreads=4)
    assert np.array_equal(a, b)


def test_oracle_rejects_bad_gates():
    psi = np.zeros(8, np.complex128)
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, ("cnot", [1], [1], []))
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, ("h", [3], [], []))
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, ("nope", [0], [], []))


# ------------------------------------------------------- the Fig. 2 example

def fig2_gates(golden, edited):
    gates = [("h", [q], [], []) for _, q in golden["net1"]]
    order = ["G6", "G7", "G10", "G9"] if edited else ["G6", "G7", "G8", "G9"]
    for k in order:
        gd = golden["gates"][k]
        gates.append(("cnot", [gd["target"]], [gd["control"]], []))
    return gates


def test_fig2_circuit_is_uniform_before_and_after_edit(golden_dir):
    golden = json.load(open(os.path.join(golden_dir, "fig2_example.json")))
    for edited in (False, True):
        psi = oracle.simulate(golden["n"], fig2_gates(golden, edited))
        assert np.max(np.abs(psi - 1 / math.sqrt(32))) <= TOL


@pytest.mark.parametrize("name", ALL_TEST_KINDS)
def test_workloads_inverse_gate_is_the_inverse(name):
    """The input generator's inverse-gate rule (used to build U then U-dagger
    circuits at full size) against the oracle: the inverse's base matrix is
    the adjoint of the gate's."""
    rng = np.random.default_rng(9)
    for _ in range(4):
        g = W.random_gate(rng, 5, kinds=[name])
        gi = W.inverse_gate(g)
        assert gi.qubits == g.qubits
        a = oracle.base_matrix(g.name, g.params)
        b = oracle.base_matrix(gi.name, gi.params)
        assert np.max(np.abs(b - a.conj().T)) <= TOL


def test_inverse_levels_undo_a_random_circuit():
    n = 8
    levels = W.random_circuit(n, 300, seed=4, p_multi=0.4)
    psi = oracle.simulate(n, W.flatten(levels) + W.flatten(W.inverse_levels(levels)))
    want = np.zeros(1 << n)
    want[0] = 1.0
    assert np.max(np.abs(psi - want)) <= 1e-12


def test_batch_circuit_shapes():
    rng = np.random.default_rng(404)
    circs = W.batch_circuits(40, rng)
    for n, levels in circs:
        assert 10 <= n <= 20 and 1 <= len(levels) <= 400
        for lv in levels:
            qs = [q for g in lv for q in g.qubits]
            assert len(qs) == len(set(qs)) and all(0 <= q < n for q in qs)
