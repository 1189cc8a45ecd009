"""Shared helpers for the GPU parity tests (inputs and comparisons only)."""
import numpy as np

import oracle
from paper_2210_01076_gb300 import binding as B
from paper_2210_01076_gb300 import workloads as W

# max-abs tolerances per amplitude against the FP64 oracle
TOL = {"c128": 1e-12, "c128df": 1e-12, "c64": 1e-5}
DTYPES = ["c128", "c128df", "c64"]


def build_circuit(n, levels, dtype, p, **opts):
    c = B.Circuit(n, dtype, p)
    for k, v in opts.items():
        c.set_option(k, v)
    ids = c.load_levels(levels)
    return c, ids


def handles_for(ids):
    m, k = {}, 0
    for lv in ids:
        for gid in lv:
            m[k] = gid
            k += 1
    return m


def prep_levels(n, seed):
    """A generic (entangled, all-amplitude) input: U3 on every qubit, a CNOT
    ladder, U3 again."""
    rng = np.random.default_rng(seed)
    gates = [W.make_gate("u3", [q], rng.uniform(0, 2 * np.pi, 3)) for q in range(n)]
    gates += [W.make_gate("cnot", [q + 1, q]) for q in range(n - 1)]
    gates += [W.make_gate("u3", [q], rng.uniform(0, 2 * np.pi, 3)) for q in range(n)]
    return W.asap_levels(n, gates)


def max_err(a, b):
    return float(np.max(np.abs(a.astype(np.complex128) - b)))


def fidelity(a, b):
    a = a.astype(np.complex128)
    return float(abs(np.vdot(b, a)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))
