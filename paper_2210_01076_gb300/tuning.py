"""Measured choice of fusion width and checkpoint spacing.

The planner's knobs trade HBM passes against per-pass work: ``tile_high``
(qubits a tile may hold above its contiguous low run -- the fusion width),
``fusion`` and ``merge``, and ``ckpt_interval`` (levels per checkpoint, which
trades memory and incremental restart distance against nothing at all in a
full run).  Which setting is fastest depends on the dtype (float-float
arithmetic is issue-bound, complex64 closer to HBM-bound) and on the circuit,
so these helpers time candidate settings on the device and keep the best
-- for complex64 also whether runs of gates on five qubits go to the tensor
cores as fused blocks (``tc_blocks``, ``tc_threshold``).
Only the timing loop is host code; every measured run is the library's.
"""
from __future__ import annotations

import itertools
from typing import Dict, Iterable, List, Optional

from . import binding as B


def _full_ms(c: "B.Circuit", repeats: int) -> float:
    c.update_state()
    best = None
    for _ in range(repeats):
        ms = c.update_state(force_full=True)["gpu_ms"]
        best = ms if best is None else min(best, ms)
    return best


def tune_circuit(n: int, dtype: str, levels, log2_partition: Optional[int] = None,
                 tile_high: Iterable[int] = (3, 4, 5), ckpt_interval: Iterable[int] = (4,),
                 fusion: Iterable[int] = (1,), merge: Iterable[int] = (0, 1), tc_threshold: Iterable[int] = (-1,),
                 repeats: int = 2) -> Dict:
    """Time a full simulation of ``levels`` for every combination of the
    candidate options; return the fastest and the whole table.
    ``tc_threshold``: -1 = no tensor-core blocks, else blocks (complex64)
    with that threshold (tenths of a dense one-qubit op)."""
    table: List[Dict] = []
    for th, ck, fu, me, tc in itertools.product(tile_high, ckpt_interval, fusion, merge, tc_threshold):
        c = B.Circuit(n, dtype, log2_partition)
        try:
            opts = {"tile_high": th, "ckpt_interval": ck, "fusion": fu, "merge": me}
            if tc >= 0:
                opts.update({"tc_blocks": 1, "tc_threshold": tc})
            for k, v in opts.items():
                c.set_option(k, v)
            c.load_levels(levels)
            ms = _full_ms(c, repeats)
            table.append({"options": opts, "full_ms": ms, "device_bytes": B.qt_device_bytes(c.h)})
        except B.QtError as e:
            table.append({"options": opts, "error": str(e)})
        finally:
            c.close()
    ok = [t for t in table if "full_ms" in t]
    best = min(ok, key=lambda t: t["full_ms"]) if ok else None
    return {"best": best, "table": table}


def tune_batch(circuits, tile_high: Iterable[int] = (3, 4, 5), repeats: int = 3) -> Dict:
    """Time batched runs of ``circuits`` with each candidate tile width set on
    every circuit; leave the fastest set and return the table."""
    table = []
    for th in tile_high:
        for c in circuits:
            c.set_option("tile_high", th)
        batch = B.Batch(circuits)
        try:
            batch.run()
            ms = min(batch.run()["gpu_ms"] for _ in range(repeats))
            table.append({"tile_high": th, "round_ms": ms})
        except B.QtError as e:
            table.append({"tile_high": th, "error": str(e)})
        finally:
            batch.close()
    ok = [t for t in table if "round_ms" in t]
    best = min(ok, key=lambda t: t["round_ms"]) if ok else None
    if best:
        for c in circuits:
            c.set_option("tile_high", best["tile_high"])
    return {"best": best, "table": table}
