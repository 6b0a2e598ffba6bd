"""Multi-GPU form of the path: independent replicas.

Every (read, window) item and every read's selection are independent, so N
GPUs each hold the whole (small) packed reference and take a share of the
reads; results are concatenated on the host.  There is no data-path
collective (the paper's V2 likewise replicates the reference on every FPGA and
hands reads to any of them, Sec. 4.2-4.3).  These helpers split a batch into
contiguous, cell-balanced shards and put the per-shard results back together.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(read_off, cand_off, c_len, world: int) -> np.ndarray:
    """Read boundaries [b0=0, b1, ..., bN=n] giving each rank a contiguous run of
    reads with about 1/world of the DP cells."""
    n = len(read_off) - 1
    m = np.diff(np.asarray(read_off, np.int64))
    counts = np.diff(np.asarray(cand_off, np.int64))
    item_m = np.repeat(m, counts)
    cells_item = item_m * np.asarray(c_len, np.int64)
    per_read = np.zeros(n, np.int64)
    if len(cells_item):
        np.add.at(per_read, np.repeat(np.arange(n), counts), cells_item)
    csum = np.concatenate([[0], np.cumsum(per_read)])
    total = csum[-1]
    bounds = [0]
    for k in range(1, world):
        bounds.append(int(np.searchsorted(csum, total * k / world, side="left")))
    bounds.append(n)
    return np.maximum.accumulate(np.array(bounds, np.int64))


def take_shard(w: dict, r0: int, r1: int) -> dict:
    """Reads [r0, r1) with their windows, offsets rebased to 0."""
    ro, co = np.asarray(w["read_off"], np.int64), np.asarray(w["cand_off"], np.int64)
    b0, b1, c0, c1 = ro[r0], ro[r1], co[r0], co[r1]
    out = dict(w)
    out.update(bases=w["bases"][b0:b1], read_off=ro[r0:r1 + 1] - b0, cand_off=co[r0:r1 + 1] - c0,
               c_ref=w["c_ref"][c0:c1], c_strand=w["c_strand"][c0:c1], c_start=w["c_start"][c0:c1],
               c_len=w["c_len"][c0:c1])
    return out


def concat_results(parts: list, item_key: str = "item") -> dict:
    """Concatenate per-shard result dicts (in rank order): per-item arrays are
    appended, winner item indices are rebased by the items before the shard,
    CIGAR offsets by the CIGAR words before it."""
    out = {}
    item_base, cig_base = 0, 0
    best, per_ref, scores, ends, cigars = [], [], [], [], []
    for p in parts:
        b = p["best"].copy()
        has = b[item_key] >= 0
        b[item_key][has] += item_base
        if "cigar_off" in b.dtype.names:
            b["cigar_off"][b["cigar_len"] > 0] += cig_base
        best.append(b)
        pr = p["best_per_ref"].copy()
        hp = pr[item_key] >= 0
        pr[item_key][hp] += item_base
        per_ref.append(pr)
        scores.append(p["item_score"])
        ends.append(p["item_end"])
        cigars.append(p["cigar"])
        item_base += len(p["item_score"])
        cig_base += len(p["cigar"])
    out["best"] = np.concatenate(best) if best else None
    out["best_per_ref"] = np.concatenate(per_ref) if per_ref else None
    out["item_score"] = np.concatenate(scores) if scores else None
    out["item_end"] = np.concatenate(ends) if ends else None
    out["cigar"] = np.concatenate(cigars) if cigars else None
    return out
