"""Helpers comparing libsr's GPU results with the oracle on the same seeded inputs."""
import numpy as np

from oracle import oracle as O


def oracle_run(w, sp=(2, 3, 5, 2), mode=0, threads=4):
    refs = [O.encode(bytes(r)) for r in w["refs"]]
    return O.run_batch(refs, w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"],
                       w["c_start"], w["c_len"], O.score_params(*sp), mode=mode, threads=threads)


def gpu_run(session, w, sp=(2, 3, 5, 2), **opts):
    from paper_1805_00106_gb300 import sr
    return session.align(w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"],
                         w["c_start"], w["c_len"], sr.score_params(*sp), sr.align_opts(**opts))


def compare(g, o, reads=None, want_cigar=True, classify=None):
    """Element-by-element comparison; returns a list of mismatch descriptions."""
    bad = []
    if not np.array_equal(g["item_score"], o["item_score"]):
        k = np.nonzero(g["item_score"] != o["item_score"])[0]
        bad.append(f"item_score differs at {len(k)} items, first {k[:5]} gpu {g['item_score'][k[:5]]} oracle {o['item_score'][k[:5]]}")
    if not np.array_equal(g["item_end"].astype(np.int64), o["item_end_j"].astype(np.int64)):
        k = np.nonzero(g["item_end"].astype(np.int64) != o["item_end_j"])[0]
        bad.append(f"item_end differs at {len(k)} items, first {k[:5]} gpu {g['item_end'][k[:5]]} oracle {o['item_end_j'][k[:5]]}")
    n = len(o["best"])
    rng = range(n) if reads is None else reads
    gb, ob = g["best"], o["best"]
    for f in ["score", "second", "n_ties", "item"]:
        gv = gb[f].astype(np.int64)[list(rng)]
        ov = ob[f].astype(np.int64)[list(rng)]
        if not np.array_equal(gv, ov):
            k = np.nonzero(gv != ov)[0]
            bad.append(f"best.{f} differs at {len(k)} reads, first {k[:5]}")
    has = ob["item"] >= 0
    for f in ["ref_id", "strand", "ref_end"]:
        gv, ov = gb[f].astype(np.int64), ob[f].astype(np.int64)
        d = np.nonzero(has & (gv != ov))[0]
        if len(d):
            bad.append(f"best.{f} differs at {len(d)} reads, first {d[:5]}")
    if want_cigar:
        for f in ["ref_start", "read_start", "read_end", "cigar_len"]:
            gv, ov = gb[f].astype(np.int64), ob[f].astype(np.int64)
            d = np.nonzero(has & (gv != ov))[0]
            if len(d):
                bad.append(f"best.{f} differs at {len(d)} reads, first {d[:5]} gpu {gv[d[:3]]} oracle {ov[d[:3]]}")
        nbad = 0
        for r in rng:
            if ob["item"][r] < 0:
                if gb["cigar_len"][r] != 0:
                    nbad += 1
                continue
            gc = g["cigar"][int(gb["cigar_off"][r]): int(gb["cigar_off"][r]) + int(gb["cigar_len"][r])]
            oc = o["cigar"][r][: int(ob["cigar_len"][r])]
            if not np.array_equal(gc, oc):
                nbad += 1
        if nbad:
            bad.append(f"CIGAR differs for {nbad} reads")
    gp, op = g["best_per_ref"], o["best_per_ref"]
    for f in ["score", "second", "n_ties", "item"]:
        if not np.array_equal(gp[f].astype(np.int64), op[f].astype(np.int64)):
            bad.append(f"best_per_ref.{f} differs")
    hp = op["item"] >= 0
    for f in ["strand", "ref_end"]:
        if np.any(hp & (gp[f].astype(np.int64) != op[f].astype(np.int64))):
            bad.append(f"best_per_ref.{f} differs")
    if classify is not None:
        min_score, margin = classify
        exp = np.array([O.classify(int(a), int(b), min_score, margin)
                        for a, b in zip(op["score"][:, 0], op["score"][:, 1])], np.uint8)
        if not np.array_equal(g["read_class"], exp):
            bad.append(f"class differs at {int(np.sum(g['read_class'] != exp))} reads")
    return bad
