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


def subset_reads(w, reads):
    """Workload restricted to `reads` (in that order), offsets rebased."""
    reads = np.asarray(reads, np.int64)
    ro, co = np.asarray(w["read_off"], np.int64), np.asarray(w["cand_off"], np.int64)
    bases = np.concatenate([w["bases"][ro[r]:ro[r + 1]] for r in reads])
    lens = ro[reads + 1] - ro[reads]
    cnts = co[reads + 1] - co[reads]
    items = np.concatenate([np.arange(co[r], co[r + 1]) for r in reads]) if cnts.sum() else np.zeros(0, np.int64)
    out = dict(refs=w["refs"], bases=bases, read_off=np.concatenate([[0], np.cumsum(lens)]),
               cand_off=np.concatenate([[0], np.cumsum(cnts)]))
    for k in ["c_ref", "c_strand", "c_start", "c_len"]:
        out[k] = np.asarray(w[k])[items]
    return out


def compare_sampled(g, w, reads, o, want_cigar=True, classify=None):
    """Compare the GPU results of a whole batch, on the sampled reads only, with
    the oracle's results `o` for the subset workload of those reads."""
    bad = []
    co = np.asarray(w["cand_off"], np.int64)
    so = 0
    for s, r in enumerate(reads):
        c0, c1 = co[r], co[r + 1]
        n = c1 - c0
        if not np.array_equal(g["item_score"][c0:c1], o["item_score"][so:so + n]):
            bad.append(f"read {r}: item scores differ")
        if not np.array_equal(g["item_end"][c0:c1].astype(np.int64), o["item_end_j"][so:so + n].astype(np.int64)):
            bad.append(f"read {r}: item ends differ")
        gb, ob = g["best"][r], o["best"][s]
        for f in ["score", "second", "n_ties"]:
            if int(gb[f]) != int(ob[f]):
                bad.append(f"read {r}: best.{f} {gb[f]} vs {ob[f]}")
        gi = int(gb["item"]) - c0 if gb["item"] >= 0 else -1
        oi = int(ob["item"]) - so if ob["item"] >= 0 else -1
        if gi != oi:
            bad.append(f"read {r}: winner {gi} vs {oi}")
        if ob["item"] >= 0:
            for f in ["ref_id", "strand", "ref_end"] + (["ref_start", "read_start", "read_end", "cigar_len"] if want_cigar else []):
                if int(gb[f]) != int(ob[f]):
                    bad.append(f"read {r}: best.{f} {gb[f]} vs {ob[f]}")
            if want_cigar:
                gc = g["cigar"][int(gb["cigar_off"]): int(gb["cigar_off"]) + int(gb["cigar_len"])]
                if not np.array_equal(gc, o["cigar"][s][: int(ob["cigar_len"])]):
                    bad.append(f"read {r}: CIGAR differs")
        for q in range(g["best_per_ref"].shape[1]):
            gp, op = g["best_per_ref"][r, q], o["best_per_ref"][s, q]
            if int(gp["score"]) != int(op["score"]) or int(gp["n_ties"]) != int(op["n_ties"]) or \
               int(gp["second"]) != int(op["second"]):
                bad.append(f"read {r}: per-ref {q} differs")
        if classify is not None:
            exp = O.classify(int(o["best_per_ref"][s, 0]["score"]), int(o["best_per_ref"][s, 1]["score"]),
                             classify[0], classify[1])
            if int(g["read_class"][r]) != exp:
                bad.append(f"read {r}: class {g['read_class'][r]} vs {exp}")
        so += n
        if len(bad) > 20:
            break
    return bad


def whole_batch_properties(g, w):
    """Properties that hold at any size: the winner's score is the read's largest
    item score, ties and second are consistent, CIGARs consume the read."""
    co = np.asarray(w["cand_off"], np.int64)
    ro = np.asarray(w["read_off"], np.int64)
    sc = g["item_score"]
    n = len(ro) - 1
    mx = np.zeros(n, np.int64)
    has = np.diff(co) > 0
    if len(sc):
        red = np.maximum.reduceat(sc.astype(np.int64), co[:-1][has]) if has.any() else np.zeros(0)
        mx[has] = red
    b = g["best"]
    bad = []
    if not np.array_equal(np.maximum(mx, 0), b["score"].astype(np.int64)):
        bad.append("best score is not the largest item score")
    pos = b["score"] > 0
    if np.any(b["n_ties"][pos] < 1) or np.any(b["n_ties"][~pos] != 0):
        bad.append("n_ties inconsistent")
    if np.any(b["second"] > b["score"]):
        bad.append("second > best")
    if np.any(sc[b["item"][pos]] != b["score"][pos]):
        bad.append("winner item does not carry the best score")
    # CIGAR lengths: M+I+S == read length for every winner
    cig = g["cigar"]
    idx = np.nonzero(pos)[0]
    for r in idx[:: max(1, len(idx) // 20000)]:
        words = cig[int(b["cigar_off"][r]): int(b["cigar_off"][r]) + int(b["cigar_len"][r])]
        ops, lens = words & 15, words >> 4
        if int(lens[(ops == 0) | (ops == 1) | (ops == 4)].sum()) != ro[r + 1] - ro[r]:
            bad.append(f"read {r}: CIGAR does not consume the read")
            break
    return bad


def edge_workload(seed=23):
    """Reads of edge lengths (1, 2, tile boundaries 15-17, 31-33, ..., 255, 256),
    each with windows clamped at both reference ends, a 1-base window, a
    512-base window, windows shorter than the read, alternating strands, and a
    read with no windows at all, on a 3 kbp reference."""
    rng = np.random.default_rng(seed)
    L = 3000
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), L)
    reads, offs = [], [0]
    cand = dict(cand_off=[0], c_ref=[], c_strand=[], c_start=[], c_len=[])
    lengths = [1, 2, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 255, 256]
    for m in lengths:
        pos = int(rng.integers(0, L - m))
        r = ref[pos:pos + m].copy()
        if m > 10:
            r[m // 2] = ord("A") if r[m // 2] != ord("A") else ord("C")
        reads.append(r)
        offs.append(offs[-1] + m)
        wins = [(pos, m), (max(0, pos - 64), min(L - max(0, pos - 64), m + 128)), (0, min(L, m + 5)),
                (L - min(L, m + 7), min(L, m + 7)), (pos, 1), (max(0, pos - 3), min(5, L)),
                (max(0, min(pos, L - 512)), 512)]
        if m > 12:
            wins.append((pos + 2, m - 10))
        for k, (st, ln) in enumerate(wins):
            cand["c_ref"].append(0)
            cand["c_strand"].append(k % 2)
            cand["c_start"].append(st)
            cand["c_len"].append(ln)
        cand["cand_off"].append(len(cand["c_ref"]))
    # a read with no windows at all
    reads.append(ref[10:90])
    offs.append(offs[-1] + 80)
    cand["cand_off"].append(len(cand["c_ref"]))
    return dict(refs=[ref], bases=np.concatenate(reads), read_off=np.array(offs),
                **{k: np.array(v) for k, v in cand.items()})
