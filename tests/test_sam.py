"""SAM writer (sr_write_sam, host code) on results built from the oracle: every
field of every line is checked against the alignment it reports (CPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_00106_gb300 import synth as S

from .parity import oracle_run

OPS = "MIDNSHP=X"


@pytest.fixture(scope="module")
def sr():
    from paper_1805_00106_gb300 import sr as _sr
    _sr.lib()
    return _sr


def _results_from_oracle(sr, o, n_refs):
    n = len(o["best"])
    best = np.zeros(n, sr.HIT_DTYPE)
    per = np.zeros((n, n_refs), sr.HIT_DTYPE)
    words, off = [], 0
    for r in range(n):
        b = o["best"][r]
        for f in ["score", "second", "n_ties", "item", "ref_id", "strand", "read_start", "read_end",
                  "ref_start", "ref_end"]:
            best[r][f] = max(int(b[f]), 0) if f not in ("score", "second", "item") else int(b[f])
        if b["item"] >= 0:
            ln = int(b["cigar_len"])
            words.append(np.asarray(o["cigar"][r][:ln], np.uint32))
            best[r]["cigar_off"], best[r]["cigar_len"] = off, ln
            off += ln
    cig = np.concatenate(words) if words else np.zeros(0, np.uint32)
    return dict(best=best, best_per_ref=per, cigar=cig, read_class=None)


def _revcomp(s):
    return s[::-1].translate(str.maketrans("ACGT", "TGCA"))


def _parse(path):
    head, lines = [], []
    for ln in open(path):
        (head if ln.startswith("@") else lines).append(ln.rstrip("\n").split("\t"))
    return head, lines


def test_sam_lines_match_the_alignments(sr, tmp_path):
    w = S.workload("c1", scale=0.02, seed=8, rc_frac=0.5)
    # a read without any window
    w["cand_off"] = np.concatenate([w["cand_off"], [w["cand_off"][-1]]])
    w["bases"] = np.concatenate([w["bases"], np.frombuffer(b"ACGTACGTAC", np.uint8)])
    w["read_off"] = np.concatenate([w["read_off"], [w["read_off"][-1] + 10]])
    o = oracle_run(w)
    res = _results_from_oracle(sr, o, 1)
    path = tmp_path / "out.sam"
    sr.write_sam(path, w["bases"], w["read_off"], res, [len(w["refs"][0])])
    head, lines = _parse(path)
    assert head[0][:2] == ["@HD", "VN:1.6"]
    assert head[1] == ["@SQ", "SN:ref0", f"LN:{len(w['refs'][0])}"]
    n = len(w["read_off"]) - 1
    assert len(lines) == n
    for r, f in enumerate(lines):
        b = o["best"][r]
        seq = bytes(w["bases"][w["read_off"][r]:w["read_off"][r + 1]]).decode()
        assert f[0] == f"r{r}"
        if b["item"] < 0:
            assert f[1:6] == ["4", "*", "0", "0", "*"] and f[9] == seq
            continue
        assert int(f[1]) == (16 if b["strand"] else 0)
        assert f[2] == "ref0" and int(f[3]) == int(b["ref_start"]) + 1
        exp_cigar = "".join(f"{int(x) >> 4}{OPS[int(x) & 15]}" for x in o["cigar"][r][:int(b["cigar_len"])])
        assert f[5] == exp_cigar
        assert f[9] == (_revcomp(seq) if b["strand"] else seq)
        assert f[10] == "*"
        tags = dict(t.split(":", 1) for t in f[11:])
        assert tags["AS"] == f"i:{int(b['score'])}" and tags["XS"] == f"i:{int(b['second'])}"
        assert tags["X0"] == f"i:{int(b['n_ties'])}"
        mq = 0 if b["n_ties"] > 1 else min(60, 60 * (int(b["score"]) - max(int(b["second"]), 0)) // int(b["score"]))
        assert int(f[4]) == mq
        # CIGAR consumes the read and spans the reported reference interval
        import re
        runs = [(int(a), c) for a, c in re.findall(r"(\d+)([MIDS])", f[5])]
        assert sum(a for a, c in runs if c in "MIS") == len(seq)
        assert sum(a for a, c in runs if c in "MD") == int(b["ref_end"]) - int(b["ref_start"]) + 1


def test_sam_names_classes_and_secondary_hits(sr, tmp_path):
    w = S.workload("c2", scale=0.0002, seed=4)
    o = oracle_run(w)
    res = _results_from_oracle(sr, o, 1)
    n = len(w["read_off"]) - 1
    res["read_class"] = np.arange(n, dtype=np.uint8) % 4
    rep_idx = O.report_batch(o, w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"], O.REPORT_BEST_N, 3)
    offs = np.concatenate([[0], np.cumsum([len(x) for x in rep_idx])]).astype(np.uint64)
    hits = np.zeros(int(offs[-1]), sr.REPORT_HIT_DTYPE)
    flat = np.concatenate(rep_idx) if len(offs) > 1 and offs[-1] else np.zeros(0, np.int64)
    if len(flat):
        hits["item"] = flat
        hits["score"] = o["item_score"][flat]
        hits["ref_id"] = np.asarray(w["c_ref"])[flat]
        hits["strand"] = np.asarray(w["c_strand"])[flat]
        hits["end_col"] = o["item_end_j"][flat]
        hits["ref_end"] = np.asarray(w["c_start"], np.int64)[flat] + o["item_end_j"][flat] - 1
    names = [f"q{r:05d}" for r in range(n)]
    path = tmp_path / "named.sam"
    sr.write_sam(path, w["bases"], w["read_off"], res, [len(w["refs"][0])], read_names=names,
                 ref_names=["chrS"], report=dict(offsets=offs, hits=hits))
    head, lines = _parse(path)
    assert head[1][1] == "SN:chrS"
    for r, f in enumerate(lines):
        assert f[0] == names[r]
        tags = dict(t.split(":", 1) for t in f[11:])
        assert tags["YC"] == "Z:" + ["UN", "A", "B", "AMB"][r % 4]
        exp = [t for t in rep_idx[r] if t != o["best"][r]["item"]]
        if exp:
            got = tags["XA"][2:].rstrip(";").split(";")
            assert got == [f"chrS,{'-' if w['c_strand'][t] else '+'}"
                           f"{int(w['c_start'][t]) + int(o['item_end_j'][t])},{int(o['item_score'][t])}"
                           for t in exp]
        else:
            assert "XA" not in tags


def test_sam_rejects_inconsistent_inputs(sr, tmp_path):
    w = S.workload("c1", scale=0.005, seed=2)
    o = oracle_run(w)
    res = _results_from_oracle(sr, o, 1)
    with pytest.raises(sr.SrError) as e:
        sr.write_sam(tmp_path / "x.sam", w["bases"], w["read_off"][:-1], res, [len(w["refs"][0])])
    assert e.value.status == sr.SR_EINVAL
    with pytest.raises(sr.SrError) as e:
        sr.write_sam(tmp_path / "no_dir" / "x.sam", w["bases"], w["read_off"], res, [len(w["refs"][0])])
    assert e.value.status == sr.SR_EIO
