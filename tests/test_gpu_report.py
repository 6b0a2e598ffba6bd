"""Score-tracker report options (Sec. 4.2: N highest-scoring CALs, all CALs tied
for the best) on the GPU vs the oracle, per read, bit-exact (-m gpu)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_00106_gb300 import synth as S

from .parity import oracle_run

pytestmark = pytest.mark.gpu

SP = (2, 3, 5, 2)


@pytest.fixture(scope="module")
def sr():
    from paper_1805_00106_gb300 import sr as _sr
    _sr.lib()
    return _sr


def _run(sr, w):
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    b = s.stage(w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"], w["c_len"])
    b.run(sr.score_params(*SP), sr.align_opts())
    return s, b


def _check(sr, b, w, o, kind, n_best):
    rep = b.report(kind, n_best)
    exp = O.report_batch(o, w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"], kind, n_best)
    offs, hits = rep["offsets"], rep["hits"]
    assert len(offs) == len(exp) + 1 and offs[0] == 0
    bad = 0
    for r, e in enumerate(exp):
        g = hits[int(offs[r]):int(offs[r + 1])]
        if not np.array_equal(g["item"].astype(np.int64), np.asarray(e, np.int64)):
            bad += 1
            continue
        if len(e):
            e = np.asarray(e)
            assert np.array_equal(g["score"], o["item_score"][e])
            assert np.array_equal(g["end_col"].astype(np.int64), o["item_end_j"][e].astype(np.int64))
            assert np.array_equal(g["ref_end"].astype(np.int64),
                                  np.asarray(w["c_start"], np.int64)[e] + o["item_end_j"][e].astype(np.int64) - 1)
            assert np.array_equal(g["ref_id"], np.asarray(w["c_ref"])[e])
            assert np.array_equal(g["strand"], np.asarray(w["c_strand"])[e])
    assert bad == 0, f"{bad} reads differ"
    return rep


@pytest.mark.parametrize("name,scale", [("c2", 0.0005), ("c5", 0.003), ("c1", 0.05)])
def test_report_vs_oracle(sr, name, scale):
    w = S.workload(name, scale=scale, seed=61)
    s, b = _run(sr, w)
    o = oracle_run(w)
    for n_best in (1, 3, 8, 256):
        _check(sr, b, w, o, sr.REPORT_BEST_N, n_best)
    rep = _check(sr, b, w, o, sr.REPORT_TIED, 1)
    # the tied report has n_ties entries per read; N = 1 is the winner
    g = b.fetch()
    cnt = np.diff(rep["offsets"].astype(np.int64))
    assert np.array_equal(cnt, g["best"]["n_ties"].astype(np.int64))
    one = b.report(sr.REPORT_BEST_N, 1)
    has = g["best"]["item"] >= 0
    assert np.array_equal(np.diff(one["offsets"].astype(np.int64)), has.astype(np.int64))
    assert np.array_equal(one["hits"]["item"], g["best"]["item"][has])


def test_report_duplicate_and_same_end_windows(sr):
    """Repeated windows and windows that end at the same reference base hold the
    same alignment: reported once."""
    rng = np.random.default_rng(5)
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), 4000)
    reads, offs = [], [0]
    cand = dict(cand_off=[0], c_ref=[], c_strand=[], c_start=[], c_len=[])
    for k in range(40):
        m = int(rng.integers(30, 120))
        pos = int(rng.integers(200, 3500))
        reads.append(ref[pos:pos + m].copy())
        offs.append(offs[-1] + m)
        wins = [(pos - 10, m + 20), (pos - 10, m + 20), (pos - 5, m + 15), (pos - 20, m + 20),
                (int(rng.integers(0, 3800)), 150), (pos + m // 2, m)]
        for st, ln in wins:
            cand["c_ref"].append(0); cand["c_strand"].append(0)
            cand["c_start"].append(st); cand["c_len"].append(ln)
        cand["cand_off"].append(len(cand["c_ref"]))
    w = dict(refs=[ref], bases=np.concatenate(reads), read_off=np.array(offs),
             **{k: np.array(v) for k, v in cand.items()})
    s, b = _run(sr, w)
    o = oracle_run(w)
    for n_best in (1, 2, 4, 6):
        _check(sr, b, w, o, sr.REPORT_BEST_N, n_best)
    _check(sr, b, w, o, sr.REPORT_TIED, 1)


def test_report_bad_arguments_and_empty(sr):
    w = S.workload("c1", scale=0.002, seed=3)
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    b = s.stage(w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"], w["c_len"])
    with pytest.raises(sr.SrError) as e:
        b.report(sr.REPORT_BEST_N, 1)  # not run yet
    assert e.value.status == sr.SR_EINVAL
    b.run(sr.score_params(*SP), sr.align_opts())
    for kind, nb in [(sr.REPORT_BEST_N, 0), (sr.REPORT_BEST_N, 257), (3, 1)]:
        with pytest.raises(sr.SrError) as e:
            b.report(kind, nb)
        assert e.value.status == sr.SR_EINVAL
    n = len(w["read_off"]) - 1
    w0 = dict(w, cand_off=np.zeros(n + 1, np.int64), c_ref=np.zeros(0, np.uint8),
              c_strand=np.zeros(0, np.uint8), c_start=np.zeros(0, np.int64), c_len=np.zeros(0, np.int32))
    b0 = s.stage(w0["bases"], w0["read_off"], w0["cand_off"], w0["c_ref"], w0["c_strand"], w0["c_start"], w0["c_len"])
    b0.run(sr.score_params(*SP), sr.align_opts())
    rep = b0.report(sr.REPORT_TIED, 1)
    assert len(rep["hits"]) == 0 and np.all(rep["offsets"] == 0)


def test_session_closed_before_its_batches(sr):
    """A batch keeps its session alive: closing the session first, then freeing
    the batch (the order a garbage collector may pick) is safe."""
    w = S.workload("c1", scale=0.002, seed=9)
    for _ in range(3):
        s, b = _run(sr, w)
        g = b.fetch()
        s.close()
        b.close()
        assert g["n_reads"] == len(w["read_off"]) - 1


def test_sam_from_gpu_results(sr, tmp_path):
    """SAM written from the device's results carries the oracle's alignments."""
    w = S.workload("c2", scale=0.0003, seed=21, rc_frac=0.5)
    s, b = _run(sr, w)
    g = b.fetch()
    rep = b.report(sr.REPORT_BEST_N, 4)
    path = tmp_path / "gpu.sam"
    sr.write_sam(path, w["bases"], w["read_off"], g, [len(w["refs"][0])], report=rep)
    o = oracle_run(w)
    lines = [ln.rstrip("\n").split("\t") for ln in open(path) if not ln.startswith("@")]
    assert len(lines) == len(w["read_off"]) - 1
    ops = "MIDNSHP=X"
    for r, f in enumerate(lines):
        ob = o["best"][r]
        if ob["item"] < 0:
            assert f[1] == "4"
            continue
        assert int(f[3]) == int(ob["ref_start"]) + 1
        assert f[5] == "".join(f"{int(x) >> 4}{ops[int(x) & 15]}" for x in o["cigar"][r][:int(ob["cigar_len"])])
        assert f"AS:i:{int(ob['score'])}" in f[11:]
