"""GPU path at the full sizes of the workloads (-m gpu), in the launch
configuration bench.py times (batched engine, default bins, winner CIGARs).

c1 is checked against the oracle on every read; c2, c3 and c5 on a random
sample of reads the oracle computes one by one, plus size-independent
properties on every read.  c3's windows come from the host index
(sr_candidates), which tests/test_host_stage.py pins to the oracle's
brute-force CAL finder on small references."""
import numpy as np
import pytest

from paper_1805_00106_gb300 import synth as S

from .parity import compare, compare_sampled, oracle_run, subset_reads, whole_batch_properties

pytestmark = pytest.mark.gpu
KEYS = ["bases", "read_off", "cand_off", "c_ref", "c_strand", "c_start", "c_len"]


@pytest.fixture(scope="module")
def sr():
    from paper_1805_00106_gb300 import sr as _sr
    _sr.lib()
    return _sr


def _run(sr, s, w, **opts):
    return s.align(*[w[k] for k in KEYS], sr.score_params(2, 3, 5, 2), sr.align_opts(**opts))


def _sampled(sr, w, g, n, seed, **kw):
    rng = np.random.default_rng(seed)
    reads = np.sort(rng.choice(len(w["read_off"]) - 1, size=min(n, len(w["read_off"]) - 1), replace=False))
    sub = subset_reads(w, reads)
    o = oracle_run(sub, threads=8)
    bad = compare_sampled(g, w, reads, o, **kw)
    assert not bad, "\n".join(bad[:20])
    bad = whole_batch_properties(g, w)
    assert not bad, bad


def test_c1_full_every_read(sr):
    w = S.workload("c1")
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    g = _run(sr, s, w)
    bad = compare(g, oracle_run(w, threads=8))
    assert not bad, bad


def test_c2_full_sampled(sr):
    w = S.workload("c2")
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    g = _run(sr, s, w)
    assert g["n_items"] > 5_900_000
    _sampled(sr, w, g, 1500, 1)


def test_c3_full_sampled_with_classification(sr):
    w = S.workload("c3")
    idx = [sr.Index.build(bytes(r), seed_len=20, address_bases=12, cal_limit=1024) for r in w["refs"]]
    w.update(sr.candidates(idx, w["bases"], w["read_off"], seed_stride=1, merge_dist=32, pad=32))
    s = sr.Session.from_indexes(idx)
    g = _run(sr, s, w, classify=True, min_score=40, margin=5)
    _sampled(sr, w, g, 1500, 2, classify=(40, 5))
    # classification against the generator's truth (informational bound)
    truth = w["t_ref"] + 1
    correct = float(np.mean(g["read_class"] == truth))
    assert correct > 0.8, correct


def test_c5_full_sampled(sr):
    w = S.workload("c5")
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    g = _run(sr, s, w)
    assert int(np.diff(w["cand_off"]).max()) == 256
    _sampled(sr, w, g, 800, 3)


def _staged(sr, s, w, **opts):
    b = s.stage(*[w[k] for k in KEYS])
    try:
        b.run(sr.score_params(2, 3, 5, 2), sr.align_opts(**opts))
        return b.fetch()
    finally:
        b.close()


def _same_results(g, h):
    assert g["n_reads"] == h["n_reads"] and g["n_items"] == h["n_items"] and g["cells"] == h["cells"]
    assert g["n_i32_items"] == h["n_i32_items"]
    for key in ("item_score", "item_end", "cigar"):
        assert np.array_equal(g[key], h[key]), key
    for f in g["best"].dtype.names:
        assert np.array_equal(g["best"][f], h["best"][f]), f
        assert np.array_equal(g["best_per_ref"][f], h["best_per_ref"][f]), f
    if h["read_class"] is not None:
        assert np.array_equal(g["read_class"], h["read_class"])


def test_c2_call_in_two_parts_equals_one_batch(sr):
    """sr_align_batch runs calls of 2^19 reads and more as two batches of
    consecutive reads on two streams; every array, window indexes and CIGAR
    offsets included, equals that of the same reads staged as one batch."""
    w = S.workload("c2")
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    g = _run(sr, s, w)
    h = _staged(sr, s, w)
    _same_results(g, h)
    # the second part's records point past the first part's windows and CIGARs
    n = len(w["read_off"]) - 1
    assert g["best"]["item"][n - 1] >= int(w["cand_off"][n // 2])
    assert g["best"]["cigar_off"][n - 1] > 0.9 * len(g["cigar"])
    # a repeat of the call gives the same arrays (the parts' arenas and pinned blocks are reused)
    _same_results(_run(sr, s, w), h)


def test_c3_call_in_two_parts_with_classification(sr):
    """Two references and classification through the two-part call."""
    w = S.workload("c3", scale=0.3)
    assert len(w["read_off"]) - 1 >= (1 << 19)
    idx = [sr.Index.build(bytes(r), seed_len=20, address_bases=12, cal_limit=1024) for r in w["refs"]]
    w.update(sr.candidates(idx, w["bases"], w["read_off"], seed_stride=1, merge_dist=32, pad=32))
    s = sr.Session.from_indexes(idx)
    opts = dict(classify=True, min_score=40, margin=5)
    _same_results(_run(sr, s, w, **opts), _staged(sr, s, w, **opts))


def test_bad_window_in_a_two_part_call_reports_the_first(sr):
    """A malformed window in either part gives the error a single batch gives:
    the first bad window (lowest index, in the caller's numbering)."""
    w = S.workload("c2", scale=0.6)
    n_items = len(w["c_len"])
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    for k1, k2 in ((n_items * 3 // 4, n_items - 1), (n_items // 4, n_items * 3 // 4)):
        bad = dict(w, c_len=w["c_len"].copy())
        bad["c_len"][k1] = 0
        bad["c_len"][k2] = 0
        with pytest.raises(sr.SrError) as e:
            _run(sr, s, bad)
        assert e.value.status == sr.SR_EINVAL
        assert f"window {k1} " in str(e.value), str(e.value)
    g = _run(sr, s, w, want_cigar=0)
    assert len(g["item_score"]) == n_items and len(g["cigar"]) == 0


def test_two_part_call_whose_last_part_has_long_cigars(sr):
    """The CIGAR block of a call in parts is sized before its last part is done,
    from the words per read so far; reads with many deletions at the end of the
    call overrun that estimate, and the results must still equal one batch's."""
    w = S.workload("c2", scale=0.55, seed=5)
    n = len(w["read_off"]) - 1
    tail = n - n // 8
    off, bases = w["read_off"].astype(np.int64), w["bases"]
    pieces, lens = [bases[: off[tail]]], []
    for r in range(tail, n):
        seq = bases[off[r]: off[r + 1]]
        keep = np.ones(len(seq), bool)
        keep[12::20] = False  # a deletion every 20 bases
        pieces.append(seq[keep])
        lens.append(int(keep.sum()))
    w = dict(w, bases=np.concatenate(pieces),
             read_off=np.concatenate([off[: tail + 1], off[tail] + np.cumsum(lens)]).astype(w["read_off"].dtype))
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    g = _run(sr, s, w)
    _same_results(g, _staged(sr, s, w))
    words = g["best"]["cigar_len"].astype(np.int64)
    # the deletion reads need several times the CIGAR words of the others
    assert words[tail:].mean() > 3 * words[:tail].mean(), (words[tail:].mean(), words[:tail].mean())
