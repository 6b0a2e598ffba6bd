"""Host stage (k-mer index + CAL finder/filter, Sec. 3.1-3.3) of libsr against
the oracle's brute-force CAL finder, bit-exactly (CPU only)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_00106_gb300 import synth as S


@pytest.fixture(scope="module")
def sr():
    from paper_1805_00106_gb300 import sr as _sr
    _sr.lib()
    return _sr


def oracle_cands(refs, w, k, stride, merge, pad, max_cands=0, cal_limit=0):
    off = [0]
    cols = {c: [] for c in ["c_ref", "c_strand", "c_start", "c_len"]}
    rc = [O.encode(bytes(r)) for r in refs]
    for r in range(len(w["read_off"]) - 1):
        read = w["bases"][w["read_off"][r]: w["read_off"][r + 1]]
        a, b, c, d = O.candidates(rc, O.encode(bytes(read)), k=k, stride=stride, merge_dist=merge,
                                  pad=pad, max_cands=max_cands, cal_limit=cal_limit)
        cols["c_ref"] += list(a); cols["c_strand"] += list(b); cols["c_start"] += list(c); cols["c_len"] += list(d)
        off.append(off[-1] + len(a))
    return dict(cand_off=np.array(off), **{k_: np.array(v, np.int64) for k_, v in cols.items()})


def same(g, o):
    assert np.array_equal(g["cand_off"], o["cand_off"])
    for k in ["c_ref", "c_strand", "c_start", "c_len"]:
        assert np.array_equal(g[k].astype(np.int64), o[k]), k


@pytest.mark.parametrize("k,stride,addr", [(20, 1, 10), (12, 12, 6), (8, 3, 4), (16, 1, 8)])
def test_candidates_match_bruteforce(sr, k, stride, addr):
    w = S.workload("c3", scale=0.0002, seed=3, rc_frac=0.5)  # two 12.8 kbp references
    w = dict(w, read_off=w["read_off"][:41], bases=w["bases"][: w["read_off"][40]])
    idx = [sr.Index.build(bytes(r), seed_len=k, address_bases=addr) for r in w["refs"]]
    g = sr.candidates(idx, w["bases"], w["read_off"], seed_stride=stride, merge_dist=24, pad=16)
    same(g, oracle_cands(w["refs"], w, k, stride, 24, 16))


def test_cal_limit_and_max_cands_match_bruteforce(sr):
    ref, _ = S.ref_repeats(30000, seed=5, rep_frac=0.5, n_families=20)
    rd = S.reads([ref], 30, 7, 100, 100, 0.01, 0.0, 0.3)
    w = dict(refs=[ref], **rd)
    for limit, maxc in [(0, 0), (3, 0), (0, 4), (2, 3)]:
        idx = [sr.Index.build(bytes(ref), seed_len=14, address_bases=7, cal_limit=limit)]
        g = sr.candidates(idx, w["bases"], w["read_off"], seed_stride=2, merge_dist=10, pad=8,
                          max_cands=maxc)
        same(g, oracle_cands([ref], w, 14, 2, 10, 8, max_cands=maxc, cal_limit=limit))


def test_index_save_load_roundtrip(sr, tmp_path):
    ref = S.ref_iid(20000, seed=9)
    idx = sr.Index.build(bytes(ref), seed_len=18, address_bases=9, cal_limit=50)
    p = tmp_path / "ref.sridx"
    idx.save(str(p))
    idx2 = sr.Index.load(str(p))
    assert idx.info() == idx2.info()
    rd = S.reads([ref], 20, 11, 90, 110)
    a = sr.candidates([idx], rd["bases"], rd["read_off"])
    b = sr.candidates([idx2], rd["bases"], rd["read_off"])
    for k in a:
        assert np.array_equal(a[k], b[k])
    raw = bytearray(p.read_bytes())
    raw[100] ^= 0xFF
    p.write_bytes(bytes(raw))
    with pytest.raises(sr.SrError) as e:
        sr.Index.load(str(p))
    assert e.value.status == sr.SR_EIO


def test_every_reference_kmer_found_and_limit(sr):
    ref = S.ref_iid(5000, seed=13)
    idx = sr.Index.build(bytes(ref), seed_len=16, address_bases=8)
    assert idx.info()["n_entries"] == 5000 - 16 + 1
    # each reference 40-mer finds its own locus on '+'
    pos = np.arange(0, 4900, 97)
    bases = np.concatenate([ref[p:p + 40] for p in pos])
    off = np.arange(len(pos) + 1) * 40
    g = sr.candidates([idx], bases, off, pad=0, merge_dist=0)
    for r, p in enumerate(pos):
        sl = slice(g["cand_off"][r], g["cand_off"][r + 1])
        assert any(s == p and st == 0 for s, st in zip(g["c_start"][sl], g["c_strand"][sl]))


def test_pigeonhole_via_index(sr):
    rng = np.random.default_rng(17)
    ref = S.ref_iid(40000, seed=15)
    idx = sr.Index.build(bytes(ref), seed_len=22, address_bases=11)
    reads, off, truth = [], [0], []
    for _ in range(60):
        p = int(rng.integers(0, 40000 - 88))
        r = ref[p:p + 88].copy()
        for q in rng.choice(88, int(rng.integers(0, 4)), replace=False):
            r[q] = [c for c in b"ACGT" if c != r[q]][int(rng.integers(0, 3))]
        reads.append(r); off.append(off[-1] + 88); truth.append(p)
    g = sr.candidates([idx], np.concatenate(reads), np.array(off), seed_stride=22, pad=0, merge_dist=0)
    for r, p in enumerate(truth):
        sl = slice(g["cand_off"][r], g["cand_off"][r + 1])
        assert p in set(g["c_start"][sl].tolist())


def test_bad_inputs(sr):
    with pytest.raises(sr.SrError) as e:
        sr.Index.build(b"ACGTNACGT" * 10, seed_len=8, address_bases=4)
    assert e.value.status == sr.SR_EBADBASE
    with pytest.raises(sr.SrError) as e:
        sr.Index.build(b"ACGT" * 10, seed_len=40, address_bases=4)
    assert e.value.status == sr.SR_EINVAL
    idx = sr.Index.build(b"ACGT" * 100, seed_len=8, address_bases=4)
    with pytest.raises(sr.SrError) as e:
        sr.candidates([idx], np.frombuffer(b"ACGTXACGTACGT", np.uint8), np.array([0, 13]))
    assert e.value.status == sr.SR_EBADBASE


def test_candidate_arrays_outlive_their_dict(sr):
    """The list's arrays are views of the library's buffers: they stay valid (and
    keep their values) after the dict and every other array are dropped, and
    many lists in a row neither leak into each other nor fail to free."""
    import gc
    w = S.workload("c3", scale=0.0002, seed=4, rc_frac=0.5)
    idx = [sr.Index.build(bytes(r), seed_len=16, address_bases=8) for r in w["refs"]]
    g = sr.candidates(idx, w["bases"], w["read_off"], seed_stride=1, merge_dist=24, pad=16)
    want = {k: np.array(v, copy=True) for k, v in g.items()}
    start, off = g["c_start"], g["cand_off"]
    assert start.dtype == np.int64 and off.dtype == np.int64 and g["c_len"].dtype == np.int32
    del g
    gc.collect()
    for _ in range(20):  # other lists allocated and freed meanwhile
        h = sr.candidates(idx, w["bases"][::-1].copy(), w["read_off"], seed_stride=2, merge_dist=0, pad=0)
        del h
    gc.collect()
    assert np.array_equal(start, want["c_start"]) and np.array_equal(off, want["cand_off"])
