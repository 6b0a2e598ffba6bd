"""Device CAL finder + filter (Sec. 3.2-3.3 on the GPU) vs the host stage,
which is itself pinned to the brute-force finder of the oracle: same windows,
same order, same hit counts, bit-exact (-m gpu)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_00106_gb300 import synth as S

pytestmark = pytest.mark.gpu

KEYS = ["cand_off", "c_ref", "c_strand", "c_start", "c_len", "c_hits"]


@pytest.fixture(scope="module")
def sr():
    from paper_1805_00106_gb300 import sr as _sr
    _sr.lib()
    return _sr


def _same(a, b):
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k], np.int64), np.asarray(b[k], np.int64)), k


# With one hash seed the device index takes its packed form (shared bucket
# starts): 16-bit keys for (20, 12) and (16, 8), 32-bit ones for (20, 10) and
# (22, 11); different hash seeds per reference take the per-reference form
@pytest.mark.parametrize("k,addr,cal_limit,seeds", [(20, 10, 1024, (0, 0)), (22, 11, 0, (0, 0)), (16, 8, 64, (0, 0)),
                                                    (20, 12, 1024, (0, 0)), (20, 12, 1024, (5, 9))])
def test_device_matches_host_xenograft(sr, k, addr, cal_limit, seeds):
    w = S.workload("c3", scale=0.002, seed=17)
    idx = [sr.Index.build(bytes(r), seed_len=k, address_bases=addr, cal_limit=cal_limit, hash_seed=hs)
           for r, hs in zip(w["refs"], seeds)]
    s = sr.Session.from_indexes(idx)
    s.attach_index(idx)
    for prm in [dict(seed_stride=1, merge_dist=32, pad=32), dict(seed_stride=k, merge_dist=32, pad=16),
                dict(seed_stride=3, merge_dist=0, pad=0), dict(seed_stride=1, merge_dist=32, pad=32, max_cands=3),
                dict(seed_stride=1, merge_dist=200, pad=64, max_cands=1)]:
        h = sr.candidates(idx, w["bases"], w["read_off"], **prm)
        d = s.candidates(w["bases"], w["read_off"], **prm)
        _same(d, h)


@pytest.mark.parametrize("heads", ["1", "0"])
def test_packed_index_with_and_without_bucket_heads(sr, monkeypatch, heads):
    """The packed index's lookups through the bucket heads (one access per seed
    for both references) and through the bucket starts and keys give the same
    list as the host stage; SR_CAL_HEADS=0 at attach time leaves the heads out."""
    monkeypatch.setenv("SR_CAL_HEADS", heads)
    w = S.workload("c3", scale=0.002, seed=23, rc_frac=0.5)
    for k, addr in [(16, 8), (20, 12), (24, 12)]:  # 16-bit keys twice, then 32-bit ones
        idx = [sr.Index.build(bytes(r), seed_len=k, address_bases=addr, cal_limit=0) for r in w["refs"]]
        s = sr.Session.from_indexes(idx)
        s.attach_index(idx)
        for prm in [dict(seed_stride=1, merge_dist=32, pad=32), dict(seed_stride=2, merge_dist=0, pad=8, max_cands=2)]:
            _same(s.candidates(w["bases"], w["read_off"], **prm), sr.candidates(idx, w["bases"], w["read_off"], **prm))


def test_device_matches_bruteforce_oracle(sr):
    rng = np.random.default_rng(3)
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), 3000)
    reads, offs = [], [0]
    for m in [15, 20, 21, 40, 77, 100, 150, 256]:
        p = int(rng.integers(0, 3000 - m))
        r = ref[p:p + m].copy()
        if rng.random() < 0.5:
            r = np.frombuffer(bytes(r)[::-1].translate(bytes.maketrans(b"ACGT", b"TGCA")), np.uint8)
        reads.append(r)
        offs.append(offs[-1] + m)
    bases = np.concatenate(reads)
    idx = [sr.Index.build(bytes(ref), seed_len=20, address_bases=10)]
    s = sr.Session.from_indexes(idx)
    s.attach_index(idx)
    d = s.candidates(bases, np.array(offs), seed_stride=1, merge_dist=32, pad=32)
    codes = [O.encode(bytes(ref))]
    for i in range(len(reads)):
        e_ref, e_str, e_st, e_len, e_hits = O.candidates(codes, O.encode(bytes(reads[i])), k=20, stride=1,
                                                        merge_dist=32, pad=32, with_hits=True)
        c0, c1 = int(d["cand_off"][i]), int(d["cand_off"][i + 1])
        got = list(zip(d["c_ref"][c0:c1].tolist(), d["c_strand"][c0:c1].tolist(), d["c_start"][c0:c1].tolist(),
                       d["c_len"][c0:c1].tolist(), d["c_hits"][c0:c1].tolist()))
        assert got == list(zip(e_ref.tolist(), e_str.tolist(), e_st.tolist(), e_len.tolist(), e_hits.tolist()))


@pytest.mark.parametrize("k,addr", [(20, 10), (16, 8)])
def test_reads_with_very_many_cals(sr, k, addr):
    """A tandem repeat gives reads tens of thousands of CALs: the large-read
    filter (global-memory sort) must agree with the host too; a shorter one
    (60 copies) gives a few thousand, the shared-memory filter of mid-size reads.
    With (16, 8) the index takes the packed form with bucket heads, and the
    repeat's buckets (hundreds of entries) spill out of their heads."""
    rng = np.random.default_rng(11)
    unit = rng.choice(np.frombuffer(b"ACGT", np.uint8), 23)
    unit2 = rng.choice(np.frombuffer(b"ACGT", np.uint8), 31)
    unit3 = rng.choice(np.frombuffer(b"ACGT", np.uint8), 37)
    ref = np.concatenate([rng.choice(np.frombuffer(b"ACGT", np.uint8), 2000), np.tile(unit, 900),
                          rng.choice(np.frombuffer(b"ACGT", np.uint8), 2000), np.tile(unit2, 60),
                          rng.choice(np.frombuffer(b"ACGT", np.uint8), 500), np.tile(unit3, 130),
                          rng.choice(np.frombuffer(b"ACGT", np.uint8), 300)])
    t2 = 2000 + 23 * 900 + 2000  # start of the 60-copy repeat
    t3 = t2 + 31 * 60 + 500  # start of the 130-copy repeat: reads of about 10k CALs (four sort tiles)
    reads, offs = [], [0]
    for st, m in [(2500, 200), (3000, 256), (100, 100), (2100, 60), (20000, 120), (t2 + 200, 150),
                  (t2 - 40, 100), (t3 + 400, 100), (t3 + 37 * 128, 120)]:
        reads.append(ref[st:st + m])
        offs.append(offs[-1] + m)
    bases = np.concatenate(reads)
    idx = [sr.Index.build(bytes(ref), seed_len=k, address_bases=addr, cal_limit=0)]
    s = sr.Session.from_indexes(idx)
    s.attach_index(idx)
    for prm in [dict(merge_dist=0, pad=8), dict(merge_dist=32, pad=32), dict(merge_dist=5, pad=0, max_cands=7)]:
        h = sr.candidates(idx, bases, np.array(offs), **prm)
        d = s.candidates(bases, np.array(offs), **prm)
        _same(d, h)
        if prm["merge_dist"] == 0 and k == 20:
            # one window per repeat copy: ~900 windows from ~200k CALs (the large-read path)
            assert int(np.max(np.diff(h["cand_off"]))) > 500
            assert int(np.max(h["c_hits"])) > 100
            # the read inside the 60-copy repeat: 131 seeds x 60 copies, between the small and large paths
            assert 30 <= int(np.diff(h["cand_off"])[5]) <= 120


def test_device_candidates_errors_and_empty(sr):
    w = S.workload("c3", scale=0.0008, seed=5)
    idx = [sr.Index.build(bytes(r), seed_len=20, address_bases=10) for r in w["refs"]]
    s = sr.Session.from_indexes(idx)
    with pytest.raises(sr.SrError) as e:
        s.candidates(w["bases"], w["read_off"])  # no index attached
    assert e.value.status == sr.SR_EINVAL
    s.attach_index(idx)
    bad = w["bases"].copy()
    bad[7] = ord("N")
    with pytest.raises(sr.SrError) as e:
        s.candidates(bad, w["read_off"])
    assert e.value.status == sr.SR_EBADBASE
    long = np.concatenate([w["bases"], np.full(300, ord("A"), np.uint8)])
    lo = np.concatenate([w["read_off"], [w["read_off"][-1] + 300]])
    with pytest.raises(sr.SrError) as e:
        s.candidates(long, lo)
    assert e.value.status == sr.SR_EINVAL
    d = s.candidates(np.zeros(0, np.uint8), np.zeros(1, np.int64))
    assert len(d["cand_off"]) == 1 and len(d["c_ref"]) == 0


def _dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()


def test_device_reads_and_device_list(sr):
    """Reads already in device memory and the list left in device memory give
    the host stage's windows; the device list feeds sr_align_batch as it is,
    with the results of the all-host pipeline."""
    import torch
    w = S.workload("c3", scale=0.002, seed=23, rc_frac=0.5)
    idx = [sr.Index.build(bytes(r), seed_len=20, address_bases=10, cal_limit=1024) for r in w["refs"]]
    s = sr.Session.from_indexes(idx)
    s.attach_index(idx)
    prm = dict(seed_stride=1, merge_dist=32, pad=32)
    h = sr.candidates(idx, w["bases"], w["read_off"], **prm)
    db, do = _dev(w["bases"], np.uint8), _dev(w["read_off"], np.int64)
    torch.cuda.synchronize()
    _same(s.candidates(db, do, **prm), h)                               # device reads, host list
    dl = s.candidates(w["bases"], w["read_off"], out_device=True, **prm)  # host reads, device list
    assert dl.n_cands == len(h["c_ref"]) and dl.n_reads == len(w["read_off"]) - 1
    _same(dl.to_numpy(), h)
    dl2 = s.candidates(db, do, out_device=True, **prm)                   # both on the device
    _same(dl2.to_numpy(), h)
    opts = sr.align_opts(classify=True)
    ref = s.align(w["bases"], w["read_off"], h["cand_off"], h["c_ref"], h["c_strand"], h["c_start"], h["c_len"],
                  sr.score_params(), opts)
    for g in (s.align_cands(db, do, dl2, sr.score_params(), opts),
              s.align_cands(w["bases"], w["read_off"], dl, sr.score_params(), opts)):
        for k in ["item_score", "item_end", "cigar", "read_class"]:
            assert np.array_equal(g[k], ref[k]), k
        assert np.array_equal(g["best"], ref["best"]) and np.array_equal(g["best_per_ref"], ref["best_per_ref"])
    # an empty batch and a read too long, from device reads
    e0 = s.candidates(_dev(np.zeros(0, np.uint8), np.uint8), _dev(np.zeros(1, np.int64), np.int64), out_device=True)
    assert e0.n_cands == 0 and e0.n_reads == 0
    lo = np.concatenate([w["read_off"], [w["read_off"][-1] + 300]])
    long = np.concatenate([w["bases"], np.full(300, ord("A"), np.uint8)])
    torch.cuda.synchronize()
    with pytest.raises(sr.SrError) as e:
        s.candidates(_dev(long, np.uint8), _dev(lo, np.int64))
    assert e.value.status == sr.SR_EINVAL


@pytest.mark.parametrize("records, keys", [(2000, 1 << 26), (1 << 27, 3000), (3000, 2500)])
def test_chunk_and_sub_chunk_cuts(sr, monkeypatch, records, keys):
    """Large calls run in chunks of kept lookups and sub-chunks of CAL bounds,
    both cut on the device where a prefix sum crosses a multiple of the limit
    (less one read's largest share, so that no piece exceeds it).  With the
    limits lowered so that a small batch is cut into many pieces, every output
    equals the uncut call's and the host stage's: host list and device list."""
    import torch
    w = S.workload("c3", scale=0.0015, seed=29, rc_frac=0.5)
    idx = [sr.Index.build(bytes(r), seed_len=20, address_bases=10, cal_limit=1024) for r in w["refs"]]
    s = sr.Session.from_indexes(idx)
    s.attach_index(idx)
    prm = dict(seed_stride=1, merge_dist=32, pad=32)
    h = sr.candidates(idx, w["bases"], w["read_off"], **prm)
    base = s.candidates(w["bases"], w["read_off"], **prm)
    _same(base, h)
    monkeypatch.setenv("SR_CAL_CHUNK_RECORDS", str(records))
    monkeypatch.setenv("SR_CAL_CHUNK_KEYS", str(keys))
    _same(s.candidates(w["bases"], w["read_off"], **prm), h)
    db, do = _dev(w["bases"], np.uint8), _dev(w["read_off"], np.int64)
    torch.cuda.synchronize()
    _same(s.candidates(db, do, out_device=True, **prm).to_numpy(), h)
