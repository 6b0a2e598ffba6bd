"""GPU path vs oracle, element by element, on seeded synthetic inputs (-m gpu).

Every case calls libsr through its C ABI (the ctypes binding) and compares item
scores and end columns, per-read winner / second / ties, per-reference bests,
winner CIGARs and classes with the oracle, bit-exactly (integer DP).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_00106_gb300 import synth as S

from .parity import compare, edge_workload, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

SP = (2, 3, 5, 2)


@pytest.fixture(scope="module")
def sr():
    from paper_1805_00106_gb300 import sr as _sr
    _sr.lib()
    return _sr


def _session(sr, w):
    return sr.Session.open([bytes(r) for r in w["refs"]])


def _check(g, o, **kw):
    bad = compare(g, o, **kw)
    assert not bad, "\n".join(bad)


@pytest.mark.parametrize("engine", [0, 1])
def test_c1_small_both_engines(sr, engine):
    w = S.workload("c1", scale=0.02, seed=3)
    s = _session(sr, w)
    g = gpu_run(s, w, engine=engine)
    _check(g, oracle_run(w))


@pytest.mark.parametrize("engine", [0, 1])
def test_c2_small_uneven_lengths(sr, engine):
    w = S.workload("c2", scale=0.0006, seed=5)
    s = _session(sr, w)
    _check(gpu_run(s, w, engine=engine), oracle_run(w))


def test_reverse_strand_reads(sr):
    w = S.workload("c2", scale=0.0004, seed=7, rc_frac=0.5)
    s = _session(sr, w)
    _check(gpu_run(s, w), oracle_run(w))


@pytest.mark.parametrize("shape", [(4, 16), (4, 20), (4, 24), (4, 28), (4, 32)] +
                         [(8, r) for r in (8, 10) + tuple(range(12, 33))] +
                         [(16, r) for r in range(5, 17)] + [(32, r) for r in range(4, 9)])
def test_forced_kernel_shapes(sr, shape):
    g_, r_ = shape
    cap = g_ * r_
    w = S.workload("c2", scale=0.0003, seed=11)
    # keep reads the shape covers
    m = np.diff(w["read_off"])
    keep = np.nonzero(m <= cap)[0]
    w = subset(w, keep)
    s = _session(sr, w)
    _check(gpu_run(s, w, lanes=g_, rows=r_), oracle_run(w))
    if shape in [(16, 16), (32, 8)]:  # the plain engine's shapes
        _check(gpu_run(s, w, lanes=g_, rows=r_, engine=1), oracle_run(w))


def test_int32_path_forced(sr):
    w = S.workload("c1", scale=0.01, seed=13)
    s = _session(sr, w)
    g = gpu_run(s, w, force_i32=True)
    _check(g, oracle_run(w))
    assert g["n_i32_items"] == g["n_items"] > 0
    assert gpu_run(s, w)["n_i32_items"] == 0


def test_overflow_promotion_large_match_score(sr):
    """match = 200: 250 identical bases score 50000 > int16; those items must be
    promoted to the int32 kernel and still agree with the oracle."""
    rng = np.random.default_rng(17)
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), 6000)
    reads, offs, cands = [], [0], dict(cand_off=[0], c_ref=[], c_strand=[], c_start=[], c_len=[])
    for k, m in enumerate([250, 200, 120, 60, 16]):
        pos = 300 + 900 * k
        reads.append(ref[pos:pos + m])
        offs.append(offs[-1] + m)
        for st in (pos - 20, pos + 400):
            cands["c_ref"].append(0); cands["c_strand"].append(0)
            cands["c_start"].append(st); cands["c_len"].append(m + 40)
        cands["cand_off"].append(len(cands["c_ref"]))
    w = dict(refs=[ref], bases=np.concatenate(reads), read_off=np.array(offs),
             **{k: np.array(v) for k, v in cands.items()})
    s = _session(sr, w)
    sp = (200, 3, 5, 2)
    o = oracle_run(w, sp=sp)
    assert o["item_score"].max() == 50000
    g = gpu_run(s, w, sp=sp)
    _check(g, o)
    # a match score this large does not fit the 16-bit kernel's tables: every window is int32
    assert g["n_i32_items"] == g["n_items"] == 10


def test_final_row_mode(sr):
    w = S.workload("c2", scale=0.0003, seed=19)
    s = _session(sr, w)
    _check(gpu_run(s, w, mode=1), oracle_run(w, mode=1))
    _check(gpu_run(s, w, mode=1, force_i32=True), oracle_run(w, mode=1))


def subset(w, keep):
    keep = np.asarray(keep)
    roff, coff = w["read_off"], w["cand_off"]
    bases = np.concatenate([w["bases"][roff[r]:roff[r + 1]] for r in keep]) if len(keep) else np.zeros(0, np.uint8)
    new_roff = np.concatenate([[0], np.cumsum([roff[r + 1] - roff[r] for r in keep])]).astype(np.int64)
    items = np.concatenate([np.arange(coff[r], coff[r + 1]) for r in keep]).astype(np.int64) if len(keep) else np.zeros(0, np.int64)
    new_coff = np.concatenate([[0], np.cumsum([coff[r + 1] - coff[r] for r in keep])]).astype(np.int64)
    out = dict(w)
    out.update(bases=bases, read_off=new_roff, cand_off=new_coff, c_ref=w["c_ref"][items],
               c_strand=w["c_strand"][items], c_start=w["c_start"][items], c_len=w["c_len"][items])
    return out


def test_edge_lengths_and_clamped_windows(sr):
    w = edge_workload()
    s = _session(sr, w)
    o = oracle_run(w)
    _check(gpu_run(s, w), o)
    _check(gpu_run(s, w, force_i32=True), o)
    _check(gpu_run(s, w, engine=1), o)


def test_empty_batches(sr):
    w = S.workload("c1", scale=0.005, seed=29)
    s = _session(sr, w)
    n = len(w["read_off"]) - 1
    # no windows for any read
    w0 = dict(w, cand_off=np.zeros(n + 1, np.int64), c_ref=np.zeros(0, np.uint8),
              c_strand=np.zeros(0, np.uint8), c_start=np.zeros(0, np.int64), c_len=np.zeros(0, np.int32))
    g = gpu_run(s, w0)
    assert np.all(g["best"]["item"] == -1) and np.all(g["best"]["score"] == 0)
    # no reads
    wz = dict(w0, bases=np.zeros(0, np.uint8), read_off=np.zeros(1, np.int64), cand_off=np.zeros(1, np.int64))
    g = gpu_run(s, wz)
    assert g["n_reads"] == 0


def test_bad_inputs_are_rejected(sr):
    w = S.workload("c1", scale=0.005, seed=31)
    s = _session(sr, w)
    bad = dict(w, bases=w["bases"].copy())
    bad["bases"][5] = ord("N")
    with pytest.raises(sr.SrError) as e:
        gpu_run(s, bad)
    assert e.value.status == sr.SR_EBADBASE
    bad = dict(w, c_start=w["c_start"].copy())
    bad["c_start"][3] = len(w["refs"][0]) - 2
    with pytest.raises(sr.SrError) as e:
        gpu_run(s, bad)
    assert e.value.status == sr.SR_EINVAL
    # a read longer than 256 bases
    long = dict(w, bases=np.concatenate([w["bases"], np.full(300, ord("A"), np.uint8)]),
                read_off=np.concatenate([w["read_off"], [w["read_off"][-1] + 300]]),
                cand_off=np.concatenate([w["cand_off"], [w["cand_off"][-1]]]))
    with pytest.raises(sr.SrError) as e:
        gpu_run(s, long)
    assert e.value.status == sr.SR_EINVAL
    with pytest.raises(sr.SrError) as e:
        gpu_run(s, w, sp=(2, 3, 5, 0))
    assert e.value.status == sr.SR_EINVAL


def test_xenograft_classification_with_host_index(sr):
    w = S.workload("c3", scale=0.0008, seed=37)
    idx = [sr.Index.build(bytes(r), seed_len=20, address_bases=10, cal_limit=1024) for r in w["refs"]]
    cd = sr.candidates(idx, w["bases"], w["read_off"], seed_stride=1, merge_dist=32, pad=32)
    w.update(cd)
    s = sr.Session.from_indexes(idx)
    g = gpu_run(s, w, classify=True, min_score=40, margin=5)
    o = oracle_run(w)
    _check(g, o, classify=(40, 5))
    # re-classification on the device with the paper's exact-tie rule
    b = s.stage(w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"], w["c_len"])
    b.run(sr.score_params(*SP), sr.align_opts())
    cls = b.classify(min_score=40, margin=1)
    exp = [O.classify(int(a), int(bb), 40, 1) for a, bb in zip(o["best_per_ref"]["score"][:, 0],
                                                                 o["best_per_ref"]["score"][:, 1])]
    assert np.array_equal(cls, np.array(exp, np.uint8))


def test_repeated_runs_and_staged_batch_identical(sr):
    w = S.workload("c2", scale=0.0003, seed=41)
    s = _session(sr, w)
    b = s.stage(w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"], w["c_len"])
    outs = []
    for _ in range(3):
        b.run(sr.score_params(*SP), sr.align_opts())
        outs.append(b.fetch())
    for o in outs[1:]:
        for k in ["item_score", "item_end", "best", "cigar"]:
            assert np.array_equal(o[k], outs[0][k])
    _check(outs[0], oracle_run(w))
    st = b.stats()
    assert st["kernels"] >= 8 and st["cells"] > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_random_reads_both_readouts(sr, mode):
    """Short, low-complexity reads and windows with several scoring schemes: many
    co-optimal cells (e.g. an earlier row holding the final row's best at the end
    column) exercise the tie rules of the end cell and of the traceback."""
    rng = np.random.default_rng(101 + mode)
    L = 5000
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), L)
    ref[1000:1600] = np.frombuffer(b"AC" * 300, np.uint8)
    ref[2000:2600] = np.frombuffer(b"AAT" * 200, np.uint8)
    reads, offs = [], [0]
    cand = dict(cand_off=[0], c_ref=[], c_strand=[], c_start=[], c_len=[])
    for k in range(1500):
        m = int(rng.integers(1, 31))
        src = int(rng.choice([rng.integers(0, L - 64), rng.integers(1000, 1540), rng.integers(2000, 2540)]))
        r = ref[src:src + m].copy()
        flips = rng.random(m) < 0.15
        r[flips] = rng.choice(np.frombuffer(b"ACGT", np.uint8), int(flips.sum()))
        reads.append(r)
        offs.append(offs[-1] + m)
        for _ in range(int(rng.integers(1, 4))):
            n = int(rng.integers(1, 41))
            st = int(min(max(0, src + int(rng.integers(-8, 9))), L - n))
            cand["c_ref"].append(0); cand["c_strand"].append(int(rng.integers(0, 2)))
            cand["c_start"].append(st); cand["c_len"].append(n)
        cand["cand_off"].append(len(cand["c_ref"]))
    w = dict(refs=[ref], bases=np.concatenate(reads), read_off=np.array(offs),
             **{k: np.array(v) for k, v in cand.items()})
    s = _session(sr, w)
    for sp in [(2, 3, 5, 2), (3, 2, 2, 1), (1, 1, 1, 1), (2, 3, 0, 2)]:
        o = oracle_run(w, sp=sp, mode=mode)
        _check(gpu_run(s, w, sp=sp, mode=mode), o)


def test_bounded_device_wait_times_out_as_a_status(sr):
    """A device wait on a barrier that nothing completes ends after its poll
    limit as SR_ETIMEOUT (status word), and the context stays usable."""
    sr.probe_wait(poll_limit=1000, arrive=True)
    with pytest.raises(sr.SrError) as e:
        sr.probe_wait(poll_limit=1000, arrive=False)
    assert e.value.status == sr.SR_ETIMEOUT
    w = S.workload("c1", scale=0.005, seed=43)
    _check(gpu_run(_session(sr, w), w), oracle_run(w))


def test_outputs_identical_across_runs_and_shapes(sr):
    """Determinism of the queues and atomics: 20 graph replays of one batch give
    byte-identical outputs, and so do other kernel shapes and the plain engine."""
    import hashlib
    w = S.workload("c2", scale=0.0005, seed=47)
    s = _session(sr, w)
    b = s.stage(w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"], w["c_len"])

    def digest(res):
        h = hashlib.sha256()
        for k in ["item_score", "item_end", "best", "best_per_ref", "cigar"]:
            h.update(np.ascontiguousarray(res[k]).tobytes())
        return h.hexdigest()

    ref = None
    for _ in range(20):
        b.run(sr.score_params(*SP), sr.align_opts())
        d = digest(b.fetch())
        ref = ref or d
        assert d == ref
    for opts in [dict(lanes=16, rows=16), dict(lanes=32, rows=8), dict(engine=1)]:
        b.run(sr.score_params(*SP), sr.align_opts(**opts))
        assert digest(b.fetch()) == ref


def _band_widths(w, o, sp=SP):
    """Traceback band width of each read's winner over every row that can end it
    (rows ceil(S / match) .. m) and with its end row known (2 g + 1)."""
    sa, _, go, ge = sp
    m = np.diff(w["read_off"]).astype(np.int64)
    b = o["best"]
    item, S = b["item"].astype(np.int64), b["score"].astype(np.int64)
    ok = (item >= 0) & (S > 0)
    jstar = np.where(ok, o["item_end_j"][np.maximum(item, 0)], 0).astype(np.int64)
    iend = b["read_end"].astype(np.int64)
    g_all = np.maximum(0, (sa * np.minimum(m, jstar) - S - go) // ge)
    w_all = m - np.maximum(1, -(-S // sa)) + 2 * g_all + 1
    g_row = np.maximum(0, (sa * np.minimum(iend, jstar) - S - go) // ge)
    return ok, w_all, 2 * g_row + 1


def test_traceback_band_classes(sr):
    """Winners in every traceback class: bands up to 32 diagonals (one lane per
    diagonal), 33-64 (two per lane), wider ones whose end row comes from the
    extension kernels' winner mode, and wider still (full rectangle)."""
    rng = np.random.default_rng(23)
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), 400_000)
    reads, offs = [], [0]
    cands = dict(cand_off=[0], c_ref=[], c_strand=[], c_start=[], c_len=[])
    for r in range(1500):
        m = int(rng.integers(60, 257))
        pos = int(rng.integers(2000, len(ref) - 2000))
        src = ref[pos:pos + m + 40].copy()
        sub, indel = [(0.0, 0.0), (0.04, 0.01), (0.10, 0.02), (0.2, 0.04)][r % 4]
        out = []
        i = 0
        while len(out) < m and i < len(src):
            u = rng.random()
            if u < indel / 2:
                i += int(rng.integers(1, 6))           # deletion from the read
            elif u < indel:
                out.extend(rng.choice(np.frombuffer(b"ACGT", np.uint8), int(rng.integers(1, 6))))
            else:
                out.append(src[i] if rng.random() >= sub else rng.choice(np.frombuffer(b"ACGT", np.uint8)))
                i += 1
        q = np.array(out[:m], np.uint8)
        if r % 7 == 0:  # only a part of the read in the window: a short local alignment
            q = np.concatenate([q[: m // 3], rng.choice(np.frombuffer(b"ACGT", np.uint8), m - m // 3)])
        reads.append(q)
        offs.append(offs[-1] + len(q))
        for d in (-32, int(rng.integers(-300, 300))):
            cands["c_ref"].append(0)
            cands["c_strand"].append(0)
            cands["c_start"].append(pos + d)
            cands["c_len"].append(len(q) + 64)
        cands["cand_off"].append(len(cands["c_ref"]))
    w = dict(refs=[ref], bases=np.concatenate(reads), read_off=np.array(offs, np.int64),
             **{k: np.array(v) for k, v in cands.items()})
    o = oracle_run(w)
    ok, w_all, w_row = _band_widths(w, o)
    assert np.sum(ok & (w_all <= 32)) > 100
    assert np.sum(ok & (w_all > 32) & (w_all <= 64)) > 50
    assert np.sum(ok & (w_all > 64) & (w_row <= 64)) > 20
    assert np.sum(ok & (w_row > 64)) > 5
    s = _session(sr, w)
    _check(gpu_run(s, w), o)


def test_traceback_reads_overhanging_the_window_start(sr):
    """Reads whose first o bases (1..40) lie before their window's start, from
    both strands: the alignment is soft-clipped at the read's start and its band
    reaches left of column 1 by about o diagonals, so the two-reads-per-thread
    kernels run rows whose first cells are virtual (in the first 16-cell slice,
    and for o > 16 in the second slice of the 32-cell rows)."""
    rng = np.random.default_rng(31)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    comp = np.zeros(256, np.uint8)
    comp[list(b"ACGT")] = list(b"TGCA")
    ref = rng.choice(acgt, 300_000)
    reads, offs, over = [], [0], []
    cands = dict(cand_off=[0], c_ref=[], c_strand=[], c_start=[], c_len=[])
    for r in range(1200):
        m = int(rng.integers(80, 257))
        o = int(rng.integers(1, 41))
        pos = int(rng.integers(1000, len(ref) - 1000))
        q = ref[pos:pos + m].copy()
        hit = rng.random(m) < [0.0, 0.01, 0.03][r % 3]
        q[hit] = rng.choice(acgt, int(hit.sum()))
        strand = r % 2
        if strand:
            q = comp[q[::-1]]  # the read as sequenced from the other strand
        reads.append(q)
        offs.append(offs[-1] + m)
        over.append(o)
        cands["c_ref"].append(0)
        cands["c_strand"].append(strand)
        cands["c_start"].append(pos + o)
        cands["c_len"].append(m + 64 - o)
        cands["cand_off"].append(len(cands["c_ref"]))
    w = dict(refs=[ref], bases=np.concatenate(reads), read_off=np.array(offs, np.int64),
             **{k: np.array(v) for k, v in cands.items()})
    o_run = oracle_run(w)
    ok, w_all, _ = _band_widths(w, o_run)
    over = np.array(over)
    assert np.sum(ok & (w_all <= 16) & (over >= 4)) > 50
    assert np.sum(ok & (w_all > 16) & (w_all <= 32) & (over > 16)) > 50
    assert np.all(o_run["best"]["read_start"][ok] > 1)
    s = _session(sr, w)
    _check(gpu_run(s, w), o_run)


def test_bad_window_in_a_large_batch_reports_the_first(sr):
    """Batches of 64k reads and more are validated in parallel on the host pool:
    the first malformed window (lowest index) is reported, before any launch."""
    w = S.workload("c2", scale=0.08, seed=41)
    assert len(w["read_off"]) - 1 >= 65536
    s = _session(sr, w)
    n_items = len(w["c_len"])
    for field, value in (("c_ref", 7), ("c_len", 0), ("c_strand", 2), ("c_start", 1 << 60)):
        bad = dict(w, **{field: w[field].copy()})
        k1, k2 = n_items // 3, (2 * n_items) // 3
        bad[field][k2] = value
        bad[field][k1] = value
        with pytest.raises(sr.SrError) as e:
            gpu_run(s, bad)
        assert e.value.status == sr.SR_EINVAL, field
        assert f"window {k1} " in str(e.value), (field, str(e.value))
    # the same batch, unmodified, still runs
    g = gpu_run(s, w, want_cigar=0)
    assert len(g["item_score"]) == n_items


@pytest.mark.parametrize("per_read", [1, 3])
def test_select_lane_groups_with_crowded_reads(sr, per_read):
    """The per-read selection runs 4, 8 or 16 lanes per read by the batch's mean
    windows per read. Batches of mostly one (or three) window per read, where a
    few reads hold 20-40 windows (each window four times, so the winner's
    duplicates must not count as its second best), take the small groups' loop
    path for those reads."""
    w = S.workload("c2", scale=0.002, seed=91, rc_frac=0.5)
    rng = np.random.default_rng(92)
    co = np.asarray(w["cand_off"], np.int64)
    n = len(co) - 1
    keep = []
    for r in range(n):
        c0, c1 = co[r], co[r + 1]
        if c1 == c0:
            keep.append([])
            continue
        if r % 97 == 5:  # a crowded read: its windows repeated, plus decoys
            idx = list(range(c0, c1)) * 4 + list(rng.integers(0, co[-1], 12))
        else:
            idx = list(range(c0, min(c1, c0 + per_read)))
        keep.append(idx)
    items = np.array([i for k in keep for i in k], np.int64)
    cand_off = np.concatenate([[0], np.cumsum([len(k) for k in keep])])
    w2 = dict(w, cand_off=cand_off, **{k: np.asarray(w[k])[items] for k in ["c_ref", "c_strand", "c_start", "c_len"]})
    assert len(items) / n <= (2 if per_read == 1 else 4)
    s = _session(sr, w2)
    o = oracle_run(w2)
    _check(gpu_run(s, w2), o)
    assert int(np.max(np.diff(cand_off))) >= 20
