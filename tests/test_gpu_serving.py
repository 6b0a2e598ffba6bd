"""Continuous batching (serving) through the C ABI (-m gpu): requests submitted
while others run are merged into shared device rounds, and each request's
results are byte-identical to aligning it alone (tolerance 0); HBM-budget
admission, bounded waits and oracle parity of served results."""
import threading
import time

import numpy as np
import pytest

from paper_1805_00106_gb300 import synth as S

from .parity import compare, oracle_run

pytestmark = pytest.mark.gpu

KEYS = ["bases", "read_off", "cand_off", "c_ref", "c_strand", "c_start", "c_len"]


def request_of(refs, n, seed):
    rd = S.reads(refs, n, seed, 75, 250, 0.009, 0.001, 0.0)
    cd = S.cands(rd, [len(r) for r in refs], seed + 1, S.COUNT_UNIFORM, 64, 32, cap_per_read=64)
    return dict(**rd, **cd)


@pytest.fixture(scope="module")
def env():
    from paper_1805_00106_gb300 import sr
    a = S.ref_iid(200_000, seed=1)
    b = S.mutate(a, seed=2, sub=0.15, indel=0.02, nblocks=3, blk_lo=1000, blk_hi=20000)
    reqs = S.serving_batches([a, b], 24, seed=3, max_batch=1500)
    return sr, [a, b], reqs


def test_results_alone_equal_results_in_the_mix(env):
    sr, refs, reqs = env
    s = sr.Session.open([bytes(r) for r in refs], hbm_budget=6 << 30)
    alone = [s.align(*[q[k] for k in KEYS], sr.score_params(), sr.align_opts(classify=True)) for q in reqs]
    s.serve_start(sr.score_params(), sr.align_opts(classify=True), max_inflight=0)
    tickets = [None] * len(reqs)

    def submit(i):
        time.sleep(0.002 * (i % 5))
        tickets[i] = s.submit(*[reqs[i][k] for k in KEYS])

    th = [threading.Thread(target=submit, args=(i,)) for i in range(len(reqs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    served = [s.wait(t, timeout_ms=120_000) for t in tickets]
    st = s.serve_stats()
    s.serve_stop()
    for a, b in zip(alone, served):
        for k in ["item_score", "item_end", "cigar", "read_class"]:
            assert np.array_equal(a[k], b[k]), k
        assert a["cells"] == b["cells"] and a["n_i32_items"] == b["n_i32_items"] == 0
        for f in a["best"].dtype.names:
            assert np.array_equal(a["best"][f], b["best"][f]), f
            assert np.array_equal(a["best_per_ref"][f], b["best_per_ref"][f]), f
    assert st["completed"] == len(reqs)
    assert st["max_round_requests"] >= 2, st  # requests shared device rounds
    assert st["rounds"] < len(reqs)
    assert st["p99_us"] >= st["p50_us"] > 0


def test_served_int32_windows_are_counted(env):
    """A served request's results count its own windows scored by the int32
    kernel, as a call of its own does."""
    sr, refs, reqs = env
    s = sr.Session.open([bytes(r) for r in refs], hbm_budget=6 << 30)
    opts = sr.align_opts(force_i32=True)
    some = reqs[:6]
    alone = [s.align(*[q[k] for k in KEYS], sr.score_params(), opts) for q in some]
    s.serve_start(sr.score_params(), opts, max_inflight=0)
    tickets = [s.submit(*[q[k] for k in KEYS]) for q in some]
    served = [s.wait(t, timeout_ms=120_000) for t in tickets]
    s.serve_stop()
    for q, a, b in zip(some, alone, served):
        assert b["n_i32_items"] == a["n_i32_items"] == len(q["c_len"])
        assert np.array_equal(a["item_score"], b["item_score"])


def test_served_results_match_oracle(env):
    sr, refs, reqs = env
    s = sr.Session.open([bytes(r) for r in refs])
    s.serve_start(sr.score_params(), sr.align_opts())
    q = reqs[0]
    t = s.submit(*[q[k] for k in KEYS])
    g = s.wait(t, timeout_ms=120_000)
    s.serve_stop()
    w = dict(q, refs=refs)
    bad = compare(g, oracle_run(w))
    assert not bad, bad


def test_budget_admission_and_bounded_wait(env):
    sr, refs, reqs = env
    s = sr.Session.open([bytes(r) for r in refs], hbm_budget=64 << 20)
    s.serve_start(sr.score_params(), sr.align_opts(), max_inflight=2)
    big = request_of(refs, 60000, 9)  # needs more than the whole budget
    with pytest.raises(sr.SrError) as e:
        s.submit(*[big[k] for k in KEYS])
    assert e.value.status == sr.SR_ENOMEM
    with pytest.raises(sr.SrError) as e:
        s.wait(987654, timeout_ms=0)
    assert e.value.status == sr.SR_EINVAL
    # several requests that each fit but not all at once: admitted as memory frees
    tickets = [s.submit(*[q[k] for k in KEYS]) for q in reqs[:8]]
    outs = [s.wait(t, timeout_ms=120_000) for t in tickets]
    assert all(o["n_reads"] == len(q["read_off"]) - 1 for o, q in zip(outs, reqs[:8]))
    s.serve_stop()


def test_wait_timeout_returns_etimeout(env):
    sr, refs, _ = env
    s = sr.Session.open([bytes(r) for r in refs])
    s.serve_start(sr.score_params(), sr.align_opts(), max_inflight=1)
    big = request_of(refs, 40000, 11)
    t1 = s.submit(*[big[k] for k in KEYS])
    t2 = s.submit(*[big[k] for k in KEYS])
    with pytest.raises(sr.SrError) as e:
        s.wait(t2, timeout_ms=0)
    assert e.value.status == sr.SR_ETIMEOUT
    a = s.wait(t1, timeout_ms=120_000)
    b = s.wait(t2, timeout_ms=120_000)
    assert np.array_equal(a["item_score"], b["item_score"])
    s.serve_stop()


def test_backlog_drains_in_bounded_rounds(env):
    """A burst totalling more than one round's read cap (131072 reads) is split
    over several rounds, and every request still gets the results it gets alone."""
    sr, refs, _ = env
    reqs = [request_of(refs, 20_000, 100 + i) for i in range(8)]  # 160k reads
    s = sr.Session.open([bytes(r) for r in refs], hbm_budget=16 << 30)
    alone = [s.align(*[q[k] for k in KEYS], sr.score_params(), sr.align_opts()) for q in reqs]
    # a long request first, so the others queue up behind its round
    s.serve_start(sr.score_params(), sr.align_opts(), max_inflight=0)
    tickets = [s.submit(*[q[k] for k in KEYS]) for q in reqs]
    served = [s.wait(t, timeout_ms=120_000) for t in tickets]
    st = s.serve_stats()
    s.serve_stop()
    for a, b in zip(alone, served):
        for k in ["item_score", "item_end", "cigar"]:
            assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a["best"], b["best"])
    assert st["completed"] == len(reqs)
    assert st["rounds"] >= 2
    assert st["max_round_requests"] <= 6  # at most 131072 reads: six requests of 20k


def test_next_round_starts_before_the_previous_one_ends(env):
    """Rounds overlap on the device: with requests arriving while others run,
    the CUDA events the server records on each round's stream show round k+1's
    first kernel finishing before round k's last kernel, and every request's
    results are still those it gets alone."""
    sr, refs, _ = env
    reqs = [request_of(refs, 3000, 300 + i) for i in range(12)]
    s = sr.Session.open([bytes(r) for r in refs], hbm_budget=8 << 30)
    alone = [s.align(*[q[k] for k in KEYS], sr.score_params(), sr.align_opts()) for q in reqs]
    s.serve_start(sr.score_params(), sr.align_opts(), max_inflight=0)
    tickets = []
    for rep in range(4):
        for q in reqs:
            tickets.append(s.submit(*[q[k] for k in KEYS]))
            time.sleep(0.0005)
    served = [s.wait(t, timeout_ms=120_000) for t in tickets]
    ov = s.serve_overlap(cap=4096)
    st = s.serve_stats()
    by_size = s.serve_stats_by_size([2048, 4096])
    s.serve_stop()
    for i, b in enumerate(served):
        a = alone[i % len(reqs)]
        for k in ["item_score", "item_end", "cigar"]:
            assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a["best"], b["best"])
    n = ov["timed_rounds"]
    assert n == st["rounds"] and n >= 2, (ov, st)
    first, last = ov["first_ms"], ov["last_ms"]
    assert np.all(last >= first)
    pairs = int(np.sum(first[1:] < last[:-1]))
    assert pairs == ov["overlapped"] >= 1, (pairs, ov["overlapped"], first[:8], last[:8])
    # every request has 3000 reads: all fall in the second size bucket
    assert by_size[0]["count"] == 0 and by_size[1]["count"] == len(tickets)
    assert by_size[1]["p50_us"] == st["p50_us"] and by_size[1]["p99_us"] == st["p99_us"]
