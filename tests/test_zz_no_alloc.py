"""sr_align_items_noalloc, the allocation-free scoring entry point (-m gpu).

It is for callers that cannot call cudaMalloc (device memory owned by another
allocator, or no tolerance for allocation latency): here PyTorch owns every
input and output buffer.  The entry point must produce, on two calls in a row,
exactly the item scores and end columns that sr_align_batch produces for the
same batch, and those of the oracle (reads on both strands, edge read lengths,
windows clamped at the reference ends); it must refuse malformed inputs with
the documented statuses and still work afterwards, and a call must leave the
device's free memory unchanged.  Kept in a file that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

from paper_1805_00106_gb300 import synth as S

from .parity import edge_workload, oracle_run

pytestmark = pytest.mark.gpu


class _Items:
    """A batch's inputs and outputs in torch device memory, and the call."""

    def __init__(self, sr, sess, w):
        import torch
        self.sr, self.sess = sr, sess
        dev = torch.device("cuda", torch.cuda.current_device())

        def t(a, dtype):
            return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).to(dev)

        self.bases = t(w["bases"], np.uint8)
        self.roff = t(w["read_off"], np.int64)
        self.coff = t(w["cand_off"], np.int64)
        self.cref = t(w["c_ref"], np.uint8)
        self.cstr = t(w["c_strand"], np.uint8)
        self.cst = t(w["c_start"], np.int64)
        self.cln = t(w["c_len"], np.int32)
        self.n_reads = len(w["read_off"]) - 1
        self.n_items = int(w["cand_off"][-1])
        self.score = torch.empty(max(self.n_items, 1), dtype=torch.int32, device=dev)
        self.end = torch.empty(max(self.n_items, 1), dtype=torch.int32, device=dev)
        self.stream = torch.cuda.current_stream(dev).cuda_stream
        self.sp = sr.score_params()

    def call(self, nr=None, ni=None):
        P = C.c_void_p
        self.score.fill_(-7)
        self.end.fill_(-7)
        return self.sr.lib().sr_align_items_noalloc(
            self.sess.h, P(self.bases.data_ptr()), P(self.roff.data_ptr()), self.n_reads if nr is None else nr,
            P(self.coff.data_ptr()), P(self.cref.data_ptr()), P(self.cstr.data_ptr()), P(self.cst.data_ptr()),
            P(self.cln.data_ptr()), self.n_items if ni is None else ni, C.byref(self.sp), P(self.score.data_ptr()),
            P(self.end.data_ptr()), P(self.stream))

    def results(self):
        return (self.score.cpu().numpy()[: self.n_items],
                self.end.cpu().numpy()[: self.n_items].astype(np.uint32))


def test_noalloc_matches_align_batch_twice():
    from paper_1805_00106_gb300 import sr

    w = S.workload("c2", scale=0.002, seed=77)  # 2000 reads, about 12k windows
    sess = sr.Session.open([bytes(r) for r in w["refs"]])
    ref = sess.align(w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"],
                     w["c_len"], sr.score_params(), sr.align_opts(want_cigar=False))
    it = _Items(sr, sess, w)
    for _ in range(2):
        st = it.call()
        assert st == 0, sr.lib().sr_last_error()
        score, end = it.results()
        assert np.array_equal(score, ref["item_score"])
        assert np.array_equal(end, ref["item_end"])

    # sizes beyond the fixed scratch are refused with a clear error
    assert it.call(nr=40000) == sr.SR_EINVAL
    assert b"at most" in sr.lib().sr_last_error()
    sess.close()


@pytest.mark.parametrize("case", ["both_strands", "edge_lengths"])
def test_noalloc_matches_the_oracle(case):
    from paper_1805_00106_gb300 import sr

    w = S.workload("c2", scale=0.0015, seed=78, rc_frac=0.5) if case == "both_strands" else edge_workload()
    sess = sr.Session.open([bytes(r) for r in w["refs"]])
    o = oracle_run(w)
    it = _Items(sr, sess, w)
    for _ in range(2):
        assert it.call() == 0, sr.lib().sr_last_error()
        score, end = it.results()
        assert np.array_equal(score, o["item_score"])
        assert np.array_equal(end.astype(np.int64), o["item_end_j"].astype(np.int64))
    if case == "both_strands":
        assert 0 < int(np.sum(w["c_strand"])) < len(w["c_strand"])
    sess.close()


def test_noalloc_refuses_bad_inputs_then_works_and_allocates_nothing():
    import torch
    from paper_1805_00106_gb300 import sr

    w = S.workload("c2", scale=0.001, seed=79)
    sess = sr.Session.open([bytes(r) for r in w["refs"]])
    o = oracle_run(w)
    n_items = int(w["cand_off"][-1])

    def expect(bad, status):
        it = _Items(sr, sess, bad)
        assert it.call() == status, sr.lib().sr_last_error()

    coff = w["cand_off"].copy()
    coff[3], coff[4] = coff[4], coff[3] - 1  # decreasing window offsets
    expect(dict(w, cand_off=coff), sr.SR_EINVAL)
    b2 = w["bases"].copy()
    b2[17] = ord("N")
    expect(dict(w, bases=b2), sr.SR_EBADBASE)
    cs = w["c_start"].copy()
    cs[n_items // 2] = len(w["refs"][0]) - 2  # a window running past the reference
    expect(dict(w, c_start=cs), sr.SR_EINVAL)
    cl = w["c_len"].copy()
    cl[n_items // 3] = 513  # longer than a window may be
    expect(dict(w, c_len=cl), sr.SR_EINVAL)

    it = _Items(sr, sess, w)
    assert it.call() == 0, sr.lib().sr_last_error()  # also loads every kernel it uses
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    assert it.call() == 0, sr.lib().sr_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    score, end = it.results()
    assert np.array_equal(score, o["item_score"])
    assert np.array_equal(end.astype(np.int64), o["item_end_j"].astype(np.int64))
    sess.close()
