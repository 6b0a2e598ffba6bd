"""sr_align_items_noalloc, the allocation-free scoring entry point (-m gpu).

It is for callers that cannot call cudaMalloc (device memory owned by another
allocator, or no tolerance for allocation latency): here PyTorch owns every
input and output buffer, and the entry point must produce, on two calls in a
row, exactly the item scores and end columns that sr_align_batch produces for
the same batch.  Kept in a file that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

from paper_1805_00106_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_noalloc_matches_align_batch_twice():
    import torch
    from paper_1805_00106_gb300 import sr

    w = S.workload("c2", scale=0.002, seed=77)  # 2000 reads, about 12k windows
    sess = sr.Session.open([bytes(r) for r in w["refs"]])
    ref = sess.align(w["bases"], w["read_off"], w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"],
                     w["c_len"], sr.score_params(), sr.align_opts(want_cigar=False))
    dev = torch.device("cuda", torch.cuda.current_device())

    def t(a, dtype):
        return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).to(dev)

    bases = t(w["bases"], np.uint8)
    roff = t(w["read_off"], np.int64)
    coff = t(w["cand_off"], np.int64)
    cref = t(w["c_ref"], np.uint8)
    cstr = t(w["c_strand"], np.uint8)
    cst = t(w["c_start"], np.int64)
    cln = t(w["c_len"], np.int32)
    n_reads = len(w["read_off"]) - 1
    n_items = int(w["cand_off"][-1])
    score = torch.empty(n_items, dtype=torch.int32, device=dev)
    end = torch.empty(n_items, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    sp = sr.score_params()
    L = sr.lib()
    P = C.c_void_p

    def call(nr=n_reads, ni=n_items):
        return L.sr_align_items_noalloc(sess.h, P(bases.data_ptr()), P(roff.data_ptr()), nr,
                                        P(coff.data_ptr()), P(cref.data_ptr()), P(cstr.data_ptr()),
                                        P(cst.data_ptr()), P(cln.data_ptr()), ni, C.byref(sp),
                                        P(score.data_ptr()), P(end.data_ptr()), P(stream))

    for _ in range(2):
        score.fill_(-7)
        end.fill_(-7)
        st = call()
        assert st == 0, L.sr_last_error()
        assert np.array_equal(score.cpu().numpy(), ref["item_score"])
        assert np.array_equal(end.cpu().numpy().astype(np.uint32), ref["item_end"])

    # sizes beyond the fixed scratch are refused with a clear error
    assert call(nr=40000) == sr.SR_EINVAL
    assert b"at most" in L.sr_last_error()
    sess.close()
