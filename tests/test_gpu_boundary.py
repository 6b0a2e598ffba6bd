"""The boundary's device-memory and classification calls (-m gpu), through the
C ABI:

* sr_align_batch on inputs flagged as device memory (CUDA tensors) gives, array
  for array, the results of the same inputs in host memory and of the oracle,
  and rejects bad inputs with the host path's statuses and indexes;
* sr_classify on an sr_results (host records from sr_align_batch or sr_wait,
  or records copied to the device, classes to host or device) equals the
  oracle's classification of the oracle's per-reference bests (Sec. 6.1-6.4).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_00106_gb300 import synth as S

from .parity import compare, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

SP = (2, 3, 5, 2)
KEYS = ["bases", "read_off", "cand_off", "c_ref", "c_strand", "c_start", "c_len"]
ARRAYS = ["item_score", "item_end", "cigar", "read_class"]


@pytest.fixture(scope="module")
def sr():
    from paper_1805_00106_gb300 import sr as _sr
    _sr.lib()
    return _sr


def _dev(w):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())

    def t(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)

    return dict(bases=t(w["bases"], np.uint8), read_off=t(w["read_off"], np.int64),
                cand_off=t(w["cand_off"], np.int64), c_ref=t(w["c_ref"], np.uint8),
                c_strand=t(w["c_strand"], np.uint8), c_start=t(w["c_start"], np.int64),
                c_len=t(w["c_len"], np.int32))


def _same(a, b):
    for k in ARRAYS:
        if a[k] is None or b[k] is None:
            assert a[k] is None and b[k] is None, k
            continue
        assert np.array_equal(a[k], b[k]), k
    for f in a["best"].dtype.names:
        assert np.array_equal(a["best"][f], b["best"][f]), f
        assert np.array_equal(a["best_per_ref"][f], b["best_per_ref"][f]), f
    assert a["cells"] == b["cells"] and a["n_i32_items"] == b["n_i32_items"]


@pytest.mark.parametrize("name,scale,rc", [("c2", 0.003, 0.5), ("c1", 0.05, 0.0)])
def test_device_inputs_equal_host_inputs_and_oracle(sr, name, scale, rc):
    import torch
    w = S.workload(name, scale=scale, seed=61, rc_frac=rc)
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    d = _dev(w)
    torch.cuda.synchronize()
    n_items = int(w["cand_off"][-1])
    for mode in (0, 1):
        g = s.align_device(*[d[k] for k in KEYS], n_items, sr.score_params(*SP), sr.align_opts(mode=mode))
        h = gpu_run(s, w, mode=mode)
        _same(g, h)
        bad = compare(g, oracle_run(w, mode=mode))
        assert not bad, "\n".join(bad)
    s.close()


def test_device_reads_with_host_candidates(sr):
    """Either struct may be on the device: device reads, host windows."""
    import ctypes as C
    import torch
    w = S.workload("c2", scale=0.002, seed=62, rc_frac=0.5)
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    d = _dev(w)
    torch.cuda.synchronize()
    keep = sr._Keep()
    reads = sr.make_reads_device(d["bases"], d["read_off"])
    cands = sr.make_cands(w["cand_off"], w["c_ref"], w["c_strand"], w["c_start"], w["c_len"], keep)
    out = C.POINTER(sr.Results)()
    st = sr.lib().sr_align_batch(s.h, C.byref(reads), C.byref(cands), C.byref(sr.score_params(*SP)),
                                 C.byref(sr.align_opts()), C.byref(out))
    assert st == 0, sr.lib().sr_last_error()
    _same(sr.results_to_numpy(out), gpu_run(s, w))
    s.close()


def test_device_inputs_bad_window_length_and_base(sr):
    """Device inputs are checked on the device with the host path's statuses,
    naming the same first bad read or window."""
    import torch
    w = S.workload("c2", scale=0.002, seed=63)
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    n_items = int(w["cand_off"][-1])

    def both(bad):
        with pytest.raises(sr.SrError) as eh:
            gpu_run(s, bad)
        d = _dev(bad)
        torch.cuda.synchronize()
        with pytest.raises(sr.SrError) as ed:
            s.align_device(*[d[k] for k in KEYS], int(bad["cand_off"][-1]), sr.score_params(*SP), sr.align_opts())
        return eh.value, ed.value

    # two bad windows: the first (lowest index) is named
    k1, k2 = n_items // 3, 2 * n_items // 3
    bad = dict(w, c_len=w["c_len"].copy())
    bad["c_len"][k2] = 0
    bad["c_start"] = w["c_start"].copy()
    bad["c_start"][k1] = len(w["refs"][0]) - 3  # runs past the reference end
    eh, ed = both(bad)
    assert eh.status == ed.status == sr.SR_EINVAL
    assert f"window {k1} " in str(eh) and f"window {k1} " in str(ed), (str(eh), str(ed))
    # a read longer than 256 bases (its neighbour absorbs the length)
    off = w["read_off"].astype(np.int64).copy()
    r = int(np.nonzero(off[2:] - off[:-2] >= 300)[0][0])  # two neighbours of 300 bases or more
    off[r + 1] = off[r] + 300
    eh, ed = both(dict(w, read_off=off))
    assert eh.status == ed.status == sr.SR_EINVAL
    assert f"read {r} " in str(eh) and f"read {r} " in str(ed), (str(eh), str(ed))
    # a non-ACGT base: found by the read-packing kernel in both paths
    b2 = w["bases"].copy()
    b2[len(b2) // 2] = ord("N")
    eh, ed = both(dict(w, bases=b2))
    assert eh.status == ed.status == sr.SR_EBADBASE
    # unknown flag bits are refused
    import ctypes as C
    d = _dev(w)
    reads = sr.make_reads_device(d["bases"], d["read_off"])
    reads.flags = 3
    cands = sr.make_cands_device(d["cand_off"], d["c_ref"], d["c_strand"], d["c_start"], d["c_len"], n_items)
    out = C.POINTER(sr.Results)()
    assert sr.lib().sr_align_batch(s.h, C.byref(reads), C.byref(cands), C.byref(sr.score_params(*SP)),
                                   C.byref(sr.align_opts()), C.byref(out)) == sr.SR_EINVAL
    # the session still aligns afterwards
    _same(gpu_run(s, w), gpu_run(s, w))
    s.close()


def _expected_classes(o, min_score, margin):
    return np.array([O.classify(int(a), int(b), min_score, margin)
                     for a, b in zip(o["best_per_ref"]["score"][:, 0], o["best_per_ref"]["score"][:, 1])], np.uint8)


def test_classify_results_host_and_device(sr):
    import torch
    w = S.workload("c3", scale=0.004, seed=64, rc_frac=0.3)
    idx = [sr.Index.build(bytes(r), seed_len=20, address_bases=12) for r in w["refs"]]
    w.update(sr.candidates(idx, w["bases"], w["read_off"]))
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    g = gpu_run(s, w)
    o = oracle_run(w)
    assert not compare(g, o)
    for min_score, margin in ((40, 5), (40, 1), (60, 3), (0, 1), (200, 5)):
        exp = _expected_classes(o, min_score, margin)
        assert np.array_equal(sr.classify(g, min_score, margin), exp), (min_score, margin)
        # records and classes in device memory
        per = torch.from_numpy(np.ascontiguousarray(g["best_per_ref"]).view(np.uint8).reshape(-1)).cuda()
        out = torch.full((len(exp),), 255, dtype=torch.uint8, device="cuda")
        sr.classify(dict(best_per_ref=per, n_reads=g["n_reads"], n_refs=g["n_refs"]), min_score, margin, out=out)
        assert np.array_equal(out.cpu().numpy(), exp), (min_score, margin)
    # every class occurs in this workload at the paper's margin of 5
    assert set(np.unique(sr.classify(g, 40, 5))) >= {sr.CLASS_A, sr.CLASS_B}
    s.close()


def test_classify_served_results(sr):
    """A result taken from the server (sr_wait) classifies like the oracle."""
    w = S.workload("c3", scale=0.002, seed=65)
    idx = [sr.Index.build(bytes(r), seed_len=20, address_bases=12) for r in w["refs"]]
    w.update(sr.candidates(idx, w["bases"], w["read_off"]))
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    s.serve_start(sr.score_params(*SP), sr.align_opts(classify=True))
    g = s.wait(s.submit(*[w[k] for k in KEYS]), timeout_ms=120_000)
    s.serve_stop()
    o = oracle_run(w)
    exp = _expected_classes(o, 40, 5)
    assert np.array_equal(g["read_class"], exp)
    assert np.array_equal(sr.classify(g, 40, 5), exp)
    assert np.array_equal(sr.classify(g, 40, 1), _expected_classes(o, 40, 1))
    s.close()


def test_classify_needs_two_references(sr):
    w = S.workload("c1", scale=0.01, seed=66)
    s = sr.Session.open([bytes(r) for r in w["refs"]])
    g = gpu_run(s, w)
    with pytest.raises(sr.SrError) as e:
        sr.classify(g)
    assert e.value.status == sr.SR_EINVAL
    s.close()
