"""The oracle -- TEST INFRASTRUCTURE ONLY.

ctypes wrapper around ``sr_oracle.c``, the plain scalar CPU restatement of the
extension step of McVicar et al., "FPGA Acceleration of Short Read Alignment"
(arXiv 1805.00106): affine-gap Smith-Waterman per (read, window) item (Sec. 3.5),
the per-read score tracker (Sec. 3.6, 4.2), winner traceback/CIGAR (Sec. 6.4)
and two-reference classification (Sec. 6.1-6.4), plus a brute-force CAL
finder/filter (Sec. 3.1-3.3).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this module.  The product package never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CIGAR_CAP = 1040
OP_M, OP_I, OP_D, OP_S = 0, 1, 2, 4
CLASS_UNALIGNED, CLASS_A, CLASS_B, CLASS_AMBIGUOUS = 0, 1, 2, 3


class Score(C.Structure):
    _fields_ = [("match", C.c_int32), ("mismatch", C.c_int32),
                ("gap_open", C.c_int32), ("gap_extend", C.c_int32)]


class Aln(C.Structure):
    _fields_ = [("score", C.c_int32), ("end_i", C.c_int32), ("end_j", C.c_int32),
                ("start_i", C.c_int32), ("start_j", C.c_int32), ("n_cigar", C.c_int32)]


class Hit(C.Structure):
    _fields_ = [("score", C.c_int32), ("second", C.c_int32), ("n_ties", C.c_uint32),
                ("item", C.c_int32), ("ref_id", C.c_int32), ("strand", C.c_int32),
                ("ref_start", C.c_int64), ("ref_end", C.c_int64),
                ("read_start", C.c_int32), ("read_end", C.c_int32), ("cigar_len", C.c_uint32)]


HIT_DTYPE = np.dtype([("score", "<i4"), ("second", "<i4"), ("n_ties", "<u4"), ("item", "<i4"),
                      ("ref_id", "<i4"), ("strand", "<i4"), ("ref_start", "<i8"),
                      ("ref_end", "<i8"), ("read_start", "<i4"), ("read_end", "<i4"),
                      ("cigar_len", "<u4"), ("_pad", "<u4")])
assert HIT_DTYPE.itemsize == C.sizeof(Hit)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vectorisation pragmas)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.or_encode.argtypes = [C.c_char_p, C.c_int64, P]
        L.or_encode.restype = C.c_int
        L.or_revcomp.argtypes = [P, C.c_int64, P]
        L.or_align.argtypes = [P, C.c_int, P, C.c_int, C.POINTER(Score), C.c_int, P, C.c_int,
                               C.POINTER(Aln)]
        L.or_align.restype = C.c_int
        L.or_select.argtypes = [C.c_int, P, P, P, P, P, C.c_int, P, P, P, P]
        L.or_report.argtypes = [C.c_int, P, P, P, P, P, C.c_int, C.c_int, C.c_int, P]
        L.or_report.restype = C.c_int
        L.or_classify.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        L.or_classify.restype = C.c_int
        L.or_candidates.argtypes = [C.c_int, P, P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_int, C.c_int, P, P, P, P, P]
        L.or_candidates.restype = C.c_int
        L.or_run_batch.argtypes = [C.c_int, P, P, C.c_int, P, P, P, P, P, P, P,
                                   C.POINTER(Score), C.c_int, P, P, P, P, P, P]
        L.or_run_batch.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def encode(seq) -> np.ndarray:
    b = seq.encode() if isinstance(seq, str) else bytes(seq)
    out = np.empty(len(b), np.uint8)
    if lib().or_encode(b, len(b), _p(out)) != 0:
        raise ValueError("non-ACGT base")
    return out


def revcomp_codes(codes: np.ndarray) -> np.ndarray:
    codes = np.ascontiguousarray(codes, np.uint8)
    out = np.empty_like(codes)
    lib().or_revcomp(_p(codes), len(codes), _p(out))
    return out


def score_params(match=2, mismatch=3, gap_open=5, gap_extend=2) -> Score:
    return Score(match, mismatch, gap_open, gap_extend)


def align(q, r, sp: Score | None = None, mode: int = 0, want_cigar: bool = True):
    """Align read q to window r (strings or code arrays).  Returns a dict with
    score, end_i, end_j, start_i, start_j and the CIGAR as a list of (len, op)."""
    sp = sp or score_params()
    qc = encode(q) if isinstance(q, (str, bytes)) else np.ascontiguousarray(q, np.uint8)
    rc = encode(r) if isinstance(r, (str, bytes)) else np.ascontiguousarray(r, np.uint8)
    cig = np.zeros(len(qc) + len(rc) + 4, np.uint32)
    a = Aln()
    lib().or_align(_p(qc), len(qc), _p(rc), len(rc), C.byref(sp), mode,
                   _p(cig) if want_cigar else None, len(cig), C.byref(a))
    ops = [(int(w) >> 4, int(w) & 15) for w in cig[: a.n_cigar]]
    return dict(score=a.score, end_i=a.end_i, end_j=a.end_j, start_i=a.start_i,
                start_j=a.start_j, cigar=ops)


def select(scores, ref_ids, strands, gends, cands=None, ref_filter=-1):
    n = len(scores)
    sc = np.ascontiguousarray(scores, np.int32)
    ri = np.ascontiguousarray(ref_ids, np.int32)
    st = np.ascontiguousarray(strands, np.int32)
    ge = np.ascontiguousarray(gends, np.int64)
    cd = np.ascontiguousarray(np.arange(n) if cands is None else cands, np.int32)
    b, s, w = C.c_int32(), C.c_int32(), C.c_int32()
    t = C.c_uint32()
    lib().or_select(n, _p(sc), _p(ri), _p(st), _p(ge), _p(cd), ref_filter,
                    C.byref(b), C.byref(s), C.byref(t), C.byref(w))
    return dict(best=b.value, second=s.value, n_ties=t.value, winner=w.value)


REPORT_BEST_N, REPORT_TIED = 1, 2


def report(scores, ref_ids, strands, gends, kind, n_best=1, cands=None, cap=256):
    """Indices of one read's reported items (Sec. 4.2 tracker options), in order."""
    n = len(scores)
    sc = np.ascontiguousarray(scores, np.int32)
    ri = np.ascontiguousarray(ref_ids, np.int32)
    st = np.ascontiguousarray(strands, np.int32)
    ge = np.ascontiguousarray(gends, np.int64)
    cd = np.ascontiguousarray(np.arange(n) if cands is None else cands, np.int32)
    out = np.zeros(max(cap, 1), np.int32)
    k = lib().or_report(n, _p(sc), _p(ri), _p(st), _p(ge), _p(cd), kind, n_best, cap, _p(out))
    return out[:k].copy()


def report_batch(res: dict, cand_off, c_ref, c_strand, c_start, kind, n_best=1, cap=256):
    """Per read, the global item indices reported from a run_batch result."""
    co = np.asarray(cand_off, np.int64)
    out = []
    for r in range(len(co) - 1):
        c0, c1 = int(co[r]), int(co[r + 1])
        ends = np.asarray(c_start[c0:c1], np.int64) + np.asarray(res["item_end_j"][c0:c1], np.int64) - 1
        idx = report(res["item_score"][c0:c1], c_ref[c0:c1], c_strand[c0:c1], ends, kind, n_best,
                     cands=np.arange(c1 - c0), cap=cap)
        out.append(idx + c0)
    return out


def classify(score_a: int, score_b: int, min_score: int = 40, margin: int = 5) -> int:
    return lib().or_classify(score_a, score_b, min_score, margin)


def candidates(refs, read, k=20, stride=1, merge_dist=32, pad=32, max_cands=0, cal_limit=0,
               cap=4096, with_hits=False):
    """Brute-force CAL finder + filter for one read against a list of references
    (strings or code arrays).  Returns (ref, strand, start, len[, hits]) arrays."""
    rcodes = [encode(r) if isinstance(r, (str, bytes)) else np.ascontiguousarray(r, np.uint8)
              for r in refs]
    q = encode(read) if isinstance(read, (str, bytes)) else np.ascontiguousarray(read, np.uint8)
    ptrs = (C.c_void_p * len(rcodes))(*[r.ctypes.data for r in rcodes])
    lens = np.array([len(r) for r in rcodes], np.int64)
    o_ref = np.zeros(cap, np.int32)
    o_str = np.zeros(cap, np.int32)
    o_st = np.zeros(cap, np.int64)
    o_len = np.zeros(cap, np.int32)
    o_hits = np.zeros(cap, np.int32)
    n = lib().or_candidates(len(rcodes), C.cast(ptrs, C.c_void_p), _p(lens), _p(q), len(q), k,
                            stride, merge_dist, pad, max_cands, cal_limit, cap,
                            _p(o_ref), _p(o_str), _p(o_st), _p(o_len), _p(o_hits))
    if n < 0:
        raise ValueError("candidate capacity exceeded")
    out = (o_ref[:n].copy(), o_str[:n].copy(), o_st[:n].copy(), o_len[:n].copy())
    return out + (o_hits[:n].copy(),) if with_hits else out


def run_batch(ref_codes, reads_bases: np.ndarray, read_off: np.ndarray, cand_off: np.ndarray,
              c_ref, c_strand, c_start, c_len, sp: Score | None = None, mode: int = 0,
              threads: int = 1):
    """Whole-batch oracle: every (read, window) item, per-read tracker and winner
    CIGAR.  ``ref_codes`` are 2-bit code arrays (``encode``).  ``threads`` splits
    the reads into contiguous ranges run concurrently (the C code itself is
    single-threaded)."""
    sp = sp or score_params()
    n_refs = len(ref_codes)
    n_reads = len(read_off) - 1
    n_items = int(cand_off[-1])
    bases = np.ascontiguousarray(reads_bases, np.uint8)
    read_off = np.ascontiguousarray(read_off, np.int64)
    cand_off = np.ascontiguousarray(cand_off, np.int64)
    c_ref = np.ascontiguousarray(c_ref, np.uint8)
    c_strand = np.ascontiguousarray(c_strand, np.uint8)
    c_start = np.ascontiguousarray(c_start, np.int64)
    c_len = np.ascontiguousarray(c_len, np.int32)
    ptrs = (C.c_void_p * n_refs)(*[r.ctypes.data for r in ref_codes])
    lens = np.array([len(r) for r in ref_codes], np.int64)
    item_score = np.zeros(n_items, np.int32)
    item_end_i = np.zeros(n_items, np.int32)
    item_end_j = np.zeros(n_items, np.int32)
    best = np.zeros(n_reads, HIT_DTYPE)
    per_ref = np.zeros(n_reads * n_refs, HIT_DTYPE)
    cigar = np.zeros(n_reads * CIGAR_CAP, np.uint32)
    L = lib()

    def run(lo, hi):
        lo, hi = int(lo), int(hi)
        if hi <= lo:
            return 0
        ro = read_off[lo:]
        co = cand_off[lo:]
        return L.or_run_batch(n_refs, C.cast(ptrs, C.c_void_p), _p(lens), hi - lo, _p(bases),
                              _p(ro), _p(co), _p(c_ref), _p(c_strand), _p(c_start), _p(c_len),
                              C.byref(sp), mode, _p(item_score), _p(item_end_i), _p(item_end_j),
                              C.c_void_p(best.ctypes.data + lo * HIT_DTYPE.itemsize),
                              C.c_void_p(per_ref.ctypes.data + lo * n_refs * HIT_DTYPE.itemsize),
                              C.c_void_p(cigar.ctypes.data + lo * CIGAR_CAP * 4))

    if threads <= 1:
        st = run(0, n_reads)
    else:
        bounds = np.linspace(0, n_reads, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            sts = list(ex.map(lambda k: run(bounds[k], bounds[k + 1]), range(threads)))
        st = min(sts) if sts else 0
    if st != 0:
        raise ValueError(f"oracle batch failed: {st}")
    return dict(item_score=item_score, item_end_i=item_end_i, item_end_j=item_end_j, best=best,
                best_per_ref=per_ref.reshape(n_reads, n_refs), cigar=cigar.reshape(n_reads, CIGAR_CAP))


def cigar_list(cigar_row: np.ndarray, n: int):
    return [(int(w) >> 4, int(w) & 15) for w in cigar_row[:n]]
