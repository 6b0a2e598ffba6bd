"""Python binding of libsr (``include/sr.h``): ctypes argument marshalling only.

Every step of the alignment path runs in libsr's CUDA kernels; this module
converts numpy arrays to the C structs and back.  If the shared library is
missing it is built in-tree; if it cannot be built or loaded, the import of the
first call raises -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

SR_OK, SR_EINVAL, SR_ENOMEM, SR_ECUDA, SR_EBADBASE, SR_ETIMEOUT, SR_EBUSY, SR_EIO = 0, -1, -2, -3, -4, -5, -6, -7
MODE_LOCAL, MODE_FINAL_ROW = 0, 1
ENGINE_BATCHED, ENGINE_PLAIN = 0, 1
CLASS_UNALIGNED, CLASS_A, CLASS_B, CLASS_AMBIGUOUS = 0, 1, 2, 3
OP_M, OP_I, OP_D, OP_S = 0, 1, 2, 4
CIGAR_STRIDE = 776
FLAG_DEVICE = 1  # sr_reads / sr_cand_list arrays are device pointers

P = C.c_void_p


class SrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsr status {status}: {msg}")
        self.status = status


class IndexParams(C.Structure):
    _fields_ = [("seed_len", C.c_uint32), ("address_bases", C.c_uint32), ("cal_limit", C.c_uint32),
                ("n_threads", C.c_uint32), ("hash_seed", C.c_uint64)]


class Reads(C.Structure):
    _fields_ = [("n_reads", C.c_uint32), ("flags", C.c_uint32), ("bases", P), ("offsets", P)]


class CandParams(C.Structure):
    _fields_ = [("seed_stride", C.c_uint32), ("merge_dist", C.c_uint32), ("pad", C.c_uint32),
                ("max_cands", C.c_uint32), ("n_threads", C.c_uint32), ("flags", C.c_uint32)]


class CandList(C.Structure):
    _fields_ = [("n_reads", C.c_uint32), ("flags", C.c_uint32), ("n_cands", C.c_uint64),
                ("offsets", P), ("ref_id", P), ("strand", P), ("win_start", P), ("win_len", P),
                ("hits", P)]


class ScoreParams(C.Structure):
    _fields_ = [("match", C.c_int32), ("mismatch", C.c_int32), ("gap_open", C.c_int32),
                ("gap_extend", C.c_int32)]


class AlignOpts(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("engine", C.c_uint32), ("want_cigar", C.c_uint32),
                ("classify", C.c_uint32), ("min_score", C.c_int32), ("margin", C.c_int32),
                ("force_i32", C.c_uint32), ("lanes", C.c_uint32), ("rows", C.c_uint32),
                ("reserved", C.c_uint32), ("cuda_stream", P)]


class Hit(C.Structure):
    _fields_ = [("score", C.c_int32), ("second", C.c_int32), ("n_ties", C.c_uint32),
                ("item", C.c_int32), ("ref_id", C.c_uint8), ("strand", C.c_uint8),
                ("reserved", C.c_uint16), ("read_start", C.c_int32), ("read_end", C.c_int32),
                ("ref_start", C.c_uint64), ("ref_end", C.c_uint64), ("cigar_off", C.c_uint32),
                ("cigar_len", C.c_uint32)]


class Results(C.Structure):
    _fields_ = [("n_reads", C.c_uint32), ("n_refs", C.c_uint32), ("n_items", C.c_uint64),
                ("best", C.POINTER(Hit)), ("best_per_ref", C.POINTER(Hit)), ("item_score", P),
                ("item_end", P), ("cigar", P), ("n_cigar", C.c_uint64), ("read_class", P),
                ("cells", C.c_uint64), ("n_i32_items", C.c_uint64)]


def _np_dtype(st):
    names, fmts, offs = [], [], []
    m = {C.c_int32: "<i4", C.c_uint32: "<u4", C.c_uint8: "u1", C.c_uint16: "<u2", C.c_uint64: "<u8"}
    for name, ty in st._fields_:
        names.append(name)
        fmts.append(m[ty])
        offs.append(getattr(st, name).offset)
    return np.dtype({"names": names, "formats": fmts, "offsets": offs, "itemsize": C.sizeof(st)})


HIT_DTYPE = _np_dtype(Hit)


class ReportHit(C.Structure):
    _fields_ = [("score", C.c_int32), ("item", C.c_int32), ("ref_id", C.c_uint8), ("strand", C.c_uint8),
                ("reserved", C.c_uint16), ("end_col", C.c_uint32), ("ref_end", C.c_uint64)]


class Report(C.Structure):
    _fields_ = [("n_reads", C.c_uint32), ("n_truncated", C.c_uint32), ("n_hits", C.c_uint64),
                ("offsets", P), ("hits", P)]


REPORT_HIT_DTYPE = _np_dtype(ReportHit)


class SamOpts(C.Structure):
    _fields_ = [("read_names", P), ("ref_names", P), ("secondary", C.POINTER(Report))]
REPORT_BEST_N, REPORT_TIED, REPORT_MAX = 1, 2, 256


def lib():
    """Load libsr.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "sr_last_error": ([], C.c_char_p), "sr_version": ([], C.c_char_p),
            "sr_index_build": ([C.c_char_p, C.c_uint64, C.POINTER(IndexParams), C.POINTER(P)], C.c_int32),
            "sr_index_save": ([P, C.c_char_p], C.c_int32),
            "sr_index_load": ([C.c_char_p, C.POINTER(P)], C.c_int32),
            "sr_index_free": ([P], None),
            "sr_index_info": ([P, P, P], C.c_int32),
            "sr_candidates": ([P, C.c_uint32, C.POINTER(Reads), C.POINTER(CandParams),
                               C.POINTER(C.POINTER(CandList))], C.c_int32),
            "sr_cand_list_alloc": ([C.c_uint32, C.c_uint64, C.POINTER(C.POINTER(CandList))], C.c_int32),
            "sr_cand_list_free": ([C.POINTER(CandList)], None),
            "sr_session_attach_index": ([P, P, C.c_uint32], C.c_int32),
            "sr_candidates_device": ([P, C.POINTER(Reads), C.POINTER(CandParams),
                                      C.POINTER(C.POINTER(CandList))], C.c_int32),
            "sr_session_open": ([P, C.c_uint32, C.c_uint64, C.POINTER(P)], C.c_int32),
            "sr_session_open_seqs": ([P, P, C.c_uint32, C.c_uint64, C.POINTER(P)], C.c_int32),
            "sr_session_close": ([P], None),
            "sr_align_batch": ([P, C.POINTER(Reads), C.POINTER(CandList), C.POINTER(ScoreParams),
                                C.POINTER(AlignOpts), C.POINTER(C.POINTER(Results))], C.c_int32),
            "sr_batch_stage": ([P, C.POINTER(Reads), C.POINTER(CandList), P, C.POINTER(P)], C.c_int32),
            "sr_batch_run": ([P, P, C.POINTER(ScoreParams), C.POINTER(AlignOpts)], C.c_int32),
            "sr_batch_run_async": ([P, P, C.POINTER(ScoreParams), C.POINTER(AlignOpts)], C.c_int32),
            "sr_batch_sync": ([P, P], C.c_int32),
            "sr_batch_fetch": ([P, P, C.POINTER(C.POINTER(Results))], C.c_int32),
            "sr_batch_free": ([P], None),
            "sr_batch_stats": ([P, P, P, P, P], C.c_int32),
            "sr_batch_timing": ([P, P, P, P], C.c_int32),
            "sr_results_free": ([C.POINTER(Results)], None),
            "sr_classify": ([P, P, P], C.c_int32),
            "sr_batch_classify": ([P, P, P, P], C.c_int32),
            "sr_batch_report": ([P, P, C.c_uint32, C.c_uint32, C.POINTER(C.POINTER(Report))], C.c_int32),
            "sr_report_free": ([C.POINTER(Report)], None),
            "sr_write_sam": ([C.POINTER(Reads), C.POINTER(Results), P, C.POINTER(SamOpts), C.c_char_p], C.c_int32),
            "sr_serve_start": ([P, C.POINTER(ScoreParams), C.POINTER(AlignOpts), C.c_uint32], C.c_int32),
            "sr_submit": ([P, C.POINTER(Reads), C.POINTER(CandList), C.POINTER(C.c_uint64)], C.c_int32),
            "sr_wait": ([P, C.c_uint64, C.c_int32, C.POINTER(C.POINTER(Results))], C.c_int32),
            "sr_serve_stats": ([P, P, P, P, P, P], C.c_int32),
            "sr_serve_stats_by_size": ([P, C.c_uint32, P, P, P, P], C.c_int32),
            "sr_serve_overlap": ([P, P, P, P, P, C.c_uint32, P, P], C.c_int32),
            "sr_serve_latencies": ([P, C.c_uint64, C.c_uint32, P, P, P, P], C.c_int32),
            "sr_serve_stop": ([P], C.c_int32),
            "sr_tune": ([P, C.POINTER(ScoreParams), C.c_uint32], C.c_int32),
            "sr_tune_save": ([C.c_char_p], C.c_int32),
            "sr_tune_load": ([C.c_char_p], C.c_int32),
            "sr_tune_get": ([P, P, P, P, C.c_uint32], C.c_int32),
            "sr_tune_set": ([C.c_uint32, P, P, P], C.c_int32),
            "sr_probe_dpx": ([P, P], C.c_int32),
            "sr_probe_wait": ([C.c_uint32, C.c_uint32], C.c_int32),
            "sr_align_items_noalloc": ([P, P, P, C.c_uint32, P, P, P, P, P, C.c_uint64,
                                        C.POINTER(ScoreParams), P, P, P], C.c_int32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def _check(st):
    if st != SR_OK:
        raise SrError(st, lib().sr_last_error().decode(errors="replace"))


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def score_params(match=2, mismatch=3, gap_open=5, gap_extend=2):
    return ScoreParams(match, mismatch, gap_open, gap_extend)


def align_opts(mode=MODE_LOCAL, engine=ENGINE_BATCHED, want_cigar=True, classify=False, min_score=40,
               margin=5, force_i32=False, lanes=0, rows=0, stream=None):
    return AlignOpts(mode, engine, int(want_cigar), int(classify), min_score, margin, int(force_i32),
                     lanes, rows, 0, stream)


class _Keep:
    """Holds numpy arrays referenced by a C struct for the duration of a call."""

    def __init__(self):
        self.refs = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.refs.append(a)
        return a


def make_reads(bases, offsets, keep: _Keep):
    b = keep.arr(np.frombuffer(bases, np.uint8) if isinstance(bases, (bytes, bytearray)) else bases, np.uint8)
    o = keep.arr(offsets, np.uint64)
    return Reads(len(o) - 1, 0, C.c_void_p(b.ctypes.data), C.c_void_p(o.ctypes.data))


def make_cands(cand_off, c_ref, c_strand, c_start, c_len, keep: _Keep):
    off = keep.arr(cand_off, np.uint64)
    ref = keep.arr(c_ref, np.uint8)
    st = keep.arr(c_strand, np.uint8)
    ws = keep.arr(c_start, np.uint64)
    wl = keep.arr(c_len, np.uint32)
    cl = CandList()
    cl.n_reads = len(off) - 1
    cl.n_cands = int(off[-1]) if len(off) else 0
    cl.offsets, cl.ref_id, cl.strand = _p(off), _p(ref), _p(st)
    cl.win_start, cl.win_len, cl.hits = _p(ws), _p(wl), None
    return cl


def _dptr(t, dtype):
    """Device address of a contiguous CUDA tensor whose elements are `dtype`-sized."""
    assert t.is_cuda and t.is_contiguous(), "device inputs must be contiguous CUDA tensors"
    assert t.element_size() == np.dtype(dtype).itemsize, (t.dtype, dtype)
    return C.c_void_p(t.data_ptr())


def make_reads_device(bases, offsets):
    """sr_reads over CUDA tensors (uint8 bases, int64 / uint64 offsets), flagged as device memory."""
    return Reads(offsets.numel() - 1, FLAG_DEVICE, _dptr(bases, np.uint8), _dptr(offsets, np.uint64))


def make_cands_device(cand_off, c_ref, c_strand, c_start, c_len, n_cands):
    """sr_cand_list over CUDA tensors (offsets and starts 8-byte, ref ids and
    strands 1-byte, lengths 4-byte integers), flagged as device memory; n_cands
    is cand_off's last value (known to the caller, not read back here)."""
    cl = CandList()
    cl.n_reads = cand_off.numel() - 1
    cl.flags = FLAG_DEVICE
    cl.n_cands = int(n_cands)
    cl.offsets, cl.ref_id = _dptr(cand_off, np.uint64), _dptr(c_ref, np.uint8)
    cl.strand, cl.win_start = _dptr(c_strand, np.uint8), _dptr(c_start, np.uint64)
    cl.win_len, cl.hits = _dptr(c_len, np.uint32), None
    return cl


class _ResultsOwner:
    """Frees an sr_results when the last array viewing it is gone."""

    def __init__(self, rp):
        self.rp = rp

    def __del__(self):
        try:
            lib().sr_results_free(self.rp)
        except Exception:
            pass


def results_to_numpy(rp) -> dict:
    """Arrays viewing the library's result buffers (no copy); the buffers are
    released with sr_results_free once no array refers to them."""
    r = rp.contents
    n, nr, ni = r.n_reads, r.n_refs, r.n_items
    owner = _ResultsOwner(rp)

    def arr(ptr, count, dtype):
        if count == 0 or not ptr:
            return np.zeros(0, dtype)
        buf = (C.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr if isinstance(ptr, int) else C.cast(ptr, C.c_void_p).value)
        buf._owner = owner
        return np.frombuffer(buf, dtype)

    out = dict(
        best=arr(C.cast(r.best, C.c_void_p).value, n, HIT_DTYPE),
        best_per_ref=arr(C.cast(r.best_per_ref, C.c_void_p).value, n * nr, HIT_DTYPE).reshape(n, nr),
        item_score=arr(r.item_score, ni, np.int32),
        item_end=arr(r.item_end, ni, np.uint32),
        cigar=arr(r.cigar, r.n_cigar, np.uint32),
        read_class=arr(r.read_class, n, np.uint8) if r.read_class else None,
        cells=int(r.cells), n_i32_items=int(r.n_i32_items),
        n_reads=n, n_refs=nr, n_items=ni,
    )
    return out


def write_sam(path, bases, read_off, res: dict, ref_lens, read_names=None, ref_names=None, report=None):
    """SAM text of aligned reads (sr_write_sam); `res` is an align/fetch result
    dict, `report` an optional Batch.report() dict for XA secondary hits."""
    keep = _Keep()
    reads = make_reads(bases, read_off, keep)
    best = keep.arr(res["best"], HIT_DTYPE)
    n = len(best)
    per = keep.arr(res["best_per_ref"], HIT_DTYPE)
    cig = keep.arr(res["cigar"], np.uint32)
    cls = keep.arr(res["read_class"], np.uint8) if res.get("read_class") is not None else None
    r = Results()
    r.n_reads, r.n_refs, r.n_items = n, len(ref_lens), 0
    r.best = C.cast(best.ctypes.data, C.POINTER(Hit))
    r.best_per_ref = C.cast(per.ctypes.data, C.POINTER(Hit))
    r.cigar, r.n_cigar = (cig.ctypes.data if len(cig) else None), len(cig)
    r.read_class = cls.ctypes.data if cls is not None else None
    lens = keep.arr(np.asarray(ref_lens), np.uint64)
    o = SamOpts()

    def names(lst):
        if lst is None:
            return None
        enc = [x.encode() for x in lst]
        arr = (C.c_char_p * len(enc))(*enc)
        keep.refs.append((enc, arr))
        return C.cast(arr, P)

    o.read_names, o.ref_names = names(read_names), names(ref_names)
    if report is not None:
        offs = keep.arr(report["offsets"], np.uint64)
        hits = keep.arr(report["hits"], REPORT_HIT_DTYPE)
        rp = Report(n, 0, len(hits), offs.ctypes.data, hits.ctypes.data if len(hits) else None)
        keep.refs.append(rp)
        o.secondary = C.pointer(rp)
    _check(lib().sr_write_sam(C.byref(reads), C.byref(r), _p(lens), C.byref(o), os.fsencode(path)))


def classify(res: dict, min_score=40, margin=5, out=None):
    """sr_classify on a results dict (align / fetch / wait): the class of every
    read between references 0 and 1, computed on the device.  res["best_per_ref"]
    may be the numpy records or a CUDA tensor holding them (n_reads x n_refs
    records of HIT_DTYPE bytes); `out` may be a CUDA uint8 tensor (filled in
    place, returned) or None (a numpy array is returned)."""
    per = res["best_per_ref"]
    keep = _Keep()
    r = Results()
    if hasattr(per, "data_ptr"):  # device records
        n, nr = int(res["n_reads"]), int(res["n_refs"])
        assert per.is_cuda and per.numel() * per.element_size() >= n * nr * HIT_DTYPE.itemsize
        r.best_per_ref = C.cast(per.data_ptr(), C.POINTER(Hit))
    else:
        per = keep.arr(per, HIT_DTYPE)
        n, nr = per.shape[0], (per.shape[1] if per.ndim == 2 else int(res["n_refs"]))
        r.best_per_ref = C.cast(per.ctypes.data, C.POINTER(Hit))
    r.n_reads, r.n_refs = n, nr
    prm = np.array([min_score, margin], np.int32)
    if out is None:
        o = np.zeros(max(n, 1), np.uint8)
        _check(lib().sr_classify(C.byref(r), _p(prm), _p(o)))
        return o[:n]
    _check(lib().sr_classify(C.byref(r), _p(prm), C.c_void_p(out.data_ptr())))
    return out


def cigar_of(res: dict, read: int):
    h = res["best"][read]
    w = res["cigar"][int(h["cigar_off"]): int(h["cigar_off"]) + int(h["cigar_len"])]
    return [(int(x) >> 4, int(x) & 15) for x in w]


class Index:
    def __init__(self, handle):
        self.h = handle

    @classmethod
    def build(cls, seq, seed_len=20, address_bases=12, cal_limit=0, threads=0, hash_seed=0):
        b = bytes(seq) if not isinstance(seq, bytes) else seq
        h = P()
        p = IndexParams(seed_len, address_bases, cal_limit, threads, hash_seed)
        _check(lib().sr_index_build(b, len(b), C.byref(p), C.byref(h)))
        return cls(h)

    @classmethod
    def load(cls, path):
        h = P()
        _check(lib().sr_index_load(os.fsencode(path), C.byref(h)))
        return cls(h)

    def save(self, path):
        _check(lib().sr_index_save(self.h, os.fsencode(path)))

    def info(self):
        a, b = C.c_uint64(), C.c_uint64()
        _check(lib().sr_index_info(self.h, C.byref(a), C.byref(b)))
        return dict(ref_len=a.value, n_entries=b.value)

    def close(self):
        if self.h:
            lib().sr_index_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def candidates(indexes, bases, read_off, seed_stride=1, merge_dist=32, pad=32, max_cands=0, threads=0):
    keep = _Keep()
    reads = make_reads(bases, read_off, keep)
    arr = (P * len(indexes))(*[ix.h for ix in indexes])
    cp = CandParams(seed_stride, merge_dist, pad, max_cands, threads, 0)
    out = C.POINTER(CandList)()
    _check(lib().sr_candidates(C.cast(arr, P), len(indexes), C.byref(reads), C.byref(cp), C.byref(out)))
    return _cand_list_to_numpy(out)


class _CandListOwner:
    """Frees a host sr_cand_list once no array viewing it is left."""

    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        if self.ptr is not None and _lib is not None:
            _lib.sr_cand_list_free(self.ptr)
        self.ptr = None


def _cand_list_to_numpy(out):
    """The list's arrays as numpy views of the library's own buffers (the list is
    freed with the last of them); cand_off and c_start read as int64, c_len as
    int32 (same bits: offsets, starts and lengths stay below 2^31 / 2^63)."""
    l = out.contents
    n, nc = l.n_reads, l.n_cands
    owner = _CandListOwner(out)

    def a(ptr, count, dt):
        if count == 0 or not ptr:
            return np.zeros(count, dt)
        buf = (C.c_char * (count * np.dtype(dt).itemsize)).from_address(ptr)
        buf._owner = owner
        return np.frombuffer(buf, dt)

    return dict(cand_off=a(l.offsets, n + 1, np.int64), c_ref=a(l.ref_id, nc, np.uint8),
                c_strand=a(l.strand, nc, np.uint8), c_start=a(l.win_start, nc, np.int64),
                c_len=a(l.win_len, nc, np.int32), c_hits=a(l.hits, nc, np.uint32))


class _CudaArray:
    """A device array of the library seen through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, n, typestr, owner):
        self.owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2}


class DeviceCandList:
    """An sr_cand_list whose arrays sit in device memory (sr_candidates_device with
    SR_FLAG_DEVICE); freed with sr_cand_list_free when this object goes away."""

    def __init__(self, ptr):
        self.ptr = ptr
        l = ptr.contents
        self.n_reads, self.n_cands = int(l.n_reads), int(l.n_cands)
        assert l.flags & FLAG_DEVICE

    def tensors(self):
        """The arrays as CUDA tensors sharing the list's memory (kept alive by them)."""
        import torch
        l = self.ptr.contents
        n, nc = self.n_reads, self.n_cands
        v = lambda p, k, t: torch.as_tensor(_CudaArray(C.cast(p, C.c_void_p).value, k, t, self), device="cuda")
        return dict(cand_off=v(l.offsets, n + 1, "<u8"), c_ref=v(l.ref_id, nc, "|u1"), c_strand=v(l.strand, nc, "|u1"),
                    c_start=v(l.win_start, nc, "<u8"), c_len=v(l.win_len, nc, "<u4"), c_hits=v(l.hits, nc, "<u4"))

    def to_numpy(self):
        """A host copy in the layout candidates() returns."""
        t = self.tensors()
        out = {k: x.cpu().numpy() for k, x in t.items()}
        out["cand_off"] = out["cand_off"].astype(np.int64)
        out["c_start"] = out["c_start"].astype(np.int64)
        out["c_len"] = out["c_len"].astype(np.int32)
        return out

    def __del__(self):
        try:
            if self.ptr:
                lib().sr_cand_list_free(self.ptr)
                self.ptr = None
        except Exception:
            pass


class Batch:
    def __init__(self, session, handle, keep):
        self.session, self.h, self._keep = session, handle, keep

    def run(self, sp=None, opts=None):
        _check(lib().sr_batch_run(self.session.h, self.h, C.byref(sp or score_params()),
                                  C.byref(opts or align_opts())))

    def run_async(self, sp=None, opts=None):
        _check(lib().sr_batch_run_async(self.session.h, self.h, C.byref(sp or score_params()),
                                        C.byref(opts or align_opts())))

    def sync(self):
        _check(lib().sr_batch_sync(self.session.h, self.h))

    def fetch(self):
        out = C.POINTER(Results)()
        _check(lib().sr_batch_fetch(self.session.h, self.h, C.byref(out)))
        return results_to_numpy(out)

    def classify(self, min_score=40, margin=5):
        n = self.n_reads
        out = np.zeros(max(n, 1), np.uint8)
        prm = np.array([min_score, margin], np.int32)
        _check(lib().sr_batch_classify(self.session.h, self.h, _p(prm), _p(out)))
        return out[:n]

    def report(self, kind=REPORT_BEST_N, n_best=1):
        """Sec. 4.2 tracker options on the device: per read, the n_best highest-scoring
        windows (REPORT_BEST_N) or all windows tied for the best (REPORT_TIED).
        Returns dict(offsets (n_reads + 1), hits (REPORT_HIT_DTYPE), n_truncated)."""
        out = C.POINTER(Report)()
        _check(lib().sr_batch_report(self.session.h, self.h, kind, n_best, C.byref(out)))
        try:
            r = out.contents
            n, nh = r.n_reads, r.n_hits
            offs = np.frombuffer((C.c_char * (8 * (n + 1))).from_address(r.offsets), np.uint64).copy()
            hits = (np.frombuffer((C.c_char * (REPORT_HIT_DTYPE.itemsize * nh)).from_address(r.hits),
                                  REPORT_HIT_DTYPE).copy() if nh else np.zeros(0, REPORT_HIT_DTYPE))
            return dict(offsets=offs, hits=hits, n_truncated=int(r.n_truncated))
        finally:
            lib().sr_report_free(out)

    def stats(self):
        k, c, i, t = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().sr_batch_stats(self.h, C.byref(k), C.byref(c), C.byref(i), C.byref(t)))
        return dict(kernels=k.value, cells=c.value, i32_items=i.value, tasks=t.value)

    def timing(self):
        """(total, extension, traceback) device milliseconds of the last run."""
        a, b, c = C.c_float(), C.c_float(), C.c_float()
        _check(lib().sr_batch_timing(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def close(self):
        if self.h:
            lib().sr_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Session:
    def __init__(self, handle):
        self.h = handle

    @classmethod
    def open(cls, refs, hbm_budget=0):
        """refs: list of ASCII sequences (bytes or uint8 arrays)."""
        keep = _Keep()
        arrs = [keep.arr(np.frombuffer(r, np.uint8) if isinstance(r, (bytes, bytearray)) else r, np.uint8) for r in refs]
        ptrs = (P * len(arrs))(*[a.ctypes.data for a in arrs])
        lens = keep.arr(np.array([len(a) for a in arrs], np.uint64), np.uint64)
        h = P()
        _check(lib().sr_session_open_seqs(C.cast(ptrs, P), _p(lens), len(arrs), hbm_budget, C.byref(h)))
        return cls(h)

    @classmethod
    def from_indexes(cls, indexes, hbm_budget=0):
        arr = (P * len(indexes))(*[ix.h for ix in indexes])
        h = P()
        _check(lib().sr_session_open(C.cast(arr, P), len(indexes), hbm_budget, C.byref(h)))
        return cls(h)

    def stage(self, bases, read_off, cand_off, c_ref, c_strand, c_start, c_len, stream=None):
        keep = _Keep()
        reads = make_reads(bases, read_off, keep)
        cands = make_cands(cand_off, c_ref, c_strand, c_start, c_len, keep)
        h = P()
        _check(lib().sr_batch_stage(self.h, C.byref(reads), C.byref(cands), stream, C.byref(h)))
        b = Batch(self, h, None)
        b.n_reads = reads.n_reads
        return b

    def align(self, bases, read_off, cand_off, c_ref, c_strand, c_start, c_len, sp=None, opts=None):
        keep = _Keep()
        reads = make_reads(bases, read_off, keep)
        cands = make_cands(cand_off, c_ref, c_strand, c_start, c_len, keep)
        out = C.POINTER(Results)()
        _check(lib().sr_align_batch(self.h, C.byref(reads), C.byref(cands), C.byref(sp or score_params()),
                                    C.byref(opts or align_opts()), C.byref(out)))
        return results_to_numpy(out)

    def align_device(self, bases, read_off, cand_off, c_ref, c_strand, c_start, c_len, n_cands, sp=None,
                     opts=None):
        """sr_align_batch on inputs that already sit in device memory (CUDA
        tensors; see make_reads_device / make_cands_device); results come back
        to host arrays as with align()."""
        reads = make_reads_device(bases, read_off)
        cands = make_cands_device(cand_off, c_ref, c_strand, c_start, c_len, n_cands)
        out = C.POINTER(Results)()
        _check(lib().sr_align_batch(self.h, C.byref(reads), C.byref(cands), C.byref(sp or score_params()),
                                    C.byref(opts or align_opts()), C.byref(out)))
        return results_to_numpy(out)

    def align_cands(self, bases, read_off, cands, sp=None, opts=None):
        """sr_align_batch with the windows of a DeviceCandList (left on the device by
        candidates(..., out_device=True)); the reads are numpy arrays or CUDA tensors."""
        keep = _Keep()
        reads = make_reads_device(bases, read_off) if hasattr(bases, "data_ptr") else make_reads(bases, read_off, keep)
        out = C.POINTER(Results)()
        _check(lib().sr_align_batch(self.h, C.byref(reads), cands.ptr, C.byref(sp or score_params()),
                                    C.byref(opts or align_opts()), C.byref(out)))
        return results_to_numpy(out)

    # device CAL finder (Sec. 3.2-3.3 on the GPU)
    def attach_index(self, indexes):
        arr = (P * len(indexes))(*[ix.h for ix in indexes])
        _check(lib().sr_session_attach_index(self.h, C.cast(arr, P), len(indexes)))

    def candidates(self, bases, read_off, seed_stride=1, merge_dist=32, pad=32, max_cands=0, out_device=False):
        """Device CAL finder.  bases / read_off: numpy arrays, or CUDA tensors (uint8,
        int64) already on the device.  Returns numpy arrays, or with out_device a
        DeviceCandList whose arrays stay in device memory."""
        keep = _Keep()
        reads = make_reads_device(bases, read_off) if hasattr(bases, "data_ptr") else make_reads(bases, read_off, keep)
        cp = CandParams(seed_stride, merge_dist, pad, max_cands, 0, FLAG_DEVICE if out_device else 0)
        out = C.POINTER(CandList)()
        _check(lib().sr_candidates_device(self.h, C.byref(reads), C.byref(cp), C.byref(out)))
        return DeviceCandList(out) if out_device else _cand_list_to_numpy(out)

    # serving
    def serve_start(self, sp=None, opts=None, max_inflight=0):
        _check(lib().sr_serve_start(self.h, C.byref(sp or score_params()), C.byref(opts or align_opts()),
                                    max_inflight))

    def submit(self, bases, read_off, cand_off, c_ref, c_strand, c_start, c_len):
        keep = _Keep()
        reads = make_reads(bases, read_off, keep)
        cands = make_cands(cand_off, c_ref, c_strand, c_start, c_len, keep)
        t = C.c_uint64()
        _check(lib().sr_submit(self.h, C.byref(reads), C.byref(cands), C.byref(t)))
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        out = C.POINTER(Results)()
        _check(lib().sr_wait(self.h, ticket, timeout_ms, C.byref(out)))
        return results_to_numpy(out)

    def serve_stats(self):
        p50, p99 = C.c_double(), C.c_double()
        n, rounds, mx = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().sr_serve_stats(self.h, C.byref(p50), C.byref(p99), C.byref(n), C.byref(rounds),
                                    C.byref(mx)))
        return dict(p50_us=p50.value, p99_us=p99.value, completed=n.value, rounds=rounds.value,
                    max_round_requests=mx.value)

    def serve_stats_by_size(self, max_reads=(256, 1024, 2048, 4096)):
        """p50/p99 latency (us) and count per request-size bucket: bucket k holds
        requests of max_reads[k-1] + 1 .. max_reads[k] reads."""
        b = np.ascontiguousarray(max_reads, np.uint32)
        p50, p99 = np.zeros(len(b)), np.zeros(len(b))
        cnt = np.zeros(len(b), np.uint64)
        _check(lib().sr_serve_stats_by_size(self.h, len(b), _p(b), _p(p50), _p(p99), _p(cnt)))
        return [dict(max_reads=int(b[k]), count=int(cnt[k]), p50_us=float(p50[k]), p99_us=float(p99[k]))
                for k in range(len(b))]

    def serve_latencies(self):
        """Every completed request in completion order: latency (us), reads and
        completion time (s after serve_start)."""
        n = C.c_uint64()
        _check(lib().sr_serve_latencies(self.h, 0, 0, None, None, None, C.byref(n)))
        k = n.value
        us, rd, t = np.zeros(max(k, 1)), np.zeros(max(k, 1), np.uint32), np.zeros(max(k, 1))
        _check(lib().sr_serve_latencies(self.h, 0, k, _p(us), _p(rd), _p(t), C.byref(n)))
        return dict(us=us[:k], reads=rd[:k], done_s=t[:k])

    def serve_overlap(self, cap=0):
        """Device timeline of completed rounds (first kernel done, last kernel
        done; ms after serve_start), rounds that overlapped the previous one,
        idle time between the others and the admissions the budget deferred."""
        n, ov, bw = C.c_uint64(), C.c_uint64(), C.c_uint64()
        idle = C.c_double()
        first, last = np.zeros(max(cap, 1), np.float32), np.zeros(max(cap, 1), np.float32)
        _check(lib().sr_serve_overlap(self.h, C.byref(n), C.byref(ov), C.byref(idle), C.byref(bw), cap,
                                      _p(first) if cap else None, _p(last) if cap else None))
        k = min(cap, n.value)
        return dict(timed_rounds=n.value, overlapped=ov.value, device_idle_ms=idle.value, budget_waits=bw.value,
                    first_ms=first[:k], last_ms=last[:k])

    def serve_stop(self):
        _check(lib().sr_serve_stop(self.h))

    def close(self):
        if self.h:
            lib().sr_session_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_get():
    n = C.c_uint32()
    up, la, ro = (np.zeros(64, np.uint32) for _ in range(3))
    _check(lib().sr_tune_get(C.byref(n), _p(up), _p(la), _p(ro), 64))
    k = min(n.value, 64)
    return [(int(up[i]), int(la[i]), int(ro[i])) for i in range(k)]


def tune_set(bins):
    up = np.array([b[0] for b in bins], np.uint32)
    la = np.array([b[1] for b in bins], np.uint32)
    ro = np.array([b[2] for b in bins], np.uint32)
    _check(lib().sr_tune_set(len(bins), _p(up), _p(la), _p(ro)))


def probe_dpx():
    r, mhz = C.c_double(), C.c_double()
    _check(lib().sr_probe_dpx(C.byref(r), C.byref(mhz)))
    return r.value, mhz.value


def probe_wait(poll_limit=1000, arrive=False):
    """Run the bounded device wait on a barrier that does (or never does) complete."""
    _check(lib().sr_probe_wait(poll_limit, 1 if arrive else 0))
