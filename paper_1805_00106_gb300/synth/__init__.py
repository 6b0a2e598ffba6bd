"""Seeded synthetic workloads shaped like the paper's (arXiv 1805.00106, Sec. 6.2,
Fig. 9): references, reads with sequencing errors and candidate windows.

Data generation only -- no alignment arithmetic lives here.  Both the oracle
(tests, CPU baseline) and the CUDA path consume these inputs.  The C core
(``synth.c``) is compiled with gcc on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

COUNT_FIXED, COUNT_POISSON, COUNT_UNIFORM, COUNT_PARETO = 0, 1, 2, 3


def build(force: bool = False) -> str:
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC,
                                   "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P, I64, I, D, U64 = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_uint64
        L.syn_ref_iid.argtypes = [U64, I64, D, P]
        L.syn_mutate.argtypes = [U64, P, I64, D, D, I, I64, I64, P, I64]
        L.syn_mutate.restype = I64
        L.syn_ref_repeats.argtypes = [U64, I64, D, I, P, P]
        L.syn_reads.argtypes = [U64, I, P, P, P, I, I, I, D, D, D, P, P, P, P, P, P]
        L.syn_cands.argtypes = [U64, I, P, P, P, P, P, I, P, I, D, D, I, I, P, P, P, P, P, P, I64]
        L.syn_cands.restype = I64
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def ref_iid(n: int, seed: int, gc: float = 0.5) -> np.ndarray:
    out = np.empty(n, np.uint8)
    _L().syn_ref_iid(seed, n, gc, _p(out))
    return out


def mutate(src: np.ndarray, seed: int, sub: float, indel: float, nblocks: int = 0,
           blk_lo: int = 10_000, blk_hi: int = 1_000_000) -> np.ndarray:
    src = np.ascontiguousarray(src, np.uint8)
    cap = int(len(src) * (1 + 2 * indel) + 1024)
    out = np.empty(cap, np.uint8)
    n = _L().syn_mutate(seed, _p(src), len(src), sub, indel, nblocks, blk_lo, blk_hi, _p(out), cap)
    return out[:n].copy()


def ref_repeats(n: int, seed: int, rep_frac: float = 0.3, n_families: int = 500):
    out = np.empty(n, np.uint8)
    mask = np.empty(n, np.uint8)
    _L().syn_ref_repeats(seed, n, rep_frac, n_families, _p(out), _p(mask))
    return out, mask


def reads(refs, n_reads: int, seed: int, len_lo: int, len_hi: int, sub: float = 0.01,
          indel: float = 0.001, rc_frac: float = 0.0, weights=None):
    refs = [np.ascontiguousarray(r, np.uint8) for r in refs]
    ptrs = (C.c_void_p * len(refs))(*[r.ctypes.data for r in refs])
    lens = np.array([len(r) for r in refs], np.int64)
    w = np.array(weights if weights is not None else [1.0] * len(refs), np.float64)
    bases = np.empty(n_reads * len_hi, np.uint8)
    off = np.empty(n_reads + 1, np.int64)
    t_ref = np.empty(n_reads, np.int32)
    t_pos = np.empty(n_reads, np.int64)
    t_strand = np.empty(n_reads, np.uint8)
    t_span = np.empty(n_reads, np.int32)
    _L().syn_reads(seed, len(refs), C.cast(ptrs, C.c_void_p), _p(lens), _p(w), n_reads, len_lo,
                   len_hi, sub, indel, rc_frac, _p(bases), _p(off), _p(t_ref), _p(t_pos),
                   _p(t_strand), _p(t_span))
    return dict(bases=bases[: off[-1]].copy(), read_off=off, t_ref=t_ref, t_pos=t_pos,
                t_strand=t_strand, t_span=t_span)


def cands(rd: dict, ref_lens, seed: int, count_kind: int, p1: float, pad: int,
          cap_per_read: int = 64, p2: float = 0.0, rep_mask=None):
    n_reads = len(rd["read_off"]) - 1
    lens = np.array(ref_lens, np.int64)
    if count_kind == COUNT_FIXED:
        cap = n_reads * int(p1)
    else:
        cap = n_reads * cap_per_read
    cap = max(int(cap), 1)
    cand_off = np.empty(n_reads + 1, np.int64)
    c_ref = np.empty(cap, np.uint8)
    c_strand = np.empty(cap, np.uint8)
    c_start = np.empty(cap, np.int64)
    c_len = np.empty(cap, np.int32)
    n = _L().syn_cands(seed, n_reads, _p(rd["read_off"]), _p(rd["t_ref"]), _p(rd["t_pos"]),
                       _p(rd["t_strand"]), _p(rd["t_span"]), len(lens), _p(lens), count_kind, p1,
                       p2, cap_per_read, pad, _p(rep_mask), _p(cand_off), _p(c_ref), _p(c_strand),
                       _p(c_start), _p(c_len), cap)
    if n < 0:
        raise RuntimeError("candidate capacity")
    return dict(cand_off=cand_off, c_ref=c_ref[:n].copy(), c_strand=c_strand[:n].copy(),
                c_start=c_start[:n].copy(), c_len=c_len[:n].copy())


# ------------------------------------------------------------------ workloads

def workload(name: str, scale: float = 1.0, seed: int = 0, rc_frac: float = 0.0) -> dict:
    """Synthetic stand-ins for the paper's data (Sec. 6.2 reads are absent).

    c1  plain small     1 Mbp uniform reference, 10k x 100 bp reads, 4 windows of
                        100 + 2*16 bp (true locus + 3 decoys)
    c2  batched uneven  100 Mbp at 41% GC, 1M reads of 75-250 bp, Poisson(6)
                        windows capped at 64, each read_len + 2*32 bp
    c3  xenograft       64 Mbp A, B = A with 15% substitutions, 2% indels, 50
                        block moves; 2M x 100 bp reads (70% A / 30% B), 1% errors;
                        candidates come from the host index, not from here
    c5  repeat heavy    200 Mbp with 30% repeats; 250 bp reads; Pareto(1.1)
                        candidate counts capped at 256, decoys mostly in repeats

    ``scale`` shrinks reference length and read count for tests.
    """
    def sz(n, lo=1):
        return max(lo, int(round(n * scale)))

    if name == "c1":
        ref = ref_iid(sz(1_000_000, 5000), seed)
        rd = reads([ref], sz(10_000, 4), seed + 1, 100, 100, 0.01, 0.001, rc_frac)
        cd = cands(rd, [len(ref)], seed + 2, COUNT_FIXED, 4, 16)
        return dict(name="c1", refs=[ref], **rd, **cd)
    if name == "c2":
        ref = ref_iid(sz(100_000_000, 20000), seed, gc=0.41)
        rd = reads([ref], sz(1_000_000, 4), seed + 1, 75, 250, 0.01, 0.001, rc_frac)
        cd = cands(rd, [len(ref)], seed + 2, COUNT_POISSON, 6.0, 32, cap_per_read=64)
        return dict(name="c2", refs=[ref], **rd, **cd)
    if name == "c3":
        a = ref_iid(sz(64_000_000, 20000), seed)
        n_blocks = 50 if scale >= 0.5 else max(1, int(50 * scale))
        blk_hi = min(1_000_000, max(100, len(a) // 20))
        blk_lo = min(10_000, blk_hi // 2)
        b = mutate(a, seed + 3, 0.15, 0.02, n_blocks, blk_lo, blk_hi)
        rd = reads([a, b], sz(2_000_000, 4), seed + 1, 100, 100, 0.009, 0.001, rc_frac,
                   weights=[0.7, 0.3])
        return dict(name="c3", refs=[a, b], **rd)
    if name == "c5":
        ref, mask = ref_repeats(sz(200_000_000, 50000), seed)
        rd = reads([ref], sz(100_000, 4), seed + 1, 250, 250, 0.009, 0.001, rc_frac)
        cd = cands(rd, [len(ref)], seed + 2, COUNT_PARETO, 1.1, 32, cap_per_read=256, p2=0.8,
                   rep_mask=mask)
        return dict(name="c5", refs=[ref], rep_mask=mask, **rd, **cd)
    raise ValueError(name)


def serving_batches(refs, n_batches: int, seed: int, max_batch: int = 4096):
    """c4 serving stream: batches of uniform [1, max_batch] reads (75-250 bp,
    1% errors) against a reference pair, with uniform [0, 64] windows each."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_batches):
        n = int(rng.integers(1, max_batch + 1))
        rd = reads(refs, n, seed * 1000 + 2 * b + 1, 75, 250, 0.009, 0.001, 0.0)
        cd = cands(rd, [len(r) for r in refs], seed * 1000 + 2 * b + 2, COUNT_UNIFORM, 64, 32,
                   cap_per_read=64)
        out.append(dict(**rd, **cd))
    return out


def splicing(scale: float = 1.0, seed: int = 0, read_len: int = 100) -> dict:
    """Alternative-splicing stand-in (the paper adds exon-junction sequences of
    Ensembl transcripts to the reference, Sec. 6.2 / Table 4): a 20 Mbp genome
    (41% GC) with genes of 4-10 exons (60-250 bp, introns 300-3000 bp); the
    junction library joins the last read_len-1 bases of exon i to the first
    read_len-1 bases of every later exon j of the same gene (exon skipping
    included), entries separated by 100 random bases.  Reads (1% errors) come
    from one random isoform per gene (inner exons kept with p = 0.7); `spans`
    marks reads crossing an exon junction of their isoform."""
    rng = np.random.default_rng(seed)
    genome = ref_iid(max(50_000, int(round(20_000_000 * scale))), seed, gc=0.41)
    n_genes = max(4, int(round(4000 * scale)))
    flank = read_len - 1
    junctions, transcripts, bounds = [], [], []
    pos = 1000
    for g in range(n_genes):
        n_ex = int(rng.integers(4, 11))
        exons = []
        p = pos
        for _ in range(n_ex):
            ln = int(rng.integers(60, 251))
            if p + ln + 1000 >= len(genome):
                break
            exons.append((p, p + ln))
            p += ln + int(rng.integers(300, 3001))
        if len(exons) < 2:
            break
        pos = p + int(rng.integers(1000, 5000))
        seqs = [genome[a:b] for a, b in exons]
        for i in range(len(seqs)):
            for j in range(i + 1, len(seqs)):
                junctions.append(np.concatenate([seqs[i][-flank:], seqs[j][:flank]]))
                junctions.append(rng.choice(np.frombuffer(b"ACGT", np.uint8), 100))
        keep = [0] + [k for k in range(1, len(seqs) - 1) if rng.random() < 0.7] + [len(seqs) - 1]
        transcripts.append(np.concatenate([seqs[k] for k in keep]))
        cut = np.cumsum([len(seqs[k]) for k in keep])[:-1]
        bounds.append(cut)
    junc = np.concatenate(junctions) if junctions else rng.choice(np.frombuffer(b"ACGT", np.uint8), 1000)
    lens = np.array([len(t) for t in transcripts], np.float64)
    rd = reads(transcripts, max(4, int(round(200_000 * scale))), seed + 1, read_len, read_len, 0.009, 0.001,
               0.0, weights=lens / lens.sum())
    spans = np.array([bool(np.any((bounds[t] > p) & (bounds[t] < p + s)))
                      for t, p, s in zip(rd["t_ref"], rd["t_pos"], rd["t_span"])])
    return dict(name="splicing", genome=genome, junctions=junc, spans=spans, n_genes=len(transcripts), **rd)
