"""Pins for the oracle against facts fixed by the paper and by the mathematics,
not by the oracle itself (CPU only).

* brute force: every local alignment of tiny strings enumerated explicitly and
  scored with the affine gap model (Sec. 3.5) -- best score, end-cell tie-break
  and the traceback's choice among co-optimal alignments;
* closed forms: identical strings, one substitution, one gap of k bases;
* invariants: score >= 0, swap symmetry, CIGAR re-scores to the score, CIGAR
  lengths, monotone in the window;
* special case: gap_open = 0 reduces to the textbook linear-gap Smith-Waterman
  (written here, independently);
* the paper's worked examples: Fig. 3 2-bit encoding, Sec. 3.1 reverse
  complement, Sec. 3.2 seed counts, Sec. 3.1 pigeonhole guarantee;
* score tracker and classification boundaries (Sec. 3.6, 4.2, 6.4).
"""
import itertools
import os
import random

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BASES = "ACGT"


def rand_seq(rng, n):
    return "".join(rng.choice(BASES) for _ in range(n))


# ---------------------------------------------------------------- brute force

def enumerate_alignments(q, r, sa, sb, go, ge):
    """Every alignment of a substring of q with a substring of r, as
    (score, start_i, start_j, end_i, end_j, ops); ops over 'M','I','D';
    a run of k gap columns costs go + k*ge."""
    m, n = len(q), len(r)
    out = []

    def rec(i, j, ops, score, last, si, sj):
        if ops:
            out.append((score, si, sj, i, j, tuple(ops)))
        if i < m and j < n:
            ops.append("M")
            rec(i + 1, j + 1, ops, score + (sa if q[i] == r[j] else -sb), "M", si, sj)
            ops.pop()
        if i < m:
            ops.append("I")
            rec(i + 1, j, ops, score - (ge if last == "I" else go + ge), "I", si, sj)
            ops.pop()
        if j < n:
            ops.append("D")
            rec(i, j + 1, ops, score - (ge if last == "D" else go + ge), "D", si, sj)
            ops.pop()

    for i0 in range(m):
        for j0 in range(n):
            rec(i0, j0, [], 0, None, i0 + 1, j0 + 1)
    return out


def backward_rank(ops):
    """Declarative form of the traceback priorities, read from the end cell
    backwards: in the match state stop < M < D < I; right after a D, closing
    the gap (M, then I) is preferred to extending it (D); right after an I,
    closing (M, then D) is preferred to extending (I)."""
    ranks = []
    state = "H"
    table = {"H": {"M": 1, "D": 2, "I": 3}, "E": {"M": 1, "I": 3, "D": 4},
             "F": {"M": 1, "D": 2, "I": 4}}
    for op in reversed(ops):
        ranks.append(table[state][op])
        state = {"M": "H", "D": "E", "I": "F"}[op]
    ranks.append(0)
    return ranks


def cigar_ops(cig):
    ops = []
    for ln, op in cig:
        if op == O.OP_S:
            continue
        ops += [{O.OP_M: "M", O.OP_I: "I", O.OP_D: "D"}[op]] * ln
    return tuple(ops)


PARAMS = [(2, 3, 5, 2), (1, 1, 1, 1), (3, 1, 2, 1), (2, 3, 1, 3), (5, 4, 3, 1)]


def _brute_cases():
    rng = random.Random(1805)
    cases = []
    for t in range(110):
        m, n = rng.randint(1, 5), rng.randint(1, 5)
        alphabet = "AC" if t % 3 == 0 else BASES  # low entropy -> many ties
        q = "".join(rng.choice(alphabet) for _ in range(m))
        r = "".join(rng.choice(alphabet) for _ in range(n))
        cases.append((q, r, PARAMS[t % len(PARAMS)]))
    cases += [("ACGTA", "ACGTA", (2, 3, 5, 2)), ("AAAAA", "AAAA", (2, 3, 5, 2)),
              ("ACAC", "CACA", (1, 1, 1, 1)), ("A", "C", (2, 3, 5, 2)), ("GATTA", "GATA", (2, 1, 1, 1))]
    return cases


@pytest.mark.parametrize("q,r,params", _brute_cases())
def test_brute_force_score_end_and_traceback(q, r, params):
    sa, sb, go, ge = params
    res = O.align(q, r, O.score_params(*params))
    alns = enumerate_alignments(q, r, sa, sb, go, ge)
    S = max([0] + [a[0] for a in alns])
    assert res["score"] == S
    if S == 0:
        assert (res["end_i"], res["end_j"]) == (0, 0)
        assert res["cigar"] == []
        return
    # end cell: smallest window column, then smallest read row, among optimal alignments
    ends = sorted({(a[4], a[3]) for a in alns if a[0] == S})
    ej, ei = ends[0]
    assert (res["end_i"], res["end_j"]) == (ei, ej)
    if go == 0:
        return  # with free gap opening adjacent gap runs tie; rule pinned for go > 0 only
    cands = [a for a in alns if a[0] == S and a[3] == ei and a[4] == ej]
    chosen = min(cands, key=lambda a: backward_rank(a[5]))
    assert (res["start_i"], res["start_j"]) == (chosen[1], chosen[2])
    assert cigar_ops(res["cigar"]) == chosen[5]


# --------------------------------------------------------------- closed forms

def test_identical_strings_score_len_times_match():
    rng = random.Random(7)
    for n in [1, 2, 17, 100, 250]:
        s = rand_seq(rng, n)
        res = O.align(s, s)
        assert res["score"] == 2 * n
        assert (res["end_i"], res["end_j"]) == (n, n)
        assert res["cigar"] == [(n, O.OP_M)]


def test_single_substitution():
    rng = random.Random(11)
    for _ in range(40):
        n = rng.randint(20, 120)
        s = rand_seq(rng, n)
        p = rng.randint(1, n)  # 1-based substituted position
        t = list(s)
        t[p - 1] = rng.choice([b for b in BASES if b != s[p - 1]])
        t = "".join(t)
        expect = max((n - 1) * 2 - 3, max(p - 1, n - p) * 2)
        assert O.align(s, t)["score"] == expect


def test_single_gap_costs_open_plus_k_extend():
    rng = random.Random(12)
    for _ in range(40):
        a, b = rand_seq(rng, rng.randint(25, 40)), rand_seq(rng, rng.randint(25, 40))
        k = rng.randint(1, 4)
        g = rand_seq(rng, k)
        q, r = a + b, a + g + b
        expect = max((len(a) + len(b)) * 2 - (5 + 2 * k), max(len(a), len(b)) * 2)
        assert O.align(q, r)["score"] == expect  # deletion from the read ('D')
        assert O.align(r, q)["score"] == expect  # insertion in the read ('I')


def test_reverse_strand_item_scores_full_length():
    rng = random.Random(13)
    ref = rand_seq(rng, 400)
    read_fwd = ref[100:200]
    read = "".join({"A": "T", "C": "G", "G": "C", "T": "A"}[c] for c in reversed(read_fwd))
    refc = O.encode(ref)
    out = O.run_batch([refc], np.frombuffer(read.encode(), np.uint8), np.array([0, 100]),
                      np.array([0, 2]), [0, 0], [0, 1], [84, 84], [132, 132])
    assert out["item_score"][1] == 200
    assert out["best"][0]["strand"] == 1 and out["best"][0]["ref_start"] == 100
    assert out["best"][0]["ref_end"] == 199


# ----------------------------------------------------------------- invariants

def rescore(q, r, res, sa=2, sb=3, go=5, ge=2):
    i, j = res["start_i"] - 1, res["start_j"] - 1
    score, last = 0, None
    for op in cigar_ops(res["cigar"]):
        if op == "M":
            score += sa if q[i] == r[j] else -sb
            i += 1
            j += 1
        elif op == "I":
            score -= ge if last == "I" else go + ge
            i += 1
        else:
            score -= ge if last == "D" else go + ge
            j += 1
        last = op
    return score, i, j


def test_invariants_random():
    rng = random.Random(21)
    for _ in range(150):
        m, n = rng.randint(1, 60), rng.randint(1, 80)
        if rng.random() < 0.5:
            q = rand_seq(rng, m)
            r = rand_seq(rng, n)
        else:  # related pair
            r = rand_seq(rng, n)
            st = rng.randint(0, max(0, n - 1))
            q = list(r[st:st + m]) or ["A"]
            for _ in range(rng.randint(0, 4)):
                p = rng.randrange(len(q))
                q[p] = rng.choice(BASES)
            if rng.random() < 0.5 and len(q) > 2:
                del q[rng.randrange(len(q))]
            q = "".join(q)
        res = O.align(q, r)
        assert res["score"] >= 0
        assert O.align(r, q)["score"] == res["score"]  # gaps are symmetric
        if res["score"] > 0:
            s, ei, ej = rescore(q, r, res)
            assert s == res["score"]
            assert (ei, ej) == (res["end_i"], res["end_j"])
            cons_read = sum(ln for ln, op in res["cigar"] if op in (O.OP_M, O.OP_I, O.OP_S))
            cons_ref = sum(ln for ln, op in res["cigar"] if op in (O.OP_M, O.OP_D))
            assert cons_read == len(q)
            assert cons_ref == res["end_j"] - res["start_j"] + 1
            assert res["cigar"][0][1] in (O.OP_M, O.OP_S) and res["cigar"][-1][1] in (O.OP_M, O.OP_S)
        # extending the window never lowers the score
        assert O.align(q, r + rand_seq(rng, 5))["score"] >= res["score"]
        assert O.align(q, rand_seq(rng, 5) + r)["score"] >= res["score"]


def linear_sw(q, r, sa, sb, ge):
    """Textbook linear-gap Smith-Waterman (each gap base costs ge)."""
    m, n = len(q), len(r)
    H = [[0] * (n + 1) for _ in range(m + 1)]
    best = 0
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            d = H[i - 1][j - 1] + (sa if q[i - 1] == r[j - 1] else -sb)
            H[i][j] = max(0, d, H[i - 1][j] - ge, H[i][j - 1] - ge)
            best = max(best, H[i][j])
    return best


def test_gap_open_zero_is_linear_gap_smith_waterman():
    rng = random.Random(31)
    for _ in range(120):
        q, r = rand_seq(rng, rng.randint(1, 40)), rand_seq(rng, rng.randint(1, 50))
        ge = rng.randint(1, 4)
        sa, sb = rng.randint(1, 4), rng.randint(1, 4)
        assert O.align(q, r, O.score_params(sa, sb, 0, ge))["score"] == linear_sw(q, r, sa, sb, ge)


def test_final_row_mode_is_read_end_anchored():
    rng = random.Random(41)
    for _ in range(60):
        q, r = rand_seq(rng, rng.randint(1, 30)), rand_seq(rng, rng.randint(1, 40))
        res = O.align(q, r, mode=1)
        if res["score"] > 0:
            assert res["end_i"] == len(q)
        # brute force for small cases
        if len(q) <= 5 and len(r) <= 5:
            alns = enumerate_alignments(q, r, 2, 3, 5, 2)
            S = max([0] + [a[0] for a in alns if a[3] == len(q)])
            assert res["score"] == S
    # mode 1 never beats the local best
    for _ in range(30):
        q, r = rand_seq(rng, 30), rand_seq(rng, 40)
        assert O.align(q, r, mode=1)["score"] <= O.align(q, r)["score"]


@pytest.mark.parametrize("q,r,params", _brute_cases())
def test_brute_force_final_row_end_column_and_traceback(q, r, params):
    """Final-row readout (Sec. 3.5-3.6: the best cell of the read's last row),
    pinned by enumeration: the score is the best over alignments that consume
    the whole read (end row m, which may end in an insertion), the end column
    is the smallest window column reaching it, and the CIGAR is the
    priority-ranked co-optimal alignment ending in that cell."""
    sa, sb, go, ge = params
    m = len(q)
    res = O.align(q, r, O.score_params(*params), mode=1)
    alns = [a for a in enumerate_alignments(q, r, sa, sb, go, ge) if a[3] == m]
    S = max([0] + [a[0] for a in alns])
    assert res["score"] == S
    if S == 0:
        assert (res["end_i"], res["end_j"]) == (0, 0)
        assert res["cigar"] == []
        return
    ej = min(a[4] for a in alns if a[0] == S)
    assert (res["end_i"], res["end_j"]) == (m, ej)
    if go == 0:
        return  # adjacent gap runs tie with free gap opening (as in the local readout)
    cands = [a for a in alns if a[0] == S and a[4] == ej]
    chosen = min(cands, key=lambda a: backward_rank(a[5]))
    assert (res["start_i"], res["start_j"]) == (chosen[1], chosen[2])
    assert cigar_ops(res["cigar"]) == chosen[5]
    # the CIGAR covers the whole read: leading soft clip only, no trailing clip
    assert res["cigar"][-1][1] != O.OP_S


# ------------------------------------------------------- paper worked examples

def _golden(name):
    kv = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(None, 1)
            kv[k] = v.strip()
    return kv


def test_fig3_two_bit_encoding():
    g = _golden("fig3_seed2.txt")
    ref, k, idx = g["reference"], int(g["seed_len"]), int(g["seed_index"])
    seed = ref[idx:idx + k]
    assert seed == g["seed"]
    bits = "".join(format(int(c), "02b") for c in O.encode(seed))
    assert len(bits) == 2 * k
    printed = g["printed_bits"]
    n_ok = int(g["agreeing_prefix_bits"])
    assert bits[:n_ok] == printed[:n_ok]
    drop = int(g["dropped_bit_index"])
    assert bits[:drop] + bits[drop + 1:] == printed


def test_reverse_complement_example():
    rc = O.revcomp_codes(O.encode("ACC"))
    assert "".join(BASES[c] for c in rc) == "GGT"


def test_seed_counts_overlapping_and_non_overlapping():
    """Sec. 3.2: L-k+1 overlapping seeds, floor(L/k) non-overlapping ones.  A
    read occurring once in a random reference collects exactly that many seed
    hits on its true CAL (Sec. 2.3's example: 81 and 5 for L=100, k=20; Sec. 3.8:
    55 for L=76, k=22)."""
    rng = random.Random(51)
    for L, k, ov, nov in [(100, 20, 81, 5), (76, 22, 55, 3), (88, 22, 67, 4)]:
        ref = rand_seq(rng, 3000)
        read = ref[1000:1000 + L]
        for stride, expect in [(1, ov), (k, nov)]:
            refs, strands, starts, lens, hits = O.candidates([ref], read, k=k, stride=stride,
                                                             pad=8, with_hits=True)
            true = [t for t in range(len(refs)) if strands[t] == 0 and starts[t] == 992]
            assert len(true) == 1
            assert hits[true[0]] == expect


def test_pigeonhole_non_overlapping_seed_guarantee():
    """Sec. 3.1: an 88-base read with fewer than 4 errors always keeps one exact
    non-overlapping 22-base seed, so its true CAL is always found."""
    rng = random.Random(61)
    for trial in range(25):
        ref = rand_seq(rng, 2500)
        pos = rng.randint(0, 2500 - 88)
        read = list(ref[pos:pos + 88])
        for p in rng.sample(range(88), rng.randint(0, 3)):
            read[p] = rng.choice([b for b in BASES if b != read[p]])
        read = "".join(read)
        refs, strands, starts, lens = O.candidates([ref], read, k=22, stride=22, pad=0,
                                                   merge_dist=0)
        assert any(strands[t] == 0 and starts[t] == pos for t in range(len(refs)))


def test_candidates_reverse_strand_and_cal_limit():
    rng = random.Random(71)
    ref = rand_seq(rng, 2000)
    fwd = ref[500:600]
    rc = "".join({"A": "T", "C": "G", "G": "C", "T": "A"}[c] for c in reversed(fwd))
    refs, strands, starts, lens = O.candidates([ref], rc, k=20, pad=10)
    assert list(zip(strands, starts)) == [(1, 490)]
    # a repeated region: every seed occurs twice; a limit of 1 drops them all
    ins = rand_seq(rng, 100)
    rep = ref[:800] + ins + ref[800:1500] + ins + ref[1500:]
    fwd = ins
    assert len(O.candidates([rep], fwd, k=20, pad=10)[0]) == 2
    assert len(O.candidates([rep], fwd, k=20, pad=10, cal_limit=1)[0]) == 0
    assert len(O.candidates([rep], fwd, k=20, pad=10, cal_limit=2)[0]) == 2
    # max_cands keeps the windows with the most seed hits
    other = fwd[:50] + rand_seq(rng, 50)
    rep2 = ref[:300] + other + ref[300:900] + fwd + ref[900:]
    refs, strands, starts, lens, hits = O.candidates([rep2], fwd, k=20, pad=0, max_cands=1,
                                                     with_hits=True)
    assert list(starts) == [300 + 100 + 600] and hits[0] == 81


# ----------------------------------------------- tracker and classification

def test_select_winner_second_and_ties():
    # score, ref, strand, global end
    sel = O.select([10, 12, 12, 12, 7], [0, 1, 0, 0, 0], [0, 0, 1, 1, 0], [50, 40, 60, 60, 10])
    # best 12; smallest ref_id wins -> items 2/3 (same end), smaller index -> 2
    assert sel["best"] == 12 and sel["winner"] == 2
    assert sel["second"] == 12  # item 1 ends elsewhere with the same score
    assert sel["n_ties"] == 2   # (1,40,+) and (0,60,-)
    # a duplicate window holding the same alignment is not a rival
    sel = O.select([9, 9, 4], [0, 0, 0], [0, 0, 0], [33, 33, 90])
    assert sel["winner"] == 0 and sel["second"] == 4 and sel["n_ties"] == 1
    # strand '+' before '-' at the same end, then candidate index
    sel = O.select([5, 5], [0, 0], [1, 0], [20, 20])
    assert sel["winner"] == 1 and sel["n_ties"] == 2 and sel["second"] == 5
    # nothing aligned
    sel = O.select([0, 0], [0, 1], [0, 0], [-1, -1])
    assert sel == dict(best=0, second=0, n_ties=0, winner=-1)
    # per-reference filter
    sel = O.select([10, 12, 8], [0, 1, 0], [0, 0, 0], [5, 6, 7], ref_filter=0)
    assert sel["best"] == 10 and sel["winner"] == 0 and sel["second"] == 8


@pytest.mark.parametrize("sa,sb,expect", [
    (39, 0, O.CLASS_UNALIGNED), (39, 39, O.CLASS_UNALIGNED), (40, 0, O.CLASS_A),
    (0, 40, O.CLASS_B), (40, 39, O.CLASS_A), (45, 40, O.CLASS_A), (44, 40, O.CLASS_AMBIGUOUS),
    (40, 44, O.CLASS_AMBIGUOUS), (40, 45, O.CLASS_B), (100, 100, O.CLASS_AMBIGUOUS),
    (100, 95, O.CLASS_A), (96, 100, O.CLASS_AMBIGUOUS)])
def test_classification_boundaries(sa, sb, expect):
    assert O.classify(sa, sb, min_score=40, margin=5) == expect


def test_classification_margin_one_is_exact_tie_rule():
    for a, b in itertools.product([40, 41, 60], repeat=2):
        c = O.classify(a, b, min_score=40, margin=1)
        assert c == (O.CLASS_AMBIGUOUS if a == b else (O.CLASS_A if a > b else O.CLASS_B))


def test_batch_matches_per_item_align_and_select():
    rng = random.Random(81)
    refs = [rand_seq(rng, 3000), rand_seq(rng, 2000)]
    rc = [O.encode(r) for r in refs]
    reads, offs, cand_off = [], [0], [0]
    c_ref, c_str, c_st, c_len = [], [], [], []
    for _ in range(20):
        m = rng.randint(20, 90)
        rr = rng.randint(0, 1)
        pos = rng.randint(0, len(refs[rr]) - m)
        read = refs[rr][pos:pos + m]
        reads.append(read)
        offs.append(offs[-1] + m)
        for _ in range(rng.randint(0, 5)):
            r2 = rng.randint(0, 1)
            st = rng.randint(0, len(refs[r2]) - 10)
            ln = min(len(refs[r2]) - st, m + 20)
            c_ref.append(r2); c_str.append(rng.randint(0, 1)); c_st.append(st); c_len.append(ln)
        c_ref.append(rr); c_str.append(0); c_st.append(max(0, pos - 10)); c_len.append(min(len(refs[rr]) - max(0, pos - 10), m + 20))
        cand_off.append(len(c_ref))
    bases = np.frombuffer("".join(reads).encode(), np.uint8)
    out = O.run_batch(rc, bases, np.array(offs), np.array(cand_off), c_ref, c_str, c_st, c_len)
    out4 = O.run_batch(rc, bases, np.array(offs), np.array(cand_off), c_ref, c_str, c_st, c_len,
                       threads=4)
    for key in ["item_score", "item_end_i", "item_end_j", "best", "best_per_ref", "cigar"]:
        assert np.array_equal(out[key], out4[key])
    for rd in range(20):
        q = reads[rd]
        qrc = "".join({"A": "T", "C": "G", "G": "C", "T": "A"}[c] for c in reversed(q))
        sc, ge_ = [], []
        for c in range(cand_off[rd], cand_off[rd + 1]):
            res = O.align(qrc if c_str[c] else q, refs[c_ref[c]][c_st[c]:c_st[c] + c_len[c]])
            assert res["score"] == out["item_score"][c]
            sc.append(res["score"])
            ge_.append(c_st[c] + res["end_j"] - 1 if res["score"] > 0 else -1)
        sl = slice(cand_off[rd], cand_off[rd + 1])
        sel = O.select(sc, c_ref[sl], c_str[sl], ge_)
        b = out["best"][rd]
        assert b["score"] == sel["best"] and b["second"] == sel["second"]
        assert b["n_ties"] == sel["n_ties"] and b["item"] == cand_off[rd] + sel["winner"]
        w = cand_off[rd] + sel["winner"]
        res = O.align(qrc if c_str[w] else q, refs[c_ref[w]][c_st[w]:c_st[w] + c_len[w]])
        assert O.cigar_list(out["cigar"][rd], b["cigar_len"]) == res["cigar"]
        assert b["ref_start"] == c_st[w] + res["start_j"] - 1
        assert b["read_start"] == res["start_i"] and b["read_end"] == res["end_i"]


# ---- score-tracker report options (Sec. 4.2: the N highest-scoring CALs, or all
# CALs tied for the highest score)

def test_report_small_example():
    # items: 0 (5, ref0, end10), 1 (9, ref0, end20), 2 duplicate of 1's alignment,
    # 3 (3, ref0, end5), 4 (9, ref1, end20), 5 scores 0 (no alignment)
    sc, ref, st, ge = [5, 9, 9, 3, 9, 0], [0, 0, 0, 0, 1, 0], [0] * 6, [10, 20, 20, 5, 20, 7]
    assert list(O.report(sc, ref, st, ge, O.REPORT_BEST_N, 3)) == [1, 4, 0]
    assert list(O.report(sc, ref, st, ge, O.REPORT_BEST_N, 10)) == [1, 4, 0, 3]
    assert list(O.report(sc, ref, st, ge, O.REPORT_TIED)) == [1, 4]
    # the '-' strand at the same end is a different alignment
    assert list(O.report([4, 4], [0, 0], [1, 0], [9, 9], O.REPORT_TIED)) == [1, 0]
    assert list(O.report([0, 0], [0, 0], [0, 0], [1, 2], O.REPORT_TIED)) == []


def _winner_key(sc, ref, ge, st, t):
    return (-int(sc[t]), int(ref[t]), int(ge[t]), int(st[t]), t)


def test_report_properties_random():
    """The report is characterised without re-deriving it: its items have
    pairwise different (ref, end, strand), come in winner order, N = 1 is the
    tracker's winner and the tied report has n_ties items; every positive item
    left out shares an alignment key with a reported one, or ranks after the
    last reported item (N best) / scores below the best (tied)."""
    rng = random.Random(77)
    for _ in range(400):
        n = rng.randint(0, 30)
        sc = [rng.choice([0, 3, 5, 5, 8, 8, 8]) for _ in range(n)]
        ref = [rng.randrange(2) for _ in range(n)]
        st = [rng.randrange(2) for _ in range(n)]
        ge = [rng.randrange(6) for _ in range(n)]
        sel = O.select(sc, ref, st, ge)
        b, ties, w = sel["best"], sel["n_ties"], sel["winner"]
        for nb in (1, 2, 5, 40):
            rep = list(O.report(sc, ref, st, ge, O.REPORT_BEST_N, nb))
            keys = [(ref[t], ge[t], st[t]) for t in rep]
            assert len(set(keys)) == len(keys)
            assert all(sc[t] > 0 for t in rep)
            ranks = [_winner_key(sc, ref, ge, st, t) for t in rep]
            assert ranks == sorted(ranks)
            assert len(rep) <= nb
            if nb == 1:
                assert rep == ([w] if w >= 0 else [])
            for t in range(n):
                if sc[t] <= 0 or t in rep:
                    continue
                if (ref[t], ge[t], st[t]) in keys:
                    continue
                assert len(rep) == nb and _winner_key(sc, ref, ge, st, t) > ranks[-1]
        tied = list(O.report(sc, ref, st, ge, O.REPORT_TIED))
        assert len(tied) == ties
        assert all(sc[t] == b for t in tied)
        tkeys = {(ref[t], ge[t], st[t]) for t in tied}
        assert all((ref[t], ge[t], st[t]) in tkeys for t in range(n) if sc[t] == b and b > 0)
