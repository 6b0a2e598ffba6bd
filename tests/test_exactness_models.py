"""Plain-Python restatements of two exactness arguments the CUDA kernels rely
on, checked against the oracle on random cases (CPU, no GPU):

1. virtual columns: lanes of the systolic sweep that run columns before a
   window (score term 0 or -1, below go + ge) keep the H = 0 border, and columns
   past an item's end never beat the best real cell, so per-lane strict-
   improvement tracking and the (score, -column) reduction still give the
   best score and its smallest end column;
2. the traceback band: a DP restricted to the diagonals that can hold any
   alignment of score S ending in column j* at a row in [ceil(S/match), m]
   (cells outside: H = 0, E = F = -inf) finds the end row (smallest i with
   H(i, j*) = S) and reproduces the full-DP traceback exactly; the band is
   the union over those end rows of each row's diagonals, and the closed form
   the kernels evaluate equals that union;
3. four bases per step in the read packing: per byte of a 32-bit word, the
   2-bit code ((c >> 1) ^ (c >> 2)) & 3 of the lower-cased byte c (the bits a
   shift brings in from the next byte are masked off), and the check that
   looking the code's letter up again gives c back, equal the per-base
   definition: A/C/G/T in either case map to 0-3, every other byte is
   rejected.

These models mirror the kernels' arithmetic order, not their code."""
import random

import pytest

from oracle import oracle as O

NEG = -(1 << 28)


def systolic_best(q, r, sa, sb, go, ge, G, R, extra, virt_sc, mode):
    goe, BIAS = go + ge, 1024
    INIT = BIAS - goe
    m, n = len(q), len(r)
    rows = [None] * (G * R - m) + q
    T = [[INIT] * R for _ in range(G)]
    E = [[INIT] * R for _ in range(G)]
    tprev, Tbot, Fbot = [INIT] * G, [INIT] * G, [INIT] * G
    best, jb = [INIT] * G, [0] * G
    for s in range(n + extra + G - 1):
        tin_all, fin_all = [INIT] + Tbot[:-1], [INIT] + Fbot[:-1]
        nTbot, nFbot = Tbot[:], Fbot[:]
        for t in range(G):
            j = s - t
            virtual = not (0 <= j < n)
            td, tup, f = tprev[t], tin_all[t], fin_all[t]
            for k in range(R):
                rr = rows[t * R + k]
                if virtual:
                    sc = virt_sc
                elif rr is None:
                    sc = goe - sb
                else:
                    sc = (sa if rr == r[j] else -sb) + goe
                tl = T[t][k]
                E[t][k] = max(E[t][k] - ge, tl)
                f = max(f - ge, tup)
                h = max(max(td + sc, E[t][k]), f, BIAS)
                td, tup = tl, h - goe
                T[t][k] = tup
            tprev[t], nTbot[t], nFbot[t] = tin_all[t], T[t][R - 1], f
            if mode == 0:
                cm = max(T[t])
            else:  # final row, virtual columns masked
                cm = T[t][R - 1] if (t == G - 1 and not virtual) else 0
            if cm > best[t]:
                best[t], jb[t] = cm, j + 1
        Tbot, Fbot = nTbot, nFbot
    key = max(((b - INIT) << 16) | (0xffff - (j if b > INIT else 0)) for b, j in zip(best, jb))
    score = key >> 16
    return score, (0xffff - (key & 0xffff)) if score else 0


def gap_bound(i, jstar, S, sa, go, ge):
    """Most gap bases an alignment of score S ending in (i, j*) can hold."""
    return max(0, (sa * min(i, jstar) - S - go) // ge)


def band_union(sa, go, ge, S, jstar, ilo, ihi):
    """(dlo, w): the diagonals j* - i - g(i) .. j* - i + g(i) of every end row
    i in ilo..ihi, united row by row."""
    lo = min(jstar - i - gap_bound(i, jstar, S, sa, go, ge) for i in range(ilo, ihi + 1))
    hi = max(jstar - i + gap_bound(i, jstar, S, sa, go, ge) for i in range(ilo, ihi + 1))
    return lo, hi - lo + 1


def band_closed_form(sa, go, ge, S, jstar, ilo, ihi):
    """The kernels' evaluation of the same union: the lower end from row ihi,
    the upper end as the largest of j* - i + g(i) at ilo, ihi, the first row with
    g > 0, j* and j* + 1 (the ends of its monotone pieces)."""
    f = lambda i: jstar - i + gap_bound(i, jstar, S, sa, go, ge)
    i1 = -(-(S + go + ge) // sa)
    cands = [ilo, ihi] + [i for i in (i1, jstar, jstar + 1) if ilo <= i <= ihi]
    dlo = jstar - ihi - gap_bound(ihi, jstar, S, sa, go, ge)
    return dlo, max(f(i) for i in cands) - dlo + 1


def band_traceback(q, r, sa, sb, go, ge, S, jstar, mode):
    goe, m = go + ge, len(q)
    ilo, ihi = (m, m) if mode == 1 else (max(1, -(-S // sa)), m)
    dlo, w = band_union(sa, go, ge, S, jstar, ilo, ihi)
    H, Ev, Fv, dirs = {}, {}, {}, {}
    for i in range(1, ihi + 1):
        for k in range(w):
            j = i + dlo + k
            hl, el = (H[(i, k - 1)], Ev[(i, k - 1)]) if k > 0 else (0, NEG)
            hu, fu = (H.get((i - 1, k + 1), 0), Fv.get((i - 1, k + 1), NEG)) if k + 1 < w else (0, NEG)
            eo, ee, fo, fe = hl - goe, el - ge, hu - goe, fu - ge
            Eh, Fh = max(eo, ee), max(fo, fe)
            if 1 <= j <= jstar:
                hs = H.get((i - 1, k), 0) + (sa if q[i - 1] == r[j - 1] else -sb)
                h = max(0, hs, Eh, Fh)
                dirs[(i, k)] = (h == hs, h == Eh, eo >= ee, fo >= fe)
                H[(i, k)], Ev[(i, k)], Fv[(i, k)] = h, Eh, Fh
            else:
                dirs[(i, k)] = (False, False, False, False)
                H[(i, k)], Ev[(i, k)], Fv[(i, k)] = 0, NEG, NEG
    # the smallest row at or above ilo (row m in final-row mode) where the band holds S
    istar = next((i for i in range(ilo, ihi + 1) if 0 <= jstar - i - dlo < w and H[(i, jstar - i - dlo)] == S),
                 None)
    if istar is None:
        return None
    i, j, k, h, state, ops = istar, jstar, jstar - istar - dlo, S, 0, []
    while True:
        assert 0 <= k < w
        if state == 0:
            if h == 0:
                break
            mb, eb, _, _ = dirs[(i, k)]
            if mb:
                ops.append("M")
                h -= sa if q[i - 1] == r[j - 1] else -sb
                i, j = i - 1, j - 1
                continue
            state = 1 if eb else 2
        elif state == 1:
            pe = dirs[(i, k)][2]
            ops.append("D")
            h += goe if pe else ge
            state = 0 if pe else 1
            j, k = j - 1, k - 1
        else:
            pf = dirs[(i, k)][3]
            ops.append("I")
            h += goe if pf else ge
            state = 0 if pf else 2
            i, k = i - 1, k + 1
    return i + 1, j + 1, istar, "".join(reversed(ops))


PARAMS = [(2, 3, 5, 2), (1, 1, 1, 1), (3, 2, 2, 1), (2, 3, 0, 2), (2, 10, 1, 1), (5, 0, 1, 1)]


def _case(rng):
    m, n = rng.randint(1, 24), rng.randint(1, 40)
    q = [rng.randrange(4) for _ in range(m)]
    r = [rng.randrange(4) for _ in range(n)]
    if rng.random() < 0.75 and n > 3:
        st = rng.randint(0, n - 1)
        for i in range(min(m, n - st)):
            r[st + i] = q[i] if rng.random() > 0.08 else rng.randrange(4)
        if rng.random() < 0.5 and n > 8 and st < n - 2:
            p = rng.randint(st, n - 2)
            if rng.random() < 0.5:
                r.insert(p, rng.randrange(4))
                r.pop()
            else:
                del r[p]
                r.append(rng.randrange(4))
    return q, r


def _s(codes):
    return "".join("ACGT"[c] for c in codes)


@pytest.mark.parametrize("seed", [1, 2])
def test_virtual_columns_keep_best_and_end(seed):
    rng = random.Random(seed)
    for _ in range(250):
        G, R = rng.choice([(4, 4), (8, 2), (2, 8), (4, 3)])
        q, r = _case(rng)
        q = q[: G * R]
        sa, sb, go, ge = rng.choice(PARAMS)
        for mode in (0, 1):
            o = O.align(_s(q), _s(r), O.score_params(sa, sb, go, ge), mode=mode)
            got = systolic_best(q, r, sa, sb, go, ge, G, R, rng.randint(0, 12), rng.choice([0, -1]), mode)
            assert got == (o["score"], o["end_j"] if o["score"] else 0), (q, r, (sa, sb, go, ge), mode)


@pytest.mark.parametrize("seed", [3, 4])
def test_band_finds_end_row_and_full_dp_path(seed):
    rng = random.Random(seed)
    for _ in range(300):
        q, r = _case(rng)
        sa, sb, go, ge = rng.choice(PARAMS)
        for mode in (0, 1):
            o = O.align(_s(q), _s(r), O.score_params(sa, sb, go, ge), mode=mode)
            if o["score"] == 0:
                continue
            got = band_traceback(q, r, sa, sb, go, ge, o["score"], o["end_j"], mode)
            ops = "".join(c * ln for ln, c in [(ln, "MID?S"[op]) for ln, op in o["cigar"]] if c != "S")
            assert got == (o["start_i"], o["start_j"], o["end_i"], ops), (q, r, (sa, sb, go, ge), mode)


@pytest.mark.parametrize("seed", [5, 6])
def test_band_closed_form_is_the_union(seed):
    rng = random.Random(seed)
    for _ in range(3000):
        sa, go, ge = rng.randint(1, 6), rng.randint(0, 12), rng.randint(1, 6)
        m = rng.randint(1, 256)
        jstar = rng.randint(1, 400)
        S = rng.randint(1, sa * min(m, jstar))
        ilo = max(1, -(-S // sa))
        if ilo > m:
            continue
        for lo, hi in ((ilo, m), (m, m), (ilo, ilo)):
            assert band_closed_form(sa, go, ge, S, jstar, lo, hi) == band_union(sa, go, ge, S, jstar, lo, hi)


def _byte_perm(x, y, sel):
    """prmt: output byte i is byte (sel >> 4i) & 7 of the eight bytes of y:x."""
    v = (y << 32) | x
    return sum(((v >> (8 * ((sel >> (4 * i)) & 7))) & 0xFF) << (8 * i) for i in range(4))


def _pack4(word, nvalid):
    """Four bytes -> (packed 2-bit codes of the first nvalid, any byte not ACGT)."""
    keep = 0xFFFFFFFF if nvalid >= 4 else (1 << (8 * nvalid)) - 1
    c = word | 0x20202020
    code = ((c >> 1) ^ (c >> 2)) & 0x03030303 & keep
    t = code | (code >> 4)
    letters = _byte_perm(0x74676361, 0, (t & 0xFF) | ((t >> 8) & 0xFF00))
    bad = ((c ^ letters) & keep) != 0
    u = code | (code >> 6)
    return (u & 0xF) | ((u >> 12) & 0xF0), bad


def _pack4_definition(bs, nvalid):
    codes = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3, ord("a"): 0, ord("c"): 1, ord("g"): 2,
             ord("t"): 3}
    v, bad = 0, False
    for i in range(nvalid):
        if bs[i] in codes:
            v |= codes[bs[i]] << (2 * i)
        else:
            bad = True
    return v, bad


def test_four_base_packing_equals_the_per_base_definition():
    # every single byte, alone in its word and followed by each letter
    for x in range(256):
        for nxt in b"ACGTN\x00\xff":
            word = x | (nxt << 8) | (0x41 << 16) | (0x74 << 24)
            v, bad = _pack4(word, 1)
            dv, dbad = _pack4_definition(bytes([x, nxt, 0x41, 0x74]), 1)
            assert bad == dbad, x
            if not bad:
                assert v == dv, x
    # random words of letters, lower case and other bytes, every count of valid bytes
    rng = random.Random(11)
    pool = list(b"ACGTacgt") * 6 + list(range(256))
    for _ in range(20000):
        bs = bytes(rng.choice(pool) for _ in range(4))
        nvalid = rng.randint(0, 4)
        v, bad = _pack4(int.from_bytes(bs, "little"), nvalid)
        dv, dbad = _pack4_definition(bs, nvalid)
        assert bad == dbad, (bs, nvalid)
        if not bad:
            assert v == dv, (bs, nvalid)
