/*
 * sr_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, obviously-correct scalar CPU restatement of what the extension
 * step of McVicar et al., "FPGA Acceleration of Short Read Alignment"
 * (arXiv 1805.00106) computes: affine-gap Smith-Waterman scoring of a read
 * against the reference window at each candidate alignment location (Sec. 3.5),
 * the per-read score tracker (Sec. 3.6, Sec. 4.2), traceback to a CIGAR
 * (Sec. 6.4, Table 5 discussion), classification between two references by the
 * higher score (Sec. 6.1, 6.2, 6.4) and, for testing the host stage, a
 * brute-force CAL finder/filter (Sec. 3.1-3.3) with no index at all.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
 * reference legs may load this library.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Full (m+1) x (n+1) int32 matrices, row-major (i = read row outer, j = window
 * column inner), no blocking or fusion.  Readings of points the paper leaves
 * open (tie-breaks, gap convention, best-cell readout) are stated at each
 * function.
 */
#include "sr_oracle.h"

#include <limits.h>
#include <stdlib.h>
#include <string.h>

#define OR_NEG (INT32_MIN / 4) /* "minus infinity" for E(i,0) and F(0,j) */

static int32_t or_max2(int32_t a, int32_t b) { return a > b ? a : b; }

/* 2-bit base codes of Fig. 3 (A=00, C=01, G=10, T=11).  Any other byte is an
 * unknown base; the paper keeps Ns out of the CAL table (Sec. 3.7), this
 * restatement rejects them (returns -1). */
int or_encode(const char* ascii, int64_t n, uint8_t* codes) {
  for (int64_t i = 0; i < n; ++i) {
    switch (ascii[i]) {
      case 'A': case 'a': codes[i] = 0; break;
      case 'C': case 'c': codes[i] = 1; break;
      case 'G': case 'g': codes[i] = 2; break;
      case 'T': case 't': codes[i] = 3; break;
      default: return -1;
    }
  }
  return 0;
}

/* Reverse complement (Sec. 3.1: "ACC" -> "GGT"): reverse the string and swap
 * A<->T, C<->G. */
void or_revcomp(const uint8_t* in, int64_t n, uint8_t* out) {
  static const uint8_t comp[4] = {3, 2, 1, 0};
  for (int64_t i = 0; i < n; ++i) out[i] = comp[in[n - 1 - i]];
}

/* Affine-gap local alignment (Sec. 3.5; the paper's ref. [12] is Gotoh's
 * recurrence).  For i = 1..m (read q), j = 1..n (window r):
 *   E(i,j) = max(H(i,j-1) - (go+ge), E(i,j-1) - ge)   gap in the read  -> 'D'
 *   F(i,j) = max(H(i-1,j) - (go+ge), F(i-1,j) - ge)   gap in the window -> 'I'
 *   H(i,j) = max(0, H(i-1,j-1) + s(q_i, r_j), E(i,j), F(i,j))
 * with H(i,0) = H(0,j) = 0, E(i,0) = F(0,j) = -inf, s = +match or -mismatch.
 *
 * Readout: mode 0 takes the best cell over the whole table (true local
 * alignment); mode 1 takes the best cell of the final row only, the readout
 * Sec. 3.5 describes for the systolic array.
 * End-cell tie-break: highest score, then smallest window column j, then
 * smallest read row i.  Score 0 means "no alignment" and the end is (0,0).
 *
 * Traceback priorities (from the end cell, state H):
 *   state H at (i,j): stop if H = 0; else diagonal ('M') if H = H(i-1,j-1)+s;
 *                     else go to state E if H = E(i,j); else state F.
 *   state E at (i,j): emit 'D'; if E(i,j) = H(i,j-1)-(go+ge) go to H (open wins
 *                     a tie), else stay in E; j -= 1.
 *   state F at (i,j): emit 'I'; if F(i,j) = H(i-1,j)-(go+ge) go to H, else
 *                     stay in F; i -= 1.
 * The CIGAR is S(start_i-1), the run-length encoded M/I/D ops, S(m-end_i).
 */
int or_align(const uint8_t* q, int m, const uint8_t* r, int n, const or_score* sp, int mode,
             uint32_t* cigar, int cigar_cap, or_aln* out) {
  memset(out, 0, sizeof(*out));
  if (m <= 0 || n <= 0) return 0;
  const int32_t sa = sp->match, sb = sp->mismatch, go = sp->gap_open, ge = sp->gap_extend;
  const int32_t goe = go + ge;
  const size_t W = (size_t)n + 1;
  const size_t cells = ((size_t)m + 1) * W;
  int32_t* H = (int32_t*)malloc(cells * sizeof(int32_t));
  int32_t* E = (int32_t*)malloc(cells * sizeof(int32_t));
  int32_t* F = (int32_t*)malloc(cells * sizeof(int32_t));
  if (!H || !E || !F) { free(H); free(E); free(F); return -1; }
#define AT(M, i, j) M[(size_t)(i) * W + (size_t)(j)]
  for (int j = 0; j <= n; ++j) { AT(H, 0, j) = 0; AT(E, 0, j) = OR_NEG; AT(F, 0, j) = OR_NEG; }
  for (int i = 0; i <= m; ++i) { AT(H, i, 0) = 0; AT(E, i, 0) = OR_NEG; AT(F, i, 0) = OR_NEG; }

  int32_t best = 0;
  int bi = 0, bj = 0;
  for (int i = 1; i <= m; ++i) {
    for (int j = 1; j <= n; ++j) {
      int32_t e = or_max2(AT(H, i, j - 1) - goe, AT(E, i, j - 1) - ge);
      int32_t f = or_max2(AT(H, i - 1, j) - goe, AT(F, i - 1, j) - ge);
      int32_t s = (q[i - 1] == r[j - 1]) ? sa : -sb;
      int32_t h = or_max2(or_max2(0, AT(H, i - 1, j - 1) + s), or_max2(e, f));
      AT(E, i, j) = e;
      AT(F, i, j) = f;
      AT(H, i, j) = h;
      if (mode == 0 || i == m) {
        int better = h > best || (h == best && h > 0 && (j < bj || (j == bj && i < bi)));
        if (better) { best = h; bi = i; bj = j; }
      }
    }
  }
  out->score = best;
  out->end_i = bi;
  out->end_j = bj;

  if (best > 0 && cigar) {
    /* walk back; ops collected in reverse order */
    int cap_ops = m + n + 2;
    uint8_t* ops = (uint8_t*)malloc((size_t)cap_ops);
    int nops = 0;
    int i = bi, j = bj, state = 0; /* 0 = H, 1 = E, 2 = F */
    for (;;) {
      if (state == 0) {
        int32_t h = AT(H, i, j);
        if (h == 0) break;
        int32_t s = (q[i - 1] == r[j - 1]) ? sa : -sb;
        if (h == AT(H, i - 1, j - 1) + s) {
          ops[nops++] = OR_OP_M;
          --i; --j;
        } else if (h == AT(E, i, j)) {
          state = 1;
        } else {
          state = 2;
        }
      } else if (state == 1) {
        ops[nops++] = OR_OP_D;
        state = (AT(E, i, j) == AT(H, i, j - 1) - goe) ? 0 : 1;
        --j;
      } else {
        ops[nops++] = OR_OP_I;
        state = (AT(F, i, j) == AT(H, i - 1, j) - goe) ? 0 : 2;
        --i;
      }
    }
    out->start_i = i + 1;
    out->start_j = j + 1;
    int nc = 0;
    if (out->start_i > 1 && nc < cigar_cap) cigar[nc++] = ((uint32_t)(out->start_i - 1) << 4) | OR_OP_S;
    for (int k = nops - 1; k >= 0;) {
      int op = ops[k], len = 0;
      while (k >= 0 && ops[k] == op) { ++len; --k; }
      if (nc < cigar_cap) cigar[nc++] = ((uint32_t)len << 4) | (uint32_t)op;
    }
    if (bi < m && nc < cigar_cap) cigar[nc++] = ((uint32_t)(m - bi) << 4) | OR_OP_S;
    out->n_cigar = nc;
    free(ops);
  }
#undef AT
  free(H); free(E); free(F);
  return 0;
}

/* Score tracker (Sec. 3.6: the read's best-scoring location is kept; Sec. 4.2
 * lists single-best, N-best and all-tied reporting modes).
 * Over the items of one read (optionally only those of one reference):
 *   winner: highest score, then smallest ref_id, then smallest global end
 *           position, then '+' before '-', then smallest candidate index;
 *   second: highest score among items whose (ref_id, global end, strand)
 *           differs from the winner's;
 *   n_ties: number of distinct (ref_id, global end, strand) reaching the best.
 * Items scoring 0 have no alignment and never win. */
void or_select(int n_items, const int32_t* score, const int32_t* ref_id, const int32_t* strand,
               const int64_t* gend, const int32_t* cand, int ref_filter,
               int32_t* best, int32_t* second, uint32_t* n_ties, int32_t* winner) {
  int w = -1;
  for (int t = 0; t < n_items; ++t) {
    if (ref_filter >= 0 && ref_id[t] != ref_filter) continue;
    if (score[t] <= 0) continue;
    if (w < 0) { w = t; continue; }
    int better;
    if (score[t] != score[w]) better = score[t] > score[w];
    else if (ref_id[t] != ref_id[w]) better = ref_id[t] < ref_id[w];
    else if (gend[t] != gend[w]) better = gend[t] < gend[w];
    else if (strand[t] != strand[w]) better = strand[t] < strand[w];
    else better = cand[t] < cand[w];
    if (better) w = t;
  }
  *winner = w;
  if (w < 0) { *best = 0; *second = 0; *n_ties = 0; return; }
  *best = score[w];
  int32_t sec = 0;
  uint32_t ties = 0;
  for (int t = 0; t < n_items; ++t) {
    if (ref_filter >= 0 && ref_id[t] != ref_filter) continue;
    if (score[t] <= 0) continue;
    int same_as_winner = ref_id[t] == ref_id[w] && gend[t] == gend[w] && strand[t] == strand[w];
    if (!same_as_winner && score[t] > sec) sec = score[t];
    if (score[t] == score[w]) {
      int seen = 0;
      for (int u = 0; u < t; ++u) {
        if (ref_filter >= 0 && ref_id[u] != ref_filter) continue;
        if (score[u] == score[w] && ref_id[u] == ref_id[t] && gend[u] == gend[t] && strand[u] == strand[t]) { seen = 1; break; }
      }
      if (!seen) ++ties;
    }
  }
  *second = sec;
  *n_ties = ties;
}

/* Score-tracker report options of Sec. 4.2: the highest-scoring CALs up to a
 * number (kind 1), or all CALs tied for the highest score (kind 2).  The items
 * with a positive score are taken in the winner order of or_select (score
 * descending, then ref_id, global end, strand, candidate index ascending); an
 * item whose (ref_id, global end, strand) equals that of an item already taken
 * reports the same alignment and is skipped.  Kind 1 stops after n_best items,
 * kind 2 at the first item scoring below the best.  At most cap indices are
 * written to out; the return value is the number written. */
int or_report(int n_items, const int32_t* score, const int32_t* ref_id, const int32_t* strand,
              const int64_t* gend, const int32_t* cand, int kind, int n_best, int cap, int32_t* out) {
  int* order = (int*)malloc(sizeof(int) * (n_items > 0 ? n_items : 1));
  int n = 0;
  for (int t = 0; t < n_items; ++t)
    if (score[t] > 0) order[n++] = t;
  /* selection sort by the winner order */
  for (int a = 0; a < n; ++a) {
    int b = a;
    for (int c = a + 1; c < n; ++c) {
      int x = order[c], y = order[b], better;
      if (score[x] != score[y]) better = score[x] > score[y];
      else if (ref_id[x] != ref_id[y]) better = ref_id[x] < ref_id[y];
      else if (gend[x] != gend[y]) better = gend[x] < gend[y];
      else if (strand[x] != strand[y]) better = strand[x] < strand[y];
      else better = cand[x] < cand[y];
      if (better) b = c;
    }
    int tmp = order[a]; order[a] = order[b]; order[b] = tmp;
  }
  int k = 0;
  for (int a = 0; a < n && k < cap; ++a) {
    int x = order[a];
    if (kind == 1 && k >= n_best) break;
    if (kind == 2 && score[x] != score[order[0]]) break;
    int seen = 0;
    for (int u = 0; u < k; ++u) {
      int y = out[u];
      if (ref_id[y] == ref_id[x] && gend[y] == gend[x] && strand[y] == strand[x]) { seen = 1; break; }
    }
    if (!seen) out[k++] = x;
  }
  free(order);
  return k;
}

/* Xenograft classification (Sec. 6.1, 6.2: the higher score decides; Sec. 6.4:
 * equal is a tie, a read aligned to one reference only counts for it, reads
 * aligned to neither with any certainty are unaligned).  min_score is the
 * certainty threshold, margin the score difference needed to decide. */
int or_classify(int32_t score_a, int32_t score_b, int32_t min_score, int32_t margin) {
  int32_t hi = score_a > score_b ? score_a : score_b;
  if (hi < min_score) return OR_CLASS_UNALIGNED;
  if (score_b < min_score) return OR_CLASS_A;
  if (score_a < min_score) return OR_CLASS_B;
  if (score_a - score_b >= margin) return OR_CLASS_A;
  if (score_b - score_a >= margin) return OR_CLASS_B;
  return OR_CLASS_AMBIGUOUS;
}

/* ---- brute-force CAL finder + filter (Sec. 3.1-3.3), no index ---- */

static int or_kmer_less(const uint8_t* a, const uint8_t* b, int k) {
  for (int t = 0; t < k; ++t) if (a[t] != b[t]) return a[t] < b[t];
  return 0;
}

/* canonical form of a k-mer: the lexicographically smaller of it and its
 * reverse complement (Sec. 3.1) */
static void or_canonical(const uint8_t* s, int k, uint8_t* rc, uint8_t* canon) {
  or_revcomp(s, k, rc);
  if (or_kmer_less(rc, s, k)) memcpy(canon, rc, (size_t)k);
  else memcpy(canon, s, (size_t)k);
}

typedef struct { int32_t ref, strand; int64_t cal; int32_t hits; } or_cal;

static int or_cal_cmp(const void* a, const void* b) {
  const or_cal* x = (const or_cal*)a;
  const or_cal* y = (const or_cal*)b;
  if (x->ref != y->ref) return x->ref < y->ref ? -1 : 1;
  if (x->strand != y->strand) return x->strand < y->strand ? -1 : 1;
  if (x->cal != y->cal) return x->cal < y->cal ? -1 : 1;
  return 0;
}

static int or_rank_cmp(const void* a, const void* b) {
  const or_cal* x = (const or_cal*)a;
  const or_cal* y = (const or_cal*)b;
  if (x->hits != y->hits) return x->hits > y->hits ? -1 : 1;
  return or_cal_cmp(a, b);
}

/* Seeds of the read start at offsets 0, stride, 2*stride, ... while a full
 * seed fits (stride 1 = overlapping, stride k = non-overlapping, Sec. 3.2).
 * For each seed, every reference position p whose k-mer has the same canonical
 * form is a hit, unless that canonical k-mer occurs more than cal_limit times
 * in the reference (cal_limit 0 = no limit; Sec. 4.1).  A hit where the
 * reference k-mer equals the seed gives a '+' CAL at p - o; one where it equals
 * the seed's reverse complement gives a '-' CAL at p - (m - o - k).  CALs are
 * sorted by (ref, strand, cal); runs whose consecutive CALs differ by at most
 * merge_dist are merged into one (Sec. 3.3), represented by the CAL value that
 * the most seeds hit (smallest on ties).
 * Each surviving CAL becomes the window [cal - pad, cal + m + pad) clamped to
 * the reference.  When max_cands > 0 and there are more windows, the ones with
 * the most seed hits are kept (ties: ref, strand, cal ascending).  Returns the
 * number of windows, or -1 if cap is too small; out_hits (optional) receives
 * the number of seed hits merged into each window. */
int or_candidates(int n_refs, const uint8_t* const* refs, const int64_t* ref_lens,
                  const uint8_t* read, int m, int k, int stride, int merge_dist, int pad,
                  int max_cands, int cal_limit, int cap, int32_t* out_ref, int32_t* out_strand,
                  int64_t* out_start, int32_t* out_len, int32_t* out_hits) {
  if (k <= 0 || stride <= 0 || m < k) return 0;
  uint8_t* rc = (uint8_t*)malloc((size_t)k);
  uint8_t* canon = (uint8_t*)malloc((size_t)k);
  uint8_t* rrc = (uint8_t*)malloc((size_t)k);
  uint8_t* rcanon = (uint8_t*)malloc((size_t)k);
  uint8_t* srev = (uint8_t*)malloc((size_t)k);
  size_t ncap = 1024, ncal = 0;
  or_cal* cals = (or_cal*)malloc(ncap * sizeof(or_cal));
  for (int o = 0; o + k <= m; o += stride) {
    const uint8_t* s = read + o;
    or_canonical(s, k, rc, canon);
    or_revcomp(s, k, srev);
    for (int r = 0; r < n_refs; ++r) {
      const uint8_t* R = refs[r];
      int64_t N = ref_lens[r];
      if (cal_limit > 0) {
        int64_t occ = 0;
        for (int64_t p = 0; p + k <= N; ++p) {
          or_canonical(R + p, k, rrc, rcanon);
          if (memcmp(rcanon, canon, (size_t)k) == 0) ++occ;
        }
        if (occ > cal_limit) continue;
      }
      for (int64_t p = 0; p + k <= N; ++p) {
        int fwd = memcmp(R + p, s, (size_t)k) == 0;
        int rev = memcmp(R + p, srev, (size_t)k) == 0;
        for (int pass = 0; pass < 2; ++pass) {
          int hit = pass == 0 ? fwd : rev;
          if (!hit) continue;
          if (ncal == ncap) { ncap *= 2; cals = (or_cal*)realloc(cals, ncap * sizeof(or_cal)); }
          cals[ncal].ref = r;
          cals[ncal].strand = pass;
          cals[ncal].cal = pass == 0 ? p - o : p - (m - o - k);
          cals[ncal].hits = 1;
          ++ncal;
        }
      }
    }
  }
  qsort(cals, ncal, sizeof(or_cal), or_cal_cmp);
  size_t nw = 0;
  for (size_t t = 0; t < ncal;) {
    size_t u = t + 1;
    while (u < ncal && cals[u].ref == cals[t].ref && cals[u].strand == cals[t].strand &&
           cals[u].cal - cals[u - 1].cal <= merge_dist)
      ++u;
    /* representative: the CAL value hit by the most seeds, smallest on ties */
    or_cal merged = cals[t];
    int32_t best_cnt = 0;
    for (size_t v = t; v < u;) {
      size_t w = v;
      while (w < u && cals[w].cal == cals[v].cal) ++w;
      if ((int32_t)(w - v) > best_cnt) { best_cnt = (int32_t)(w - v); merged.cal = cals[v].cal; }
      v = w;
    }
    merged.hits = (int32_t)(u - t);
    cals[nw++] = merged;
    t = u;
  }
  if (max_cands > 0 && nw > (size_t)max_cands) {
    qsort(cals, nw, sizeof(or_cal), or_rank_cmp);
    nw = (size_t)max_cands;
    qsort(cals, nw, sizeof(or_cal), or_cal_cmp);
  }
  int ret = (int)nw;
  if (nw > (size_t)cap) ret = -1;
  else {
    for (size_t t = 0; t < nw; ++t) {
      int64_t N = ref_lens[cals[t].ref];
      int64_t lo = cals[t].cal - pad, hi = cals[t].cal + m + pad;
      if (lo < 0) lo = 0;
      if (hi > N) hi = N;
      out_ref[t] = cals[t].ref;
      out_strand[t] = cals[t].strand;
      out_start[t] = lo;
      out_len[t] = (int32_t)(hi - lo);
      if (out_hits) out_hits[t] = cals[t].hits;
    }
  }
  free(cals); free(rc); free(canon); free(rrc); free(rcanon); free(srev);
  return ret;
}

/* ---- whole batch: every (read, window) item, per-read tracker, winner CIGAR ---- */

/* For each read: encode it (reverse-complement it for '-' windows: Sec. 3.1
 * keeps a strand bit per CAL so the final alignment runs on the matching
 * strand), align it to each of its
 * windows, select per read and per reference, and trace back the overall
 * winner.  Outputs are indexed by the global item index (cand_off CSR). */
int or_run_batch(int n_refs, const uint8_t* const* refs, const int64_t* ref_lens,
                 int n_reads, const char* bases, const int64_t* read_off,
                 const int64_t* cand_off, const uint8_t* c_ref, const uint8_t* c_strand,
                 const int64_t* c_start, const int32_t* c_len, const or_score* sp, int mode,
                 int32_t* item_score, int32_t* item_end_i, int32_t* item_end_j,
                 or_hit* best, or_hit* best_per_ref, uint32_t* cigar) {
  int rc_status = 0;
  for (int rd = 0; rd < n_reads; ++rd) {
    int m = (int)(read_off[rd + 1] - read_off[rd]);
    uint8_t* fwd = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
    uint8_t* rev = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
    if (or_encode(bases + read_off[rd], m, fwd) != 0) { free(fwd); free(rev); return -2; }
    or_revcomp(fwd, m, rev);
    int64_t c0 = cand_off[rd], c1 = cand_off[rd + 1];
    int nit = (int)(c1 - c0);
    int32_t* sc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nit > 0 ? nit : 1));
    int32_t* rid = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nit > 0 ? nit : 1));
    int32_t* str = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nit > 0 ? nit : 1));
    int32_t* cix = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nit > 0 ? nit : 1));
    int64_t* ge = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nit > 0 ? nit : 1));
    for (int t = 0; t < nit; ++t) {
      int64_t c = c0 + t;
      item_end_i[c] = 0;
      item_end_j[c] = 0;
      if (c_ref[c] >= n_refs || c_strand[c] > 1 || c_len[c] <= 0 ||
          c_start[c] < 0 || c_start[c] + c_len[c] > ref_lens[c_ref[c]]) { rc_status = -3; sc[t] = 0; }
      else {
        or_aln a;
        const uint8_t* q = c_strand[c] ? rev : fwd;
        or_align(q, m, refs[c_ref[c]] + c_start[c], c_len[c], sp, mode, NULL, 0, &a);
        sc[t] = a.score;
        item_end_i[c] = a.end_i;
        item_end_j[c] = a.end_j;
      }
      item_score[c] = sc[t];
      rid[t] = c_ref[c];
      str[t] = c_strand[c];
      cix[t] = t;
      ge[t] = sc[t] > 0 ? c_start[c] + item_end_j[c] - 1 : -1;
    }
    or_hit* h = &best[rd];
    memset(h, 0, sizeof(*h));
    int32_t w;
    or_select(nit, sc, rid, str, ge, cix, -1, &h->score, &h->second, &h->n_ties, &w);
    h->item = w >= 0 ? (int32_t)(c0 + w) : -1;
    if (w >= 0) {
      int64_t c = c0 + w;
      or_aln a;
      const uint8_t* q = c_strand[c] ? rev : fwd;
      or_align(q, m, refs[c_ref[c]] + c_start[c], c_len[c], sp, mode,
               cigar + (size_t)rd * OR_CIGAR_CAP, OR_CIGAR_CAP, &a);
      h->ref_id = c_ref[c];
      h->strand = c_strand[c];
      h->ref_start = c_start[c] + a.start_j - 1;
      h->ref_end = c_start[c] + a.end_j - 1;
      h->read_start = a.start_i;
      h->read_end = a.end_i;
      h->cigar_len = (uint32_t)a.n_cigar;
    }
    for (int r = 0; r < n_refs; ++r) {
      or_hit* hr = &best_per_ref[(size_t)rd * n_refs + r];
      memset(hr, 0, sizeof(*hr));
      int32_t wr;
      or_select(nit, sc, rid, str, ge, cix, r, &hr->score, &hr->second, &hr->n_ties, &wr);
      hr->item = wr >= 0 ? (int32_t)(c0 + wr) : -1;
      if (wr >= 0) {
        hr->ref_id = r;
        hr->strand = str[wr];
        hr->ref_end = ge[wr];
      }
    }
    free(fwd); free(rev); free(sc); free(rid); free(str); free(cix); free(ge);
  }
  return rc_status;
}
