/*
 * synth.c -- seeded synthetic inputs shaped like the paper's workloads
 * (McVicar et al., arXiv 1805.00106, Sec. 6.2: 100 bp RNA-seq reads against
 * large references; Fig. 9: most reads have few CALs, with a long tail).
 *
 * This module generates data only: references, reads with sequencing errors,
 * and candidate windows around the true locus plus decoys.  It holds none of
 * the aligner's arithmetic, and both the oracle and the CUDA path consume its
 * output.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014).  Every stream is derived from
 * (seed, purpose) so outputs are reproducible on any host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static void rng_init(rng_t* r, uint64_t seed, uint64_t stream) {
  uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ull);
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return result;
}

static double rng_unif(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [lo, hi] */
static int64_t rng_range(rng_t* r, int64_t lo, int64_t hi) {
  if (hi <= lo) return lo;
  uint64_t span = (uint64_t)(hi - lo) + 1;
  return lo + (int64_t)(rng_next(r) % span);
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

static char comp(char c) {
  switch (c) { case 'A': return 'T'; case 'C': return 'G'; case 'G': return 'C'; default: return 'A'; }
}

static char rand_base(rng_t* r) { return BASES[rng_next(r) >> 62]; }

static char other_base(rng_t* r, char c) {
  for (;;) {
    char b = rand_base(r);
    if (b != c) return b;
  }
}

/* i.i.d. reference with P(C)=P(G)=gc/2, P(A)=P(T)=(1-gc)/2 */
void syn_ref_iid(uint64_t seed, int64_t n, double gc, char* out) {
  rng_t r;
  rng_init(&r, seed, 1);
  for (int64_t i = 0; i < n; ++i) {
    double u = rng_unif(&r);
    if (u < gc * 0.5) out[i] = 'C';
    else if (u < gc) out[i] = 'G';
    else if (u < gc + (1.0 - gc) * 0.5) out[i] = 'A';
    else out[i] = 'T';
  }
}

/* A diverged copy of src: per-base substitution with probability sub, indel
 * events at per-base rate indel (insertion or deletion 50/50, length uniform
 * 1..3), then nblocks block moves (a block of length uniform [blk_lo, blk_hi]
 * is cut and reinserted at a uniform position, reverse-complemented with
 * probability 1/2).  Returns the length written (<= cap). */
int64_t syn_mutate(uint64_t seed, const char* src, int64_t n, double sub, double indel, int nblocks,
                   int64_t blk_lo, int64_t blk_hi, char* out, int64_t cap) {
  rng_t r;
  rng_init(&r, seed, 2);
  int64_t o = 0;
  for (int64_t i = 0; i < n && o < cap;) {
    if (rng_unif(&r) < indel) {
      int len = (int)rng_range(&r, 1, 3);
      if (rng_next(&r) & 1) {
        for (int t = 0; t < len && o < cap; ++t) out[o++] = rand_base(&r);
      } else {
        i += len;
        continue;
      }
    }
    char c = src[i++];
    if (rng_unif(&r) < sub) c = other_base(&r, c);
    if (o < cap) out[o++] = c;
  }
  char* tmp = NULL;
  if (nblocks > 0 && o > blk_hi + 1) tmp = (char*)malloc((size_t)blk_hi);
  for (int b = 0; b < nblocks && tmp; ++b) {
    int64_t len = rng_range(&r, blk_lo, blk_hi);
    if (len >= o) break;
    int64_t from = rng_range(&r, 0, o - len);
    memcpy(tmp, out + from, (size_t)len);
    memmove(out + from, out + from + len, (size_t)(o - from - len));
    int64_t rest = o - len;
    int64_t to = rng_range(&r, 0, rest);
    memmove(out + to + len, out + to, (size_t)(rest - to));
    if (rng_next(&r) & 1) {
      for (int64_t t = 0; t < len; ++t) out[to + t] = comp(tmp[len - 1 - t]);
    } else {
      memcpy(out + to, tmp, (size_t)len);
    }
  }
  free(tmp);
  return o;
}

/* Repeat-rich reference of length n: a fraction rep_frac of the bases comes
 * from repeats, half tandem (a unit of length uniform 2..300 repeated to fill a
 * block of 1-10 kb) and half interspersed (copies of one of n_families
 * consensus units of length uniform 2..300, each copy with 5% divergence); the
 * rest is uniform random in segments of 1-10 kb.  is_rep[i] = 1 marks repeat
 * bases. */
void syn_ref_repeats(uint64_t seed, int64_t n, double rep_frac, int n_families, char* out,
                     uint8_t* is_rep) {
  rng_t r;
  rng_init(&r, seed, 3);
  int fam_cap = 300;
  char* fam = (char*)malloc((size_t)n_families * (size_t)fam_cap);
  int* fam_len = (int*)malloc(sizeof(int) * (size_t)n_families);
  for (int f = 0; f < n_families; ++f) {
    fam_len[f] = (int)rng_range(&r, 2, 300);
    for (int t = 0; t < fam_len[f]; ++t) fam[(size_t)f * fam_cap + t] = rand_base(&r);
  }
  int64_t o = 0, n_tandem = 0, n_inter = 0;
  char unit[300];
  while (o < n) {
    double rep_now = (double)(n_tandem + n_inter) / (double)(o > 0 ? o : 1);
    int kind;
    if (rep_now < rep_frac) kind = (n_tandem <= n_inter) ? 1 : 2;
    else kind = 0;
    if (kind == 0) {
      int64_t len = rng_range(&r, 1000, 10000);
      for (int64_t t = 0; t < len && o < n; ++t) { out[o] = rand_base(&r); is_rep[o++] = 0; }
    } else if (kind == 1) {
      int ul = (int)rng_range(&r, 2, 300);
      for (int t = 0; t < ul; ++t) unit[t] = rand_base(&r);
      int64_t len = rng_range(&r, 1000, 10000);
      for (int64_t t = 0; t < len && o < n; ++t) { out[o] = unit[t % ul]; is_rep[o++] = 1; ++n_tandem; }
    } else {
      int f = (int)rng_range(&r, 0, n_families - 1);
      for (int t = 0; t < fam_len[f] && o < n; ++t) {
        char c = fam[(size_t)f * fam_cap + t];
        if (rng_unif(&r) < 0.05) c = other_base(&r, c);
        out[o] = c;
        is_rep[o++] = 1;
        ++n_inter;
      }
    }
  }
  free(fam);
  free(fam_len);
}

/* Reads: for each read pick a reference by weight, a length uniform in
 * [len_lo, len_hi] and a uniform start; copy the reference with per-base
 * substitution rate sub and indel events at per-base rate indel (insertion or
 * deletion 50/50, length uniform 1..3) until the read has its length; with
 * probability rc_frac the read is reverse-complemented ('-' strand).
 * Truth: reference, start, strand and the number of reference bases spanned. */
void syn_reads(uint64_t seed, int n_refs, const char* const* refs, const int64_t* ref_lens,
               const double* ref_weights, int n_reads, int len_lo, int len_hi, double sub,
               double indel, double rc_frac, char* out_bases, int64_t* out_off, int32_t* t_ref,
               int64_t* t_pos, uint8_t* t_strand, int32_t* t_span) {
  rng_t r;
  rng_init(&r, seed, 4);
  double wsum = 0;
  for (int k = 0; k < n_refs; ++k) wsum += ref_weights[k];
  char* buf = (char*)malloc((size_t)len_hi + 8);
  int64_t o = 0;
  out_off[0] = 0;
  for (int rd = 0; rd < n_reads; ++rd) {
    double u = rng_unif(&r) * wsum;
    int k = 0;
    while (k < n_refs - 1 && u >= ref_weights[k]) { u -= ref_weights[k]; ++k; }
    int L = (int)rng_range(&r, len_lo, len_hi);
    int64_t N = ref_lens[k];
    int64_t slack = L / 8 + 8;
    int64_t pos = rng_range(&r, 0, N - L - slack > 0 ? N - L - slack : 0);
    const char* R = refs[k];
    int len = 0;
    int64_t p = pos;
    while (len < L && p < N) {
      if (rng_unif(&r) < indel) {
        int il = (int)rng_range(&r, 1, 3);
        if (rng_next(&r) & 1) {
          for (int t = 0; t < il && len < L; ++t) buf[len++] = rand_base(&r);
          continue;
        }
        p += il;
        if (p >= N) break;
      }
      char c = R[p++];
      if (rng_unif(&r) < sub) c = other_base(&r, c);
      buf[len++] = c;
    }
    while (len < L) buf[len++] = rand_base(&r); /* ran off the end: pad randomly */
    int rc = rng_unif(&r) < rc_frac;
    char* dst = out_bases + o;
    if (rc) for (int t = 0; t < L; ++t) dst[t] = comp(buf[L - 1 - t]);
    else memcpy(dst, buf, (size_t)L);
    o += L;
    out_off[rd + 1] = o;
    t_ref[rd] = k;
    t_pos[rd] = pos;
    t_strand[rd] = (uint8_t)rc;
    t_span[rd] = (int32_t)((p < N ? p : N) - pos);
  }
  free(buf);
}

static int poisson(rng_t* r, double mean) {
  double L = exp(-mean), p = 1.0;
  int k = 0;
  do { ++k; p *= rng_unif(r); } while (p > L);
  return k - 1;
}

/* Candidate windows per read.  count_kind: 0 = fixed p1; 1 = Poisson(p1);
 * 2 = uniform integer in [0, p1]; 3 = floor(Pareto(x_m = 1, alpha = p1)); all
 * capped at cap_per_read.  When the count is >= 1 the first window is the true
 * locus [pos - pad, pos + span + pad); the others are decoys [p - pad, p + m +
 * pad) at a uniform reference and position (with probability p2 drawn from a
 * base flagged in rep_mask of reference 0 when rep_mask is given), strand
 * uniform.  Windows are clamped to the reference.  Returns the number of
 * windows, or -1 if cap is too small. */
int64_t syn_cands(uint64_t seed, int n_reads, const int64_t* read_off, const int32_t* t_ref,
                  const int64_t* t_pos, const uint8_t* t_strand, const int32_t* t_span,
                  int n_refs, const int64_t* ref_lens, int count_kind, double p1, double p2,
                  int cap_per_read, int pad, const uint8_t* rep_mask, int64_t* cand_off,
                  uint8_t* c_ref, uint8_t* c_strand, int64_t* c_start, int32_t* c_len,
                  int64_t cap) {
  rng_t r;
  rng_init(&r, seed, 5);
  int64_t o = 0;
  cand_off[0] = 0;
  for (int rd = 0; rd < n_reads; ++rd) {
    int m = (int)(read_off[rd + 1] - read_off[rd]);
    int cnt;
    switch (count_kind) {
      case 0: cnt = (int)p1; break;
      case 1: cnt = poisson(&r, p1); break;
      case 2: cnt = (int)rng_range(&r, 0, (int64_t)p1); break;
      default: {
        double u = rng_unif(&r);
        double x = 1.0 / pow(1.0 - u, 1.0 / p1);
        cnt = x > 1e9 ? 1000000000 : (int)floor(x);
      }
    }
    if (cnt > cap_per_read) cnt = cap_per_read;
    if (o + cnt > cap) return -1;
    for (int t = 0; t < cnt; ++t) {
      int k;
      int64_t lo, hi;
      uint8_t st;
      if (t == 0) {
        k = t_ref[rd];
        lo = t_pos[rd] - pad;
        hi = t_pos[rd] + t_span[rd] + pad;
        st = t_strand[rd];
      } else {
        k = (int)rng_range(&r, 0, n_refs - 1);
        int64_t N = ref_lens[k];
        int64_t p = rng_range(&r, 0, N > m ? N - m : 0);
        if (rep_mask && k == 0 && rng_unif(&r) < p2) {
          for (int tries = 0; tries < 64; ++tries) {
            int64_t q = rng_range(&r, 0, N > m ? N - m : 0);
            if (rep_mask[q]) { p = q; break; }
          }
        }
        lo = p - pad;
        hi = p + m + pad;
        st = (uint8_t)(rng_next(&r) & 1);
      }
      if (lo < 0) lo = 0;
      if (hi > ref_lens[k]) hi = ref_lens[k];
      if (hi <= lo) { lo = 0; hi = ref_lens[k] < 1 ? 1 : (ref_lens[k] < m ? ref_lens[k] : m); }
      c_ref[o] = (uint8_t)k;
      c_strand[o] = st;
      c_start[o] = lo;
      c_len[o] = (int32_t)(hi - lo);
      ++o;
    }
    cand_off[rd + 1] = o;
  }
  return o;
}
