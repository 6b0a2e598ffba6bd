/*
 * sr_oracle.h -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * Declarations of the plain, slow, scalar CPU restatement of the extension
 * step of the seed-and-extend short-read aligner of McVicar et al., "FPGA
 * Acceleration of Short Read Alignment" (arXiv 1805.00106).  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs may load
 * the oracle library.  It shares no code with the CUDA path (paper_1805_00106_gb300).
 *
 * Encoding (Sec. 3.1, Fig. 3): A=0, C=1, G=2, T=3.
 * Scores (Sec. 3.5, affine gap): a gap of k bases costs gap_open + k*gap_extend.
 */
#ifndef SR_ORACLE_H
#define SR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_CIGAR_CAP 1040 /* CIGAR words per read: >= 2*max_read_len + 2 for reads <= 512 bp */

/* BAM-style CIGAR op codes, word = (len << 4) | op */
enum { OR_OP_M = 0, OR_OP_I = 1, OR_OP_D = 2, OR_OP_S = 4 };

enum { OR_CLASS_UNALIGNED = 0, OR_CLASS_A = 1, OR_CLASS_B = 2, OR_CLASS_AMBIGUOUS = 3 };

typedef struct {
  int32_t match, mismatch, gap_open, gap_extend;
} or_score;

typedef struct {
  int32_t score;
  int32_t end_i, end_j;     /* 1-based end cell, (0,0) when score == 0 */
  int32_t start_i, start_j; /* 1-based first aligned cell, (0,0) when score == 0 */
  int32_t n_cigar;          /* words written to the CIGAR buffer */
} or_aln;

typedef struct {
  int32_t score, second;
  uint32_t n_ties;
  int32_t item;             /* index into the batch's item list, -1 = none */
  int32_t ref_id, strand;
  int64_t ref_start, ref_end; /* 0-based inclusive on the forward reference */
  int32_t read_start, read_end; /* 1-based, on the read as aligned (revcomp for '-') */
  uint32_t cigar_len;
} or_hit;

int or_encode(const char* ascii, int64_t n, uint8_t* codes);
void or_revcomp(const uint8_t* in, int64_t n, uint8_t* out);

int or_align(const uint8_t* q, int m, const uint8_t* r, int n, const or_score* sp, int mode,
             uint32_t* cigar, int cigar_cap, or_aln* out);

void or_select(int n_items, const int32_t* score, const int32_t* ref_id, const int32_t* strand,
               const int64_t* gend, const int32_t* cand, int ref_filter,
               int32_t* best, int32_t* second, uint32_t* n_ties, int32_t* winner);

int or_report(int n_items, const int32_t* score, const int32_t* ref_id, const int32_t* strand,
              const int64_t* gend, const int32_t* cand, int kind, int n_best, int cap, int32_t* out);

int or_classify(int32_t score_a, int32_t score_b, int32_t min_score, int32_t margin);

int or_candidates(int n_refs, const uint8_t* const* refs, const int64_t* ref_lens,
                  const uint8_t* read, int m, int k, int stride, int merge_dist, int pad,
                  int max_cands, int cal_limit, int cap, int32_t* out_ref, int32_t* out_strand,
                  int64_t* out_start, int32_t* out_len, int32_t* out_hits);

int or_run_batch(int n_refs, const uint8_t* const* refs, const int64_t* ref_lens,
                 int n_reads, const char* bases, const int64_t* read_off,
                 const int64_t* cand_off, const uint8_t* c_ref, const uint8_t* c_strand,
                 const int64_t* c_start, const int32_t* c_len, const or_score* sp, int mode,
                 int32_t* item_score, int32_t* item_end_i, int32_t* item_end_j,
                 or_hit* best, or_hit* best_per_ref, uint32_t* cigar);

#ifdef __cplusplus
}
#endif
#endif
