/*
 * sr.h -- C ABI of libsr, a GB300 (sm_103a) short-read extension library.
 *
 * It implements the data-parallel hot path of the seed-and-extend aligner of
 * McVicar et al., "FPGA Acceleration of Short Read Alignment" (arXiv 1805.00106):
 * affine-gap Smith-Waterman scoring of every read against the reference window
 * of each candidate alignment location (CAL, Sec. 3.5), per-read best /
 * second-best / tie tracking (Sec. 3.6, 4.2), traceback to a CIGAR for the
 * winner (Sec. 4.2, 6.4) and classification of each read between two
 * references by score (Sec. 6.1, 6.2, 6.4).  The k-mer index and CAL
 * finder/filter (Sec. 3.1-3.3, 4.1-4.2) are a host stage.
 *
 * Conventions
 *  - Every call returns sr_status (SR_OK = 0, negative on error); no C++
 *    exception crosses this boundary.  sr_last_error() returns a thread-local
 *    message for the last failure on the calling thread.
 *  - Bases are ASCII A/C/G/T (either case).  Any other byte is SR_EBADBASE.
 *    The 2-bit code is A=0, C=1, G=2, T=3 (Sec. 3.1, Fig. 3).
 *  - Inputs are caller-owned and only read during the call (sr_submit copies
 *    them).  Objects returned through an `out` pointer are owned by the caller
 *    and released with the matching sr_*_free / sr_*_close.
 *  - Scores: match +match, mismatch -mismatch, a gap of k bases costs
 *    gap_open + k*gap_extend (Sec. 3.5; the paper leaves the constants open).
 *  - Positions are 0-based on the forward strand of the reference; read
 *    coordinates (read_start/read_end, 1-based) refer to the read as aligned,
 *    i.e. reverse-complemented for '-' strand windows (Sec. 3.1 strand bit).
 *  - All device work runs in libsr's own CUDA kernels on the current CUDA
 *    device; no CPU fallback exists.  A build without a usable GPU returns
 *    SR_ECUDA from every call that needs one.
 */
#ifndef SR_H
#define SR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sr_status;
enum {
  SR_OK = 0,
  SR_EINVAL = -1,   /* bad argument, size or parameter */
  SR_ENOMEM = -2,   /* host or device allocation failed, or HBM budget exceeded */
  SR_ECUDA = -3,    /* CUDA runtime error (message in sr_last_error) */
  SR_EBADBASE = -4, /* a read or reference byte is not A/C/G/T */
  SR_ETIMEOUT = -5, /* a bounded wait ran out (sr_wait, device queue poll) */
  SR_EBUSY = -6,    /* resource in use (e.g. serving queue full) */
  SR_EIO = -7       /* file I/O or format error */
};

#define SR_MAX_READ_LEN 256u /* longest read the device path accepts */
#define SR_MAX_WIN_LEN 512u  /* longest reference window */
#define SR_MAX_REFS 16u      /* references per session */
#define SR_CIGAR_STRIDE 776u /* CIGAR words reserved per read (>= 3*256+4 runs) */

const char* sr_last_error(void);
const char* sr_version(void);

/* ------------------------------------------------------------------ index
 * Pointer table + CAL table over the canonical (lexicographically smaller of a
 * k-mer and its reverse complement) seeds of every reference position (Sec. 3.1,
 * 4.1).  The whole seed is put through an invertible hash; the top
 * 2*address_bases bits address the pointer table, the rest is the key stored in
 * the CAL table (Sec. 3.1).  Canonical seeds occurring more than cal_limit times
 * are dropped (0 = no limit; Sec. 4.1, Table 5).
 * seed_len in [4, 32]; address_bases in [1, min(seed_len, 14)] and
 * 2*(seed_len - address_bases) <= 32.  n_threads 0 = all host cores. */
typedef struct sr_index sr_index;
typedef struct {
  uint32_t seed_len;      /* default 20 */
  uint32_t address_bases; /* default 12 */
  uint32_t cal_limit;     /* 0 = unlimited */
  uint32_t n_threads;     /* 0 = hardware concurrency */
  uint64_t hash_seed;     /* mixes the invertible seed hash */
} sr_index_params;

/* Build from `len` ASCII bases (copied).  Errors: SR_EINVAL (params), SR_EBADBASE,
 * SR_ENOMEM. */
sr_status sr_index_build(const char* seq, uint64_t len, const sr_index_params* params,
                         sr_index** out);
/* Flat binary file: header (magic, params, sizes), tables, packed reference,
 * checksum.  Errors: SR_EIO. */
sr_status sr_index_save(const sr_index* idx, const char* path);
sr_status sr_index_load(const char* path, sr_index** out);
void sr_index_free(sr_index* idx);
/* Reference length and number of CAL-table entries. */
sr_status sr_index_info(const sr_index* idx, uint64_t* ref_len, uint64_t* n_entries);

/* ------------------------------------------------------------------ reads
 * CSR batch of reads: read r is bases[offsets[r] .. offsets[r+1]).
 * flags: 0 = host memory; SR_FLAG_DEVICE = bases and offsets are device
 * pointers on the current device (for example torch tensors' data_ptr()).
 * Device inputs are accepted by sr_batch_stage and sr_align_batch only (the
 * other calls that take reads or candidates return SR_EINVAL for them); they
 * are read on the call's stream (sr_batch_stage's cuda_stream, sr_align_opts
 * cuda_stream, else the session's stream), so whatever produces them must have
 * finished or run on that stream.  The library copies them into its own device
 * buffers and never frees them. */
enum { SR_FLAG_DEVICE = 1 };
typedef struct {
  uint32_t n_reads;
  uint32_t flags;          /* 0 or SR_FLAG_DEVICE */
  const char* bases;
  const uint64_t* offsets; /* n_reads + 1 entries, offsets[0] = 0 */
} sr_reads;

/* ------------------------------------------------------------- candidates
 * CAL finder + filter (Sec. 3.2, 3.3).  Seeds start at 0, seed_stride,
 * 2*seed_stride, ... (1 = overlapping, seed_len = non-overlapping).  A hit at
 * reference position p from the seed at read offset o gives a '+' CAL p - o when
 * the reference k-mer equals the seed, a '-' CAL p - (m - o - k) when it equals
 * the seed's reverse complement.  CALs of one (ref, strand) whose consecutive
 * values differ by <= merge_dist merge into one, represented by the CAL value
 * hit by the most seeds (smallest on ties).  Each merged CAL becomes the window
 * [cal - pad, cal + m + pad) clamped to the reference.  With max_cands > 0 only
 * the max_cands windows with the most seed hits are kept (ties: ref, strand,
 * cal ascending).  Windows are listed per read by (ref, strand, cal). */
typedef struct {
  uint32_t seed_stride; /* default 1 */
  uint32_t merge_dist;  /* default 32 */
  uint32_t pad;         /* default 32 */
  uint32_t max_cands;   /* 0 = all */
  uint32_t n_threads;   /* 0 = hardware concurrency */
  uint32_t flags;       /* sr_candidates_device only: SR_FLAG_DEVICE = leave the list in device
                           memory (flagged so, ready for sr_align_batch); sr_candidates: 0 */
} sr_cand_params;

typedef struct {
  uint32_t n_reads;
  uint32_t flags;     /* 0 or SR_FLAG_DEVICE: offsets, ref_id, strand, win_start and
                         win_len are device pointers (as for sr_reads) */
  uint64_t n_cands;
  uint64_t* offsets;  /* n_reads + 1: read r owns windows offsets[r] .. offsets[r+1] */
  uint8_t* ref_id;    /* reference index per window */
  uint8_t* strand;    /* 0 = '+', 1 = '-' (read is reverse-complemented) */
  uint64_t* win_start;
  uint32_t* win_len;  /* 1 .. SR_MAX_WIN_LEN */
  uint32_t* hits;     /* seed hits merged into the window (may be NULL on input) */
} sr_cand_list;

/* idx[0..n_refs) are the references' indexes (same seed_len).  Errors:
 * SR_EINVAL, SR_EBADBASE (read bytes), SR_ENOMEM. */
sr_status sr_candidates(const sr_index* const* idx, uint32_t n_refs, const sr_reads* reads,
                        const sr_cand_params* params, sr_cand_list** out);
/* Allocate an empty list the caller fills (for windows chosen elsewhere). */
sr_status sr_cand_list_alloc(uint32_t n_reads, uint64_t n_cands, sr_cand_list** out);
/* Frees a list the library allocated: host arrays, or device arrays when the
 * list is flagged SR_FLAG_DEVICE. */
void sr_cand_list_free(sr_cand_list* list);

/* ---------------------------------------------------------------- scoring */
typedef struct {
  int32_t match, mismatch, gap_open, gap_extend;
} sr_score_params;

/* Readout (Sec. 3.5): 0 = best cell anywhere (local alignment, default);
 * 1 = best cell of the read's final row. */
enum { SR_MODE_LOCAL = 0, SR_MODE_FINAL_ROW = 1 };
/* Engines: BATCHED = length-binned, LPT-ordered persistent kernels replayed as
 * one CUDA graph (default); PLAIN = one ordinary launch per batch over the items
 * in input order, one fixed kernel shape. */
enum { SR_ENGINE_BATCHED = 0, SR_ENGINE_PLAIN = 1 };

typedef struct {
  uint32_t mode;        /* SR_MODE_* */
  uint32_t engine;      /* SR_ENGINE_* */
  uint32_t want_cigar;  /* 1 = trace back each read's winner */
  uint32_t classify;    /* 1 = classify each read between references 0 and 1 */
  int32_t min_score;    /* classification certainty threshold (default 40) */
  int32_t margin;       /* classification score margin (default 5) */
  uint32_t force_i32;   /* 1 = use the int32 kernel for every item */
  uint32_t lanes;       /* 0 = auto; else lanes per alignment (1,2,4,8,16,32) */
  uint32_t rows;        /* 0 = auto; else read rows per lane */
  uint32_t reserved;
  void* cuda_stream;    /* cudaStream_t to run on; NULL = the library's stream */
} sr_align_opts;

/* One reported alignment.  For a read without any positive-scoring window,
 * score = 0, item = -1 and the other fields are 0. */
typedef struct {
  int32_t score;      /* best score */
  int32_t second;     /* best score at a different (ref, end, strand) */
  uint32_t n_ties;    /* distinct (ref, end, strand) reaching `score` */
  int32_t item;       /* winning window (global candidate index), -1 = none */
  uint8_t ref_id, strand;
  uint16_t reserved;
  int32_t read_start, read_end; /* 1-based on the aligned read (winner only) */
  uint64_t ref_start, ref_end;  /* 0-based inclusive on the reference */
  uint32_t cigar_off, cigar_len; /* into sr_results.cigar (winner only) */
} sr_hit;

enum { SR_CLASS_UNALIGNED = 0, SR_CLASS_A = 1, SR_CLASS_B = 2, SR_CLASS_AMBIGUOUS = 3 };

typedef struct {
  uint32_t n_reads, n_refs;
  uint64_t n_items;
  sr_hit* best;          /* n_reads: the read's winner over all references */
  sr_hit* best_per_ref;  /* n_reads * n_refs: per reference (score, second,
                            n_ties, item, strand, ref_end; no CIGAR) */
  int32_t* item_score;   /* n_items: score of every (read, window) item */
  uint32_t* item_end;    /* n_items: 1-based window column of the end cell, 0 if score 0 */
  uint32_t* cigar;       /* BAM-style words (len << 4 | op), M=0 I=1 D=2 S=4 */
  uint64_t n_cigar;
  uint8_t* read_class;   /* n_reads, SR_CLASS_* (NULL unless classified) */
  uint64_t cells;        /* DP cells of all items (sum of m*n) */
  uint64_t n_i32_items;  /* items scored by the int32 kernel */
} sr_results;

void sr_results_free(sr_results* res);

/* -------------------------------------------------------------- session
 * A session keeps the references 2-bit packed in device memory (packed by a
 * kernel) for as long as it is open.  hbm_budget bounds the device bytes the
 * session may hold for batches and serving (0 = no limit). */
typedef struct sr_session sr_session;
sr_status sr_session_open(const sr_index* const* refs, uint32_t n_refs, uint64_t hbm_budget,
                          sr_session** out);
sr_status sr_session_open_seqs(const char* const* seqs, const uint64_t* lens, uint32_t n_refs,
                               uint64_t hbm_budget, sr_session** out);
/* Closing a session stops its server; its device memory is released once the
 * last batch staged on it has been freed as well (a batch keeps its session
 * alive, so sessions and batches may be released in either order).  After
 * close, the session handle must not be passed to any call. */
void sr_session_close(sr_session* s);

/* The same CAL finder and filter on the GPU (the paper runs it on the host,
 * Sec. 4.1-4.2; here the index lives in HBM next to the references).
 * sr_session_attach_index uploads idx[r], the index of the session's reference
 * r (same length; all with one seed_len and address_bases), once; replacing an
 * attached set is allowed.  When the indexes share one hash_seed and each has
 * under 2^32 entries and at most 2^30 bases, the device copy is packed (bucket
 * starts of all references interleaved in 32 bits, keys in 16 bits when 2 *
 * (seed_len - address_bases) <= 16 and in 32 bits otherwise, position and
 * orientation in one word: 6 or 8 bytes per entry and 4 per bucket); otherwise
 * each reference's tables are copied as they are (9 bytes per entry and 8 per
 * bucket).  A packed copy of one or two references with at most 2^26 buckets and
 * at most 13 (16-bit keys) or 8 (32-bit keys) entries per bucket on average also
 * gets 64-byte bucket heads (both references' starts and counts and up to 26 or
 * 13 keys, built on the device; left out if they cannot be allocated, or with
 * SR_CAL_HEADS=0 in the environment).
 * sr_candidates_device then returns exactly the list
 * sr_candidates returns for those indexes (same windows, order and hits): one
 * warp per read looks up its seeds, one warp or block per read sorts and
 * merges its CALs, and reads of more than 8192 CALs are emitted, sorted and
 * merged by many blocks each.  The reads may be host memory or, flagged SR_FLAG_DEVICE, device
 * memory (read on the session's stream); params->flags = SR_FLAG_DEVICE leaves
 * the list in device memory (its arrays device pointers, the list flagged
 * SR_FLAG_DEVICE), so that reads, windows and the alignment stay on the device
 * (sr_align_batch takes such a list as it is).  The call's scratch (kept seed
 * lookups, 8 bytes per seed and reference, up to 1 GiB; CAL keys and window
 * arrays, 24 bytes per CAL bound, up to 64M bounds; a few words per read; for a
 * host list, the list itself, 8 bytes per read and 18 per window, built on the
 * device and copied out once through a pinned block of the session's pool)
 * stays allocated in the session for the next call and is released by
 * sr_session_close; calls on one session run one at a time.  Reads
 * longer than SR_MAX_READ_LEN or with decreasing offsets are SR_EINVAL,
 * non-ACGT bases SR_EBADBASE, no attached index SR_EINVAL.  params->n_threads
 * is unused. */
sr_status sr_session_attach_index(sr_session* s, const sr_index* const* idx, uint32_t n_refs);
sr_status sr_candidates_device(sr_session* s, const sr_reads* reads, const sr_cand_params* params,
                               sr_cand_list** out);

/* Whole batch: stage (inputs to the device), run, fetch (results to host
 * buffers).  Inputs are host memory or, flagged SR_FLAG_DEVICE, device memory
 * (then copied device to device and checked by a kernel, with the same errors).
 * Errors: SR_EINVAL (shapes, windows past the reference, read or window too
 * long, parameters), SR_EBADBASE, SR_ENOMEM, SR_ECUDA.
 * A call of 2^19 reads or more with host inputs and opts->cuda_stream NULL (batched engine)
 * runs as three batches of consecutive reads (1/10, 8/10 and 1/10 of the windows)
 * on three streams of the session, so that staging and fetching overlap the
 * other parts' compute.  The results, errors included, are those of one batch:
 * window indexes and CIGAR offsets refer to the whole call.  The CIGAR words
 * then sit in a host block of their own; sr_results_free releases both. */
sr_status sr_align_batch(sr_session* s, const sr_reads* reads, const sr_cand_list* cands,
                         const sr_score_params* sp, const sr_align_opts* opts, sr_results** out);

/* The same in three steps, so the device part can be timed and repeated with
 * inputs resident in HBM.  stage copies inputs to device buffers (no kernels);
 * run enqueues every kernel of the path on the stream (pack, work list and
 * bins, extension, per-read selection, traceback, classification) and waits
 * for it; run_async only enqueues (check with sr_batch_sync); fetch copies the
 * results back. */
typedef struct sr_batch sr_batch;
sr_status sr_batch_stage(sr_session* s, const sr_reads* reads, const sr_cand_list* cands,
                         void* cuda_stream, sr_batch** out);
sr_status sr_batch_run(sr_session* s, sr_batch* b, const sr_score_params* sp,
                       const sr_align_opts* opts);
sr_status sr_batch_run_async(sr_session* s, sr_batch* b, const sr_score_params* sp,
                             const sr_align_opts* opts);
sr_status sr_batch_sync(sr_session* s, sr_batch* b);
sr_status sr_batch_fetch(sr_session* s, sr_batch* b, sr_results** out);
void sr_batch_free(sr_batch* b);
/* Device-side statistics of the last run: kernels launched, cells, items per
 * kernel variant.  Any pointer may be NULL. */
sr_status sr_batch_stats(const sr_batch* b, uint64_t* kernels, uint64_t* cells,
                         uint64_t* i32_items, uint64_t* tasks);

/* Score-tracker report options of Sec. 4.2 for a batch that has run: per read,
 * the highest-scoring windows up to n_best (SR_REPORT_BEST_N), or every window
 * tied for the read's best score (SR_REPORT_TIED; n_best is ignored).  Windows
 * are taken in the winner order of sr_hit (score descending, then ref_id,
 * reference end, strand '+' first, candidate index); a window whose
 * (ref_id, reference end, strand) repeats that of a window already reported
 * holds the same alignment and is skipped, so a read's tied report has n_ties
 * entries.  Windows scoring 0 are never reported.  At most SR_REPORT_MAX entries
 * per read: n_best must be 1..SR_REPORT_MAX (else SR_EINVAL), and reads with more
 * tied alignments are cut at SR_REPORT_MAX and counted in n_truncated.
 * Selection, counting and compaction run on the device; the result is
 * allocated by the library and released with sr_report_free.  Fails with
 * SR_EINVAL if the batch has not run. */
enum { SR_REPORT_BEST_N = 1, SR_REPORT_TIED = 2 };
#define SR_REPORT_MAX 256u
typedef struct {
  int32_t score;
  int32_t item;       /* global candidate index */
  uint8_t ref_id, strand;
  uint16_t reserved;
  uint32_t end_col;   /* 1-based last window column of the alignment */
  uint64_t ref_end;   /* 0-based inclusive end on the reference */
} sr_report_hit;
typedef struct {
  uint32_t n_reads;
  uint32_t n_truncated;  /* reads whose tied set was cut at SR_REPORT_MAX */
  uint64_t n_hits;
  uint64_t* offsets;     /* n_reads + 1: read r's entries are hits[offsets[r] .. offsets[r+1]) */
  sr_report_hit* hits;
} sr_report;
sr_status sr_batch_report(sr_session* s, sr_batch* b, uint32_t kind, uint32_t n_best, sr_report** out);
void sr_report_free(sr_report* rep);

/* SAM 1.6 text of a batch's results (the paper's host formats its output "into
 * a standard format like SAM", Sec. 4.2).  Header: @HD, one @SQ per reference
 * (ref_lens[n_refs]), @PG.  One line per read, in read order:
 *   QNAME  read_names[r], or "r<index>"
 *   FLAG   0, 16 for a '-' strand winner (SEQ is then the reverse complement), 4 unmapped
 *   RNAME / POS  reference name (ref_names, or "ref<id>") and ref_start + 1
 *   MAPQ   0 when n_ties > 1, else 60 * (score - second) / score (at most 60)
 *   CIGAR  the winner's CIGAR (reference orientation, soft clips included)
 *   RNEXT PNEXT TLEN QUAL  * 0 0 *
 *   tags   AS:i score, XS:i second, X0:i n_ties; YC:Z class (UN/A/B/AMB) when the
 *          results carry classes; XA:Z ref,+end,score; (or -end for '-' strand)
 *          for every other window of `secondary` (an SR_REPORT_* report of the
 *          same batch; end is the 1-based last reference base; the secondary
 *          alignments carry no CIGAR).
 * Host code (parallel formatting).  Errors: SR_EINVAL (inconsistent inputs),
 * SR_EIO (file). */
typedef struct {
  const char* const* read_names;  /* n_reads names or NULL */
  const char* const* ref_names;   /* n_refs names or NULL */
  const sr_report* secondary;     /* or NULL */
} sr_sam_opts;
sr_status sr_write_sam(const sr_reads* reads, const sr_results* res, const uint64_t* ref_lens,
                       const sr_sam_opts* opts, const char* path);

/* Device time of the last run of a batch, from CUDA events recorded on the
 * launching stream (inside the replayed graph): the whole path, the extension
 * kernels alone, the traceback + CIGAR kernels.  Call after sr_batch_sync /
 * sr_batch_run.  Any pointer may be NULL. */
sr_status sr_batch_timing(const sr_batch* b, float* total_ms, float* extend_ms, float* traceback_ms);

/* Classification of each read between references 0 and 1 (Sec. 6.1, 6.2, 6.4,
 * Table 2): the reference with the higher best score wins when it leads by at
 * least `margin`; equal-enough scores are SR_CLASS_AMBIGUOUS (margin 1 = the
 * paper's exact-tie rule); a read under min_score on one reference counts for
 * the other; under min_score on both it is SR_CLASS_UNALIGNED.
 * sr_classify reads res->best_per_ref (n_reads x n_refs records, n_refs >= 2;
 * the score field of references 0 and 1) and writes n_reads SR_CLASS_* bytes
 * to class_out (caller-owned).  Either may be host memory (results from
 * sr_align_batch, sr_batch_fetch or sr_wait; pinned or not) or device memory
 * (found with cudaPointerGetAttributes); the classes are computed by a kernel
 * on the current device either way (host records are copied over first).  The
 * work runs on the per-thread default stream, which waits for the legacy
 * default stream; device records or a device class array that work on other
 * streams writes must be finished before the call.  It returns when the
 * classes are in class_out.  params NULL = defaults.  Errors: SR_EINVAL (fewer
 * than 2 references, null arrays), SR_ECUDA. */
typedef struct {
  int32_t min_score; /* default 40 */
  int32_t margin;    /* default 5; 1 = the paper's exact-tie rule */
} sr_classify_params;
sr_status sr_classify(const sr_results* res, const sr_classify_params* params, uint8_t* class_out);
/* The same for a batch that has run, from its device-resident records, with
 * other thresholds; class_out is host memory (n_reads bytes). */
sr_status sr_batch_classify(sr_session* s, sr_batch* b, const sr_classify_params* params,
                            uint8_t* class_out);

/* -------------------------------------------------------------- serving
 * Continuous batching (reads are handed to the aligners as they arrive,
 * Sec. 4.2): sr_submit copies a request and returns a ticket at once.  A
 * scheduler thread admits queued requests in arrival order while their device
 * footprint fits the session's hbm_budget, merges them into the next device
 * round (up to 131072 reads and half the budget; a single larger request runs
 * alone), stages it and
 * launches all its kernels on a stream of its own while the previous round is
 * still on the device: two rounds are in flight at once.  The new round's read
 * packing and length binning run beside the previous round's last kernels; its
 * extension kernels wait on the device for that round's last kernel.  A second
 * thread completes the rounds in order: it copies a round's results back and
 * splits them per request while the next round computes.  sr_wait blocks up to
 * timeout_ms (< 0 = forever) and returns SR_ETIMEOUT when the limit runs out.
 * A request larger than the whole budget is rejected with SR_ENOMEM.  The
 * score parameters and options of every request are the ones given to
 * sr_serve_start (opts NULL: CIGARs on, no classification; the batched engine
 * only, else SR_EINVAL; opts->cuda_stream is ignored). */
sr_status sr_serve_start(sr_session* s, const sr_score_params* sp, const sr_align_opts* opts,
                         uint32_t max_inflight_requests);
sr_status sr_submit(sr_session* s, const sr_reads* reads, const sr_cand_list* cands,
                    uint64_t* ticket);
sr_status sr_wait(sr_session* s, uint64_t ticket, int32_t timeout_ms, sr_results** out);
/* Latency of completed requests, submit to completion, in microseconds:
 * p50, p99, count; rounds run and the largest number of requests in a round. */
sr_status sr_serve_stats(sr_session* s, double* p50_us, double* p99_us, uint64_t* completed,
                         uint64_t* rounds, uint64_t* max_round_requests);
/* The same latency split by request size: bucket k holds the requests of
 * max_reads[k-1] + 1 .. max_reads[k] reads (bucket 0: 0 .. max_reads[0]);
 * bounds must increase.  p50_us, p99_us and count have n_buckets entries each
 * (any may be NULL). */
sr_status sr_serve_stats_by_size(sr_session* s, uint32_t n_buckets, const uint32_t* max_reads,
                                 double* p50_us, double* p99_us, uint64_t* count);
/* Every completed request in completion order, from index `first` on: up to
 * cap entries of latency (us, submit to completion), size (reads) and
 * completion time (s after sr_serve_start); n_out receives the number of
 * requests completed so far. */
sr_status sr_serve_latencies(sr_session* s, uint64_t first, uint32_t cap, double* us, uint32_t* reads,
                             double* done_s, uint64_t* n_out);
/* Device timeline of the completed rounds, from CUDA events the server records
 * on each round's stream: first_ms[k] when round k's first kernel finished,
 * last_ms[k] when its last kernel finished, both in ms after sr_serve_start
 * (rounds in launch order; up to cap entries written, 65536 rounds kept).
 * overlapped counts the rounds whose first kernel finished before the previous
 * round's last kernel; device_idle_ms sums, over the other consecutive pairs,
 * the time from one round's last kernel to the end of the next one's first
 * kernel (it includes the time when no request was waiting).  budget_waits
 * counts the admissions the HBM budget deferred.  Any pointer may be NULL
 * (first_ms / last_ms only when cap is 0). */
sr_status sr_serve_overlap(sr_session* s, uint64_t* timed_rounds, uint64_t* overlapped,
                           double* device_idle_ms, uint64_t* budget_waits, uint32_t cap,
                           float* first_ms, float* last_ms);
/* Stops the server after every queued request has run; results not yet taken
 * with sr_wait are freed. */
sr_status sr_serve_stop(sr_session* s);

/* ------------------------------------------------------------ autotuner
 * Measures candidate kernel shapes (lanes per alignment x rows per lane) for
 * each read-length bin on a synthetic sample of sample_reads reads (0: 4096)
 * with 6 windows each on the current GPU and keeps the fastest, unless the
 * bin's current shape is within 1.5% of it (then the current shape stays); the
 * table is used by SR_ENGINE_BATCHED.  save/load use a small text
 * file keyed by device name.  sr_tune_get writes up to cap entries of
 * (bin upper read length, lanes, rows). */
sr_status sr_tune(sr_session* s, const sr_score_params* sp, uint32_t sample_reads);
sr_status sr_tune_save(const char* path);
sr_status sr_tune_load(const char* path);
sr_status sr_tune_get(uint32_t* n_bins, uint32_t* upper, uint32_t* lanes, uint32_t* rows,
                      uint32_t cap);
sr_status sr_tune_set(uint32_t n_bins, const uint32_t* upper, const uint32_t* lanes,
                      const uint32_t* rows);

/* ------------------------------------------------ allocation-free scoring
 * No counterpart in the paper: a service entry point of this library.
 * Scores every (read, window) item whose inputs already sit in device memory
 * and writes each item's score and 1-based end column (0 when the score is 0)
 * into caller-owned device buffers, without allocating anything.  It is meant
 * for callers that cannot call cudaMalloc: a process whose device memory is
 * already held by another allocator, or a latency-sensitive caller that must
 * not pay for allocation (cudaMalloc/cudaFree can synchronize the device and
 * can fail under fragmentation).  Its scratch (work-queue counters, status
 * word, packed read rows, read lengths, item-to-read map) is a fixed
 * file-scope device array of about 3.3 MiB that every GPU loading libsr keeps
 * until the process exits; calls with more than SR_NOALLOC_MAX_READS reads or
 * SR_NOALLOC_MAX_ITEMS windows are rejected with SR_EINVAL.
 *  - Inputs: d_bases/d_read_off (CSR ASCII reads, offsets from 0), d_cand_off
 *    (n_reads + 1 window offsets from 0 ending at n_items) and the per-window
 *    d_ref_id/d_strand/d_win_start/d_win_len, all device pointers; references
 *    come from the session.  Outputs: d_item_score, d_item_end (n_items each).
 *  - Scores must fit the packed 16-bit kernel (match + gap_open + 2*gap_extend
 *    small, match * 256 <= 31743); otherwise SR_EINVAL (use sr_align_batch).
 *  - Runs on cuda_stream (NULL = default stream) and returns when the work is
 *    done; bad offsets, reads or windows give SR_EINVAL / SR_EBADBASE.  The
 *    current device must be the one the session was opened on (else SR_EINVAL).
 *  - The first call on a device looks up the scratch array's device address
 *    with that device current; make that first call before any stream capture.
 *  - All calls share the one scratch array: calls whose work overlaps on the
 *    GPU (two host threads, or two streams) race on it. */
#define SR_NOALLOC_MAX_READS 32768u
#define SR_NOALLOC_MAX_ITEMS 262144u
sr_status sr_align_items_noalloc(sr_session* s, const char* d_bases, const uint64_t* d_read_off,
                                 uint32_t n_reads, const uint64_t* d_cand_off,
                                 const uint8_t* d_ref_id, const uint8_t* d_strand,
                                 const uint64_t* d_win_start, const uint32_t* d_win_len,
                                 uint64_t n_items, const sr_score_params* sp,
                                 int32_t* d_item_score, uint32_t* d_item_end, void* cuda_stream);

/* ------------------------------------------------------- measurement
 * Issue-rate probe of the packed 16-bit DPX max/add-max instructions: returns
 * lane-operations per clock per SM measured with CUDA events (and the clock
 * attribute), used as the integer roofline denominator. */
sr_status sr_probe_dpx(double* lane_ops_per_clk_per_sm, double* sm_clock_mhz);

/* Check of the bounded device waits (no counterpart in the paper).  The
 * extension kernels wait for their window copies on an mbarrier for a bounded
 * number of polls, after which they record a timeout in the batch's status word
 * and return (the batch then fails with SR_ETIMEOUT).  This probe runs that
 * polling on a barrier that receives its arrival (arrive != 0: SR_OK) or never
 * does (arrive == 0: SR_ETIMEOUT after poll_limit polls, 1..2^24, else
 * SR_EINVAL); the context stays usable either way. */
sr_status sr_probe_wait(uint32_t poll_limit, uint32_t arrive);

#ifdef __cplusplus
}
#endif
#endif /* SR_H */
