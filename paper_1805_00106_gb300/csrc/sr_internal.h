// sr_internal.h -- device data layout and kernel launchers shared inside libsr.
//
// Layout in HBM (all buffers 256-byte aligned by cudaMalloc):
//   reference k : uint32 words, 16 bases per word, base p in bits 2*(p&15)..+1 of
//                 word p>>4 (A=0 C=1 G=2 T=3, Sec. 3.1 Fig. 3 codes), followed by
//                 >= 64 bytes of padding so 16-byte TMA copies of any window stay
//                 inside the allocation;
//   reads       : one 64-byte row per read (16 words = 256 bases), same packing;
//   items       : one per (read, window) candidate, structure of arrays indexed
//                 by the global candidate index.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sr.h"

namespace sr {

constexpr int kMaxReadLen = 256;
constexpr int kMaxWinLen = 512;
constexpr int kMaxRefs = 16;
constexpr int kReadWords = 16;     // words per packed read row
constexpr int kCigarStride = 776;  // CIGAR words reserved per read (>= 3*256 + 4 runs)
static_assert(kMaxReadLen == SR_MAX_READ_LEN && kMaxWinLen == SR_MAX_WIN_LEN && kMaxRefs == SR_MAX_REFS &&
                  kCigarStride == SR_CIGAR_STRIDE && kReadWords * 16 == kMaxReadLen,
              "device limits agree with the public header");
constexpr int kNumBins = 23;       // read-length bins of the batched engine (8-row steps above 96)
constexpr int kNumClasses = kNumBins + 1;  // + the int32 class
constexpr int kI32Class = kNumBins;
constexpr int kKeysPerClass = kMaxWinLen;  // sort key = class*512 + (512 - n)
constexpr int kNumKeys = kNumClasses * kKeysPerClass;
constexpr int kBias = 1024;        // bias of packed 16-bit DP values (keeps halves >= 0)

// status word bits (device -> host)
enum : uint32_t {
  kStBadBase = 1u << 0,
  kStBadRead = 1u << 1,    // read length 0 or > kMaxReadLen
  kStBadWindow = 1u << 2,  // window outside its reference / bad ref id / length
  kStTimeout = 1u << 3,    // a bounded wait (TMA mbarrier) ran out
  kStOverflow = 1u << 4,   // int16 guard tripped (never expected: routing is exact)
  kStInternal = 1u << 5,
};

struct DevRefs {
  const uint32_t* words[kMaxRefs];
  uint64_t len[kMaxRefs];
  int n;
};

struct ScoreConst {
  int32_t sa, sb, go, ge;
};

// per-read result slot (device); index read * (1 + n_refs) + (0 = overall, 1 + r = ref r)
struct DevHit {
  int32_t score, second;
  uint32_t n_ties;
  int32_t item;
  int32_t read_start, read_end;  // winner only (1-based rows of the aligned read)
  uint32_t start_j, cigar_len;   // winner only: 1-based first window column, CIGAR words
};

struct BatchDev {
  // staged inputs
  const char* bases = nullptr;
  const uint64_t* read_off = nullptr;
  const uint64_t* cand_off = nullptr;
  const uint8_t* c_ref = nullptr;
  const uint8_t* c_strand = nullptr;
  const uint64_t* c_start = nullptr;
  const uint32_t* c_len = nullptr;
  uint32_t n_reads = 0;
  uint64_t n_items = 0;
  // derived
  uint32_t* rpack = nullptr;      // n_reads * 16
  uint32_t* rlen = nullptr;       // n_reads
  uint32_t* item_read = nullptr;  // n_items
  uint16_t* item_key = nullptr;   // n_items
  uint32_t* order = nullptr;      // n_items, sorted by key
  uint32_t* hist = nullptr;       // kNumKeys
  uint32_t* cursor = nullptr;     // kNumKeys
  uint32_t* class_range = nullptr;  // 2 * kNumClasses
  uint32_t* queue = nullptr;      // kNumClasses + 8 counters
  unsigned long long* cells = nullptr;  // 1 counter
  uint32_t* status = nullptr;     // 1 word
  // outputs
  int32_t* item_score = nullptr;
  uint32_t* item_end = nullptr;
  DevHit* hits = nullptr;         // n_reads * (1 + n_refs)
  uint32_t* cigar_slots = nullptr;  // n_reads * kCigarStride
  uint32_t* item_iend = nullptr;  // n_items: end row of winning items (traceback)
  uint32_t* wcount = nullptr;     // kNumClasses: winners per class
  uint32_t* wrange = nullptr;     // 2 * kNumClasses: winner ranges in `order`
  uint32_t* wqueue = nullptr;     // kNumClasses + 8: winner-pass task counters
  uint8_t* tb_flag = nullptr;     // n_reads: how the winner's end row is found (kTbFlag*)
  uint32_t* tb_list = nullptr;    // 2 * n_reads: per-read sort code, then reads sorted by code
  uint32_t* tb_count = nullptr;   // kTbCountWords: code histogram, cursors, bucket ranges
  uint32_t* tb_dirs = nullptr;    // tb_dirs_words(n_reads): narrow-band direction words
  uint32_t* tb_dirs32 = nullptr;  // tb_dirs32_words(n_reads): direction words of 17-32-diagonal bands
  uint32_t* cigar_off = nullptr;  // n_reads + 1 (exclusive scan of lengths)
  uint32_t* cigar = nullptr;      // compacted, n_reads * kCigarStride capacity
  uint8_t* read_class = nullptr;  // n_reads
  uint32_t* scan_tmp = nullptr;   // block sums for scans
  sr_hit* out_best = nullptr;     // n_reads: results in the public layout (fetch)
  sr_hit* out_per_ref = nullptr;  // n_reads * n_refs
  void* check = nullptr;          // staging checks of device inputs (a StageCheck)
};

// traceback routing.  A winner's end row i* is searched inside the band
// (kTbFlagBand), comes from the extension kernels' winner mode (kTbFlagRow:
// the band over every possible end row would be wider than 64 diagonals), or is
// found by the full-rectangle kernel (kTbFlagFull: int32-class winners).
enum : uint8_t { kTbFlagBand = 0, kTbFlagFull = 1, kTbFlagRow = 2 };
constexpr int kTbBuckets = 8;                        // band <= 1 / 2 / 4 / 8 / 16 / 32 / 64 diagonals, full
constexpr int kTbCodes = kTbBuckets * kMaxReadLen;   // code = bucket * 256 + (256 - last row)
constexpr int kTbCountWords = 2 * kTbCodes + 2 * kTbBuckets + 8;
constexpr int kTbMaxBand = 64;
// warps of the one-thread-per-read narrow-band traceback (each owns a scratch
// of 256 rows x 32 lanes of direction words): 152 SMs x 32, its register-bound
// residency on GB300
constexpr uint32_t kTbThreadMaxWarps = 4864;
inline uint32_t tb_thread_warps(uint32_t n_reads) {
  const uint32_t w = (n_reads + 31u) / 32u;
  return w < kTbThreadMaxWarps ? (w ? w : 1u) : kTbThreadMaxWarps;
}
// warps of the two-reads-per-thread traceback for bands of at most 16 diagonals
// (64 reads per warp; each owns a scratch of 256 rows x 4 words x 32 lanes):
// 152 SMs x 24, its residency on GB300
constexpr uint32_t kTbPairMaxWarps = 3648;
constexpr uint64_t kTbPairWarpWords = 256ull * 4 * 32;
inline uint32_t tb_pair_warps(uint32_t n_reads) {
  const uint32_t w = (n_reads + 63u) / 64u;
  return w < kTbPairMaxWarps ? (w ? w : 1u) : kTbPairMaxWarps;
}
// warps of its 32-cell variant (bands of 17-32 diagonals: a few percent of
// short reads, more of long ones; warps for up to half of the batch's reads,
// more take more rounds, each a latency-bound pass; each warp owns 256 rows x 8
// words x 32 lanes)
constexpr uint32_t kTbPair32MaxWarps = 2432;  // 152 SMs x 16, its residency on GB300
constexpr uint64_t kTbPair32WarpWords = 256ull * 8 * 32;
inline uint32_t tb_pair32_warps(uint32_t n_reads) {
  const uint32_t w = (n_reads + 127u) / 128u;
  return w < kTbPair32MaxWarps ? (w ? w : 1u) : kTbPair32MaxWarps;
}
inline uint64_t tb_dirs32_words(uint32_t n_reads) {
  return static_cast<uint64_t>(tb_pair32_warps(n_reads)) * kTbPair32WarpWords;
}
// the narrow-band scratch serves whichever of the two kernels runs
inline uint64_t tb_dirs_words(uint32_t n_reads) {
  const uint64_t a = static_cast<uint64_t>(tb_thread_warps(n_reads)) * 256 * 32;
  const uint64_t b = static_cast<uint64_t>(tb_pair_warps(n_reads)) * kTbPairWarpWords;
  return a > b ? a : b;
}

// Diagonal band of a winner (score S >= 1 ending in column j*) whose end row lies
// in [ilo, ihi]: every alignment of score S ending at (i, j*) has at most
// g(i) = (sa * min(i, j*) - S - go) / ge gap bases (each gap run costs go plus ge
// per base and at most min(i, j*) bases can match), so it stays within the
// diagonals j - i in [j* - ihi - g(ihi), j* - ilo + g(ihi)] (g grows with i).
struct TbBand {
  int ilo, ihi, g, w, dlo;
};
#ifdef __CUDACC__
__host__ __device__ inline TbBand tb_band(int32_t sa, int32_t go, int32_t ge, int32_t S, uint32_t jstar,
                                          uint32_t ilo, uint32_t ihi) {
  // g(i): the most gap bases an alignment of score S ending in (i, j*) can
  // hold; it lies in diagonals j* - i - g(i) .. j* - i + g(i).  The band is the
  // union over the end rows ilo..ihi.  Its lower end is row ihi's.  On the upper
  // end, j* - i + g(i) falls while g = 0, is monotone while g > 0 and i <= j*,
  // and falls again past j*, so its maximum is at ilo or at an end of the middle
  // piece.
  const int64_t J = jstar, lo = ilo, hi = ihi;
  auto g = [&](int64_t i) -> int64_t {
    const int64_t v = (static_cast<int64_t>(sa) * (i < J ? i : J) - S - go) / ge;
    return v > 0 ? v : 0;
  };
  auto f = [&](int64_t i) { return J - i + g(i); };
  const int64_t i1 = (static_cast<int64_t>(S) + go + ge + sa - 1) / sa;  // first row with g > 0 (below j*)
  int64_t up = f(lo);
  if (i1 > lo && i1 <= hi) up = f(i1) > up ? f(i1) : up;
  if (J >= lo && J <= hi) up = f(J) > up ? f(J) : up;
  if (J + 1 > lo && J + 1 <= hi) up = f(J + 1) > up ? f(J + 1) : up;
  up = f(hi) > up ? f(hi) : up;
  TbBand b;
  b.ilo = static_cast<int>(ilo);
  b.ihi = static_cast<int>(ihi);
  b.g = static_cast<int>(g(hi));
  b.dlo = static_cast<int>(J - hi - b.g);
  b.w = static_cast<int>(up - b.dlo + 1);
  return b;
}
// smallest row that can end an alignment of score S (S <= sa * i)
__host__ __device__ inline uint32_t tb_min_row(int32_t sa, int32_t S) {
  return static_cast<uint32_t>((S + sa - 1) / sa);
}
#endif

// Independent kernels of one phase (the length bins, the traceback buckets)
// run on side streams forked from the launching stream and joined back, so a
// bin's tail overlaps the next bins and small batches do not pay the bins'
// latencies one after another.  Events: one fork and kSide joins per phase.
// Small batches spread over all kSide streams (latency); large ones over four,
// where more concurrent kernels only contend.
constexpr int kSide = 8;
inline int fan_width(uint32_t n_reads) { return n_reads >= (1u << 18) ? 4 : kSide; }
struct Fanout {
  cudaStream_t side[kSide];
  cudaEvent_t fork;
  cudaEvent_t join[kSide];
};
// record the fork on st and make every side stream wait for it
int fanout_begin(const Fanout& f, cudaStream_t st);
// make st wait for everything enqueued on the side streams
int fanout_end(const Fanout& f, cudaStream_t st);

struct TuneBin {
  uint32_t upper;  // largest read length in the bin
  uint32_t lanes;  // G: lanes per alignment (power of two)
  uint32_t rows;   // R: read rows per lane
};

// launchers (each returns the number of kernels it enqueued, or -1 on error)
int launch_pack_refs(const char* ascii, uint64_t len, uint32_t* words, uint32_t* status,
                     cudaStream_t st);
int launch_prepare(const BatchDev& b, const DevRefs& refs, cudaStream_t st);
int launch_bins(const BatchDev& b, const ScoreConst& sc, const TuneBin* bins, int n_bins,
                bool force_i32, bool plain, cudaStream_t st);
// class_items: items per length class (host; nullptr = launch every class);
// fan: side streams for the per-class kernels (nullptr = all on st)
int launch_extend(const BatchDev& b, const DevRefs& refs, const ScoreConst& sc,
                  const TuneBin* bins, int n_bins, int mode, bool plain, uint32_t lanes,
                  uint32_t rows, cudaStream_t st, const uint64_t* class_items = nullptr,
                  const Fanout* fan = nullptr);
int launch_select(const BatchDev& b, int n_refs, cudaStream_t st);
int launch_winners(const BatchDev& b, const ScoreConst& sc, int mode, int n_refs, bool plain,
                   cudaStream_t st);
// end rows of the winners compacted by k_winners: one launch (lanes x rows, 0 = 16 x 16)
int launch_winner_rows(const BatchDev& b, const DevRefs& refs, const ScoreConst& sc, uint32_t lanes,
                       uint32_t rows, cudaStream_t st);
int launch_traceback(const BatchDev& b, const DevRefs& refs, const ScoreConst& sc, int mode,
                     int n_refs, cudaStream_t st, const Fanout* fan = nullptr);
int launch_cigar_compact(const BatchDev& b, int n_refs, cudaStream_t st);
// records in the public layout; a batch holding one part of a larger result
// adds item_base to its window indexes and cigar_base to its CIGAR offsets
int launch_assemble(const BatchDev& b, int n_refs, bool want_cigar, int32_t item_base, uint32_t cigar_base,
                    cudaStream_t st);
// checks of a batch whose inputs were staged from device memory
struct StageCheck {
  unsigned long long cells;
  unsigned long long bad;      // (read << 3) | reason of the first bad read, ~0 if none
                               // (1 offsets, 2 read length, 3 window count, 4 a window)
  unsigned long long bad_win;  // the first bad window of that read (reason 4), ~0 if none
  uint32_t max_m;
  uint32_t pad;
  unsigned long long by_len[kMaxReadLen + 1];  // windows per read length
};
int launch_stage_check(const BatchDev& b, const DevRefs& refs, StageCheck* out, cudaStream_t st);
int launch_first_bad_window(const BatchDev& b, const DevRefs& refs, uint32_t read, StageCheck* out,
                            cudaStream_t st);
// off[0..n) -= base
int launch_rebase_offsets(uint64_t* off, uint64_t n, uint64_t base, cudaStream_t st);
// exclusive scan of n counts into out[0..n] (out[n] = total) with a scratch of
// n / 1024 + 1 words (sr_report.cu)
int launch_scan_u32(const uint32_t* in, uint32_t n, uint32_t* out, uint32_t* sums, cudaStream_t st);

// device copy of the host index of each reference (sr_cal.cu, Sec. 3.1-3.3)
struct DevIndex {
  const uint64_t* ptr[kMaxRefs];
  const uint32_t* key[kMaxRefs];
  const uint32_t* pos[kMaxRefs];
  const uint8_t* orient[kMaxRefs];
  // packed form (packed = 1; ptr, pos and orient unset): the bucket starts of
  // all references interleaved as 32-bit values, jptr[b * n_refs + r], so that
  // one sector holds a seed's bucket in every reference; 16-bit keys in key16
  // when they fit (2 (k - a) <= 16, key_bits 16), else 32-bit ones in key
  // (key_bits 32); each entry's position with its orientation bits in the top
  // two (posor), one load per entry.  Used when the references share one hash
  // seed and each has under 2^32 entries and at most 2^30 bases.
  const uint32_t* jptr;
  const uint16_t* key16[kMaxRefs];
  const uint32_t* posor[kMaxRefs];
  int packed, key_bits;
  // bucket heads (packed form, one or two references; nullptr otherwise): 64
  // bytes per bucket, read with one access: its first entry in references 0 and
  // 1 (words 0, 1), their entry counts (word 2, 16 bits each) and up to
  // kHeadKeys 16-bit keys (two per word, low half first) or kHeadKeys32 32-bit
  // ones, reference 0's then reference 1's in entry order (words 3-15).  Word 2
  // is kHeadSpill where they do not fit: that bucket is looked up in jptr and
  // the keys.
  const uint4* heads;
  uint64_t ref_len[kMaxRefs];
  uint64_t hash_seed[kMaxRefs];
  int n_refs, k, a;
};
constexpr uint32_t kCalSmallKeys = 1024;  // reads up to this many CALs: small-block filter (24 KB)
constexpr uint32_t kCalSmemKeys = 8192;   // up to this many: filtered in shared memory (192 KB)
// shared or scratch words (u64) the filter of a read of up to P CALs uses (P a
// power of two): its keys, each window's best run, run and window start positions
__host__ __device__ constexpr uint64_t cal_filter_words(uint64_t P) { return 3 * P + 1; }
// count pass (cals == nullptr: an upper bound of the CALs of each read into
// count, exact unless a seed is its own reverse complement; reads with bad
// offsets or over kMaxReadLen bases set kStBadRead) or emit pass (CAL keys of
// read r0 + i into cals[off[i] ...], their number into actual[i]) over reads
// r0 .. r0 + nr
// Seed lookups the count pass keeps for the emit pass: records start at
// seed_off[r - rbase] for read r (seeds x references of it, from
// launch_cal_slots); recount[r - rbase] = 1 where they could not be kept
struct CalRanges {
  uint64_t* ranges = nullptr;
  const uint32_t* seed_off = nullptr;
  uint8_t* recount = nullptr;
  uint32_t rbase = 0;
};
constexpr int kHeadKeys = 26;
constexpr int kHeadKeys32 = 13;
constexpr uint32_t kHeadSpill = 0xffffffffu;
// the bucket heads of a packed index (nbuckets buckets, n_refs <= 2) into heads
int launch_cal_heads(const DevIndex& di, uint64_t nbuckets, uint4* heads, cudaStream_t st);
// Emit pass of the large reads (device list big, n_big of them: over
// kCalSmemKeys CAL bounds) whose lookups were kept, by many blocks per read,
// after launch_cal_seeds' emit pass (given the bounds as count, it leaves those
// reads out); its part tables take cal_sort_words(n_big) words after the
// filter's scratch_words
int launch_cal_emit_big(const DevIndex& di, const uint64_t* read_off, uint32_t r0, uint32_t nr, uint32_t stride,
                        const uint32_t* bound, const uint64_t* off, uint64_t* cals, const CalRanges& kept,
                        const uint32_t* big, uint32_t n_big, uint64_t* scratch, uint64_t scratch_words,
                        cudaStream_t st);
int launch_cal_seeds(const DevIndex& di, const char* bases, const uint64_t* read_off, uint32_t r0, uint32_t nr,
                     uint32_t stride, uint32_t* count, const uint64_t* off, uint64_t* cals, uint32_t* actual,
                     uint32_t* status, const CalRanges& kept, cudaStream_t st);
// lookup records of each of n reads (seeds x n_refs); bad offsets or reads
// over kMaxReadLen bases set kStBadRead
int launch_cal_slots(const uint64_t* read_off, uint32_t n, int k, uint32_t stride, int n_refs, uint32_t* slots,
                     uint32_t* status, cudaStream_t st);
// windows of each read at off[i] (nwin[i] of them).  Reads with up to
// kCalSmallKeys CALs (largest: max_small) and up to kCalSmemKeys (largest:
// max_mid, 0 = none) sort in shared memory; the n_big others (device list big
// of indices into the chunk) sort in scratch from slot big_soff[b] (pow2 of
// their count each, scratch_words in all), followed by
// cal_sort_words(n_big, scratch_words) words of the large-read tables
int launch_cal_filter(const DevIndex& di, const uint64_t* read_off, uint32_t r0, uint32_t nr, uint32_t merge_dist,
                      uint32_t pad, uint32_t max_cands, const uint32_t* count, const uint32_t* actual,
                      const uint64_t* off, uint64_t* cals, uint32_t max_small, uint32_t max_mid, const uint32_t* big,
                      const uint64_t* big_soff, uint32_t n_big, uint64_t* scratch, uint64_t scratch_words,
                      uint32_t* nwin, uint64_t* wkey, uint32_t* whits, uint32_t* wlen, cudaStream_t st);
// keys per tile of the large-read sort and merge
constexpr uint32_t kCalSortTile = 4096;
// words after a filter's scratch (scratch_words) for the tables of the
// large-read emit (the reads' chunk counts, their prefix and its block sums)
// and, later, of the large-read sort and merge (class counts and fills, the
// reads in class order; run and window starts per tile, their prefixes and
// block sums, for at most scratch_words / (3 kCalSortTile) + 1 tiles)
constexpr uint64_t cal_sort_words(uint64_t n_big, uint64_t scratch_words) {
  const uint64_t nt = scratch_words / (3ull * kCalSortTile) + 1;
  const uint64_t emit = (n_big + 1) / 2 + 1 + (n_big + 1) + n_big / 1024 + 2;
  const uint64_t merge = 20 + (n_big + 1) / 2 + 1 + nt + 2 * (nt + 1) + nt / 1024 + 2;
  return (emit > merge ? emit : merge) + 8;
}
// out[i] = base + woff[i] for i = 0 .. nr (a chunk's window offsets in the whole list)
int launch_cal_offsets(const uint32_t* woff, uint32_t nr, uint64_t base, uint64_t* out, cudaStream_t st);
// exclusive 64-bit scan of n counts into out[0..n] (out[n] = the total) with a
// scratch of n / 1024 + 1 words (sr_cal.cu)
int launch_scan_u64(const uint32_t* in, uint32_t n, uint64_t* out, uint64_t* sums, cudaStream_t st);
// The CAL filter's routing of nr reads by their CAL bounds: reads over
// kCalSmemKeys CALs listed in big (indices into the reads, in any order) with
// their scratch offsets in big_soff, and the largest small, mid-size and
// overall bound; big = nullptr takes the maxima only.  plan must be zeroed.
struct CalPlan {
  unsigned long long scratch;  // scratch words of the listed large reads
  unsigned int n_big, max_small, max_mid, max_all;
};
int launch_cal_route(const uint32_t* count, uint32_t nr, uint32_t* big, uint64_t* big_soff, CalPlan* plan,
                     cudaStream_t st);
// cuts of a prefix sum pre[0..nr) into pieces of span: bounds[j] = the first
// index whose prefix lies in [j span, (j + 1) span) (every j up to
// pre[nr - 1] / span has one when no single count reaches span)
int launch_cal_bounds(const uint64_t* pre, uint32_t nr, uint64_t span, uint32_t* bounds, cudaStream_t st);
// a piece's prefix sums from 0: out[i] = pre[a + i] - pre[a] for i = 0 .. cnt
// into out64 or, when it is nullptr, out32
int launch_cal_rebase(const uint64_t* pre, uint32_t a, uint32_t cnt, uint64_t* out64, uint32_t* out32,
                      cudaStream_t st);
int launch_cal_compact(uint32_t nr, const uint64_t* off, const uint32_t* nwin, const uint32_t* woff,
                       const uint64_t* wkey, const uint32_t* whits, const uint32_t* wlen, uint8_t* o_ref,
                       uint8_t* o_strand, uint64_t* o_start, uint32_t* o_len, uint32_t* o_hits, cudaStream_t st);

// report options (sr_report.cu): count pass + scan into a scratch of
// report_scratch_words(n_reads) words, then the write pass
uint64_t report_scratch_words(uint32_t n_reads);
int launch_report_count(const BatchDev& b, int n_refs, int kind, uint32_t n_best, uint32_t* scratch,
                        cudaStream_t st);
int launch_report_write(const BatchDev& b, int n_refs, int kind, uint32_t n_best, const uint32_t* scratch,
                        sr_report_hit* out, cudaStream_t st);
int launch_classify(const BatchDev& b, int n_refs, int32_t min_score, int32_t margin,
                    cudaStream_t st);
// the same on public records in device memory: per_ref holds n_reads * n_refs
// sr_hit (n_refs >= 2), classes of references 0 and 1 into out[n_reads]
int launch_classify_hits(const sr_hit* per_ref, uint32_t n_reads, uint32_t n_refs, int32_t min_score,
                         int32_t margin, uint8_t* out, cudaStream_t st);
bool extend_config_supported(uint32_t lanes, uint32_t rows);
// the built (lanes, rows) shapes; returns how many there are
int extend_shapes(uint32_t* lanes, uint32_t* rows, int cap);
// Loading every kernel of the library at session open (cudaFuncGetAttributes
// loads a kernel's module): with lazy module loading the first launch of a
// rarely used kernel (the winner end-row pass, the int32 path, a selection
// width) would otherwise stall the host in the middle of enqueuing a batch.
// One per source file; each returns the number of kernels touched.
int preload_mode0();
int preload_mode1();
int preload_mode2();
int preload_extend();
int preload_kernels();
int preload_traceback();
int preload_cal();
int preload_report();
int preload_noalloc();
#define SR_TOUCH(k)                                                             \
  do {                                                                          \
    cudaFuncAttributes fa_;                                                     \
    if (cudaFuncGetAttributes(&fa_, reinterpret_cast<const void*>(&(k))) == cudaSuccess) ++n_; \
  } while (0)
int probe_dpx(double* lane_ops_per_clk_per_sm, double* clk_mhz);
// bounded mbarrier wait with (arrive = 1) or without its arrival; status word out
int probe_wait(uint32_t poll_limit, int arrive, uint32_t* status_out);

}  // namespace sr
