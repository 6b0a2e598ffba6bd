// sr_kernels.cu -- the non-DP kernels of the path: 2-bit packing (Sec. 3.1,
// Fig. 3), work list + length bins, per-read score tracker (Sec. 3.6, 4.2),
// classification (Sec. 6.1-6.4) and CIGAR compaction.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xffffffffu;

// ASCII -> 2-bit code (A=0 C=1 G=2 T=3, either case); returns 4 for anything else
__device__ __forceinline__ uint32_t ascii_code(uint32_t ch) {
  const uint32_t c = ch | 0x20u;
  const bool ok = c == 'a' || c == 'c' || c == 'g' || c == 't';
  return ok ? (((c >> 1) ^ (c >> 2)) & 3u) : 4u;
}

// one thread per 16-base word of the reference; `words` has room for the padding
__global__ void k_pack_ref(const char* ascii, uint64_t len, uint64_t n_words_alloc, uint32_t* words,
                           uint32_t* status) {
  for (uint64_t w = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; w < n_words_alloc;
       w += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    uint32_t v = 0;
    bool bad = false;
    const uint64_t p0 = w * 16;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      if (p0 + b < len) {
        uint32_t c = ascii_code(static_cast<uint8_t>(ascii[p0 + b]));
        bad |= c > 3u;
        v |= (c & 3u) << (2 * b);
      }
    }
    words[w] = v;
    if (bad) atomicOr(status, kStBadBase);
  }
}

// 16 threads per read, one packed word each; validates length and bases
__global__ void k_pack_reads(const char* bases, const uint64_t* off, uint32_t n_reads,
                             uint32_t* rpack, uint32_t* rlen, uint32_t* status) {
  const uint64_t gt = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const uint64_t r = gt >> 4;
  const uint32_t w = static_cast<uint32_t>(gt & 15u);
  if (r >= n_reads) return;
  const uint64_t o0 = off[r], o1 = off[r + 1];
  const uint64_t m = o1 - o0;
  const bool len_ok = o1 > o0 && m <= static_cast<uint64_t>(kMaxReadLen);
  uint32_t v = 0;
  bool bad = false;
  if (len_ok && 16u * w < m) {
    // this word's bases as aligned 32-bit loads (an aligned word holding a valid
    // byte never crosses a page), realigned by a funnel shift
    const uint32_t nv = static_cast<uint32_t>(m - 16u * w < 16u ? m - 16u * w : 16u);  // valid bases
    const uintptr_t at = reinterpret_cast<uintptr_t>(bases + o0 + 16u * w);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(at & ~static_cast<uintptr_t>(3));
    const uint32_t lead = static_cast<uint32_t>(at & 3u);
    uint32_t x[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) x[k] = 4u * k < lead + nv ? src[k] : 0u;
    // four bases at a time: per byte the code of ascii_code (((c >> 1) ^ (c >> 2)) & 3
    // of the lower-cased byte; bits shifted in from the next byte are masked
    // off), checked by looking the code's letter up again and comparing
    uint32_t diff = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t y = __funnelshift_r(x[k], x[k + 1], 8u * lead);
      const int left = static_cast<int>(nv) - 4 * k;  // valid bytes of y: min(max(left, 0), 4)
      const uint32_t keep = left >= 4 ? 0xffffffffu : (left <= 0 ? 0u : (1u << (8 * left)) - 1u);
      const uint32_t c = y | 0x20202020u;
      const uint32_t code = ((c >> 1) ^ (c >> 2)) & 0x03030303u & keep;
      const uint32_t t = code | (code >> 4);                       // codes as nibbles 0..3
      const uint32_t letters = __byte_perm(0x74676361u, 0u, (t & 0xffu) | ((t >> 8) & 0xff00u));
      diff |= (c ^ letters) & keep;                                // 'a' 'c' 'g' 't'
      const uint32_t u = code | (code >> 6);                       // codes as 2-bit fields
      v |= ((u & 0xfu) | ((u >> 12) & 0xf0u)) << (8 * k);
    }
    bad = diff != 0;
  }
  rpack[r * kReadWords + w] = v;
  if (w == 0) {
    rlen[r] = len_ok ? static_cast<uint32_t>(m) : 0u;
    if (!len_ok) atomicOr(status, kStBadRead);
  }
  if (bad) atomicOr(status, kStBadBase);
}

// eight lanes per read: item -> read map and window validation
__global__ void k_items(const uint64_t* cand_off, uint32_t n_reads, const uint8_t* c_ref,
                        const uint8_t* c_strand, const uint64_t* c_start, const uint32_t* c_len,
                        DevRefs refs, uint32_t* item_read, uint32_t* status) {
  const uint64_t r = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 3;
  const int lane = threadIdx.x & 7;
  if (r >= n_reads) return;
  const uint64_t c0 = cand_off[r], c1 = cand_off[r + 1];
  bool bad = c1 < c0;
  for (uint64_t c = c0 + lane; c < c1 && !bad; c += 8) {
    item_read[c] = static_cast<uint32_t>(r);
    const uint32_t k = c_ref[c];
    const uint32_t n = c_len[c];
    bool ok = k < static_cast<uint32_t>(refs.n) && c_strand[c] <= 1u && n >= 1u &&
              n <= static_cast<uint32_t>(kMaxWinLen);
    if (ok) ok = c_start[c] + n <= refs.len[k];
    bad |= !ok;
  }
  if (bad) atomicOr(status, kStBadWindow);
}

struct BinArgs {
  uint8_t cls_of_len[kMaxReadLen + 1];  // read length -> class (kI32Class for int32 items)
};

// sort key per item: class * 512 + (512 - n); shared-memory histogram
__global__ void k_keys(const uint32_t* item_read, const uint32_t* rlen, const uint32_t* c_len,
                       uint64_t n_items, BinArgs ba, uint16_t* item_key, uint32_t* hist) {
  __shared__ uint32_t sh[kNumKeys];
  for (int k = threadIdx.x; k < kNumKeys; k += blockDim.x) sh[k] = 0;
  __syncthreads();
  for (uint64_t c = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; c < n_items;
       c += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t m = min(rlen[item_read[c]], static_cast<uint32_t>(kMaxReadLen));
    const uint32_t n = min(max(c_len[c], 1u), static_cast<uint32_t>(kMaxWinLen));
    const uint32_t key = static_cast<uint32_t>(ba.cls_of_len[m]) * kKeysPerClass + (kMaxWinLen - n);
    item_key[c] = static_cast<uint16_t>(key);
    atomicAdd(&sh[key], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kNumKeys; k += blockDim.x)
    if (sh[k]) atomicAdd(&hist[k], sh[k]);
}

// one block: exclusive scan of the histogram -> cursor, class ranges
__global__ void k_scan_keys(const uint32_t* hist, uint32_t* cursor, uint32_t* class_range) {
  __shared__ uint32_t part[1024];
  constexpr int per = (kNumKeys + 1023) / 1024;
  const int t = threadIdx.x;
  uint32_t loc[per];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < per; ++i) {
    const int k = t * per + i;
    loc[i] = k < kNumKeys ? hist[k] : 0u;
    sum += loc[i];
  }
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    uint32_t v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = part[t] - sum;
#pragma unroll
  for (int i = 0; i < per; ++i) {
    const int k = t * per + i;
    if (k < kNumKeys) {
      cursor[k] = run;
      if (k % kKeysPerClass == 0) class_range[2 * (k / kKeysPerClass)] = run;
      if (k % kKeysPerClass == kKeysPerClass - 1) class_range[2 * (k / kKeysPerClass) + 1] = run + loc[i];
    }
    run += loc[i];
  }
}

// scatter items into key order; warp-aggregated atomics per equal key
__global__ void k_scatter(const uint16_t* item_key, uint64_t n_items, uint32_t* cursor,
                          uint32_t* order) {
  const uint64_t c = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const bool live = c < n_items;
  const uint32_t key = live ? item_key[c] : 0xffffffffu;
  const uint32_t act = __ballot_sync(FULL, live);
  if (!live) return;
  const uint32_t peers = __match_any_sync(act, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&cursor[key], static_cast<uint32_t>(__popc(peers)));
  base = __shfl_sync(peers, base, leader);
  const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
  order[base + rank] = static_cast<uint32_t>(c);
}

// ---- per-read tracker (Sec. 3.6, 4.2): winner, second best, ties, per reference

// G lanes per read (a group; two reads per warp for G = 16)
template <int G>
__device__ __forceinline__ unsigned long long gmin64(uint32_t gm, unsigned long long v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    unsigned long long x = __shfl_xor_sync(gm, v, o, G);
    v = x < v ? x : v;
  }
  return v;
}

template <int G>
__global__ void k_select(const uint64_t* cand_off, uint32_t n_reads, const int32_t* item_score,
                         const uint32_t* item_end, const uint8_t* c_ref, const uint8_t* c_strand,
                         const uint64_t* c_start, int n_refs, DevHit* hits) {
  static_assert(G == 4 || G == 8 || G == 16 || G == 32, "groups of 4, 8, 16 or 32 lanes");
  const uint64_t r = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) / G;
  const int wl = threadIdx.x & 31;                       // lane in the warp
  const int l = wl % G;                                  // lane in the group
  const uint32_t gm = G == 32 ? FULL : (((1u << G) - 1u) << (wl & (32 - G)));  // the group's lanes
  if (r >= n_reads) return;
  const uint64_t c0 = cand_off[r], c1 = cand_off[r + 1];
  const int slots = 1 + n_refs;
  // with one reference its record is the overall one: computed once, stored twice
  const int f_end = n_refs == 1 ? 0 : n_refs;
  if (c1 - c0 <= static_cast<uint64_t>(G)) {
    // up to G windows: one per lane, loaded once; the same rules as below
    const bool has = c0 + l < c1;
    const uint64_t c = c0 + l;
    const int32_t s = has ? item_score[c] : 0;
    const uint32_t ref = has ? c_ref[c] : 0u, str = has ? c_strand[c] : 0u;
    const unsigned long long gend = has ? c_start[c] + item_end[c] - 1 : 0ull;
    const unsigned long long locus = (static_cast<unsigned long long>(ref) << 60) | (gend << 20) |
                                     (static_cast<unsigned long long>(str) << 19);
    for (int f = -1; f < f_end; ++f) {
      const bool in = has && (f < 0 || ref == static_cast<uint32_t>(f));
      const int32_t best = __reduce_max_sync(gm, in ? max(s, 0) : 0);
      DevHit h{};
      h.item = -1;
      if (best > 0) {
        const bool top = in && s == best;
        const unsigned long long wk = gmin64<G>(gm, top ? locus | static_cast<unsigned long long>(l) : ~0ull);
        const int win = static_cast<int>(wk & 0x7ffffull);
        const unsigned long long wlocus = wk & ~0x7ffffull;
        h.score = best;
        h.second = __reduce_max_sync(gm, (in && s > 0 && locus != wlocus) ? s : 0);
        // ties: distinct loci among the best-scoring windows
        const uint32_t tops = __ballot_sync(gm, top);
        const uint32_t same = __match_any_sync(gm, top ? locus : ~0ull);
        h.n_ties = static_cast<uint32_t>(
            __popc(__ballot_sync(gm, top && (same & tops & ((1u << wl) - 1u)) == 0u)));
        h.item = static_cast<int32_t>(c0 + static_cast<uint64_t>(win));
      }
      if (l == 0) {
        hits[r * slots + (f + 1)] = h;
        if (f_end == 0) hits[r * slots + 1] = h;
      }
    }
    return;
  }
  for (int f = -1; f < f_end; ++f) {
    // best score
    int32_t best = 0;
    for (uint64_t c = c0 + l; c < c1; c += G) {
      if (f >= 0 && c_ref[c] != f) continue;
      best = max(best, item_score[c]);
    }
    best = __reduce_max_sync(gm, best);
    DevHit h{};
    h.item = -1;
    if (best > 0) {
      // winner: smallest (ref, global end, strand, candidate index) among the best
      unsigned long long wk = ~0ull;
      for (uint64_t c = c0 + l; c < c1; c += G) {
        if ((f >= 0 && c_ref[c] != f) || item_score[c] != best) continue;
        const unsigned long long gend = c_start[c] + item_end[c] - 1;
        const unsigned long long k = (static_cast<unsigned long long>(c_ref[c]) << 60) |
                                     (gend << 20) |
                                     (static_cast<unsigned long long>(c_strand[c]) << 19) |
                                     static_cast<unsigned long long>(c - c0);
        wk = k < wk ? k : wk;
      }
      wk = gmin64<G>(gm, wk);
      const uint64_t wc = c0 + (wk & 0x7ffffull);
      const uint32_t wref = c_ref[wc], wstr = c_strand[wc];
      const unsigned long long wend = c_start[wc] + item_end[wc] - 1;
      int32_t second = 0;
      uint32_t ties = 0;
      for (uint64_t c = c0 + l; c < c1; c += G) {
        if (f >= 0 && c_ref[c] != f) continue;
        const int32_t s = item_score[c];
        if (s <= 0) continue;
        const unsigned long long ge = c_start[c] + item_end[c] - 1;
        const bool same = c_ref[c] == wref && ge == wend && c_strand[c] == wstr;
        if (!same) second = max(second, s);
        if (s == best) {
          bool seen = false;
          for (uint64_t u = c0; u < c && !seen; ++u) {
            if (f >= 0 && c_ref[u] != f) continue;
            seen = item_score[u] == best && c_ref[u] == c_ref[c] && c_strand[u] == c_strand[c] &&
                   c_start[u] + item_end[u] - 1 == ge;
          }
          ties += seen ? 0u : 1u;
        }
      }
      h.score = best;
      h.second = __reduce_max_sync(gm, second);
      h.n_ties = __reduce_add_sync(gm, ties);
      h.item = static_cast<int32_t>(wc);
    }
    if (l == 0) {
      hits[r * slots + (f + 1)] = h;
      if (f_end == 0) hits[r * slots + 1] = h;
    }
  }
}

// How each read's winner finds its end row for the traceback.  int32-class
// winners go to the full-rectangle kernel.  Otherwise the band that covers every
// row able to end the alignment (rows ceil(S / match) .. m in local mode, row m
// in final-row mode) is searched directly when it is at most 64 diagonals wide;
// wider ones first get their end row from the extension kernels' winner mode,
// for which they are compacted into the front of `order` (one range for all
// read lengths: there are few, and one launch costs less than one per bin).
__global__ void k_winners(uint32_t n_reads, int slots, const DevHit* hits, const uint16_t* item_key,
                          const uint32_t* class_range, const uint32_t* rlen, const uint32_t* item_read,
                          const uint32_t* item_end, ScoreConst sc, int mode, bool plain,
                          uint32_t* wcount, uint32_t* order, uint8_t* tb_flag) {
  const uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (r >= n_reads) return;
  const DevHit h = hits[r * slots];
  uint8_t flag = kTbFlagBand;
  if (h.item >= 0 && h.score > 0) {
    const uint32_t cls = plain ? 0u : static_cast<uint32_t>(item_key[h.item]) / kKeysPerClass;
    if (cls >= static_cast<uint32_t>(kNumBins)) {
      flag = kTbFlagFull;
    } else if (mode == 0) {
      const uint32_t m = rlen[item_read[h.item]];
      const uint32_t ilo = tb_min_row(sc.sa, h.score);
      const TbBand b = tb_band(sc.sa, sc.go, sc.ge, h.score, item_end[h.item], ilo < 1u ? 1u : ilo, m);
      if (b.w > kTbMaxBand) {
        flag = kTbFlagRow;
        order[atomicAdd(&wcount[0], 1u)] = static_cast<uint32_t>(h.item);
      }
    }
  }
  tb_flag[r] = flag;
}

__global__ void k_wrange(const uint32_t* wcount, uint32_t* wrange) {
  const int c = threadIdx.x;
  if (c >= kNumClasses) return;
  wrange[2 * c] = 0u;
  wrange[2 * c + 1] = c == 0 ? wcount[0] : 0u;
}

// Classification of each read between references 0 and 1 (Sec. 6.1-6.4): the
// higher score wins by at least `margin`; a read under min_score on one
// reference counts for the other; under min_score on both it is unaligned.
// Scores are read with a stride (in 32-bit words) so that both the device hit
// slots and the public sr_hit records can be classified in place.
__global__ void k_classify(uint32_t n_reads, const int32_t* score_a, const int32_t* score_b, uint64_t stride,
                           int32_t min_score, int32_t margin, uint8_t* cls) {
  const uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (r >= n_reads) return;
  const int32_t a = score_a ? score_a[r * stride] : 0;
  const int32_t b = score_b ? score_b[r * stride] : 0;
  uint8_t c;
  if (max(a, b) < min_score) c = 0;
  else if (b < min_score) c = 1;
  else if (a < min_score) c = 2;
  else if (a - b >= margin) c = 1;
  else if (b - a >= margin) c = 2;
  else c = 3;
  cls[r] = c;
}

// ---- CIGAR compaction: exclusive scan of per-read lengths, then gather
__global__ void k_scan_block(const DevHit* hits, int slots, uint32_t n, uint32_t* out,
                             uint32_t* block_sums) {
  __shared__ uint32_t sh[1024];
  const uint32_t i = blockIdx.x * 1024u + threadIdx.x;
  const uint32_t v = i < n ? hits[static_cast<uint64_t>(i) * slots].cigar_len : 0u;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    uint32_t x = threadIdx.x >= static_cast<unsigned>(off) ? sh[threadIdx.x - off] : 0u;
    __syncthreads();
    sh[threadIdx.x] += x;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == 1023) block_sums[blockIdx.x] = sh[1023];
}

__global__ void k_scan_sums(uint32_t* block_sums, uint32_t nb, uint32_t* total_out) {
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  __shared__ uint32_t sh[1024];
  for (uint32_t base = 0; base < nb; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < nb ? block_sums[i] : 0u;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      uint32_t x = threadIdx.x >= static_cast<unsigned>(off) ? sh[threadIdx.x - off] : 0u;
      __syncthreads();
      sh[threadIdx.x] += x;
      __syncthreads();
    }
    if (i < nb) block_sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_cigar_gather(const DevHit* hits, int slots, uint32_t n, const uint32_t* block_sums,
                               uint32_t* off, const uint32_t* slots_buf, uint32_t* cigar) {
  const uint32_t r = blockIdx.x * static_cast<uint32_t>(blockDim.x) + threadIdx.x;
  if (r >= n) return;
  const uint32_t o = off[r] + block_sums[r >> 10];
  off[r] = o;
  const uint32_t len = hits[static_cast<uint64_t>(r) * slots].cigar_len;
  const uint32_t* src = slots_buf + static_cast<uint64_t>(r) * kCigarStride;
  for (uint32_t k = 0; k < len; ++k) cigar[o + k] = src[k];
}

}  // namespace

int launch_pack_refs(const char* ascii, uint64_t len, uint32_t* words, uint32_t* status,
                     cudaStream_t st) {
  const uint64_t nw = ((len + 63) / 64) * 4 + 16;
  const int threads = 256;
  const uint64_t blocks = (nw + threads - 1) / threads;
  k_pack_ref<<<static_cast<unsigned>(blocks < 65535 * 16 ? blocks : 65535 * 16), threads, 0, st>>>(
      ascii, len, nw, words, status);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_prepare(const BatchDev& b, const DevRefs& refs, cudaStream_t st) {
  if (b.n_reads == 0) return 0;
  const uint64_t t = static_cast<uint64_t>(b.n_reads) * 16;
  k_pack_reads<<<static_cast<unsigned>((t + 255) / 256), 256, 0, st>>>(
      b.bases, b.read_off, b.n_reads, b.rpack, b.rlen, b.status);
  const uint64_t tw = static_cast<uint64_t>(b.n_reads) * 8;
  k_items<<<static_cast<unsigned>((tw + 255) / 256), 256, 0, st>>>(
      b.cand_off, b.n_reads, b.c_ref, b.c_strand, b.c_start, b.c_len, refs, b.item_read, b.status);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int launch_bins(const BatchDev& b, const ScoreConst& sc, const TuneBin* bins, int n_bins,
                bool force_i32, bool plain, cudaStream_t st) {
  if (plain || b.n_items == 0) return 0;
  BinArgs ba;
  const int32_t goe = sc.go + sc.ge;
  const bool tables_fit = sc.sa + goe <= 127 && goe - sc.sb >= -128 && goe + sc.ge + 256 < kBias;
  for (int m = 0; m <= kMaxReadLen; ++m) {
    int c = n_bins - 1;
    for (int k = 0; k < n_bins; ++k)
      if (static_cast<uint32_t>(m) <= bins[k].upper) {
        c = k;
        break;
      }
    const bool i16_ok = tables_fit && static_cast<int64_t>(sc.sa) * m <= 32767 - kBias;
    ba.cls_of_len[m] = static_cast<uint8_t>((force_i32 || !i16_ok) ? kI32Class : c);
  }
  cudaMemsetAsync(b.hist, 0, sizeof(uint32_t) * kNumKeys, st);
  cudaMemsetAsync(b.queue, 0, sizeof(uint32_t) * (kNumClasses + 8), st);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t blocks_needed = (b.n_items + 1023) / 1024;
  const unsigned kb = static_cast<unsigned>(blocks_needed < static_cast<uint64_t>(nsm) * 4
                                                ? blocks_needed
                                                : static_cast<uint64_t>(nsm) * 4);
  k_keys<<<kb, 1024, 0, st>>>(b.item_read, b.rlen, b.c_len, b.n_items, ba, b.item_key, b.hist);
  k_scan_keys<<<1, 1024, 0, st>>>(b.hist, b.cursor, b.class_range);
  k_scatter<<<static_cast<unsigned>((b.n_items + 255) / 256), 256, 0, st>>>(b.item_key, b.n_items,
                                                                            b.cursor, b.order);
  return cudaPeekAtLastError() == cudaSuccess ? 3 : -1;
}

int launch_select(const BatchDev& b, int n_refs, cudaStream_t st) {
  if (b.n_reads == 0) return 0;
  // G lanes per read, by the batch's windows per read: a read with up to G
  // windows is handled one window per lane, more in a loop.  Half a warp when
  // reads hold several windows (c2: Poisson(6)); 4 or 8 lanes when they hold one
  // or two (index candidates on a diverged reference pair: 1.3 per read), so
  // that fewer lanes idle.
  const uint64_t wpr = (b.n_items + b.n_reads - 1) / b.n_reads;  // mean windows per read, rounded up
  auto go = [&](auto kern, int G) {
    const uint64_t t = static_cast<uint64_t>(b.n_reads) * G;
    kern<<<static_cast<unsigned>((t + 255) / 256), 256, 0, st>>>(b.cand_off, b.n_reads, b.item_score, b.item_end,
                                                                 b.c_ref, b.c_strand, b.c_start, n_refs, b.hits);
  };
  if (wpr <= 2) go(k_select<4>, 4);
  else if (wpr <= 4) go(k_select<8>, 8);
  else go(k_select<16>, 16);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_winners(const BatchDev& b, const ScoreConst& sc, int mode, int n_refs, bool plain,
                   cudaStream_t st) {
  if (b.n_reads == 0) return 0;
  if (cudaMemsetAsync(b.wcount, 0, sizeof(uint32_t) * kNumClasses, st) != cudaSuccess) return -1;
  if (cudaMemsetAsync(b.wqueue, 0, sizeof(uint32_t) * (kNumClasses + 8), st) != cudaSuccess) return -1;
  k_winners<<<(b.n_reads + 255) / 256, 256, 0, st>>>(b.n_reads, 1 + n_refs, b.hits, b.item_key,
                                                     b.class_range, b.rlen, b.item_read, b.item_end, sc,
                                                     mode, plain, b.wcount, b.order, b.tb_flag);
  k_wrange<<<1, 32, 0, st>>>(b.wcount, b.wrange);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

// Results in the public sr_hit layout: reference, strand and reference
// coordinates of each read's overall winner (with its CIGAR offset) and of its
// best window per reference.
__global__ void k_assemble(uint32_t n_reads, int slots, const DevHit* hits, const uint8_t* c_ref,
                           const uint8_t* c_strand, const uint64_t* c_start, const uint32_t* item_end,
                           const uint32_t* cigar_off, bool want_cigar, int32_t item_base, uint32_t cigar_base,
                           sr_hit* best, sr_hit* per_ref) {
  const uint64_t x = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (x >= static_cast<uint64_t>(n_reads) * slots) return;
  const uint64_t i = x / slots;
  const int sl = static_cast<int>(x - i * slots);
  const DevHit h = hits[x];
  sr_hit o;
  o.score = h.score;
  o.second = h.second;
  o.n_ties = h.n_ties;
  o.item = h.item >= 0 ? h.item + item_base : h.item;
  o.ref_id = 0;
  o.strand = 0;
  o.reserved = 0;
  o.read_start = 0;
  o.read_end = 0;
  o.ref_start = 0;
  o.ref_end = 0;
  o.cigar_off = 0;
  o.cigar_len = 0;
  if (h.item >= 0) {
    const uint64_t it = static_cast<uint64_t>(h.item);
    o.ref_id = c_ref[it];
    o.strand = c_strand[it];
    o.ref_end = c_start[it] + item_end[it] - 1;
    if (sl == 0 && want_cigar) {
      o.read_start = h.read_start;
      o.read_end = h.read_end;
      o.ref_start = c_start[it] + h.start_j - 1;
      o.cigar_off = cigar_base + cigar_off[i];
      o.cigar_len = h.cigar_len;
    }
  }
  if (sl == 0) best[i] = o;
  else per_ref[i * (slots - 1) + (sl - 1)] = o;
}

int launch_assemble(const BatchDev& b, int n_refs, bool want_cigar, int32_t item_base, uint32_t cigar_base,
                    cudaStream_t st) {
  if (b.n_reads == 0) return 0;
  const uint64_t total = static_cast<uint64_t>(b.n_reads) * (1 + n_refs);
  k_assemble<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(
      b.n_reads, 1 + n_refs, b.hits, b.c_ref, b.c_strand, b.c_start, b.item_end, b.cigar_off, want_cigar,
      item_base, cigar_base, b.out_best, b.out_per_ref);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// A batch staged from a read range [r0, r1) of the caller's arrays receives
// the range's offsets as they are; they are made batch-relative here.
// ---- checks of a batch staged from device memory (the host path runs the same
// checks on the caller's host arrays): per read, its offsets, length, window
// count and windows; the first bad read (lowest index) with the reason, and for
// good batches the DP cells, the longest read and the windows per read length.
__global__ void k_stage_check(const uint64_t* read_off, const uint64_t* cand_off, uint32_t n, uint64_t nc,
                              const uint8_t* c_ref, const uint8_t* c_strand, const uint64_t* c_start,
                              const uint32_t* c_len, DevRefs refs, StageCheck* out) {
  __shared__ uint32_t hist[kMaxReadLen + 1];
  __shared__ unsigned long long cells_sh;
  for (int k = threadIdx.x; k <= kMaxReadLen; k += blockDim.x) hist[k] = 0;
  if (threadIdx.x == 0) cells_sh = 0;
  __syncthreads();
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cells = 0;
  if (r < n) {
    const uint64_t a0 = read_off[r], a1 = read_off[r + 1], c0 = cand_off[r], c1 = cand_off[r + 1];
    uint32_t why = 0;
    if (a1 < a0 || c1 < c0 || c1 > nc) why = 1;
    else if (a1 - a0 == 0 || a1 - a0 > static_cast<uint64_t>(kMaxReadLen)) why = 2;
    else if (c1 - c0 >= (1ull << 19)) why = 3;
    if (!why) {
      const uint64_t m = a1 - a0;
      uint64_t suml = 0;
      for (uint64_t k = c0; k < c1; ++k) {
        const uint32_t ref = c_ref[k], len = c_len[k];
        const uint64_t w0 = c_start[k];
        const bool ok = ref < static_cast<uint32_t>(refs.n) && c_strand[k] <= 1 && len >= 1 &&
                        len <= static_cast<uint32_t>(kMaxWinLen) && w0 <= refs.len[ref] && w0 + len <= refs.len[ref];
        if (!ok) {
          why = 4;
          break;
        }
        suml += len;
      }
      if (!why) {
        cells = m * suml;
        if (c1 > c0) atomicAdd(&hist[m], static_cast<uint32_t>(c1 - c0));
        atomicMax(&out->max_m, static_cast<uint32_t>(m));
      }
    }
    if (why) atomicMin(&out->bad, (static_cast<unsigned long long>(r) << 3) | why);
  }
  for (int o = 16; o; o >>= 1) cells += __shfl_xor_sync(0xffffffffu, cells, o);
  if ((threadIdx.x & 31) == 0 && cells) atomicAdd(&cells_sh, cells);
  __syncthreads();
  for (int k = threadIdx.x; k <= kMaxReadLen; k += blockDim.x)
    if (hist[k]) atomicAdd(&out->by_len[k], static_cast<unsigned long long>(hist[k]));
  if (threadIdx.x == 0 && cells_sh) atomicAdd(&out->cells, cells_sh);
}

// the first bad window of read r (after k_stage_check found one there)
__global__ void k_first_bad_window(uint32_t r, const uint64_t* cand_off, const uint8_t* c_ref, const uint8_t* c_strand,
                                   const uint64_t* c_start, const uint32_t* c_len, DevRefs refs, StageCheck* out) {
  const uint64_t c0 = cand_off[r], c1 = cand_off[r + 1];
  for (uint64_t k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
    const uint32_t ref = c_ref[k], len = c_len[k];
    const uint64_t w0 = c_start[k];
    const bool ok = ref < static_cast<uint32_t>(refs.n) && c_strand[k] <= 1 && len >= 1 &&
                    len <= static_cast<uint32_t>(kMaxWinLen) && w0 <= refs.len[ref] && w0 + len <= refs.len[ref];
    if (!ok) atomicMin(&out->bad_win, static_cast<unsigned long long>(k));
  }
}

int launch_stage_check(const BatchDev& b, const DevRefs& refs, StageCheck* out, cudaStream_t st) {
  if (cudaMemsetAsync(out, 0, sizeof(StageCheck), st) != cudaSuccess) return -1;
  if (cudaMemsetAsync(&out->bad, 0xff, 2 * sizeof(unsigned long long), st) != cudaSuccess) return -1;
  if (b.n_reads == 0) return 0;
  k_stage_check<<<(b.n_reads + 255) / 256, 256, 0, st>>>(b.read_off, b.cand_off, b.n_reads, b.n_items, b.c_ref,
                                                         b.c_strand, b.c_start, b.c_len, refs, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_first_bad_window(const BatchDev& b, const DevRefs& refs, uint32_t read, StageCheck* out,
                            cudaStream_t st) {
  k_first_bad_window<<<1, 256, 0, st>>>(read, b.cand_off, b.c_ref, b.c_strand, b.c_start, b.c_len, refs, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

__global__ void k_rebase_offsets(uint64_t* off, uint64_t n, uint64_t base) {
  const uint64_t x = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (x < n) off[x] -= base;
}

int launch_rebase_offsets(uint64_t* off, uint64_t n, uint64_t base, cudaStream_t st) {
  if (n == 0 || base == 0) return 0;
  k_rebase_offsets<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(off, n, base);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_classify(const BatchDev& b, int n_refs, int32_t min_score, int32_t margin,
                    cudaStream_t st) {
  if (b.n_reads == 0) return 0;
  static_assert(sizeof(DevHit) % 4 == 0, "hit slots are whole words");
  const uint64_t stride = (1ull + n_refs) * sizeof(DevHit) / 4;
  k_classify<<<(b.n_reads + 255) / 256, 256, 0, st>>>(b.n_reads, n_refs > 0 ? &b.hits[1].score : nullptr,
                                                      n_refs > 1 ? &b.hits[2].score : nullptr, stride, min_score,
                                                      margin, b.read_class);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_classify_hits(const sr_hit* per_ref, uint32_t n_reads, uint32_t n_refs, int32_t min_score,
                         int32_t margin, uint8_t* out, cudaStream_t st) {
  if (n_reads == 0) return 0;
  static_assert(sizeof(sr_hit) % 4 == 0, "sr_hit records are whole words");
  const uint64_t stride = static_cast<uint64_t>(n_refs) * sizeof(sr_hit) / 4;
  k_classify<<<(n_reads + 255) / 256, 256, 0, st>>>(n_reads, &per_ref[0].score, &per_ref[1].score, stride, min_score,
                                                    margin, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_cigar_compact(const BatchDev& b, int n_refs, cudaStream_t st) {
  if (b.n_reads == 0) return 0;
  const int slots = 1 + n_refs;
  const uint32_t nb = (b.n_reads + 1023) / 1024;
  k_scan_block<<<nb, 1024, 0, st>>>(b.hits, slots, b.n_reads, b.cigar_off, b.scan_tmp);
  k_scan_sums<<<1, 1024, 0, st>>>(b.scan_tmp, nb, b.cigar_off + b.n_reads);
  k_cigar_gather<<<(b.n_reads + 255) / 256, 256, 0, st>>>(b.hits, slots, b.n_reads, b.scan_tmp,
                                                          b.cigar_off, b.cigar_slots, b.cigar);
  return cudaPeekAtLastError() == cudaSuccess ? 3 : -1;
}

int preload_kernels() {
  int n_ = 0;
  SR_TOUCH(k_pack_ref);
  SR_TOUCH(k_pack_reads);
  SR_TOUCH(k_items);
  SR_TOUCH(k_keys);
  SR_TOUCH(k_scan_keys);
  SR_TOUCH(k_scatter);
  SR_TOUCH(k_select<4>);
  SR_TOUCH(k_select<8>);
  SR_TOUCH(k_select<16>);
  SR_TOUCH(k_select<32>);
  SR_TOUCH(k_winners);
  SR_TOUCH(k_wrange);
  SR_TOUCH(k_classify);
  SR_TOUCH(k_scan_block);
  SR_TOUCH(k_scan_sums);
  SR_TOUCH(k_cigar_gather);
  SR_TOUCH(k_assemble);
  SR_TOUCH(k_stage_check);
  SR_TOUCH(k_first_bad_window);
  SR_TOUCH(k_rebase_offsets);
  return n_;
}

}  // namespace sr
