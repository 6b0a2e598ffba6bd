// sr_cal.cu -- the CAL finder and filter on the device (McVicar et al., arXiv
// 1805.00106, Sec. 3.2 CAL finder, Sec. 3.3 CAL filter; the paper's V2 keeps
// them on the host, Sec. 4.1-4.2).  Same windows, in the same order, as the host
// stage sr_candidates.
//
//   count / emit  one warp per read: the read's 2-bit codes packed in shared
//                 memory (with its reverse complement), each lane takes seeds
//                 o = lane*stride, (lane+32)*stride, ...; per reference the
//                 hashed canonical seed picks a bucket, its key is found among
//                 the bucket's (key, position)-sorted entries (or, with bucket
//                 heads, in the bucket's 64-byte head), and every matching entry
//                 gives a '+' and/or '-' CAL by its orientation bits.  The count
//                 pass keeps each lookup for the emit pass.  CALs are packed keys
//                 ref << 60 | strand << 59 | (cal + 1024).
//   filter        per read: a sort of its CAL keys, then the merge of
//                 consecutive CALs <= merge_dist apart into windows represented
//                 by their most frequent CAL (smallest on ties), the max_cands
//                 cut by hit count, and the clamped window [cal - pad, cal + m +
//                 pad).  One warp per read up to 128 CALs, one block up to 8192
//                 (shared memory); larger reads are emitted, sorted and merged by
//                 many blocks each, in tiles of 4096 keys.
//   compact       per-read windows to contiguous arrays.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sr_internal.h"
#include "sr_seed.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kCalWarps = 4;
constexpr uint64_t kCalBias = 1024;
constexpr uint64_t kCalMask = (1ull << 59) - 1;
constexpr uint64_t kNoKey = ~0ull;

__device__ __forceinline__ uint64_t cal_key(uint32_t ref, uint32_t strand, int64_t cal) {
  return (static_cast<uint64_t>(ref) << 60) | (static_cast<uint64_t>(strand) << 59) |
         static_cast<uint64_t>(cal + static_cast<int64_t>(kCalBias));
}

// ASCII -> 2-bit code; 4 for a non-ACGT byte
__device__ __forceinline__ uint32_t code_of(char ch) {
  switch (static_cast<unsigned>(static_cast<unsigned char>(ch)) | 0x20u) {
    case 'a': return 0;
    case 'c': return 1;
    case 'g': return 2;
    case 't': return 3;
    default: return 4;
  }
}

// entries [l, e) of the sorted keys K[s0 .. s1) equal to key
template <typename KT>
__device__ __forceinline__ void key_range(const KT* K, uint64_t s0, uint64_t s1, uint32_t key, uint64_t* lo,
                                          uint64_t* hi) {
  uint64_t l = s0, u = s1;
  while (l < u) {
    const uint64_t mid = l + ((u - l) >> 1);
    if (K[mid] < key) l = mid + 1;
    else u = mid;
  }
  uint64_t e = l;
  while (e < s1 && K[e] == key) ++e;
  *lo = l;
  *hi = e;
}

// packed index: entries [lo, hi) of reference r with key `key` in bucket b
// (16-bit keys in key16, 32-bit ones in key)
__device__ __forceinline__ void lookup_packed(const DevIndex& di, uint64_t b, uint32_t key, int r, uint64_t* lo,
                                              uint64_t* hi) {
  const uint64_t s0 = di.jptr[b * di.n_refs + r], s1 = di.jptr[(b + 1) * di.n_refs + r];
  if (di.key_bits == 16) key_range(di.key16[r], s0, s1, key, lo, hi);
  else key_range(di.key[r], s0, s1, key, lo, hi);
}

// 32-bit keys: the head holds up to kHeadKeys32, one per word
__device__ __forceinline__ bool head_range32(const uint4 v0, const uint4 v1, const uint4 v2, const uint4 v3,
                                             uint32_t key, uint32_t* lo0, uint32_t* hi0, uint32_t* lo1,
                                             uint32_t* hi1) {
  const uint32_t w[13] = {v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w, v3.x, v3.y, v3.z, v3.w};
  uint32_t eq = 0;
#pragma unroll
  for (int j = 0; j < 13; ++j) eq |= (w[j] == key ? 1u : 0u) << j;
  const uint32_t n0 = v0.z & 0xffffu, n1 = v0.z >> 16;
  const uint32_t m0 = (1u << n0) - 1u, m1 = ((1u << (n0 + n1)) - 1u) & ~m0;
  const uint32_t e0 = eq & m0, e1 = eq & m1;
  *lo0 = v0.x + (e0 ? __ffs(e0) - 1u : 0u);
  *hi0 = *lo0 + __popc(e0);
  *lo1 = v0.y + (e1 ? __ffs(e1) - 1u - n0 : 0u);
  *hi1 = *lo1 + __popc(e1);
  return true;
}

// packed index with bucket heads: entries [lo0, hi0) of reference 0 and [lo1,
// hi1) of reference 1 with key `key` in bucket b, from the bucket's head alone
// (an empty range may start anywhere); false when the bucket spilled (its
// entries are then looked up in jptr / key16)
__device__ __forceinline__ bool lookup_head(const uint4* heads, uint64_t b, uint32_t key, int key_bits,
                                            uint32_t* lo0, uint32_t* hi0, uint32_t* lo1, uint32_t* hi1) {
  const uint4* h = heads + b * 4;
  const uint4 v0 = __ldg(h), v1 = __ldg(h + 1), v2 = __ldg(h + 2), v3 = __ldg(h + 3);
  if (v0.z == kHeadSpill) return false;
  if (key_bits != 16) return head_range32(v0, v1, v2, v3, key, lo0, hi0, lo1, hi1);
  const uint32_t w[13] = {v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w, v3.x, v3.y, v3.z, v3.w};
  // bit i: the head's key i equals the seed's, two keys per word: a 16-bit half
  // of w ^ (key, key) is zero exactly when adding 0x7fff to its low 15 bits
  // leaves its top bit clear and its top bit was clear
  const uint32_t kk = key | (key << 16);
  uint32_t eq = 0;
#pragma unroll
  for (int j = 0; j < 13; ++j) {
    const uint32_t x = w[j] ^ kk;
    const uint32_t z = ~(((x & 0x7fff7fffu) + 0x7fff7fffu) | x) & 0x80008000u;
    eq |= (((z >> 15) & 1u) | (z >> 30)) << (2 * j);
  }
  // equal keys are consecutive within each reference's run of sorted keys
  const uint32_t n0 = v0.z & 0xffffu, n1 = v0.z >> 16;
  const uint32_t m0 = (1u << n0) - 1u, m1 = ((1u << (n0 + n1)) - 1u) & ~m0;
  const uint32_t e0 = eq & m0, e1 = eq & m1;
  *lo0 = v0.x + (e0 ? __ffs(e0) - 1u : 0u);
  *hi0 = *lo0 + __popc(e0);
  *lo1 = v0.y + (e1 ? __ffs(e1) - 1u - n0 : 0u);
  *hi1 = *lo1 + __popc(e1);
  return true;
}

// entries [lo, hi) of reference r whose key equals the seed's
__device__ __forceinline__ void lookup(const DevIndex& di, int r, uint64_t canon, uint64_t* lo, uint64_t* hi) {
  const int kb = 2 * (di.k - di.a);
  const uint64_t h = seed_hash(canon, di.k, di.hash_seed[r]);
  const uint64_t b = h >> kb;
  const uint32_t key = static_cast<uint32_t>(h & mask_bits(kb));
  uint64_t s0 = di.ptr[r][b], s1 = di.ptr[r][b + 1];
  const uint32_t* K = di.key[r];
  // lower bound of key in the bucket
  uint64_t l = s0, u = s1;
  while (l < u) {
    const uint64_t mid = l + ((u - l) >> 1);
    if (K[mid] < key) l = mid + 1;
    else u = mid;
  }
  uint64_t e = l;
  while (e < s1 && K[e] == key) ++e;
  *lo = l;
  *hi = e;
}

// read r's codes into shared memory; false (and status) on a non-ACGT base
__device__ __forceinline__ bool load_codes(const char* bases, uint64_t o0, uint32_t m, uint8_t* q, int lane,
                                           uint32_t* status) {
  bool bad = false;
  for (uint32_t t = lane; t < m; t += 32) {
    const uint32_t c = code_of(bases[o0 + t]);
    bad |= c > 3;
    q[t] = static_cast<uint8_t>(c & 3);
  }
  bad = __any_sync(FULL, bad);
  if (bad && lane == 0) atomicOr(status, kStBadBase);
  __syncwarp();
  return !bad;
}

// The read's codes as 2-bit fields, first base highest, in kPackWords 32-bit
// words (kMaxReadLen bases and two words of padding): Pk for the read, Rk for
// the reverse complement of the read padded to kMaxReadLen bases, so that a
// seed's forward and reverse-complement k-mers (Kmer's fwd and rc) are each
// read with two funnel shifts.  Bases past the read's end are never extracted.
constexpr int kPackWords = kMaxReadLen / 16 + 2;

// q: the codes (one byte each, 4-byte aligned); lanes 0-15 pack word j
__device__ __forceinline__ void pack_codes(const uint8_t* q, uint32_t* Pk, uint32_t* Rk, int lane) {
  const uint32_t* q32 = reinterpret_cast<const uint32_t*>(q);
  uint32_t w = 0;
  if (lane < kMaxReadLen / 16) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // four codes, first in byte 0, to one byte with the first code highest
      const uint32_t x = __byte_perm(q32[4 * lane + i] & 0x03030303u, 0, 0x0123);
      const uint32_t t = (x | (x >> 6)) & 0x000F000Fu;
      w = (w << 8) | ((t | (t >> 12)) & 0xFFu);
    }
  }
  // the reverse complement: words in reverse order, 2-bit fields reversed, complemented
  const uint32_t src = __shfl_sync(FULL, w, (kMaxReadLen / 16 - 1 - lane) & 31);
  uint32_t r = __brev(~src);
  r = ((r >> 1) & 0x55555555u) | ((r << 1) & 0xAAAAAAAAu);
  if (lane < kMaxReadLen / 16) {
    Pk[lane] = w;
    Rk[lane] = r;
  } else if (lane < kPackWords) {
    Pk[lane] = 0;
    Rk[lane] = 0;
  }
  __syncwarp();
}

// the k bases at o of a packed string, first base highest (k <= 32)
__device__ __forceinline__ uint64_t kmer_at(const uint32_t* W, uint32_t o, int k) {
  const uint32_t b = 2 * o, j = b >> 5, s = b & 31;
  const uint32_t w0 = W[j], w1 = W[j + 1], w2 = W[j + 2];
  const uint64_t win = (static_cast<uint64_t>(__funnelshift_l(w1, w0, s)) << 32) | __funnelshift_l(w2, w1, s);
  return win >> (64 - 2 * k);
}

struct SeedArgs {
  DevIndex di;
  const char* bases;
  const uint64_t* read_off;
  uint32_t r0, nr;        // reads r0 .. r0 + nr
  uint32_t stride;
  uint32_t* count;        // count pass: an upper bound of the CALs of each read (indexed r - r0)
  const uint64_t* off;    // emit pass: first slot of each read (indexed r - r0)
  uint64_t* cals;         // emit pass
  uint32_t* actual;       // emit pass: the CALs written for each read (indexed r - r0)
  uint32_t* status;
  // Seed lookups kept from the count pass for the emit pass (nullptr: the emit
  // pass looks its seeds up again): per read (indexed r - rbase) its records
  // start at seed_off, one per (seed, reference) in that order; recount (per
  // read) marks the reads whose records could not hold a lookup
  uint64_t* ranges;
  const uint32_t* seed_off;
  uint8_t* recount;
  uint32_t rbase;
};

// a kept lookup: first matching entry (38 bits), their number (24 bits) and the
// seed's orientation bits (2)
constexpr uint32_t kRangeCntMax = (1u << 24) - 1u;
constexpr uint64_t kRangeLoMax = (1ull << 38) - 1ull;
__device__ __forceinline__ uint64_t range_pack(uint64_t lo, uint32_t cnt, uint32_t rori) {
  return (lo << 26) | (static_cast<uint64_t>(cnt) << 2) | rori;
}

// seeds x references of each read (the lookup records the count pass keeps);
// reads with decreasing offsets or over kMaxReadLen bases set kStBadRead
__global__ void k_cal_slots(const uint64_t* read_off, uint32_t n, int k, uint32_t stride, int n_refs,
                            uint32_t* slots, uint32_t* status) {
  const uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (r >= n) return;
  const uint64_t o0 = read_off[r], o1 = read_off[r + 1];
  if (o1 < o0 || o1 - o0 > static_cast<uint64_t>(kMaxReadLen)) {
    atomicOr(status, kStBadRead);
    slots[r] = 0;
    return;
  }
  const uint32_t m = static_cast<uint32_t>(o1 - o0);
  slots[r] = m >= static_cast<uint32_t>(k) ? ((m - k) / stride + 1u) * static_cast<uint32_t>(n_refs) : 0u;
}

// 12 blocks per SM: 40 registers, no spills (48 warps per SM)
template <bool EMIT>
__global__ void __launch_bounds__(32 * kCalWarps, 12) k_cal_seeds(SeedArgs a) {
  __shared__ __align__(16) uint8_t qs[kCalWarps][kMaxReadLen];
  __shared__ uint32_t pk_s[kCalWarps][kPackWords], rk_s[kCalWarps][kPackWords];
  __shared__ uint32_t ctr[kCalWarps];
  __shared__ uint32_t incl_s[kCalWarps][32];  // inclusive scan of the lanes' entry counts
  __shared__ uint64_t lo_s[kCalWarps][32];     // each lane's first matching entry
  __shared__ uint32_t o_s[kCalWarps][32];      // its seed offset and orientation bits
  __shared__ uint32_t ro_s[kCalWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* q = qs[warp];
  uint32_t* incl = incl_s[warp];
  const int k = a.di.k;
  for (uint32_t rr = blockIdx.x * kCalWarps + warp; rr < a.nr; rr += gridDim.x * kCalWarps) {
    const uint32_t r = a.r0 + rr;
    const uint64_t o0 = a.read_off[r], o1 = a.read_off[r + 1];
    const uint32_t m = static_cast<uint32_t>(o1 - o0);
    if (lane == 0) ctr[warp] = 0;
    __syncwarp();
    uint32_t n = 0;
    // offsets and lengths: checked on the host for host reads, here for device reads
    const bool len_ok = o1 >= o0 && o1 - o0 <= static_cast<uint64_t>(kMaxReadLen);
    if (!len_ok && lane == 0) atomicOr(a.status, kStBadRead);
    // the emit pass takes the count pass's lookups when they were kept for this read
    const bool kept = EMIT && a.ranges && !a.recount[r - a.rbase];
    // emit pass: a read of more CALs than kCalSmemKeys whose lookups were kept
    // is left to k_cal_emit_big (its bound, in count, is then its exact count)
    const bool split = kept && a.count && a.count[rr] > kCalSmemKeys;
    uint64_t* rec = a.ranges ? a.ranges + (len_ok ? a.seed_off[r - a.rbase] : 0u) : nullptr;
    bool fits = true;
    if (!split && len_ok && (kept || load_codes(a.bases, o0, m, q, lane, a.status)) &&
        m >= static_cast<uint32_t>(k)) {
      if (!kept) pack_codes(q, pk_s[warp], rk_s[warp], lane);
      const uint64_t base = EMIT ? a.off[rr] : 0;
      // 32 seeds per round, one per lane; the matching entries of all of them
      // are then shared out over the warp (a repeat seed may have thousands)
      for (uint32_t o_base = 0, si_base = 0; o_base + k <= m; o_base += 32 * a.stride, si_base += 32) {
        const uint32_t o = o_base + lane * a.stride;
        const uint32_t si = si_base + lane;  // the seed's index in the read
        const bool live = o + k <= m;
        uint64_t canon = 0;
        uint32_t rori = 0;
        if (!kept) {
          // Kmer's fwd and rc of the seed (the reverse complement's k-mer at
          // kMaxReadLen - o - k of the padded reverse complement)
          const uint64_t fwd = live ? kmer_at(pk_s[warp], o, k) : 0;
          const uint64_t rc = live ? kmer_at(rk_s[warp], kMaxReadLen - o - k, k) : 0;
          canon = fwd < rc ? fwd : rc;
          rori = (fwd == canon ? 1u : 0u) | (rc == canon ? 2u : 0u);
        }
        // packed index: one hash (the references share its seed) gives the bucket
        // and key in every reference
        uint64_t pb = 0;
        uint32_t pkey = 0;
        if (a.di.packed && !kept && live) {
          const int kb = 2 * (k - a.di.a);
          const uint64_t h = seed_hash(canon, k, a.di.hash_seed[0]);
          pb = h >> kb;
          pkey = static_cast<uint32_t>(h & mask_bits(kb));
        }
        // with bucket heads, one access answers both references (at most two);
        // the count pass only (the emit pass reads the lookups it kept)
        uint32_t hl0 = 0, hh0 = 0, hl1 = 0, hh1 = 0;
        bool head = false;
        if (!EMIT && a.di.heads && live)
          head = lookup_head(a.di.heads, pb, pkey, a.di.key_bits, &hl0, &hh0, &hl1, &hh1);
        for (int r2 = 0; r2 < a.di.n_refs; ++r2) {
          uint64_t lo = 0, hi = 0;
          if (kept) {
            if (live) {
              const uint64_t x = rec[static_cast<uint64_t>(si) * a.di.n_refs + r2];
              lo = x >> 26;
              hi = lo + ((x >> 2) & kRangeCntMax);
              rori = static_cast<uint32_t>(x & 3u);
            }
          } else if (live) {
            if (head) {
              lo = r2 ? hl1 : hl0;
              hi = r2 ? hh1 : hh0;
            } else if (a.di.packed) {
              lookup_packed(a.di, pb, pkey, r2, &lo, &hi);
            } else {
              lookup(a.di, r2, canon, &lo, &hi);
            }
          }
          uint32_t cnt = static_cast<uint32_t>(hi - lo);
          if (!EMIT) {
            // an entry gives one CAL unless the seed is its own reverse complement
            // (then at most two): a bound that needs no entry loads
            n += rori == 3u ? 2u * cnt : cnt;
            if (rec && live) {
              const bool ok = hi - lo <= kRangeCntMax && lo <= kRangeLoMax;
              fits = fits && ok;
              rec[static_cast<uint64_t>(si) * a.di.n_refs + r2] = ok ? range_pack(lo, cnt, rori) : 0ull;
            }
            continue;
          }
          uint32_t sc = cnt;
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const uint32_t x = __shfl_up_sync(FULL, sc, off);
            if (lane >= off) sc += x;
          }
          const uint32_t total = __shfl_sync(FULL, sc, 31);
          if (total == 0) continue;
          // owner values (shared memory: lanes that finish early still serve them)
          incl[lane] = sc;
          lo_s[warp][lane] = lo;
          o_s[warp][lane] = o;
          ro_s[warp][lane] = rori;
          __syncwarp();
          // entry j belongs to the first lane whose inclusive count exceeds j
          for (uint32_t j = lane; j < total; j += 32) {
            int lo_l = 0, hi_l = 31;
            while (lo_l < hi_l) {
              const int mid = (lo_l + hi_l) >> 1;
              if (incl[mid] > j) hi_l = mid;
              else lo_l = mid + 1;
            }
            const int own = lo_l;
            const uint32_t before = own ? incl[own - 1] : 0u;
            const uint64_t e = lo_s[warp][own] + (j - before);
            const uint32_t so = o_s[warp][own], sro = ro_s[warp][own];
            // packed index: position and orientation bits in one word
            const uint32_t po = a.di.packed ? a.di.posor[r2][e] : 0u;
            const uint32_t fo = a.di.packed ? po >> 30 : a.di.orient[r2][e];
            const bool plus = ((fo & 1u) && (sro & 1u)) || ((fo & 2u) && (sro & 2u));
            const bool minus = ((fo & 1u) && (sro & 2u)) || ((fo & 2u) && (sro & 1u));
            if (EMIT) {
              const int64_t p = a.di.packed ? (po & 0x3fffffffu) : a.di.pos[r2][e];
              if (plus) a.cals[base + atomicAdd(&ctr[warp], 1u)] = cal_key(r2, 0, p - so);
              if (minus) a.cals[base + atomicAdd(&ctr[warp], 1u)] =
                  cal_key(r2, 1, p - static_cast<int64_t>(m - so - k));
            } else {
              n += (plus ? 1u : 0u) + (minus ? 1u : 0u);
            }
          }
          __syncwarp();
        }
      }
    }
    if (!EMIT) {
      n = __reduce_add_sync(FULL, n);
      if (lane == 0) a.count[rr] = n;
      if (a.ranges) {
        const bool all_fit = __all_sync(FULL, fits);
        if (lane == 0) a.recount[r - a.rbase] = all_fit ? 0 : 1;
      }
    } else if (lane == 0) {
      a.actual[rr] = split ? a.count[rr] : ctr[warp];
    }
    __syncwarp();
  }
}

// block-wide bitonic sort of P (a power of two) keys, ascending
__device__ void bitonic(uint64_t* s, uint32_t P) {
  for (uint32_t size = 2; size <= P; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
        const uint32_t lo = 2 * i - (i & (stride - 1));
        const uint32_t hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t x = s[lo], y = s[hi];
        if ((x > y) == up) {
          s[lo] = y;
          s[hi] = x;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ uint32_t pow2_at_least(uint32_t n) {
  uint32_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

// the large read (index into big) and the part of it (tile or chunk) this block
// takes, from the exclusive prefix tpre of the reads' parts; false for blocks
// past the last part
__device__ __forceinline__ bool block_item(const uint64_t* tpre, uint32_t n_big, uint32_t* b, uint32_t* ti) {
  __shared__ uint32_t sb, st;
  if (threadIdx.x == 0) {
    const uint64_t t = blockIdx.x;
    uint32_t lo = 0, hi = n_big;  // the last read whose first tile is <= t
    while (lo + 1 < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (tpre[mid] <= t) lo = mid;
      else hi = mid;
    }
    const bool in = t < tpre[n_big];
    sb = in ? lo : 0xffffffffu;
    st = in ? static_cast<uint32_t>(t - tpre[lo]) : 0u;
  }
  __syncthreads();
  *b = sb;
  *ti = st;
  return sb != 0xffffffffu;
}

struct FilterArgs {
  DevIndex di;
  const uint64_t* read_off;
  uint32_t r0, nr;
  uint32_t merge_dist, pad, max_cands;
  const uint32_t* count;  // upper bound of the CALs of each read (routes it to a kernel, sizes its space)
  const uint32_t* actual; // CALs of each read
  const uint64_t* off;    // first slot of each read in cals / the window arrays
  uint64_t* cals;
  uint32_t smem_cap;      // reads with more CALs are left to the large-read kernel
  uint32_t* nwin;         // windows per read
  uint64_t* wkey;         // window CAL key (then reused for the start)
  uint32_t* whits;
  uint32_t* wlen;
};

// Block-wide exclusive prefix sum of one 64-bit value per thread; *total gets
// the block's sum.  (Two 32-bit counts packed as high:low add without carries
// while each total stays below 2^32.)
__device__ uint64_t block_exscan(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_sum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
  if (w == 0) {
    uint64_t t = lane < nw ? warp_sum[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(FULL, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_sum[lane] = t;
  }
  __syncthreads();
  const uint64_t before = (w ? warp_sum[w - 1] : 0ull) + x - v;
  *total = warp_sum[nw - 1];
  __syncthreads();
  return before;
}

// The filter of one read (whole block).  keys has room for P CALs (P the power
// of two at or above n) followed by the merge's work space: cal_filter_words(P)
// words in all.
//
// The merge (Sec. 3.3) in parallel: in the sorted CALs, a window starts where
// the (ref, strand) changes or the gap to the previous CAL exceeds merge_dist,
// and a run of equal values starts where the value changes.  One prefix sum
// numbers both; every run offers (length, position in its window) to its
// window by an atomic max, so each window keeps its most frequent value and,
// among equally frequent ones, the first (smallest) -- the rule a serial scan
// of the sorted CALs applies.
__device__ void filter_finish(const FilterArgs& a, uint32_t rr, uint64_t* keys, uint32_t nw);
__device__ __forceinline__ void window_clamp(const FilterArgs& a, uint64_t base, uint32_t m, uint32_t i);

// keys: the read's work space (keys, then the window and run arrays)
__device__ void filter_read(const FilterArgs& a, uint32_t rr, uint64_t* keys, uint32_t n) {
  __shared__ uint32_t s_nw;
  const uint64_t base = a.off[rr];
  const uint32_t P = pow2_at_least(n);
  unsigned long long* wbest = reinterpret_cast<unsigned long long*>(keys + P);  // P per window
  uint32_t* pos_run = reinterpret_cast<uint32_t*>(keys + 2 * P);                // P + 1 run starts
  uint32_t* pos_win = pos_run + P + 1;                                          // P + 1 window starts
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) keys[i] = i < n ? a.cals[base + i] : kNoKey;
  __syncthreads();
  bitonic(keys, P);
  const uint32_t T = blockDim.x;
  const uint32_t per = (n + T - 1) / T;  // each thread a contiguous slice of the sorted CALs
  const uint32_t i0 = min(n, threadIdx.x * per), i1 = min(n, i0 + per);
  const uint64_t md = a.merge_dist;
  auto starts = [&](uint32_t i, bool* rs, bool* ws) {
    const uint64_t k = keys[i];
    if (i == 0) {
      *rs = *ws = true;
      return;
    }
    const uint64_t p = keys[i - 1];
    *rs = k != p;
    *ws = (k >> 59) != (p >> 59) || k - p > md;
  };
  uint64_t cnt = 0;
  for (uint32_t i = i0; i < i1; ++i) {
    bool rs, ws;
    starts(i, &rs, &ws);
    cnt += (static_cast<uint64_t>(ws) << 32) | static_cast<uint64_t>(rs);
  }
  uint64_t tot = 0;
  const uint64_t pre = block_exscan(cnt, &tot);
  const uint32_t nruns = static_cast<uint32_t>(tot), nwin = static_cast<uint32_t>(tot >> 32);
  {
    uint32_t rk = static_cast<uint32_t>(pre), wk = static_cast<uint32_t>(pre >> 32);
    for (uint32_t i = i0; i < i1; ++i) {
      bool rs, ws;
      starts(i, &rs, &ws);
      if (rs) pos_run[rk++] = i;
      if (ws) pos_win[wk++] = i;
    }
  }
  if (threadIdx.x == 0) {
    pos_run[nruns] = n;
    pos_win[nwin] = n;
  }
  for (uint32_t j = threadIdx.x; j < nwin; j += T) wbest[j] = 0ull;
  __syncthreads();
  {
    uint32_t rk = static_cast<uint32_t>(pre), wk = static_cast<uint32_t>(pre >> 32);
    for (uint32_t i = i0; i < i1; ++i) {
      bool rs, ws;
      starts(i, &rs, &ws);
      wk += ws ? 1u : 0u;
      if (rs) {
        const uint32_t w = wk - 1;  // the window holding this run
        const uint32_t len = pos_run[rk + 1] - i, at = i - pos_win[w];
        atomicMax(&wbest[w], (static_cast<unsigned long long>(len) << 32) | (0xffffffffu - at));
        ++rk;
      }
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < nwin; j += T) {
    const uint32_t at = 0xffffffffu - static_cast<uint32_t>(wbest[j] & 0xffffffffull);
    a.wkey[base + j] = keys[pos_win[j] + at];
    a.whits[base + j] = pos_win[j + 1] - pos_win[j];
  }
  if (threadIdx.x == 0) s_nw = nwin;
  __syncthreads();
  filter_finish(a, rr, keys, s_nw);
}

// the end of a read's filter once its nw windows have their key and hits: the
// max_cands cut (keys: work space of at least the power of two of nw), the
// window clamping and the window count
__device__ void filter_finish(const FilterArgs& a, uint32_t rr, uint64_t* keys, uint32_t nw) {
  const uint32_t r = a.r0 + rr;
  const uint64_t base = a.off[rr];
  const uint32_t m = static_cast<uint32_t>(a.read_off[r + 1] - a.read_off[r]);
  if (a.max_cands && nw > a.max_cands) {
    // keep the max_cands windows with most hits (ties: smaller key), in key order
    const uint32_t P2 = pow2_at_least(nw);
    for (uint32_t i = threadIdx.x; i < P2; i += blockDim.x)
      keys[i] = i < nw ? (static_cast<uint64_t>(0xffffffffu - a.whits[base + i]) << 32) | i : kNoKey;
    __syncthreads();
    bitonic(keys, P2);
    for (uint32_t i = threadIdx.x; i < P2; i += blockDim.x)
      keys[i] = i < a.max_cands ? (keys[i] & 0xffffffffull) : kNoKey;
    __syncthreads();
    bitonic(keys, P2);
    if (threadIdx.x == 0) {
      for (uint32_t j = 0; j < a.max_cands; ++j) {
        const uint32_t src = static_cast<uint32_t>(keys[j]);
        a.wkey[base + j] = a.wkey[base + src];
        a.whits[base + j] = a.whits[base + src];
      }
    }
    nw = a.max_cands;
    __syncthreads();
  }
  for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) window_clamp(a, base, m, i);
  if (threadIdx.x == 0) a.nwin[rr] = nw;
  __syncthreads();
}

// window i of the read at base: [cal - pad, cal + m + pad) clamped to the reference
__device__ __forceinline__ void window_clamp(const FilterArgs& a, uint64_t base, uint32_t m, uint32_t i) {
  const uint64_t key = a.wkey[base + i];
  const uint32_t ref = static_cast<uint32_t>(key >> 60);
  const int64_t cal = static_cast<int64_t>(key & kCalMask) - static_cast<int64_t>(kCalBias);
  const int64_t N = static_cast<int64_t>(a.di.ref_len[ref]);
  int64_t lo = cal - static_cast<int64_t>(a.pad), hi = cal + m + static_cast<int64_t>(a.pad);
  if (lo < 0) lo = 0;
  if (hi > N) hi = N;
  a.wlen[base + i] = static_cast<uint32_t>(hi - lo);
  // the key's ref and strand bits stay for the compaction; the start replaces the CAL
  a.wkey[base + i] = (key & ~kCalMask) | static_cast<uint64_t>(lo);
}

// The same filter for a read of at most 32 E CALs on one warp, without block
// barriers: element e = 32 h + lane of the warp's E registers per lane.  A
// bitonic network sorts the keys (partners in other lanes by shuffle, in the
// same lane by register); run and window starts become ballot masks; each run
// offers (its length, its position in its window) to its window by an atomic
// max in shared memory; the max_cands cut keeps the windows of rank below it
// (most hits first, then the smaller key), in key order.
constexpr int kFilterWarps = 8;
template <int E>
__global__ void __launch_bounds__(32 * kFilterWarps) k_cal_filter_warp(FilterArgs a, uint32_t lo, uint32_t hi) {
  constexpr int P = 32 * E;
  __shared__ uint64_t sk_s[kFilterWarps][P];                 // sorted keys
  __shared__ unsigned long long sb_s[kFilterWarps][P];       // per window: (run length << 32) | ~position
  __shared__ uint32_t sp_s[kFilterWarps][P + 1];             // window starts, then n
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  uint64_t* sk = sk_s[wi];
  unsigned long long* sb = sb_s[wi];
  uint32_t* sp = sp_s[wi];
  const uint32_t le = (2u << lane) - 1u;  // lanes at or below this one (lane 31: all)
  for (uint32_t rr = blockIdx.x * kFilterWarps + wi; rr < a.nr; rr += gridDim.x * kFilterWarps) {
    const uint32_t c = a.count[rr];
    if (c < lo || c > hi) continue;
    const uint32_t n = a.actual[rr];
    const uint32_t r = a.r0 + rr;
    const uint64_t base = a.off[rr];
    const uint32_t m = static_cast<uint32_t>(a.read_off[r + 1] - a.read_off[r]);
    uint64_t k[E];
#pragma unroll
    for (int h = 0; h < E; ++h) {
      const uint32_t e = 32 * h + lane;
      k[h] = e < n ? a.cals[base + e] : kNoKey;
    }
    // bitonic sort, ascending: the lower index of a pair keeps the minimum in
    // ascending runs ((e & size) == 0), the maximum in descending ones
#pragma unroll
    for (int size = 2; size <= P; size <<= 1) {
#pragma unroll
      for (int stride = size / 2; stride > 0; stride >>= 1) {
        if (stride >= 32) {
          const int hs = stride / 32;
#pragma unroll
          for (int h = 0; h < E; ++h) {
            if (h & hs) continue;
            const uint32_t e = 32 * h + lane;
            const bool up = (e & size) == 0;
            const uint64_t x = k[h], y = k[h | hs];
            if ((x > y) == up) {
              k[h] = y;
              k[h | hs] = x;
            }
          }
        } else {
#pragma unroll
          for (int h = 0; h < E; ++h) {
            const uint32_t e = 32 * h + lane;
            const uint64_t y = __shfl_xor_sync(FULL, k[h], stride);
            const bool up = (e & size) == 0, low = (lane & stride) == 0;
            k[h] = (low == up) ? (k[h] < y ? k[h] : y) : (k[h] > y ? k[h] : y);
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < E; ++h) sk[32 * h + lane] = k[h];
    __syncwarp();
    // run starts (value changes) and window starts ((ref, strand) changes or a
    // gap over merge_dist), as masks of the E groups of 32 elements
    uint32_t rm[E], wm[E];
    uint32_t nwin = 0;
#pragma unroll
    for (int h = 0; h < E; ++h) {
      const uint32_t e = 32 * h + lane;
      bool rs = false, ws = false;
      if (e < n) {
        if (e == 0) {
          rs = ws = true;
        } else {
          const uint64_t p = sk[e - 1];
          rs = k[h] != p;
          ws = (k[h] >> 59) != (p >> 59) || k[h] - p > a.merge_dist;
        }
      }
      rm[h] = __ballot_sync(FULL, rs);
      wm[h] = __ballot_sync(FULL, ws);
      nwin += __popc(wm[h]);
    }
    for (uint32_t j = lane; j < nwin; j += 32) sb[j] = 0ull;
    __syncwarp();
    uint32_t wbefore = 0;  // window starts in the groups before h
#pragma unroll
    for (int h = 0; h < E; ++h) {
      const uint32_t e = 32 * h + lane;
      if ((wm[h] >> lane) & 1u) sp[wbefore + __popc(wm[h] & (le >> 1))] = e;
      if ((rm[h] >> lane) & 1u) {
        // the window holding this run, the next run start, this run's window start
        const uint32_t w = wbefore + __popc(wm[h] & le) - 1u;
        uint32_t next = n;
        const uint32_t above = rm[h] & ~le;
        if (above) {
          next = 32 * h + __ffs(above) - 1;
        } else {
#pragma unroll
          for (int h2 = E - 1; h2 > h; --h2)
            if (rm[h2]) next = 32 * h2 + __ffs(rm[h2]) - 1;
        }
        uint32_t wst = 0;
        const uint32_t below = wm[h] & le;
        if (below) {
          wst = 32 * h + 31 - __clz(below);
        } else {
#pragma unroll
          for (int h2 = 0; h2 < h; ++h2)
            if (wm[h2]) wst = 32 * h2 + 31 - __clz(wm[h2]);
        }
        atomicMax(&sb[w], (static_cast<unsigned long long>(next - e) << 32) | (0xffffffffu - (e - wst)));
      }
      wbefore += __popc(wm[h]);
    }
    if (lane == 0) sp[nwin] = n;
    __syncwarp();
    // windows kept (all, or the max_cands of rank below it) in key order, each
    // clamped to [cal - pad, cal + m + pad) within its reference
    const bool cut = a.max_cands && nwin > a.max_cands;
    uint32_t kept_before = 0;
    for (uint32_t j0 = 0; j0 < nwin; j0 += 32) {
      const uint32_t j = j0 + lane;
      const bool in = j < nwin;
      const uint32_t hits = in ? sp[j + 1] - sp[j] : 0u;
      bool keep = in;
      if (cut && in) {
        uint32_t rank = 0;
        for (uint32_t q = 0; q < nwin; ++q) {
          const uint32_t hq = sp[q + 1] - sp[q];
          rank += (hq > hits || (hq == hits && q < j)) ? 1u : 0u;
        }
        keep = rank < a.max_cands;
      }
      const uint32_t km = __ballot_sync(FULL, keep);
      if (keep) {
        const uint32_t dst = kept_before + __popc(km & (le >> 1));
        const uint32_t at = 0xffffffffu - static_cast<uint32_t>(sb[j] & 0xffffffffull);
        const uint64_t key = sk[sp[j] + at];
        const uint32_t ref = static_cast<uint32_t>(key >> 60);
        const int64_t cal = static_cast<int64_t>(key & kCalMask) - static_cast<int64_t>(kCalBias);
        const int64_t N = static_cast<int64_t>(a.di.ref_len[ref]);
        int64_t wlo = cal - static_cast<int64_t>(a.pad), whi = cal + m + static_cast<int64_t>(a.pad);
        if (wlo < 0) wlo = 0;
        if (whi > N) whi = N;
        a.wkey[base + dst] = (key & ~kCalMask) | static_cast<uint64_t>(wlo);
        a.whits[base + dst] = hits;
        a.wlen[base + dst] = static_cast<uint32_t>(whi - wlo);
      }
      kept_before += __popc(km);
    }
    if (lane == 0) a.nwin[rr] = kept_before;
    __syncwarp();
  }
}

// reads with lo <= count <= hi, keys in shared memory
__global__ void __launch_bounds__(256) k_cal_filter(FilterArgs a, uint32_t lo, uint32_t hi) {
  extern __shared__ uint64_t skeys[];
  for (uint32_t rr = blockIdx.x; rr < a.nr; rr += gridDim.x) {
    const uint32_t n = a.count[rr];
    if (n < lo || n > hi) continue;
    filter_read(a, rr, skeys, a.actual[rr]);
  }
}

// one block per large read (big[b]), keys in a global scratch from slot soff[b]
// reads of more than kCalSmemKeys CALs, one block each, once the large-read
// merge below has given them their windows: the max_cands cut where it applies
// (the merge has clamped the windows of the others)
__global__ void __launch_bounds__(1024) k_cal_filter_big(FilterArgs a, const uint32_t* big, const uint64_t* soff,
                                                         uint64_t* scratch) {
  const uint32_t rr = big[blockIdx.x];
  const uint32_t nw = a.nwin[rr];
  if (!(a.max_cands && nw > a.max_cands)) return;
  filter_finish(a, rr, scratch + soff[blockIdx.x], nw);
}

// The large-read sort: the keys of every large read (a power of two of them
// with kNoKey padding, at least one tile) bitonic-sorted by many blocks at once.
// A block takes one tile of kSortTile keys: stages with strides below a tile
// run in shared memory, those of a tile or more as passes over global memory
// (one block per tile of lower partners); each compare-exchange sorts up where
// its lower index has bit `size` clear, the order of one whole bitonic network.
constexpr uint32_t kSortTile = kCalSortTile;

__device__ __forceinline__ uint32_t big_sort_len(const FilterArgs& a, uint32_t rr) {
  const uint32_t P = pow2_at_least(a.actual[rr]);
  return P > kSortTile ? P : kSortTile;
}

// The large reads in classes of equal sort length, longest first, so that a
// pass over the tiles of the reads at least `size` long covers a prefix of the
// tiles: perm lists the reads (indices into big) class by class.
constexpr int kSortLgMin = 12;    // log2 kSortTile
constexpr int kSortClasses = 20;  // sort lengths 2^12 .. 2^31
static_assert((1u << kSortLgMin) == kSortTile, "sort classes start at one tile");
struct SortClasses {
  uint32_t n;                     // classes present
  uint32_t lg[kSortClasses];      // log2 of their sort length, decreasing
  uint32_t read0[kSortClasses];   // position of their first read in perm
  uint32_t count[kSortClasses];   // their reads
  uint64_t tile0[kSortClasses];   // their first tile
};

__device__ __forceinline__ uint32_t sort_lg(const FilterArgs& a, uint32_t rr) {
  return 31u - static_cast<uint32_t>(__clz(big_sort_len(a, rr)));
}

__global__ void k_bsort_hist(FilterArgs a, const uint32_t* big, uint32_t n_big, uint32_t* hist) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n_big) atomicAdd(&hist[sort_lg(a, big[b]) - kSortLgMin], 1u);
}

__global__ void k_bsort_order(FilterArgs a, const uint32_t* big, uint32_t n_big, SortClasses c, uint32_t* fill,
                              uint32_t* perm) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_big) return;
  const uint32_t lg = sort_lg(a, big[b]);
  for (uint32_t ci = 0; ci < c.n; ++ci)
    if (c.lg[ci] == lg) perm[c.read0[ci] + atomicAdd(&fill[ci], 1u)] = b;
}

// the large read (index into big) and tile of this block
__device__ __forceinline__ bool sort_tile(const SortClasses& c, const uint32_t* perm, uint32_t* b, uint32_t* ti,
                                          uint32_t* P) {
  const uint64_t t = blockIdx.x;
  for (uint32_t ci = 0; ci < c.n; ++ci) {
    const uint32_t tpr = 1u << (c.lg[ci] - kSortLgMin);  // tiles per read
    if (t < c.tile0[ci] + static_cast<uint64_t>(c.count[ci]) * tpr) {
      const uint64_t x = t - c.tile0[ci];
      *b = perm[c.read0[ci] + static_cast<uint32_t>(x >> (c.lg[ci] - kSortLgMin))];
      *ti = static_cast<uint32_t>(x & (tpr - 1u));
      *P = 1u << c.lg[ci];
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ void cmp_swap(uint64_t& x, uint64_t& y, bool up) {
  if ((x > y) == up) {
    const uint64_t t = x;
    x = y;
    y = t;
  }
}

// all stages of sizes 2 .. kSortTile, each tile in shared memory, from the CALs into the scratch
__global__ void __launch_bounds__(1024) k_bsort_local(FilterArgs a, const uint32_t* big, const uint64_t* soff,
                                                      SortClasses c, const uint32_t* perm, uint64_t* scratch) {
  __shared__ uint64_t sk[kSortTile];
  uint32_t b, ti, P;
  if (!sort_tile(c, perm, &b, &ti, &P)) return;
  const uint32_t rr = big[b], n = a.actual[rr];
  const uint64_t base = a.off[rr];
  const uint32_t g0 = ti * kSortTile;
  for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x)
    sk[i] = g0 + i < n ? a.cals[base + g0 + i] : kNoKey;
  __syncthreads();
  for (uint32_t size = 2; size <= kSortTile; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t p = threadIdx.x; p < kSortTile / 2; p += blockDim.x) {
        const uint32_t lo = 2 * p - (p & (stride - 1));
        cmp_swap(sk[lo], sk[lo + stride], ((g0 + lo) & size) == 0);
      }
      __syncthreads();
    }
  }
  uint64_t* keys = scratch + soff[b];
  for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x) keys[g0 + i] = sk[i];
}

// one stage of size `size` and a stride of a tile or more, over global memory
__global__ void __launch_bounds__(1024) k_bsort_global(FilterArgs a, const uint32_t* big, const uint64_t* soff,
                                                       SortClasses c, const uint32_t* perm, uint64_t* scratch,
                                                       uint32_t size, uint32_t stride) {
  uint32_t b, ti, P;
  if (!sort_tile(c, perm, &b, &ti, &P)) return;
  const uint32_t g0 = ti * kSortTile;
  if (P < size || (g0 & stride)) return;  // sorted already, or an upper partner
  uint64_t* keys = scratch + soff[b];
  for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x) {
    const uint32_t lo = g0 + i;
    uint64_t x = keys[lo], y = keys[lo + stride];
    const bool up = (lo & size) == 0;
    if ((x > y) == up) {
      keys[lo] = y;
      keys[lo + stride] = x;
    }
  }
}

// the stages of size `size` with strides below a tile, each tile in shared memory
__global__ void __launch_bounds__(1024) k_bsort_tail(FilterArgs a, const uint32_t* big, const uint64_t* soff,
                                                     SortClasses c, const uint32_t* perm, uint64_t* scratch,
                                                     uint32_t size) {
  __shared__ uint64_t sk[kSortTile];
  uint32_t b, ti, P;
  if (!sort_tile(c, perm, &b, &ti, &P)) return;
  if (P < size) return;
  const uint32_t g0 = ti * kSortTile;
  uint64_t* keys = scratch + soff[b];
  for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x) sk[i] = keys[g0 + i];
  __syncthreads();
  const bool up = (g0 & size) == 0;  // size > kSortTile: one direction for the whole tile
  for (uint32_t stride = kSortTile / 2; stride > 0; stride >>= 1) {
    for (uint32_t p = threadIdx.x; p < kSortTile / 2; p += blockDim.x) {
      const uint32_t lo = 2 * p - (p & (stride - 1));
      cmp_swap(sk[lo], sk[lo + stride], up);
    }
    __syncthreads();
  }
  for (uint32_t i = threadIdx.x; i < kSortTile; i += blockDim.x) keys[g0 + i] = sk[i];
}

__global__ void k_cal_compact(uint32_t nr, const uint64_t* off, const uint32_t* nwin, const uint32_t* woff,
                              const uint64_t* wkey, const uint32_t* whits, const uint32_t* wlen,
                              uint8_t* o_ref, uint8_t* o_strand, uint64_t* o_start, uint32_t* o_len,
                              uint32_t* o_hits) {
  const uint32_t rr = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (rr >= nr) return;
  const uint64_t base = off[rr];
  const uint32_t d0 = woff[rr];
  for (uint32_t i = lane; i < nwin[rr]; i += 32) {
    const uint64_t key = wkey[base + i];
    o_ref[d0 + i] = static_cast<uint8_t>(key >> 60);
    o_strand[d0 + i] = static_cast<uint8_t>((key >> 59) & 1u);
    o_start[d0 + i] = key & kCalMask;
    o_len[d0 + i] = wlen[base + i];
    o_hits[d0 + i] = whits[base + i];
  }
}

}  // namespace

int launch_cal_slots(const uint64_t* read_off, uint32_t n, int k, uint32_t stride, int n_refs, uint32_t* slots,
                     uint32_t* status, cudaStream_t st) {
  if (n == 0) return 0;
  k_cal_slots<<<(n + 255) / 256, 256, 0, st>>>(read_off, n, k, stride, n_refs, slots, status);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// one thread per bucket: its head from jptr and key16 / key (the layout at DevIndex)
__global__ void k_cal_heads(DevIndex di, uint64_t nb, uint4* heads) {
  const uint64_t b = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (b >= nb) return;
  const int R = di.n_refs;
  const uint32_t s0 = di.jptr[b * R], e0 = di.jptr[(b + 1) * R];
  const uint32_t s1 = R > 1 ? di.jptr[b * R + 1] : 0u, e1 = R > 1 ? di.jptr[(b + 1) * R + 1] : 0u;
  const uint64_t n0 = e0 - s0, n1 = e1 - s1;
  uint32_t w[16];
  for (int i = 0; i < 16; ++i) w[i] = 0;
  w[0] = s0;
  w[1] = s1;
  if (di.key_bits == 16 && n0 + n1 <= static_cast<uint64_t>(kHeadKeys)) {
    w[2] = static_cast<uint32_t>(n0 | (n1 << 16));
    for (uint32_t i = 0; i < n0 + n1; ++i) {
      const uint32_t kk = i < n0 ? di.key16[0][s0 + i] : di.key16[1][s1 + (i - n0)];
      w[3 + (i >> 1)] |= kk << (16 * (i & 1));
    }
  } else if (di.key_bits != 16 && n0 + n1 <= static_cast<uint64_t>(kHeadKeys32)) {
    w[2] = static_cast<uint32_t>(n0 | (n1 << 16));
    for (uint32_t i = 0; i < n0 + n1; ++i) w[3 + i] = i < n0 ? di.key[0][s0 + i] : di.key[1][s1 + (i - n0)];
  } else {
    w[2] = kHeadSpill;
  }
  for (int j = 0; j < 4; ++j) heads[b * 4 + j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
}

int launch_cal_heads(const DevIndex& di, uint64_t nbuckets, uint4* heads, cudaStream_t st) {
  if (!di.packed || di.n_refs < 1 || di.n_refs > 2) return -1;
  if (nbuckets == 0) return 0;
  k_cal_heads<<<static_cast<unsigned>((nbuckets + 255) / 256), 256, 0, st>>>(di, nbuckets, heads);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Emit pass of the large reads whose lookups were kept, by many blocks per read.
// Their count bound is exact: a matching entry gives one CAL, two (the '+' one,
// then the '-' one) when the seed is its own reverse complement.  So a CAL's
// slot follows from the prefix of the CAL counts of the read's records (seed x
// reference, in order), and each block takes kEmitChunk consecutive slots of
// one read: it scans the read's records in shared memory, finds each slot's
// record by binary search and writes the CAL of that entry.
constexpr uint32_t kEmitChunk = 8192;
constexpr uint32_t kEmitRecs = static_cast<uint32_t>(kMaxReadLen) * kMaxRefs;

__global__ void k_emit_count(const uint32_t* bound, const uint32_t* big, uint32_t n_big, uint32_t* chunks) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n_big) chunks[b] = (bound[big[b]] + kEmitChunk - 1) / kEmitChunk;
}

__global__ void __launch_bounds__(512) k_cal_emit_big(SeedArgs a, const uint32_t* big, uint32_t n_big,
                                                      const uint64_t* cpre) {
  __shared__ uint32_t spre[kEmitRecs + 1];
  uint32_t b, ci;
  if (!block_item(cpre, n_big, &b, &ci)) return;
  const uint32_t rr = big[b], r = a.r0 + rr;
  if (a.recount[r - a.rbase]) return;  // looked up again and emitted by k_cal_seeds
  const uint32_t m = static_cast<uint32_t>(a.read_off[r + 1] - a.read_off[r]);
  const int k = a.di.k;
  const uint32_t nref = static_cast<uint32_t>(a.di.n_refs);
  const uint32_t nrec = ((m - k) / a.stride + 1) * nref;  // the read has CALs, so m >= k
  const uint64_t* rec = a.ranges + a.seed_off[r - a.rbase];
  // exclusive prefix of the records' CAL counts
  const uint32_t per = (nrec + blockDim.x - 1) / blockDim.x, q0 = min(nrec, threadIdx.x * per),
                 q1 = min(nrec, q0 + per);
  uint64_t sum = 0;
  for (uint32_t q = q0; q < q1; ++q) {
    const uint64_t x = rec[q];
    sum += ((x >> 2) & kRangeCntMax) << ((x & 3u) == 3u ? 1 : 0);
  }
  uint64_t tot = 0;
  uint64_t pre = block_exscan(sum, &tot);
  for (uint32_t q = q0; q < q1; ++q) {
    spre[q] = static_cast<uint32_t>(pre);
    const uint64_t x = rec[q];
    pre += ((x >> 2) & kRangeCntMax) << ((x & 3u) == 3u ? 1 : 0);
  }
  if (threadIdx.x == 0) spre[nrec] = static_cast<uint32_t>(tot);
  __syncthreads();
  const uint32_t s1 = min(static_cast<uint32_t>(tot), (ci + 1) * kEmitChunk);
  const uint64_t base = a.off[rr];
  for (uint32_t sl = ci * kEmitChunk + threadIdx.x; sl < s1; sl += blockDim.x) {
    uint32_t lo = 0, hi = nrec;  // the last record whose first slot is <= sl (it has CALs)
    while (lo + 1 < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (spre[mid] <= sl) lo = mid;
      else hi = mid;
    }
    const uint64_t x = rec[lo];
    const uint32_t rori = static_cast<uint32_t>(x & 3u), u = sl - spre[lo];
    const bool two = rori == 3u;
    const uint64_t e = (x >> 26) + (two ? u >> 1 : u);
    const uint32_t si = lo / nref, r2 = lo - si * nref, so = si * a.stride;
    const uint32_t po = a.di.packed ? a.di.posor[r2][e] : 0u;
    const uint32_t fo = a.di.packed ? po >> 30 : a.di.orient[r2][e];
    const int64_t p = a.di.packed ? static_cast<int64_t>(po & 0x3fffffffu) : static_cast<int64_t>(a.di.pos[r2][e]);
    const bool plus = two ? (u & 1u) == 0u : ((fo & 1u) && (rori & 1u)) || ((fo & 2u) && (rori & 2u));
    a.cals[base + sl] = plus ? cal_key(r2, 0, p - so) : cal_key(r2, 1, p - static_cast<int64_t>(m - so - k));
  }
}

int launch_cal_emit_big(const DevIndex& di, const uint64_t* read_off, uint32_t r0, uint32_t nr, uint32_t stride,
                        const uint32_t* bound, const uint64_t* off, uint64_t* cals, const CalRanges& kept,
                        const uint32_t* big, uint32_t n_big, uint64_t* scratch, uint64_t scratch_words,
                        cudaStream_t st) {
  if (nr == 0 || n_big == 0 || !kept.ranges) return 0;
  SeedArgs a{di, nullptr, read_off, r0, nr, stride, const_cast<uint32_t*>(bound), off, cals, nullptr, nullptr,
             kept.ranges, kept.seed_off, kept.recount, kept.rbase};
  uint32_t* chunks = reinterpret_cast<uint32_t*>(scratch + scratch_words);
  uint64_t* cpre = scratch + scratch_words + (n_big + 1) / 2 + 1;
  uint64_t* sums = cpre + n_big + 1;
  k_emit_count<<<(n_big + 255) / 256, 256, 0, st>>>(bound, big, n_big, chunks);
  if (launch_scan_u64(chunks, n_big, cpre, sums, st) < 0) return -1;
  // a large read's bound is at most the power of two of its scratch (3 of them per read)
  const uint32_t grid = static_cast<uint32_t>(scratch_words / (3ull * kEmitChunk)) + n_big + 1u;
  k_cal_emit_big<<<grid, 512, 0, st>>>(a, big, n_big, cpre);
  return cudaPeekAtLastError() == cudaSuccess ? 5 : -1;
}

int launch_cal_seeds(const DevIndex& di, const char* bases, const uint64_t* read_off, uint32_t r0, uint32_t nr,
                     uint32_t stride, uint32_t* count, const uint64_t* off, uint64_t* cals, uint32_t* actual,
                     uint32_t* status, const CalRanges& kept, cudaStream_t st) {
  if (nr == 0) return 0;
  SeedArgs a{di, bases, read_off, r0, nr, stride, count, off, cals, actual, status,
             kept.ranges, kept.seed_off, kept.recount, kept.rbase};
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t need = (nr + kCalWarps - 1) / kCalWarps;
  const uint32_t grid = need < static_cast<uint32_t>(nsm) * 32 ? need : static_cast<uint32_t>(nsm) * 32;
  if (cals) k_cal_seeds<true><<<grid, 32 * kCalWarps, 0, st>>>(a);
  else k_cal_seeds<false><<<grid, 32 * kCalWarps, 0, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// The large-read merge, over the sorted keys by the same tiles: run starts (the
// value changes) and window starts ((reference, strand) changes, or a gap over
// merge_dist) are counted per tile, numbered by scans over the tiles, and each
// run offers (its length, its position in its window) to its window by an
// atomic max: the rule of filter_read, by many blocks.  The layout of a read's
// work space is filter_read's (keys, window bests, run starts, window starts).
struct MergeTabs {
  uint32_t *trs, *tws;  // run and window starts per tile
  uint64_t *prs, *pws;  // their exclusive prefixes over all tiles (tiles + 1 entries)
};

// this thread's four keys g0 + 4 t .. + 3 (those below n): run and window start bits
__device__ __forceinline__ uint32_t merge_flags(const uint64_t* K, uint32_t g0, uint32_t n, uint64_t md) {
  uint32_t f = 0;
  const uint32_t i0 = g0 + 4 * threadIdx.x;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const uint32_t i = i0 + u;
    if (i >= n) break;
    if (i == 0) {
      f |= 3u << (2 * u);
      continue;
    }
    const uint64_t k = K[i], p = K[i - 1];
    f |= ((k != p ? 1u : 0u) | (((k >> 59) != (p >> 59) || k - p > md) ? 2u : 0u)) << (2 * u);
  }
  return f;
}

__device__ __forceinline__ uint64_t merge_counts(uint32_t f) {
  uint64_t c = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) c += (static_cast<uint64_t>((f >> (2 * u + 1)) & 1u) << 32) | ((f >> (2 * u)) & 1u);
  return c;
}

__global__ void __launch_bounds__(1024) k_bmerge_count(FilterArgs a, const uint32_t* big, const uint64_t* soff,
                                                       SortClasses c, const uint32_t* perm, uint64_t* scratch,
                                                       MergeTabs t) {
  uint32_t b, ti, P;
  if (!sort_tile(c, perm, &b, &ti, &P)) return;
  const uint32_t rr = big[b];
  const uint32_t f = merge_flags(scratch + soff[b], ti * kSortTile, a.actual[rr], a.merge_dist);
  uint64_t tot = 0;
  block_exscan(merge_counts(f), &tot);
  if (threadIdx.x == 0) {
    t.trs[blockIdx.x] = static_cast<uint32_t>(tot);
    t.tws[blockIdx.x] = static_cast<uint32_t>(tot >> 32);
  }
}

// PASS 0: run and window starts written (window bests cleared), the read's
// ends and window count by its last tile; PASS 1: each run's offer to its window
template <int PASS>
__global__ void __launch_bounds__(1024) k_bmerge_pos(FilterArgs a, const uint32_t* big, const uint64_t* soff,
                                                     SortClasses c, const uint32_t* perm, uint64_t* scratch,
                                                     MergeTabs t) {
  uint32_t b, ti, P;
  if (!sort_tile(c, perm, &b, &ti, &P)) return;
  const uint32_t rr = big[b], n = a.actual[rr];
  uint64_t* K = scratch + soff[b];
  unsigned long long* wbest = reinterpret_cast<unsigned long long*>(K + P);
  uint32_t* pos_run = reinterpret_cast<uint32_t*>(K + 2 * P);
  uint32_t* pos_win = pos_run + P + 1;
  const uint32_t g0 = ti * kSortTile, t0 = blockIdx.x - ti;  // the read's tiles are consecutive
  const uint32_t f = merge_flags(K, g0, n, a.merge_dist);
  uint64_t tot = 0;
  const uint64_t pre = block_exscan(merge_counts(f), &tot);
  uint32_t rk = static_cast<uint32_t>(t.prs[blockIdx.x] - t.prs[t0]) + static_cast<uint32_t>(pre);
  uint32_t wk = static_cast<uint32_t>(t.pws[blockIdx.x] - t.pws[t0]) + static_cast<uint32_t>(pre >> 32);
  const uint32_t i0 = g0 + 4 * threadIdx.x;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const bool rs = (f >> (2 * u)) & 1u, ws = (f >> (2 * u + 1)) & 1u;
    const uint32_t i = i0 + u;
    if (PASS == 0) {
      if (rs) pos_run[rk++] = i;
      if (ws) {
        wbest[wk] = 0ull;
        pos_win[wk++] = i;
      }
    } else {
      wk += ws ? 1u : 0u;
      if (rs) {
        const uint32_t w = wk - 1;  // the window holding this run
        const uint32_t len = pos_run[rk + 1] - i, at = i - pos_win[w];
        atomicMax(&wbest[w], (static_cast<unsigned long long>(len) << 32) | (0xffffffffu - at));
        ++rk;
      }
    }
  }
  if (PASS == 0 && threadIdx.x == 0 && ti == (P / kSortTile) - 1) {
    const uint32_t te = t0 + P / kSortTile;
    const uint32_t nruns = static_cast<uint32_t>(t.prs[te] - t.prs[t0]), nwin = static_cast<uint32_t>(t.pws[te] - t.pws[t0]);
    pos_run[nruns] = n;
    pos_win[nwin] = n;
    a.nwin[rr] = nwin;
  }
}

// each window's key (its most frequent CAL, the first of equally frequent) and
// hits; clamped here unless the max_cands cut (k_cal_filter_big) still applies
__global__ void __launch_bounds__(1024) k_bmerge_out(FilterArgs a, const uint32_t* big, const uint64_t* soff,
                                                     SortClasses c, const uint32_t* perm, uint64_t* scratch) {
  uint32_t b, ti, P;
  if (!sort_tile(c, perm, &b, &ti, &P)) return;
  const uint32_t rr = big[b], r = a.r0 + rr, nwin = a.nwin[rr];
  const uint64_t* K = scratch + soff[b];
  const unsigned long long* wbest = reinterpret_cast<const unsigned long long*>(K + P);
  const uint32_t* pos_win = reinterpret_cast<const uint32_t*>(K + 2 * P) + P + 1;
  const uint64_t base = a.off[rr];
  const uint32_t m = static_cast<uint32_t>(a.read_off[r + 1] - a.read_off[r]);
  const bool cut = a.max_cands && nwin > a.max_cands;
  for (uint32_t j = ti * kSortTile + threadIdx.x; j < min(nwin, (ti + 1) * kSortTile); j += blockDim.x) {
    const uint32_t at = 0xffffffffu - static_cast<uint32_t>(wbest[j] & 0xffffffffull);
    a.wkey[base + j] = K[pos_win[j] + at];
    a.whits[base + j] = pos_win[j + 1] - pos_win[j];
    if (!cut) window_clamp(a, base, m, j);
  }
}

int launch_cal_filter(const DevIndex& di, const uint64_t* read_off, uint32_t r0, uint32_t nr, uint32_t merge_dist,
                      uint32_t pad, uint32_t max_cands, const uint32_t* count, const uint32_t* actual,
                      const uint64_t* off, uint64_t* cals, uint32_t max_small, uint32_t max_mid, const uint32_t* big,
                      const uint64_t* big_soff, uint32_t n_big, uint64_t* scratch, uint64_t scratch_words,
                      uint32_t* nwin, uint64_t* wkey, uint32_t* whits, uint32_t* wlen, cudaStream_t st) {
  if (nr == 0) return 0;
  FilterArgs a{di, read_off, r0, nr, merge_dist, pad, max_cands, count, actual, off, cals, kCalSmemKeys,
               nwin, wkey, whits, wlen};
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_cal_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(cal_filter_words(kCalSmemKeys) * sizeof(uint64_t))) != cudaSuccess)
      return -1;
    attr = true;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  auto p2 = [](uint32_t n) {
    uint32_t p = 1;
    while (p < n) p <<= 1;
    return p;
  };
  int launched = 0;
  // reads of at most 64 and of 65-128 CALs: one warp each
  {
    const uint32_t warps = static_cast<uint32_t>(nsm) * 8 * kFilterWarps;
    const uint32_t grid = (std::min(nr, warps) + kFilterWarps - 1) / kFilterWarps;
    k_cal_filter_warp<2><<<grid, 32 * kFilterWarps, 0, st>>>(a, 0u, 64u);
    ++launched;
    if (max_small > 64) {
      k_cal_filter_warp<4><<<grid, 32 * kFilterWarps, 0, st>>>(a, 65u, 128u);
      ++launched;
    }
  }
  // the other small reads: 24 KB or less of shared memory per block, many blocks per SM
  if (max_small > 128) {
    const size_t smem = static_cast<size_t>(cal_filter_words(p2(max_small))) * sizeof(uint64_t);
    const uint32_t grid = nr < static_cast<uint32_t>(nsm) * 32 ? nr : static_cast<uint32_t>(nsm) * 32;
    k_cal_filter<<<grid, 128, smem, st>>>(a, 129u, kCalSmallKeys);
    ++launched;
  }
  if (max_mid) {
    const size_t smem = static_cast<size_t>(cal_filter_words(p2(max_mid))) * sizeof(uint64_t);
    const uint32_t grid = static_cast<uint32_t>(nsm) * 2;
    k_cal_filter<<<grid, 256, smem, st>>>(a, kCalSmallKeys + 1, kCalSmemKeys);
    ++launched;
  }
  if (n_big) {
    // the large reads' keys sorted by the whole GPU, then each read's windows by
    // one block; the reads' classes of sort length come back to the host, which
    // sizes each pass to the tiles of the reads it still has to sort
    uint32_t* hist = reinterpret_cast<uint32_t*>(scratch + scratch_words);
    uint32_t* fill = hist + kSortClasses;
    uint32_t* perm = fill + kSortClasses;
    uint32_t h[kSortClasses] = {};
    if (cudaMemsetAsync(hist, 0, 2 * kSortClasses * sizeof(uint32_t), st) != cudaSuccess) return -1;
    k_bsort_hist<<<(n_big + 255) / 256, 256, 0, st>>>(a, big, n_big, hist);
    if (cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return -1;
    SortClasses c{};
    uint32_t rank = 0;
    uint64_t tiles = 0;
    for (int lg = kSortLgMin + kSortClasses - 1; lg >= kSortLgMin; --lg) {
      const uint32_t cnt = h[lg - kSortLgMin];
      if (!cnt) continue;
      c.lg[c.n] = static_cast<uint32_t>(lg);
      c.read0[c.n] = rank;
      c.count[c.n] = cnt;
      c.tile0[c.n] = tiles;
      ++c.n;
      rank += cnt;
      tiles += static_cast<uint64_t>(cnt) << (lg - kSortLgMin);
    }
    // tiles of the reads at least `size` long: a prefix
    auto tiles_ge = [&](uint32_t size) {
      for (uint32_t ci = 0; ci < c.n; ++ci)
        if ((1ull << c.lg[ci]) < size) return c.tile0[ci];
      return tiles;
    };
    k_bsort_order<<<(n_big + 255) / 256, 256, 0, st>>>(a, big, n_big, c, fill, perm);
    k_bsort_local<<<static_cast<uint32_t>(tiles), 1024, 0, st>>>(a, big, big_soff, c, perm, scratch);
    launched += 3;
    const uint32_t pmax = c.n ? 1u << c.lg[0] : kSortTile;
    for (uint32_t size = 2 * kSortTile; size <= pmax && size != 0; size <<= 1) {
      const uint32_t grid = static_cast<uint32_t>(tiles_ge(size));
      for (uint32_t stride = size / 2; stride >= kSortTile; stride >>= 1, ++launched)
        k_bsort_global<<<grid, 1024, 0, st>>>(a, big, big_soff, c, perm, scratch, size, stride);
      k_bsort_tail<<<grid, 1024, 0, st>>>(a, big, big_soff, c, perm, scratch, size);
      ++launched;
    }
    // the merge by the same tiles, then the max_cands cut, one block per read that needs it
    const uint32_t nt = static_cast<uint32_t>(tiles);
    uint64_t* mt = scratch + scratch_words + kSortClasses + (n_big + 1) / 2 + 1;
    MergeTabs t{reinterpret_cast<uint32_t*>(mt), reinterpret_cast<uint32_t*>(mt) + nt, mt + nt + 1, nullptr};
    t.pws = t.prs + nt + 1;
    uint64_t* sums = t.pws + nt + 1;
    k_bmerge_count<<<nt, 1024, 0, st>>>(a, big, big_soff, c, perm, scratch, t);
    if (launch_scan_u64(t.trs, nt, t.prs, sums, st) < 0 || launch_scan_u64(t.tws, nt, t.pws, sums, st) < 0)
      return -1;
    k_bmerge_pos<0><<<nt, 1024, 0, st>>>(a, big, big_soff, c, perm, scratch, t);
    k_bmerge_pos<1><<<nt, 1024, 0, st>>>(a, big, big_soff, c, perm, scratch, t);
    k_bmerge_out<<<nt, 1024, 0, st>>>(a, big, big_soff, c, perm, scratch);
    k_cal_filter_big<<<n_big, 1024, 0, st>>>(a, big, big_soff, scratch);
    launched += 11;
  }
  return cudaPeekAtLastError() == cudaSuccess ? launched : -1;
}

__global__ void k_cal_offsets(const uint32_t* woff, uint32_t nr, uint64_t base, uint64_t* out) {
  const uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (i <= nr) out[i] = base + woff[i];
}

namespace {
constexpr int kScanBlock64 = 1024;

// per block: exclusive scan of the counts (64-bit), the block's total into sums
__global__ void __launch_bounds__(kScanBlock64) k_scan64_a(const uint32_t* in, uint32_t n, uint64_t* out,
                                                         uint64_t* sums) {
  __shared__ uint64_t sh[kScanBlock64];
  const uint32_t i = blockIdx.x * kScanBlock64 + threadIdx.x;
  const uint64_t v = i < n ? in[i] : 0u;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int d = 1; d < kScanBlock64; d <<= 1) {
    const uint64_t x = threadIdx.x >= static_cast<unsigned>(d) ? sh[threadIdx.x - d] : 0ull;
    __syncthreads();
    sh[threadIdx.x] += x;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == kScanBlock64 - 1) sums[blockIdx.x] = sh[threadIdx.x];
}

// one block: exclusive scan of the block totals in place, the total into *end
__global__ void __launch_bounds__(kScanBlock64) k_scan64_b(uint64_t* sums, uint32_t nb, uint64_t* end) {
  __shared__ uint64_t sh[kScanBlock64];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nb; b0 += kScanBlock64) {
    const uint32_t i = b0 + threadIdx.x;
    const uint64_t v = i < nb ? sums[i] : 0ull;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int d = 1; d < kScanBlock64; d <<= 1) {
      const uint64_t x = threadIdx.x >= static_cast<unsigned>(d) ? sh[threadIdx.x - d] : 0ull;
      __syncthreads();
      sh[threadIdx.x] += x;
      __syncthreads();
    }
    if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += sh[kScanBlock64 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *end = carry;
}

__global__ void k_scan64_c(uint64_t* out, uint32_t n, const uint64_t* sums) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[i / kScanBlock64];
}

// the filter's routing of reads by their CAL bounds (big: nullptr to take the
// maxima only)
__global__ void k_cal_route(const uint32_t* count, uint32_t nr, uint32_t* big, uint64_t* big_soff, CalPlan* plan) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t c = i < nr ? count[i] : 0u;
  uint32_t small = 0, mid = 0;
  if (i < nr) {
    if (c > kCalSmemKeys) {
      if (big) {
        const uint32_t b = atomicAdd(&plan->n_big, 1u);
        big[b] = i;
        big_soff[b] = atomicAdd(&plan->scratch, static_cast<unsigned long long>(cal_filter_words(pow2_at_least(c))));
      }
    } else if (c > kCalSmallKeys) {
      mid = c;
    } else {
      small = c;
    }
  }
  const uint32_t all = __reduce_max_sync(FULL, c);
  small = __reduce_max_sync(FULL, small);
  mid = __reduce_max_sync(FULL, mid);
  if ((threadIdx.x & 31) == 0) {
    if (small) atomicMax(&plan->max_small, small);
    if (mid) atomicMax(&plan->max_mid, mid);
    if (all) atomicMax(&plan->max_all, all);
  }
}

// bounds[p / span] = the first read whose prefix p = pre[r] falls in that span
__global__ void k_cal_bounds(const uint64_t* pre, uint32_t nr, uint64_t span, uint32_t* bounds) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nr) return;
  const uint64_t j = pre[r] / span;
  if (r == 0 || pre[r - 1] / span != j) bounds[j] = r;
}

// out[i] = pre[a + i] - pre[a], i = 0 .. cnt, 64- or 32-bit
__global__ void k_cal_rebase(const uint64_t* pre, uint32_t a, uint32_t cnt, uint64_t* out64, uint32_t* out32) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > cnt) return;
  const uint64_t v = pre[a + i] - pre[a];
  if (out64) out64[i] = v;
  else out32[i] = static_cast<uint32_t>(v);
}
}  // namespace

int launch_scan_u64(const uint32_t* in, uint32_t n, uint64_t* out, uint64_t* sums, cudaStream_t st) {
  const uint32_t nb = (n + kScanBlock64 - 1) / kScanBlock64;
  if (nb) k_scan64_a<<<nb, kScanBlock64, 0, st>>>(in, n, out, sums);
  k_scan64_b<<<1, kScanBlock64, 0, st>>>(sums, nb, out + n);
  if (nb) k_scan64_c<<<(n + 255) / 256, 256, 0, st>>>(out, n, sums);
  return cudaPeekAtLastError() == cudaSuccess ? 3 : -1;
}

int launch_cal_route(const uint32_t* count, uint32_t nr, uint32_t* big, uint64_t* big_soff, CalPlan* plan,
                     cudaStream_t st) {
  if (nr == 0) return 0;
  k_cal_route<<<(nr + 255) / 256, 256, 0, st>>>(count, nr, big, big_soff, plan);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_cal_bounds(const uint64_t* pre, uint32_t nr, uint64_t span, uint32_t* bounds, cudaStream_t st) {
  if (nr == 0) return 0;
  k_cal_bounds<<<(nr + 255) / 256, 256, 0, st>>>(pre, nr, span, bounds);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_cal_rebase(const uint64_t* pre, uint32_t a, uint32_t cnt, uint64_t* out64, uint32_t* out32,
                      cudaStream_t st) {
  k_cal_rebase<<<(cnt + 256) / 256, 256, 0, st>>>(pre, a, cnt, out64, out32);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_cal_offsets(const uint32_t* woff, uint32_t nr, uint64_t base, uint64_t* out, cudaStream_t st) {
  k_cal_offsets<<<(nr + 256) / 256, 256, 0, st>>>(woff, nr, base, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_cal_compact(uint32_t nr, const uint64_t* off, const uint32_t* nwin, const uint32_t* woff,
                       const uint64_t* wkey, const uint32_t* whits, const uint32_t* wlen, uint8_t* o_ref,
                       uint8_t* o_strand, uint64_t* o_start, uint32_t* o_len, uint32_t* o_hits, cudaStream_t st) {
  if (nr == 0) return 0;
  k_cal_compact<<<(nr + 7) / 8, 256, 0, st>>>(nr, off, nwin, woff, wkey, whits, wlen, o_ref, o_strand, o_start,
                                             o_len, o_hits);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int preload_cal() {
  int n_ = 0;
  SR_TOUCH(k_cal_slots);
  SR_TOUCH(k_cal_heads);
  SR_TOUCH(k_cal_seeds<false>);
  SR_TOUCH(k_cal_seeds<true>);
  SR_TOUCH(k_cal_filter);
  SR_TOUCH(k_cal_filter_big);
  SR_TOUCH(k_emit_count);
  SR_TOUCH(k_cal_emit_big);
  SR_TOUCH(k_bmerge_count);
  SR_TOUCH(k_bmerge_pos<0>);
  SR_TOUCH(k_bmerge_pos<1>);
  SR_TOUCH(k_bmerge_out);
  SR_TOUCH(k_bsort_hist);
  SR_TOUCH(k_bsort_order);
  SR_TOUCH(k_bsort_local);
  SR_TOUCH(k_bsort_global);
  SR_TOUCH(k_bsort_tail);
  SR_TOUCH(k_cal_filter_warp<2>);
  SR_TOUCH(k_cal_filter_warp<4>);
  SR_TOUCH(k_cal_compact);
  SR_TOUCH(k_cal_offsets);
  SR_TOUCH(k_scan64_a);
  SR_TOUCH(k_scan64_b);
  SR_TOUCH(k_scan64_c);
  SR_TOUCH(k_cal_route);
  SR_TOUCH(k_cal_bounds);
  SR_TOUCH(k_cal_rebase);
  return n_;
}

}  // namespace sr
