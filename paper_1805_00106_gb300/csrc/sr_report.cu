// sr_report.cu -- the score tracker's report options (McVicar et al., arXiv
// 1805.00106, Sec. 4.2: the single highest-scoring CAL, some number of the
// highest-scoring CALs, or all CALs tied for the highest score).
//
// One warp per read picks, round by round, the next window in the winner order
// (score descending, then reference, reference end, strand, candidate index)
// that ranks after the previous pick and whose (reference, end, strand) is not
// yet reported; a count pass, an exclusive scan of the counts and a write pass
// give the compacted per-read lists.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kRepWarps = 4;
constexpr int kRepMax = static_cast<int>(SR_REPORT_MAX);
constexpr int kScanBlock = 1024;

struct Cand {
  int32_t score;
  uint32_t ref, strand, item;
  uint64_t gend;
};

// a ranks before b in the winner order
__device__ __forceinline__ bool before(const Cand& a, const Cand& b) {
  if (a.score != b.score) return a.score > b.score;
  if (a.ref != b.ref) return a.ref < b.ref;
  if (a.gend != b.gend) return a.gend < b.gend;
  if (a.strand != b.strand) return a.strand < b.strand;
  return a.item < b.item;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int off) {
  Cand o;
  o.score = __shfl_xor_sync(FULL, c.score, off);
  o.ref = __shfl_xor_sync(FULL, c.ref, off);
  o.strand = __shfl_xor_sync(FULL, c.strand, off);
  o.item = __shfl_xor_sync(FULL, c.item, off);
  o.gend = __shfl_xor_sync(FULL, c.gend, off);
  return o;
}

struct RepArgs {
  uint32_t n_reads;
  const uint64_t* cand_off;
  const int32_t* item_score;
  const uint32_t* item_end;
  const uint8_t* c_ref;
  const uint8_t* c_strand;
  const uint64_t* c_start;
  const DevHit* hits;
  int slots;
  int kind;
  uint32_t n_best;
  uint32_t* count;          // count pass: entries per read
  const uint32_t* offsets;  // write pass: exclusive scan of count
  sr_report_hit* out;       // write pass
  uint32_t* truncated;
};

__global__ void __launch_bounds__(32 * kRepWarps) k_report(RepArgs a) {
  __shared__ uint64_t kg[kRepWarps][kRepMax];
  __shared__ uint32_t kr[kRepWarps][kRepMax];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool write = a.out != nullptr;
  for (uint64_t r = blockIdx.x * static_cast<uint64_t>(kRepWarps) + warp; r < a.n_reads;
       r += static_cast<uint64_t>(gridDim.x) * kRepWarps) {
    const DevHit h = a.hits[r * a.slots];
    const uint64_t c0 = a.cand_off[r], c1 = a.cand_off[r + 1];
    uint32_t limit;
    if (h.item < 0 || h.score <= 0) {
      limit = 0;
    } else if (a.kind == SR_REPORT_TIED) {
      limit = h.n_ties < static_cast<uint32_t>(kRepMax) ? h.n_ties : static_cast<uint32_t>(kRepMax);
      if (!write && lane == 0 && h.n_ties > static_cast<uint32_t>(kRepMax)) atomicAdd(a.truncated, 1u);
    } else {
      limit = a.n_best;
    }
    Cand prev{};
    uint32_t k = 0;
    for (; k < limit; ++k) {
      bool have = false;
      Cand best{};
      for (uint64_t c = c0 + lane; c < c1; c += 32) {
        Cand x;
        x.score = a.item_score[c];
        if (x.score <= 0 || (a.kind == SR_REPORT_TIED && x.score != h.score)) continue;
        x.ref = a.c_ref[c];
        x.strand = a.c_strand[c];
        x.item = static_cast<uint32_t>(c);
        x.gend = a.c_start[c] + a.item_end[c] - 1;
        if (k > 0 && !before(prev, x)) continue;
        bool dup = false;
        const uint32_t rs = (x.ref << 1) | x.strand;
        for (uint32_t u = 0; u < k && !dup; ++u) dup = kg[warp][u] == x.gend && kr[warp][u] == rs;
        if (dup) continue;
        if (!have || before(x, best)) {
          best = x;
          have = true;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const bool oh = __shfl_xor_sync(FULL, have, off);
        const Cand o = shfl_cand(best, off);
        if (oh && (!have || before(o, best))) {
          best = o;
          have = true;
        }
      }
      if (!have) break;
      if (lane == 0) {
        kg[warp][k] = best.gend;
        kr[warp][k] = (best.ref << 1) | best.strand;
        if (write) {
          sr_report_hit o;
          o.score = best.score;
          o.item = static_cast<int32_t>(best.item);
          o.ref_id = static_cast<uint8_t>(best.ref);
          o.strand = static_cast<uint8_t>(best.strand);
          o.reserved = 0;
          o.end_col = a.item_end[best.item];
          o.ref_end = best.gend;
          a.out[a.offsets[r] + k] = o;
        }
      }
      prev = best;
      __syncwarp();
    }
    if (!write && lane == 0) a.count[r] = k;
    __syncwarp();
  }
}

// exclusive scan of n counts into out[0..n] (out[n] = total), three passes
__global__ void __launch_bounds__(kScanBlock) k_scan_a(const uint32_t* in, uint32_t n, uint32_t* out,
                                                      uint32_t* sums) {
  __shared__ uint32_t sh[kScanBlock];
  const uint32_t i = blockIdx.x * kScanBlock + threadIdx.x;
  const uint32_t v = i < n ? in[i] : 0u;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    const uint32_t x = threadIdx.x >= static_cast<unsigned>(off) ? sh[threadIdx.x - off] : 0u;
    __syncthreads();
    sh[threadIdx.x] += x;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void __launch_bounds__(kScanBlock) k_scan_b(uint32_t* sums, uint32_t nb, uint32_t* total) {
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  __shared__ uint32_t sh[kScanBlock];
  for (uint32_t base = 0; base < nb; base += kScanBlock) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < nb ? sums[i] : 0u;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
      const uint32_t x = threadIdx.x >= static_cast<unsigned>(off) ? sh[threadIdx.x - off] : 0u;
      __syncthreads();
      sh[threadIdx.x] += x;
      __syncthreads();
    }
    if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += sh[kScanBlock - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_c(uint32_t* out, uint32_t n, const uint32_t* sums) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[i / kScanBlock];
}

}  // namespace

int launch_scan_u32(const uint32_t* in, uint32_t n, uint32_t* out, uint32_t* sums, cudaStream_t st) {
  const uint32_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (nb == 0) return cudaMemsetAsync(out, 0, 4, st) == cudaSuccess ? 0 : -1;
  k_scan_a<<<nb, kScanBlock, 0, st>>>(in, n, out, sums);
  k_scan_b<<<1, kScanBlock, 0, st>>>(sums, nb, out + n);
  k_scan_c<<<(n + 255) / 256, 256, 0, st>>>(out, n, sums);
  return cudaPeekAtLastError() == cudaSuccess ? 3 : -1;
}

// scratch: count n, offsets n + 1, sums n / 1024 + 1, one truncation counter
uint64_t report_scratch_words(uint32_t n_reads) {
  return 2ull * n_reads + 1 + n_reads / kScanBlock + 1 + 1;
}

int launch_report_count(const BatchDev& b, int n_refs, int kind, uint32_t n_best, uint32_t* scratch,
                        cudaStream_t st) {
  const uint32_t n = b.n_reads;
  uint32_t* count = scratch;
  uint32_t* offsets = scratch + n;
  uint32_t* sums = offsets + n + 1;
  uint32_t* trunc = sums + n / kScanBlock + 1;
  if (cudaMemsetAsync(trunc, 0, 4, st) != cudaSuccess) return -1;
  RepArgs a{n, b.cand_off, b.item_score, b.item_end, b.c_ref, b.c_strand, b.c_start, b.hits, 1 + n_refs,
            kind, n_best, count, nullptr, nullptr, trunc};
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t need = (static_cast<uint64_t>(n) + kRepWarps - 1) / kRepWarps;
  const uint32_t grid = static_cast<uint32_t>(need < static_cast<uint64_t>(nsm) * 16 ? (need ? need : 1) : nsm * 16);
  k_report<<<grid, 32 * kRepWarps, 0, st>>>(a);
  const int t = launch_scan_u32(count, n, offsets, sums, st);
  if (t < 0) return -1;
  return cudaPeekAtLastError() == cudaSuccess ? 1 + t : -1;
}

int launch_report_write(const BatchDev& b, int n_refs, int kind, uint32_t n_best, const uint32_t* scratch,
                        sr_report_hit* out, cudaStream_t st) {
  const uint32_t n = b.n_reads;
  RepArgs a{n, b.cand_off, b.item_score, b.item_end, b.c_ref, b.c_strand, b.c_start, b.hits, 1 + n_refs,
            kind, n_best, nullptr, scratch + n, out, nullptr};
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t need = (static_cast<uint64_t>(n) + kRepWarps - 1) / kRepWarps;
  const uint32_t grid = static_cast<uint32_t>(need < static_cast<uint64_t>(nsm) * 16 ? (need ? need : 1) : nsm * 16);
  k_report<<<grid, 32 * kRepWarps, 0, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int preload_report() {
  int n_ = 0;
  SR_TOUCH(k_report);
  SR_TOUCH(k_scan_a);
  SR_TOUCH(k_scan_b);
  SR_TOUCH(k_scan_c);
  return n_;
}

}  // namespace sr
