// sr_traceback.cu -- CIGAR of each read's winning window (McVicar et al.,
// arXiv 1805.00106: the reported alignment of Sec. 4.2 / SAM output, whose
// traceback the paper runs on the host, Sec. 6.4).
//
// Most winners are traced by k_tb_band (below), which needs the end row i*
// found by the extension kernel's winner mode.  Winners whose band is wider
// than 32 diagonals, and int32-class winners, use k_traceback: one warp per
// read recomputes the DP of the winning window in
// exact int32 over rows 1..m and columns 1..j* only (j* = the end column found
// by the extension kernels; cells right of j* cannot influence the path) with
// the same systolic sweep (8 rows per lane), and records per cell a 4-bit
// direction code in shared memory:
//   bit 0  E came from opening (H(i,j-1)-(go+ge) >= E(i,j-1)-ge)
//   bit 1  F came from opening (H(i-1,j)-(go+ge) >= F(i-1,j)-ge)
//   bit 2  H(i-1,j-1)+s >= E(i,j)
//   bit 3  max(H(i-1,j-1)+s, E(i,j)) >= F(i,j)
// Lane 0 then walks back from the end cell with the fixed priorities
// (diagonal, then E, then F; gap open before extend), tracking the exact cell
// value so it stops where H reaches 0.  The end row i* is the smallest row with
// H(i*, j*) equal to the score (final row in read-end-anchored mode).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kTbRows = 8;  // rows per lane (32 lanes x 8 = 256 rows)

__device__ __forceinline__ uint32_t base_at(const uint32_t* w, uint64_t p) {
  return (w[p >> 4] >> ((p & 15u) * 2u)) & 3u;
}

struct TbArgs {
  const uint32_t* rpack;
  const uint32_t* rlen;
  const uint8_t* c_ref;
  const uint8_t* c_strand;
  const uint64_t* c_start;
  const uint32_t* c_len;
  const uint32_t* item_read;
  const uint32_t* item_end;
  DevRefs refs;
  const uint32_t* item_iend;
  uint8_t* need_full;
  DevHit* hits;
  uint32_t* cigar_slots;
  uint32_t* status;
  uint32_t n_reads;
  int slots;
  int mode;
  int32_t sa, sb, go, ge;
};

__global__ void __launch_bounds__(32) k_traceback(TbArgs a, const uint32_t* list, const uint32_t* count_ptr) {
  extern __shared__ uint32_t dirs[];  // [j][lane], j < j*
  __shared__ uint8_t rcode[kMaxWinLen];
  __shared__ uint8_t qcode[kMaxReadLen];
  __shared__ uint8_t ops[kMaxReadLen + kMaxWinLen + 4];
  const int lane = threadIdx.x;
  const int32_t goe = a.go + a.ge;
  constexpr int32_t NEG = -(1 << 28);
  const uint32_t count = *count_ptr;
  for (uint32_t li = blockIdx.x; li < count; li += gridDim.x) {
    const uint32_t r = list[li];
    DevHit* hp = a.hits + static_cast<uint64_t>(r) * a.slots;
    const int32_t item = hp->item;
    const int32_t S = hp->score;
    const uint32_t rd = a.item_read[item];
    const uint32_t m = a.rlen[rd];
    const uint32_t strand = a.c_strand[item];
    const uint64_t ws = a.c_start[item];
    const uint32_t jstar = a.item_end[item];
    const uint32_t* ref = a.refs.words[a.c_ref[item]];
    const uint32_t* row = a.rpack + static_cast<uint64_t>(rd) * kReadWords;
    for (uint32_t j = lane; j < jstar; j += 32) rcode[j] = static_cast<uint8_t>(base_at(ref, ws + j));
    for (uint32_t i = lane; i < m; i += 32)
      qcode[i] = static_cast<uint8_t>(strand ? 3u - base_at(row, m - 1u - i) : base_at(row, i));
    __syncwarp();
    uint32_t qc[kTbRows];
#pragma unroll
    for (int k = 0; k < kTbRows; ++k) {
      const uint32_t i = lane * kTbRows + k;
      qc[k] = i < m ? qcode[i] : 4u;
    }
    int32_t H[kTbRows], E[kTbRows];
#pragma unroll
    for (int k = 0; k < kTbRows; ++k) {
      H[k] = 0;
      E[k] = NEG;
    }
    int32_t hprev = 0, Hbot = 0, Fbot = NEG;
    uint32_t icand = 0xffffffffu;  // smallest 1-based row with H(i, j*) == S
    const int nsteps = static_cast<int>(jstar) + 31;
    for (int s = 0; s < nsteps; ++s) {
      int32_t hin = __shfl_up_sync(FULL, Hbot, 1);
      int32_t fin = __shfl_up_sync(FULL, Fbot, 1);
      if (lane == 0) {
        hin = 0;
        fin = NEG;
      }
      const int j = s - lane;
      if (j >= 0 && j < static_cast<int>(jstar)) {
        const uint32_t rc = rcode[j];
        int32_t hd = hprev, hup = hin, f = fin;
        uint32_t word = 0;
#pragma unroll
        for (int k = 0; k < kTbRows; ++k) {
          const int32_t hl = H[k];
          const int32_t eo = hl - goe, ee = E[k] - a.ge;
          const uint32_t pe = eo >= ee;
          E[k] = max(eo, ee);
          const int32_t fo = hup - goe, fe = f - a.ge;
          const uint32_t pf = fo >= fe;
          f = max(fo, fe);
          const int32_t d = hd + (qc[k] == rc ? a.sa : -a.sb);
          const uint32_t px = d >= E[k];
          const int32_t x = max(d, E[k]);
          const uint32_t ph = x >= f;
          const int32_t h = max(max(x, f), 0);
          word |= (pe | (pf << 1) | (px << 2) | (ph << 3)) << (4 * k);
          hd = hl;
          H[k] = h;
          hup = h;
          const uint32_t i1 = lane * kTbRows + k + 1;
          if (j == static_cast<int>(jstar) - 1 && h == S && i1 <= m && i1 < icand) icand = i1;
        }
        dirs[j * 32 + lane] = word;
        hprev = hin;
        Hbot = H[kTbRows - 1];
        Fbot = f;
      }
    }
    icand = __reduce_min_sync(FULL, icand);
    __syncwarp();
    if (lane == 0) {
      uint32_t istar = a.mode == 1 ? m : icand;
      int i = static_cast<int>(istar), j = static_cast<int>(jstar);
      int32_t h = S;
      int state = 0, nops = 0;
      bool bad = istar > m || istar == 0;
      const int limit = static_cast<int>(m + jstar) + 2;
      while (!bad) {
        if (nops > limit || i < 0 || j < 0) {
          bad = true;
          break;
        }
        if (state == 0) {
          if (h == 0) break;
          if (i < 1 || j < 1) {
            bad = true;
            break;
          }
          const uint32_t nib = (dirs[(j - 1) * 32 + (i - 1) / kTbRows] >> (4 * ((i - 1) % kTbRows))) & 15u;
          if ((nib & 4u) && (nib & 8u)) {
            ops[nops++] = 0;  // M
            h -= qcode[i - 1] == rcode[j - 1] ? a.sa : -a.sb;
            --i;
            --j;
          } else if (nib & 8u) {
            state = 1;
          } else {
            state = 2;
          }
        } else {
          if (i < 1 || j < 1) {
            bad = true;
            break;
          }
          const uint32_t nib = (dirs[(j - 1) * 32 + (i - 1) / kTbRows] >> (4 * ((i - 1) % kTbRows))) & 15u;
          if (state == 1) {
            ops[nops++] = 2;  // D
            if (nib & 1u) {
              h += goe;
              state = 0;
            } else {
              h += a.ge;
            }
            --j;
          } else {
            ops[nops++] = 1;  // I
            if (nib & 2u) {
              h += goe;
              state = 0;
            } else {
              h += a.ge;
            }
            --i;
          }
        }
      }
      uint32_t* out = a.cigar_slots + static_cast<uint64_t>(r) * kCigarStride;
      uint32_t nc = 0;
      if (bad) {
        atomicOr(a.status, kStInternal);
      } else {
        const uint32_t start_i = static_cast<uint32_t>(i) + 1u;
        if (start_i > 1) out[nc++] = ((start_i - 1u) << 4) | 4u;
        for (int k = nops - 1; k >= 0;) {
          const uint32_t op = ops[k];
          uint32_t len = 0;
          while (k >= 0 && ops[k] == op) {
            ++len;
            --k;
          }
          out[nc++] = (len << 4) | op;
        }
        if (istar < m) out[nc++] = ((m - istar) << 4) | 4u;
        hp->read_start = static_cast<int32_t>(start_i);
        hp->read_end = static_cast<int32_t>(istar);
        hp->start_j = static_cast<uint32_t>(j) + 1u;
      }
      hp->cigar_len = nc;
    }
    __syncwarp();
  }
}

// Banded traceback.  The winning path's total gap length is at most
// g = (match * min(i*, j*) - S - gap_open) / gap_extend when it has a gap at all
// (every gap run costs gap_open plus gap_extend per base, and at most
// min(i*, j*) bases can match), so the path lies in the diagonals
// [d* - g, d* + g] around its end diagonal d* = j* - i*.  A DP restricted to
// those diagonals (cells outside count as H = 0, E = F = -inf) gives values no
// larger than the full DP's, and equal ones on every cell of the path (the
// path's own prefixes stay inside); each traceback decision there compares a
// path value with a value that is either also on the path or lower in both
// DPs, so the banded DP reproduces the full-DP path exactly.
//
// Schedule: a segment of SEG lanes holds one read, lane k the band diagonal
// dlo + k.  Lane k computes row i at step 2(i-1) + k, so its left neighbour
// (lane k-1, same row) and its upper neighbour (lane k+1, row above) were both
// computed at the previous step and its diagonal neighbour (itself, row above)
// two steps before: one shuffle each, no dependency chain within a step.  Each
// cell stores 4 bits: H came from the diagonal, H equals E, E opened, F opened.
// The walk jumps along runs of diagonal steps, checking SEG cells per
// iteration with a prefix sum of their scores.
constexpr int kTbWarps = 4;

template <int SEG>
__global__ void __launch_bounds__(32 * kTbWarps) k_tb_wave(TbArgs a, const uint32_t* list,
                                                           const uint32_t* count_ptr) {
  constexpr int NSEG = 32 / SEG;
  __shared__ uint8_t dirs_s[kTbWarps][NSEG][kMaxReadLen * SEG];
  __shared__ uint8_t rcode_s[kTbWarps][NSEG][kMaxWinLen];
  __shared__ uint8_t qcode_s[kTbWarps][NSEG][kMaxReadLen];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int seg = lane / SEG;
  const int k = lane % SEG;
  const uint32_t seg_mask = SEG == 32 ? FULL : (((1u << SEG) - 1u) << (seg * SEG));
  uint8_t* dirs = dirs_s[warp][seg];
  uint8_t* rcode = rcode_s[warp][seg];
  uint8_t* qcode = qcode_s[warp][seg];
  const int32_t goe = a.go + a.ge;
  constexpr int32_t NEG = -(1 << 28);
  const uint32_t count = *count_ptr;
  const uint32_t stride = gridDim.x * kTbWarps * NSEG;
  for (uint32_t base = (blockIdx.x * kTbWarps + warp) * NSEG; base < count; base += stride) {
    const uint32_t li = base + seg;
    const bool has = li < count;
    uint32_t r = 0, m = 0, istar = 0, jstar = 0, strand = 0;
    int32_t S = 0, item = -1;
    int g = 0, w = 0, dlo = 0;
    uint64_t ws = 0;
    const uint32_t* ref = nullptr;
    if (has) {
      r = list[li];
      const DevHit* hp = a.hits + static_cast<uint64_t>(r) * a.slots;
      item = hp->item;
      S = hp->score;
      const uint32_t rd = a.item_read[item];
      m = a.rlen[rd];
      jstar = a.item_end[item];
      istar = a.mode == 1 ? m : a.item_iend[item];
      const int64_t gl = (static_cast<int64_t>(a.sa) * min(istar, jstar) - S - a.go) / a.ge;
      g = gl > 0 ? static_cast<int>(gl) : 0;
      w = 2 * g + 1;
      dlo = static_cast<int>(jstar) - static_cast<int>(istar) - g;
      strand = a.c_strand[item];
      ws = a.c_start[item];
      ref = a.refs.words[a.c_ref[item]];
      const uint32_t* row = a.rpack + static_cast<uint64_t>(rd) * kReadWords;
      for (uint32_t j = k; j < jstar; j += SEG) rcode[j] = static_cast<uint8_t>(base_at(ref, ws + j));
      for (uint32_t i = k; i < istar; i += SEG)
        qcode[i] = static_cast<uint8_t>(strand ? 3u - base_at(row, m - 1u - i) : base_at(row, i));
    }
    __syncwarp();
    // ---- banded DP, skew-2 wavefront
    const int nsteps = has ? 2 * (static_cast<int>(istar) - 1) + w : 0;
    const int nmax = static_cast<int>(__reduce_max_sync(FULL, static_cast<uint32_t>(nsteps)));
    int32_t Hc = 0, Ec = NEG, Fc = NEG;
    for (int t = 0; t < nmax; ++t) {
      int32_t hl = __shfl_up_sync(FULL, Hc, 1, SEG);
      int32_t el = __shfl_up_sync(FULL, Ec, 1, SEG);
      int32_t hu = __shfl_down_sync(FULL, Hc, 1, SEG);
      int32_t fu = __shfl_down_sync(FULL, Fc, 1, SEG);
      if (k == 0) {
        hl = 0;
        el = NEG;
      }
      if (k + 1 >= w) {
        hu = 0;
        fu = NEG;
      }
      const int tk = t - k;
      if (has && k < w && tk >= 0 && !(tk & 1) && tk / 2 < static_cast<int>(istar)) {
        const int i = tk / 2 + 1;
        const int j = i + dlo + k;
        const int32_t eo = hl - goe, ee = el - a.ge, fo = hu - goe, fe = fu - a.ge;
        const int32_t E = max(eo, ee), F = max(fo, fe);
        uint32_t nib = 0;
        if (j >= 1 && j <= static_cast<int>(jstar)) {
          const int32_t hs = Hc + (qcode[i - 1] == rcode[j - 1] ? a.sa : -a.sb);
          const int32_t H = max(max(0, hs), max(E, F));
          nib = static_cast<uint32_t>(H == hs) | (static_cast<uint32_t>(H == E) << 1) |
                (static_cast<uint32_t>(eo >= ee) << 2) | (static_cast<uint32_t>(fo >= fe) << 3);
          Hc = H;
          Ec = E;
          Fc = F;
        } else {
          Hc = 0;
          Ec = NEG;
          Fc = NEG;
        }
        dirs[(i - 1) * SEG + k] = static_cast<uint8_t>(nib);
      }
    }
    __syncwarp();
    // ---- walk back (per segment)
    if (has) {
      uint32_t* out = a.cigar_slots + static_cast<uint64_t>(r) * kCigarStride;
      int i = static_cast<int>(istar), j = static_cast<int>(jstar), kk = g;
      int32_t h = S;
      int state = 0;
      uint32_t nr = 0, cur_op = 0xffu, cur_len = 0;
      bool bad = false;
      const int limit = static_cast<int>(istar + jstar) + 4;
      for (int it = 0;; ++it) {
        if (it > limit || kk < 0 || kk >= w) {
          bad = true;
          break;
        }
        if (state == 0) {
          if (h == 0) break;
          const int ii = i - k, jj = j - k;
          const bool v = ii >= 1 && jj >= 1;
          const uint32_t nib = v ? dirs[(ii - 1) * SEG + kk] : 0u;
          const int32_t st = v ? (qcode[ii - 1] == rcode[jj - 1] ? a.sa : -a.sb) : 0;
          int32_t incl = st;
#pragma unroll
          for (int off = 1; off < SEG; off <<= 1) {
            const int32_t x = __shfl_up_sync(seg_mask, incl, off, SEG);
            if (k >= off) incl += x;
          }
          const bool stop = !(v && (h - (incl - st)) != 0 && (nib & 1u));
          const uint32_t bal = (__ballot_sync(seg_mask, stop) & seg_mask) >> (SEG == 32 ? 0 : seg * SEG);
          const int L = bal ? __ffs(bal) - 1 : SEG;
          if (L > 0) {
            const int32_t used = __shfl_sync(seg_mask, incl, L - 1, SEG);
            h -= used;
            i -= L;
            j -= L;
            if (cur_op == 0u) {
              cur_len += static_cast<uint32_t>(L);
            } else {
              if (nr + 4 >= static_cast<uint32_t>(kCigarStride)) {
                bad = true;
                break;
              }
              if (cur_len && k == 0) out[1 + nr] = (cur_len << 4) | cur_op;
              nr += cur_len ? 1u : 0u;
              cur_op = 0u;
              cur_len = static_cast<uint32_t>(L);
            }
            continue;
          }
          const uint32_t nib0 = __shfl_sync(seg_mask, nib, 0, SEG);
          state = (nib0 & 2u) ? 1 : 2;
        } else {
          if (i < 1 || j < 1) {
            bad = true;
            break;
          }
          const uint32_t nib = dirs[(i - 1) * SEG + kk];
          const uint32_t op = state == 1 ? 2u : 1u;  // D : I
          if (cur_op == op) {
            ++cur_len;
          } else {
            if (nr + 4 >= static_cast<uint32_t>(kCigarStride)) {
              bad = true;
              break;
            }
            if (cur_len && k == 0) out[1 + nr] = (cur_len << 4) | cur_op;
            nr += cur_len ? 1u : 0u;
            cur_op = op;
            cur_len = 1;
          }
          const bool open = state == 1 ? (nib & 4u) : (nib & 8u);
          h += open ? goe : a.ge;
          if (open) state = 0;
          if (op == 2u) {
            --j;
            --kk;
          } else {
            --i;
            ++kk;
          }
        }
      }
      if (k == 0) {
        DevHit* hp = a.hits + static_cast<uint64_t>(r) * a.slots;
        if (bad || nr + 3 > static_cast<uint32_t>(kCigarStride)) {
          atomicOr(a.status, kStInternal);
          hp->cigar_len = 0;
        } else {
          if (cur_len) out[1 + nr++] = (cur_len << 4) | cur_op;
          // runs sit reversed in out[1 .. nr]; put them in order after the soft clip
          for (uint32_t x = 0; x < nr / 2; ++x) {
            const uint32_t t0 = out[1 + x];
            out[1 + x] = out[nr - x];
            out[nr - x] = t0;
          }
          const uint32_t start_i = static_cast<uint32_t>(i) + 1u;
          uint32_t nc;
          if (start_i > 1) {
            out[0] = ((start_i - 1u) << 4) | 4u;
            nc = nr + 1;
          } else {
            for (uint32_t x = 0; x < nr; ++x) out[x] = out[x + 1];
            nc = nr;
          }
          if (istar < m) out[nc++] = ((m - istar) << 4) | 4u;
          hp->read_start = static_cast<int32_t>(start_i);
          hp->read_end = static_cast<int32_t>(istar);
          hp->start_j = static_cast<uint32_t>(j) + 1u;
          hp->cigar_len = nc;
        }
      }
    }
    __syncwarp();
  }
}

// Routing: clears reads without a winner and sorts winners by band width into
// lists for k_tb_wave<8|16|32>; wider bands and int32-class winners go to the
// full-rectangle kernel.
__global__ void k_tb_route(TbArgs a, uint32_t* lists, uint32_t* counts) {
  const uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const bool live = r < a.n_reads;
  int bucket = -1;
  if (live) {
    DevHit* hp = a.hits + r * a.slots;
    const int32_t item = hp->item, S = hp->score;
    if (item < 0 || S <= 0) {
      hp->read_start = hp->read_end = 0;
      hp->start_j = 0;
      hp->cigar_len = 0;
    } else if (a.need_full[r]) {
      bucket = 3;
    } else {
      const uint32_t m = a.rlen[a.item_read[item]];
      const uint32_t jstar = a.item_end[item];
      const uint32_t istar = a.mode == 1 ? m : a.item_iend[item];
      if (istar == 0 || istar > m || jstar == 0) {
        atomicOr(a.status, kStInternal);
        hp->cigar_len = 0;
      } else {
        const int64_t gl = (static_cast<int64_t>(a.sa) * min(istar, jstar) - S - a.go) / a.ge;
        const int64_t w = 2 * (gl > 0 ? gl : 0) + 1;
        bucket = w <= 8 ? 0 : (w <= 16 ? 1 : (w <= 32 ? 2 : 3));
      }
    }
  }
  const uint32_t act = __ballot_sync(FULL, live && bucket >= 0);
  if (!(live && bucket >= 0)) return;
  const uint32_t peers = __match_any_sync(act, static_cast<uint32_t>(bucket));
  const int ln = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t b0 = 0;
  if (ln == leader) b0 = atomicAdd(&counts[bucket], static_cast<uint32_t>(__popc(peers)));
  b0 = __shfl_sync(peers, b0, leader);
  lists[static_cast<uint64_t>(bucket) * a.n_reads + b0 + __popc(peers & ((1u << ln) - 1u))] =
      static_cast<uint32_t>(r);
}

}  // namespace

int launch_traceback(const BatchDev& b, const DevRefs& refs, const ScoreConst& sc, int mode,
                     int n_refs, cudaStream_t st) {
  if (b.n_reads == 0) return 0;
  TbArgs a{};
  a.rpack = b.rpack;
  a.rlen = b.rlen;
  a.c_ref = b.c_ref;
  a.c_strand = b.c_strand;
  a.c_start = b.c_start;
  a.c_len = b.c_len;
  a.item_read = b.item_read;
  a.item_end = b.item_end;
  a.item_iend = b.item_iend;
  a.need_full = b.need_full;
  a.refs = refs;
  a.hits = b.hits;
  a.cigar_slots = b.cigar_slots;
  a.status = b.status;
  a.n_reads = b.n_reads;
  a.slots = 1 + n_refs;
  a.mode = mode;
  a.sa = sc.sa;
  a.sb = sc.sb;
  a.go = sc.go;
  a.ge = sc.ge;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMemsetAsync(b.tb_count, 0, 4 * sizeof(uint32_t), st) != cudaSuccess) return -1;
  k_tb_route<<<(b.n_reads + 255) / 256, 256, 0, st>>>(a, b.tb_list, b.tb_count);
  int launched = 1;
  auto wave = [&](auto kern, int bucket, int per_warp) -> bool {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kTbWarps, 0) != cudaSuccess) return false;
    const uint32_t g0 = static_cast<uint32_t>(nsm) * static_cast<uint32_t>(per_sm > 0 ? per_sm : 1);
    const uint32_t need = (b.n_reads + kTbWarps * per_warp - 1) / (kTbWarps * per_warp);
    kern<<<need < g0 ? need : g0, 32 * kTbWarps, 0, st>>>(a, b.tb_list + static_cast<uint64_t>(bucket) * b.n_reads,
                                                        b.tb_count + bucket);
    ++launched;
    return cudaPeekAtLastError() == cudaSuccess;
  };
  if (!wave(k_tb_wave<8>, 0, 4) || !wave(k_tb_wave<16>, 1, 2) || !wave(k_tb_wave<32>, 2, 1)) return -1;
  const size_t smem = static_cast<size_t>(kMaxWinLen) * 32 * sizeof(uint32_t);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_traceback, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return -1;
    attr = true;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traceback, 32, smem) != cudaSuccess) return -1;
  const uint32_t grid = static_cast<uint32_t>(nsm) * static_cast<uint32_t>(per_sm > 0 ? per_sm : 1);
  k_traceback<<<grid, 32, smem, st>>>(a, b.tb_list + 3ull * b.n_reads, b.tb_count + 3);
  ++launched;
  return cudaPeekAtLastError() == cudaSuccess ? launched : -1;
}

}  // namespace sr
