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

__global__ void __launch_bounds__(32) k_traceback(TbArgs a) {
  extern __shared__ uint32_t dirs[];  // [j][lane], j < j*
  __shared__ uint8_t rcode[kMaxWinLen];
  __shared__ uint8_t qcode[kMaxReadLen];
  __shared__ uint8_t ops[kMaxReadLen + kMaxWinLen + 4];
  const int lane = threadIdx.x;
  const int32_t goe = a.go + a.ge;
  constexpr int32_t NEG = -(1 << 28);
  for (uint32_t r = blockIdx.x; r < a.n_reads; r += gridDim.x) {
    DevHit* hp = a.hits + static_cast<uint64_t>(r) * a.slots;
    const int32_t item = hp->item;
    const int32_t S = hp->score;
    if (item < 0 || S <= 0) continue;  // cleared by the banded kernel
    if (!a.need_full[r]) continue;     // traced by the banded kernel
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
// g = (match * min(i*, j*) - S) / gap_extend (every gap base costs at least
// gap_extend and at most min(i*, j*) bases can match), so the path lies in the
// diagonals [d* - g, d* + g] around its end diagonal d* = j* - i*.  A DP
// restricted to those diagonals (cells outside count as H = 0, E = F = -inf)
// gives values no larger than the full DP's, and equal ones on every cell of
// the path (the path's own prefixes stay inside); each traceback decision
// there compares a path value with a value that is either also on the path or
// lower in both DPs, so the banded DP reproduces the full-DP path exactly.
// One lane per diagonal (bands up to 32 wide), rows in order: F comes from the
// row above by a shuffle, E by an exclusive max-plus prefix scan over the row,
//   E(i, d) = max_{d' < d} (H'(i, d') + d'*ge) - go - d*ge,
// with H' the cell value without E.  Wider bands go to k_traceback.
constexpr int kBandW = 32;
constexpr int kBandWarps = 4;

__global__ void __launch_bounds__(32 * kBandWarps) k_tb_band(TbArgs a) {
  __shared__ uint8_t dirs_s[kBandWarps][kMaxReadLen * kBandW];
  __shared__ uint8_t rcode_s[kBandWarps][kMaxWinLen];
  __shared__ uint8_t qcode_s[kBandWarps][kMaxReadLen];
  __shared__ uint8_t ops_s[kBandWarps][kMaxReadLen + kMaxWinLen + 4];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  uint8_t* dirs = dirs_s[warp];
  uint8_t* rcode = rcode_s[warp];
  uint8_t* qcode = qcode_s[warp];
  uint8_t* ops = ops_s[warp];
  const int32_t goe = a.go + a.ge;
  constexpr int32_t NEG = -(1 << 28);
  for (uint32_t r = blockIdx.x * kBandWarps + warp; r < a.n_reads; r += gridDim.x * kBandWarps) {
    DevHit* hp = a.hits + static_cast<uint64_t>(r) * a.slots;
    const int32_t item = hp->item;
    const int32_t S = hp->score;
    if (item < 0 || S <= 0) {
      if (lane == 0) {
        hp->read_start = hp->read_end = 0;
        hp->start_j = 0;
        hp->cigar_len = 0;
      }
      continue;
    }
    if (a.need_full[r]) continue;
    const uint32_t rd = a.item_read[item];
    const uint32_t m = a.rlen[rd];
    const uint32_t jstar = a.item_end[item];
    const uint32_t istar = a.mode == 1 ? m : a.item_iend[item];
    if (istar == 0 || istar > m || jstar == 0) {
      if (lane == 0) {
        atomicOr(a.status, kStInternal);
        hp->cigar_len = 0;
      }
      continue;
    }
    const int64_t gl = (static_cast<int64_t>(a.sa) * min(istar, jstar) - S) / a.ge;
    if (gl < 0 || 2 * gl + 1 > kBandW) {
      if (lane == 0) a.need_full[r] = 1;
      continue;
    }
    const int g = static_cast<int>(gl);
    const int w = 2 * g + 1;
    const int dlo = static_cast<int>(jstar) - static_cast<int>(istar) - g;
    const uint32_t strand = a.c_strand[item];
    const uint64_t ws = a.c_start[item];
    const uint32_t* ref = a.refs.words[a.c_ref[item]];
    const uint32_t* row = a.rpack + static_cast<uint64_t>(rd) * kReadWords;
    for (uint32_t j = lane; j < jstar; j += 32) rcode[j] = static_cast<uint8_t>(base_at(ref, ws + j));
    for (uint32_t i = lane; i < istar; i += 32)
      qcode[i] = static_cast<uint8_t>(strand ? 3u - base_at(row, m - 1u - i) : base_at(row, i));
    __syncwarp();
    const int d = dlo + lane;
    const bool inband = lane < w;
    int32_t H = 0, F = NEG;
    for (int i = 1; i <= static_cast<int>(istar); ++i) {
      const int j = i + d;
      const bool valid = inband && j >= 1 && j <= static_cast<int>(jstar);
      int32_t hup = __shfl_down_sync(FULL, H, 1);
      int32_t fup = __shfl_down_sync(FULL, F, 1);
      if (lane + 1 >= w) {
        hup = 0;
        fup = NEG;
      }
      const int32_t fo = hup - goe, fe = fup - a.ge;
      const uint32_t pf = fo >= fe;
      const int32_t Fn = max(fo, fe);
      const int32_t sc = valid ? (qcode[i - 1] == rcode[j - 1] ? a.sa : -a.sb) : 0;
      const int32_t hs = H + sc;
      const int32_t hpr = valid ? max(max(0, hs), Fn) : 0;
      int32_t inc = hpr + lane * a.ge;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int32_t t = __shfl_up_sync(FULL, inc, off);
        if (lane >= off) inc = max(inc, t);
      }
      int32_t exc = __shfl_up_sync(FULL, inc, 1);
      exc = lane == 0 ? -a.ge : max(exc, -a.ge);
      const int32_t E = exc - a.go - lane * a.ge;
      const int32_t Hn = valid ? max(hpr, E) : 0;
      int32_t hl = __shfl_up_sync(FULL, Hn, 1);
      if (lane == 0) hl = 0;
      const uint32_t mb = valid && Hn == hs;
      const uint32_t eb = Hn == E;
      const uint32_t pe = E == hl - goe;
      dirs[(i - 1) * kBandW + lane] = static_cast<uint8_t>(mb | (eb << 1) | (pe << 2) | (pf << 3));
      H = Hn;
      F = valid ? Fn : NEG;
    }
    __syncwarp();
    if (lane == 0) {
      int i = static_cast<int>(istar), j = static_cast<int>(jstar), k = g;
      int32_t h = S;
      int state = 0, nops = 0;
      bool bad = false;
      const int limit = static_cast<int>(istar + jstar) + 2;
      for (;;) {
        if (nops > limit || k < 0 || k >= w) {
          bad = true;
          break;
        }
        if (state == 0 && h == 0) break;
        if (i < 1 || j < 1) {
          bad = true;
          break;
        }
        const uint32_t nib = dirs[(i - 1) * kBandW + k];
        if (state == 0) {
          if (nib & 1u) {
            ops[nops++] = 0;  // M
            h -= qcode[i - 1] == rcode[j - 1] ? a.sa : -a.sb;
            --i;
            --j;
          } else {
            state = (nib & 2u) ? 1 : 2;
          }
        } else if (state == 1) {
          ops[nops++] = 2;  // D
          if (nib & 4u) {
            h += goe;
            state = 0;
          } else {
            h += a.ge;
          }
          --j;
          --k;
        } else {
          ops[nops++] = 1;  // I
          if (nib & 8u) {
            h += goe;
            state = 0;
          } else {
            h += a.ge;
          }
          --i;
          ++k;
        }
      }
      uint32_t* out = a.cigar_slots + static_cast<uint64_t>(r) * kCigarStride;
      uint32_t nc = 0;
      if (bad) {
        atomicOr(a.status, kStInternal);
      } else {
        const uint32_t start_i = static_cast<uint32_t>(i) + 1u;
        if (start_i > 1) out[nc++] = ((start_i - 1u) << 4) | 4u;
        for (int q = nops - 1; q >= 0;) {
          const uint32_t op = ops[q];
          uint32_t len = 0;
          while (q >= 0 && ops[q] == op) {
            ++len;
            --q;
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
  {
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tb_band, 32 * kBandWarps, 0) != cudaSuccess)
      return -1;
    const uint32_t need = (b.n_reads + kBandWarps - 1) / kBandWarps;
    const uint32_t g0 = static_cast<uint32_t>(nsm) * static_cast<uint32_t>(per_sm > 0 ? per_sm : 1);
    k_tb_band<<<need < g0 ? need : g0, 32 * kBandWarps, 0, st>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
  }
  const size_t smem = static_cast<size_t>(kMaxWinLen) * 32 * sizeof(uint32_t);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_traceback, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return -1;
    attr = true;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traceback, 32, smem) != cudaSuccess)
    return -1;
  const uint32_t grid0 = static_cast<uint32_t>(nsm) * static_cast<uint32_t>(per_sm > 0 ? per_sm : 1);
  const uint32_t grid = grid0 < b.n_reads ? grid0 : b.n_reads;
  k_traceback<<<grid, 32, smem, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

}  // namespace sr
