// sr_traceback.cu -- CIGAR of each read's winning window (McVicar et al.,
// arXiv 1805.00106: the reported alignment of Sec. 4.2 / SAM output, whose
// traceback the paper runs on the host, Sec. 6.4).
//
// Most winners are traced by a banded DP that also finds the end row i*: two
// reads per thread in the 16-bit halves of each value, swept row by row, for
// bands of at most 16 diagonals (k_tb_pair<16>) and of 17-32 (k_tb_pair<32>);
// when the scores do not fit those 16-bit values, one thread per read for at
// most 8 diagonals (k_tb_thread) and a wavefront over the band's diagonals for
// 9-32 (k_tb_wave); two diagonals per lane for 33-64 (k_tb_wave2).  Winners
// whose band is wider than 64 diagonals, and int32-class winners, use
// k_traceback: one warp
// per read recomputes the DP of the winning window in exact int32 over rows
// 1..m and columns 1..j* only (j* = the end column found by the extension
// kernels; cells right of j* cannot influence the path) with the same systolic
// sweep (8 rows per lane), and records per cell a 4-bit direction code in
// shared memory:
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

#include <algorithm>

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
  const uint8_t* tb_flag;
  DevHit* hits;
  uint32_t* cigar_slots;
  uint32_t* status;
  uint32_t n_reads;
  int slots;
  int mode;
  int32_t sa, sb, go, ge;
  uint32_t k2;  // 2, passed at run time (multiply-adds by it stay on the FMA pipe)
};

__global__ void __launch_bounds__(32) k_traceback(TbArgs a, const uint32_t* list, const uint32_t* range) {
  extern __shared__ uint32_t dirs[];  // [j][lane], j < j*
  __shared__ uint8_t rcode[kMaxWinLen];
  __shared__ uint8_t qcode[kMaxReadLen];
  __shared__ uint8_t ops[kMaxReadLen + kMaxWinLen + 4];
  const int lane = threadIdx.x;
  const int32_t goe = a.go + a.ge;
  constexpr int32_t NEG = -(1 << 28);
  const uint32_t begin = range[0], count = range[1] - range[0];
  for (uint32_t li = blockIdx.x; li < count; li += gridDim.x) {
    const uint32_t r = list[begin + li];
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

// Banded traceback.  The winner's end cell is (i*, j*): j* from the extension
// kernels, i* the smallest row with H(i*, j*) = S.  Every alignment of score S
// ending in column j* at a row in [ilo, ihi] lies in the band of tb_band(), so a
// DP restricted to those diagonals (cells outside count as H = 0, E = F = -inf)
// gives values no larger than the full DP's and equal ones on every cell of
// such an alignment (its prefixes stay inside).  Column j* of the band thus
// holds S exactly at the rows where the full DP does, which gives i*; and each
// traceback decision compares a path value with a value that is either also on
// the path or lower in both DPs, so the banded DP reproduces the full-DP path.
//
// Schedule: a segment of SEG lanes holds two reads, lane k the band diagonal
// dlo + k of each.  Lane k computes row i of read A at step 2(i-1) + k and row i
// of read B one step later, so every lane computes one cell per step, of A and B
// in turn.  A cell's left neighbour (lane k-1, same row) and upper neighbour
// (lane k+1, row above) belong to the same read and were computed at the
// previous step, its diagonal neighbour (itself, row above) two steps before.
// Each cell computes the E of its right neighbour and the F of its lower one
// (open from its H or extend its own gap value), so a step takes two shuffles
// and no dependency chain.  Each cell stores 4 bits (H came from the diagonal,
// H equals E, it opened its right neighbour's E, it opened its lower neighbour's
// F); read A's in the low and read B's in the high nibble of one byte per (row,
// lane).  The walk jumps along runs of diagonal steps, checking SEG cells per
// iteration with a prefix sum of their scores; a gap step reads the open flag
// at the cell it steps to.
constexpr int kTbWarps = 2;  // static shared memory stays below 48 KB per block
constexpr int kTbRowPad = 16;  // rows before row 1 / after row 256 a lane may reach (SEG / 2)
constexpr uint32_t kNoRow = 0xffffffffu;

struct TbRead {
  bool has;
  uint32_t r, m, jstar, strand, rd;
  int32_t S, item;
  int ilo, ihi, g, w, dlo;
  uint64_t ws;
  const uint32_t* ref;
};

// rows that may end the winner's alignment: row m in final-row mode, the row the
// extension kernels' winner mode found, or every row from ceil(S / match) to m
__device__ __forceinline__ bool tb_rows(const TbArgs& a, uint32_t r, int32_t item, int32_t S, uint32_t m,
                                        uint32_t* ilo, uint32_t* ihi) {
  if (a.mode == 1) {
    *ilo = *ihi = m;
    return m >= 1;
  }
  if (a.tb_flag[r] == kTbFlagRow) {
    const uint32_t i = a.item_iend[item];
    *ilo = *ihi = i;
    return i >= 1 && i <= m;
  }
  uint32_t lo = tb_min_row(a.sa, S);
  if (lo < 1) lo = 1;
  *ilo = lo;
  *ihi = m;
  return lo <= m;
}

__device__ __forceinline__ TbRead tb_load(const TbArgs& a, bool has, uint32_t r) {
  TbRead t{};
  t.has = has;
  if (!has) return t;
  t.r = r;
  const DevHit* hp = a.hits + static_cast<uint64_t>(r) * a.slots;
  t.item = hp->item;
  t.S = hp->score;
  t.rd = a.item_read[t.item];
  t.m = a.rlen[t.rd];
  t.jstar = a.item_end[t.item];
  uint32_t ilo = 1, ihi = 1;
  tb_rows(a, r, t.item, t.S, t.m, &ilo, &ihi);  // checked by the routing kernel
  const TbBand b = tb_band(a.sa, a.go, a.ge, t.S, t.jstar, ilo, ihi);
  t.ilo = b.ilo;
  t.ihi = b.ihi;
  t.g = b.g;
  t.w = b.w;
  t.dlo = b.dlo;
  t.strand = a.c_strand[t.item];
  t.ws = a.c_start[t.item];
  t.ref = a.refs.words[a.c_ref[t.item]];
  return t;
}

// What the walk needs of one read.
struct WalkRead {
  int32_t has, r, m, jstar, ihi, w, dlo, S;
};

__device__ __forceinline__ WalkRead walk_of(const TbRead& t) {
  return WalkRead{t.has ? 1 : 0, static_cast<int32_t>(t.r), static_cast<int32_t>(t.m),
                  static_cast<int32_t>(t.jstar), t.ihi, t.w, t.dlo, t.S};
}

// Byte codes of a read and its window in shared memory, addressed by 32-bit
// offsets into the kernel's flat arrays.
struct Codes {
  const uint8_t* qb;
  const uint8_t* rb;
  __device__ __forceinline__ bool match(uint32_t qo, uint32_t ro, uint32_t i0, uint32_t j0) const {
    return qb[qo + i0] == rb[ro + j0];
  }
};

// walk back from (i*, j*) through one read's nibbles (shift 0: read A, 4: read B)
// with a group of WG lanes (lane k of the group); dirs rows have SEG bytes
// (dirs entries of type DT hold the read's nibble at `shift`, its bits inverted
// when INV = 15; cd.match(qo, ro, i0, j0) compares query row i0 with window
// column j0, both 0-based)
template <int SEG, int WG, typename CD, typename DT = uint8_t, uint32_t INV = 0>
__device__ __forceinline__ void tb_walk(const TbArgs& a, const WalkRead& t, uint32_t istar, int shift,
                                        const DT* dirs, const CD& cd, uint32_t qo, uint32_t ro,
                                        int k, uint32_t gmask, int gshift) {
  if (!t.has) return;
  const int32_t goe = a.go + a.ge;
  uint32_t* out = a.cigar_slots + static_cast<uint64_t>(t.r) * kCigarStride;
  int i = static_cast<int>(istar), j = t.jstar;
  int kk = j - i - t.dlo;
  int32_t h = t.S;
  int state = 0;
  uint32_t nr = 0, cur_op = 0xffu, cur_len = 0;
  bool bad = istar == kNoRow;
  const int limit = t.ihi + t.jstar + 4;
  for (int it = 0; !bad; ++it) {
    if (it > limit || kk < 0 || kk >= t.w) {
      bad = true;
      break;
    }
    if (state == 0) {
      if (h == 0) break;
      const int ii = i - k, jj = j - k;
      const bool v = ii >= 1 && jj >= 1;
      const uint32_t nib = v ? ((static_cast<uint32_t>(dirs[(ii - 1) * SEG + kk]) >> shift) ^ INV) & 15u : 0u;
      const int32_t st = v ? (cd.match(qo, ro, ii - 1, jj - 1) ? a.sa : -a.sb) : 0;
      int32_t incl = st;
#pragma unroll
      for (int off = 1; off < WG; off <<= 1) {
        const int32_t x = __shfl_up_sync(gmask, incl, off, WG);
        if (k >= off) incl += x;
      }
      const bool stop = !(v && (h - (incl - st)) != 0 && (nib & 1u));
      const uint32_t bal = (__ballot_sync(gmask, stop) & gmask) >> gshift;
      const int L = bal ? __ffs(bal) - 1 : WG;
      if (L > 0) {
        const int32_t used = __shfl_sync(gmask, incl, L - 1, WG);
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
      const uint32_t nib0 = __shfl_sync(gmask, nib, 0, WG);
      state = (nib0 & 2u) ? 1 : 2;
    } else {
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
      if (op == 2u) {
        --j;
        --kk;
      } else {
        --i;
        ++kk;
      }
      // the cell the gap came from holds whether it was opened there
      if (i < 1 || j < 1 || kk < 0 || kk >= t.w) {
        bad = true;
        break;
      }
      const uint32_t nib = ((static_cast<uint32_t>(dirs[(i - 1) * SEG + kk]) >> shift) ^ INV) & 15u;
      const bool open = op == 2u ? (nib & 4u) : (nib & 8u);
      h += open ? goe : a.ge;
      if (open) state = 0;
    }
  }
  if (k == 0) {
    DevHit* hp = a.hits + static_cast<uint64_t>(t.r) * a.slots;
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
      if (istar < static_cast<uint32_t>(t.m)) out[nc++] = ((t.m - istar) << 4) | 4u;
      hp->read_start = static_cast<int32_t>(start_i);
      hp->read_end = static_cast<int32_t>(istar);
      hp->start_j = static_cast<uint32_t>(j) + 1u;
      hp->cigar_len = nc;
    }
  }
}

// One read's band diagonal q (column = row + c, c = dlo + q) as a lane runs
// it: the rows where it is inside the window [rlo, rlo + cnt), the code offsets
// (packed: the slot's word offsets; bytes: offsets that index the codes by
// row), the row where it crosses the end column, the lower band edge flag.
struct TbSub {
  uint32_t rlo, cnt, qa, ra;
  int c, icr;
  bool bd;
};

__device__ __forceinline__ TbSub tb_sub(const TbRead& x, int q, uint32_t qslot, uint32_t rslot) {
  TbSub u;
  const int c = x.dlo + q;
  const int lo = max(1, 1 - c), hi = min(x.ihi, static_cast<int>(x.jstar) - c);
  const bool on = x.has && q < x.w && hi >= lo;
  u.rlo = static_cast<uint32_t>(lo);
  u.cnt = on ? static_cast<uint32_t>(hi - lo + 1) : 0u;
  u.qa = qslot - 1u;
  u.ra = rslot + static_cast<uint32_t>(c - 1);
  u.c = c;
  const int ir = static_cast<int>(x.jstar) - c;
  u.icr = (on && ir >= x.ilo && ir >= lo && ir <= hi) ? ir : -(1 << 20);
  u.bd = q + 1 >= x.w;
  return u;
}

// The byte codes of row i of a diagonal; outside the window they load from
// index 0 (no branch) and never match.  The loops load a row's codes one pair
// of steps ahead, so the loads' latency is off the wavefront's critical path.
struct TbLd {
  uint32_t q, r;
  bool in;
  __device__ __forceinline__ bool eq() const { return in & (q == r); }
};
__device__ __forceinline__ TbLd tb_ld_bytes(const TbSub& sb, int i, const uint8_t* qb, const uint8_t* rb) {
  const uint32_t ui = static_cast<uint32_t>(i);
  const bool in = ui - sb.rlo < sb.cnt;
  const uint32_t qi = in ? sb.qa + ui : 0u, ri = in ? sb.ra + ui : 0u;
  return TbLd{qb[qi], rb[ri], in};
}

// One cell.  E and F arrive complete from the left and upper neighbours, which
// computed them from their own cells (gap opened from their H or extended from
// their own gap value), and this cell does the same for its right (En) and
// lower (Fn) neighbour.  Cells outside the window score a mismatch: with the top
// and left borders at H = 0 and gap values at most -(go+ge) they keep H = 0,
// which is the border itself; cells right of j* or below the last row only feed
// cells that are never read.  Returns the 4 bits: H came from the diagonal, H
// equals E, this cell opened its right neighbour's E, this cell opened its lower
// neighbour's F.  hd holds the diagonal's previous H and becomes this one.
__device__ __forceinline__ uint32_t tb_cell(const TbArgs& a, int32_t goe, bool eq, int32_t E, int32_t F,
                                            bool cross, int32_t& hd, int32_t& En, int32_t& Fn, int32_t& hcr) {
  const int32_t hs = hd + (eq ? a.sa : -a.sb);
  const int32_t H = max(max(hs, 0), max(E, F));
  const int32_t g = H - goe, ee = E - a.ge, fe = F - a.ge;
  En = max(g, ee);
  Fn = max(g, fe);
  if (cross) hcr = H;
  hd = H;
  return static_cast<uint32_t>(H == hs) | (static_cast<uint32_t>(H == E) << 1) |
         (static_cast<uint32_t>(g >= ee) << 2) | (static_cast<uint32_t>(g >= fe) << 3);
}

// A read's codes as bytes (query rows up to ihi, window columns up to j*),
// staged by the lanes k, k + step, ...
__device__ __forceinline__ void tb_stage_bytes(const TbArgs& a, const TbRead& x, uint8_t* qc, uint8_t* rc,
                                               uint32_t k, uint32_t step) {
  const uint32_t* row = a.rpack + static_cast<uint64_t>(x.rd) * kReadWords;
  for (uint32_t j = k; j < x.jstar; j += step) rc[j] = static_cast<uint8_t>(base_at(x.ref, x.ws + j));
  for (uint32_t i = k; i < static_cast<uint32_t>(x.ihi); i += step)
    qc[i] = static_cast<uint8_t>(x.strand ? 3u - base_at(row, x.m - 1u - i) : base_at(row, i));
}

template <int SEG>
__global__ void __launch_bounds__(32 * kTbWarps) k_tb_wave(TbArgs a, const uint32_t* list,
                                                           const uint32_t* range) {
  static_assert(SEG >= 8, "narrow bands run one thread per read (k_tb_thread)");
  constexpr int NSEG = 32 / SEG;
  constexpr int kQB = kMaxReadLen;  // byte codes per read
  constexpr int kRB = kMaxWinLen;
  constexpr int kSlots = kTbWarps * NSEG * 2;  // reads resident per block
  // direction bytes of rows 1 - kTbRowPad .. kMaxReadLen + kTbRowPad + 1: the
  // wavefront's first and last steps run lanes above row 1 and below row m
  __shared__ uint8_t dirs_s[kTbWarps][NSEG][(kMaxReadLen + 2 * kTbRowPad + 1) * SEG];
  __shared__ uint8_t qbyte_s[kSlots * kQB];
  __shared__ uint8_t rbyte_s[kSlots * kRB];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int seg = lane / SEG;
  const int k = lane % SEG;
  const uint32_t seg_mask = SEG == 32 ? FULL : (((1u << SEG) - 1u) << (seg * SEG));
  uint8_t* dirs = dirs_s[warp][seg] + kTbRowPad * SEG;
  const Codes cd{qbyte_s, rbyte_s};
  const int32_t goe = a.go + a.ge;
  const uint32_t begin = range[0];
  const uint32_t count = range[1] - begin;
  constexpr uint32_t kPerWarp = 2 * NSEG;
  const uint32_t stride = gridDim.x * kTbWarps * kPerWarp;
  // slot of read X of this segment, and its code offsets
  auto slot = [&](int sg, int X) { return (warp * NSEG + sg) * 2 + X; };
  for (uint32_t base = (blockIdx.x * kTbWarps + warp) * kPerWarp; base < count; base += stride) {
    TbRead rd[2];
#pragma unroll
    for (int X = 0; X < 2; ++X) {
      const uint32_t li = base + 2 * seg + X;
      rd[X] = tb_load(a, li < count, li < count ? list[begin + li] : 0u);
      if (rd[X].has) {
        const int sl = slot(seg, X);
        tb_stage_bytes(a, rd[X], qbyte_s + sl * kQB, rbyte_s + sl * kRB, static_cast<uint32_t>(k), SEG);
      }
    }
    __syncwarp();
    // ---- banded DP of both reads, interleaved skew-2 wavefront.  Lane k runs
    // read (k & 1) at even steps and the other read at odd steps, so a pair of
    // steps has a fixed read per half-step and the per-read terms are set once.
    const int stA = rd[0].has ? 2 * (rd[0].ihi - 1) + rd[0].w : 0;
    const int stB = rd[1].has ? 2 * (rd[1].ihi - 1) + rd[1].w : 0;
    const int nmax = static_cast<int>(__reduce_max_sync(FULL, static_cast<uint32_t>(max(stA, stB) + 1)));
    const int p = k & 1;
    // the read of each half-step on this lane's diagonal
    const int slA = slot(seg, 0), slB = slot(seg, 1);
    const TbSub uA = tb_sub(rd[0], k, static_cast<uint32_t>(slA * kQB), static_cast<uint32_t>(slA * kRB));
    const TbSub uB = tb_sub(rd[1], k, static_cast<uint32_t>(slB * kQB), static_cast<uint32_t>(slB * kRB));
    const TbSub s0 = p ? uB : uA, s1 = p ? uA : uB;
    auto cell = [&](const TbSub& sb, int i, const TbLd& ld, int32_t E, int32_t F, int32_t& hd, int32_t& En,
                    int32_t& Fn, uint32_t& nib, int32_t& hcr) {
      nib = tb_cell(a, goe, ld.eq(), E, F, i == sb.icr, hd, En, Fn, hcr);
    };
    auto load = [&](const TbSub& sb, int i) { return tb_ld_bytes(sb, i, qbyte_s, rbyte_s); };
    // what each half-step sent last: gap values for the neighbours, own H
    int32_t Ha = 0, Hb = 0, Ena = -goe, Fna = -goe, Enb = -goe, Fnb = -goe;
    int32_t hcr0 = -1, hcr1 = -1;
    uint32_t pend = 0;
    int ia = 1 - ((k + p) >> 1);  // row of half-step 0 in this pair
    uint8_t* drow = dirs + (ia - 1) * SEG + k;  // this lane's byte of row ia
    TbLd L0 = load(s0, ia), L1 = load(s1, ia + p);
    for (int t = 0; t < nmax; t += 2, ++ia, drow += SEG) {
      const TbLd N0 = load(s0, ia + 1), N1 = load(s1, ia + 1 + p);
      uint32_t nib;
      {
        int32_t E = __shfl_up_sync(FULL, Enb, 1, SEG);
        int32_t F = __shfl_down_sync(FULL, Fnb, 1, SEG);
        if (k == 0) E = -goe;
        if (s0.bd) F = -goe;
        cell(s0, ia, L0, E, F, Ha, Ena, Fna, nib, hcr0);
        // A row's byte is read A's nibble (low) and read B's (high).  Every
        // half-step stores the byte of its row with the other read's last
        // nibble; the half-step that runs read B writes it last, and the
        // earlier store of read A's half-step is overwritten (lanes with p = 1
        // run read A one row ahead, so theirs goes to the next row).
        *drow = static_cast<uint8_t>(pend + (nib << 4));
        pend = nib;
      }
      {
        int32_t E = __shfl_up_sync(FULL, Ena, 1, SEG);
        int32_t F = __shfl_down_sync(FULL, Fna, 1, SEG);
        if (k == 0) E = -goe;
        if (s1.bd) F = -goe;
        cell(s1, ia + p, L1, E, F, Hb, Enb, Fnb, nib, hcr1);
        drow[p ? SEG : 0] = static_cast<uint8_t>(pend + (nib << 4));
        pend = nib;
      }
      L0 = N0;
      L1 = N1;
    }
    const uint32_t ic0 = (s0.icr > 0 && hcr0 == (p ? rd[1].S : rd[0].S)) ? static_cast<uint32_t>(s0.icr) : kNoRow;
    const uint32_t ic1 = (s1.icr > 0 && hcr1 == (p ? rd[0].S : rd[1].S)) ? static_cast<uint32_t>(s1.icr) : kNoRow;
    uint32_t icA = p ? ic1 : ic0, icB = p ? ic0 : ic1;
#pragma unroll
    for (int off = SEG / 2; off > 0; off >>= 1) {
      icA = min(icA, __shfl_xor_sync(FULL, icA, off, SEG));
      icB = min(icB, __shfl_xor_sync(FULL, icB, off, SEG));
    }
    __syncwarp();
    // ---- walk back: read A, then read B of each segment, walked by the segment's lanes
    tb_walk<SEG, SEG, Codes>(a, walk_of(rd[0]), icA, 0, dirs, cd, static_cast<uint32_t>(slot(seg, 0) * kQB),
                              static_cast<uint32_t>(slot(seg, 0) * kRB), k, seg_mask, SEG == 32 ? 0 : seg * SEG);
    __syncwarp(seg_mask);
    tb_walk<SEG, SEG, Codes>(a, walk_of(rd[1]), icB, 4, dirs, cd, static_cast<uint32_t>(slot(seg, 1) * kQB),
                              static_cast<uint32_t>(slot(seg, 1) * kRB), k, seg_mask, SEG == 32 ? 0 : seg * SEG);
    __syncwarp();
  }
}

// byte permute (prmt.b32) and a multiply-add that stays a multiply-add
__device__ __forceinline__ uint32_t tb_prmt(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t imad_u32(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// whether the packed (two reads per thread) kernels hold these scores:
// byte-table scores, and every cell value (>= -(go+ge), <= the int16-class
// score) inside 16 bits
bool tb_pair_fits(int32_t sa, int32_t sb, int32_t go, int32_t ge) {
  return sa >= 1 && sa <= 127 && sb >= 1 && sb <= 128 && static_cast<int64_t>(go) + ge <= 8192;
}

// The same wavefront for bands of 33-64 diagonals: lane k runs band diagonals k
// and k + 32 of both reads, the second 16 rows behind the first (its step for
// row i is 32 later).  Diagonal 31's right neighbour (32) and diagonal 32's left
// neighbour (31) sit on lanes 0 and 31, so the gap values that cross between the
// lane's two diagonals go by rotating shuffles.
constexpr int kTb2Diags = 64;
constexpr int kTb2RowPad = 32;  // rows before row 1 the second diagonal reaches
constexpr int kTb2Rows = kMaxReadLen + 2 * kTb2RowPad + 1;

__global__ void __launch_bounds__(32 * kTbWarps) k_tb_wave2(TbArgs a, const uint32_t* list, const uint32_t* range) {
  constexpr int V = kTb2Diags;
  constexpr int kSlots = kTbWarps * 2;
  constexpr int kLag = 16 * V - 32;  // bytes from diagonal k's row i to diagonal k + 32's row i - 16
  __shared__ uint8_t dirs_s[kTbWarps][kTb2Rows * V];
  __shared__ uint8_t qbyte_s[kSlots * kMaxReadLen];
  __shared__ uint8_t rbyte_s[kSlots * kMaxWinLen];
  const int k = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  uint8_t* dirs = dirs_s[warp] + kTb2RowPad * V;
  const Codes cd{qbyte_s, rbyte_s};
  const int32_t goe = a.go + a.ge;
  const uint32_t begin = range[0];
  const uint32_t count = range[1] - begin;
  const uint32_t stride = gridDim.x * kTbWarps * 2;
  const int up = (k + 31) & 31, dn = (k + 1) & 31;
  for (uint32_t base = (blockIdx.x * kTbWarps + warp) * 2; base < count; base += stride) {
    TbRead rd[2];
#pragma unroll
    for (int X = 0; X < 2; ++X) {
      const uint32_t li = base + X;
      rd[X] = tb_load(a, li < count, li < count ? list[begin + li] : 0u);
      const int sl = warp * 2 + X;
      if (rd[X].has) tb_stage_bytes(a, rd[X], qbyte_s + sl * kMaxReadLen, rbyte_s + sl * kMaxWinLen, k, 32);
    }
    __syncwarp();
    const int stA = rd[0].has ? 2 * (rd[0].ihi - 1) + rd[0].w : 0;
    const int stB = rd[1].has ? 2 * (rd[1].ihi - 1) + rd[1].w : 0;
    const int nmax = static_cast<int>(__reduce_max_sync(FULL, static_cast<uint32_t>(max(stA, stB) + 1)));
    const int p = k & 1;
    const uint32_t qA = warp * 2 * kMaxReadLen, rA = warp * 2 * kMaxWinLen;
    const uint32_t qB = qA + kMaxReadLen, rB = rA + kMaxWinLen;
    // [read of the half-step][diagonal k, k + 32]
    const TbSub uA0 = tb_sub(rd[0], k, qA, rA), uA1 = tb_sub(rd[0], k + 32, qA, rA);
    const TbSub uB0 = tb_sub(rd[1], k, qB, rB), uB1 = tb_sub(rd[1], k + 32, qB, rB);
    const TbSub s00 = p ? uB0 : uA0, s01 = p ? uB1 : uA1, s10 = p ? uA0 : uB0, s11 = p ? uA1 : uB1;
    int32_t Ha0 = 0, Ha1 = 0, Hb0 = 0, Hb1 = 0;
    int32_t Ena0 = -goe, Ena1 = -goe, Fna0 = -goe, Fna1 = -goe;
    int32_t Enb0 = -goe, Enb1 = -goe, Fnb0 = -goe, Fnb1 = -goe;
    int32_t hcr00 = -1, hcr01 = -1, hcr10 = -1, hcr11 = -1;
    uint32_t pend0 = 0, pend1 = 0;
    int ia = 1 - ((k + p) >> 1);  // diagonal k's row at half-step 0
    uint8_t* drow = dirs + (ia - 1) * V + k;
    const int o1 = p ? V : 0;     // half-step 1 runs read A one row ahead on odd lanes
    // (loading the codes a step ahead, as k_tb_wave does, costs this kernel
    // more in registers than it saves)
    for (int t = 0; t < nmax; t += 2, ++ia, drow += V) {
      {
        int32_t E0 = __shfl_up_sync(FULL, Enb0, 1);
        const int32_t E1 = __shfl_sync(FULL, k == 31 ? Enb0 : Enb1, up);
        int32_t F0 = __shfl_sync(FULL, k == 0 ? Fnb1 : Fnb0, dn);
        int32_t F1 = __shfl_down_sync(FULL, Fnb1, 1);
        if (k == 0) E0 = -goe;
        if (s00.bd) F0 = -goe;
        if (s01.bd) F1 = -goe;
        const uint32_t n0 = tb_cell(a, goe, tb_ld_bytes(s00, ia, qbyte_s, rbyte_s).eq(), E0, F0, ia == s00.icr, Ha0,
                                    Ena0, Fna0, hcr00);
        const uint32_t n1 = tb_cell(a, goe, tb_ld_bytes(s01, ia - 16, qbyte_s, rbyte_s).eq(), E1, F1,
                                    ia - 16 == s01.icr, Ha1, Ena1, Fna1, hcr01);
        // bytes as in k_tb_wave: read A's nibble low, read B's high
        drow[0] = static_cast<uint8_t>(pend0 + (n0 << 4));
        drow[-kLag] = static_cast<uint8_t>(pend1 + (n1 << 4));
        pend0 = n0;
        pend1 = n1;
      }
      {
        int32_t E0 = __shfl_up_sync(FULL, Ena0, 1);
        const int32_t E1 = __shfl_sync(FULL, k == 31 ? Ena0 : Ena1, up);
        int32_t F0 = __shfl_sync(FULL, k == 0 ? Fna1 : Fna0, dn);
        int32_t F1 = __shfl_down_sync(FULL, Fna1, 1);
        if (k == 0) E0 = -goe;
        if (s10.bd) F0 = -goe;
        if (s11.bd) F1 = -goe;
        const int ib = ia + p;
        const uint32_t n0 = tb_cell(a, goe, tb_ld_bytes(s10, ib, qbyte_s, rbyte_s).eq(), E0, F0, ib == s10.icr, Hb0,
                                    Enb0, Fnb0, hcr10);
        const uint32_t n1 = tb_cell(a, goe, tb_ld_bytes(s11, ib - 16, qbyte_s, rbyte_s).eq(), E1, F1,
                                    ib - 16 == s11.icr, Hb1, Enb1, Fnb1, hcr11);
        drow[o1] = static_cast<uint8_t>(pend0 + (n0 << 4));
        drow[o1 - kLag] = static_cast<uint8_t>(pend1 + (n1 << 4));
        pend0 = n0;
        pend1 = n1;
      }
    }
    auto ic = [&](const TbSub& u, int32_t hcr, int32_t S) {
      return (u.icr > 0 && hcr == S) ? static_cast<uint32_t>(u.icr) : kNoRow;
    };
    const int32_t S0 = p ? rd[1].S : rd[0].S, S1 = p ? rd[0].S : rd[1].S;
    const uint32_t ic0 = min(ic(s00, hcr00, S0), ic(s01, hcr01, S0));
    const uint32_t ic1 = min(ic(s10, hcr10, S1), ic(s11, hcr11, S1));
    const uint32_t icA = __reduce_min_sync(FULL, p ? ic1 : ic0);
    const uint32_t icB = __reduce_min_sync(FULL, p ? ic0 : ic1);
    __syncwarp();
    tb_walk<V, 32, Codes>(a, walk_of(rd[0]), icA, 0, dirs, cd, qA, rA, k, FULL, 0);
    __syncwarp();
    tb_walk<V, 32, Codes>(a, walk_of(rd[1]), icB, 4, dirs, cd, qB, rB, k, FULL, 0);
    __syncwarp();
  }
}

// ---- Narrow bands (at most W diagonals): one thread per read.  A band this
// narrow leaves most lanes of a wavefront idle, so each thread sweeps its read
// row by row, the W cells of a row in registers (E runs along the row, F and
// the diagonal come from the previous row), and writes the row's W nibbles
// (from the diagonal, H = E, E opened here, F opened here) as one word to a
// per-warp scratch laid out [row][lane], so a warp's stores coalesce.  The
// read's query words and its window (realigned to column 1) are staged in
// shared memory, 17 / 33 words per lane so the lanes' loads hit distinct banks.
constexpr int kTbTQW = kReadWords + 1;       // query words per lane (padded)
constexpr int kTbTRW = kMaxWinLen / 16 + 1;  // window words per lane (33: odd, conflict-free)
constexpr int kTbTWarps = 4;

// One read on its thread (bands of at most W diagonals): the band DP row by row,
// then the walk; qw / rw are the read's staged query and window words.
template <int W>
__device__ __forceinline__ void tb_thread_read(const TbArgs& a, const TbRead& t, uint32_t* dirs, const uint32_t* qw,
                                               const uint32_t* rw) {
  static_assert(W >= 1 && W <= 8, "one 32-bit word of nibbles per row");
  const int32_t goe = a.go + a.ge;
  constexpr int32_t NEG = -(1 << 28);
  auto qcode = [&](int i) {  // query code of row i (1-based)
    const uint32_t p = t.strand ? t.m - static_cast<uint32_t>(i) : static_cast<uint32_t>(i - 1);
    const uint32_t c = (qw[p >> 4] >> ((p & 15u) * 2u)) & 3u;
    return t.strand ? 3u - c : c;
  };
  auto rcode = [&](int j) {  // window code of column j (1-based, 1 <= j <= j*)
    const uint32_t p = static_cast<uint32_t>(j - 1);
    return (rw[p >> 4] >> ((p & 15u) * 2u)) & 3u;
  };
  // ---- the band DP, row by row
  int32_t Hp[W + 1], Fp[W + 1];  // previous row; index W is outside the band
#pragma unroll
  for (int k = 0; k <= W; ++k) {
    Hp[k] = 0;
    Fp[k] = NEG;
  }
  uint32_t istar = kNoRow;
  const int rows = t.has ? t.ihi : 0;
  const int w = t.w;
  const uint32_t wmask = w >= W ? 0xffffffffu : ((1u << w) - 1u);  // cells inside the band
  for (int i = 1; i <= rows; ++i) {
    const int c0 = i + t.dlo;  // column of cell 0 (1-based)
    // cells whose column lies in 1..j*
    const int klo = 1 - c0, khi = static_cast<int>(t.jstar) - c0;  // inclusive
    uint32_t vm = wmask;
    vm &= klo > 0 ? (klo >= 32 ? 0u : ~((1u << klo) - 1u)) : 0xffffffffu;
    vm &= khi < 31 ? (khi < 0 ? 0u : ((2u << khi) - 1u)) : 0xffffffffu;
    // the row's window codes, cell k at bits 2k; a match clears both bits of x
    const int cs = c0 - 1;
    const int rb = min(max(cs, 0), kMaxWinLen - 1);  // word (rb >> 4) + 1 <= 32 is staged space
    const uint32_t sh = static_cast<uint32_t>(rb & 15) * 2u;
    const uint32_t r0 = rw[rb >> 4], r1 = rw[(rb >> 4) + 1];
    uint32_t rbits = sh ? (r0 >> sh) | (r1 << (32u - sh)) : r0;
    if (cs < 0) rbits = -cs >= 16 ? 0u : rbits << (2 * -cs);
    const uint32_t x = rbits ^ (qcode(i) * 0x55555555u);
    const uint32_t mm = ~(x | (x >> 1));  // bit 2k: cell k matches
    int32_t H[W], E[W];
    int32_t Fn[W];
    uint32_t word = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const int32_t hl = k > 0 ? H[k - 1] : 0, el = k > 0 ? E[k - 1] : NEG;
      const bool up_in = k + 1 < w;
      const int32_t hu = up_in ? Hp[k + 1] : 0, fu = up_in ? Fp[k + 1] : NEG;
      const int32_t eo = hl - goe, ee = el - a.ge, fo = hu - goe, fe = fu - a.ge;
      const int32_t Eh = max(eo, ee), Fh = max(fo, fe);
      const bool in = (vm >> k) & 1u;
      const int32_t hs = Hp[k] + (((mm >> (2 * k)) & 1u) ? a.sa : -a.sb);
      const int32_t h = max(max(hs, 0), max(Eh, Fh));
      word |= in ? (static_cast<uint32_t>(h == hs) | (static_cast<uint32_t>(h == Eh) << 1) |
                    (static_cast<uint32_t>(eo >= ee) << 2) | (static_cast<uint32_t>(fo >= fe) << 3))
                       << (4 * k)
                 : 0u;
      H[k] = in ? h : 0;
      E[k] = in ? Eh : NEG;
      Fn[k] = in ? Fh : NEG;
    }
    dirs[(i - 1) * 32] = word;
    // end row: the smallest row at or past ilo whose cell in column j* holds S
    const int kc = khi;  // cell of column j*
    if (istar == kNoRow && i >= t.ilo && kc >= 0 && kc < w) {
      int32_t hc = 0;
#pragma unroll
      for (int k = 0; k < W; ++k) hc = k == kc ? H[k] : hc;
      if (hc == t.S) istar = static_cast<uint32_t>(i);
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      Hp[k] = H[k];
      Fp[k] = Fn[k];
    }
  }
  if (a.mode == 1 && t.has) istar = (istar == static_cast<uint32_t>(t.m)) ? istar : kNoRow;
  // ---- walk back from (i*, j*)
  if (t.has) {
    uint32_t* out = a.cigar_slots + static_cast<uint64_t>(t.r) * kCigarStride;
    int i = static_cast<int>(istar), j = static_cast<int>(t.jstar);
    int32_t h = t.S;
    int state = 0;
    uint32_t nr = 0, cur_op = 0xffu, cur_len = 0;
    bool bad = istar == kNoRow;
    const int limit = t.ihi + static_cast<int>(t.jstar) + 4;
    for (int it = 0; !bad; ++it) {
      const int k = j - i - t.dlo;
      if (it > limit || k < 0 || k >= w || i < 1 || j < 1) {
        bad = !(state == 0 && h == 0);
        break;
      }
      if (state == 0 && h == 0) break;
      const uint32_t nib = (dirs[(i - 1) * 32] >> (4 * k)) & 15u;
      uint32_t op;
      if (state == 0) {
        if (nib & 1u) {
          op = 0u;  // M
          h -= qcode(i) == rcode(j) ? a.sa : -a.sb;
          --i;
          --j;
        } else {
          state = (nib & 2u) ? 1 : 2;
          continue;
        }
      } else if (state == 1) {
        op = 2u;  // D
        const bool open = nib & 4u;
        h += open ? goe : a.ge;
        if (open) state = 0;
        --j;
      } else {
        op = 1u;  // I
        const bool open = nib & 8u;
        h += open ? goe : a.ge;
        if (open) state = 0;
        --i;
      }
      if (op == cur_op) {
        ++cur_len;
      } else {
        if (nr + 4 >= static_cast<uint32_t>(kCigarStride)) {
          bad = true;
          break;
        }
        if (cur_len) out[1 + nr++] = (cur_len << 4) | cur_op;
        cur_op = op;
        cur_len = 1;
      }
    }
    DevHit* hp = a.hits + static_cast<uint64_t>(t.r) * a.slots;
    if (bad || nr + 3 > static_cast<uint32_t>(kCigarStride)) {
      atomicOr(a.status, kStInternal);
      hp->cigar_len = 0;
    } else {
      if (cur_len) out[1 + nr++] = (cur_len << 4) | cur_op;
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
      if (istar < t.m) out[nc++] = ((t.m - istar) << 4) | 4u;
      hp->read_start = static_cast<int32_t>(start_i);
      hp->read_end = static_cast<int32_t>(istar);
      hp->start_j = static_cast<uint32_t>(j) + 1u;
      hp->cigar_len = nc;
    }
  }
}

// Reads of bands up to 8 diagonals, in band-width order: each warp runs the
// narrowest cell count that holds its 32 reads.
__global__ void __launch_bounds__(32 * kTbTWarps) k_tb_thread(TbArgs a, const uint32_t* list, const uint32_t* range_lo,
                                                            const uint32_t* range_hi, uint32_t* scratch,
                                                            uint32_t n_warps) {
  __shared__ uint32_t q_s[kTbTWarps][32 * kTbTQW];
  __shared__ uint32_t r_s[kTbTWarps][32 * kTbTRW];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint32_t gw = blockIdx.x * kTbTWarps + warp;
  if (gw >= n_warps) return;
  uint32_t* dirs = scratch + static_cast<uint64_t>(gw) * kMaxReadLen * 32 + lane;  // [row][lane]
  uint32_t* qw = q_s[warp] + lane * kTbTQW;
  uint32_t* rw = r_s[warp] + lane * kTbTRW;
  const uint32_t first = range_lo[0];
  const uint32_t count = range_hi[1] - first;
  for (uint32_t base = gw * 32u; base < count; base += n_warps * 32u) {
    const uint32_t li = base + lane;
    const TbRead t = tb_load(a, li < count, li < count ? list[first + li] : 0u);
    // stage this read's words: the query row as packed, the window from column 1
    if (t.has) {
      const uint32_t* row = a.rpack + static_cast<uint64_t>(t.rd) * kReadWords;
      for (int w = 0; w < kReadWords; ++w) qw[w] = row[w];
      const int nwin = static_cast<int>((t.jstar + 15) / 16);
      for (int w = 0; w < nwin; ++w) {
        const uint64_t idx = t.ws + 16ull * w;
        const uint32_t sh = static_cast<uint32_t>(idx & 15u) * 2u;
        const uint32_t* src = t.ref + (idx >> 4);
        rw[w] = sh ? (src[0] >> sh) | (src[1] << (32u - sh)) : src[0];
      }
    }
    const uint32_t wmax = __reduce_max_sync(FULL, t.has ? static_cast<uint32_t>(t.w) : 0u);
    if (wmax <= 1)
      tb_thread_read<1>(a, t, dirs, qw, rw);
    else if (wmax <= 2)
      tb_thread_read<2>(a, t, dirs, qw, rw);
    else if (wmax <= 4)
      tb_thread_read<4>(a, t, dirs, qw, rw);
    else
      tb_thread_read<8>(a, t, dirs, qw, rw);
  }
}

// ---- Bands of at most 16 (or 32) diagonals: two reads per thread, one in each
// 16-bit half (DPX s16x2 arithmetic), each pair swept row by row with the row's
// W cells in registers.  Cell k of row i is band diagonal dlo + k (column
// i + dlo + k); its left neighbour is cell k - 1 of the same row, its upper one
// cell k + 1 and its diagonal cell k of the row above.  As in the wavefront
// (tb_cell), E and F arrive complete, the cell computes its right
// neighbour's E and its lower neighbour's F (gap opened from its H or extended)
// and stores 4 bits, inverted (1 = not equal): H = diagonal value, H = E,
// En = the opened gap value, Fn = the opened gap value.  Cells that are not
// needed still compute: the band they form is wider than the winner's, and the
// banded DP is exact for any band holding every alignment of the score (cells
// left of column 1 score a mismatch and so stay at the H = 0 border; cells right
// of j* feed only cells right of j*).
//
// Scores: per row and read, the window codes of the row's W cells come from one
// funnel shift of the staged window words; XOR with the row's query code gives
// 2 bits per cell (0: match), folded to one mismatch bit per cell.  Four cells'
// bits are spread to four bytes (0x80 + 0x11 n: the prmt selector nibbles n,
// n | 8 that pick byte n of the score table sign-extended), and per cell one
// prmt takes read A's byte and read B's into the selector of a second prmt that
// picks both scores.  Direction words, one per 4 cells and row, hold read A's 4
// nibbles in the low half and read B's in the high half, in a per-warp scratch
// laid out [row][word][lane] so that a warp's stores coalesce.
constexpr int kTbPWarps = 4;                     // warps per block
constexpr int kTbPQ = kReadWords;                // staged query words per read
// staged window words per read for rows of at most MAXW cells (band offsets
// 0 .. 255 + MAXW - 1, read by funnel shifts of consecutive words)
template <int MAXW>
__host__ __device__ constexpr int tbp_rwords() { return (kMaxReadLen + MAXW - 1) / 16 + 1; }
// per-lane shared words [query A][query B][window A][window B] (odd: conflict-free)
template <int MAXW>
__host__ __device__ constexpr int tbp_lane() { return 2 * kTbPQ + 2 * tbp_rwords<MAXW>() + 1; }
static_assert(tbp_lane<16>() % 2 == 1 && tbp_lane<32>() % 2 == 1, "odd per-lane stride");

struct TbPairConst {
  uint32_t NEG2, ONE2, NGOE2, NGE2, tab;
  uint32_t K2, KN[3];  // 2, 16, 256, 4096 held in registers: the multiply-adds stay on the FMA pipe
};

// codes 0..3 of query row i (1-based) of a staged read, complemented for the
// '-' strand by the caller's mask
__device__ __forceinline__ uint32_t tbp_qcode(const uint32_t* q, const TbRead& t, int i) {
  const int p = t.strand ? max(static_cast<int>(t.m) - i, 0) : i - 1;
  return (q[p >> 4] >> ((p & 15) * 2)) & 3u;
}
// window code of band offset u (column u + dlo + 1)
__device__ __forceinline__ uint32_t tbp_rcode(const uint32_t* r, int u) { return (r[u >> 4] >> ((u & 15) * 2)) & 3u; }

// walk read X (0: low half, 1: high half) back from (i*, j*) through the scratch
// of direction words with Q words per row
__device__ __forceinline__ void tbp_walk(const TbArgs& a, const TbRead& t, uint32_t istar, int X, const uint32_t* dirs,
                                         int Q, const uint32_t* q, const uint32_t* r) {
  const int32_t goe = a.go + a.ge;
  uint32_t* out = a.cigar_slots + static_cast<uint64_t>(t.r) * kCigarStride;
  const uint32_t cm = t.strand ? 3u : 0u;
  int i = static_cast<int>(istar), j = static_cast<int>(t.jstar);
  int kk = j - i - t.dlo;
  int32_t h = t.S;
  int state = 0;
  uint32_t nr = 0, cur_op = 0xffu, cur_len = 0;
  bool bad = istar == kNoRow;
  const int limit = t.ihi + static_cast<int>(t.jstar) + 4;
  const int sh0 = 16 * X;
  auto nib_at = [&](int ii, int k) {
    const uint32_t wd = dirs[(static_cast<uint32_t>((ii - 1) * Q + (k >> 2))) * 32u];
    return ((wd >> (sh0 + 4 * (k & 3))) & 15u) ^ 15u;
  };
  for (int it = 0; !bad; ++it) {
    if (it > limit || kk < 0 || kk >= t.w || i < 1 || j < 1) {
      bad = !(state == 0 && h == 0);
      break;
    }
    uint32_t op;
    if (state == 0) {
      if (h == 0) break;
      // a run of up to 8 diagonal steps: the words of band cell kk in rows
      // i .. i - 7 load together, so a run pays one memory latency, not eight
      uint32_t wv[8];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        wv[c] = i - c >= 1 ? dirs[static_cast<uint32_t>((i - 1 - c) * Q + (kk >> 2)) * 32u] : 0u;
      const int sh = sh0 + 4 * (kk & 3);
      int L = 0;
      bool run = true;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (run) {
          const int ii = i - c, jj = j - c;
          const uint32_t nib = ((wv[c] >> sh) & 15u) ^ 15u;
          if (ii < 1 || jj < 1 || h == 0 || !(nib & 1u)) {
            run = false;
          } else {
            h -= (tbp_qcode(q, t, ii) ^ cm) == tbp_rcode(r, jj - 1 - t.dlo) ? a.sa : -a.sb;
            ++L;
          }
        }
      }
      if (L == 0) {  // (i, j) did not come from the diagonal: a gap ends here
        state = ((((wv[0] >> sh) & 15u) ^ 15u) & 2u) ? 1 : 2;
        continue;
      }
      i -= L;
      j -= L;
      if (cur_op == 0u) {
        cur_len += static_cast<uint32_t>(L);
      } else {
        if (nr + 4 >= static_cast<uint32_t>(kCigarStride)) {
          bad = true;
          break;
        }
        if (cur_len) out[1 + nr++] = (cur_len << 4) | cur_op;
        cur_op = 0u;  // M
        cur_len = static_cast<uint32_t>(L);
      }
      continue;
    } else {
      op = state == 1 ? 2u : 1u;  // D : I
      if (op == 2u) {
        --j;
        --kk;
      } else {
        --i;
        ++kk;
      }
      // the cell the gap came from holds whether it was opened there
      if (i < 1 || j < 1 || kk < 0 || kk >= t.w) {
        bad = true;
        break;
      }
      const uint32_t nib = nib_at(i, kk);
      const bool open = op == 2u ? (nib & 4u) : (nib & 8u);
      h += open ? goe : a.ge;
      if (open) state = 0;
    }
    if (op == cur_op) {
      ++cur_len;
    } else {
      if (nr + 4 >= static_cast<uint32_t>(kCigarStride)) {
        bad = true;
        break;
      }
      if (cur_len) out[1 + nr++] = (cur_len << 4) | cur_op;
      cur_op = op;
      cur_len = 1;
    }
  }
  DevHit* hp = a.hits + static_cast<uint64_t>(t.r) * a.slots;
  if (bad || nr + 3 > static_cast<uint32_t>(kCigarStride)) {
    atomicOr(a.status, kStInternal);
    hp->cigar_len = 0;
    return;
  }
  if (cur_len) out[1 + nr++] = (cur_len << 4) | cur_op;
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
  if (istar < t.m) out[nc++] = ((t.m - istar) << 4) | 4u;
  hp->read_start = static_cast<int32_t>(start_i);
  hp->read_end = static_cast<int32_t>(istar);
  hp->start_j = static_cast<uint32_t>(j) + 1u;
  hp->cigar_len = nc;
}

// the band DP of a thread's two reads (W cells per row), then both walks; RW
// window words are staged per read
template <int W, int RW>
__device__ __forceinline__ void tb_pair_reads(const TbArgs& a, const TbRead (&t)[2], uint32_t* dirs,
                                              const uint32_t* sq, const uint32_t* sr, const TbPairConst& c) {
  static_assert(W == 4 || W == 8 || W == 16 || W == 32, "cells per row");
  constexpr int Q = W / 4;                 // direction words per row
  constexpr int NS = W > 16 ? 2 : 1;       // 16-cell code slices per row
  const int rows = max(t[0].has ? t[0].ihi : 0, t[1].has ? t[1].ihi : 0);
  uint32_t Hp[W], Fp[W];  // the row above: H, and the F it sends down-left
#pragma unroll
  for (int k = 0; k < W; ++k) {
    Hp[k] = 0u;
    Fp[k] = c.NGOE2;
  }
  // per read: the complement mask of its query codes, the shift of its
  // virtual-cell mask, the rows where the band crosses column j* inside
  // [ilo, ihi], and i*
  uint32_t cmask[2], ist[2];
  int lsh[2], clo[2], chi[2];
#pragma unroll
  for (int X = 0; X < 2; ++X) {
    cmask[X] = t[X].strand ? 0xffffffffu : 0u;
    // cells k < 1 - i - dlo lie left of column 1: in a row's first slice they are
    // the low cells of 0x55555555 shifted right by 32 - 2 (1 - i - dlo) (clamped
    // to 0 .. 32), in the second slice by 32 more
    lsh[X] = 32 + 2 * t[X].dlo;
    const int jd = static_cast<int>(t[X].jstar) - t[X].dlo;  // row where cell 0 is column j*
    clo[X] = t[X].has ? max(t[X].ilo, jd - W + 1) : 1;
    chi[X] = t[X].has ? min(t[X].ihi, jd) : 0;
    ist[X] = kNoRow;
  }
  const uint32_t* q0 = sq;
  const uint32_t* q1 = sq + kTbPQ;
  const uint32_t* r0 = sr;
  const uint32_t* r1 = sr + RW;
  for (int i = 1; i <= rows; ++i) {
    // mismatch bits of the row (slice s, bit 2k: cell 16 s + k), per read
    uint32_t nb[2][NS];
#pragma unroll
    for (int X = 0; X < 2; ++X) {
      const uint32_t* q = X ? q1 : q0;
      const uint32_t* r = X ? r1 : r0;
      const int u = i - 1;  // band offset of cell 0
      const uint32_t qr = imad_u32(tbp_qcode(q, t[X], i), 0x55555555u, 0u) ^ cmask[X];
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const uint32_t cw = __funnelshift_r(r[(u >> 4) + sl], r[(u >> 4) + sl + 1], (u & 15) * 2);
        const uint32_t lm = __funnelshift_rc(0x55555555u, 0u, static_cast<uint32_t>(max(lsh[X] + 32 * sl, 0)));
        const uint32_t x = (cw ^ qr) | lm;
        nb[X][sl] = (x | (x >> 1)) & 0x55555555u;
      }
      lsh[X] += 2;
    }
    uint32_t E = c.NGOE2;  // arriving at cell 0 from outside the band
    uint32_t acc = 0u, sA = 0u, sB = 0u;
    uint32_t* drow = dirs + static_cast<uint32_t>((i - 1) * Q) * 32u;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      if ((k & 3) == 0) {
        // cells k .. k + 3: mismatch bits at 0, 2, 4, 6 -> bytes 0x80 + 0x11 n
        const uint32_t sel4 = 0x4440u | static_cast<uint32_t>((k >> 2) & 3);
        const uint32_t bA = tb_prmt(nb[0][k >> 4], 0u, sel4);
        const uint32_t bB = tb_prmt(nb[1][k >> 4], 0u, sel4);
        sA = imad_u32(imad_u32(bA, 0x41041u, 0u) & 0x01010101u, 0x11u, 0x80808080u);
        sB = imad_u32(imad_u32(bB, 0x41041u, 0u) & 0x01010101u, 0x11u, 0x80808080u);
      }
      const uint32_t sel = tb_prmt(sA, sB, static_cast<uint32_t>((k & 3) | ((4 + (k & 3)) << 4)));
      const uint32_t sc = tb_prmt(c.tab, 0u, sel);
      const uint32_t F = k + 1 < W ? Fp[k + 1] : c.NGOE2;
      const uint32_t hs = __viaddmax_s16x2(Hp[k], sc, c.NEG2);
      const uint32_t H = __vimax3_s16x2_relu(hs, E, F);
      const uint32_t g = __viaddmax_s16x2(H, c.NGOE2, c.NEG2);
      const uint32_t En = __viaddmax_s16x2(E, c.NGE2, g);
      const uint32_t Fn = __viaddmax_s16x2(F, c.NGE2, g);
      // bits (inverted) by Horner steps: Fn, En, H = E, H = diagonal
      uint32_t z = imad_u32(__vimin3_u16x2(Fn ^ g, c.ONE2, c.ONE2), c.K2, __vimin3_u16x2(En ^ g, c.ONE2, c.ONE2));
      z = imad_u32(z, c.K2, __vimin3_u16x2(H ^ E, c.ONE2, c.ONE2));
      z = imad_u32(z, c.K2, __vimin3_u16x2(H ^ hs, c.ONE2, c.ONE2));
      acc = (k & 3) ? imad_u32(z, c.KN[(k & 3) - 1], acc) : z;
      if ((k & 3) == 3) drow[(k >> 2) * 32] = acc;
      Hp[k] = H;
      Fp[k] = Fn;
      E = En;
    }
    // end rows: the smallest row in [ilo, ihi] whose cell in column j* holds S
#pragma unroll
    for (int X = 0; X < 2; ++X) {
      if (ist[X] == kNoRow && i >= clo[X] && i <= chi[X]) {
        const int kc = static_cast<int>(t[X].jstar) - i - t[X].dlo;
        uint32_t hc = 0u;
#pragma unroll
        for (int k = 0; k < W; ++k) hc = k == kc ? Hp[k] : hc;
        const int32_t v = X ? static_cast<int16_t>(hc >> 16) : static_cast<int16_t>(hc & 0xffffu);
        if (v == t[X].S) ist[X] = static_cast<uint32_t>(i);
      }
    }
  }
  if (t[0].has) tbp_walk(a, t[0], ist[0], 0, dirs, Q, q0, r0);
  if (t[1].has) tbp_walk(a, t[1], ist[1], 1, dirs, Q, q1, r1);
}

// Reads of bands up to MAXW diagonals (16: buckets 0-4, each warp running the
// narrowest row width, 4, 8 or 16 cells, that holds its reads; 32: bucket 5),
// in band-width order, 64 per warp.
template <int MAXW>
__global__ void __launch_bounds__(32 * kTbPWarps) k_tb_pair(TbArgs a, const uint32_t* list, const uint32_t* range_lo,
                                                          const uint32_t* range_hi, uint32_t* scratch,
                                                          uint32_t n_warps) {
  constexpr int RW = tbp_rwords<MAXW>();
  constexpr int LANE = tbp_lane<MAXW>();
  __shared__ uint32_t s_s[kTbPWarps][32 * LANE];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint32_t gw = blockIdx.x * kTbPWarps + warp;
  if (gw >= n_warps) return;
  uint32_t* dirs = scratch + static_cast<uint64_t>(gw) * kMaxReadLen * (MAXW / 4) * 32 + lane;
  uint32_t* sq = s_s[warp] + lane * LANE;  // [query A][query B][window A][window B]
  uint32_t* sr = sq + 2 * kTbPQ;
  auto pack2 = [](int32_t v) { return (static_cast<uint32_t>(v) & 0xffffu) * 0x10001u; };
  const int32_t goe = a.go + a.ge;
  TbPairConst c;
  c.NEG2 = 0x80008000u;
  c.ONE2 = 0x00010001u;
  c.NGOE2 = pack2(-goe);
  c.NGE2 = pack2(-a.ge);
  c.tab = (static_cast<uint32_t>(a.sa) & 0xffu) | ((static_cast<uint32_t>(-a.sb) & 0xffu) << 8);
  c.K2 = a.k2;
  c.KN[0] = a.k2 << 3;
  c.KN[1] = a.k2 << 7;
  c.KN[2] = a.k2 << 11;
  const uint32_t first = range_lo[0];
  const uint32_t count = range_hi[1] - first;
  for (uint32_t base = gw * 64u; base < count; base += n_warps * 64u) {
    TbRead t[2];
#pragma unroll
    for (int X = 0; X < 2; ++X) {
      const uint32_t li = base + 2 * lane + X;
      t[X] = tb_load(a, li < count, li < count ? list[first + li] : 0u);
      if (t[X].has && t[X].w > MAXW) {  // routed by band width, so never expected: keep the scratch in bounds
        atomicOr(a.status, kStInternal);
        t[X].has = false;
      }
      uint32_t* q = sq + X * kTbPQ;
      uint32_t* r = sr + X * RW;
      if (!t[X].has) continue;
      const uint32_t* row = a.rpack + static_cast<uint64_t>(t[X].rd) * kReadWords;
      for (int w = 0; w < kTbPQ; ++w) q[w] = row[w];
      // band offsets 16 w .. 16 w + 15 hold window positions dlo + 16 w + b:
      // reference words realigned; positions before the reference start or past
      // j* (never needed) read as 0
      const int64_t nref = static_cast<int64_t>((t[X].ws + t[X].jstar) >> 4) + 1;
      for (int w = 0; w < RW; ++w) {
        const int64_t P = static_cast<int64_t>(t[X].ws) + t[X].dlo + 16 * w;
        uint32_t v = 0u;
        if (t[X].dlo + 16 * w <= static_cast<int>(t[X].jstar)) {
          const int64_t wi = P >> 4;  // floor
          const uint32_t sh = static_cast<uint32_t>(P & 15) * 2u;
          const uint32_t lo = (wi >= 0 && wi <= nref) ? t[X].ref[wi] : 0u;
          const uint32_t hi = (wi + 1 >= 0 && wi + 1 <= nref) ? t[X].ref[wi + 1] : 0u;
          v = __funnelshift_r(lo, hi, sh);
        }
        r[w] = v;
      }
    }
    if (MAXW == 32) {
      tb_pair_reads<32, RW>(a, t, dirs, sq, sr, c);
    } else {
      uint32_t wmax = 0;
#pragma unroll
      for (int X = 0; X < 2; ++X) wmax = max(wmax, t[X].has ? static_cast<uint32_t>(t[X].w) : 0u);
      wmax = __reduce_max_sync(FULL, wmax);
      if (wmax <= 4)
        tb_pair_reads<4, RW>(a, t, dirs, sq, sr, c);
      else if (wmax <= 8)
        tb_pair_reads<8, RW>(a, t, dirs, sq, sr, c);
      else
        tb_pair_reads<16, RW>(a, t, dirs, sq, sr, c);
    }
  }
}

// Routing: clears reads without a winner, writes the CIGAR of reads matched
// base for base (no DP needed), picks each other winner's traceback kernel
// (band <= 1 / 2 / 4 / 8 / 16 / 32 / 64 diagonals, else the full-rectangle kernel) and counts the
// sort code bucket * 256 + (256 - last row), so that each kernel's reads come
// sorted by the number of rows their DP runs, longest first.
__global__ void __launch_bounds__(1024) k_tb_route(TbArgs a, uint32_t* code, uint32_t* hist) {
  __shared__ uint32_t sh[kTbCodes];
  for (int c = threadIdx.x; c < kTbCodes; c += blockDim.x) sh[c] = 0;
  __syncthreads();
  const uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (r < a.n_reads) {
    uint32_t cd = kNoRow;
    DevHit* hp = a.hits + r * a.slots;
    const int32_t item = hp->item, S = hp->score;
    if (item < 0 || S <= 0) {
      hp->read_start = hp->read_end = 0;
      hp->start_j = 0;
      hp->cigar_len = 0;
    } else {
      const uint32_t m = a.rlen[a.item_read[item]];
      const uint32_t jstar = a.item_end[item];
      int bucket = -1;
      uint32_t last = m;
      if (m >= 1 && jstar >= m && static_cast<int64_t>(S) == static_cast<int64_t>(a.sa) * m) {
        // every base matched: any mismatch or gap scores below match * m, so the
        // alignment is the whole read on one diagonal ending at (m, j*)
        a.cigar_slots[static_cast<uint64_t>(r) * kCigarStride] = m << 4;  // m M
        hp->read_start = 1;
        hp->read_end = static_cast<int32_t>(m);
        hp->start_j = jstar - m + 1u;
        hp->cigar_len = 1;
      } else if (a.tb_flag[r] == kTbFlagFull) {
        bucket = kTbBuckets - 1;
      } else {
        uint32_t ilo = 0, ihi = 0;
        if (jstar == 0 || m == 0 || m > kMaxReadLen || !tb_rows(a, static_cast<uint32_t>(r), item, S, m, &ilo, &ihi)) {
          atomicOr(a.status, kStInternal);
          hp->cigar_len = 0;
        } else {
          const TbBand b = tb_band(a.sa, a.go, a.ge, S, jstar, ilo, ihi);
          bucket = b.w <= 1 ? 0 : b.w <= 2 ? 1 : b.w <= 4 ? 2 : b.w <= 8 ? 3 : b.w <= 16 ? 4
                 : b.w <= 32 ? 5 : b.w <= kTbMaxBand ? 6 : kTbBuckets - 1;
          last = ihi;
        }
      }
      if (bucket >= 0) {
        cd = static_cast<uint32_t>(bucket) * kMaxReadLen + (kMaxReadLen - last);
        atomicAdd(&sh[cd], 1u);
      }
    }
    code[r] = cd;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kTbCodes; c += blockDim.x)
    if (sh[c]) atomicAdd(&hist[c], sh[c]);
}

// exclusive offsets of the codes (one block, two codes per thread) and each
// bucket's [begin, end) in the sorted list
constexpr int kTbScanThreads = (kTbCodes + 1) / 2;
static_assert(kTbScanThreads <= 1024, "traceback code scan block");
__global__ void __launch_bounds__(kTbScanThreads) k_tb_scan(uint32_t* cnt) {
  __shared__ uint32_t sh[kTbScanThreads];
  const int t = threadIdx.x;
  const uint32_t v0 = 2 * t < kTbCodes ? cnt[2 * t] : 0u;
  const uint32_t v1 = 2 * t + 1 < kTbCodes ? cnt[2 * t + 1] : 0u;
  sh[t] = v0 + v1;
  __syncthreads();
  for (int off = 1; off < kTbScanThreads; off <<= 1) {
    const uint32_t x = t >= off ? sh[t - off] : 0u;
    __syncthreads();
    sh[t] += x;
    __syncthreads();
  }
  const uint32_t ex0 = sh[t] - v0 - v1;
  if (2 * t < kTbCodes) cnt[kTbCodes + 2 * t] = ex0;
  if (2 * t + 1 < kTbCodes) cnt[kTbCodes + 2 * t + 1] = ex0 + v0;
  __syncthreads();
  if (t < kTbBuckets) {
    // bucket t spans codes [t * 256, (t + 1) * 256): begin = exclusive offset of its first code
    const int c0 = t * kMaxReadLen, c1 = (t + 1) * kMaxReadLen;
    cnt[2 * kTbCodes + 2 * t] = cnt[kTbCodes + c0];
    cnt[2 * kTbCodes + 2 * t + 1] = cnt[kTbCodes + c1 - 1] + cnt[c1 - 1];
  }
}

__global__ void k_tb_scatter(uint32_t n_reads, const uint32_t* code, uint32_t* cursor, uint32_t* list) {
  const uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const uint32_t cd = r < n_reads ? code[r] : kNoRow;
  const bool live = cd != kNoRow;
  const uint32_t act = __ballot_sync(FULL, live);
  if (!live) return;
  const uint32_t peers = __match_any_sync(act, cd);
  const int ln = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t b0 = 0;
  if (ln == leader) b0 = atomicAdd(&cursor[cd], static_cast<uint32_t>(__popc(peers)));
  b0 = __shfl_sync(peers, b0, leader);
  list[b0 + __popc(peers & ((1u << ln) - 1u))] = static_cast<uint32_t>(r);
}

}  // namespace

int launch_traceback(const BatchDev& b, const DevRefs& refs, const ScoreConst& sc, int mode,
                     int n_refs, cudaStream_t st, const Fanout* fan) {
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
  a.tb_flag = b.tb_flag;
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
  a.k2 = 2u;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  uint32_t* code = b.tb_list;
  uint32_t* list = b.tb_list + b.n_reads;
  uint32_t* hist = b.tb_count;
  uint32_t* cursor = b.tb_count + kTbCodes;
  const uint32_t* ranges = b.tb_count + 2 * kTbCodes;
  if (cudaMemsetAsync(hist, 0, kTbCodes * sizeof(uint32_t), st) != cudaSuccess) return -1;
  k_tb_route<<<(b.n_reads + 1023) / 1024, 1024, 0, st>>>(a, code, hist);
  k_tb_scan<<<1, kTbScanThreads, 0, st>>>(b.tb_count);
  k_tb_scatter<<<(b.n_reads + 255) / 256, 256, 0, st>>>(b.n_reads, code, cursor, list);
  int launched = 3;
  if (fan && fanout_begin(*fan, st) < 0) return -1;
  int next = 0;
  const int width = fan_width(b.n_reads);
  auto lane_of = [&]() { return fan ? fan->side[next++ % width] : st; };
  auto wave = [&](auto kern, int bucket, int per_warp) -> bool {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kTbWarps, 0) != cudaSuccess) return false;
    const uint32_t g0 = static_cast<uint32_t>(nsm) * static_cast<uint32_t>(per_sm > 0 ? per_sm : 1);
    const uint32_t need = (b.n_reads + kTbWarps * per_warp - 1) / (kTbWarps * per_warp);
    kern<<<need < g0 ? need : g0, 32 * kTbWarps, 0, lane_of()>>>(a, list, ranges + 2 * bucket);
    ++launched;
    return cudaPeekAtLastError() == cudaSuccess;
  };
  // bands of at most 8 diagonals (buckets 0-3, adjacent in the sorted list): one
  // thread per read, one launch
  auto threads = [&]() -> bool {
    const uint32_t nw = tb_thread_warps(b.n_reads);
    k_tb_thread<<<(nw + kTbTWarps - 1) / kTbTWarps, 32 * kTbTWarps, 0, lane_of()>>>(
        a, list, ranges + 2 * 0, ranges + 2 * 3, b.tb_dirs, nw);
    ++launched;
    return cudaPeekAtLastError() == cudaSuccess;
  };
  // bands of at most 16 diagonals (buckets 0-4) with packed scores: two reads
  // per thread, one launch
  // bands of at most 16 diagonals (buckets 0-4) and of 17-32 (bucket 5) with
  // packed scores: two reads per thread, one launch each, each with a scratch of
  // its own
  auto pairs = [&](auto kern, int b0, int b1, uint32_t nw_max, uint32_t* scratch) -> bool {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kTbPWarps, 0) != cudaSuccess)
      return false;
    const uint32_t cap = static_cast<uint32_t>(nsm) * static_cast<uint32_t>(per_sm > 0 ? per_sm : 1) * kTbPWarps;
    const uint32_t nw = std::min(nw_max, cap);  // within the carved scratch
    kern<<<(nw + kTbPWarps - 1) / kTbPWarps, 32 * kTbPWarps, 0, lane_of()>>>(a, list, ranges + 2 * b0,
                                                                          ranges + 2 * b1, scratch, nw);
    ++launched;
    return cudaPeekAtLastError() == cudaSuccess;
  };
  // widest bands (longest kernels) first
  const bool pair = tb_pair_fits(a.sa, a.sb, a.go, a.ge);
  if (!wave(k_tb_wave2, 6, 2) ||
      !(pair ? pairs(k_tb_pair<32>, 5, 5, tb_pair32_warps(b.n_reads), b.tb_dirs32)
             : wave(k_tb_wave<32>, 5, 2)) ||
      !(pair ? pairs(k_tb_pair<16>, 0, 4, tb_pair_warps(b.n_reads), b.tb_dirs)
             : (wave(k_tb_wave<16>, 4, 4) && threads())))
    return -1;
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
  k_traceback<<<grid, 32, smem, lane_of()>>>(a, list, ranges + 2 * (kTbBuckets - 1));
  ++launched;
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  if (fan && fanout_end(*fan, st) < 0) return -1;
  return launched;
}

int preload_traceback() {
  int n_ = 0;
  SR_TOUCH(k_traceback);
  SR_TOUCH(k_tb_wave<16>);
  SR_TOUCH(k_tb_wave<32>);
  SR_TOUCH(k_tb_wave2);
  SR_TOUCH(k_tb_thread);
  SR_TOUCH(k_tb_pair<16>);
  SR_TOUCH(k_tb_pair<32>);
  SR_TOUCH(k_tb_route);
  SR_TOUCH(k_tb_scan);
  SR_TOUCH(k_tb_scatter);
  return n_;
}

}  // namespace sr
