// sr_extend.cuh -- score-only affine-gap Smith-Waterman extension of every
// (read, window) item (McVicar et al., arXiv 1805.00106, Sec. 3.5).
//
// Kernel shape: the GPU form of the paper's 1-D systolic array (Sec. 3.5,
// Fig. 6).  A group of G lanes holds the read, R rows per lane; the window
// streams through the group, lane t working on column j = step - t, so the
// group sweeps anti-diagonal wavefronts.  Each step a lane receives the bottom
// row of the lane above (H and F at column j) by a warp shuffle.  Each lane
// carries two independent items in the 16-bit halves of every register
// (s16x2) and updates them with packed DPX instructions:
//
//   E(i,j) = max(E(i,j-1) - ge, H(i,j-1) - (go+ge))
//   F(i,j) = max(F(i-1,j) - ge, H(i-1,j) - (go+ge))
//   H(i,j) = max(0, H(i-1,j-1) + s(q_i, r_j), E(i,j), F(i,j))
//
// Values are stored as T = H - (go+ge) plus a bias of kBias, so every half
// stays positive (the subtraction is a plain 32-bit add without cross-half
// borrow, which issues at full rate beside the half-rate DPX and PRMT) and the
// zero floor of H becomes a max with the bias.  The
// substitution score s + (go+ge) comes from a per-row 8-byte table held in two
// registers and is picked with one byte permute (prmt.b32) whose selector encodes
// the two items' window bases at column j (sign-extended int8 -> int16).
//
// The best cell: per lane, the max over its rows of each column is compared
// with the running best; a strict improvement records the column, so the
// smallest column reaching the best wins; the group then reduces
// (score, -column) keys.  The keys and the top-border substitution of lane 0
// are built with integer multiply-adds, which issue on the FMA pipe, so that
// the ALU pipe carries the recurrence, the column maximum and two key maxima.  Rows beyond the read are added at the top with
// mismatch scores; they stay at H = 0 and leave the recurrence unchanged
// (they act like the H = 0 / F = -inf top border).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sr_internal.h"

#pragma once

namespace sr {

struct ExtArgs {
  const uint32_t* rpack;
  const uint32_t* rlen;
  const uint8_t* c_ref;
  const uint8_t* c_strand;
  const uint64_t* c_start;
  const uint32_t* c_len;
  const uint32_t* item_read;
  const uint32_t* order;        // sorted item list (batched); nullptr = identity
  const uint32_t* class_range;  // begin/end of this class in `order` (batched)
  uint32_t* queue;              // this class's task counter (persistent)
  DevRefs refs;
  int32_t* item_score;
  uint32_t* item_end;
  uint32_t* item_iend;          // winner end-row search (mode 2): smallest row at the end column
  uint32_t* status;
  uint64_t n_items;             // plain engine: items in input order
  int cls;
  int32_t sa, sb, go, ge;
  // 65536, passed at run time so that the per-column key arithmetic stays
  // multiply-adds (the FMA pipe) instead of being folded into shifts and
  // byte permutes on the ALU pipe, which the recurrence saturates
  uint32_t k16;
};

// kernel shapes (lanes per alignment, rows per lane) instantiated for the batched
// engine; the plain engine uses the 256-row shapes only
#define SR_SHAPES(X)                                                                         \
  X(4, 16) X(4, 20) X(4, 24) X(4, 28) X(4, 32) X(8, 8) X(8, 10) X(8, 12) X(8, 13) X(8, 14)   \
      X(8, 15) X(8, 16) X(8, 17) X(8, 18) X(8, 19) X(8, 20) X(8, 21) X(8, 22) X(8, 23)      \
      X(8, 24) X(8, 25) X(8, 26) X(8, 27) X(8, 28) X(8, 29) X(8, 30) X(8, 31) X(8, 32)      \
      X(16, 5) X(16, 6) X(16, 7) X(16, 8) X(16, 9) X(16, 10) X(16, 11) X(16, 12) X(16, 13)  \
      X(16, 14) X(16, 15) X(16, 16) X(32, 4) X(32, 5) X(32, 6) X(32, 7) X(32, 8)
#define SR_PLAIN_SHAPES(X) X(16, 16) X(32, 8)

// launch the int16 kernel of one shape and readout mode; -1 if the shape is not built
int dispatch_mode0(bool persist, uint32_t lanes, uint32_t rows, const ExtArgs& a, cudaStream_t st,
                   uint64_t plain_tasks);
int dispatch_mode1(bool persist, uint32_t lanes, uint32_t rows, const ExtArgs& a, cudaStream_t st,
                   uint64_t plain_tasks);
int dispatch_mode2(uint32_t lanes, uint32_t rows, const ExtArgs& a, cudaStream_t st);

namespace {


constexpr uint32_t FULL = 0xffffffffu;
constexpr int kStageWords = 40;      // >= 36 words needed for a 512-base window
constexpr long kWaitLimit = 1 << 22; // bounded mbarrier polls
constexpr int kColLead = 32;         // >= G - 1 virtual columns before column 0

// Selector of a real column: the low half of the result is byte b_lo of the lo
// table sign-extended, the high half byte 4 + b_hi (the hi table) sign-extended.
// A virtual half picks the sign of a byte for both of its bytes, so its score
// term is 0 or -1, below go + ge.  With it, a lane may run columns outside an
// item's window: before column 0 every value stays at the H = 0 border
// (H(i-1,j-1) + s - (go+ge) < 0), and past the last column every value is
// strictly below the best real cell already seen (each term subtracts ge or
// more from a real value), so neither changes the tracked best.
constexpr uint32_t kSelLo = 0x0080u, kSelHi = 0xC400u;
constexpr uint32_t kVirtLo = 0x0088u, kVirtHi = 0xCC00u;

struct __align__(16) GroupSmem {
  uint32_t stage[2][kStageWords];  // 16-byte aligned TMA destinations
  unsigned long long mbar;
  uint32_t pad[2];
  // per column j (stored at j + kColLead): PRMT selector of the two items' bases;
  // columns before the window and past each item's end hold the virtual selector
  uint16_t col[kMaxWinLen + 2 * kColLead];
};
static_assert(sizeof(GroupSmem) % 16 == 0, "group smem alignment");


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false if the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// a * b + c and the high word of a * b as 32-bit integer multiply-adds (issued
// on the FMA pipe, beside the ALU pipe that runs the DPX recurrence)
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t imulhi(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// byte permute, default mode: selector nibble bits 2:0 pick one of the 8 bytes
// of {b, a}; bit 3 replicates that byte's sign bit (PTX prmt.b32)
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// 2-bit code of base p of a packed word array
__device__ __forceinline__ uint32_t base_at(const uint32_t* w, uint32_t p) {
  return (w[p >> 4] >> ((p & 15u) * 2u)) & 3u;
}

// word range [w0, w0 + nw) holding window [ws, ws + n), 16-byte aligned
__device__ __forceinline__ void window_words(uint64_t ws, uint32_t n, uint64_t* w0,
                                             uint32_t* nw) {
  uint64_t a = (ws >> 6) << 2;
  uint64_t b = ((ws + n + 63) >> 6) << 2;
  *w0 = a;
  *nw = static_cast<uint32_t>(b - a);
}

struct ItemDesc {
  uint32_t item, read, m, n, strand, ref;
  uint64_t ws;
};

__device__ __forceinline__ ItemDesc load_item(const ExtArgs& a, uint32_t item, bool to_end) {
  ItemDesc d;
  d.item = item;
  d.read = a.item_read[item];
  d.m = a.rlen[d.read];
  d.n = to_end ? a.item_end[item] : a.c_len[item];
  d.strand = a.c_strand[item];
  d.ref = a.c_ref[item];
  d.ws = a.c_start[item];
  return d;
}

// read base (2-bit code) of real row i (0-based) as aligned: '-' strand reads
// are reverse-complemented (Sec. 3.1 strand bit).
__device__ __forceinline__ uint32_t read_code(const uint32_t* row, uint32_t m, uint32_t strand,
                                              uint32_t i) {
  return strand ? 3u - base_at(row, m - 1u - i) : base_at(row, i);
}

// Blocks of 128 threads per SM the register budget is cut for (the sweep is
// bound by the ALU pipe and the latency of its DPX chains, so resident warps
// count).  Persistent kernels: up to 12 rows per lane fit 80 registers (6
// blocks, 24 warps per SM), up to 17 rows 96 (16 in final-row mode, which keeps
// more per row; 5 blocks), up to 24 rows (22) 128 (4 blocks), up to 32 rows
// (30) 168 (3 blocks), more up to 255.  The one-launch (plain) kernels keep the 128
// register budget up to 24 rows.  None of them spills.
template <int R, int MODE, bool PERSIST>
constexpr int ext_min_blocks() {
  return (PERSIST && R <= 12) ? 6
         : (PERSIST && R <= (MODE == 1 ? 16 : 17)) ? 5
         : R <= (MODE == 1 ? 22 : 24) ? 4
         : (R <= (MODE == 1 ? 30 : 32) ? 3 : 2);
}

template <int G, int R, int MODE, bool PERSIST>
__global__ void __launch_bounds__(128, ext_min_blocks<R, MODE, PERSIST>()) k_extend16(ExtArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int GPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int glane = lane & (G - 1);
  const int gidx = lane / G;
  GroupSmem* gs = reinterpret_cast<GroupSmem*>(smem_raw) + (warp * GPW + gidx);

  const int32_t goe = a.go + a.ge;
  const uint32_t GOE2 = static_cast<uint32_t>(goe) * 0x10001u;
  const uint32_t NGE2 = (static_cast<uint32_t>(-a.ge) & 0xffffu) * 0x10001u;
  const uint32_t BIAS2 = static_cast<uint32_t>(kBias) * 0x10001u;
  const uint32_t INIT = static_cast<uint32_t>(kBias - goe) * 0x10001u;  // T of H = 0
  const uint32_t mis_b = static_cast<uint32_t>(goe - a.sb) & 0xffu;
  const uint32_t hit_b = static_cast<uint32_t>(a.sa + goe) & 0xffu;
  const uint32_t MIS4 = mis_b * 0x01010101u;

  if (glane == 0) {
    mbar_init(&gs->mbar, 1);
    fence_mbar_init();
  }
  for (int c = glane; c < kColLead; c += G) gs->col[c] = static_cast<uint16_t>(kVirtLo | kVirtHi);
  __syncwarp();
  uint32_t phase = 0;

  uint32_t begin = 0, count;
  if (PERSIST) {
    begin = a.class_range[2 * a.cls];
    count = a.class_range[2 * a.cls + 1] - begin;
  } else {
    count = static_cast<uint32_t>(a.n_items);
  }
  const uint32_t n_tasks = (count + 1) / 2;
  const uint32_t warps_per_block = blockDim.x >> 5;

  for (uint32_t round = 0;; ++round) {
    uint32_t base;
    if (PERSIST) {
      uint32_t b0 = 0;
      if (lane == 0) b0 = atomicAdd(a.queue + a.cls, static_cast<uint32_t>(GPW));
      base = __shfl_sync(FULL, b0, 0);
    } else {
      if (round > 0) break;
      base = (blockIdx.x * warps_per_block + warp) * GPW;
    }
    if (base >= n_tasks) break;
    const uint32_t task = base + gidx;
    const bool has_task = task < n_tasks;

    // ---- the pair of items of this group
    ItemDesc lo{}, hi{};
    bool hi_valid = false;
    if (has_task) {
      uint32_t p0 = begin + 2 * task;
      uint32_t i0 = a.order ? a.order[p0] : p0;
      lo = load_item(a, i0, MODE == 2);
      if (2 * task + 1 < count) {
        uint32_t i1 = a.order ? a.order[p0 + 1] : p0 + 1;
        hi = load_item(a, i1, MODE == 2);
        hi_valid = true;
      } else {
        hi = lo;
      }
    }

    // ---- stage both windows into shared memory with TMA bulk copies (a3)
    uint64_t w0lo = 0, w0hi = 0;
    uint32_t nwlo = 0, nwhi = 0;
    if (has_task) {
      window_words(lo.ws, lo.n, &w0lo, &nwlo);
      window_words(hi.ws, hi.n, &w0hi, &nwhi);
      if (glane == 0) {
        fence_proxy_async();
        mbar_expect_tx(&gs->mbar, (nwlo + nwhi) * 4u);
        tma_load_1d(gs->stage[0], a.refs.words[lo.ref] + w0lo, nwlo * 4u, &gs->mbar);
        tma_load_1d(gs->stage[1], a.refs.words[hi.ref] + w0hi, nwhi * 4u, &gs->mbar);
      }
    }

    // ---- per-row substitution tables (a4: query profile in registers)
    uint32_t TL[R], TH[R];
    const int padlo = G * R - static_cast<int>(lo.m);
    const int padhi = G * R - static_cast<int>(hi.m);
    {
      const uint32_t* rowlo = a.rpack + static_cast<size_t>(lo.read) * kReadWords;
      const uint32_t* rowhi = a.rpack + static_cast<size_t>(hi.read) * kReadWords;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int r = glane * R + k;
        uint32_t tl = MIS4, th = MIS4;
        if (has_task && r >= padlo) {
          uint32_t c = read_code(rowlo, lo.m, lo.strand, static_cast<uint32_t>(r - padlo));
          tl = (MIS4 & ~(0xffu << (8 * c))) | (hit_b << (8 * c));
        }
        if (has_task && r >= padhi) {
          uint32_t c = read_code(rowhi, hi.m, hi.strand, static_cast<uint32_t>(r - padhi));
          th = (MIS4 & ~(0xffu << (8 * c))) | (hit_b << (8 * c));
        }
        TL[k] = tl;
        TH[k] = th;
      }
    }

    // ---- wait for the windows, build the column stream
    bool ok = true;
    if (has_task) {
      ok = mbar_wait_bounded(&gs->mbar, phase);
      if (!ok) {
        atomicOr(a.status, kStTimeout);
        mbar_wait_bounded(&gs->mbar, phase);  // let copies in flight land
      }
      phase ^= 1u;
    }
    if (__any_sync(FULL, !ok)) break;
    const uint32_t nmax = has_task ? max(lo.n, hi.n) : 0u;
    const uint32_t nlo = has_task ? lo.n : 0u, nhi = has_task ? hi.n : 0u;
    const uint32_t wmax = __reduce_max_sync(FULL, nmax);
    const int nsteps = static_cast<int>(wmax) + G - 1;
    {
      // real columns, then virtual ones up to the last column any lane of the warp reaches
      const uint32_t offlo = static_cast<uint32_t>(lo.ws - (w0lo << 4));
      const uint32_t offhi = static_cast<uint32_t>(hi.ws - (w0hi << 4));
      const uint32_t ncol = wmax + G - 1;
      for (uint32_t j = glane; j < ncol; j += G) {
        const uint32_t vlo = j < nlo ? kSelLo + base_at(gs->stage[0], offlo + j) * 0x11u : kVirtLo;
        const uint32_t vhi = j < nhi ? kSelHi + base_at(gs->stage[1], offhi + j) * 0x1100u : kVirtHi;
        gs->col[kColLead + j] = static_cast<uint16_t>(vlo | vhi);
      }
    }
    __syncwarp();

    // ---- the systolic sweep (a5)
    uint32_t T[R], E[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      T[k] = INIT;
      E[k] = INIT;
    }
    uint32_t tprev = INIT, Tbot = INIT, Fbot = INIT;
    // best cell per half as the key (T << 16) | (0xffff - column): the max keeps the
    // highest score and, among equal scores, the smallest (first) column
    const uint32_t KINIT = (INIT & 0xffffu) << 16;
    uint32_t kbl = KINIT, kbh = KINIT;
    // 0x7fff - (column of step s), column = s - glane + 1: in 0x7fff - 544 .. 0x7fff + 31,
    // so it never carries into a key's score half
    const uint32_t jn = 0x7ffeu + static_cast<uint32_t>(glane);
    const uint32_t K16 = a.k16;
    // lane 0's row above is the top border (H = 0, F = -inf): its shuffled-in
    // values v become (v - INIT) * nz + INIT, with nz = 0 on lane 0, else 1
    const uint32_t nz = glane == 0 ? 0u : 1u;
    // mode 2: biased T value of the winner's score in each half, rows found
    uint32_t tgt_lo = 0, tgt_hi = 0, ilo = 0xffffffffu, ihi = 0xffffffffu;
    if (MODE == 2 && has_task) {
      tgt_lo = static_cast<uint32_t>(a.item_score[lo.item] - goe + kBias);
      tgt_hi = static_cast<uint32_t>(a.item_score[hi.item] - goe + kBias);
    }
    const uint32_t lastmask = (MODE == 1 && glane == G - 1) ? FULL : 0u;
    const uint16_t* colp = gs->col + kColLead - glane;  // colp[s] = column s - glane
    for (int s = 0; s < nsteps; ++s) {
      // lane 0's row above is the top border (H = 0, F = -inf): tin = fin = INIT
      const uint32_t tin = imad(__shfl_up_sync(FULL, Tbot, 1, G) - INIT, nz, INIT);
      const uint32_t fin = imad(__shfl_up_sync(FULL, Fbot, 1, G) - INIT, nz, INIT);
      const int j = s - glane;
      {
        const uint32_t sel = colp[s];
        uint32_t td = tprev, tup = tin, f = fin;
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const uint32_t sc = prmt(TL[k], TH[k], sel);
          const uint32_t tl = T[k];
          E[k] = __viaddmax_s16x2(E[k], NGE2, tl);        // E(i,j) = max(E(i,j-1) - ge, T(i,j-1))
          f = __viaddmax_s16x2(f, NGE2, tup);             // F(i,j) = max(F(i-1,j) - ge, T(i-1,j))
          const uint32_t x = __viaddmax_s16x2(td, sc, E[k]);  // max(H(i-1,j-1) + s, E)
          const uint32_t h = __vimax3_s16x2(x, f, BIAS2);     // H = max(x, F, 0)
          td = tl;
          tup = h - GOE2;  // plain add: each half stays >= 0
          T[k] = tup;
        }
        tprev = tin;
        Tbot = T[R - 1];
        Fbot = f;
        if (MODE == 2) {
          if (j == static_cast<int>(lo.n) - 1) {
#pragma unroll
            for (int k = R - 1; k >= 0; --k)
              if ((T[k] & 0xffffu) == tgt_lo) ilo = static_cast<uint32_t>(glane * R + k - padlo + 1);
          }
          if (j == static_cast<int>(hi.n) - 1) {
#pragma unroll
            for (int k = R - 1; k >= 0; --k)
              if ((T[k] >> 16) == tgt_hi) ihi = static_cast<uint32_t>(glane * R + k - padhi + 1);
          }
          continue;
        }
        uint32_t cm;
        if (MODE == 1) {
          cm = T[R - 1] & lastmask;
        } else {
          cm = T[0];
#pragma unroll
          for (int k = 1; k < R; k += 2) cm = __vimax3_s16x2(cm, T[k], T[k + 1 < R ? k + 1 : k]);
        }
        // final-row readout: virtual columns may exceed the final row's best, mask them
        if (MODE == 1)
          cm &= (static_cast<uint32_t>(j) < nlo ? 0xffffu : 0u) |
                (static_cast<uint32_t>(j) < nhi ? 0xffff0000u : 0u);
        // strict improvement per half records the (1-based) column: keys
        // (half << 16) | (0x7fff - column)
        const uint32_t jc = jn - static_cast<uint32_t>(s);
        kbl = max(kbl, imad(cm, K16, jc));
        kbh = max(kbh, imad(imulhi(cm, K16), K16, jc));
      }
    }

    if (MODE == 2) {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) {
        ilo = min(ilo, __shfl_xor_sync(FULL, ilo, off, G));
        ihi = min(ihi, __shfl_xor_sync(FULL, ihi, off, G));
      }
      if (has_task && glane == 0) {
        a.item_iend[lo.item] = ilo;
        if (hi_valid) a.item_iend[hi.item] = ihi;
      }
      __syncwarp();
      continue;
    }
    // ---- group reduction of (score, -column) and write-back
    const uint32_t base_t = static_cast<uint32_t>(kBias - goe) << 16;
    uint32_t klo = kbl - base_t, khi = kbh - base_t;  // (score << 16) | (0xffff - column)
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      klo = max(klo, __shfl_xor_sync(FULL, klo, off, G));
      khi = max(khi, __shfl_xor_sync(FULL, khi, off, G));
    }
    if (has_task && glane == 0) {
      const uint32_t sl = klo >> 16, sh = khi >> 16;
      a.item_score[lo.item] = static_cast<int32_t>(sl);
      a.item_end[lo.item] = sl ? 0x7fffu - (klo & 0xffffu) : 0u;
      if (hi_valid) {
        a.item_score[hi.item] = static_cast<int32_t>(sh);
        a.item_end[hi.item] = sh ? 0x7fffu - (khi & 0xffffu) : 0u;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- int32 path
// Items whose best score could exceed the int16 range (match * read length >
// 32767 - bias) or whose scores do not fit the int8 tables run here: one item
// per 32-lane group, 8 rows per lane, exact int32 arithmetic.
template <int MODE>
__global__ void __launch_bounds__(128) k_extend32(ExtArgs a) {
  constexpr int G = 32, R = 8;
  __shared__ uint8_t colc[4][kMaxWinLen];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int32_t goe = a.go + a.ge;
  const int32_t smatch = a.sa + goe, smis = goe - a.sb;
  uint32_t begin = a.class_range[2 * a.cls];
  uint32_t count = a.class_range[2 * a.cls + 1] - begin;
  for (;;) {
    uint32_t t0 = 0;
    if (lane == 0) t0 = atomicAdd(a.queue + a.cls, 1u);
    const uint32_t task = __shfl_sync(FULL, t0, 0);
    if (task >= count) break;
    const ItemDesc it = load_item(a, a.order[begin + task], false);
    const uint32_t* row = a.rpack + static_cast<size_t>(it.read) * kReadWords;
    const uint32_t* ref = a.refs.words[it.ref];
    for (uint32_t j = lane; j < it.n; j += 32) {
      const uint64_t p = it.ws + j;
      colc[warp][j] = static_cast<uint8_t>((ref[p >> 4] >> ((p & 15u) * 2u)) & 3u);
    }
    uint32_t qc[R];
    const int pad = G * R - static_cast<int>(it.m);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = lane * R + k;
      qc[k] = r >= pad ? read_code(row, it.m, it.strand, static_cast<uint32_t>(r - pad)) : 4u;
    }
    __syncwarp();
    int32_t T[R], E[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      T[k] = -goe;
      E[k] = -goe;
    }
    int32_t tprev = -goe, Tbot = -goe, Fbot = -goe, best = -goe;
    uint32_t jb = 0;
    const int nsteps = static_cast<int>(it.n) + G - 1;
    for (int s = 0; s < nsteps; ++s) {
      int32_t tin = __shfl_up_sync(FULL, Tbot, 1);
      int32_t fin = __shfl_up_sync(FULL, Fbot, 1);
      if (lane == 0) {
        tin = -goe;
        fin = -goe;
      }
      const int j = s - lane;
      if (j >= 0 && j < static_cast<int>(it.n)) {
        const uint32_t rc = colc[warp][j];
        int32_t td = tprev, tup = tin, f = fin;
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const int32_t sc = qc[k] == rc ? smatch : smis;
          const int32_t tl = T[k];
          E[k] = __viaddmax_s32(E[k], -a.ge, tl);
          f = __viaddmax_s32(f, -a.ge, tup);
          const int32_t x = __viaddmax_s32(td, sc, E[k]);
          const int32_t h = __vimax_s32_relu(x, f);
          td = tl;
          tup = h - goe;
          T[k] = tup;
        }
        tprev = tin;
        Tbot = T[R - 1];
        Fbot = f;
        int32_t cm;
        if (MODE == 1) {
          cm = lane == G - 1 ? T[R - 1] : -goe;
        } else {
          cm = T[0];
#pragma unroll
          for (int k = 1; k < R; ++k) cm = max(cm, T[k]);
        }
        if (cm > best) {
          best = cm;
          jb = static_cast<uint32_t>(j + 1);
        }
      }
    }
    const int32_t score = best + goe;
    unsigned long long key =
        (static_cast<unsigned long long>(static_cast<uint32_t>(score)) << 32) |
        (0xffffffffu - (score ? jb : 0u));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      unsigned long long o = __shfl_xor_sync(FULL, key, off);
      key = o > key ? o : key;
    }
    if (lane == 0) {
      const int32_t sc = static_cast<int32_t>(key >> 32);
      a.item_score[it.item] = sc;
      a.item_end[it.item] = sc ? 0xffffffffu - static_cast<uint32_t>(key & 0xffffffffu) : 0u;
    }
    __syncwarp();
  }
}

template <int G, int R, int MODE, bool PERSIST>
int launch16(const ExtArgs& a, cudaStream_t st, uint64_t plain_tasks) {
  constexpr int kThreads = 128;
  constexpr int groups = (kThreads / 32) * (32 / G);
  const size_t smem = sizeof(GroupSmem) * groups;
  auto kern = k_extend16<G, R, MODE, PERSIST>;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return -1;
    attr_set = true;
  }
  int grid;
  if (PERSIST) {
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) !=
        cudaSuccess)
      return -1;
    grid = nsm * (per_sm > 0 ? per_sm : 1);
  } else {
    uint64_t g = (plain_tasks + groups - 1) / groups;
    if (g == 0) return 0;
    grid = static_cast<int>(g);
  }
  kern<<<grid, kThreads, smem, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}


}  // namespace
}  // namespace sr
