// sr_noalloc.cu -- sr_align_items_noalloc: scores (read, window) items that
// already live in device memory without allocating anything.
//
// Who needs this: a caller whose device memory is already owned by another
// allocator (for example a framework's caching allocator that has reserved the
// GPU), or a latency-sensitive caller that cannot afford cudaMalloc/cudaFree,
// which can synchronize the whole device and can fail under fragmentation.
// Such a caller passes its own device buffers for inputs and outputs; the
// scratch this path needs (the work-queue counters, the status word, the
// packed read rows, the read lengths and the item-to-read map) lives in the
// fixed file-scope array below, which every GPU that loads libsr holds for the
// life of the process.
//
// It runs the same kernels as sr_batch_run's batched engine with one kernel
// shape (16 lanes x 16 rows, which covers every read up to 256 bases) and the
// items in input order, after a validation kernel; it returns only when the
// work is done.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current; make that first call before
// any stream capture.  All calls share the one array: two calls whose work
// overlaps on the GPU (from two host threads, or two streams) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "sr_host.h"
#include "sr_internal.h"

namespace sr {
const DevRefs& session_refs(sr_session* s);
uint32_t session_n_refs(sr_session* s);
int session_device(sr_session* s);
sr_status set_error(sr_status st, const char* fmt, ...);
}  // namespace sr

namespace {

constexpr uint32_t kNaMaxReads = SR_NOALLOC_MAX_READS;
constexpr uint32_t kNaMaxItems = SR_NOALLOC_MAX_ITEMS;
// word layout of the scratch array
constexpr size_t kNaUp32(size_t x) { return (x + 31) / 32 * 32; }
constexpr size_t kNaQueue = 0;                                          // kNumClasses + 8 counters
constexpr size_t kNaRange = kNaUp32(sr::kNumClasses + 8);               // 2 * kNumClasses
constexpr size_t kNaStatus = kNaUp32(kNaRange + 2 * sr::kNumClasses);   // 1 word
constexpr size_t kNaRlen = kNaUp32(kNaStatus + 1) + 64;                 // kNaMaxReads
constexpr size_t kNaRpack = kNaRlen + kNaMaxReads;          // kNaMaxReads * 16
constexpr size_t kNaItemRead = kNaRpack + static_cast<size_t>(kNaMaxReads) * sr::kReadWords;
constexpr size_t kNaWords = kNaItemRead + kNaMaxItems;      // about 3.3 MiB in all

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNaWords];

std::mutex g_na_mu;
uint32_t* g_na_ptr[64] = {};

// read_off / cand_off must be monotone CSR offsets starting at 0 that end at
// the stated totals, with read lengths 1..256; sets status bits otherwise.
__global__ void k_noalloc_check(const uint64_t* read_off, const uint64_t* cand_off, uint32_t n_reads,
                                uint64_t n_items, uint32_t* status) {
  const uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  if (r > n_reads) return;
  if (r == 0) {
    if (read_off[0] != 0 || cand_off[0] != 0 || cand_off[n_reads] != n_items) atomicOr(status, sr::kStBadWindow);
    return;
  }
  const uint64_t m = read_off[r] - read_off[r - 1];
  if (read_off[r] < read_off[r - 1] || m == 0 || m > static_cast<uint64_t>(sr::kMaxReadLen))
    atomicOr(status, sr::kStBadRead);
  if (cand_off[r] < cand_off[r - 1] || cand_off[r] > n_items || cand_off[r] - cand_off[r - 1] >= (1ull << 19))
    atomicOr(status, sr::kStBadWindow);
}

sr_status status_error(uint32_t st) {
  if (st & sr::kStBadBase) return sr::set_error(SR_EBADBASE, "sr_align_items_noalloc: read has a non-ACGT base");
  if (st & sr::kStBadRead) return sr::set_error(SR_EINVAL, "sr_align_items_noalloc: bad read offsets or a read length outside 1..256");
  if (st & sr::kStBadWindow) return sr::set_error(SR_EINVAL, "sr_align_items_noalloc: bad window offsets, or a window outside its reference or longer than 512");
  if (st & sr::kStTimeout) return sr::set_error(SR_ETIMEOUT, "sr_align_items_noalloc: device wait for a window copy ran out");
  return sr::set_error(SR_ECUDA, "sr_align_items_noalloc: device check failed (status %u)", st);
}

sr_status cuda_fail(const char* what, cudaError_t e) {
  return sr::set_error(SR_ECUDA, "sr_align_items_noalloc: %s: %s", what, cudaGetErrorString(e));
}

}  // namespace

extern "C" sr_status sr_align_items_noalloc(sr_session* s, const char* d_bases, const uint64_t* d_read_off,
                                            uint32_t n_reads, const uint64_t* d_cand_off, const uint8_t* d_ref_id,
                                            const uint8_t* d_strand, const uint64_t* d_win_start,
                                            const uint32_t* d_win_len, uint64_t n_items,
                                            const sr_score_params* sp, int32_t* d_item_score,
                                            uint32_t* d_item_end, void* cuda_stream) {
  using namespace sr;
  if (!s || !sp || !d_read_off || !d_cand_off || (n_reads && !d_bases) ||
      (n_items && (!d_ref_id || !d_strand || !d_win_start || !d_win_len || !d_item_score || !d_item_end)))
    return set_error(SR_EINVAL, "sr_align_items_noalloc: null argument");
  if (n_reads > kNaMaxReads || n_items > kNaMaxItems)
    return set_error(SR_EINVAL, "sr_align_items_noalloc: at most %u reads and %u windows per call (got %u, %llu)",
                     kNaMaxReads, kNaMaxItems, n_reads, static_cast<unsigned long long>(n_items));
  const int32_t goe = sp->gap_open + sp->gap_extend;
  if (sp->match < 1 || sp->mismatch < 1 || sp->gap_open < 0 || sp->gap_extend < 1 || sp->match + goe > 127 ||
      goe - sp->mismatch < -128 || goe + sp->gap_extend + 256 >= kBias ||
      static_cast<int64_t>(sp->match) * kMaxReadLen > 32767 - kBias)
    return set_error(SR_EINVAL, "sr_align_items_noalloc: scores must fit the packed 16-bit kernel (use sr_align_batch)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return cuda_fail("device", e);
  // the session's references live on its device; kernels run on the current one
  if (dev != session_device(s))
    return set_error(SR_EINVAL, "sr_align_items_noalloc: current device %d is not the session's device %d", dev,
                     session_device(s));
  uint32_t* base;
  {
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return cuda_fail("cudaGetSymbolAddress", e);
      g_na_ptr[dev] = static_cast<uint32_t*>(p);
    }
    base = g_na_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t* status = base + kNaStatus;
  // counters and the status word must start at zero on every call
  e = cudaMemsetAsync(base, 0, kNaRlen * sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail("clear", e);
  if (n_reads == 0) return cudaStreamSynchronize(st) == cudaSuccess ? SR_OK : cuda_fail("sync", cudaGetLastError());
  k_noalloc_check<<<(n_reads + 256) / 256, 256, 0, st>>>(d_read_off, d_cand_off, n_reads, n_items, status);
  uint32_t hst = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("offset check", e);
  if (hst) return status_error(hst);

  BatchDev d{};
  d.bases = d_bases;
  d.read_off = d_read_off;
  d.cand_off = d_cand_off;
  d.c_ref = d_ref_id;
  d.c_strand = d_strand;
  d.c_start = d_win_start;
  d.c_len = d_win_len;
  d.n_reads = n_reads;
  d.n_items = n_items;
  d.rpack = base + kNaRpack;
  d.rlen = base + kNaRlen;
  d.item_read = base + kNaItemRead;
  d.status = status;
  d.queue = base + kNaQueue;
  d.class_range = base + kNaRange;
  d.order = nullptr;  // items in input order
  d.item_score = d_item_score;
  d.item_end = d_item_end;
  const DevRefs& refs = session_refs(s);
  // pack reads into the scratch rows and validate every window
  if (launch_prepare(d, refs, st) < 0) return cuda_fail("prepare", cudaGetLastError());
  e = cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("validation", e);
  if (hst) return status_error(hst);
  if (n_items == 0) return SR_OK;
  // every item in the first length bin, run with the 16 x 16 shape
  uint32_t range[2 * kNumClasses];
  for (int c = 0; c < kNumClasses; ++c) {
    range[2 * c] = c == 0 ? 0u : static_cast<uint32_t>(n_items);
    range[2 * c + 1] = static_cast<uint32_t>(n_items);
  }
  e = cudaMemcpyAsync(d.class_range, range, sizeof(range), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail("ranges", e);
  TuneBin bins[kNumBins];
  for (int c = 0; c < kNumBins; ++c) bins[c] = TuneBin{kMaxReadLen, 16, 16};
  const ScoreConst sc{sp->match, sp->mismatch, sp->gap_open, sp->gap_extend};
  // only the first class holds items: one persistent 16 x 16 grid, no int32 grid
  uint64_t class_items[kNumClasses] = {};
  class_items[0] = n_items;
  if (launch_extend(d, refs, sc, bins, kNumBins, 0, false, 16, 16, st, class_items) < 0)
    return cuda_fail("extension", cudaGetLastError());
  e = cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("extension", e);
  if (hst) return status_error(hst);
  return SR_OK;
}

namespace sr {
int preload_noalloc() {
  int n_ = 0;
  SR_TOUCH(k_noalloc_check);
  return n_;
}
}  // namespace sr
