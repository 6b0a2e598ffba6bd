// sr_session.cpp -- sessions (device-resident references), batches (staging,
// the device pipeline as one CUDA graph, fetch), classification, the
// autotuner table and the C ABI glue of libsr.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sr_host.h"
#include "sr_internal.h"
#include "sr_serve.h"

namespace sr {

static thread_local std::string g_err;

sr_status set_error(sr_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

static sr_status cuda_error(const char* where, cudaError_t e) {
  return set_error(SR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// ---- autotuner table (read-length bins -> kernel shape)
static std::mutex g_tune_mu;
// defaults = the autotuner's picks on GB300 for the c2 score parameters
static TuneBin g_bins[kNumBins] = {
    {64, 4, 16},   {80, 8, 10},   {96, 8, 12},   {104, 8, 13},  {112, 8, 14},  {120, 8, 15},
    {128, 8, 16},  {136, 8, 17},  {144, 8, 18},  {152, 8, 19},  {160, 8, 20},  {168, 8, 21},
    {176, 8, 22},  {184, 8, 23},  {192, 8, 24},  {200, 8, 25},  {208, 8, 26},  {216, 8, 27},
    {224, 8, 28},  {232, 8, 29},  {240, 8, 30},  {248, 8, 31},  {256, 8, 32}};

void tune_get_bins(TuneBin* out) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  memcpy(out, g_bins, sizeof(g_bins));
}
void tune_set_bins(const TuneBin* in) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  memcpy(g_bins, in, sizeof(g_bins));
}

static sr_status check_score(const sr_score_params* sp) {
  if (!sp) return set_error(SR_EINVAL, "null score params");
  const int lim = 1 << 20;
  if (sp->match < 1 || sp->mismatch < 1 || sp->gap_open < 0 || sp->gap_extend < 1 ||
      sp->match > lim || sp->mismatch > lim || sp->gap_open > lim || sp->gap_extend > lim)
    return set_error(SR_EINVAL,
                     "score params: need match >= 1, mismatch >= 1, gap_open >= 0, gap_extend >= 1, each <= 2^20");
  return SR_OK;
}

static sr_align_opts default_opts() {
  sr_align_opts o{};
  o.mode = SR_MODE_LOCAL;
  o.engine = SR_ENGINE_BATCHED;
  o.want_cigar = 1;
  o.classify = 0;
  o.min_score = 40;
  o.margin = 5;
  return o;
}

}  // namespace sr

using namespace sr;

namespace {
// A batch's timing events and the side streams and fork/join events of its
// fan-out phases.  Creating streams and events costs tens of microseconds, so
// the session keeps those of freed batches for the next ones.
struct BatchRes {
  cudaEvent_t ev[6] = {};  // around: whole path, extension kernels, traceback
  Fanout fan[2] = {};      // extension and traceback phases (the same side streams)
};

void res_destroy(BatchRes& r) {
  for (auto ev : r.ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& f : r.fan) {
    if (f.fork) cudaEventDestroy(f.fork);
    for (auto j : f.join)
      if (j) cudaEventDestroy(j);
  }
  for (auto x : r.fan[0].side)
    if (x) {
      cudaStreamSynchronize(x);
      cudaStreamDestroy(x);
    }
  r = BatchRes{};
}

bool res_create(BatchRes& r) {
  bool ok = true;
  for (auto& ev : r.ev) ok = ok && cudaEventCreate(&ev) == cudaSuccess;
  cudaStream_t side[kSide] = {};
  for (auto& x : side) ok = ok && cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) == cudaSuccess;
  for (auto& f : r.fan) {
    for (int i = 0; i < kSide; ++i) f.side[i] = side[i];
    ok = ok && cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) == cudaSuccess;
    for (auto& j : f.join) ok = ok && cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) res_destroy(r);
  return ok;
}
constexpr size_t kResPool = 16;
constexpr size_t kKeptArenas = 3;
// a positive integer from the environment, else dflt
uint64_t env_u64(const char* name, uint64_t dflt) {
  const char* v = getenv(name);
  if (!v || !*v) return dflt;
  char* end = nullptr;
  const unsigned long long x = strtoull(v, &end, 10);
  return (end && *end == 0 && x > 0) ? static_cast<uint64_t>(x) : dflt;
}
// roles of the device CAL finder's cached scratch buffers
enum CalBuf : int {
  kCbBases, kCbRoff, kCbCount, kCbActual, kCbStatus, kCbSlots, kCbPre, kCbSums, kCbBounds, kCbPlan,
  kCbRanges, kCbSeedOff, kCbRecount, kCbCpre, kCbOff, kCbNwin, kCbWoff, kCbWsums, kCbBig, kCbBigOff,
  kCbCals, kCbWkey, kCbWhits, kCbWlen, kCbScratch, kCbLoff, kCbLref, kCbLstr, kCbLstart, kCbLlen, kCbLhits,
  kCalBufs
};
}  // namespace

struct sr_session {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t part_stream[3] = {};  // the parts of a large sr_align_batch call
  uint32_t n_refs = 0;
  std::vector<uint32_t*> d_words;
  std::vector<uint64_t> lens;
  DevRefs refs{};
  uint64_t hbm_budget = 0;
  std::atomic<uint64_t> hbm_used{0};
  Server* server = nullptr;
  // the handle plus one per live batch: a batch keeps its session alive, so the
  // two may be released in either order
  std::atomic<int> live{1};
  // device copy of the references' indexes (sr_session_attach_index)
  DevIndex didx{};
  std::vector<void*> idx_bufs;
  // pinned host blocks that held fetched results, kept for the next fetch
  std::mutex pool_mu;
  std::vector<std::pair<void*, uint64_t>> pool;
  // arenas of freed batches, kept for the next ones (not counted in hbm_used):
  // up to kKeptArenas, so that neither a two-deep serving pipeline nor the
  // parts of a large sr_align_batch call allocate anything in steady state
  std::mutex spare_mu;
  std::vector<std::pair<void*, uint64_t>> spares;
  // streams and events of freed batches
  std::mutex res_mu;
  std::vector<BatchRes> res_pool;
  // scratch of the device CAL finder by role, kept between calls and grown on
  // demand (not counted in hbm_used); one sr_candidates_device call at a time
  std::mutex cal_mu;
  void* cal_buf[kCalBufs] = {};
  uint64_t cal_bytes[kCalBufs] = {};
};

struct sr_batch {
  sr_session* s = nullptr;
  cudaStream_t stream = nullptr;
  BatchDev d{};
  void* arena = nullptr;
  uint64_t bytes = 0;        // carved size (counted in the session's hbm_used)
  uint64_t arena_bytes = 0;  // allocated size (>= bytes: a kept arena, or allocated with headroom)
  uint32_t n_reads = 0;
  uint64_t n_items = 0;
  uint64_t cells = 0;
  uint64_t items_by_len[kMaxReadLen + 1] = {};  // windows per read length
  uint32_t max_m = 0;
  cudaGraphExec_t graph = nullptr;
  sr_score_params g_sp{};
  sr_align_opts g_opts{};
  TuneBin g_bins[kNumBins]{};
  uint64_t kernels = 0;
  uint64_t i32_items = 0;
  bool ran = false;
  bool assembled = false;  // the last run also assembled the result records (serving rounds)
  sr_align_opts last_opts{};
  BatchRes res{};  // events, side streams (from the session's pool)
  bool res_ok = false;
};

extern "C" const char* sr_last_error(void) { return g_err.c_str(); }
extern "C" const char* sr_version(void) { return "libsr 0.1 (sm_103a)"; }

// ------------------------------------------------------------------ session
// every kernel of the library loaded once per device (see preload_kernels)
static void preload_all(int dev) {
  static std::mutex mu;
  static bool done[64] = {};
  std::lock_guard<std::mutex> g(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  preload_mode0();
  preload_mode1();
  preload_mode2();
  preload_extend();
  preload_kernels();
  preload_traceback();
  preload_cal();
  preload_report();
  preload_noalloc();
  cudaGetLastError();
  done[dev] = true;
}

static sr_status open_common(const uint8_t* const* codes, const char* const* ascii,
                             const uint64_t* lens, uint32_t n_refs, uint64_t budget,
                             sr_session** out) {
  if (!out || n_refs == 0 || n_refs > SR_MAX_REFS) return set_error(SR_EINVAL, "session: 1..16 references");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return set_error(SR_ECUDA, "session: no CUDA device available");
  auto* s = new sr_session;
  cudaGetDevice(&s->device);
  preload_all(s->device);
  e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  for (auto& x : s->part_stream)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (s->stream) cudaStreamDestroy(s->stream);
    for (auto x : s->part_stream)
      if (x) cudaStreamDestroy(x);
    delete s;
    return cuda_error("session stream", e);
  }
  s->hbm_budget = budget;
  s->n_refs = n_refs;
  uint32_t* d_status = nullptr;
  e = cudaMalloc(&d_status, 4);
  if (e != cudaSuccess) {
    sr_session_close(s);
    return cuda_error("session status", e);
  }
  cudaMemsetAsync(d_status, 0, 4, s->stream);
  for (uint32_t r = 0; r < n_refs; ++r) {
    const uint64_t len = lens[r];
    if (len == 0 || len >= (1ull << 40)) {
      cudaFree(d_status);
      sr_session_close(s);
      return set_error(SR_EINVAL, "session: reference length out of range");
    }
    const uint64_t nw = ((len + 63) / 64) * 4 + 16;
    uint32_t* w = nullptr;
    e = cudaMalloc(&w, nw * 4);
    if (e != cudaSuccess) {
      cudaFree(d_status);
      sr_session_close(s);
      return cuda_error("session reference", e);
    }
    s->d_words.push_back(w);
    s->lens.push_back(len);
    // upload ASCII in chunks and pack on the device (a1)
    const uint64_t chunk = 1ull << 28;  // 256 MiB, a multiple of 64 bases
    char* d_ascii = nullptr;
    e = cudaMalloc(&d_ascii, std::min(len, chunk));
    if (e != cudaSuccess) {
      cudaFree(d_status);
      sr_session_close(s);
      return cuda_error("session staging", e);
    }
    std::vector<char> tmp;
    for (uint64_t off = 0; off < len; off += chunk) {
      const uint64_t n = std::min(chunk, len - off);
      const char* src;
      if (ascii) {
        src = ascii[r] + off;
      } else {
        tmp.resize(n);
        static const char L[4] = {'A', 'C', 'G', 'T'};
        for (uint64_t i = 0; i < n; ++i) tmp[i] = L[codes[r][off + i] & 3];
        src = tmp.data();
      }
      e = cudaMemcpyAsync(d_ascii, src, n, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess && launch_pack_refs(d_ascii, n, w + off / 16, d_status, s->stream) < 0)
        e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) break;
    }
    cudaFree(d_ascii);
    if (e != cudaSuccess) {
      cudaFree(d_status);
      sr_session_close(s);
      return cuda_error("session pack", e);
    }
    s->refs.words[r] = w;
    s->refs.len[r] = len;
  }
  s->refs.n = static_cast<int>(n_refs);
  uint32_t st = 0;
  cudaMemcpy(&st, d_status, 4, cudaMemcpyDeviceToHost);
  cudaFree(d_status);
  if (st & kStBadBase) {
    sr_session_close(s);
    return set_error(SR_EBADBASE, "session: reference has a non-ACGT base");
  }
  *out = s;
  return SR_OK;
}

extern "C" sr_status sr_session_open(const sr_index* const* refs, uint32_t n_refs, uint64_t hbm_budget,
                                     sr_session** out) {
  if (!refs) return set_error(SR_EINVAL, "sr_session_open: null refs");
  std::vector<const uint8_t*> codes(n_refs);
  std::vector<uint64_t> lens(n_refs);
  for (uint32_t r = 0; r < n_refs; ++r) {
    if (!refs[r]) return set_error(SR_EINVAL, "sr_session_open: null index");
    codes[r] = index_codes(refs[r], &lens[r]);
  }
  return open_common(codes.data(), nullptr, lens.data(), n_refs, hbm_budget, out);
}

extern "C" sr_status sr_session_open_seqs(const char* const* seqs, const uint64_t* lens, uint32_t n_refs,
                                          uint64_t hbm_budget, sr_session** out) {
  if (!seqs || !lens) return set_error(SR_EINVAL, "sr_session_open_seqs: null argument");
  return open_common(nullptr, seqs, lens, n_refs, hbm_budget, out);
}

static void session_release(sr_session* s) {
  if (s->live.fetch_sub(1) != 1) return;
  for (auto* w : s->d_words) cudaFree(w);
  for (auto* p : s->idx_bufs) cudaFree(p);
  for (auto& b : s->pool) cudaFreeHost(b.first);
  for (auto& r : s->res_pool) res_destroy(r);
  for (auto& a : s->spares) cudaFree(a.first);
  for (void* p : s->cal_buf)
    if (p) cudaFree(p);
  if (s->stream) cudaStreamDestroy(s->stream);
  for (auto x : s->part_stream)
    if (x) cudaStreamDestroy(x);
  delete s;
}

extern "C" void sr_session_close(sr_session* s) {
  if (!s) return;
  if (s->server) {
    serve_destroy(s->server);
    s->server = nullptr;
  }
  session_release(s);
}

namespace sr {
cudaStream_t session_stream(sr_session* s) { return s->stream; }
uint64_t session_budget(sr_session* s) { return s->hbm_budget; }
std::atomic<uint64_t>& session_used(sr_session* s) { return s->hbm_used; }
Server*& session_server(sr_session* s) { return s->server; }
uint32_t session_n_refs(sr_session* s) { return s->n_refs; }
const DevRefs& session_refs(sr_session* s) { return s->refs; }
int session_device(sr_session* s) { return s->device; }
}  // namespace sr

// ------------------------------------------------------------------ batches
namespace {

struct Carve {
  uint64_t off = 0;
  template <class T>
  void take(T*& p, uint64_t count) {
    off = (off + 255) & ~255ull;
    p = reinterpret_cast<T*>(off);
    off += (count ? count : 1) * sizeof(T);
  }
};

template <class T>
void rebase(T*& p, char* base) {
  p = reinterpret_cast<T*>(base + reinterpret_cast<uint64_t>(p));
}
template <class T>
void rebase_c(const T*& p, char* base) {
  p = reinterpret_cast<const T*>(base + reinterpret_cast<uint64_t>(p));
}

}  // namespace

namespace sr {
namespace {
// Lays out a batch's arena: every pointer of d becomes an offset from the
// arena's start; returns the bytes the arena needs.
uint64_t carve_batch(BatchDev& d, uint32_t n, uint64_t nb, uint64_t nc, uint32_t n_refs) {
  Carve c;
  char* p1;
  c.take(p1, nb);
  d.bases = p1;
  uint64_t* p8;
  c.take(p8, n + 1ull);
  d.read_off = p8;
  c.take(p8, n + 1ull);
  d.cand_off = p8;
  uint8_t* pu8;
  c.take(pu8, nc);
  d.c_ref = pu8;
  c.take(pu8, nc);
  d.c_strand = pu8;
  c.take(p8, nc);
  d.c_start = p8;
  uint32_t* p4;
  c.take(p4, nc);
  d.c_len = p4;
  c.take(d.rpack, n * 16ull);
  c.take(d.rlen, n);
  c.take(d.item_read, nc);
  c.take(d.item_key, nc);
  c.take(d.order, nc);
  c.take(d.hist, kNumKeys);
  c.take(d.cursor, kNumKeys);
  c.take(d.class_range, 2 * kNumClasses);
  c.take(d.queue, kNumClasses + 8);
  c.take(d.status, 4);
  c.take(d.item_score, nc);
  c.take(d.item_end, nc);
  c.take(d.hits, static_cast<uint64_t>(n) * (1 + n_refs));
  c.take(d.cigar_slots, static_cast<uint64_t>(n) * kCigarStride);
  c.take(d.cigar_off, n + 1ull);
  c.take(d.cigar, static_cast<uint64_t>(n) * kCigarStride);
  c.take(d.read_class, n);
  c.take(d.scan_tmp, n / 1024 + 4ull);
  c.take(d.item_iend, nc);
  c.take(d.wcount, kNumClasses);
  c.take(d.wrange, 2 * kNumClasses);
  c.take(d.wqueue, kNumClasses + 8);
  c.take(d.tb_flag, n);
  c.take(d.tb_list, 2ull * n);
  c.take(d.tb_count, kTbCountWords);
  c.take(d.tb_dirs, tb_dirs_words(n));
  c.take(d.tb_dirs32, tb_dirs32_words(n));
  c.take(d.out_best, n);
  c.take(d.out_per_ref, static_cast<uint64_t>(n) * n_refs);
  StageCheck* pc;
  c.take(pc, 1);
  d.check = pc;
  return c.off + 256;
}

void rebase_batch(BatchDev& d, char* base) {
  rebase_c(d.bases, base);
  rebase_c(d.read_off, base);
  rebase_c(d.cand_off, base);
  rebase_c(d.c_ref, base);
  rebase_c(d.c_strand, base);
  rebase_c(d.c_start, base);
  rebase_c(d.c_len, base);
  rebase(d.rpack, base);
  rebase(d.rlen, base);
  rebase(d.item_read, base);
  rebase(d.item_key, base);
  rebase(d.order, base);
  rebase(d.hist, base);
  rebase(d.cursor, base);
  rebase(d.class_range, base);
  rebase(d.queue, base);
  rebase(d.status, base);
  rebase(d.item_score, base);
  rebase(d.item_end, base);
  rebase(d.hits, base);
  rebase(d.cigar_slots, base);
  rebase(d.cigar_off, base);
  rebase(d.cigar, base);
  rebase(d.read_class, base);
  rebase(d.scan_tmp, base);
  rebase(d.item_iend, base);
  rebase(d.wcount, base);
  rebase(d.wrange, base);
  rebase(d.wqueue, base);
  rebase(d.tb_flag, base);
  rebase(d.tb_list, base);
  rebase(d.tb_count, base);
  rebase(d.tb_dirs, base);
  rebase(d.tb_dirs32, base);
  rebase(d.out_best, base);
  rebase(d.out_per_ref, base);
  rebase(d.check, base);
}
}  // namespace

uint64_t batch_bytes_estimate(uint32_t n_reads, uint64_t n_items, uint64_t n_bases, uint32_t n_refs) {
  BatchDev d;
  return carve_batch(d, n_reads, n_bases, n_items, n_refs);
}
}  // namespace sr

namespace {
// A batch of n reads, nb bases and nc windows on `stream`, its arena taken from
// the session's kept arenas or allocated, and its events and side streams from
// the session's pool.  Counts its bytes in the session's hbm_used.
sr_status batch_alloc(sr_session* s, uint32_t n, uint64_t nb, uint64_t nc, cudaStream_t stream, bool check_budget,
                      sr_batch** out) {
  BatchDev d;
  const uint64_t bytes = carve_batch(d, n, nb, nc, s->n_refs);
  if (check_budget && s->hbm_budget && s->hbm_used.load() + bytes > s->hbm_budget)
    return set_error(SR_ENOMEM, "sr_batch_stage: batch needs %llu bytes, over the HBM budget",
                     static_cast<unsigned long long>(bytes));
  auto* b = new sr_batch;
  b->s = s;
  s->live.fetch_add(1);
  b->stream = stream;
  b->n_reads = n;
  b->n_items = nc;
  b->bytes = bytes;
  {
    // the smallest kept arena that holds this batch
    std::lock_guard<std::mutex> lk(s->spare_mu);
    int pick = -1;
    for (int i = 0; i < static_cast<int>(s->spares.size()); ++i)
      if (s->spares[i].second >= b->bytes && (pick < 0 || s->spares[i].second < s->spares[pick].second)) pick = i;
    if (pick >= 0) {
      b->arena = s->spares[pick].first;
      b->arena_bytes = s->spares[pick].second;
      s->spares.erase(s->spares.begin() + pick);
    }
  }
  if (!b->arena) {
    // a quarter of headroom, so batches a little larger later reuse this arena
    uint64_t want = b->bytes + b->bytes / 4;
    cudaError_t e = cudaMalloc(&b->arena, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      want = b->bytes;
      e = cudaMalloc(&b->arena, want);
    }
    if (e != cudaSuccess) {
      // the kept arenas may be what is in the way
      cudaGetLastError();
      std::vector<std::pair<void*, uint64_t>> sp;
      {
        std::lock_guard<std::mutex> lk(s->spare_mu);
        sp.swap(s->spares);
      }
      if (!sp.empty()) {
        for (auto& a : sp) cudaFree(a.first);
        e = cudaMalloc(&b->arena, want);
      }
      if (e != cudaSuccess) {
        b->arena = nullptr;
        sr_batch_free(b);
        cudaGetLastError();
        return set_error(SR_ENOMEM, "sr_batch_stage: device allocation of %llu bytes failed",
                         static_cast<unsigned long long>(bytes));
      }
    }
    b->arena_bytes = want;
  }
  rebase_batch(d, static_cast<char*>(b->arena));
  d.n_reads = n;
  d.n_items = nc;
  b->d = d;
  s->hbm_used += b->bytes;
  {
    std::lock_guard<std::mutex> lk(s->res_mu);
    if (!s->res_pool.empty()) {
      b->res = s->res_pool.back();
      s->res_pool.pop_back();
      b->res_ok = true;
    }
  }
  if (!b->res_ok) {
    if (!res_create(b->res)) {
      sr_batch_free(b);
      return cuda_error("sr_batch_stage streams", cudaGetLastError());
    }
    b->res_ok = true;
  }
  *out = b;
  return SR_OK;
}

// Stages a batch whose reads or candidates (sr_reads / sr_cand_list flags) sit
// in device memory: the header is read with two small copies, every array is
// copied into the arena (device to device, or host to device for the other
// struct) and checked there by a kernel, which also counts the cells and the
// windows per read length.  Errors name the same read and window as the host
// checks do.
sr_status stage_device(sr_session* s, const sr_reads* reads, const sr_cand_list* cands, cudaStream_t st,
                       bool check_budget, sr_batch** out) {
  const uint32_t n = reads->n_reads;
  const bool rdev = (reads->flags & SR_FLAG_DEVICE) != 0, cdev = (cands->flags & SR_FLAG_DEVICE) != 0;
  if (n > (8u << 20)) return set_error(SR_EINVAL, "sr_batch_stage: more than 8M reads in one batch");
  if (!reads->offsets || !cands->offsets || (n && !reads->bases))
    return set_error(SR_EINVAL, "sr_batch_stage: null arrays");
  // offsets[0] and offsets[n] of both lists
  uint64_t ends[4] = {};
  cudaError_t e = cudaSuccess;
  auto get = [&](uint64_t* dst, const uint64_t* src, bool dev) {
    if (!dev) *dst = *src;
    else if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, 8, cudaMemcpyDefault, st);
  };
  get(&ends[0], reads->offsets, rdev);
  get(&ends[1], reads->offsets + n, rdev);
  get(&ends[2], cands->offsets, cdev);
  get(&ends[3], cands->offsets + n, cdev);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error("sr_batch_stage offsets", e);
  if (ends[0] != 0 || ends[2] != 0) return set_error(SR_EINVAL, "sr_batch_stage: offsets must start at 0");
  const uint64_t nb = ends[1], nc = ends[3];
  if (nc != cands->n_cands) return set_error(SR_EINVAL, "sr_batch_stage: n_cands != offsets[n_reads]");
  if (nc >= (1ull << 32)) return set_error(SR_EINVAL, "sr_batch_stage: too many windows");
  if (nc && (!cands->ref_id || !cands->strand || !cands->win_start || !cands->win_len))
    return set_error(SR_EINVAL, "sr_batch_stage: null candidate arrays");
  if (nb > static_cast<uint64_t>(n) * SR_MAX_READ_LEN)
    return set_error(SR_EINVAL, "sr_batch_stage: %llu bases in %u reads: some read is longer than %d",
                     static_cast<unsigned long long>(nb), n, SR_MAX_READ_LEN);
  sr_batch* b = nullptr;
  sr_status rs = batch_alloc(s, n, nb, nc, st, check_budget, &b);
  if (rs != SR_OK) return rs;
  BatchDev& d = b->d;
  auto copy = [&](const void* dst, const void* src, uint64_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyDefault, st);
  };
  copy(d.bases, reads->bases, nb);
  copy(d.read_off, reads->offsets, (n + 1ull) * 8);
  copy(d.cand_off, cands->offsets, (n + 1ull) * 8);
  copy(d.c_ref, cands->ref_id, nc);
  copy(d.c_strand, cands->strand, nc);
  copy(d.c_start, cands->win_start, nc * 8);
  copy(d.c_len, cands->win_len, nc * 4);
  StageCheck* dc = static_cast<StageCheck*>(d.check);
  if (e == cudaSuccess && launch_stage_check(d, s->refs, dc, st) < 0) e = cudaGetLastError();
  StageCheck hc{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, dc, sizeof(hc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && hc.bad != ~0ull && (hc.bad & 7) == 4) {
    if (launch_first_bad_window(d, s->refs, static_cast<uint32_t>(hc.bad >> 3), dc, st) < 0) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc.bad_win, &dc->bad_win, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(st);
    sr_batch_free(b);
    return cuda_error("sr_batch_stage copy", e);
  }
  if (hc.bad != ~0ull) {
    sr_batch_free(b);
    const uint32_t r = static_cast<uint32_t>(hc.bad >> 3);
    switch (hc.bad & 7) {
      case 1:
        return set_error(SR_EINVAL, "sr_batch_stage: decreasing or out-of-range offsets at read %u", r);
      case 2:
        return set_error(SR_EINVAL, "sr_batch_stage: read %u has a length outside 1..256", r);
      case 3:
        return set_error(SR_EINVAL, "sr_batch_stage: read %u has more than 2^19-1 windows", r);
      default:
        return set_error(SR_EINVAL, "sr_batch_stage: window %llu is outside its reference or malformed",
                         static_cast<unsigned long long>(hc.bad_win));
    }
  }
  b->cells = hc.cells;
  b->max_m = hc.max_m;
  for (int m = 0; m <= kMaxReadLen; ++m) b->items_by_len[m] = hc.by_len[m];
  *out = b;
  return SR_OK;
}
}  // namespace

extern "C" sr_status sr_batch_stage(sr_session* s, const sr_reads* reads, const sr_cand_list* cands,
                                    void* cuda_stream, sr_batch** out) {
  return batch_stage_internal(s, reads, cands, cuda_stream, true, out);
}

sr_status sr::batch_stage_internal(sr_session* s, const sr_reads* reads, const sr_cand_list* cands,
                                   void* cuda_stream, bool check_budget, sr_batch** out) {
  return batch_stage_range(s, reads, cands, 0, reads ? reads->n_reads : 0, cuda_stream, check_budget, out);
}

// Stages reads [r0, r1) of the caller's arrays (and their windows) as one
// batch: the whole list's header is checked, the range's arrays are copied and
// its offsets made batch-relative on the device.  Reads and windows named in
// error messages keep their indexes in the caller's arrays.
sr_status sr::batch_stage_range(sr_session* s, const sr_reads* reads, const sr_cand_list* cands, uint32_t r0,
                                uint32_t r1, void* cuda_stream, bool check_budget, sr_batch** out) {
  Trace trace_("sr_batch_stage");
  if (!s || !reads || !cands || !out) return set_error(SR_EINVAL, "sr_batch_stage: null argument");
  *out = nullptr;
  const uint32_t n_all = reads->n_reads;
  if (cands->n_reads != n_all) return set_error(SR_EINVAL, "sr_batch_stage: reads and candidates differ in n_reads");
  if ((reads->flags | cands->flags) & ~static_cast<uint32_t>(SR_FLAG_DEVICE))
    return set_error(SR_EINVAL, "sr_batch_stage: unknown flags");
  const cudaStream_t stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : s->stream;
  if ((reads->flags | cands->flags) & SR_FLAG_DEVICE) {
    if (r0 != 0 || r1 != n_all) return set_error(SR_EINVAL, "sr_batch_stage: device inputs are staged whole");
    return stage_device(s, reads, cands, stream, check_budget, out);
  }
  if (r0 > r1 || r1 > n_all) return set_error(SR_EINVAL, "sr_batch_stage: bad read range");
  const uint32_t n = r1 - r0;
  if (n > (8u << 20)) return set_error(SR_EINVAL, "sr_batch_stage: more than 8M reads in one batch");
  if (n_all && (!reads->offsets || !reads->bases || !cands->offsets))
    return set_error(SR_EINVAL, "sr_batch_stage: null arrays");
  const uint64_t nc_all = n_all ? cands->offsets[n_all] : 0;
  if (n_all && (reads->offsets[0] != 0 || cands->offsets[0] != 0))
    return set_error(SR_EINVAL, "sr_batch_stage: offsets must start at 0");
  if (nc_all != cands->n_cands) return set_error(SR_EINVAL, "sr_batch_stage: n_cands != offsets[n_reads]");
  if (nc_all >= (1ull << 32)) return set_error(SR_EINVAL, "sr_batch_stage: too many windows");
  if (nc_all && (!cands->ref_id || !cands->strand || !cands->win_start || !cands->win_len))
    return set_error(SR_EINVAL, "sr_batch_stage: null candidate arrays");
  // the range's first base and window, and its sizes
  const uint64_t rb = n ? reads->offsets[r0] : 0, cb = n ? cands->offsets[r0] : 0;
  const uint64_t re = n ? reads->offsets[r1] : 0, ce = n ? cands->offsets[r1] : 0;
  if (re < rb || ce < cb || ce > nc_all)
    return set_error(SR_EINVAL, "sr_batch_stage: decreasing or out-of-range offsets in reads %u..%u", r0, r1);
  const uint64_t nb = re - rb;
  const uint64_t nc = ce - cb;
  if (nb > static_cast<uint64_t>(n) * SR_MAX_READ_LEN)
    return set_error(SR_EINVAL, "sr_batch_stage: %llu bases in %u reads: some read is longer than %d",
                     static_cast<unsigned long long>(nb), n, SR_MAX_READ_LEN);
  sr_batch* b = nullptr;
  sr_status rs = batch_alloc(s, n, nb, nc, stream, check_budget, &b);
  if (rs != SR_OK) return rs;
  const BatchDev& d = b->d;
  cudaError_t e = cudaSuccess;
  cudaStream_t st = b->stream;
  if (nb) e = cudaMemcpyAsync(const_cast<char*>(d.bases), reads->bases + rb, nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<uint64_t*>(d.read_off), reads->offsets + r0, (n + 1ull) * 8,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<uint64_t*>(d.cand_off), cands->offsets + r0, (n + 1ull) * 8,
                        cudaMemcpyHostToDevice, st);
  if (nc) {
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<uint8_t*>(d.c_ref), cands->ref_id + cb, nc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<uint8_t*>(d.c_strand), cands->strand + cb, nc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<uint64_t*>(d.c_start), cands->win_start + cb, nc * 8, cudaMemcpyHostToDevice,
                          st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<uint32_t*>(d.c_len), cands->win_len + cb, nc * 4, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess && n && (launch_rebase_offsets(const_cast<uint64_t*>(d.read_off), n + 1ull, rb, st) < 0 ||
                                launch_rebase_offsets(const_cast<uint64_t*>(d.cand_off), n + 1ull, cb, st) < 0))
    e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaStreamSynchronize(st);
    sr_batch_free(b);
    return cuda_error("sr_batch_stage copy", e);
  }
  // host-side validation, while the copies run: every kernel relies on these
  // bounds (window copies, shared-memory column streams, packed read rows).
  // Read ranges are checked in parallel; the first bad read (lowest index) is
  // reported.  The same pass counts the DP cells and the windows per read length.
  struct Part {
    uint64_t cells = 0;
    uint32_t max_m = 0;
    uint64_t by_len[kMaxReadLen + 1] = {};
    uint32_t bad_read = UINT32_MAX;
    int why = 0;  // 1 offsets, 2 read length, 3 window count, 4 window
    uint64_t bad_win = 0;
  };
  const uint32_t nthr = (n < 65536u) ? 1u : 4u * host_threads();
  std::vector<Part> parts(nthr);
  static_assert((kMaxRefs & (kMaxRefs - 1)) == 0, "ref_id masking");
  uint64_t lens16[kMaxRefs] = {};  // reference lengths, indexed by ref_id & (kMaxRefs - 1)
  for (uint32_t q = 0; q < s->n_refs && q < static_cast<uint32_t>(kMaxRefs); ++q) lens16[q] = s->lens[q];
  const uint32_t nref = s->n_refs;
  auto check = [&](uint32_t t) {
    Part& P = parts[t];
    const uint32_t p0 = static_cast<uint32_t>(static_cast<uint64_t>(n) * t / nthr);
    const uint32_t p1 = static_cast<uint32_t>(static_cast<uint64_t>(n) * (t + 1) / nthr);
    for (uint32_t r = r0 + p0; r < r0 + p1; ++r) {
      const uint64_t a0 = reads->offsets[r], a1 = reads->offsets[r + 1];
      const uint64_t c0 = cands->offsets[r], c1 = cands->offsets[r + 1];
      if (a1 < a0 || c1 < c0 || c1 > ce) {
        P.bad_read = r;
        P.why = 1;
        return;
      }
      const uint64_t m = a1 - a0;
      if (m == 0 || m > SR_MAX_READ_LEN) {
        P.bad_read = r;
        P.why = 2;
        return;
      }
      if (c1 - c0 >= (1ull << 19)) {
        P.bad_read = r;
        P.why = 3;
        return;
      }
      // all of a read's windows without a branch, then the first bad one if any
      uint64_t suml = 0;
      uint32_t bad = 0;
      for (uint64_t k = c0; k < c1; ++k) {
        const uint32_t ref = cands->ref_id[k], len = cands->win_len[k];
        const uint64_t L = lens16[ref & (kMaxRefs - 1)], w0 = cands->win_start[k];
        bad |= static_cast<uint32_t>(ref >= nref) | static_cast<uint32_t>(cands->strand[k] > 1) |
               static_cast<uint32_t>(len - 1u >= static_cast<uint32_t>(SR_MAX_WIN_LEN)) |
               static_cast<uint32_t>(w0 > L) | static_cast<uint32_t>(w0 + len > L);
        suml += len;
      }
      if (bad) {
        for (uint64_t k = c0; k < c1; ++k) {
          const uint32_t ref = cands->ref_id[k], len = cands->win_len[k];
          if (ref >= nref || cands->strand[k] > 1 || len < 1 || len > SR_MAX_WIN_LEN ||
              cands->win_start[k] > s->lens[ref] || cands->win_start[k] + len > s->lens[ref]) {
            P.bad_read = r;
            P.why = 4;
            P.bad_win = k;
            return;
          }
        }
      }
      P.cells += m * suml;
      P.by_len[m] += c1 - c0;
      P.max_m = std::max<uint32_t>(P.max_m, static_cast<uint32_t>(m));
    }
  };
  parallel_for(nthr, check);
  uint64_t cells = 0;
  uint32_t max_m = 0;
  uint64_t by_len[kMaxReadLen + 1] = {};
  const Part* worst = nullptr;
  for (const Part& P : parts) {
    if (P.bad_read != UINT32_MAX && (!worst || P.bad_read < worst->bad_read)) worst = &P;
    cells += P.cells;
    max_m = std::max(max_m, P.max_m);
    for (int m = 0; m <= kMaxReadLen; ++m) by_len[m] += P.by_len[m];
  }
  if (worst) {
    // the copies may still be reading the caller's arrays
    cudaStreamSynchronize(st);
    sr_batch_free(b);
    const uint32_t r = worst->bad_read;
    switch (worst->why) {
      case 1:
        return set_error(SR_EINVAL, "sr_batch_stage: decreasing or out-of-range offsets at read %u", r);
      case 2:
        return set_error(SR_EINVAL, "sr_batch_stage: read %u has length %llu, must be 1..256", r,
                         static_cast<unsigned long long>(reads->offsets[r + 1] - reads->offsets[r]));
      case 3:
        return set_error(SR_EINVAL, "sr_batch_stage: read %u has more than 2^19-1 windows", r);
      default:
        return set_error(SR_EINVAL, "sr_batch_stage: window %llu is outside its reference or malformed",
                         static_cast<unsigned long long>(worst->bad_win));
    }
  }
  // the caller may reuse its arrays once this returns
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    sr_batch_free(b);
    return cuda_error("sr_batch_stage copy", e);
  }
  b->cells = cells;
  b->max_m = max_m;
  std::memcpy(b->items_by_len, by_len, sizeof(by_len));
  *out = b;
  return SR_OK;
}

extern "C" void sr_batch_free(sr_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->res_ok) {
    // idle side streams before the next batch gets them
    bool idle = true;
    for (auto x : b->res.fan[0].side) idle = idle && cudaStreamSynchronize(x) == cudaSuccess;
    bool kept = false;
    if (idle) {
      std::lock_guard<std::mutex> lk(b->s->res_mu);
      if (b->s->res_pool.size() < kResPool) {
        b->s->res_pool.push_back(b->res);
        kept = true;
      }
    }
    if (!kept) res_destroy(b->res);
  }
  if (b->arena) {
    cudaStreamSynchronize(b->stream);
    // keep this arena for the next batches; past kKeptArenas kept, drop the smallest
    void* drop = nullptr;
    {
      std::lock_guard<std::mutex> lk(b->s->spare_mu);
      auto& sp = b->s->spares;
      sp.emplace_back(b->arena, b->arena_bytes);
      if (sp.size() > kKeptArenas) {
        auto it = std::min_element(sp.begin(), sp.end(),
                                   [](const std::pair<void*, uint64_t>& x, const std::pair<void*, uint64_t>& y) {
                                     return x.second < y.second;
                                   });
        drop = it->first;
        sp.erase(it);
      }
    }
    if (drop) cudaFree(drop);
    b->s->hbm_used -= b->bytes;
  }
  sr_session* s = b->s;
  delete b;
  if (s) session_release(s);
}

namespace sr {

// enqueue every kernel of the path for one batch; returns kernels launched or -1.
// Serving rounds pass ev_first (recorded once the first kernel is done),
// wait_extend (the extension kernels and everything after them wait for it:
// the previous round's last kernel) and assemble (the result records are built
// at the end, so fetching them needs copies only).
static int enqueue(sr_batch* b, const sr_score_params& sp, const sr_align_opts& o,
                   const TuneBin* bins, cudaStream_t st, cudaEvent_t ev_first = nullptr,
                   cudaEvent_t wait_extend = nullptr, bool assemble = false) {
  const BatchDev& d = b->d;
  const ScoreConst sc{sp.match, sp.mismatch, sp.gap_open, sp.gap_extend};
  const bool plain = o.engine == SR_ENGINE_PLAIN;
  const int nr = static_cast<int>(b->s->n_refs);
  int k = 0, t;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  const unsigned evf = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  auto mark = [&](int i) { return cudaEventRecordWithFlags(b->res.ev[i], st, evf) == cudaSuccess; };
  if (!mark(0)) return -1;
  if (cudaMemsetAsync(d.status, 0, 4, st) != cudaSuccess) return -1;
  if ((t = launch_prepare(d, b->s->refs, st)) < 0) return -1;
  k += t;
  if (ev_first && cudaEventRecord(ev_first, st) != cudaSuccess) return -1;
  // windows per length class (as launch_bins will route them): empty classes launch nothing
  uint64_t class_items[kNumClasses] = {};
  {
    const int32_t goe = sp.gap_open + sp.gap_extend;
    const bool tables_fit = sp.match + goe <= 127 && goe - sp.mismatch >= -128 && goe + sp.gap_extend + 256 < kBias;
    for (int m = 0; m <= kMaxReadLen; ++m) {
      if (!b->items_by_len[m]) continue;
      int c = kNumBins - 1;
      for (int q = 0; q < kNumBins; ++q)
        if (static_cast<uint32_t>(m) <= bins[q].upper) {
          c = q;
          break;
        }
      const bool i16_ok = tables_fit && static_cast<int64_t>(sp.match) * m <= 32767 - kBias;
      class_items[(o.force_i32 || !i16_ok) ? kI32Class : c] += b->items_by_len[m];
    }
  }
  if (b->n_items) {
    if ((t = launch_bins(d, sc, bins, kNumBins, o.force_i32 != 0, plain, st)) < 0) return -1;
    k += t;
    if (wait_extend && cudaStreamWaitEvent(st, wait_extend, 0) != cudaSuccess) return -1;
    if (!mark(2)) return -1;
    if ((t = launch_extend(d, b->s->refs, sc, bins, kNumBins, static_cast<int>(o.mode), plain, o.lanes,
                           o.rows, st, class_items, &b->res.fan[0])) < 0)
      return -1;
    if (!mark(3)) return -1;
    k += t;
  } else {
    if (wait_extend && cudaStreamWaitEvent(st, wait_extend, 0) != cudaSuccess) return -1;
    if (!mark(2) || !mark(3)) return -1;
  }
  if ((t = launch_select(d, nr, st)) < 0) return -1;
  k += t;
  if (!mark(4)) return -1;
  if (o.want_cigar) {
    if ((t = launch_winners(d, sc, static_cast<int>(o.mode), nr, plain, st)) < 0) return -1;
    k += t;
    if (o.mode == SR_MODE_LOCAL && b->n_items) {
      if ((t = launch_winner_rows(d, b->s->refs, sc, o.lanes, o.rows, st)) < 0)
        return -1;
      k += t;
    }
    if ((t = launch_traceback(d, b->s->refs, sc, static_cast<int>(o.mode), nr, st, &b->res.fan[1])) < 0) return -1;
    k += t;
    if ((t = launch_cigar_compact(d, nr, st)) < 0) return -1;
    k += t;
  }
  if (!mark(5)) return -1;
  if (o.classify) {
    if ((t = launch_classify(d, nr, o.min_score, o.margin, st)) < 0) return -1;
    k += t;
  }
  if (!mark(1)) return -1;
  if (assemble) {
    if ((t = launch_assemble(d, nr, o.want_cigar != 0, 0, 0, st)) < 0) return -1;
    k += t;
  }
  return k;
}

static bool same_opts(const sr_align_opts& a, const sr_align_opts& b) {
  return a.mode == b.mode && a.engine == b.engine && a.want_cigar == b.want_cigar && a.classify == b.classify &&
         a.min_score == b.min_score && a.margin == b.margin && a.force_i32 == b.force_i32 &&
         a.lanes == b.lanes && a.rows == b.rows;
}

uint32_t i32_min_read_len(const sr_score_params& sp, const sr_align_opts& o) {
  if (o.engine == SR_ENGINE_PLAIN) return kMaxReadLen + 1;
  const int32_t goe = sp.gap_open + sp.gap_extend;
  const bool i16_tables = sp.match + goe <= 127 && goe - sp.mismatch >= -128 && goe + sp.gap_extend + 256 < kBias;
  if (o.force_i32 || !i16_tables) return 0;
  for (uint32_t m = 1; m <= static_cast<uint32_t>(kMaxReadLen); ++m)
    if (static_cast<int64_t>(sp.match) * m > 32767 - kBias) return m;
  return kMaxReadLen + 1;
}

// checks a run's arguments against the batch; o receives the options to use
static sr_status run_args(sr_session* s, sr_batch* b, const sr_score_params* sp, const sr_align_opts* opts,
                          sr_align_opts& o) {
  if (!s || !b || b->s != s) return set_error(SR_EINVAL, "sr_batch_run: bad session/batch");
  sr_status st = check_score(sp);
  if (st != SR_OK) return st;
  o = opts ? *opts : default_opts();
  if (o.mode > 1 || o.engine > 1) return set_error(SR_EINVAL, "sr_batch_run: bad mode/engine");
  if ((o.lanes || o.rows) && !extend_config_supported(o.lanes, o.rows))
    return set_error(SR_EINVAL, "sr_batch_run: unsupported lanes x rows shape");
  if (o.engine == SR_ENGINE_PLAIN && o.lanes && !((o.lanes == 16 && o.rows == 16) || (o.lanes == 32 && o.rows == 8)))
    return set_error(SR_EINVAL, "sr_batch_run: the plain engine runs the 16x16 or 32x8 shape");
  if (o.lanes && o.lanes * o.rows < std::max<uint32_t>(b->max_m, 1))
    return set_error(SR_EINVAL, "sr_batch_run: lanes*rows must cover the longest read of the batch");
  if (o.classify && s->n_refs < 2) return set_error(SR_EINVAL, "sr_batch_run: classification needs 2 references");
  const int32_t goe = sp->gap_open + sp->gap_extend;
  const bool i16_tables = sp->match + goe <= 127 && goe - sp->mismatch >= -128 && goe + sp->gap_extend + 256 < kBias;
  if (o.engine == SR_ENGINE_PLAIN &&
      (!i16_tables || o.force_i32 || static_cast<int64_t>(sp->match) * b->max_m > 32767 - kBias))
    return set_error(SR_EINVAL, "sr_batch_run: the plain engine runs the int16 kernel only; use the batched engine");
  return SR_OK;
}

static void count_i32_items(sr_batch* b, const sr_score_params& sp, const sr_align_opts& o) {
  uint64_t n32 = 0;
  for (uint32_t m = i32_min_read_len(sp, o); m <= static_cast<uint32_t>(kMaxReadLen); ++m) n32 += b->items_by_len[m];
  b->i32_items = n32;
}

sr_status batch_run_serving(sr_session* s, sr_batch* b, const sr_score_params* sp, const sr_align_opts* opts,
                            cudaEvent_t ev_first, cudaEvent_t wait_extend) {
  Trace trace_("sr_batch_run serving");
  sr_align_opts o;
  sr_status st = run_args(s, b, sp, opts, o);
  if (st != SR_OK) return st;
  if (o.engine != SR_ENGINE_BATCHED) return set_error(SR_EINVAL, "serving runs the batched engine");
  cudaStream_t stream = o.cuda_stream ? static_cast<cudaStream_t>(o.cuda_stream) : b->stream;
  TuneBin bins[kNumBins];
  tune_get_bins(bins);
  count_i32_items(b, *sp, o);
  const int k = enqueue(b, *sp, o, bins, stream, ev_first, wait_extend, true);
  if (k < 0) return cuda_error("serving round launch", cudaGetLastError());
  b->kernels = static_cast<uint64_t>(k);
  b->ran = true;
  b->assembled = true;
  b->last_opts = o;
  return SR_OK;
}

sr_status batch_run_async(sr_session* s, sr_batch* b, const sr_score_params* sp, const sr_align_opts* opts) {
  Trace trace_("sr_batch_run");
  sr_align_opts o;
  sr_status st = run_args(s, b, sp, opts, o);
  if (st != SR_OK) return st;
  cudaStream_t stream = o.cuda_stream ? static_cast<cudaStream_t>(o.cuda_stream) : b->stream;
  TuneBin bins[kNumBins];
  tune_get_bins(bins);
  count_i32_items(b, *sp, o);
  const bool plain = o.engine == SR_ENGINE_PLAIN;
  if (plain) {
    const int k = enqueue(b, *sp, o, bins, stream);
    if (k < 0) return cuda_error("sr_batch_run launch", cudaGetLastError());
    b->kernels = static_cast<uint64_t>(k);
  } else if (!b->ran) {
    // a batch's first run launches the kernels directly: a batch run once (one
    // sr_align_batch call, one serving round) would not earn back a graph's
    // capture and instantiation
    const int k = enqueue(b, *sp, o, bins, stream);
    if (k < 0) return cuda_error("sr_batch_run launch", cudaGetLastError());
    b->kernels = static_cast<uint64_t>(k);
  } else {
    // later runs replay the whole path as one CUDA graph
    const bool reuse = b->graph && same_opts(b->g_opts, o) && memcmp(&b->g_sp, sp, sizeof(*sp)) == 0 &&
                       memcmp(b->g_bins, bins, sizeof(bins)) == 0;
    if (!reuse) {
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_error("sr_batch_run capture", e);
      const int k = enqueue(b, *sp, o, bins, stream);
      e = cudaStreamEndCapture(stream, &g);
      if (k < 0 || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_error("sr_batch_run capture", e != cudaSuccess ? e : cudaGetLastError());
      }
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_error("sr_batch_run instantiate", e);
      }
      b->g_opts = o;
      b->g_sp = *sp;
      memcpy(b->g_bins, bins, sizeof(bins));
      b->kernels = static_cast<uint64_t>(k);
    }
    cudaError_t e = cudaGraphLaunch(b->graph, stream);
    if (e != cudaSuccess) return cuda_error("sr_batch_run graph launch", e);
  }
  b->ran = true;
  b->assembled = false;
  b->last_opts = o;
  return SR_OK;
}

sr_status batch_sync(sr_batch* b, cudaStream_t stream) {
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_error("sr_batch_sync", e);
  uint32_t st = 0;
  e = cudaMemcpy(&st, b->d.status, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error("sr_batch_sync status", e);
  if (st & kStBadBase) return set_error(SR_EBADBASE, "read has a non-ACGT base");
  if (st & kStBadRead) return set_error(SR_EINVAL, "read length must be 1..256");
  if (st & kStBadWindow) return set_error(SR_EINVAL, "window outside its reference, bad ref id/strand or length not in 1..512");
  if (st & kStTimeout) return set_error(SR_ETIMEOUT, "device wait for a window copy ran out");
  if (st & (kStOverflow | kStInternal)) return set_error(SR_ECUDA, "device internal check failed (status %u)", st);
  return SR_OK;
}

}  // namespace sr

extern "C" sr_status sr_batch_run_async(sr_session* s, sr_batch* b, const sr_score_params* sp,
                                        const sr_align_opts* opts) {
  return batch_run_async(s, b, sp, opts);
}

extern "C" sr_status sr_batch_sync(sr_session* s, sr_batch* b) {
  if (!s || !b) return set_error(SR_EINVAL, "sr_batch_sync: null argument");
  cudaStream_t st = b->last_opts.cuda_stream ? static_cast<cudaStream_t>(b->last_opts.cuda_stream) : b->stream;
  return batch_sync(b, st);
}

extern "C" sr_status sr_batch_run(sr_session* s, sr_batch* b, const sr_score_params* sp,
                                  const sr_align_opts* opts) {
  sr_status st = batch_run_async(s, b, sp, opts);
  if (st != SR_OK) return st;
  return sr_batch_sync(s, b);
}

extern "C" sr_status sr_batch_stats(const sr_batch* b, uint64_t* kernels, uint64_t* cells, uint64_t* i32_items,
                                    uint64_t* tasks) {
  if (!b) return set_error(SR_EINVAL, "sr_batch_stats: null batch");
  if (kernels) *kernels = b->kernels;
  if (cells) *cells = b->cells;
  if (i32_items) *i32_items = b->i32_items;
  if (tasks) *tasks = (b->n_items + 1) / 2;
  return SR_OK;
}

extern "C" sr_status sr_batch_timing(const sr_batch* b, float* total_ms, float* extend_ms, float* traceback_ms) {
  if (!b || !b->ran) return set_error(SR_EINVAL, "sr_batch_timing: batch has not run");
  float t = 0;
  if (total_ms) {
    if (cudaEventElapsedTime(&t, b->res.ev[0], b->res.ev[1]) != cudaSuccess) return cuda_error("sr_batch_timing", cudaGetLastError());
    *total_ms = t;
  }
  if (extend_ms) {
    if (cudaEventElapsedTime(&t, b->res.ev[2], b->res.ev[3]) != cudaSuccess) return cuda_error("sr_batch_timing", cudaGetLastError());
    *extend_ms = t;
  }
  if (traceback_ms) {
    if (cudaEventElapsedTime(&t, b->res.ev[4], b->res.ev[5]) != cudaSuccess) return cuda_error("sr_batch_timing", cudaGetLastError());
    *traceback_ms = t;
  }
  return SR_OK;
}

namespace sr {
// Every sr_results is the head of a ResultsBox.  Fetched results keep all
// their arrays in one pinned host block of the session's pool (fast D2H, no
// page faults, no unmapping at free); the block goes back to the pool when the
// results are freed, and the results hold a reference to the session meanwhile.
struct ResultsBox {
  sr_results pub;
  sr_session* pool_of = nullptr;
  void* block = nullptr;
  uint64_t block_bytes = 0;
  void* cig_block = nullptr;  // the CIGAR words, when they sit in a block of their own
  uint64_t cig_block_bytes = 0;
};

sr_results* results_alloc() {
  auto* b = static_cast<ResultsBox*>(calloc(1, sizeof(ResultsBox)));
  return b ? &b->pub : nullptr;
}

static void* pool_take(sr_session* s, uint64_t bytes, uint64_t* got) {
  {
    std::lock_guard<std::mutex> lk(s->pool_mu);
    int pick = -1;
    for (size_t i = 0; i < s->pool.size(); ++i)
      if (s->pool[i].second >= bytes && s->pool[i].second <= 2 * bytes + (64ull << 20) &&
          (pick < 0 || s->pool[i].second < s->pool[pick].second))
        pick = static_cast<int>(i);
    if (pick >= 0) {
      void* p = s->pool[pick].first;
      *got = s->pool[pick].second;
      s->pool.erase(s->pool.begin() + pick);
      return p;
    }
  }
  // new blocks in whole units of 64 MiB: pinning pages costs time on the caller's
  // path (the serving completer), so a pool of a few such blocks covers the
  // result sizes that follow instead of growing by every larger round
  constexpr uint64_t kUnit = 64ull << 20;
  const uint64_t want = (bytes + kUnit - 1) / kUnit * kUnit;
  void* p = nullptr;
  if (cudaMallocHost(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *got = want;
  return p;
}

static void pool_give(sr_session* s, void* p, uint64_t bytes) {
  void* drop = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->pool_mu);
    s->pool.emplace_back(p, bytes);
    if (s->pool.size() > 8) {  // keep the eight most recent blocks (results a caller still holds take some)
      drop = s->pool.front().first;
      s->pool.erase(s->pool.begin());
    }
  }
  if (drop) cudaFreeHost(drop);
}
}  // namespace sr

extern "C" void sr_results_free(sr_results* r) {
  if (!r) return;
  auto* box = reinterpret_cast<ResultsBox*>(r);
  if (box->block) {
    sr_session* s = box->pool_of;
    pool_give(s, box->block, box->block_bytes);
    if (box->cig_block) pool_give(s, box->cig_block, box->cig_block_bytes);
    free(box);
    session_release(s);
    return;
  }
  free(r->best);
  free(r->best_per_ref);
  free(r->item_score);
  free(r->item_end);
  free(r->cigar);
  free(r->read_class);
  free(box);
}

extern "C" sr_status sr_batch_fetch(sr_session* s, sr_batch* b, sr_results** out) {
  Trace trace_("sr_batch_fetch");
  if (!s || !b || !out) return set_error(SR_EINVAL, "sr_batch_fetch: null argument");
  if (!b->ran) return set_error(SR_EINVAL, "sr_batch_fetch: batch has not run");
  *out = nullptr;
  cudaStream_t stream = b->last_opts.cuda_stream ? static_cast<cudaStream_t>(b->last_opts.cuda_stream) : b->stream;
  sr_status st = batch_sync(b, stream);
  if (st != SR_OK) return st;
  const uint32_t n = b->n_reads, nr = s->n_refs;
  const uint64_t nc = b->n_items;
  sr_results* r = results_alloc();
  if (!r) return set_error(SR_ENOMEM, "sr_batch_fetch: out of memory");
  r->n_reads = n;
  r->n_refs = nr;
  r->n_items = nc;
  r->cells = b->cells;
  r->n_i32_items = b->i32_items;
  // records in the public layout are assembled on the device, then every array
  // comes back with one copy each on the batch's stream and a single wait
  const bool cig = b->last_opts.want_cigar != 0;
  const bool cls = b->last_opts.classify != 0;
  if (!b->assembled && launch_assemble(b->d, static_cast<int>(nr), cig, 0, 0, stream) < 0) {
    sr_results_free(r);
    return cuda_error("sr_batch_fetch assemble", cudaGetLastError());
  }
  uint32_t total = 0;
  cudaError_t e = cudaSuccess;
  if (n && cig) {
    e = cudaMemcpyAsync(&total, b->d.cigar_off + n, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  }
  if (e != cudaSuccess) {
    sr_results_free(r);
    return cuda_error("sr_batch_fetch copy", e);
  }
  // one block for every array, 256-byte aligned parts
  uint64_t off = 0;
  auto part = [&](uint64_t bytes) {
    const uint64_t at = off;
    off = (off + (bytes ? bytes : 1) + 255) & ~255ull;
    return at;
  };
  const uint64_t o_best = part(static_cast<uint64_t>(n) * sizeof(sr_hit));
  const uint64_t o_per = part(static_cast<uint64_t>(n) * (nr ? nr : 1) * sizeof(sr_hit));
  const uint64_t o_sc = part(nc * 4);
  const uint64_t o_end = part(nc * 4);
  const uint64_t o_cig = cig ? part(static_cast<uint64_t>(total) * 4) : 0;
  const uint64_t o_cls = cls ? part(n) : 0;
  uint64_t got = 0;
  // small results (serving rounds) use plain memory: pinning costs more than it saves
  char* blk = off >= (16ull << 20) ? static_cast<char*>(pool_take(s, off, &got)) : nullptr;
  if (blk) {
    auto* box = reinterpret_cast<ResultsBox*>(r);
    box->pool_of = s;
    box->block = blk;
    box->block_bytes = got;
    s->live.fetch_add(1);
    r->best = reinterpret_cast<sr_hit*>(blk + o_best);
    r->best_per_ref = reinterpret_cast<sr_hit*>(blk + o_per);
    r->item_score = reinterpret_cast<int32_t*>(blk + o_sc);
    r->item_end = reinterpret_cast<uint32_t*>(blk + o_end);
    if (cig) r->cigar = reinterpret_cast<uint32_t*>(blk + o_cig);
    if (cls) r->read_class = reinterpret_cast<uint8_t*>(blk + o_cls);
  } else {  // no pinned memory: plain allocations
    r->best = static_cast<sr_hit*>(malloc(static_cast<size_t>(n ? n : 1) * sizeof(sr_hit)));
    r->best_per_ref = static_cast<sr_hit*>(malloc(static_cast<size_t>(n ? n : 1) * (nr ? nr : 1) * sizeof(sr_hit)));
    r->item_score = static_cast<int32_t*>(malloc((nc ? nc : 1) * 4));
    r->item_end = static_cast<uint32_t*>(malloc((nc ? nc : 1) * 4));
    if (cig) r->cigar = static_cast<uint32_t*>(malloc((total ? total : 1) * 4ull));
    if (cls) r->read_class = static_cast<uint8_t*>(malloc(n ? n : 1));
    if (!r->best || !r->best_per_ref || !r->item_score || !r->item_end || (cig && !r->cigar) ||
        (cls && !r->read_class)) {
      sr_results_free(r);
      return set_error(SR_ENOMEM, "sr_batch_fetch: out of memory");
    }
  }
  if (cig) r->n_cigar = total;
  auto copy = [&](void* dst, const void* src, uint64_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, stream);
  };
  copy(r->item_score, b->d.item_score, nc * 4);
  copy(r->item_end, b->d.item_end, nc * 4);
  copy(r->best, b->d.out_best, static_cast<uint64_t>(n) * sizeof(sr_hit));
  copy(r->best_per_ref, b->d.out_per_ref, static_cast<uint64_t>(n) * nr * sizeof(sr_hit));
  if (cig) copy(r->cigar, b->d.cigar, static_cast<uint64_t>(total) * 4);
  if (cls) copy(r->read_class, b->d.read_class, n);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    sr_results_free(r);
    return cuda_error("sr_batch_fetch copy", e);
  }
  *out = r;
  return SR_OK;
}

// ------------------------------------------------------------------ device CAL finder
extern "C" sr_status sr_session_attach_index(sr_session* s, const sr_index* const* idx, uint32_t n_refs) {
  if (!s || !idx || n_refs != s->n_refs || n_refs == 0)
    return set_error(SR_EINVAL, "sr_session_attach_index: one index per session reference");
  std::vector<IndexTables> t(n_refs);
  for (uint32_t r = 0; r < n_refs; ++r) {
    if (!idx[r]) return set_error(SR_EINVAL, "sr_session_attach_index: null index");
    t[r] = index_tables(idx[r]);
    if (t[r].ref_len != s->lens[r])
      return set_error(SR_EINVAL, "sr_session_attach_index: index %u is of another reference", r);
    if (t[r].seed_len != t[0].seed_len || t[r].address_bases != t[0].address_bases)
      return set_error(SR_EINVAL, "sr_session_attach_index: indexes differ in seed layout");
  }
  for (auto* p : s->idx_bufs) cudaFree(p);
  s->idx_bufs.clear();
  s->didx = DevIndex{};
  auto up = [&](const void* src, uint64_t bytes, void** dst) -> bool {
    void* d = nullptr;
    if (cudaMalloc(&d, bytes ? bytes : 1) != cudaSuccess) return false;
    s->idx_bufs.push_back(d);
    if (bytes && cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return false;
    *dst = d;
    return true;
  };
  auto fail = [&]() -> sr_status {
    for (auto* p : s->idx_bufs) cudaFree(p);
    s->idx_bufs.clear();
    s->didx = DevIndex{};
    cudaGetLastError();
    return set_error(SR_ENOMEM, "sr_session_attach_index: device upload failed");
  };
  // the packed device form when the references allow it (see DevIndex)
  const bool keys16 = 2 * (static_cast<int>(t[0].seed_len) - static_cast<int>(t[0].address_bases)) <= 16;
  bool packed = true;
  for (uint32_t r = 0; r < n_refs && packed; ++r)
    packed = t[r].hash_seed == t[0].hash_seed && t[r].n_ptr == t[0].n_ptr && t[r].n_entries < (1ull << 32) &&
             t[r].ref_len <= (1ull << 30);
  if (packed) {
    const uint64_t nb = t[0].n_ptr;  // buckets + 1, the same in every reference
    std::vector<uint32_t> jp(nb * n_refs);
    for (uint64_t b = 0; b < nb; ++b)
      for (uint32_t r = 0; r < n_refs; ++r) jp[b * n_refs + r] = static_cast<uint32_t>(t[r].ptr[b]);
    void* pj;
    if (!up(jp.data(), jp.size() * 4, &pj)) return fail();
    s->didx.jptr = static_cast<const uint32_t*>(pj);
    for (uint32_t r = 0; r < n_refs; ++r) {
      std::vector<uint16_t> k16(keys16 ? t[r].n_entries : 0);
      std::vector<uint32_t> po(t[r].n_entries);
      for (uint64_t i = 0; i < t[r].n_entries; ++i) {
        if (keys16) k16[i] = static_cast<uint16_t>(t[r].key[i]);
        po[i] = t[r].pos[i] | (static_cast<uint32_t>(t[r].orient[i] & 3u) << 30);
      }
      void *pk, *pp;
      if (keys16 ? !up(k16.data(), k16.size() * 2, &pk) : !up(t[r].key, t[r].n_entries * 4, &pk)) return fail();
      if (!up(po.data(), po.size() * 4, &pp)) return fail();
      if (keys16) s->didx.key16[r] = static_cast<const uint16_t*>(pk);
      else s->didx.key[r] = static_cast<const uint32_t*>(pk);
      s->didx.posor[r] = static_cast<const uint32_t*>(pp);
      s->didx.ref_len[r] = t[r].ref_len;
      s->didx.hash_seed[r] = t[r].hash_seed;
    }
    s->didx.packed = 1;
    s->didx.key_bits = keys16 ? 16 : 32;
  } else {
    for (uint32_t r = 0; r < n_refs; ++r) {
      void *pp, *pk, *ps, *po;
      if (!up(t[r].ptr, t[r].n_ptr * 8, &pp) || !up(t[r].key, t[r].n_entries * 4, &pk) ||
          !up(t[r].pos, t[r].n_entries * 4, &ps) || !up(t[r].orient, t[r].n_entries, &po))
        return fail();
      s->didx.ptr[r] = static_cast<const uint64_t*>(pp);
      s->didx.key[r] = static_cast<const uint32_t*>(pk);
      s->didx.pos[r] = static_cast<const uint32_t*>(ps);
      s->didx.orient[r] = static_cast<const uint8_t*>(po);
      s->didx.ref_len[r] = t[r].ref_len;
      s->didx.hash_seed[r] = t[r].hash_seed;
    }
  }
  s->didx.n_refs = static_cast<int>(n_refs);
  s->didx.k = static_cast<int>(t[0].seed_len);
  s->didx.a = static_cast<int>(t[0].address_bases);
  // bucket heads, built on the device from the packed tables: where buckets are
  // small (on average at most half a head's 16-bit keys, or 8 of its 13 32-bit
  // ones, so that few spill) a seed's lookup in both references is one 64-byte
  // access instead of three dependent ones (SR_CAL_HEADS=0 leaves them out)
  const uint64_t nbk = t[0].n_ptr ? t[0].n_ptr - 1 : 0;
  uint64_t entries = 0;
  for (uint32_t r = 0; r < n_refs; ++r) entries += t[r].n_entries;
  const uint64_t per_bucket = keys16 ? kHeadKeys / 2 : 8;
  if (packed && n_refs <= 2 && nbk && nbk <= (1ull << 26) && entries <= nbk * per_bucket &&
      env_u64("SR_CAL_HEADS", 1) != 0) {
    void* ph = nullptr;
    if (cudaMalloc(&ph, nbk * 64) == cudaSuccess) {
      s->idx_bufs.push_back(ph);
      if (launch_cal_heads(s->didx, nbk, static_cast<uint4*>(ph), s->stream) < 0 ||
          cudaStreamSynchronize(s->stream) != cudaSuccess)
        return fail();
      s->didx.heads = static_cast<const uint4*>(ph);
    } else {
      cudaGetLastError();  // the heads are optional: without them the lookups read jptr / key16
    }
  }
  return SR_OK;
}

extern "C" sr_status sr_candidates_device(sr_session* s, const sr_reads* reads, const sr_cand_params* params,
                                          sr_cand_list** out) {
  Trace trace_("sr_candidates_device");
  if (!s || !reads || !out) return set_error(SR_EINVAL, "sr_candidates_device: null argument");
  *out = nullptr;
  if (s->didx.n_refs == 0) return set_error(SR_EINVAL, "sr_candidates_device: no index attached to the session");
  sr_cand_params cp{};
  if (params) cp = *params;
  if (!cp.seed_stride) cp.seed_stride = 1;
  if ((reads->flags | cp.flags) & ~static_cast<uint32_t>(SR_FLAG_DEVICE))
    return set_error(SR_EINVAL, "sr_candidates_device: unknown flags");
  const bool in_dev = (reads->flags & SR_FLAG_DEVICE) != 0, out_dev = (cp.flags & SR_FLAG_DEVICE) != 0;
  const uint32_t n = reads->n_reads;
  if (!reads->offsets || (n && !reads->bases)) return set_error(SR_EINVAL, "sr_candidates_device: null reads");
  cudaStream_t st = s->stream;
  uint64_t nb = 0;
  if (in_dev) {
    // the read lengths are checked by the count kernel
    uint64_t ends[2] = {};
    cudaError_t e = cudaMemcpyAsync(&ends[0], reads->offsets, 8, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], reads->offsets + n, 8, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error("sr_candidates_device offsets", e);
    if (ends[0] != 0) return set_error(SR_EINVAL, "sr_candidates_device: offsets must start at 0");
    nb = ends[1];
    if (nb > static_cast<uint64_t>(n) * SR_MAX_READ_LEN)
      return set_error(SR_EINVAL, "sr_candidates_device: some read is longer than %u bases", SR_MAX_READ_LEN);
  } else {
    if (reads->offsets[0] != 0) return set_error(SR_EINVAL, "sr_candidates_device: offsets must start at 0");
    for (uint32_t r = 0; r < n; ++r) {
      if (reads->offsets[r + 1] < reads->offsets[r])
        return set_error(SR_EINVAL, "sr_candidates_device: decreasing read offsets");
      if (reads->offsets[r + 1] - reads->offsets[r] > SR_MAX_READ_LEN)
        return set_error(SR_EINVAL, "sr_candidates_device: read %u longer than %u bases", r, SR_MAX_READ_LEN);
    }
    nb = reads->offsets[n];
  }
  // the call's scratch comes from the session's cache (grown with a quarter of
  // headroom when a call needs more), so steady-state calls allocate only
  // their result list
  std::lock_guard<std::mutex> cal_lock(s->cal_mu);
  cudaError_t e = cudaSuccess;
  auto cbuf = [&](int role, uint64_t bytes) -> void* {
    if (e != cudaSuccess) return nullptr;
    bytes = std::max<uint64_t>(bytes, 16);
    if (s->cal_bytes[role] < bytes) {
      if (s->cal_buf[role]) {
        // earlier launches of this call may still use the smaller buffer
        e = cudaStreamSynchronize(st);
        cudaFree(s->cal_buf[role]);
        s->cal_buf[role] = nullptr;
        s->cal_bytes[role] = 0;
        if (e != cudaSuccess) return nullptr;
      }
      const uint64_t want = bytes + bytes / 4;
      e = cudaMalloc(&s->cal_buf[role], want);
      if (e != cudaSuccess) {
        s->cal_buf[role] = nullptr;
        return nullptr;
      }
      s->cal_bytes[role] = want;
    }
    return s->cal_buf[role];
  };
  // The list is built on the device in either case: in the caller's list arrays
  // (device output, grown chunk by chunk), or in the session's cached arrays
  // (host output: copied out once at the end, through a pinned block).
  sr_cand_list* l = static_cast<sr_cand_list*>(calloc(1, sizeof(sr_cand_list)));
  if (!l) return set_error(SR_ENOMEM, "sr_candidates_device: out of memory");
  l->n_reads = n;
  l->flags = out_dev ? static_cast<uint32_t>(SR_FLAG_DEVICE) : 0u;
  struct {
    uint64_t* off;
    uint8_t *ref, *str;
    uint64_t* start;
    uint32_t *len, *hits;
  } L{};
  uint64_t cap_out = 0;  // windows the device result arrays hold
  auto done = [&](sr_status stt, const char* msg) -> sr_status {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    if (stt == SR_OK) return static_cast<sr_status>(SR_OK);
    sr_cand_list_free(l);  // host output: its arrays are still unset
    if (stt == SR_ECUDA) return cuda_error(msg, e == cudaSuccess ? cudaErrorUnknown : e);
    return set_error(stt, "%s", msg);
  };
  if (out_dev) {
    if (cudaMalloc(&l->offsets, (n + 1ull) * 8) != cudaSuccess) {
      e = cudaGetLastError();
      return done(SR_ENOMEM, "sr_candidates_device: device allocation failed");
    }
    L.off = l->offsets;
  } else {
    L.off = static_cast<uint64_t*>(cbuf(kCbLoff, (n + 1ull) * 8));
    if (e != cudaSuccess) return done(SR_ENOMEM, "sr_candidates_device: device allocation failed");
  }
  if (n == 0 && cudaMemsetAsync(L.off, 0, 8, st) != cudaSuccess) {
    e = cudaGetLastError();
    return done(SR_ECUDA, "sr_candidates_device offsets");
  }
  // a cached array grown to `need` bytes, its first `keep` bytes kept
  auto cgrow = [&](int role, uint64_t need, uint64_t keep) -> void* {
    if (s->cal_bytes[role] >= need) return s->cal_buf[role];
    void* p = nullptr;
    const uint64_t want = need + need / 4;
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    if (keep && s->cal_buf[role] &&
        cudaMemcpyAsync(p, s->cal_buf[role], keep, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(p);
      return nullptr;
    }
    cudaStreamSynchronize(st);
    if (s->cal_buf[role]) cudaFree(s->cal_buf[role]);
    s->cal_buf[role] = p;
    s->cal_bytes[role] = want;
    return p;
  };
  // grows the device result arrays to hold `need` windows, keeping the first `keep`
  auto grow_out = [&](uint64_t need, uint64_t keep) -> bool {
    if (need <= cap_out) return true;
    const uint64_t c = std::max<uint64_t>(need, cap_out + cap_out / 2);
    if (!out_dev) {
      L.ref = static_cast<uint8_t*>(cgrow(kCbLref, c, keep));
      L.str = static_cast<uint8_t*>(cgrow(kCbLstr, c, keep));
      L.start = static_cast<uint64_t*>(cgrow(kCbLstart, c * 8, keep * 8));
      L.len = static_cast<uint32_t*>(cgrow(kCbLlen, c * 4, keep * 4));
      L.hits = static_cast<uint32_t*>(cgrow(kCbLhits, c * 4, keep * 4));
      if (!L.ref || !L.str || !L.start || !L.len || !L.hits) return false;
      cap_out = c;
      return true;
    }
    void *r8 = nullptr, *s8 = nullptr, *st64 = nullptr, *ln32 = nullptr, *h32 = nullptr;
    bool ok = cudaMalloc(&r8, c) == cudaSuccess && cudaMalloc(&s8, c) == cudaSuccess &&
              cudaMalloc(&st64, c * 8) == cudaSuccess && cudaMalloc(&ln32, c * 4) == cudaSuccess &&
              cudaMalloc(&h32, c * 4) == cudaSuccess;
    if (ok && keep) {
      ok = cudaMemcpyAsync(r8, l->ref_id, keep, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(s8, l->strand, keep, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(st64, l->win_start, keep * 8, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(ln32, l->win_len, keep * 4, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(h32, l->hits, keep * 4, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaStreamSynchronize(st) == cudaSuccess;
    }
    void* old[5] = {l->ref_id, l->strand, l->win_start, l->win_len, l->hits};
    void* fresh[5] = {r8, s8, st64, ln32, h32};
    if (!ok) {
      for (void* p : fresh)
        if (p) cudaFree(p);
      cudaGetLastError();
      return false;
    }
    for (void* p : old)
      if (p) cudaFree(p);
    l->ref_id = static_cast<uint8_t*>(r8);
    l->strand = static_cast<uint8_t*>(s8);
    l->win_start = static_cast<uint64_t*>(st64);
    l->win_len = static_cast<uint32_t*>(ln32);
    l->hits = static_cast<uint32_t*>(h32);
    L.ref = l->ref_id;
    L.str = l->strand;
    L.start = l->win_start;
    L.len = l->win_len;
    L.hits = l->hits;
    cap_out = c;
    return true;
  };
  uint64_t total_w = 0;
  if (n) {
    const char* d_bases = in_dev ? reads->bases : static_cast<const char*>(cbuf(kCbBases, nb));
    const uint64_t* d_roff = in_dev ? reads->offsets : static_cast<const uint64_t*>(cbuf(kCbRoff, (n + 1ull) * 8));
    uint32_t* d_count = static_cast<uint32_t*>(cbuf(kCbCount, n * 4ull));
    uint32_t* d_actual = static_cast<uint32_t*>(cbuf(kCbActual, n * 4ull));
    uint32_t* d_status = static_cast<uint32_t*>(cbuf(kCbStatus, 4));
    // per read: its lookup records (seeds x references), then their prefix sums
    uint32_t* d_slots = static_cast<uint32_t*>(cbuf(kCbSlots, n * 4ull));
    uint64_t* d_pre = static_cast<uint64_t*>(cbuf(kCbPre, (n + 1ull) * 8));
    uint64_t* d_sums = static_cast<uint64_t*>(cbuf(kCbSums, (n / 1024 + 2ull) * 8));
    uint32_t* d_bounds = static_cast<uint32_t*>(cbuf(kCbBounds, (n + 1ull) * 4));
    CalPlan* d_plan = static_cast<CalPlan*>(cbuf(kCbPlan, sizeof(CalPlan)));
    if (e != cudaSuccess) return done(SR_ENOMEM, "sr_candidates_device: device allocation failed");
    if (!in_dev) {
      if (nb) e = cudaMemcpyAsync(const_cast<char*>(d_bases), reads->bases, nb, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<uint64_t*>(d_roff), reads->offsets, (n + 1ull) * 8, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, 4, st);
    if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device copy");
    // The count pass keeps each seed's lookup (one record per seed and
    // reference) for the emit pass.  Reads run in chunks of at most
    // kRangeRecords records: a chunk is cut where the records' prefix sum crosses
    // a multiple of kRangeRecords less one read's most records, so that no chunk
    // exceeds it; all cuts are made on the device.
    const uint64_t rec_read = (static_cast<uint64_t>(kMaxReadLen) / cp.seed_stride + 1) * s->didx.n_refs;
    // 1 GiB of kept lookups at most; SR_CAL_CHUNK_RECORDS lowers it (tests of the cuts)
    const uint64_t kRangeRecords = std::max<uint64_t>(env_u64("SR_CAL_CHUNK_RECORDS", 128ull << 20), 2 * rec_read);
    const uint64_t rec_span = kRangeRecords - rec_read;
    uint64_t ends[2] = {};  // prefix of the last read, total records
    uint32_t status = 0;
    if (launch_cal_slots(d_roff, n, s->didx.k, cp.seed_stride, s->didx.n_refs, d_slots, d_status, st) < 0 ||
        launch_scan_u64(d_slots, n, d_pre, d_sums, st) < 0 || launch_cal_bounds(d_pre, n, rec_span, d_bounds, st) < 0) {
      e = cudaGetLastError();
      return done(SR_ECUDA, "sr_candidates_device slots");
    }
    e = cudaMemcpyAsync(ends, d_pre + n - 1, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device slots copy");
    if (status & kStBadRead) return done(SR_EINVAL, "sr_candidates_device: decreasing read offsets or a read longer than 256 bases");
    const uint32_t n_chunks = static_cast<uint32_t>(ends[0] / rec_span) + 1;
    std::vector<uint32_t> rchunk(n_chunks + 1ull);
    e = cudaMemcpyAsync(rchunk.data(), d_bounds, n_chunks * 4ull, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device chunks");
    rchunk[n_chunks] = n;
    uint32_t max_reads = 0;
    uint64_t max_rec = 0;
    for (uint32_t c = 0; c < n_chunks; ++c) max_reads = std::max(max_reads, rchunk[c + 1] - rchunk[c]);
    max_rec = std::min<uint64_t>(ends[1], kRangeRecords);
    uint64_t* d_ranges = static_cast<uint64_t*>(cbuf(kCbRanges, std::max<uint64_t>(max_rec, 1) * 8));
    uint32_t* d_seed_off = static_cast<uint32_t*>(cbuf(kCbSeedOff, (max_reads + 1ull) * 4));
    uint8_t* d_recount = static_cast<uint8_t*>(cbuf(kCbRecount, max_reads + 1ull));
    // per chunk: the prefix sums of its reads' CAL bounds, a sub-chunk's offsets
    // (from 0) and its large-read list
    uint64_t* d_cpre = static_cast<uint64_t*>(cbuf(kCbCpre, (max_reads + 1ull) * 8));
    uint64_t* d_off = static_cast<uint64_t*>(cbuf(kCbOff, (max_reads + 1ull) * 8));
    uint32_t* d_nwin = static_cast<uint32_t*>(cbuf(kCbNwin, max_reads * 4ull + 4));
    uint32_t* d_woff = static_cast<uint32_t*>(cbuf(kCbWoff, (max_reads + 1ull) * 4));
    uint32_t* d_wsums = static_cast<uint32_t*>(cbuf(kCbWsums, (max_reads / 1024 + 2ull) * 4));
    uint32_t* d_big = static_cast<uint32_t*>(cbuf(kCbBig, max_reads * 4ull + 4));
    uint64_t* d_bigoff = static_cast<uint64_t*>(cbuf(kCbBigOff, max_reads * 8ull + 8));
    if (e != cudaSuccess) return done(SR_ENOMEM, "sr_candidates_device: device allocation failed");
    // the emit / filter buffers, sized for the largest sub-chunk so far
    uint64_t cap = 0;
    uint64_t *d_cals = nullptr, *d_wkey = nullptr;
    uint32_t *d_whits = nullptr, *d_wlen = nullptr;
    uint64_t* d_scratch = nullptr;
    uint64_t scratch_keys = 0;
    std::vector<uint32_t> sub;
    // one sub-chunk (reads r0 .. r0 + nr of the chunk at R0, offsets in d_off):
    // routing, emit, filter, window offsets and the compacted windows
    auto run_sub = [&](uint32_t r0, uint32_t nr, const CalRanges& kept) -> sr_status {
      CalPlan plan{};
      e = cudaMemsetAsync(d_plan, 0, sizeof(CalPlan), st);
      if (e != cudaSuccess || launch_cal_route(d_count + r0, nr, d_big, d_bigoff, d_plan, st) < 0)
        return done(SR_ECUDA, "sr_candidates_device route");
      e = cudaMemcpyAsync(&plan, d_plan, sizeof(CalPlan), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device route copy");
      const uint64_t scratch_need = plan.scratch + (plan.n_big ? cal_sort_words(plan.n_big, plan.scratch) : 0);
      if (scratch_need > scratch_keys) {
        d_scratch = static_cast<uint64_t*>(cbuf(kCbScratch, scratch_need * 8));
        if (e != cudaSuccess) return done(SR_ENOMEM, "sr_candidates_device: device allocation failed");
        scratch_keys = scratch_need;
      }
      if (launch_cal_seeds(s->didx, d_bases, d_roff, r0, nr, cp.seed_stride, d_count + r0, d_off, d_cals, d_actual,
                           d_status, kept, st) < 0 ||
          launch_cal_emit_big(s->didx, d_roff, r0, nr, cp.seed_stride, d_count + r0, d_off, d_cals, kept, d_big,
                              plan.n_big, d_scratch, plan.scratch, st) < 0 ||
          launch_cal_filter(s->didx, d_roff, r0, nr, cp.merge_dist, cp.pad, cp.max_cands, d_count + r0, d_actual,
                            d_off, d_cals, std::max(plan.max_small, 1u), plan.max_mid, d_big, d_bigoff, plan.n_big,
                            d_scratch, plan.scratch, d_nwin, d_wkey, d_whits, d_wlen, st) < 0 ||
          launch_scan_u32(d_nwin, nr, d_woff, d_wsums, st) < 0) {
        e = cudaGetLastError();
        return done(SR_ECUDA, "sr_candidates_device filter");
      }
      uint32_t nw32 = 0;
      e = cudaMemcpyAsync(&nw32, d_woff + nr, 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device window count");
      const uint64_t nw = nw32;
      // this sub-chunk's offsets in the whole list, its windows compacted
      // straight into the list's arrays after the windows so far
      if (launch_cal_offsets(d_woff, nr, total_w, L.off + r0, st) < 0) {
        e = cudaGetLastError();
        return done(SR_ECUDA, "sr_candidates_device offsets");
      }
      if (!grow_out(total_w + nw, total_w)) return done(SR_ENOMEM, "sr_candidates_device: device allocation failed");
      if (launch_cal_compact(nr, d_off, d_nwin, d_woff, d_wkey, d_whits, d_wlen, L.ref + total_w, L.str + total_w,
                             L.start + total_w, L.len + total_w, L.hits + total_w, st) < 0) {
        e = cudaGetLastError();
        return done(SR_ECUDA, "sr_candidates_device compact");
      }
      total_w += nw;
      return static_cast<sr_status>(SR_OK);
    };
    for (uint32_t ci = 0; ci < n_chunks; ++ci) {
      const uint32_t R0 = rchunk[ci], R1 = rchunk[ci + 1], nrc = R1 - R0;
      // this chunk's record offsets from 0, then its count pass (which keeps the lookups)
      if (launch_cal_rebase(d_pre, R0, nrc, nullptr, d_seed_off, st) < 0) {
        e = cudaGetLastError();
        return done(SR_ECUDA, "sr_candidates_device records");
      }
      const CalRanges kept{d_ranges, d_seed_off, d_recount, R0};
      // the chunk's CAL bounds: their prefix sums and largest
      CalPlan whole{};
      uint64_t cends[2] = {};  // prefix of the last read, total
      e = cudaMemsetAsync(d_plan, 0, sizeof(CalPlan), st);
      if (e != cudaSuccess ||
          launch_cal_seeds(s->didx, d_bases, d_roff, R0, nrc, cp.seed_stride, d_count + R0, nullptr, nullptr,
                           nullptr, d_status, kept, st) < 0 ||
          launch_scan_u64(d_count + R0, nrc, d_cpre, d_sums, st) < 0 ||
          launch_cal_route(d_count + R0, nrc, nullptr, nullptr, d_plan, st) < 0) {
        e = cudaGetLastError();
        return done(SR_ECUDA, "sr_candidates_device count");
      }
      e = cudaMemcpyAsync(cends, d_cpre + nrc - 1, 16, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&whole, d_plan, sizeof(CalPlan), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device count copy");
      if (status & kStBadRead) return done(SR_EINVAL, "sr_candidates_device: decreasing read offsets or a read longer than 256 bases");
      if (status & kStBadBase) return done(SR_EBADBASE, "sr_candidates_device: read has a non-ACGT base");
      // sub-chunks of at most kCalChunkKeys CAL bounds (more only for a read that
      // alone has more), cut where the prefix sum crosses multiples of that less
      // the largest read's bound
      // SR_CAL_CHUNK_KEYS lowers it (tests of the cuts)
      const uint64_t kCalChunkKeys = std::max<uint64_t>(env_u64("SR_CAL_CHUNK_KEYS", 64ull << 20), 1);
      const uint64_t one = whole.max_all;
      const uint64_t want = std::max<uint64_t>(std::min<uint64_t>(std::max<uint64_t>(cends[1], 1), kCalChunkKeys), 2 * one);
      if (want > cap) {
        cap = want;
        d_cals = static_cast<uint64_t*>(cbuf(kCbCals, cap * 8));
        d_wkey = static_cast<uint64_t*>(cbuf(kCbWkey, cap * 8));
        d_whits = static_cast<uint32_t*>(cbuf(kCbWhits, cap * 4));
        d_wlen = static_cast<uint32_t*>(cbuf(kCbWlen, cap * 4));
        if (e != cudaSuccess) return done(SR_ENOMEM, "sr_candidates_device: device allocation failed");
      }
      if (cends[1] <= cap) {
        // the whole chunk in one sub-chunk: its prefix sums are its offsets
        e = cudaMemcpyAsync(d_off, d_cpre, (nrc + 1ull) * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device offsets");
        const sr_status r = run_sub(R0, nrc, kept);
        if (r != SR_OK) return r;
        continue;
      }
      const uint64_t span = cap - one;
      const uint32_t n_sub = static_cast<uint32_t>(cends[0] / span) + 1;
      sub.assign(n_sub + 1ull, 0);
      if (launch_cal_bounds(d_cpre, nrc, span, d_bounds, st) < 0) {
        e = cudaGetLastError();
        return done(SR_ECUDA, "sr_candidates_device sub-chunks");
      }
      e = cudaMemcpyAsync(sub.data(), d_bounds, n_sub * 4ull, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device sub-chunks");
      sub[n_sub] = nrc;
      for (uint32_t si = 0; si < n_sub; ++si) {
        const uint32_t a0 = sub[si], a1 = sub[si + 1];
        if (launch_cal_rebase(d_cpre, a0, a1 - a0, d_off, nullptr, st) < 0) {
          e = cudaGetLastError();
          return done(SR_ECUDA, "sr_candidates_device offsets");
        }
        const sr_status r = run_sub(R0 + a0, a1 - a0, kept);
        if (r != SR_OK) return r;
      }
    }
    // the device result arrays must be complete before the call returns
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(SR_ECUDA, "sr_candidates_device");
  }
  l->n_cands = total_w;
  if (out_dev) {
    if (!grow_out(std::max<uint64_t>(total_w, 1), total_w)) return done(SR_ENOMEM, "sr_candidates_device: device allocation failed");
    sr_status stt = done(SR_OK, "");
    if (stt != SR_OK) return stt;
    *out = l;
    return SR_OK;
  }
  // host output: the device list copied out through one pinned block, then
  // spread over the host threads into the list's own arrays
  sr_cand_list* h = nullptr;
  const sr_status sa = sr_cand_list_alloc(n, total_w, &h);
  if (sa != SR_OK) return done(sa, "sr_candidates_device: out of memory");
  const uint64_t part_bytes[6] = {(n + 1ull) * 8, total_w, total_w, total_w * 8, total_w * 4, total_w * 4};
  const void* src[6] = {L.off, L.ref, L.str, L.start, L.len, L.hits};
  void* dst[6] = {h->offsets, h->ref_id, h->strand, h->win_start, h->win_len, h->hits};
  uint64_t at[7] = {0};
  for (int k = 0; k < 6; ++k) at[k + 1] = (at[k] + part_bytes[k] + 255) & ~255ull;
  uint64_t got = 0;
  char* blk = static_cast<char*>(pool_take(s, at[6], &got));
  if (!blk) {
    // no pinned block to be had: copy straight into the list's own arrays
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
      if (part_bytes[k]) e = cudaMemcpyAsync(dst[k], src[k], part_bytes[k], cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      sr_cand_list_free(h);
      return done(SR_ECUDA, "sr_candidates_device list copy");
    }
    const sr_status stt = done(SR_OK, "");
    sr_cand_list_free(l);
    if (stt != SR_OK) {
      sr_cand_list_free(h);
      return stt;
    }
    *out = h;
    return SR_OK;
  }
  for (int k = 0; k < 6 && e == cudaSuccess; ++k)
    if (part_bytes[k]) e = cudaMemcpyAsync(blk + at[k], src[k], part_bytes[k], cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    pool_give(s, blk, got);
    sr_cand_list_free(h);
    return done(SR_ECUDA, "sr_candidates_device list copy");
  }
  constexpr uint64_t kSlice = 4ull << 20;  // bytes per host copy task
  std::vector<std::pair<int, uint64_t>> tasks;
  for (int k = 0; k < 6; ++k)
    for (uint64_t o = 0; o < part_bytes[k]; o += kSlice) tasks.emplace_back(k, o);
  parallel_for(static_cast<uint32_t>(tasks.size()), [&](uint32_t t) {
    const int k = tasks[t].first;
    const uint64_t o = tasks[t].second, len = std::min(kSlice, part_bytes[k] - o);
    std::memcpy(static_cast<char*>(dst[k]) + o, blk + at[k] + o, len);
  });
  pool_give(s, blk, got);
  const sr_status stt = done(SR_OK, "");
  sr_cand_list_free(l);
  if (stt != SR_OK) {
    sr_cand_list_free(h);
    return stt;
  }
  *out = h;
  return SR_OK;
}

extern "C" void sr_report_free(sr_report* rep) {
  if (!rep) return;
  free(rep->offsets);
  free(rep->hits);
  free(rep);
}

extern "C" sr_status sr_batch_report(sr_session* s, sr_batch* b, uint32_t kind, uint32_t n_best, sr_report** out) {
  Trace trace_("sr_batch_report");
  if (!s || !b || !out || b->s != s) return set_error(SR_EINVAL, "sr_batch_report: bad argument");
  *out = nullptr;
  if (!b->ran) return set_error(SR_EINVAL, "sr_batch_report: batch has not run");
  if (kind != SR_REPORT_BEST_N && kind != SR_REPORT_TIED)
    return set_error(SR_EINVAL, "sr_batch_report: kind must be SR_REPORT_BEST_N or SR_REPORT_TIED");
  if (kind == SR_REPORT_BEST_N && (n_best < 1 || n_best > SR_REPORT_MAX))
    return set_error(SR_EINVAL, "sr_batch_report: n_best must be 1..%u", SR_REPORT_MAX);
  cudaStream_t stream = b->last_opts.cuda_stream ? static_cast<cudaStream_t>(b->last_opts.cuda_stream) : b->stream;
  sr_status st = batch_sync(b, stream);
  if (st != SR_OK) return st;
  const uint32_t n = b->n_reads;
  const int nr = static_cast<int>(s->n_refs);
  auto* rep = static_cast<sr_report*>(calloc(1, sizeof(sr_report)));
  if (!rep) return set_error(SR_ENOMEM, "sr_batch_report: out of memory");
  rep->n_reads = n;
  rep->offsets = static_cast<uint64_t*>(calloc(n + 1ull, sizeof(uint64_t)));
  if (!rep->offsets) {
    sr_report_free(rep);
    return set_error(SR_ENOMEM, "sr_batch_report: out of memory");
  }
  if (n == 0) {
    *out = rep;
    return SR_OK;
  }
  uint32_t* scratch = nullptr;
  sr_report_hit* d_hits = nullptr;
  const uint64_t sw = report_scratch_words(n);
  cudaError_t e = cudaMalloc(&scratch, sw * 4);
  auto fail = [&](const char* where) {
    cudaGetLastError();
    if (scratch) cudaFree(scratch);
    if (d_hits) cudaFree(d_hits);
    sr_report_free(rep);
    return cuda_error(where, e == cudaSuccess ? cudaErrorUnknown : e);
  };
  if (e != cudaSuccess) return fail("sr_batch_report alloc");
  const int kd = static_cast<int>(kind);
  if (launch_report_count(b->d, nr, kd, n_best, scratch, stream) < 0) {
    e = cudaGetLastError();
    return fail("sr_batch_report count");
  }
  uint32_t tail[2] = {0, 0};  // total entries, truncated reads
  const uint32_t* d_off = scratch + n;
  e = cudaMemcpyAsync(&tail[0], d_off + n, 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&tail[1], scratch + sw - 1, 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail("sr_batch_report total");
  const uint64_t total = tail[0];
  rep->n_truncated = tail[1];
  rep->n_hits = total;
  rep->hits = static_cast<sr_report_hit*>(malloc((total ? total : 1) * sizeof(sr_report_hit)));
  std::vector<uint32_t> off32(n + 1ull);
  if (!rep->hits) {
    e = cudaErrorMemoryAllocation;
    return fail("sr_batch_report host alloc");
  }
  if (total) {
    e = cudaMalloc(&d_hits, total * sizeof(sr_report_hit));
    if (e != cudaSuccess) return fail("sr_batch_report alloc");
    if (launch_report_write(b->d, nr, kd, n_best, scratch, d_hits, stream) < 0) {
      e = cudaGetLastError();
      return fail("sr_batch_report write");
    }
    e = cudaMemcpyAsync(rep->hits, d_hits, total * sizeof(sr_report_hit), cudaMemcpyDeviceToHost, stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(off32.data(), d_off, (n + 1ull) * 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail("sr_batch_report copy");
  for (uint64_t i = 0; i <= n; ++i) rep->offsets[i] = off32[i];
  cudaFree(scratch);
  if (d_hits) cudaFree(d_hits);
  *out = rep;
  return SR_OK;
}

namespace sr {
// sr_align_batch calls of at least this many reads run as kParts batches
constexpr uint32_t kPartMinReads = 1u << 19;
constexpr int kParts = 3;
// where the parts end, in tenths of the call's windows: a small first part
// (whose staging nobody hides) and a small last part (whose fetch nobody hides)
constexpr uint64_t kPartEnd[kParts] = {1, 9, 10};

// One large sr_align_batch call as kParts batches of consecutive reads, each on
// a stream of its own.  A part's copies and host checks run while the parts
// before it compute, and its results come back while the parts after it
// compute.  A read's windows all stay in its part, so every result is the one a
// single batch gives; a later part's window indexes and CIGAR offsets are
// shifted on the device as its records are assembled.  An input error or a
// device error (bad base, window, timeout) is returned as it stands: staging
// checks the parts in read order and reports indexes in the caller's arrays, so
// the status and message are those of an unsplit call.  Only when a resource
// runs out (device arena, pinned host block, the call's shape does not split)
// does it return kRunAsOne, with nothing left allocated; the caller then runs
// the call as one batch.
constexpr sr_status kRunAsOne = 1;
static sr_status align_in_parts(sr_session* s, const sr_reads* reads, const sr_cand_list* cands,
                                const sr_score_params* sp, const sr_align_opts& o, sr_results** out) {
  Trace trace_("sr_align_batch parts");
  static_assert(kParts <= static_cast<int>(sizeof(sr_session::part_stream) / sizeof(cudaStream_t)), "streams");
  const uint32_t n = reads->n_reads;
  const uint64_t nc = cands->n_cands;
  if (!reads->offsets || !cands->offsets || cands->n_reads != n || cands->offsets[n] != nc) return kRunAsOne;
  // part k ends at the first read whose windows start at or past its share
  uint32_t rr[kParts + 1] = {0};
  for (int k = 0; k < kParts; ++k) {
    const uint64_t want = nc / kPartEnd[kParts - 1] * kPartEnd[k];
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo) / 2;
      if (cands->offsets[mid] < want) lo = mid + 1;
      else hi = mid;
    }
    rr[k + 1] = k == kParts - 1 ? n : lo;
    if (rr[k + 1] <= rr[k]) return kRunAsOne;
  }
  sr_align_opts oo = o;
  oo.cuda_stream = nullptr;
  sr_batch* b[kParts] = {};
  auto drop_parts = [&]() {
    for (auto*& x : b)
      if (x) {
        sr_batch_free(x);
        x = nullptr;
      }
  };
  for (int k = 0; k < kParts; ++k) {
    sr_status st = batch_stage_range(s, reads, cands, rr[k], rr[k + 1], s->part_stream[k], true, &b[k]);
    if (st == SR_OK) st = batch_run_async(s, b[k], sp, &oo);
    if (st != SR_OK) {
      drop_parts();
      return st == SR_ENOMEM ? kRunAsOne : st;
    }
  }
  const uint32_t nr = s->n_refs;
  const bool cig = o.want_cigar != 0, cls = o.classify != 0;
  // one pinned block for the arrays whose sizes are known now; the CIGAR
  // words get a second one (below)
  uint64_t off = 0;
  auto part = [&](uint64_t bytes) {
    const uint64_t at = off;
    off = (off + (bytes ? bytes : 1) + 255) & ~255ull;
    return at;
  };
  const uint64_t o_best = part(static_cast<uint64_t>(n) * sizeof(sr_hit));
  const uint64_t o_per = part(static_cast<uint64_t>(n) * nr * sizeof(sr_hit));
  const uint64_t o_sc = part(nc * 4);
  const uint64_t o_end = part(nc * 4);
  const uint64_t o_cls = cls ? part(n) : 0;
  uint64_t got = 0;
  char* blk = static_cast<char*>(pool_take(s, off, &got));
  sr_results* r = blk ? results_alloc() : nullptr;
  if (!r) {
    if (blk) pool_give(s, blk, got);
    drop_parts();
    return kRunAsOne;
  }
  auto* box = reinterpret_cast<ResultsBox*>(r);
  box->pool_of = s;
  box->block = blk;
  box->block_bytes = got;
  s->live.fetch_add(1);
  r->n_reads = n;
  r->n_refs = nr;
  r->n_items = nc;
  for (auto* x : b) {
    r->cells += x->cells;
    r->n_i32_items += x->i32_items;
  }
  r->best = reinterpret_cast<sr_hit*>(blk + o_best);
  r->best_per_ref = reinterpret_cast<sr_hit*>(blk + o_per);
  r->item_score = reinterpret_cast<int32_t*>(blk + o_sc);
  r->item_end = reinterpret_cast<uint32_t*>(blk + o_end);
  if (cls) r->read_class = reinterpret_cast<uint8_t*>(blk + o_cls);
  // st_fail: the status to return (kRunAsOne when a host block ran out)
  auto fail = [&](sr_status st_fail) {
    for (auto* x : b)
      if (x) cudaStreamSynchronize(x->stream);
    cudaGetLastError();
    sr_results_free(r);
    drop_parts();
    return st_fail;
  };
  cudaError_t e = cudaSuccess;
  auto copy = [&](void* dst, const void* src, uint64_t bytes, cudaStream_t st) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
  };
  uint32_t total[kParts] = {};
  uint64_t i0 = 0, c0 = 0;  // windows and CIGAR words of the parts before
  // The CIGAR block is taken once every part but the last is done, sized for
  // their words plus an estimate of the last part's (its reads at 1.25x the
  // words per read so far), so the earlier parts' CIGARs come back while the
  // last part computes.  An estimate that falls short is replaced at the end by
  // a block of the exact size, into which every part is copied again.
  int cig_parts = 0;  // parts whose CIGARs are copied into the block
  uint64_t cig_cap = 0;
  auto take_cigar_block = [&](uint64_t words) -> bool {
    uint64_t got_c = 0;
    void* p = pool_take(s, std::max<uint64_t>(words * 4, 256), &got_c);
    if (!p) return false;
    box->cig_block = p;
    box->cig_block_bytes = got_c;
    r->cigar = static_cast<uint32_t*>(p);
    cig_cap = got_c / 4;
    return true;
  };
  auto copy_cigars = [&](int upto) {
    uint64_t at = 0;
    for (int k = 0; k < upto; ++k) {
      if (k >= cig_parts) copy(r->cigar + at, b[k]->d.cigar, static_cast<uint64_t>(total[k]) * 4, b[k]->stream);
      at += total[k];
    }
    cig_parts = upto;
  };
  for (int k = 0; k < kParts; ++k) {
    sr_batch* x = b[k];
    cudaStream_t st = x->stream;
    const sr_status sst = batch_sync(x, st);
    if (sst != SR_OK) return fail(sst);
    const uint32_t r0 = rr[k];
    if (i0 > static_cast<uint64_t>(INT32_MAX) || c0 > UINT32_MAX)
      return fail(set_error(SR_EINVAL, "sr_align_batch: more than 2^31 windows or 2^32 CIGAR words"));
    if (launch_assemble(x->d, static_cast<int>(nr), cig, static_cast<int32_t>(i0), static_cast<uint32_t>(c0),
                        st) < 0)
      return fail(cuda_error("sr_align_batch assemble", cudaGetLastError()));
    if (cig) {
      e = cudaMemcpyAsync(&total[k], x->d.cigar_off + x->n_reads, 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    // this part's results come back while the later parts compute
    copy(r->item_score + i0, x->d.item_score, x->n_items * 4, st);
    copy(r->item_end + i0, x->d.item_end, x->n_items * 4, st);
    copy(r->best + r0, x->d.out_best, static_cast<uint64_t>(x->n_reads) * sizeof(sr_hit), st);
    copy(r->best_per_ref + static_cast<uint64_t>(r0) * nr, x->d.out_per_ref,
         static_cast<uint64_t>(x->n_reads) * nr * sizeof(sr_hit), st);
    if (cls) copy(r->read_class + r0, x->d.read_class, x->n_reads, st);
    if (e != cudaSuccess) return fail(cuda_error("sr_align_batch copy", e));
    i0 += x->n_items;
    c0 += total[k];
    if (cig && k == kParts - 2) {
      const uint64_t n_done = rr[k + 1], n_last = n - n_done;
      if (!take_cigar_block(c0 + c0 * n_last * 5 / (4 * n_done) + 4096)) return fail(kRunAsOne);
      copy_cigars(k + 1);
      if (e != cudaSuccess) return fail(cuda_error("sr_align_batch copy", e));
    }
  }
  if (cig) {
    if (c0 > cig_cap) {
      // the estimate fell short: wait for the copies into the first block, then
      // copy every part into one of the exact size
      for (int k = 0; k < cig_parts; ++k)
        if (e == cudaSuccess) e = cudaStreamSynchronize(b[k]->stream);
      if (e != cudaSuccess) return fail(cuda_error("sr_align_batch copy", e));
      pool_give(s, box->cig_block, box->cig_block_bytes);
      box->cig_block = nullptr;
      cig_parts = 0;
      if (!take_cigar_block(c0)) return fail(kRunAsOne);
    }
    copy_cigars(kParts);
    r->n_cigar = c0;
  }
  for (auto* x : b)
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return fail(cuda_error("sr_align_batch copy", e));
  drop_parts();
  *out = r;
  return SR_OK;
}
}  // namespace sr

extern "C" sr_status sr_align_batch(sr_session* s, const sr_reads* reads, const sr_cand_list* cands,
                                    const sr_score_params* sp, const sr_align_opts* opts, sr_results** out) {
  Trace trace_("sr_align_batch");
  if (!out) return set_error(SR_EINVAL, "sr_align_batch: null out");
  *out = nullptr;
  // inputs in device memory are staged as one batch: with no host copies to hide, parts gain nothing
  if (s && reads && cands && sp && reads->n_reads >= kPartMinReads && !((reads->flags | cands->flags) & SR_FLAG_DEVICE)) {
    const sr_align_opts o = opts ? *opts : default_opts();
    if (!o.cuda_stream && o.engine != SR_ENGINE_PLAIN) {
      const sr_status st = align_in_parts(s, reads, cands, sp, o, out);
      if (st != kRunAsOne) return st;
    }
  }
  sr_batch* b = nullptr;
  sr_status st = sr_batch_stage(s, reads, cands, opts ? opts->cuda_stream : nullptr, &b);
  if (st != SR_OK) return st;
  st = sr_batch_run(s, b, sp, opts);
  if (st == SR_OK) st = sr_batch_fetch(s, b, out);
  sr_batch_free(b);
  return st;
}

extern "C" sr_status sr_batch_classify(sr_session* s, sr_batch* b, const sr_classify_params* params,
                                       uint8_t* class_out) {
  if (!s || !b || !class_out) return set_error(SR_EINVAL, "sr_batch_classify: null argument");
  if (!b->ran) return set_error(SR_EINVAL, "sr_batch_classify: batch has not run");
  if (s->n_refs < 2) return set_error(SR_EINVAL, "sr_batch_classify: needs 2 references");
  const int32_t ms = params ? params->min_score : 40, mg = params ? params->margin : 5;
  cudaStream_t stream = b->stream;
  if (launch_classify(b->d, static_cast<int>(s->n_refs), ms, mg, stream) < 0)
    return cuda_error("sr_batch_classify launch", cudaGetLastError());
  cudaError_t e = cudaMemcpyAsync(class_out, b->d.read_class, b->n_reads, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_error("sr_batch_classify", e);
  return SR_OK;
}

namespace {
// device (or managed) memory, as opposed to host memory, pinned or not
bool on_device(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" sr_status sr_classify(const sr_results* res, const sr_classify_params* params, uint8_t* class_out) {
  Trace trace_("sr_classify");
  if (!res || !class_out) return set_error(SR_EINVAL, "sr_classify: null argument");
  if (res->n_refs < 2) return set_error(SR_EINVAL, "sr_classify: needs results over 2 references");
  const uint32_t n = res->n_reads, nr = res->n_refs;
  if (n == 0) return SR_OK;
  if (!res->best_per_ref) return set_error(SR_EINVAL, "sr_classify: results have no per-reference records");
  const int32_t ms = params ? params->min_score : 40, mg = params ? params->margin : 5;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return set_error(SR_ECUDA, "sr_classify: no CUDA device available");
  }
  cudaStream_t st = cudaStreamPerThread;
  const bool hits_dev = on_device(res->best_per_ref), out_dev = on_device(class_out);
  const uint64_t hit_bytes = static_cast<uint64_t>(n) * nr * sizeof(sr_hit);
  const sr_hit* d_hits = res->best_per_ref;
  uint8_t* d_out = class_out;
  void* tmp_hits = nullptr;
  void* tmp_out = nullptr;
  cudaError_t e = cudaSuccess;
  if (!hits_dev) {
    e = cudaMallocAsync(&tmp_hits, hit_bytes, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp_hits, res->best_per_ref, hit_bytes, cudaMemcpyHostToDevice, st);
    d_hits = static_cast<const sr_hit*>(tmp_hits);
  }
  if (e == cudaSuccess && !out_dev) {
    e = cudaMallocAsync(&tmp_out, n, st);
    d_out = static_cast<uint8_t*>(tmp_out);
  }
  if (e == cudaSuccess && launch_classify_hits(d_hits, n, nr, ms, mg, d_out, st) < 0) e = cudaGetLastError();
  if (e == cudaSuccess && !out_dev) e = cudaMemcpyAsync(class_out, d_out, n, cudaMemcpyDeviceToHost, st);
  if (tmp_hits) cudaFreeAsync(tmp_hits, st);
  if (tmp_out) cudaFreeAsync(tmp_out, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_error("sr_classify", e);
  return SR_OK;
}

// ------------------------------------------------------------------ tuning table
extern "C" sr_status sr_tune_get(uint32_t* n_bins, uint32_t* upper, uint32_t* lanes, uint32_t* rows, uint32_t cap) {
  TuneBin b[kNumBins];
  tune_get_bins(b);
  if (n_bins) *n_bins = kNumBins;
  for (uint32_t i = 0; i < kNumBins && i < cap; ++i) {
    if (upper) upper[i] = b[i].upper;
    if (lanes) lanes[i] = b[i].lanes;
    if (rows) rows[i] = b[i].rows;
  }
  return SR_OK;
}

extern "C" sr_status sr_tune_set(uint32_t n_bins, const uint32_t* upper, const uint32_t* lanes, const uint32_t* rows) {
  if (n_bins != kNumBins || !upper || !lanes || !rows) return set_error(SR_EINVAL, "sr_tune_set: need %d bins", kNumBins);
  TuneBin b[kNumBins];
  for (uint32_t i = 0; i < kNumBins; ++i) {
    if (!extend_config_supported(lanes[i], rows[i]) || lanes[i] * rows[i] < upper[i] ||
        (i > 0 && upper[i] <= upper[i - 1]) || upper[i] > SR_MAX_READ_LEN)
      return set_error(SR_EINVAL, "sr_tune_set: bin %u: unsupported shape or bad bound", i);
    b[i] = TuneBin{upper[i], lanes[i], rows[i]};
  }
  if (b[kNumBins - 1].upper != SR_MAX_READ_LEN) return set_error(SR_EINVAL, "sr_tune_set: last bin must end at 256");
  tune_set_bins(b);
  return SR_OK;
}

extern "C" sr_status sr_tune_save(const char* path) {
  if (!path) return set_error(SR_EINVAL, "sr_tune_save: null path");
  TuneBin b[kNumBins];
  tune_get_bins(b);
  cudaDeviceProp p{};
  int dev = 0;
  cudaGetDevice(&dev);
  const bool have = cudaGetDeviceProperties(&p, dev) == cudaSuccess;
  FILE* f = fopen(path, "w");
  if (!f) return set_error(SR_EIO, "sr_tune_save: cannot open");
  fprintf(f, "# libsr tune table: device %s\n", have ? p.name : "unknown");
  for (int i = 0; i < kNumBins; ++i) fprintf(f, "%u %u %u\n", b[i].upper, b[i].lanes, b[i].rows);
  return fclose(f) == 0 ? SR_OK : set_error(SR_EIO, "sr_tune_save: write failed");
}

extern "C" sr_status sr_tune_load(const char* path) {
  if (!path) return set_error(SR_EINVAL, "sr_tune_load: null path");
  FILE* f = fopen(path, "r");
  if (!f) return set_error(SR_EIO, "sr_tune_load: cannot open");
  uint32_t up[kNumBins], la[kNumBins], ro[kNumBins];
  char line[256];
  int n = 0;
  while (n < kNumBins && fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    if (sscanf(line, "%u %u %u", &up[n], &la[n], &ro[n]) == 3) ++n;
  }
  fclose(f);
  if (n != kNumBins) return set_error(SR_EIO, "sr_tune_load: expected %d bins", kNumBins);
  return sr_tune_set(kNumBins, up, la, ro);
}

// Autotuner: for each read-length bin, time every supported kernel shape whose
// rows cover the bin on a synthetic sample (reads of the bin's longest length,
// 6 windows of length m + 64 each at random positions of reference 0) and keep
// the fastest.
extern "C" sr_status sr_tune(sr_session* s, const sr_score_params* sp, uint32_t sample_reads) {
  Trace trace_("sr_tune");
  if (!s) return set_error(SR_EINVAL, "sr_tune: null session");
  sr_status st = check_score(sp);
  if (st != SR_OK) return st;
  if (sample_reads == 0) sample_reads = 4096;
  uint32_t sh_lanes[64], sh_rows[64];
  const int n_shapes = std::min(64, extend_shapes(sh_lanes, sh_rows, 64));
  const bool verbose = getenv("SR_TUNE_VERBOSE") != nullptr;
  TuneBin cur[kNumBins];
  tune_get_bins(cur);
  uint64_t rng = 0x9E3779B97F4A7C15ull;
  auto next = [&]() {
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return rng;
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int bi = 0; bi < kNumBins; ++bi) {
    // reads of lengths spread over the bin (row padding counts as it will in use)
    const uint32_t m = cur[bi].upper;
    const uint32_t m_lo = (bi ? cur[bi - 1].upper : 0u) + 1u;
    const uint32_t nw = 6;
    std::vector<uint64_t> roff(sample_reads + 1ull), coff(sample_reads + 1ull);
    std::vector<uint32_t> mlen(sample_reads);
    roff[0] = 0;
    for (uint32_t r = 0; r < sample_reads; ++r) {
      mlen[r] = m_lo + static_cast<uint32_t>(next() % (m - m_lo + 1));
      roff[r + 1] = roff[r] + mlen[r];
      coff[r + 1] = static_cast<uint64_t>(r + 1) * nw;
    }
    coff[0] = 0;
    std::vector<char> bases(roff[sample_reads]);
    for (auto& c : bases) c = "ACGT"[next() & 3];
    std::vector<uint8_t> cref(static_cast<size_t>(sample_reads) * nw, 0), cstr(cref.size(), 0);
    std::vector<uint64_t> cst(cref.size());
    std::vector<uint32_t> cln(cref.size());
    const uint64_t L = s->lens[0];
    for (size_t k = 0; k < cref.size(); ++k) {
      const uint32_t wl = static_cast<uint32_t>(std::min<uint64_t>(mlen[k / nw] + 64, L));
      cln[k] = wl;
      cst[k] = (L > wl) ? next() % (L - wl) : 0;
    }
    sr_reads rd{sample_reads, 0, bases.data(), roff.data()};
    sr_cand_list cl{};
    cl.n_reads = sample_reads;
    cl.n_cands = cref.size();
    cl.offsets = coff.data();
    cl.ref_id = cref.data();
    cl.strand = cstr.data();
    cl.win_start = cst.data();
    cl.win_len = cln.data();
    sr_batch* b = nullptr;
    st = batch_stage_internal(s, &rd, &cl, nullptr, false, &b);
    if (st != SR_OK) break;
    float best_ms = 1e30f, cur_ms = -1.0f;
    TuneBin pick = cur[bi];
    for (int q = 0; q < n_shapes; ++q) {
      const uint32_t sh[2] = {sh_lanes[q], sh_rows[q]};
      if (sh[0] * sh[1] < m || sh[0] * sh[1] > 2 * m + 64) continue;
      sr_align_opts o = default_opts();
      o.want_cigar = 0;
      o.lanes = sh[0];
      o.rows = sh[1];
      float tot = 0;
      bool ok = true;
      for (int rep = 0; rep < 7 && ok; ++rep) {
        if (rep == 2) cudaEventRecord(e0, b->stream);
        ok = batch_run_async(s, b, sp, &o) == SR_OK;
      }
      cudaEventRecord(e1, b->stream);
      if (ok) ok = batch_sync(b, b->stream) == SR_OK;
      if (!ok) continue;
      cudaEventElapsedTime(&tot, e0, e1);
      if (verbose)
        fprintf(stderr, "sr_tune bin<=%u lanes %u rows %u: %.3f ms for 5 runs\n", m, sh[0], sh[1], tot);
      if (sh[0] == cur[bi].lanes && sh[1] == cur[bi].rows) cur_ms = tot;
      if (tot < best_ms) {
        best_ms = tot;
        pick = TuneBin{m, sh[0], sh[1]};
      }
    }
    sr_batch_free(b);
    // the bin's current shape stays unless a candidate beats it by more than
    // 1.5%: a persistent grid's tail on the sample is about that size, and the
    // sample runs alone where the batch's bins share the device
    if (cur_ms > 0.0f && best_ms > cur_ms / 1.015f) pick = cur[bi];
    cur[bi] = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SR_OK) return st;
  tune_set_bins(cur);
  return SR_OK;
}

extern "C" sr_status sr_probe_wait(uint32_t poll_limit, uint32_t arrive) {
  if (poll_limit == 0 || poll_limit > (1u << 24)) return set_error(SR_EINVAL, "sr_probe_wait: poll_limit 1..2^24");
  uint32_t st = 0;
  if (probe_wait(poll_limit, arrive ? 1 : 0, &st) != 0) return cuda_error("sr_probe_wait", cudaGetLastError());
  if (st & kStTimeout) return set_error(SR_ETIMEOUT, "sr_probe_wait: the bounded wait ran out (status word)");
  return SR_OK;
}

extern "C" sr_status sr_probe_dpx(double* rate, double* mhz) {
  if (!rate || !mhz) return set_error(SR_EINVAL, "sr_probe_dpx: null argument");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return set_error(SR_ECUDA, "no CUDA device");
  if (probe_dpx(rate, mhz) != 0) return cuda_error("sr_probe_dpx", cudaGetLastError());
  return SR_OK;
}
