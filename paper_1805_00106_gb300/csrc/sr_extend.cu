// sr_extend.cu -- launchers of the extension kernels (see sr_extend.cuh), the
// int32 path and the DPX issue-rate probe.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sr_extend.cuh"

namespace sr {
namespace {

ExtArgs make_args(const BatchDev& b, const DevRefs& refs, const ScoreConst& sc) {
  ExtArgs a{};
  a.rpack = b.rpack;
  a.rlen = b.rlen;
  a.c_ref = b.c_ref;
  a.c_strand = b.c_strand;
  a.c_start = b.c_start;
  a.c_len = b.c_len;
  a.item_read = b.item_read;
  a.order = b.order;
  a.class_range = b.class_range;
  a.queue = b.queue;
  a.refs = refs;
  a.item_score = b.item_score;
  a.item_end = b.item_end;
  a.item_iend = b.item_iend;
  a.status = b.status;
  a.n_items = b.n_items;
  a.sa = sc.sa;
  a.sb = sc.sb;
  a.go = sc.go;
  a.ge = sc.ge;
  a.k16 = 65536u;
  return a;
}


}  // namespace

int fanout_begin(const Fanout& f, cudaStream_t st) {
  if (cudaEventRecord(f.fork, st) != cudaSuccess) return -1;
  for (int i = 0; i < kSide; ++i)
    if (cudaStreamWaitEvent(f.side[i], f.fork, 0) != cudaSuccess) return -1;
  return 0;
}

int fanout_end(const Fanout& f, cudaStream_t st) {
  for (int i = 0; i < kSide; ++i) {
    if (cudaEventRecord(f.join[i], f.side[i]) != cudaSuccess) return -1;
    if (cudaStreamWaitEvent(st, f.join[i], 0) != cudaSuccess) return -1;
  }
  return 0;
}

int launch_winner_rows(const BatchDev& b, const DevRefs& refs, const ScoreConst& sc, uint32_t lanes,
                       uint32_t rows, cudaStream_t st) {
  ExtArgs a = make_args(b, refs, sc);
  a.order = b.order;  // winners of every read length in one range (class 0)
  a.class_range = b.wrange;
  a.queue = b.wqueue;
  a.item_iend = b.item_iend;
  a.cls = 0;
  // one shape that holds every read length (256 rows)
  const int k = dispatch_mode2(lanes ? lanes : 16u, rows ? rows : 16u, a, st);
  return k < 0 ? -1 : k;
}

int extend_shapes(uint32_t* lanes, uint32_t* rows, int cap) {
  int n = 0;
#define SR_LIST(g, r)     \
  if (n < cap) {          \
    lanes[n] = g;         \
    rows[n] = r;          \
  }                       \
  ++n;
  SR_SHAPES(SR_LIST)
#undef SR_LIST
  return n;
}

bool extend_config_supported(uint32_t lanes, uint32_t rows) {
#define SR_CHK(g, r) \
  if (lanes == g && rows == r) return true;
  SR_SHAPES(SR_CHK)
#undef SR_CHK
  return false;
}

int launch_extend(const BatchDev& b, const DevRefs& refs, const ScoreConst& sc,
                  const TuneBin* bins, int n_bins, int mode, bool plain, uint32_t lanes,
                  uint32_t rows, cudaStream_t st, const uint64_t* class_items, const Fanout* fan) {
  ExtArgs a = make_args(b, refs, sc);
  int launched = 0;
  if (plain) {
    // one ordinary launch over the items in input order, one kernel shape
    a.order = nullptr;
    a.cls = 0;
    uint32_t g = lanes ? lanes : 16, r = rows ? rows : 16;
    uint64_t tasks = (b.n_items + 1) / 2;
    int k = mode == 1 ? dispatch_mode1(false, g, r, a, st, tasks)
                      : dispatch_mode0(false, g, r, a, st, tasks);
    return k < 0 ? -1 : k;
  }
  if (fan && fanout_begin(*fan, st) < 0) return -1;
  int next = 0;
  const int width = fan_width(b.n_reads);
  // longest reads first: each side stream starts on a large bin
  for (int c = n_bins - 1; c >= 0; --c) {
    if (class_items && class_items[c] == 0) continue;
    a.cls = c;
    uint32_t g = lanes ? lanes : bins[c].lanes, r = rows ? rows : bins[c].rows;
    const cudaStream_t s = fan ? fan->side[next++ % width] : st;
    int k = mode == 1 ? dispatch_mode1(true, g, r, a, s, 0) : dispatch_mode0(true, g, r, a, s, 0);
    if (k < 0) return -1;
    launched += k;
  }
  a.cls = kI32Class;
  if (!class_items || class_items[kI32Class] != 0) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const cudaStream_t s = fan ? fan->side[next++ % width] : st;
    if (mode == 1) k_extend32<1><<<nsm * 4, 128, 0, s>>>(a);
    else k_extend32<0><<<nsm * 4, 128, 0, s>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    ++launched;
  }
  if (fan && fanout_end(*fan, st) < 0) return -1;
  return launched;
}

// ---------------------------------------------------------------- DPX probe
// Issue rate of the packed 16-bit add-max: 8 independent chains per thread,
// 4 co-resident blocks of 256 threads per SM; each block times itself in SM
// clock cycles, so the rate is per clock whatever the clock was.
__global__ void k_probe_dpx(uint32_t* out, unsigned long long* cycles, uint32_t seed, int iters) {
  uint32_t x[8], y[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    x[c] = seed * (threadIdx.x + 7u * c + 1u);
    y[c] = x[c] ^ 0x00050003u;
  }
  const uint32_t k1 = seed | 0x00010001u;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = __viaddmax_s16x2(x[c], k1, y[c]);
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) r ^= x[c] + y[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
  __syncthreads();
  if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(clock64() - t0);
}

// ---------------------------------------------------------------- bounded wait probe
// The window copies of the extension kernels complete on an mbarrier that a
// kernel polls a bounded number of times before it records kStTimeout and
// returns.  This probe runs the same polling on a barrier that gets its one
// arrival (arrive = 1) or none (a flag nothing sets), so a test can check that
// a wait that never completes ends as a status, not a hang.
__global__ void k_probe_wait(uint32_t poll_limit, int arrive, uint32_t* status) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    bool done = false;
    for (uint32_t it = 0; it < poll_limit && !done; ++it) done = mbar_try_wait(&bar, 0);
    if (!done) atomicOr(status, kStTimeout);
  }
}

int probe_wait(uint32_t poll_limit, int arrive, uint32_t* status_out) {
  uint32_t* d = nullptr;
  if (cudaMalloc(&d, 4) != cudaSuccess) return -1;
  cudaMemset(d, 0, 4);
  k_probe_wait<<<1, 32>>>(poll_limit, arrive, d);
  cudaError_t e = cudaMemcpy(status_out, d, 4, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int probe_dpx(double* lane_ops_per_clk_per_sm, double* clk_mhz) {
  int dev = 0, nsm = 0, clk_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int bs = 256, bpsm = 4, iters = 8192;
  const int grid = nsm * bpsm;
  uint32_t* d = nullptr;
  unsigned long long* cyc = nullptr;
  if (cudaMalloc(&d, static_cast<size_t>(grid) * bs * 4) != cudaSuccess) return -1;
  if (cudaMalloc(&cyc, static_cast<size_t>(grid) * 8) != cudaSuccess) {
    cudaFree(d);
    return -1;
  }
  for (int w = 0; w < 3; ++w) k_probe_dpx<<<grid, bs>>>(d, cyc, 3u + w, iters);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  k_probe_dpx<<<grid, bs>>>(d, cyc, 7u, iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  unsigned long long* h = new unsigned long long[grid];
  cudaMemcpy(h, cyc, static_cast<size_t>(grid) * 8, cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  cudaFree(cyc);
  if (cudaGetLastError() != cudaSuccess || ms <= 0) {
    delete[] h;
    return -1;
  }
  unsigned long long mx = 0;
  for (int i = 0; i < grid; ++i) mx = h[i] > mx ? h[i] : mx;
  delete[] h;
  const double ops_per_sm = static_cast<double>(bpsm) * bs * 8.0 * iters;
  *lane_ops_per_clk_per_sm = ops_per_sm / static_cast<double>(mx);
  // effective SM clock over the timed launch
  *clk_mhz = static_cast<double>(mx) / (ms * 1e3);
  (void)clk_khz;
  return 0;
}

int preload_extend() {
  int n_ = 0;
  SR_TOUCH(k_extend32<0>);
  SR_TOUCH(k_extend32<1>);
  SR_TOUCH(k_probe_dpx);
  SR_TOUCH(k_probe_wait);
  return n_;
}

}  // namespace sr
