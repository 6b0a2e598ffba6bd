// sr_host.h -- helpers shared by libsr's host translation units.
#pragma once
#include <stdint.h>

#include <functional>

#include "../../include/sr.h"
#include <nvtx3/nvToolsExt.h>

namespace sr {
// records a thread-local message for sr_last_error() and returns `st`
sr_status set_error(sr_status st, const char* fmt, ...);
// ASCII bases -> 2-bit codes (A=0 C=1 G=2 T=3); -1 on a non-ACGT byte
int encode_ascii(const char* s, uint64_t n, uint8_t* out);
// the index's reference as 2-bit codes
const uint8_t* index_codes(const sr_index* idx, uint64_t* len);
// the index's tables (pointer table of 4^address_bases + 1 bucket starts; per
// entry the hashed seed's key bits, reference position and orientation bits)
struct IndexTables {
  uint32_t seed_len, address_bases;
  uint64_t hash_seed, ref_len;
  const uint64_t* ptr;
  uint64_t n_ptr;
  const uint32_t* key;
  const uint32_t* pos;
  const uint8_t* orient;
  uint64_t n_entries;
};
IndexTables index_tables(const sr_index* idx);
// a zeroed sr_results whose arrays the caller allocates with malloc (released by sr_results_free)
sr_results* results_alloc();
// threads of the host pool (workers + the caller), at most 16
unsigned host_threads();
// fn(0) .. fn(n - 1) spread over the pool's threads; returns when all are done
void parallel_for(uint32_t n, const std::function<void(uint32_t)>& fn);
// NVTX range over a host stage (visible in profiler timelines; free without a tool attached)
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
};
}  // namespace sr
