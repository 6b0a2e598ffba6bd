// sr_serve.h -- continuous-batching request server of libsr (internal).
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "sr_host.h"

namespace sr {
struct Server;
void serve_destroy(Server* sv);  // stops the scheduler and frees the server
uint64_t batch_bytes_estimate(uint32_t n_reads, uint64_t n_items, uint64_t n_bases, uint32_t n_refs);
cudaStream_t session_stream(sr_session* s);
uint64_t session_budget(sr_session* s);
std::atomic<uint64_t>& session_used(sr_session* s);
Server*& session_server(sr_session* s);
uint32_t session_n_refs(sr_session* s);
sr_status batch_stage_internal(sr_session* s, const sr_reads* reads, const sr_cand_list* cands,
                               void* stream, bool check_budget, sr_batch** out);
// the shortest read length whose windows the int32 kernel scores under these
// parameters (0: every window; SR_MAX_READ_LEN + 1: none)
uint32_t i32_min_read_len(const sr_score_params& sp, const sr_align_opts& o);
// a serving round: every kernel of the path plus the result records, launched
// directly on the batch's stream; ev_first is recorded once the first kernel is
// done, and the extension kernels (and all after them) wait for wait_extend
// (either may be null)
sr_status batch_run_serving(sr_session* s, sr_batch* b, const sr_score_params* sp, const sr_align_opts* opts,
                            cudaEvent_t ev_first, cudaEvent_t wait_extend);
sr_status batch_stage_range(sr_session* s, const sr_reads* reads, const sr_cand_list* cands, uint32_t r0,
                            uint32_t r1, void* stream, bool check_budget, sr_batch** out);
}  // namespace sr
