// sr_serve.cpp -- continuous batching for libsr.
//
// Requests (a read batch plus its candidate windows) are copied at submit and
// queued.  Two threads keep the device busy:
//  - the scheduler admits every queued request whose device footprint still
//    fits the session's HBM budget (FIFO, bounded by max_inflight and by
//    kMaxRoundReads reads per round), merges them into the next round, stages
//    its inputs and launches every kernel of the round on a stream of its own,
//    as long as fewer than kDepth rounds are in flight;
//  - the completer waits for the oldest round, copies its results back, splits
//    them per request (window and CIGAR indexes rebased) and completes those
//    requests, freeing their budget and the round's slot.
// So round k+1 is on the device before round k ends: its first kernels (read
// packing, work list, length bins) run beside round k's last ones, and its
// extension kernels wait on the device (not on the host) for round k's last
// kernel, so that round k's latency-bound tail (selection, traceback, result
// records) is not crowded out by round k+1's persistent kernels.  Round k's
// copies back, the split and the frees run while round k+1 computes.
// Each read's result depends only on that read and its windows, so a request
// gets identical results alone or in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "sr_host.h"
#include "sr_serve.h"

namespace sr {
namespace {
using Clock = std::chrono::steady_clock;
constexpr uint64_t kMaxRoundReads = 131072;
// rounds in flight (launched, not yet completed): one computing, the next
// queued behind it on the device
constexpr int kDepth = 2;
// device timelines of the most recent rounds kept for sr_serve_overlap
constexpr size_t kTimelineCap = 1u << 16;

struct Request {
  uint64_t ticket = 0;
  std::vector<char> bases;
  std::vector<uint64_t> roff, coff, cstart;
  std::vector<uint8_t> cref, cstr;
  std::vector<uint32_t> clen;
  uint64_t bytes = 0, cells = 0;
  uint32_t n_reads = 0;
  Clock::time_point t_submit, t_done;
  sr_results* res = nullptr;
  sr_status status = SR_OK;
  bool done = false;
};

// a round's stream and the events that time it on the device
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t first = nullptr;  // after the round's first kernel
  cudaEvent_t last = nullptr;   // after its last kernel
  bool busy = false;
};

struct Round {
  std::vector<Request*> reqs;
  sr_batch* b = nullptr;
  sr_status status = SR_OK;
  int slot = -1;
  bool timed = false;  // its events were recorded
};

}  // namespace

struct Server {
  sr_session* s = nullptr;
  int device = 0;
  sr_score_params sp{};
  sr_align_opts opts{};
  uint32_t max_inflight = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_round;
  std::deque<Request*> pending;
  std::map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  uint64_t reserved = 0;
  uint64_t inflight = 0;
  bool stop = false;
  bool sched_done = false;
  std::thread th_sched, th_done;
  // completed requests, in completion order: latency (us), size (reads) and
  // completion time (s after sr_serve_start)
  std::vector<double> lat_us;
  std::vector<uint32_t> lat_reads;
  std::vector<double> lat_done_s;
  Clock::time_point t_start = Clock::now();
  uint64_t rounds = 0, rounds_done = 0, max_round = 0, budget_waits = 0;
  // rounds launched and not yet completed, oldest first (the completer's queue)
  std::deque<Round> launched;
  Slot slots[kDepth];
  cudaEvent_t t0 = nullptr;      // device time origin of the timelines
  int last_slot = -1;            // slot of the round launched last
  // per completed round: (first kernel done, last kernel done) in ms after t0
  std::vector<std::pair<float, float>> timeline;
};

namespace {

sr_results* slice_results(const sr_results* all, uint32_t r0, uint32_t r1, uint64_t i0, uint64_t i1,
                          uint64_t cells, uint64_t i32_items) {
  const uint32_t n = r1 - r0, nr = all->n_refs;
  const uint64_t ni = i1 - i0;
  sr_results* r = results_alloc();
  if (!r) return nullptr;
  r->n_reads = n;
  r->n_refs = nr;
  r->n_items = ni;
  r->cells = cells;
  r->n_i32_items = i32_items;
  r->best = static_cast<sr_hit*>(malloc((n ? n : 1) * sizeof(sr_hit)));
  r->best_per_ref = static_cast<sr_hit*>(malloc(static_cast<size_t>(n ? n : 1) * nr * sizeof(sr_hit)));
  r->item_score = static_cast<int32_t*>(malloc((ni ? ni : 1) * 4));
  r->item_end = static_cast<uint32_t*>(malloc((ni ? ni : 1) * 4));
  uint64_t cw0 = 0, cw1 = 0;
  if (all->cigar) {
    for (uint32_t k = r0; k < r1; ++k)
      if (all->best[k].cigar_len) {
        cw0 = all->best[k].cigar_off;
        break;
      }
    cw1 = cw0;
    for (uint32_t k = r0; k < r1; ++k)
      if (all->best[k].cigar_len) cw1 = all->best[k].cigar_off + all->best[k].cigar_len;
    r->n_cigar = cw1 - cw0;
    r->cigar = static_cast<uint32_t*>(malloc((r->n_cigar ? r->n_cigar : 1) * 4));
    if (r->cigar && r->n_cigar) memcpy(r->cigar, all->cigar + cw0, r->n_cigar * 4);
  }
  if (all->read_class) {
    r->read_class = static_cast<uint8_t*>(malloc(n ? n : 1));
    if (r->read_class && n) memcpy(r->read_class, all->read_class + r0, n);
  }
  if (!r->best || !r->best_per_ref || !r->item_score || !r->item_end || (all->cigar && !r->cigar) ||
      (all->read_class && !r->read_class)) {
    sr_results_free(r);
    return nullptr;
  }
  auto fix = [&](sr_hit h, bool with_cigar) {
    if (h.item >= 0) h.item -= static_cast<int32_t>(i0);
    if (with_cigar && h.cigar_len) h.cigar_off -= static_cast<uint32_t>(cw0);
    else if (!h.cigar_len) h.cigar_off = 0;
    return h;
  };
  for (uint32_t k = 0; k < n; ++k) {
    r->best[k] = fix(all->best[r0 + k], true);
    for (uint32_t q = 0; q < nr; ++q)
      r->best_per_ref[static_cast<size_t>(k) * nr + q] = fix(all->best_per_ref[static_cast<size_t>(r0 + k) * nr + q], false);
  }
  if (ni) {
    memcpy(r->item_score, all->item_score + i0, ni * 4);
    memcpy(r->item_end, all->item_end + i0, ni * 4);
  }
  return r;
}

void finish(Server* sv, Round& rd, sr_results* merged) {
  uint32_t r0 = 0;
  uint64_t i0 = 0;
  const auto now = Clock::now();
  std::vector<std::pair<Request*, sr_results*>> outs;
  const uint32_t m32 = i32_min_read_len(sv->sp, sv->opts);
  for (Request* q : rd.reqs) {
    const uint32_t n = q->n_reads;
    const uint64_t ni = q->coff.back();
    uint64_t n32 = 0;
    for (uint32_t r = 0; r < n; ++r)
      if (q->roff[r + 1] - q->roff[r] >= m32) n32 += q->coff[r + 1] - q->coff[r];
    sr_results* part = nullptr;
    if (rd.status == SR_OK && merged) part = slice_results(merged, r0, r0 + n, i0, i0 + ni, q->cells, n32);
    outs.emplace_back(q, part);
    r0 += n;
    i0 += ni;
  }
  std::lock_guard<std::mutex> g(sv->mu);
  for (auto& o : outs) {
    Request* q = o.first;
    q->res = o.second;
    q->status = rd.status != SR_OK ? rd.status : (o.second ? SR_OK : SR_ENOMEM);
    q->t_done = now;
    q->done = true;
    sv->reserved -= q->bytes;
    --sv->inflight;
    sv->lat_us.push_back(std::chrono::duration<double, std::micro>(now - q->t_submit).count());
    sv->lat_reads.push_back(q->n_reads);
    sv->lat_done_s.push_back(std::chrono::duration<double>(now - sv->t_start).count());
  }
  sv->cv_done.notify_all();
  sv->cv_work.notify_all();
}

sr_batch* stage_round(Server* sv, Round& rd, cudaStream_t stream) {
  uint32_t n = 0;
  uint64_t nb = 0, ni = 0;
  for (Request* q : rd.reqs) {
    n += q->n_reads;
    nb += q->roff.back();
    ni += q->coff.back();
  }
  std::vector<char> bases(nb ? nb : 1);
  std::vector<uint64_t> roff(n + 1ull), coff(n + 1ull), cstart(ni ? ni : 1);
  std::vector<uint8_t> cref(ni ? ni : 1), cstr(ni ? ni : 1);
  std::vector<uint32_t> clen(ni ? ni : 1);
  uint32_t r = 0;
  uint64_t ob = 0, oi = 0;
  for (Request* q : rd.reqs) {
    const uint32_t qn = q->n_reads;
    if (q->roff.back()) memcpy(bases.data() + ob, q->bases.data(), q->roff.back());
    for (uint32_t k = 0; k < qn; ++k) {
      roff[r + k] = ob + q->roff[k];
      coff[r + k] = oi + q->coff[k];
    }
    const uint64_t qi = q->coff.back();
    if (qi) {
      memcpy(cstart.data() + oi, q->cstart.data(), qi * 8);
      memcpy(cref.data() + oi, q->cref.data(), qi);
      memcpy(cstr.data() + oi, q->cstr.data(), qi);
      memcpy(clen.data() + oi, q->clen.data(), qi * 4);
    }
    r += qn;
    ob += q->roff.back();
    oi += qi;
  }
  roff[n] = ob;
  coff[n] = oi;
  sr_reads reads{n, 0, bases.data(), roff.data()};
  sr_cand_list cl{};
  cl.n_reads = n;
  cl.n_cands = ni;
  cl.offsets = coff.data();
  cl.ref_id = cref.data();
  cl.strand = cstr.data();
  cl.win_start = cstart.data();
  cl.win_len = clen.data();
  sr_batch* b = nullptr;
  rd.status = batch_stage_internal(sv->s, &reads, &cl, stream, false, &b);
  return rd.status == SR_OK ? b : nullptr;
}

// Admits, stages and launches rounds while fewer than kDepth are in flight.
void scheduler(Server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    Round next;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      auto free_slot = [&] {
        for (int i = 0; i < kDepth; ++i)
          if (!sv->slots[i].busy) return i;
        return -1;
      };
      // on stop, the queued requests are still run before the scheduler exits
      sv->cv_work.wait(lk, [&] {
        return (sv->stop && sv->pending.empty()) || (!sv->pending.empty() && free_slot() >= 0);
      });
      if (sv->pending.empty()) break;
      const uint64_t budget = session_budget(sv->s);
      uint64_t round_reads = 0, round_bytes = 0;
      while (!sv->pending.empty()) {
        Request* q = sv->pending.front();
        if (budget && sv->reserved + q->bytes > budget) {
          ++sv->budget_waits;
          break;
        }
        if (sv->max_inflight && sv->inflight >= sv->max_inflight) break;
        // a round stays at most kMaxRoundReads reads (one request may exceed it alone),
        // so a backlog drains in rounds of bounded latency and device memory
        if (!next.reqs.empty() && round_reads + q->n_reads > kMaxRoundReads) break;
        // and at most half the budget (one larger request runs alone), so that the
        // next round always fits beside a running one: under memory pressure the
        // device still has a round queued instead of idling until one completes
        if (budget && !next.reqs.empty() && round_bytes + q->bytes > budget / 2) break;
        round_reads += q->n_reads;
        round_bytes += q->bytes;
        sv->pending.pop_front();
        sv->reserved += q->bytes;
        ++sv->inflight;
        next.reqs.push_back(q);
      }
      if (next.reqs.empty()) {
        // the front request does not fit: rounds are in flight (an empty device
        // admits any request under the budget), and their completion frees budget
        const uint64_t seen = sv->rounds_done;
        sv->cv_work.wait(lk, [&] { return sv->rounds_done != seen; });
        continue;
      }
      next.slot = free_slot();
      sv->slots[next.slot].busy = true;
    }
    Slot& sl = sv->slots[next.slot];
    next.b = stage_round(sv, next, sl.stream);
    if (next.status == SR_OK) {
      sr_align_opts o = sv->opts;
      o.cuda_stream = sl.stream;
      // the previous round's last kernel (its slot still holds that record)
      cudaEvent_t prev = sv->last_slot >= 0 ? sv->slots[sv->last_slot].last : nullptr;
      next.status = batch_run_serving(sv->s, next.b, &sv->sp, &o, sl.first, prev);
      if (next.status == SR_OK && cudaEventRecord(sl.last, sl.stream) == cudaSuccess) {
        next.timed = true;
        sv->last_slot = next.slot;
      }
    }
    std::lock_guard<std::mutex> g(sv->mu);
    ++sv->rounds;
    sv->max_round = std::max<uint64_t>(sv->max_round, next.reqs.size());
    sv->launched.push_back(std::move(next));
    sv->cv_round.notify_all();
  }
  std::lock_guard<std::mutex> g(sv->mu);
  sv->sched_done = true;
  sv->cv_round.notify_all();
}

// Completes the launched rounds in order: waits for each, copies its results
// back (the records were built on the device), splits them per request.
void completer(Server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    Round rd;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_round.wait(lk, [&] { return !sv->launched.empty() || sv->sched_done; });
      if (sv->launched.empty()) break;  // the scheduler has exited and every round is complete
      rd = std::move(sv->launched.front());
      sv->launched.pop_front();
    }
    sr_results* merged = nullptr;
    if (rd.status == SR_OK) rd.status = sr_batch_fetch(sv->s, rd.b, &merged);
    const Slot& sl = sv->slots[rd.slot];
    float a = 0, z = 0;
    const bool timed = rd.timed && rd.status == SR_OK && cudaEventElapsedTime(&a, sv->t0, sl.first) == cudaSuccess &&
                       cudaEventElapsedTime(&z, sv->t0, sl.last) == cudaSuccess;
    cudaGetLastError();
    if (timed) {
      // before the requests complete, so a caller that has all its results sees this round
      std::lock_guard<std::mutex> g(sv->mu);
      if (sv->timeline.size() < kTimelineCap) sv->timeline.emplace_back(a, z);
    }
    finish(sv, rd, merged);
    sr_results_free(merged);
    sr_batch_free(rd.b);
    std::lock_guard<std::mutex> g(sv->mu);
    sv->slots[rd.slot].busy = false;
    ++sv->rounds_done;
    sv->cv_work.notify_all();
  }
}

}  // namespace

void serve_destroy(Server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->th_sched.joinable()) sv->th_sched.join();
  if (sv->th_done.joinable()) sv->th_done.join();
  for (auto& kv : sv->all) {
    sr_results_free(kv.second->res);
    delete kv.second;
  }
  for (auto& sl : sv->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.first) cudaEventDestroy(sl.first);
    if (sl.last) cudaEventDestroy(sl.last);
  }
  if (sv->t0) cudaEventDestroy(sv->t0);
  delete sv;
}

}  // namespace sr

using namespace sr;

extern "C" sr_status sr_serve_start(sr_session* s, const sr_score_params* sp, const sr_align_opts* opts,
                                    uint32_t max_inflight_requests) {
  if (!s || !sp) return set_error(SR_EINVAL, "sr_serve_start: null argument");
  if (session_server(s)) return set_error(SR_EBUSY, "sr_serve_start: already serving");
  if (opts && opts->engine != SR_ENGINE_BATCHED) return set_error(SR_EINVAL, "sr_serve_start: serving runs the batched engine");
  auto* sv = new Server;
  sv->s = s;
  cudaGetDevice(&sv->device);
  sv->sp = *sp;
  if (opts) {
    sv->opts = *opts;
    sv->opts.cuda_stream = nullptr;
  } else {
    sv->opts.want_cigar = 1;
    sv->opts.min_score = 40;
    sv->opts.margin = 5;
  }
  sv->max_inflight = max_inflight_requests;
  bool ok = cudaEventCreate(&sv->t0) == cudaSuccess;
  for (auto& sl : sv->slots) {
    ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreate(&sl.first) == cudaSuccess && cudaEventCreate(&sl.last) == cudaSuccess;
  }
  // the origin of the round timelines, recorded before any round
  ok = ok && cudaEventRecord(sv->t0, sv->slots[0].stream) == cudaSuccess &&
       cudaEventSynchronize(sv->t0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    serve_destroy(sv);
    return set_error(SR_ECUDA, "sr_serve_start: stream or event creation failed");
  }
  session_server(s) = sv;
  sv->th_sched = std::thread(scheduler, sv);
  sv->th_done = std::thread(completer, sv);
  return SR_OK;
}

extern "C" sr_status sr_serve_stop(sr_session* s) {
  if (!s) return set_error(SR_EINVAL, "sr_serve_stop: null session");
  Server* sv = session_server(s);
  if (!sv) return SR_OK;
  serve_destroy(sv);
  session_server(s) = nullptr;
  return SR_OK;
}

extern "C" sr_status sr_submit(sr_session* s, const sr_reads* reads, const sr_cand_list* cands, uint64_t* ticket) {
  if (!s || !reads || !cands || !ticket) return set_error(SR_EINVAL, "sr_submit: null argument");
  Server* sv = session_server(s);
  if (!sv) return set_error(SR_EINVAL, "sr_submit: call sr_serve_start first");
  const uint32_t n = reads->n_reads;
  if (cands->n_reads != n) return set_error(SR_EINVAL, "sr_submit: reads and candidates differ in n_reads");
  if (reads->flags || cands->flags) return set_error(SR_EINVAL, "sr_submit: requests are copied from host memory (flags 0)");
  if (n && (!reads->offsets || !reads->bases || !cands->offsets)) return set_error(SR_EINVAL, "sr_submit: null arrays");
  auto* q = new Request;
  q->roff.assign(reads->offsets, reads->offsets + n + 1);
  q->coff.assign(cands->offsets, cands->offsets + n + 1);
  q->n_reads = n;
  if (n == 0) {
    q->roff.assign(1, 0);
    q->coff.assign(1, 0);
  }
  if (q->roff[0] != 0 || q->coff[0] != 0 || q->coff.back() != cands->n_cands) {
    delete q;
    return set_error(SR_EINVAL, "sr_submit: bad offsets");
  }
  for (uint32_t r = 0; r < n; ++r)
    if (q->roff[r + 1] < q->roff[r] || q->coff[r + 1] < q->coff[r]) {
      delete q;
      return set_error(SR_EINVAL, "sr_submit: decreasing offsets");
    }
  const uint64_t nb = q->roff.back(), ni = q->coff.back();
  q->bases.assign(reads->bases, reads->bases + nb);
  if (ni) {
    q->cstart.assign(cands->win_start, cands->win_start + ni);
    q->cref.assign(cands->ref_id, cands->ref_id + ni);
    q->cstr.assign(cands->strand, cands->strand + ni);
    q->clen.assign(cands->win_len, cands->win_len + ni);
  }
  for (uint32_t r = 0; r < n; ++r)
    for (uint64_t k = q->coff[r]; k < q->coff[r + 1]; ++k) q->cells += (q->roff[r + 1] - q->roff[r]) * q->clen[k];
  q->bytes = batch_bytes_estimate(n, ni, nb, session_n_refs(s));
  const uint64_t budget = session_budget(s);
  if (budget && q->bytes > budget) {
    delete q;
    return set_error(SR_ENOMEM, "sr_submit: request needs more than the whole HBM budget");
  }
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(sv->mu);
    q->ticket = sv->next_ticket++;
    sv->all[q->ticket] = q;
    sv->pending.push_back(q);
  }
  sv->cv_work.notify_all();
  *ticket = q->ticket;
  return SR_OK;
}

extern "C" sr_status sr_wait(sr_session* s, uint64_t ticket, int32_t timeout_ms, sr_results** out) {
  if (!s || !out) return set_error(SR_EINVAL, "sr_wait: null argument");
  *out = nullptr;
  Server* sv = session_server(s);
  if (!sv) return set_error(SR_EINVAL, "sr_wait: not serving");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return set_error(SR_EINVAL, "sr_wait: unknown ticket");
  Request* q = it->second;
  auto ready = [&] { return q->done; };
  if (timeout_ms < 0) {
    sv->cv_done.wait(lk, ready);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return set_error(SR_ETIMEOUT, "sr_wait: request not finished within %d ms", timeout_ms);
  }
  sv->all.erase(it);
  sr_status st = q->status;
  *out = q->res;
  q->res = nullptr;
  lk.unlock();
  delete q;
  if (st != SR_OK) return set_error(st, "sr_wait: request failed (status %d)", st);
  return SR_OK;
}

namespace {
double percentile(std::vector<double>& v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t k = static_cast<size_t>(p * (v.size() - 1) + 0.5);
  return v[std::min(k, v.size() - 1)];
}
}  // namespace

extern "C" sr_status sr_serve_stats(sr_session* s, double* p50_us, double* p99_us, uint64_t* completed,
                                    uint64_t* rounds, uint64_t* max_round_requests) {
  if (!s) return set_error(SR_EINVAL, "sr_serve_stats: null session");
  Server* sv = session_server(s);
  if (!sv) return set_error(SR_EINVAL, "sr_serve_stats: not serving");
  std::vector<double> v;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    v = sv->lat_us;
    if (rounds) *rounds = sv->rounds;
    if (max_round_requests) *max_round_requests = sv->max_round;
  }
  if (completed) *completed = v.size();
  const double p50 = percentile(v, 0.50), p99 = percentile(v, 0.99);
  if (p50_us) *p50_us = p50;
  if (p99_us) *p99_us = p99;
  return SR_OK;
}

extern "C" sr_status sr_serve_stats_by_size(sr_session* s, uint32_t n_buckets, const uint32_t* max_reads,
                                            double* p50_us, double* p99_us, uint64_t* count) {
  if (!s || (n_buckets && !max_reads)) return set_error(SR_EINVAL, "sr_serve_stats_by_size: null argument");
  for (uint32_t k = 1; k < n_buckets; ++k)
    if (max_reads[k] <= max_reads[k - 1]) return set_error(SR_EINVAL, "sr_serve_stats_by_size: bucket bounds must increase");
  Server* sv = session_server(s);
  if (!sv) return set_error(SR_EINVAL, "sr_serve_stats_by_size: not serving");
  std::vector<double> lat;
  std::vector<uint32_t> sz;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    lat = sv->lat_us;
    sz = sv->lat_reads;
  }
  for (uint32_t k = 0; k < n_buckets; ++k) {
    std::vector<double> v;
    const uint32_t lo = k ? max_reads[k - 1] : 0;
    for (size_t i = 0; i < lat.size(); ++i)
      if ((k == 0 || sz[i] > lo) && sz[i] <= max_reads[k]) v.push_back(lat[i]);
    if (count) count[k] = v.size();
    const double p50 = percentile(v, 0.50), p99 = percentile(v, 0.99);
    if (p50_us) p50_us[k] = p50;
    if (p99_us) p99_us[k] = p99;
  }
  return SR_OK;
}

extern "C" sr_status sr_serve_latencies(sr_session* s, uint64_t first, uint32_t cap, double* us, uint32_t* reads,
                                        double* done_s, uint64_t* n_out) {
  if (!s || (cap && (!us || !reads || !done_s)) || !n_out) return set_error(SR_EINVAL, "sr_serve_latencies: null argument");
  Server* sv = session_server(s);
  if (!sv) return set_error(SR_EINVAL, "sr_serve_latencies: not serving");
  std::lock_guard<std::mutex> g(sv->mu);
  const uint64_t n = sv->lat_us.size();
  uint64_t k = 0;
  for (uint64_t i = first; i < n && k < cap; ++i, ++k) {
    us[k] = sv->lat_us[i];
    reads[k] = sv->lat_reads[i];
    done_s[k] = sv->lat_done_s[i];
  }
  *n_out = n;
  return SR_OK;
}

extern "C" sr_status sr_serve_overlap(sr_session* s, uint64_t* timed_rounds, uint64_t* overlapped,
                                      double* device_idle_ms, uint64_t* budget_waits, uint32_t cap,
                                      float* first_ms, float* last_ms) {
  if (!s || (cap && (!first_ms || !last_ms))) return set_error(SR_EINVAL, "sr_serve_overlap: null argument");
  Server* sv = session_server(s);
  if (!sv) return set_error(SR_EINVAL, "sr_serve_overlap: not serving");
  std::vector<std::pair<float, float>> t;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    t = sv->timeline;
    if (budget_waits) *budget_waits = sv->budget_waits;
  }
  uint64_t ov = 0;
  double idle = 0;
  for (size_t k = 1; k < t.size(); ++k) {
    if (t[k].first < t[k - 1].second) ++ov;
    else idle += t[k].first - t[k - 1].second;
  }
  if (timed_rounds) *timed_rounds = t.size();
  if (overlapped) *overlapped = ov;
  if (device_idle_ms) *device_idle_ms = idle;
  const size_t n = std::min<size_t>(cap, t.size());
  for (size_t k = 0; k < n; ++k) {
    first_ms[k] = t[k].first;
    last_ms[k] = t[k].second;
  }
  return SR_OK;
}
