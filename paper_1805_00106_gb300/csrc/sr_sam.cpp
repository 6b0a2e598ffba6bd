// sr_sam.cpp -- SAM text output of a batch's results (the paper's V2 formats its
// results "into a standard format like SAM", Sec. 4.2).  Host code: formatting
// runs in parallel chunks of reads, written in read order.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "sr_host.h"

using namespace sr;

namespace {

const char kOps[] = "MIDNSHP=X";

void append_int(std::string& s, long long v) {
  char buf[32];
  const int n = std::snprintf(buf, sizeof(buf), "%lld", v);
  s.append(buf, static_cast<size_t>(n));
}

char comp(char c) {
  switch (c | 0x20) {
    case 'a': return 'T';
    case 'c': return 'G';
    case 'g': return 'C';
    case 't': return 'A';
    default: return 'N';
  }
}

// mapping quality from the winner's margin over the second best (a reading:
// the paper reports none): 0 when the best score is tied at another place,
// else 60 * (best - second) / best, capped at 60
int mapq(const sr_hit& h) {
  if (h.score <= 0 || h.n_ties > 1) return 0;
  const long long q = 60LL * (h.score - std::max(h.second, 0)) / h.score;
  return static_cast<int>(std::min<long long>(60, std::max<long long>(0, q)));
}

void format_read(const sr_reads* reads, const sr_results* res, const sr_sam_opts* o,
                 uint32_t r, std::string& out) {
  const uint64_t o0 = reads->offsets[r], o1 = reads->offsets[r + 1];
  const char* seq = reads->bases + o0;
  const uint64_t m = o1 - o0;
  const sr_hit& h = res->best[r];
  if (o && o->read_names && o->read_names[r]) out += o->read_names[r];
  else {
    out += 'r';
    append_int(out, r);
  }
  const bool mapped = h.item >= 0 && h.score > 0;
  const bool rev = mapped && h.strand;
  out += '\t';
  append_int(out, mapped ? (rev ? 16 : 0) : 4);
  out += '\t';
  if (mapped) {
    if (o && o->ref_names && o->ref_names[h.ref_id]) out += o->ref_names[h.ref_id];
    else {
      out += "ref";
      append_int(out, h.ref_id);
    }
  } else {
    out += '*';
  }
  out += '\t';
  append_int(out, mapped ? static_cast<long long>(h.ref_start) + 1 : 0);
  out += '\t';
  append_int(out, mapped ? mapq(h) : 0);
  out += '\t';
  if (mapped && res->cigar && h.cigar_len) {
    for (uint32_t t = 0; t < h.cigar_len; ++t) {
      const uint32_t w = res->cigar[h.cigar_off + t];
      append_int(out, w >> 4);
      out += kOps[(w & 15u) < 9 ? (w & 15u) : 0];
    }
  } else {
    out += '*';
  }
  out += "\t*\t0\t0\t";
  if (rev) {
    for (uint64_t t = m; t-- > 0;) out += comp(seq[t]);
  } else {
    for (uint64_t t = 0; t < m; ++t) out += static_cast<char>(seq[t] & ~0x20);
  }
  out += "\t*";
  if (mapped) {
    out += "\tAS:i:";
    append_int(out, h.score);
    out += "\tXS:i:";
    append_int(out, h.second);
    out += "\tX0:i:";
    append_int(out, h.n_ties);
  }
  if (res->read_class) {
    static const char* cls[] = {"UN", "A", "B", "AMB"};
    out += "\tYC:Z:";
    out += cls[res->read_class[r] & 3u];
  }
  // secondary hits of a report: XA:Z:ref,+end,score;... (end 1-based, sign = strand)
  if (o && o->secondary && r < o->secondary->n_reads) {
    const sr_report* rep = o->secondary;
    bool first = true;
    for (uint64_t t = rep->offsets[r]; t < rep->offsets[r + 1]; ++t) {
      const sr_report_hit& x = rep->hits[t];
      if (x.item == h.item) continue;
      out += first ? "\tXA:Z:" : "";
      first = false;
      if (o->ref_names && o->ref_names[x.ref_id]) out += o->ref_names[x.ref_id];
      else {
        out += "ref";
        append_int(out, x.ref_id);
      }
      out += ',';
      out += x.strand ? '-' : '+';
      append_int(out, static_cast<long long>(x.ref_end) + 1);
      out += ',';
      append_int(out, x.score);
      out += ';';
    }
  }
  out += '\n';
}

}  // namespace

extern "C" sr_status sr_write_sam(const sr_reads* reads, const sr_results* res, const uint64_t* ref_lens,
                                  const sr_sam_opts* opts, const char* path) {
  Trace trace_("sr_write_sam");
  if (!reads || !res || !path || (res->n_refs && !ref_lens))
    return set_error(SR_EINVAL, "sr_write_sam: null argument");
  if (reads->n_reads != res->n_reads) return set_error(SR_EINVAL, "sr_write_sam: reads and results differ");
  if (reads->flags) return set_error(SR_EINVAL, "sr_write_sam: reads must be in host memory (flags 0)");
  const uint32_t n = res->n_reads;
  if (n && (!reads->bases || !reads->offsets || !res->best)) return set_error(SR_EINVAL, "sr_write_sam: null arrays");
  for (uint32_t r = 0; r < n; ++r) {
    const sr_hit& h = res->best[r];
    if (h.item >= 0 && h.score > 0) {
      if (h.ref_id >= res->n_refs) return set_error(SR_EINVAL, "sr_write_sam: read %u has a bad reference id", r);
      if (res->cigar && static_cast<uint64_t>(h.cigar_off) + h.cigar_len > res->n_cigar)
        return set_error(SR_EINVAL, "sr_write_sam: read %u has a CIGAR outside the results", r);
    }
  }
  if (opts && opts->secondary && opts->secondary->n_reads != n)
    return set_error(SR_EINVAL, "sr_write_sam: the report is of another batch");
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_error(SR_EIO, "sr_write_sam: cannot open %s", path);
  std::string head = "@HD\tVN:1.6\tSO:unsorted\n";
  for (uint32_t q = 0; q < res->n_refs; ++q) {
    head += "@SQ\tSN:";
    if (opts && opts->ref_names && opts->ref_names[q]) head += opts->ref_names[q];
    else {
      head += "ref";
      append_int(head, q);
    }
    head += "\tLN:";
    append_int(head, static_cast<long long>(ref_lens[q]));
    head += '\n';
  }
  head += "@PG\tID:libsr\tPN:libsr\tVN:0.1\n";
  bool ok = std::fwrite(head.data(), 1, head.size(), f) == head.size();
  const uint32_t nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  const uint32_t chunk = 65536;
  std::vector<std::string> bufs(nt);
  for (uint32_t c0 = 0; c0 < n && ok; c0 += chunk * nt) {
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < nt; ++t) {
      th.emplace_back([&, t]() {
        std::string& s = bufs[t];
        s.clear();
        const uint32_t a = c0 + t * chunk, b = std::min<uint32_t>(n, a + chunk);
        for (uint32_t r = a; r < b; ++r) format_read(reads, res, opts, r, s);
      });
    }
    for (auto& x : th) x.join();
    for (uint32_t t = 0; t < nt && ok; ++t) ok = std::fwrite(bufs[t].data(), 1, bufs[t].size(), f) == bufs[t].size();
  }
  if (std::fclose(f) != 0) ok = false;
  return ok ? SR_OK : set_error(SR_EIO, "sr_write_sam: write to %s failed", path);
}
