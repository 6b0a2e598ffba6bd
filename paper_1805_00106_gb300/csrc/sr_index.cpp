// sr_index.cpp -- host stage: k-mer index (pointer table + CAL table) and the
// CAL finder / filter of McVicar et al., arXiv 1805.00106, Sec. 3.1-3.3 and
// 4.1-4.2.  Its output (candidate windows) feeds the device path.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sr_host.h"
#include "sr_seed.h"

struct sr_index {
  sr_index_params p{};
  std::vector<uint8_t> codes;  // 2-bit codes of the reference, one per byte
  std::vector<uint64_t> ptr;   // 4^address_bases + 1 bucket starts
  std::vector<uint32_t> key;   // CAL table: key bits of the hashed canonical seed
  std::vector<uint32_t> pos;   // CAL table: reference position
  std::vector<uint8_t> orient; // bit0: k-mer is the canonical form; bit1: its revcomp is
};

namespace sr {

int encode_ascii(const char* s, uint64_t n, uint8_t* out) {
  for (uint64_t i = 0; i < n; ++i) {
    const unsigned c = static_cast<unsigned char>(s[i]) | 0x20u;
    switch (c) {
      case 'a': out[i] = 0; break;
      case 'c': out[i] = 1; break;
      case 'g': out[i] = 2; break;
      case 't': out[i] = 3; break;
      default: return -1;
    }
  }
  return 0;
}

namespace {

int n_threads_of(uint32_t req) {
  unsigned hc = std::thread::hardware_concurrency();
  int n = req ? static_cast<int>(req) : static_cast<int>(hc ? hc : 1);
  return n < 1 ? 1 : (n > 256 ? 256 : n);
}

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" sr_status sr_index_build(const char* seq, uint64_t len, const sr_index_params* params,
                                    sr_index** out) {
  Trace trace_("sr_index_build");
  if (!seq || !out) return set_error(SR_EINVAL, "sr_index_build: null argument");
  *out = nullptr;
  sr_index_params p{};
  if (params) p = *params;
  if (!p.seed_len) p.seed_len = 20;
  if (!p.address_bases) p.address_bases = 12;
  const int k = static_cast<int>(p.seed_len), a = static_cast<int>(p.address_bases);
  if (k < 4 || k > 32 || a < 1 || a > 14 || a > k || 2 * (k - a) > 32)
    return set_error(SR_EINVAL, "sr_index_build: seed_len in [4,32], address_bases in [1,min(k,14)], 2*(k-a) <= 32");
  if (len >= (1ull << 32)) return set_error(SR_EINVAL, "sr_index_build: reference longer than 2^32");
  auto* idx = new (std::nothrow) sr_index;
  if (!idx) return set_error(SR_ENOMEM, "sr_index_build: out of host memory");
  idx->p = p;
  try {
    idx->codes.resize(len);
    if (encode_ascii(seq, len, idx->codes.data()) != 0) {
      delete idx;
      return set_error(SR_EBADBASE, "sr_index_build: reference has a non-ACGT base");
    }
    const uint64_t nb = 1ull << (2 * a);
    const int kb = 2 * (k - a);
    const uint64_t kmask = mask_bits(kb);
    const uint64_t npos = len >= static_cast<uint64_t>(k) ? len - k + 1 : 0;
    // pass 1: hashed canonical seed of every position
    std::vector<uint64_t> hv(npos);
    std::vector<uint8_t> ori(npos);
    {
      Kmer km;
      for (uint64_t i = 0; i < len; ++i) {
        kmer_push(km, idx->codes[i], k);
        if (i + 1 >= static_cast<uint64_t>(k)) {
          const uint64_t p0 = i + 1 - k;
          const uint64_t canon = std::min(km.fwd, km.rc);
          hv[p0] = seed_hash(canon, k, p.hash_seed);
          ori[p0] = static_cast<uint8_t>((km.fwd == canon ? 1 : 0) | (km.rc == canon ? 2 : 0));
        }
      }
    }
    // pass 2: counting sort by address
    std::vector<uint64_t> cnt(nb + 1, 0);
    for (uint64_t q = 0; q < npos; ++q) ++cnt[(hv[q] >> kb) + 1];
    for (uint64_t b = 0; b < nb; ++b) cnt[b + 1] += cnt[b];
    std::vector<uint64_t> cur(cnt.begin(), cnt.end() - 1);
    std::vector<uint32_t> sorted(npos);
    for (uint64_t q = 0; q < npos; ++q) sorted[cur[hv[q] >> kb]++] = static_cast<uint32_t>(q);
    // pass 3: per bucket order by (key, pos), drop keys above cal_limit
    idx->ptr.assign(nb + 1, 0);
    idx->key.reserve(npos);
    idx->pos.reserve(npos);
    idx->orient.reserve(npos);
    std::vector<std::pair<uint64_t, uint32_t>> tmp;
    for (uint64_t b = 0; b < nb; ++b) {
      idx->ptr[b] = idx->key.size();
      const uint64_t s0 = cnt[b], s1 = cnt[b + 1];
      if (s1 == s0) continue;
      tmp.clear();
      for (uint64_t t = s0; t < s1; ++t) tmp.emplace_back(hv[sorted[t]] & kmask, sorted[t]);
      std::sort(tmp.begin(), tmp.end());
      for (size_t t = 0; t < tmp.size();) {
        size_t u = t;
        while (u < tmp.size() && tmp[u].first == tmp[t].first) ++u;
        if (p.cal_limit == 0 || u - t <= p.cal_limit) {
          for (size_t v = t; v < u; ++v) {
            idx->key.push_back(static_cast<uint32_t>(tmp[v].first));
            idx->pos.push_back(tmp[v].second);
            idx->orient.push_back(ori[tmp[v].second]);
          }
        }
        t = u;
      }
    }
    idx->ptr[nb] = idx->key.size();
  } catch (const std::bad_alloc&) {
    delete idx;
    return set_error(SR_ENOMEM, "sr_index_build: out of host memory");
  }
  *out = idx;
  return SR_OK;
}

void sr_index_free(sr_index* idx) { delete idx; }

extern "C" sr_status sr_index_info(const sr_index* idx, uint64_t* ref_len, uint64_t* n_entries) {
  if (!idx) return set_error(SR_EINVAL, "sr_index_info: null index");
  if (ref_len) *ref_len = idx->codes.size();
  if (n_entries) *n_entries = idx->key.size();
  return SR_OK;
}

namespace sr {
const uint8_t* index_codes(const sr_index* idx, uint64_t* len) {
  *len = idx->codes.size();
  return idx->codes.data();
}

IndexTables index_tables(const sr_index* idx) {
  IndexTables t;
  t.seed_len = idx->p.seed_len;
  t.address_bases = idx->p.address_bases;
  t.hash_seed = idx->p.hash_seed;
  t.ref_len = idx->codes.size();
  t.ptr = idx->ptr.data();
  t.n_ptr = idx->ptr.size();
  t.key = idx->key.data();
  t.pos = idx->pos.data();
  t.orient = idx->orient.data();
  t.n_entries = idx->key.size();
  return t;
}
}  // namespace sr

// ---- save / load: header, arrays, FNV-1a checksum of everything before it
namespace {
constexpr char kMagic[8] = {'S', 'R', 'I', 'D', 'X', '0', '0', '1'};

struct Fnv {
  uint64_t h = 0xcbf29ce484222325ull;
  void add(const void* p, size_t n) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 0x100000001b3ull;
    }
  }
};

template <class T>
bool write_vec(FILE* f, Fnv& fnv, const std::vector<T>& v) {
  const uint64_t n = v.size();
  fnv.add(&n, 8);
  if (fwrite(&n, 8, 1, f) != 1) return false;
  if (n) {
    fnv.add(v.data(), n * sizeof(T));
    if (fwrite(v.data(), sizeof(T), n, f) != n) return false;
  }
  return true;
}

template <class T>
bool read_vec(FILE* f, Fnv& fnv, std::vector<T>& v, uint64_t max_n) {
  uint64_t n = 0;
  if (fread(&n, 8, 1, f) != 1 || n > max_n) return false;
  fnv.add(&n, 8);
  v.resize(n);
  if (n) {
    if (fread(v.data(), sizeof(T), n, f) != n) return false;
    fnv.add(v.data(), n * sizeof(T));
  }
  return true;
}
}  // namespace

extern "C" sr_status sr_index_save(const sr_index* idx, const char* path) {
  if (!idx || !path) return set_error(SR_EINVAL, "sr_index_save: null argument");
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(SR_EIO, "sr_index_save: cannot open file");
  Fnv fnv;
  bool ok = fwrite(kMagic, 8, 1, f) == 1;
  fnv.add(kMagic, 8);
  ok = ok && fwrite(&idx->p, sizeof(idx->p), 1, f) == 1;
  fnv.add(&idx->p, sizeof(idx->p));
  ok = ok && write_vec(f, fnv, idx->codes) && write_vec(f, fnv, idx->ptr) &&
       write_vec(f, fnv, idx->key) && write_vec(f, fnv, idx->pos) && write_vec(f, fnv, idx->orient);
  ok = ok && fwrite(&fnv.h, 8, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  return ok ? SR_OK : set_error(SR_EIO, "sr_index_save: write failed");
}

extern "C" sr_status sr_index_load(const char* path, sr_index** out) {
  if (!path || !out) return set_error(SR_EINVAL, "sr_index_load: null argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(SR_EIO, "sr_index_load: cannot open file");
  auto* idx = new (std::nothrow) sr_index;
  if (!idx) {
    fclose(f);
    return set_error(SR_ENOMEM, "sr_index_load: out of memory");
  }
  Fnv fnv;
  char mg[8];
  bool ok = fread(mg, 8, 1, f) == 1 && memcmp(mg, kMagic, 8) == 0;
  fnv.add(kMagic, 8);
  ok = ok && fread(&idx->p, sizeof(idx->p), 1, f) == 1;
  if (ok) fnv.add(&idx->p, sizeof(idx->p));
  const uint64_t lim = 1ull << 34;
  try {
    ok = ok && read_vec(f, fnv, idx->codes, lim) && read_vec(f, fnv, idx->ptr, lim) &&
         read_vec(f, fnv, idx->key, lim) && read_vec(f, fnv, idx->pos, lim) &&
         read_vec(f, fnv, idx->orient, lim);
  } catch (const std::bad_alloc&) {
    ok = false;
  }
  uint64_t chk = 0;
  ok = ok && fread(&chk, 8, 1, f) == 1 && chk == fnv.h;
  const int k = static_cast<int>(idx->p.seed_len), a = static_cast<int>(idx->p.address_bases);
  ok = ok && k >= 4 && k <= 32 && a >= 1 && a <= 14 && idx->ptr.size() == (1ull << (2 * a)) + 1 &&
       idx->key.size() == idx->pos.size() && idx->pos.size() == idx->orient.size() &&
       idx->ptr.back() == idx->key.size();
  fclose(f);
  if (!ok) {
    delete idx;
    return set_error(SR_EIO, "sr_index_load: bad or corrupt index file");
  }
  *out = idx;
  return SR_OK;
}

// ---- CAL finder + filter
namespace {
struct Cal {
  uint32_t ref, strand;
  int64_t cal;
};

struct Win {
  uint32_t ref, strand;
  int64_t cal;
  uint32_t hits;
  uint64_t start;
  uint32_t len;
};

void find_read(const sr_index* const* idx, uint32_t n_refs, const uint8_t* q, int m,
               const sr_cand_params& cp, std::vector<Cal>& cals, std::vector<Win>& out) {
  cals.clear();
  out.clear();
  const int k = static_cast<int>(idx[0]->p.seed_len);
  if (m < k) return;
  const int a = static_cast<int>(idx[0]->p.address_bases);
  const int kb = 2 * (k - a);
  const uint64_t kmask = mask_bits(kb);
  const int stride = static_cast<int>(cp.seed_stride ? cp.seed_stride : 1);
  for (int o = 0; o + k <= m; o += stride) {
    Kmer km;
    for (int t = 0; t < k; ++t) kmer_push(km, q[o + t], k);
    const uint64_t canon = std::min(km.fwd, km.rc);
    const uint32_t rori = (km.fwd == canon ? 1u : 0u) | (km.rc == canon ? 2u : 0u);
    for (uint32_t r = 0; r < n_refs; ++r) {
      const sr_index* ix = idx[r];
      const uint64_t h = seed_hash(canon, k, ix->p.hash_seed);
      const uint64_t b = h >> kb;
      const uint32_t key = static_cast<uint32_t>(h & kmask);
      const uint64_t s0 = ix->ptr[b], s1 = ix->ptr[b + 1];
      // keys are sorted within a bucket
      const uint32_t* kb0 = ix->key.data() + s0;
      const uint32_t* kb1 = ix->key.data() + s1;
      const uint32_t* lo = std::lower_bound(kb0, kb1, key);
      for (const uint32_t* e = lo; e < kb1 && *e == key; ++e) {
        const uint64_t t = static_cast<uint64_t>(e - ix->key.data());
        const uint32_t fo = ix->orient[t];
        const int64_t p = ix->pos[t];
        const bool plus = ((fo & 1u) && (rori & 1u)) || ((fo & 2u) && (rori & 2u));
        const bool minus = ((fo & 1u) && (rori & 2u)) || ((fo & 2u) && (rori & 1u));
        if (plus) cals.push_back({r, 0u, p - o});
        if (minus) cals.push_back({r, 1u, p - (m - o - k)});
      }
    }
  }
  std::sort(cals.begin(), cals.end(), [](const Cal& x, const Cal& y) {
    if (x.ref != y.ref) return x.ref < y.ref;
    if (x.strand != y.strand) return x.strand < y.strand;
    return x.cal < y.cal;
  });
  for (size_t t = 0; t < cals.size();) {
    size_t u = t + 1;
    while (u < cals.size() && cals[u].ref == cals[t].ref && cals[u].strand == cals[t].strand &&
           cals[u].cal - cals[u - 1].cal <= static_cast<int64_t>(cp.merge_dist))
      ++u;
    Win w{cals[t].ref, cals[t].strand, cals[t].cal, static_cast<uint32_t>(u - t), 0, 0};
    uint32_t best = 0;
    for (size_t v = t; v < u;) {
      size_t x = v;
      while (x < u && cals[x].cal == cals[v].cal) ++x;
      if (x - v > best) {
        best = static_cast<uint32_t>(x - v);
        w.cal = cals[v].cal;
      }
      v = x;
    }
    out.push_back(w);
    t = u;
  }
  if (cp.max_cands && out.size() > cp.max_cands) {
    std::sort(out.begin(), out.end(), [](const Win& x, const Win& y) {
      if (x.hits != y.hits) return x.hits > y.hits;
      if (x.ref != y.ref) return x.ref < y.ref;
      if (x.strand != y.strand) return x.strand < y.strand;
      return x.cal < y.cal;
    });
    out.resize(cp.max_cands);
    std::sort(out.begin(), out.end(), [](const Win& x, const Win& y) {
      if (x.ref != y.ref) return x.ref < y.ref;
      if (x.strand != y.strand) return x.strand < y.strand;
      return x.cal < y.cal;
    });
  }
  for (auto& w : out) {
    const int64_t N = static_cast<int64_t>(idx[w.ref]->codes.size());
    int64_t lo = w.cal - static_cast<int64_t>(cp.pad), hi = w.cal + m + static_cast<int64_t>(cp.pad);
    if (lo < 0) lo = 0;
    if (hi > N) hi = N;
    w.start = static_cast<uint64_t>(lo);
    w.len = static_cast<uint32_t>(hi - lo);
  }
}
}  // namespace

extern "C" sr_status sr_cand_list_alloc(uint32_t n_reads, uint64_t n_cands, sr_cand_list** out) {
  if (!out) return set_error(SR_EINVAL, "sr_cand_list_alloc: null out");
  auto* l = static_cast<sr_cand_list*>(calloc(1, sizeof(sr_cand_list)));
  if (!l) return set_error(SR_ENOMEM, "sr_cand_list_alloc: out of memory");
  l->n_reads = n_reads;
  l->n_cands = n_cands;
  l->offsets = static_cast<uint64_t*>(calloc(static_cast<size_t>(n_reads) + 1, 8));
  const size_t nc = n_cands ? n_cands : 1;
  l->ref_id = static_cast<uint8_t*>(malloc(nc));
  l->strand = static_cast<uint8_t*>(malloc(nc));
  l->win_start = static_cast<uint64_t*>(malloc(nc * 8));
  l->win_len = static_cast<uint32_t*>(malloc(nc * 4));
  l->hits = static_cast<uint32_t*>(malloc(nc * 4));
  if (!l->offsets || !l->ref_id || !l->strand || !l->win_start || !l->win_len || !l->hits) {
    sr_cand_list_free(l);
    return set_error(SR_ENOMEM, "sr_cand_list_alloc: out of memory");
  }
  *out = l;
  return SR_OK;
}

extern "C" void sr_cand_list_free(sr_cand_list* l) {
  if (!l) return;
  if (l->flags & SR_FLAG_DEVICE) {
    // a list sr_candidates_device left on the device
    void* arrays[6] = {l->offsets, l->ref_id, l->strand, l->win_start, l->win_len, l->hits};
    for (void* p : arrays)
      if (p) cudaFree(p);
    free(l);
    return;
  }
  free(l->offsets);
  free(l->ref_id);
  free(l->strand);
  free(l->win_start);
  free(l->win_len);
  free(l->hits);
  free(l);
}

extern "C" sr_status sr_candidates(const sr_index* const* idx, uint32_t n_refs, const sr_reads* reads,
                                   const sr_cand_params* params, sr_cand_list** out) {
  Trace trace_("sr_candidates");
  if (!idx || !reads || !out || n_refs == 0 || n_refs > SR_MAX_REFS)
    return set_error(SR_EINVAL, "sr_candidates: bad arguments");
  *out = nullptr;
  if (reads->flags) return set_error(SR_EINVAL, "sr_candidates: reads must be in host memory (flags 0)");
  for (uint32_t r = 0; r < n_refs; ++r) {
    if (!idx[r]) return set_error(SR_EINVAL, "sr_candidates: null index");
    if (idx[r]->p.seed_len != idx[0]->p.seed_len || idx[r]->p.address_bases != idx[0]->p.address_bases)
      return set_error(SR_EINVAL, "sr_candidates: indexes differ in seed layout");
  }
  sr_cand_params cp{};
  if (params) cp = *params;
  if (!cp.seed_stride) cp.seed_stride = 1;
  const uint32_t n = reads->n_reads;
  if (n && (!reads->bases || !reads->offsets)) return set_error(SR_EINVAL, "sr_candidates: null reads");
  const int nt = std::min<int>(n_threads_of(cp.n_threads), static_cast<int>(n ? n : 1));
  std::vector<std::vector<Win>> per_read(n);
  std::atomic<int> bad{0};
  std::atomic<uint32_t> next{0};
  auto work = [&]() {
    std::vector<Cal> cals;
    std::vector<uint8_t> q;
    for (;;) {
      const uint32_t r0 = next.fetch_add(256);
      if (r0 >= n) break;
      const uint32_t r1 = std::min<uint32_t>(n, r0 + 256);
      for (uint32_t r = r0; r < r1; ++r) {
        const uint64_t o0 = reads->offsets[r], o1 = reads->offsets[r + 1];
        if (o1 < o0) {
          bad = 2;
          continue;
        }
        const int m = static_cast<int>(o1 - o0);
        q.resize(static_cast<size_t>(m));
        if (encode_ascii(reads->bases + o0, static_cast<uint64_t>(m), q.data()) != 0) {
          bad = 1;
          continue;
        }
        find_read(idx, n_refs, q.data(), m, cp, cals, per_read[r]);
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  if (bad == 1) return set_error(SR_EBADBASE, "sr_candidates: read has a non-ACGT base");
  if (bad == 2) return set_error(SR_EINVAL, "sr_candidates: decreasing read offsets");
  uint64_t total = 0;
  for (auto& v : per_read) total += v.size();
  sr_cand_list* l = nullptr;
  sr_status st = sr_cand_list_alloc(n, total, &l);
  if (st != SR_OK) return st;
  uint64_t o = 0;
  for (uint32_t r = 0; r < n; ++r) {
    l->offsets[r] = o;
    for (const Win& w : per_read[r]) {
      l->ref_id[o] = static_cast<uint8_t>(w.ref);
      l->strand[o] = static_cast<uint8_t>(w.strand);
      l->win_start[o] = w.start;
      l->win_len[o] = w.len;
      l->hits[o] = w.hits;
      ++o;
    }
  }
  l->offsets[n] = o;
  *out = l;
  return SR_OK;
}
