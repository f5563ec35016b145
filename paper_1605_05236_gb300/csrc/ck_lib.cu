// ck_lib.cu -- host side of libck.so: the C ABI declared in include/ck.h.
// Table memory layout, parameter checks, kernel dispatch and counters.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "ck.h"
#include "ck_launch.cuh"

using namespace ck;

struct ck_table {
  DevTable dt;
  void* buf;
  size_t bytes;
  bool owns;
  int device;
  int sm_count;
  cudaStream_t last;
  uint64_t load_base;    // keys submitted for insertion minus keys submitted for deletion
  uint32_t overlap;      // insert launches may overlap their predecessor
  uint32_t block;
  uint32_t policy_code;  // as passed by the caller (policy | ghost flag)
  uint64_t max_inflight; // insertions in flight per insert launch at most (0: as many as fit)
  uint32_t search_warp;  // BFS searches run by a whole warp (ck_warp.cuh) ...
  uint32_t search_warp_load;  // ... in launches that start at a load of at least this / 1000
};

namespace {

constexpr size_t ALIGN = 256;
constexpr uint32_t SEARCHERS_MAX = 160 * 1024;  // concurrent searches a table provisions scratch for

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

bool shape_ok(uint64_t bins, uint32_t B, uint32_t d, uint32_t policy) {
  uint32_t pol = policy & 0xFF;
  bool ghost = (policy & CK_GHOST) != 0;
  if ((policy & ~0x1FFu) != 0) return false;
  if (bins < 2 || bins >= (1ull << 32)) return false;
  if (d == 2) {
    if (B != 4 && B != 8) return false;
    if (pol > CK_QUEUE && pol != CK_HYBRID) return false;
  } else if (d == 3 || d == 4) {
    if (B != 1 || ghost) return false;
    if (pol == CK_QUEUE || pol > CK_HYBRID) return false;  // d-ary: random/rattle kicking, the searches
  } else {
    return false;
  }
  if (bins < d) return false;
  return true;
}

bool is_search(uint32_t policy) {
  uint32_t pol = policy & 0xFF;
  return pol == CK_BFS || pol == CK_SORTED || pol == CK_HYBRID;
}

uint32_t searchers_for(uint64_t bins) {
  uint64_t s = bins < 1024 ? 1024 : bins;
  if (s > SEARCHERS_MAX) s = SEARCHERS_MAX;
  return (uint32_t)((s + 255) / 256 * 256);
}

// scratch plans for chains longer than a thread's local plan (and for the
// serial replay): a few per table, more for large tables.  d-ary random
// kicking walks past the local plan often near its load limits (chains of
// ~1,500-2,300 at 0.90 / 0.96), so it gets up to 4096 plans, enough for the
// long walks a full GPU has in flight at once.
uint32_t long_plans_for(uint64_t bins, uint32_t B, uint32_t policy) {
  const uint64_t most = (B == 1 && (policy & 0xFF) == CK_RANDOM) ? 4096 : 1024;
  uint64_t k = bins / 4096;
  if (k < 8) k = 8;
  if (k > most) k = most;
  return (uint32_t)k;
}

struct Layout {
  size_t slots, meta, counters, busy, slab_busy, long_plans, scratch, total;
};

Layout layout(uint64_t bins, uint32_t B, uint32_t policy) {
  Layout L;
  L.slots = 0;
  size_t off = align_up(bins * B * sizeof(uint64_t));
  L.meta = off;
  off = align_up(off + bins * sizeof(uint32_t));
  L.counters = off;
  off = align_up(off + COUNTER_WORDS * sizeof(uint64_t));
  L.busy = off;
  off = align_up(off + long_plans_for(bins, B, policy) * sizeof(uint32_t));
  L.slab_busy = off;
  if (is_search(policy)) off = align_up(off + (searchers_for(bins) / SLAB) * sizeof(uint32_t));
  L.long_plans = off;
  off = align_up(off + (size_t)long_plans_for(bins, B, policy) * LONG_REGION);
  L.scratch = off;
  if (is_search(policy)) off = align_up(off + (size_t)searchers_for(bins) * SEARCH_REGION);
  L.total = off;
  return L;
}

int check(cudaError_t e) { return e == cudaSuccess ? CK_OK : CK_ECUDA; }

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int clear_on(ck_table* t, cudaStream_t s) {
  Layout L = layout(t->dt.n_bins, t->dt.B, t->policy_code);
  uint8_t* base = static_cast<uint8_t*>(t->buf);
  if (cudaMemsetAsync(base + L.slots, 0xFF, t->dt.n_bins * t->dt.B * sizeof(uint64_t), s) != cudaSuccess)
    return CK_ECUDA;
  if (cudaMemsetAsync(base + L.meta, 0, t->dt.n_bins * sizeof(uint32_t), s) != cudaSuccess) return CK_ECUDA;
  if (cudaMemsetAsync(base + L.counters, 0, L.long_plans - L.counters, s) != cudaSuccess) return CK_ECUDA;
  t->last = s;
  t->load_base = 0;
  return CK_OK;
}

int init_table(ck_table* t, void* buf, size_t bytes, bool owns, uint64_t bins, uint32_t B, uint32_t d,
               uint32_t policy, uint64_t seed) {
  Layout L = layout(bins, B, policy);
  uint8_t* base = static_cast<uint8_t*>(buf);
  DevTable& dt = t->dt;
  std::memset(&dt, 0, sizeof(dt));
  dt.slots = reinterpret_cast<uint64_t*>(base + L.slots);
  dt.meta = reinterpret_cast<uint32_t*>(base + L.meta);
  dt.counters = reinterpret_cast<unsigned long long*>(base + L.counters);
  dt.scratch = is_search(policy) ? base + L.scratch : nullptr;
  dt.long_scratch = base + L.long_plans;
  dt.long_busy = reinterpret_cast<uint32_t*>(base + L.busy);
  dt.slab_busy = is_search(policy) ? reinterpret_cast<uint32_t*>(base + L.slab_busy) : nullptr;
  dt.n_long = long_plans_for(bins, B, policy);
  dt.n_bins = bins;
  dt.total_slots = bins * B;
  dt.rng_seed = seed;
  dt.bin_mask = (bins & (bins - 1)) == 0 ? (uint32_t)(bins - 1) : 0u;
  dt.B = B;
  dt.d = d;
  dt.policy = policy & 0xFF;
  dt.ghost = (policy & CK_GHOST) ? 1 : 0;
  dt.cap = 500;
  dt.max_retries = 1024;
  dt.ordered_writes = 0;  // see CK_PARAM_ORDERED_WRITES
  dt.spawn_k = 1;
  dt.tie_resident = 0;
  dt.n_searchers = is_search(policy) ? searchers_for(bins) : 0;
  dt.seeds[0] = 0x9E3779B9u;
  dt.seeds[1] = 0x85EBCA6Bu;
  dt.seeds[2] = 0xC2B2AE35u;
  dt.seeds[3] = 0x27D4EB2Fu;
  t->buf = buf;
  t->bytes = bytes;
  t->owns = owns;
  t->last = nullptr;
  // measured on one GB300 (fill of 2^24 x 4 or 2^23 x 8 to 0.95-0.99): 4-slot
  // queue-kicking tables fill 3-5% faster with 256-thread blocks, 8-slot
  // tables and random kicking with 128
  t->block = (B == 4 && (policy & 0xFF) == CK_QUEUE) ? 256u : 128u;
  t->overlap = 1;
  t->load_base = 0;
  t->policy_code = policy;
  t->max_inflight = 0;
  t->search_warp = 0;
  t->search_warp_load = 0;
  if (cudaGetDevice(&t->device) != cudaSuccess) return CK_ECUDA;
  if (cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->device) != cudaSuccess)
    return CK_ECUDA;
  return CK_OK;
}

// ---- kernel dispatch -------------------------------------------------

InsertFn pick_insert(const ck_table* t) {
  const DevTable& d = t->dt;
  if (d.B == 1) return pick_insert_b1(d.policy);
  if (d.B == 4) return pick_insert_b4(d.policy, d.ghost != 0);
  if (d.B == 8) return pick_insert_b8(d.policy, d.ghost != 0);
  return nullptr;
}

unsigned grid_for(uint64_t n, uint32_t block) {
  uint64_t g = (n + block - 1) / block;
  if (g == 0) g = 1;
  if (g > 0x7FFFFFFFull) g = 0x7FFFFFFFull;
  return (unsigned)g;
}

}  // namespace

// Device view of a handle, for the other translation units of the library.
const ck::DevTable* ck_internal_devtable(const ck_table* t) { return &t->dt; }

// Keys submitted for insertion so far (the bins-viewed histogram's load).
uint64_t ck_internal_load_base(const ck_table* t) { return t->load_base; }

// Bookkeeping of an insert launch made by another translation unit: the
// handle's readers wait for its stream, and the load base moves on.
void ck_internal_note_insert(ck_table* t, void* stream, uint64_t n) {
  t->last = S(stream);
  t->load_base += n;
}

// The stream that host-side reads of the table (stats, export) wait for;
// the serving loop hands it back when it lets go of the table.
void* ck_internal_swap_last(ck_table* t, void* s) {
  void* old = t->last;
  t->last = S(s);
  return old;
}

// The single-table insert launch for a bare device view (the batched form's
// one-launch-per-table reference path): concurrent mode, overlapping launches,
// at most max_threads insertions in flight.
int ck_internal_launch_insert(const DevTable& dt, uint32_t block, int sm_count, const uint32_t* keys,
                              const uint32_t* vals, uint64_t n, uint8_t* status, cudaStream_t s,
                              uint64_t max_threads) {
  if (dt.policy != CK_QUEUE && dt.policy != CK_RANDOM) return CK_ENOTSUP;
  InsertFn fn = dt.B == 4 ? pick_insert_b4(dt.policy, dt.ghost != 0)
                          : dt.B == 8 ? pick_insert_b8(dt.policy, dt.ghost != 0) : nullptr;
  if (!fn) return CK_ECUDA;
  const InsertLaunch l{&dt, block, sm_count, true, 0, max_threads};
  return fn(l, keys, vals, n, status, nullptr, false, 0u, s) == cudaSuccess ? CK_OK : CK_ECUDA;
}

extern "C" {

size_t ck_required_bytes(uint64_t bins, uint32_t slots_per_bin, uint32_t d, uint32_t policy) {
  if (!shape_ok(bins, slots_per_bin, d, policy)) return 0;
  return layout(bins, slots_per_bin, policy).total;
}

int ck_create(ck_table** out, uint64_t bins, uint32_t slots_per_bin, uint32_t d, uint32_t policy,
              uint64_t seed) {
  if (!out) return CK_EINVAL;
  *out = nullptr;
  if (!shape_ok(bins, slots_per_bin, d, policy)) return CK_EINVAL;
  size_t bytes = layout(bins, slots_per_bin, policy).total;
  void* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return CK_ENOMEM;
  }
  ck_table* t = new (std::nothrow) ck_table();
  if (!t) {
    cudaFree(buf);
    return CK_ENOMEM;
  }
  int rc = init_table(t, buf, bytes, true, bins, slots_per_bin, d, policy, seed);
  if (rc == CK_OK && is_search(policy)) rc = check(cudaMemset(t->dt.scratch, 0, (size_t)t->dt.n_searchers * SEARCH_REGION));
  if (rc == CK_OK) rc = clear_on(t, nullptr);
  if (rc == CK_OK) rc = check(cudaDeviceSynchronize());
  if (rc != CK_OK) {
    cudaFree(buf);
    delete t;
    return rc;
  }
  *out = t;
  return CK_OK;
}

int ck_create_on(ck_table** out, void* dev_buf, size_t bytes, uint64_t bins, uint32_t slots_per_bin, uint32_t d,
                 uint32_t policy, uint64_t seed, void* stream) {
  if (!out) return CK_EINVAL;
  *out = nullptr;
  if (!dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) % ALIGN) != 0) return CK_EINVAL;
  if (!shape_ok(bins, slots_per_bin, d, policy)) return CK_EINVAL;
  if (bytes < layout(bins, slots_per_bin, policy).total) return CK_ENOMEM;
  ck_table* t = new (std::nothrow) ck_table();
  if (!t) return CK_ENOMEM;
  int rc = init_table(t, dev_buf, bytes, false, bins, slots_per_bin, d, policy, seed);
  if (rc == CK_OK && is_search(policy))
    rc = check(cudaMemsetAsync(t->dt.scratch, 0, (size_t)t->dt.n_searchers * SEARCH_REGION, S(stream)));
  if (rc == CK_OK) rc = clear_on(t, S(stream));
  if (rc != CK_OK) {
    delete t;
    return rc;
  }
  *out = t;
  return CK_OK;
}

int ck_set_param(ck_table* t, int key, int64_t value) {
  if (!t) return CK_EINVAL;
  DevTable& d = t->dt;
  switch (key) {
    case CK_PARAM_CHAIN_CAP: {
      int64_t hi = is_search(t->policy_code) ? MAX_GROUPS : LONG_CHAIN - 8;
      if (value < 1 || value > hi) return CK_EINVAL;
      d.cap = (uint32_t)value;
      return CK_OK;
    }
    case CK_PARAM_MAX_RETRIES:
      if (value < 1 || value > (1 << 20)) return CK_EINVAL;
      d.max_retries = (uint32_t)value;
      return CK_OK;
    case CK_PARAM_RNG_SEED:
      d.rng_seed = (uint64_t)value;
      return CK_OK;
    case CK_PARAM_BLOCK:
      if (value != 32 && value != 64 && value != 128 && value != 256) return CK_EINVAL;
      t->block = (uint32_t)value;
      return CK_OK;
    case CK_PARAM_RATTLE_TIE_RESIDENT:
      d.tie_resident = value ? 1 : 0;
      return CK_OK;
    case CK_PARAM_ORDERED_WRITES:
      d.ordered_writes = value ? 1 : 0;
      return CK_OK;
    case CK_PARAM_OVERLAP:
      t->overlap = value ? 1 : 0;
      return CK_OK;
    case CK_PARAM_SPAWN_K:
      if (value < 1 || value > 8) return CK_EINVAL;
      d.spawn_k = (uint32_t)value;
      return CK_OK;
    case CK_PARAM_MAX_INFLIGHT:
      if (value < 0 || value > (1ll << 40)) return CK_EINVAL;
      t->max_inflight = (uint64_t)value;
      return CK_OK;
    case CK_PARAM_SEARCH_WARP:
      if (value != 0 && value != 1) return CK_EINVAL;
      if (value && (d.B == 1 || d.ghost || d.policy != CK_BFS)) return CK_EINVAL;
      t->search_warp = (uint32_t)value;
      return CK_OK;
    case CK_PARAM_SEARCH_WARP_LOAD:
      if (value < 0 || value > 1000) return CK_EINVAL;
      t->search_warp_load = (uint32_t)value;
      return CK_OK;
    case CK_PARAM_HASH_FAMILY:
      if (value != 0 && value != 1) return CK_EINVAL;
      d.hash_family = (uint32_t)value;
      return CK_OK;
    default:
      if (key >= CK_PARAM_HASH_SEED0 && key < CK_PARAM_HASH_SEED0 + (int)d.d) {
        if (value < 0 || value > 0xFFFFFFFFll) return CK_EINVAL;
        d.seeds[key - CK_PARAM_HASH_SEED0] = (uint32_t)value;
        return CK_OK;
      }
      return CK_EINVAL;
  }
}

int ck_insert_batch_ex(ck_table* t, const uint32_t* d_keys, const uint32_t* d_vals, uint64_t n, uint8_t* d_status,
                       uint32_t* d_viewed, uint32_t flags, void* stream) {
  if (!t) return CK_EINVAL;
  if (n == 0) return CK_OK;
  if (!d_keys || !d_vals) return CK_EINVAL;
  if (flags & ~(uint32_t)(CK_INS_SERIAL | CK_INS_UPSERT)) return CK_EINVAL;
  InsertFn fn = pick_insert(t);
  if (t->search_warp && t->dt.spawn_k == 1 && !(flags & (CK_INS_SERIAL | CK_INS_UPSERT)) &&
      t->load_base * 1000 >= (uint64_t)t->search_warp_load * t->dt.total_slots)
    fn = t->dt.B == 4 ? pick_insert_warp_b4() : pick_insert_warp_b8();
  if (!fn) return CK_ENOTSUP;
  const InsertLaunch l{&t->dt, t->block, t->sm_count, t->overlap != 0, t->load_base,
                       t->max_inflight ? t->max_inflight : ~0ull};
  cudaError_t e = fn(l, d_keys, d_vals, n, d_status, d_viewed, (flags & CK_INS_SERIAL) != 0,
                     (flags & CK_INS_UPSERT) ? 1u : 0u, S(stream));
  t->last = S(stream);
  t->load_base += n;
  return check(e);
}

int ck_insert_batch(ck_table* t, const uint32_t* d_keys, const uint32_t* d_vals, uint64_t n, uint8_t* d_status,
                    void* stream) {
  return ck_insert_batch_ex(t, d_keys, d_vals, n, d_status, nullptr, 0, stream);
}

int ck_lookup_batch(ck_table* t, const uint32_t* d_keys, uint64_t n, uint32_t* d_vals_out, uint8_t* d_found,
                    void* stream) {
  if (!t) return CK_EINVAL;
  if (n == 0) return CK_OK;
  if (!d_keys) return CK_EINVAL;
  unsigned grid = grid_for(n, 256);
  if (t->dt.B == 4) k_lookup2<4><<<grid, 256, 0, S(stream)>>>(t->dt, d_keys, n, d_vals_out, d_found);
  else if (t->dt.B == 8) k_lookup2<8><<<grid, 256, 0, S(stream)>>>(t->dt, d_keys, n, d_vals_out, d_found);
  else k_lookup_dary<<<grid, 256, 0, S(stream)>>>(t->dt, d_keys, n, d_vals_out, d_found);
  t->last = S(stream);
  return check(cudaGetLastError());
}

int ck_delete_batch(ck_table* t, const uint32_t* d_keys, uint64_t n, uint8_t* d_found, void* stream) {
  if (!t) return CK_EINVAL;
  if (n == 0) return CK_OK;
  if (!d_keys) return CK_EINVAL;
  unsigned grid = grid_for(n, 256);
  if (t->dt.B == 4) k_delete<4><<<grid, 256, 0, S(stream)>>>(t->dt, d_keys, n, d_found);
  else if (t->dt.B == 8) k_delete<8><<<grid, 256, 0, S(stream)>>>(t->dt, d_keys, n, d_found);
  else k_delete<1><<<grid, 256, 0, S(stream)>>>(t->dt, d_keys, n, d_found);
  t->load_base = t->load_base > n ? t->load_base - n : 0;
  t->last = S(stream);
  return check(cudaGetLastError());
}

int ck_stats(ck_table* t, ck_stats_t* out) {
  if (!t || !out) return CK_EINVAL;
  unsigned long long c[C_N];
  if (cudaStreamSynchronize(t->last) != cudaSuccess) return CK_ECUDA;
  if (cudaMemcpy(c, t->dt.counters, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return CK_ECUDA;
  std::memset(out, 0, sizeof(*out));
  out->inserts_ok = c[C_INS_OK];
  out->inserts_failed = c[C_INS_FAILED];
  out->inserts_aborted = c[C_INS_ABORTED];
  out->bins_viewed = c[C_VIEWED];
  out->kicks = c[C_KICKS];
  out->chain_max = c[C_CHAIN_MAX];
  out->aborts = c[C_ABORTS];
  out->ghost_pairs_made = c[C_GHOSTS_MADE];
  out->dup_evictions = c[C_DUP_EVICT];
  out->size = c[C_SIZE];
  out->live_ghosts = c[C_LIVE_GHOSTS];
  out->lookups = c[C_LOOKUPS];
  out->lookup_hits = c[C_LOOKUP_HITS];
  out->deletes = c[C_DELETES];
  out->delete_hits = c[C_DELETE_HITS];
  out->delete_aborts = c[C_DELETE_ABORTS];
  out->conflict_views = c[C_REVIEWS];
  out->bins_viewed_all = c[C_VIEWED_ALL];
  out->total_slots = t->dt.total_slots;
  out->load = (double)out->size / (double)out->total_slots;
  uint64_t ins = out->inserts_ok + out->inserts_failed + out->inserts_aborted;
  out->bins_viewed_per_insert = ins ? (double)out->bins_viewed / (double)ins : 0.0;
  out->aborts_per_insert = ins ? (double)out->aborts / (double)ins : 0.0;
  out->updates = c[C_UPDATES];
  return CK_OK;
}

int ck_load_histogram(ck_table* t, uint64_t* views, uint64_t* inserts) {
  if (!t || !views || !inserts) return CK_EINVAL;
  if (cudaStreamSynchronize(t->last) != cudaSuccess) return CK_ECUDA;
  if (cudaMemcpy(views, t->dt.counters + C_N, HIST_BUCKETS * sizeof(uint64_t), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return CK_ECUDA;
  if (cudaMemcpy(inserts, t->dt.counters + C_N + HIST_BUCKETS, HIST_BUCKETS * sizeof(uint64_t),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return CK_ECUDA;
  return CK_OK;
}

int ck_chain_histogram(ck_table* t, uint64_t* counts) {
  if (!t || !counts) return CK_EINVAL;
  if (cudaStreamSynchronize(t->last) != cudaSuccess) return CK_ECUDA;
  if (cudaMemcpy(counts, t->dt.counters + CHAIN_HIST, CHAIN_BUCKETS * sizeof(uint64_t), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return CK_ECUDA;
  return CK_OK;
}

int ck_reset_stats(ck_table* t) {
  if (!t) return CK_EINVAL;
  // keep the size and the live ghost pairs: they describe the table, not the run
  unsigned long long keep[2];
  if (cudaStreamSynchronize(t->last) != cudaSuccess) return CK_ECUDA;
  if (cudaMemcpy(keep, t->dt.counters + C_SIZE, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return CK_ECUDA;
  if (cudaMemset(t->dt.counters, 0, COUNTER_WORDS * sizeof(uint64_t)) != cudaSuccess) return CK_ECUDA;
  if (cudaMemcpy(t->dt.counters + C_SIZE, keep, 2 * sizeof(unsigned long long), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return CK_ECUDA;
  return CK_OK;
}

int ck_clear(ck_table* t, void* stream) {
  if (!t) return CK_EINVAL;
  return clear_on(t, S(stream));
}

int ck_export(ck_table* t, uint64_t* h_slots, uint32_t* h_meta) {
  if (!t) return CK_EINVAL;
  if (cudaStreamSynchronize(t->last) != cudaSuccess) return CK_ECUDA;
  if (h_slots && cudaMemcpy(h_slots, t->dt.slots, t->dt.total_slots * sizeof(uint64_t), cudaMemcpyDeviceToHost) !=
                     cudaSuccess)
    return CK_ECUDA;
  if (h_meta &&
      cudaMemcpy(h_meta, t->dt.meta, t->dt.n_bins * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CK_ECUDA;
  return CK_OK;
}

int ck_import(ck_table* t, const uint64_t* h_slots, const uint32_t* h_meta) {
  if (!t || !h_slots || !h_meta) return CK_EINVAL;
  const uint64_t nb = t->dt.n_bins;
  const uint32_t B = t->dt.B;
  // a snapshot of a quiescent table: no claim flags, duplicate marks only on
  // occupied slots and in pairs, no reserved key stored
  uint64_t occupied = 0, dups = 0;
  for (uint64_t b = 0; b < nb; b++) {
    const uint32_t m = h_meta[b];
    const uint32_t dmask = B > 1 ? (m >> DUP_SHIFT) & 0xFFu : 0u;
    if (B > 1 ? (m & 0xFFu) != 0 : (m & 1u) != 0) return CK_EINVAL;
    if (B > 1 && (dmask >> B) != 0) return CK_EINVAL;
    for (uint32_t s = 0; s < B; s++) {
      const uint64_t rec = h_slots[b * B + s];
      const bool dup = (dmask >> s) & 1u;
      if (rec == EMPTY) {
        if (dup) return CK_EINVAL;
        continue;
      }
      if ((uint32_t)(rec >> 32) == RESERVED_KEY) return CK_EINVAL;
      occupied++;
      dups += dup;
    }
  }
  if (dups & 1) return CK_EINVAL;
  if (cudaStreamSynchronize(t->last) != cudaSuccess) return CK_ECUDA;
  if (cudaMemcpy(t->dt.slots, h_slots, t->dt.total_slots * sizeof(uint64_t), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(t->dt.meta, h_meta, nb * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(t->dt.counters, 0, COUNTER_WORDS * sizeof(uint64_t)) != cudaSuccess)
    return CK_ECUDA;
  // a ghost pair is one key stored twice, both copies marked
  const unsigned long long size_ghosts[2] = {occupied - dups / 2, dups / 2};
  static_assert(C_LIVE_GHOSTS == C_SIZE + 1, "size and live ghosts are adjacent counters");
  if (cudaMemcpy(t->dt.counters + C_SIZE, size_ghosts, sizeof(size_ghosts), cudaMemcpyHostToDevice) != cudaSuccess)
    return CK_ECUDA;
  return CK_OK;
}

int ck_debug_claims(ck_table* t, uint64_t bin, uint32_t set_mask, uint32_t clear_mask) {
  if (!t || bin >= t->dt.n_bins) return CK_EINVAL;
  const uint32_t claim_bits = t->dt.B > 1 ? (1u << t->dt.B) - 1 : 1u;
  if ((set_mask | clear_mask) & ~claim_bits) return CK_EINVAL;
  if (cudaStreamSynchronize(t->last) != cudaSuccess) return CK_ECUDA;
  uint32_t m = 0;
  if (cudaMemcpy(&m, t->dt.meta + bin, sizeof(m), cudaMemcpyDeviceToHost) != cudaSuccess) return CK_ECUDA;
  m = (m & ~clear_mask) | set_mask;
  return cudaMemcpy(t->dt.meta + bin, &m, sizeof(m), cudaMemcpyHostToDevice) == cudaSuccess ? CK_OK : CK_ECUDA;
}

void ck_destroy(ck_table* t) {
  if (!t) return;
  if (t->last) cudaStreamSynchronize(t->last);
  if (t->owns) cudaFree(t->buf);
  delete t;
}

int ck_shape(const ck_table* t, uint64_t* bins, uint32_t* slots_per_bin, uint32_t* d, uint32_t* policy) {
  if (!t) return CK_EINVAL;
  if (bins) *bins = t->dt.n_bins;
  if (slots_per_bin) *slots_per_bin = t->dt.B;
  if (d) *d = t->dt.d;
  if (policy) *policy = t->policy_code;
  return CK_OK;
}

const char* ck_strerror(int code) {
  switch (code) {
    case CK_OK: return "ok";
    case CK_EINVAL: return "invalid argument";
    case CK_ENOMEM: return "out of memory or buffer too small";
    case CK_ECUDA: return "CUDA runtime error";
    case CK_EBUSY: return "busy: admission refused";
    case CK_ENOTSUP: return "not supported";
    default: return "unknown error";
  }
}

}  // extern "C"
