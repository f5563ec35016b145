// ck_multi.cu -- the batched form: many independent two-choice cuckoo tables
// of uneven sizes filled in one persistent launch.
//
// Each table is a full table (slots, metadata, counters) of its own and is
// filled with exactly the per-insertion code of the single-table path
// (insert_one: the kick-out policies of Sec. 3-7 with claim flags and
// back-to-front chains, Sec. 8), so a key set gives the same key->value map
// per table either way.  What the batched form changes is scheduling: the
// keys of all tables are cut into tiles, a tile list is built once, and a
// persistent grid pulls tiles from one global counter and keys within a
// tile from a shared-memory counter.  Small tables no longer leave the GPU
// idle and 4096 launches become one.  The reference path,
// ck_multi_insert_per_table, launches the single-table kernel once per
// table.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "ck.h"
#include "ck_kernels.cuh"

using namespace ck;

// per-table path: the single-table launcher of ck_lib.cu
int ck_internal_launch_insert(const DevTable& dt, uint32_t block, int sm_count, const uint32_t* keys,
                              const uint32_t* vals, uint64_t n, uint8_t* status, cudaStream_t s,
                              uint64_t max_threads);

namespace {

constexpr size_t ALIGN = 256;
size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Tile {
  uint32_t table;
  uint32_t pad;
  uint64_t lo, hi;  // key range in the shared key/value arrays
};

constexpr uint32_t MULTI_LONG_PLANS = 1024;

}  // namespace

struct ck_multi {
  uint32_t n_tables;
  uint32_t policy;
  std::vector<ck_multi_desc> desc;
  std::vector<DevTable> host_tables;  // host copies of the device descriptors
  DevTable* d_tables;
  Tile* d_tiles;
  unsigned long long* d_tile_ctr;
  uint8_t* buf;
  size_t bytes;
  uint32_t n_tiles;
  uint32_t tile;
  uint32_t block;
  uint32_t blocks_per_sm;  // 0: as many as fit
  uint32_t cap;
  int sm_count;
  cudaStream_t last;
  std::vector<size_t> table_off;  // byte offset of each table's slots
  size_t pool_off, busy_off, tables_off, tiles_off, ctr_off;
};

namespace {

struct MultiLayout {
  std::vector<size_t> off;  // per table: slots; meta and counters follow
  size_t tables, tiles, ctr, busy, pool, total;
  uint32_t n_tiles;
};

size_t table_bytes(const ck_multi_desc& d) {
  size_t b = align_up(d.bins * d.slots_per_bin * sizeof(uint64_t));
  b += align_up(d.bins * sizeof(uint32_t));
  b += align_up(COUNTER_WORDS * sizeof(uint64_t));
  return b;
}

uint32_t count_tiles(const ck_multi_desc* d, uint32_t n, uint32_t tile) {
  uint64_t t = 0;
  for (uint32_t i = 0; i < n; i++) t += (d[i].n_keys + tile - 1) / tile;
  return (uint32_t)t;
}

bool desc_ok(const ck_multi_desc* d, uint32_t n) {
  if (!d || n == 0) return false;
  for (uint32_t i = 0; i < n; i++) {
    if (d[i].bins < 2 || d[i].bins >= (1ull << 32)) return false;
    if (d[i].slots_per_bin != 4 && d[i].slots_per_bin != 8) return false;
  }
  return true;
}

// The tile list is sized for the smallest tile the autotuner may pick.
constexpr uint32_t MIN_TILE = 256;

MultiLayout multi_layout(const ck_multi_desc* d, uint32_t n) {
  MultiLayout L;
  size_t off = 0;
  L.off.resize(n);
  for (uint32_t i = 0; i < n; i++) {
    L.off[i] = off;
    off += table_bytes(d[i]);
  }
  L.tables = off;
  off = align_up(off + (size_t)n * sizeof(DevTable));
  L.n_tiles = count_tiles(d, n, MIN_TILE);
  L.tiles = off;
  off = align_up(off + (size_t)L.n_tiles * sizeof(Tile));
  L.ctr = off;
  off = align_up(off + (n + 1) * sizeof(unsigned long long));
  L.busy = off;
  off = align_up(off + MULTI_LONG_PLANS * sizeof(uint32_t));
  L.pool = off;
  off = align_up(off + (size_t)MULTI_LONG_PLANS * LONG_REGION);
  L.total = off;
  return L;
}

// Persistent batched insert: blocks pull tiles, threads pull keys.
template <int POL, bool GHOST>
__global__ void __launch_bounds__(256, 4) k_multi_insert(const DevTable* __restrict__ tables,
                                                      const Tile* __restrict__ tiles, uint32_t n_tiles,
                                                      unsigned long long* tile_ctr,
                                                      const uint32_t* __restrict__ keys,
                                                      const uint32_t* __restrict__ vals,
                                                      uint8_t* __restrict__ status) {
  __shared__ unsigned long long s_next, s_hi;
  __shared__ uint32_t s_tile, s_table;
  __shared__ unsigned long long bc[C_N];
  PlanStore<MAX_CHAIN> store;
  for (;;) {
    if (threadIdx.x == 0) {
      unsigned long long k = atomicAdd(tile_ctr, 1ull);
      s_tile = k < n_tiles ? (uint32_t)k : n_tiles;
      if (k < n_tiles) {
        Tile tl = tiles[k];
        s_table = tl.table;
        s_next = tl.lo;
        s_hi = tl.hi;
      }
    }
    for (int i = threadIdx.x; i < C_N; i += blockDim.x) bc[i] = 0;
    __syncthreads();
    if (s_tile >= n_tiles) break;
    const DevTable t = tables[s_table];
    const unsigned long long hi = s_hi;
    uint32_t ok = 0, failed = 0, aborted = 0, viewed = 0, viewed_all = 0, kicks = 0;  // per tile
    uint32_t aborts = 0, chain_max = 0, ghosts = 0, dupev = 0;
    for (;;) {
      unsigned long long i = atomicAdd(&s_next, 1ull);
      if (i >= hi) break;
      uint32_t key = keys[i];
      if (key == RESERVED_KEY) {
        if (status) status[i] = ST_INVALID;
        continue;
      }
      Ctx c;
      c.key = key;
      c.krec = ((uint64_t)key << 32) | vals[i];
      c.viewed = 0;
      c.reviews = 0;
      int st = t.B == 4 ? insert_one<4, POL, GHOST>(t, c, nullptr, aborts, store.e, MAX_CHAIN, true)
                        : insert_one<8, POL, GHOST>(t, c, nullptr, aborts, store.e, MAX_CHAIN, true);
      if (st == ST_OK) {
        ok++;
        kicks += c.kicks;
        chain_max = max(chain_max, c.kicks);
        ghosts += c.ghosts_made;
        dupev += c.dup_evict;
      } else if (st == ST_FAILED) {
        failed++;
      } else {
        aborted++;
      }
      viewed += c.viewed - c.viewed0;
      viewed_all += c.viewed;
      if (status) status[i] = (uint8_t)st;
    }
    if (ok) atomicAdd(&bc[C_INS_OK], ok);
    if (failed) atomicAdd(&bc[C_INS_FAILED], failed);
    if (aborted) atomicAdd(&bc[C_INS_ABORTED], aborted);
    if (viewed) atomicAdd(&bc[C_VIEWED], viewed);
    if (viewed_all) atomicAdd(&bc[C_VIEWED_ALL], viewed_all);
    if (kicks) atomicAdd(&bc[C_KICKS], kicks);
    if (aborts) atomicAdd(&bc[C_ABORTS], (unsigned long long)aborts);
    if (ghosts) atomicAdd(&bc[C_GHOSTS_MADE], (unsigned long long)ghosts);
    if (dupev) atomicAdd(&bc[C_DUP_EVICT], (unsigned long long)dupev);
    if (chain_max) atomicMax(&bc[C_CHAIN_MAX], (unsigned long long)chain_max);
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 0; k < C_N; k++) {
        if (!bc[k]) continue;
        if (k == C_CHAIN_MAX) atomicMax(t.counters + k, bc[k]);
        else atomicAdd(t.counters + k, bc[k]);
      }
      if (bc[C_INS_OK]) atomicAdd(t.counters + C_SIZE, bc[C_INS_OK]);
      long long dg = (long long)bc[C_GHOSTS_MADE] - (long long)bc[C_DUP_EVICT];
      if (dg) atomicAdd(t.counters + C_LIVE_GHOSTS, (unsigned long long)dg);
    }
    __syncthreads();
  }
}

// Lookups across tables: key i belongs to table tab[i].
__global__ void __launch_bounds__(256) k_multi_lookup(const DevTable* __restrict__ tables,
                                                      const uint32_t* __restrict__ tab,
                                                      const uint32_t* __restrict__ keys, uint64_t n,
                                                      uint32_t* __restrict__ vals_out,
                                                      uint8_t* __restrict__ found_out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const DevTable& t = tables[tab[i]];
    uint32_t key = keys[i];
    uint32_t val = 0;
    bool f = false;
    if (key != RESERVED_KEY) {
      uint32_t b0, b1;
      bins2(t, key, b0, b1);
      if (t.B == 4) {
        uint64_t s0[4], s1[4];
        load_bin_nc<4>(t, b0, s0);
        load_bin_nc<4>(t, b1, s1);
        f = match_bin<4>(s0, key, val);
        if (!f) f = match_bin<4>(s1, key, val);
      } else {
        uint64_t s0[8], s1[8];
        load_bin_nc<8>(t, b0, s0);
        load_bin_nc<8>(t, b1, s1);
        f = match_bin<8>(s0, key, val);
        if (!f) f = match_bin<8>(s1, key, val);
      }
    }
    if (vals_out) vals_out[i] = val;
    if (found_out) found_out[i] = (uint8_t)f;
  }
}

using MultiFn = void (*)(const ck_multi*, const uint32_t*, const uint32_t*, uint8_t*, cudaStream_t, unsigned,
                         unsigned);

template <int POL, bool GHOST>
void launch_multi(const ck_multi* m, const uint32_t* k, const uint32_t* v, uint8_t* st, cudaStream_t s,
                  unsigned grid, unsigned block) {
  k_multi_insert<POL, GHOST><<<grid, block, 0, s>>>(m->d_tables, m->d_tiles, m->n_tiles, m->d_tile_ctr, k, v, st);
}

MultiFn pick_multi(uint32_t policy) {
  bool g = (policy & CK_GHOST) != 0;
  switch (policy & 0xFF) {
    case CK_RANDOM: return g ? launch_multi<P_RANDOM, true> : launch_multi<P_RANDOM, false>;
    case CK_QUEUE: return g ? launch_multi<P_QUEUE, true> : launch_multi<P_QUEUE, false>;
    default: return nullptr;
  }
}

int occupancy_blocks(uint32_t policy, uint32_t block) {
  int per_sm = 0;
  cudaError_t e = cudaErrorInvalidValue;
  bool g = (policy & CK_GHOST) != 0;
  if ((policy & 0xFF) == CK_QUEUE)
    e = g ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_insert<P_QUEUE, true>, block, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_insert<P_QUEUE, false>, block, 0);
  else
    e = g ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_insert<P_RANDOM, true>, block, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_insert<P_RANDOM, false>, block, 0);
  if (e != cudaSuccess || per_sm < 1) return 1;
  return per_sm;
}

// Build the tile list for the current tile size and upload it.  Tiles are
// interleaved round-robin over the tables (tile r of every table, then tile
// r+1, ...): the GPU works on many tables at once and each table keeps only
// a few tiles in flight, so its load grows in order and its insertions
// rarely meet each other's claims.
int build_tiles(ck_multi* m, cudaStream_t s) {
  std::vector<Tile> tiles;
  tiles.reserve(count_tiles(m->desc.data(), m->n_tables, m->tile));
  for (uint64_t r = 0;; r++) {
    bool any = false;
    for (uint32_t i = 0; i < m->n_tables; i++) {
      const ck_multi_desc& d = m->desc[i];
      uint64_t lo = r * m->tile;
      if (lo >= d.n_keys) continue;
      any = true;
      Tile t;
      t.table = i;
      t.pad = 0;
      t.lo = d.key_offset + lo;
      t.hi = d.key_offset + (lo + m->tile < d.n_keys ? lo + m->tile : d.n_keys);
      tiles.push_back(t);
    }
    if (!any) break;
  }
  m->n_tiles = (uint32_t)tiles.size();
  if (cudaMemcpyAsync(m->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return CK_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? CK_OK : CK_ECUDA;
}

int clear_tables(ck_multi* m, cudaStream_t s) {
  for (uint32_t i = 0; i < m->n_tables; i++) {
    const DevTable& t = m->host_tables[i];
    if (cudaMemsetAsync(t.slots, 0xFF, t.total_slots * sizeof(uint64_t), s) != cudaSuccess) return CK_ECUDA;
    if (cudaMemsetAsync(t.meta, 0, t.n_bins * sizeof(uint32_t), s) != cudaSuccess) return CK_ECUDA;
    if (cudaMemsetAsync(t.counters, 0, COUNTER_WORDS * sizeof(uint64_t), s) != cudaSuccess)
      return CK_ECUDA;
  }
  m->last = s;
  return CK_OK;
}

}  // namespace

extern "C" {

size_t ck_multi_required_bytes(const ck_multi_desc* h_desc, uint32_t n_tables) {
  if (!desc_ok(h_desc, n_tables)) return 0;
  return multi_layout(h_desc, n_tables).total;
}

int ck_multi_create_on(ck_multi** out, void* dev_buf, size_t bytes, const ck_multi_desc* h_desc, uint32_t n_tables,
                       uint32_t policy, uint64_t seed, void* stream) {
  if (!out) return CK_EINVAL;
  *out = nullptr;
  if (!desc_ok(h_desc, n_tables)) return CK_EINVAL;
  uint32_t pol = policy & 0xFF;
  if ((policy & ~0x1FFu) != 0 || (pol != CK_RANDOM && pol != CK_QUEUE)) return CK_ENOTSUP;
  if (!dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) % ALIGN) != 0) return CK_EINVAL;
  MultiLayout L = multi_layout(h_desc, n_tables);
  if (bytes < L.total) return CK_ENOMEM;
  ck_multi* m = new (std::nothrow) ck_multi();
  if (!m) return CK_ENOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  m->n_tables = n_tables;
  m->policy = policy;
  m->desc.assign(h_desc, h_desc + n_tables);
  m->buf = static_cast<uint8_t*>(dev_buf);
  m->bytes = bytes;
  m->tile = 4096;
  m->block = 128;
  m->blocks_per_sm = 0;
  m->cap = 500;
  m->last = s;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete m;
    return CK_ECUDA;
  }
  m->d_tables = reinterpret_cast<DevTable*>(m->buf + L.tables);
  m->d_tiles = reinterpret_cast<Tile*>(m->buf + L.tiles);
  m->d_tile_ctr = reinterpret_cast<unsigned long long*>(m->buf + L.ctr);
  uint32_t* busy = reinterpret_cast<uint32_t*>(m->buf + L.busy);
  uint8_t* pool = m->buf + L.pool;
  m->host_tables.resize(n_tables);
  for (uint32_t i = 0; i < n_tables; i++) {
    const ck_multi_desc& d = h_desc[i];
    DevTable& t = m->host_tables[i];
    std::memset(&t, 0, sizeof(t));
    uint8_t* base = m->buf + L.off[i];
    size_t so = align_up(d.bins * d.slots_per_bin * sizeof(uint64_t));
    size_t mo = so + align_up(d.bins * sizeof(uint32_t));
    t.slots = reinterpret_cast<uint64_t*>(base);
    t.meta = reinterpret_cast<uint32_t*>(base + so);
    t.counters = reinterpret_cast<unsigned long long*>(base + mo);
    t.scratch = nullptr;
    t.long_scratch = pool;
    t.long_busy = busy;
    t.slab_busy = nullptr;
    t.n_bins = d.bins;
    t.total_slots = d.bins * d.slots_per_bin;
    t.rng_seed = seed + i;
    t.bin_mask = (d.bins & (d.bins - 1)) == 0 ? (uint32_t)(d.bins - 1) : 0u;
    t.B = d.slots_per_bin;
    t.d = 2;
    t.policy = pol;
    t.ghost = (policy & CK_GHOST) ? 1 : 0;
    t.cap = m->cap;
    t.max_retries = 1024;
    t.ordered_writes = 0;
    t.spawn_k = 1;
    t.n_searchers = 0;
    t.n_long = MULTI_LONG_PLANS;
    t.hash_family = 0;
    t.seeds[0] = 0x9E3779B9u;
    t.seeds[1] = 0x85EBCA6Bu;
    t.seeds[2] = 0xC2B2AE35u;
    t.seeds[3] = 0x27D4EB2Fu;
  }
  int rc = CK_OK;
  if (cudaMemcpyAsync(m->d_tables, m->host_tables.data(), n_tables * sizeof(DevTable), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(busy, 0, MULTI_LONG_PLANS * sizeof(uint32_t), s) != cudaSuccess)
    rc = CK_ECUDA;
  if (rc == CK_OK) rc = clear_tables(m, s);
  if (rc == CK_OK) rc = build_tiles(m, s);
  if (rc != CK_OK) {
    delete m;
    return rc;
  }
  *out = m;
  return CK_OK;
}

int ck_multi_set_param(ck_multi* m, int key, int64_t value) {
  if (!m) return CK_EINVAL;
  switch (key) {
    case CK_MULTI_TILE:
      if (value < MIN_TILE || value > (1 << 22)) return CK_EINVAL;
      m->tile = (uint32_t)value;
      return build_tiles(m, m->last);
    case CK_MULTI_BLOCK:
      if (value != 64 && value != 128 && value != 256) return CK_EINVAL;
      m->block = (uint32_t)value;
      return CK_OK;
    case CK_MULTI_BLOCKS_PER_SM:
      if (value < 0 || value > 32) return CK_EINVAL;
      m->blocks_per_sm = (uint32_t)value;
      return CK_OK;
    case CK_MULTI_CHAIN_CAP: {
      if (value < 1 || value > LONG_CHAIN - 8) return CK_EINVAL;
      m->cap = (uint32_t)value;
      for (auto& t : m->host_tables) t.cap = m->cap;
      if (cudaMemcpyAsync(m->d_tables, m->host_tables.data(), m->n_tables * sizeof(DevTable), cudaMemcpyHostToDevice,
                          m->last) != cudaSuccess)
        return CK_ECUDA;
      return CK_OK;
    }
    default:
      return CK_EINVAL;
  }
}

int ck_multi_insert(ck_multi* m, const uint32_t* d_keys, const uint32_t* d_vals, uint8_t* d_status, void* stream) {
  if (!m || !d_keys || !d_vals) return CK_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MultiFn fn = pick_multi(m->policy);
  if (!fn) return CK_ENOTSUP;
  int per_sm = occupancy_blocks(m->policy, m->block);
  if (m->blocks_per_sm && (int)m->blocks_per_sm < per_sm) per_sm = (int)m->blocks_per_sm;
  unsigned grid = (unsigned)(per_sm * m->sm_count);
  if (grid > m->n_tiles) grid = m->n_tiles ? m->n_tiles : 1;
  if (cudaMemsetAsync(m->d_tile_ctr, 0, sizeof(unsigned long long), s) != cudaSuccess) return CK_ECUDA;
  fn(m, d_keys, d_vals, d_status, s, grid, m->block);
  m->last = s;
  return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

int ck_multi_insert_per_table(ck_multi* m, const uint32_t* d_keys, const uint32_t* d_vals, uint8_t* d_status,
                              void* stream) {
  if (!m || !d_keys || !d_vals) return CK_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (uint32_t i = 0; i < m->n_tables; i++) {
    const ck_multi_desc& d = m->desc[i];
    if (!d.n_keys) continue;
    // in flight at once: at most 1/16 of the table's slots (one block at
    // least), the operating range of the claim protocol (Sec. 8 runs a few
    // threads on a large table); launches of different tables overlap
    uint64_t max_threads = d.bins * d.slots_per_bin / 16;
    if (max_threads < m->block) max_threads = m->block;
    int rc = ck_internal_launch_insert(m->host_tables[i], m->block, m->sm_count, d_keys + d.key_offset,
                                       d_vals + d.key_offset, d.n_keys, d_status ? d_status + d.key_offset : nullptr,
                                       s, max_threads);
    if (rc != CK_OK) return rc;
  }
  m->last = s;
  return CK_OK;
}

int ck_multi_lookup(ck_multi* m, const uint32_t* d_table, const uint32_t* d_keys, uint64_t n, uint32_t* d_vals_out,
                    uint8_t* d_found, void* stream) {
  if (!m) return CK_EINVAL;
  if (n == 0) return CK_OK;
  if (!d_table || !d_keys) return CK_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint64_t g = (n + 255) / 256;
  if (g > 0x7FFFFFFFull) g = 0x7FFFFFFFull;
  k_multi_lookup<<<(unsigned)g, 256, 0, s>>>(m->d_tables, d_table, d_keys, n, d_vals_out, d_found);
  m->last = s;
  return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

int ck_multi_table_stats(ck_multi* m, uint32_t table, ck_stats_t* out) {
  if (!m || !out || table >= m->n_tables) return CK_EINVAL;
  unsigned long long c[C_N];
  if (cudaStreamSynchronize(m->last) != cudaSuccess) return CK_ECUDA;
  if (cudaMemcpy(c, m->host_tables[table].counters, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return CK_ECUDA;
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
  out->conflict_views = c[C_REVIEWS];
  out->bins_viewed_all = c[C_VIEWED_ALL];
  out->total_slots = m->host_tables[table].total_slots;
  out->load = out->total_slots ? (double)out->size / (double)out->total_slots : 0.0;
  uint64_t ins = out->inserts_ok + out->inserts_failed + out->inserts_aborted;
  out->bins_viewed_per_insert = ins ? (double)out->bins_viewed / (double)ins : 0.0;
  out->aborts_per_insert = ins ? (double)out->aborts / (double)ins : 0.0;
  return CK_OK;
}

int ck_multi_stats(ck_multi* m, ck_stats_t* out) {
  if (!m || !out) return CK_EINVAL;
  ck_stats_t sum;
  std::memset(&sum, 0, sizeof(sum));
  uint64_t chain_max = 0;
  for (uint32_t i = 0; i < m->n_tables; i++) {
    ck_stats_t s;
    int rc = ck_multi_table_stats(m, i, &s);
    if (rc != CK_OK) return rc;
    sum.inserts_ok += s.inserts_ok;
    sum.inserts_failed += s.inserts_failed;
    sum.inserts_aborted += s.inserts_aborted;
    sum.bins_viewed += s.bins_viewed;
    sum.kicks += s.kicks;
    sum.aborts += s.aborts;
    sum.ghost_pairs_made += s.ghost_pairs_made;
    sum.dup_evictions += s.dup_evictions;
    sum.size += s.size;
    sum.live_ghosts += s.live_ghosts;
    sum.conflict_views += s.conflict_views;
    sum.bins_viewed_all += s.bins_viewed_all;
    sum.total_slots += s.total_slots;
    if (s.chain_max > chain_max) chain_max = s.chain_max;
  }
  sum.chain_max = chain_max;
  sum.load = sum.total_slots ? (double)sum.size / (double)sum.total_slots : 0.0;
  uint64_t ins = sum.inserts_ok + sum.inserts_failed + sum.inserts_aborted;
  sum.bins_viewed_per_insert = ins ? (double)sum.bins_viewed / (double)ins : 0.0;
  sum.aborts_per_insert = ins ? (double)sum.aborts / (double)ins : 0.0;
  *out = sum;
  return CK_OK;
}

int ck_multi_export(ck_multi* m, uint32_t table, uint64_t* h_slots, uint32_t* h_meta) {
  if (!m || table >= m->n_tables) return CK_EINVAL;
  if (cudaStreamSynchronize(m->last) != cudaSuccess) return CK_ECUDA;
  const DevTable& t = m->host_tables[table];
  if (h_slots && cudaMemcpy(h_slots, t.slots, t.total_slots * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CK_ECUDA;
  if (h_meta && cudaMemcpy(h_meta, t.meta, t.n_bins * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CK_ECUDA;
  return CK_OK;
}

int ck_multi_clear(ck_multi* m, void* stream) {
  if (!m) return CK_EINVAL;
  return clear_tables(m, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

// A captured fill of a batched form: the graph and its executable.
struct ck_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  ck_multi* m;
};

extern "C" {

int ck_multi_capture(ck_multi* m, const uint32_t* d_keys, const uint32_t* d_vals, uint8_t* d_status,
                     uint32_t flags, void* stream, ck_graph** out) {
  if (!out) return CK_EINVAL;
  *out = nullptr;
  if (!m || !d_keys || !d_vals) return CK_EINVAL;
  if (flags & ~(uint32_t)(CK_MULTI_CAPTURE_CLEAR | CK_MULTI_CAPTURE_PER_TABLE)) return CK_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bool own = false;
  if (!s) {  // the legacy default stream cannot be captured: use a stream of our own
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return CK_ECUDA;
    own = true;
  }
  const cudaStream_t last = m->last;
  int rc = CK_OK;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = CK_ECUDA;
  if (rc == CK_OK) {
    if (flags & CK_MULTI_CAPTURE_CLEAR) rc = clear_tables(m, s);
    if (rc == CK_OK)
      rc = (flags & CK_MULTI_CAPTURE_PER_TABLE) ? ck_multi_insert_per_table(m, d_keys, d_vals, d_status, s)
                                                : ck_multi_insert(m, d_keys, d_vals, d_status, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);  // always ends the capture, even after an error
    if (rc == CK_OK && (e != cudaSuccess || !g)) rc = CK_ECUDA;
    ck_graph* h = nullptr;
    if (rc == CK_OK) {
      h = new (std::nothrow) ck_graph();
      if (!h) rc = CK_ENOMEM;
    }
    if (rc == CK_OK && cudaGraphInstantiate(&h->exec, g, 0) != cudaSuccess) rc = CK_ECUDA;
    if (rc == CK_OK) {
      h->graph = g;
      h->m = m;
      *out = h;
    } else {
      if (g) cudaGraphDestroy(g);
      delete h;
      cudaGetLastError();
    }
  }
  m->last = last;  // nothing ran yet: the handle's readers keep waiting where they did
  if (own) cudaStreamDestroy(s);
  return rc;
}

int ck_graph_launch(ck_graph* g, void* stream) {
  if (!g) return CK_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaGraphLaunch(g->exec, s) != cudaSuccess) return CK_ECUDA;
  g->m->last = s;
  return CK_OK;
}

void ck_graph_destroy(ck_graph* g) {
  if (!g) return;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
}

void ck_multi_destroy(ck_multi* m) {
  if (!m) return;
  if (m->last) cudaStreamSynchronize(m->last);
  delete m;
}

}  // extern "C"
