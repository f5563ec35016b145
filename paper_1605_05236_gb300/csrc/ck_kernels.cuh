// ck_kernels.cuh -- the bulk kernels of the GB300 cuckoo table: insert
// (every policy), lookup and delete (Kuszmaul, arXiv:1605.05236, Sec. 1,
// Sec. 3-8), plus their per-batch counters.
#pragma once
#include "ck_search.cuh"

namespace ck {

// Block-wide accumulation of per-thread counts, then one global add each.
struct BlockCounters {
  unsigned long long v[C_N];
};

__device__ __forceinline__ void flush_counter(unsigned long long* shared_slot, unsigned long long x) {
  if (x) atomicAdd(shared_slot, x);
}

// Randomised exponential backoff after a conflict: [w, 2w) ns with w =
// 64 << attempt, up to 32-64 us, so that long walks that keep meeting each
// other (small tables with most keys in flight) drift apart.  Measured on
// the 2^14 x 4 table with all 62,259 keys in flight at once (1.3 claim
// conflicts per key): capping w at 32 us rather than 1 ms fills it about 9%
// faster; the large fills do not change.
__device__ __forceinline__ void backoff(uint32_t attempt, uint32_t key) {
  uint32_t w = 64u << (attempt < 9 ? attempt : 9);
  __nanosleep(w + (fmix32(key ^ attempt) & (w - 1)));
}

template <int B, int POL, bool GHOST>
__device__ __forceinline__ int attempt_insert(const DevTable& t, Ctx& c, uint8_t* region) {
  if constexpr (B == 1) {
    if constexpr (POL == P_RATTLE) return insert_rattle(t, c);
    else if constexpr (POL == P_RANDOM) return insert_random_dary(t, c);
    else return insert_search_dary<POL>(t, c, region);
  } else if constexpr (POL == P_QUEUE) {
    return insert_queue<B, GHOST>(t, c);
  } else if constexpr (POL == P_BFS || POL == P_SORTED || POL == P_HYBRID) {
    return insert_search<B, POL, GHOST>(t, c, region);
  } else {
    return insert_random2<B, GHOST>(t, c);
  }
}

// A block's search scratch: ceil(blockDim / SLAB) slabs of SLAB consecutive
// per-thread regions, taken together at block start (all or none: a block
// never waits while holding a slab, so blocks of overlapping launches cannot
// hold each other up) and returned at block end.  A block of the next launch
// may wait for slabs while the previous launch drains; the wait is bounded
// (about 10 ms), after which the block reports its keys as aborted.
__device__ __forceinline__ bool acquire_slabs(const DevTable& t, int* out, int need) {
  const uint32_t n_slabs = t.n_searchers / SLAB;
  if (n_slabs < (uint32_t)need) return false;
  for (uint32_t round = 0; round < 4096; round++) {
    int got = 0;
    uint32_t start = (blockIdx.x * (uint32_t)need + round * 7919u) % n_slabs;
    for (uint32_t k = 0; k < n_slabs && got < need; k++) {
      uint32_t r = start + k;
      if (r >= n_slabs) r -= n_slabs;
      if (*(volatile uint32_t*)(t.slab_busy + r) == 0 && atomicCAS(t.slab_busy + r, 0u, 1u) == 0u) out[got++] = (int)r;
    }
    if (got == need) return true;
    for (int j = 0; j < got; j++) atomicExch(t.slab_busy + out[j], 0u);
    __nanosleep(2000);
  }
  return false;
}

// One insertion with bounded retries after claim conflicts.  A chain that
// outgrows the local plan continues in a scratch plan.  retry_failed: a
// random walk that failed in concurrent mode is tried again with new draws
// (up to 3 times): its path depended on the timing of other insertions.
template <int B, int POL, bool GHOST>
__device__ __forceinline__ int insert_one(const DevTable& t, Ctx& c, uint8_t* region, uint32_t& aborts,
                                          uint64_t* local_e, int local_cap, bool retry_failed = false) {
  c.long_id = -1;
  c.big_id = -1;
  int st;
  uint32_t fails = 0;
  for (uint32_t attempt = 0;;) {
    c.attempt = attempt;
    c.kicks = 0;
    c.draws = 0;
    c.viewed0 = c.viewed;
    c.ghosts_made = 0;
    c.dup_evict = 0;
    c.foreign = 0;
    c.capped = 0;
    if (c.long_id < 0) {
      c.pe = local_e;
      c.pcap = local_cap;
    }
    c.pn = 0;
    st = attempt_insert<B, POL, GHOST>(t, c, region);
    bool undone = false;
    if (st == ST_OK) {
      if (commit<B>(t, c)) break;
      st = ST_CONFLICT;  // a slot no longer held what the plan expected: its writes were undone
      undone = true;
    }
    release_all(t, c, undone);
    if (st == ST_LONG) {  // a search path longer than the local plan
      if (c.long_id >= 0 || !grow_plan(t, c)) { st = c.long_id >= 0 ? ST_FAILED : ST_ABORTED; break; }
      continue;
    }
    // a walk or search that ran out is retried at most six times, or 32
    // times while it meets other insertions' claims on the way (they
    // finish meanwhile); then the key is FAILED
    const bool ran_out = st == ST_FAILED || (st == ST_CONFLICT && c.capped);
    if (ran_out) {
      if (!retry_failed || ++fails > (st == ST_FAILED ? 6u : 32u)) {
        st = ST_FAILED;
        break;
      }
      // a search out of budget tries again in a larger space (search_space)
      if (region && c.big_id < 0 && (POL == P_BFS || POL == P_SORTED || POL == P_HYBRID)) {
        c.big_id = acquire_long(t, c.key ^ 0x5bd1e995u);
        if (c.big_id >= 0) {
          uint64_t* vis = reinterpret_cast<uint64_t*>(t.long_scratch + (uint64_t)c.big_id * LONG_REGION + SEARCH_HDR +
                                                      BIG_GROUPS * sizeof(Group));
          for (int i = 0; i < BIG_VISITED; i++) vis[i] = 0;  // the region held a plan: no stale tags
        }
      }
    } else {
      aborts++;
    }
    if (++attempt >= t.max_retries) { st = ST_ABORTED; break; }
    // a failed attempt waits longer before its retry: the walks and claims
    // of the insertions around it, which made it fail, finish meanwhile
    backoff(ran_out ? 6 + 2 * fails : attempt, c.key);
  }
  if (c.long_id >= 0) release_long(t, c.long_id);
  if (c.big_id >= 0) release_long(t, c.big_id);
  return st;
}

// ------------------------------------------------------------------
// deletes (Sec. 1): every copy goes, each under its claim flag (Sec. 8)
// ------------------------------------------------------------------
// The copies a delete removes (at most d bins of B slots).
struct DelPlan {
  uint32_t bin[16];
  uint8_t slot[16];
  uint8_t old_r[16];  // two-choice: duplicate mark; d-ary: rattle counter
  uint64_t rec;       // the record the copies held when viewed (every copy holds the same)
  int n;
};

// Replace the record in every claimed copy of p by `to`, each by a 64-bit
// compare-and-swap from the record seen when the copies were viewed: a
// claim validates a view through the metadata word only, and that word can
// come back to an earlier value.  If a copy no longer holds the record, the
// copies already replaced get it back and the call returns false.
template <int B>
__device__ __forceinline__ bool swap_copies(const DevTable& t, const DelPlan& p, uint64_t to) {
  int done = 0;
  for (; done < p.n; done++)
    if (!cas_slot(t.slots + (uint64_t)p.bin[done] * B + p.slot[done], p.rec, to)) break;
  if (done == p.n) return true;
  for (int i = 0; i < done; i++) st_slot(t.slots + (uint64_t)p.bin[i] * B + p.slot[i], p.rec);
  fence_release();
  return false;
}

// One delete: find the key in its bins and claim the slots holding it
// (every copy: a ghost pair has two), clear them, release.  A miss is
// reported only when the bins were seen unclaimed and unchanged across the
// read (unchanged_since), so a delete running beside insertions on another
// stream never misses a key that is being moved.  Slots claimed by a
// writer are waited out with backoff, at most DELETE_ATTEMPTS times
// (status 2).
constexpr int DELETE_ATTEMPTS = 1024;

template <int B>
__device__ __forceinline__ int delete_one(const DevTable& t, uint32_t key, DelPlan& p, uint32_t& ghost_removed) {
  uint32_t b[4];
  bins_of(t, key, b);
  const uint32_t nb = t.d;
  constexpr uint32_t CLAIM_BITS = (1u << B) - 1;
  for (int attempt = 0; attempt < DELETE_ATTEMPTS; attempt++) {
    p.n = 0;
    bool conflict = false, any = false;
    int dup_copies = 0;
    uint32_t seen[4];
    for (uint32_t j = 0; j < nb && !conflict; j++) {
      View<B> v;
      load_view<B>(t, b[j], v);
      uint32_t m = v.m;
      seen[j] = m;
      uint32_t add = 0;
#pragma unroll
      for (int s = 0; s < B; s++) {
        if (v.s[s] != EMPTY && key_of(v.s[s]) == key) {
          if ((m >> s) & 1u) { conflict = true; break; }  // a writer holds it
          add |= 1u << s;
        }
      }
      if (conflict || !add) continue;
      uint64_t r0 = slot_of<B>(v, lowest(add));
      if (any && r0 != p.rec) { conflict = true; break; }  // copies that differ: a writer is active
      if (!cas_acquire(t.meta + b[j], m, m + add)) { conflict = true; break; }
      any = true;
      p.rec = r0;
      for (int s = 0; s < B; s++) {
        if ((add >> s) & 1u) {
          int i = p.n++;
          p.bin[i] = b[j];
          p.slot[i] = (uint8_t)s;
          p.old_r[i] = (uint8_t)((B == 1) ? rattle_of(m) : ((m >> (DUP_SHIFT + s)) & 1u));
          dup_copies += (B > 1) ? p.old_r[i] : 0;
        }
      }
    }
    if (!conflict && !any) {
      if (unchanged_since(t.meta, b, seen, nb, CLAIM_BITS)) return 0;
      conflict = true;  // a writer was active in the key's bins: look again
    }
    bool undone = false;
    if (!conflict && !swap_copies<B>(t, p, EMPTY)) conflict = undone = true;
    if (conflict) {
      for (int i = 0; i < p.n; i++) add_relaxed(t.meta + p.bin[i], (undone ? VER_ONE : 0u) - (1u << p.slot[i]));
      p.n = 0;
      uint32_t w = 128u << (attempt < 13 ? attempt : 13);
      __nanosleep(w + (fmix32(key ^ attempt) & (w - 1)));
      continue;
    }
    for (int i = 0; i < p.n; i++) {
      uint32_t delta = VER_ONE - (1u << p.slot[i]);
      if (B == 1) delta -= (uint32_t)p.old_r[i] << RATTLE_SHIFT;        // the bin forgets r(x)
      else if (p.old_r[i]) delta -= 1u << (DUP_SHIFT + p.slot[i]);       // duplicate mark goes too
      add_release(t.meta + p.bin[i], delta);
    }
    ghost_removed += dup_copies >= 2 ? 1 : 0;
    return 1;
  }
  return 2;
}

// Overwrite the value of a present key (CK_INS_UPSERT): claim every slot
// holding it (both copies of a ghost pair), store the new record, release
// with a version bump; the duplicate marks stay.  Returns 1 if updated, 0 if
// the key is absent (a miss proven as delete_one proves it), 2 if claimed
// slots were not released within DELETE_ATTEMPTS tries.
template <int B>
__device__ __forceinline__ int update_one(const DevTable& t, uint32_t key, uint64_t rec, DelPlan& p) {
  uint32_t b[4];
  bins_of(t, key, b);
  const uint32_t nb = t.d;
  constexpr uint32_t CLAIM_BITS = (1u << B) - 1;
  for (int attempt = 0; attempt < DELETE_ATTEMPTS; attempt++) {
    p.n = 0;
    bool conflict = false, any = false;
    uint32_t seen[4];
    for (uint32_t j = 0; j < nb && !conflict; j++) {
      View<B> v;
      load_view<B>(t, b[j], v);
      uint32_t m = v.m;
      seen[j] = m;
      uint32_t add = 0;
#pragma unroll
      for (int s = 0; s < B; s++) {
        if (v.s[s] != EMPTY && key_of(v.s[s]) == key) {
          if ((m >> s) & 1u) { conflict = true; break; }  // a writer holds it
          add |= 1u << s;
        }
      }
      if (conflict || !add) continue;
      uint64_t r0 = slot_of<B>(v, lowest(add));
      if (any && r0 != p.rec) { conflict = true; break; }  // copies that differ: a writer is active
      if (!cas_acquire(t.meta + b[j], m, m + add)) { conflict = true; break; }
      any = true;
      p.rec = r0;
      for (int s = 0; s < B; s++) {
        if ((add >> s) & 1u) {
          int i = p.n++;
          p.bin[i] = b[j];
          p.slot[i] = (uint8_t)s;
        }
      }
    }
    if (!conflict && !any) {
      if (unchanged_since(t.meta, b, seen, nb, CLAIM_BITS)) return 0;
      conflict = true;
    }
    bool undone = false;
    if (!conflict && !swap_copies<B>(t, p, rec)) conflict = undone = true;
    if (conflict) {
      for (int i = 0; i < p.n; i++) add_relaxed(t.meta + p.bin[i], (undone ? VER_ONE : 0u) - (1u << p.slot[i]));
      p.n = 0;
      uint32_t w = 128u << (attempt < 13 ? attempt : 13);
      __nanosleep(w + (fmix32(key ^ attempt) & (w - 1)));
      continue;
    }
    fence_release();
    for (int i = 0; i < p.n; i++) red_relaxed(t.meta + p.bin[i], VER_ONE - (1u << p.slot[i]));
    return 1;
  }
  return 2;
}

// Insert kernel.  Concurrent mode: each block takes a contiguous range of
// the batch and its threads pull keys from it, one insertion per thread at
// a time, plans in local memory.  Serial mode (SERIAL, one
// thread): keys in batch order, one insertion in flight, a scratch-backed
// plan; this replays the paper's serial algorithms exactly.
//
// Consecutive insert launches may overlap (programmatic dependent launch):
// each block lets the next launch start at once, and each thread waits for
// the previous launch to finish before it exits, so a launch completes only
// after its predecessor.  Insertions of distinct absent keys commute under
// the claim protocol, so the overlap changes no result.  `load_base` is the
// number of keys the table held before this batch (for the histogram).
// Registers: at most 64 (4 blocks of 256 or 8 of 128 threads per SM) for
// most policies, 80 for 4-slot queue-kicking (3 blocks of 256).  Measured on
// one GB300, fill of 2^24 x 4 to 0.95: queue-kicking 10.36-10.52 ms at 80
// registers (no spills) vs 10.56-10.74 at 64 (92 bytes spilled); random
// kicking 25.1 ms at 80 vs 24.0-24.4 at 64: the kernel is bound by random
// accesses in flight, and only the queue kernel's spills cost more than the
// warps a larger register file takes away.
template <int B, int POL>
constexpr int insert_blocks_per_sm() { return (B == 4 && POL == P_QUEUE) ? 3 : 4; }

template <int B, int POL, bool GHOST, bool SERIAL>
__global__ void __launch_bounds__(256, insert_blocks_per_sm<B, POL>()) k_insert(DevTable t, const uint32_t* __restrict__ keys,
                                                const uint32_t* __restrict__ vals, uint64_t n,
                                                uint8_t* __restrict__ status,
                                                uint32_t* __restrict__ viewed_out, uint64_t load_base,
                                                uint32_t upsert) {
  asm volatile("griddepcontrol.launch_dependents;");
  __shared__ unsigned int h_views[HIST_BUCKETS];
  __shared__ unsigned int h_cnt[HIST_BUCKETS];
  __shared__ unsigned int h_chain[CHAIN_BUCKETS];
  __shared__ unsigned long long bc[C_N];
  __shared__ unsigned long long s_next;  // next key of this block's range
  __shared__ int s_slab[SLABS_PER_BLOCK], s_long;
  for (int i = threadIdx.x; i < HIST_BUCKETS; i += blockDim.x) h_views[i] = h_cnt[i] = 0;
  for (int i = threadIdx.x; i < CHAIN_BUCKETS; i += blockDim.x) h_chain[i] = 0;
  for (int i = threadIdx.x; i < C_N; i += blockDim.x) bc[i] = 0;
  // each block owns a contiguous range of the batch; its threads pull keys
  // from it one at a time, so a thread held up by a long chain does not
  // hold up the others
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t lo = min(n, (uint64_t)blockIdx.x * per), hi = min(n, lo + per);
  if (threadIdx.x == 0) {
    s_next = lo;
    const int need = (int)((blockDim.x + SLAB - 1) / SLAB);
    if (!t.scratch || !acquire_slabs(t, s_slab, need)) s_slab[0] = -1;
    s_long = SERIAL ? acquire_long(t, 0) : -1;
  }
  __syncthreads();

  PlanStore<SERIAL ? 1 : MAX_CHAIN> store;
  uint64_t* local_e = store.e;
  int local_cap = SERIAL ? 1 : MAX_CHAIN;
  bool usable = true;
  if (SERIAL) {
    if (s_long >= 0) {
      local_e = reinterpret_cast<uint64_t*>(t.long_scratch + (uint64_t)s_long * LONG_REGION);
      local_cap = LONG_CHAIN;
    } else {
      usable = false;
    }
  }
  uint8_t* region = s_slab[0] >= 0 ? t.scratch + ((uint64_t)s_slab[threadIdx.x / SLAB] * SLAB + threadIdx.x % SLAB) *
                                                   SEARCH_REGION
                                   : nullptr;
  if (t.scratch && !region) usable = false;
  const unsigned long long size_base = load_base;

  // per-thread tallies of the counts every key adds to (32-bit: a thread
  // handles far fewer than 2^32 keys or bin views in one launch), flushed
  // into the block's 64-bit counters at the end; the rarer counts go to the
  // block's counters as they happen, which keeps them out of registers for
  // the whole loop
  uint32_t ok = 0, viewed = 0, viewed_all = 0;
  for (;;) {
    uint64_t i = atomicAdd(&s_next, 1ull);
    if (i >= hi) break;
    uint32_t key = keys[i];
    if (key == RESERVED_KEY) {
      if (status) status[i] = ST_INVALID;
      if (viewed_out) viewed_out[i] = 0;
      continue;
    }
    Ctx c;
    c.key = key;
    c.krec = ((uint64_t)key << 32) | vals[i];
    if (upsert) {  // a present key is overwritten in place, not inserted again
      DelPlan up;
      int r = update_one<B>(t, key, c.krec, up);
      if (r != 0) {
        atomicAdd(&bc[r == 1 ? C_UPDATES : C_INS_ABORTED], 1ull);
        if (status) status[i] = (uint8_t)(r == 1 ? ST_UPDATED : ST_ABORTED);
        if (viewed_out) viewed_out[i] = 0;
        continue;
      }
    }
    c.viewed = 0;
    c.reviews = 0;
    uint32_t aborts = 0;
    // concurrent mode retries a failed attempt (up to three times): other
    // insertions moved records meanwhile, so the next walk or search differs;
    // the serial replay never retries
    int st = usable ? insert_one<B, POL, GHOST>(t, c, region, aborts, local_e, local_cap, !SERIAL)
                    : (int)ST_ABORTED;
    if (st == ST_OK) {
      ok++;
      if (c.kicks) {
        atomicAdd(&bc[C_KICKS], (unsigned long long)c.kicks);
        atomicMax(&bc[C_CHAIN_MAX], (unsigned long long)c.kicks);
      }
      atomicAdd(&h_chain[chain_bucket(c.kicks)], 1u);
      if (c.ghosts_made) atomicAdd(&bc[C_GHOSTS_MADE], (unsigned long long)c.ghosts_made);
      if (c.dup_evict) atomicAdd(&bc[C_DUP_EVICT], (unsigned long long)c.dup_evict);
    } else {
      atomicAdd(&bc[st == ST_FAILED ? C_INS_FAILED : C_INS_ABORTED], 1ull);
    }
    if (aborts) atomicAdd(&bc[C_ABORTS], (unsigned long long)aborts);
    if (c.reviews) atomicAdd(&bc[C_REVIEWS], (unsigned long long)c.reviews);
    // bins viewed by the attempt that was applied (or failed), and by all
    // attempts including those abandoned after claim conflicts
    uint32_t v_final = c.viewed - c.viewed0;
    viewed += v_final;
    viewed_all += c.viewed;
    if (status) status[i] = (uint8_t)st;
    if (viewed_out) viewed_out[i] = v_final;
    uint64_t bucket = ((size_base + i) * HIST_BUCKETS) / t.total_slots;
    if (bucket >= HIST_BUCKETS) bucket = HIST_BUCKETS - 1;
    atomicAdd(&h_views[bucket], v_final);
    atomicAdd(&h_cnt[bucket], 1u);
  }
  flush_counter(&bc[C_INS_OK], ok);
  flush_counter(&bc[C_VIEWED], viewed);
  flush_counter(&bc[C_VIEWED_ALL], viewed_all);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < C_N; k++) {
      if (!bc[k]) continue;
      if (k == C_CHAIN_MAX) atomicMax(t.counters + k, bc[k]);
      else atomicAdd(t.counters + k, bc[k]);
    }
    // size and live ghosts follow from the counts above
    if (bc[C_INS_OK]) atomicAdd(t.counters + C_SIZE, bc[C_INS_OK]);
    long long dg = (long long)bc[C_GHOSTS_MADE] - (long long)bc[C_DUP_EVICT];
    if (dg) atomicAdd(t.counters + C_LIVE_GHOSTS, (unsigned long long)dg);
  }
  unsigned long long* hist = t.counters + C_N;
  for (int i = threadIdx.x; i < HIST_BUCKETS; i += blockDim.x) {
    if (h_cnt[i]) {
      atomicAdd(hist + i, (unsigned long long)h_views[i]);
      atomicAdd(hist + HIST_BUCKETS + i, (unsigned long long)h_cnt[i]);
    }
  }
  for (int i = threadIdx.x; i < CHAIN_BUCKETS; i += blockDim.x)
    if (h_chain[i]) atomicAdd(t.counters + CHAIN_HIST + i, (unsigned long long)h_chain[i]);
  if (threadIdx.x == 0) {
    if (s_slab[0] >= 0) {
      __threadfence();
      for (int j = 0; j < (int)((blockDim.x + SLAB - 1) / SLAB); j++) atomicExch(t.slab_busy + s_slab[j], 0u);
    }
    if (s_long >= 0) release_long(t, s_long);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------
// lookups (Sec. 1: a present key sits in one of its d bins)
// ------------------------------------------------------------------

// Read-only 32-byte sector load through the non-coherent path: lookups run
// with no writer in flight on the table.
__device__ __forceinline__ void ld_bin4_nc(const uint64_t* p, uint64_t* s) {
  asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3]) : "l"(p));
}

__device__ __forceinline__ uint64_t ld_slot_nc(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.global.nc.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

template <int B>
__device__ __forceinline__ bool match_bin(const uint64_t* s, uint32_t key, uint32_t& val) {
  bool f = false;
#pragma unroll
  for (int q = 0; q < B; q++) {
    if (!f && key_of(s[q]) == key) { f = true; val = (uint32_t)s[q]; }
  }
  return f;
}

template <int B>
__device__ __forceinline__ void load_bin_nc(const DevTable& t, uint32_t bin, uint64_t* s) {
  const uint64_t* p = t.slots + (uint64_t)bin * B;
#pragma unroll
  for (int q = 0; q < B; q += 4) ld_bin4_nc(p + q, s + q);
}

// Two-choice lookup: both bins are fetched at once (two independent sector
// loads in flight per key).
template <int B>
__global__ void __launch_bounds__(256) k_lookup2(DevTable t, const uint32_t* __restrict__ keys, uint64_t n,
                                                 uint32_t* __restrict__ vals_out,
                                                 uint8_t* __restrict__ found_out) {
  __shared__ unsigned long long hits_sh, cnt_sh;
  if (threadIdx.x == 0) hits_sh = cnt_sh = 0;
  __syncthreads();
  uint32_t hits = 0, cnt = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t key = __ldcs(keys + i);
    uint32_t val = 0;
    bool f = false;
    if (key != RESERVED_KEY) {
      uint32_t b0, b1;
      bins2(t, key, b0, b1);
      uint64_t s0[B], s1[B];
      load_bin_nc<B>(t, b0, s0);
      load_bin_nc<B>(t, b1, s1);
      f = match_bin<B>(s0, key, val);
      if (!f) f = match_bin<B>(s1, key, val);
    }
    hits += f;
    cnt++;
    if (vals_out) __stcs(vals_out + i, val);
    if (found_out) __stcs(found_out + i, (uint8_t)f);
  }
  hits = __reduce_add_sync(0xffffffffu, hits);
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0) {
    if (hits) atomicAdd(&hits_sh, (unsigned long long)hits);
    if (cnt) atomicAdd(&cnt_sh, (unsigned long long)cnt);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (hits_sh) atomicAdd(t.counters + C_LOOKUP_HITS, hits_sh);
    if (cnt_sh) atomicAdd(t.counters + C_LOOKUPS, cnt_sh);
  }
}

// d-ary lookup: the d single-slot bins are fetched at once.
static __global__ void __launch_bounds__(256) k_lookup_dary(DevTable t, const uint32_t* __restrict__ keys, uint64_t n,
                                                     uint32_t* __restrict__ vals_out,
                                                     uint8_t* __restrict__ found_out) {
  __shared__ unsigned long long hits_sh, cnt_sh;
  if (threadIdx.x == 0) hits_sh = cnt_sh = 0;
  __syncthreads();
  uint32_t hits = 0, cnt = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t key = __ldcs(keys + i);
    uint32_t val = 0;
    bool f = false;
    if (key != RESERVED_KEY) {
      uint32_t b[4];
      bins_of(t, key, b);
      uint64_t s[4];
#pragma unroll
      for (int j = 0; j < 4; j++) s[j] = j < (int)t.d ? ld_slot_nc(t.slots + b[j]) : EMPTY;
#pragma unroll
      for (int j = 0; j < 4; j++)
        if (!f && key_of(s[j]) == key) { f = true; val = (uint32_t)s[j]; }
    }
    hits += f;
    cnt++;
    if (vals_out) __stcs(vals_out + i, val);
    if (found_out) __stcs(found_out + i, (uint8_t)f);
  }
  hits = __reduce_add_sync(0xffffffffu, hits);
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0) {
    if (hits) atomicAdd(&hits_sh, (unsigned long long)hits);
    if (cnt) atomicAdd(&cnt_sh, (unsigned long long)cnt);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (hits_sh) atomicAdd(t.counters + C_LOOKUP_HITS, hits_sh);
    if (cnt_sh) atomicAdd(t.counters + C_LOOKUPS, cnt_sh);
  }
}

template <int B>
__global__ void __launch_bounds__(256) k_delete(DevTable t, const uint32_t* __restrict__ keys, uint64_t n,
                                                uint8_t* __restrict__ found_out) {
  __shared__ unsigned long long bc[4];
  if (threadIdx.x < 4) bc[threadIdx.x] = 0;
  __syncthreads();
  DelPlan p;
  uint32_t hits = 0, aborts = 0, ghosts = 0, cnt = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t key = keys[i];
    int r = key == RESERVED_KEY ? 0 : delete_one<B>(t, key, p, ghosts);
    hits += r == 1;
    aborts += r == 2;
    cnt++;
    if (found_out) found_out[i] = (uint8_t)r;
  }
  if (hits) atomicAdd(&bc[0], (unsigned long long)hits);
  if (aborts) atomicAdd(&bc[1], (unsigned long long)aborts);
  if (ghosts) atomicAdd(&bc[2], (unsigned long long)ghosts);
  if (cnt) atomicAdd(&bc[3], (unsigned long long)cnt);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bc[0]) {
      atomicAdd(t.counters + C_DELETE_HITS, bc[0]);
      atomicAdd(t.counters + C_SIZE, 0ull - bc[0]);
    }
    if (bc[1]) atomicAdd(t.counters + C_DELETE_ABORTS, bc[1]);
    if (bc[2]) atomicAdd(t.counters + C_LIVE_GHOSTS, 0ull - bc[2]);
    if (bc[3]) atomicAdd(t.counters + C_DELETES, bc[3]);
  }
}

}  // namespace ck
