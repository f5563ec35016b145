// ck_warp.cuh -- breadth-first search by a whole warp (Kuszmaul,
// arXiv:1605.05236, Sec. 5), for two-choice tables without ghosts: the
// CK_PARAM_SEARCH_WARP form of CK_BFS.
//
// Each lane inserts its own key as in k_insert: it views the key's two
// bins and takes a free slot if there is one.  A key whose bins are both
// full is searched for by all 32 lanes together, one key at a time: the
// candidates of the breadth-first order (the records of the groups, a
// group per bin viewed, groups in viewing order, a group's records in slot
// order) are taken 32 at a time, one per lane; each lane computes its
// record's other bin, drops it if a group already holds that bin or an
// earlier lane of the round spawns the same bin (__match_any_sync), and
// views it; the lowest lane whose bin has a free slot ends the search
// (__ballot_sync), so the path found is the one the serial search finds
// when nothing changes meanwhile.  The groups live in shared memory (bin,
// metadata word as viewed, parent, and the other bin of each record, taken
// from the view), so a search reads and writes nothing but the table.
//
// A round views every candidate of its 32 that spawns, also those after
// the lane that ends the search: this form views more bins than the serial
// search (counted as viewed), and in exchange takes one round trip for up
// to 32 of them.  The owner lane claims the path and its terminal exactly
// as the per-thread search does (ck_search.cuh) and commits with the same
// code.  A search that needs more groups than shared memory holds (128),
// runs out of budget, or finds no way on (with other insertions' claims in
// its path or not) is handed to the per-thread search, with that search's
// retries (in a larger space), so every key ends as it would in k_insert.
#pragma once
#include "ck_kernels.cuh"

namespace ck {

// groups one warp search keeps in shared memory: 128 keeps the 4-slot
// kernel at 8 blocks (32 warps) per SM; 256 (6 blocks) made the 2^24 x 4
// BFS fill with the warp form 14% slower
template <int B>
__host__ __device__ constexpr int warp_groups() { return 128; }
constexpr unsigned FULL_MASK = 0xFFFFFFFFu;
constexpr int WARP_BLOCK = 128;        // threads per block of k_insert_warp

template <int B>
struct WarpGroups {
  uint32_t bin[warp_groups<B>()];
  uint32_t meta[warp_groups<B>()];     // metadata word as viewed
  uint16_t par[warp_groups<B>()];      // (group << 3) | slot of the record that led here; NO_PARENT at a root
  uint32_t y[warp_groups<B>() * B];    // other bin of each record, NO_BIN if the slot was empty (bins < 2^32 - 1)
  // each lane's two root groups, staged until its search (bins, words, other bins)
  uint32_t root_bin[64];
  uint32_t root_meta[64];
  uint32_t root_y[64 * B];
  // the view of the bin with room that ended the search
  uint64_t win_s[B];
  uint32_t win_m;
};

// The other bin of each record of a view (NO_BIN for an empty slot).
template <int B>
__device__ __forceinline__ void other_bins(const DevTable& t, uint32_t bin, const View<B>& v, uint32_t* y) {
#pragma unroll
  for (int q = 0; q < B; q++) y[q] = v.s[q] == EMPTY ? NO_BIN : other_bin2(t, v.s[q], bin);
}

// Group `g` of the search: bin `bin` as viewed in `v` (one lane writes it).
template <int B>
__device__ __forceinline__ void put_group(const DevTable& t, WarpGroups<B>& W, uint32_t g, uint32_t bin,
                                          const View<B>& v, uint32_t par) {
  W.bin[g] = bin;
  W.meta[g] = v.m;
  W.par[g] = (uint16_t)par;
  other_bins<B>(t, bin, v, W.y + g * B);
}

// Result of a warp search (the same in every lane).
struct WarpFound {
  int st;          // ST_OK: a path; ST_FAILED / ST_CONFLICT: none (claims seen: conflict); ST_LONG: too many groups
  uint32_t views;  // bins the search viewed
  int lane;        // ST_OK: the lane whose bin has room
  uint32_t g, s, y;  // ST_OK: the candidate (group, slot) and its bin y
};

// The search itself; roots (groups 0 and 1) already in W.  `used`: bins
// the attempt viewed before the search (the roots).  Every lane calls it.
template <int B>
__device__ __forceinline__ WarpFound warp_bfs(const DevTable& t, WarpGroups<B>& W, uint32_t used) {
  const uint32_t lane = threadIdx.x & 31u;
  View<B> vy;
  const uint32_t below = (1u << lane) - 1u;
  WarpFound f;
  f.views = 0;
  uint32_t ng = 2, c0 = 0, foreign = 0;
  for (;;) {
    const uint32_t cend = min(c0 + 32u, ng * (uint32_t)B);
    if (c0 >= cend) {  // no candidate left
      f.st = __any_sync(FULL_MASK, foreign) ? ST_CONFLICT : ST_FAILED;
      return f;
    }
    const uint32_t cand = c0 + lane;
    const uint32_t g = cand / B, s = cand % B;
    uint32_t y = NO_BIN;
    bool spawn = false;
    if (cand < cend) {
      if ((W.meta[g] >> s) & 1u) {
        foreign = 1;  // claimed by another insertion: ignore it (Sec. 8)
      } else {
        y = W.y[cand];
        spawn = y != NO_BIN;
      }
    }
    // a bin a group already holds was viewed before (the visited set)
    bool seen = false;
    for (uint32_t q = 0; q < ng; q++) seen |= W.bin[q] == y;
    spawn &= !seen;
    // among this round's candidates spawning the same bin, the first spawns
    const unsigned same = __match_any_sync(FULL_MASK, spawn ? (uint64_t)y : (1ull << 32) | lane);
    spawn &= (same & below) == 0;
    // the budget: spawns past it view nothing and end the search
    const unsigned sm0 = __ballot_sync(FULL_MASK, spawn);
    const uint32_t rank = __popc(sm0 & below);
    const bool cut = spawn && used + f.views + rank >= t.cap;
    spawn &= !cut;
    const bool any_cut = __any_sync(FULL_MASK, cut);
    bool room = false;
    if (spawn) {
      load_view_fast<B>(t, y, vy);
      if (claimed_mask<B>(vy)) foreign = 1;
      room = free_mask<B>(vy) != 0;
    }
    const unsigned sm = __ballot_sync(FULL_MASK, spawn);
    const unsigned rm = __ballot_sync(FULL_MASK, room);
    f.views += __popc(sm);
    if (rm) {
      f.st = ST_OK;
      f.lane = __ffs(rm) - 1;
      f.g = __shfl_sync(FULL_MASK, g, f.lane);
      f.s = __shfl_sync(FULL_MASK, s, f.lane);
      f.y = __shfl_sync(FULL_MASK, y, f.lane);
      if ((int)lane == f.lane) {
#pragma unroll
        for (int q = 0; q < B; q++) W.win_s[q] = vy.s[q];
        W.win_m = vy.m;
      }
      __syncwarp();
      return f;
    }
    // every spawned bin is full: each becomes a group, in candidate order
    const uint32_t n_new = __popc(sm);
    if (ng + n_new > (uint32_t)warp_groups<B>()) {
      f.st = ST_LONG;
      return f;
    }
    if (spawn) put_group<B>(t, W, ng + __popc(sm & below), y, vy, (g << 3) | s);
    __syncwarp();
    ng += n_new;
    if (any_cut) {
      f.st = __any_sync(FULL_MASK, foreign) ? ST_CONFLICT : ST_FAILED;
      return f;
    }
    c0 = cend;
  }
}

// The owner lane: claim the path root -> ... -> (g, s) in chain order from
// the metadata words as viewed, re-reading each claimed record (it must be
// the record the search saw: it belongs to the next bin of the path), then
// the free slot of y (as insert_search).
template <int B>
__device__ __forceinline__ int warp_claim_path(const DevTable& t, Ctx& c, const WarpGroups<B>& W,
                                               const WarpFound& f) {
  uint32_t depth = 1;
  for (uint32_t q = f.g; W.par[q] != NO_PARENT; q = W.par[q] >> 3) depth++;
  if ((int)depth + 4 > c.pcap) return ST_LONG;
  {
    uint32_t q = f.g, qs = f.s;
    for (int e = (int)depth - 1; e >= 0; e--) {
      set_entry(c, e, pack_entry(W.bin[q], (int)qs, K_MOVE, false, 0, 0), q);
      const uint32_t par = W.par[q];
      if (par != NO_PARENT) {
        qs = par & 7u;
        q = par >> 3;
      }
    }
  }
  c.pn = 0;
  for (uint32_t e = 0; e < depth; e++) {
    const uint32_t q = (uint32_t)content_at(c, (int)e);
    const uint32_t sl = e_slot(desc_at(c, (int)e));
    if (!cas_acquire(t.meta + W.bin[q], W.meta[q], W.meta[q] + (1u << sl))) return ST_CONFLICT;
    c.pn = (int)e + 1;
    const uint64_t r = reread<B>(t, W.bin[q], sl);
    const uint32_t to = e + 1 < depth ? W.bin[(uint32_t)content_at(c, (int)e + 1)] : f.y;
    set_content(c, (int)e, r);
    if (!belongs<B>(t, r, to)) return ST_CONFLICT;
  }
  c.kicks = depth;
  View<B> vy;
#pragma unroll
  for (int q = 0; q < B; q++) vy.s[q] = W.win_s[q];
  vy.m = W.win_m;
  return take_free<B>(t, c, f.y, vy, lowest(free_mask<B>(vy)), false);
}

// What the per-thread search did with a key the warp search handed over.
struct Handover {
  int st;
  uint32_t kicks, viewed, reviews, aborts;
};

// The per-thread insertion (k_insert's, with its larger-space retry) of a
// key whose warp search needed more groups than shared memory holds or ran
// out of budget.  Out of line: it is rare, and inlined it would hold its
// registers across the whole warp kernel.
template <int B>
__device__ __noinline__ Handover hand_over(const DevTable& t, uint32_t key, uint64_t krec, uint8_t* region,
                                           uint64_t* local_e) {
  Ctx c;
  c.key = key;
  c.krec = krec;
  c.viewed = 0;
  c.reviews = 0;
  uint32_t aborts = 0;
  Handover h;
  h.st = insert_one<B, P_BFS, false>(t, c, region, aborts, local_e, MAX_CHAIN, true);
  h.kicks = c.kicks;
  h.viewed = c.viewed;
  h.reviews = c.reviews;
  h.aborts = aborts;
  return h;
}

template <int B>
__global__ void __launch_bounds__(WARP_BLOCK, 8) k_insert_warp(DevTable t, const uint32_t* __restrict__ keys,
                                                               const uint32_t* __restrict__ vals, uint64_t n,
                                                               uint8_t* __restrict__ status,
                                                               uint32_t* __restrict__ viewed_out, uint64_t load_base) {
  asm volatile("griddepcontrol.launch_dependents;");
  __shared__ WarpGroups<B> ws[WARP_BLOCK / 32];
  __shared__ unsigned int h_views[HIST_BUCKETS];
  __shared__ unsigned int h_cnt[HIST_BUCKETS];
  __shared__ unsigned int h_chain[CHAIN_BUCKETS];
  __shared__ unsigned long long bc[C_N];
  __shared__ unsigned long long s_next;
  __shared__ int s_slab[SLABS_PER_BLOCK];
  for (int i = threadIdx.x; i < HIST_BUCKETS; i += blockDim.x) h_views[i] = h_cnt[i] = 0;
  for (int i = threadIdx.x; i < CHAIN_BUCKETS; i += blockDim.x) h_chain[i] = 0;
  for (int i = threadIdx.x; i < C_N; i += blockDim.x) bc[i] = 0;
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t lo = min(n, (uint64_t)blockIdx.x * per), hi = min(n, lo + per);
  if (threadIdx.x == 0) {
    s_next = lo;
    const int need = (int)((blockDim.x + SLAB - 1) / SLAB);
    if (!t.scratch || !acquire_slabs(t, s_slab, need)) s_slab[0] = -1;
  }
  __syncthreads();
  WarpGroups<B>& W = ws[threadIdx.x / 32];
  const uint32_t lane = threadIdx.x & 31u;
  PlanStore<MAX_CHAIN> store;
  uint8_t* region = s_slab[0] >= 0 ? t.scratch + ((uint64_t)s_slab[threadIdx.x / SLAB] * SLAB + threadIdx.x % SLAB) *
                                                   SEARCH_REGION
                                   : nullptr;

  uint32_t ok = 0, viewed = 0, viewed_all = 0;
  bool have = false;
  uint64_t i = 0;
  uint32_t attempt = 0, fails = 0, aborts = 0;
  Ctx c;
  for (;;) {
    int st = -1;  // the key's final status once known
    bool need = false;
    if (!have) {
      i = atomicAdd(&s_next, 1ull);
      have = i < hi;
      if (have) {
        const uint32_t key = keys[i];
        if (key == RESERVED_KEY) {
          if (status) status[i] = ST_INVALID;
          if (viewed_out) viewed_out[i] = 0;
          have = false;
        } else {
          c.key = key;
          c.krec = ((uint64_t)key << 32) | vals[i];
          c.viewed = 0;
          c.reviews = 0;
          c.long_id = -1;
          c.big_id = -1;
          attempt = 0;
          fails = 0;
          aborts = 0;
        }
      }
    }
    if (!__any_sync(FULL_MASK, have)) break;
    // one attempt per lane holding a key: its two bins, a free slot if any
    int at = -1;  // the attempt's outcome (ST_*), -1 while it waits for a search
    View<B> v0, v1;
    uint32_t b0 = 0, b1 = 0;
    if (have) {
      if (!region) {
        st = ST_ABORTED;
      } else {
        c.attempt = attempt;
        c.kicks = 0;
        c.draws = 0;
        c.viewed0 = c.viewed;
        c.ghosts_made = 0;
        c.dup_evict = 0;
        c.foreign = 0;
        c.capped = 0;
        c.pe = store.e;
        c.pcap = MAX_CHAIN;
        c.pn = 0;
        bins2(t, c.key, b0, b1);
        load_view_fast<B>(t, b0, v0);
        load_view_fast<B>(t, b1, v1);
        c.viewed += 2;
        const uint32_t g0 = free_mask<B>(v0), g1 = free_mask<B>(v1);
        if (g0) {
          at = place_direct<B>(t, c, b0, lowest(g0), false) ? (int)ST_OK : (int)ST_CONFLICT;
        } else if (g1) {
          at = place_direct<B>(t, c, b1, lowest(g1), false) ? (int)ST_OK : (int)ST_CONFLICT;
        } else {
          fence_acquire();
          load_slots<B>(t, b0, v0);
          load_slots<B>(t, b1, v1);
          const uint32_t f0 = free_mask<B>(v0), f1 = free_mask<B>(v1);
          if (f0) {
            at = take_free<B>(t, c, b0, v0, lowest(f0), false);
          } else if (f1) {
            at = take_free<B>(t, c, b1, v1, lowest(f1), false);
          } else {  // both full: stage the roots for the search
            need = true;
            W.root_bin[2 * lane] = b0;
            W.root_bin[2 * lane + 1] = b1;
            W.root_meta[2 * lane] = v0.m;
            W.root_meta[2 * lane + 1] = v1.m;
            other_bins<B>(t, b0, v0, W.root_y + 2 * lane * B);
            other_bins<B>(t, b1, v1, W.root_y + (2 * lane + 1) * B);
          }
        }
      }
    }
    // the searches, one key at a time, all lanes
    unsigned nm = __ballot_sync(FULL_MASK, need);
    __syncwarp();
    for (; nm; nm &= nm - 1) {
      const int L = __ffs(nm) - 1;
      if (lane < 2) {
        W.bin[lane] = W.root_bin[2 * L + lane];
        W.meta[lane] = W.root_meta[2 * L + lane];
        W.par[lane] = (uint16_t)NO_PARENT;
      }
      if (lane < 2 * B) W.y[lane] = W.root_y[2 * L * B + lane];
      __syncwarp();
      const uint32_t used = __shfl_sync(FULL_MASK, c.viewed - c.viewed0, L);
      const WarpFound f = warp_bfs<B>(t, W, used);
      if ((int)lane == L) {
        c.viewed += f.views;
        // a search that found nothing (claims seen on the way or not) or
        // outgrew shared memory goes to the per-thread search
        at = f.st == ST_OK ? warp_claim_path<B>(t, c, W, f) : f.st == ST_CONFLICT ? (int)ST_FAILED : f.st;
      }
      __syncwarp();
    }
    // finish the attempt as insert_one does
    if (have && st < 0) {
      bool undone = false;
      if (at == ST_OK) {
        if (commit<B>(t, c)) st = ST_OK;
        else {
          at = ST_CONFLICT;  // a slot no longer held what the plan expected: its writes were undone
          undone = true;
        }
      }
      if (st < 0) {
        release_all(t, c, undone);
        if (at == ST_LONG || at == ST_FAILED) {
          // the per-thread search takes over (with its larger-space retry)
          const Handover h = hand_over<B>(t, c.key, c.krec, region, store.e);
          st = h.st;
          c.kicks = h.kicks;
          c.viewed0 = c.viewed;
          c.viewed += h.viewed;
          c.reviews += h.reviews;
          aborts += h.aborts;
        } else {
          aborts++;
          if (++attempt >= t.max_retries) st = ST_ABORTED;
          else backoff(attempt, c.key);
        }
      }
    }
    if (have && st >= 0) {
      if (st == ST_OK) {
        ok++;
        if (c.kicks) {
          atomicAdd(&bc[C_KICKS], (unsigned long long)c.kicks);
          atomicMax(&bc[C_CHAIN_MAX], (unsigned long long)c.kicks);
        }
        atomicAdd(&h_chain[chain_bucket(c.kicks)], 1u);
      } else {
        atomicAdd(&bc[st == ST_FAILED ? C_INS_FAILED : C_INS_ABORTED], 1ull);
      }
      if (aborts) atomicAdd(&bc[C_ABORTS], (unsigned long long)aborts);
      if (c.reviews) atomicAdd(&bc[C_REVIEWS], (unsigned long long)c.reviews);
      const uint32_t v_final = c.viewed - c.viewed0;
      viewed += v_final;
      viewed_all += c.viewed;
      if (status) status[i] = (uint8_t)st;
      if (viewed_out) viewed_out[i] = v_final;
      uint64_t bucket = ((load_base + i) * HIST_BUCKETS) / t.total_slots;
      if (bucket >= HIST_BUCKETS) bucket = HIST_BUCKETS - 1;
      atomicAdd(&h_views[bucket], v_final);
      atomicAdd(&h_cnt[bucket], 1u);
      have = false;
    }
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
    if (bc[C_INS_OK]) atomicAdd(t.counters + C_SIZE, bc[C_INS_OK]);
  }
  unsigned long long* hist = t.counters + C_N;
  for (int k = threadIdx.x; k < HIST_BUCKETS; k += blockDim.x) {
    if (h_cnt[k]) {
      atomicAdd(hist + k, (unsigned long long)h_views[k]);
      atomicAdd(hist + HIST_BUCKETS + k, (unsigned long long)h_cnt[k]);
    }
  }
  for (int k = threadIdx.x; k < CHAIN_BUCKETS; k += blockDim.x)
    if (h_chain[k]) atomicAdd(t.counters + CHAIN_HIST + k, (unsigned long long)h_chain[k]);
  if (threadIdx.x == 0 && s_slab[0] >= 0) {
    __threadfence();
    for (int j = 0; j < (int)((blockDim.x + SLAB - 1) / SLAB); j++) atomicExch(t.slab_busy + s_slab[j], 0u);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace ck
