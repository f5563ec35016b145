// ck_device.cuh -- device-side building blocks of the GB300 cuckoo table:
// hashing, counter-based draws, bin views, claims and the back-to-front
// commit of a planned kick-out chain (Kuszmaul, arXiv:1605.05236, Sec. 1,
// Sec. 4-8).
//
// Memory layout of one table (all in HBM):
//   slots[n_bins * B]  uint64  key << 32 | value; all-ones = empty
//   meta[n_bins]       uint32  per-bin metadata word:
//       two-choice: bits 0-7 claim flags (Sec. 8), 8-15 duplicate marks
//       (Sec. 4), 16-19 spawn count (Sec. 5), 20-27 hit counter (Sec. 6),
//       28-31 version;  d-ary: bit 0 claim flag, bits 8-15 rattle counter of
//       the resident key (Sec. 7), 28-31 version.
//
// Every write to an occupied slot happens while its claim flag is held.  A
// claim is a compare-and-swap of the whole metadata word from the value read
// when the bin was viewed, so a successful claim also shows that nothing in
// the bin changed since the view -- every release adds one to the version
// field (the release also folds in the duplicate/rattle update of the slot),
// and the hit counter of queue-kicking moves on every insertion -- unless
// the word came back to the value seen (the 4-bit version wraps after 16
// releases).  The writes themselves are therefore 64-bit compare-and-swaps
// from the records the plan saw, undone if one fails, which closes that
// gap.  The metadata word is read with acquire semantics before the slots,
// so the slots seen are at least as new as that word.
#pragma once
#include <cstdint>
#include <cuda/atomic>

namespace ck {

constexpr uint64_t EMPTY = ~0ull;
constexpr uint32_t NO_BIN = 0xFFFFFFFFu;
constexpr uint32_t RESERVED_KEY = 0xFFFFFFFFu;

constexpr int MAX_B = 8;
constexpr int MAX_CHAIN = 512;    // plan entries kept in local memory by the concurrent kernel
constexpr int LONG_CHAIN = 4104;  // plan entries of a scratch-backed plan (walk cap <= 4096)
constexpr int LONG_REGION = 65792;  // bytes of one scratch plan (16 * LONG_CHAIN, 256-aligned)
constexpr int MAX_GROUPS = 512;   // bins a search can view (budget <= MAX_GROUPS)
constexpr int VISITED_SLOTS = 1024;
constexpr int SLAB = 64;          // search regions per slab (a block holds ceil(blockDim / SLAB) slabs)
constexpr int SLABS_PER_BLOCK = 4; // blockDim <= 256

constexpr uint32_t DUP_SHIFT = 8;
constexpr uint32_t SPAWN_SHIFT = 16;
constexpr uint32_t HIT_SHIFT = 20;
constexpr uint32_t VER_SHIFT = 28;
constexpr uint32_t RATTLE_SHIFT = 8;
constexpr uint32_t HIT_ONE = 1u << HIT_SHIFT;
constexpr uint32_t VER_ONE = 1u << VER_SHIFT;

enum Policy : uint32_t { P_RANDOM = 0, P_BFS = 1, P_SORTED = 2, P_QUEUE = 3, P_RATTLE = 4, P_HYBRID = 5 };
// ST_CONFLICT: a claim lost a race, retry; ST_LONG: the local plan is full,
// continue with a scratch-backed plan.
enum Status : int {
  ST_OK = 0, ST_FAILED = 1, ST_ABORTED = 2, ST_INVALID = 3, ST_UPDATED = 5, ST_CONFLICT = 100, ST_LONG = 101
};

// device counters (uint64 each)
enum Counter : int {
  C_INS_OK = 0, C_INS_FAILED, C_INS_ABORTED, C_VIEWED, C_KICKS, C_CHAIN_MAX, C_ABORTS,
  C_GHOSTS_MADE, C_DUP_EVICT, C_SIZE, C_LIVE_GHOSTS /* C_SIZE + 1 */, C_LOOKUPS, C_LOOKUP_HITS, C_DELETES,
  C_DELETE_HITS, C_DELETE_ABORTS, C_REVIEWS, C_VIEWED_ALL, C_UPDATES, C_N = 24
};
constexpr int HIST_BUCKETS = 200;
// chain-length histogram of successful insertions: kick-outs k < 32 exact,
// then one bucket per power of two (32-63, ..., 2048-4095), then >= 4096
constexpr int CHAIN_BUCKETS = 40;
// the counter block of a table: C_N counters, the bins-viewed histogram by
// load (2 x HIST_BUCKETS), the chain-length histogram
constexpr int COUNTER_WORDS = C_N + 2 * HIST_BUCKETS + CHAIN_BUCKETS;
constexpr int CHAIN_HIST = C_N + 2 * HIST_BUCKETS;

__host__ __device__ inline uint32_t chain_bucket(uint32_t kicks) {
  if (kicks < 32) return kicks;
  uint32_t lg = 31;
  while (!((kicks >> lg) & 1u)) lg--;  // floor(log2(kicks)), 5 <= lg <= 31
  uint32_t b = 27 + lg;
  return b < CHAIN_BUCKETS - 1 ? b : CHAIN_BUCKETS - 1;
}

struct DevTable {
  uint64_t* slots;
  uint32_t* meta;
  unsigned long long* counters;  // COUNTER_WORDS: C_N counters, then the histograms
  uint8_t* scratch;              // search scratch, SEARCH_REGION bytes per searcher
  uint8_t* long_scratch;         // n_long plans of LONG_REGION bytes
  uint32_t* long_busy;           // n_long flags: plan region in use
  uint32_t* slab_busy;           // n_searchers / SLAB flags: a block's slab of search regions is in use
  uint64_t n_bins;
  uint64_t total_slots;
  uint64_t rng_seed;
  uint32_t bin_mask;             // n_bins - 1 when n_bins is a power of two, else 0
  uint32_t B, d, policy, ghost;
  uint32_t cap, max_retries;
  uint32_t ordered_writes, tie_resident;
  uint32_t n_searchers;
  uint32_t n_long;
  uint32_t hash_family;          // 0: fmix32(k ^ seed_i); 1: decorrelated (see bin_hash)
  uint32_t spawn_k;              // searches: spawns per round, their bins fetched together (1..8)
  uint32_t seeds[4];
};

// ------------------------------------------------------------------
// hashing and draws
// ------------------------------------------------------------------

// MurmurHash3's 32-bit finalizer (Appleby, public domain).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// SplitMix64 output for generator state x (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Draw number `i` of the insertion of `key`, attempt `attempt`; attempt 0
// replays the serial order exactly.
__device__ __forceinline__ uint64_t draw(const DevTable& t, uint32_t key, uint32_t i, uint32_t attempt) {
  return splitmix64_at(t.rng_seed ^ (uint64_t)key ^ ((uint64_t)i << 32) ^ ((uint64_t)attempt << 48));
}

__device__ __forceinline__ uint32_t reduce_bin(const DevTable& t, uint32_t h) {
  return t.bin_mask ? (h & t.bin_mask) : (uint32_t)((uint64_t)h % t.n_bins);
}

__device__ __forceinline__ uint32_t next_bin(const DevTable& t, uint32_t b) {
  return (uint64_t)(b + 1) == t.n_bins ? 0u : b + 1;
}

// Hash i of a key.  Family 0: fmix32(key ^ seed_i), the stated workload's
// hash.  Its d functions are not independent: key ^ seed_i ^ seed_j has
// key's h_i and h_j swapped, so such pairs share two bins, which single-slot
// d-ary tables feel at scale.  Family 1 keeps fmix32 but decorrelates the
// functions: fmix32(fmix32(key + seed_i) ^ (seed_i * 0x27D4EB2F)), closer to
// the independent uniform hashes the paper assumes (Sec. 3).
__device__ __forceinline__ uint32_t bin_hash(const DevTable& t, uint32_t key, uint32_t i) {
  uint32_t s = t.seeds[i];
  return t.hash_family ? fmix32(fmix32(key + s) ^ (s * 0x27D4EB2Fu)) : fmix32(key ^ s);
}

// The d bins of a key: h_i mod n_bins; a choice equal to an earlier one
// moves to the next bin, so the choices are distinct (Sec. 1).
__device__ __forceinline__ void bins_of(const DevTable& t, uint32_t key, uint32_t* b) {
  b[0] = reduce_bin(t, bin_hash(t, key, 0));
  for (uint32_t i = 1; i < t.d; i++) {
    uint32_t x = reduce_bin(t, bin_hash(t, key, i));
    for (;;) {
      bool clash = false;
      for (uint32_t j = 0; j < i; j++) clash |= (b[j] == x);
      if (!clash) break;
      x = next_bin(t, x);
    }
    b[i] = x;
  }
}

__device__ __forceinline__ void bins2(const DevTable& t, uint32_t key, uint32_t& b0, uint32_t& b1) {
  b0 = reduce_bin(t, bin_hash(t, key, 0));
  b1 = reduce_bin(t, bin_hash(t, key, 1));
  if (b1 == b0) b1 = next_bin(t, b1);
}

__device__ __forceinline__ uint32_t key_of(uint64_t rec) { return (uint32_t)(rec >> 32); }

__device__ __forceinline__ uint32_t other_bin2(const DevTable& t, uint64_t rec, uint32_t here) {
  uint32_t b0, b1;
  bins2(t, key_of(rec), b0, b1);
  return b0 == here ? b1 : b0;
}

// ------------------------------------------------------------------
// memory access
// ------------------------------------------------------------------

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One 32-byte sector of four slots, relaxed at GPU scope (bypasses L1).
__device__ __forceinline__ void ld_bin4(const uint64_t* p, uint64_t* s) {
  asm volatile("ld.relaxed.gpu.global.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3]) : "l"(p) : "memory");
}

__device__ __forceinline__ uint64_t ld_slot(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_slot(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void fence_release() {
  cuda::atomic_thread_fence(cuda::memory_order_release, cuda::thread_scope_device);
}

__device__ __forceinline__ void fence_acquire() {
  cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// A read of a bin's slots that saw no claim bit in the bin's metadata word,
// and finds the word unchanged when it is read again after the slots, saw
// no key move: every move (a chain step, a delete) happens under a claim,
// and every release advances the bin's version.  The one write without a
// claim, a new key taking a free slot, adds a key and moves none.  This is
// how a miss is proven while insertions run (a key moving between its own
// bins is written to the new bin before it leaves the old one, but two
// separate reads can still fall on either side of the move).
__device__ __forceinline__ bool unchanged_since(const uint32_t* meta, const uint32_t* bins, const uint32_t* seen,
                                                uint32_t nb, uint32_t claim_bits) {
  fence_acquire();
  bool ok = true;
  for (uint32_t j = 0; j < nb; j++) {
    uint32_t now = ld_relaxed(meta + bins[j]);
    ok &= now == seen[j] && (seen[j] & claim_bits) == 0;
  }
  return ok;
}

__device__ __forceinline__ bool cas_acquire(uint32_t* p, uint32_t expected, uint32_t desired) {
  uint32_t old;
  asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;"
               : "=r"(old) : "l"(p), "r"(expected), "r"(desired) : "memory");
  return old == expected;
}

__device__ __forceinline__ uint32_t add_release(uint32_t* p, uint32_t delta) {
  cuda::atomic_ref<uint32_t, cuda::thread_scope_device> a(*p);
  return a.fetch_add(delta, cuda::memory_order_release);
}

// Fire-and-forget atomic add (no value returned).
// 64-bit compare-and-swap of one slot (relaxed): the unclaimed placement
// of a new key into a free slot, and a chain's write of its terminal free
// slot, both of which must not overwrite a key another thread placed there.
__device__ __forceinline__ uint64_t cas_slot_old(uint64_t* p, uint64_t expected, uint64_t desired) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(old) : "l"(p), "l"(expected), "l"(desired) : "memory");
  return old;
}

__device__ __forceinline__ bool cas_slot(uint64_t* p, uint64_t expected, uint64_t desired) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(old) : "l"(p), "l"(expected), "l"(desired) : "memory");
  return old == expected;
}

__device__ __forceinline__ void red_relaxed(uint32_t* p, uint32_t delta) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(delta) : "memory");
}

__device__ __forceinline__ uint32_t add_relaxed(uint32_t* p, uint32_t delta) {
  cuda::atomic_ref<uint32_t, cuda::thread_scope_device> a(*p);
  return a.fetch_add(delta, cuda::memory_order_relaxed);
}

// A view of one bin: its metadata word, then its B slots.
template <int B>
struct View {
  uint64_t s[B];
  uint32_t m;
};

template <int B>
__device__ __forceinline__ void load_view(const DevTable& t, uint32_t bin, View<B>& v) {
  v.m = ld_acquire(t.meta + bin);
  const uint64_t* p = t.slots + (uint64_t)bin * B;
  if constexpr (B == 1) {
    v.s[0] = ld_slot(p);
  } else {
#pragma unroll
    for (int q = 0; q < B; q += 4) ld_bin4(p + q, v.s + q);
  }
}

template <int B>
__device__ __forceinline__ void load_slots(const DevTable& t, uint32_t bin, View<B>& v) {
  const uint64_t* p = t.slots + (uint64_t)bin * B;
  if constexpr (B == 1) {
    v.s[0] = ld_slot(p);
  } else {
#pragma unroll
    for (int q = 0; q < B; q += 4) ld_bin4(p + q, v.s + q);
  }
}

// A view without ordering between the metadata word and the slots, in one
// round trip.  Insertions plan on such views: a free slot they take is
// written by a compare-and-swap from empty, and every record they move is
// read again after its claim (reread) -- so a view whose slots are older or
// newer than its word costs a retry, never a wrong move.  Deletes, which
// prove misses from their views, use load_view.
template <int B>
__device__ __forceinline__ void load_view_fast(const DevTable& t, uint32_t bin, View<B>& v) {
  v.m = ld_relaxed(t.meta + bin);
  load_slots<B>(t, bin, v);
}

// Views of a key's two bins in one round trip (unordered, as load_view_fast).
template <int B>
__device__ __forceinline__ void load_view2_fast(const DevTable& t, uint32_t b0, uint32_t b1, View<B>& v0,
                                                View<B>& v1) {
  v0.m = ld_relaxed(t.meta + b0);
  v1.m = ld_relaxed(t.meta + b1);
  load_slots<B>(t, b0, v0);
  load_slots<B>(t, b1, v1);
}

// Slot s of a view, s known only at run time: a chain of selects keeps the
// view in registers (indexing the array would move it to local memory).
template <int B>
__device__ __forceinline__ uint64_t slot_of(const View<B>& v, int s) {
  uint64_t r = v.s[0];
#pragma unroll
  for (int q = 1; q < B; q++) r = (s == q) ? v.s[q] : r;
  return r;
}

// slot predicates on a view (claim bits cover every in-flight writer)
template <int B>
__device__ __forceinline__ uint32_t claimed_mask(const View<B>& v) { return v.m & ((1u << B) - 1); }

template <int B>
__device__ __forceinline__ uint32_t free_mask(const View<B>& v) {
  uint32_t m = 0;
#pragma unroll
  for (int s = 0; s < B; s++) m |= (v.s[s] == EMPTY ? 1u : 0u) << s;
  return m & ~claimed_mask(v);
}

// Empty slots whatever their claim bits (a view that read no metadata word).
template <int B>
__device__ __forceinline__ uint32_t empty_mask(const View<B>& v) {
  uint32_t m = 0;
#pragma unroll
  for (int s = 0; s < B; s++) m |= (v.s[s] == EMPTY ? 1u : 0u) << s;
  return m;
}

template <int B>
__device__ __forceinline__ uint32_t dup_mask(const View<B>& v) {
  uint32_t m = 0;
#pragma unroll
  for (int s = 0; s < B; s++) m |= (v.s[s] != EMPTY ? 1u : 0u) << s;
  return m & (v.m >> DUP_SHIFT) & ~claimed_mask(v) & ((1u << B) - 1);
}

__device__ __forceinline__ int lowest(uint32_t mask) { return mask ? __ffs(mask) - 1 : -1; }

// first set bit of `mask` at or after `start`, cyclically over B bits
template <int B>
__device__ __forceinline__ int first_from(uint32_t mask, uint32_t start) {
  uint32_t rot = ((mask >> start) | (mask << (B - start))) & ((1u << B) - 1);
  if (!rot) return -1;
  return (int)((start + (__ffs(rot) - 1)) % B);
}

// i-th set bit (0-based) of a mask
__device__ __forceinline__ int nth_bit(uint32_t mask, uint32_t i) {
  for (uint32_t k = 0; k < i; k++) mask &= mask - 1;
  return __ffs(mask) - 1;
}

__device__ __forceinline__ uint32_t spawn_of(uint32_t m) { return (m >> SPAWN_SHIFT) & 15u; }
__device__ __forceinline__ uint32_t hit_of(uint32_t m) { return (m >> HIT_SHIFT) & 255u; }
__device__ __forceinline__ uint32_t rattle_of(uint32_t m) { return (m >> RATTLE_SHIFT) & 255u; }

}  // namespace ck
