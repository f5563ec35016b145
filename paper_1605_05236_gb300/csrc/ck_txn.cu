// ck_txn.cu -- the transactional multi-writer cuckoo table of Sec. 8
// (Kuszmaul, arXiv:1605.05236): transactions of inserts, reads,
// overwrites and deletes under the SILO-style optimistic concurrency scheme
// the paper describes, with its abort-reducing mechanisms as switches: local
// retries, queue-kicking with hit counters, system-transaction kick-outs
// and claim flags.
//
// A table here is `trials` independent cuckoo tables of n bins x B slots
// (packed key << 32 | value, all-ones empty), run in one launch: the Sec. 8
// experiments average many trials, and on this GPU the trials run side by
// side.  Trial r hashes with its own salted seed pair, so its hash pairs are
// independent of the other trials'.
//
// Every slot and every bin has a 64-bit word: version << 2 | claim << 1 |
// lock (bins never carry a claim).  A version is the ID of the transaction
// that last wrote the slot or bin.
//
// One warp is one worker (one of the paper's threads; lane 0 does the
// work, so workers run concurrently and not interleaved inside one warp).
// A worker runs its transactions in order.  One attempt of a transaction:
//  Stage 1, planning.  An operation that finds its key records the slot's
//    version: in the read set for a read, in the write set (with the record
//    to store) for an overwrite or delete.  An operation whose key is absent
//    records the versions of the key's two bins in the read set, with the
//    key.  An insert records its two bins that way, then plans its
//    placement: a free slot of the less full bin (load balancing), or a
//    kick-out chain when both are full; the chain's slots join the write
//    set with the records they will hold, and every bin that gains a record
//    joins the write set too.  Nothing is written to the table.
//      Queue-kicking: the slot a record goes to in a bin is the bin's hit
//    counter (fetch-and-add) modulo B, whether or not it is free.
//      Claim flags: every slot that joins the write set is claimed at once
//    (compare-and-swap of the claim bit); inserts and chains pass over
//    claimed slots, and an overwrite or delete that meets one aborts.
//      System-transaction kick-outs: a chain is carried out during planning,
//    last move first, each move a small transaction of its own; only the
//    slot it frees joins the write set.
//  Stage 2, locking and verification.  The write set is locked in one
//    global order (bins before slots, then by index); a write-set version
//    that moved aborts, except that with local retries a bin that moved is
//    accepted once the keys whose absence it vouches for are found still
//    absent (the check runs under the bin's lock).  Then the read set is
//    checked.  With local retries a read-set bin that moved releases the
//    locks, checks the key is still absent there, takes the new version and
//    runs Stage 2 again; without them, and for a slot, it aborts.
//  Stage 3, apply and commit.  The transaction ID is one more than every
//    version seen and than the worker's previous ID; the planned records
//    are stored, and every written slot and bin takes the ID as its version
//    when its lock is released.
// An aborted attempt releases its locks and claims and runs again.  Every
// wait is bounded: a lock not obtained within the bound aborts the attempt.
//
// GPU shape: a bin is read as one view -- its B words, then its B records,
// then the words again, each a 32-byte vector load -- and a slot's record
// counts only if its word was unlocked and unchanged (up to a claim) across
// the view.  The read and write sets live in global scratch; which slots
// and bins they hold is kept in a hash set in shared memory, so the checks
// planning makes on every candidate slot cost one shared-memory probe.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "ck.h"
#include "ck_device.cuh"

using namespace ck;

namespace {

constexpr unsigned long long W_LOCK = 1ull, W_CLAIM = 2ull;
constexpr int RS_MAX = 512;        // read-set entries per transaction
constexpr int WS_MAX = 1024;       // write-set entries per transaction
constexpr int HS = 2048;           // hash-set buckets per worker (power of two)
constexpr int WORKERS_PER_BLOCK = 2;
constexpr int CHAIN_SLOTS = 512;   // kick-out chain slots one insert plans (kicks <= 500)
// Polls of a locked word before giving up (about 30 ms).  Locks are taken
// in one global order and a lock holder never waits on a transaction that
// is still planning, so every wait ends; the bound only keeps a fault from
// hanging the GPU, and an abort it causes is counted as TXS_ABORT_LOCK.
constexpr int LOCK_POLLS = 1 << 15;
// Stage 2 runs again after each round of read-set local retries; the paper
// sets no limit, and under a burst of concurrent commits (every worker's
// first transaction inserts into the same empty table) tens of rounds are
// common.  Past this many the attempt aborts (TXS_ABORT_RS).
constexpr int STAGE2_PASSES = 4096;
constexpr uint32_t ATTEMPTS_MAX = 100000;
constexpr uint32_t OVERFLOWS_MAX = 4;     // attempts that overflowed a read or write set before giving up
constexpr uint32_t CHAIN_ABORTS_MAX = 64; // attempts that found no eligible slot for an insert
constexpr uint64_t TIME_BUDGET_NS = 120ull * 1000 * 1000 * 1000;  // per worker and launch
constexpr uint32_t BIN_KEY = 0x80000000u;  // hash-set keys: slot index, or bin index | BIN_KEY
constexpr size_t SMEM_BYTES = (size_t)WORKERS_PER_BLOCK * HS * (8 + 4);

enum TxStat : int {
  TXS_COMMITS = 0,
  TXS_ATTEMPTS = 1,
  TXS_ABORT_CLAIMED = 2,   // met a slot claimed by another transaction
  TXS_ABORT_LOCK = 3,      // a lock was not obtained (or not released by another) within the bound
  TXS_ABORT_WS = 4,        // a write-set version moved
  TXS_ABORT_RS = 5,        // a read-set version moved (or a key appeared in a bin)
  TXS_ABORT_CHAIN = 6,     // no eligible slot for an insert or chain step
  TXS_ABORT_OVERFLOW = 7,  // read or write set full
  TXS_LOCAL_RETRIES = 8,
  TXS_FAILED = 9,          // transactions given up (attempt or time bound, or no placement)
  TXS_MINI_TXNS = 10,      // chain moves done as system transactions
  TXS_MINI_ABORTS = 11,
  TXS_KICKS = 12,          // records moved by committed plans and system moves
  TXS_N = 16
};
static_assert(TXS_N == CK_TXN_COUNTERS, "counter count");

struct TxDev {
  DevTable h;                 // hashing: n_bins (per trial), bin_mask, seeds (family 0, d = 2)
  uint64_t* slots;            // trials * n_bins * B
  unsigned long long* sver;   // per slot: version << 2 | claim << 1 | lock
  unsigned long long* bver;   // per bin: version << 2 | lock
  unsigned int* hit;          // per bin: hit counter (queue-kicking)
  unsigned long long* stats;  // TXS_N counters, summed over trials
  unsigned long long* order;  // per trial: commits so far
  uint64_t bins_per_trial;
  uint32_t B, flags, cap, trials;
  uint64_t rng_seed;
};

// A recorded word.  kind 0: slot, 1: bin.  Read-set bins carry the key
// whose absence their version vouches for.
struct Ent {
  uint32_t idx;              // global slot or bin index
  uint32_t key;
  unsigned long long ver;    // version seen, as version << 2
  unsigned long long lockw;  // the word the lock replaced (write set)
  uint64_t rec;              // write-set slots: the record to store
  uint8_t kind, claimed, locked, stale;
  uint32_t pad;
};
static_assert(sizeof(Ent) == 40, "entry is 40 bytes");

struct Scratch {  // one per worker, in global memory
  Ent rs[RS_MAX];
  Ent ws[WS_MAX];
  uint64_t lock_order[WS_MAX];  // sort key << 16 | write-set index
  // the kick-out chain being planned: slot, its bin, its word, its record
  uint32_t path[CHAIN_SLOTS], pbin[CHAIN_SLOTS];
  unsigned long long pword[CHAIN_SLOTS];
  uint64_t pold[CHAIN_SLOTS];
};

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

struct Txn {
  Scratch* sc;
  unsigned long long* hkey;  // HS buckets: epoch << 32 | set key (epoch 0: never used)
  uint32_t* hval;            // bit 0: a read-set slot; bits 1..: write-set index + 1
  uint32_t epoch;            // the current attempt's tag; other tags count as empty
  int nrs, nws;
  uint32_t trial;
  uint32_t bin0;  // first bin of this trial's table
  uint64_t rng;   // draw state
  int cause;      // TxStat of the abort
  DevTable h;     // this trial's hashing
};

__device__ __forceinline__ uint64_t next_draw(Txn& x) {
  x.rng += 0x9E3779B97F4A7C15ull;
  return splitmix64_at(x.rng);
}

// ---- the attempt's hash set of slots and bins in its read/write sets ----

static_assert(HS == 1 << 11, "hs_home takes 11 bits");
__device__ __forceinline__ uint32_t hs_home(uint32_t k) { return (k * 0x9E3779B1u) >> (32 - 11); }

// Bucket holding k, or -1.
__device__ int hs_find(const Txn& x, uint32_t k) {
  const unsigned long long want = ((unsigned long long)x.epoch << 32) | k;
  uint32_t b = hs_home(k);
  for (int p = 0; p < HS; p++, b = (b + 1) & (HS - 1)) {
    const unsigned long long c = x.hkey[b];
    if (c == want) return (int)b;
    if ((uint32_t)(c >> 32) != x.epoch) return -1;  // an empty bucket ends the probe
  }
  return -1;
}

// Bucket holding k, added (value 0) if absent; -1 if the set is full.
__device__ int hs_add(Txn& x, uint32_t k) {
  const unsigned long long want = ((unsigned long long)x.epoch << 32) | k;
  uint32_t b = hs_home(k);
  for (int p = 0; p < HS; p++, b = (b + 1) & (HS - 1)) {
    const unsigned long long c = x.hkey[b];
    if (c == want) return (int)b;
    if ((uint32_t)(c >> 32) != x.epoch) {
      x.hkey[b] = want;
      x.hval[b] = 0;
      return (int)b;
    }
  }
  return -1;
}

__device__ int ws_slot_at(const Txn& x, uint32_t idx) {
  const int b = hs_find(x, idx);
  return b < 0 ? -1 : (int)(x.hval[b] >> 1) - 1;
}

// The write-set entry for the word of e (same kind and index), or -1.
__device__ int ws_entry_of(const Txn& x, const Ent& e) {
  const int b = hs_find(x, e.kind ? (e.idx | BIN_KEY) : e.idx);
  return b < 0 ? -1 : (int)(x.hval[b] >> 1) - 1;
}

// The write-set slot whose planned record has `key`, or -1.
__device__ int ws_planned_key(const Txn& x, uint32_t key) {
  for (int i = 0; i < x.nws; i++) {
    const Ent& e = x.sc->ws[i];
    if (e.kind == 0 && e.rec != EMPTY && key_of(e.rec) == key) return i;
  }
  return -1;
}

__device__ bool add_rs(Txn& x, uint32_t idx, uint8_t kind, uint32_t key, unsigned long long word) {
  if (x.nrs >= RS_MAX) {
    x.cause = TXS_ABORT_OVERFLOW;
    return false;
  }
  if (kind == 0) {
    const int b = hs_add(x, idx);
    if (b < 0) {
      x.cause = TXS_ABORT_OVERFLOW;
      return false;
    }
    x.hval[b] |= 1u;
  }
  Ent& e = x.sc->rs[x.nrs++];
  e.idx = idx;
  e.key = key;
  e.ver = word & ~3ull;
  e.lockw = 0;
  e.rec = 0;
  e.kind = kind;
  e.claimed = e.locked = e.stale = 0;
  return true;
}

// Add a slot (kind 0, with the record to store) or a bin (kind 1; a bin
// already in the write set keeps its first entry).
__device__ bool add_ws(Txn& x, uint32_t idx, uint8_t kind, unsigned long long word, uint64_t rec, bool claimed) {
  const int b = hs_add(x, kind ? (idx | BIN_KEY) : idx);
  if (b < 0 || (kind == 0 && (x.hval[b] >> 1)) || x.nws >= WS_MAX) {
    x.cause = TXS_ABORT_OVERFLOW;  // (a slot planned twice cannot happen: eligible() excludes it)
    return false;
  }
  if (x.hval[b] >> 1) return true;  // the bin is recorded already
  x.hval[b] |= (uint32_t)(x.nws + 1) << 1;
  Ent& e = x.sc->ws[x.nws++];
  e.idx = idx;
  e.key = 0;
  e.ver = word & ~3ull;
  e.lockw = 0;
  e.rec = rec;
  e.kind = kind;
  e.claimed = claimed ? 1 : 0;
  e.locked = e.stale = 0;
  return true;
}

// ---- reading the table ----

struct BinView {
  uint64_t rec[8];
  uint64_t w[8];
};

// One try at a consistent view of a bin: every slot's word unlocked and
// unchanged (up to a claim) from before its record was read to after.
__device__ bool view_once(const TxDev& t, uint32_t bin, BinView& v) {
  const uint64_t* sp = t.slots + (uint64_t)bin * t.B;
  const uint64_t* wp = reinterpret_cast<const uint64_t*>(t.sver) + (uint64_t)bin * t.B;
  uint64_t w1[8];
#pragma unroll
  for (int q = 0; q < 8; q += 4)
    if (q < (int)t.B) ld_bin4(wp + q, w1 + q);
  fence_acquire();
#pragma unroll
  for (int q = 0; q < 8; q += 4)
    if (q < (int)t.B) ld_bin4(sp + q, v.rec + q);
  fence_acquire();
#pragma unroll
  for (int q = 0; q < 8; q += 4)
    if (q < (int)t.B) ld_bin4(wp + q, v.w + q);
  bool ok = true;
#pragma unroll
  for (int s = 0; s < 8; s++)
    if (s < (int)t.B) ok = ok && !(w1[s] & W_LOCK) && ((w1[s] | W_CLAIM) == (v.w[s] | W_CLAIM));
  return ok;
}

// A consistent view, waiting out locks.  false: a slot stayed locked or
// kept changing.
__device__ bool view_bin(const TxDev& t, uint32_t bin, BinView& v) {
  for (int k = 0; k < LOCK_POLLS; k++) {
    if (view_once(t, bin, v)) return true;
    __nanosleep(128);
  }
  return false;
}

// A bin's word once unlocked.  false: it stayed locked.
__device__ bool read_bin(const TxDev& t, uint32_t bin, unsigned long long& word) {
  for (int k = 0; k < LOCK_POLLS; k++) {
    const unsigned long long w = ld_word(t.bver + bin);
    if (!(w & W_LOCK)) {
      word = w;
      return true;
    }
    __nanosleep(128);
  }
  return false;
}

// Claim a slot whose word was read as `word`.  Fails if it is claimed or
// locked, or has changed since.
__device__ bool claim_slot(const TxDev& t, uint32_t idx, unsigned long long word) {
  if (word & (W_CLAIM | W_LOCK)) return false;
  return atomicCAS(t.sver + idx, word, word | W_CLAIM) == word;
}

__device__ __forceinline__ void unclaim(const TxDev& t, uint32_t idx) { atomicAnd(t.sver + idx, ~W_CLAIM); }

// Unlock every locked write-set word, restoring what the lock replaced
// (claims stay).
__device__ void unlock_all(const TxDev& t, Txn& x) {
  bool fenced = false;
  for (int i = 0; i < x.nws; i++) {
    Ent& e = x.sc->ws[i];
    if (!e.locked) continue;
    if (!fenced) {
      __threadfence();
      fenced = true;
    }
    atomicExch(e.kind == 0 ? t.sver + e.idx : t.bver + e.idx, e.lockw);
    e.locked = 0;
  }
}

// Abort: unlock, then drop every claim.
__device__ void release(const TxDev& t, Txn& x) {
  unlock_all(t, x);
  for (int i = 0; i < x.nws; i++) {
    Ent& e = x.sc->ws[i];
    if (e.claimed) {
      unclaim(t, e.idx);
      e.claimed = 0;
    }
  }
}

// Is `key` absent from `bin`?  -1: the bin could not be viewed.  Stable
// when the caller holds the bin's lock: nothing moves into it then.
__device__ int absent_scan(const TxDev& t, uint32_t bin, uint32_t key) {
  BinView v;
  if (!view_bin(t, bin, v)) return -1;
#pragma unroll
  for (int s = 0; s < 8; s++)
    if (s < (int)t.B && v.rec[s] != EMPTY && key_of(v.rec[s]) == key) return 0;
  return 1;
}

// Is `key` absent from `bin`, with the bin's version unchanged around the
// scan?  1 absent (word set), 0 present, -1 a lock stayed held.
__device__ int absent_versioned(const TxDev& t, uint32_t bin, uint32_t key, unsigned long long& word) {
  for (int tries = 0; tries < 16; tries++) {
    unsigned long long v1, v2;
    if (!read_bin(t, bin, v1)) return -1;
    const int a = absent_scan(t, bin, key);
    if (a <= 0) return a;
    if (!read_bin(t, bin, v2)) return -1;
    if ((v1 >> 2) == (v2 >> 2)) {
      word = v1;
      return 1;
    }
  }
  return -1;
}

// absent_versioned without waiting: 1 absent (word set), 0 present, -1 a
// lock or a change was seen.  Safe while holding locks: it waits on nobody.
__device__ int try_absent(const TxDev& t, uint32_t bin, uint32_t key, unsigned long long& word) {
  const unsigned long long v1 = ld_word(t.bver + bin);
  if (v1 & W_LOCK) return -1;
  BinView v;
  if (!view_once(t, bin, v)) return -1;
#pragma unroll
  for (int s = 0; s < 8; s++)
    if (s < (int)t.B && v.rec[s] != EMPTY && key_of(v.rec[s]) == key) return 0;
  const unsigned long long v2 = ld_word(t.bver + bin);
  if (v2 != v1) return -1;
  word = v1;
  return 1;
}

// Find `key` in its bins.  >= 0: its slot (rec, word set).  -1: absent,
// with the two bins' words, unchanged across the scan.  -2: a lock stayed
// held.
__device__ int find_key(const TxDev& t, uint32_t key, uint32_t b0, uint32_t b1, uint64_t& rec,
                        unsigned long long& word, unsigned long long& bw0, unsigned long long& bw1) {
  for (int tries = 0; tries < 16; tries++) {
    if (!read_bin(t, b0, bw0) || !read_bin(t, b1, bw1)) return -2;
    for (int j = 0; j < 2; j++) {
      const uint32_t bin = j ? b1 : b0;
      BinView v;
      if (!view_bin(t, bin, v)) return -2;
#pragma unroll
      for (int s = 0; s < 8; s++)
        if (s < (int)t.B && v.rec[s] != EMPTY && key_of(v.rec[s]) == key) {
          rec = v.rec[s];
          word = v.w[s];
          return (int)(bin * t.B + s);
        }
    }
    unsigned long long c0, c1;
    if (!read_bin(t, b0, c0) || !read_bin(t, b1, c1)) return -2;
    if ((c0 >> 2) == (bw0 >> 2) && (c1 >> 2) == (bw1 >> 2)) return -1;
  }
  return -2;
}

// May the transaction plan a write into slot idx (word w)?  Not if it
// already reads or writes it, or (claim flags) another holds its claim.
__device__ bool eligible(const TxDev& t, const Txn& x, uint32_t idx, unsigned long long w) {
  if ((t.flags & CK_TXF_CLAIM) && (w & W_CLAIM)) return false;
  const int b = hs_find(x, idx);
  return b < 0 || x.hval[b] == 0;
}

// The slot on the chain being planned?
__device__ bool on_path(const uint32_t* path, int np, uint32_t idx) {
  for (int q = 0; q < np; q++)
    if (path[q] == idx) return true;
  return false;
}

// Free eligible slots of `bin` not on the chain being planned: the lowest
// one (-1 if none; -2 if the bin could not be viewed) and how many.
__device__ int free_slots(const TxDev& t, const Txn& x, uint32_t bin, const uint32_t* path, int np,
                          unsigned long long& word, int& count) {
  int first = -1;
  count = 0;
  BinView v;
  if (!view_bin(t, bin, v)) return -2;
#pragma unroll
  for (int s = 0; s < 8; s++) {
    if (s >= (int)t.B || v.rec[s] != EMPTY) continue;
    const uint32_t idx = bin * t.B + s;
    if (!eligible(t, x, idx, v.w[s]) || on_path(path, np, idx)) continue;
    if (first < 0) {
      first = (int)idx;
      word = v.w[s];
    }
    count++;
  }
  return first;
}

// The slot a record goes to in `bin` when planning needs one beyond the
// plain free-slot rule.  Queue-kicking: one fetch-and-add of the bin's hit
// counter gives h; the first free eligible slot from h mod B, else the
// first eligible occupied one from h mod B (in a bin filled without
// deletes and without aborted plans, slot h mod B itself: the record that
// has been there longest).  Concurrent planners draw different h, so they
// start from different slots.  Otherwise (random kicking): a uniformly
// drawn slot, or the next eligible one after it.  With claim flags the slot
// is claimed here; a claim lost meanwhile passes the slot over.  -1: none
// found; -3: none found, but slots other transactions hold claimed were
// passed over (contention, not a full bin); -2: the bin could not be viewed.
__device__ int target_slot(const TxDev& t, Txn& x, uint32_t bin, const uint32_t* path, int np, uint64_t& rec,
                           unsigned long long& word) {
  const bool queue = t.flags & CK_TXF_QUEUE;
  const bool claim = t.flags & CK_TXF_CLAIM;
  const uint32_t start = queue ? atomicAdd(t.hit + bin, 1u) % t.B : (uint32_t)(next_draw(x) % t.B);
  BinView v;
  if (!view_bin(t, bin, v)) return -2;
  bool foreign = false;
  for (int pass = queue ? 0 : 1; pass < 2; pass++) {  // queue: free slots first
    for (uint32_t k = 0; k < t.B; k++) {
      const uint32_t s = (start + k) % t.B;
      const uint32_t idx = bin * t.B + s;
      if (pass == 0 && v.rec[s] != EMPTY) continue;
      if (!eligible(t, x, idx, v.w[s]) || on_path(path, np, idx)) {
        if (claim && (v.w[s] & W_CLAIM) && !on_path(path, np, idx) && hs_find(x, idx) < 0) foreign = true;
        continue;
      }
      if (claim && !claim_slot(t, idx, v.w[s])) {
        foreign = true;
        continue;
      }
      rec = v.rec[s];
      word = v.w[s] | (claim ? W_CLAIM : 0ull);
      return (int)idx;
    }
  }
  return foreign ? -3 : -1;
}

// A system transaction moving record r from slot src to the empty slot dst
// of bin dbin.  ws_/wd are the words read when the chain was planned (with
// claim flags the chain holds both claims).  The destination bin and both
// slots are locked, the contents checked, the record moved, and all three
// take a new version.  The source keeps its claim (the next move, or the
// insert, fills it); the destination's ends.
__device__ bool mini_move(const TxDev& t, uint32_t src, unsigned long long ws_, uint32_t dst,
                          unsigned long long wd, uint32_t dbin, uint64_t r) {
  unsigned long long bw;
  if (!read_bin(t, dbin, bw)) return false;
  if (atomicCAS(t.bver + dbin, bw, bw | W_LOCK) != bw) return false;
  const bool src_first = src < dst;
  const uint32_t lo = src_first ? src : dst, hi = src_first ? dst : src;
  const unsigned long long wlo = src_first ? ws_ : wd, whi = src_first ? wd : ws_;
  const bool ok_lo = atomicCAS(t.sver + lo, wlo, wlo | W_LOCK) == wlo;
  bool ok_hi = ok_lo && atomicCAS(t.sver + hi, whi, whi | W_LOCK) == whi;
  if (ok_hi) {
    __threadfence();
    ok_hi = ld_slot(t.slots + src) == r && ld_slot(t.slots + dst) == EMPTY;
    if (!ok_hi) atomicExch(t.sver + hi, whi);
  }
  if (!ok_hi) {
    if (ok_lo) atomicExch(t.sver + lo, wlo);
    atomicExch(t.bver + dbin, bw);
    return false;
  }
  unsigned long long v = ws_ >> 2;
  v = max(v, wd >> 2);
  v = max(v, bw >> 2);
  const unsigned long long nv = (v + 1) << 2;
  st_slot(t.slots + dst, r);
  st_slot(t.slots + src, EMPTY);
  __threadfence();
  atomicExch(t.sver + dst, nv);
  atomicExch(t.sver + src, nv | (ws_ & W_CLAIM));
  atomicExch(t.bver + dbin, nv);
  return true;
}

// Plan an insert of `rec` (its absence from b0, b1 already in the read
// set).  0 planned, 1 abort (cause set), 2 no placement within the chain
// cap.
__device__ int plan_insert(const TxDev& t, Txn& x, uint64_t rec, uint32_t b0, uint32_t b1) {
  const bool claim = t.flags & CK_TXF_CLAIM;
  const bool sys = t.flags & CK_TXF_SYSTEM;
  const bool queue = t.flags & CK_TXF_QUEUE;
  uint32_t* path = x.sc->path;
  uint32_t* pbin = x.sc->pbin;
  unsigned long long* pword = x.sc->pword;
  uint64_t* pold = x.sc->pold;
  for (int round = 0; round < 8; round++) {
    int n0, n1;
    unsigned long long w0 = 0, w1 = 0;
    const int f0 = free_slots(t, x, b0, path, 0, w0, n0);
    const int f1 = free_slots(t, x, b1, path, 0, w1, n1);
    if (f0 == -2 || f1 == -2) {
      x.cause = TXS_ABORT_LOCK;
      return 1;
    }
    uint32_t bin;
    if (f0 >= 0 || f1 >= 0)  // load balancing: the bin with more free slots (b0 on ties)
      bin = (f0 >= 0 && n0 >= n1) ? b0 : b1;
    else  // both full: a uniformly drawn bin (no hit balancing)
      bin = (next_draw(x) & 1) ? b1 : b0;
    // path[0]: the slot the new record goes to
    int s;
    uint64_t occ = EMPTY;
    unsigned long long sw = 0;
    if (!queue && (f0 >= 0 || f1 >= 0)) {
      s = bin == b0 ? f0 : f1;
      sw = bin == b0 ? w0 : w1;
      if (claim) {
        if (!claim_slot(t, (uint32_t)s, sw)) continue;  // taken meanwhile: look again
        sw |= W_CLAIM;
      }
    } else {
      s = target_slot(t, x, bin, path, 0, occ, sw);
      if (s < 0) {
        x.cause = s == -2 ? TXS_ABORT_LOCK : s == -3 ? TXS_ABORT_CLAIMED : TXS_ABORT_CHAIN;
        return 1;
      }
    }
    path[0] = (uint32_t)s;
    pbin[0] = bin;
    pword[0] = sw;
    pold[0] = occ;
    int np = 1;
    // while the chain's last slot is occupied, its record moves to a slot
    // of its other bin
    int result = 0;
    while (pold[np - 1] != EMPTY) {
      if (np >= CHAIN_SLOTS || np > (int)t.cap) {
        result = 2;
        break;
      }
      uint32_t c0, c1;
      bins2(x.h, key_of(pold[np - 1]), c0, c1);
      c0 += x.bin0;
      c1 += x.bin0;
      const uint32_t y = c0 == pbin[np - 1] ? c1 : c0;
      int ns = -1, cnt;
      uint64_t nocc = EMPTY;
      unsigned long long nw = 0;
      if (!queue) {
        // a free slot of y; with claim flags, one lost to another claim
        // meanwhile is passed over like any claimed slot
        for (uint32_t k = 0; k < t.B; k++) {
          ns = free_slots(t, x, y, path, np, nw, cnt);
          if (ns < 0 || !claim || claim_slot(t, (uint32_t)ns, nw)) break;
          ns = -1;
        }
        if (ns == -2) {
          x.cause = TXS_ABORT_LOCK;
          result = 1;
          break;
        }
        if (ns >= 0 && claim) nw |= W_CLAIM;
      }
      if (ns < 0) {
        ns = target_slot(t, x, y, path, np, nocc, nw);
        if (ns < 0) {
          x.cause = ns == -2 ? TXS_ABORT_LOCK : ns == -3 ? TXS_ABORT_CLAIMED : TXS_ABORT_CHAIN;
          result = 1;
          break;
        }
      }
      path[np] = (uint32_t)ns;
      pbin[np] = y;
      pword[np] = nw;
      pold[np] = nocc;
      np++;
    }
    if (result != 0) {
      if (claim)
        for (int q = 0; q < np; q++) unclaim(t, path[q]);
      return result;
    }
    if (!sys) {
      // the write set: every chain slot with the record it will hold, and
      // every bin gaining a record
      for (int q = 0; q < np; q++) {
        unsigned long long bw;
        bool ok = read_bin(t, pbin[q], bw);
        if (!ok) x.cause = TXS_ABORT_LOCK;
        ok = ok && add_ws(x, pbin[q], 1, bw, 0, false) &&
             add_ws(x, path[q], 0, pword[q], q == 0 ? rec : pold[q - 1], claim);
        if (!ok) {
          if (claim)
            for (int r = q; r < np; r++) unclaim(t, path[r]);
          return 1;
        }
      }
      return 0;
    }
    // system-transaction kick-outs: last move first, each its own
    // transaction
    bool moved_all = true;
    for (int q = np - 1; q >= 1; q--) {
      if (!mini_move(t, path[q - 1], pword[q - 1], path[q], pword[q], pbin[q], pold[q - 1])) {
        moved_all = false;
        atomicAdd(t.stats + TXS_MINI_ABORTS, 1ull);
        if (claim)
          for (int r = 0; r < q; r++) unclaim(t, path[r]);
        break;
      }
      atomicAdd(t.stats + TXS_MINI_TXNS, 1ull);
      atomicAdd(t.stats + TXS_KICKS, 1ull);
      // path[q-1] is empty now, with a new version (and still the claim)
      pword[q - 1] = ld_word(t.sver + path[q - 1]) & ~W_LOCK;
      pold[q - 1] = EMPTY;
    }
    if (!moved_all) continue;  // plan the insert again
    unsigned long long bw;
    bool ok = read_bin(t, pbin[0], bw);
    if (!ok) x.cause = TXS_ABORT_LOCK;
    ok = ok && add_ws(x, pbin[0], 1, bw, 0, false) && add_ws(x, path[0], 0, pword[0], rec, claim);
    if (!ok) {
      if (claim) unclaim(t, path[0]);
      return 1;
    }
    return 0;
  }
  x.cause = TXS_ABORT_CHAIN;
  return 1;
}

// The write set's lock order, bins before slots, then by index: sort keys
// (1 - kind) << 48 | index << 16 | entry, Shell-sorted (Ciura's gaps).
__device__ void sort_lock_order(Txn& x) {
  uint64_t* o = x.sc->lock_order;
  const int n = x.nws;
  for (int i = 0; i < n; i++) {
    const Ent& e = x.sc->ws[i];
    o[i] = ((uint64_t)(1 - e.kind) << 48) | ((uint64_t)e.idx << 16) | (uint64_t)i;
  }
  const int gaps[8] = {301, 132, 57, 23, 10, 4, 1, 0};
  for (int g = 0; gaps[g] > 0; g++) {
    const int gap = gaps[g];
    for (int i = gap; i < n; i++) {
      const uint64_t v = o[i];
      int j = i;
      while (j >= gap && o[j - gap] > v) {
        o[j] = o[j - gap];
        j -= gap;
      }
      o[j] = v;
    }
  }
}

// Lock the write set in the global order.  false: abort (cause set).
__device__ bool lock_ws(const TxDev& t, Txn& x) {
  const bool local = t.flags & CK_TXF_LOCAL_RETRY;
  for (int j = 0; j < x.nws; j++) {
    Ent& e = x.sc->ws[x.sc->lock_order[j] & 0xFFFF];
    unsigned long long* p = e.kind == 0 ? t.sver + e.idx : t.bver + e.idx;
    bool got = false;
    unsigned long long cur = 0;
    for (int k = 0; k < LOCK_POLLS && !got; k++) {
      cur = ld_word(p);
      if (cur & W_LOCK) {
        __nanosleep(128);
        continue;
      }
      if (e.kind == 0 && (cur >> 2) != (e.ver >> 2)) {  // a slot that moved: abort
        x.cause = TXS_ABORT_WS;
        return false;
      }
      if (e.kind == 0 && ((cur & W_CLAIM) != 0) != (e.claimed != 0)) {
        x.cause = TXS_ABORT_CLAIMED;  // claimed by another since it was planned
        return false;
      }
      got = atomicCAS(p, cur, cur | W_LOCK) == cur;
    }
    if (!got) {
      x.cause = TXS_ABORT_LOCK;
      return false;
    }
    e.locked = 1;
    e.lockw = cur;
    if (e.kind == 1 && (cur >> 2) != (e.ver >> 2)) {
      // a bin that moved.  With local retries (its lock is ours, so nothing
      // moves into it): are the keys whose absence it vouches for still
      // absent from it?
      if (!local) {
        x.cause = TXS_ABORT_WS;
        return false;
      }
      for (int q = 0; q < x.nrs; q++) {
        Ent& r = x.sc->rs[q];
        if (r.kind != 1 || r.idx != e.idx) continue;
        const int a = absent_scan(t, e.idx, r.key);
        if (a <= 0) {
          x.cause = a < 0 ? TXS_ABORT_LOCK : TXS_ABORT_WS;
          return false;
        }
        r.ver = cur & ~3ull;
      }
      e.ver = cur & ~3ull;
      atomicAdd(t.stats + TXS_LOCAL_RETRIES, 1ull);
    }
  }
  return true;
}

// Stage 2.  true: every version holds, with the write set locked.
//
// A read-set bin that moved (local retries) is checked again at once when
// that needs no waiting (try_absent), keeping the locks; a validation pass
// that then finds every version unchanged is a point at which every read
// holds with the write set locked.  Only a bin that is locked by another
// transaction, or changing, makes the transaction release its locks, wait
// for the check, and lock again (the paper's local retry; waiting while
// holding locks could deadlock).
__device__ bool stage2(const TxDev& t, Txn& x) {
  const bool local = t.flags & CK_TXF_LOCAL_RETRY;
  sort_lock_order(x);
  int passes = 0;
  while (passes < STAGE2_PASSES) {
    if (!lock_ws(t, x)) return false;
    bool relock = false;
    while (!relock) {
      if (++passes > STAGE2_PASSES) {
        x.cause = TXS_ABORT_RS;
        return false;
      }
      bool retry = false;
      // the read set, eight words in flight at a time
      for (int i0 = 0; i0 < x.nrs; i0 += 8) {
        unsigned long long cur[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const Ent& e = x.sc->rs[min(i0 + u, x.nrs - 1)];
          cur[u] = ld_word(e.kind == 0 ? t.sver + e.idx : t.bver + e.idx);
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
          if (i0 + u >= x.nrs) break;
          Ent& e = x.sc->rs[i0 + u];
          bool locked_other = false;
          if (cur[u] & W_LOCK) {
            const int w = ws_entry_of(x, e);
            locked_other = w < 0 || !x.sc->ws[w].locked;
          }
          if (!locked_other && (cur[u] >> 2) == (e.ver >> 2)) continue;
          if (e.kind == 1 && local) {
            e.stale = 1;
            retry = true;
            continue;
          }
          x.cause = TXS_ABORT_RS;
          return false;
        }
      }
      if (!retry) return true;
      for (int i = 0; i < x.nrs; i++) {
        Ent& e = x.sc->rs[i];
        if (!e.stale) continue;
        unsigned long long w;
        const int a = try_absent(t, e.idx, e.key, w);
        if (a == 0) {
          x.cause = TXS_ABORT_RS;
          return false;
        }
        if (a < 0) {
          relock = true;
          continue;
        }
        e.stale = 0;
        e.ver = w & ~3ull;
        atomicAdd(t.stats + TXS_LOCAL_RETRIES, 1ull);
      }
    }
    // a moved bin is busy: release the locks, confirm the key still absent
    // under the bin's new version, and run Stage 2 again
    unlock_all(t, x);
    for (int i = 0; i < x.nrs; i++) {
      Ent& e = x.sc->rs[i];
      if (!e.stale) continue;
      e.stale = 0;
      unsigned long long w;
      const int a = absent_versioned(t, e.idx, e.key, w);
      if (a <= 0) {
        x.cause = a < 0 ? TXS_ABORT_LOCK : TXS_ABORT_RS;
        return false;
      }
      e.ver = w & ~3ull;
      atomicAdd(t.stats + TXS_LOCAL_RETRIES, 1ull);
    }
  }
  x.cause = TXS_ABORT_RS;
  return false;
}

// Stage 3.  Returns the transaction ID; `pos` gets the commit's position
// in its trial.
__device__ unsigned long long stage3(const TxDev& t, Txn& x, unsigned long long last_tid, unsigned long long& pos) {
  unsigned long long v = last_tid;
  for (int i = 0; i < x.nrs; i++) v = max(v, x.sc->rs[i].ver >> 2);
  for (int i = 0; i < x.nws; i++) v = max(v, x.sc->ws[i].ver >> 2);
  const unsigned long long tid = v + 1;
  pos = atomicAdd(t.order + x.trial, 1ull);
  __threadfence();  // the locks are visible before any record changes
  uint32_t moved = 0;
  for (int i = 0; i < x.nws; i++) {
    const Ent& e = x.sc->ws[i];
    if (e.kind != 0) continue;
    const uint64_t old = ld_slot(t.slots + e.idx);
    if (old != EMPTY && e.rec != EMPTY && key_of(old) != key_of(e.rec)) moved++;
    st_slot(t.slots + e.idx, e.rec);
  }
  __threadfence();
  for (int i = 0; i < x.nws; i++) {
    Ent& e = x.sc->ws[i];
    atomicExch(e.kind == 0 ? t.sver + e.idx : t.bver + e.idx, tid << 2);
    e.locked = 0;
    e.claimed = 0;
  }
  if (moved) atomicAdd(t.stats + TXS_KICKS, (unsigned long long)moved);
  return tid;
}

// One attempt.  0 committed, 1 aborted (cause set), 2 failed (an insert
// found no placement within the chain cap).
__device__ int attempt(const TxDev& t, Txn& x, const uint8_t* op, const uint32_t* key, const uint32_t* val,
                       uint32_t L, uint8_t* st_out, uint32_t* val_out, unsigned long long& tid,
                       unsigned long long& pos) {
  x.nrs = x.nws = 0;
  x.epoch++;  // empties the hash set
  x.cause = TXS_ABORT_CHAIN;
  const bool claim = t.flags & CK_TXF_CLAIM;
  for (uint32_t j = 0; j < L; j++) {
    const uint32_t k = key[j];
    uint32_t b0, b1;
    bins2(x.h, k, b0, b1);
    b0 += x.bin0;
    b1 += x.bin0;
    uint64_t rec = EMPTY;
    unsigned long long w = 0, bw0 = 0, bw1 = 0;
    const int at = find_key(t, k, b0, b1, rec, w, bw0, bw1);
    if (at == -2) {
      x.cause = TXS_ABORT_LOCK;
      release(t, x);
      return 1;
    }
    uint8_t st = 0;
    uint32_t v = 0;
    const uint8_t o = op[j];
    if (at < 0) {  // absent: the two bins' versions vouch for it
      if (!add_rs(x, b0, 1, k, bw0) || !add_rs(x, b1, 1, k, bw1)) {
        release(t, x);
        return 1;
      }
      if (o == CK_TX_INSERT) {
        const int r = plan_insert(t, x, ((uint64_t)k << 32) | val[j], b0, b1);
        if (r != 0) {
          release(t, x);
          return r;
        }
      }
    } else if (o == CK_TX_INSERT) {
      st = 1;  // present already: nothing to insert
    } else {
      st = 1;
      if (ws_slot_at(x, (uint32_t)at) >= 0) {
        // the slot is on one of this transaction's chains, so the record is
        // planned to move: read it as it is, or edit it where it goes
        const int to = ws_planned_key(x, k);
        if (o == CK_TX_READ) {
          v = (uint32_t)rec;
        } else if (to >= 0) {
          x.sc->ws[to].rec = o == CK_TX_DELETE ? EMPTY : (((uint64_t)k << 32) | val[j]);
        } else {
          release(t, x);
          return 1;
        }
      } else if (o == CK_TX_READ) {
        if (!add_rs(x, (uint32_t)at, 0, k, w)) {
          release(t, x);
          return 1;
        }
        v = (uint32_t)rec;
      } else {  // overwrite or delete: the slot joins the write set
        if (claim) {
          if (!claim_slot(t, (uint32_t)at, w)) {
            x.cause = TXS_ABORT_CLAIMED;
            release(t, x);
            return 1;
          }
          w |= W_CLAIM;
        }
        const uint64_t nrec = o == CK_TX_DELETE ? EMPTY : (((uint64_t)k << 32) | val[j]);
        if (!add_ws(x, (uint32_t)at, 0, w, nrec, claim)) {
          if (claim) unclaim(t, (uint32_t)at);
          release(t, x);
          return 1;
        }
      }
    }
    if (st_out) st_out[j] = st;
    if (val_out) val_out[j] = v;
  }
  if (!stage2(t, x)) {
    release(t, x);
    return 1;
  }
  tid = stage3(t, x, tid, pos);
  return 0;
}

// One warp per worker (lane 0 works; the warp first clears the worker's
// hash set).  Worker w of trial r runs transactions w*T .. w*T+T-1 of the
// shared operation arrays.
__global__ void __launch_bounds__(32 * WORKERS_PER_BLOCK) k_txn_run(
    TxDev t, const uint8_t* __restrict__ op, const uint32_t* __restrict__ key, const uint32_t* __restrict__ val,
    uint32_t n_workers, uint32_t T, uint32_t L, Scratch* scratch, uint8_t* status, uint32_t* value,
    uint32_t* attempts_out, unsigned long long* tid_out, unsigned long long* pos_out) {
  extern __shared__ unsigned long long smem[];
  const uint32_t wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long* hkey = smem + (size_t)wl * HS;
  uint32_t* hval = reinterpret_cast<uint32_t*>(smem + (size_t)WORKERS_PER_BLOCK * HS) + (size_t)wl * HS;
  for (int i = lane; i < HS; i += 32) {
    hkey[i] = 0;
    hval[i] = 0;
  }
  __syncwarp();
  const uint64_t g = (uint64_t)blockIdx.x * WORKERS_PER_BLOCK + wl;
  if (lane != 0 || g >= (uint64_t)n_workers * t.trials) return;
  const uint32_t trial = (uint32_t)(g / n_workers), w = (uint32_t)(g % n_workers);
  Txn x;
  x.sc = scratch + g;
  x.hkey = hkey;
  x.hval = hval;
  x.epoch = 0;
  x.trial = trial;
  x.bin0 = (uint32_t)(trial * t.bins_per_trial);
  x.rng = t.rng_seed ^ (g << 24);
  x.h = t.h;
  const uint32_t salt = (uint32_t)splitmix64_at(t.rng_seed + trial);
  x.h.seeds[0] ^= salt;  // the same salt on both seeds keeps them distinct
  x.h.seeds[1] ^= salt;
  const uint64_t n_ops = (uint64_t)n_workers * T * L;
  unsigned long long last = 0;
  const uint64_t start = now_ns();
  for (uint32_t i = 0; i < T; i++) {
    const uint64_t tx = (uint64_t)w * T + i;
    const uint64_t base = tx * L;
    const uint64_t out = (uint64_t)trial * n_ops + base;
    int rc = 1;
    uint32_t a = 0, overflows = 0, chain_aborts = 0;
    unsigned long long tid = last, pos = ~0ull;
    while (rc == 1 && a < ATTEMPTS_MAX && now_ns() - start < TIME_BUDGET_NS) {
      a++;
      tid = last;
      rc = attempt(t, x, op + base, key + base, val + base, L, status ? status + out : nullptr,
                   value ? value + out : nullptr, tid, pos);
      if (rc == 1) {
        atomicAdd(t.stats + x.cause, 1ull);
        // a transaction too large for its read or write set overflows on
        // every attempt, and one whose inserts cannot all be placed finds no
        // eligible slot on every attempt: give those up
        if (x.cause == TXS_ABORT_OVERFLOW && ++overflows == OVERFLOWS_MAX) rc = 2;
        else if (x.cause == TXS_ABORT_CHAIN && ++chain_aborts == CHAIN_ABORTS_MAX) rc = 2;
        else if (a > 16) __nanosleep(64u << (a < 24 ? a - 16 : 8));
      }
    }
    atomicAdd(t.stats + TXS_ATTEMPTS, (unsigned long long)a);
    if (rc == 0) {
      last = tid;
      atomicAdd(t.stats + TXS_COMMITS, 1ull);
    } else {
      atomicAdd(t.stats + TXS_FAILED, 1ull);
      if (status)
        for (uint32_t j = 0; j < L; j++) status[out + j] = 255;
    }
    const uint64_t to = (uint64_t)trial * n_workers * T + tx;
    if (attempts_out) attempts_out[to] = a;
    if (tid_out) tid_out[to] = rc == 0 ? tid : 0;
    if (pos_out) pos_out[to] = rc == 0 ? pos : ~0ull;
  }
}

__global__ void k_txn_clear(uint64_t* slots, unsigned long long* sver, uint64_t n_slots, unsigned long long* bver,
                            unsigned int* hit, uint64_t n_bins) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += stride) {
    slots[i] = EMPTY;
    sver[i] = 0;
  }
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_bins; i += stride) {
    bver[i] = 0;
    hit[i] = 0;
  }
}

}  // namespace

struct ck_txn_table {
  TxDev t;
  void* buf;
  Scratch* scratch;
  uint64_t scratch_workers;
  uint64_t n_bins_all;
};

namespace {

int clear_all(ck_txn_table* x) {
  TxDev& t = x->t;
  k_txn_clear<<<1024, 256>>>(t.slots, t.sver, x->n_bins_all * t.B, t.bver, t.hit, x->n_bins_all);
  if (cudaGetLastError() != cudaSuccess) return CK_ECUDA;
  if (cudaMemset(t.stats, 0, TXS_N * 8) != cudaSuccess) return CK_ECUDA;
  if (cudaMemset(t.order, 0, (size_t)t.trials * 8) != cudaSuccess) return CK_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? CK_OK : CK_ECUDA;
}

}  // namespace

extern "C" {

int ck_txn_create(ck_txn_table** out, uint64_t bins, uint32_t slots_per_bin, uint32_t trials, uint64_t seed) {
  if (!out) return CK_EINVAL;
  *out = nullptr;
  if (bins < 2 || trials == 0 || (slots_per_bin != 4 && slots_per_bin != 8)) return CK_EINVAL;
  if (bins > (1ull << 32) || trials > (1u << 20)) return CK_EINVAL;
  const uint64_t all = bins * trials;
  if (all * slots_per_bin > 0x7FFFFFFFull) return CK_EINVAL;  // slot indices below BIN_KEY
  ck_txn_table* x = new (std::nothrow) ck_txn_table();
  if (!x) return CK_ENOMEM;
  const uint64_t ns = all * slots_per_bin;
  const size_t bytes = ns * 16 + all * 8 + TXS_N * 8 + (size_t)trials * 8 + all * 4;
  if (cudaMalloc(&x->buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete x;
    return CK_ENOMEM;
  }
  uint8_t* p = static_cast<uint8_t*>(x->buf);
  TxDev& t = x->t;
  std::memset(&t, 0, sizeof(t));
  t.slots = reinterpret_cast<uint64_t*>(p);  // 32-byte aligned bins: the buffer is, and B * 8 is 32 or 64
  p += ns * 8;
  t.sver = reinterpret_cast<unsigned long long*>(p);
  p += ns * 8;
  t.bver = reinterpret_cast<unsigned long long*>(p);
  p += all * 8;
  t.stats = reinterpret_cast<unsigned long long*>(p);
  p += TXS_N * 8;
  t.order = reinterpret_cast<unsigned long long*>(p);
  p += (size_t)trials * 8;
  t.hit = reinterpret_cast<unsigned int*>(p);
  t.h.n_bins = bins;
  t.h.total_slots = bins * slots_per_bin;
  t.h.bin_mask = (bins & (bins - 1)) == 0 ? (uint32_t)(bins - 1) : 0u;
  t.h.d = 2;
  t.h.B = slots_per_bin;
  t.h.hash_family = 0;
  t.h.seeds[0] = 0x9E3779B9u;
  t.h.seeds[1] = 0x85EBCA6Bu;
  t.bins_per_trial = bins;
  t.B = slots_per_bin;
  t.cap = 500;
  t.trials = trials;
  t.rng_seed = seed;
  x->n_bins_all = all;
  x->scratch = nullptr;
  x->scratch_workers = 0;
  const int rc = clear_all(x);
  if (rc != CK_OK) {
    cudaFree(x->buf);
    delete x;
    return rc;
  }
  *out = x;
  return CK_OK;
}

int ck_txn_reset(ck_txn_table* x) {
  if (!x) return CK_EINVAL;
  return clear_all(x);
}

int ck_txn_run(ck_txn_table* x, uint32_t flags, const uint8_t* d_op, const uint32_t* d_key, const uint32_t* d_val,
               uint32_t n_workers, uint32_t txns_per_worker, uint32_t ops_per_txn, uint8_t* d_status,
               uint32_t* d_value, uint32_t* d_attempts, uint64_t* d_tid, uint64_t* d_order, void* stream) {
  if (!x) return CK_EINVAL;
  if (flags & ~(uint32_t)(CK_TXF_LOCAL_RETRY | CK_TXF_QUEUE | CK_TXF_SYSTEM | CK_TXF_CLAIM)) return CK_EINVAL;
  if (n_workers == 0 || txns_per_worker == 0) return CK_OK;
  if (!d_op || !d_key || !d_val) return CK_EINVAL;
  if (ops_per_txn == 0 || ops_per_txn > (uint32_t)CK_TXN_MAX_OPS) return CK_EINVAL;
  const uint64_t workers = (uint64_t)n_workers * x->t.trials;
  if (workers > (1ull << 22)) return CK_EINVAL;
  if (x->scratch_workers < workers) {
    cudaFree(x->scratch);
    x->scratch = nullptr;
    x->scratch_workers = 0;
    if (cudaMalloc(&x->scratch, (size_t)workers * sizeof(Scratch)) != cudaSuccess) {
      cudaGetLastError();
      return CK_ENOMEM;
    }
    x->scratch_workers = workers;
  }
  if (cudaFuncSetAttribute(k_txn_run, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES) !=
      cudaSuccess)
    return CK_ECUDA;
  TxDev t = x->t;
  t.flags = flags;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)((workers + WORKERS_PER_BLOCK - 1) / WORKERS_PER_BLOCK);
  k_txn_run<<<grid, 32 * WORKERS_PER_BLOCK, SMEM_BYTES, s>>>(
      t, d_op, d_key, d_val, n_workers, txns_per_worker, ops_per_txn, x->scratch, d_status, d_value, d_attempts,
      reinterpret_cast<unsigned long long*>(d_tid), reinterpret_cast<unsigned long long*>(d_order));
  return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

int ck_txn_stats(ck_txn_table* x, uint64_t* h_counters, uint32_t n) {
  if (!x || !h_counters || n > (uint32_t)TXS_N) return CK_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return CK_ECUDA;
  return cudaMemcpy(h_counters, x->t.stats, (size_t)n * 8, cudaMemcpyDeviceToHost) == cudaSuccess ? CK_OK
                                                                                                    : CK_ECUDA;
}

int ck_txn_export(ck_txn_table* x, uint32_t trial, uint64_t* h_slots) {
  if (!x || !h_slots || trial >= x->t.trials) return CK_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return CK_ECUDA;
  const size_t n = (size_t)x->t.bins_per_trial * x->t.B;
  return cudaMemcpy(h_slots, x->t.slots + (size_t)trial * n, n * 8, cudaMemcpyDeviceToHost) == cudaSuccess
             ? CK_OK
             : CK_ECUDA;
}

void ck_txn_destroy(ck_txn_table* x) {
  if (!x) return;
  cudaDeviceSynchronize();
  cudaFree(x->scratch);
  cudaFree(x->buf);
  delete x;
}

}  // extern "C"
