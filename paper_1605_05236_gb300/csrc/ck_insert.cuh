// ck_insert.cuh -- one insertion on the GPU: plan a kick-out chain with
// claim flags, then apply it back to front (Kuszmaul, arXiv:1605.05236,
// Sec. 8 "System-Transaction Kick-Outs" and "Claim Flags"), for every
// kick-out policy of Sec. 3-7 and the ghost insertions of Sec. 4.
//
// A plan is a list of claimed slots.  Chain entries come first, in chain
// order: entry 0 receives the new record, entry i receives the record that
// entry i-1 displaced, and the last chain entry is the free slot or the
// duplicate that ends the chain.  A ghost insertion is two entries that both
// receive the new record; overwriting a duplicate adds an entry for its
// twin, whose duplicate mark is cleared.  Nothing is written until every
// slot of the plan is claimed, so an attempt that hits its cap or a claimed
// slot is abandoned by releasing its claims, and the table is unchanged.
//
// With one insertion in flight the claim flags seen in a bin are exactly
// the chain's own, and every decision below reduces to the serial order of
// the paper's definitions; with many in flight a slot claimed by another
// insertion is ignored (Sec. 8) and a bin whose metadata changed between
// view and claim is viewed again.
#pragma once
#include "ck_device.cuh"

namespace ck {

enum Kind : uint8_t { K_MOVE = 0, K_DUPTERM = 1, K_TWIN = 2, K_GHOST = 3 };

// A plan: one 16-byte entry per chain step or claimed slot, stored as two
// 64-bit words: a packed descriptor -- bits 0-31 bin, 32-34 slot, 35-36
// kind, 37 hit-counter increment, 38 revisit, 39 superseded; single-slot
// bins: 40-47 rattle counter of the displaced key, 48-55 rattle counter of
// the incoming key; bucketized bins: 40-55 the previous entry of a revisit
// -- and the record the slot held when the step was planned.  A revisit is
// a queue-kicking step into a slot the plan already holds (the walk came
// back to a bin): it takes no claim of its own, its record is the one the
// plan placed there, and the earlier entry for that slot is marked
// superseded (its write is replaced by the revisit's).  Beyond the first REG_ENTRIES (registers), entries live in
// local memory (MAX_CHAIN of them, the concurrent kernel) or in table
// scratch (LONG_CHAIN: the serial replay and chains longer than MAX_CHAIN).
template <int N>
struct PlanStore {
  alignas(16) uint64_t e[2 * N];  // entries are stored as 16-byte vectors
};

__device__ __forceinline__ uint64_t pack_entry(uint32_t bin, int slot, int kind, bool hit, uint32_t old_r,
                                               uint32_t new_r) {
  return (uint64_t)bin | ((uint64_t)slot << 32) | ((uint64_t)kind << 35) | ((uint64_t)(hit ? 1 : 0) << 37) |
         ((uint64_t)(old_r & 255u) << 40) | ((uint64_t)(new_r & 255u) << 48);
}
__device__ __forceinline__ uint32_t e_bin(uint64_t e) { return (uint32_t)e; }
__device__ __forceinline__ uint32_t e_slot(uint64_t e) { return (uint32_t)(e >> 32) & 7u; }
__device__ __forceinline__ uint32_t e_kind(uint64_t e) { return (uint32_t)(e >> 35) & 3u; }
__device__ __forceinline__ bool e_hit(uint64_t e) { return (e >> 37) & 1u; }
__device__ __forceinline__ uint32_t e_old_r(uint64_t e) { return (uint32_t)(e >> 40) & 255u; }
__device__ __forceinline__ uint32_t e_new_r(uint64_t e) { return (uint32_t)(e >> 48) & 255u; }
constexpr uint64_t E_REVISIT = 1ull << 38;
constexpr uint64_t E_SUPERSEDED = 1ull << 39;
__device__ __forceinline__ bool e_rev(uint64_t e) { return (e & E_REVISIT) != 0; }
__device__ __forceinline__ bool e_sup(uint64_t e) { return (e & E_SUPERSEDED) != 0; }
__device__ __forceinline__ int e_prev(uint64_t e) { return (int)((e >> 40) & 0xFFFFu); }

// The first REG_ENTRIES entries of a plan stay in registers (most chains
// are one or two slots long); the rest go to memory at pe, indexed by entry
// number (the first REG_ENTRIES places there stay unused).
constexpr int REG_ENTRIES = 1;  // measured: 1 is as fast as 2 and frees registers
static_assert(REG_ENTRIES >= 0 && REG_ENTRIES <= 2, "at most two plan entries in registers");

struct Ctx {
  uint32_t key;
  uint64_t krec;
  uint32_t attempt;
  uint32_t viewed;   // bins viewed, all attempts
  uint32_t viewed0;  // `viewed` when the current attempt started
  uint32_t reviews;  // bins viewed again because a claim lost a race (part of `viewed`)
  uint32_t foreign;  // the attempt ignored a slot another insertion had claimed
  uint32_t capped;   // the attempt ended at its cap or budget, or at a dead end of its own (out_of_cap, dead_end)
  uint32_t kicks;    // kick-outs of the current attempt
  uint32_t draws;    // random draws of the current attempt
  uint32_t ghosts_made;
  uint32_t dup_evict;
  // the plan, by value so the context can live in registers: entries
  // 0 .. REG_ENTRIES-1 in r*, the others at pe (16-byte aligned); pn of pcap used
  uint64_t r0d, r0c, r1d, r1c;
  uint64_t* pe;
  int pn;
  int pcap;
  int long_id;    // scratch plan in use (index in the table's pool), or -1
  int big_id;     // scratch plan region lent to a search as its larger space, or -1
  uint64_t held;  // d-ary walks: the record in hand
};

__device__ __forceinline__ void set_entry(Ctx& c, int i, uint64_t desc, uint64_t content) {
  if (REG_ENTRIES > 0 && i == 0) {
    c.r0d = desc;
    c.r0c = content;
  } else if (REG_ENTRIES > 1 && i == 1) {
    c.r1d = desc;
    c.r1c = content;
  } else {
    ulonglong2 v;
    v.x = desc;
    v.y = content;
    *reinterpret_cast<ulonglong2*>(c.pe + 2 * i) = v;
  }
}
__device__ __forceinline__ void set_content(Ctx& c, int i, uint64_t content) {
  if (REG_ENTRIES > 0 && i == 0) c.r0c = content;
  else if (REG_ENTRIES > 1 && i == 1) c.r1c = content;
  else c.pe[2 * i + 1] = content;
}
__device__ __forceinline__ void put_entry(Ctx& c, uint64_t desc, uint64_t content) {
  set_entry(c, c.pn, desc, content);
  c.pn++;
}
__device__ __forceinline__ uint64_t desc_at(const Ctx& c, int i) {
  if (REG_ENTRIES > 0 && i == 0) return c.r0d;
  if (REG_ENTRIES > 1 && i == 1) return c.r1d;
  return c.pe[2 * i];
}
__device__ __forceinline__ uint64_t content_at(const Ctx& c, int i) {
  if (REG_ENTRIES > 0 && i == 0) return c.r0c;
  if (REG_ENTRIES > 1 && i == 1) return c.r1c;
  return c.pe[2 * i + 1];
}

// Scratch plans for chains longer than a thread's local plan: a pool with a
// busy flag per plan.  Taking one never waits unboundedly: after a bounded
// number of sweeps it gives up (the attempt is then retried).
__device__ __forceinline__ int acquire_long(const DevTable& t, uint32_t key) {
  for (uint32_t round = 0; round < 256; round++) {
    uint32_t start = fmix32(key + round) % t.n_long;
    for (uint32_t k = 0; k < t.n_long; k++) {
      uint32_t r = start + k;
      if (r >= t.n_long) r -= t.n_long;
      if (*(volatile uint32_t*)(t.long_busy + r) == 0 && atomicCAS(t.long_busy + r, 0u, 1u) == 0u) return (int)r;
    }
    __nanosleep(1000);
  }
  return -1;
}

__device__ __forceinline__ void release_long(const DevTable& t, int r) {
  __threadfence();
  atomicExch(t.long_busy + r, 0u);
}

// The local plan is full: copy the chain into a scratch plan and go on.
__device__ __forceinline__ bool grow_plan(const DevTable& t, Ctx& c) {
  if (c.long_id >= 0) return false;
  int id = acquire_long(t, c.key);
  if (id < 0) return false;
  uint64_t* le = reinterpret_cast<uint64_t*>(t.long_scratch + (uint64_t)id * LONG_REGION);
  for (int i = 2 * REG_ENTRIES; i < 2 * c.pn; i++) le[i] = c.pe[i];
  c.pe = le;
  c.pcap = LONG_CHAIN;
  c.long_id = id;
  return true;
}

// Room for the next few entries: 0, or the status to give up with (a full
// scratch plan cannot happen under the cap; no free scratch plan: retry).
__device__ __forceinline__ int plan_room(const DevTable& t, Ctx& c) {
  if (c.pn < c.pcap - 4) return 0;
  if (grow_plan(t, c)) return 0;
  return c.long_id >= 0 ? (int)ST_FAILED : (int)ST_CONFLICT;
}

// Claim slot s of `bin` by CAS from the viewed metadata word m (hit: the
// claim also advances queue-kicking's hit counter) and append the entry.
__device__ __forceinline__ bool claim(const DevTable& t, Ctx& c, uint32_t bin, uint32_t m, int s, uint8_t kind,
                                      bool hit, uint64_t content, uint32_t old_r = 0, uint32_t new_r = 0) {
  uint32_t desired = m + (hit ? HIT_ONE : 0u) + (1u << s);
  if (!cas_acquire(t.meta + bin, m, desired)) return false;
  put_entry(c, pack_entry(bin, s, kind, hit, old_r, new_r), content);
  return true;
}

// The record in slot s of `bin`, read after this insertion claimed the slot.
// It must be the record the plan saw there: a claim validates its view
// through the bin's metadata word, which can come back to the value seen (a
// 4-bit version wraps after 16 releases); once the claim is held the slot
// cannot change, so this one read settles it.  Walks issue it together with
// the next step's loads and compare after them.
template <int B>
__device__ __forceinline__ uint64_t reread(const DevTable& t, uint32_t bin, uint32_t s) {
  return ld_slot(t.slots + (uint64_t)bin * B + s);
}

// Slots of `bin` this plan holds claims on (revisits hold none of their own).
__device__ __forceinline__ uint32_t own_slots(const Ctx& c, uint32_t bin) {
  uint32_t m = 0;
  for (int i = 0; i < c.pn; i++) {
    uint64_t e = desc_at(c, i);
    if (e_bin(e) == bin && !e_rev(e)) m |= 1u << e_slot(e);
  }
  return m;
}

// The plan's latest entry for slot s of `bin`, or -1.
__device__ __forceinline__ int last_entry_for(const Ctx& c, uint32_t bin, uint32_t s) {
  for (int i = c.pn - 1; i >= 0; i--) {
    uint64_t e = desc_at(c, i);
    if (e_bin(e) == bin && e_slot(e) == s) return i;
  }
  return -1;
}

// The record chain entry j receives: the new record, or the record entry
// j - 1 displaced.
__device__ __forceinline__ uint64_t placed_by(const Ctx& c, int j) {
  return j == 0 ? c.krec : content_at(c, j - 1);
}

// A queue-kicking step into slot s of `bin`, which the plan already holds
// (entry j placed the record there): the hit counter advances by CAS from
// the viewed metadata word, which also validates the view, and the new
// entry takes over entry j's write.
__device__ __forceinline__ bool claim_again(const DevTable& t, Ctx& c, uint32_t bin, uint32_t m, int s, int j,
                                            uint64_t victim) {
  if (!cas_acquire(t.meta + bin, m, m + HIT_ONE)) return false;
  set_entry(c, j, desc_at(c, j) | E_SUPERSEDED, content_at(c, j));
  put_entry(c, pack_entry(bin, s, K_MOVE, true, 0, 0) | E_REVISIT | ((uint64_t)j << 40), victim);
  return true;
}

// A new key straight into free slot s of `bin` (tables without ghosts):
// one 64-bit compare-and-swap of the slot from empty to the record, and for
// queue-kicking a relaxed add that advances the bin's hit counter (Sec. 6:
// every placement into a bin counts).  No claim is taken and the version
// does not move: the key moves nothing, so no reader that proves a miss and
// no planner's claim depends on it (a chain that had claimed this slot as
// its terminal finds it taken when its compare-and-swap commits, and starts
// again).  With one insertion in flight the slot and the policy's metadata
// end exactly as a claim and its release would leave them.
template <int B>
__device__ __forceinline__ bool place_direct(const DevTable& t, Ctx& c, uint32_t bin, int s, bool hit) {
  if (!cas_slot(t.slots + (uint64_t)bin * B + s, EMPTY, c.krec)) return false;
  if (hit) red_relaxed(t.meta + bin, HIT_ONE);
  return true;
}

// Abandon the plan: drop every claim (and hit increment).  Nothing was
// written, or (bump) every write was undone: then the version moves too, so
// that a reader validating a miss across the undone writes looks again.
__device__ __forceinline__ void release_all(const DevTable& t, Ctx& c, bool bump = false) {
  for (int i = 0; i < c.pn; i++) {
    uint64_t e = desc_at(c, i);
    red_relaxed(t.meta + e_bin(e),
                (bump ? VER_ONE : 0u) - ((e_rev(e) ? 0u : 1u << e_slot(e)) + (e_hit(e) ? HIT_ONE : 0u)));
  }
  c.pn = 0;
}

// The record `rec` may live in `bin`: it is a record (not an empty slot)
// and `bin` is one of its key's bins (Sec. 1).
template <int B>
__device__ __forceinline__ bool belongs(const DevTable& t, uint64_t rec, uint32_t bin) {
  if (rec == EMPTY) return false;
  if constexpr (B == 1) {
    uint32_t b[4];
    bins_of(t, key_of(rec), b);
    bool ok = false;
    for (uint32_t j = 0; j < t.d; j++) ok |= b[j] == bin;
    return ok;
  } else {
    uint32_t b0, b1;
    bins2(t, key_of(rec), b0, b1);
    return bin == b0 || bin == b1;
  }
}

// Chain entry i's slot.
template <int B>
__device__ __forceinline__ uint64_t* slot_at(const DevTable& t, uint64_t e) {
  return t.slots + (uint64_t)e_bin(e) * B + e_slot(e);
}

// Apply the plan back to front, then release every claim (Sec. 8).  Entry 0
// of the chain receives the new record, entry i the record entry i-1 held.
//
// Every slot of the plan was validated when it was claimed: a claim is a
// compare-and-swap of the bin's metadata word from the value seen when the
// bin was viewed, and since that word can come back to an earlier value (its
// version field wraps), the slot itself is read once more after the claim
// and must still hold the record the plan saw (reread; a search
// reads its path's records after claiming them and checks that each belongs
// to the bin it moves into).  A claimed slot holding a record cannot change
// until its claim is released, so the writes below need no further check --
// except the chain's terminal, the first write: a free terminal can be taken
// by a new key without a claim (place_direct), so it is written by a
// compare-and-swap, and if that fails nothing has been written and the
// caller abandons the plan (false).  With ordered writes a release fence
// separates consecutive writes, so a key is never absent for a concurrent
// reader; one fence then orders all writes before the relaxed releases, each
// of which also moves the version, duplicate mark or rattle counter of its
// slot.
template <int B>
__device__ __forceinline__ bool commit(const DevTable& t, Ctx& c) {
  if (c.pn == 0) return true;  // placed directly (place_direct)
  int n_chain = 0;
  while (n_chain < c.pn && (e_kind(desc_at(c, n_chain)) == K_MOVE || e_kind(desc_at(c, n_chain)) == K_DUPTERM))
    n_chain++;
  for (int i = n_chain - 1; i >= 0; i--) {
    const uint64_t e = desc_at(c, i);
    if (e_sup(e)) continue;  // a later revisit of this slot writes it
    const uint64_t rec = (i == 0) ? c.krec : content_at(c, i - 1);
    uint64_t* p = slot_at<B>(t, e);
    if (i == n_chain - 1) {
      if (!cas_slot(p, content_at(c, i), rec)) return false;
    } else {
      st_slot(p, rec);
    }
    if (t.ordered_writes && i > 0) fence_release();  // the copy lands before its source is overwritten
  }
  // ghost pairs (Sec. 4): the new record into both free slots
  for (int i = n_chain; i < c.pn; i++) {
    const uint64_t e = desc_at(c, i);
    if (e_kind(e) != K_GHOST) continue;
    if (!cas_slot(slot_at<B>(t, e), EMPTY, c.krec)) {
      for (int j = n_chain; j < i; j++) {
        const uint64_t f = desc_at(c, j);
        if (e_kind(f) == K_GHOST) st_slot(slot_at<B>(t, f), EMPTY);
      }
      fence_release();
      return false;
    }
  }
  fence_release();
  for (int i = 0; i < c.pn; i++) {
    uint64_t ei = desc_at(c, i);
    uint32_t sl = e_slot(ei);
    uint32_t delta = VER_ONE - (e_rev(ei) ? 0u : 1u << sl);
    if (B == 1) {
      delta += (e_new_r(ei) - e_old_r(ei)) << RATTLE_SHIFT;
    } else if (e_kind(ei) == K_GHOST) {
      delta += 1u << (DUP_SHIFT + sl);
    } else if (e_kind(ei) == K_DUPTERM || e_kind(ei) == K_TWIN) {
      delta -= 1u << (DUP_SHIFT + sl);
    }
    red_relaxed(t.meta + e_bin(ei), delta);
  }
  return true;
}

// A walk or search reached its cap or budget.  Without having met another
// insertion's claim that is the serial algorithm's failure; after detours
// around claims it is a conflict, retried.  Either way insert_one counts it
// as a failed attempt (capped), so a key that keeps running out ends FAILED
// after the failed-attempt retries instead of spending every conflict
// retry -- and the waits between them.
__device__ __forceinline__ int out_of_cap(Ctx& c) {
  c.capped = 1;
  return c.foreign ? ST_CONFLICT : ST_FAILED;
}

// No way on: every candidate slot or bin is claimed or already this
// chain's.  With other insertions' claims among them the key is blocked, a
// conflict like any other (retried up to max_retries); with none, the
// serial algorithm's failure.
__device__ __forceinline__ int dead_end(Ctx& c) {
  if (c.foreign) return ST_CONFLICT;
  c.capped = 1;
  return ST_FAILED;
}

// Claim both free slots of a ghost pair (Sec. 4), the lower bin first: two
// insertions whose keys hash to the same two bins in opposite order would
// otherwise each claim its first bin, fail on the other's, release, and
// meet again on every retry.
__device__ __forceinline__ bool claim_ghost_pair(const DevTable& t, Ctx& c, uint32_t b0, uint32_t m0, int s0,
                                                 uint32_t b1, uint32_t m1, int s1, bool hit) {
  if (b1 < b0) {
    if (!claim(t, c, b1, m1, s1, K_GHOST, hit, EMPTY)) return false;
    return claim(t, c, b0, m0, s0, K_GHOST, hit, EMPTY);
  }
  if (!claim(t, c, b0, m0, s0, K_GHOST, hit, EMPTY)) return false;
  return claim(t, c, b1, m1, s1, K_GHOST, hit, EMPTY);
}

__device__ __forceinline__ bool plan_has_bin(const Ctx& c, uint32_t bin) {
  for (int i = 0; i < c.pn; i++)
    if (e_bin(desc_at(c, i)) == bin) return true;
  return false;
}

// Every claimed slot of this view belongs to our own plan.
template <int B>
__device__ __forceinline__ bool claims_all_ours(const Ctx& c, uint32_t bin, uint32_t claimed) {
  uint32_t ours = 0;
  for (int i = 0; i < c.pn; i++)
    if (e_bin(desc_at(c, i)) == bin) ours |= 1u << e_slot(desc_at(c, i));
  return (claimed & ~ours) == 0;
}

// Claim the twin of the duplicate `g`, which lives in bin y (Sec. 4: the
// other copy loses its duplicate mark).  The twin's bin is read but not
// counted as viewed: only its metadata changes.
template <int B>
__device__ __forceinline__ bool claim_twin(const DevTable& t, Ctx& c, uint64_t g, uint32_t y) {
  for (int tries = 0; tries < 4; tries++) {
    View<B> v;
    load_view_fast<B>(t, y, v);
    uint32_t dm = dup_mask<B>(v);
    int s = -1;
#pragma unroll
    for (int u = 0; u < B; u++)
      if (s < 0 && ((dm >> u) & 1u) && v.s[u] == g) s = u;
    if (s < 0) return false;
    if (claim(t, c, y, v.m, s, K_TWIN, false, g)) return reread<B>(t, y, (uint32_t)s) == g;
  }
  return false;
}

// ------------------------------------------------------------------
// terminal moves shared by the two-choice policies
// ------------------------------------------------------------------

// Place the record into free slot s of a bin (terminal of a chain, or the
// new key directly).  Re-views the bin on a metadata change.
template <int B>
__device__ __forceinline__ int take_free(const DevTable& t, Ctx& c, uint32_t bin, View<B>& v, int s,
                                         bool hit) {
  for (int tries = 0;; tries++) {
    if (claim(t, c, bin, v.m, s, K_MOVE, hit, EMPTY)) return ST_OK;
    if (tries == 3) return ST_CONFLICT;
    load_view_fast<B>(t, bin, v);
    c.viewed++;
    c.reviews++;
    if (((free_mask<B>(v) >> s) & 1u) == 0) return ST_CONFLICT;
  }
}

// Overwrite the duplicate in slot s and unmark its twin.  The two copies
// are claimed lower bin first, so two insertions that each want one copy of
// the same ghost pair cannot hold one each and retry forever.
template <int B>
__device__ __forceinline__ int take_dup(const DevTable& t, Ctx& c, uint32_t bin, View<B>& v, int s,
                                        bool hit) {
  uint64_t g = slot_of<B>(v, s);
  uint32_t y = other_bin2(t, g, bin);
  if (y < bin) {
    if (!claim_twin<B>(t, c, g, y)) return ST_CONFLICT;
    if (!claim(t, c, bin, v.m, s, K_DUPTERM, hit, g)) return ST_CONFLICT;
    // keep the chain entries contiguous: the twin goes after the terminal
    const int a = c.pn - 2, b = c.pn - 1;
    uint64_t td = desc_at(c, a), tc = content_at(c, a);
    set_entry(c, a, desc_at(c, b), content_at(c, b));
    set_entry(c, b, td, tc);
  } else {
    if (!claim(t, c, bin, v.m, s, K_DUPTERM, hit, g)) return ST_CONFLICT;
    if (!claim_twin<B>(t, c, g, y)) return ST_CONFLICT;
  }
  c.dup_evict++;
  return ST_OK;
}

// Displace the record in slot s (a chain step).  On a metadata change the
// bin is viewed again and the step retried while slot s is still usable.
template <int B>
__device__ __forceinline__ int take_victim(const DevTable& t, Ctx& c, uint32_t bin, View<B>& v, int s,
                                           bool hit) {
  for (int tries = 0;; tries++) {
    if (claim(t, c, bin, v.m, s, K_MOVE, hit, slot_of<B>(v, s))) return ST_OK;
    if (tries == 3) return ST_CONFLICT;
    load_view_fast<B>(t, bin, v);
    c.viewed++;
    c.reviews++;
    uint32_t usable = ~claimed_mask<B>(v) & ~(v.m >> DUP_SHIFT);
    if (((usable >> s) & 1u) == 0 || slot_of<B>(v, s) == EMPTY) return ST_CONFLICT;
  }
}

// ------------------------------------------------------------------
// random kicking, two bins of B slots (Sec. 1; ghosts Sec. 4)
// ------------------------------------------------------------------
template <int B, bool GHOST>
__device__ int insert_random2(const DevTable& t, Ctx& c) {
  constexpr uint32_t FULL = (1u << B) - 1;
  uint32_t b0, b1;
  bins2(t, c.key, b0, b1);
  View<B> v0, v1;
  if (!GHOST) {
    // the first free slot of b0, then of b1, placed by a compare-and-swap
    // of the slot on unordered views
    load_view_fast<B>(t, b0, v0);
    c.viewed++;
    int s = lowest(free_mask<B>(v0));
    if (s >= 0) return place_direct<B>(t, c, b0, s, false) ? (int)ST_OK : (int)ST_CONFLICT;
    load_view_fast<B>(t, b1, v1);
    c.viewed++;
    s = lowest(free_mask<B>(v1));
    if (s >= 0) return place_direct<B>(t, c, b1, s, false) ? (int)ST_OK : (int)ST_CONFLICT;
    // both full: the views as read serve the walk (unordered metadata and
    // slots are fine: every move is re-validated after its claim)
  } else {
    load_view2_fast<B>(t, b0, b1, v0, v1);
    c.viewed += 2;
    uint32_t f0 = free_mask<B>(v0), f1 = free_mask<B>(v1);
    if (f0 && f1) {
      if (!claim_ghost_pair(t, c, b0, v0.m, lowest(f0), b1, v1.m, lowest(f1), false)) return ST_CONFLICT;
      c.ghosts_made++;
      return ST_OK;
    }
    if (f0) return take_free<B>(t, c, b0, v0, lowest(f0), false);
    if (f1) return take_free<B>(t, c, b1, v1, lowest(f1), false);
    uint32_t d0 = dup_mask<B>(v0), d1 = dup_mask<B>(v1);
    if (d0) return take_dup<B>(t, c, b0, v0, lowest(d0), false);
    if (d1) return take_dup<B>(t, c, b1, v1, lowest(d1), false);
  }
  // first victim: uniform over the usable slots of b0 then b1
  uint32_t e0 = FULL & ~claimed_mask<B>(v0) & ~(v0.m >> DUP_SHIFT);
  uint32_t e1 = FULL & ~claimed_mask<B>(v1) & ~(v1.m >> DUP_SHIFT);
  uint32_t n0 = __popc(e0), ne = n0 + __popc(e1);
  if (ne == 0) return ST_CONFLICT;
  uint32_t idx = (uint32_t)(draw(t, c.key, c.draws++, c.attempt) % ne);
  uint32_t x;
  int s;
  View<B> vx;
  if (idx < n0) { x = b0; vx = v0; s = nth_bit(e0, idx); }
  else { x = b1; vx = v1; s = nth_bit(e1, idx - n0); }
  // One kick a round trip: the victim's claim goes out together with the
  // view of the bin it moves to (metadata word and slots, unordered) and the
  // re-read of the slot the previous kick claimed (reread; that claim has
  // completed), which is compared once the claim is back.
  const uint64_t* pend = nullptr;
  uint64_t pend_v = 0;
  for (;;) {
    if (c.kicks == t.cap) return ST_FAILED;
    uint64_t victim = slot_of<B>(vx, s);
    uint32_t xn = other_bin2(t, victim, x);
    const uint64_t chk = pend ? ld_slot(pend) : 0;
    View<B> vn;
    load_view_fast<B>(t, xn, vn);
    int st = take_victim<B>(t, c, x, vx, s, false);
    if (st != ST_OK) return st;
    if (pend && chk != pend_v) return ST_CONFLICT;
    if (slot_of<B>(vx, s) != victim) {  // x was viewed again: another record is moving
      victim = slot_of<B>(vx, s);
      xn = other_bin2(t, victim, x);
      load_view_fast<B>(t, xn, vn);
    }
    c.kicks++;
    pend = t.slots + (uint64_t)x * B + s;
    pend_v = victim;
    x = xn;
    vx = vn;
    c.viewed++;
    uint32_t fm = free_mask<B>(vx);
    if (fm) {
      const uint64_t chk_last = ld_slot(pend);
      const int r = take_free<B>(t, c, x, vx, lowest(fm), false);
      return (r == ST_OK && chk_last != pend_v) ? (int)ST_CONFLICT : r;
    }
    if (GHOST) {
      uint32_t dm = dup_mask<B>(vx);
      if (dm) {
        const uint64_t chk_last = ld_slot(pend);
        const int r = take_dup<B>(t, c, x, vx, lowest(dm), false);
        return (r == ST_OK && chk_last != pend_v) ? (int)ST_CONFLICT : r;
      }
    }
    uint32_t claimed = claimed_mask<B>(vx);
    uint32_t e = FULL & ~claimed & ~(vx.m >> DUP_SHIFT);
    if (!e) return claims_all_ours<B>(c, x, claimed) ? ST_FAILED : ST_CONFLICT;
    if (int r0 = plan_room(t, c)) return r0;
    uint64_t r = draw(t, c.key, c.draws++, c.attempt);
    s = nth_bit(e, (uint32_t)(r % __popc(e)));
  }
}

// ------------------------------------------------------------------
// queue-kicking with hit counters and hit balancing (Sec. 6)
// ------------------------------------------------------------------
// Every placement into a bin takes its hit counter h and increments it (the
// claim of a kicked slot and the increment are one compare-and-swap, the GPU
// form of the paper's fetch-and-add scheduling).  A record goes to the
// lowest free slot (in insert-only tables the bin fills in slot order, so
// this is slot h mod B); a full bin gives up the record at h mod B, the one
// that has been there longest -- also when this chain placed it there on an
// earlier visit -- skipping only slots another insertion holds.
template <int B, bool GHOST>
__device__ int insert_queue(const DevTable& t, Ctx& c) {
  constexpr uint32_t FULL = (1u << B) - 1;
  uint32_t b0, b1;
  bins2(t, c.key, b0, b1);
  View<B> v0, v1;
  if (!GHOST) {
    // the common case first: the lowest empty slot of the less full bin,
    // taken by a compare-and-swap of the slot; only the two bins' slots are
    // read (an empty slot another insertion claimed as its chain's end is
    // taken all the same: that chain finds it gone when it commits)
    load_slots<B>(t, b0, v0);
    load_slots<B>(t, b1, v1);
    c.viewed += 2;
    uint32_t g0 = empty_mask<B>(v0), g1 = empty_mask<B>(v1);
    if (g0 | g1) {
      bool first = __popc(g0) >= __popc(g1);
      uint32_t x = first ? b0 : b1;
      int s = lowest(first ? g0 : g1);
      return place_direct<B>(t, c, x, s, true) ? (int)ST_OK : (int)ST_CONFLICT;
    }
    // both full: the metadata words, with the slots as read (unordered is
    // fine: every move is re-validated after its claim)
    v0.m = ld_relaxed(t.meta + b0);
    v1.m = ld_relaxed(t.meta + b1);
  } else {
    load_view2_fast<B>(t, b0, b1, v0, v1);
    c.viewed += 2;
  }
  uint32_t fm0 = free_mask<B>(v0), fm1 = free_mask<B>(v1);
  int f0 = __popc(fm0), f1 = __popc(fm1);
  if (GHOST && f0 > 0 && f1 > 0) {
    int s0 = lowest(fm0);
    int s1 = lowest(fm1);
    if (!claim_ghost_pair(t, c, b0, v0.m, s0, b1, v1.m, s1, true)) return ST_CONFLICT;
    c.ghosts_made++;
    return ST_OK;
  }
  uint32_t x;
  View<B> vx;
  if (f0 > 0 || f1 > 0) {
    bool first = f0 >= f1;
    x = first ? b0 : b1;
    vx = first ? v0 : v1;
  } else if (GHOST && (dup_mask<B>(v0) || dup_mask<B>(v1))) {
    bool first = dup_mask<B>(v0) != 0;
    x = first ? b0 : b1;
    vx = first ? v0 : v1;
  } else {
    bool first = hit_of(v0.m) <= hit_of(v1.m);
    x = first ? b0 : b1;
    vx = first ? v0 : v1;
  }
  // One kick a round trip: the claim goes out together with the view of
  // the next bin (metadata word and slots, unordered) and the re-read of the
  // slot the previous kick claimed (reread; that claim has completed),
  // compared once the claim is back.
  const uint64_t* pend = nullptr;
  uint64_t pend_v = 0;
  for (;;) {
    int tries = 0;
    for (;;) {  // one step at bin x: free slot, duplicate, or victim from hit mod B
      uint32_t h = hit_of(vx.m) % B;
      uint32_t fm = free_mask<B>(vx);
      const uint64_t chk = pend ? ld_slot(pend) : 0;
      if (fm) {
        if (claim(t, c, x, vx.m, lowest(fm), K_MOVE, true, EMPTY))
          return (pend && chk != pend_v) ? (int)ST_CONFLICT : (int)ST_OK;
      } else if (GHOST && dup_mask<B>(vx)) {
        const int r = take_dup<B>(t, c, x, vx, first_from<B>(dup_mask<B>(vx), h), true);
        return (r == ST_OK && pend && chk != pend_v) ? (int)ST_CONFLICT : r;
      } else {
        // the victim: the record at slot h mod B, skipping slots another
        // insertion holds; a slot this chain already wrote is taken again
        // (the walk came back to the bin; its queue has moved on), with the
        // record the chain put there
        uint32_t claimed = claimed_mask<B>(vx);
        uint32_t own = claimed ? own_slots(c, x) : 0u;
        uint32_t foreign = claimed & ~own;
        uint32_t um = FULL & ~foreign & ~((vx.m >> DUP_SHIFT) & ~own);
        // a detour around another insertion's claim: reaching the cap after
        // one is not the serial algorithm's failure
        if (foreign) c.foreign = 1;
        int s = first_from<B>(um, h);
        if (s < 0) return dead_end(c);
        if (c.kicks == t.cap) return out_of_cap(c);
        if (int r0 = plan_room(t, c)) return r0;
        const bool rev = (own >> s) & 1u;
        const int jprev = rev ? last_entry_for(c, x, (uint32_t)s) : -1;
        const uint64_t victim = rev ? placed_by(c, jprev) : slot_of<B>(vx, s);
        const uint32_t xn = other_bin2(t, victim, x);
        View<B> vn;
        load_view_fast<B>(t, xn, vn);
        if (rev ? claim_again(t, c, x, vx.m, s, jprev, victim) : claim(t, c, x, vx.m, s, K_MOVE, true, victim)) {
          if (pend && chk != pend_v) return ST_CONFLICT;
          c.kicks++;
          // a slot the chain holds already carries the plan's record: no re-read
          pend = rev ? nullptr : t.slots + (uint64_t)x * B + s;
          pend_v = victim;
          x = xn;
          vx = vn;
          break;
        }
      }
      if (++tries == 4) return ST_CONFLICT;
      load_view_fast<B>(t, x, vx);
      c.viewed++;
      c.reviews++;
    }
    c.viewed++;
  }
}

// ------------------------------------------------------------------
// d-ary tables, single-slot bins (Sec. 7)
// ------------------------------------------------------------------

// Random kicking: view h_0.. in order until an empty bin; when all d are
// full displace the occupant of a uniformly drawn h_j, which moves to a
// uniformly drawn bin of its own that the chain has not written, and so on.
__device__ inline int insert_random_dary(const DevTable& t, Ctx& c) {
  uint32_t b[4];
  bins_of(t, c.key, b);
  View<1> v[4];
#pragma unroll
  for (int i = 0; i < 4; i++)
    if (i < (int)t.d) load_view_fast<1>(t, b[i], v[i]);  // the d loads overlap
  for (uint32_t i = 0; i < t.d; i++) {
    c.viewed++;
    if (free_mask<1>(v[i]) && take_free<1>(t, c, b[i], v[i], 0, false) == ST_OK) return ST_OK;
  }
  // Every bin of the record in hand is full: displace the occupant of a
  // uniformly drawn candidate -- one of the record's bins whose claim flag
  // is clear.  With one insertion in flight the set claims are exactly this
  // chain's own, so these are the bins the chain has not written.  The
  // candidates' slots are fetched together; only the drawn one counts as
  // viewed.  A candidate another insertion took meanwhile is dropped and the
  // draw repeated.
  uint32_t cb[4], nc = 0;
  View<1> cv[4];
  for (uint32_t i = 0; i < t.d; i++) {
    if (!claimed_mask<1>(v[i])) { cb[nc] = b[i]; cv[nc] = v[i]; nc++; }
    else c.foreign = 1;  // no claim of ours exists before the first kick
  }
  bool counted = true;  // the first candidates were counted above
  uint32_t holder = NO_BIN;  // the bin whose record is in hand (the last one claimed)
  // One kick a round trip: the displaced record's other bins are viewed
  // together with its claim, and the slot the previous kick claimed is read
  // again (reread) in the same round trip.
  const uint64_t* pend = nullptr;
  uint64_t pend_v = 0;
  uint32_t vb[4];
  View<1> w[4];
  for (uint32_t waits = 0;;) {
    if (nc == 0 && c.foreign && holder != NO_BIN && waits < 8) {
      // every candidate is held by other insertions, which release their
      // claims within microseconds: view the candidates again rather than
      // abandon the whole walk (a bounded wait, so no deadlock)
      __nanosleep(256u << waits);
      waits++;
      bins_of(t, key_of(c.held), vb);
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (i < (int)t.d && vb[i] != holder) load_view_fast<1>(t, vb[i], w[i]);
      for (uint32_t i = 0; i < t.d; i++) {
        if (vb[i] == holder) continue;
        if (!claimed_mask<1>(w[i])) { cb[nc] = vb[i]; cv[nc] = w[i]; nc++; }
      }
      c.reviews += nc;
      continue;
    }
    if (nc == 0) return dead_end(c);
    uint32_t k = (uint32_t)(draw(t, c.key, c.draws++, c.attempt) % nc);
    uint32_t x = cb[k];
    View<1> vx = cv[k];
    if (!counted) c.viewed++;
    bool kicked = false, lost = false;
    for (int tries = 0; tries < 4 && !kicked && !lost; tries++) {
      if (tries) {  // lost a race for x: view it again
        load_view_fast<1>(t, x, vx);
        c.viewed++;
        c.reviews++;
      }
      if (claimed_mask<1>(vx)) { lost = true; break; }
      const uint64_t chk = pend ? ld_slot(pend) : 0;
      if (vx.s[0] == EMPTY) {
        if (claim(t, c, x, vx.m, 0, K_MOVE, false, EMPTY))
          return (pend && chk != pend_v) ? (int)ST_CONFLICT : (int)ST_OK;
        continue;
      }
      if (c.kicks == t.cap) return ST_FAILED;
      if (int r = plan_room(t, c)) return r;
      bins_of(t, key_of(vx.s[0]), vb);
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (i < (int)t.d && vb[i] != x) load_view_fast<1>(t, vb[i], w[i]);
      kicked = claim(t, c, x, vx.m, 0, K_MOVE, false, vx.s[0]);
      if (kicked && pend && chk != pend_v) return ST_CONFLICT;
    }
    if (!kicked) {
      c.foreign = 1;
      cb[k] = cb[nc - 1];
      cv[k] = cv[nc - 1];
      nc--;
      continue;
    }
    c.kicks++;
    holder = x;
    c.held = vx.s[0];
    pend = t.slots + x;
    pend_v = c.held;
    nc = 0;
    for (uint32_t i = 0; i < t.d; i++) {
      if (vb[i] == x) continue;  // just claimed by this chain
      if (!claimed_mask<1>(w[i])) { cb[nc] = vb[i]; cv[nc] = w[i]; nc++; }
      else if (!plan_has_bin(c, vb[i])) c.foreign = 1;
    }
    counted = false;
  }
}

// Rattle-kicking with rattle balancing (Sec. 7).  r counts the bins a key
// has tried; the key tries h_{r mod d}, r increments (saturating at 255);
// the larger counter keeps the bin, the incoming key on a tie (or the
// resident, under the debug reading); the loser tries its next bin.  The
// counter of a resident key lives in its bin's metadata word.
__device__ inline int insert_rattle(const DevTable& t, Ctx& c) {
  uint64_t cur = c.krec;
  uint32_t rc = 0;
  const uint64_t* pend = nullptr;  // the slot the last kick claimed, re-read with the next view (reread)
  uint64_t pend_v = 0;
  for (uint32_t tries = 0;; tries++) {
    if (tries == t.cap) return out_of_cap(c);
    if (int r = plan_room(t, c)) return r;
    uint32_t vb[4];
    bins_of(t, key_of(cur), vb);
    uint32_t x = vb[rc % t.d];
    rc = rc < 255 ? rc + 1 : 255;
    View<1> vx;
    const uint64_t chk = pend ? ld_slot(pend) : 0;
    load_view_fast<1>(t, x, vx);
    if (pend) {
      if (chk != pend_v) return ST_CONFLICT;
      pend = nullptr;
    }
    if (claimed_mask<1>(vx)) {
      // this chain's own bin: skipped, not viewed; another insertion's:
      // viewed and ignored (Sec. 8)
      if (!plan_has_bin(c, x)) {
        c.viewed++;
        c.foreign = 1;
      }
      continue;
    }
    c.viewed++;
    bool moved = false, skip = false;
    for (int k = 0; k < 4 && !moved && !skip; k++) {
      if (k) {
        load_view_fast<1>(t, x, vx);
        c.viewed++;
        c.reviews++;
        if (claimed_mask<1>(vx)) {
          c.foreign = 1;
          skip = true;
          break;
        }
      }
      if (vx.s[0] == EMPTY) {
        if (claim(t, c, x, vx.m, 0, K_MOVE, false, EMPTY, rattle_of(vx.m), rc)) return ST_OK;
        continue;
      }
      uint32_t ry = rattle_of(vx.m);
      bool incoming_stays = t.tie_resident ? (rc > ry) : (rc >= ry);
      if (!incoming_stays) { skip = true; break; }
      if (claim(t, c, x, vx.m, 0, K_MOVE, false, vx.s[0], ry, rc)) {
        c.kicks++;
        cur = vx.s[0];
        rc = ry;
        moved = true;
        pend = t.slots + x;
        pend_v = cur;
      }
    }
    if (!moved && !skip) return ST_CONFLICT;
  }
}

}  // namespace ck
