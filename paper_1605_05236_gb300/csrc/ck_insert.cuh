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

// A plan: parallel arrays of claimed slots.  The arrays live in local
// memory (MAX_CHAIN entries, the concurrent kernel) or in table scratch
// (LONG_CHAIN entries, the serial replay and the pass for long chains).
struct Plan {
  uint64_t* content;  // record the slot held when claimed (EMPTY for a free slot)
  uint32_t* bin;
  uint8_t* slot;
  uint8_t* kind;
  uint8_t* hit;       // the claim also advanced the hit counter
  uint8_t* old_r;     // d-ary: rattle counter stored with the displaced key
  uint8_t* new_r;     // d-ary: rattle counter stored with the incoming key
  int n;
  int cap;            // entries the arrays hold
};

template <int N>
struct PlanStore {
  uint64_t content[N];
  uint32_t bin[N];
  uint8_t slot[N], kind[N], hit[N], old_r[N], new_r[N];
  __device__ __forceinline__ Plan view() {
    Plan p{content, bin, slot, kind, hit, old_r, new_r, 0, N};
    return p;
  }
};

// Plan arrays carved from a scratch region of LONG_REGION bytes.
__device__ __forceinline__ Plan plan_in(uint8_t* r) {
  Plan p;
  p.content = reinterpret_cast<uint64_t*>(r);
  p.bin = reinterpret_cast<uint32_t*>(r + 8 * LONG_CHAIN);
  p.slot = r + 12 * LONG_CHAIN;
  p.kind = r + 13 * LONG_CHAIN;
  p.hit = r + 14 * LONG_CHAIN;
  p.old_r = r + 15 * LONG_CHAIN;
  p.new_r = r + 16 * LONG_CHAIN;
  p.n = 0;
  p.cap = LONG_CHAIN;
  return p;
}

struct Ctx {
  uint32_t key;
  uint64_t krec;
  uint32_t attempt;
  uint32_t viewed;   // bins viewed, all attempts
  uint32_t viewed0;  // `viewed` when the current attempt started
  uint32_t reviews;  // bins viewed again because a claim lost a race (part of `viewed`)
  uint32_t foreign;  // the attempt ignored a slot another insertion had claimed
  uint32_t kicks;    // kick-outs of the current attempt
  uint32_t draws;    // random draws of the current attempt
  uint32_t ghosts_made;
  uint32_t dup_evict;
  Plan* plan;
};

// Claim slot s of `bin` by CAS from the viewed metadata word m (extra: the
// hit-counter increment of queue-kicking) and append the entry.
__device__ __forceinline__ bool claim(const DevTable& t, Ctx& c, uint32_t bin, uint32_t m, int s,
                                      uint64_t content, uint8_t kind, bool hit,
                                      uint8_t old_r = 0, uint8_t new_r = 0) {
  uint32_t desired = m + (hit ? HIT_ONE : 0u) + (1u << s);
  if (!cas_acquire(t.meta + bin, m, desired)) return false;
  Plan& p = *c.plan;
  int i = p.n++;
  p.content[i] = content;
  p.bin[i] = bin;
  p.slot[i] = (uint8_t)s;
  p.kind[i] = kind;
  p.hit[i] = hit ? 1 : 0;
  p.old_r[i] = old_r;
  p.new_r[i] = new_r;
  return true;
}

// Abandon the plan: drop every claim (and hit increment); nothing was written.
__device__ __forceinline__ void release_all(const DevTable& t, Ctx& c) {
  Plan& p = *c.plan;
  for (int i = 0; i < p.n; i++)
    add_relaxed(t.meta + p.bin[i], 0u - ((1u << p.slot[i]) + (p.hit[i] ? HIT_ONE : 0u)));
  p.n = 0;
}

// Apply the plan back to front, then release every claim with one atomic
// per slot that also moves the version, duplicate mark and rattle counter.
template <int B>
__device__ __forceinline__ void commit(const DevTable& t, Ctx& c) {
  Plan& p = *c.plan;
  int n_chain = 0;
  while (n_chain < p.n && (p.kind[n_chain] == K_MOVE || p.kind[n_chain] == K_DUPTERM)) n_chain++;
  for (int i = n_chain - 1; i >= 0; i--) {
    uint64_t rec = (i == 0) ? c.krec : p.content[i - 1];
    st_slot(t.slots + (uint64_t)p.bin[i] * B + p.slot[i], rec);
    if (t.ordered_writes && i > 0) fence_release();  // the copy lands before its source is overwritten
  }
  for (int i = n_chain; i < p.n; i++)
    if (p.kind[i] == K_GHOST) st_slot(t.slots + (uint64_t)p.bin[i] * B + p.slot[i], c.krec);
  for (int i = 0; i < p.n; i++) {
    uint32_t delta = VER_ONE - (1u << p.slot[i]);
    if (B == 1) {
      delta += ((uint32_t)p.new_r[i] - (uint32_t)p.old_r[i]) << RATTLE_SHIFT;
    } else if (p.kind[i] == K_GHOST) {
      delta += 1u << (DUP_SHIFT + p.slot[i]);
    } else if (p.kind[i] == K_DUPTERM || p.kind[i] == K_TWIN) {
      delta -= 1u << (DUP_SHIFT + p.slot[i]);
    }
    add_release(t.meta + p.bin[i], delta);
  }
}

// A cap reached without meeting another insertion's claim is a genuine
// failure; one reached after detours around claims is retried instead.
__device__ __forceinline__ bool claims_none_foreign(const Ctx& c) { return !c.foreign; }

__device__ __forceinline__ bool plan_has_bin(const Plan& p, uint32_t bin) {
  for (int i = 0; i < p.n; i++)
    if (p.bin[i] == bin) return true;
  return false;
}

// Every claimed slot of this view belongs to our own plan.
template <int B>
__device__ __forceinline__ bool claims_all_ours(const Plan& p, uint32_t bin, uint32_t claimed) {
  uint32_t ours = 0;
  for (int i = 0; i < p.n; i++)
    if (p.bin[i] == bin) ours |= 1u << p.slot[i];
  return (claimed & ~ours) == 0;
}

// Claim the twin of the duplicate `g`, which lives in bin y (Sec. 4: the
// other copy loses its duplicate mark).  The twin's bin is read but not
// counted as viewed: only its metadata changes.
template <int B>
__device__ __forceinline__ bool claim_twin(const DevTable& t, Ctx& c, uint64_t g, uint32_t y) {
  for (int tries = 0; tries < 4; tries++) {
    View<B> v;
    load_view<B>(t, y, v);
    uint32_t dm = dup_mask<B>(v);
    int s = -1;
#pragma unroll
    for (int u = 0; u < B; u++)
      if (s < 0 && ((dm >> u) & 1u) && v.s[u] == g) s = u;
    if (s < 0) return false;
    if (claim(t, c, y, v.m, s, g, K_TWIN, false)) return true;
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
    if (claim(t, c, bin, v.m, s, EMPTY, K_MOVE, hit)) return ST_OK;
    if (tries == 3) return ST_CONFLICT;
    load_view<B>(t, bin, v);
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
  uint64_t g = v.s[s];
  uint32_t y = other_bin2(t, g, bin);
  if (y < bin) {
    if (!claim_twin<B>(t, c, g, y)) return ST_CONFLICT;
    if (!claim(t, c, bin, v.m, s, g, K_DUPTERM, hit)) return ST_CONFLICT;
    // keep the chain entries contiguous: the twin goes after the terminal
    Plan& p = *c.plan;
    int a = p.n - 2, b = p.n - 1;
    uint64_t tc = p.content[a]; p.content[a] = p.content[b]; p.content[b] = tc;
    uint32_t tb = p.bin[a]; p.bin[a] = p.bin[b]; p.bin[b] = tb;
    uint8_t t8;
    t8 = p.slot[a]; p.slot[a] = p.slot[b]; p.slot[b] = t8;
    t8 = p.kind[a]; p.kind[a] = p.kind[b]; p.kind[b] = t8;
    t8 = p.hit[a]; p.hit[a] = p.hit[b]; p.hit[b] = t8;
    t8 = p.old_r[a]; p.old_r[a] = p.old_r[b]; p.old_r[b] = t8;
    t8 = p.new_r[a]; p.new_r[a] = p.new_r[b]; p.new_r[b] = t8;
  } else {
    if (!claim(t, c, bin, v.m, s, g, K_DUPTERM, hit)) return ST_CONFLICT;
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
    if (claim(t, c, bin, v.m, s, v.s[s], K_MOVE, hit)) return ST_OK;
    if (tries == 3) return ST_CONFLICT;
    load_view<B>(t, bin, v);
    c.viewed++;
    c.reviews++;
    uint32_t usable = ~claimed_mask<B>(v) & ~(v.m >> DUP_SHIFT);
    if (((usable >> s) & 1u) == 0 || v.s[s] == EMPTY) return ST_CONFLICT;
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
    load_view<B>(t, b0, v0);
    c.viewed++;
    int s = lowest(free_mask<B>(v0));
    if (s >= 0) return take_free<B>(t, c, b0, v0, s, false);
    load_view<B>(t, b1, v1);
    c.viewed++;
    s = lowest(free_mask<B>(v1));
    if (s >= 0) return take_free<B>(t, c, b1, v1, s, false);
  } else {
    load_view<B>(t, b0, v0);
    load_view<B>(t, b1, v1);
    c.viewed += 2;
    uint32_t f0 = free_mask<B>(v0), f1 = free_mask<B>(v1);
    if (f0 && f1) {
      if (!claim(t, c, b0, v0.m, lowest(f0), EMPTY, K_GHOST, false)) return ST_CONFLICT;
      if (!claim(t, c, b1, v1.m, lowest(f1), EMPTY, K_GHOST, false)) return ST_CONFLICT;
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
  for (;;) {
    if (c.kicks == t.cap) return ST_FAILED;
    int st = take_victim<B>(t, c, x, vx, s, false);
    if (st != ST_OK) return st;
    c.kicks++;
    uint64_t victim = vx.s[s];
    x = other_bin2(t, victim, x);
    load_view<B>(t, x, vx);
    c.viewed++;
    uint32_t fm = free_mask<B>(vx);
    if (fm) return take_free<B>(t, c, x, vx, lowest(fm), false);
    if (GHOST) {
      uint32_t dm = dup_mask<B>(vx);
      if (dm) return take_dup<B>(t, c, x, vx, lowest(dm), false);
    }
    uint32_t claimed = claimed_mask<B>(vx);
    uint32_t e = FULL & ~claimed & ~(vx.m >> DUP_SHIFT);
    if (!e) return claims_all_ours<B>(*c.plan, x, claimed) ? ST_FAILED : ST_CONFLICT;
    if (c.plan->n >= c.plan->cap - 4) return ST_LONG;
    uint64_t r = draw(t, c.key, c.draws++, c.attempt);
    s = nth_bit(e, (uint32_t)(r % __popc(e)));
  }
}

// ------------------------------------------------------------------
// queue-kicking with hit counters and hit balancing (Sec. 6)
// ------------------------------------------------------------------
// The claim of a slot and the increment of the bin's hit counter are one
// compare-and-swap, the GPU form of the paper's fetch-and-add scheduling:
// B insertions arriving at one bin are handed B different slots.
template <int B, bool GHOST>
__device__ int insert_queue(const DevTable& t, Ctx& c) {
  constexpr uint32_t FULL = (1u << B) - 1;
  uint32_t b0, b1;
  bins2(t, c.key, b0, b1);
  View<B> v0, v1;
  load_view<B>(t, b0, v0);
  load_view<B>(t, b1, v1);
  c.viewed += 2;
  uint32_t fm0 = free_mask<B>(v0), fm1 = free_mask<B>(v1);
  int f0 = __popc(fm0), f1 = __popc(fm1);
  if (GHOST && f0 > 0 && f1 > 0) {
    int s0 = first_from<B>(fm0, hit_of(v0.m) % B);
    int s1 = first_from<B>(fm1, hit_of(v1.m) % B);
    if (!claim(t, c, b0, v0.m, s0, EMPTY, K_GHOST, true)) return ST_CONFLICT;
    if (!claim(t, c, b1, v1.m, s1, EMPTY, K_GHOST, true)) return ST_CONFLICT;
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
  for (;;) {
    int tries = 0;
    for (;;) {  // one step at bin x: free slot, duplicate, or victim from hit mod B
      uint32_t h = hit_of(vx.m) % B;
      uint32_t fm = free_mask<B>(vx);
      if (fm) {
        if (claim(t, c, x, vx.m, first_from<B>(fm, h), EMPTY, K_MOVE, true)) return ST_OK;
      } else if (GHOST && dup_mask<B>(vx)) {
        return take_dup<B>(t, c, x, vx, first_from<B>(dup_mask<B>(vx), h), true);
      } else {
        uint32_t claimed = claimed_mask<B>(vx);
        uint32_t um = FULL & ~claimed & ~(vx.m >> DUP_SHIFT);
        int s = first_from<B>(um, h);
        if (s < 0) return claims_all_ours<B>(*c.plan, x, claimed) ? ST_FAILED : ST_CONFLICT;
        if (c.kicks == t.cap) return ST_FAILED;
        if (c.plan->n >= c.plan->cap - 4) return ST_LONG;
        if (claim(t, c, x, vx.m, s, vx.s[s], K_MOVE, true)) {
          c.kicks++;
          x = other_bin2(t, vx.s[s], x);
          break;
        }
      }
      if (++tries == 4) return ST_CONFLICT;
      load_view<B>(t, x, vx);
      c.viewed++;
      c.reviews++;
    }
    load_view<B>(t, x, vx);
    c.viewed++;
  }
}

// ------------------------------------------------------------------
// d-ary tables, single-slot bins (Sec. 7)
// ------------------------------------------------------------------

// Random kicking: view h_0.. in order until an empty bin; when all d are
// full displace the occupant of a uniformly drawn h_j, which moves to a
// uniformly drawn bin of its own that the chain has not written, and so on.
__device__ int insert_random_dary(const DevTable& t, Ctx& c) {
  uint32_t b[4];
  bins_of(t, c.key, b);
  View<1> v[4];
#pragma unroll
  for (int i = 0; i < 4; i++)
    if (i < (int)t.d) load_view<1>(t, b[i], v[i]);  // the d loads overlap
  for (uint32_t i = 0; i < t.d; i++) {
    c.viewed++;
    if (free_mask<1>(v[i])) return take_free<1>(t, c, b[i], v[i], 0, false);
  }
  // all d full: a uniform unclaimed h_j (claimed bins are ignored, Sec. 8)
  uint32_t elig[4], ne = 0;
  for (uint32_t i = 0; i < t.d; i++)
    if (!claimed_mask<1>(v[i])) elig[ne++] = i;
  if (ne == 0) return ST_CONFLICT;
  uint32_t j = elig[draw(t, c.key, c.draws++, c.attempt) % ne];
  uint32_t x = b[j];
  View<1> vx = v[j];
  for (;;) {
    if (c.kicks == t.cap) return ST_FAILED;
    if (c.plan->n >= c.plan->cap - 4) return ST_LONG;
    int st = take_victim<1>(t, c, x, vx, 0, false);
    if (st != ST_OK) return st;
    c.kicks++;
    uint64_t victim = vx.s[0];
    uint32_t vb[4], cand[4], nc = 0;
    bins_of(t, key_of(victim), vb);
    for (uint32_t i = 0; i < t.d; i++)
      if (!plan_has_bin(*c.plan, vb[i])) cand[nc++] = vb[i];
    // a uniform bin of the victim's own that this chain has not written;
    // one another insertion holds is dropped and the draw repeated
    for (;;) {
      if (nc == 0) return claims_none_foreign(c) ? ST_FAILED : ST_CONFLICT;
      uint32_t k = (uint32_t)(draw(t, c.key, c.draws++, c.attempt) % nc);
      x = cand[k];
      load_view<1>(t, x, vx);
      c.viewed++;
      if (!claimed_mask<1>(vx)) break;
      c.foreign = 1;
      cand[k] = cand[--nc];
    }
    if (free_mask<1>(vx)) return take_free<1>(t, c, x, vx, 0, false);
  }
}

// Rattle-kicking with rattle balancing (Sec. 7).  r counts the bins a key
// has tried; the key tries h_{r mod d}, r increments (saturating at 255);
// the larger counter keeps the bin, the incoming key on a tie (or the
// resident, under the debug reading); the loser tries its next bin.  The
// counter of a resident key lives in its bin's metadata word.
__device__ int insert_rattle(const DevTable& t, Ctx& c) {
  uint64_t cur = c.krec;
  uint32_t rc = 0;
  for (uint32_t tries = 0;; tries++) {
    if (tries == t.cap) return claims_none_foreign(c) ? ST_FAILED : ST_CONFLICT;
    if (c.plan->n >= c.plan->cap - 4) return ST_LONG;
    uint32_t vb[4];
    bins_of(t, key_of(cur), vb);
    uint32_t x = vb[rc % t.d];
    rc = rc < 255 ? rc + 1 : 255;
    if (plan_has_bin(*c.plan, x)) continue;
    View<1> vx;
    load_view<1>(t, x, vx);
    c.viewed++;
    bool moved = false, skip = false;
    for (int k = 0; k < 4 && !moved && !skip; k++) {
      if (k) {
        load_view<1>(t, x, vx);
        c.viewed++;
        c.reviews++;
      }
      if (claimed_mask<1>(vx)) {  // another insertion holds it: ignore the bin (Sec. 8)
        c.foreign = 1;
        skip = true;
        break;
      }
      if (vx.s[0] == EMPTY) {
        if (claim(t, c, x, vx.m, 0, EMPTY, K_MOVE, false, (uint8_t)rattle_of(vx.m), (uint8_t)rc)) return ST_OK;
        continue;
      }
      uint32_t ry = rattle_of(vx.m);
      bool incoming_stays = t.tie_resident ? (rc > ry) : (rc >= ry);
      if (!incoming_stays) { skip = true; break; }
      if (claim(t, c, x, vx.m, 0, vx.s[0], K_MOVE, false, (uint8_t)ry, (uint8_t)rc)) {
        c.kicks++;
        cur = vx.s[0];
        rc = ry;
        moved = true;
      }
    }
    if (!moved && !skip) return ST_CONFLICT;
  }
}

}  // namespace ck
