// ck_search.cuh -- breadth-first search, sorted search and their hybrid
// for a kick-out chain (Kuszmaul, arXiv:1605.05236, Sec. 5), with ghost
// insertions (Sec. 4) and claim flags (Sec. 8).
//
// Candidates are the records of the bins viewed so far that have not been
// spawned, kept as groups (one per viewed bin, in viewing order; a group's
// records pop in slot order).  Spawning a record views its other bin; a
// free slot there (or, with ghosts, a duplicate) ends the search.  A bin
// already viewed is never viewed again (the small visited set of Sec. 5,
// bin index as hash).  BFS pops the oldest candidate; sorted search pops the
// candidate with the smallest spawn count, oldest first among equals, where
// a candidate's count is its bin's spawn count when the bin was viewed
// (the bucket-sort key of Sec. 5).  Spawning a record increments the spawn
// count of its bin (4 bits, saturating), and the increment stays even if
// the search fails.  The hybrid (end of Sec. 5) orders candidates by the
// depth at which they were spawn victims (records of b0 and b1: 0), then
// by that spawn count, oldest first among equals, and counts spawns like
// sorted search.
//
// The search itself takes no claims.  When it succeeds, every slot of the
// path is claimed by CAS from the metadata word read when its bin was
// viewed; a bin that changed since then aborts the attempt, and so does a
// record, read after its claim, that does not belong to the bin the path
// moves it into (the word came back to its viewed value meanwhile).
//
// Per-searcher scratch (global memory, SEARCH_REGION bytes): a header
// holding a generation counter and the bucket queues that give sorted
// search and the hybrid their next candidate in constant time, MAX_GROUPS
// group records, and an open-addressed visited set tagged with the
// generation (cleared only when the generation wraps).  The d-ary BFS
// keeps the record of the group it spawns from, with its bins and their
// visited tests, in registers (GroupCache).  In concurrent mode a search that spent its budget
// without meeting another insertion's claim is retried with four times the
// budget in a larger space borrowed from the table's scratch plans
// (search_space): the layout concurrent filling produces differs from the
// serial one, and a key the serial order places within the budget can need
// more in it.  The serial replay never retries, so it keeps the budget.
#pragma once
#include "ck_insert.cuh"

namespace ck {

struct Group {
  uint32_t bin;
  uint32_t meta;    // metadata word as viewed (updated by our own spawn increments)
  uint16_t parent;  // (group << 3) | slot of the record that led here; NO_PARENT at a root
  uint16_t link;    // sorted search, hybrid: the next group in the same bucket
  uint8_t next;     // next slot to pop
  uint8_t stale;    // the bin changed under us: a path through it aborts
  uint16_t key;     // sort key: spawn count when viewed (hybrid: depth * 16 + that count)
};
static_assert(sizeof(Group) == 16, "group record is 16 bytes");
constexpr uint32_t NO_PARENT = 0xFFFFu;

// Region header: the generation word, then (sorted search, hybrid) the
// bucket queues of candidate groups, 32 heads and 32 tails of 16 bits.
constexpr size_t SEARCH_HDR = 16 + 64 * sizeof(uint16_t);
constexpr size_t SEARCH_REGION = SEARCH_HDR + MAX_GROUPS * sizeof(Group) + VISITED_SLOTS * 8;

// A larger search space for the retry of a search that ran out of budget in
// concurrent mode: a scratch plan region (LONG_REGION bytes) holds the
// header, BIG_GROUPS group records and a visited set of BIG_VISITED slots.
constexpr int BIG_GROUPS = 2048;
constexpr int BIG_VISITED = 4096;
static_assert(SEARCH_HDR + BIG_GROUPS * 16 + BIG_VISITED * 8 <= LONG_REGION, "a big search fits a scratch plan region");
static_assert(((BIG_GROUPS - 1) << 3 | 7) < NO_PARENT, "a parent reference fits 16 bits");
static_assert((1 << 10) == VISITED_SLOTS && (1 << 12) == BIG_VISITED, "visited sets are powers of two");

// Where one search keeps its state, and how much it may use.
struct SearchSpace {
  uint32_t* hdr;
  Group* G;
  uint64_t* vis;
  uint32_t max_groups;
  uint32_t vis_bits;  // the visited set has 2^vis_bits slots
  uint32_t budget;    // bins viewed
};

// The ordinary space (the searcher's region, the table's budget), or, when
// the insertion holds a big region (c.big_id), that region with four times
// the budget.
__device__ __forceinline__ SearchSpace search_space(const DevTable& t, const Ctx& c, uint8_t* region) {
  SearchSpace s;
  if (c.big_id >= 0) {
    uint8_t* r = t.long_scratch + (uint64_t)c.big_id * LONG_REGION;
    s.hdr = reinterpret_cast<uint32_t*>(r);
    s.G = reinterpret_cast<Group*>(r + SEARCH_HDR);
    s.vis = reinterpret_cast<uint64_t*>(r + SEARCH_HDR + BIG_GROUPS * sizeof(Group));
    s.max_groups = BIG_GROUPS;
    s.vis_bits = 12;
    s.budget = min(4u * t.cap, (uint32_t)BIG_GROUPS - 8u);
  } else {
    s.hdr = reinterpret_cast<uint32_t*>(region);
    s.G = reinterpret_cast<Group*>(region + SEARCH_HDR);
    s.vis = reinterpret_cast<uint64_t*>(region + SEARCH_HDR + MAX_GROUPS * sizeof(Group));
    s.max_groups = MAX_GROUPS;
    s.vis_bits = 10;
    s.budget = t.cap;
  }
  return s;
}

__device__ __forceinline__ uint32_t vis_hash(uint32_t bin, uint32_t bits) { return (bin * 0x9E3779B1u) >> (32 - bits); }

// Bring a bin's slots and metadata word toward L2 ahead of its view.
template <int B>
__device__ __forceinline__ void prefetch_bin(const DevTable& t, uint32_t bin) {
  const uint64_t* p = t.slots + (uint64_t)bin * B;
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  if (B == 8) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 4));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(t.meta + bin));
}

// The generation of a new search in a region: one more than the last.  When
// the 32-bit count wraps, the visited set is cleared (generation 0 marks a
// free entry and is never used), so a tag left 2^32 searches ago cannot
// match.
__device__ __forceinline__ uint32_t next_generation(uint32_t* hdr, uint64_t* vis, uint32_t bits) {
  uint32_t gen = hdr[0] + 1;
  if (gen == 0) {
    for (uint32_t i = 0; i < (1u << bits); i++) vis[i] = 0;
    gen = 1;
  }
  hdr[0] = gen;
  return gen;
}

// Insert `bin` into the visited set; returns false if it was already there.
__device__ __forceinline__ bool vis_insert(uint64_t* vis, uint32_t bits, uint32_t gen, uint32_t bin) {
  uint64_t tag = ((uint64_t)gen << 32) | bin;
  for (uint32_t h = vis_hash(bin, bits);; h = (h + 1) & ((1u << bits) - 1)) {
    uint64_t e = vis[h];
    if (e == tag) return false;
    if ((uint32_t)(e >> 32) != gen) { vis[h] = tag; return true; }
  }
}

__device__ __forceinline__ bool vis_has(const uint64_t* vis, uint32_t bits, uint32_t gen, uint32_t bin) {
  uint64_t tag = ((uint64_t)gen << 32) | bin;
  for (uint32_t h = vis_hash(bin, bits);; h = (h + 1) & ((1u << bits) - 1)) {
    uint64_t e = vis[h];
    if (e == tag) return true;
    if ((uint32_t)(e >> 32) != gen) return false;
  }
}

// vis_has, given the entry at the bin's hash position already loaded (so
// the probes for a group's records overlap).
__device__ __forceinline__ bool vis_has_from(const uint64_t* vis, uint32_t bits, uint32_t gen, uint32_t bin,
                                             uint64_t e) {
  const uint64_t tag = ((uint64_t)gen << 32) | bin;
  for (uint32_t h = vis_hash(bin, bits);;) {
    if (e == tag) return true;
    if ((uint32_t)(e >> 32) != gen) return false;
    h = (h + 1) & ((1u << bits) - 1);
    e = vis[h];
  }
}

// a[s] for s known only at run time, kept in registers (a chain of selects)
template <int N>
__device__ __forceinline__ uint32_t pick(const uint32_t (&a)[N], uint32_t s) {
  uint32_t r = a[0];
#pragma unroll
  for (int q = 1; q < N; q++) r = (s == (uint32_t)q) ? a[q] : r;
  return r;
}

// The group a d-ary BFS spawns from: its record's d bins (y[j]: the bin of
// hash function j) and which of them may be tried, taken when the search
// reaches the group, the visited-set probes of the d bins overlapping.  `ok`
// bit j: the record is present, y[j] is not its own bin, and y[j] was
// unvisited then.  Until the search moves on to the next group, the only
// bins it marks visited are those its tries from this group view
// (`spawned`), so ok and spawned together give exactly the visited test the
// search makes try by try.
template <int N>
struct GroupCache {
  uint32_t g;  // group index (~0u: none yet)
  uint32_t bin, meta, next;
  uint32_t y[N];
  uint32_t ok, spawned;
};

// Was y viewed by a spawn from the cached group since it was taken?
template <int N>
__device__ __forceinline__ bool spawned_to(const GroupCache<N>& k, uint32_t y) {
  bool hit = false;
#pragma unroll
  for (int q = 0; q < N; q++) hit |= ((k.spawned >> q) & 1u) && k.y[q] == y;
  return hit;
}

__device__ __forceinline__ void take_group_dary(const DevTable& t, const Group* G, uint32_t g, const uint64_t* vis,
                                                uint32_t vb, uint32_t gen, GroupCache<4>& k) {
  const Group gr = G[g];
  k.g = g;
  k.bin = gr.bin;
  k.meta = gr.meta;
  k.next = gr.next;
  k.spawned = 0;
  k.ok = 0;
  const uint64_t rec = ld_slot(t.slots + gr.bin);
  if (rec == EMPTY) return;
  bins_of(t, key_of(rec), k.y);
  uint64_t e[4];
#pragma unroll
  for (int j = 0; j < 4; j++) e[j] = j < (int)t.d && k.y[j] != gr.bin ? vis[vis_hash(k.y[j], vb)] : 0;
#pragma unroll
  for (int j = 0; j < 4; j++)
    if (j < (int)t.d && k.y[j] != gr.bin && !vis_has_from(vis, vb, gen, k.y[j], e[j])) k.ok |= 1u << j;
}

// Bucket queues of candidate groups for sorted search and the hybrid.  A
// group's key never changes (the spawn count of its bin when viewed; the
// hybrid adds 16 x its depth), so the candidate with the smallest key,
// oldest first among equals, is the head of the lowest non-empty bucket,
// each bucket a list in push order.  Sorted search: bucket = key (0-15).
// Hybrid: depth-major order means only two depths have candidates at once
// (the one being spawned from and the next), so bucket = 16 x (depth & 1) +
// spawn count, and the search looks at the half of its current depth
// first.  `mask` bit b: bucket b holds a group.
struct Buckets {
  uint16_t* q;  // q[b]: head of bucket b, q[32 + b]: its tail
  uint32_t mask;
  uint32_t depth;  // hybrid: the depth being spawned from
};

__device__ __forceinline__ uint32_t bucket_of(int order, uint32_t key) {
  return order == P_HYBRID ? ((key >> 4) & 1u) * 16u + (key & 15u) : key;
}

__device__ __forceinline__ void bucket_push(Buckets& bq, Group* G, uint32_t b, uint32_t g) {
  if ((bq.mask >> b) & 1u) G[bq.q[32 + b]].link = (uint16_t)g;
  else bq.q[b] = (uint16_t)g;
  bq.q[32 + b] = (uint16_t)g;
  bq.mask |= 1u << b;
}

// The bucket to spawn from, or -1 when no candidate is left.
__device__ __forceinline__ int bucket_min(int order, Buckets& bq) {
  if (bq.mask == 0) return -1;
  if (order != P_HYBRID) return __ffs(bq.mask) - 1;
  uint32_t half = (bq.depth & 1u) ? (bq.mask >> 16) : (bq.mask & 0xFFFFu);
  if (half == 0) {  // this depth is exhausted: the next one
    bq.depth++;
    half = (bq.depth & 1u) ? (bq.mask >> 16) : (bq.mask & 0xFFFFu);
  }
  return (int)((bq.depth & 1u) * 16u) + __ffs(half) - 1;
}

// Group g, the head of bucket b, has no record left to spawn.
__device__ __forceinline__ void bucket_pop(Buckets& bq, const Group* G, uint32_t b, uint32_t g) {
  if (bq.q[32 + b] == (uint16_t)g) bq.mask &= ~(1u << b);
  else bq.q[b] = G[g].link;
}

// ORDER: P_BFS, P_SORTED or P_HYBRID
template <int B, int ORDER, bool GHOST>
__device__ int insert_search(const DevTable& t, Ctx& c, uint8_t* region) {
  uint32_t b0, b1;
  bins2(t, c.key, b0, b1);
  View<B> v0, v1;
  if (!GHOST) {
    // a free slot of b0, then of b1, placed by a compare-and-swap of the
    // slot on unordered views; the search needs ordered ones
    load_view_fast<B>(t, b0, v0);
    load_view_fast<B>(t, b1, v1);
    c.viewed += 2;
    uint32_t g0 = free_mask<B>(v0), g1 = free_mask<B>(v1);
    if (g0) return place_direct<B>(t, c, b0, lowest(g0), false) ? (int)ST_OK : (int)ST_CONFLICT;
    if (g1) return place_direct<B>(t, c, b1, lowest(g1), false) ? (int)ST_OK : (int)ST_CONFLICT;
    fence_acquire();
    load_slots<B>(t, b0, v0);
    load_slots<B>(t, b1, v1);
  } else {
    load_view2_fast<B>(t, b0, b1, v0, v1);
    c.viewed += 2;
  }
  uint32_t f0 = free_mask<B>(v0), f1 = free_mask<B>(v1);
  if (GHOST) {
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
  } else {
    if (f0) return take_free<B>(t, c, b0, v0, lowest(f0), false);
    if (f1) return take_free<B>(t, c, b1, v1, lowest(f1), false);
  }

  const SearchSpace sp = search_space(t, c, region);
  Group* G = sp.G;
  uint64_t* vis = sp.vis;
  const uint32_t vb = sp.vis_bits;
  const uint32_t gen = next_generation(sp.hdr, vis, vb);

  uint32_t ng = 0, head = 0;
  Buckets bq;
  bq.q = reinterpret_cast<uint16_t*>(sp.hdr + 4);
  bq.mask = 0;
  bq.depth = 0;
  auto push = [&](uint32_t bin, uint32_t m, uint32_t parent) {
    Group g;
    g.bin = bin;
    g.meta = m;
    g.parent = (uint16_t)parent;
    g.link = 0;
    g.next = 0;
    uint32_t depth = (ORDER == P_HYBRID && parent != NO_PARENT) ? (G[parent >> 3].key >> 4) + 1u : 0u;
    g.key = (uint16_t)(depth * 16 + spawn_of(m));
    g.stale = 0;
    G[ng] = g;
    if (ORDER != P_BFS) bucket_push(bq, G, bucket_of(ORDER, g.key), ng);
    ng++;
    vis_insert(vis, vb, gen, bin);
  };
  push(b0, v0.m, NO_PARENT);
  push(b1, v1.m, NO_PARENT);

  for (;;) {
    // one round: up to spawn_k spawns in candidate order, their bins
    // prefetched together (Sec. 5: spawning the k best records at a time
    // lets the fetches overlap); the first of them with room ends the
    // search, the others join as groups.  spawn_k = 1: the plain search.
    uint32_t rg[8], ry[8];
    uint8_t rs[8];
    uint32_t nr = 0;
    bool out = false;  // budget spent during the round
    while (nr < t.spawn_k) {
      uint32_t g;
      int bk = 0;
      if (ORDER == P_BFS) {  // the oldest group with a record left
        while (head < ng && G[head].next >= B) head++;
        if (head == ng) break;  // nothing left to spawn
        g = head;
      } else {  // the smallest key, oldest first among equals
        bk = bucket_min(ORDER, bq);
        if (bk < 0) break;
        g = bq.q[bk];
      }
      Group gr = G[g];
      uint32_t s = gr.next;
      G[g].next = (uint8_t)(s + 1);
      if (ORDER != P_BFS && s + 1 >= B) bucket_pop(bq, G, (uint32_t)bk, g);
      if ((gr.meta >> s) & 1u) {  // claimed by another insertion: ignore it (Sec. 8)
        c.foreign = 1;
        continue;
      }
      uint64_t rec = ld_slot(t.slots + (uint64_t)gr.bin * B + s);
      if (rec == EMPTY) continue;
      uint32_t y = other_bin2(t, rec, gr.bin);
      if (vis_has(vis, vb, gen, y)) continue;
      if (ORDER != P_BFS && spawn_of(gr.meta) < 15) {
        uint32_t nm = gr.meta + (1u << SPAWN_SHIFT);
        if (cas_acquire(t.meta + gr.bin, gr.meta, nm)) {
          G[g].meta = nm;
        } else {
          G[g].stale = 1;
          uint32_t m = ld_acquire(t.meta + gr.bin);
          for (int k = 0; k < 64 && spawn_of(m) < 15; k++) {  // bounded: a lost count is harmless
            if (cas_acquire(t.meta + gr.bin, m, m + (1u << SPAWN_SHIFT))) break;
            m = ld_acquire(t.meta + gr.bin);
          }
        }
      }
      if (c.viewed - c.viewed0 >= sp.budget || ng + nr >= sp.max_groups) { out = true; break; }  // budget spent
      vis_insert(vis, vb, gen, y);
      c.viewed++;
      prefetch_bin<B>(t, y);
      rg[nr] = g;
      rs[nr] = (uint8_t)s;
      ry[nr] = y;
      nr++;
    }
    if (nr == 0) return dead_end(c);
    for (uint32_t i = 0; i < nr; i++) {
      const uint32_t g = rg[i], s = rs[i], y = ry[i];
      View<B> vy;
      load_view_fast<B>(t, y, vy);
      if (claimed_mask<B>(vy)) c.foreign = 1;
      uint32_t fm = free_mask<B>(vy);
      int term = lowest(fm);
      bool isdup = false;
      if (term < 0 && GHOST) {
        term = lowest(dup_mask<B>(vy));
        isdup = term >= 0;
      }
      if (term < 0) {
        push(y, vy.m, (g << 3) | s);
        continue;
      }
      // path root -> ... -> (g, s): depth entries in chain order
      uint32_t depth = 1;
      for (uint32_t q = g; G[q].parent != NO_PARENT; q = G[q].parent >> 3) depth++;
      if ((int)depth + 4 > c.pcap) return ST_LONG;
      {
        // entries in chain order; the group index rides in the content word
        // until the slot is claimed
        uint32_t q = g, qs = s;
        for (int e = (int)depth - 1; e >= 0; e--) {
          set_entry(c, e, pack_entry(G[q].bin, (int)qs, K_MOVE, false, 0, 0), q);
          uint32_t par = G[q].parent;
          if (par != NO_PARENT) { qs = par & 7u; q = par >> 3; }
        }
      }
      // claim the path in chain order; each CAS checks its bin is as viewed,
      // so the record read after the claim is the one the search saw
      c.pn = 0;
      for (uint32_t e = 0; e < depth; e++) {
        Group gq = G[(uint32_t)content_at(c, (int)e)];
        uint32_t sl = e_slot(desc_at(c, (int)e));
        if (gq.stale) return ST_CONFLICT;
        if (!cas_acquire(t.meta + gq.bin, gq.meta, gq.meta + (1u << sl))) return ST_CONFLICT;
        c.pn = (int)e + 1;
        // the record must move into the next bin of the path: it is the one
        // the search saw unless the bin's word came back to its viewed value
        const uint64_t r = reread<B>(t, gq.bin, sl);
        const uint32_t to = e + 1 < depth ? G[(uint32_t)content_at(c, (int)e + 1)].bin : y;
        set_content(c, (int)e, r);
        if (!belongs<B>(t, r, to)) return ST_CONFLICT;
      }
      c.kicks = depth;
      if (isdup) return take_dup<B>(t, c, y, vy, term, false);
      return take_free<B>(t, c, y, vy, term, false);
    }
    if (out) return out_of_cap(c);
  }
}

// ------------------------------------------------------------------
// d-ary tables (Sec. 7 evaluates BFS and sorted search on them): one record
// per bin.  The first step is random kicking's (h_0, h_1, .. viewed until
// an empty bin).  Then the key's d bins are the root groups; popping a
// group tries its record's next hash function j (the record's own bin and
// bins already viewed are skipped without a view or a spawn); a try is a
// spawn (the group's bin gets its spawn count incremented for sorted
// search and the hybrid) and views the record's j-th bin: empty ends the
// search, full makes it a group.  Same group order, budget and claiming of
// the path as the two-choice searches above.
// ------------------------------------------------------------------
template <int ORDER>
__device__ int insert_search_dary(const DevTable& t, Ctx& c, uint8_t* region) {
  const uint32_t d = t.d;
  uint32_t b[4];
  bins_of(t, c.key, b);
  View<1> v[4];
#pragma unroll
  for (int i = 0; i < 4; i++)
    if (i < (int)d) load_view_fast<1>(t, b[i], v[i]);  // the d loads overlap
  for (uint32_t i = 0; i < d; i++) {
    c.viewed++;
    if (free_mask<1>(v[i])) return take_free<1>(t, c, b[i], v[i], 0, false);
  }

  const SearchSpace sp = search_space(t, c, region);
  Group* G = sp.G;
  uint64_t* vis = sp.vis;
  const uint32_t vb = sp.vis_bits;
  const uint32_t gen = next_generation(sp.hdr, vis, vb);

  uint32_t ng = 0, head = 0;
  Buckets bq;
  bq.q = reinterpret_cast<uint16_t*>(sp.hdr + 4);
  bq.mask = 0;
  bq.depth = 0;
  auto push = [&](uint32_t bin, uint32_t m, uint32_t parent) {
    Group g;
    g.bin = bin;
    g.meta = m;
    g.parent = (uint16_t)parent;
    g.link = 0;
    g.next = 0;
    uint32_t depth = (ORDER == P_HYBRID && parent != NO_PARENT) ? (G[parent >> 3].key >> 4) + 1u : 0u;
    g.key = (uint16_t)(depth * 16 + spawn_of(m));
    g.stale = 0;
    G[ng] = g;
    if (ORDER != P_BFS) bucket_push(bq, G, bucket_of(ORDER, g.key), ng);
    ng++;
    vis_insert(vis, vb, gen, bin);
  };
  for (uint32_t i = 0; i < d; i++) push(b[i], v[i].m, NO_PARENT);

  GroupCache<4> k;  // BFS: the head group's record, its bins and which of them may be tried
  k.g = ~0u;
  for (;;) {
    // rounds of spawn_k tries, as in the two-choice searches
    uint32_t rg[8], ry[8];
    uint32_t nr = 0;
    bool out = false;
    while (nr < t.spawn_k) {
      uint32_t g, j, y;
      if (ORDER == P_BFS) {  // the oldest group, until its hash functions run out
        if (k.g == head && k.next >= d) head++;
        if (head == ng) break;  // nothing left to try
        if (k.g != head) take_group_dary(t, G, head, vis, vb, gen, k);
        g = head;
        j = k.next++;
        if (k.meta & 1u) {  // claimed by another insertion: ignore it (Sec. 8)
          c.foreign = 1;
          continue;
        }
        // empty, the record's own bin, or a bin already viewed
        if (!((k.ok >> j) & 1u)) continue;
        y = pick<4>(k.y, j);
        if (spawned_to<4>(k, y)) continue;
      } else {  // the smallest key, oldest first among equals
        const int bk = bucket_min(ORDER, bq);
        if (bk < 0) break;
        g = bq.q[bk];
        Group gr = G[g];
        j = gr.next;
        G[g].next = (uint8_t)(j + 1);
        if (j + 1 >= d) bucket_pop(bq, G, (uint32_t)bk, g);
        if (gr.meta & 1u) {
          c.foreign = 1;
          continue;
        }
        uint64_t rec = ld_slot(t.slots + gr.bin);
        if (rec == EMPTY) continue;
        uint32_t rb[4];
        bins_of(t, key_of(rec), rb);
        y = rb[j];
        if (y == gr.bin || vis_has(vis, vb, gen, y)) continue;
        if (spawn_of(gr.meta) < 15) {
          uint32_t nm = gr.meta + (1u << SPAWN_SHIFT);
          if (cas_acquire(t.meta + gr.bin, gr.meta, nm)) {
            G[g].meta = nm;
          } else {
            G[g].stale = 1;
            uint32_t m = ld_acquire(t.meta + gr.bin);
            for (int q = 0; q < 64 && spawn_of(m) < 15; q++) {  // bounded: a lost count is harmless
              if (cas_acquire(t.meta + gr.bin, m, m + (1u << SPAWN_SHIFT))) break;
              m = ld_acquire(t.meta + gr.bin);
            }
          }
        }
      }
      if (c.viewed - c.viewed0 >= sp.budget || ng + nr >= sp.max_groups) { out = true; break; }  // budget spent
      vis_insert(vis, vb, gen, y);
      if (ORDER == P_BFS) k.spawned |= 1u << j;
      c.viewed++;
      prefetch_bin<1>(t, y);
      rg[nr] = g;
      ry[nr] = y;
      nr++;
    }
    if (nr == 0) return dead_end(c);
    for (uint32_t i = 0; i < nr; i++) {
      const uint32_t g = rg[i], y = ry[i];
      View<1> vy;
      load_view_fast<1>(t, y, vy);
      if (claimed_mask<1>(vy)) c.foreign = 1;
      if (!free_mask<1>(vy)) {
        push(y, vy.m, g << 3);
        continue;
      }
      // path: root group -> ... -> group g, one record each, in chain order
      uint32_t depth = 1;
      for (uint32_t q = g; G[q].parent != NO_PARENT; q = G[q].parent >> 3) depth++;
      if ((int)depth + 4 > c.pcap) return ST_LONG;
      {
        uint32_t q = g;
        for (int e = (int)depth - 1; e >= 0; e--) {
          set_entry(c, e, pack_entry(G[q].bin, 0, K_MOVE, false, 0, 0), q);
          if (G[q].parent != NO_PARENT) q = G[q].parent >> 3;
        }
      }
      // claim the path in chain order from the metadata words as viewed; the
      // record read after a claim is the one the search saw
      c.pn = 0;
      for (uint32_t e = 0; e < depth; e++) {
        Group gq = G[(uint32_t)content_at(c, (int)e)];
        if (gq.stale) return ST_CONFLICT;
        if (!cas_acquire(t.meta + gq.bin, gq.meta, gq.meta + 1u)) return ST_CONFLICT;
        c.pn = (int)e + 1;
        const uint64_t r = reread<1>(t, gq.bin, 0);
        const uint32_t to = e + 1 < depth ? G[(uint32_t)content_at(c, (int)e + 1)].bin : y;
        set_content(c, (int)e, r);
        if (!belongs<1>(t, r, to)) return ST_CONFLICT;
      }
      c.kicks = depth;
      return take_free<1>(t, c, y, vy, 0, false);
    }
    if (out) return out_of_cap(c);
  }
}

}  // namespace ck
