/*
 * ck_oracle.c -- serial CPU oracle for the cuckoo-table hot path of
 * Kuszmaul, "Fast Concurrent Cuckoo Kick-out Eviction Schemes for
 * High-Density Tables" (arXiv:1605.05236).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Every insertion is simulated forward, one kick-out at a time, exactly in
 * the order the paper describes (Sec. 1: place into a free slot of one of the
 * two bins, otherwise kick a victim out and re-insert it).  Every change is
 * written to an undo log, so a failed insertion (chain cap or search budget
 * reached) leaves the table exactly as it was: the homeless record is always
 * the new key (system-transaction kick-outs are planned before they are
 * applied, Sec. 8 "System-Transaction Kick-Outs").
 *
 * Claim flags (Sec. 8 "Claim Flags"): a chain claims every slot it writes
 * and ignores claimed slots.  With one insertion in flight the only claims
 * are the chain's own, so here "claimed" means "already written by the
 * current chain".  A chain therefore never writes one slot twice.
 *
 * Per-slot state is kept in plain arrays (record, duplicate flag, rattle
 * counter) and per-bin state likewise (hit counter, spawn count); no bit
 * packing.
 *
 * Readings of points the paper leaves open are listed beside the code that
 * takes them.  Every operation here is pinned by the tests named
 * tests/test_oracle_*.py against values fixed by the paper or by
 * mathematics (brute-force matching, invariants, published hash and
 * generator test vectors, hand-worked fixtures); none is left unpinned.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

#define ORC_EMPTY 0xFFFFFFFFFFFFFFFFull
#define ORC_RESERVED_KEY 0xFFFFFFFFu

/* policy codes: the same numbering the library's C ABI uses */
#define ORC_RANDOM 0
#define ORC_BFS 1
#define ORC_SORTED 2
#define ORC_QUEUE 3
#define ORC_RATTLE 4
#define ORC_HYBRID 5
#define ORC_GHOST 0x100

#define ORC_OK 0
#define ORC_FAILED 1
#define ORC_INVALID 3

/* stats indices (exported with orc_stats) */
enum {
  OS_INSERTS_OK = 0,
  OS_INSERTS_FAILED,
  OS_BINS_VIEWED,       /* over every insertion, failed ones included */
  OS_KICKS,             /* records displaced by successful insertions */
  OS_CHAIN_MAX,
  OS_GHOST_PAIRS_MADE,  /* ghost insertions (Sec. 4) */
  OS_DUP_EVICTIONS,     /* duplicates overwritten */
  OS_SIZE,              /* distinct live keys */
  OS_LIVE_GHOSTS,       /* live ghost pairs */
  OS_LOOKUPS,
  OS_LOOKUP_HITS,
  OS_DELETES,
  OS_DELETE_HITS,
  OS_PROP41_VIOLATIONS, /* Prop. 4.1 checks that failed */
  OS_PROP41_CHECKS,
  OS_UPDATES,
  OS_N
};

typedef struct {
  uint64_t slot;
  uint64_t old_rec;
  uint8_t old_dup;
  uint8_t old_rattle;
} undo_slot_t;

typedef struct {
  uint64_t bin;
  uint8_t old_hit;
} undo_hit_t;

typedef struct {
  uint64_t bin;
  int32_t parent;   /* index of the group whose record led here, -1 at a root */
  int32_t pslot;    /* slot (in the parent's bin) of that record */
  uint32_t next;    /* next slot of this bin not yet spawned */
  uint32_t skey;    /* spawn count of the bin when its records joined the list */
  uint32_t depth;   /* spawns between the new key and this bin's records (roots: 0) */
} group_t;

typedef struct orc_table {
  uint64_t n;          /* bins */
  uint32_t B;          /* slots per bin */
  uint32_t d;          /* hash functions */
  uint32_t policy;     /* ORC_RANDOM .. ORC_HYBRID */
  uint32_t ghost;      /* ghost insertions on (Sec. 4) */
  uint32_t cap;        /* kick-out cap (walks), try cap (rattle), bin budget (search) */
  uint32_t rattle_tie_resident; /* debug reading: resident wins rattle ties */
  uint32_t hash_family;  /* 0: fmix32(key ^ seed_i); 1: fmix32(fmix32(key + seed_i) ^ seed_i*0x27D4EB2F) */
  uint32_t spawn_k;      /* searches: spawns per round, their bins viewed together (Sec. 5); 1 = plain */
  uint64_t rng_seed;
  uint32_t seeds[4];

  uint64_t *rec;       /* n*B slots, key<<32 | value, ORC_EMPTY when free */
  uint8_t *dup;        /* n*B duplicate marks (Sec. 4) */
  uint8_t *rattle;     /* n*B rattle counters r(x) of resident keys (Sec. 7) */
  uint8_t *hit;        /* n hit counters (Sec. 6) */
  uint8_t *spawn;      /* n spawn counts, 0..15 (Sec. 5) */

  /* per-insertion working state */
  uint8_t *claimed;    /* n*B: written by the current chain */
  uint64_t *claimed_list;
  uint64_t n_claimed, claimed_capacity;
  undo_slot_t *undo_s;
  uint64_t n_undo_s, undo_s_capacity;
  undo_hit_t *undo_h;
  uint64_t n_undo_h, undo_h_capacity;
  uint8_t *visited;    /* n: bin viewed by the current search */
  uint64_t *visited_list;
  uint64_t n_visited, visited_capacity;
  group_t *groups;
  uint64_t n_groups, groups_capacity;

  uint64_t cur_viewed;
  uint64_t cur_kicks;
  uint64_t cur_draw;
  uint32_t cur_key;    /* key whose insertion is running (seeds the draws) */

  /* explicit bin choices for hand-worked fixtures (keys sorted) */
  uint32_t *ov_keys;
  uint64_t *ov_bins;   /* d per key */
  uint64_t n_ov;

  uint64_t stats[OS_N];
} orc_table;

/* ------------------------------------------------------------------ */
/* hashing and random draws                                            */
/* ------------------------------------------------------------------ */

/* MurmurHash3's 32-bit finalizer (Appleby, public domain): an invertible
 * avalanche mix standing in for Sec. 3's uniformly random hashes. */
static uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output produced from
 * generator state x, i.e. mix(x + golden gamma). */
static uint64_t splitmix64_at(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint32_t orc_fmix32(uint32_t h) { return fmix32(h); }
uint64_t orc_splitmix64_at(uint64_t x) { return splitmix64_at(x); }

/* The draw-th random number of the insertion of key k: a counter-based
 * stream so that a run with one insertion in flight can be replayed. */
static uint64_t draw(orc_table *t) {
  uint64_t x = t->rng_seed ^ (uint64_t)t->cur_key ^ (t->cur_draw << 32);
  t->cur_draw++;
  return splitmix64_at(x);
}

static int ov_find(const orc_table *t, uint32_t key) {
  uint64_t lo = 0, hi = t->n_ov;
  while (lo < hi) {
    uint64_t mid = (lo + hi) / 2;
    if (t->ov_keys[mid] < key) lo = mid + 1; else hi = mid;
  }
  if (lo < t->n_ov && t->ov_keys[lo] == key) return (int)lo;
  return -1;
}

/* The d bins of a key (Sec. 1: two different bins per key; Sec. 7 for d
 * hash functions).  h_i = fmix32(key ^ seed_i) mod n (family
 * 0, the stated workload's hash), or, in family 1, a decorrelated form of
 * the same mix: fmix32(fmix32(key + seed_i) ^ (seed_i * 0x27D4EB2F)) mod n
 * (family 0's functions are not independent: key ^ seed_i ^ seed_j gets
 * key's h_i and h_j swapped).  A collision with an earlier choice moves to
 * the next bin (mod n), so the d choices are distinct as the paper requires. */
static void bins_of(const orc_table *t, uint32_t key, uint64_t *out) {
  if (t->n_ov) {
    int i = ov_find(t, key);
    if (i >= 0) {
      for (uint32_t j = 0; j < t->d; j++) out[j] = t->ov_bins[(uint64_t)i * t->d + j];
      return;
    }
  }
  for (uint32_t i = 0; i < t->d; i++) {
    uint32_t s = t->seeds[i];
    uint32_t h = t->hash_family ? fmix32(fmix32(key + s) ^ (uint32_t)(s * 0x27D4EB2Fu)) : fmix32(key ^ s);
    uint64_t b = (uint64_t)h % t->n;
    for (;;) {
      int clash = 0;
      for (uint32_t j = 0; j < i; j++) if (out[j] == b) clash = 1;
      if (!clash) break;
      b = (b + 1) % t->n;
    }
    out[i] = b;
  }
}

void orc_bins(const orc_table *t, uint32_t key, uint64_t *out) { bins_of(t, key, out); }

static uint32_t key_of(uint64_t rec) { return (uint32_t)(rec >> 32); }

/* The bin of a two-choice record other than `here`. */
static uint64_t other_bin(const orc_table *t, uint64_t rec, uint64_t here) {
  uint64_t b[4];
  bins_of(t, key_of(rec), b);
  return b[0] == here ? b[1] : b[0];
}

/* ------------------------------------------------------------------ */
/* table lifetime                                                     */
/* ------------------------------------------------------------------ */

static void *xcalloc(uint64_t n, uint64_t sz) {
  void *p = calloc(n ? n : 1, sz);
  if (!p) { fprintf(stderr, "ck_oracle: out of memory\n"); abort(); }
  return p;
}

static void grow(void **p, uint64_t *cap, uint64_t need, uint64_t sz) {
  if (need <= *cap) return;
  uint64_t c = *cap ? *cap : 64;
  while (c < need) c *= 2;
  void *q = realloc(*p, c * sz);
  if (!q) { fprintf(stderr, "ck_oracle: out of memory\n"); abort(); }
  *p = q;
  *cap = c;
}

orc_table *orc_create(uint64_t n_bins, uint32_t B, uint32_t d, uint32_t policy,
                      uint64_t rng_seed, uint32_t cap, const uint32_t *seeds) {
  if (n_bins < d || d < 2 || d > 4) return NULL;
  orc_table *t = (orc_table *)xcalloc(1, sizeof(orc_table));
  t->n = n_bins;
  t->B = B;
  t->d = d;
  t->policy = policy & 0xFF;
  t->ghost = (policy & ORC_GHOST) ? 1 : 0;
  t->cap = cap;
  t->spawn_k = 1;
  t->rng_seed = rng_seed;
  for (uint32_t i = 0; i < d; i++) t->seeds[i] = seeds[i];
  uint64_t ns = n_bins * B;
  t->rec = (uint64_t *)malloc(ns * sizeof(uint64_t));
  if (!t->rec) { free(t); return NULL; }
  for (uint64_t i = 0; i < ns; i++) t->rec[i] = ORC_EMPTY;
  t->dup = (uint8_t *)xcalloc(ns, 1);
  t->rattle = (uint8_t *)xcalloc(ns, 1);
  t->claimed = (uint8_t *)xcalloc(ns, 1);
  t->hit = (uint8_t *)xcalloc(n_bins, 1);
  t->spawn = (uint8_t *)xcalloc(n_bins, 1);
  t->visited = (uint8_t *)xcalloc(n_bins, 1);
  return t;
}

void orc_destroy(orc_table *t) {
  if (!t) return;
  free(t->rec); free(t->dup); free(t->rattle); free(t->claimed);
  free(t->hit); free(t->spawn); free(t->visited);
  free(t->claimed_list); free(t->undo_s); free(t->undo_h);
  free(t->visited_list); free(t->groups);
  free(t->ov_keys); free(t->ov_bins);
  free(t);
}

void orc_set_rattle_tie_resident(orc_table *t, int on) { t->rattle_tie_resident = on ? 1 : 0; }
void orc_set_hash_family(orc_table *t, int f) { t->hash_family = f ? 1 : 0; }
int orc_set_spawn_k(orc_table *t, uint32_t k) {
  if (k < 1 || k > 8) return -1;
  t->spawn_k = k;
  return 0;
}
/* Fixtures: start a bin with a given spawn count (as left by earlier searches). */
int orc_set_spawn(orc_table *t, uint64_t bin, uint32_t count) {
  if (bin >= t->n || count > 15) return -1;
  t->spawn[bin] = (uint8_t)count;
  return 0;
}

/* Fixtures: give `n` keys explicit bin choices (d per key, distinct). */
int orc_set_bins_override(orc_table *t, const uint32_t *keys, const uint64_t *bins, uint64_t n) {
  free(t->ov_keys); free(t->ov_bins);
  t->ov_keys = (uint32_t *)xcalloc(n, 4);
  t->ov_bins = (uint64_t *)xcalloc(n * t->d, 8);
  /* insertion sort by key: fixtures are tiny */
  for (uint64_t i = 0; i < n; i++) {
    uint64_t j = i;
    while (j > 0 && t->ov_keys[j - 1] > keys[i]) {
      t->ov_keys[j] = t->ov_keys[j - 1];
      memcpy(t->ov_bins + j * t->d, t->ov_bins + (j - 1) * t->d, 8 * t->d);
      j--;
    }
    t->ov_keys[j] = keys[i];
    memcpy(t->ov_bins + j * t->d, bins + i * t->d, 8 * t->d);
    for (uint32_t a = 0; a < t->d; a++) {
      if (bins[i * t->d + a] >= t->n) return -1;
      for (uint32_t b = 0; b < a; b++)
        if (bins[i * t->d + a] == bins[i * t->d + b]) return -1;
    }
  }
  t->n_ov = n;
  return 0;
}

/* ------------------------------------------------------------------ */
/* per-insertion working state: own claims, undo log                  */
/* ------------------------------------------------------------------ */

static void begin_insert(orc_table *t, uint32_t key) {
  t->n_claimed = 0;
  t->n_undo_s = 0;
  t->n_undo_h = 0;
  t->cur_viewed = 0;
  t->cur_kicks = 0;
  t->cur_draw = 0;
  t->cur_key = key;
}

static void mark_claimed(orc_table *t, uint64_t slot) {
  if (t->claimed[slot]) return;
  t->claimed[slot] = 1;
  grow((void **)&t->claimed_list, &t->claimed_capacity, t->n_claimed + 1, 8);
  t->claimed_list[t->n_claimed++] = slot;
}

static void end_insert(orc_table *t) {
  for (uint64_t i = 0; i < t->n_claimed; i++) t->claimed[t->claimed_list[i]] = 0;
  t->n_claimed = 0;
  for (uint64_t i = 0; i < t->n_visited; i++) t->visited[t->visited_list[i]] = 0;
  t->n_visited = 0;
}

static void log_slot(orc_table *t, uint64_t slot) {
  grow((void **)&t->undo_s, &t->undo_s_capacity, t->n_undo_s + 1, sizeof(undo_slot_t));
  undo_slot_t *u = &t->undo_s[t->n_undo_s++];
  u->slot = slot;
  u->old_rec = t->rec[slot];
  u->old_dup = t->dup[slot];
  u->old_rattle = t->rattle[slot];
}

/* Write `rec` into `slot` (claiming it) and return the record it held. */
static uint64_t put(orc_table *t, uint64_t slot, uint64_t rec, uint8_t dup, uint8_t r) {
  log_slot(t, slot);
  uint64_t old = t->rec[slot];
  t->rec[slot] = rec;
  t->dup[slot] = dup;
  t->rattle[slot] = r;
  mark_claimed(t, slot);
  return old;
}

/* Hit counter of a bin: read then incremented, one byte (Sec. 6 footnote). */
static uint32_t hit_take(orc_table *t, uint64_t bin) {
  grow((void **)&t->undo_h, &t->undo_h_capacity, t->n_undo_h + 1, sizeof(undo_hit_t));
  t->undo_h[t->n_undo_h].bin = bin;
  t->undo_h[t->n_undo_h].old_hit = t->hit[bin];
  t->n_undo_h++;
  uint32_t h = t->hit[bin];
  t->hit[bin] = (uint8_t)(h + 1);
  return h;
}

static void rollback(orc_table *t) {
  for (uint64_t i = t->n_undo_s; i-- > 0;) {
    undo_slot_t *u = &t->undo_s[i];
    t->rec[u->slot] = u->old_rec;
    t->dup[u->slot] = u->old_dup;
    t->rattle[u->slot] = u->old_rattle;
  }
  for (uint64_t i = t->n_undo_h; i-- > 0;) t->hit[t->undo_h[i].bin] = t->undo_h[i].old_hit;
  t->n_undo_s = t->n_undo_h = 0;
}

/* ------------------------------------------------------------------ */
/* slot predicates inside one bin                                     */
/* ------------------------------------------------------------------ */

static void view(orc_table *t) { t->cur_viewed++; }

static int is_free(const orc_table *t, uint64_t slot) {
  return t->rec[slot] == ORC_EMPTY && !t->claimed[slot];
}

static int is_dup(const orc_table *t, uint64_t slot) {
  return t->rec[slot] != ORC_EMPTY && t->dup[slot] && !t->claimed[slot];
}

/* lowest-index free slot of a bin, or -1 */
static int lowest_free(const orc_table *t, uint64_t bin) {
  for (uint32_t s = 0; s < t->B; s++) if (is_free(t, bin * t->B + s)) return (int)s;
  return -1;
}

static int count_free(const orc_table *t, uint64_t bin) {
  int c = 0;
  for (uint32_t s = 0; s < t->B; s++) c += is_free(t, bin * t->B + s);
  return c;
}

static int lowest_dup(const orc_table *t, uint64_t bin) {
  for (uint32_t s = 0; s < t->B; s++) if (is_dup(t, bin * t->B + s)) return (int)s;
  return -1;
}

/* first slot from `start` onwards (cyclically) satisfying the predicate */
static int first_dup_from(const orc_table *t, uint64_t bin, uint32_t start) {
  for (uint32_t i = 0; i < t->B; i++) {
    uint32_t s = (start + i) % t->B;
    if (is_dup(t, bin * t->B + s)) return (int)s;
  }
  return -1;
}

/* Overwrite the duplicate at `slot` with `rec` and clear the duplicate mark
 * of its twin (Sec. 4: removing one copy leaves the other as a plain
 * record).  Unmarking the twin is a metadata write, not a bin view. */
static void evict_dup(orc_table *t, uint64_t bin, uint32_t s, uint64_t rec) {
  uint64_t slot = bin * t->B + s;
  uint64_t g = put(t, slot, rec, 0, 0);
  uint64_t y = other_bin(t, g, bin);
  for (uint32_t u = 0; u < t->B; u++) {
    uint64_t ts = y * t->B + u;
    if (t->rec[ts] == g && t->dup[ts]) {
      log_slot(t, ts);
      t->dup[ts] = 0;
      mark_claimed(t, ts);
      break;
    }
  }
  t->stats[OS_DUP_EVICTIONS]++;
  t->stats[OS_LIVE_GHOSTS]--;
}

/* Ghost insertion (Sec. 4): the new record into both bins, marked duplicate. */
static void put_ghost_pair(orc_table *t, uint64_t b0, uint32_t s0, uint64_t b1, uint32_t s1, uint64_t rec) {
  put(t, b0 * t->B + s0, rec, 1, 0);
  put(t, b1 * t->B + s1, rec, 1, 0);
  t->stats[OS_GHOST_PAIRS_MADE]++;
  t->stats[OS_LIVE_GHOSTS]++;
}

/* Prop. 4.1 check: in an insert-only ghost table the last bin of a kick-out
 * chain held a duplicate before the chain.  Slots the chain itself wrote
 * held plain victims, so only unclaimed slots can carry that duplicate. */
static int had_deletes_flag(const orc_table *t) { return t->stats[OS_DELETE_HITS] != 0; }

static void prop41_check(orc_table *t, uint64_t bin) {
  if (!t->ghost || t->cur_kicks == 0 || had_deletes_flag(t)) return;
  int ok = 0;
  for (uint32_t s = 0; s < t->B; s++) if (is_dup(t, bin * t->B + s)) ok = 1;
  t->stats[OS_PROP41_CHECKS]++;
  if (!ok) t->stats[OS_PROP41_VIOLATIONS]++;
}

/* Displace the record at (bin, s) by `cur`; return the displaced record. */
static uint64_t kick(orc_table *t, uint64_t bin, uint32_t s, uint64_t cur) {
  t->cur_kicks++;
  return put(t, bin * t->B + s, cur, 0, 0);
}

/* ------------------------------------------------------------------ */
/* random kicking, two bins of B slots (Sec. 1; Sec. 3 Fig. A/B)      */
/* ------------------------------------------------------------------ */
/* Without ghosts the new key goes to the first of its two bins that has a
 * free slot (Sec. 1), viewing b0 and only then b1.  With ghosts both bins
 * are viewed first (Sec. 4): room in both gives a ghost pair, room in one a
 * single copy, otherwise a duplicate in b0 (then b1) is overwritten.
 * Otherwise a victim is drawn uniformly from the 2B slots of the two bins,
 * it moves to its other bin, and so on: each later victim is drawn
 * uniformly from the slots of the current bin the chain has not written.
 * Each bin the chain reaches is one more bin viewed. */
static int insert_random2(orc_table *t, uint64_t krec, const uint64_t *b) {
  uint64_t b0 = b[0], b1 = b[1];
  int s0, s1;
  if (!t->ghost) {
    view(t);
    if ((s0 = lowest_free(t, b0)) >= 0) { put(t, b0 * t->B + s0, krec, 0, 0); return ORC_OK; }
    view(t);
    if ((s1 = lowest_free(t, b1)) >= 0) { put(t, b1 * t->B + s1, krec, 0, 0); return ORC_OK; }
  } else {
    view(t); view(t);
    s0 = lowest_free(t, b0);
    s1 = lowest_free(t, b1);
    if (s0 >= 0 && s1 >= 0) { put_ghost_pair(t, b0, s0, b1, s1, krec); return ORC_OK; }
    if (s0 >= 0) { put(t, b0 * t->B + s0, krec, 0, 0); return ORC_OK; }
    if (s1 >= 0) { put(t, b1 * t->B + s1, krec, 0, 0); return ORC_OK; }
    if ((s0 = lowest_dup(t, b0)) >= 0) { evict_dup(t, b0, s0, krec); return ORC_OK; }
    if ((s1 = lowest_dup(t, b1)) >= 0) { evict_dup(t, b1, s1, krec); return ORC_OK; }
  }
  /* first victim: uniform over the 2B slots of b0 then b1 */
  uint64_t r = draw(t);
  uint32_t idx = (uint32_t)(r % (2ull * t->B));
  uint64_t x = idx < t->B ? b0 : b1;
  uint32_t s = idx % t->B;
  uint64_t cur = krec;
  for (;;) {
    if (t->cur_kicks == t->cap) return ORC_FAILED;
    cur = kick(t, x, s, cur);
    x = other_bin(t, cur, x);
    view(t);
    int f = lowest_free(t, x);
    if (f >= 0) { prop41_check(t, x); put(t, x * t->B + f, cur, 0, 0); return ORC_OK; }
    if (t->ghost) {
      int g = lowest_dup(t, x);
      if (g >= 0) { prop41_check(t, x); evict_dup(t, x, g, cur); return ORC_OK; }
    }
    /* uniform over the unclaimed slots of x, in slot order */
    uint32_t elig[8], ne = 0;
    for (uint32_t u = 0; u < t->B; u++) if (!t->claimed[x * t->B + u]) elig[ne++] = u;
    if (ne == 0) return ORC_FAILED;
    r = draw(t);
    s = elig[r % ne];
  }
}

/* ------------------------------------------------------------------ */
/* queue-kicking with hit counters and hit balancing (Sec. 6)          */
/* ------------------------------------------------------------------ */
/* Each insertion into a bin takes the bin's hit counter h and increments
 * it; the record goes to slot h mod B, kicking out its occupant (the record
 * that has been in the bin longest).  Readings: when the bin still has a
 * free slot the record takes the lowest free slot (in insert-only tables
 * the bin fills in slot order, so this is slot h mod B itself; after
 * deletes a free slot wins over kicking); with ghosts a duplicate, searched from
 * h mod B, is overwritten before any plain record is kicked; a walk that
 * comes back to a bin kicks out the record at h mod B even if this chain
 * placed it there (the walk has no memory of its path; only the cap ends
 * it).  The new key views both bins and takes
 * the less full one (load balancing, Sec. 2), b0 on ties; when both are
 * full it takes the one with the smaller hit counter (hit balancing), b0 on
 * ties.  With ghosts, room in both bins gives a ghost pair. */
static int insert_queue(orc_table *t, uint64_t krec, const uint64_t *b) {
  uint64_t b0 = b[0], b1 = b[1];
  view(t); view(t);
  int f0 = count_free(t, b0), f1 = count_free(t, b1);
  if (t->ghost && f0 > 0 && f1 > 0) {
    hit_take(t, b0);
    int s0 = lowest_free(t, b0);
    hit_take(t, b1);
    int s1 = lowest_free(t, b1);
    put_ghost_pair(t, b0, s0, b1, s1, krec);
    return ORC_OK;
  }
  uint64_t x;
  if (f0 > 0 || f1 > 0) x = (f0 >= f1) ? b0 : b1;
  else if (t->ghost && (lowest_dup(t, b0) >= 0 || lowest_dup(t, b1) >= 0)) x = lowest_dup(t, b0) >= 0 ? b0 : b1;
  else x = (t->hit[b0] <= t->hit[b1]) ? b0 : b1;
  uint64_t cur = krec;
  for (;;) {
    uint32_t h = hit_take(t, x) % t->B;
    int s = lowest_free(t, x);
    if (s >= 0) { prop41_check(t, x); put(t, x * t->B + s, cur, 0, 0); return ORC_OK; }
    if (t->ghost && (s = first_dup_from(t, x, h)) >= 0) { prop41_check(t, x); evict_dup(t, x, s, cur); return ORC_OK; }
    /* the record at slot h mod B, whoever placed it: a walk that comes
     * back to a bin displaces the next record in the bin's queue, which
     * may be one this chain put there (the walk keeps no memory of its
     * path; the hit counter has moved on since its last visit) */
    s = (int)h;
    if (t->cur_kicks == t->cap) return ORC_FAILED;
    cur = kick(t, x, (uint32_t)s, cur);
    x = other_bin(t, cur, x);
    view(t);
  }
}

/* ------------------------------------------------------------------ */
/* breadth-first search and sorted search (Sec. 5)                     */
/* ------------------------------------------------------------------ */
/* Candidates are the records of the bins viewed so far that have not been
 * spawned.  Spawning a record views its other bin (its children).  A free
 * slot there (or, with ghosts, a duplicate) ends the search, and the chain
 * root -> ... -> spawned record -> that slot is applied.  Otherwise the new
 * bin's B records become candidates.  A bin already viewed by this search
 * is never viewed again (the small visited set of Sec. 5); popping a record
 * whose other bin was viewed is skipped without a view and without a spawn.
 *
 * BFS pops the oldest candidate.  Sorted search pops the candidate with
 * the smallest spawn count; ties go to the oldest candidate, so equal
 * counts reduce to BFS.  Reading: where a candidate sits in the priority
 * order is fixed when it joins the list, by the spawn count its bin has at that
 * moment (the bucket sort of Sec. 5 keys each entry once).  Spawning a
 * record increments the spawn count of the bin holding it, saturating at 15
 * (four bits, Sec. 5); these increments persist even when the search fails
 * (the count covers the whole life of the table, Sec. 5).
 *
 * The sorted search / BFS hybrid (end of Sec. 5) orders candidates first by
 * the depth at which they were spawn victims (the records of b0 and b1:
 * depth 0, the records of a bin viewed by spawning a depth-k record: k + 1)
 * and then by spawn count, oldest first on ties; it updates spawn counts as
 * sorted search does.  Reading: the paper notes the hybrid needs no cycle
 * monitoring; it keeps the same visited set anyway, so that all three
 * searches count bins viewed the same way.
 *
 * Candidates are kept as groups, one per viewed bin, in the order the bins
 * were viewed; a group's records are popped in slot order.  The budget is
 * the number of bins viewed (b0 and b1 included). */
static int pick_group(const orc_table *t) {
  /* a two-choice group spawns its B records; a d-ary group (one record)
   * tries its record's d bins */
  const uint32_t width = t->B == 1 ? t->d : t->B;
  int best = -1;
  for (uint64_t g = 0; g < t->n_groups; g++) {
    const group_t *q = &t->groups[g];
    if (q->next >= width) continue;
    if (t->policy == ORC_BFS) return (int)g;
    if (best < 0) { best = (int)g; continue; }
    const group_t *b = &t->groups[best];
    if (t->policy == ORC_HYBRID) {
      if (q->depth < b->depth || (q->depth == b->depth && q->skey < b->skey)) best = (int)g;
    } else if (q->skey < b->skey) {
      best = (int)g;
    }
  }
  return best;
}

static void mark_visited(orc_table *t, uint64_t bin) {
  if (t->visited[bin]) return;
  grow((void **)&t->visited_list, &t->visited_capacity, t->n_visited + 1, 8);
  t->visited[bin] = 1;
  t->visited_list[t->n_visited++] = bin;
}

static void push_group(orc_table *t, uint64_t bin, int32_t parent, int32_t pslot) {
  grow((void **)&t->groups, &t->groups_capacity, t->n_groups + 1, sizeof(group_t));
  group_t *g = &t->groups[t->n_groups++];
  g->bin = bin;
  g->parent = parent;
  g->pslot = pslot;
  g->next = 0;
  g->skey = t->spawn[bin];
  g->depth = parent < 0 ? 0 : t->groups[parent].depth + 1;
  mark_visited(t, bin);
}

static int insert_search(orc_table *t, uint64_t krec, const uint64_t *b) {
  uint64_t b0 = b[0], b1 = b[1];
  view(t); view(t);
  int s0 = lowest_free(t, b0), s1 = lowest_free(t, b1);
  if (t->ghost) {
    if (s0 >= 0 && s1 >= 0) { put_ghost_pair(t, b0, s0, b1, s1, krec); return ORC_OK; }
    if (s0 >= 0) { put(t, b0 * t->B + s0, krec, 0, 0); return ORC_OK; }
    if (s1 >= 0) { put(t, b1 * t->B + s1, krec, 0, 0); return ORC_OK; }
    if ((s0 = lowest_dup(t, b0)) >= 0) { evict_dup(t, b0, s0, krec); return ORC_OK; }
    if ((s1 = lowest_dup(t, b1)) >= 0) { evict_dup(t, b1, s1, krec); return ORC_OK; }
  } else {
    if (s0 >= 0) { put(t, b0 * t->B + s0, krec, 0, 0); return ORC_OK; }
    if (s1 >= 0) { put(t, b1 * t->B + s1, krec, 0, 0); return ORC_OK; }
  }
  t->n_groups = 0;
  push_group(t, b0, -1, -1);
  push_group(t, b1, -1, -1);
  for (;;) {
    /* one round: up to spawn_k spawns in candidate order, their bins viewed
     * together (Sec. 5: spawning the k best records at a time lets the
     * fetches overlap); the first of them, in that order, with room ends
     * the search, the others join as groups.  spawn_k = 1: the plain search. */
    int rg[8];
    uint32_t rs[8];
    uint64_t ry[8];
    uint32_t nr = 0;
    int out = 0;  /* budget spent during the round */
    while (nr < t->spawn_k) {
      int g = pick_group(t);
      if (g < 0) break;                              /* nothing left to spawn */
      uint64_t gb = t->groups[g].bin;
      uint32_t s = t->groups[g].next++;
      uint64_t r = t->rec[gb * t->B + s];
      uint64_t y = other_bin(t, r, gb);
      if (t->visited[y]) continue;
      if ((t->policy == ORC_SORTED || t->policy == ORC_HYBRID) && t->spawn[gb] < 15) t->spawn[gb]++;
      if (t->cur_viewed == t->cap) { out = 1; break; } /* budget spent */
      view(t);
      mark_visited(t, y);
      rg[nr] = g; rs[nr] = s; ry[nr] = y; nr++;
    }
    if (nr == 0) return ORC_FAILED;
    for (uint32_t i = 0; i < nr; i++) {
      int g = rg[i];
      uint32_t s = rs[i];
      uint64_t y = ry[i];
      uint64_t gb = t->groups[g].bin;
      int f = lowest_free(t, y);
      int isdup = 0;
      if (f < 0 && t->ghost) { f = lowest_dup(t, y); isdup = f >= 0; }
      if (f >= 0) {
        /* path from the root group to the spawned record */
        uint32_t depth = 1;
        for (int32_t q = g; t->groups[q].parent >= 0; q = t->groups[q].parent) depth++;
        uint64_t *path_bin = (uint64_t *)xcalloc(depth, 8);
        uint32_t *path_slot = (uint32_t *)xcalloc(depth, 4);
        uint32_t len = 0;
        path_bin[len] = gb; path_slot[len] = s; len++;
        int32_t p = g;
        while (t->groups[p].parent >= 0) {
          path_bin[len] = t->groups[t->groups[p].parent].bin;
          path_slot[len] = (uint32_t)t->groups[p].pslot;
          len++;
          p = t->groups[p].parent;
        }
        /* apply the chain from the root: the new key into the root slot, each
         * displaced record into the next slot, the last into y */
        uint64_t cur = krec;
        for (uint32_t j = len; j-- > 0;) cur = kick(t, path_bin[j], path_slot[j], cur);
        free(path_bin);
        free(path_slot);
        prop41_check(t, y);
        if (isdup) evict_dup(t, y, (uint32_t)f, cur);
        else put(t, y * t->B + f, cur, 0, 0);
        return ORC_OK;
      }
    }
    for (uint32_t i = 0; i < nr; i++) push_group(t, ry[i], rg[i], (int32_t)rs[i]);
    if (out) return ORC_FAILED;
  }
}

/* ------------------------------------------------------------------ */
/* d-ary BFS, sorted search and hybrid (Sec. 7 evaluates them; Sec. 5   */
/* defines them)                                                       */
/* ------------------------------------------------------------------ */
/* Readings (Sec. 7 names the searches for d-ary tables without restating
 * them): the first step is random kicking's, bins h_0 .. h_{d-1} viewed in
 * order until an empty one.  If all d are full, the search starts from
 * the key's d bins, each a group of one record.  Popping a group tries its
 * record's next hash function (j = 0 .. d-1); the record's own bin and
 * bins this search already viewed are skipped without a view or a spawn.
 * Otherwise the try is a spawn: the bin holding the record gets its spawn
 * count incremented (sorted search and hybrid; saturating at 15) and the
 * record's j-th bin is viewed; empty ends the search with the chain
 * root -> ... -> that bin, full makes it a new group.  Group order and the
 * budget (bins viewed, first step included) are those of Sec. 5 above. */
static int insert_search_dary(orc_table *t, uint64_t krec, const uint64_t *b) {
  for (uint32_t i = 0; i < t->d; i++) {
    view(t);
    if (is_free(t, b[i])) { put(t, b[i], krec, 0, 0); return ORC_OK; }
  }
  t->n_groups = 0;
  for (uint32_t i = 0; i < t->d; i++) push_group(t, b[i], -1, -1);
  for (;;) {
    /* rounds of spawn_k tries, as in the two-choice searches */
    int rg[8];
    uint32_t rj[8];
    uint64_t ry[8];
    uint32_t nr = 0;
    int out = 0;
    while (nr < t->spawn_k) {
      int g = pick_group(t);
      if (g < 0) break;                              /* nothing left to try */
      uint64_t gb = t->groups[g].bin;
      uint32_t j = t->groups[g].next++;
      uint64_t r = t->rec[gb];
      uint64_t rb[4];
      bins_of(t, key_of(r), rb);
      uint64_t y = rb[j];
      if (y == gb || t->visited[y]) continue;
      if ((t->policy == ORC_SORTED || t->policy == ORC_HYBRID) && t->spawn[gb] < 15) t->spawn[gb]++;
      if (t->cur_viewed == t->cap) { out = 1; break; } /* budget spent */
      view(t);
      mark_visited(t, y);
      rg[nr] = g; rj[nr] = j; ry[nr] = y; nr++;
    }
    if (nr == 0) return ORC_FAILED;
    for (uint32_t i = 0; i < nr; i++) {
      int g = rg[i];
      uint64_t y = ry[i];
      if (is_free(t, y)) {
        /* the chain from the root bin: the new key into the root, each
         * displaced record into the next bin of the path, the last into y */
        uint32_t depth = 1;
        for (int32_t q = g; t->groups[q].parent >= 0; q = t->groups[q].parent) depth++;
        uint64_t *path = (uint64_t *)xcalloc(depth, 8);
        uint32_t len = 0;
        for (int32_t q = g; q >= 0; q = t->groups[q].parent) path[len++] = t->groups[q].bin;
        uint64_t cur = krec;
        for (uint32_t j = len; j-- > 0;) {
          cur = put(t, path[j], cur, 0, 0);
          t->cur_kicks++;
        }
        free(path);
        put(t, y, cur, 0, 0);
        return ORC_OK;
      }
    }
    for (uint32_t i = 0; i < nr; i++) push_group(t, ry[i], rg[i], (int32_t)rj[i]);
    if (out) return ORC_FAILED;
  }
}

/* ------------------------------------------------------------------ */
/* d-ary tables: single-slot bins, d hash functions (Sec. 7)           */
/* ------------------------------------------------------------------ */
/* Random kicking: bins h_0 .. h_{d-1} are viewed in order until one is
 * empty (so a near-empty table views fewer than d bins, Sec. 7).  When all
 * d are full the occupant of a uniformly drawn h_j is displaced; it moves
 * to a uniformly drawn bin among its own d bins that the chain has not
 * written (which excludes the bin it was displaced from), displacing that
 * bin's occupant unless the bin is empty, and so on. */
static int insert_random_dary(orc_table *t, uint64_t krec, const uint64_t *b) {
  for (uint32_t i = 0; i < t->d; i++) {
    view(t);
    if (is_free(t, b[i])) { put(t, b[i], krec, 0, 0); return ORC_OK; }
  }
  uint64_t x = b[draw(t) % t->d];
  uint64_t cur = krec;
  for (;;) {
    if (t->cur_kicks == t->cap) return ORC_FAILED;
    t->cur_kicks++;
    cur = put(t, x, cur, 0, 0);
    uint64_t vb[4], elig[4];
    uint32_t ne = 0;
    bins_of(t, key_of(cur), vb);
    for (uint32_t i = 0; i < t->d; i++) if (!t->claimed[vb[i]]) elig[ne++] = vb[i];
    if (ne == 0) return ORC_FAILED;
    x = elig[draw(t) % ne];
    view(t);
    if (is_free(t, x)) { put(t, x, cur, 0, 0); return ORC_OK; }
  }
}

/* Rattle-kicking (Sec. 7).  r(x) counts the bins x has tried; a new key
 * starts at 0.  A key tries bin h_{r mod d} and r is incremented (saturating
 * at 255, one byte per key).  An empty bin takes it.  Otherwise the key with
 * the larger counter keeps the bin (rattle balancing) and the other one
 * tries its next bin.  Readings: counters are compared after the
 * increment; on a tie the incoming key stays and the resident is displaced
 * (the classic cuckoo move; the opposite reading is a debug switch); the
 * paper's "h_0, h_2, ..." is read as h_0, h_1, ...; a bin the chain already
 * wrote is skipped without a view; the cap counts tries. */
static int insert_rattle(orc_table *t, uint64_t krec, const uint64_t *bnew) {
  (void)bnew;
  uint64_t cur = krec;
  uint32_t rc = 0;
  uint64_t tries = 0;
  for (;;) {
    if (tries == t->cap) return ORC_FAILED;
    tries++;
    uint64_t vb[4];
    bins_of(t, key_of(cur), vb);
    uint64_t x = vb[rc % t->d];
    rc = rc < 255 ? rc + 1 : 255;
    if (t->claimed[x]) continue;
    view(t);
    if (t->rec[x] == ORC_EMPTY) { put(t, x, cur, 0, (uint8_t)rc); return ORC_OK; }
    uint32_t ry = t->rattle[x];
    int incoming_stays = t->rattle_tie_resident ? (rc > ry) : (rc >= ry);
    if (incoming_stays) {
      t->cur_kicks++;
      cur = put(t, x, cur, 0, (uint8_t)rc);
      rc = ry;
    }
  }
}

/* ------------------------------------------------------------------ */
/* public operations                                                  */
/* ------------------------------------------------------------------ */

/* Insert one key assumed absent (Sec. 3: insertions do not check
 * presence).  Returns ORC_OK or ORC_FAILED (table unchanged). */
static int insert_one(orc_table *t, uint32_t key, uint32_t val, uint32_t *viewed, uint32_t *kicks) {
  if (key == ORC_RESERVED_KEY) { if (viewed) *viewed = 0; if (kicks) *kicks = 0; return ORC_INVALID; }
  uint64_t b[4];
  bins_of(t, key, b);
  uint64_t krec = ((uint64_t)key << 32) | val;
  begin_insert(t, key);
  int st;
  if (t->B == 1) {
    if (t->policy == ORC_RATTLE) st = insert_rattle(t, krec, b);
    else if (t->policy == ORC_RANDOM) st = insert_random_dary(t, krec, b);
    else st = insert_search_dary(t, krec, b);
  } else if (t->policy == ORC_QUEUE) {
    st = insert_queue(t, krec, b);
  } else if (t->policy == ORC_BFS || t->policy == ORC_SORTED || t->policy == ORC_HYBRID) {
    st = insert_search(t, krec, b);
  } else {
    st = insert_random2(t, krec, b);
  }
  t->stats[OS_BINS_VIEWED] += t->cur_viewed;
  if (st == ORC_OK) {
    t->stats[OS_INSERTS_OK]++;
    t->stats[OS_KICKS] += t->cur_kicks;
    t->stats[OS_SIZE]++;
    if (t->cur_kicks > t->stats[OS_CHAIN_MAX]) t->stats[OS_CHAIN_MAX] = t->cur_kicks;
  } else {
    rollback(t);
    t->stats[OS_INSERTS_FAILED]++;
  }
  if (viewed) *viewed = (uint32_t)t->cur_viewed;
  if (kicks) *kicks = st == ORC_OK ? (uint32_t)t->cur_kicks : 0;
  end_insert(t);
  return st;
}

void orc_insert_batch(orc_table *t, const uint32_t *keys, const uint32_t *vals, uint64_t n,
                      uint8_t *status, uint32_t *viewed, uint32_t *kicks) {
  for (uint64_t i = 0; i < n; i++) {
    int st = insert_one(t, keys[i], vals[i], viewed ? viewed + i : NULL, kicks ? kicks + i : NULL);
    if (status) status[i] = (uint8_t)st;
  }
}

/* Lookup of one key (Sec. 1: a present key is in one of its d bins).
 * Returns 1 and the value if found.  Reads the table only. */
static int lookup_one(const orc_table *t, uint32_t key, uint32_t *val) {
  uint64_t b[4];
  *val = 0;
  if (key == ORC_RESERVED_KEY) return 0;
  bins_of(t, key, b);
  for (uint32_t j = 0; j < t->d; j++)
    for (uint32_t s = 0; s < t->B; s++) {
      uint64_t r = t->rec[b[j] * t->B + s];
      if (r != ORC_EMPTY && key_of(r) == key) { *val = (uint32_t)r; return 1; }
    }
  return 0;
}

/* Delete of one key (Sec. 1): every copy goes; a ghost pair loses both.
 * Returns found (bit 0) and whether the key was a ghost pair (bit 1).
 * Writes only the slots holding the key. */
static int delete_one(orc_table *t, uint32_t key) {
  uint64_t b[4];
  int f = 0, was_ghost = 0;
  if (key == ORC_RESERVED_KEY) return 0;
  bins_of(t, key, b);
  for (uint32_t j = 0; j < t->d; j++)
    for (uint32_t s = 0; s < t->B; s++) {
      uint64_t slot = b[j] * t->B + s;
      if (t->rec[slot] != ORC_EMPTY && key_of(t->rec[slot]) == key) {
        if (t->dup[slot]) was_ghost = 1;
        t->rec[slot] = ORC_EMPTY;
        t->dup[slot] = 0;
        t->rattle[slot] = 0;
        f = 1;
      }
    }
  return f | (was_ghost << 1);
}

void orc_lookup_batch(orc_table *t, const uint32_t *keys, uint64_t n, uint32_t *vals, uint8_t *found) {
  for (uint64_t i = 0; i < n; i++) {
    uint32_t v;
    int f = lookup_one(t, keys[i], &v);
    t->stats[OS_LOOKUPS]++;
    t->stats[OS_LOOKUP_HITS] += f;
    if (vals) vals[i] = v;
    if (found) found[i] = (uint8_t)f;
  }
}

void orc_delete_batch(orc_table *t, const uint32_t *keys, uint64_t n, uint8_t *found) {
  for (uint64_t i = 0; i < n; i++) {
    int r = delete_one(t, keys[i]);
    t->stats[OS_DELETES]++;
    if (r & 1) {
      t->stats[OS_DELETE_HITS]++;
      t->stats[OS_SIZE]--;
      if (r & 2) t->stats[OS_LIVE_GHOSTS]--;
    }
    if (found) found[i] = (uint8_t)(r & 1);
  }
}

/* The same lookups and deletes split over `threads` host threads, one
 * contiguous range of the batch each (the CPU baseline on all cores).
 * Lookups only read the table.  Deletes of distinct keys write disjoint
 * slots (every copy of a key lives in that key's own bins), so the ranges
 * never write the same slot; the keys must be distinct.  Each thread keeps
 * its own counts, added to the table's counters after the join. */
typedef struct {
  orc_table *t;
  const uint32_t *keys;
  uint64_t lo, hi;
  uint32_t *vals;
  uint8_t *found;
  int del;
  uint64_t hits, ghosts;
} range_job;

static void *range_worker(void *arg) {
  range_job *j = (range_job *)arg;
  for (uint64_t i = j->lo; i < j->hi; i++) {
    if (j->del) {
      int r = delete_one(j->t, j->keys[i]);
      j->hits += (uint64_t)(r & 1);
      j->ghosts += (uint64_t)((r >> 1) & 1);
      if (j->found) j->found[i] = (uint8_t)(r & 1);
    } else {
      uint32_t v;
      int f = lookup_one(j->t, j->keys[i], &v);
      j->hits += (uint64_t)f;
      if (j->vals) j->vals[i] = v;
      if (j->found) j->found[i] = (uint8_t)f;
    }
  }
  return NULL;
}

static int run_ranges(orc_table *t, const uint32_t *keys, uint64_t n, uint32_t *vals, uint8_t *found, int del,
                      uint32_t threads) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  range_job jobs[256];
  pthread_t tid[256];
  uint32_t started = 0;
  for (uint32_t k = 0; k < threads; k++) {
    range_job *j = &jobs[k];
    j->t = t;
    j->keys = keys;
    j->lo = n * k / threads;
    j->hi = n * (k + 1) / threads;
    j->vals = vals;
    j->found = found;
    j->del = del;
    j->hits = j->ghosts = 0;
  }
  for (uint32_t k = 1; k < threads; k++) {
    if (pthread_create(&tid[k], NULL, range_worker, &jobs[k]) != 0) break;
    started = k;
  }
  range_worker(&jobs[0]);
  for (uint32_t k = 1; k <= started; k++) pthread_join(tid[k], NULL);
  for (uint32_t k = started + 1; k < threads; k++) range_worker(&jobs[k]);  /* threads that did not start */
  uint64_t hits = 0, ghosts = 0;
  for (uint32_t k = 0; k < threads; k++) { hits += jobs[k].hits; ghosts += jobs[k].ghosts; }
  if (del) {
    t->stats[OS_DELETES] += n;
    t->stats[OS_DELETE_HITS] += hits;
    t->stats[OS_SIZE] -= hits;
    t->stats[OS_LIVE_GHOSTS] -= ghosts;
  } else {
    t->stats[OS_LOOKUPS] += n;
    t->stats[OS_LOOKUP_HITS] += hits;
  }
  return (int)(started + 1);
}

int orc_lookup_batch_threads(orc_table *t, const uint32_t *keys, uint64_t n, uint32_t *vals, uint8_t *found,
                             uint32_t threads) {
  return run_ranges(t, keys, n, vals, found, 0, threads);
}

int orc_delete_batch_threads(orc_table *t, const uint32_t *keys, uint64_t n, uint8_t *found, uint32_t threads) {
  return run_ranges(t, keys, n, NULL, found, 1, threads);
}

/* Insert with the absent-key assumption of Sec. 3 lifted (upsert): a key
 * already present gets the new value in every copy (a ghost pair keeps its
 * duplicate marks) and status 5; an absent key is inserted as by
 * orc_insert_batch.  Keys are taken in order, so a key repeated in the batch
 * is inserted once and then updated. */
void orc_upsert_batch(orc_table *t, const uint32_t *keys, const uint32_t *vals, uint64_t n, uint8_t *status) {
  for (uint64_t i = 0; i < n; i++) {
    uint64_t b[4];
    int f = 0;
    if (keys[i] != ORC_RESERVED_KEY) {
      bins_of(t, keys[i], b);
      for (uint32_t j = 0; j < t->d; j++)
        for (uint32_t s = 0; s < t->B; s++) {
          uint64_t slot = b[j] * t->B + s;
          if (t->rec[slot] != ORC_EMPTY && key_of(t->rec[slot]) == keys[i]) {
            t->rec[slot] = ((uint64_t)keys[i] << 32) | vals[i];
            f = 1;
          }
        }
    }
    if (f) {
      t->stats[OS_UPDATES]++;
      if (status) status[i] = 5;
      continue;
    }
    int st = insert_one(t, keys[i], vals[i], NULL, NULL);
    if (status) status[i] = (uint8_t)st;
  }
}

void orc_stats(const orc_table *t, uint64_t *out) { memcpy(out, t->stats, sizeof(t->stats)); }
uint32_t orc_n_stats(void) { return OS_N; }

/* Copy out the state: records, duplicate marks, rattle counters (per slot);
 * hit counters, spawn counts (per bin).  Any pointer may be NULL. */
void orc_export(const orc_table *t, uint64_t *rec, uint8_t *dup, uint8_t *rattle, uint8_t *hit, uint8_t *spawn) {
  uint64_t ns = t->n * t->B;
  if (rec) memcpy(rec, t->rec, ns * 8);
  if (dup) memcpy(dup, t->dup, ns);
  if (rattle) memcpy(rattle, t->rattle, ns);
  if (hit) memcpy(hit, t->hit, t->n);
  if (spawn) memcpy(spawn, t->spawn, t->n);
}

/* Structural invariants: every key in one of its bins; a duplicate in
 * exactly both of its bins, each copy marked; plain keys exactly once;
 * size and ghost counters match; spawn counts at most 15.  Returns 0 when
 * all hold, else the number of violations (first one described in msg). */
int orc_check_invariants(const orc_table *t, char *msg, uint64_t msglen) {
  int bad = 0;
  uint64_t keys = 0, ghosts = 0;
  uint64_t ns = t->n * t->B;
  for (uint64_t slot = 0; slot < ns; slot++) {
    uint64_t r = t->rec[slot];
    uint64_t here = slot / t->B;
    if (r == ORC_EMPTY) {
      if (t->dup[slot]) { if (!bad && msg) snprintf(msg, msglen, "empty slot %llu marked duplicate", (unsigned long long)slot); bad++; }
      continue;
    }
    uint64_t b[4];
    bins_of(t, key_of(r), b);
    int mine = 0;
    for (uint32_t j = 0; j < t->d; j++) if (b[j] == here) mine = 1;
    if (!mine) { if (!bad && msg) snprintf(msg, msglen, "key %u in bin %llu outside its bins", key_of(r), (unsigned long long)here); bad++; }
    /* count copies over all d bins */
    int copies = 0, marked = 0, bins_with_copy = 0;
    for (uint32_t j = 0; j < t->d; j++) {
      int in_bin = 0;
      for (uint32_t s = 0; s < t->B; s++) {
        uint64_t o = b[j] * t->B + s;
        if (t->rec[o] != ORC_EMPTY && key_of(t->rec[o]) == key_of(r)) { copies++; in_bin++; marked += t->dup[o]; }
      }
      bins_with_copy += in_bin > 0;
    }
    if (copies == 1 && marked == 0) keys++;
    else if (copies == 2 && marked == 2 && t->d == 2 && bins_with_copy == 2) { if (here == b[0]) { keys++; ghosts++; } }
    else { if (!bad && msg) snprintf(msg, msglen, "key %u has %d copies, %d marked", key_of(r), copies, marked); bad++; }
  }
  if (keys != t->stats[OS_SIZE]) { if (!bad && msg) snprintf(msg, msglen, "size %llu != counted %llu", (unsigned long long)t->stats[OS_SIZE], (unsigned long long)keys); bad++; }
  if (ghosts != t->stats[OS_LIVE_GHOSTS]) { if (!bad && msg) snprintf(msg, msglen, "ghosts %llu != counted %llu", (unsigned long long)t->stats[OS_LIVE_GHOSTS], (unsigned long long)ghosts); bad++; }
  for (uint64_t x = 0; x < t->n; x++) if (t->spawn[x] > 15) { if (!bad && msg) snprintf(msg, msglen, "spawn > 15"); bad++; }
  return bad;
}
