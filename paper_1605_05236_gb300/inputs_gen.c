/*
 * inputs_gen.c -- seeded synthetic inputs (keys, values, orders) shared by
 * the tests, the benchmark and the oracle.  No cuckoo-table arithmetic
 * lives here: only the SplitMix64 generator, a set used to drop repeated
 * keys, and Fisher-Yates shuffles.
 *
 * Key stream of seed s: output i (i = 0, 1, ...) of SplitMix64 seeded with
 * s (state s + (i+1)*0x9E3779B97F4A7C15, then mixed), high 32 bits.  A key
 * equal to 0xFFFFFFFF, to an earlier accepted key, or to a key of the
 * exclusion list is skipped.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ull
#define RESERVED 0xFFFFFFFFu

static uint64_t sm64_out(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * GAMMA;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

typedef struct {
  uint32_t *v;
  uint64_t mask;
  int shift;
} kset;

static int set_init(kset *s, uint64_t n) {
  uint64_t cap = 1024;
  int bits = 10;
  while (cap < 2 * n + 16) { cap <<= 1; bits++; }
  s->v = (uint32_t *)malloc(cap * sizeof(uint32_t));
  if (!s->v) return -1;
  memset(s->v, 0xFF, cap * sizeof(uint32_t));
  s->mask = cap - 1;
  s->shift = 64 - bits;
  return 0;
}

/* returns 1 if inserted, 0 if it was present */
static int set_add(kset *s, uint32_t k) {
  uint64_t h = ((uint64_t)k * 0x9E3779B97F4A7C15ull) >> s->shift;
  for (;;) {
    uint32_t e = s->v[h];
    if (e == k) return 0;
    if (e == RESERVED) { s->v[h] = k; return 1; }
    h = (h + 1) & s->mask;
  }
}

/* n distinct keys from the stream of `seed` starting at output `start`,
 * skipping the n_ex keys of `exclude`.  Writes out[0..n) and returns the
 * stream index just after the last accepted key (or -1 on allocation
 * failure). */
int64_t gen_distinct_keys(uint64_t seed, uint64_t start, uint64_t n, const uint32_t *exclude,
                          uint64_t n_ex, uint32_t *out) {
  kset s;
  if (set_init(&s, n + n_ex)) return -1;
  for (uint64_t i = 0; i < n_ex; i++) set_add(&s, exclude[i]);
  uint64_t i = start, got = 0;
  while (got < n) {
    uint32_t k = (uint32_t)(sm64_out(seed, i) >> 32);
    i++;
    if (k == RESERVED) continue;
    if (!set_add(&s, k)) continue;
    out[got++] = k;
  }
  free(s.v);
  return (int64_t)i;
}

/* First k entries of a forward Fisher-Yates shuffle of 0..n-1 driven by
 * the stream of `seed`: for i < k, swap a[i] with a[i + out_i mod (n-i)]. */
int gen_permutation(uint64_t seed, uint64_t n, uint64_t k, uint64_t *out) {
  uint64_t *a = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
  if (!a) return -1;
  for (uint64_t i = 0; i < n; i++) a[i] = i;
  if (k > n) k = n;
  for (uint64_t i = 0; i < k && i + 1 < n; i++) {
    uint64_t j = i + sm64_out(seed, i) % (n - i);
    uint64_t t = a[i];
    a[i] = a[j];
    a[j] = t;
  }
  memcpy(out, a, k * sizeof(uint64_t));
  free(a);
  return 0;
}

/* gather: out[i] = src[idx[i]] (uint32) */
void gen_gather_u32(const uint32_t *src, const uint64_t *idx, uint64_t n, uint32_t *out) {
  for (uint64_t i = 0; i < n; i++) out[i] = src[idx[i]];
}
