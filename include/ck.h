/*
 * ck.h -- C ABI of libck.so, GB300 (sm_103a) cuckoo hash tables with the
 * kick-out eviction policies and claim flags of W. Kuszmaul, "Fast
 * Concurrent Cuckoo Kick-out Eviction Schemes for High-Density Tables"
 * (arXiv:1605.05236).
 *
 * Problem statement (Sec. 1): each key maps to distinct bins by hash
 * functions; an insertion places the key into a free slot of one of its
 * bins, otherwise it kicks a resident record out and re-inserts it,
 * forming a kick-out chain.  Reads, overwrites and deletes touch only the
 * key's own bins.  Tables are either two hash functions over bins of B = 4
 * or 8 slots (Sec. 1, Sec. 3) or d = 3 or 4 hash functions over single-slot
 * bins (d-ary cuckoo hashing, Sec. 7).
 *
 * Conventions for every call:
 *   - Return value: CK_OK (0) or a negative CK_E* code; nothing is launched
 *     when a call returns an error before launching.  ck_strerror() names a
 *     code.
 *   - Key/value/status pointers of the *_batch calls are DEVICE pointers
 *     owned by the caller; they must stay valid until the stream reaches
 *     the work.  Keys are uint32; 0xFFFFFFFF is reserved (it marks an empty
 *     slot) and is rejected per key with CK_ST_INVALID.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Batch
 *     calls are asynchronous on it.  Calls on one table must be ordered by
 *     the caller (one stream, or events); a table handle is not safe for
 *     concurrent use from several host threads.
 *   - Layout in device memory (one buffer per table): slots (n_bins * B
 *     uint64, key << 32 | value, all-ones when empty), then one uint32
 *     metadata word per bin, then device counters, then search scratch.
 */
#ifndef CK_H
#define CK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define CK_OK 0
#define CK_EINVAL (-1)   /* bad argument (sizes, policy/shape mix, null) */
#define CK_ENOMEM (-2)   /* device or host allocation failed / buffer too small */
#define CK_ECUDA (-3)    /* a CUDA runtime call failed */
#define CK_EBUSY (-4)    /* admission refused (serving form) */
#define CK_ENOTSUP (-5)  /* combination not implemented */

/* ---- per-key status written by ck_insert_batch ---- */
#define CK_ST_OK 0       /* inserted */
#define CK_ST_FAILED 1   /* chain cap / search budget reached; key absent, table as before */
#define CK_ST_ABORTED 2  /* claim conflicts exceeded the retry limit; key absent */
#define CK_ST_INVALID 3  /* reserved key 0xFFFFFFFF */
#define CK_ST_UPDATED 5  /* CK_INS_UPSERT: the key was present; every copy now holds the new value */

/* ---- kick-out policies (Sec. 3-7), ghost insertions OR-able (Sec. 4) ---- */
#define CK_RANDOM 0      /* random kicking (Sec. 1) */
#define CK_BFS 1         /* breadth-first search (Sec. 1, Sec. 5) */
#define CK_SORTED 2      /* sorted search by spawn count (Sec. 5) */
#define CK_QUEUE 3       /* queue-kicking, hit counters, hit balancing (Sec. 6) */
#define CK_RATTLE 4      /* rattle-kicking, d-ary only (Sec. 7) */
#define CK_HYBRID 5      /* sorted search / BFS hybrid: depth first, then spawn count (Sec. 5, end) */
#define CK_GHOST 0x100   /* ghost insertions; with RANDOM/BFS/SORTED/QUEUE/HYBRID, two-choice only */

/* ---- runtime parameters for ck_set_param ---- */
#define CK_PARAM_CHAIN_CAP 1     /* kick-outs (walks), tries (rattle), bins viewed (search); default 500 */
#define CK_PARAM_MAX_RETRIES 2   /* attempts per key after claim conflicts; default 1024 */
#define CK_PARAM_RNG_SEED 3      /* seed of the counter-based kick-out draws */
#define CK_PARAM_HASH_SEED0 10   /* + i for seed_i, i < d (defaults 0x9E3779B9, 0x85EBCA6B, 0xC2B2AE35, 0x27D4EB2F) */
#define CK_PARAM_BLOCK 20        /* threads per block of the insert kernels: 32, 64, 128 or 256;
                                    default 256 for 4-slot queue-kicking tables, else 128 */
#define CK_PARAM_RATTLE_TIE_RESIDENT 30 /* 1: the resident wins rattle ties (debug reading) */
#define CK_PARAM_ORDERED_WRITES 31      /* chains are always written back to front (Sec. 8);
                                           1: a release fence between consecutive writes makes
                                           that order visible, so a reader that does not
                                           validate never misses a moving key.  0 (default):
                                           one fence per chain -- every reader in this library
                                           either validates against claims (server lookups,
                                           deletes) or does not overlap writers (bulk lookups) */
#define CK_PARAM_OVERLAP 32     /* 1 (default): an insert launch may start while the previous
                                   one on the stream finishes its longest chains */
#define CK_PARAM_SPAWN_K 34     /* searches (BFS, sorted, hybrid): spawns per round, 1..8
                                   (default 1).  Sec. 5: spawning the k best candidates at a
                                   time lets their bins be fetched together; every bin of a
                                   round counts as viewed, and the first with room, in
                                   candidate order, ends the search. */
#define CK_PARAM_MAX_INFLIGHT 35 /* insertions one insert launch keeps in flight at most
                                    (0, the default: as many threads as fit on the GPU --
                                    nine tenths of that for random kicking and queue-kicking,
                                    eight tenths for rattle-kicking, when launches overlap,
                                    so that the next launch starts beside this one's longest
                                    walks; else
                                    whole blocks, one at least).  Claim conflicts grow with the
                                    share of a table's slots in flight, so a small table can
                                    fill faster with fewer insertions at once, each thread
                                    taking more keys. */
#define CK_PARAM_SEARCH_WARP 36 /* 1: breadth-first search on a two-choice table without ghosts
                                   is run by a whole warp per key (spawn_k 1 only): the
                                   candidates of the search order are viewed 32 at a time and
                                   the first with room in that order ends the search, so it
                                   views more bins (all counted) in fewer round trips; the
                                   search state stays in shared memory.  Searches longer than
                                   128 groups or out of budget continue as CK_BFS does.
                                   Concurrent inserts only (CK_INS_SERIAL and CK_INS_UPSERT
                                   run the per-thread kernel).  Default 0; CK_EINVAL for any
                                   other table. */
#define CK_PARAM_SEARCH_WARP_LOAD 37 /* with CK_PARAM_SEARCH_WARP: the warp form runs only the
                                        insert calls that start with the table at least this
                                        full, in thousandths (0..1000; default 0: every call);
                                        the calls before run the per-thread kernel. */
#define CK_PARAM_HASH_FAMILY 33 /* 0 (default): h_i = fmix32(k ^ seed_i); 1: decorrelated
                                   h_i = fmix32(fmix32(k + seed_i) ^ (seed_i * 0x27D4EB2F)).
                                   Set before the first insertion. */

/* ---- ck_insert_batch_ex flags ---- */
#define CK_INS_SERIAL 1  /* one insertion in flight, keys in batch order (debug/parity) */
#define CK_INS_UPSERT 2  /* lift the absent-key assumption (Sec. 3): a present key gets its value
                            overwritten in place (CK_ST_UPDATED), an absent one is inserted; keys
                            must be distinct within the batch and not written by another call
                            running at the same time */

/* ---- counters returned by ck_stats (device totals since the last reset) ---- */
typedef struct ck_stats_t {
  uint64_t inserts_ok;
  uint64_t inserts_failed;      /* CK_ST_FAILED */
  uint64_t inserts_aborted;     /* CK_ST_ABORTED */
  uint64_t bins_viewed;         /* bins examined by the attempt of each insertion that was
                                   applied or failed (the Sec. 3 metric) */
  uint64_t kicks;               /* records displaced by successful insertions */
  uint64_t chain_max;           /* longest kick-out chain */
  uint64_t aborts;              /* attempts abandoned on a claim conflict (Sec. 8) */
  uint64_t ghost_pairs_made;    /* ghost insertions (Sec. 4) */
  uint64_t dup_evictions;       /* duplicates overwritten */
  uint64_t size;                /* distinct live keys */
  uint64_t live_ghosts;         /* live ghost pairs */
  uint64_t lookups, lookup_hits;
  uint64_t deletes, delete_hits, delete_aborts;
  uint64_t conflict_views;      /* bins viewed again after a lost claim race */
  uint64_t bins_viewed_all;     /* bins examined by all attempts, abandoned ones included */
  uint64_t total_slots;         /* n_bins * B */
  double load;                  /* size / total_slots */
  double bins_viewed_per_insert;/* bins_viewed / (inserts_ok + failed + aborted) */
  double aborts_per_insert;
  uint64_t updates;             /* CK_INS_UPSERT: present keys overwritten (CK_ST_UPDATED) */
} ck_stats_t;

typedef struct ck_table ck_table; /* opaque; owned by the library */

/* Bytes of device memory a table needs (slots, metadata, counters and,
 * for the search policies, scratch).  0 when the shape is invalid. */
size_t ck_required_bytes(uint64_t bins, uint32_t slots_per_bin, uint32_t d, uint32_t policy);

/* Create a table whose device memory the library allocates (cudaMalloc on
 * the current device) and clears.  bins: n_bins >= d, < 2^32; slots_per_bin:
 * 4 or 8 with d = 2, 1 with d = 3 or 4; policy: CK_* above.  seed: the
 * kick-out draw seed.  *out receives the handle.  Synchronous. */
int ck_create(ck_table **out, uint64_t bins, uint32_t slots_per_bin, uint32_t d,
              uint32_t policy, uint64_t seed);

/* Same, over caller-owned device memory (e.g. a torch tensor): dev_buf must
 * be 256-byte aligned and at least ck_required_bytes(...) long; it stays
 * owned by the caller and must outlive the table.  Cleared on `stream`. */
int ck_create_on(ck_table **out, void *dev_buf, size_t bytes, uint64_t bins,
                 uint32_t slots_per_bin, uint32_t d, uint32_t policy, uint64_t seed,
                 void *stream);

/* Set a CK_PARAM_*; CK_EINVAL for an unknown key or out-of-range value. */
int ck_set_param(ck_table *t, int key, int64_t value);

/* Insert n keys with values (Sec. 1; the paper assumes each key is absent
 * and distinct, Sec. 3 -- a key already present gets a second copy).
 * Concurrent insertions claim every slot they will write with a one-bit
 * claim flag and skip slots others claimed (Sec. 8 "Claim Flags"); chains
 * are executed back to front (Sec. 8 "System-Transaction Kick-Outs"), so a
 * failed or aborted insertion changes nothing.  d_status (nullable): n
 * CK_ST_* bytes. */
int ck_insert_batch(ck_table *t, const uint32_t *d_keys, const uint32_t *d_vals, uint64_t n,
                    uint8_t *d_status, void *stream);

/* As ck_insert_batch, plus d_viewed (nullable): bins viewed by each key,
 * and flags (CK_INS_SERIAL). */
int ck_insert_batch_ex(ck_table *t, const uint32_t *d_keys, const uint32_t *d_vals, uint64_t n,
                       uint8_t *d_status, uint32_t *d_viewed, uint32_t flags, void *stream);

/* Look up n keys (Sec. 1: a present key is in one of its bins).  Writes
 * d_vals_out[i] (0 when absent) and d_found[i] in {0,1}; either nullable.
 * The reads are not validated against writers: call it while no insertion
 * or delete on this table is in flight on another stream (the serving
 * form's lookups are validated and may overlap writers). */
int ck_lookup_batch(ck_table *t, const uint32_t *d_keys, uint64_t n, uint32_t *d_vals_out,
                    uint8_t *d_found, void *stream);

/* Delete n keys (Sec. 1), every copy of a ghost pair included.  d_found[i]
 * (nullable) = 1 if this call removed the key, 0 if it was absent.  Safe
 * beside insertions running on other streams: a slot claimed by an
 * in-flight insertion (Sec. 8) is waited out with backoff, and a miss is
 * reported only after the key's bins were read unclaimed and unchanged;
 * after 1024 such retries the key gets 2 (not resolved). */
int ck_delete_batch(ck_table *t, const uint32_t *d_keys, uint64_t n, uint8_t *d_found,
                    void *stream);

/* Copy the device counters (synchronises the table's last stream). */
int ck_stats(ck_table *t, ck_stats_t *out);

/* Bins-viewed histogram by load before each insertion, 200 buckets of
 * 0.5%: views[i], inserts[i] for load in [i/200, (i+1)/200).  Host arrays
 * of 200 uint64 each; synchronous. */
int ck_load_histogram(ck_table *t, uint64_t *views, uint64_t *inserts);

/* Chain lengths of the successful insertions since the last reset (Fig. D
 * of the paper plots their distribution for walks and searches):
 * counts[i] = insertions with i kick-outs for i < 32, with 2^(i-27) ..
 * 2^(i-26) - 1 kick-outs for 32 <= i < 39, and with >= 4096 for i = 39.
 * A search counts the length of the path it applied; a ghost pair 0.
 * counts: host array of 40 uint64.  Synchronous. */
#define CK_CHAIN_BUCKETS 40
int ck_chain_histogram(ck_table *t, uint64_t *counts);

/* Zero the counters (asynchronous on the last stream used). */
int ck_reset_stats(ck_table *t);

/* Empty the table and zero the counters (asynchronous). */
int ck_clear(ck_table *t, void *stream);

/* Copy the table to host memory (synchronous): slots (n_bins*B uint64) and
 * meta (n_bins uint32: bits 0-7 claim, 8-15 duplicate, 16-19 spawn count,
 * 20-27 hit counter, 28-31 version; d-ary: bit 0 claim, 8-15 rattle
 * counter).  Either pointer may be NULL. */
int ck_export(ck_table *t, uint64_t *h_slots, uint32_t *h_meta);

/* Restore a table from a snapshot ck_export wrote (synchronous): slots and
 * meta in the layout above, from host memory, for a table of the same shape
 * (the caller's responsibility; the sizes are this table's).  Checked first:
 * no claim flag set (the snapshot must come from a table with no call in
 * flight), duplicate marks only on occupied slots and an even number of
 * them, no stored key 0xFFFFFFFF -- CK_EINVAL otherwise, and the table is
 * left untouched.  Counters restart at zero except size and live ghost
 * pairs, which are recomputed from the snapshot.  Spawn counts, hit
 * counters, rattle counters and versions are restored as they were, so
 * insertions continue exactly as they would have in the exported table
 * (transaction IDs help logging and snapshots, Sec. 8). */
int ck_import(ck_table *t, const uint64_t *h_slots, const uint32_t *h_meta);

/* Free the table (and its memory, when ck_create allocated it). */
void ck_destroy(ck_table *t);

/* Shape of a table: any pointer may be NULL. */
int ck_shape(const ck_table *t, uint64_t *bins, uint32_t *slots_per_bin, uint32_t *d,
             uint32_t *policy);

const char *ck_strerror(int code);

/* ---- insertion without allocation (the paper has no counterpart) ----
 *
 * For callers that must not allocate device memory on their insertion path:
 * services whose device memory budget is fixed up front, real-time sections
 * where an allocation's latency is not acceptable, libraries embedding this
 * one that own no device allocator.  Same operation and per-key status as
 * ck_insert_batch (the key -> value map it leaves is the one ck_insert_batch
 * leaves for the same keys; the slot layout may differ, as between any two
 * concurrent runs), but the per-search scratch of breadth-first and sorted search comes from a fixed
 * array compiled into libck.so (CK_NOALLOC_MAX_KEYS regions of 16,528 bytes,
 * 8.1 MiB, in the memory of every GPU that loads the library, kept until the
 * process exits), one region per key, and the call allocates nothing.
 *   - n > CK_NOALLOC_MAX_KEYS: returns CK_EINVAL and launches nothing.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call uses the same array: calls whose kernels overlap on the GPU
 *     (other streams, other tables) race on it and must be ordered by the
 *     caller.  The array keeps the last call's contents; nothing in it has
 *     to start at zero.
 *   - The table's counters, bins-viewed-by-load histogram and chain-length
 *     histogram are updated as ck_insert_batch updates them, and the
 *     handle's readers (ck_stats, the histograms, ck_export) wait for this
 *     call's stream.
 *   - Insertions are concurrent (one thread per key) as in ck_insert_batch's
 *     concurrent mode, failed walks retried the same way; the launch does
 *     not overlap the previous insert launch. */
#define CK_NOALLOC_MAX_KEYS 512
int ck_insert_batch_noalloc(ck_table *t, const uint32_t *d_keys, const uint32_t *d_vals, uint64_t n,
                            uint8_t *d_status, void *stream);

/* ---- batched form: many independent two-choice tables, one launch ----
 *
 * Thousands of independent tables of uneven sizes in one device buffer,
 * filled by one persistent launch (a queue of key tiles over all tables)
 * instead of one launch per table.  Each table behaves exactly like a
 * ck_table with the same shape and policy: the same kick-out policies
 * (RANDOM or QUEUE, optionally | GHOST), claim flags and back-to-front
 * chains (Sec. 3-8), the default hash seeds, and the draw seed seed + i for
 * table i.  Keys of table i are key_offset .. key_offset + n_keys - 1 of the
 * shared key/value/status arrays (device pointers). */
typedef struct ck_multi_desc {
  uint64_t bins;          /* n_bins of this table (>= 2, < 2^32; need not be a power of two) */
  uint32_t slots_per_bin; /* 4 or 8 */
  uint32_t pad;
  uint64_t key_offset;
  uint64_t n_keys;
} ck_multi_desc;

typedef struct ck_multi ck_multi;

/* Device bytes for n tables with these descriptors (0 when invalid). */
size_t ck_multi_required_bytes(const ck_multi_desc *h_desc, uint32_t n_tables);

/* Create the tables in one caller-owned device buffer (256-byte aligned,
 * >= ck_multi_required_bytes); clears them on `stream`. */
int ck_multi_create_on(ck_multi **out, void *dev_buf, size_t bytes, const ck_multi_desc *h_desc,
                       uint32_t n_tables, uint32_t policy, uint64_t seed, void *stream);

/* Launch-shape knobs (chosen by the autotuner): keys per tile (>= 256),
 * threads per block (64/128/256), resident blocks per SM (0 = as many as
 * fit), chain cap of every table. */
#define CK_MULTI_TILE 1
#define CK_MULTI_BLOCK 2
#define CK_MULTI_BLOCKS_PER_SM 3
#define CK_MULTI_CHAIN_CAP 4
int ck_multi_set_param(ck_multi *m, int key, int64_t value);

/* Insert every table's keys: one persistent launch; blocks take tiles in
 * the order of a list interleaved over the tables.  Asynchronous. */
int ck_multi_insert(ck_multi *m, const uint32_t *d_keys, const uint32_t *d_vals, uint8_t *d_status,
                    void *stream);

/* The reference path: one single-table insert launch per table (the same
 * per-insertion code), for comparison. */
int ck_multi_insert_per_table(ck_multi *m, const uint32_t *d_keys, const uint32_t *d_vals,
                              uint8_t *d_status, void *stream);

/* Look up n keys, key i in table d_table[i] (outputs as ck_lookup_batch). */
int ck_multi_lookup(ck_multi *m, const uint32_t *d_table, const uint32_t *d_keys, uint64_t n,
                    uint32_t *d_vals_out, uint8_t *d_found, void *stream);

/* Counters of one table / summed over all tables (synchronise). */
int ck_multi_table_stats(ck_multi *m, uint32_t table, ck_stats_t *out);
int ck_multi_stats(ck_multi *m, ck_stats_t *out);

/* Copy one table out (as ck_export; synchronous). */
int ck_multi_export(ck_multi *m, uint32_t table, uint64_t *h_slots, uint32_t *h_meta);

/* Empty every table (asynchronous) / free the handle (not the buffer). */
int ck_multi_clear(ck_multi *m, void *stream);
void ck_multi_destroy(ck_multi *m);

/* A batched fill captured once and replayed as a CUDA graph: launching the
 * thousands of operations of a fill (a clear is three copies per table;
 * the per-table path launches one kernel per table) costs the host more
 * than the GPU spends on them, and a graph replays them with one call.
 * ck_multi_capture records, on `stream` (NULL: a stream of the library's
 * own), an optional clear of every table (CK_MULTI_CAPTURE_CLEAR) followed
 * by ck_multi_insert -- or ck_multi_insert_per_table with
 * CK_MULTI_CAPTURE_PER_TABLE -- of the given device arrays, and
 * instantiates it; nothing runs until ck_graph_launch.  The graph keeps the
 * pointers and launch shape of the capture: replaying it fills the same
 * arrays into the same tables (capture again after ck_multi_set_param or
 * for other arrays).  Capture mode is thread-local, so other host threads
 * may use CUDA meanwhile; `stream` must not be capturing already.
 * Returns CK_EINVAL for bad arguments or flags, CK_ECUDA if the capture or
 * instantiation fails (no handle is returned then).  ck_graph_launch is
 * asynchronous on `stream`; the batched handle's readers then wait for that
 * stream.  ck_graph_destroy frees the graph (not the tables). */
typedef struct ck_graph ck_graph;
#define CK_MULTI_CAPTURE_CLEAR 1u
#define CK_MULTI_CAPTURE_PER_TABLE 2u
int ck_multi_capture(ck_multi *m, const uint32_t *d_keys, const uint32_t *d_vals, uint8_t *d_status,
                     uint32_t flags, void *stream, ck_graph **out);
int ck_graph_launch(ck_graph *g, void *stream);
void ck_graph_destroy(ck_graph *g);

/* ---- serving form: a continuous-batching request loop ----
 *
 * A server owns a resident table (created with ck_create/ck_create_on)
 * and two host threads.  Requests (lookup, insert or delete of n keys in
 * host memory) are submitted as they arrive; the scheduler merges every
 * pending request that fits into the next free wave slot (keys copied into
 * pinned staging, one device batch per kind), launches the three kinds on
 * three streams, and goes on forming the next wave while earlier ones run
 * (continuous batching).  A completion thread copies results out and
 * timestamps each request.  Inserts are admitted only while the table's
 * load (live keys + admitted inserts) stays at or below load_hi; an insert
 * that waits longer than max_defer_us completes with CK_ST_BUSY.  Wave
 * staging is sized to fit in hbm_fraction of the device memory free at
 * creation (fewer slots if needed).  Lookups in the server validate their
 * reads against concurrent writers: a miss counts only when the key's bins
 * were unclaimed and unchanged across the read (status 2 after 1024
 * retries: not resolved).  The table must not be used by other calls while
 * a server owns it.  The paper has no serving loop; it is the continuous
 * form of its bulk operations (Sec. 8 concurrency). */
#define CK_OP_LOOKUP 0
#define CK_OP_INSERT 1
#define CK_OP_DELETE 2
#define CK_ST_BUSY 4     /* insert not admitted: the table stayed above load_hi */

typedef struct ck_server_config {
  uint64_t wave_keys;    /* keys per kind per wave (default 2^20; a request may not exceed it) */
  uint32_t wave_slots;   /* waves in flight (default 4) */
  uint32_t pad;
  double load_hi;        /* admission bound for inserts (default 0.97) */
  uint64_t max_defer_us; /* longest wait of a deferred insert (default 20000) */
  double hbm_fraction;   /* share of free device memory the staging may take (default 0.25) */
} ck_server_config;

typedef struct ck_server ck_server;

/* cfg may be NULL for the defaults.  Synchronises the table's stream. */
int ck_server_create(ck_server **out, ck_table *t, const ck_server_config *cfg);

/* Queue a request; h_* are host buffers that must stay valid until the
 * request completes.  t_arrive_ns (0 = now, ck_now_ns clock) is the arrival
 * time latency is measured from.  *ticket is waited on with ck_server_wait. */
int ck_server_submit(ck_server *s, uint32_t op, const uint32_t *h_keys, const uint32_t *h_vals, uint64_t n,
                     uint32_t *h_vals_out, uint8_t *h_status_out, int64_t t_arrive_ns, void **ticket);

/* Block until the request is done (frees the ticket); *latency_ns =
 * completion - arrival. */
int ck_server_wait(ck_server *s, void *ticket, int64_t *latency_ns);

/* Monotonic clock of the server, nanoseconds. */
int64_t ck_now_ns(void);

/* Open-loop replay of a trace: request i (op[i]; keys key_off[i] ..
 * key_off[i] + n_keys[i] - 1 of the host arrays) is submitted at
 * arrive_ns[i] after the call starts; waits for all; per-request latency. */
int ck_server_replay(ck_server *s, uint64_t n_req, const uint32_t *op, const uint64_t *key_off,
                     const uint64_t *n_keys, const int64_t *arrive_ns, const uint32_t *keys,
                     const uint32_t *vals, uint32_t *vals_out, uint8_t *status_out, int64_t *latency_ns);

/* The same trace as plain sequential bulk calls on one stream (request i
 * starts once it has arrived and request i-1 is done): the reference. */
int ck_replay_sequential(ck_table *t, uint64_t n_req, const uint32_t *op, const uint64_t *key_off,
                         const uint64_t *n_keys, const int64_t *arrive_ns, const uint32_t *keys,
                         const uint32_t *vals, uint32_t *vals_out, uint8_t *status_out,
                         int64_t *latency_ns, void *stream);

/* Waves launched, inserts refused, current load, wave slots. */
int ck_server_info(ck_server *s, uint64_t *waves, uint64_t *busy_rejects, double *load, uint32_t *wave_slots);

/* Stop the threads (after draining) and free the server (not the table). */
void ck_server_destroy(ck_server *s);

/* ---- transactional layer (Sec. 8) ----
 *
 * Transactions of inserts, reads, overwrites and deletes on two-choice
 * tables of n bins x B slots, under the optimistic concurrency scheme of
 * Sec. 8 (read and write sets of version IDs; Stage 1 plans, Stage 2 locks
 * the write set in a global order and verifies both sets, Stage 3 applies
 * and stamps every written slot and bin with the transaction ID), with the
 * mechanisms of Sec. 8 that reduce aborts as flags.
 *
 * One handle holds `trials` independent tables, run side by side by one
 * launch: trial r hashes with its own salted seed pair, and all trials run
 * the same operation arrays.  A worker (the paper's thread) is one warp and
 * runs its transactions in order; workers run concurrently.  Every wait on a
 * lock is bounded; a lock not obtained within the bound aborts the attempt,
 * and an aborted attempt runs again: at most 100,000 attempts, and none
 * once the worker has run 120 s in this launch (its remaining transactions
 * are given up).
 *
 * Operations (d_op): CK_TX_INSERT (key, val): adds the record; status 0,
 * or 1 if the key was present already (nothing written).  CK_TX_READ: status
 * 1 and the value if present, else status 0.  CK_TX_OVERWRITE /
 * CK_TX_DELETE: status 1 if the key was present (value replaced / record
 * removed), else 0.  A transaction names each key at most once.  A
 * transaction given up (attempt or time bound, an insert with no
 * placement within 500 kick-outs, four attempts that overflowed the read
 * set of 512 or the write set of 1024 entries, or 64 attempts whose inserts
 * found no eligible slot) gets status 255 on all its operations and writes
 * nothing.  Each operation takes up to 2 read-set
 * entries; an insert takes 2 write-set entries plus 2 per kick-out. */
#define CK_TX_INSERT 0
#define CK_TX_READ 1
#define CK_TX_OVERWRITE 2
#define CK_TX_DELETE 3

/* Mechanisms (Sec. 8 "Mechanisms for Reducing Aborts"; queue-kicking with
 * hit counters, Sec. 5).  No flag: the naive scheme (random kicking). */
#define CK_TXF_LOCAL_RETRY 1u  /* a moved bin version: re-check the key's absence, not abort */
#define CK_TXF_QUEUE 2u        /* the slot a record takes is the bin's hit counter mod B */
#define CK_TXF_SYSTEM 4u       /* kick-out chains done in Stage 1, last move first, one small transaction each */
#define CK_TXF_CLAIM 8u        /* slots joining a write set are claimed; chains pass over claimed slots */

#define CK_TXN_MAX_OPS 256     /* operations per transaction */
#define CK_TXN_COUNTERS 16
/* counters of ck_txn_stats, summed over trials since the last create/reset */
#define CK_TXS_COMMITS 0
#define CK_TXS_ATTEMPTS 1
#define CK_TXS_ABORT_CLAIMED 2   /* an overwrite/delete or a planned slot met another's claim */
#define CK_TXS_ABORT_LOCK 3      /* a lock not obtained within the bound */
#define CK_TXS_ABORT_WS 4        /* a write-set version moved */
#define CK_TXS_ABORT_RS 5        /* a read-set version moved / a key appeared */
#define CK_TXS_ABORT_CHAIN 6     /* no eligible slot for an insert or chain step */
#define CK_TXS_ABORT_OVERFLOW 7  /* read set (512) or write set (1024) full */
#define CK_TXS_LOCAL_RETRIES 8
#define CK_TXS_FAILED 9
#define CK_TXS_MINI_TXNS 10      /* chain moves done as small transactions (CK_TXF_SYSTEM) */
#define CK_TXS_MINI_ABORTS 11
#define CK_TXS_KICKS 12

typedef struct ck_txn_table ck_txn_table;

/* `trials` empty tables of `bins` bins x `slots_per_bin` (4 or 8) slots
 * each; trials * bins * slots_per_bin < 2^31.  Device memory: 16 bytes per
 * slot and 12 per bin, plus 81,920 bytes of transaction scratch per worker
 * at the first ck_txn_run.  Synchronous. */
int ck_txn_create(ck_txn_table **out, uint64_t bins, uint32_t slots_per_bin, uint32_t trials, uint64_t seed);

/* Empty every trial's table and zero the counters.  Synchronous. */
int ck_txn_reset(ck_txn_table *x);

/* Run n_workers workers on every trial: worker w runs transactions
 * w*T .. w*T + T - 1 (T = txns_per_worker) in order; transaction i is
 * operations i*L .. i*L + L - 1 (L = ops_per_txn <= CK_TXN_MAX_OPS) of the
 * device arrays d_op, d_key, d_val (n_workers*T*L entries, shared by all
 * trials; keys != 0xFFFFFFFF).  Outputs, all device memory and each
 * optional (NULL: not written): d_status, d_value per operation and trial
 * (trials*n_workers*T*L, trial-major); per transaction and trial
 * (trials*n_workers*T): d_attempts (attempts made), d_tid (the committed
 * transaction ID; per worker strictly increasing) and d_order (its position
 * among its trial's commits; all ~0 for a transaction given up).  Flags:
 * CK_TXF_*.  Asynchronous on `stream`. */
int ck_txn_run(ck_txn_table *x, uint32_t flags, const uint8_t *d_op, const uint32_t *d_key,
               const uint32_t *d_val, uint32_t n_workers, uint32_t txns_per_worker, uint32_t ops_per_txn,
               uint8_t *d_status, uint32_t *d_value, uint32_t *d_attempts, uint64_t *d_tid, uint64_t *d_order,
               void *stream);

/* The first n (<= CK_TXN_COUNTERS) counters into host memory.  Synchronous. */
int ck_txn_stats(ck_txn_table *x, uint64_t *h_counters, uint32_t n);

/* Trial `trial`'s slots (bins*slots_per_bin packed records) into host
 * memory.  Synchronous. */
int ck_txn_export(ck_txn_table *x, uint32_t trial, uint64_t *h_slots);

void ck_txn_destroy(ck_txn_table *x);

/* Testing aid (not an operation of the paper): set, then clear, claim
 * flags of one bin directly (bits 0..B-1; bit 0 for single-slot bins).  A
 * set flag stands in for an insertion that claimed the slot and never
 * released it -- a writer that died mid-chain.  Every wait on a claim is
 * bounded, so such a flag turns into per-key statuses, not a hang:
 * insertions that need the slot end CK_ST_ABORTED after their claim
 * retries, deletes of a key in it report 2, lookups are unaffected.
 * Synchronous; call with no work on the table in flight.  CK_EINVAL for a
 * bin out of range or a mask beyond the claim bits. */
int ck_debug_claims(ck_table *t, uint64_t bin, uint32_t set_mask, uint32_t clear_mask);

/* Measurement helper (not an operation of the paper): n_reads independent
 * random reads of `width` bytes (8, 32 or 64: one single-slot, 4-slot or
 * 8-slot bin) from a device buffer of `bytes` bytes (64-byte aligned), the
 * access pattern of lookups and insertions.  Timing it gives the measured
 * random-gather roofline the table kernels are reported against.  d_sink:
 * 8 KB of device memory the kernel may write.  Asynchronous. */
int ck_gather_probe(const void *d_buf, size_t bytes, uint32_t width, uint64_t n_reads,
                    uint64_t seed, void *d_sink, void *stream);

/* The same reads with the launch shape given, for finding the fastest one
 * (the roofline is the best the memory system gives this pattern):
 * per_thread independent reads in flight per thread (1, 2, 4 or 8), `block`
 * threads per block (a multiple of 32, at most 1024), at most `max_blocks`
 * blocks striding over the reads (0: as many blocks as it takes for one
 * pass).  ck_gather_probe is per_thread 8, block 256, max_blocks 152 * 64.
 * CK_EINVAL for any other value, and for a block larger than the probe
 * kernel of that width and per_thread can run (64-byte reads, 8 in flight:
 * at most 256 threads); asynchronous. */
int ck_gather_probe_ex(const void *d_buf, size_t bytes, uint32_t width, uint64_t n_reads, uint64_t seed,
                       uint32_t per_thread, uint32_t block, uint32_t max_blocks, void *d_sink, void *stream);

/* Measurement helper (not an operation of the paper): n_ops independent
 * random atomics over a device buffer of `bytes` bytes (64-byte aligned),
 * the read-modify-writes insertions issue.  kind 0: a 32-bit add with no
 * result (red; a metadata update); 1: a 32-bit add whose result is used
 * (a claim-style round trip); 2: a 64-bit compare-and-swap whose result is
 * used (a slot write).  The buffer's contents change.  d_sink: 8 KB of
 * device memory the kernel may write.  Asynchronous. */
int ck_atomic_probe(void *d_buf, size_t bytes, uint32_t kind, uint64_t n_ops, uint64_t seed,
                    void *d_sink, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CK_H */
