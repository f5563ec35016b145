// ck_noalloc.cu -- ck_insert_batch_noalloc: insertion for callers that
// cannot allocate device memory while they run.
//
// Breadth-first and sorted search keep per-search state (the candidate
// groups and the visited set) in scratch memory.  The ordinary insert path
// takes that scratch from the table's own buffer, which ck_required_bytes
// sizes for ~10^5 concurrent searches.  Some callers cannot size or
// allocate such a buffer when they insert: services whose device memory
// budget is fixed up front, real-time sections where an allocation's
// latency is not acceptable, or libraries embedding this one that own no
// device allocator.  For them this variant takes the search scratch from a
// fixed array compiled into libck.so instead, and allocates nothing.  The
// first call on a device looks up the array's device address; that first
// call should come before any stream capture.
//
// The array: NOALLOC_REGIONS = 512 search regions of 16,528 bytes, 8.1 MiB in
// all, in device memory of every GPU that loads the library, held until the
// process exits.  One region per key, so a call takes at most 512 keys.
#include <cuda_runtime.h>

#include <mutex>

#include "ck.h"
#include "ck_kernels.cuh"

using namespace ck;

// the device view of a table handle, and the bookkeeping of an insert
// launch on it (defined in ck_lib.cu)
const ck::DevTable* ck_internal_devtable(const ck_table* t);
uint64_t ck_internal_load_base(const ck_table* t);
void ck_internal_note_insert(ck_table* t, void* stream, uint64_t n);

namespace {

constexpr int NOALLOC_REGIONS = CK_NOALLOC_MAX_KEYS;
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_REGIONS * SEARCH_REGION;

// One search region per key of a call.  Contents persist between calls;
// nothing in a region needs to start at zero: each search stamps its visited
// set with a new generation number (the region's first word), so entries
// left by earlier searches do not match, and the set is cleared whenever the
// 32-bit generation wraps; the group records are written before they are
// read.
static __device__ __align__(256) uint8_t g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the array on the current device, looked up once per
// device.  The host-side name g_noalloc_scratch is not a device address.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CK_ECUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return CK_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CK_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CK_OK;
}

// One thread per key; thread i searches in region i of the array.  Each
// insertion runs as in ck_insert_batch's concurrent mode (insert_one with
// failed walks retried), and the same counters and histograms are kept:
// bins viewed by load (load_base: keys the table held before the call) and
// kick-out chain lengths.
template <int B, int POL, bool GHOST>
__global__ void __launch_bounds__(128) k_insert_noalloc(DevTable t, uint8_t* scratch,
                                                        const uint32_t* __restrict__ keys,
                                                        const uint32_t* __restrict__ vals, uint64_t n,
                                                        uint8_t* __restrict__ status, uint64_t load_base) {
  __shared__ unsigned long long bc[C_N];
  for (int i = threadIdx.x; i < C_N; i += blockDim.x) bc[i] = 0;
  __syncthreads();
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    PlanStore<MAX_CHAIN> store;
    uint8_t* region = scratch + i * SEARCH_REGION;
    uint32_t key = keys[i];
    int st = ST_INVALID;
    Ctx c;
    c.viewed = 0;
    c.viewed0 = 0;
    c.reviews = 0;
    c.kicks = 0;
    c.ghosts_made = 0;
    c.dup_evict = 0;
    uint32_t aborts = 0;
    if (key != RESERVED_KEY) {
      c.key = key;
      c.krec = ((uint64_t)key << 32) | vals[i];
      st = insert_one<B, POL, GHOST>(t, c, region, aborts, store.e, MAX_CHAIN, true);
    }
    if (status) status[i] = (uint8_t)st;
    if (st != ST_INVALID) {
      const uint32_t v_final = c.viewed - c.viewed0;
      atomicAdd(&bc[st == ST_OK ? C_INS_OK : st == ST_FAILED ? C_INS_FAILED : C_INS_ABORTED], 1ull);
      atomicAdd(&bc[C_VIEWED], (unsigned long long)v_final);
      atomicAdd(&bc[C_VIEWED_ALL], (unsigned long long)c.viewed);
      if (aborts) atomicAdd(&bc[C_ABORTS], (unsigned long long)aborts);
      if (c.reviews) atomicAdd(&bc[C_REVIEWS], (unsigned long long)c.reviews);
      if (st == ST_OK) {
        atomicAdd(&bc[C_KICKS], (unsigned long long)c.kicks);
        atomicMax(&bc[C_CHAIN_MAX], (unsigned long long)c.kicks);
        if (c.ghosts_made) atomicAdd(&bc[C_GHOSTS_MADE], (unsigned long long)c.ghosts_made);
        if (c.dup_evict) atomicAdd(&bc[C_DUP_EVICT], (unsigned long long)c.dup_evict);
        atomicAdd(t.counters + CHAIN_HIST + chain_bucket(c.kicks), 1ull);
      }
      uint64_t bucket = ((load_base + i) * HIST_BUCKETS) / t.total_slots;
      if (bucket >= HIST_BUCKETS) bucket = HIST_BUCKETS - 1;
      atomicAdd(t.counters + C_N + bucket, (unsigned long long)v_final);
      atomicAdd(t.counters + C_N + HIST_BUCKETS + bucket, 1ull);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < C_N; k++) {
      if (!bc[k]) continue;
      if (k == C_CHAIN_MAX) atomicMax(t.counters + k, bc[k]);
      else atomicAdd(t.counters + k, bc[k]);
    }
    if (bc[C_INS_OK]) atomicAdd(t.counters + C_SIZE, bc[C_INS_OK]);
    long long dg = (long long)bc[C_GHOSTS_MADE] - (long long)bc[C_DUP_EVICT];
    if (dg) atomicAdd(t.counters + C_LIVE_GHOSTS, (unsigned long long)dg);
  }
}

template <int B, int POL, bool GHOST>
void launch(const DevTable& dt, uint8_t* scratch, const uint32_t* k, const uint32_t* v, uint64_t n,
            uint8_t* st, uint64_t lb, cudaStream_t s) {
  unsigned grid = (unsigned)((n + 127) / 128);
  k_insert_noalloc<B, POL, GHOST><<<grid, 128, 0, s>>>(dt, scratch, k, v, n, st, lb);
}

template <int B>
int dispatch2(const DevTable& dt, uint8_t* sp, const uint32_t* k, const uint32_t* v, uint64_t n, uint8_t* st,
              uint64_t lb, cudaStream_t s) {
  bool g = dt.ghost != 0;
  switch (dt.policy) {
    case CK_RANDOM: g ? launch<B, P_RANDOM, true>(dt, sp, k, v, n, st, lb, s) : launch<B, P_RANDOM, false>(dt, sp, k, v, n, st, lb, s); break;
    case CK_BFS: g ? launch<B, P_BFS, true>(dt, sp, k, v, n, st, lb, s) : launch<B, P_BFS, false>(dt, sp, k, v, n, st, lb, s); break;
    case CK_SORTED: g ? launch<B, P_SORTED, true>(dt, sp, k, v, n, st, lb, s) : launch<B, P_SORTED, false>(dt, sp, k, v, n, st, lb, s); break;
    case CK_HYBRID: g ? launch<B, P_HYBRID, true>(dt, sp, k, v, n, st, lb, s) : launch<B, P_HYBRID, false>(dt, sp, k, v, n, st, lb, s); break;
    case CK_QUEUE: g ? launch<B, P_QUEUE, true>(dt, sp, k, v, n, st, lb, s) : launch<B, P_QUEUE, false>(dt, sp, k, v, n, st, lb, s); break;
    default: return CK_ENOTSUP;
  }
  return CK_OK;
}

}  // namespace

extern "C" int ck_insert_batch_noalloc(ck_table* t, const uint32_t* d_keys, const uint32_t* d_vals, uint64_t n,
                                       uint8_t* d_status, void* stream) {
  if (!t) return CK_EINVAL;
  if (n > (uint64_t)CK_NOALLOC_MAX_KEYS) return CK_EINVAL;  // one scratch region per key
  if (n == 0) return CK_OK;
  if (!d_keys || !d_vals) return CK_EINVAL;
  void* sp = nullptr;
  int rc = scratch_address(&sp);
  if (rc != CK_OK) return rc;
  const DevTable& dt = *ck_internal_devtable(t);
  const uint64_t lb = ck_internal_load_base(t);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint8_t* scratch = static_cast<uint8_t*>(sp);
  if (dt.B == 4) rc = dispatch2<4>(dt, scratch, d_keys, d_vals, n, d_status, lb, s);
  else if (dt.B == 8) rc = dispatch2<8>(dt, scratch, d_keys, d_vals, n, d_status, lb, s);
  else if (dt.policy == CK_RATTLE) launch<1, P_RATTLE, false>(dt, scratch, d_keys, d_vals, n, d_status, lb, s);
  else if (dt.policy == CK_BFS) launch<1, P_BFS, false>(dt, scratch, d_keys, d_vals, n, d_status, lb, s);
  else if (dt.policy == CK_SORTED) launch<1, P_SORTED, false>(dt, scratch, d_keys, d_vals, n, d_status, lb, s);
  else if (dt.policy == CK_HYBRID) launch<1, P_HYBRID, false>(dt, scratch, d_keys, d_vals, n, d_status, lb, s);
  else launch<1, P_RANDOM, false>(dt, scratch, d_keys, d_vals, n, d_status, lb, s);
  if (rc != CK_OK) return rc;
  if (cudaGetLastError() != cudaSuccess) return CK_ECUDA;
  // the handle's readers (ck_stats, histograms, export) now wait for this stream
  ck_internal_note_insert(t, stream, n);
  return CK_OK;
}
