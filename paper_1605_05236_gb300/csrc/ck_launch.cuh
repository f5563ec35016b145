// ck_launch.cuh -- host-side launch of the insert kernel, shared by the
// translation units that instantiate it (ck_insert_b1.cu, ck_insert_b4.cu,
// ck_insert_b8.cu: one bin size each, so they compile in parallel).
#pragma once
#include <cuda_runtime.h>

#include "ck.h"
#include "ck_kernels.cuh"
#include "ck_warp.cuh"

namespace ck {

// The host-side parameters of one insert launch (a table handle's fields).
struct InsertLaunch {
  const DevTable* dt;
  uint32_t block;
  int sm_count;
  bool overlap;          // the launch may start while its predecessor finishes
  uint64_t load_base;    // keys already in the table (the bins-viewed histogram's load)
  uint64_t max_threads;  // insertions in flight at most
};

using InsertFn = cudaError_t (*)(const InsertLaunch& l, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                                 uint8_t* st, uint32_t* viewed, bool serial, uint32_t upsert, cudaStream_t s);

// The launch function for a policy, or nullptr (one definition per bin size).
InsertFn pick_insert_b1(uint32_t policy);
InsertFn pick_insert_b4(uint32_t policy, bool ghost);
InsertFn pick_insert_b8(uint32_t policy, bool ghost);
InsertFn pick_insert_warp_b4();  // BFS by a warp per search (CK_PARAM_SEARCH_WARP)
InsertFn pick_insert_warp_b8();

template <int B, int POL, bool GHOST>
cudaError_t launch_insert(const InsertLaunch& l, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                          uint8_t* st, uint32_t* viewed, bool serial, uint32_t upsert, cudaStream_t s) {
  const DevTable& dt = *l.dt;
  const uint64_t load_base = l.load_base;
  if (serial) {
    k_insert<B, POL, GHOST, true><<<1, 1, 0, s>>>(dt, keys, vals, n, st, viewed, load_base, upsert);
    return cudaGetLastError();
  }
  const uint32_t block = l.block;
  // persistent launch: at most the blocks that fit on the GPU at once
  static int cached_block = 0, cached_per_sm = 0;
  if (cached_block != (int)block) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_insert<B, POL, GHOST, false>, block, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    cached_per_sm = per_sm;
    cached_block = (int)block;
  }
  uint64_t grid = (n + block - 1) / block;
  uint64_t resident = (uint64_t)cached_per_sm * l.sm_count;
  // Walks whose launches overlap leave part of the GPU to the next launch:
  // its blocks start while this launch's longest walks finish.  Measured
  // (whole fills, one GB300): two-choice queue-kicking 10.18 ms against
  // 10.45-10.50 with every block resident (2^24 x 4 to 0.95) and 12.4
  // against 14.1-14.3 (2^23 x 8 to 0.99), random kicking 22.8 against 24.5
  // and 34.4 against 38.3; 3-ary random kicking 204.5 against 207.9 (2^26
  // bins to 0.90); rattle-kicking keeps 0.8 of the blocks, 51.6 against
  // 58.4 (4-ary to 0.96).  Searches, which need every thread they can get,
  // are slower that way (BFS 22.5 against 20.8) and keep the full grid.  A
  // limit the caller sets (CK_PARAM_MAX_INFLIGHT) replaces this one.
  constexpr uint64_t tenths = (POL == P_QUEUE || POL == P_RANDOM) ? 9 : POL == P_RATTLE ? 8 : 10;
  if (tenths < 10 && l.overlap && l.max_threads == ~0ull) {
    const uint64_t most = resident * tenths / 10;
    resident = most > 0 ? most : 1;
  }
  if (grid > resident) grid = resident;
  uint64_t by_threads = l.max_threads / block;  // insertions in flight at once
  if (grid > by_threads) grid = by_threads > 0 ? by_threads : 1;
  if (dt.scratch) {
    uint64_t cap_blocks = (dt.n_searchers / SLAB) / ((block + SLAB - 1) / SLAB);
    if (grid > cap_blocks) grid = cap_blocks;
  }
  if (grid > 0x7FFFFFFFull) grid = 0x7FFFFFFFull;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = l.overlap ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_insert<B, POL, GHOST, false>, dt, keys, vals, n, st, viewed, load_base, upsert);
}

// The warp-search form of BFS (two-choice, no ghosts, concurrent only).
template <int B>
cudaError_t launch_insert_warp(const InsertLaunch& l, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                               uint8_t* st, uint32_t* viewed, bool, uint32_t, cudaStream_t s) {
  const DevTable& dt = *l.dt;
  static int cached_per_sm = 0;
  if (cached_per_sm == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_insert_warp<B>, WARP_BLOCK, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    cached_per_sm = per_sm;
  }
  uint64_t grid = (n + WARP_BLOCK - 1) / WARP_BLOCK;
  const uint64_t resident = (uint64_t)cached_per_sm * l.sm_count;
  if (grid > resident) grid = resident;
  const uint64_t by_threads = l.max_threads / WARP_BLOCK;
  if (grid > by_threads) grid = by_threads > 0 ? by_threads : 1;
  const uint64_t cap_blocks = (dt.n_searchers / SLAB) / ((WARP_BLOCK + SLAB - 1) / SLAB);
  if (grid > cap_blocks) grid = cap_blocks;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(WARP_BLOCK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = l.overlap ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_insert_warp<B>, dt, keys, vals, n, st, viewed, l.load_base);
}

// The two-choice policies for one bin size.
template <int B>
InsertFn pick_two_choice(uint32_t pol, bool ghost) {
  switch (pol) {
    case CK_RANDOM: return ghost ? launch_insert<B, P_RANDOM, true> : launch_insert<B, P_RANDOM, false>;
    case CK_BFS: return ghost ? launch_insert<B, P_BFS, true> : launch_insert<B, P_BFS, false>;
    case CK_SORTED: return ghost ? launch_insert<B, P_SORTED, true> : launch_insert<B, P_SORTED, false>;
    case CK_HYBRID: return ghost ? launch_insert<B, P_HYBRID, true> : launch_insert<B, P_HYBRID, false>;
    case CK_QUEUE: return ghost ? launch_insert<B, P_QUEUE, true> : launch_insert<B, P_QUEUE, false>;
    default: return nullptr;
  }
}

}  // namespace ck
