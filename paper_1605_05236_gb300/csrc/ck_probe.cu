// ck_probe.cu -- random-access microbenchmarks: the measured rooflines for
// the table's access patterns over a buffer the size of the table.
// Gathers: independent random reads of one sector-sized record (8 B for a
// single-slot bin, 32 B for a 4-slot bin, 64 B for an 8-slot bin).
// Atomics: independent random read-modify-writes of the kinds insertions
// issue (a fire-and-forget 32-bit add on a metadata word, a returning
// 32-bit add, a returning 64-bit compare-and-swap on a slot).
#include <cuda_runtime.h>

#include <cstdint>

#include "ck.h"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// U independent random reads in flight per thread, each of one W-byte
// record (8, 32 or 64 bytes).  A grid of gridDim.x blocks strides over the
// reads; a grid that covers every read once makes each thread do one pass.
template <int W, int U>
__global__ void k_gather(const uint64_t* __restrict__ buf, uint64_t n_records, uint64_t mask, uint64_t n_reads,
                         uint64_t seed, uint64_t* __restrict__ sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t acc = 0;
  for (uint64_t i = tid * U; i < n_reads; i += stride * U) {  // U consecutive indices per thread
    uint64_t v[U][W / 8];
#pragma unroll
    for (int u = 0; u < U; u++) {
      uint64_t h = mix64(seed ^ (i + u));
      uint64_t r = mask ? (h & mask) : h % n_records;
      const uint64_t* p = buf + r * (W / 8);
      if (i + u < n_reads) {
        if constexpr (W == 8) {
          asm volatile("ld.global.nc.u64 %0, [%1];" : "=l"(v[u][0]) : "l"(p));
        } else {
#pragma unroll
          for (int q = 0; q < W / 8; q += 4)
            asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(v[u][q]), "=l"(v[u][q + 1]), "=l"(v[u][q + 2]), "=l"(v[u][q + 3])
                         : "l"(p + q));
        }
      } else {
#pragma unroll
        for (int q = 0; q < W / 8; q++) v[u][q] = 0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
      for (int q = 0; q < W / 8; q++) acc ^= v[u][q];
  }
  if (acc == 0x0123456789ABCDEFull) sink[tid & 1023] = acc;  // keeps the loads live
}

// The probe kernel for a width and reads in flight per thread.
template <int W>
using GatherKernel = void (*)(const uint64_t*, uint64_t, uint64_t, uint64_t, uint64_t, uint64_t*);

template <int W>
GatherKernel<W> gather_kernel(uint32_t per_thread) {
  switch (per_thread) {
    case 1: return k_gather<W, 1>;
    case 2: return k_gather<W, 2>;
    case 4: return k_gather<W, 4>;
    default: return k_gather<W, 8>;
  }
}

// CK_EINVAL when the block is larger than the kernel can run with (its
// registers: 64-byte reads, 8 in flight, take 140 a thread, so 512-thread
// blocks do not fit); else the launch's result.
template <int W>
int launch_gather(uint32_t per_thread, unsigned grid, unsigned block, cudaStream_t s, const uint64_t* b,
                  uint64_t n_records, uint64_t mask, uint64_t n_reads, uint64_t seed, uint64_t* k) {
  const GatherKernel<W> fn = gather_kernel<W>(per_thread);
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) return CK_ECUDA;
  if ((int)block > a.maxThreadsPerBlock) return CK_EINVAL;
  fn<<<grid, block, 0, s>>>(b, n_records, mask, n_reads, seed, k);
  return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

// KIND 0: red.add.u32 (no result), 1: atom.add.u32 (result used),
// 2: atom.cas.b64 against 0 on an all-ones-free buffer (result used).
template <int KIND>
__global__ void __launch_bounds__(256) k_atomic(uint64_t* __restrict__ buf, uint64_t n_words, uint64_t mask,
                                                uint64_t n_ops, uint64_t seed, uint64_t* __restrict__ sink) {
  constexpr int U = 8;  // independent operations in flight per thread
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t acc = 0;
  for (uint64_t i = tid * U; i < n_ops; i += stride * U) {
    uint64_t v[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      v[u] = 0;
      if (i + u >= n_ops) continue;
      const uint64_t h = mix64(seed ^ (i + u));
      const uint64_t r = mask ? (h & mask) : h % n_words;
      if constexpr (KIND == 0) {
        unsigned int* p = reinterpret_cast<unsigned int*>(buf) + r;
        asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
      } else if constexpr (KIND == 1) {
        unsigned int* p = reinterpret_cast<unsigned int*>(buf) + r;
        v[u] = atomicAdd(p, 1u);
      } else {
        v[u] = atomicCAS(reinterpret_cast<unsigned long long*>(buf) + r, 0ull, 1ull);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) acc ^= v[u];
  }
  if (acc == 0x0123456789ABCDEFull) sink[tid & 1023] = acc;  // keeps the results live
}

}  // namespace

extern "C" int ck_atomic_probe(void* d_buf, size_t bytes, uint32_t kind, uint64_t n_ops, uint64_t seed,
                               void* d_sink, void* stream) {
  if (!d_buf || !d_sink || kind > 2) return CK_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_buf) % 64) != 0 || bytes < 64) return CK_EINVAL;
  const uint64_t word = kind == 2 ? 8 : 4;
  const uint64_t n_words = bytes / word;
  const uint64_t mask = (n_words & (n_words - 1)) == 0 ? n_words - 1 : 0;
  uint64_t grid = ((n_ops + 7) / 8 + 255) / 256;
  if (grid > 152ull * 64) grid = 152ull * 64;
  if (grid == 0) grid = 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint64_t* b = static_cast<uint64_t*>(d_buf);
  uint64_t* k = static_cast<uint64_t*>(d_sink);
  if (kind == 0) k_atomic<0><<<(unsigned)grid, 256, 0, s>>>(b, n_words, mask, n_ops, seed, k);
  else if (kind == 1) k_atomic<1><<<(unsigned)grid, 256, 0, s>>>(b, n_words, mask, n_ops, seed, k);
  else k_atomic<2><<<(unsigned)grid, 256, 0, s>>>(b, n_words, mask, n_ops, seed, k);
  return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

extern "C" int ck_gather_probe_ex(const void* d_buf, size_t bytes, uint32_t width, uint64_t n_reads, uint64_t seed,
                                  uint32_t per_thread, uint32_t block, uint32_t max_blocks, void* d_sink,
                                  void* stream) {
  if (!d_buf || !d_sink || (width != 8 && width != 32 && width != 64)) return CK_EINVAL;
  if (per_thread != 1 && per_thread != 2 && per_thread != 4 && per_thread != 8) return CK_EINVAL;
  if (block < 32 || block > 1024 || (block % 32) != 0) return CK_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_buf) % 64) != 0 || bytes < 64) return CK_EINVAL;
  uint64_t n_records = bytes / width;
  uint64_t mask = (n_records & (n_records - 1)) == 0 ? n_records - 1 : 0;
  uint64_t threads = (n_reads + per_thread - 1) / per_thread;
  uint64_t grid = (threads + block - 1) / block;
  if (max_blocks && grid > max_blocks) grid = max_blocks;  // grid-stride beyond max_blocks
  if (grid > 0x7FFFFFFFull) grid = 0x7FFFFFFFull;
  if (grid == 0) grid = 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t* b = static_cast<const uint64_t*>(d_buf);
  uint64_t* k = static_cast<uint64_t*>(d_sink);
  if (width == 8) return launch_gather<8>(per_thread, (unsigned)grid, block, s, b, n_records, mask, n_reads, seed, k);
  if (width == 32) return launch_gather<32>(per_thread, (unsigned)grid, block, s, b, n_records, mask, n_reads, seed, k);
  return launch_gather<64>(per_thread, (unsigned)grid, block, s, b, n_records, mask, n_reads, seed, k);
}

extern "C" int ck_gather_probe(const void* d_buf, size_t bytes, uint32_t width, uint64_t n_reads,
                               uint64_t seed, void* d_sink, void* stream) {
  // 8 reads in flight per thread, 256-thread blocks, at most 64 blocks per SM of 152
  return ck_gather_probe_ex(d_buf, bytes, width, n_reads, seed, 8, 256, 152u * 64u, d_sink, stream);
}
