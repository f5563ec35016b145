// ck_serve.cu -- the serving form: a request loop over one resident table
// that merges lookup/insert/delete requests of different sizes into device
// waves as they arrive (continuous batching), keeps several waves in flight
// on separate streams so their work overlaps on the GPU, admits inserts by
// the table's load, and timestamps every request for latency.
//
// Correctness under overlap rests on the table's own protocol: insertions
// and deletes claim every slot they write (Sec. 8 "Claim Flags") and apply
// chains back to front with release-ordered stores, and lookups here use a
// validated read: the metadata words of the key's bins are read before and
// after the slots, and a read that saw a claim or a change is repeated, so
// a lookup never reports a key absent that was present throughout.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ck.h"
#include "ck_kernels.cuh"

using namespace ck;

const ck::DevTable* ck_internal_devtable(const ck_table* t);
void* ck_internal_swap_last(ck_table* t, void* s);

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// ---------------------------------------------------------------------------
// validated lookups (safe while insertions and deletes run)
// ---------------------------------------------------------------------------

// found_out: 1 present, 0 absent, 2 not resolved within the retry bound.
// A hit is final at once (a slot holding the key is a real record of it);
// a miss only when unchanged_since proves no writer touched the bins.
constexpr int LOOKUP_ATTEMPTS = 1024;

template <int B>
__global__ void __launch_bounds__(256) k_lookup_validated(DevTable t, const uint32_t* __restrict__ keys,
                                                          uint64_t n, uint32_t* __restrict__ vals_out,
                                                          uint8_t* __restrict__ found_out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  constexpr uint32_t CLAIM_BITS = (1u << B) - 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t key = keys[i];
    uint32_t val = 0;
    int f = 0;
    if (key != RESERVED_KEY) {
      uint32_t b[4];
      uint32_t nb = B == 1 ? t.d : 2;
      if (B == 1) bins_of(t, key, b);
      else bins2(t, key, b[0], b[1]);
      f = 2;
      for (int attempt = 0; attempt < LOOKUP_ATTEMPTS && f == 2; attempt++) {
        uint32_t seen[4];
        bool hit = false;
        uint32_t v = 0;
        for (uint32_t j = 0; j < nb; j++) {
          View<B> vw;
          load_view<B>(t, b[j], vw);
          seen[j] = vw.m;
#pragma unroll
          for (int q = 0; q < B; q++)
            if (!hit && vw.s[q] != EMPTY && key_of(vw.s[q]) == key) { hit = true; v = (uint32_t)vw.s[q]; }
        }
        if (hit || unchanged_since(t.meta, b, seen, nb, CLAIM_BITS)) {
          f = hit ? 1 : 0;
          val = v;
        } else {
          uint32_t w = 64u << (attempt < 14 ? attempt : 14);
          __nanosleep(w + (fmix32(key ^ attempt) & (w - 1)));
        }
      }
    }
    if (vals_out) vals_out[i] = val;
    if (found_out) found_out[i] = (uint8_t)f;
  }
}

int launch_validated_lookup(const DevTable& dt, const uint32_t* keys, uint64_t n, uint32_t* vals, uint8_t* found,
                            cudaStream_t s) {
  if (n == 0) return CK_OK;
  uint64_t g = (n + 255) / 256;
  if (g > 0x7FFFFFFFull) g = 0x7FFFFFFFull;
  if (dt.B == 4) k_lookup_validated<4><<<(unsigned)g, 256, 0, s>>>(dt, keys, n, vals, found);
  else if (dt.B == 8) k_lookup_validated<8><<<(unsigned)g, 256, 0, s>>>(dt, keys, n, vals, found);
  else k_lookup_validated<1><<<(unsigned)g, 256, 0, s>>>(dt, keys, n, vals, found);
  return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

// ---------------------------------------------------------------------------
// the server
// ---------------------------------------------------------------------------

struct Request {
  uint32_t op;
  const uint32_t* keys;
  const uint32_t* vals;
  uint64_t n;
  uint32_t* vals_out;
  uint8_t* status_out;
  int64_t t_arrive;
  int64_t t_done;
  std::atomic<int> done;
};

constexpr int N_OPS = 3;  // CK_OP_LOOKUP, CK_OP_INSERT, CK_OP_DELETE

struct WaveSlot {
  // per op: device keys/vals/outputs, pinned host staging
  uint32_t* d_keys[N_OPS];
  uint32_t* d_vals[N_OPS];
  uint32_t* d_vout[N_OPS];
  uint8_t* d_st[N_OPS];
  uint32_t* h_keys[N_OPS];
  uint32_t* h_vals[N_OPS];
  uint32_t* h_vout[N_OPS];
  uint8_t* h_st[N_OPS];
  cudaEvent_t done[N_OPS];
  bool used[N_OPS];
  std::vector<Request*> reqs;
  std::vector<uint64_t> offs;  // offset of each request in its op's staging
  bool busy;
};

}  // namespace

struct ck_server {
  ck_table* table;
  DevTable dt;
  ck_server_config cfg;
  cudaStream_t streams[N_OPS];
  std::vector<WaveSlot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_slot, cv_done;
  std::deque<Request*> pending;
  std::deque<Request*> deferred;
  std::deque<int> inflight;  // wave slot indices in launch order
  std::atomic<bool> stop;
  std::thread scheduler, completer;
  int device;
  void* table_last;  // the table's own stream, handed back at destroy
  // load accounting (keys), updated at completion; inserts in flight are
  // counted when admitted so admission never overshoots
  int64_t live;
  int64_t admitted_inserts;
  uint64_t total_slots;
  uint64_t waves, busy_rejects;
  int error;
};

namespace {

void free_slots(ck_server* s) {
  for (auto& w : s->slots) {
    for (int o = 0; o < N_OPS; o++) {
      cudaFree(w.d_keys[o]);
      cudaFree(w.d_vals[o]);
      cudaFree(w.d_vout[o]);
      cudaFree(w.d_st[o]);
      cudaFreeHost(w.h_keys[o]);
      cudaFreeHost(w.h_vals[o]);
      cudaFreeHost(w.h_vout[o]);
      cudaFreeHost(w.h_st[o]);
      if (w.done[o]) cudaEventDestroy(w.done[o]);
    }
  }
  s->slots.clear();
}

void complete(Request* r, int64_t t) {
  r->t_done = t;
  r->done.store(1, std::memory_order_release);
}

// Launch one wave: every request in w.reqs, grouped by op.
int launch_wave(ck_server* s, WaveSlot& w) {
  uint64_t fill[N_OPS] = {0, 0, 0};
  w.offs.resize(w.reqs.size());
  for (size_t i = 0; i < w.reqs.size(); i++) {
    Request* r = w.reqs[i];
    w.offs[i] = fill[r->op];
    std::memcpy(w.h_keys[r->op] + fill[r->op], r->keys, r->n * sizeof(uint32_t));
    if (r->op == CK_OP_INSERT) std::memcpy(w.h_vals[r->op] + fill[r->op], r->vals, r->n * sizeof(uint32_t));
    fill[r->op] += r->n;
  }
  // deletes first, then inserts, then lookups: independent streams
  const int order[N_OPS] = {CK_OP_DELETE, CK_OP_INSERT, CK_OP_LOOKUP};
  for (int oi = 0; oi < N_OPS; oi++) {
    int o = order[oi];
    w.used[o] = fill[o] > 0;
    if (!w.used[o]) continue;
    cudaStream_t st = s->streams[o];
    uint64_t n = fill[o];
    if (cudaMemcpyAsync(w.d_keys[o], w.h_keys[o], n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) return CK_ECUDA;
    int rc = CK_OK;
    if (o == CK_OP_INSERT) {
      if (cudaMemcpyAsync(w.d_vals[o], w.h_vals[o], n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) return CK_ECUDA;
      rc = ck_insert_batch(s->table, w.d_keys[o], w.d_vals[o], n, w.d_st[o], st);
      if (rc == CK_OK && cudaMemcpyAsync(w.h_st[o], w.d_st[o], n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = CK_ECUDA;
    } else if (o == CK_OP_DELETE) {
      rc = ck_delete_batch(s->table, w.d_keys[o], n, w.d_st[o], st);
      if (rc == CK_OK && cudaMemcpyAsync(w.h_st[o], w.d_st[o], n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = CK_ECUDA;
    } else {
      rc = launch_validated_lookup(s->dt, w.d_keys[o], n, w.d_vout[o], w.d_st[o], st);
      if (rc == CK_OK && (cudaMemcpyAsync(w.h_vout[o], w.d_vout[o], n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                          cudaMemcpyAsync(w.h_st[o], w.d_st[o], n, cudaMemcpyDeviceToHost, st) != cudaSuccess))
        rc = CK_ECUDA;
    }
    if (rc != CK_OK) return rc;
    if (cudaEventRecord(w.done[o], st) != cudaSuccess) return CK_ECUDA;
  }
  return CK_OK;
}

void scheduler_loop(ck_server* s) {
  cudaSetDevice(s->device);
  const double hi = s->cfg.load_hi;
  for (;;) {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_work.wait(lk, [&] { return s->stop.load() || !s->pending.empty() || !s->deferred.empty(); });
    if (s->stop.load() && s->pending.empty() && s->deferred.empty()) return;
    // a free wave slot (continuous batching: never wait for a wave to finish
    // while another slot is free)
    int slot = -1;
    s->cv_slot.wait(lk, [&] {
      for (size_t i = 0; i < s->slots.size(); i++)
        if (!s->slots[i].busy) { slot = (int)i; return true; }
      return s->stop.load();
    });
    if (slot < 0) return;
    WaveSlot& w = s->slots[slot];
    w.reqs.clear();
    uint64_t fill[N_OPS] = {0, 0, 0};
    int64_t t = now_ns();
    // deferred inserts first (oldest first), then new arrivals in order
    std::deque<Request*> still;
    auto admit = [&](Request* r) -> bool {
      if (fill[r->op] + r->n > s->cfg.wave_keys) return false;  // next wave
      if (r->op == CK_OP_INSERT) {
        double load = (double)(s->live + s->admitted_inserts + (int64_t)r->n) / (double)s->total_slots;
        if (load > hi) {
          if ((uint64_t)(t - r->t_arrive) > s->cfg.max_defer_us * 1000ull) {
            if (r->status_out) std::memset(r->status_out, CK_ST_BUSY, r->n);
            s->busy_rejects++;
            complete(r, t);
            return true;
          }
          still.push_back(r);
          return true;
        }
        s->admitted_inserts += (int64_t)r->n;
      }
      w.reqs.push_back(r);
      fill[r->op] += r->n;
      return true;
    };
    while (!s->deferred.empty()) {
      Request* r = s->deferred.front();
      if (!admit(r)) break;
      s->deferred.pop_front();
    }
    while (!s->pending.empty()) {
      Request* r = s->pending.front();
      if (!admit(r)) break;
      s->pending.pop_front();
    }
    for (Request* r : still) s->deferred.push_back(r);
    if (w.reqs.empty()) {
      // only deferred inserts: wait for completions to change the load
      s->cv_done.wait_for(lk, std::chrono::microseconds(50));
      continue;
    }
    w.busy = true;
    s->waves++;
    lk.unlock();
    int rc = launch_wave(s, w);  // events recorded before the completer may look
    lk.lock();
    if (rc != CK_OK) s->error = rc;
    s->inflight.push_back(slot);
    s->cv_done.notify_all();
  }
}

void completer_loop(ck_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<int> ready;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_done.wait_for(lk, std::chrono::microseconds(20), [&] { return s->stop.load() || !s->inflight.empty(); });
      if (s->stop.load() && s->inflight.empty() && s->pending.empty() && s->deferred.empty()) return;
      for (auto it = s->inflight.begin(); it != s->inflight.end();) {
        WaveSlot& w = s->slots[*it];
        bool all = true;
        for (int o = 0; o < N_OPS && all; o++)
          if (w.used[o] && cudaEventQuery(w.done[o]) == cudaErrorNotReady) all = false;
        if (all) {
          ready.push_back(*it);
          it = s->inflight.erase(it);
        } else {
          ++it;
        }
      }
    }
    if (ready.empty()) continue;
    int64_t t = now_ns();
    int64_t d_live = 0, d_admitted = 0;
    for (int slot : ready) {
      WaveSlot& w = s->slots[slot];
      for (size_t i = 0; i < w.reqs.size(); i++) {
        Request* r = w.reqs[i];
        uint64_t off = w.offs[i];
        const uint8_t* st = w.h_st[r->op] + off;
        if (r->status_out) std::memcpy(r->status_out, st, r->n);
        if (r->op == CK_OP_LOOKUP && r->vals_out) std::memcpy(r->vals_out, w.h_vout[r->op] + off, r->n * 4);
        if (r->op == CK_OP_INSERT) {
          d_admitted -= (int64_t)r->n;
          for (uint64_t k = 0; k < r->n; k++) d_live += st[k] == CK_ST_OK;
        } else if (r->op == CK_OP_DELETE) {
          for (uint64_t k = 0; k < r->n; k++) d_live -= st[k] == 1;
        }
        complete(r, t);
      }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->live += d_live;
    s->admitted_inserts += d_admitted;
    for (int slot : ready) s->slots[slot].busy = false;
    s->cv_slot.notify_all();
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int ck_server_create(ck_server** out, ck_table* t, const ck_server_config* cfg_in) {
  if (!out || !t) return CK_EINVAL;
  *out = nullptr;
  ck_server_config cfg;
  cfg.wave_keys = 1ull << 20;
  cfg.wave_slots = 4;
  cfg.load_hi = 0.97;
  cfg.max_defer_us = 20000;
  cfg.hbm_fraction = 0.25;
  if (cfg_in) cfg = *cfg_in;
  if (cfg.wave_keys < 1024 || cfg.wave_slots < 1 || cfg.wave_slots > 64 || cfg.load_hi <= 0 || cfg.load_hi > 1)
    return CK_EINVAL;
  // admission by free HBM: the staging of all wave slots must fit in the
  // given fraction of the memory free now
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return CK_ECUDA;
  size_t per_slot = (size_t)cfg.wave_keys * N_OPS * (4 + 4 + 4 + 1);
  size_t budget = (size_t)(cfg.hbm_fraction * (double)free_b);
  if (per_slot * cfg.wave_slots > budget) {
    uint64_t fit = budget / per_slot;
    if (fit < 1) return CK_ENOMEM;
    cfg.wave_slots = (uint32_t)fit;
  }
  ck_server* s = new (std::nothrow) ck_server();
  if (!s) return CK_ENOMEM;
  s->table = t;
  s->dt = *ck_internal_devtable(t);
  s->cfg = cfg;
  s->stop = false;
  s->error = CK_OK;
  s->waves = s->busy_rejects = 0;
  s->admitted_inserts = 0;
  cudaGetDevice(&s->device);
  ck_stats_t st;
  int rc = ck_stats(t, &st);
  if (rc != CK_OK) {
    delete s;
    return rc;
  }
  s->live = (int64_t)st.size;
  s->table_last = ck_internal_swap_last(t, nullptr);
  ck_internal_swap_last(t, s->table_last);
  s->total_slots = st.total_slots;
  for (int o = 0; o < N_OPS; o++) cudaStreamCreateWithFlags(&s->streams[o], cudaStreamNonBlocking);
  s->slots.resize(cfg.wave_slots);
  bool ok = true;
  for (auto& w : s->slots) {
    w.busy = false;
    for (int o = 0; o < N_OPS; o++) {
      w.d_keys[o] = w.d_vals[o] = w.d_vout[o] = nullptr;
      w.d_st[o] = nullptr;
      w.h_keys[o] = w.h_vals[o] = w.h_vout[o] = nullptr;
      w.h_st[o] = nullptr;
      w.done[o] = nullptr;
      size_t n = cfg.wave_keys;
      ok &= cudaMalloc(&w.d_keys[o], n * 4) == cudaSuccess;
      ok &= cudaMalloc(&w.d_vals[o], n * 4) == cudaSuccess;
      ok &= cudaMalloc(&w.d_vout[o], n * 4) == cudaSuccess;
      ok &= cudaMalloc(&w.d_st[o], n) == cudaSuccess;
      ok &= cudaMallocHost(&w.h_keys[o], n * 4) == cudaSuccess;
      ok &= cudaMallocHost(&w.h_vals[o], n * 4) == cudaSuccess;
      ok &= cudaMallocHost(&w.h_vout[o], n * 4) == cudaSuccess;
      ok &= cudaMallocHost(&w.h_st[o], n) == cudaSuccess;
      ok &= cudaEventCreateWithFlags(&w.done[o], cudaEventDisableTiming) == cudaSuccess;
      w.used[o] = false;
    }
  }
  if (!ok) {
    free_slots(s);
    for (int o = 0; o < N_OPS; o++) cudaStreamDestroy(s->streams[o]);
    delete s;
    cudaGetLastError();
    return CK_ENOMEM;
  }
  s->scheduler = std::thread(scheduler_loop, s);
  s->completer = std::thread(completer_loop, s);
  *out = s;
  return CK_OK;
}

int ck_server_submit(ck_server* s, uint32_t op, const uint32_t* h_keys, const uint32_t* h_vals, uint64_t n,
                     uint32_t* h_vals_out, uint8_t* h_status_out, int64_t t_arrive_ns, void** ticket) {
  if (!s || !ticket || op >= N_OPS || (n && !h_keys) || (op == CK_OP_INSERT && n && !h_vals)) return CK_EINVAL;
  if (n > s->cfg.wave_keys) return CK_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return CK_ENOMEM;
  r->op = op;
  r->keys = h_keys;
  r->vals = h_vals;
  r->n = n;
  r->vals_out = h_vals_out;
  r->status_out = h_status_out;
  r->t_arrive = t_arrive_ns ? t_arrive_ns : now_ns();
  r->t_done = 0;
  r->done.store(0);
  *ticket = r;
  if (n == 0) {
    complete(r, now_ns());
    return CK_OK;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending.push_back(r);
  }
  s->cv_work.notify_one();
  return CK_OK;
}

// Wait for a request; on return *t_done_ns holds its completion time.  The
// ticket is freed.
int ck_server_wait(ck_server* s, void* ticket, int64_t* latency_ns) {
  if (!s || !ticket) return CK_EINVAL;
  Request* r = static_cast<Request*>(ticket);
  while (!r->done.load(std::memory_order_acquire)) {
    std::this_thread::sleep_for(std::chrono::microseconds(5));
    if (s->error != CK_OK) return s->error;
  }
  if (latency_ns) *latency_ns = r->t_done - r->t_arrive;
  delete r;
  return s->error;
}

int64_t ck_now_ns(void) { return now_ns(); }

int ck_server_replay(ck_server* s, uint64_t n_req, const uint32_t* op, const uint64_t* key_off, const uint64_t* n_keys,
                     const int64_t* arrive_ns, const uint32_t* keys, const uint32_t* vals, uint32_t* vals_out,
                     uint8_t* status_out, int64_t* latency_ns) {
  if (!s || !op || !key_off || !n_keys || !arrive_ns || !keys) return CK_EINVAL;
  std::vector<void*> tickets(n_req);
  int64_t t0 = now_ns();
  for (uint64_t i = 0; i < n_req; i++) {
    int64_t due = t0 + arrive_ns[i];
    while (now_ns() < due) {
    }
    int rc = ck_server_submit(s, op[i], keys + key_off[i], vals ? vals + key_off[i] : nullptr, n_keys[i],
                              vals_out ? vals_out + key_off[i] : nullptr, status_out ? status_out + key_off[i] : nullptr,
                              due, &tickets[i]);
    if (rc != CK_OK) return rc;
  }
  int err = CK_OK;
  for (uint64_t i = 0; i < n_req; i++) {
    int64_t lat = 0;
    int rc = ck_server_wait(s, tickets[i], &lat);
    if (rc != CK_OK) err = rc;
    if (latency_ns) latency_ns[i] = lat;
  }
  return err;
}

// The same trace as plain sequential bulk calls on one stream: request i
// starts when it has arrived and request i-1 has finished.
int ck_replay_sequential(ck_table* t, uint64_t n_req, const uint32_t* op, const uint64_t* key_off,
                         const uint64_t* n_keys, const int64_t* arrive_ns, const uint32_t* keys, const uint32_t* vals,
                         uint32_t* vals_out, uint8_t* status_out, int64_t* latency_ns, void* stream) {
  if (!t || !op || !key_off || !n_keys || !arrive_ns || !keys) return CK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint64_t maxn = 0;
  for (uint64_t i = 0; i < n_req; i++) maxn = n_keys[i] > maxn ? n_keys[i] : maxn;
  if (maxn == 0) return CK_OK;
  uint32_t *dk = nullptr, *dv = nullptr, *dvo = nullptr, *hk = nullptr, *hv = nullptr, *hvo = nullptr;
  uint8_t *ds = nullptr, *hs = nullptr;
  bool ok = cudaMalloc(&dk, maxn * 4) == cudaSuccess && cudaMalloc(&dv, maxn * 4) == cudaSuccess &&
            cudaMalloc(&dvo, maxn * 4) == cudaSuccess && cudaMalloc(&ds, maxn) == cudaSuccess &&
            cudaMallocHost(&hk, maxn * 4) == cudaSuccess && cudaMallocHost(&hv, maxn * 4) == cudaSuccess &&
            cudaMallocHost(&hvo, maxn * 4) == cudaSuccess && cudaMallocHost(&hs, maxn) == cudaSuccess;
  int rc = ok ? CK_OK : CK_ENOMEM;
  const DevTable dt = *ck_internal_devtable(t);
  int64_t t0 = now_ns();
  for (uint64_t i = 0; i < n_req && rc == CK_OK; i++) {
    int64_t due = t0 + arrive_ns[i];
    while (now_ns() < due) {
    }
    uint64_t n = n_keys[i], off = key_off[i];
    if (n) {
      std::memcpy(hk, keys + off, n * 4);
      cudaMemcpyAsync(dk, hk, n * 4, cudaMemcpyHostToDevice, st);
      if (op[i] == CK_OP_INSERT) {
        std::memcpy(hv, vals + off, n * 4);
        cudaMemcpyAsync(dv, hv, n * 4, cudaMemcpyHostToDevice, st);
        rc = ck_insert_batch(t, dk, dv, n, ds, st);
      } else if (op[i] == CK_OP_DELETE) {
        rc = ck_delete_batch(t, dk, n, ds, st);
      } else {
        rc = launch_validated_lookup(dt, dk, n, dvo, ds, st);
        cudaMemcpyAsync(hvo, dvo, n * 4, cudaMemcpyDeviceToHost, st);
      }
      cudaMemcpyAsync(hs, ds, n, cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) rc = CK_ECUDA;
      if (status_out) std::memcpy(status_out + off, hs, n);
      if (vals_out && op[i] == CK_OP_LOOKUP) std::memcpy(vals_out + off, hvo, n * 4);
    }
    if (latency_ns) latency_ns[i] = now_ns() - due;
  }
  cudaFree(dk);
  cudaFree(dv);
  cudaFree(dvo);
  cudaFree(ds);
  cudaFreeHost(hk);
  cudaFreeHost(hv);
  cudaFreeHost(hvo);
  cudaFreeHost(hs);
  return rc;
}

int ck_server_info(ck_server* s, uint64_t* waves, uint64_t* busy_rejects, double* load, uint32_t* wave_slots) {
  if (!s) return CK_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (waves) *waves = s->waves;
  if (busy_rejects) *busy_rejects = s->busy_rejects;
  if (load) *load = (double)s->live / (double)s->total_slots;
  if (wave_slots) *wave_slots = (uint32_t)s->slots.size();
  return s->error;
}

void ck_server_destroy(ck_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_slot.notify_all();
  s->cv_done.notify_all();
  if (s->scheduler.joinable()) s->scheduler.join();
  if (s->completer.joinable()) s->completer.join();
  for (int o = 0; o < N_OPS; o++) cudaStreamSynchronize(s->streams[o]);
  ck_internal_swap_last(s->table, s->table_last);
  free_slots(s);
  for (int o = 0; o < N_OPS; o++) cudaStreamDestroy(s->streams[o]);
  delete s;
}

}  // extern "C"
