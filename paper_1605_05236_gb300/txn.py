"""Binding of the transactional layer (ck_txn_* in include/ck.h; Sec. 8):
transactions of inserts, reads, overwrites and deletes under the paper's
optimistic concurrency scheme, with its abort-reducing mechanisms as flags.
Argument marshalling only: every step runs in the CUDA library."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import ck

TX_INSERT, TX_READ, TX_OVERWRITE, TX_DELETE = 0, 1, 2, 3
LOCAL_RETRY, QUEUE, SYSTEM, CLAIM = 1, 2, 4, 8
MAX_OPS = 256
N_COUNTERS = 16
ST_GIVEN_UP = 255

COUNTER_NAMES = ("commits", "attempts", "abort_claimed", "abort_lock", "abort_ws", "abort_rs", "abort_chain",
                 "abort_overflow", "local_retries", "failed", "mini_txns", "mini_aborts", "kicks")

# The six implementations compared in Sec. 8's experiments, in the paper's order.
VARIANTS = (
    ("naive", 0),
    ("local_retries", LOCAL_RETRY),
    ("queue", LOCAL_RETRY | QUEUE),
    ("queue_system", LOCAL_RETRY | QUEUE | SYSTEM),
    ("claim", LOCAL_RETRY | CLAIM),
    ("claim_system", LOCAL_RETRY | CLAIM | SYSTEM),
)

_bound = False


def _lib():
    global _bound
    L = ck.load()
    if not _bound:
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        L.ck_txn_create.argtypes = [ctypes.POINTER(vp), u64, u32, u32, u64]
        L.ck_txn_reset.argtypes = [vp]
        L.ck_txn_run.argtypes = [vp, u32, vp, vp, vp, u32, u32, u32, vp, vp, vp, vp, vp, vp]
        L.ck_txn_stats.argtypes = [vp, vp, u32]
        L.ck_txn_export.argtypes = [vp, u32, vp]
        L.ck_txn_destroy.argtypes = [vp]
        L.ck_txn_destroy.restype = None
        _bound = True
    return L


class TxnTable:
    """`trials` independent transactional tables of `bins` x `slots_per_bin`."""

    def __init__(self, bins: int, slots_per_bin: int = 8, trials: int = 1, seed: int = 1):
        L = _lib()
        h = ctypes.c_void_p()
        ck._check(L.ck_txn_create(ctypes.byref(h), bins, slots_per_bin, trials, seed), "ck_txn_create")
        self._h = h
        self.bins, self.B, self.trials = bins, slots_per_bin, trials

    def close(self):
        if getattr(self, "_h", None):
            _lib().ck_txn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        ck._check(_lib().ck_txn_reset(self._h), "ck_txn_reset")

    def run(self, op: torch.Tensor, key: torch.Tensor, val: torch.Tensor, n_workers: int, txns_per_worker: int,
            ops_per_txn: int, flags: int = 0, want_values=True, want_status=True, stream=None):
        """Runs the workload on every trial (asynchronously on `stream`).
        Returns dict of device tensors: status (uint8) and value (int32 bit
        patterns), per trial and operation; attempts (int32), tid and order
        (int64 bit patterns) per trial and transaction."""
        n = n_workers * txns_per_worker * ops_per_txn
        if op.numel() != n or key.numel() != n or val.numel() != n:
            raise ValueError("operation arrays must hold n_workers * txns_per_worker * ops_per_txn entries")
        if op.dtype != torch.uint8:
            raise ValueError("op must be uint8")
        dev = op.device
        nt = n_workers * txns_per_worker
        out = {
            "status": torch.empty(self.trials * n, dtype=torch.uint8, device=dev) if want_status else None,
            "value": torch.empty(self.trials * n, dtype=torch.int32, device=dev) if want_values else None,
            "attempts": torch.empty(self.trials * nt, dtype=torch.int32, device=dev),
            "tid": torch.empty(self.trials * nt, dtype=torch.int64, device=dev),
            "order": torch.empty(self.trials * nt, dtype=torch.int64, device=dev),
        }
        rc = _lib().ck_txn_run(self._h, flags, ck._ptr(op), ck._ptr(ck._u32_view(key)), ck._ptr(ck._u32_view(val)),
                               n_workers, txns_per_worker, ops_per_txn, ck._ptr(out["status"]),
                               ck._ptr(out["value"]), ck._ptr(out["attempts"]), ck._ptr(out["tid"]),
                               ck._ptr(out["order"]), ck._stream(stream))
        ck._check(rc, "ck_txn_run")
        return out

    def stats(self) -> dict:
        c = np.zeros(N_COUNTERS, dtype=np.uint64)
        ck._check(_lib().ck_txn_stats(self._h, ctypes.c_void_p(c.ctypes.data), N_COUNTERS), "ck_txn_stats")
        return {name: int(c[i]) for i, name in enumerate(COUNTER_NAMES)}

    def export(self, trial: int = 0) -> np.ndarray:
        s = np.zeros(self.bins * self.B, dtype=np.uint64)
        ck._check(_lib().ck_txn_export(self._h, trial, ctypes.c_void_p(s.ctypes.data)), "ck_txn_export")
        return s


def aborts_by_density(status: np.ndarray, op: np.ndarray, attempts: np.ndarray, order: np.ndarray,
                      ops_per_txn: int, capacity: int, densities):
    """Aborts and attempts over a table's lifetime up to each density
    (Sec. 8's figures): commits are taken in their commit order, the table's
    size after each is the running sum of the transactions' net inserts
    (inserts that added a record, less deletes that removed one, from the
    statuses), and the aborts (attempts) counted up to density q are those
    of the transactions committed before the size first reached
    q * capacity (-1 where it never did).  One trial's arrays; returns
    (aborts, attempts) as int64 arrays over `densities`."""
    st = status.reshape(-1, ops_per_txn)
    o = op.reshape(-1, ops_per_txn)
    delta = ((o == TX_INSERT) & (st == 0)).sum(1).astype(np.int64) - ((o == TX_DELETE) & (st == 1)).sum(1)
    ok = order >= 0
    idx = np.argsort(np.where(ok, order, np.iinfo(np.int64).max), kind="stable")[: int(ok.sum())]
    size = np.cumsum(delta[idx])
    att = np.cumsum(attempts[idx].astype(np.int64))
    ab = att - np.arange(1, len(idx) + 1)
    aborts, attempts_to = [], []
    for q in densities:
        hit = np.nonzero(size >= q * capacity)[0]
        aborts.append(ab[hit[0]] if len(hit) else -1)
        attempts_to.append(att[hit[0]] if len(hit) else -1)
    return np.array(aborts, dtype=np.int64), np.array(attempts_to, dtype=np.int64)
