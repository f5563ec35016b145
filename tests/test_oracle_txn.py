"""The serial replay of transactional workloads (oracle/txn.py) against a
hand-worked example, and the workload generator's promises."""
import numpy as np

from oracle import txn
from paper_1605_05236_gb300 import inputs

I, R, O, D = txn.TX_INSERT, txn.TX_READ, txn.TX_OVERWRITE, txn.TX_DELETE


def test_replay_hand_worked():
    # two workers, two transactions of three operations each; worked by hand
    work = {"op": np.array([I, I, R,   O, R, D,   I, R, I,   D, R, O], dtype=np.uint8),
            "key": np.array([1, 2, 3,   1, 2, 2,   9, 1, 8,   9, 9, 8], dtype=np.uint32),
            "val": np.array([10, 20, 0, 11, 0, 0,  90, 0, 80,  0, 0, 81], dtype=np.uint32)}
    st, v, final = txn.replay(work)
    assert st.tolist() == [0, 0, 0,  1, 1, 1,  0, 1, 0,  1, 0, 1]
    assert v.tolist() == [0, 0, 0,  0, 20, 0,  0, 11, 0,  0, 0, 0]
    assert final == {1: 11, 8: 81}


def test_workload_keeps_keys_per_worker_and_targets_live_keys():
    W, T, L = 5, 40, 20
    work = inputs.txn_workload(W, T, L, (2, 1, 2, 2), seed=3)
    op, key = work["op"], work["key"]
    owner = {}
    for w in range(W):
        live = set()
        for t in range(T):
            base = (w * T + t) * L
            ks = key[base:base + L]
            assert len(set(ks.tolist())) == L  # a key at most once per transaction
            dead, born = [], []
            for j in range(L):
                k, o = int(ks[j]), int(op[base + j])
                if o == I:
                    assert k not in owner  # fresh
                    owner[k] = w
                    born.append(k)
                else:
                    assert owner[k] == w and k in live  # own, live, earlier transaction
                    if o == D:
                        dead.append(k)
            live -= set(dead)
            live |= set(born)
    st, _, _ = txn.replay(work)
    assert (st[op != I] == 1).all()  # every read / overwrite / delete finds its key
