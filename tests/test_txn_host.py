"""Host-side logic of the transactional layer's binding: the lifetime abort
count by table density (the x axis of Sec. 8's figures), on a hand-worked
example.  No GPU."""
import numpy as np

from paper_1605_05236_gb300 import txn

I, R, O, D = txn.TX_INSERT, txn.TX_READ, txn.TX_OVERWRITE, txn.TX_DELETE


def test_aborts_by_density_hand_worked():
    # four transactions of two operations; net inserts +2, +1, -1 (one delete hits), +2
    op = np.array([I, I,  I, R,  D, D,  I, I], dtype=np.uint8)
    st = np.array([0, 0,  0, 1,  1, 0,  0, 0], dtype=np.uint8)
    attempts = np.array([1, 3, 2, 1], dtype=np.int32)
    # committed in the order 1, 0, 3, 2: sizes after each 1, 3, 5, 4
    order = np.array([1, 0, 3, 2], dtype=np.int64)
    ab, att = txn.aborts_by_density(st, op, attempts, order, 2, 10, [0.1, 0.3, 0.5, 0.6])
    assert ab.tolist() == [2, 2, 2, -1]     # txn 1 (2 aborts) reaches size 1; txn 3 reaches 5; 6 never
    assert att.tolist() == [3, 4, 5, -1]


def test_aborts_by_density_skips_given_up_transactions():
    op = np.array([I, I, I, I], dtype=np.uint8)
    st = np.array([0, 0, 255, 255], dtype=np.uint8)
    attempts = np.array([4, 9], dtype=np.int32)
    order = np.array([0, -1], dtype=np.int64)
    ab, att = txn.aborts_by_density(st, op, attempts, order, 2, 4, [0.5, 1.0])
    assert ab.tolist() == [3, -1] and att.tolist() == [4, -1]
