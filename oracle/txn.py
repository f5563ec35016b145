"""Serial replay of a transactional workload (Sec. 8): the results every
transaction's operations must have in any serializable execution.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The workloads (inputs.txn_workload) give each worker keys of its own, so
transactions of different workers never touch the same key and every
serialization gives the same results; a worker's transactions take effect
in its own order.  The replay is the plain definition of the operations of
Sec. 1 on a key -> value map: an insert adds the key (status 0), a read
returns the value (status 1) or reports absence (status 0), an overwrite
replaces the value and a delete removes the key (status 1 if the key was
present, 0 if not)."""
from __future__ import annotations

import numpy as np

TX_INSERT, TX_READ, TX_OVERWRITE, TX_DELETE = 0, 1, 2, 3


def replay(work):
    """Returns (status uint8[n], value uint32[n], final dict key -> value)."""
    op, key, val = work["op"], work["key"], work["val"]
    n = len(op)
    status = np.zeros(n, dtype=np.uint8)
    value = np.zeros(n, dtype=np.uint32)
    table = {}
    # worker-major order: a worker's transactions in order, workers one after another
    for i in range(n):
        k, v, o = int(key[i]), int(val[i]), int(op[i])
        if o == TX_INSERT:
            table[k] = v
            status[i] = 0
        elif o == TX_READ:
            if k in table:
                status[i], value[i] = 1, table[k]
        elif o == TX_OVERWRITE:
            if k in table:
                table[k] = v
                status[i] = 1
        elif o == TX_DELETE:
            if k in table:
                del table[k]
                status[i] = 1
        else:
            raise ValueError("unknown operation %d" % o)
    return status, value, table
