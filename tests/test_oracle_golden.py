"""Hand-worked fixtures (tests/golden/*.txt) pin the oracle's policies step
by step: each fixture cites the paper section whose definition it works
through, gives every key's bins explicitly and states the expected status,
bins viewed, kick-outs and final table state.

Policies that draw random numbers state the draws a step uses as premises
(`draw key=K i=I mod M = R`: draw I of key K's insertion, reduced mod M, is
R).  Each premise is checked against SplitMix64, the generator the draws
come from (pinned to its published outputs in test_oracle_hash.py), so the
hand-worked steps rest on the stated residues alone."""
import glob
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
POLICIES = {"RANDOM": oracle.RANDOM, "BFS": oracle.BFS, "SORTED": oracle.SORTED,
            "QUEUE": oracle.QUEUE, "RATTLE": oracle.RATTLE, "HYBRID": oracle.HYBRID, "GHOST": oracle.GHOST}
STATUS = {"OK": oracle.ST_OK, "FAILED": oracle.ST_FAILED}


def parse(path):
    table, steps, keybins = None, [], {}
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        head, rest = line.split(None, 1)
        if head == "table":
            kv = dict(x.split("=") for x in rest.split())
            pol = 0
            for p in kv["policy"].split("|"):
                pol |= POLICIES[p]
            table = dict(bins=int(kv["bins"]), B=int(kv["B"]), d=int(kv["d"]), policy=pol,
                         cap=int(kv["cap"]), spawn_k=int(kv.get("spawn_k", 1)),
                         tie_resident=kv.get("tie", "incoming") == "resident")
        elif head == "insert":
            lhs, rhs = rest.split("->")
            kv = dict(x.split("=") for x in lhs.split())
            key, val = int(kv["key"]), int(kv["val"])
            keybins[key] = [int(b) for b in kv["bins"].split(",")]
            r = rhs.split()
            exp = dict(x.split("=") for x in r[1:])
            steps.append(("insert", key, val, STATUS[r[0]], int(exp["viewed"]), int(exp["kicks"])))
        elif head == "draw":  # draw key=K i=I mod M = R: a premise about the draws
            kv = dict(x.split("=") for x in rest.split("mod")[0].split())
            mod, res = rest.split("mod")[1].split("=")
            steps.append(("draw", int(kv["key"]), int(kv["i"]), int(mod), int(res)))
        elif head == "set":  # set spawn <bin> = <count>: a starting state of the fixture
            what, rhs = rest.split("=")
            what = what.split()
            steps.append(("set", what, int(rhs)))
        elif head == "expect":
            what, rhs = rest.split("=")
            what = what.split()
            steps.append(("expect", what, rhs.strip()))
        else:
            raise ValueError(line)
    return table, steps, keybins


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))),
                         ids=lambda p: os.path.basename(p))
def test_golden(path):
    table, steps, keybins = parse(path)
    t = oracle.OracleTable(table["bins"], table["B"], table["d"], table["policy"], rng_seed=0,
                           cap=table["cap"])
    keys = sorted(keybins)
    t.set_bins(np.array(keys, dtype=np.uint32), np.array([keybins[k] for k in keys], dtype=np.uint64))
    t.set_spawn_k(table["spawn_k"])
    if table["tie_resident"]:
        t.set_rattle_tie_resident(True)
    for step in steps:
        if step[0] == "draw":
            # the fixture table's draw seed is 0: draw i of key k is the
            # SplitMix64 output for state k ^ (i << 32)
            _, key, i, mod, res = step
            assert oracle.lib().orc_splitmix64_at(key ^ (i << 32)) % mod == res, (path, step)
        elif step[0] == "insert":
            _, key, val, st, viewed, kicks = step
            s, v, k = t.insert([key], [val], trace=True)
            assert (int(s[0]), int(v[0]), int(k[0])) == (st, viewed, kicks), (path, key)
            assert t.check_invariants()[0] == 0, t.check_invariants()
        elif step[0] == "set":
            _, what, value = step
            assert what[0] == "spawn", what
            t.set_spawn(int(what[1]), value)
        else:
            _, what, rhs = step
            e = t.export()
            if what[0] == "rec":
                b = int(what[1])
                got = []
                for s in range(t.B):
                    r = int(e["rec"][b * t.B + s])
                    got.append("-" if r == 0xFFFFFFFFFFFFFFFF else str(r >> 32))
                    if r != 0xFFFFFFFFFFFFFFFF:
                        # the value travels with its key
                        assert (r & 0xFFFFFFFF) == (r >> 32) * 10
                assert ",".join(got) == rhs, (path, what)
            elif what[0] == "dup":
                b = int(what[1])
                got = ",".join(str(int(x)) for x in e["dup"][b * t.B:(b + 1) * t.B])
                assert got == rhs, (path, what)
            elif what[0] == "rattle":
                assert int(e["rattle"][int(what[1])]) == int(rhs), (path, what)
            elif what[0] in ("hit", "spawn"):
                assert int(e[what[0]][int(what[1])]) == int(rhs), (path, what)
            elif what[0] == "stat":
                assert t.stats()[what[1]] == int(rhs), (path, what)
            else:
                raise ValueError(what)
