"""Reader and runner for the hand-derived worked examples in tests/golden/.

A fixture is a list of lines `op args -> expectations`.  `run_sv` / `run_mv` drive any
adapter object with the oracle's method names (insert, retrieve, erase, size,
count_values, retrieve_multi) so the same fixture checks the oracle and the GPU path.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FLAG_BITS = {"DUP": 1, "INV": 2}


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            yield line


def _expect(rhs):
    exp = {}
    for tok in rhs.split():
        k, _, v = tok.partition("=")
        exp[k] = v
    return exp


def _flags(s):
    bits = 0
    for name in filter(None, s.split(",")):
        bits |= FLAG_BITS[name]
    return bits


def _vals(s, nf):
    return [nf if t == "NF" else int(t) for t in s.split(",")]


def run_sv(name, make_table, nf=0xFFFFFFFF):
    t = make_table()
    checked = 0
    for line in _lines(name):
        lhs, _, rhs = line.partition("->")
        op, *args = lhs.split()
        exp = _expect(rhs)
        flags = None
        if op == "insert":
            ks = [int(a.split(":")[0]) for a in args]
            vs = [int(a.split(":")[1]) for a in args]
            flags = t.insert(np.array(ks, dtype=np.uint64), np.array(vs, dtype=np.uint64))
        elif op == "erase":
            flags = t.erase(np.array([int(a) for a in args], dtype=np.uint64))
        elif op == "retrieve":
            out, found, flags = t.retrieve(np.array([int(a) for a in args], dtype=np.uint64))
            assert [int(x) for x in out] == _vals(exp["values"], nf), line
            assert [int(x) for x in found] == [int(x) for x in exp["found"].split(",")], line
        else:
            raise ValueError(op)
        if "flags" in exp:
            assert flags == _flags(exp["flags"]), (line, flags)
        if "size" in exp:
            assert t.size() == int(exp["size"]), (line, t.size())
        checked += 1
    return checked


def run_mv(name, make_table):
    t = make_table()
    checked = 0
    for line in _lines(name):
        if line == "reset":
            t = make_table()
            continue
        lhs, _, rhs = line.partition("->")
        op, *args = lhs.split()
        if op == "insert":
            ks = [int(a.split(":")[0]) for a in args]
            vs = [int(a.split(":")[1]) for a in args]
            t.insert(np.array(ks, dtype=np.uint64), np.array(vs, dtype=np.uint64))
            assert t.size() == int(_expect(rhs)["size"]), line
        elif op == "erase":
            t.erase(np.array([int(a) for a in args], dtype=np.uint64))
            assert t.size() == int(_expect(rhs)["size"]), line
        elif op == "count":
            offs, _ = t.count_values(np.array([int(a) for a in args], dtype=np.uint64))
            want = [int(x) for x in _expect(rhs)["offsets"].split(",")]
            assert [int(x) for x in offs] == want, line
        elif op == "retrieve_multi":
            q = np.array([int(a) for a in args], dtype=np.uint64)
            offs, _ = t.count_values(q)
            out, _ = t.retrieve_multi(q, offs)
            segs_txt = rhs.split("segments=", 1)[1]
            want = [sorted(int(x) for x in s.split()) for s in segs_txt.split("|")]
            assert len(want) == len(args), line
            got = [sorted(int(x) for x in out[int(offs[i]):int(offs[i + 1])]) for i in range(len(args))]
            assert got == want, (line, got)
        else:
            raise ValueError(op)
        checked += 1
    return checked
