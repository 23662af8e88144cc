"""Readers for the text fixtures under tests/golden/ (each cites its passage)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for raw in fh:
            line = raw.split("#", 1)[0].strip()
            if line:
                yield line.split()


def bfs_example():
    d = {"rows": {}, "frontiers": {}}
    for tok in _lines("paper_bfs_example.txt"):
        key, vals = tok[0], tok[1:]
        if key == "row":
            d["rows"][int(vals[0])] = [int(x) for x in vals[1:]]
        elif key == "frontier":
            d["frontiers"][int(vals[0])] = [int(x) for x in vals[1:]]
        elif key in ("n", "root"):
            d[key] = int(vals[0])
        else:
            d[key] = [int(x) for x in vals]
    n = d["n"]
    A = np.array([d["rows"][r] for r in range(n)], dtype=np.uint8)
    d["A"] = A
    src, dst = np.nonzero(np.triu(A))          # each undirected edge once
    d["src"] = src.astype(np.int32)
    d["dst"] = dst.astype(np.int32)
    return d


def directory_example():
    d = {}
    for tok in _lines("paper_directory_example.txt"):
        key, vals = tok[0], [int(x) for x in tok[1:]]
        d[key] = vals if len(vals) != 1 else vals[0]
    return d


def wah_examples():
    out, cur = {}, None
    for tok in _lines("paper_wah_examples.txt"):
        key, vals = tok[0], tok[1:]
        if key == "example":
            cur = out.setdefault(vals[0], {})
        elif key == "runs":
            bits = []
            for r in vals:
                cnt, b = r.split(":")
                bits += [int(b)] * int(cnt)
            cur["bits"] = np.array(bits, dtype=np.uint8)
        elif key == "words":
            cur["words"] = [int(x, 16) for x in vals]
        else:
            cur[key] = int(vals[0])
    return out


def row_buffer_example():
    """{p: [[word per slot] per level]} of paper_row_buffers.txt."""
    out = {}
    for tok in _lines("paper_row_buffers.txt"):
        if tok[0] != "words":
            continue
        p, k = int(tok[1]), int(tok[2])
        lv = out.setdefault(p, [])
        assert len(lv) == k
        lv.append([int(x, 16) for x in tok[3:]])
    return out
