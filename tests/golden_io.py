"""Readers of the text fixtures under tests/golden/."""
import os

import numpy as np

from paper_2111_09947_gb300.synth import Csr

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_sections(name):
    secs, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                secs[cur] = []
                continue
            secs[cur].append(line)
    return secs


def rows_to_csr(lines, ncols, dtype):
    rp, ci, v = [0], [], []
    for line in lines:
        _, rest = line.split(":", 1)
        for tok in rest.split():
            c, x = tok.split(":")
            ci.append(int(c))
            v.append(dtype(x))
        rp.append(len(ci))
    return Csr(len(lines), ncols, np.array(rp, np.int32), np.array(ci, np.int32),
               np.array(v, np.float32 if dtype is float else np.int64))


def worked_example():
    s = read_sections("worked_example_4x4.txt")
    out = {}
    for k, lines in s.items():
        out[k] = rows_to_csr(lines, 4, int)
    return out


def triangle_forms():
    rows = []
    with open(os.path.join(GOLDEN, "triangle_closed_forms.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                parts = line.split()
                rows.append((parts[0], [int(x) for x in parts[1:-1]], int(parts[-1])))
    return rows


def family_edges(kind, params):
    if kind == "complete":
        n = params[0]
        return n, [(i, j) for i in range(n) for j in range(i + 1, n)]
    if kind == "bipartite":
        a, b = params
        return a + b, [(i, a + j) for i in range(a) for j in range(b)]
    if kind == "cycle":
        n = params[0]
        return n, [(i, (i + 1) % n) for i in range(n)]
    if kind == "wheel":
        r = params[0]
        return r + 1, [(0, 1 + i) for i in range(r)] + [(1 + i, 1 + (i + 1) % r) for i in range(r)]
    raise ValueError(kind)
