"""Hand-derived worked examples under tests/golden/ and the check of a LOD
result against them.

Each fixture holds a tiny input, the leaf threshold and depth cap, the
sampling modes it covers (filtered, pick, and the neighbourhood-weighted
average of Section 4.2.4 and first come of Section 4.2.1, which only the
oracle computes so far), and the
whole expected result worked out by hand from the method's definitions
(every file's header shows the derivation and cites the sections and
readings it follows).  The expected values come from neither the oracle
nor the CUDA path, so the same check pins both."""
from __future__ import annotations

import glob
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NONE = 0xFFFFFFFF
MODES = {"filtered": 0, "pick": 1, "weighted": 2, "first": 3}


def pack(r, g, b, a):
    return (int(r) & 255) | (int(g) & 255) << 8 | (int(b) & 255) << 16 | (int(a) & 255) << 24


def u32(v):
    return NONE if int(v) == -1 else int(v)


def load(path):
    fx = {"points": [], "nodes": [], "leaves": {}, "voxels": {0: {}, 1: {}, 2: {}, 3: {}}, "name": os.path.basename(path)}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        w = line.split()
        tag, v = w[0], w[1:]
        if tag == "T":
            fx["T"] = int(v[0])
        elif tag == "max_depth":
            fx["max_depth"] = int(v[0])
        elif tag == "modes":  # the modes whose voxels the file states
            fx["modes"] = sorted(MODES[t] for t in v)
        elif tag == "point":
            x, y, z, r, g, b = (int(t) for t in v)
            fx["points"].append((x, y, z, pack(r, g, b, 255)))
        elif tag == "node":
            fx["nodes"].append([int(t) for t in v])
        elif tag == "leaf":
            fx["leaves"][int(v[0])] = sorted(int(t) for t in v[1:])
        elif tag == "voxel":
            mode, node = MODES[v[0]], int(v[1])
            cell, r, g, b, a, cnt, pick = (int(t) for t in v[2:])
            fx["voxels"][mode].setdefault(node, []).append((cell, pack(r, g, b, a), cnt, u32(pick)))
        else:
            raise ValueError(f"{path}: unknown line {line!r}")
    p = np.array(fx["points"], dtype=np.int64).reshape(-1, 4)
    fx["input"] = np.ascontiguousarray(p.astype(np.uint32).view(np.int32).reshape(-1, 4) if len(p) else
                                       np.zeros((0, 4), np.int32))
    return fx


def fixtures():
    return sorted(glob.glob(os.path.join(HERE, "*.txt")))


def cases(modes=(0, 1, 2, 3)):
    """(path, mode) for every fixture and every stated mode among ``modes``."""
    return [(p, m) for p in fixtures() for m in load(p)["modes"] if m in modes]


def check(res: dict, fx: dict, mode: int) -> None:
    """Every node field, every leaf's points (and indices where the result
    keeps them) and every inner node's voxels equal the worked example."""
    name = fx["name"]
    nodes = fx["nodes"]
    assert len(res["level"]) == len(nodes), f"{name}: {len(res['level'])} nodes, expected {len(nodes)}"
    for row in nodes:
        i, mx, my, mz, level, lg, mask, flags, parent, first, off, cnt = row
        got = (tuple(int(t) for t in res["min"][i]), int(res["level"][i]), int(res["log2_size"][i]),
               int(res["child_mask"][i]), int(res["flags"][i]), int(res["parent"][i]), int(res["first_child"][i]),
               int(res["point_offset"][i]), int(res["point_count"][i]))
        want = ((mx, my, mz), level, lg, mask, flags, u32(parent), u32(first), off, cnt)
        assert got == want, f"{name} node {i}: {got} != {want}"
        nvox = len(fx["voxels"][mode].get(i, []))
        assert int(res["voxel_count"][i]) == nvox, f"{name} node {i}: voxel_count"
    inp = fx["input"]
    for i, idx in fx["leaves"].items():
        a, c = int(res["point_offset"][i]), int(res["point_count"][i])
        have = np.asarray(res["points"][a:a + c]).astype(np.int64)
        want = inp[idx].astype(np.int64)
        key = lambda m: m[np.lexsort(m.T[::-1])]
        assert np.array_equal(key(have), key(want)), f"{name} leaf {i}: points"
        if res.get("index") is not None:
            assert sorted(int(t) for t in res["index"][a:a + c]) == idx, f"{name} leaf {i}: indices"
    vox = np.asarray(res["voxels"]).reshape(-1, 4).astype(np.uint32)
    for i, rows in fx["voxels"][mode].items():
        a, c = int(res["voxel_offset"][i]), int(res["voxel_count"][i])
        have = sorted(tuple(int(t) for t in r) for r in vox[a:a + c])
        assert have == sorted(rows), f"{name} node {i}: voxels {have} != {sorted(rows)}"
