"""Pins for the CPU BVH build (``oracle/lbvh_ref.cpp``), the twin the GPU
builder is checked against bit for bit.

The paper leaves the acceleration structure unspecified (Sec. 7.2 only says
rays are traced through the scene), so what pins the twin is validity plus
the rule of the clustering method it states (PLOC, Meister and Bittner 2018),
checked here by code that shares nothing with it:

  * Morton keys: the centroid's 10-bit cell per axis interleaved (x highest),
    recomputed from the definition with numpy float32 arithmetic and a
    bit-by-bit interleave; keys sorted, their low words a permutation;
  * structure: every internal node has two children, every node but the root
    and every leaf slot is referenced exactly once, and the tree is connected
    from root 0 (hence every triangle sits in exactly one leaf);
  * boxes: every stored child box equals, bit for bit, the float min/max of
    the vertices of that child's subtree;
  * clustering rule: replaying the rounds from the leaves, each round's
    merges are exactly the mutual nearest-neighbour pairs by merged-box half
    surface area within +-8 positions (ties to the lower position), created
    in position order;
  * closest hits: rays walked through the tree (every triangle whose
    ancestor boxes the ray enters) find the same closest hit as an exhaustive
    scan of all triangles.

The last tests plant mistakes in the twin's output (a box one ulp short, a
leaf dropped, two children swapped between rounds) and check that the
validator rejects each one.
"""
import numpy as np
import pytest

from paper_2303_15762_gb300 import scenegen as sg

LEAF = np.int64(0x80000000)


def _cases():
    return ["one", "two", "three", "grating", "small", "medium", "large"]


def _scene(case):
    if case in ("one", "two", "three"):
        n = {"one": 1, "two": 2, "three": 3}[case]
        rng = np.random.default_rng(n)
        return rng.uniform(-1, 1, (n, 3, 3)).astype(np.float32)
    if case == "grating":
        return np.asarray(sg.grating_scene()["verts"], dtype=np.float32).reshape(-1, 3, 3)
    if case == "small":
        s = sg.procedural_scene(seed=5, n_objects=4, target_tris=2100)
    elif case == "medium":
        s = sg.procedural_scene(seed=6, n_objects=16, target_tris=20000)
    else:
        s = sg.procedural_scene(seed=2)
    return np.asarray(s["verts"], dtype=np.float32).reshape(-1, 3, 3)


# ------------------------------------------------------------------ checks
def _morton_expected(verts):
    """Sorted 64-bit keys from the definition: float32 centroid ((v0 + v1) +
    v2) / 3, cell trunc((c - lo) / (hi - lo) * 1024) clamped to [0, 1023] per
    axis, bits interleaved x, y, z from the top, key = code << 32 | id."""
    v = verts.astype(np.float32)
    c = ((v[:, 0] + v[:, 1]) + v[:, 2]) / np.float32(3.0)
    lo, hi = c.min(axis=0), c.max(axis=0)
    ext = hi - lo
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(ext > 0, (c - lo) / np.where(ext > 0, ext, np.float32(1)), np.float32(0))
    q = np.clip((t * np.float32(1024.0)).astype(np.int64), 0, 1023)
    code = np.zeros(len(v), dtype=np.uint64)
    for bit in range(9, -1, -1):        # most significant cell bit first
        for a in range(3):              # x, then y, then z
            code = (code << np.uint64(1)) | ((q[:, a] >> bit) & 1).astype(np.uint64)
    keys = (code << np.uint64(32)) | np.arange(len(v), dtype=np.uint64)
    return np.sort(keys)


def _structure(n, children):
    """Checks the node graph; returns the leaf mask and child indices [n-1][2]."""
    ch = children.astype(np.int64) & 0xFFFFFFFF
    assert ch.shape == (n - 1, 2)
    is_leaf = (ch & LEAF) != 0
    idx = np.where(is_leaf, ch & 0x7FFFFFFF, ch)
    leaf_refs = idx[is_leaf]
    node_refs = idx[~is_leaf]
    assert np.all(leaf_refs < n), "leaf slot out of range"
    assert np.array_equal(np.sort(leaf_refs), np.arange(n)), "a leaf slot is missing or repeated"
    assert np.all((node_refs >= 1) & (node_refs < n - 1)), "child node reference out of range"
    assert np.array_equal(np.sort(node_refs), np.arange(1, n - 1)), "a node is missing, repeated or the root is a child"
    # connected from the root (the counts above plus reachability exclude cycles)
    seen = np.zeros(n - 1, dtype=bool)
    stack = [0]
    while stack:
        x = stack.pop()
        assert not seen[x], "cycle"
        seen[x] = True
        for c in range(2):
            if not is_leaf[x, c]:
                stack.append(int(idx[x, c]))
    assert seen.all(), "tree not connected from root 0"
    return is_leaf, idx


def _subtree_boxes(n, verts, keys, is_leaf, idx):
    """Exact float32 min/max of every child's subtree, [n-1][2][2][3]."""
    tri_of_slot = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    v = verts[tri_of_slot]                       # [slot][3 vertices][xyz]
    leaf_lo, leaf_hi = v.min(axis=1), v.max(axis=1)
    node_lo = np.zeros((n - 1, 3), np.float32)
    node_hi = np.zeros((n - 1, 3), np.float32)
    out = np.zeros((n - 1, 2, 2, 3), np.float32)
    # every child node is referenced by one parent; visit children first
    order = []
    stack = [(0, False)]
    while stack:
        x, done = stack.pop()
        if done:
            order.append(x)
            continue
        stack.append((x, True))
        for c in range(2):
            if not is_leaf[x, c]:
                stack.append((int(idx[x, c]), False))
    for x in order:
        for c in range(2):
            j = int(idx[x, c])
            lo, hi = (leaf_lo[j], leaf_hi[j]) if is_leaf[x, c] else (node_lo[j], node_hi[j])
            out[x, c, 0], out[x, c, 1] = lo, hi
        node_lo[x] = np.minimum(out[x, 0, 0], out[x, 1, 0])
        node_hi[x] = np.maximum(out[x, 0, 1], out[x, 1, 1])
    return out


def _half_area(lo, hi):
    d = (hi - lo).astype(np.float32)
    return (d[..., 0] * d[..., 1] + d[..., 1] * d[..., 2]) + d[..., 2] * d[..., 0]


def _replay_ploc(n, verts, keys, children):
    """Replays the clustering from the sorted leaves and checks that each
    round merges exactly its mutual nearest neighbours (+-8 positions, least
    merged half area in float32, ties to the lower position), numbering the
    new nodes (n - 2) - creation index in position order."""
    tri_of_slot = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    v = verts[tri_of_slot]
    lo, hi = v.min(axis=1), v.max(axis=1)
    ref = np.arange(n, dtype=np.int64) | LEAF
    ch = children.astype(np.int64) & 0xFFFFFFFF
    created = 0
    R = 8
    while len(ref) > 1:
        m = len(ref)
        best = np.full(m, -1, np.int64)
        barea = np.full(m, np.inf, np.float32)
        for off in range(-R, R + 1):           # ascending j: strict < keeps the lower j on ties
            if off == 0:
                continue
            i = np.arange(max(0, -off), min(m, m - off))
            j = i + off
            a = _half_area(np.minimum(lo[i], lo[j]), np.maximum(hi[i], hi[j]))
            better = a < barea[i]
            barea[i[better]] = a[better]
            best[i[better]] = j[better]
        pos = np.arange(m)
        mutual = (best >= 0) & (best[np.maximum(best, 0)] == pos)
        first = mutual & (best > pos)
        keep = ~(mutual & (best < pos))
        x_of = np.full(m, -1, np.int64)
        for i in np.nonzero(first)[0]:
            x = (n - 2) - created
            created += 1
            assert 0 <= x < n - 1, "more merges than internal nodes"
            assert ch[x, 0] == ref[i] and ch[x, 1] == ref[best[i]], \
                "node %d is not the merge of mutual neighbours %d, %d" % (x, i, best[i])
            x_of[i] = x
        new_lo = np.where(first[:, None], np.minimum(lo, lo[np.maximum(best, 0)]), lo)
        new_hi = np.where(first[:, None], np.maximum(hi, hi[np.maximum(best, 0)]), hi)
        new_ref = np.where(first, x_of, ref)
        lo, hi, ref = new_lo[keep], new_hi[keep], new_ref[keep]
        assert int(first.sum()) > 0, "a round without merges"
    assert created == n - 1


def _tri_hits(o, d, tv):
    """Moller-Trumbore in FP64 for rays o, d [r][3] against triangles tv
    [r][3][3] pairwise; t (inf on a miss)."""
    e1 = tv[:, 1] - tv[:, 0]
    e2 = tv[:, 2] - tv[:, 0]
    p = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, p)
    ok = np.abs(det) > 1e-300
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    s = o - tv[:, 0]
    u = np.einsum("ij,ij->i", s, p) * inv
    q = np.cross(s, e1)
    w = np.einsum("ij,ij->i", d, q) * inv
    t = np.einsum("ij,ij->i", e2, q) * inv
    hit = ok & (u >= 0) & (w >= 0) & (u + w <= 1) & (t > 1e-9)
    return np.where(hit, t, np.inf)


def _closest_exhaustive(o, d, tri):
    best_t = np.full(len(o), np.inf)
    best_i = np.full(len(o), -1, np.int64)
    for k in range(len(tri)):
        t = _tri_hits(o, d, np.broadcast_to(tri[k], (len(o), 3, 3)))
        better = t < best_t
        best_t[better] = t[better]
        best_i[better] = k
    return best_t, best_i


def _closest_through_tree(o, d, verts64, n, keys, is_leaf, idx, boxes):
    """Walks every ray through every child box it enters (all rays at once,
    level by level; boxes widened by 1e-9 so that the FP64 slab test cannot
    miss a box a hit lies in), then tests the triangles of the leaves reached."""
    tri_of_slot = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    inv = 1.0 / np.where(d == 0.0, 1e-300, d)
    rays = np.zeros(len(o) if n > 1 else 0, np.int64) + np.arange(len(o) if n > 1 else 0)
    nodes = np.zeros(len(rays), np.int64)
    cand_r, cand_s = [], []
    if n == 1:
        cand_r.append(np.arange(len(o)))
        cand_s.append(np.zeros(len(o), np.int64))
    while len(rays):
        nr, nn = [], []
        for c in range(2):
            b = boxes[nodes, c].astype(np.float64)
            lo = b[:, 0] - 1e-9 * (1 + np.abs(b[:, 0]))
            hi = b[:, 1] + 1e-9 * (1 + np.abs(b[:, 1]))
            t0 = (lo - o[rays]) * inv[rays]
            t1 = (hi - o[rays]) * inv[rays]
            tmin = np.minimum(t0, t1).max(axis=1)
            tmax = np.maximum(t0, t1).min(axis=1)
            enter = (tmax >= np.maximum(tmin, 0.0))
            leaf = is_leaf[nodes, c]
            sel = enter & leaf
            cand_r.append(rays[sel])
            cand_s.append(idx[nodes[sel], c])
            sel = enter & ~leaf
            nr.append(rays[sel])
            nn.append(idx[nodes[sel], c])
        rays = np.concatenate(nr)
        nodes = np.concatenate(nn)
    r = np.concatenate(cand_r)
    s = np.concatenate(cand_s)
    best_t = np.full(len(o), np.inf)
    best_i = np.full(len(o), -1, np.int64)
    tri_ids = tri_of_slot[s]
    t = _tri_hits(o[r], d[r], verts64[tri_ids])
    order = np.lexsort((tri_ids, t))     # per ray: least t, then least id
    r, t, tri_ids = r[order], t[order], tri_ids[order]
    first = np.unique(r, return_index=True)[1]
    fin = np.isfinite(t[first])
    best_t[r[first][fin]] = t[first][fin]
    best_i[r[first][fin]] = tri_ids[first][fin]
    return best_t, best_i


def _validate(verts, keys, children, boxes):
    n = len(verts)
    assert np.array_equal(keys, _morton_expected(verts)), "Morton keys differ from the definition"
    if n == 1:
        return None
    is_leaf, idx = _structure(n, children)
    sub = _subtree_boxes(n, verts, keys, is_leaf, idx)
    stored = boxes.reshape(n - 1, 2, 2, 3)
    assert np.array_equal(stored.view(np.uint32), sub.view(np.uint32)), \
        "a child box is not the exact float min/max of its subtree"
    _replay_ploc(n, verts, keys, children)
    return is_leaf, idx


def _random_rays(verts, count, seed):
    rng = np.random.default_rng(seed)
    v = verts.reshape(-1, 3).astype(np.float64)
    lo, hi = v.min(axis=0), v.max(axis=0)
    c, ext = (lo + hi) / 2, np.maximum(hi - lo, 1e-3)
    o = c + (rng.uniform(-0.75, 0.75, (count, 3)) * ext)
    # half the rays aim at random triangle points (so that most hit), half are isotropic
    aim_t = rng.integers(0, len(verts), count)
    bc = rng.dirichlet([1, 1, 1], count)
    aim = np.einsum("ij,ijk->ik", bc, verts[aim_t].astype(np.float64))
    d = aim - o
    iso = rng.normal(size=(count, 3))
    d[count // 2:] = iso[count // 2:]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d


# ------------------------------------------------------------------ tests
@pytest.mark.parametrize("case", _cases())
def test_twin_is_a_valid_ploc_bvh(oracle, case):
    verts = _scene(case)
    keys, children, boxes = oracle.lbvh_build(verts.reshape(-1, 9))
    _validate(verts, keys, children, boxes)


@pytest.mark.parametrize("case,count", [("three", 2000), ("grating", 20000), ("small", 20000), ("medium", 4000)])
def test_twin_closest_hits_equal_exhaustive_scan(oracle, case, count):
    verts = _scene(case)
    n = len(verts)
    keys, children, boxes = oracle.lbvh_build(verts.reshape(-1, 9))
    is_leaf, idx = _structure(n, children) if n > 1 else (None, None)
    v64 = verts.astype(np.float64)
    o, d = _random_rays(verts, count, seed=n)
    t_ex, i_ex = _closest_exhaustive(o, d, v64)
    t_bv, i_bv = _closest_through_tree(o, d, v64, n, keys, is_leaf, idx, boxes.reshape(max(n - 1, 0), 2, 2, 3))
    assert np.isfinite(t_ex).mean() > 0.3, "too few rays hit anything"
    assert np.array_equal(i_bv, i_ex)
    assert np.array_equal(t_bv, t_ex)


def test_validator_rejects_planted_mistakes(oracle):
    """Mistakes planted in the twin's output must fail the checks above."""
    verts = _scene("small")
    n = len(verts)
    keys, children, boxes = oracle.lbvh_build(verts.reshape(-1, 9))
    _validate(verts, keys, children, boxes)

    # a child box one ulp short on one face
    bad = boxes.copy().reshape(n - 1, 12)
    bad[n // 3, 3] = np.nextafter(bad[n // 3, 3], np.float32(-np.inf))
    with pytest.raises(AssertionError, match="exact float min/max"):
        _validate(verts, keys, children, bad.reshape(boxes.shape))

    # a leaf dropped: its reference replaced by another leaf's
    bad_c = children.copy()
    leaf_pos = np.argwhere((bad_c.astype(np.int64) & 0xFFFFFFFF & LEAF) != 0)
    (a0, a1), (b0, b1) = leaf_pos[5], leaf_pos[6]
    bad_c[a0, a1] = bad_c[b0, b1]
    with pytest.raises(AssertionError, match="leaf slot is missing"):
        _validate(verts, keys, bad_c, boxes)

    # two internal nodes' child pairs exchanged (structure and boxes moved
    # together, so only the clustering rule can notice)
    bad_c = children.copy()
    bad_b = boxes.copy().reshape(n - 1, 12)
    x, y = 1, n - 2
    bad_c[[x, y]] = bad_c[[y, x]]
    bad_b[[x, y]] = bad_b[[y, x]]
    with pytest.raises(AssertionError):
        _validate(verts, keys, bad_c, bad_b.reshape(boxes.shape))

    # keys not sorted by their Morton codes
    bad_k = keys.copy()
    bad_k[[3, 4]] = bad_k[[4, 3]]
    with pytest.raises(AssertionError, match="Morton"):
        _validate(verts, bad_k, children, boxes)


def test_walk_detects_a_dropped_triangle(oracle):
    """With one leaf's triangle removed from the walk, some ray's closest hit
    differs from the exhaustive scan."""
    verts = _scene("grating")
    n = len(verts)
    keys, children, boxes = oracle.lbvh_build(verts.reshape(-1, 9))
    is_leaf, idx = _structure(n, children)
    v64 = verts.astype(np.float64)
    o, d = _random_rays(verts, 4000, seed=3)
    t_ex, i_ex = _closest_exhaustive(o, d, v64)
    # point the leaf that holds slot 0 at slot 1 instead (slot 0's triangle vanishes)
    idx2 = idx.copy()
    where = np.argwhere(is_leaf & (idx == 0))[0]
    idx2[where[0], where[1]] = 1
    t_bv, i_bv = _closest_through_tree(o, d, v64, n, keys, is_leaf, idx2, boxes.reshape(n - 1, 2, 2, 3))
    assert not np.array_equal(i_bv, i_ex)
