"""Seeded synthetic street-canyon meshes (input generation only).

This module builds the unstructured triangular meshes that stand in for the
Gmsh meshes of Section 3 (Fig. 1: ~12,000 cells, wall-refined, elliptic
relaxation; Fig. 2: ~500 cells with the y+ < 30 wall strip removed, wall
functions). It holds none of the method's arithmetic: it only lays out nodes
and triangles, tags boundary edges and pairs the periodic nodes. Both the
CUDA path and the CPU oracle consume its output.

Geometry (Section 3): a periodic row of street canyons. One period of length
``L = B + W`` holds a building of width ``B`` (split across the periodic seam)
and a canyon of width ``W`` centred at ``x = L/2``; buildings have height
``H`` and the domain top is at ``y = T``.  With ``offset = d > 0`` the no-slip
walls are moved a distance ``d`` into the fluid, the stripped domain of the
wall-function case (Fig. 2 caption; Section 3 on y+ = 30).

Construction: a tensor-product set of grid lines (uniform, or geometrically
graded toward the walls for the fully resolved case), restricted to the fluid
polygon, interior nodes jittered by a seeded random fraction of the local
spacing, every quadrilateral split along a seeded random diagonal. The result
is conforming by construction (every wall is a union of grid-line segments),
periodic-x node pairs share their y coordinate, and elements are numbered in
Morton order of their centroids so that element-sorted particles touch nearby
memory.

Conventions of the returned mesh (the C-ABI ``pdf_init_mesh`` takes these):
  xy[nnode, 2]      float64 node coordinates
  tri[ntri, 3]      int32, counter-clockwise
  edge_tag[ntri, 3] int32, edge k is the edge opposite vertex k:
                    0 interior, 1 wall, 2 top (symmetry), 3 periodic
  periodic_pair[nnode] int32, partner node across the seam or -1
"""
from __future__ import annotations

import numpy as np

EDGE_INTERIOR, EDGE_WALL, EDGE_TOP, EDGE_PERIODIC = 0, 1, 2, 3


def _graded_between(a: float, b: float, h_a: float, h_b: float, h_max: float,
                    growth: float) -> np.ndarray:
    """Points in [a, b] whose spacing starts at h_a at a (h_b at b), grows by
    ``growth`` per cell away from each end, and is capped at h_max.
    ``h_a``/``h_b`` of None mean "no refinement at that end"."""
    length = b - a
    if length <= 0:
        return np.array([a])

    def ramp(h0):
        if h0 is None:
            return np.zeros(0)
        d, s, out = 0.0, h0, []
        while s < h_max and d + s < 0.5 * length:
            d += s
            out.append(d)
            s *= growth
        return np.array(out)

    ra, rb = ramp(h_a), ramp(h_b)
    da = ra[-1] if ra.size else 0.0
    db = rb[-1] if rb.size else 0.0
    mid_len = length - da - db
    nmid = max(1, int(np.ceil(mid_len / h_max)))
    mid = da + np.linspace(0.0, mid_len, nmid + 1)
    pts = np.concatenate([[0.0], ra, mid, length - rb[::-1], [length]])
    pts = np.unique(np.round(pts, 14))
    out = a + pts
    out[0], out[-1] = a, b
    return out


def _merge_lines(*parts: np.ndarray) -> np.ndarray:
    """Union of sorted line sets, dropping near-duplicates (keeps exact ends)."""
    allp = np.concatenate(parts)
    allp.sort()
    keep = [allp[0]]
    for v in allp[1:]:
        if v - keep[-1] > 1e-12:
            keep.append(v)
        elif v in [p[0] for p in parts] or v in [p[-1] for p in parts]:
            keep[-1] = v
    return np.array(keep)


def _morton_key(x: np.ndarray, y: np.ndarray, bits: int = 16) -> np.ndarray:
    xs = ((x - x.min()) / max(np.ptp(x), 1e-300) * ((1 << bits) - 1)).astype(np.uint64)
    ys = ((y - y.min()) / max(np.ptp(y), 1e-300) * ((1 << bits) - 1)).astype(np.uint64)
    key = np.zeros_like(xs)
    for i in range(bits):
        key |= ((xs >> np.uint64(i)) & np.uint64(1)) << np.uint64(2 * i)
        key |= ((ys >> np.uint64(i)) & np.uint64(1)) << np.uint64(2 * i + 1)
    return key


def canyon_mesh(*, H: float = 1.0, W: float = 1.0, B: float = 2.0, T: float = 2.0,
                offset: float = 0.0, h: float = 0.07, y1: float | None = None,
                growth: float = 1.2, jitter: float = 0.2, seed: int = 0) -> dict:
    """Build one canyon mesh.

    h       target spacing away from walls (uniform mesh when y1 is None)
    y1      first-cell height at the no-slip walls (graded mesh), or None
    growth  geometric growth ratio of the graded spacing
    jitter  interior nodes move by up to +-jitter x the local spacing
    """
    rng = np.random.default_rng(seed)
    L = B + W
    xl, xr = 0.5 * (L - W), 0.5 * (L + W)
    d = offset
    xwl, xwr = xl + d, xr - d            # canyon side walls
    yf, yr = d, H + d                    # canyon floor, roof level
    if not (0 < xwl < xwr < L and 0 <= yf < yr < T):
        raise ValueError("degenerate canyon geometry")
    ref = y1  # None -> uniform
    # x lines: refined toward the canyon side walls from both sides
    xs = _merge_lines(
        _graded_between(0.0, xwl, None, ref, h, growth),
        _graded_between(xwl, xwr, ref, ref, h, growth),
        _graded_between(xwr, L, ref, None, h, growth))
    # y lines: refined toward the floor and toward the roof level (both sides)
    ys = _merge_lines(
        _graded_between(yf, yr, ref, ref, h, growth),
        _graded_between(yr, T, ref, None, h, growth))
    nx, ny = xs.size, ys.size

    def fluid_cell(i, j):  # cell [xs[i],xs[i+1]] x [ys[j],ys[j+1]]
        xc, yc = 0.5 * (xs[i] + xs[i + 1]), 0.5 * (ys[j] + ys[j + 1])
        return yc > yr or (xwl < xc < xwr)

    cells = [(i, j) for j in range(ny - 1) for i in range(nx - 1) if fluid_cell(i, j)]
    used = np.zeros((nx, ny), dtype=bool)
    for i, j in cells:
        used[i, j] = used[i + 1, j] = used[i, j + 1] = used[i + 1, j + 1] = True
    gid = -np.ones((nx, ny), dtype=np.int64)
    gid[used] = np.arange(int(used.sum()))
    I, J = np.nonzero(used)
    px, py = xs[I].copy(), ys[J].copy()

    # boundary nodes keep their coordinates; interior nodes are jittered
    def on_boundary(i, j):
        x, y = xs[i], ys[j]
        if i == 0 or i == nx - 1 or j == ny - 1:
            return True
        if y == yf or (y == yr and not (xwl < x < xwr)):
            return True
        if (x == xwl or x == xwr) and y <= yr:
            return True
        return False

    for n, (i, j) in enumerate(zip(I, J)):
        if on_boundary(i, j):
            continue
        sx = min(xs[i] - xs[i - 1], xs[i + 1] - xs[i])
        sy = min(ys[j] - ys[j - 1], ys[j + 1] - ys[j])
        px[n] += jitter * sx * (2 * rng.random() - 1)
        py[n] += jitter * sy * (2 * rng.random() - 1)

    tris = []
    flips = rng.random(len(cells)) < 0.5
    for (i, j), f in zip(cells, flips):
        a, b, c, e = gid[i, j], gid[i + 1, j], gid[i + 1, j + 1], gid[i, j + 1]
        if f:
            tris += [(a, b, c), (a, c, e)]
        else:
            tris += [(a, b, e), (b, c, e)]
    tri = np.array(tris, dtype=np.int64)

    # node renumbering: Morton order of nodes; element order: Morton of centroid
    nkey = _morton_key(px, py)
    norder = np.argsort(nkey, kind="stable")
    newid = np.empty_like(norder)
    newid[norder] = np.arange(norder.size)
    xy = np.stack([px[norder], py[norder]], axis=1)
    tri = newid[tri]
    cx, cy = xy[tri, 0].mean(axis=1), xy[tri, 1].mean(axis=1)
    tri = tri[np.argsort(_morton_key(cx, cy), kind="stable")]
    # counter-clockwise orientation
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    area2 = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    cw = area2 < 0
    tri[cw] = tri[cw][:, [0, 2, 1]]
    tri = tri.astype(np.int32)

    # edge tags (edge k opposite vertex k)
    ntri = tri.shape[0]
    e0 = tri[:, [1, 2, 0]]
    e1 = tri[:, [2, 0, 1]]
    lo = np.minimum(e0, e1).ravel().astype(np.int64)
    hi = np.maximum(e0, e1).ravel().astype(np.int64)
    key = lo * xy.shape[0] + hi
    uniq, counts = np.unique(key, return_counts=True)
    cnt = counts[np.searchsorted(uniq, key)]
    edge_tag = np.zeros(3 * ntri, dtype=np.int32)
    bnd = np.nonzero(cnt == 1)[0]
    mx = 0.5 * (xy[lo[bnd], 0] + xy[hi[bnd], 0])
    my = 0.5 * (xy[lo[bnd], 1] + xy[hi[bnd], 1])
    same_x = xy[lo[bnd], 0] == xy[hi[bnd], 0]
    per = same_x & ((mx == 0.0) | (mx == L))
    top = (~per) & (my == T)
    tag = np.full(bnd.size, EDGE_WALL, dtype=np.int32)
    tag[per] = EDGE_PERIODIC
    tag[top] = EDGE_TOP
    edge_tag[bnd] = tag
    if np.any(cnt > 2):
        raise RuntimeError("non-manifold edge")
    edge_tag = edge_tag.reshape(ntri, 3)

    # periodic pairs: nodes on x = 0 and x = L with equal y
    pair = -np.ones(xy.shape[0], dtype=np.int32)
    left = np.nonzero(xy[:, 0] == 0.0)[0]
    right = np.nonzero(xy[:, 0] == L)[0]
    ry = {float(xy[r, 1]): r for r in right}
    for l_ in left:
        r = ry[float(xy[l_, 1])]
        pair[l_], pair[r] = r, l_

    return dict(xy=np.ascontiguousarray(xy, dtype=np.float64), tri=np.ascontiguousarray(tri),
                edge_tag=np.ascontiguousarray(edge_tag), periodic_pair=pair,
                L=L, H=H, W=W, T=T, offset=d, x_canyon=(xwl, xwr), y_floor=yf, y_roof=yr)


def inradius(mesh: dict) -> np.ndarray:
    """Inradius of every triangle (geometry only)."""
    xy, tri = mesh["xy"], mesh["tri"]
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    la = np.hypot(*(b - c).T)
    lb = np.hypot(*(c - a).T)
    lc = np.hypot(*(a - b).T)
    area = 0.5 * np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    return 2.0 * area / (la + lb + lc)
