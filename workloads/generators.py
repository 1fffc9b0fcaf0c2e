"""Seeded synthetic workloads for the dynamic max-flow path.

Both sides of every parity check read their inputs from here: the CPU oracle
(``oracle/``) and the CUDA library (``paper_2511_05895_gb300``).  This module
holds no max-flow arithmetic at all -- it only draws graphs, capacities and
update batches.

Random numbers come from one counter-based generator, splitmix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value ``i`` of a stream with key ``k`` is ``mix64(k + (i + 1) * 0x9E3779B97F4A7C15)``.
It is written out here with numpy uint64 arithmetic, so the same seed gives
the same integers on every machine and every numpy version.

Workload shapes (the paper's real graphs are not available, so these stand in
for them):

* ``random_graph``   -- uniform directed graph with a guaranteed s->t path
                        (the paper's integer weights drawn from 1..100, Sec. 6.1).
* ``rmat``           -- RMAT power-law graph (a, b, c, d quadrant recursion),
                        standing in for the social/web graphs of Table 1.
* ``grid_segmentation`` -- 4-connected image grid with terminal arcs, the
                        image-segmentation use named in Sec. 1.
* ``mixed_batch``    -- distinct uniformly chosen edges, half raised and half
                        lowered (clamped at 0): the mixed updates of Sec. 6.4.
* ``grid_rect_batch``-- rewrite of the terminal capacities inside a rectangle.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    tmp = z >> np.uint64(30)
    z ^= tmp
    z *= _M1
    np.right_shift(z, np.uint64(27), out=tmp)
    z ^= tmp
    z *= _M2
    np.right_shift(z, np.uint64(31), out=tmp)
    z ^= tmp
    return z


def _fnv1a(text: str) -> int:
    h = 0xCBF29CE484222325
    for b in text.encode():
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


class Stream:
    """One named splitmix64 stream derived from (seed, name)."""

    def __init__(self, seed: int, name: str):
        base = np.array([(int(seed) * 0x9E3779B97F4A7C15 + _fnv1a(name)) & 0xFFFFFFFFFFFFFFFF],
                        dtype=np.uint64)
        self.key = _mix64(base)[0]
        self.pos = 0

    def u64(self, count: int) -> np.ndarray:
        z = self.u64_at(self.pos, count)
        self.pos += count
        return z

    def u64_at(self, offset: int, count: int) -> np.ndarray:
        """Values offset .. offset + count - 1 of the stream (position unchanged)."""
        z = np.arange(offset + 1, offset + 1 + count, dtype=np.uint64)
        z *= _GOLDEN
        z += self.key
        return _mix64(z)

    def integers(self, count: int, lo: int, hi: int) -> np.ndarray:
        """Integers uniform in [lo, hi] (inclusive) by the multiply-shift map."""
        span = int(hi) - int(lo) + 1
        assert 0 < span <= (1 << 32)
        x = self.u64(count) >> np.uint64(32)
        return (int(lo) + ((x * np.uint64(span)) >> np.uint64(32)).astype(np.int64))

    def uniform(self, count: int) -> np.ndarray:
        """Floats uniform in [0, 1) with 53 random bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def permutation(self, count: int) -> np.ndarray:
        """A seeded permutation of range(count) (sort by random 64-bit keys)."""
        return np.argsort(self.u64(count), kind="stable").astype(np.int64)


@dataclass
class Graph:
    """A directed graph in CSR form.  Edge id == CSR position."""

    n: int
    row_ptr: np.ndarray  # int64 [n + 1]
    col: np.ndarray      # int32 [m]
    cap: np.ndarray      # int32 [m]
    s: int
    t: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def tails(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.row_ptr)).astype(np.int32)


def from_edges(n: int, tails, heads, caps, s: int, t: int, name: str = "") -> Graph:
    """Build CSR (stable order by tail) from an edge list."""
    tails = np.asarray(tails, dtype=np.int64)
    heads = np.asarray(heads, dtype=np.int64)
    caps = np.asarray(caps, dtype=np.int64)
    m = tails.shape[0]
    assert n < (1 << 31) and m < (1 << 32)
    # stable order by tail: sort the unique keys tail * 2**32 + position
    keys = (tails << np.int64(32)) | np.arange(m, dtype=np.int64)
    keys.sort()
    order = keys & np.int64(0xFFFFFFFF)
    counts = np.bincount(tails, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(n=n, row_ptr=row_ptr, col=heads[order].astype(np.int32),
                 cap=caps[order].astype(np.int32), s=int(s), t=int(t), name=name)


def random_graph(n: int = 1000, m: int = 8000, cap_lo: int = 1, cap_hi: int = 100,
                 seed: int = 0, s: int = 0, t: int | None = None) -> Graph:
    """Uniform random directed graph with no self-loops plus a guaranteed path.

    The path is s -> v1 -> v2 -> t with v1, v2 distinct and outside {s, t};
    the other m - 3 edges have uniform endpoints (self-loops are re-mapped by
    drawing the head as tail + 1 + U[0, n - 2] mod n).  Capacities are uniform
    integers in [cap_lo, cap_hi].  Parallel and antiparallel edges may occur.
    """
    t = n - 1 if t is None else t
    assert n >= 4 and m >= 3 and s != t
    st = Stream(seed, "random_graph")
    others = np.array([v for v in range(n) if v not in (s, t)], dtype=np.int64)
    i1 = int(st.integers(1, 0, len(others) - 1)[0])
    i2 = int(st.integers(1, 0, len(others) - 2)[0])
    if i2 >= i1:
        i2 += 1
    v1, v2 = int(others[i1]), int(others[i2])
    u = st.integers(m - 3, 0, n - 1)
    v = (u + 1 + st.integers(m - 3, 0, n - 2)) % n
    tails = np.concatenate([[s, v1, v2], u])
    heads = np.concatenate([[v1, v2, t], v])
    caps = st.integers(m, cap_lo, cap_hi)
    g = from_edges(n, tails, heads, caps, s, t, name=f"random_n{n}_m{m}_seed{seed}")
    g.meta.update(kind="random", seed=seed)
    return g


def rmat(scale: int = 20, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, cap_lo: int = 1, cap_hi: int = 1000, seed: int = 0) -> Graph:
    """RMAT graph: edge_factor * 2**scale draws of the (a, b, c, d) recursion.

    Each level picks a quadrant by one 32-bit uniform compared with the
    cumulative thresholds floor(p * 2**32).  Vertex ids are then relabelled by
    a seeded permutation (no artificial locality), self-loops are dropped and
    duplicate edges kept.  s is the vertex of highest out-degree and t the
    second highest (ties go to the lower id).
    """
    n = 1 << scale
    draws = edge_factor * n
    st = Stream(seed, "rmat")
    th_a = np.uint32(int(a * 2 ** 32))
    th_ab = np.uint32(int((a + b) * 2 ** 32))
    th_abc = np.uint32(int((a + b + c) * 2 ** 32))
    u = np.zeros(draws, dtype=np.uint32)
    v = np.zeros(draws, dtype=np.uint32)
    pairs = (scale + 1) // 2   # one 64-bit value per draw feeds two levels

    def levels(c0: int, c1: int) -> None:
        # draws [c0, c1): level 2k uses the high and level 2k + 1 the low 32
        # bits of value k * draws + i of the stream
        uu = u[c0:c1]
        vv = v[c0:c1]
        level = 0
        for k in range(pairs):
            x = st.u64_at(k * draws + c0, c1 - c0)
            for half in (x >> np.uint64(32), x & np.uint64(0xFFFFFFFF)):
                if level >= scale:
                    break
                half = half.astype(np.uint32)
                bu = half >= th_ab                                        # quadrants c, d
                bv = ((half >= th_a) & ~bu) | (half >= th_abc)           # b, d
                uu <<= np.uint32(1)
                uu |= bu
                vv <<= np.uint32(1)
                vv |= bv
                level += 1

    chunk = 1 << 20
    bounds = [(c0, min(draws, c0 + chunk)) for c0 in range(0, draws, chunk)]
    if len(bounds) > 1:
        from concurrent.futures import ThreadPoolExecutor   # numpy releases the GIL
        import os
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(lambda cb: levels(*cb), bounds))
    else:
        levels(0, draws)
    st.pos = pairs * draws
    perm = st.permutation(n)
    u = perm[u.astype(np.int64)]
    v = perm[v.astype(np.int64)]
    keep = u != v
    u, v = u[keep], v[keep]
    caps = st.integers(u.shape[0], cap_lo, cap_hi)
    outdeg = np.bincount(u, minlength=n)
    order = np.lexsort((np.arange(n), -outdeg))
    s, t = int(order[0]), int(order[1])
    g = from_edges(n, u, v, caps, s, t, name=f"rmat{scale}_ef{edge_factor}_seed{seed}")
    g.meta.update(kind="rmat", seed=seed, scale=scale)
    return g


def _grid_intensity(W: int, H: int, st: Stream, n_blobs: int) -> np.ndarray:
    xs = np.arange(W, dtype=np.float64)
    ys = np.arange(H, dtype=np.float64)
    img = np.full((H, W), 40.0)
    cx = st.uniform(n_blobs) * W
    cy = st.uniform(n_blobs) * H
    rad = (st.uniform(n_blobs) * (1.0 / 6 - 1.0 / 32) + 1.0 / 32) * min(W, H)
    amp = 60.0 + st.uniform(n_blobs) * 100.0
    for k in range(n_blobs):
        gx = np.exp(-((xs - cx[k]) ** 2) / (2.0 * rad[k] ** 2))
        gy = np.exp(-((ys - cy[k]) ** 2) / (2.0 * rad[k] ** 2))
        img += amp[k] * np.outer(gy, gx)
    img += (st.uniform(W * H).reshape(H, W) - 0.5) * 10.0   # mild sensor noise
    return np.clip(img, 0.0, 255.0)


def _nll(img: np.ndarray, mu: float, sd: float) -> np.ndarray:
    return 0.5 * ((img - mu) / sd) ** 2 + np.log(sd)


def grid_segmentation(W: int = 4096, H: int = 4096, sigma: float = 10.0, n_blobs: int = 24,
                      seed: int = 0) -> Graph:
    """4-connected pixel grid with terminal arcs (image segmentation).

    Pixel (x, y) is vertex y * W + x; s = W * H and t = W * H + 1.  Each pixel
    has an n-link edge to each existing 4-neighbour with capacity
    round(100 * exp(-dI**2 / (2 sigma**2))), an edge p -> t with capacity
    round(1000 * NLL_fg(p) / Lmax) and an edge s -> p with capacity
    round(1000 * NLL_bg(p) / Lmax), where NLL_* are Gaussian negative
    log-likelihoods of the pixel intensity under the foreground/background
    models and Lmax is the largest of them over the image.
    Row order: pixel rows hold right, left, down, up n-links then the t-link;
    s's row holds s -> p for p = 0 .. W*H - 1; t's row is empty.
    """
    st = Stream(seed, "grid")
    img = _grid_intensity(W, H, st, n_blobs)
    mu_b = 30.0 + 40.0 * st.uniform(1)[0]
    mu_f = 150.0 + 50.0 * st.uniform(1)[0]
    sd_b = 20.0 + 20.0 * st.uniform(1)[0]
    sd_f = 20.0 + 20.0 * st.uniform(1)[0]
    nll_f = _nll(img, mu_f, sd_f)
    nll_b = _nll(img, mu_b, sd_b)
    lmax = float(max(nll_f.max(), nll_b.max()))
    P = W * H
    s, t = P, P + 1
    n = P + 2
    pid = np.arange(P, dtype=np.int64).reshape(H, W)
    inv2s2 = 1.0 / (2.0 * sigma * sigma)
    heads = np.full((H, W, 5), -1, dtype=np.int64)
    caps = np.zeros((H, W, 5), dtype=np.int64)
    # right, left, down, up
    heads[:, :-1, 0] = pid[:, 1:]
    caps[:, :-1, 0] = np.rint(100.0 * np.exp(-((img[:, :-1] - img[:, 1:]) ** 2) * inv2s2))
    heads[:, 1:, 1] = pid[:, :-1]
    caps[:, 1:, 1] = np.rint(100.0 * np.exp(-((img[:, 1:] - img[:, :-1]) ** 2) * inv2s2))
    heads[:-1, :, 2] = pid[1:, :]
    caps[:-1, :, 2] = np.rint(100.0 * np.exp(-((img[:-1, :] - img[1:, :]) ** 2) * inv2s2))
    heads[1:, :, 3] = pid[:-1, :]
    caps[1:, :, 3] = np.rint(100.0 * np.exp(-((img[1:, :] - img[:-1, :]) ** 2) * inv2s2))
    heads[:, :, 4] = t
    caps[:, :, 4] = np.rint(1000.0 * nll_f / lmax)
    valid = heads.reshape(P, 5) >= 0
    deg = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:P + 1])
    row_ptr[P + 1] = row_ptr[P] + P   # s's row
    row_ptr[P + 2] = row_ptr[P + 1]   # t's row (empty)
    col = np.concatenate([heads.reshape(P, 5)[valid], np.arange(P, dtype=np.int64)])
    cap_s = np.rint(1000.0 * nll_b / lmax).reshape(P)
    cap = np.concatenate([caps.reshape(P, 5)[valid], cap_s])
    g = Graph(n=n, row_ptr=row_ptr, col=col.astype(np.int32), cap=cap.astype(np.int32),
              s=s, t=t, name=f"grid{W}x{H}_seed{seed}")
    g.meta.update(kind="grid", seed=seed, W=W, H=H, img=img, lmax=lmax,
                  models=(mu_f, sd_f, mu_b, sd_b))
    return g


def choose_distinct(st: Stream, count: int, m: int) -> np.ndarray:
    """count distinct ids uniform in [0, m), in random draw order."""
    assert 0 <= count <= m
    picked = np.zeros(0, dtype=np.int64)
    while picked.shape[0] < count:
        need = count - picked.shape[0]
        cand = st.integers(int(need * 1.25) + 64, 0, m - 1)
        allc = np.concatenate([picked, cand])
        _, first = np.unique(allc, return_index=True)
        picked = allc[np.sort(first)]
    return picked[:count]


@dataclass
class Batch:
    edge_id: np.ndarray   # int32 [k], distinct
    new_cap: np.ndarray   # int32 [k], absolute new capacity >= 0


def mixed_batch(cur_cap: np.ndarray, k: int, lo: int, hi: int, seed: int, index: int) -> Batch:
    """k distinct uniform edges: the first ceil(k/2) get +U[lo, hi], the rest
    -U[lo, hi] clamped at 0.  ``cur_cap`` holds the current (cumulative) edge
    capacities; it is not modified."""
    st = Stream(seed, f"mixed_batch_{index}")
    ids = choose_distinct(st, k, cur_cap.shape[0])
    amt = st.integers(k, lo, hi)
    ninc = (k + 1) // 2
    old = cur_cap[ids].astype(np.int64)
    new = old.copy()
    new[:ninc] = old[:ninc] + amt[:ninc]
    new[ninc:] = np.maximum(0, old[ninc:] - amt[ninc:])
    return Batch(edge_id=ids.astype(np.int32), new_cap=new.astype(np.int32))


def grid_rect_batch(g: Graph, seed: int, index: int, side_lo: int = 64, side_hi: int = 512) -> Batch:
    """Re-draw the intensities inside a random rectangle (a new blob) and
    rewrite the s->p and p->t capacities of every pixel in it.  The image in
    ``g.meta['img']`` is updated in place so that batches accumulate."""
    W, H = g.meta["W"], g.meta["H"]
    img = g.meta["img"]
    mu_f, sd_f, mu_b, sd_b = g.meta["models"]
    lmax = g.meta["lmax"]
    st = Stream(seed, f"grid_rect_{index}")
    w = int(min(W, st.integers(1, side_lo, side_hi)[0]))
    h = int(min(H, st.integers(1, side_lo, side_hi)[0]))
    x0 = int(st.integers(1, 0, W - w)[0])
    y0 = int(st.integers(1, 0, H - h)[0])
    sign = 1.0 if st.integers(1, 0, 1)[0] else -1.0
    amp = sign * (40.0 + 80.0 * st.uniform(1)[0])
    rad = max(w, h) / 3.0
    xs = np.arange(x0, x0 + w, dtype=np.float64) - (x0 + w / 2.0)
    ys = np.arange(y0, y0 + h, dtype=np.float64) - (y0 + h / 2.0)
    blob = amp * np.outer(np.exp(-ys ** 2 / (2 * rad * rad)), np.exp(-xs ** 2 / (2 * rad * rad)))
    sub = np.clip(img[y0:y0 + h, x0:x0 + w] + blob, 0.0, 255.0)
    img[y0:y0 + h, x0:x0 + w] = sub
    cap_t = np.clip(np.rint(1000.0 * _nll(sub, mu_f, sd_f) / lmax), 0, 1000).astype(np.int64)
    cap_s = np.clip(np.rint(1000.0 * _nll(sub, mu_b, sd_b) / lmax), 0, 1000).astype(np.int64)
    pix = (np.arange(y0, y0 + h, dtype=np.int64)[:, None] * W
           + np.arange(x0, x0 + w, dtype=np.int64)[None, :]).reshape(-1)
    P = W * H
    tlink = g.row_ptr[pix + 1] - 1           # last edge of each pixel row is p -> t
    slink = g.row_ptr[P] + pix               # s's row lists s -> p in pixel order
    ids = np.concatenate([slink, tlink])
    new = np.concatenate([cap_s.reshape(-1), cap_t.reshape(-1)])
    return Batch(edge_id=ids.astype(np.int32), new_cap=new.astype(np.int32))


def apply_batch(cur_cap: np.ndarray, batch: Batch) -> None:
    """Write a batch's absolute capacities into the host copy of the caps."""
    cur_cap[batch.edge_id.astype(np.int64)] = batch.new_cap


def bipartite(left: int = 1 << 20, right: int = 1 << 20, m: int = 16 << 20, seed: int = 0) -> Graph:
    """Unit-capacity assignment graph: s -> every left vertex, m uniform
    left -> right edges, every right vertex -> t (max flow = maximum
    matching).  Vertices: left 0 .. L-1, right L .. L+R-1, s = L+R, t = L+R+1."""
    st = Stream(seed, "bipartite")
    L, R = left, right
    s, t = L + R, L + R + 1
    lu = st.integers(m, 0, L - 1)
    rv = L + st.integers(m, 0, R - 1)
    tails = np.concatenate([np.full(L, s, np.int64), lu, np.arange(L, L + R, dtype=np.int64)])
    heads = np.concatenate([np.arange(L, dtype=np.int64), rv, np.full(R, t, np.int64)])
    g = from_edges(L + R + 2, tails, heads, np.ones(tails.shape[0], np.int64), s, t,
                   name=f"bipartite{L}x{R}_m{m}_seed{seed}")
    g.meta.update(kind="bipartite", seed=seed)
    return g
