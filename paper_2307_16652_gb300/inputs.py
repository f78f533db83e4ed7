"""Seeded synthetic workloads for the PaLD triplet passes.

This module only draws points and turns them into FP32 distance matrices.
It contains none of the method's arithmetic (no focus sizes, no cohesion),
so both the CUDA path and the CPU oracle can take their inputs from it.

Every matrix follows one recipe: points are drawn in FP64 from a seeded
Gaussian mixture, d_ij is the FP64 Euclidean distance rounded once to FP32,
the matrix is made exactly symmetric by mirroring the upper triangle, and
the diagonal is +0.0.  The paper only says it used "randomly generated
distance matrices" (Sec. 5, Sec. 6.1); the mixtures below stand in for
that, and for the text and SNAP data the paper used (Sec. 7, App. C), which
are not available here.

Seeds come from ``numpy.random.SeedSequence([20230731, config, index])``
and the bit generator is PCG64, so a workload is a pure function of its
name (and, for the batched workload, the matrix index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 20230731

# Workload names, in the order the configurations are listed.
PLAIN_512 = "plain-512"
TIE_HEAVY_4096 = "tie-heavy-4096"
PRECISION_16384 = "precision-16384"
BATCHED_2000 = "batched-2000"
PAPER_65536 = "paper-65536"
WORKLOADS = (PLAIN_512, TIE_HEAVY_4096, PRECISION_16384, BATCHED_2000, PAPER_65536)
_CONFIG_INDEX = {name: i + 1 for i, name in enumerate(WORKLOADS)}


def rng_for(config: int, index: int = 0) -> np.random.Generator:
    """PCG64 generator for workload ``config`` (1-based) and sub-index."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE, config, index])))


# ----------------------------------------------------------------------------
# points -> FP32 distances
# ----------------------------------------------------------------------------

def _mirror_upper(d: np.ndarray) -> np.ndarray:
    """Copy the strict upper triangle onto the lower one; +0.0 diagonal."""
    n = d.shape[0]
    iu = np.triu_indices(n, 1)
    d[(iu[1], iu[0])] = d[iu]
    np.fill_diagonal(d, 0.0)
    return d


def euclidean_fp32(points: np.ndarray, block: int = 256) -> np.ndarray:
    """FP64 Euclidean distances of ``points`` (n x dim), rounded once to FP32.

    Computed from explicit coordinate differences (no |p|^2+|q|^2-2pq
    expansion, which cancels), row block by row block.
    """
    p = np.ascontiguousarray(points, dtype=np.float64)
    n = p.shape[0]
    out = np.empty((n, n), dtype=np.float32)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        diff = p[r0:r1, None, :] - p[None, :, :]
        out[r0:r1] = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff)).astype(np.float32)
    return _mirror_upper(out)


def euclidean_fp32_torch(points: np.ndarray, device: str = "cuda", block: int = 1024):
    """Same recipe as :func:`euclidean_fp32`, computed by torch on ``device``.

    Used for the n = 65536 workload, whose 17 GB matrix is built directly in
    device memory.  The FP64 distances come from explicit differences
    (``torch.cdist`` without the matmul expansion) and the upper triangle
    is mirrored block by block, so the result is exactly symmetric.
    """
    import torch

    p = torch.as_tensor(np.ascontiguousarray(points, dtype=np.float64), device=device)
    n = p.shape[0]
    d = torch.empty((n, n), dtype=torch.float32, device=device)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        blk = torch.cdist(p[r0:r1], p[r0:], compute_mode="donot_use_mm_for_euclid_dist")
        d[r0:r1, r0:] = blk.to(torch.float32)
        del blk
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        # lower part of this block-row <- transpose of the upper block-column
        if r0 > 0:
            d[r0:r1, :r0] = d[:r0, r0:r1].transpose(0, 1)
        sub = d[r0:r1, r0:r1]
        iu = torch.triu_indices(r1 - r0, r1 - r0, 1, device=device)
        sub[iu[1], iu[0]] = sub[iu[0], iu[1]]
        sub.fill_diagonal_(0.0)
    return d


# ----------------------------------------------------------------------------
# mixtures
# ----------------------------------------------------------------------------

@dataclass
class Mixture:
    sizes: np.ndarray      # points per component (sums to n)
    means: np.ndarray      # (k, dim)
    stds: np.ndarray       # (k,)

    def sample(self, rng: np.random.Generator, shuffle: bool = True) -> np.ndarray:
        dim = self.means.shape[1]
        parts = [self.means[c] + self.stds[c] * rng.standard_normal((int(s), dim))
                 for c, s in enumerate(self.sizes)]
        pts = np.concatenate(parts, axis=0)
        if shuffle:
            pts = pts[rng.permutation(pts.shape[0])]
        return pts


def largest_remainder(weights: np.ndarray, total: int) -> np.ndarray:
    """Integer sizes proportional to ``weights`` that sum exactly to ``total``."""
    w = np.asarray(weights, dtype=np.float64)
    raw = w / w.sum() * total
    base = np.floor(raw).astype(np.int64)
    rest = total - int(base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:rest]] += 1
    return base


def log_uniform(rng: np.random.Generator, lo: float, hi: float, size) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def plain_points(n: int = 512) -> np.ndarray:
    """R^2, four equal components, stds 0.1/0.5/1.0/3.0, means on a radius-10
    circle at angles k*pi/2 (the angles are this project's reading)."""
    rng = rng_for(_CONFIG_INDEX[PLAIN_512])
    k = 4
    ang = np.arange(k) * (math.pi / 2)
    means = 10.0 * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    mix = Mixture(largest_remainder(np.ones(k), n), means, np.array([0.1, 0.5, 1.0, 3.0]))
    return mix.sample(rng)


def plain_matrix(n: int = 512) -> np.ndarray:
    return euclidean_fp32(plain_points(n))


def tie_heavy_matrix(n: int = 4096, lo: int = 1, hi: int = 20, seed_index: int = 0) -> np.ndarray:
    """Symmetric integer distances drawn uniformly from [lo, hi], stored as
    FP32, +0.0 diagonal: every comparison has many exact ties."""
    rng = rng_for(_CONFIG_INDEX[TIE_HEAVY_4096], seed_index)
    d = rng.integers(lo, hi + 1, size=(n, n)).astype(np.float32)
    return _mirror_upper(d)


def precision_points(n: int = 16384, dim: int = 16, k: int = 16) -> np.ndarray:
    """R^16, 16 components with Zipf(1.2) sizes (largest remainder to n),
    stds log-uniform in [0.05, 5], means uniform in [-10, 10]^16."""
    rng = rng_for(_CONFIG_INDEX[PRECISION_16384])
    sizes = largest_remainder(np.arange(1, k + 1, dtype=np.float64) ** -1.2, n)
    stds = log_uniform(rng, 0.05, 5.0, k)
    means = rng.uniform(-10.0, 10.0, (k, dim))
    return Mixture(sizes, means, stds).sample(rng)


def precision_matrix(n: int = 16384) -> np.ndarray:
    return euclidean_fp32(precision_points(n))


def batched_sizes(count: int = 2000, lo: int = 32, hi: int = 1024) -> np.ndarray:
    """Matrix orders of the batched workload, uniform on [lo, hi]."""
    rng = rng_for(_CONFIG_INDEX[BATCHED_2000], 0)
    return rng.integers(lo, hi + 1, size=count).astype(np.int64)


def batched_points(i: int, n: int, dim: int = 8) -> np.ndarray:
    """Matrix ``i`` of the batched workload: R^8, 2..8 components with equal
    multinomial sizes, stds log-uniform in [0.1, 3], means in [-10, 10]^8."""
    rng = rng_for(_CONFIG_INDEX[BATCHED_2000], i + 1)
    k = int(rng.integers(2, 9))
    sizes = rng.multinomial(n, np.full(k, 1.0 / k))
    stds = log_uniform(rng, 0.1, 3.0, k)
    means = rng.uniform(-10.0, 10.0, (k, dim))
    return Mixture(sizes, means, stds).sample(rng)


def batched_matrices(count: int = 2000, lo: int = 32, hi: int = 1024):
    """Yield (index, n_i, D_i) for the batched workload."""
    ns = batched_sizes(count, lo, hi)
    for i, n in enumerate(ns):
        yield i, int(n), euclidean_fp32(batched_points(i, int(n)))


def packed_offsets(ns) -> np.ndarray:
    """Element offsets of n_i x n_i matrices stored back to back.

    Each offset is rounded up to a multiple of 4 elements (16 bytes) so that
    every matrix starts on a 16-byte boundary."""
    off = np.zeros(len(ns), dtype=np.int64)
    pos = 0
    for i, n in enumerate(ns):
        off[i] = pos
        pos += (int(n) * int(n) + 3) // 4 * 4
    return off, pos


def paper_points(n: int = 65536, dim: int = 32, k: int = 64) -> np.ndarray:
    """R^32, 64 equal components, stds log-uniform in [0.1, 10], means
    uniform in [-20, 20]^32 (varying densities)."""
    rng = rng_for(_CONFIG_INDEX[PAPER_65536])
    sizes = largest_remainder(np.ones(k), n)
    stds = log_uniform(rng, 0.1, 10.0, k)
    means = rng.uniform(-20.0, 20.0, (k, dim))
    return Mixture(sizes, means, stds).sample(rng)


def small_tie_heavy(rng: np.random.Generator, n: int, hi: int = 4, dup: bool = False) -> np.ndarray:
    """Tiny symmetric integer matrix for brute-force checks.

    With ``dup`` some pairs of points are made duplicates (d = 0 off the
    diagonal); their rows are copied so the matrix stays a consistent
    pseudometric on the duplicated pair."""
    d = rng.integers(1, hi + 1, size=(n, n)).astype(np.float32)
    d = _mirror_upper(d)
    if dup and n >= 3:
        a, b = rng.choice(n, size=2, replace=False)
        d[b, :] = d[a, :]
        d[:, b] = d[:, a]
        d[a, b] = d[b, a] = 0.0
        d[b, b] = 0.0
    return d


def small_points_matrix(rng: np.random.Generator, n: int, dim: int = 3) -> np.ndarray:
    """Tiny Euclidean matrix from standard normal points (ties unlikely)."""
    return euclidean_fp32(rng.standard_normal((n, dim)))


def planted_tie_matrix(rng: np.random.Generator, n: int, ties: int, dim: int = 3) -> np.ndarray:
    """Euclidean FP32 matrix with `ties` planted one-sided ties.

    Each tie copies an entry into another entry of the same row:
    d_xz = d_zx := d_xy for random distinct x, y, z, so row x holds the same
    value at columns y and z (the case that decides between pass 2's short
    and long inner loops).  The matrix stays exactly symmetric with a +0
    diagonal; it no longer needs to be a metric."""
    d = small_points_matrix(rng, n, dim=dim)
    if n < 3:
        return d
    for _ in range(ties):
        x, y, z = rng.choice(n, size=3, replace=False)
        d[x, z] = d[z, x] = d[x, y]
    return d


# ----------------------------------------------------------------------------
# graph distances: stand-in for the SNAP collaboration networks (Sec. 7)
# ----------------------------------------------------------------------------
#
# The paper's scaling study runs PaLD on all-pairs shortest-path distances of
# three co-authorship networks (5,242 to 23,133 authors).  Those files are not
# available; this recipe grows a graph of the same kind: paper i (one per
# author) joins a team of 2..5 distinct authors into a clique: author i and
# co-authors chosen with preferential attachment (probability proportional to
# 1 + the papers they already have).  Each component other than the largest
# is then tied to a random author of the largest by one edge, so every
# distance is finite and the diameter stays small.  d_ij is the hop count (an
# integer, exact in FP32); the matrices are very tie-heavy.

GRAPH_CONFIG = len(WORKLOADS) + 1  # seed config of the graph workloads ("graph-<n>")


def collaboration_edges(rng: np.random.Generator, n: int, team_lo: int = 2, team_hi: int = 5) -> np.ndarray:
    """Undirected edges (m x 2, u < v) of a connected co-authorship graph on n >= 2 authors."""
    if n < 2:
        raise ValueError("a graph workload needs n >= 2")
    pool = list(range(n))  # author a appears 1 + (papers of a) times
    edges = set()
    for lead in range(n):
        k = int(rng.integers(team_lo, min(team_hi, n) + 1))
        team = {lead}
        while len(team) < k:
            team.add(pool[int(rng.integers(len(pool)))])
        members = sorted(team)
        for i, a in enumerate(members):
            for b in members[i + 1:]:
                edges.add((a, b))
        pool.extend(members)
    e = np.array(sorted(edges), dtype=np.int64).reshape(-1, 2)
    # tie every other component to a random author of the largest one
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    adj = coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
    ncomp, labels = connected_components(adj, directed=False)
    if ncomp > 1:
        big = int(np.argmax(np.bincount(labels)))
        in_big = np.flatnonzero(labels == big)
        links = []
        for c in range(ncomp):
            if c != big:
                a = int(np.flatnonzero(labels == c)[0])
                b = int(in_big[int(rng.integers(len(in_big)))])
                links.append((min(a, b), max(a, b)))
        e = np.concatenate([e, np.array(links, dtype=np.int64)])
    return e


def hop_distances_fp32(n: int, edges: np.ndarray, block: int = 1024) -> np.ndarray:
    """All-pairs hop counts of the undirected graph (breadth-first search from
    every vertex, a block of sources at a time) as an FP32 n x n matrix; the
    graph must be connected."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path

    adj = csr_matrix((np.ones(len(edges)), (edges[:, 0], edges[:, 1])), shape=(n, n))
    adj = adj + adj.T
    D = np.empty((n, n), np.float32)
    for r0 in range(0, n, block):
        rows = np.arange(r0, min(n, r0 + block))
        d = shortest_path(adj, method="D", directed=False, unweighted=True, indices=rows)
        if not np.all(np.isfinite(d)):
            raise ValueError("the graph is not connected")
        D[rows] = d.astype(np.float32)
    np.fill_diagonal(D, 0.0)
    return D


def graph_matrix(n: int, index: int = 0) -> np.ndarray:
    """Hop-distance matrix of the seeded collaboration graph on n authors."""
    return hop_distances_fp32(n, collaboration_edges(rng_for(GRAPH_CONFIG, index), n))
