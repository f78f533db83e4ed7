"""The graph-distance workload (stand-in for the collaboration networks of
Sec. 7): a valid PaLD input, hop counts equal to a plain breadth-first
search, and the oracle's invariants on it."""
from collections import deque

import numpy as np
import pytest

import oracle
from paper_2307_16652_gb300 import inputs

pytest.importorskip("scipy")


def test_graph_matrix_is_a_valid_input():
    n = 300
    D = inputs.graph_matrix(n)
    assert D.dtype == np.float32 and D.shape == (n, n)
    assert np.array_equal(D.view(np.uint32), D.T.view(np.uint32)), "not exactly symmetric"
    assert np.all(D.diagonal().view(np.uint32) == 0), "diagonal must be +0.0"
    off = D[~np.eye(n, dtype=bool)]
    assert np.all(np.isfinite(off)) and off.min() >= 1.0
    assert np.array_equal(off, np.round(off)), "hop counts are integers"
    assert D.max() <= 12, "collaboration graphs have a small diameter"
    assert np.array_equal(D, inputs.graph_matrix(n)), "the workload must be a pure function of its seed"


def test_hop_distances_match_a_plain_breadth_first_search():
    n = 150
    e = inputs.collaboration_edges(inputs.rng_for(inputs.GRAPH_CONFIG, 3), n)
    D = inputs.hop_distances_fp32(n, e)
    nbrs = [[] for _ in range(n)]
    for a, b in e:
        nbrs[a].append(b)
        nbrs[b].append(a)
    for s in range(n):
        dist = [-1] * n
        dist[s] = 0
        q = deque([s])
        while q:
            v = q.popleft()
            for w in nbrs[v]:
                if dist[w] < 0:
                    dist[w] = dist[v] + 1
                    q.append(w)
        assert min(dist) == 0 and dist.count(0) == 1, "the graph must be connected"
        assert np.array_equal(D[s], np.array(dist, dtype=np.float32)), f"source {s}"


def test_collaboration_degrees_are_heavy_tailed():
    n = 2000
    e = inputs.collaboration_edges(inputs.rng_for(inputs.GRAPH_CONFIG, 0), n)
    assert np.all(e[:, 0] < e[:, 1]) and len(np.unique(e, axis=0)) == len(e)
    deg = np.bincount(e.ravel(), minlength=n)
    assert deg.min() >= 1 and deg.max() >= 5 * deg.mean()


def test_oracle_invariants_on_a_graph_matrix():
    n = 200
    D = inputs.graph_matrix(n, index=1)
    U, C = oracle.focus_and_cohesion(D)
    off = ~np.eye(n, dtype=bool)
    assert np.array_equal(U, U.T)
    assert U[off].min() >= 2 and U[off].max() <= n
    assert C.min() >= 0.0
    assert abs(C.sum() - n / 2) < 1e-9 * n
    rows = C.sum(axis=1)
    assert rows.min() >= 0.0 and rows.max() <= 1.0 + 1e-12
