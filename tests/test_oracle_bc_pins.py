"""Pins of the betweenness-centrality oracle (Alg. 3 forward sweep + dependency back-propagation)
against facts that do not come from its own formula: closed forms on paths, stars and complete
graphs, path counts on grids (binomials) and hypercubes (factorials), the identity that a source's
dependencies add up to the interior length of its shortest paths, an explicit enumeration of all
shortest paths on tiny digraphs, and an independent library implementation."""
import itertools
import math

import numpy as np
import pytest

import graphgen as gg
import oracle


def _csr(g):
    rp, ci = g.numpy()
    return g.V, rp, ci


@pytest.mark.parametrize("n", [2, 3, 7, 30])
def test_path_closed_form(n):
    """Undirected path: vertex i lies inside every shortest path between a vertex left of it and
    one right of it, i * (n-1-i) pairs, counted in both directions."""
    V, rp, ci = _csr(gg.path(n))
    want = np.array([2.0 * i * (n - 1 - i) for i in range(n)])
    np.testing.assert_array_equal(oracle.bc(V, rp, ci), want)


@pytest.mark.parametrize("n", [1, 2, 5, 40])
def test_star_closed_form(n):
    """Undirected star: the hub is the middle of the only shortest path between any two leaves."""
    V, rp, ci = _csr(gg.star(n))
    s = oracle.bc(V, rp, ci)
    assert s[0] == n * (n - 1)
    assert np.all(s[1:] == 0.0)


def test_complete_graph_has_no_intermediates():
    V, rp, ci = _csr(gg.complete(9))
    assert np.all(oracle.bc(V, rp, ci) == 0.0)


def test_grid_path_counts_are_binomials():
    """On a full grid the shortest paths from a corner to (i, j) are the monotone lattice paths:
    C(i+j, i) of them, at depth i+j."""
    rows, cols = 9, 12
    V, rp, ci = _csr(gg.grid2d(rows, cols, drop=0.0))
    depth, sigma = oracle.bc_forward(V, rp, ci, 0)
    for i in range(rows):
        for j in range(cols):
            v = i * cols + j
            assert depth[v] == i + j
            assert sigma[v] == math.comb(i + j, i)


def test_hypercube_path_counts_are_factorials():
    """In the k-cube every shortest path from 0 to x flips the set bits of x in some order."""
    k = 7
    edges = [(x, x ^ (1 << b)) for x in range(1 << k) for b in range(k)]
    V, rp, ci = _csr(gg.from_edge_list(1 << k, edges))
    depth, sigma = oracle.bc_forward(V, rp, ci, 0)
    for x in range(1 << k):
        h = bin(x).count("1")
        assert depth[x] == h and sigma[x] == math.factorial(h)


def test_unreachable_vertices():
    V, rp, ci = _csr(gg.path(6, directed=True))
    depth, sigma = oracle.bc_forward(V, rp, ci, 3)
    assert list(depth) == [-1, -1, -1, 0, 1, 2] and list(sigma) == [0, 0, 0, 1, 1, 1]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dependencies_sum_to_interior_path_length(seed):
    """For one source s, the dependencies of all vertices add up to sum over reachable t of
    (d(s, t) - 1): each shortest s-t path has d(s, t) - 1 interior vertices, and the path
    fractions through them add up to exactly that.  Distances come from the BFS oracle."""
    V, rp, ci = _csr(gg.random_small(300, 1500, seed))
    for s in (0, 17, 111):
        d = oracle.bfs(V, rp, ci, s)
        want = float(sum(int(x) - 1 for t, x in enumerate(d) if x > 0))
        got = oracle.bc(V, rp, ci, [s]).sum()
        assert abs(got - want) <= 1e-9 * max(1.0, want)


def _brute_force_bc(V, edges):
    """Enumerate every shortest path of a tiny digraph explicitly."""
    adj = [[] for _ in range(V)]
    for u, v in edges:
        adj[u].append(v)
    score = [0.0] * V
    for s in range(V):
        for t in range(V):
            if s == t:
                continue
            # all paths s -> t of increasing length until some exist: those are the shortest
            found = []
            frontier = [[s]]
            while frontier and not found:
                nxt = []
                for p in frontier:
                    for w in adj[p[-1]]:
                        if w in p:
                            continue
                        (found if w == t else nxt).append(p + [w])
                frontier = nxt
            if not found:
                continue
            for p in found:
                for v in p[1:-1]:
                    score[v] += 1.0 / len(found)
    return np.array(score)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_enumeration(seed):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(4, 9))
    edges = sorted({(int(u), int(v)) for u, v in rng.integers(0, V, size=(3 * V, 2)) if u != v})
    g = gg.from_edge_list(V, edges)
    V_, rp, ci = _csr(g)
    np.testing.assert_allclose(oracle.bc(V_, rp, ci), _brute_force_bc(V, edges), rtol=1e-12, atol=1e-12)


def test_matches_networkx_brandes():
    nx = pytest.importorskip("networkx")
    g = gg.random_small(200, 900, 9)
    V, rp, ci = _csr(g)
    G = nx.DiGraph()
    G.add_nodes_from(range(V))
    src = np.repeat(np.arange(V), np.diff(rp))
    G.add_edges_from(zip(src.tolist(), ci.tolist()))
    ref = nx.betweenness_centrality(G, normalized=False)
    np.testing.assert_allclose(oracle.bc(V, rp, ci), [ref[v] for v in range(V)], rtol=1e-10, atol=1e-9)


def test_sources_subset_adds_up():
    """Scores are additive over sources: the all-source score is the sum of single-source ones."""
    V, rp, ci = _csr(gg.random_small(60, 240, 4))
    total = oracle.bc(V, rp, ci)
    parts = sum(oracle.bc(V, rp, ci, [s]) for s in range(V))
    np.testing.assert_allclose(total, parts, rtol=1e-12, atol=1e-12)
    assert all(x == 0 for x in itertools.islice(oracle.bc(V, rp, ci, []), 5))
