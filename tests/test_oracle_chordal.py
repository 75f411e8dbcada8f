"""Pins of the oracle's chordal extension (oracle/chordal.py), without a GPU.

Independent checks: networkx's chordality test and maximal-clique enumeration (library routines) on
the extended pattern, closed forms (a chordal block-arrow pattern gains nothing and keeps its
cliques; a cycle C_n gains n-3 chords and has n-2 triangles), containment of every original edge,
and planted mistakes in the elimination that the checks catch.
"""

import itertools

import numpy as np
import pytest

from oracle import chordal as ch

nx = pytest.importorskip("networkx")


def graph_of(n, rows, cols):
    g = nx.Graph()
    g.add_nodes_from(range(n))
    g.add_edges_from((int(r), int(c)) for r, c in zip(rows, cols) if r != c)
    return g


def extended_graph(n, rows, cols, cliques):
    g = graph_of(n, rows, cols)
    for cl in cliques:
        g.add_edges_from(itertools.combinations(cl, 2))
    return g


def check(n, rows, cols):
    cliques, fill = ch.chordal_extension(n, rows, cols)
    g0 = graph_of(n, rows, cols)
    g = extended_graph(n, rows, cols, cliques)
    assert nx.is_chordal(g)
    # the cliques cover every vertex and every edge of the extension, and are its maximal cliques
    want = sorted(sorted(c) for c in nx.find_cliques(g))
    assert sorted(cliques) == want
    assert all(g.has_edge(*e) for e in g0.edges)
    assert g.number_of_edges() - g0.number_of_edges() == fill
    assert set(itertools.chain.from_iterable(cliques)) == set(range(n))
    return cliques, fill


def test_block_arrow_is_kept():
    from sdp_inputs import config_instance
    inst = config_instance(0)
    cliques, fill = check(inst.n, inst.pat_row, inst.pat_col)
    assert fill == 0
    assert sorted(map(tuple, cliques)) == sorted(tuple(int(v) for v in c) for c in inst.cliques)


@pytest.mark.parametrize("n", [4, 5, 9, 16])
def test_cycle_gets_n_minus_3_chords(n):
    rows = np.arange(n)
    cols = (rows + 1) % n
    r, c = np.maximum(rows, cols), np.minimum(rows, cols)
    cliques, fill = check(n, r, c)
    assert fill == n - 3
    assert len(cliques) == n - 2 and all(len(x) == 3 for x in cliques)


def test_random_patterns_against_networkx():
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = int(rng.integers(1, 30))
        dens = rng.uniform(0.02, 0.4)
        rows, cols = np.tril_indices(n, -1)
        keep = rng.random(len(rows)) < dens
        check(n, rows[keep], cols[keep])


def test_tree_and_interval_graphs_gain_nothing():
    # a path and a star are trees (chordal); an interval graph is chordal
    n = 12
    path = (np.arange(1, n), np.arange(0, n - 1))
    star = (np.arange(1, n), np.zeros(n - 1, int))
    iv = [(i, j) for i in range(n) for j in range(i) if i - j <= 3]
    for rows, cols in (path, star, (np.array([a for a, _ in iv]), np.array([b for _, b in iv]))):
        _, fill = check(n, rows, cols)
        assert fill == 0


def test_planted_mistake_is_caught(monkeypatch):
    """Dropping the children's contribution in the symbolic elimination leaves a non-chordal
    pattern on a cycle, which the networkx check catches."""
    orig = ch.symbolic_elimination

    def broken(adj, order):
        n = len(adj)
        pos = {v: i for i, v in enumerate(order)}
        higher = [None] * n
        parent = [-1] * n
        children = [[] for _ in range(n)]
        for v in order:
            h = {u for u in adj[v] if pos[u] > pos[v]}
            higher[v] = h
            if h:
                parent[v] = min(h, key=lambda u: pos[u])
                children[parent[v]].append(v)
        return higher, parent, children, [pos[v] for v in range(n)]

    monkeypatch.setattr(ch, "symbolic_elimination", broken)
    n = 6
    rows = np.arange(n)
    cols = (rows + 1) % n
    r, c = np.maximum(rows, cols), np.minimum(rows, cols)
    with pytest.raises(AssertionError):
        check(n, r, c)
    monkeypatch.setattr(ch, "symbolic_elimination", orig)
