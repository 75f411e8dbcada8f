"""Plain CPU reference of the chordal extension and maximal-clique extraction (Section II.A,
"chordal extension"; Section III.A takes the maximal cliques of a chordal pattern as given).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by ``tests/`` and nothing else.

The paper says only that a non-chordal pattern is first extended to a chordal one by adding edges,
and that finding a minimal extension is NP-complete, so heuristics are used. The reading taken
here, written out step by step:

1. Ordering by maximum cardinality search (Tarjan and Yannakakis): vertices are numbered from the
   last to the first; each step numbers the unnumbered vertex with the most numbered neighbours
   (ties: the smallest vertex index). The elimination order is the order of the numbers, so the
   first vertex picked is eliminated last. On a chordal pattern this is a perfect elimination
   ordering and adds no edge.
2. Symbolic elimination in that order: the higher neighbours of v in the extended pattern are its
   own higher neighbours together with those of every vertex whose parent is v, without v; the
   parent of v is its first higher neighbour. The extension adds exactly the pairs that appear here
   and not in the pattern.
3. Every v gives the clique {v} ∪ higher(v) of the extension; it is maximal unless a vertex whose
   parent is v has one more higher neighbour (its clique then contains v's). Maximal cliques are
   listed in elimination order of their defining vertex, vertices ascending.
"""

from __future__ import annotations

import numpy as np


def adjacency(n: int, rows, cols) -> list:
    """Neighbour sets of the undirected graph of a symmetric pattern (diagonal dropped)."""
    adj = [set() for _ in range(n)]
    for r, c in zip(np.asarray(rows).tolist(), np.asarray(cols).tolist()):
        if r != c:
            adj[r].add(c)
            adj[c].add(r)
    return adj


def mcs_order(adj: list) -> list:
    """Elimination order from maximum cardinality search (step 1)."""
    n = len(adj)
    count = [0] * n
    numbered = [False] * n
    picked = []
    for _ in range(n):
        best, vbest = -1, -1
        for v in range(n):
            if not numbered[v] and count[v] > best:
                best, vbest = count[v], v
        numbered[vbest] = True
        picked.append(vbest)
        for u in adj[vbest]:
            if not numbered[u]:
                count[u] += 1
    return picked[::-1]


def symbolic_elimination(adj: list, order: list):
    """Higher neighbours of every vertex in the extension, and the parent of every vertex (step 2)."""
    n = len(adj)
    pos = [0] * n
    for i, v in enumerate(order):
        pos[v] = i
    higher = [None] * n
    parent = [-1] * n
    children = [[] for _ in range(n)]
    for v in order:
        h = {u for u in adj[v] if pos[u] > pos[v]}
        for ch in children[v]:
            h |= higher[ch] - {v}
        higher[v] = h
        if h:
            parent[v] = min(h, key=lambda u: pos[u])
            children[parent[v]].append(v)
    return higher, parent, children, pos


def chordal_extension(n: int, rows, cols):
    """(cliques, fill): maximal cliques of the extension (ascending vertex lists, in elimination
    order of their defining vertex) and the number of added lower pairs (step 3)."""
    adj = adjacency(n, rows, cols)
    order = mcs_order(adj)
    higher, parent, children, pos = symbolic_elimination(adj, order)
    cliques = []
    for v in order:
        if any(len(higher[ch]) == len(higher[v]) + 1 for ch in children[v]):
            continue
        cliques.append(sorted({v} | higher[v]))
    fill = sum(len(higher[v] - adj[v]) for v in range(n))
    return cliques, fill
