// Chordal extension of a sparse symmetric pattern and the maximal cliques of the extension
// (Section II.A: a non-chordal aggregate pattern is first extended to a chordal one; Section III.A
// then takes the maximal cliques as given). The paper leaves the extension to heuristics:
//   1. ordering by maximum cardinality search: vertices are numbered from the last to the first,
//      each step taking the unnumbered vertex with the most numbered neighbours (ties: smallest
//      index); elimination follows the numbers. On a chordal pattern this is a perfect elimination
//      ordering and adds nothing;
//   2. symbolic elimination: the higher neighbours of v in the extension are its own higher
//      neighbours and those of every vertex whose parent (first higher neighbour) is v, without v;
//   3. {v} with its higher neighbours is a clique of the extension, maximal unless a vertex whose
//      parent is v has one more higher neighbour. Cliques are listed in elimination order of
//      their defining vertex, vertices ascending.
#include <algorithm>
#include <set>
#include <string>
#include <vector>

#include "sdp_internal.h"

namespace cadmm {

int chordal_cliques(int n, long long nnz, const int* row, const int* col, std::vector<int>& clique_ptr,
                    std::vector<int>& clique_vtx, long long& fill, std::string& err) {
    if (n <= 0) {
        err = "n must be positive";
        return SDP_ERR_ARG;
    }
    if (nnz < 0 || (nnz > 0 && (!row || !col))) {
        err = "bad pattern arrays";
        return SDP_ERR_ARG;
    }
    // ---- undirected adjacency (CSR, sorted, no duplicates, no diagonal)
    std::vector<long long> deg(n + 1, 0);
    for (long long t = 0; t < nnz; ++t) {
        const int r = row[t], c = col[t];
        if (r < 0 || r >= n || c < 0 || c >= n) {
            err = "pattern index out of range";
            return SDP_ERR_ARG;
        }
        if (r != c) {
            deg[r + 1]++;
            deg[c + 1]++;
        }
    }
    for (int v = 0; v < n; ++v) deg[v + 1] += deg[v];
    std::vector<int> adj(deg[n]);
    {
        std::vector<long long> fp(deg.begin(), deg.end() - 1);
        for (long long t = 0; t < nnz; ++t) {
            const int r = row[t], c = col[t];
            if (r == c) continue;
            adj[fp[r]++] = c;
            adj[fp[c]++] = r;
        }
    }
    std::vector<long long> ap(n + 1, 0);
    {
        long long w = 0;
        for (int v = 0; v < n; ++v) {
            const long long lo = deg[v], hi = deg[v + 1];
            std::sort(adj.begin() + lo, adj.begin() + hi);
            ap[v] = w;
            for (long long t = lo; t < hi; ++t)
                if (t == lo || adj[t] != adj[t - 1]) adj[w++] = adj[t];
        }
        ap[n] = w;
        adj.resize(w);
    }

    // ---- 1. maximum cardinality search: buckets of unnumbered vertices by numbered-neighbour count
    std::vector<int> count(n, 0), order(n);
    std::vector<char> numbered(n, 0);
    std::vector<std::set<int>> bucket(1);
    for (int v = 0; v < n; ++v) bucket[0].insert(v);
    int top = 0;
    for (int k = n - 1; k >= 0; --k) {
        while (bucket[top].empty()) --top;
        const int v = *bucket[top].begin();
        bucket[top].erase(bucket[top].begin());
        numbered[v] = 1;
        order[k] = v;
        for (long long t = ap[v]; t < ap[v + 1]; ++t) {
            const int u = adj[t];
            if (numbered[u]) continue;
            bucket[count[u]].erase(u);
            ++count[u];
            if ((int)bucket.size() <= count[u]) bucket.resize(count[u] + 1);
            bucket[count[u]].insert(u);
            top = std::max(top, count[u]);
        }
    }
    std::vector<int> pos(n);
    for (int i = 0; i < n; ++i) pos[order[i]] = i;

    // ---- 2. symbolic elimination
    std::vector<std::vector<int>> higher(n);
    std::vector<std::vector<int>> children(n);
    std::vector<int> stamp(n, -1);
    fill = 0;
    for (int i = 0; i < n; ++i) {
        const int v = order[i];
        std::vector<int>& h = higher[v];
        stamp[v] = v;
        for (long long t = ap[v]; t < ap[v + 1]; ++t) {
            const int u = adj[t];
            if (pos[u] > i && stamp[u] != v) {
                stamp[u] = v;
                h.push_back(u);
            }
        }
        const size_t own = h.size();
        for (int c : children[v])
            for (int u : higher[c])
                if (stamp[u] != v) {
                    stamp[u] = v;
                    h.push_back(u);
                }
        fill += (long long)(h.size() - own);
        std::sort(h.begin(), h.end());
        if (!h.empty()) {
            int par = h[0];
            for (int u : h)
                if (pos[u] < pos[par]) par = u;
            children[par].push_back(v);
        }
    }

    // ---- 3. maximal cliques
    clique_ptr.assign(1, 0);
    clique_vtx.clear();
    for (int i = 0; i < n; ++i) {
        const int v = order[i];
        bool maximal = true;
        for (int c : children[v])
            if (higher[c].size() == higher[v].size() + 1) {
                maximal = false;
                break;
            }
        if (!maximal) continue;
        std::vector<int> cl(higher[v]);
        cl.push_back(v);
        std::sort(cl.begin(), cl.end());
        clique_vtx.insert(clique_vtx.end(), cl.begin(), cl.end());
        clique_ptr.push_back((int)clique_vtx.size());
    }
    return SDP_OK;
}

}  // namespace cadmm
