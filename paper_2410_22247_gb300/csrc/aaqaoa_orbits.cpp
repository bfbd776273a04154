// Edge orbits for H_red, computed natively on the host (Sec. 4, Algorithm 1).
//
// The paper takes generators of Aut(G) from a third-party tool and closes the
// edge set under them breadth first. Here the generators come from this
// project's individualisation-refinement search:
//   * colour refinement to the coarsest equitable ordered partition (new
//     colours ranked by (old colour, sorted neighbour colours));
//   * a first path of individualisations (first vertex of the first
//     non-singleton cell) down to a discrete partition: the reference leaf;
//   * for every level of that path, deepest first, each sibling of the path
//     vertex not yet in its orbit (under the generators found so far) is
//     individualised and searched for a leaf that differs from the reference
//     leaf by an automorphism, pruning nodes whose cell sizes leave the path's.
// The automorphisms found (one transversal element per level of the
// stabiliser chain) generate Aut(G); each is checked to map E onto E.
// The edge classes are the orbits, on unordered edges, of the group the
// generators span (the method of Sec. 4, Algorithm 1): a breadth-first closure
// seeds a class with each unclassified edge, in the caller's edge order, and
// adds the images of its members under every generator (normalised to
// (min, max)). The seed is the
// class representative and the class size its weight. With integer edge
// weights (weighted MaxCut) refinement counts neighbours per edge weight and
// only weight-preserving automorphisms are accepted.
#include <algorithm>
#include <cstdint>
#include <deque>
#include <map>
#include <numeric>
#include <vector>

#include "aaqaoa.h"

namespace {

using Col = std::vector<int>;

struct G {
    int n;
    std::vector<std::vector<int>> adj;
    std::vector<std::vector<int>> wt;  // weight of each adjacency entry (all 1 when unweighted)
    std::vector<uint64_t> nb;          // neighbour masks (n <= 64)
    bool weighted = false;
    std::map<std::pair<int, int>, int> w;  // edge (u < v) -> weight
    Col init;  // initial vertex colours (vertex fields ranked), or empty for one colour
};

Col rank_keys(const std::vector<std::vector<int>> &keys)
{
    std::vector<int> idx(keys.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return keys[a] < keys[b]; });
    Col r(keys.size());
    int c = -1;
    for (size_t i = 0; i < idx.size(); i++) {
        if (i == 0 || keys[idx[i]] != keys[idx[i - 1]])
            c++;
        r[idx[i]] = c;
    }
    return r;
}

int count_cells(const Col &c) { return c.empty() ? 0 : *std::max_element(c.begin(), c.end()) + 1; }

Col refine(const G &g, Col col)
{
    int cells = count_cells(col);
    for (;;) {
        std::vector<std::vector<int>> sig(g.n);
        for (int v = 0; v < g.n; v++) {
            std::vector<int> s;
            if (!g.weighted) {
                s.reserve(g.adj[v].size() + 1);
                for (int u : g.adj[v])
                    s.push_back(col[u]);
                std::sort(s.begin(), s.end());
            } else {  // neighbours as (colour, edge weight) pairs, sorted
                std::vector<std::pair<int, int>> pr;
                for (size_t i = 0; i < g.adj[v].size(); i++)
                    pr.push_back({col[g.adj[v][i]], g.wt[v][i]});
                std::sort(pr.begin(), pr.end());
                for (auto &q : pr) {
                    s.push_back(q.first);
                    s.push_back(q.second);
                }
            }
            s.insert(s.begin(), col[v]);
            sig[v] = std::move(s);
        }
        Col nw = rank_keys(sig);
        const int k = count_cells(nw);
        if (k == cells)
            return nw;
        col = std::move(nw);
        cells = k;
    }
}

Col individualise(const G &g, const Col &col, int v)
{
    std::vector<std::vector<int>> keys(g.n);
    for (int u = 0; u < g.n; u++)
        keys[u] = {col[u], u == v ? 0 : 1};
    return refine(g, rank_keys(keys));
}

// members of the first (lowest colour) cell with more than one vertex
std::vector<int> target_cell(const Col &col)
{
    const int k = count_cells(col);
    std::vector<std::vector<int>> cells(k);
    for (int v = 0; v < (int)col.size(); v++)
        cells[col[v]].push_back(v);
    for (auto &c : cells)
        if (c.size() > 1)
            return c;
    return {};
}

std::vector<int> cell_sizes(const Col &col)
{
    std::vector<int> s(col.size(), 0);
    for (int c : col)
        s[c]++;
    return s;
}

bool is_automorphism(const G &g, const std::vector<int> &perm)
{
    for (int u = 0; u < g.n; u++)
        for (int v : g.adj[u])
            if (!((g.nb[perm[u]] >> perm[v]) & 1ull))
                return false;
    if (g.weighted)
        for (auto &kv : g.w) {
            const int a = perm[kv.first.first], b = perm[kv.first.second];
            if (g.w.at({std::min(a, b), std::max(a, b)}) != kv.second)
                return false;
        }
    if (!g.init.empty())
        for (int u = 0; u < g.n; u++)
            if (g.init[perm[u]] != g.init[u])
                return false;
    return true;
}

std::vector<int> orbit_ids(int n, const std::vector<std::vector<int>> &gens)
{
    std::vector<int> parent(n);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int a) {
        while (parent[a] != a) {
            parent[a] = parent[parent[a]];
            a = parent[a];
        }
        return a;
    };
    for (auto &gp : gens)
        for (int a = 0; a < n; a++) {
            const int ra = find(a), rb = find(gp[a]);
            if (ra != rb)
                parent[ra] = rb;
        }
    std::vector<int> r(n);
    for (int a = 0; a < n; a++)
        r[a] = find(a);
    return r;
}

struct Search {
    const G &g;
    Col leaf0;
    std::vector<std::vector<int>> depth_sizes;

    std::vector<int> leaf_map(const Col &leaf) const
    {
        std::vector<int> inv(g.n), perm(g.n);
        for (int v = 0; v < g.n; v++)
            inv[leaf[v]] = v;
        for (int u = 0; u < g.n; u++)
            perm[u] = inv[leaf0[u]];
        return perm;
    }

    bool run(const Col &col, int depth, std::vector<int> &out) const
    {
        if (cell_sizes(col) != depth_sizes[depth])
            return false;
        const std::vector<int> cell = target_cell(col);
        if (cell.empty()) {
            std::vector<int> p = leaf_map(col);
            if (is_automorphism(g, p)) {
                out = p;
                return true;
            }
            return false;
        }
        for (int x : cell)
            if (run(individualise(g, col, x), depth + 1, out))
                return true;
        return false;
    }
};

std::vector<std::vector<int>> generators(const G &g)
{
    std::vector<std::vector<int>> gens;
    if (g.n == 0)
        return gens;
    Col col = refine(g, g.init.empty() ? Col(g.n, 0) : g.init);
    struct Level {
        Col col;
        std::vector<int> cell;
        int v;
    };
    std::vector<Level> path;
    for (;;) {
        std::vector<int> cell = target_cell(col);
        if (cell.empty())
            break;
        path.push_back({col, cell, cell[0]});
        col = individualise(g, col, cell[0]);
    }
    Search s{g, col, {}};
    for (auto &lv : path)
        s.depth_sizes.push_back(cell_sizes(lv.col));
    s.depth_sizes.push_back(cell_sizes(col));
    for (int level = (int)path.size() - 1; level >= 0; level--) {
        const Level &lv = path[level];
        for (int w : lv.cell) {
            if (w == lv.v)
                continue;
            const std::vector<int> orb = orbit_ids(g.n, gens);
            if (orb[w] == orb[lv.v])
                continue;
            std::vector<int> p;
            if (s.run(individualise(g, lv.col, w), level + 1, p))
                gens.push_back(p);
        }
    }
    return gens;
}

// Edge orbits of the group the generators span (Sec. 4, Algorithm 1): a
// breadth-first closure of each unclassified seed edge, in the given edge
// order. Returns the number of classes.
int edge_closure(const std::vector<std::vector<int>> &gens, int num_edges, const int32_t *edges,
                 const std::map<std::pair<int, int>, int> &index, int32_t *edge_orbit, int32_t *orbit_rep,
                 int32_t *orbit_weight)
{
    std::vector<int> cls(num_edges, -1);
    int classes = 0;
    for (int seed = 0; seed < num_edges; seed++) {
        if (cls[seed] >= 0)
            continue;
        const int c = classes++;
        cls[seed] = c;
        orbit_rep[c] = seed;
        int size = 1;
        std::deque<std::pair<int, int>> q;
        int su = edges[2 * seed], sv = edges[2 * seed + 1];
        q.push_back({std::min(su, sv), std::max(su, sv)});
        while (!q.empty()) {
            const auto e = q.front();
            q.pop_front();
            for (auto &gp : gens) {
                const int a = gp[e.first], b = gp[e.second];
                auto it = index.find({std::min(a, b), std::max(a, b)});
                if (it != index.end() && cls[it->second] < 0) {
                    cls[it->second] = c;
                    size++;
                    q.push_back(it->first);
                }
            }
        }
        orbit_weight[c] = size;
    }
    for (int i = 0; i < num_edges; i++)
        edge_orbit[i] = cls[i];
    return classes;
}

}  // namespace

extern "C" int aaqaoa_edge_orbits(int n, int num_edges, const int32_t *edges, const int32_t *edge_weight,
                                  int32_t *edge_orbit, int32_t *num_orbits, int32_t *orbit_rep, int32_t *orbit_weight)
{
    if (n < 1 || n > 64 || num_edges < 0 || (num_edges > 0 && !edges) || !num_orbits ||
        (num_edges > 0 && (!edge_orbit || !orbit_rep || !orbit_weight)))
        return AAQAOA_ERR_INVALID_ARG;
    G g;
    g.n = n;
    g.adj.assign(n, {});
    g.wt.assign(n, {});
    g.nb.assign(n, 0);
    g.weighted = edge_weight != nullptr;
    std::map<std::pair<int, int>, int> index;
    for (int i = 0; i < num_edges; i++) {
        int u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v)
            return AAQAOA_ERR_INVALID_ARG;
        if (u > v)
            std::swap(u, v);
        if (!index.emplace(std::make_pair(u, v), i).second)
            return AAQAOA_ERR_INVALID_ARG;  // repeated edge
        const int wi = edge_weight ? edge_weight[i] : 1;
        if (wi < 1)
            return AAQAOA_ERR_INVALID_ARG;
        g.w[{u, v}] = wi;
        g.adj[u].push_back(v);
        g.adj[v].push_back(u);
        g.wt[u].push_back(wi);
        g.wt[v].push_back(wi);
        g.nb[u] |= 1ull << v;
        g.nb[v] |= 1ull << u;
    }
    const std::vector<std::vector<int>> gens = generators(g);
    *num_orbits = edge_closure(gens, num_edges, edges, index, edge_orbit, orbit_rep, orbit_weight);
    return AAQAOA_OK;
}

// Ising-form objectives: the same search with the distinct real couplings as
// edge-weight classes and the distinct fields as initial vertex colours, so
// only automorphisms that keep both are found; vertex orbits are numbered by
// their smallest vertex.
extern "C" int aaqaoa_ising_orbits(int n, int num_edges, const int32_t *edges, const double *edge_weight,
                                   const double *field, int32_t *edge_orbit, int32_t *num_orbits, int32_t *orbit_rep,
                                   int32_t *orbit_weight, int32_t *vertex_orbit, int32_t *num_vorbits,
                                   int32_t *vorbit_rep, int32_t *vorbit_weight)
{
    if (n < 1 || n > 64 || num_edges < 0 || (num_edges > 0 && (!edges || !edge_weight)) || !num_orbits ||
        (num_edges > 0 && (!edge_orbit || !orbit_rep || !orbit_weight)) || !vertex_orbit || !num_vorbits ||
        !vorbit_rep || !vorbit_weight)
        return AAQAOA_ERR_INVALID_ARG;
    std::vector<double> wv(edge_weight, edge_weight + num_edges);
    std::vector<double> distinct = wv;
    std::sort(distinct.begin(), distinct.end());
    distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
    G g;
    g.n = n;
    g.adj.assign(n, {});
    g.wt.assign(n, {});
    g.nb.assign(n, 0);
    g.weighted = true;
    std::map<std::pair<int, int>, int> index;
    for (int i = 0; i < num_edges; i++) {
        int u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v || !(wv[i] == wv[i]))
            return AAQAOA_ERR_INVALID_ARG;
        if (u > v)
            std::swap(u, v);
        if (!index.emplace(std::make_pair(u, v), i).second)
            return AAQAOA_ERR_INVALID_ARG;
        const int wi = 1 + (int)(std::lower_bound(distinct.begin(), distinct.end(), wv[i]) - distinct.begin());
        g.w[{u, v}] = wi;
        g.adj[u].push_back(v);
        g.adj[v].push_back(u);
        g.wt[u].push_back(wi);
        g.wt[v].push_back(wi);
        g.nb[u] |= 1ull << v;
        g.nb[v] |= 1ull << u;
    }
    if (field) {
        std::vector<std::vector<int>> keys(n);
        std::vector<double> hv(field, field + n), hd = hv;
        std::sort(hd.begin(), hd.end());
        hd.erase(std::unique(hd.begin(), hd.end()), hd.end());
        for (int u = 0; u < n; u++) {
            if (!(hv[u] == hv[u]))
                return AAQAOA_ERR_INVALID_ARG;
            keys[u] = {(int)(std::lower_bound(hd.begin(), hd.end(), hv[u]) - hd.begin())};
        }
        g.init = rank_keys(keys);
    }
    const std::vector<std::vector<int>> gens = generators(g);
    *num_orbits = edge_closure(gens, num_edges, edges, index, edge_orbit, orbit_rep, orbit_weight);
    const std::vector<int> root = orbit_ids(n, gens);
    std::map<int, int> cls;  // root -> class, in order of smallest member
    int k = 0;
    for (int u = 0; u < n; u++) {
        auto it = cls.find(root[u]);
        if (it == cls.end()) {
            it = cls.emplace(root[u], k).first;
            vorbit_rep[k] = u;
            vorbit_weight[k] = 0;
            k++;
        }
        vertex_orbit[u] = it->second;
        vorbit_weight[it->second]++;
    }
    *num_vorbits = k;
    return AAQAOA_OK;
}
