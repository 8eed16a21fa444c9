// Locality reordering before encoding (host code; no CUDA call). §4.3 puts a
// dummy word wherever two consecutive columns of a row are 2^D or more apart,
// and names a locality-improving ordering of the matrix as the way to fewer
// dummies (left to future work, §7). A reordering also gathers rows of
// similar length into the same slices, which cuts SELL padding at small sigma.
//
// packsell_reorder_rcm: reverse Cuthill-McKee on the symmetrised pattern
// A + A^T. Every connected component starts from a pseudo-peripheral vertex
// (George-Liu: from a vertex of least degree, repeat a breadth-first search
// from a least-degree vertex of the last level while the number of levels
// grows); the breadth-first search appends each vertex's unvisited neighbours
// in increasing degree (ties by index); the whole order is then reversed.
// packsell_permute_csr: B = P A P^T for that order, columns sorted per row.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace packsell {
namespace {

struct Graph {
    std::vector<int64_t> start;  // [n + 1]
    std::vector<int32_t> adj;    // neighbours of v: adj[start[v] .. start[v + 1]), ascending
    int32_t degree(int32_t v) const { return (int32_t)(start[v + 1] - start[v]); }
};

// Symmetrised pattern without the diagonal: v ~ w if a_vw or a_wv is stored.
Graph symmetrise(int32_t n, const int64_t *rowptr, const int32_t *col) {
    Graph g;
    std::vector<int64_t> cnt(n + 1, 0);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q)
            if (col[q] != i) {
                ++cnt[i + 1];
                ++cnt[col[q] + 1];
            }
    for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> all(cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q)
            if (col[q] != i) {
                all[fill[i]++] = col[q];
                all[fill[col[q]]++] = i;
            }
    g.start.assign(n + 1, 0);
    g.adj.reserve(all.size());
    for (int32_t v = 0; v < n; ++v) {
        auto b = all.begin() + cnt[v], e = all.begin() + cnt[v + 1];
        std::sort(b, e);
        e = std::unique(b, e);
        g.adj.insert(g.adj.end(), b, e);
        g.start[v + 1] = (int64_t)g.adj.size();
    }
    return g;
}

// Breadth-first levels of the component of `root` among unplaced vertices;
// `mark` holds the search's stamp. Returns the number of levels and leaves
// the last level in `last`.
int bfs_levels(const Graph &g, int32_t root, const std::vector<uint8_t> &placed,
               std::vector<int64_t> &mark, int64_t stamp, std::vector<int32_t> &queue,
               std::vector<int32_t> &last) {
    queue.clear();
    queue.push_back(root);
    mark[root] = stamp;
    size_t head = 0;
    int levels = 0;
    while (head < queue.size()) {
        const size_t end = queue.size();
        last.assign(queue.begin() + head, queue.begin() + end);
        ++levels;
        for (; head < end; ++head) {
            const int32_t v = queue[head];
            for (int64_t q = g.start[v]; q < g.start[v + 1]; ++q) {
                const int32_t w = g.adj[q];
                if (!placed[w] && mark[w] != stamp) {
                    mark[w] = stamp;
                    queue.push_back(w);
                }
            }
        }
    }
    return levels;
}

int32_t least_degree(const Graph &g, const std::vector<int32_t> &vs) {
    int32_t best = vs[0];
    for (int32_t v : vs)
        if (g.degree(v) < g.degree(best) || (g.degree(v) == g.degree(best) && v < best)) best = v;
    return best;
}

}  // namespace
}  // namespace packsell

using namespace packsell;

extern "C" {

packsell_status packsell_reorder_rcm(int64_t n, const int64_t *rowptr, const int32_t *col,
                                     int32_t *perm) {
    clear_error();
    if (n < 0 || n >= (1ll << 31) || (n > 0 && (!rowptr || !col || !perm)))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_reorder_rcm: bad argument");
    if (rowptr && rowptr[0] != 0)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_reorder_rcm: rowptr[0] must be 0");
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i])
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_reorder_rcm: rowptr decreases");
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q)
            if (col[q] < 0 || col[q] >= n)
                return fail(PACKSELL_ERR_RANGE, "packsell_reorder_rcm: column out of range (the "
                                                "matrix must be square)");
    }
    try {
        const int32_t N = (int32_t)n;
        const Graph g = symmetrise(N, rowptr, col);
        std::vector<uint8_t> placed(N, 0);
        std::vector<int64_t> mark(N, -1);
        std::vector<int32_t> queue, last, nbr;
        queue.reserve(N);
        int64_t stamp = 0;
        int32_t out = 0;
        for (int32_t seed = 0; seed < N; ++seed) {
            if (placed[seed]) continue;
            if (g.degree(seed) == 0) {  // a component of one vertex
                placed[seed] = 1;
                perm[out++] = seed;
                continue;
            }
            // least-degree vertex of this component
            bfs_levels(g, seed, placed, mark, stamp++, queue, last);
            int32_t root = least_degree(g, queue);
            int levels = bfs_levels(g, root, placed, mark, stamp++, queue, last);
            for (;;) {  // pseudo-peripheral vertex
                const int32_t cand = least_degree(g, last);
                const int lv = bfs_levels(g, cand, placed, mark, stamp++, queue, last);
                if (lv <= levels) break;
                root = cand;
                levels = lv;
            }
            // Cuthill-McKee order of the component
            const int32_t first = out;
            perm[out++] = root;
            placed[root] = 1;
            for (int32_t head = first; head < out; ++head) {
                const int32_t v = perm[head];
                nbr.clear();
                for (int64_t q = g.start[v]; q < g.start[v + 1]; ++q)
                    if (!placed[g.adj[q]]) nbr.push_back(g.adj[q]);
                std::sort(nbr.begin(), nbr.end(), [&](int32_t a, int32_t b) {
                    return g.degree(a) != g.degree(b) ? g.degree(a) < g.degree(b) : a < b;
                });
                for (int32_t w : nbr) {
                    placed[w] = 1;
                    perm[out++] = w;
                }
            }
        }
        std::reverse(perm, perm + N);
    } catch (const std::bad_alloc &) {
        return fail(PACKSELL_ERR_NO_MEMORY, "packsell_reorder_rcm: host memory");
    }
    return PACKSELL_OK;
}

packsell_status packsell_permute_csr(int64_t n, const int64_t *rowptr, const int32_t *col,
                                     const void *val, int32_t val_is_f64, const int32_t *perm,
                                     int64_t *out_rowptr, int32_t *out_col, void *out_val) {
    clear_error();
    if (n < 0 || n >= (1ll << 31) ||
        (n > 0 && (!rowptr || !col || !perm || !out_rowptr || !out_col)) ||
        (val != nullptr) != (out_val != nullptr))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_permute_csr: bad argument");
    if (n == 0) {
        if (out_rowptr) out_rowptr[0] = 0;
        return PACKSELL_OK;
    }
    const size_t vb = val_is_f64 ? 8 : 4;
    try {
        std::vector<int32_t> inv(n, -1);
        for (int64_t k = 0; k < n; ++k) {
            if (perm[k] < 0 || perm[k] >= n || inv[perm[k]] >= 0)
                return fail(PACKSELL_ERR_INVALID_ARG, "packsell_permute_csr: perm is not a permutation");
            inv[perm[k]] = (int32_t)k;
        }
        std::vector<std::pair<int32_t, int64_t>> row;  // (new column, old position)
        out_rowptr[0] = 0;
        for (int64_t k = 0; k < n; ++k) {
            const int64_t i = perm[k];
            row.clear();
            for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                if (col[q] < 0 || col[q] >= n)
                    return fail(PACKSELL_ERR_RANGE, "packsell_permute_csr: column out of range");
                row.emplace_back(inv[col[q]], q);
            }
            std::sort(row.begin(), row.end());
            int64_t o = out_rowptr[k];
            for (const auto &e : row) {
                out_col[o] = e.first;
                if (val)
                    std::memcpy((char *)out_val + vb * o, (const char *)val + vb * e.second, vb);
                ++o;
            }
            out_rowptr[k + 1] = o;
        }
    } catch (const std::bad_alloc &) {
        return fail(PACKSELL_ERR_NO_MEMORY, "packsell_permute_csr: host memory");
    }
    return PACKSELL_OK;
}

}  // extern "C"
