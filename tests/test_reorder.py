"""Locality reordering before encoding (host code in the library, no GPU):
reverse Cuthill-McKee and the symmetric CSR permutation. The order is not
unique (ties), so the tests check what defines it - a breadth-first search
from each component's root that appends unvisited neighbours in increasing
degree, reversed - plus exact cases (a path, components), the permutation
against numpy, and the word counts of the oracle's encoder before and after."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I
from paper_2604_13433_gb300 import packsell as ps


def _sym_adjacency(rowptr, col, n):
    adj = [set() for _ in range(n)]
    for i in range(n):
        for j in col[rowptr[i]:rowptr[i + 1]]:
            if j != i:
                adj[i].add(int(j))
                adj[int(j)].add(i)
    return adj


def _check_cuthill_mckee(perm, adj):
    """perm reversed must be a Cuthill-McKee order: components contiguous,
    each a breadth-first search from its first vertex in which every vertex's
    unvisited neighbours follow in increasing degree (ties by index)."""
    n = len(adj)
    assert sorted(perm.tolist()) == list(range(n))
    cm = perm[::-1]
    pos = np.empty(n, np.int64)
    pos[cm] = np.arange(n)
    deg = np.array([len(a) for a in adj])
    k = 0
    while k < n:
        # one component: the vertices reachable from cm[k]
        seen, stack = {int(cm[k])}, [int(cm[k])]
        while stack:
            for w in adj[stack.pop()]:
                if w not in seen:
                    seen.add(w)
                    stack.append(w)
        end = k + len(seen)
        assert set(cm[k:end].tolist()) == seen, "component not contiguous"
        # children of each vertex, in order of appearance
        prev_parent, prev_key = -1, None
        for t in range(k + 1, end):
            v = int(cm[t])
            parent = min(pos[w] for w in adj[v] if pos[w] < t)
            assert parent >= prev_parent, "not a breadth-first order"
            key = (deg[v], v)
            if parent == prev_parent:
                assert key > prev_key, "children not in increasing degree"
            prev_parent, prev_key = parent, key
        k = end


def _random_pattern(n, density, seed, isolated=()):
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        cols = set()
        if i not in isolated:
            cols = set(rng.choice(n, rng.binomial(n, density), replace=False).tolist())
            cols -= set(isolated)
        cols.add(i)
        rows.append(sorted(cols))
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], np.int32)
    return rowptr, col


@pytest.mark.parametrize("seed,density", [(1, 0.004), (2, 0.01), (3, 0.03)])
def test_rcm_is_a_cuthill_mckee_order(seed, density):
    n = 300
    rowptr, col = _random_pattern(n, density, seed, isolated=(5, 77, 299))
    perm = ps.packsell_reorder_rcm(rowptr, col)
    _check_cuthill_mckee(perm, _sym_adjacency(rowptr, col, n))


def test_rcm_path_starts_at_an_end():
    # a path with shuffled labels: the order walks it from one end (bandwidth 1)
    n = 500
    rng = np.random.default_rng(4)
    label = rng.permutation(n)
    nbr = [[] for _ in range(n)]
    for a in range(n - 1):
        u, v = label[a], label[a + 1]
        nbr[u].append(v)
        nbr[v].append(u)
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(x) for x in nbr])
    col = np.array([c for x in nbr for c in sorted(x)], np.int32)
    perm = ps.packsell_reorder_rcm(rowptr, col)
    assert perm[0] in (label[0], label[-1]) and perm[-1] in (label[0], label[-1])
    rp, cl, _ = ps.packsell_permute_csr(rowptr, col, None, perm)
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.abs(rows - cl).max() == 1


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_permute_csr_matches_numpy(dtype):
    csr = I.random_csr(400, 400, 0.02, seed=7, dtype=dtype)
    perm = np.random.default_rng(8).permutation(400).astype(np.int32)
    rp, cl, vl = ps.packsell_permute_csr(csr.rowptr, csr.col, csr.val, perm)
    dense = np.zeros((400, 400), dtype)
    dense[np.repeat(np.arange(400), np.diff(csr.rowptr)), csr.col] = csr.val
    ref = dense[perm][:, perm]
    r, c = np.nonzero(ref)
    assert np.array_equal(np.diff(rp), np.bincount(r, minlength=400))
    assert np.array_equal(cl, c.astype(np.int32))
    assert vl.dtype == dtype and np.array_equal(vl, ref[r, c])


def test_reorder_errors():
    rowptr = np.array([0, 1, 2], np.int64)
    with pytest.raises(ps.PackSELLError) as e:
        ps.packsell_reorder_rcm(rowptr, np.array([0, 2], np.int32))  # column 2 of a 2 x 2
    assert e.value.code == 4
    with pytest.raises(ps.PackSELLError) as e:
        ps.packsell_permute_csr(rowptr, np.array([0, 1], np.int32), None,
                                np.array([1, 1], np.int32))
    assert e.value.code == 1
    assert ps.packsell_reorder_rcm(np.zeros(1, np.int64), np.zeros(0, np.int32)).size == 0


def _words(rowptr, col, n, D, sigma=256):
    csr = SimpleNamespace(n=n, m=n, rowptr=rowptr, col=col, val=np.ones(col.size))
    return O.encode(csr, C=32, sigma=sigma, D=D, fmt=O.FMT_E8MY if D != 15 else O.FMT_FP16).n_words


def test_rcm_word_counts():
    """Measured on the oracle's encoder. Power-law rows: at sigma = 256 the
    order gathers rows of similar length into slices (2^16 rows: 4,022,080 ->
    2,065,472 words). 7-point grid 32^3 at D = 9 (the plane of 1,024 columns
    against 2^9, as 65,536 against 2^15 on 256^3): the diagonal level sets
    narrow part of the plane gaps (289,248 -> 275,840 words)."""
    csr = I.zipf_irregular(1 << 16, seed=0)
    perm = ps.packsell_reorder_rcm(csr.rowptr, csr.col)
    rp, cl, _ = ps.packsell_permute_csr(csr.rowptr, csr.col, None, perm)
    before, after = _words(csr.rowptr, csr.col, csr.n, 15), _words(rp, cl, csr.n, 15)
    assert (before, after) == (4_022_080, 2_065_472)
    g = I.poisson7_varcoef(32, seed=0)
    perm = ps.packsell_reorder_rcm(g.rowptr, g.col)
    rp, cl, _ = ps.packsell_permute_csr(g.rowptr, g.col, None, perm)
    assert (_words(g.rowptr, g.col, g.n, 9), _words(rp, cl, g.n, 9)) == (289_248, 275_840)


def test_reordered_system_solves_the_original():
    """The documented use: B = P A P^T, b_new = b[perm], x[perm] = x_new. With
    B x_new = b_new the scattered x solves A x = b (FP64 dense solves of a
    small SPD matrix; the product identity B x[perm] = (A x)[perm] on the
    oracle's FP64 CSR product)."""
    csr, _ = I.poisson5_varcoef(12, seed=31)
    perm = ps.packsell_reorder_rcm(csr.rowptr, csr.col)
    rp, cl, vl = ps.packsell_permute_csr(csr.rowptr, csr.col, csr.val, perm)
    B = SimpleNamespace(n=csr.n, m=csr.m, rowptr=rp, col=cl, val=vl)
    x = I.uniform(csr.n, seed=32).astype(np.float64)
    assert np.allclose(O.csr_spmv_f64(B, vl, x[perm]), O.csr_spmv_f64(csr, csr.val, x)[perm],
                       rtol=1e-14, atol=1e-14)
    dense = np.zeros((csr.n, csr.n))
    dense[np.repeat(np.arange(csr.n), np.diff(rp)), cl] = vl
    b = I.uniform(csr.n, seed=33).astype(np.float64)
    x_new = np.linalg.solve(dense, b[perm])
    xs = np.empty_like(x_new)
    xs[perm] = x_new
    A = np.zeros((csr.n, csr.n))
    A[np.repeat(np.arange(csr.n), np.diff(csr.rowptr)), csr.col] = csr.val
    assert np.allclose(A @ xs, b, rtol=1e-10, atol=1e-10)
