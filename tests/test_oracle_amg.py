"""Pins of the oracle's smoothed-aggregation AMG (Eq. prec2, Sec. 4) against
brute force, dense linear algebra and textbook multigrid properties."""
import numpy as np
import pytest
import scipy.sparse as sp

import gl_inputs as gi

BH3 = gi.WORKLOADS["cube128"][3]


def to_scipy(rp, ci, v, n, m=None):
    return sp.csr_matrix((v, ci, rp), shape=(n, m if m is not None else n))


def graph_adj(rp, ci, n):
    return [set(int(c) for c in ci[rp[i]:rp[i + 1]] if c != i) for i in range(n)]


def random_graph(n, deg, seed):
    g = gi.rng(seed)
    rows, cols = [], []
    for i in range(n):
        for j in g.integers(0, n, deg):
            if j != i:
                rows += [i, j]
                cols += [j, i]
    A = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n)) + sp.eye(n)
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32)


def key(oracle_mod, i):
    return (oracle_mod.hash32(i) << 32) | i


def lattice_graph(oracle_mod, dim, N):
    m = oracle_mod.Mesh(dim, N, 1.0)
    rp, ci, _ = m.khat_csr()
    return rp, ci


GRAPHS = [("lattice2", 2, 23), ("lattice3", 3, 9), ("random", 0, 400)]


@pytest.mark.parametrize("kind,dim,N", GRAPHS)
def test_aggregation_roots_are_greedy_mis2(oracle_mod, kind, dim, N):
    """Synchronous Luby rounds with fixed priorities give the lexicographically first
    maximal independent set of the distance-2 graph (Blelloch, Fineman & Shun 2012):
    brute-force greedy over nodes in descending priority must give the same roots."""
    rp, ci = lattice_graph(oracle_mod, dim, N) if kind != "random" else random_graph(N, 3, 5)
    n = len(rp) - 1
    nagg, agg = oracle_mod.aggregate(rp, ci)
    adj = graph_adj(rp, ci, n)
    n2 = [set().union(adj[i], *[adj[j] for j in adj[i]]) - {i} for i in range(n)]
    chosen = set()
    for i in sorted(range(n), key=lambda i: -key(oracle_mod, i)):
        if not (n2[i] & chosen):
            chosen.add(i)
    roots = sorted(chosen)
    assert nagg == len(roots)
    # roots get ids in ascending node order and lead their aggregate
    for a, r in enumerate(roots):
        assert agg[r] == a
    # every neighbour of a root is in the root's aggregate
    for r in roots:
        for j in adj[r]:
            assert agg[j] == agg[r]
    # the remaining nodes join the neighbouring (distance-1) aggregate with the smallest id
    first = {i: agg[i] for i in range(n) if i in chosen or (adj[i] & chosen)}
    for i in range(n):
        if i not in first:
            cands = [first[j] for j in adj[i] if j in first]
            assert cands and agg[i] == min(cands)
    # aggregates are connected
    for a in range(nagg):
        members = set(np.nonzero(agg == a)[0].tolist())
        seen, stack = {roots[a]}, [roots[a]]
        while stack:
            u = stack.pop()
            for w in adj[u]:
                if w in members and w not in seen:
                    seen.add(w)
                    stack.append(w)
        assert seen == members


@pytest.mark.parametrize("kind,dim,N", GRAPHS)
def test_jp_colouring_characterisation(oracle_mod, kind, dim, N):
    """Jones-Plassmann: a proper colouring where each node's colour is the smallest
    colour not taken by its higher-priority neighbours."""
    rp, ci = lattice_graph(oracle_mod, dim, N) if kind != "random" else random_graph(N, 3, 5)
    n = len(rp) - 1
    ncol, col = oracle_mod.color_jp(rp, ci)
    adj = graph_adj(rp, ci, n)
    assert col.min() == 0 and col.max() == ncol - 1
    for i in range(n):
        higher = {int(col[j]) for j in adj[i] if key(oracle_mod, j) > key(oracle_mod, i)}
        c = 0
        while c in higher:
            c += 1
        assert col[i] == c
        assert all(col[j] != col[i] for j in adj[i])


@pytest.mark.parametrize("kind,dim,N", GRAPHS + [("coarse3", 3, 20)])
def test_smallest_last_colouring(oracle_mod, kind, dim, N):
    """Smallest-last greedy colouring (Matula & Beck): the reversed colouring order
    removes, at every step, a vertex of minimum degree among those left; each
    colour is the smallest not taken by neighbours coloured before; the colouring
    is proper and uses at most degeneracy + 1 colours (the degeneracy counted by
    brute force)."""
    if kind == "coarse3":
        m = oracle_mod.Mesh(3, N, 1.0, BH3)
        P = oracle_mod.Precond(m, np.ones(m.n, complex), max_coarse=64, coloring=oracle_mod.COLOR_JP)
        rp, ci, _ = P.level_matrix(1)
    elif kind == "random":
        rp, ci = random_graph(N, 3, 5)
    else:
        rp, ci = lattice_graph(oracle_mod, dim, N)
    n = len(rp) - 1
    ncol, col, order = oracle_mod.color_sl(rp, ci)
    adj = graph_adj(rp, ci, n)
    assert sorted(order) == list(range(n))
    left = set(range(n))
    deg = {v: len(adj[v]) for v in range(n)}
    degeneracy = 0
    for v in order[::-1]:
        v = int(v)
        assert deg[v] == min(deg[u] for u in left), v
        degeneracy = max(degeneracy, deg[v])
        left.remove(v)
        for u in adj[v]:
            if u in left:
                deg[u] -= 1
    pos = np.empty(n, np.int64)
    pos[order] = np.arange(n)
    for v in range(n):
        before = {int(col[u]) for u in adj[v] if pos[u] < pos[v]}
        c = 0
        while c in before:
            c += 1
        assert col[v] == c
        assert all(col[u] != col[v] for u in adj[v])
    assert col.max() == ncol - 1 and ncol <= degeneracy + 1
    if kind == "coarse3":
        # fewer colours than Jones-Plassmann on a coarse AMG level
        assert ncol < oracle_mod.color_jp(rp, ci)[0]


@pytest.mark.parametrize("kind,dim,N", GRAPHS + [("coarse3", 3, 20)])
def test_round_smallest_last_colouring(oracle_mod, kind, dim, N):
    """Smallest-last colouring in removal rounds: the levels come from removing, in
    each round, every remaining vertex whose remaining degree is within the slack
    of the round's minimum (checked by a brute-force replay of the rounds); each
    colour is the smallest not taken by the neighbours that come earlier in
    decreasing (level, priority) order; proper; never more colours than
    Jones-Plassmann, and within one of the one-at-a-time smallest-last colouring
    on a coarse AMG level."""
    if kind == "coarse3":
        m = oracle_mod.Mesh(3, N, 1.0, BH3)
        P = oracle_mod.Precond(m, np.ones(m.n, complex), max_coarse=64, coloring=oracle_mod.COLOR_JP)
        rp, ci, _ = P.level_matrix(1)
    elif kind == "random":
        rp, ci = random_graph(N, 3, 5)
    else:
        rp, ci = lattice_graph(oracle_mod, dim, N)
    n = len(rp) - 1
    ncol, col, level = oracle_mod.color_psl(rp, ci)
    adj = graph_adj(rp, ci, n)
    # replay the removal rounds
    left = set(range(n))
    deg = {v: len(adj[v]) for v in range(n)}
    r = 0
    while left:
        dmin = min(deg[v] for v in left)
        out = {v for v in left if deg[v] <= dmin + oracle_mod.PSL_SLACK}
        assert {int(v) for v in np.nonzero(level == r)[0]} == out, r
        left -= out
        for v in out:
            for u in adj[v]:
                if u in left:
                    deg[u] -= 1
        r += 1
    assert level.max() == r - 1
    for v in range(n):
        kv = (int(level[v]), key(oracle_mod, v))
        earlier = {int(col[u]) for u in adj[v] if (int(level[u]), key(oracle_mod, u)) > kv}
        c = 0
        while c in earlier:
            c += 1
        assert col[v] == c
        assert all(col[u] != col[v] for u in adj[v])
    assert col.max() == ncol - 1
    assert ncol <= oracle_mod.color_jp(rp, ci)[0]
    if kind == "coarse3":
        assert ncol <= oracle_mod.color_sl(rp, ci)[0] + 1


@pytest.fixture(scope="module")
def prec2d(oracle_mod):
    m = oracle_mod.Mesh(2, 32, 1.5)
    psi = gi.disk(m.n, 1)
    P = oracle_mod.Precond(m, psi, max_coarse=40)
    return m, psi, P


@pytest.fixture(scope="module")
def prec3d(oracle_mod):
    m = oracle_mod.Mesh(3, 11, 1.0, BH3)
    psi = gi.disk(m.n, 4)
    P = oracle_mod.Precond(m, psi, max_coarse=40)
    return m, psi, P


@pytest.mark.parametrize("which", ["prec2d", "prec3d"])
def test_hierarchy_galerkin_and_hermitian(oracle_mod, which, request):
    """Level 0 is P-hat = K-hat + 2 D |psi|^2 (Eq. prec2); each coarse operator is the
    Galerkin product P^H A P (checked against dense products) and is Hermitian
    positive definite; colourings are proper; tentative columns are orthonormal."""
    m, psi, P = request.getfixturevalue(which)
    assert P.nlevels >= 3
    K = m.khat_dense()
    A0 = K + np.diag(2 * m.volumes() * np.abs(psi) ** 2)
    rp, ci, v = P.level_matrix(0)
    np.testing.assert_allclose(to_scipy(rp, ci, v, m.n).toarray(), A0, atol=1e-13)
    for l in range(P.nlevels - 1):
        info, cinfo = P.level_info(l), P.level_info(l + 1)
        A = to_scipy(*P.level_matrix(l), info["n"]).toarray()
        Pm = to_scipy(*P.level_P(l), info["n"], cinfo["n"]).toarray()
        Ac = to_scipy(*P.level_matrix(l + 1), cinfo["n"]).toarray()
        ref = Pm.conj().T @ A @ Pm
        assert np.abs(Ac - ref).max() < 1e-12 * np.abs(ref).max()
        assert np.abs(Ac - Ac.conj().T).max() == 0
        assert np.linalg.eigvalsh(Ac).min() > 0
        # P = (I - omega D^-1 A) P_tent with orthonormal tentative columns
        agg = P.aggregates(l)
        assert agg.min() == 0 and agg.max() == cinfo["n"] - 1
        d = np.real(np.diag(A))
        Pt = np.linalg.solve(np.eye(info["n"]) - info["omega"] * A / d[:, None], Pm)
        assert np.abs(Pt.conj().T @ Pt - np.eye(cinfo["n"])).max() < 1e-9
        assert np.all(np.abs(Pt[np.arange(info["n"]), agg]) > 0)
        Pt[np.arange(info["n"]), agg] = 0
        assert np.abs(Pt).max() < 1e-9
        # omega = 4 / (3 rho) with rho a lower estimate of the spectral radius of D^-1 A
        rho = np.abs(np.linalg.eigvals(A / d[:, None])).max()
        rho_est = 4.0 / (3.0 * info["omega"])
        assert 0.85 * rho <= rho_est <= rho * (1 + 1e-12)
        col = P.colors(l)
        for i, nbrs in enumerate(graph_adj(*P.level_matrix(l)[:2], info["n"])):
            assert all(col[j] != col[i] for j in nbrs)


@pytest.mark.parametrize("which", ["prec2d", "prec3d"])
def test_vcycle_symmetric_positive_definite_convergent(oracle_mod, which, request):
    """AMG_1 of a Hermitian problem is Hermitian (Sec. 4.1) and positive definite; as a
    stationary iteration it converges (error-propagation spectral radius < 1)."""
    m, psi, P = request.getfixturevalue(which)
    n = m.n
    cols = [gi.complex_normal(n, 100 + s) for s in range(4)]
    Vc = [P.vcycle(0, c) for c in cols]
    for a in range(4):
        assert np.vdot(cols[a], Vc[a]).real > 0
        for b in range(4):
            lhs, rhs = np.vdot(cols[a], Vc[b]), np.conj(np.vdot(cols[b], Vc[a]))
            assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(cols[a]) * np.linalg.norm(Vc[b])
    A = to_scipy(*P.level_matrix(0), n)
    e = gi.complex_normal(n, 7)
    rates = []
    for _ in range(12):
        e_new = e - P.vcycle(0, A @ e)
        rates.append(np.linalg.norm(e_new) / np.linalg.norm(e))
        e = e_new
    assert rates[-1] < 0.8, rates


def test_precond_is_self_adjoint_in_discrete_inner_product(oracle_mod, prec2d):
    """R_1 = AMG_1(K-hat + 2D|psi|^2, D .) is self-adjoint in <.,.>_D (Eq. prec2)."""
    m, psi, P = prec2d
    vol = m.volumes()
    x, y = gi.complex_normal(m.n, 1), gi.complex_normal(m.n, 2)
    a = np.vdot(vol * x, P.apply(y))
    b = np.vdot(vol * P.apply(x), y)
    assert abs(a - b) < 1e-12 * abs(a)


def test_single_level_is_exact_inverse(oracle_mod):
    """With one level (n <= max_coarse) R_1 is the exact P^-1 = (K-hat + 2D|psi|^2)^-1 D
    (Eq. prec1)."""
    m = oracle_mod.Mesh(2, 12, 1.0)
    psi = gi.disk(m.n, 3)
    P = oracle_mod.Precond(m, psi)
    assert P.nlevels == 1
    A0 = m.khat_dense() + np.diag(2 * m.volumes() * np.abs(psi) ** 2)
    v = gi.complex_normal(m.n, 4)
    np.testing.assert_allclose(P.apply(v), np.linalg.solve(A0, m.volumes() * v), rtol=1e-10, atol=1e-12)


def test_multigrid_factor_zero_field(oracle_mod):
    """Textbook behaviour on the A = 0, psi = 1 problem (Neumann Laplacian + 2 D): the
    two-level method contracts the energy-norm error by a factor below 1/2 that does
    not depend on h; the full V-cycle still contracts."""
    facs = []
    for N in (33, 65, 129):
        m = oracle_mod.Mesh(2, N, 0.0)
        for ml in (2, 10):
            P = oracle_mod.Precond(m, np.ones(m.n, complex), max_coarse=32, max_levels=ml)
            A = to_scipy(*P.level_matrix(0), m.n)
            e = gi.complex_normal(m.n, 11)
            for _ in range(12):
                e_new = e - P.vcycle(0, A @ e)
                f = np.sqrt(np.vdot(e_new, A @ e_new).real / np.vdot(e, A @ e).real)
                e = e_new
            if ml == 2:
                facs.append(f)
            else:
                assert f < 0.8
    assert max(facs) < 0.45, facs
    assert max(facs) - min(facs) < 0.05, facs
