"""The host symbolic analysis (cs_symbolic_pattern; no device) against definitions
written here: the fill pattern equals a brute-force elimination in the returned
order, every step eliminates a vertex of minimum current degree (smaller bus index
among equals) with the reference held back to the end, the elimination-tree
heights are consistent, and the block-update count is the sum over columns of
r(r+1)/2.  The 118-bus figures quoted for the study network are pinned too."""
import numpy as np
import pytest

from paper_2512_08465_gb300 import cs, synth


def _graphs():
    yield synth.case118()
    for seed, (nb, nbr) in enumerate([(9, 12), (14, 20), (30, 45), (57, 80)]):
        yield synth.make_network(nb, nbr, 3, nb // 2, 0, seed=seed)


def _eliminate(n, f, t, perm, ref):
    """Brute force: eliminating v joins its remaining neighbours into a clique.
    Returns the rows (new indices) of each column and checks the ordering rule."""
    adj = [set() for _ in range(n)]
    for a, b in zip(f, t):
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    iperm = np.empty(n, np.int64)
    iperm[perm] = np.arange(n)
    alive = set(range(n))
    cols = []
    for step, v in enumerate(perm):
        cand = [u for u in alive if u != ref or len(alive) == 1]
        dmin = min(len(adj[u]) for u in cand)
        assert len(adj[v]) == dmin and v == min(u for u in cand if len(adj[u]) == dmin), step
        nbrs = adj[v]
        cols.append(sorted(int(iperm[u]) for u in nbrs))
        for a in nbrs:
            adj[a].discard(v)
            adj[a] |= nbrs - {a}
        adj[v] = set()
        alive.discard(v)
    return cols


@pytest.mark.parametrize("k", range(5))
def test_pattern_is_the_elimination_of_its_order(k):
    net = list(_graphs())[k]
    n = net.n_bus
    r = cs.symbolic_pattern(n, net.f, net.t, net.ref_bus)
    perm = r["perm"].astype(np.int64)
    assert sorted(perm) == list(range(n)) and perm[-1] == net.ref_bus
    cols = _eliminate(n, net.f, net.t, perm, net.ref_bus)
    cp, row = r["col_ptr"], r["row"]
    for j in range(n):
        assert list(row[cp[j]:cp[j + 1]]) == cols[j], j
    iperm = np.empty(n, np.int64)
    iperm[perm] = np.arange(n)
    for a, b in zip(net.f, net.t):                     # every branch inside the pattern
        lo, hi = sorted((iperm[a], iperm[b]))
        assert hi in cols[lo]
    # elimination tree: parent = first row; heights increase strictly towards the root
    lev = r["level"]
    kids = [[] for _ in range(n)]
    for j in range(n):
        if cols[j]:
            kids[cols[j][0]].append(j)
    for j in range(n):
        assert lev[j] == (1 + max(lev[c] for c in kids[j]) if kids[j] else 0), j
    assert r["levels"] == lev.max() + 1 and r["blocks"] == cp[n]
    assert r["updates"] == sum(len(c) * (len(c) + 1) // 2 for c in cols)


def test_study_network_figures():
    net = synth.case118()
    r = cs.symbolic_pattern(net.n_bus, net.f, net.t, net.ref_bus)
    assert (r["blocks"], r["levels"], r["updates"]) == (475, 26, 1961)


def test_invalid_graphs_are_rejected():
    with pytest.raises(cs.CSError):
        cs.symbolic_pattern(3, [0, 1], [1, 1], -1)      # self loop
    with pytest.raises(cs.CSError):
        cs.symbolic_pattern(3, [0], [3], -1)            # end out of range
    with pytest.raises(cs.CSError):
        cs.symbolic_pattern(3, [0], [1], 3)             # reference out of range
    r = cs.symbolic_pattern(4, [0, 0, 1], [1, 1, 2], -1)  # parallel branch, isolated bus 3
    assert r["blocks"] == 2
