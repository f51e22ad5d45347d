// Host symbolic analysis (runs once per network in cs_load_network).
//
// The Newton matrix of every scenario of a network, reduced to one 4x4 block
// per bus, and the network admittance matrix of the small-signal model share
// the sparsity pattern of the bus graph with every branch in service (an
// outaged branch only zeroes values).  One ordering and one fill pattern
// therefore serve all contingencies:
//  * ordering: exact minimum degree on the elimination graph (ties broken by
//    the smaller bus index), computed on explicit adjacency sets, with the
//    reference bus eliminated last.  Its reduced-KKT block has the angle row
//    replaced by the identity, so without a generator at that bus the block
//    alone is singular; as the last pivot it is the Schur complement of the
//    whole system, which is nonsingular whenever the system is;
//  * pattern: the neighbours of each bus when it is eliminated are the rows of
//    its column of L;
//  * elimination tree (parent = first row of the column) and its heights; the
//    columns of one height are independent, so each height is one parallel
//    step of the numeric kernels;
//  * left-looking update lists: for target block (i, j), i >= j, every k < j
//    with L(i,k) and L(j,k) nonzero, so that A(i,j) -= L(i,k) U(j,k)^T.
#include "symbolic.h"

#include <algorithm>
#include <map>
#include <set>

std::string symbolic_analysis(int n, const std::vector<int>& f, const std::vector<int>& t, int last,
                              Symbolic& S) {
    if (n <= 0) return "network has no bus";
    if (last >= n) return "reference bus out of range";
    std::vector<std::set<int>> adj(n);
    for (size_t k = 0; k < f.size(); ++k) {
        const int a = f[k], b = t[k];
        if (a < 0 || a >= n || b < 0 || b >= n) return "branch end out of range";
        if (a == b) return "branch with both ends on one bus";
        adj[a].insert(b);
        adj[b].insert(a);
    }
    S.n = n;
    S.perm.assign(n, -1);
    S.iperm.assign(n, -1);
    std::vector<char> alive(n, 1);
    std::vector<std::vector<int>> colrows(n);   // in old indices, filled at elimination
    for (int step = 0; step < n; ++step) {
        int best = -1;
        size_t bdeg = 0;
        for (int v = 0; v < n; ++v) {
            if (!alive[v] || (v == last && step < n - 1)) continue;
            if (best < 0 || adj[v].size() < bdeg) {
                best = v;
                bdeg = adj[v].size();
            }
        }
        const int v = best;
        std::vector<int> nb(adj[v].begin(), adj[v].end());
        for (int a : nb) {
            adj[a].erase(v);
            for (int b : nb)
                if (b != a) adj[a].insert(b);
        }
        adj[v].clear();
        alive[v] = 0;
        S.perm[step] = v;
        S.iperm[v] = step;
        colrows[step] = nb;   // old indices, converted below
    }
    // CSC of L in new indices
    S.Lcolptr.assign(n + 1, 0);
    for (int j = 0; j < n; ++j) {
        std::vector<int>& r = colrows[j];
        for (int& v : r) v = S.iperm[v];
        std::sort(r.begin(), r.end());
        for (int v : r)
            if (v <= j) return "internal: fill row above the diagonal";
        S.Lcolptr[j + 1] = S.Lcolptr[j] + (int)r.size();
    }
    const int nL = S.Lcolptr[n];
    S.Lrow.resize(nL);
    S.Lcol.resize(nL);
    std::vector<std::map<int, int>> blk_of(n);   // per column: row -> block id
    for (int j = 0; j < n; ++j)
        for (int q = 0; q < (int)colrows[j].size(); ++q) {
            const int id = S.Lcolptr[j] + q;
            S.Lrow[id] = colrows[j][q];
            S.Lcol[id] = j;
            blk_of[j][colrows[j][q]] = id;
        }
    // CSR of L
    S.Lrowptr.assign(n + 1, 0);
    for (int id = 0; id < nL; ++id) S.Lrowptr[S.Lrow[id] + 1]++;
    for (int i = 0; i < n; ++i) S.Lrowptr[i + 1] += S.Lrowptr[i];
    S.Lrowcol.resize(nL);
    S.Lrowblk.resize(nL);
    {
        std::vector<int> fill(S.Lrowptr.begin(), S.Lrowptr.end() - 1);
        for (int j = 0; j < n; ++j)           // columns ascending -> rows' entries sorted by column
            for (int id = S.Lcolptr[j]; id < S.Lcolptr[j + 1]; ++id) {
                const int i = S.Lrow[id];
                S.Lrowcol[fill[i]] = j;
                S.Lrowblk[fill[i]] = id;
                fill[i]++;
            }
    }
    // elimination tree heights and levels
    std::vector<int> height(n, 0);
    for (int j = 0; j < n; ++j) {
        if (S.Lcolptr[j + 1] > S.Lcolptr[j]) {
            const int p = S.Lrow[S.Lcolptr[j]];
            height[p] = std::max(height[p], height[j] + 1);
        }
    }
    int H = 0;
    for (int j = 0; j < n; ++j) H = std::max(H, height[j] + 1);
    S.nlevels = H;
    S.lev_ptr.assign(H + 1, 0);
    for (int j = 0; j < n; ++j) S.lev_ptr[height[j] + 1]++;
    for (int h = 0; h < H; ++h) S.lev_ptr[h + 1] += S.lev_ptr[h];
    S.lev_col.resize(n);
    {
        std::vector<int> fill(S.lev_ptr.begin(), S.lev_ptr.end() - 1);
        for (int j = 0; j < n; ++j) S.lev_col[fill[height[j]]++] = j;
    }
    // factor targets per level: the diagonal of each column, then its blocks
    S.tgt_ptr.assign(H + 1, 0);
    S.tgt.clear();
    for (int h = 0; h < H; ++h) {
        for (int w = S.lev_ptr[h]; w < S.lev_ptr[h + 1]; ++w) {
            const int j = S.lev_col[w];
            S.tgt.push_back(j);
            for (int id = S.Lcolptr[j]; id < S.Lcolptr[j + 1]; ++id) S.tgt.push_back(n + id);
        }
        S.tgt_ptr[h + 1] = (int)S.tgt.size();
    }
    // left-looking update lists per target
    std::vector<std::vector<std::pair<int, int>>> upd(n + nL);
    for (int k = 0; k < n; ++k) {
        const int c0 = S.Lcolptr[k], c1 = S.Lcolptr[k + 1];
        for (int pb = c0; pb < c1; ++pb) {          // row b = j
            const int j = S.Lrow[pb];
            for (int pa = pb; pa < c1; ++pa) {      // row a = i >= j
                const int i = S.Lrow[pa];
                int target;
                if (i == j) {
                    target = j;
                } else {
                    auto it = blk_of[j].find(i);
                    if (it == blk_of[j].end()) return "internal: missing fill block";
                    target = n + it->second;
                }
                upd[target].emplace_back(pa, pb);   // A(i,j) -= L(i,k) U(j,k)^T
            }
        }
    }
    S.upd_ptr.assign(n + nL + 1, 0);
    S.upd_a.clear();
    S.upd_b.clear();
    S.block_updates = 0;
    for (int q = 0; q < n + nL; ++q) {
        for (auto& pr : upd[q]) {
            S.upd_a.push_back(pr.first);
            S.upd_b.push_back(pr.second);
        }
        S.upd_ptr[q + 1] = (int)S.upd_a.size();
        S.block_updates += (long long)upd[q].size();
    }
    // within a level, targets with similar update counts sit next to each other, so
    // that the threads sharing a warp run loops of similar length
    for (int h = 0; h < H; ++h)
        std::stable_sort(S.tgt.begin() + S.tgt_ptr[h], S.tgt.begin() + S.tgt_ptr[h + 1], [&](int x, int y) {
            return upd[x].size() > upd[y].size();
        });
    // block -> branches whose off-diagonal pair it holds
    std::vector<std::vector<int>> bb(nL);
    for (size_t k = 0; k < f.size(); ++k) {
        const int F = S.iperm[f[k]], T = S.iperm[t[k]];
        const int r = std::max(F, T), c = std::min(F, T);
        auto it = blk_of[c].find(r);
        if (it == blk_of[c].end()) return "internal: branch outside the pattern";
        bb[it->second].push_back((int)k);
    }
    S.blk_br_ptr.assign(nL + 1, 0);
    S.blk_br.clear();
    for (int q = 0; q < nL; ++q) {
        for (int b : bb[q]) S.blk_br.push_back(b);
        S.blk_br_ptr[q + 1] = (int)S.blk_br.size();
    }
    return std::string();
}
