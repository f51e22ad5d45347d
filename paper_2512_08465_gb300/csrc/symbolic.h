// Host symbolic analysis of the bus graph, shared by every scenario of a network.
#pragma once

#include <string>
#include <vector>

struct Symbolic {
    int n = 0;                         // buses
    std::vector<int> perm, iperm;      // new -> old, old -> new
    std::vector<int> Lcolptr, Lrow, Lcol;
    std::vector<int> Lrowptr, Lrowcol, Lrowblk;
    int nlevels = 0;
    std::vector<int> lev_ptr, lev_col;
    std::vector<int> tgt_ptr, tgt;
    std::vector<int> upd_ptr, upd_a, upd_b;
    std::vector<int> blk_br_ptr, blk_br;
    long long block_updates = 0;       // sum over targets of update pairs
};

// Minimum-degree elimination of the graph (n nodes, undirected edges f[k]-t[k],
// parallel edges allowed, self loops rejected) with node `last` (the reference
// bus, -1 for none) held back to the end, symbolic block factorisation,
// elimination-tree levels and left-looking update lists.  Returns an empty
// string on success, an error message otherwise.
std::string symbolic_analysis(int n, const std::vector<int>& f, const std::vector<int>& t, int last,
                              Symbolic& S);
