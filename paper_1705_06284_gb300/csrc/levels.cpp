// Evaluation levels of a plan (host code); see levels.h.
#include "levels.h"

#include <algorithm>
#include <cmath>
#include <cstdint>

namespace fbs {

int grid_above(const std::vector<int> &grids, int S, int N) {
    for (int M : grids)
        if (M > S && M <= N) return M;
    return N;
}

namespace {

struct Sets {
    uint64_t bins[2] = {0, 0};
    std::vector<uint64_t> outer, inner;  // bitsets over nb*nb pairs
};

int popc(const std::vector<uint64_t> &v) {
    int n = 0;
    for (uint64_t w : v) n += __builtin_popcountll(w);
    return n;
}

// Work model of one level on grid M, in units of one contraction row over one
// point (~0.62 ps at 512^3): every bin is inverse transformed (4.5 units per
// point on grids with compile-time-radix stages, 12.7 otherwise); the
// tensor-core pass costs a full 128-row tile per point for every tile of
// outer pairs (~0.7 of the distinct (b, c) pairs remain after the pair cover)
// plus one unit per inner row (the single bins, and ~0.4 of the distinct
// inner pairs after the quadruplet cover); plus `per_level` for the level's
// launches (1e8 by default, about 60 us).  The weights are the measured
// per-point times of these stages at 512^3 (inverse stages 2.8 ps per bin and
// point, 7.9 ps on grids with run-time factors; 78 ps per tile and 0.66 ps per
// inner row in the contraction), rounded.
double level_cost(int M, const Sets &s, const std::vector<int> &fast, double per_level) {
    const double pts = (double)M * M * M;
    const int nbins = __builtin_popcountll(s.bins[0]) + __builtin_popcountll(s.bins[1]);
    const int outer = popc(s.outer), inner_pairs = popc(s.inner);
    const double tiles = outer > 0 ? std::ceil(0.7 * outer / 128.0) : 0.0;
    const double rows = 128.0 * tiles + (outer > 0 ? nbins + 0.4 * inner_pairs : 0.0);
    const bool f = std::find(fast.begin(), fast.end(), M) != fast.end();
    return pts * ((f ? 4.5 : 12.7) * nbins + rows) + per_level;
}

}  // namespace

LevelChoice choose_levels(int N, int nb, const std::vector<int> &R, std::vector<LevelItem> items, int single_M,
                          const std::vector<int> &fast, int max_levels, double per_level, int min_grid) {
    LevelChoice out;
    std::vector<int> admissible;
    for (int M = 8; M <= N; ++M) {
        int m = M;
        if (m % 2) continue;
        while (m % 2 == 0) m /= 2;
        while (m % 3 == 0) m /= 3;
        if (m == 1) admissible.push_back(M);
    }
    const int floor_M = min_grid > 0 ? grid_above(admissible, min_grid - 1, N) : 0;
    std::vector<int> needs;
    for (auto &it : items) {
        if (single_M > 0) it.need = single_M;
        it.need = std::max(it.need, floor_M);
        needs.push_back(it.need);
    }
    std::sort(needs.begin(), needs.end());
    needs.erase(std::unique(needs.begin(), needs.end()), needs.end());
    const int G = (int)needs.size();
    if (G <= 1) {
        out.grids = needs;
    } else {
        // per distinct need: its bins and pairs
        const size_t words = ((size_t)nb * nb + 63) / 64;
        std::vector<Sets> grp(G);
        for (auto &g : grp) {
            g.outer.assign(words, 0);
            g.inner.assign(words, 0);
        }
        for (const auto &it : items) {
            const int gi = (int)(std::lower_bound(needs.begin(), needs.end(), it.need) - needs.begin());
            Sets &g = grp[gi];
            for (int k = 0; k < it.arity; ++k) g.bins[it.b[k] >> 6] |= 1ull << (it.b[k] & 63);
            const size_t op = (size_t)it.b[it.arity - 2] * nb + it.b[it.arity - 1];
            g.outer[op >> 6] |= 1ull << (op & 63);
            if (it.arity == 4) {
                const size_t ip = (size_t)it.b[0] * nb + it.b[1];
                g.inner[ip >> 6] |= 1ull << (ip & 63);
            }
        }
        // cost of one level holding the needs (lo .. hi] on grid needs[hi]
        std::vector<std::vector<double>> span(G, std::vector<double>(G, 0.0));
        for (int lo = 0; lo < G; ++lo) {
            Sets acc;
            acc.outer.assign(words, 0);
            acc.inner.assign(words, 0);
            for (int hi = lo; hi < G; ++hi) {
                acc.bins[0] |= grp[hi].bins[0];
                acc.bins[1] |= grp[hi].bins[1];
                for (size_t w = 0; w < words; ++w) {
                    acc.outer[w] |= grp[hi].outer[w];
                    acc.inner[w] |= grp[hi].inner[w];
                }
                span[lo][hi] = level_cost(needs[hi], acc, fast, per_level);
            }
        }
        // best[k][j]: cheapest cover of needs 0..j by k levels, the last on needs[j]
        const double inf = 1e300;
        std::vector<std::vector<double>> best(max_levels + 1, std::vector<double>(G, inf));
        std::vector<std::vector<int>> from(max_levels + 1, std::vector<int>(G, -1));
        for (int j = 0; j < G; ++j) best[1][j] = span[0][j];
        for (int k = 2; k <= max_levels; ++k)
            for (int j = 0; j < G; ++j)
                for (int i = 0; i < j; ++i)
                    if (best[k - 1][i] + span[i + 1][j] < best[k][j]) {
                        best[k][j] = best[k - 1][i] + span[i + 1][j];
                        from[k][j] = i;
                    }
        int kbest = 1;
        for (int k = 2; k <= max_levels; ++k)
            if (best[k][G - 1] < best[kbest][G - 1]) kbest = k;
        for (int k = kbest, j = G - 1; k >= 1 && j >= 0; j = from[k][j], --k) out.grids.push_back(needs[j]);
        std::reverse(out.grids.begin(), out.grids.end());
    }
    auto level_of = [&](int M) {
        return (int)(std::lower_bound(out.grids.begin(), out.grids.end(), M) - out.grids.begin());
    };
    // items to levels; each bin's P from the lowest level that evaluates it
    out.item_level.resize(items.size());
    out.bin_level.assign(nb, -1);
    for (size_t i = 0; i < items.size(); ++i) {
        const int l = level_of(items[i].need);
        out.item_level[i] = l;
        for (int k = 0; k < items[i].arity; ++k) {
            int &bl = out.bin_level[items[i].b[k]];
            if (bl < 0 || l < bl) bl = l;
        }
    }
    // a non-empty bin in no item still needs P: the lowest grid above 2 R
    // (a new level when every chosen grid is too small)
    for (int b = 0; b < nb; ++b) {
        if (R[b] < 0 || out.bin_level[b] >= 0) continue;
        const int need = single_M > 0 ? single_M : std::max(floor_M, grid_above(admissible, 2 * R[b], N));
        int l = level_of(need);
        if (l == (int)out.grids.size()) {
            out.grids.push_back(need);
            // the new grid is above every other: no index shifts
        }
        out.bin_level[b] = l;
    }
    // bins of each level
    std::vector<std::vector<char>> in(out.grids.size(), std::vector<char>(nb, 0));
    for (size_t i = 0; i < items.size(); ++i)
        for (int k = 0; k < items[i].arity; ++k) in[out.item_level[i]][items[i].b[k]] = 1;
    for (int b = 0; b < nb; ++b)
        if (out.bin_level[b] >= 0) in[out.bin_level[b]][b] = 1;
    out.bins.assign(out.grids.size(), {});
    for (size_t l = 0; l < out.grids.size(); ++l)
        for (int b = 0; b < nb; ++b)
            if (in[l][b]) out.bins[l].push_back(b);
    return out;
}

}  // namespace fbs
