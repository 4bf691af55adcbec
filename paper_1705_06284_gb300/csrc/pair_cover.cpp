// Greedy pair covers for the outer rows of the tensor-core contraction.
#include "pair_cover.h"

#include <algorithm>

namespace fbs {

std::vector<int> cover_triplet_pairs(int nb, const std::vector<std::array<int, 3>> &trip) {
    const int T = (int)trip.size();
    auto keys = [&](const std::array<int, 3> &tr, int *k) {  // distinct pairs of a triplet
        int n = 0;
        const int cand[3] = {tr[0] * nb + tr[1], tr[0] * nb + tr[2], tr[1] * nb + tr[2]};
        for (int j = 0; j < 3; ++j) {
            bool seen = false;
            for (int m = 0; m < n; ++m) seen |= (k[m] == cand[j]);
            if (!seen) k[n++] = cand[j];
        }
        return n;
    };
    std::vector<int> cnt((size_t)nb * nb, 0);
    std::vector<std::vector<int>> of((size_t)nb * nb);
    for (int i = 0; i < T; ++i) {
        int k[3];
        const int n = keys(trip[i], k);
        for (int m = 0; m < n; ++m) {
            of[k[m]].push_back(i);
            ++cnt[k[m]];
        }
    }
    std::vector<int> assigned(T, -1);
    int left = T;
    while (left > 0) {
        int best = -1;
        for (int q = 0; q < nb * nb; ++q)
            if (cnt[q] > 0 && (best < 0 || cnt[q] > cnt[best])) best = q;
        for (int i : of[best]) {
            if (assigned[i] >= 0) continue;
            assigned[i] = best;
            --left;
            int k[3];
            const int n = keys(trip[i], k);
            for (int m = 0; m < n; ++m) --cnt[k[m]];
        }
    }
    return assigned;
}

// Quadruplet pairings: sum_x I_a I_b I_c I_d is the same for the three
// pairings {ab, cd}, {ac, bd}, {ad, bc} and either pair as the inner row.
// cover_quad_pairings picks, for every quadruplet (sorted 4-tuples q), an
// (inner pair, outer pair) so that the outer pairs, together with the
// triplets' outer pairs `fixed`, fill at most one 128-row tile and the inner
// pairs are few: the outer set first takes pairs until every quadruplet can
// be served (greedy), then the pairs that can serve the most quadruplets up
// to the tile; a greedy set cover then chooses the inner pairs.  Pair keys
// are x * nb + y with x <= y.  Returns false when no assignment fits.
bool cover_quad_pairings(int nb, const std::vector<std::array<int, 4>> &q, const std::vector<int> &fixed,
                         std::vector<std::pair<int, int>> &assign) {
    const int P = nb * nb;
    auto options = [&](const std::array<int, 4> &t, std::pair<int, int> *o) {  // distinct (inner, outer)
        const int pr[3][4] = {{t[0], t[1], t[2], t[3]}, {t[0], t[2], t[1], t[3]}, {t[0], t[3], t[1], t[2]}};
        int n = 0;
        for (int k = 0; k < 3; ++k) {
            const int u = pr[k][0] * nb + pr[k][1], v = pr[k][2] * nb + pr[k][3];
            const std::pair<int, int> cand[2] = {{u, v}, {v, u}};
            for (const auto &c : cand) {
                bool seen = false;
                for (int m = 0; m < n; ++m) seen |= (o[m] == c);
                if (!seen) o[n++] = c;
            }
        }
        return n;
    };
    std::vector<char> in_o(P, 0);
    int no = 0;
    for (int f : fixed)
        if (!in_o[f]) { in_o[f] = 1; ++no; }
    std::vector<int> useful(P, 0);
    for (const auto &t : q) {
        std::pair<int, int> o[6];
        const int n = options(t, o);
        std::vector<int> outs;
        for (int m = 0; m < n; ++m)
            if (std::find(outs.begin(), outs.end(), o[m].second) == outs.end()) outs.push_back(o[m].second);
        for (int v : outs) ++useful[v];
    }
    // outer pairs until every quadruplet can be served (greedy cover by
    // outer pairs), then the most useful pairs up to one tile
    {
        const int Q0 = (int)q.size();
        std::vector<char> served(Q0, 0);
        int unserved = 0;
        std::vector<std::vector<int>> outs_of(Q0);
        for (int i = 0; i < Q0; ++i) {
            std::pair<int, int> o[6];
            const int n = options(q[i], o);
            for (int m = 0; m < n; ++m)
                if (std::find(outs_of[i].begin(), outs_of[i].end(), o[m].second) == outs_of[i].end())
                    outs_of[i].push_back(o[m].second);
            for (int v : outs_of[i]) served[i] |= in_o[v];
            unserved += !served[i];
        }
        while (unserved > 0) {
            std::vector<int> c(P, 0);
            for (int i = 0; i < Q0; ++i)
                if (!served[i])
                    for (int v : outs_of[i]) ++c[v];
            int best = (int)(std::max_element(c.begin(), c.end()) - c.begin());
            in_o[best] = 1;
            ++no;
            for (int i = 0; i < Q0; ++i)
                if (!served[i] && std::find(outs_of[i].begin(), outs_of[i].end(), best) != outs_of[i].end()) {
                    served[i] = 1;
                    --unserved;
                }
        }
        if (no > 128) return false;
    }
    std::vector<int> order(P);
    for (int i = 0; i < P; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return useful[x] > useful[y]; });
    for (int v : order) {
        if (no >= 128 || useful[v] == 0) break;
        if (!in_o[v]) { in_o[v] = 1; ++no; }
    }
    // greedy cover of the quadruplets by inner pairs whose partner is in the outer set
    const int Q = (int)q.size();
    std::vector<int> cnt(P, 0);
    std::vector<std::vector<int>> of(P);
    for (int i = 0; i < Q; ++i) {
        std::pair<int, int> o[6];
        const int n = options(q[i], o);
        bool any = false;
        for (int m = 0; m < n; ++m)
            if (in_o[o[m].second]) {
                any = true;
                if (of[o[m].first].empty() || of[o[m].first].back() != i) {
                    of[o[m].first].push_back(i);
                    ++cnt[o[m].first];
                }
            }
        if (!any) return false;
    }
    assign.assign(Q, {-1, -1});
    int left = Q;
    while (left > 0) {
        int best = -1;
        for (int u = 0; u < P; ++u)
            if (cnt[u] > 0 && (best < 0 || cnt[u] > cnt[best])) best = u;
        if (best < 0) return false;
        for (int i : of[best]) {
            if (assign[i].first >= 0) continue;
            std::pair<int, int> o[6];
            const int n = options(q[i], o);
            for (int m = 0; m < n; ++m)
                if (o[m].first == best && in_o[o[m].second]) {
                    assign[i] = o[m];
                    break;
                }
            --left;
            std::vector<int> seen;
            for (int m = 0; m < n; ++m)
                if (in_o[o[m].second] && std::find(seen.begin(), seen.end(), o[m].first) == seen.end()) {
                    seen.push_back(o[m].first);
                    --cnt[o[m].first];
                }
        }
    }
    return true;
}

}  // namespace fbs
