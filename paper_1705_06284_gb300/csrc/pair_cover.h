// Greedy pair covers for the outer rows of the tensor-core contraction
// (host code).  Pair keys are x * nb + y with x <= y.
#pragma once

#include <array>
#include <utility>
#include <vector>

namespace fbs {

// Triplets (a <= b <= c, distinct tuples): the key of the pair that carries
// each.  sum_x I_a I_b I_c is the same whichever two fields form the pair
// product; a greedy set cover (the pair carrying the most uncovered triplets
// first, ties to the smaller key) keeps the number of distinct pairs small.
std::vector<int> cover_triplet_pairs(int nb, const std::vector<std::array<int, 3>> &trip);

// Quadruplets (sorted 4-tuples): an (inner pair, outer pair) of each, one of
// its three pairings in either role, with the outer pairs together with
// `fixed` within one 128-row tile and few inner pairs.  False when no such
// assignment exists.
bool cover_quad_pairings(int nb, const std::vector<std::array<int, 4>> &q, const std::vector<int> &fixed,
                         std::vector<std::pair<int, int>> &assign);

}  // namespace fbs
