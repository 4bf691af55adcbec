// Evaluation levels of a plan (host code).
//
// An item (a triplet or quadruplet of bins) sums exactly on any grid M above
// the degree of its product of shell fields, R_a + R_b + R_c (+ R_d), where
// R_b is the largest component a mode of bin b can have; M must also exceed
// 2 R_b of each of its bins so that every shell field is free of aliasing on
// the grid.  A plan groups its items into levels: a few grids, each item on
// the smallest chosen grid it fits, chosen to minimise a work model of the
// inverse transforms (per bin and point) and the contractions (per row and
// point).
#pragma once

#include <vector>

namespace fbs {

struct LevelItem {
    int arity;  // 3 or 4
    int b[4];   // bins, ascending
    int need;   // smallest admissible grid
};

struct LevelChoice {
    std::vector<int> grids;       // level grids, ascending
    std::vector<int> item_level;  // level of every item
    std::vector<int> bin_level;   // level providing P of each bin (-1: empty bin)
    std::vector<std::vector<int>> bins;  // bins evaluated by each level, ascending
};

// Smallest even 2^a 3^b grid M > S from `grids` (ascending, the admissible
// sizes up to N); N when none is larger.
int grid_above(const std::vector<int> &grids, int S, int N);

// Levels for items over nb bins.  R[b] < 0 marks an empty bin.  With
// single_M > 0 every item and bin goes to that one grid.  `fast` lists the
// grids with compile-time-radix inverse stages (cheaper in the model);
// `per_level` is the model's fixed cost of a level (its launches), in the
// units of one contraction row over one point.  No level grid is below
// `min_grid` (rounded up to an admissible grid, at most N): a sum over fewer
// points averages the per-product rounding of the split-precision
// contraction over fewer terms.
LevelChoice choose_levels(int N, int nb, const std::vector<int> &R, std::vector<LevelItem> items,
                          int single_M, const std::vector<int> &fast, int max_levels = 4,
                          double per_level = 1e8, int min_grid = 0);

}  // namespace fbs
