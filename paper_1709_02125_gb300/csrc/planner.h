// Tile planner (planner.cpp): chain features, the candidate grid of (tile height, depth)
// shared by the exhaustive autotuner and the learned predictor.
#pragma once

#include <cstdint>
#include <vector>

#include "oc_internal.h"

namespace oc {

constexpr int kGridN = 8;
constexpr float kPlannerMargin = 0.03f;  // log2 time ratio an alternative must win by
constexpr float kPlannerMaxZ = 4.0f;     // standardised feature beyond which the network abstains
extern const double kGridFrac[kGridN];   // tile height as a fraction of the largest fitting one

void chain_features(const std::vector<Loop>& loops, const std::vector<Dat>& dats, long long budget, float f[8]);
int grid_height(int hmax, int idx);
bool planner_load(const float* params, const float* mean, const float* stdv);
bool planner_loaded();
// The learned choice (grid index, depth); false when no network is loaded.
bool planner_predict(const float feat[8], int& grid_idx, int& depth);
void planner_reset();

}  // namespace oc
