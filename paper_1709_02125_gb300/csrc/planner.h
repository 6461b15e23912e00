// Tile planner (planner.cpp): chain features, the candidate grid of (tile height, depth)
// shared by the exhaustive autotuner and the learned predictor.
#pragma once

#include <cstdint>
#include <vector>

#include "oc_internal.h"

namespace oc {

constexpr int kGridN = 4;
constexpr int kResN = 4;
constexpr float kPlannerMargin = 0.03f;  // log2 time ratio an alternative must win by
constexpr float kPlannerMaxZ = 4.0f;     // standardised feature beyond which the network abstains
extern const double kGridFrac[kGridN];   // tile height as a fraction of the largest fitting one
extern const double kResLevel[kResN];    // share of the budget for datasets kept resident

// One candidate of the planner grid: tile height hmax * kGridFrac[grid], pipeline depth,
// residency level kResLevel[res].
struct PlanChoice {
    int grid = 0, depth = 3, res = 0;
};
// The fixed rule (the method without a planner): largest fitting height, depth 3, no
// dataset kept resident.
constexpr PlanChoice kFixedChoice{0, 3, 0};

void chain_features(const std::vector<Loop>& loops, const std::vector<Dat>& dats, long long budget, float f[8]);
int grid_height(int hmax, int idx);
bool planner_load(const float* params, const float* mean, const float* stdv);
bool planner_loaded();
// The two alternatives to the fixed rule whose gains the network predicts.
void planner_set_alternatives(const PlanChoice alt[2]);
void planner_alternatives(PlanChoice alt[2]);
// The learned choice; false when no network is loaded or the chain lies outside the
// network's training features.
bool planner_predict(const float feat[8], PlanChoice& out);
void planner_reset();

}  // namespace oc
