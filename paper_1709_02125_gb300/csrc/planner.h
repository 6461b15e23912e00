// Tile planner: chooses (tile height, pipeline depth) for a chain. The exhaustive
// autotuner and the learned (MLP) predictor live in planner.cpp.
#pragma once

#include <cstdint>
#include <vector>

#include "oc_internal.h"

namespace oc {

// Returns true and sets (h, depth) when the planner has a choice for this chain;
// false lets the executor fall back to the fixed rule.
bool planner_choose(const std::vector<Loop>& loops, const std::vector<Dat>& dats,
                    const std::vector<int>& red_ops, uint32_t flags, long long budget, int mode,
                    int& h, int& depth);
void planner_reset();

}  // namespace oc
