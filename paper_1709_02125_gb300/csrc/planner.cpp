// Tile planner (placeholder until the autotuner and the MLP are wired in).
#include "planner.h"

namespace oc {

bool planner_choose(const std::vector<Loop>&, const std::vector<Dat>&, const std::vector<int>&, uint32_t,
                    long long, int, int&, int&)
{
    return false;
}

void planner_reset() {}

}  // namespace oc
