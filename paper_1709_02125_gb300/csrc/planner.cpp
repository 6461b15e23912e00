// Tile planner: chain features, the learned (MLP) choice of tile height and pipeline
// depth, and the candidate grid shared with the exhaustive autotuner (runtime.cu).
//
// Features of a chain (inputs of the network, before standardisation):
//   0 log2(loops)   1 datasets used   2 slow-axis stencil radius   3 bytes per cell
//   4 budget / footprint   5 dimensions   6 log2(footprint bytes)   7 log2(slow rows)
// The network is a cost model of two alternatives to the fixed rule (largest fitting
// height hmax, depth 3, nothing kept resident): output k is the predicted log2(t(fixed) /
// t(alternative k)). The alternatives are candidates of the planner grid (height
// fraction, depth, residency level) named when the network is installed; by default the
// fixed tiling with a quarter and with half of the budget given to resident datasets.
// The planner keeps the fixed rule unless an alternative is predicted to be faster by
// more than kPlannerMargin, otherwise it takes the alternative with the larger gain.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "../../include/oc.h"
#include "mlp.h"
#include "planner.h"

namespace oc {

const double kGridFrac[kGridN] = {1.0, 0.75, 0.5, 0.25};
const double kResLevel[kResN] = {0.0, 0.25, 0.5, 0.75};

namespace {

struct Learned {
    bool loaded = false;
    std::vector<float> params, mean, stdv;
    PlanChoice alt[2] = {{0, 3, 1}, {0, 3, 2}};
};

Learned& learned()
{
    static Learned L;
    return L;
}

}  // namespace

void chain_features(const std::vector<Loop>& loops, const std::vector<Dat>& dats, long long budget, float f[8])
{
    std::vector<char> used(dats.size(), 0);
    int radius = 0, nd = 2, Y0 = INT_MAX, Y1 = INT_MIN;
    for (const Loop& lp : loops) {
        const int sa = lp.ndim - 1;
        nd = lp.ndim;
        Y0 = std::min(Y0, lp.lo[sa]);
        Y1 = std::max(Y1, lp.hi[sa]);
        for (const Arg& ar : lp.args) {
            if (ar.access == OC_REDUCE) continue;
            used[ar.dat] = 1;
            radius = std::max(radius, std::max(-ar.rmin[sa], ar.rmax[sa]));
        }
    }
    double nds = 0, bpc = 0, fp = 0;
    for (size_t d = 0; d < dats.size(); ++d)
        if (used[d]) {
            nds += 1;
            bpc += dats[d].esz;
            fp += (double)dats[d].bytes();
        }
    f[0] = (float)std::log2(std::max<size_t>(1, loops.size()));
    f[1] = (float)nds;
    f[2] = (float)radius;
    f[3] = (float)bpc;
    f[4] = (float)(fp > 0 ? (double)budget / fp : 1.0);
    f[5] = (float)nd;
    f[6] = (float)std::log2(std::max(1.0, fp));
    f[7] = (float)std::log2((double)std::max(1, Y1 - Y0));
}

int grid_height(int hmax, int idx) { return std::max(1, (int)std::lround(hmax * kGridFrac[idx])); }

bool planner_load(const float* params, const float* mean, const float* stdv)
{
    Learned& L = learned();
    L.params.assign(params, params + mlp_nparams());
    L.mean.assign(mean, mean + 8);
    L.stdv.assign(stdv, stdv + 8);
    L.loaded = true;
    return true;
}

bool planner_loaded() { return learned().loaded; }

void planner_set_alternatives(const PlanChoice alt[2])
{
    learned().alt[0] = alt[0];
    learned().alt[1] = alt[1];
}

void planner_alternatives(PlanChoice alt[2])
{
    alt[0] = learned().alt[0];
    alt[1] = learned().alt[1];
}

bool planner_predict(const float feat[8], PlanChoice& out)
{
    Learned& L = learned();
    if (!L.loaded) return false;
    float x[8], y[2];
    for (int k = 0; k < 8; ++k) {
        x[k] = (feat[k] - L.mean[k]) / (L.stdv[k] > 0 ? L.stdv[k] : 1.0f);
        // a chain unlike those the network was trained on: no prediction (the caller
        // falls back to the autotuner)
        if (!(std::fabs(x[k]) <= kPlannerMaxZ)) return false;
    }
    if (mlp_forward(L.params.data(), x, 1, y) != cudaSuccess) return false;
    out = kFixedChoice;
    if (std::max(y[0], y[1]) > kPlannerMargin) out = y[0] >= y[1] ? L.alt[0] : L.alt[1];
    return true;
}

void planner_reset()
{
    Learned& L = learned();
    const PlanChoice a0 = L.alt[0], a1 = L.alt[1];
    L = Learned();
    L.alt[0] = a0;
    L.alt[1] = a1;
}

}  // namespace oc
