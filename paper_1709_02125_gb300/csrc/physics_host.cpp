// Host-side description of the PDE kernels (include/oc_physics.h): argument layouts,
// fixed stencils and parameter counts, checked when a loop is enqueued so that the
// tiling analysis sees exactly the reach the kernel uses.
#include <algorithm>
#include <array>
#include <string>
#include <vector>

#include "../../include/oc.h"
#include "../../include/oc_physics.h"
#include "physics.h"

namespace oc {

namespace {

using Off = std::array<int, 3>;
using Stencil = std::vector<Off>;

struct ArgSpec {
    int access;       // OC_READ / OC_WRITE / OC_RW; -1: WRITE or RW
    Stencil pts;
};

const Stencil kP0 = {{0, 0, 0}};

Stencil cross9()
{
    return {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {2, 0, 0}, {-2, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 2, 0}, {0, -2, 0}};
}

Stencil star12()
{
    Stencil s;
    for (int a = 0; a < 3; ++a)
        for (int k : {-2, -1, 1, 2}) {
            Off o = {0, 0, 0};
            o[a] = k;
            s.push_back(o);
        }
    return s;
}

void add(std::vector<ArgSpec>& v, int n, int access, const Stencil& pts)
{
    for (int i = 0; i < n; ++i) v.push_back({access, pts});
}

// Returns the expected arguments of a kernel (without a trailing REDUCE argument),
// its dimensionality, parameter count and whether it carries a reduction.
bool layout(int k, int nargs, std::vector<ArgSpec>& a, int& ndim, int& nparams, bool& reduces)
{
    reduces = false;
    switch (k) {
    case OC_K_EULER_PRIM: ndim = 2; nparams = 1; add(a, 4, OC_READ, kP0); add(a, 3, OC_WRITE, kP0); return true;
    case OC_K_EULER_FLUX: ndim = 2; nparams = 0; add(a, 7, OC_READ, kP0); add(a, 8, OC_WRITE, kP0); return true;
    case OC_K_EULER_PRED:
        ndim = 2; nparams = 2;
        add(a, 4, OC_READ, kP0);
        add(a, 4, OC_READ, {{0, 0, 0}, {1, 0, 0}});
        add(a, 4, OC_READ, {{0, 0, 0}, {0, 1, 0}});
        add(a, 4, OC_WRITE, kP0);
        return true;
    case OC_K_EULER_CORR:
        ndim = 2; nparams = 4;
        add(a, 4, OC_READ, cross9());
        add(a, 4, OC_READ, kP0);
        add(a, 4, OC_READ, {{0, 0, 0}, {-1, 0, 0}});
        add(a, 4, OC_READ, {{0, 0, 0}, {0, -1, 0}});
        add(a, 4, OC_WRITE, kP0);
        return true;
    case OC_K_EULER_DT:
        ndim = 2; nparams = 3; reduces = true;
        add(a, nargs == 9 ? 8 : 4, OC_READ, kP0);
        return true;
    case OC_K_NS_PRIM: ndim = 3; nparams = 2; add(a, 5, OC_READ, kP0); add(a, 5, OC_WRITE, kP0); return true;
    case OC_K_NS_GRAD: ndim = 3; nparams = 3; add(a, 4, OC_READ, star12()); add(a, 12, OC_WRITE, kP0); return true;
    case OC_K_NS_RHS:
        ndim = 3; nparams = 9;
        add(a, 5 + 4 + 12, OC_READ, star12());
        add(a, 5, -1, kP0);
        return true;
    case OC_K_NS_UPDATE: ndim = 3; nparams = 1; add(a, 5, OC_RW, kP0); add(a, 5, OC_READ, kP0); return true;
    case OC_K_NS_FLUX: ndim = 3; nparams = 4; add(a, 21, OC_READ, kP0); add(a, 15, OC_WRITE, kP0); return true;
    case OC_K_NS_DIV:
        ndim = 3; nparams = 5;
        for (int m = 0; m < 5; ++m)
            for (int ax = 0; ax < 3; ++ax) {
                Stencil st;
                for (int k : {-2, -1, 1, 2}) {
                    Off o = {0, 0, 0};
                    o[ax] = k;
                    st.push_back(o);
                }
                add(a, 1, OC_READ, st);
            }
        add(a, 5, -1, kP0);
        return true;
    default: return false;
    }
}

bool same_set(Stencil a, Stencil b)
{
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    return a == b;
}

}  // namespace

bool physics_kernel_known(int k)
{
    std::vector<ArgSpec> a;
    int nd, np;
    bool r;
    return layout(k, 0, a, nd, np, r);
}

bool physics_kernel_reduces(int k) { return k == OC_K_EULER_DT; }

bool physics_validate(const Loop& lp, const std::vector<Dat>&, std::string& msg)
{
    std::vector<ArgSpec> want;
    int ndim = 0, nparams = 0;
    bool reduces = false;
    const int nargs = (int)lp.args.size();
    if (!layout(lp.kernel, nargs, want, ndim, nparams, reduces)) {
        msg = "unknown kernel";
        return false;
    }
    const int expect_args = (int)want.size() + (reduces ? 1 : 0);
    if (nargs != expect_args) {
        msg = "kernel " + std::to_string(lp.kernel) + " takes " + std::to_string(expect_args) + " arguments";
        return false;
    }
    if (lp.ndim != ndim) {
        msg = "kernel " + std::to_string(lp.kernel) + " works on " + std::to_string(ndim) + "-D datasets";
        return false;
    }
    if ((int)lp.params.size() != nparams) {
        msg = "kernel " + std::to_string(lp.kernel) + " takes " + std::to_string(nparams) + " parameters";
        return false;
    }
    for (size_t j = 0; j < want.size(); ++j) {
        const Arg& ar = lp.args[j];
        const bool acc_ok = want[j].access < 0 ? (ar.access == OC_WRITE || ar.access == OC_RW)
                                               : ar.access == want[j].access;
        if (!acc_ok) {
            msg = "kernel " + std::to_string(lp.kernel) + ": argument " + std::to_string(j) + " has the wrong access mode";
            return false;
        }
        Stencil got(ar.off.begin(), ar.off.end());
        if (!same_set(got, want[j].pts)) {
            msg = "kernel " + std::to_string(lp.kernel) + ": argument " + std::to_string(j) +
                  " must carry the kernel's stencil";
            return false;
        }
    }
    if (reduces && lp.args.back().access != OC_REDUCE) {
        msg = "kernel " + std::to_string(lp.kernel) + ": last argument must be a reduction";
        return false;
    }
    if (lp.kernel == OC_K_NS_RHS || lp.kernel == OC_K_NS_DIV) {
        const int first = lp.kernel == OC_K_NS_RHS ? 21 : 15;
        const int acc0 = lp.args[first].access;
        for (int j = first + 1; j < first + 5; ++j)
            if (lp.args[j].access != acc0) {
                msg = "NS_RHS: the five dU arguments share one access mode";
                return false;
            }
    }
    return true;
}

}  // namespace oc
