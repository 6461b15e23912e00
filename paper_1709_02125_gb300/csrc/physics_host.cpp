// Host-side description of the PDE kernels (filled in with the Euler and
// Navier-Stokes kernels).
#include "physics.h"

namespace oc {

bool physics_kernel_known(int) { return false; }
bool physics_kernel_reduces(int) { return false; }
bool physics_validate(const Loop&, const std::vector<Dat>&, std::string& msg)
{
    msg = "unknown kernel";
    return false;
}

}  // namespace oc
