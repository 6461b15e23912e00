// Host-side checks of the PDE loop kernels (Euler, Navier-Stokes): which kernel ids
// exist, which carry a reduction, and whether a loop's arguments match the kernel.
#pragma once

#include <string>
#include <vector>

#include "oc_internal.h"

namespace oc {

bool physics_kernel_known(int kernel_id);
bool physics_kernel_reduces(int kernel_id);
bool physics_validate(const Loop& lp, const std::vector<Dat>& dats, std::string& msg);

}  // namespace oc
