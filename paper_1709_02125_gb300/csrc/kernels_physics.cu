// PDE loop kernels (Euler, Navier-Stokes); dispatch entry.
#include <cuda_runtime.h>

#include "launch.h"

namespace oc {

cudaError_t launch_physics(const LaunchDesc&, cudaStream_t) { return cudaErrorInvalidValue; }

}  // namespace oc
