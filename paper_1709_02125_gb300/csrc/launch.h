// Launch descriptors passed from the executor (runtime.cu) to the kernels.
// Plain structs: device pointers, sizes and per-launch constants only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace oc {

constexpr int kLaunchMaxArgs = 40;
constexpr int kLaunchMaxSamples = 64;

// Device view of one dataset argument inside one launch. A slow row s lives at
// slab slot  slot0 + (s - W0)  (minus S if >= S); every row a launch touches lies in
// [W0, W0 + S), so one conditional subtraction replaces the modulo. Element
// (x, yl, s) is at base + slot*row_elems + (yl + oy)*pitch + ox + x, where yl is the
// y index of a 3-D dataset (0 in 2-D).
struct DView {
    char* base;
    long long row_elems;
    long long pitch;
    int ox, oy;
    int S, W0, slot0;
    int nx, ny;        // interior extents of the two fast axes (periodic wrap)
    int periodic;      // bit 0: x wraps modulo nx, bit 1 (3-D): y wraps modulo ny
    int pad_;
};

// Per-sample addressing precomputed on the host for the lean LINCOMB / COPY kernels:
// element (x, yl) of the sample's row for launch row r is at
// p0 + yl * pitch + x + slot * row_elems, slot = sl0 + r (minus S if >= S).
struct SampleRec {
    const char* p0;
    long long row_elems;
    long long pitch;
    int S;
    int sl0;
};

struct LaunchDesc {
    int kernel;
    int ndim;
    int dtype;                 // 0 = f64, 1 = f32 (all dataset arguments share it)
    int lo[3], hi[3];          // iteration range of this launch; slow axis = this tile's rows
    int nargs;
    int npts[kLaunchMaxArgs];  // stencil points per argument
    int access[kLaunchMaxArgs];
    DView v[kLaunchMaxArgs];
    int nsamp;                 // total stencil samples of the READ arguments
    int sarg[kLaunchMaxSamples];
    int soff[kLaunchMaxSamples][3];
    const double* params;      // device pointer to this loop's parameters
    const float* paramsf;      // the same parameters rounded to float (FP32 kernels)
    int nparams;
    double* part;              // reduction partials of this loop (row part_row0 first)
    int part_row0;
    int chunks;                // partials per slow row
    int red_op;                // OC_SUM / OC_MAX / OC_MIN
    int lean;                  // 1: no argument wraps a fast axis; srec / orec are valid
    int ring;                  // 1: every slab's element offsets fit 32 bits (ring kernels)
    int o32;                   // 1: every view's slot * row_elems fits 32 bits (PDE kernels)
    int uni;                   // 1 (with o32): every dataset argument has the same fast-axis
                               //    extents, periodicity, pitch and origin (PDE kernels
                               //    then share one in-row offset per point)
    int ore;                   // output row stride in elements (ring launches)
    int sre[kLaunchMaxSamples];// sample row strides in elements (ring launches)
    SampleRec orec;            // output argument (arg 0) of LINCOMB / COPY
    SampleRec srec[kLaunchMaxSamples];
};

// Strided host-to-device copies done by SM threads that read the pinned host store
// through its device mapping (the copy engines move narrow strips -- a few bytes per
// x-line -- one line at a time). Job j copies `lines` lines of `words` 32-bit words:
// line i from src + i * pitch to dst + i * pitch.
struct StripJob {
    const char* src;
    char* dst;
    long long pitch;
    int lines;
    int words;
};
constexpr int kStripJobs = 96;
struct StripBatch {
    int njobs;
    int pad_;
    StripJob job[kStripJobs];
};
cudaError_t launch_strips(const StripBatch& b, cudaStream_t stream);

// Launch one loop tile on `stream`. Returns cudaSuccess or the launch error.
cudaError_t launch_loop(const LaunchDesc& d, cudaStream_t stream);
// Fold `n` partials of one reduction into *out (deterministic, single block).
cudaError_t launch_combine(const double* part, long long n, int op, double* out,
                           cudaStream_t stream);
// Launch a PDE kernel (Euler / Navier-Stokes ids); kernels_physics.cu.
cudaError_t launch_physics(const LaunchDesc& d, cudaStream_t stream);
int kernels_compiled_arch();
// Launch-shape tables (occupancy of the kernel instantiations); call before any capture.
void kernels_prepare();

}  // namespace oc
