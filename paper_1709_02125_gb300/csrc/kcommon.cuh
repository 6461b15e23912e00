// Device helpers shared by the kernel translation units: slab addressing through a
// launch view (launch.h), periodic wrap of the fast axes, and the fixed-shape block
// fold used by every reduction.
#pragma once

#include <cuda_runtime.h>

#include "../../include/oc.h"
#include "launch.h"

namespace oc {
namespace dev {

constexpr int kThreadsX = 128;
constexpr int kRedThreads = 256;

// Programmatic dependent launch (sm_90 and later). The executor launches the kernels of a
// tile with programmatic stream serialisation, so a kernel may be launched while its
// predecessor on the stream is still running. Every such kernel calls this first: it lets
// its own successor launch at once (the successor's blocks are placed once all of this
// grid's blocks have started), then waits until the predecessor grid has completed and its
// writes are visible. Nothing is read or written before the wait, so each kernel still
// sees every earlier kernel's results. Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch switch for the above, read once by kernels_prepare (OC_PDL=0 in the environment
// turns the attribute off; the kernels are the same either way).
extern bool g_pdl;

// Launch of a tile kernel on `st` with programmatic stream serialisation.
template <typename... P, typename... A>
cudaError_t launch_tile_kernel(void (*kern)(P...), dim3 grid, int threads, cudaStream_t st, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = g_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}
// points of a slow row per reduction partial (the host's kRedChunk)
constexpr int kRedPoints = 4096;

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Slot of slow row s in the view's slab: every row a launch touches lies in
// [W0, W0 + S), so one conditional subtraction replaces the modulo.
__device__ __forceinline__ int first_slot(const DView& v, int s)
{
    int slot = v.slot0 + (s - v.W0);
    return slot >= v.S ? slot - v.S : slot;
}

// Pointer to element x of x-line yl (periodic fast axes wrap) in slot 0 of the view.
template <typename T>
__device__ __forceinline__ const T* col_ptr(const DView& v, int x, int yl)
{
    if (v.periodic & 1) x = wrap1(x, v.nx);
    if (v.periodic & 2) yl = wrap1(yl, v.ny);
    return reinterpret_cast<const T*>(v.base) + (long long)(yl + v.oy) * v.pitch + v.ox + x;
}

// Element (x, yl, s) of a view.
template <typename T>
__device__ __forceinline__ const T* elem(const DView& v, int x, int yl, int s)
{
    return col_ptr<T>(v, x, yl) + (long long)first_slot(v, s) * v.row_elems;
}

// The same element with 32-bit offset arithmetic, for launches whose views all keep
// slot * row_elems below 2^31 (LaunchDesc::o32).
template <typename T>
__device__ __forceinline__ const T* elem32(const DView& v, int x, int yl, int s)
{
    if (v.periodic & 1) x = wrap1(x, v.nx);
    if (v.periodic & 2) yl = wrap1(yl, v.ny);
    const int off = first_slot(v, s) * (int)v.row_elems + (yl + v.oy) * (int)v.pitch + v.ox + x;
    return reinterpret_cast<const T*>(v.base) + off;
}

template <typename T, bool O32 = false>
__device__ __forceinline__ T ld(const DView& v, int x, int yl, int s)
{
    return __ldg(O32 ? elem32<T>(v, x, yl, s) : elem<T>(v, x, yl, s));
}

template <typename T, bool O32 = false>
__device__ __forceinline__ void st(const DView& v, int x, int yl, int s, T val)
{
    *const_cast<T*>(O32 ? elem32<T>(v, x, yl, s) : elem<T>(v, x, yl, s)) = val;
}

template <typename T>
__device__ __forceinline__ const T* params_of(const LaunchDesc& d);
template <>
__device__ __forceinline__ const float* params_of<float>(const LaunchDesc& d) { return d.paramsf; }
template <>
__device__ __forceinline__ const double* params_of<double>(const LaunchDesc& d) { return d.params; }

__device__ __forceinline__ double red_identity(int op)
{
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    return op == OC_SUM ? 0.0 : (op == OC_MAX ? -inf : inf);
}

__device__ __forceinline__ double red_apply(int op, double a, double b)
{
    if (op == OC_SUM) return a + b;
    if (op == OC_MAX) return b > a ? b : a;
    return b < a ? b : a;
}

// Fixed-shape block fold: a fixed shuffle tree per warp, then a fixed tree over the
// warps; the result is valid in thread 0. Blocks have kRedThreads threads.
__device__ __forceinline__ double block_fold(double acc, int op)
{
    __shared__ double sm[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = red_apply(op, acc, __shfl_down_sync(0xffffffffu, acc, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = acc;
    __syncthreads();
    if (w == 0) {
        acc = l < kRedThreads / 32 ? sm[l] : red_identity(op);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) acc = red_apply(op, acc, __shfl_down_sync(0xffffffffu, acc, o));
    }
    return acc;
}

// Per-row reduction partial: the block (chunk c, row s) folds the points of its chunk
// of row s with value(x, yl, s) and stores the result at part[(s - row0) * chunks + c].
// The chunk's points are taken line by line (x fastest), so no point index is divided.
template <typename F>
__device__ __forceinline__ void row_partial(const LaunchDesc& d, F value)
{
    const int sa = d.ndim - 1;
    const int s = d.lo[sa] + (int)blockIdx.y;
    const int nxr = d.hi[0] - d.lo[0];
    const long long plane = d.ndim == 3 ? (long long)nxr * (d.hi[1] - d.lo[1]) : (long long)nxr;
    const long long q0 = (long long)blockIdx.x * kRedPoints;
    const long long q1 = q0 + kRedPoints < plane ? q0 + kRedPoints : plane;
    double acc = red_identity(d.red_op);
    if (q1 > q0) {
        const int l0 = (int)(q0 / nxr), l1 = (int)((q1 - 1) / nxr);
        for (int l = l0; l <= l1; ++l) {
            const long long lq = (long long)l * nxr;
            const int x0 = l == l0 ? (int)(q0 - lq) : 0;
            const int x1 = l == l1 ? (int)(q1 - lq) : nxr;
            const int yl = d.ndim == 3 ? d.lo[1] + l : 0;
            for (int x = x0 + (int)threadIdx.x; x < x1; x += kRedThreads)
                acc = red_apply(d.red_op, acc, value(d.lo[0] + x, yl, s));
        }
    }
    acc = block_fold(acc, d.red_op);
    if (threadIdx.x == 0) d.part[(long long)(s - d.part_row0) * d.chunks + blockIdx.x] = acc;
}

}  // namespace dev
}  // namespace oc
