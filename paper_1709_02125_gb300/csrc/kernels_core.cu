// Generic stencil-loop kernels of the executor: COPY, LINCOMB, REDUCE (with the
// deterministic partial combine) and the compensated HILO_ADD update.
//
// arXiv 1709.02125, Sec. 3: a parallel loop applies a kernel at every point of its
// range; points are independent, so each thread owns one x column and R consecutive
// slow rows of the tile. Datasets are read through their cyclic slab (launch.h):
// the slot of a row is advanced with one compare-and-subtract per row, never a
// modulo. x is the fastest axis, so a warp reads 32 consecutive elements of one
// x-line (coalesced); rows of neighbouring samples are shared through L1/L2.
//
// Arithmetic follows the evaluation order stated in include/oc.h for every point.
// The library is compiled with -fmad=false, so the only fused multiply-adds are the
// explicit ones (__fma_rn) that the stated order allows; a tiled and an untiled run
// execute the same instructions per point and agree bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <type_traits>

#include "../../include/oc.h"
#include "kcommon.cuh"
#include "launch.h"

namespace oc {

namespace {

using namespace dev;
constexpr int kRows = 4;

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }

// Division of the LINCOMB nonlinear term: IEEE for FP64; for FP32 the fast division
// (at most 2 ulp), the FP32 form's error budget being far larger.
__device__ __forceinline__ double nl_div(double a, double b) { return a / b; }
__device__ __forceinline__ float nl_div(float a, float b) { return __fdividef(a, b); }


// One stencil sample m for the R rows of this thread: load, then accumulate.
template <typename T, int R>
__device__ __forceinline__ void lincomb_sample(const LaunchDesc& d, const T* cp, int m, int x, int yl,
                                               int s0, int shi, T (&acc)[R], T (&x0)[R], T (&x1)[R],
                                               T (&x2)[R])
{
    const int sa = d.ndim - 1;
    const DView& v = d.v[d.sarg[m]];
    const T c = cp[1 + m];
    const T* col = col_ptr<T>(v, x + d.soff[m][0], yl + (d.ndim == 3 ? d.soff[m][1] : 0));
    int slot = first_slot(v, s0 + d.soff[m][sa]);
    T val[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        val[r] = T(0);
        if (s0 + r < shi) val[r] = __ldg(col + (long long)slot * v.row_elems);
        if (++slot == v.S) slot = 0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (m == 0) { acc[r] = c * val[r]; x0[r] = val[r]; }
        else {
            acc[r] = fma_t(c, val[r], acc[r]);
            if (m == 1) x1[r] = val[r];
            if (m == 2) x2[r] = val[r];
        }
    }
}

// LINCOMB (include/oc.h): acc = c0 x0, acc = c_m x_m + acc (fused), then the bounded
// nonlinear term. M > 0: the sample count is a compile-time constant, so the loop is
// fully unrolled and all R*M loads of a thread are independent; M == 0: any count.
template <typename T, int R, int M>
__global__ void __launch_bounds__(kThreadsX) k_lincomb(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    const int x = d.lo[0] + blockIdx.x * kThreadsX + threadIdx.x;
    if (x >= d.hi[0]) return;
    const int sa = d.ndim - 1;
    const int yl = d.ndim == 3 ? d.lo[1] + (int)blockIdx.y : 0;
    const int s0 = d.lo[sa] + (int)blockIdx.z * R;
    const int shi = d.hi[sa];
    const int nM = M > 0 ? M : d.nsamp;
    const T* cp = params_of<T>(d);

    T acc[R], x0[R], x1[R], x2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { acc[r] = T(0); x0[r] = x1[r] = x2[r] = T(0); }
    if (M > 0) {
#pragma unroll
        for (int m = 0; m < M; ++m) lincomb_sample<T, R>(d, cp, m, x, yl, s0, shi, acc, x0, x1, x2);
    } else {
#pragma unroll 1
        for (int m = 0; m < nM; ++m) lincomb_sample<T, R>(d, cp, m, x, yl, s0, shi, acc, x0, x1, x2);
    }
    const T alpha = cp[0];
    if (alpha != T(0)) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T a = x0[r];
            const T b = nM > 1 ? x1[r] : x0[r];
            const T c = nM > 2 ? x2[r] : x0[r];
            acc[r] = acc[r] + nl_div((alpha * a) * b, T(1) + c * c);
        }
    }
    const DView& o = d.v[0];
    T* ocol = const_cast<T*>(col_ptr<T>(o, x, yl));
    int slot = first_slot(o, s0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (s0 + r < shi) ocol[(long long)slot * o.row_elems] = acc[r];
        if (++slot == o.S) slot = 0;
    }
}

// Lean LINCOMB: the same samples in the same order as k_lincomb, but every sample's
// addressing (row base of x = 0, slab slot of the launch's first row) comes precomputed
// from the host (launch.h SampleRec), so a sample costs a few integer operations per
// row. Each thread takes one x column and R rows; full row groups skip the row guard.
template <typename T, int R, int M>
__global__ void __launch_bounds__(kThreadsX) k_lincomb_lean(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    const int x = d.lo[0] + blockIdx.x * kThreadsX + threadIdx.x;
    if (x >= d.hi[0]) return;
    const int sa = d.ndim - 1;
    const long long yl = d.ndim == 3 ? d.lo[1] + (int)blockIdx.y : 0;
    const int r0 = (int)blockIdx.z * R;
    const int nr = d.hi[sa] - d.lo[sa] - r0;
    const T* cp = params_of<T>(d);

    T acc[R], x0[R], x1[R], x2[R];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const SampleRec& sr = d.srec[m];
        const T c = cp[1 + m];
        const T* p = reinterpret_cast<const T*>(sr.p0) + yl * sr.pitch + x;
        int slot = sr.sl0 + r0;
        if (slot >= sr.S) slot -= sr.S;
        T val[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int sl = slot + r >= sr.S ? slot + r - sr.S : slot + r;
            val[r] = (R <= nr || r < nr) ? __ldg(p + (long long)sl * sr.row_elems) : T(0);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (m == 0) { acc[r] = c * val[r]; x0[r] = val[r]; }
            else {
                acc[r] = fma_t(c, val[r], acc[r]);
                if (m == 1) x1[r] = val[r];
                if (m == 2) x2[r] = val[r];
            }
        }
    }
    const T alpha = cp[0];
    if (alpha != T(0)) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T a = x0[r];
            const T b = M > 1 ? x1[r] : x0[r];
            const T c = M > 2 ? x2[r] : x0[r];
            acc[r] = acc[r] + nl_div((alpha * a) * b, T(1) + c * c);
        }
    }
    const SampleRec& o = d.orec;
    T* op = const_cast<T*>(reinterpret_cast<const T*>(o.p0)) + yl * o.pitch + x;
    int slot = o.sl0 + r0;
    if (slot >= o.S) slot -= o.S;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int sl = slot + r >= o.S ? slot + r - o.S : slot + r;
        if (R <= nr || r < nr) op[(long long)sl * o.row_elems] = acc[r];
    }
}

// Row of a block-row window in a cyclic slab with 32-bit element offsets. `rel` is the
// slot of the window's first row; rows r >= S - rel wrap to the slab start. The wrap
// test is uniform over the block, so only the one window per slab that straddles the
// slab end takes the per-row select.
template <typename T, int R>
__device__ __forceinline__ void ring_rows(const T* base, int sl0, int r0, int S, int re, int nr, T (&val)[R])
{
    int rel = sl0 + r0;
    if (rel >= S) rel -= S;
    const T* q = base + rel * re;
    const int w = S - rel;
    if (w >= R) {
#pragma unroll
        for (int r = 0; r < R; ++r) val[r] = (R <= nr || r < nr) ? __ldg(q + r * re) : T(0);
    } else {
        const int sre = S * re;
#pragma unroll
        for (int r = 0; r < R; ++r)
            val[r] = (R <= nr || r < nr) ? __ldg(q + (r * re - (r >= w ? sre : 0))) : T(0);
    }
}

// LINCOMB with ring addressing (launch.h: `ring`): the samples and their order are
// those of k_lincomb; each sample's rows come from ring_rows.
template <typename T, int R, int M>
__global__ void __launch_bounds__(kThreadsX) k_lincomb_ring(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    const int x = d.lo[0] + blockIdx.x * kThreadsX + threadIdx.x;
    if (x >= d.hi[0]) return;
    const int sa = d.ndim - 1;
    const long long yl = d.ndim == 3 ? d.lo[1] + (int)blockIdx.y : 0;
    const int r0 = (int)blockIdx.z * R;
    const int nr = d.hi[sa] - d.lo[sa] - r0;
    const T* cp = params_of<T>(d);

    T acc[R], x0[R], x1[R], x2[R];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const SampleRec& sr = d.srec[m];
        const T c = cp[1 + m];
        const T* p = reinterpret_cast<const T*>(sr.p0) + yl * sr.pitch + x;
        T val[R];
        ring_rows<T, R>(p, sr.sl0, r0, sr.S, d.sre[m], nr, val);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (m == 0) { acc[r] = c * val[r]; x0[r] = val[r]; }
            else {
                acc[r] = fma_t(c, val[r], acc[r]);
                if (m == 1) x1[r] = val[r];
                if (m == 2) x2[r] = val[r];
            }
        }
    }
    const T alpha = cp[0];
    if (alpha != T(0)) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T a = x0[r];
            const T b = M > 1 ? x1[r] : x0[r];
            const T c = M > 2 ? x2[r] : x0[r];
            acc[r] = acc[r] + nl_div((alpha * a) * b, T(1) + c * c);
        }
    }
    const SampleRec& od = d.orec;
    T* op = const_cast<T*>(reinterpret_cast<const T*>(od.p0)) + yl * od.pitch + x;
    int rel = od.sl0 + r0;
    if (rel >= od.S) rel -= od.S;
    const int re = d.ore;
    T* q = op + rel * re;
    const int w = od.S - rel;
    const int sre = od.S * re;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (R <= nr || r < nr) q[r * re - (r >= w ? sre : 0)] = acc[r];
}

template <typename T, int R>
__global__ void __launch_bounds__(kThreadsX) k_copy_lean(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    const int x = d.lo[0] + blockIdx.x * kThreadsX + threadIdx.x;
    if (x >= d.hi[0]) return;
    const int sa = d.ndim - 1;
    const long long yl = d.ndim == 3 ? d.lo[1] + (int)blockIdx.y : 0;
    const int r0 = (int)blockIdx.z * R;
    const int nr = d.hi[sa] - d.lo[sa] - r0;
    const SampleRec& sr = d.srec[0];
    const SampleRec& o = d.orec;
    const T* p = reinterpret_cast<const T*>(sr.p0) + yl * sr.pitch + x;
    T* op = const_cast<T*>(reinterpret_cast<const T*>(o.p0)) + yl * o.pitch + x;
    int si = sr.sl0 + r0, so = o.sl0 + r0;
    if (si >= sr.S) si -= sr.S;
    if (so >= o.S) so -= o.S;
    T val[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int sl = si + r >= sr.S ? si + r - sr.S : si + r;
        val[r] = (R <= nr || r < nr) ? __ldg(p + (long long)sl * sr.row_elems) : T(0);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int sl = so + r >= o.S ? so + r - o.S : so + r;
        if (R <= nr || r < nr) op[(long long)sl * o.row_elems] = val[r];
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(kThreadsX) k_copy(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    const int x = d.lo[0] + blockIdx.x * kThreadsX + threadIdx.x;
    if (x >= d.hi[0]) return;
    const int sa = d.ndim - 1;
    const int yl = d.ndim == 3 ? d.lo[1] + (int)blockIdx.y : 0;
    const int s0 = d.lo[sa] + (int)blockIdx.z * R;
    const int shi = d.hi[sa];
    const DView& v = d.v[1];
    const T* col = col_ptr<T>(v, x + d.soff[0][0], yl + (d.ndim == 3 ? d.soff[0][1] : 0));
    int slot = first_slot(v, s0 + d.soff[0][sa]);
    T val[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        val[r] = T(0);
        if (s0 + r < shi) val[r] = __ldg(col + (long long)slot * v.row_elems);
        if (++slot == v.S) slot = 0;
    }
    const DView& o = d.v[0];
    T* ocol = const_cast<T*>(col_ptr<T>(o, x, yl));
    slot = first_slot(o, s0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (s0 + r < shi) ocol[(long long)slot * o.row_elems] = val[r];
        if (++slot == o.S) slot = 0;
    }
}

// (hi, lo) += (float)scale * du, compensated (TwoSum, then Fast2Sum renormalisation).
template <int R>
__global__ void __launch_bounds__(kThreadsX) k_hilo_add(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    const int x = d.lo[0] + blockIdx.x * kThreadsX + threadIdx.x;
    if (x >= d.hi[0]) return;
    const int sa = d.ndim - 1;
    const int yl = d.ndim == 3 ? d.lo[1] + (int)blockIdx.y : 0;
    const int s0 = d.lo[sa] + (int)blockIdx.z * R;
    const int shi = d.hi[sa];
    const float scale = d.paramsf[0];
    float* hp = const_cast<float*>(col_ptr<float>(d.v[0], x, yl));
    float* lp = const_cast<float*>(col_ptr<float>(d.v[1], x, yl));
    const float* up = col_ptr<float>(d.v[2], x, yl);
    int sh = first_slot(d.v[0], s0), sl = first_slot(d.v[1], s0), su = first_slot(d.v[2], s0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (s0 + r < shi) {
            const long long ih = (long long)sh * d.v[0].row_elems;
            const long long il = (long long)sl * d.v[1].row_elems;
            const float hi = hp[ih], lo = lp[il];
            const float y = scale * __ldg(up + (long long)su * d.v[2].row_elems);
            const float s = hi + y;
            const float z = s - hi;
            const float e = (hi - (s - z)) + (y - z);
            const float l = lo + e;
            const float h2 = s + l;
            hp[ih] = h2;
            lp[il] = l - (h2 - s);
        }
        if (++sh == d.v[0].S) sh = 0;
        if (++sl == d.v[1].S) sl = 0;
        if (++su == d.v[2].S) su = 0;
    }
}

template <typename T> struct VecOf;
template <> struct VecOf<float> { using V = float4; static constexpr int N = 4; };
template <> struct VecOf<double> { using V = double2; static constexpr int N = 2; };

__device__ __forceinline__ double red_mode(double v, int mode)
{
    return mode == 1 ? fabs(v) : (mode == 2 ? v * v : v);
}

// Per-thread accumulators of a REDUCE (value v, mode 0: v, 1: |v|, 2: v * v).
// FP64: every term folded in FP64.
struct RedAccD {
    double a;
    __device__ __forceinline__ void init(int op) { a = red_identity(op); }
    __device__ __forceinline__ void add(int op, int mode, double v) { a = red_apply(op, a, red_mode(v, mode)); }
    __device__ __forceinline__ void add2(int op, int mode, double u, double v) { add(op, mode, u + v); }
    __device__ __forceinline__ double value(int, int) const { return a; }
};

// FP32 data without FP64 arithmetic per element (GB300's FP64 rate is a small fraction
// of its FP32 rate). A sum is kept as an unevaluated FP32 pair s + c: every term goes in
// by Knuth's TwoSum, whose rounding error is exact and collects in c, and a square v * v
// enters as its exact split p + e (p = fl(v * v), e = fma(v, v, -p)); the pairs are
// folded over the warp the same way and become one FP64 value per warp. Extremes of v or |v| are exact in FP32 and a mode-2 extreme
// is squared in FP64 at the end, which gives the FP64 fold's value. Only single-source
// reductions and plain sums of two sources (hi + lo, added term by term) take this form.
struct RedAccF {
    float s, c;
    __device__ __forceinline__ void init(int op)
    {
        s = op == OC_SUM ? 0.0f : (op == OC_MAX ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000));
        c = 0.0f;
    }
    __device__ __forceinline__ void two_sum(float t)
    {
        const float u = s + t;
        const float bp = u - s;
        c += (s - (u - bp)) + (t - bp);
        s = u;
    }
    __device__ __forceinline__ void add(int op, int mode, float v)
    {
        if (op == OC_SUM) {
            if (mode == 2) {
                const float p = v * v;
                two_sum(p);
                two_sum(fmaf(v, v, -p));
            } else {
                two_sum(mode == 1 ? fabsf(v) : v);
            }
        } else {
            const float m = mode == 0 ? v : fabsf(v);
            s = op == OC_MAX ? (m > s ? m : s) : (m < s ? m : s);
        }
    }
    __device__ __forceinline__ void add2(int, int, float u, float v)
    {
        two_sum(u);
        two_sum(v);
    }
    __device__ __forceinline__ double value(int op, int mode) const
    {
        if (op == OC_SUM) return (double)s + (double)c;
        return mode == 2 && !isinf(s) ? (double)s * (double)s : (double)s;
    }
    // Fixed shuffle tree over the warp, still in FP32: pairs are added with TwoSum of their
    // leading parts (the error and both trailing parts go to c); lane 0 ends with the fold.
    __device__ __forceinline__ void warp_fold(int op)
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, o);
            const float c2 = __shfl_down_sync(0xffffffffu, c, o);
            if (op == OC_SUM) {
                const float u = s + s2;
                const float bp = u - s;
                c = (c + c2) + ((s - (u - bp)) + (s2 - bp));
                s = u;
            } else {
                s = op == OC_MAX ? (s2 > s ? s2 : s) : (s2 < s ? s2 : s);
            }
        }
    }
};

// Block fold of warp-folded FP32 accumulators (valid in lane 0 of each warp) to one FP64
// value in thread 0: the warps' values are folded in FP64 with a fixed tree.
__device__ __forceinline__ double block_value(const RedAccF& acc, int op, int mode)
{
    __shared__ double sm[kRedThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = acc.value(op, mode);
    __syncthreads();
    double v = red_identity(op);
    if (w == 0) {
        v = l < kRedThreads / 32 ? sm[l] : red_identity(op);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v = red_apply(op, v, __shfl_down_sync(0xffffffffu, v, o));
    }
    return v;
}

// Fold n consecutive elements pa[0..n) (+ pb[0..n) when pb is set) into this thread's
// accumulator: a scalar head up to the first 16-byte boundary of pa, 16-byte vectors,
// a scalar tail. Thread k of the block takes head element k, vectors k, k + 256, ...
// and tail element k (+ 256...), each in that order, so the association is fixed by the
// segment alone. Both sources go vector only if they share their offset modulo 16.
template <typename T, typename A>
__device__ __forceinline__ void seg_fold(const T* pa, const T* pb, int n, int mode, int op, A& acc)
{
    using V = typename VecOf<T>::V;
    constexpr int N = VecOf<T>::N;
    const uintptr_t ua = reinterpret_cast<uintptr_t>(pa);
    const bool vec = (ua % sizeof(T)) == 0 && (!pb || ((reinterpret_cast<uintptr_t>(pb) ^ ua) & 15) == 0);
    int head = vec ? (int)(((16 - (ua & 15)) & 15) / sizeof(T)) : n;
    if (head > n) head = n;
    for (int i = threadIdx.x; i < head; i += kRedThreads) {
        if (pb) acc.add2(op, mode, __ldg(pa + i), __ldg(pb + i));
        else acc.add(op, mode, __ldg(pa + i));
    }
    const int nv = (n - head) / N;
    const V* va = reinterpret_cast<const V*>(pa + head);
    const V* vb = reinterpret_cast<const V*>(pb ? pb + head : pa);
    // unrolled so that a thread's independent 16-byte loads are in flight together
#pragma unroll 4
    for (int i = threadIdx.x; i < nv; i += kRedThreads) {
        T ea[N], eb[N];
        *reinterpret_cast<V*>(ea) = __ldg(va + i);
        if (pb) *reinterpret_cast<V*>(eb) = __ldg(vb + i);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (pb) acc.add2(op, mode, ea[k], eb[k]);
            else acc.add(op, mode, ea[k]);
        }
    }
    for (int i = head + nv * N + threadIdx.x; i < n; i += kRedThreads) {
        if (pb) acc.add2(op, mode, __ldg(pa + i), __ldg(pb + i));
        else acc.add(op, mode, __ldg(pa + i));
    }
}

// One block per (chunk of kRedPoints points of a slow row, group of slow rows): block
// (c, g) folds chunk c of rows s = lo + g, lo + g + gridDim.y, ... The points of a row
// are its x-lines in order (one line in 2-D, the y-lines of a z-plane in 3-D), so chunk c
// covers whole or partial lines; each line segment is contiguous (a REDUCE reads at
// offset 0 inside the range, which never wraps a periodic axis). Each thread folds its
// elements into its accumulator, the block folds the threads' values with a fixed tree,
// and the partial of row s, chunk c is stored at part[(s - part_row0) * chunks + c],
// independent of the tiling, so tiled and untiled runs fold the same partials in the same
// order.
template <typename T, typename A>
__device__ __forceinline__ void reduce_rows(const LaunchDesc& d)
{
    const int sa = d.ndim - 1;
    const int nxr = d.hi[0] - d.lo[0];
    const int nyl = d.ndim == 3 ? d.hi[1] - d.lo[1] : 1;
    const long long plane = (long long)nxr * nyl;
    const long long q0 = (long long)blockIdx.x * kRedPoints;
    const long long q1 = q0 + kRedPoints < plane ? q0 + kRedPoints : plane;
    const int op = d.red_op;
    const int mode = (int)d.params[0];
    const bool two = d.nargs == 3;
    const DView& a = d.v[0];
    const DView& b = d.v[1];
    // lines touched by the chunk: one division per block
    const int l0 = q1 > q0 ? (int)(q0 / nxr) : 0;
    const int l1 = q1 > q0 ? (int)((q1 - 1) / nxr) : -1;
    for (int s = d.lo[sa] + (int)blockIdx.y; s < d.hi[sa]; s += (int)gridDim.y) {
        const long long ra = (long long)first_slot(a, s) * a.row_elems;
        const long long rb = two ? (long long)first_slot(b, s) * b.row_elems : 0;
        auto fold = [&](auto& acc) {
            using Acc = typename std::remove_reference<decltype(acc)>::type;
            acc.init(op);
            for (int l = l0; l <= l1; ++l) {
                const long long lq = (long long)l * nxr;
                const int x0 = l == l0 ? (int)(q0 - lq) : 0;
                const int x1 = l == l1 ? (int)(q1 - lq) : nxr;
                const int yl = d.ndim == 3 ? d.lo[1] + l : 0;
                const T* pa = col_ptr<T>(a, d.lo[0] + x0, yl) + ra;
                const T* pb = two ? col_ptr<T>(b, d.lo[0] + x0, yl) + rb : nullptr;
                seg_fold<T, Acc>(pa, pb, x1 - x0, mode, op, acc);
            }
        };
        double v;
        if constexpr (std::is_same<A, RedAccF>::value) {
            RedAccF acc;
            fold(acc);
            acc.warp_fold(op);
            // a sum beyond FP32's range (or an inf / NaN term) anywhere in the block: the
            // block folds this chunk again in FP64, which gives the FP64 form's value
            const bool out = (threadIdx.x & 31) == 0 && op == OC_SUM && !(isfinite(acc.s) && isfinite(acc.c));
            if (__syncthreads_or(out)) {
                RedAccD acd;
                fold(acd);
                v = block_fold(acd.a, op);
            } else {
                v = block_value(acc, op, mode);
            }
        } else {
            A acc;
            fold(acc);
            v = block_fold(acc.a, op);
        }
        if (threadIdx.x == 0) d.part[(long long)(s - d.part_row0) * d.chunks + blockIdx.x] = v;
        __syncthreads();   // the fold's shared slots are reused by the next row
    }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_reduce(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    if constexpr (std::is_same<T, float>::value) {
        // the FP32 form for single sources and plain two-source sums (uniform branch)
        if (d.nargs != 3 || (d.red_op == OC_SUM && (int)d.params[0] == 0)) {
            reduce_rows<float, RedAccF>(d);
            return;
        }
    }
    reduce_rows<T, RedAccD>(d);
}

__global__ void __launch_bounds__(kRedThreads) k_combine(const double* __restrict__ part, long long n,
                                                        int op, double* out)
{
    pdl_enter();
    const long long per = (n + kRedThreads - 1) / kRedThreads;
    const long long a = per * threadIdx.x;
    const long long b = a + per < n ? a + per : n;
    double acc = red_identity(op);
    for (long long i = a; i < b; ++i) acc = red_apply(op, acc, part[i]);
    acc = block_fold(acc, op);
    if (threadIdx.x == 0) *out = acc;
}

// Halo-strip upload (launch.h StripBatch): block row y = job, threads stride over the
// job's (line, word) pairs. Host memory is read with cache-volatile loads, so a line
// the copy engines wrote back to the host since is fetched again.
constexpr int kStripThreads = 256;
__global__ void __launch_bounds__(kStripThreads) k_strip_copy(const __grid_constant__ StripBatch b)
{
    const StripJob& j = b.job[blockIdx.y];
    const long long n = (long long)j.lines * j.words;
    for (long long i = (long long)blockIdx.x * kStripThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kStripThreads) {
        const long long line = i / j.words;
        const long long o = line * j.pitch + 4 * (i - line * j.words);
        *reinterpret_cast<unsigned int*>(j.dst + o) = __ldcv(reinterpret_cast<const unsigned int*>(j.src + o));
    }
}

template <typename F>
cudaError_t launch_pointwise(const LaunchDesc& d, cudaStream_t st, F kern)
{
    const int sa = d.ndim - 1;
    const int nx = d.hi[0] - d.lo[0];
    const int ns = d.hi[sa] - d.lo[sa];
    if (nx <= 0 || ns <= 0 || (d.ndim == 3 && d.hi[1] <= d.lo[1])) return cudaSuccess;
    dim3 grid((nx + kThreadsX - 1) / kThreadsX, d.ndim == 3 ? d.hi[1] - d.lo[1] : 1,
              (ns + kRows - 1) / kRows);
    return launch_tile_kernel(kern, grid, kThreadsX, st, d);
}

constexpr int kLeanRows = 8;

template <typename K>
cudaError_t launch_rows(const LaunchDesc& d, cudaStream_t st, K kern, int rows)
{
    const int sa = d.ndim - 1;
    const int nx = d.hi[0] - d.lo[0];
    const int ns = d.hi[sa] - d.lo[sa];
    if (nx <= 0 || ns <= 0 || (d.ndim == 3 && d.hi[1] <= d.lo[1])) return cudaSuccess;
    dim3 grid((nx + kThreadsX - 1) / kThreadsX, d.ndim == 3 ? d.hi[1] - d.lo[1] : 1, (ns + rows - 1) / rows);
    return launch_tile_kernel(kern, grid, kThreadsX, st, d);
}

// Resident blocks per SM of the ring LINCOMB instantiations ([f32][R = 4, 8][M]) and the
// SM count, filled once by kernels_prepare() (before any stream capture).
constexpr int kRingMaxM = 20;
int g_ring_occ[2][2][kRingMaxM + 1] = {};
int g_sms = 0;

template <typename T, int M>
void ring_occupancy()
{
    const int f = std::is_same<T, float>::value ? 1 : 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_ring_occ[f][0][M], k_lincomb_ring<T, 4, M>, kThreadsX, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_ring_occ[f][1][M], k_lincomb_ring<T, kLeanRows, M>, kThreadsX, 0);
}

// Rows per thread of a ring LINCOMB launch: 8, or 4 when that fills the resident block
// slots of the GPU better. A launch of B blocks with C resident blocks per SM on S SMs
// runs ceil(B / (C S)) waves; its last wave leaves slots idle. Short tile launches (a few
// hundred rows) are one or two waves, where this matters; the arithmetic of every point is
// the same for both choices, so results do not depend on it.
template <typename T, int M>
int ring_rows_for(const LaunchDesc& d)
{
    const int f = std::is_same<T, float>::value ? 1 : 0;
    const int c4 = g_ring_occ[f][0][M], c8 = g_ring_occ[f][1][M];
    if (g_sms <= 0 || c4 <= 0 || c8 <= 0) return kLeanRows;
    const int sa = d.ndim - 1;
    const long long bx = (d.hi[0] - d.lo[0] + kThreadsX - 1) / kThreadsX;
    const long long by = d.ndim == 3 ? d.hi[1] - d.lo[1] : 1;
    const long long ns = d.hi[sa] - d.lo[sa];
    auto eff = [&](int R, int c) {
        const double w = (double)(bx * by * ((ns + R - 1) / R)) / ((double)c * g_sms);
        return w / std::ceil(w);
    };
    return eff(4, c4) > eff(kLeanRows, c8) + 0.05 ? 4 : kLeanRows;
}

template <typename T, int M>
cudaError_t lincomb_m(const LaunchDesc& d, cudaStream_t st)
{
    if constexpr (M > 0) {
        if (d.ring) {
            if (ring_rows_for<T, M>(d) == 4) return launch_rows(d, st, k_lincomb_ring<T, 4, M>, 4);
            return launch_rows(d, st, k_lincomb_ring<T, kLeanRows, M>, kLeanRows);
        }
        if (d.lean) return launch_rows(d, st, k_lincomb_lean<T, kLeanRows, M>, kLeanRows);
    }
    return launch_pointwise(d, st, k_lincomb<T, kRows, M>);
}

// Dispatch on the number of samples: 1..20 get a fully unrolled instance.
template <typename T>
cudaError_t launch_lincomb(const LaunchDesc& d, cudaStream_t st)
{
    switch (d.nsamp) {
#define OC_LC(M) case M: return lincomb_m<T, M>(d, st);
        OC_LC(1) OC_LC(2) OC_LC(3) OC_LC(4) OC_LC(5) OC_LC(6) OC_LC(7) OC_LC(8) OC_LC(9) OC_LC(10)
        OC_LC(11) OC_LC(12) OC_LC(13) OC_LC(14) OC_LC(15) OC_LC(16) OC_LC(17) OC_LC(18) OC_LC(19) OC_LC(20)
#undef OC_LC
    default: return lincomb_m<T, 0>(d, st);
    }
}

}  // namespace

cudaError_t launch_loop(const LaunchDesc& d, cudaStream_t st)
{
    const bool f32 = d.dtype == OC_F32;
    switch (d.kernel) {
    case OC_K_COPY:
        if (d.lean)
            return f32 ? launch_rows(d, st, k_copy_lean<float, kLeanRows>, kLeanRows)
                       : launch_rows(d, st, k_copy_lean<double, kLeanRows>, kLeanRows);
        return f32 ? launch_pointwise(d, st, k_copy<float, kRows>) : launch_pointwise(d, st, k_copy<double, kRows>);
    case OC_K_LINCOMB:
        return f32 ? launch_lincomb<float>(d, st) : launch_lincomb<double>(d, st);
    case OC_K_HILO_ADD:
        return launch_pointwise(d, st, k_hilo_add<kRows>);
    case OC_K_REDUCE: {
        const int sa = d.ndim - 1;
        const int ns = d.hi[sa] - d.lo[sa];
        if (ns <= 0) return cudaSuccess;
        dim3 grid(d.chunks, std::min(ns, 65535), 1);
        return f32 ? launch_tile_kernel(k_reduce<float>, grid, kRedThreads, st, d)
                   : launch_tile_kernel(k_reduce<double>, grid, kRedThreads, st, d);
    }
    default:
        return launch_physics(d, st);
    }
}

cudaError_t launch_strips(const StripBatch& b, cudaStream_t st)
{
    if (b.njobs <= 0) return cudaSuccess;
    long long most = 1;
    for (int k = 0; k < b.njobs; ++k) most = std::max(most, (long long)b.job[k].lines * b.job[k].words);
    const int bx = (int)std::min<long long>(64, (most + kStripThreads - 1) / kStripThreads);
    k_strip_copy<<<dim3(bx, b.njobs), kStripThreads, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_combine(const double* part, long long n, int op, double* out, cudaStream_t st)
{
    return launch_tile_kernel(k_combine, dim3(1, 1, 1), kRedThreads, st, part, n, op, out);
}

int kernels_compiled_arch() { return 1030; }

namespace dev {
bool g_pdl = true;
}

void kernels_prepare()
{
    const char* pdl = getenv("OC_PDL");
    dev::g_pdl = !(pdl && pdl[0] == '0');
    if (g_sms > 0) return;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
#define OC_OCC(M) ring_occupancy<float, M>(); ring_occupancy<double, M>();
    OC_OCC(1) OC_OCC(2) OC_OCC(3) OC_OCC(4) OC_OCC(5) OC_OCC(6) OC_OCC(7) OC_OCC(8) OC_OCC(9) OC_OCC(10)
    OC_OCC(11) OC_OCC(12) OC_OCC(13) OC_OCC(14) OC_OCC(15) OC_OCC(16) OC_OCC(17) OC_OCC(18) OC_OCC(19) OC_OCC(20)
#undef OC_OCC
    cudaGetLastError();
    g_sms = sms;
}

}  // namespace oc
