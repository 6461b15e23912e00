// PDE loop kernels: 2-D Euler (MacCormack with fourth-order dissipation) and 3-D
// Navier-Stokes (fourth-order central differences, low-storage RK3). Definitions,
// argument layouts and evaluation order: include/oc_physics.h.
//
// Every kernel is pointwise: one thread per point, x fastest across the threads of a
// block (coalesced x-lines), blockIdx.y over y-lines of a 3-D plane, blockIdx.z over
// the slow rows of the tile. Stencil neighbours come through L1/L2. Fast periodic axes
// wrap in the address computation; the slow axis is read through the cyclic slab.
// The arithmetic of each point follows the stated order with separately rounded
// operations (the library is built with -fmad=false), in FP64 or FP32 by the
// datasets' element type.
#include <cuda_runtime.h>

#include "../../include/oc.h"
#include "../../include/oc_physics.h"
#include "kcommon.cuh"
#include "launch.h"

namespace oc {

namespace {

using namespace dev;

// A point of the launch. With uniform argument geometry (LaunchDesc::uni) the in-row
// offset (y line and x) is shared by all arguments and computed once; `xin` / `yin` say
// that the +-2 neighbours along x / y need no periodic wrap.
struct Pt {
    int x, yl, s;
    int inrow;
    bool fast, xin, yin;
};

__device__ __forceinline__ bool point_of(const LaunchDesc& d, Pt& p)
{
    p.x = d.lo[0] + (int)(blockIdx.x * kThreadsX + threadIdx.x);
    if (p.x >= d.hi[0]) return false;
    const int sa = d.ndim - 1;
    p.yl = d.ndim == 3 ? d.lo[1] + (int)blockIdx.y : 0;
    p.s = d.lo[sa] + (int)blockIdx.z;
    const DView& v = d.v[0];
    p.fast = d.uni != 0;
    p.inrow = (p.yl + v.oy) * (int)v.pitch + v.ox + p.x;
    p.xin = !(v.periodic & 1) || (p.x >= 2 && p.x < v.nx - 2);
    p.yin = !(v.periodic & 2) || (p.yl >= 2 && p.yl < v.ny - 2);
    return true;
}

// neighbour of p at distance k along axis a (a = 0 x, 1 y, 2 slow axis in 3-D;
// in 2-D axis 1 is the slow axis); its addresses are then computed in full
__device__ __forceinline__ Pt shift(const LaunchDesc& d, Pt p, int a, int k)
{
    if (a == 0) p.x += k;
    else if (a == 1 && d.ndim == 3) p.yl += k;
    else p.s += k;
    p.fast = false;
    return p;
}

// Address of argument `arg` at point p.
template <typename T, bool O>
__device__ __forceinline__ const T* C(const LaunchDesc& d, int arg, const Pt& p)
{
    const DView& v = d.v[arg];
    if (O && p.fast)
        return reinterpret_cast<const T*>(v.base) + (first_slot(v, p.s) * (int)v.row_elems + p.inrow);
    return O ? elem32<T>(v, p.x, p.yl, p.s) : elem<T>(v, p.x, p.yl, p.s);
}

template <typename T, bool O>
__device__ __forceinline__ T L(const LaunchDesc& d, int arg, const Pt& p)
{
    return __ldg(C<T, O>(d, arg, p));
}

template <typename T, bool O>
__device__ __forceinline__ void S(const LaunchDesc& d, int arg, const Pt& p, T v)
{
    *const_cast<T*>(C<T, O>(d, arg, p)) = v;
}

// Neighbour at distance k along axis a of the point whose address is c: an offset
// from the centre (x: elements, y: x-lines, slow axis: slab slots), the full periodic
// wrap only where a fast periodic axis crosses its end.
template <typename T, bool O>
__device__ __forceinline__ T Lk(const LaunchDesc& d, int arg, const Pt& p, const T* c, int a, int k)
{
    const DView& v = d.v[arg];
    if (a == 0) {
        const bool wraps = p.fast ? !p.xin : ((v.periodic & 1) && (p.x + k < 0 || p.x + k >= v.nx));
        if (wraps) return L<T, O>(d, arg, shift(d, p, 0, k));
        return __ldg(c + k);
    }
    if (a == 1 && d.ndim == 3) {
        const bool wraps = p.fast ? !p.yin : ((v.periodic & 2) && (p.yl + k < 0 || p.yl + k >= v.ny));
        if (wraps) return L<T, O>(d, arg, shift(d, p, 1, k));
        return __ldg(c + k * (int)v.pitch);
    }
    const int s0 = first_slot(v, p.s);
    int s1 = s0 + k;
    if (s1 >= v.S) s1 -= v.S;
    else if (s1 < 0) s1 += v.S;
    if (O) return __ldg(c + (s1 - s0) * (int)v.row_elems);
    return __ldg(c + (long long)(s1 - s0) * v.row_elems);
}

// ------------------------------------------------------------------ Euler -----
template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_euler_prim(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T gamma = params_of<T>(d)[0];
    const T r = L<T, O>(d, 0, p), mx = L<T, O>(d, 1, p), my = L<T, O>(d, 2, p), E = L<T, O>(d, 3, p);
    const T u = mx / r, v = my / r;
    const T pr = (gamma - T(1)) * (E - T(0.5) * (mx * u + my * v));
    S<T, O>(d, 4, p, u);
    S<T, O>(d, 5, p, v);
    S<T, O>(d, 6, p, pr);
}

template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_euler_flux(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T mx = L<T, O>(d, 1, p), my = L<T, O>(d, 2, p), E = L<T, O>(d, 3, p);
    const T u = L<T, O>(d, 4, p), v = L<T, O>(d, 5, p), pr = L<T, O>(d, 6, p);
    const T ep = E + pr;
    S<T, O>(d, 7, p, mx);
    S<T, O>(d, 8, p, mx * u + pr);
    S<T, O>(d, 9, p, mx * v);
    S<T, O>(d, 10, p, ep * u);
    S<T, O>(d, 11, p, my);
    S<T, O>(d, 12, p, my * u);
    S<T, O>(d, 13, p, my * v + pr);
    S<T, O>(d, 14, p, ep * v);
}

template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_euler_pred(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T lx = params_of<T>(d)[0], ly = params_of<T>(d)[1];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T U = L<T, O>(d, k, p);
        const T* cF = C<T, O>(d, 4 + k, p);
        const T* cG = C<T, O>(d, 8 + k, p);
        const T F = __ldg(cF), Fp = Lk<T, O>(d, 4 + k, p, cF, 0, 1);
        const T G = __ldg(cG), Gp = Lk<T, O>(d, 8 + k, p, cG, 1, 1);
        S<T, O>(d, 12 + k, p, (U - lx * (Fp - F)) - ly * (Gp - G));
    }
}

template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_euler_corr(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T* pm = params_of<T>(d);
    const T lx = pm[0], ly = pm[1], eps4 = pm[2];
    const bool inc = pm[3] != T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T* cU = C<T, O>(d, k, p);
        const T U = __ldg(cU);
        const T d4x = (((Lk<T, O>(d, k, p, cU, 0, -2) - T(4) * Lk<T, O>(d, k, p, cU, 0, -1)) + T(6) * U) -
                       T(4) * Lk<T, O>(d, k, p, cU, 0, 1)) + Lk<T, O>(d, k, p, cU, 0, 2);
        const T d4y = (((Lk<T, O>(d, k, p, cU, 1, -2) - T(4) * Lk<T, O>(d, k, p, cU, 1, -1)) + T(6) * U) -
                       T(4) * Lk<T, O>(d, k, p, cU, 1, 1)) + Lk<T, O>(d, k, p, cU, 1, 2);
        const T Us = L<T, O>(d, 4 + k, p);
        const T* cH = C<T, O>(d, 8 + k, p);
        const T* cK = C<T, O>(d, 12 + k, p);
        const T A = lx * (__ldg(cH) - Lk<T, O>(d, 8 + k, p, cH, 0, -1));
        const T B = ly * (__ldg(cK) - Lk<T, O>(d, 12 + k, p, cK, 1, -1));
        const T first = inc ? (Us - U) : (U + Us);
        S<T, O>(d, 16 + k, p, T(0.5) * ((first - A) - B) - eps4 * (d4x + d4y));
    }
}

// CFL candidate of one point; with the low parts present the state is hi + lo.
template <typename T, bool O>
__global__ void __launch_bounds__(kRedThreads) k_euler_dt(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    const T* pm = params_of<T>(d);
    const T gamma = pm[0], dx = pm[1], dy = pm[2];
    const bool lo = d.nargs == 9;
    row_partial(d, [&](int x, int yl, int s) -> double {
        T U[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            U[k] = ld<T, O>(d.v[k], x, yl, s);
            if (lo) U[k] = U[k] + ld<T, O>(d.v[4 + k], x, yl, s);
        }
        const T r = U[0], u = U[1] / r, v = U[2] / r;
        const T pr = (gamma - T(1)) * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
        const T c = sqrt(gamma * pr / r);
        const T a = dx / (fabs(u) + c), b = dy / (fabs(v) + c);
        return (double)(a < b ? a : b);
    });
}

// --------------------------------------------------------------- Navier-Stokes --
template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_ns_prim(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T gamma = params_of<T>(d)[0], Ma = params_of<T>(d)[1];
    const T r = L<T, O>(d, 0, p), ru = L<T, O>(d, 1, p), rv = L<T, O>(d, 2, p), rw = L<T, O>(d, 3, p), rE = L<T, O>(d, 4, p);
    const T u = ru / r, v = rv / r, w = rw / r;
    const T pr = (gamma - T(1)) * (rE - T(0.5) * ((ru * u + rv * v) + rw * w));
    S<T, O>(d, 5, p, u);
    S<T, O>(d, 6, p, v);
    S<T, O>(d, 7, p, w);
    S<T, O>(d, 8, p, pr);
    S<T, O>(d, 9, p, ((gamma * Ma) * Ma) * pr / r);
}

template <typename T, bool O>
__device__ __forceinline__ T d1(const LaunchDesc& d, int arg, const Pt& p, const T* c, int a, T h12)
{
    const T fm2 = Lk<T, O>(d, arg, p, c, a, -2), fm1 = Lk<T, O>(d, arg, p, c, a, -1);
    const T fp1 = Lk<T, O>(d, arg, p, c, a, 1), fp2 = Lk<T, O>(d, arg, p, c, a, 2);
    return ((fm2 - T(8) * fm1) + (T(8) * fp1 - fp2)) / h12;
}

template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_ns_grad(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T* pm = params_of<T>(d);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const T* c = C<T, O>(d, f, p);
#pragma unroll
        for (int a = 0; a < 3; ++a) S<T, O>(d, 4 + 3 * f + a, p, d1<T, O>(d, f, p, c, a, T(12) * pm[a]));
    }
}

// The 21 inputs of the fluxes at point q (arguments 0-4 U, 5-8 u v w p, 9-20 the
// gradients d(u,v,w,T)/d(x,y,z) in that order), loaded once.
template <typename T, bool O>
__device__ __forceinline__ void ns_inputs(const LaunchDesc& d, const Pt& q, T (&in)[21])
{
#pragma unroll
    for (int k = 0; k < 21; ++k) in[k] = L<T, O>(d, k, q);
}

// The five fluxes in direction a from the inputs of one point.
template <typename T>
__device__ __forceinline__ void ns_fluxes(const T (&in)[21], int a, T mu, T kc, T (&f)[5])
{
    const T vel[3] = {in[5], in[6], in[7]};
    const T pr = in[8];
    const T div = (in[9] + in[13]) + in[17];
    T tau[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const T s = in[9 + 3 * b + a] + in[9 + 3 * a + b];
        tau[b] = mu * (b == a ? s - (T(2) / T(3)) * div : s);
    }
    f[0] = in[1 + a];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const T uu = in[1 + i] * vel[a];
        f[1 + i] = (i == a ? uu + pr : uu) - tau[i];
    }
    f[4] = ((in[4] + pr) * vel[a] - ((vel[0] * tau[0] + vel[1] * tau[1]) + vel[2] * tau[2])) - kc * in[18 + a];
}

template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_ns_rhs(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T* pd = params_of<T>(d);
    const T gamma = pd[0], Ma = pd[1], Re = pd[2], Pr = pd[3];
    const T A = pd[7], dt = pd[8];
    const T mu = Re > T(0) ? T(1) / Re : T(0);
    const T kc = mu / ((((gamma - T(1)) * Ma) * Ma) * Pr);
    T R[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
        const T h12 = T(12) * pd[4 + a];
        T fm2[5], fm1[5], fp1[5], fp2[5], in[21];
        ns_inputs<T, O>(d, shift(d, p, a, -2), in);
        ns_fluxes<T>(in, a, mu, kc, fm2);
        ns_inputs<T, O>(d, shift(d, p, a, -1), in);
        ns_fluxes<T>(in, a, mu, kc, fm1);
        ns_inputs<T, O>(d, shift(d, p, a, 1), in);
        ns_fluxes<T>(in, a, mu, kc, fp1);
        ns_inputs<T, O>(d, shift(d, p, a, 2), in);
        ns_fluxes<T>(in, a, mu, kc, fp2);
#pragma unroll
        for (int m = 0; m < 5; ++m) R[m] = R[m] - ((fm2[m] - T(8) * fm1[m]) + (T(8) * fp1[m] - fp2[m])) / h12;
    }
    const bool rw = d.access[21] == OC_RW;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const T du = rw ? A * L<T, O>(d, 21 + m, p) + dt * R[m] : dt * R[m];
        S<T, O>(d, 21 + m, p, du);
    }
}

// The 15 fluxes of the point (same evaluation as the fused kernel's ns_fluxes).
template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_ns_flux(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T* pd = params_of<T>(d);
    const T gamma = pd[0], Ma = pd[1], Re = pd[2], Pr = pd[3];
    const T mu = Re > T(0) ? T(1) / Re : T(0);
    const T kc = mu / ((((gamma - T(1)) * Ma) * Ma) * Pr);
    T in[21];
    ns_inputs<T, O>(d, p, in);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T f[5];
        ns_fluxes<T>(in, a, mu, kc, f);
#pragma unroll
        for (int m = 0; m < 5; ++m) S<T, O>(d, 21 + 3 * m + a, p, f[m]);
    }
}

// R_m = - sum_a D_a(F_{m,a}) from stored fluxes, then the low-storage RK register.
template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_ns_div(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T* pd = params_of<T>(d);
    const T A = pd[3], dt = pd[4];
    const bool rw = d.access[15] == OC_RW;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        T r = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int arg = 3 * m + a;
            const T* c = C<T, O>(d, arg, p);
            const T fm2 = Lk<T, O>(d, arg, p, c, a, -2), fm1 = Lk<T, O>(d, arg, p, c, a, -1);
            const T fp1 = Lk<T, O>(d, arg, p, c, a, 1), fp2 = Lk<T, O>(d, arg, p, c, a, 2);
            r = r - ((fm2 - T(8) * fm1) + (T(8) * fp1 - fp2)) / (T(12) * pd[a]);
        }
        const T du = rw ? A * L<T, O>(d, 15 + m, p) + dt * r : dt * r;
        S<T, O>(d, 15 + m, p, du);
    }
}

template <typename T, bool O>
__global__ void __launch_bounds__(kThreadsX) k_ns_update(const __grid_constant__ LaunchDesc d)
{
    pdl_enter();
    Pt p;
    if (!point_of(d, p)) return;
    const T B = params_of<T>(d)[0];
#pragma unroll
    for (int m = 0; m < 5; ++m) S<T, O>(d, m, p, L<T, O>(d, m, p) + B * L<T, O>(d, 5 + m, p));
}

template <typename K>
cudaError_t launch_pt(const LaunchDesc& d, cudaStream_t st, K kern)
{
    const int sa = d.ndim - 1;
    const int nx = d.hi[0] - d.lo[0], ns = d.hi[sa] - d.lo[sa];
    const int ny = d.ndim == 3 ? d.hi[1] - d.lo[1] : 1;
    if (nx <= 0 || ns <= 0 || ny <= 0) return cudaSuccess;
    dim3 grid((nx + kThreadsX - 1) / kThreadsX, ny, ns);
    return launch_tile_kernel(kern, grid, kThreadsX, st, d);
}

}  // namespace

cudaError_t launch_physics(const LaunchDesc& d, cudaStream_t st)
{
    const bool f = d.dtype == OC_F32;
    const bool o = d.o32 != 0;
#define OC_PT(K) (f ? (o ? launch_pt(d, st, K<float, true>) : launch_pt(d, st, K<float, false>)) \
                    : (o ? launch_pt(d, st, K<double, true>) : launch_pt(d, st, K<double, false>)))
    switch (d.kernel) {
    case OC_K_EULER_PRIM: return OC_PT(k_euler_prim);
    case OC_K_EULER_FLUX: return OC_PT(k_euler_flux);
    case OC_K_EULER_PRED: return OC_PT(k_euler_pred);
    case OC_K_EULER_CORR: return OC_PT(k_euler_corr);
    case OC_K_EULER_DT: {
        const int sa = d.ndim - 1, ns = d.hi[sa] - d.lo[sa];
        if (ns <= 0) return cudaSuccess;
        dim3 grid(d.chunks, ns, 1);
        if (f) {
            return o ? launch_tile_kernel(k_euler_dt<float, true>, grid, kRedThreads, st, d)
                     : launch_tile_kernel(k_euler_dt<float, false>, grid, kRedThreads, st, d);
        } else {
            return o ? launch_tile_kernel(k_euler_dt<double, true>, grid, kRedThreads, st, d)
                     : launch_tile_kernel(k_euler_dt<double, false>, grid, kRedThreads, st, d);
        }
    }
    case OC_K_NS_PRIM: return OC_PT(k_ns_prim);
    case OC_K_NS_GRAD: return OC_PT(k_ns_grad);
    case OC_K_NS_RHS: return OC_PT(k_ns_rhs);
    case OC_K_NS_UPDATE: return OC_PT(k_ns_update);
    case OC_K_NS_FLUX: return OC_PT(k_ns_flux);
    case OC_K_NS_DIV: return OC_PT(k_ns_div);
    default: return cudaErrorInvalidValue;
    }
#undef OC_PT
}

}  // namespace oc
