/*
 * oc_physics.h -- PDE loop kernels of liboc.so (kernel_id values for oc_enqueue_loop).
 *
 * They are the loops of the two compressible-flow workloads that stand in for the
 * paper's applications (arXiv 1709.02125, Sec. 5.1: CloverLeaf -- Euler equations,
 * explicit second-order scheme -- and OpenSBLI -- Navier-Stokes, fourth-order finite
 * differences, third-order Runge-Kutta, no reductions inside a step). Each kernel is
 * pointwise with a fixed stencil; enqueueing checks that the arguments carry exactly
 * the stencil below (so the tiling analysis sees the true reach), the access modes,
 * one element type for all datasets, and the parameter count. Fast axes of datasets
 * declared periodic wrap inside the kernels; the slow (tiled) axis is periodic through
 * deep ghost rows (oc_decl_dat). "cross9" = {(0,0), (+-1,0), (+-2,0), (0,+-1), (0,+-2)};
 * "star12" = the twelve points at +-1 and +-2 along each of x, y, z.
 *
 * Euler, 2-D, conserved U = (rho, mx, my, E), gamma-law gas:
 *   u = mx/rho, v = my/rho, p = (gamma - 1)(E - 0.5 (mx u + my v)).
 * OC_K_EULER_PRIM  [R rho, R mx, R my, R E, W u, W v, W p]              params [gamma]
 * OC_K_EULER_FLUX  [R rho, mx, my, E, u, v, p, W F0..F3, W G0..G3]       params []
 *                  F = (mx, mx u + p, mx v, (E + p) u), G = (my, my u, my v + p, (E + p) v)
 * OC_K_EULER_PRED  [R U0..U3, R F0..F3 at {(0,0),(1,0)}, R G0..G3 at {(0,0),(0,1)},
 *                   W S0..S3]                                             params [lx, ly]
 *                  S = (U - lx (F(x+1) - F)) - ly (G(y+1) - G)          (MacCormack predictor)
 * OC_K_EULER_CORR  [R U0..U3 at cross9, R S0..S3, R H0..H3 at {(0,0),(-1,0)},
 *                   R K0..K3 at {(0,0),(0,-1)}, W out0..out3]             params [lx, ly, eps4, mode]
 *                  A = lx (H - H(x-1)), B = ly (K - K(y-1)), H, K the fluxes of S,
 *                  d4 = d4x U + d4y U, d4x U = (((U(x-2) - 4U(x-1)) + 6U) - 4U(x+1)) + U(x+2);
 *                  mode 0: out = 0.5 (((U + S) - A) - B) - eps4 d4      (new state)
 *                  mode 1: out = 0.5 (((S - U) - A) - B) - eps4 d4      (increment, for the
 *                          compensated hi/lo update of the mixed-precision form)
 * OC_K_EULER_DT    [R U0..U3, (optional R L0..L3), REDUCE h (MIN)]       params [gamma, dx, dy]
 *                  value = min(dx / (|u| + c), dy / (|v| + c)), c = sqrt(gamma p / rho), from U
 *                  (or from U + L when the low parts are given), folded into h.
 *
 * Navier-Stokes, 3-D, conserved U = (rho, rho u, rho v, rho w, rho E), nondimensional:
 *   p = (gamma - 1)(rho E - 0.5 (ru u + rv v + rw w)), T = gamma Ma^2 p / rho,
 *   mu = 1/Re (0 if Re <= 0), k = mu / ((gamma - 1) Ma^2 Pr),
 *   D f = ((f(-2) - 8 f(-1)) + (8 f(+1) - f(+2))) / (12 h)  (fourth-order central).
 * OC_K_NS_PRIM     [R rho, ru, rv, rw, rE, W u, v, w, p, T]              params [gamma, Ma]
 * OC_K_NS_GRAD     [R u, v, w, T at star12, W du/dx, du/dy, du/dz, dv/dx, ..., dT/dz]
 *                                                                         params [hx, hy, hz]
 * OC_K_NS_RHS      [R U0..U4 at star12, R u, v, w, p at star12, R the 12 gradients at star12,
 *                   W or RW dU0..dU4]                       params [gamma, Ma, Re, Pr, hx, hy, hz, A, dt]
 *                  R_m = - sum over axes a = x, y, z (in that order) of D_a(flux_{m,a}), with
 *                  flux_{0,a} = U_{a+1}, flux_{i,a} = U_i u_a + p delta_ia - tau_ia,
 *                  flux_{4,a} = (rho E + p) u_a - (u tau_xa + v tau_ya + w tau_za) - k dT/dx_a,
 *                  tau_ba = mu (d u_b/dx_a + d u_a/dx_b - 2/3 delta_ab div u);
 *                  dU = A dU + dt R (with W access: dU = dt R, the first low-storage stage).
 * OC_K_NS_UPDATE   [RW U0..U4, R dU0..dU4]                                params [B]
 *                  U = U + B dU.
 * OC_K_NS_FLUX     [R U0..U4, R u, v, w, p, R the 12 gradients (all at offset 0),
 *                   W F_{m,a} for m = 0..4, a = x, y, z (15, m-major)]   params [gamma, Ma, Re, Pr]
 *                  F_{m,a} = flux_{m,a} of OC_K_NS_RHS at the point.
 * OC_K_NS_DIV      [R F_{m,a} (15, m-major) each at +-1, +-2 along its own axis a,
 *                   W or RW dU0..dU4]                                    params [hx, hy, hz, A, dt]
 *                  R_m = - sum over a = x, y, z (in order) of D_a(F_{m,a}); dU as NS_RHS.
 *                  NS_FLUX followed by NS_DIV computes exactly what NS_RHS computes, with
 *                  each flux evaluated once per point instead of at four neighbours.
 */
#ifndef OC_PHYSICS_H
#define OC_PHYSICS_H

#define OC_K_EULER_PRIM 10
#define OC_K_EULER_FLUX 11
#define OC_K_EULER_PRED 12
#define OC_K_EULER_CORR 13
#define OC_K_EULER_DT   14
#define OC_K_NS_PRIM    20
#define OC_K_NS_GRAD    21
#define OC_K_NS_RHS     22
#define OC_K_NS_UPDATE  23
#define OC_K_NS_FLUX    24
#define OC_K_NS_DIV     25

#endif /* OC_PHYSICS_H */
