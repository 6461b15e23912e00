"""Kernel ids of the PDE loops (include/oc_physics.h) for the binding."""
KERNELS = {
    "euler_prim": 10, "euler_flux": 11, "euler_pred": 12, "euler_corr": 13, "euler_dt": 14,
    "ns_prim": 20, "ns_grad": 21, "ns_rhs": 22, "ns_update": 23, "ns_flux": 24, "ns_div": 25,
}
