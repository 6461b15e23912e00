"""Loop-level oracle of the PDE kernels: each Euler / Navier-Stokes loop evaluated over
its iteration range on full-extent FP64 fields (numpy, elementwise, no fused operations).

TEST INFRASTRUCTURE (see the package docstring). The formulas are those of the two
workloads standing in for the applications of arXiv 1709.02125 Sec. 5.1 -- the
MacCormack step with fourth-order dissipation (Euler) and the fourth-order central,
low-storage RK3 Navier-Stokes step -- split into the loops a user of the executor
enqueues (include/oc_physics.h lists them). The whole-step definitions are
`oracle.physics` (physics.c); the tests check that the loops of one step, run in program
order with the deep-ghost rule of the periodic slow axis (ghost row y takes interior
row y mod n at the start of a chain), reproduce those steps.

Fields are `oracle.Field` objects; a field's `periodic` axes other than the slowest have
no halo and wrap modulo the interior size.
"""
from __future__ import annotations

from typing import Dict

import numpy as np

KERNELS = ("euler_prim", "euler_flux", "euler_pred", "euler_corr", "euler_dt",
           "ns_prim", "ns_grad", "ns_flux", "ns_div", "ns_rhs", "ns_update")


def _index(f, lo, hi, off):
    """Index arrays of the range [lo, hi) shifted by `off`, slowest axis first."""
    per = getattr(f, "periodic", ())
    nd = f.ndim
    idx = []
    for a in reversed(range(nd)):
        r = np.arange(lo[a], hi[a]) + (off[a] if a < len(off) else 0)
        if a in per and a < nd - 1:
            r = np.mod(r, f.size[a])
        r = r + f.halo_lo[a]
        ext = f.size[a] + f.halo_lo[a] + f.halo_hi[a]
        if r.size and (r.min() < 0 or r.max() >= ext):
            raise IndexError("stencil access outside the allocated extent")
        idx.append(r)
    return np.ix_(*idx)


def _get(f, lo, hi, off=(0, 0, 0)):
    return f.a[_index(f, lo, hi, off)]


def _put(f, lo, hi, v):
    f.a[_index(f, lo, hi, (0, 0, 0))] = v


def _unit(a, k):
    o = [0, 0, 0]
    o[a] = k
    return tuple(o)


def _d1(f, lo, hi, a, h):
    """fourth-order central first difference along axis a:
    ((f(-2) - 8 f(-1)) + (8 f(+1) - f(+2))) / (12 h)"""
    fm2, fm1 = _get(f, lo, hi, _unit(a, -2)), _get(f, lo, hi, _unit(a, -1))
    fp1, fp2 = _get(f, lo, hi, _unit(a, 1)), _get(f, lo, hi, _unit(a, 2))
    return ((fm2 - 8.0 * fm1) + (8.0 * fp1 - fp2)) / (12.0 * h)


# --------------------------------------------------------------------- Euler ----
def _euler_prim(rho, mx, my, E, gamma):
    u = mx / rho
    v = my / rho
    p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v))
    return u, v, p


def _euler(lp, F, reds, red_ops):
    k, lo, hi, A, P = lp.kernel, lp.lo, lp.hi, lp.args, lp.params
    g = [F[a.name] for a in A if a.access != "red"]
    if k == "euler_prim":
        u, v, p = _euler_prim(*[_get(x, lo, hi) for x in g[:4]], P[0])
        for x, val in zip(g[4:7], (u, v, p)):
            _put(x, lo, hi, val)
    elif k == "euler_flux":
        rho, mx, my, E, u, v, p = [_get(x, lo, hi) for x in g[:7]]
        Fv = (mx, mx * u + p, mx * v, (E + p) * u)
        Gv = (my, my * u, my * v + p, (E + p) * v)
        for x, val in zip(g[7:15], Fv + Gv):
            _put(x, lo, hi, val)
    elif k == "euler_pred":
        lx, ly = P
        for c in range(4):
            U = _get(g[c], lo, hi)
            dF = _get(g[4 + c], lo, hi, (1, 0)) - _get(g[4 + c], lo, hi)
            dG = _get(g[8 + c], lo, hi, (0, 1)) - _get(g[8 + c], lo, hi)
            _put(g[12 + c], lo, hi, (U - lx * dF) - ly * dG)
    elif k == "euler_corr":
        lx, ly, eps4, mode = P
        for c in range(4):
            Uf = g[c]
            U = _get(Uf, lo, hi)
            S = _get(g[4 + c], lo, hi)
            Aa = lx * (_get(g[8 + c], lo, hi) - _get(g[8 + c], lo, hi, (-1, 0)))
            Bb = ly * (_get(g[12 + c], lo, hi) - _get(g[12 + c], lo, hi, (0, -1)))
            d4 = []
            for ax in (0, 1):
                m2, m1 = _get(Uf, lo, hi, _unit(ax, -2)), _get(Uf, lo, hi, _unit(ax, -1))
                p1, p2 = _get(Uf, lo, hi, _unit(ax, 1)), _get(Uf, lo, hi, _unit(ax, 2))
                d4.append((((m2 - 4.0 * m1) + 6.0 * U) - 4.0 * p1) + p2)
            d4 = d4[0] + d4[1]
            first = (U + S) if mode == 0.0 else (S - U)
            _put(g[16 + c], lo, hi, 0.5 * ((first - Aa) - Bb) - eps4 * d4)
    elif k == "euler_dt":
        gamma, dx, dy = P
        rho, mx, my, E = [_get(x, lo, hi) for x in g[:4]]
        if len(g) == 8:
            rho, mx, my, E = [a + _get(x, lo, hi) for a, x in zip((rho, mx, my, E), g[4:8])]
        u, v, p = _euler_prim(rho, mx, my, E, gamma)
        c = np.sqrt(gamma * p / rho)
        val = np.minimum(dx / (np.abs(u) + c), dy / (np.abs(v) + c))
        red = [a.name for a in A if a.access == "red"][0]
        m = float(val.min()) if val.size else float("inf")
        reds[red] = min(reds[red], m) if red in reds else m


# ------------------------------------------------------------- Navier-Stokes ----
def _ns_consts(gamma, Ma, Re, Pr):
    mu = 1.0 / Re if Re > 0 else 0.0
    kc = mu / ((gamma - 1.0) * Ma * Ma * Pr)
    return mu, kc


def _ns_flux(Uv, W, D, mu, kc, m, a):
    """flux of conserved component m along axis a from the state U (5), the primitives
    W = (u, v, w, p) and the 12 gradients D[3 f + b] = d(u, v, w, T)_f / dx_b"""
    vel = W[:3]
    p = W[3]
    div = (D[0] + D[4]) + D[8]
    tau = [mu * ((D[3 * b + a] + D[3 * a + b]) - ((2.0 / 3.0) * div if b == a else 0.0)) for b in range(3)]
    if m == 0:
        return Uv[a + 1]
    if m <= 3:
        base = Uv[m] * vel[a]
        if m - 1 == a:
            base = base + p
        return base - tau[m - 1]
    work = (vel[0] * tau[0] + vel[1] * tau[1]) + vel[2] * tau[2]
    return ((Uv[4] + p) * vel[a] - work) - kc * D[9 + a]


def _ns(lp, F, reds, red_ops):
    k, lo, hi, A, P = lp.kernel, lp.lo, lp.hi, lp.args, lp.params
    g = [F[a.name] for a in A if a.access != "red"]
    acc = [a.access for a in A if a.access != "red"]
    if k == "ns_prim":
        gamma, Ma = P
        rho, ru, rv, rw, rE = [_get(x, lo, hi) for x in g[:5]]
        u, v, w = ru / rho, rv / rho, rw / rho
        p = (gamma - 1.0) * (rE - 0.5 * ((ru * u + rv * v) + rw * w))
        T = gamma * Ma * Ma * p / rho
        for x, val in zip(g[5:10], (u, v, w, p, T)):
            _put(x, lo, hi, val)
    elif k == "ns_grad":
        h = P
        for f in range(4):
            for a in range(3):
                _put(g[4 + 3 * f + a], lo, hi, _d1(g[f], lo, hi, a, h[a]))
    elif k == "ns_flux":
        gamma, Ma, Re, Pr = P
        mu, kc = _ns_consts(gamma, Ma, Re, Pr)
        Uv = [_get(x, lo, hi) for x in g[:5]]
        W = [_get(x, lo, hi) for x in g[5:9]]
        D = [_get(x, lo, hi) for x in g[9:21]]
        for m in range(5):
            for a in range(3):
                _put(g[21 + 3 * m + a], lo, hi, _ns_flux(Uv, W, D, mu, kc, m, a))
    elif k in ("ns_div", "ns_rhs"):
        if k == "ns_div":
            h, (Acoef, dt) = P[:3], P[3:]
            first = 15
        else:
            gamma, Ma, Re, Pr = P[:4]
            h, (Acoef, dt) = P[4:7], P[7:]
            mu, kc = _ns_consts(gamma, Ma, Re, Pr)
            first = 21
        for m in range(5):
            r = np.zeros([hi[a] - lo[a] for a in (2, 1, 0)])
            for a in range(3):
                if k == "ns_div":
                    r = r - _d1(g[3 * m + a], lo, hi, a, h[a])
                else:
                    vals = {}
                    for s in (-2, -1, 1, 2):
                        o = _unit(a, s)
                        Uv = [_get(x, lo, hi, o) for x in g[:5]]
                        W = [_get(x, lo, hi, o) for x in g[5:9]]
                        D = [_get(x, lo, hi, o) for x in g[9:21]]
                        vals[s] = _ns_flux(Uv, W, D, mu, kc, m, a)
                    r = r - ((vals[-2] - 8.0 * vals[-1]) + (8.0 * vals[1] - vals[2])) / (12.0 * h[a])
            out = g[first + m]
            if acc[first + m] == "rw":
                _put(out, lo, hi, Acoef * _get(out, lo, hi) + dt * r)
            else:
                _put(out, lo, hi, dt * r)
    elif k == "ns_update":
        B = P[0]
        for m in range(5):
            _put(g[m], lo, hi, _get(g[m], lo, hi) + B * _get(g[5 + m], lo, hi))


def run_loop(lp, fields: Dict, reds: Dict[str, float], red_ops: Dict[str, str]):
    """Evaluate one PDE loop (a `workloads.spec.Loop`) in place on `fields`."""
    if lp.kernel.startswith("euler_"):
        _euler(lp, fields, reds, red_ops)
    elif lp.kernel.startswith("ns_"):
        _ns(lp, fields, reds, red_ops)
    else:
        raise NotImplementedError(lp.kernel)


def refresh_ghosts(fields: Dict, names=None):
    """Deep ghosts of the periodic slow axis: every halo row y of a field periodic along
    its slowest axis takes interior row y mod n."""
    for nm, f in fields.items():
        if names is not None and nm not in names:
            continue
        sa = f.ndim - 1
        if sa not in getattr(f, "periodic", ()):
            continue
        n, h0 = f.size[sa], f.halo_lo[sa]
        for r in range(f.a.shape[0]):
            y = r - h0
            if y < 0 or y >= n:
                f.a[r] = f.a[(y % n) + h0]
