"""Forward-mode gradient of the smooth CVA_0 in FP64 dual numbers.

TEST INFRASTRUCTURE ONLY (part of the oracle): the tests use it to check the CUDA
adjoint; the product path never imports it.

The smooth CVA_0 is the exact discrete form of the intensity formula eq.
(eq:CVAint) at the first pricing date,

    CVA_0 = mean_k sum_c sum_{j=1..n} (1 - R_c) beta_j (MtM^c_j)^+ (e^{-Lambda^c_{j-1}} - e^{-Lambda^c_j}),

on the model of Sec. 4.1 and App. B: Hull-White short rates r^e with the quanto drift
under Q^0, lognormal FX rates chi^e, CIR intensities gamma^c with full truncation,
Euler-Maruyama sub-steps with left-point integrals (Remark rem:finecoarse), and swaps
priced by the three-case formula of App. B with the Hull-White zero-coupon closed
form. Its arithmetic follows the C oracle (cva_oracle.c) step by step, with every
quantity carried as a value and its tangents: the derivative along each of the
parameter directions, propagated by the chain rule of each operation (forward-mode
automatic differentiation, one pass for all directions). The standard normals are the
oracle's own (Philox4x32-10, Box-Muller), so the value equals the C oracle's smooth
CVA_0 up to rounding order, which pins the restatement; the tangents are then exact
derivatives of that same arithmetic.

Directions, in the order of the CUDA library's gradient: curve levels f_e (E), rate
volatilities sigma^r_e (E), FX volatilities sigma^chi_e for e = 1..E-1, CIR kappa_c,
theta_c, nu_c (C each); then, beyond it, the recoveries R_c (C). The swaps' fixed
rates are held fixed (the portfolio must carry them), as are gamma_0, the mean
reversions a_e and the correlations.
"""
from __future__ import annotations

from typing import Dict

import numpy as np

from . import normals as _normals


class Dual:
    """A value v (shape (1,) or (M,)) and its tangents d (shape (P, 1) or (P, M))."""
    __slots__ = ("v", "d")

    def __init__(self, v, d):
        self.v = v
        self.d = d

    def __add__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v + o.v, self.d + o.d)
        return Dual(self.v + o, self.d)

    __radd__ = __add__

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __sub__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v - o.v, self.d - o.d)
        return Dual(self.v - o, self.d)

    def __rsub__(self, o):
        return Dual(o - self.v, -self.d)

    def __mul__(self, o):
        if isinstance(o, Dual):   # (a b)' = a' b + a b'
            return Dual(self.v * o.v, self.d * o.v + o.d * self.v)
        return Dual(self.v * o, self.d * o)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, Dual):   # (a / b)' = (a' b - a b') / b^2
            return Dual(self.v / o.v, (self.d * o.v - o.d * self.v) / (o.v * o.v))
        return Dual(self.v / o, self.d / o)

    def __rtruediv__(self, o):    # (c / b)' = -c b' / b^2
        return Dual(o / self.v, -o * self.d / (self.v * self.v))


def exp(x: Dual) -> Dual:
    e = np.exp(x.v)
    return Dual(e, x.d * e)


def sqrt(x: Dual) -> Dual:
    """sqrt with the derivative d / (2 sqrt(v)) where v > 0 and 0 at v = 0 (the
    truncated CIR intensity has a zero tangent there)."""
    s = np.sqrt(x.v)
    safe = np.where(s > 0.0, s, 1.0)
    return Dual(s, np.where(x.v > 0.0, x.d / (2.0 * safe), 0.0))


def pos(x: Dual) -> Dual:
    """x^+ = max(x, 0), derivative 1 where x > 0 and 0 elsewhere."""
    return Dual(np.where(x.v > 0.0, x.v, 0.0), np.where(x.v > 0.0, x.d, 0.0))


def n_directions(model) -> int:
    """3E - 1 + 3C directions of the CUDA gradient, then C recoveries."""
    return 3 * model.E - 1 + 4 * model.C


def _param(value: float, i: int, P: int) -> Dual:
    d = np.zeros((P, 1))
    d[i, 0] = 1.0
    return Dual(np.array([float(value)]), d)


def _const(value: float, P: int) -> Dual:
    return Dual(np.array([float(value)]), np.zeros((P, 1)))


def smooth_cva0_grad(model, pf, grid, M: int, seed: int, k0: int = 0) -> Dict[str, np.ndarray]:
    """Smooth CVA_0 over outer paths [k0, k0 + M) and its derivatives.

    Returns {"cva0": float, "grad": [3E - 1 + 3C] (the CUDA gradient's order),
    "grad_recovery": [C], "cva0_c": [C] (each counterparty's share of CVA_0)}.
    """
    if getattr(pf, "fixed_rate", None) is None:
        raise ValueError("the portfolio must carry its fixed rates (trade terms held fixed)")
    E, C = model.E, model.C
    n, S = grid.n_steps, grid.substeps
    P = n_directions(model)
    Delta = grid.horizon / n
    ds = Delta / S
    sqds = np.sqrt(ds)
    ppp = int(round(pf.delta / Delta))
    if ppp < 1 or abs(pf.delta / Delta - ppp) > 1e-9 * ppp:
        raise ValueError("reset dates must lie on the pricing grid")

    # parameters as duals (tangent = unit direction) and constants
    f = [_param(model.curve[e], e, P) for e in range(E)]
    sr = [_param(model.hw_sigma[e], E + e, P) for e in range(E)]
    sx = [_const(0.0, P)] + [_param(model.fx_vol[e], 2 * E + e - 1, P) for e in range(1, E)]
    o = 3 * E - 1
    kap = [_param(model.cir_kappa[c], o + c, P) for c in range(C)]
    the = [_param(model.cir_theta[c], o + C + c, P) for c in range(C)]
    nu = [_param(model.cir_nu[c], o + 2 * C + c, P) for c in range(C)]
    rec = [_param(model.recovery[c], o + 3 * C + c, P) for c in range(C)]
    a = np.asarray(model.hw_a, dtype=np.float64)
    corr = np.asarray(model.corr, dtype=np.float64)

    # factor positions in the correlated normal vector
    pos_r = list(range(E))
    pos_x = [-1] + list(range(E, 2 * E - 1))
    pos_g, p = [], 2 * E - 1
    for c in range(C):
        if model.cir_nu[c] > 0.0:
            pos_g.append(p)
            p += 1
        else:
            pos_g.append(-1)
    F = p
    L = np.linalg.cholesky(corr)

    def zc_hw(e: int, t: float, T: float, r: Dual) -> Dual:
        """Hull-White zero-coupon bond of App. B for the flat curve f_e."""
        B = (1.0 - np.exp(-a[e] * (T - t))) / a[e]
        lnA = f[e] * (-(T - t) + B) - sr[e] * sr[e] * ((1.0 - np.exp(-2.0 * a[e] * t)) * B * B / (4.0 * a[e]))
        return exp(lnA - r * B)

    def hw_theta(e: int, t: float) -> Dual:
        return f[e] * a[e] + sr[e] * sr[e] * ((1.0 - np.exp(-2.0 * a[e] * t)) / (2.0 * a[e]))

    # the portfolio's swaps, each priced on its own
    ccy = np.asarray(pf.ccy)
    cpty = np.asarray(pf.cpty)
    nper = np.asarray(pf.n_periods)
    w = np.asarray(pf.omega) * np.asarray(pf.notional, dtype=np.float64)
    Sig = np.asarray(pf.fixed_rate, dtype=np.float64)
    delta = float(pf.delta)

    # standard normals of every fine step: z[q] is [M, F]
    paths = range(k0, k0 + M)
    z = np.stack([np.stack([_normals(seed, k, q, F) for k in paths]) for q in range(n * S)])

    r = [f[e] * np.ones(M) for e in range(E)]
    lchi = [_const(np.log(model.fx0[e]), P) * np.ones(M) for e in range(E)]
    rfix = list(r)
    gam = [_const(model.gamma0[c], P) * np.ones(M) for c in range(C)]
    Lam_prev = [_const(0.0, P) * np.ones(M) for _ in range(C)]
    Iacc = _const(0.0, P) * np.ones(M)
    share = [_const(0.0, P) * np.ones(M) for _ in range(C)]
    q_rho = [corr[pos_r[e], pos_x[e]] if e > 0 else 0.0 for e in range(E)]

    for j in range(n + 1):
        Lam = list(Lam_prev)
        if j > 0:
            for s in range(S):
                q = (j - 1) * S + s
                t = q * ds
                W = z[q] @ L.T                                     # [M, F]
                dr = []
                for e in range(E):
                    drift = hw_theta(e, t) - r[e] * a[e]
                    if e > 0:   # quanto adjustment Q^e -> Q^0 (App. B)
                        drift = drift - sx[e] * sr[e] * q_rho[e]
                    dr.append(drift * ds + sr[e] * (sqds * W[:, pos_r[e]]))
                dl = [None] + [(r[0] - r[e] - sx[e] * sx[e] * 0.5) * ds + sx[e] * (sqds * W[:, pos_x[e]])
                               for e in range(1, E)]
                dg = []
                for c in range(C):
                    if pos_g[c] < 0:
                        dg.append(None)
                        continue
                    gp = pos(gam[c])
                    dg.append((the[c] - gp) * kap[c] * ds + nu[c] * sqrt(gp) * (sqds * W[:, pos_g[c]]))
                Iacc = Iacc + r[0] * ds                           # left-point integrals
                for c in range(C):
                    Lam[c] = Lam[c] + pos(gam[c]) * ds
                r = [r[e] + dr[e] for e in range(E)]
                lchi = [lchi[0]] + [lchi[e] + dl[e] for e in range(1, E)]
                gam = [gam[c] + dg[c] if dg[c] is not None else gam[c] for c in range(C)]

        # pricing date t_j: MtM of each counterparty, swap by swap (App. B)
        t = j * Delta
        on_reset = (j % ppp) == 0
        qp = j // ppp
        mtm = [_const(0.0, P) * np.ones(M) for _ in range(C)]
        memo = {}

        def zc(e, t0, T, rr, tag):   # the date's bond prices, each computed once
            key = (e, tag, t0, T)
            if key not in memo:
                memo[key] = zc_hw(e, t0, T, rr)
            return memo[key]

        for sw in range(len(ccy)):
            e, npr = int(ccy[sw]), int(nper[sw])
            tbar = npr * delta
            if on_reset and qp == 0:
                ann = zc(e, 0.0, delta, r[e], 0)
                for g in range(2, npr + 1):
                    ann = ann + zc(e, 0.0, g * delta, r[e], 0)
                pv = 1.0 - zc(e, 0.0, tbar, r[e], 0) - ann * (delta * Sig[sw])
            elif on_reset:
                if qp > npr:
                    continue
                t_minus = (qp - 1) * delta
                ann = _const(1.0, P) * np.ones(M)   # ZC_t(t) = 1, the coupon paid today
                for g in range(qp + 1, npr + 1):
                    ann = ann + zc(e, t, g * delta, r[e], 0)
                pv = 1.0 / zc(e, t_minus, t, rfix[e], 1) - zc(e, t, tbar, r[e], 0) - ann * (delta * Sig[sw])
            else:
                if qp + 1 > npr:
                    continue
                t_minus, t_plus = qp * delta, (qp + 1) * delta
                ann = zc(e, t, (qp + 1) * delta, r[e], 0)
                for g in range(qp + 2, npr + 1):
                    ann = ann + zc(e, t, g * delta, r[e], 0)
                pv = zc(e, t, t_plus, r[e], 0) / zc(e, t_minus, t_plus, rfix[e], 1) - zc(e, t, tbar, r[e], 0) \
                    - ann * (delta * Sig[sw])
            val = pv * w[sw] if e == 0 else exp(lchi[e]) * pv * w[sw]
            mtm[int(cpty[sw])] = mtm[int(cpty[sw])] + val
        if on_reset:
            rfix = list(r)
        if j > 0:   # the j-th term of the smooth form: (1 - R_c) beta_j MtM^+ (e^{-Lam_{j-1}} - e^{-Lam_j})
            beta = exp(-Iacc)
            for c in range(C):
                V = (1.0 - rec[c]) * beta * pos(mtm[c])
                share[c] = share[c] + V * (exp(-Lam_prev[c]) - exp(-Lam[c]))
        Lam_prev = Lam

    cva0_c = np.array([float(np.mean(sc.v)) for sc in share])
    tot = share[0]
    for c in range(1, C):
        tot = tot + share[c]
    g = np.mean(tot.d, axis=1)
    nc = 3 * E - 1 + 3 * C
    return {"cva0": float(np.mean(tot.v)), "grad": g[:nc], "grad_recovery": g[nc:], "cva0_c": cva0_c}
