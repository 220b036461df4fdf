"""Primal-dual interior-point method for Eq. 1, FP64, dense: the oracle's solver.

TEST INFRASTRUCTURE ONLY.

Eq. 1 is min f(v) s.t. c(v) = 0 with bounds on v; Eq. 2 is the Newton system of such a method,
    [ W + alpha   A^T ] [ dv ]      [ grad f + A^T lambda + beta ]
    [ A           0   ] [ dl ]  = - [ c                          ],
with W the Hessian of the Lagrangian (Eq. 6 for the network part).  The paper leaves alpha and
beta unstated.  They are read here as the terms of the primal-dual barrier method of IPOPT
(Waechter & Biegler 2006, cited for the solver):  alpha = Sigma + delta_w I with
Sigma = Z_L (V - L)^-1 + Z_U (U - V)^-1 and delta_w the inertia correction, and beta the barrier
terms -mu/(v - L) + mu/(U - v) plus the bound multipliers they replace.  The steps, in order:

  start    push v into the bounds (kappa_1 = kappa_2 = 1e-2), z = 1, lambda = 0, mu = mu_0 = 0.1
  each iteration
    1  evaluate f, grad f, c, A, and the scaled optimality error E_mu (s_max = 100); stop when
       E_0 <= tol = 1e-6; while E_mu <= kappa_eps mu (kappa_eps = 10) lower
       mu <- max(tol/10, min(kappa_mu mu, mu^theta_mu)) with kappa_mu = 0.2, theta_mu = 1.5
    2  W = grad^2 f + sum_i lambda_i grad^2 c_i
    3  KKT matrix [[W + Sigma + delta_w I, A^T], [A, -delta_c I]]; its inertia must be
       (n, m, 0) (n positive, m negative, no zero eigenvalues); otherwise raise delta_w
       (first 1e-4, or a third of the last value; then x8, or x100 if no earlier value), and
       use delta_c = 1e-8 mu^(1/4) if the matrix is singular
    4  solve for (dv, dl); dz_L = mu/(v-L) - z_L - Sigma_L dv, dz_U = mu/(U-v) - z_U + Sigma_U dv
    5  fraction to the boundary with tau = max(0.99, 1 - mu) for v (alpha_max) and z (alpha_z)
    6  backtracking line search on the exact-penalty merit function
       phi(v) = f(v) - mu sum ln(v - L) - mu sum ln(U - v) + nu ||c(v)||_1  (Armijo 1e-4, halving),
       nu raised so that the step is a descent direction
    7  v += alpha dv, lambda += alpha dl, z += alpha_z dz; keep z within a factor
       kappa_Sigma = 1e10 of mu / slack.
A warm start (a predicted point v, lambda) replaces the start: v pushed into the bounds as above,
lambda as given, mu = warm_mu0 = 1e-3 and z = mu / slack, so every complementarity product starts
at mu.
The inertia here is the plain definition (signs of the eigenvalues, numpy eigvalsh, taken on a
congruent diagonally scaled copy so that the zero test is scale-invariant); the solve is numpy's
dense solver.  Iteration counts need not match IPOPT's (no filter, no
second-order correction, no restoration phase).
"""
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

OPTIMAL, MAX_ITER, LINESEARCH_FAILED, NONFINITE, INERTIA_FAILED = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "optimal", 1: "max_iter", 2: "linesearch_failed", 3: "nonfinite",
                4: "inertia_failed"}


@dataclass
class Options:
    tol: float = 1e-6
    max_iter: int = 300
    mu0: float = 0.1
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    kappa_eps: float = 10.0
    tau_min: float = 0.99
    kappa1: float = 1e-2
    kappa2: float = 1e-2
    s_max: float = 100.0
    eta: float = 1e-4
    delta_w0: float = 1e-4
    delta_w_min: float = 1e-20
    delta_w_max: float = 1e40
    kappa_w_plus: float = 8.0
    kappa_w_plus_bar: float = 100.0
    kappa_w_minus: float = 1.0 / 3.0
    kappa_sigma: float = 1e10
    max_backtracks: int = 40
    max_ls_failures: int = 5
    warm_mu0: float = 1e-3


@dataclass
class Problem:
    """min f(v) s.t. c(v) = 0, lb <= v <= ub (entries may be +-inf)."""
    n: int
    m: int
    lb: np.ndarray
    ub: np.ndarray
    v0: np.ndarray
    f: Callable
    grad_f: Callable
    hess_f: Callable            # v -> dense n x n
    c: Callable                 # v -> m
    jac_c: Callable             # v -> dense m x n
    hess_c: Callable            # (v, lam) -> dense n x n, sum_i lam_i grad^2 c_i


@dataclass
class Result:
    status: int
    v: np.ndarray
    lam: np.ndarray
    zL: np.ndarray
    zU: np.ndarray
    obj: float
    iters: int
    kkt_error: float
    history: list = field(default_factory=list)


def _errors(p, v, lam, zL, zU, mu, g, cval, A, hasL, hasU, s_max):
    rd = g + (A.T @ lam if p.m else 0.0) - zL + zU
    nb = int(hasL.sum() + hasU.sum())
    s_d = max(s_max, (np.abs(lam).sum() + np.abs(zL).sum() + np.abs(zU).sum()) / max(1, p.m + nb)) / s_max
    s_c = max(s_max, (np.abs(zL).sum() + np.abs(zU).sum()) / max(1, nb)) / s_max
    sL = np.where(hasL, v - np.where(hasL, p.lb, 0.0), 0.0)
    sU = np.where(hasU, np.where(hasU, p.ub, 0.0) - v, 0.0)
    compL = np.where(hasL, sL * zL - mu, 0.0) if hasL.any() else np.zeros(1)
    compU = np.where(hasU, sU * zU - mu, 0.0) if hasU.any() else np.zeros(1)
    cinf = np.abs(cval).max() if p.m else 0.0
    return max(np.abs(rd).max() / s_d, cinf, max(np.abs(compL).max(), np.abs(compU).max()) / s_c)


def _inertia(K, tol=0.0):
    """(positive, negative, zero) eigenvalue counts of K.  The signs are taken after a symmetric
    diagonal scaling D K D (D_ii = 1 / sqrt(max_j |K_ij|)): a congruence, so by Sylvester's law of
    inertia the counts are those of K, while the zero test (relative to the largest eigenvalue)
    no longer mistakes the small negative eigenvalues of a badly scaled KKT matrix (barrier terms
    of order 1e10 next to constraint rows of order 1) for zeros."""
    rmax = np.abs(K).max(axis=1)
    d = 1.0 / np.sqrt(np.where(rmax > 0.0, rmax, 1.0))
    ev = np.linalg.eigvalsh(K * d[:, None] * d[None, :])
    scale = max(1.0, np.abs(ev).max())
    zero = np.abs(ev) <= 1e-14 * scale
    return int(((ev > 0) & ~zero).sum()), int(((ev < 0) & ~zero).sum()), int(zero.sum())


def solve(p: Problem, opt: Optional[Options] = None, callback=None, warm=None) -> Result:
    """warm = (v_start, lam_start) starts from a predicted point (a learned warm start): v_start
    is pushed into the bounds like any start, lambda = lam_start, mu = warm_mu0 and every bound
    multiplier is rebuilt as z = mu / slack."""
    opt = opt or Options()
    n, m = p.n, p.m
    lb, ub = np.asarray(p.lb, float), np.asarray(p.ub, float)
    hasL, hasU = np.isfinite(lb), np.isfinite(ub)
    # --- start: push v0 into the bounds
    v = np.array(p.v0 if warm is None else warm[0], dtype=np.float64)
    width = np.where(hasL & hasU, ub - lb, np.inf)
    pL = np.minimum(opt.kappa1 * np.maximum(1.0, np.abs(np.where(hasL, lb, 0.0))), opt.kappa2 * width)
    pU = np.minimum(opt.kappa1 * np.maximum(1.0, np.abs(np.where(hasU, ub, 0.0))), opt.kappa2 * width)
    v = np.where(hasL, np.maximum(v, lb + pL), v)
    v = np.where(hasU, np.minimum(v, ub - pU), v)
    zL = np.where(hasL, 1.0, 0.0)
    zU = np.where(hasU, 1.0, 0.0)
    lam = np.zeros(m)
    mu = opt.mu0
    if warm is not None:
        lam = np.array(warm[1], dtype=np.float64)
        mu = opt.warm_mu0
        zL = np.where(hasL, mu / np.where(hasL, v - np.where(hasL, lb, 0.0), 1.0), 0.0)
        zU = np.where(hasU, mu / np.where(hasU, np.where(hasU, ub, 0.0) - v, 1.0), 0.0)
    tau = max(opt.tau_min, 1.0 - mu)
    nu = 1.0
    delta_w_last = 0.0
    ls_fail = 0
    hist = []
    lb0, ub0 = np.where(hasL, lb, 0.0), np.where(hasU, ub, 0.0)
    slackL = lambda vv: np.where(hasL, vv - lb0, 1.0)  # noqa: E731
    slackU = lambda vv: np.where(hasU, ub0 - vv, 1.0)  # noqa: E731

    def barrier_merit(vv, fv, cv, nu_):
        sL, sU = slackL(vv), slackU(vv)
        if np.any(sL[hasL] <= 0) or np.any(sU[hasU] <= 0):
            return np.inf
        return fv - mu * np.log(sL[hasL]).sum() - mu * np.log(sU[hasU]).sum() + nu_ * (np.abs(cv).sum() if m else 0.0)

    status = MAX_ITER
    E0 = np.inf
    it = 0
    for it in range(opt.max_iter + 1):
        fv, g = p.f(v), p.grad_f(v)
        cval = p.c(v) if m else np.zeros(0)
        A = p.jac_c(v) if m else np.zeros((0, n))
        if not (np.isfinite(fv) and np.all(np.isfinite(g)) and np.all(np.isfinite(cval)) and np.all(np.isfinite(A))):
            status = NONFINITE
            break
        E0 = _errors(p, v, lam, zL, zU, 0.0, g, cval, A, hasL, hasU, opt.s_max)
        hist.append(dict(it=it, f=fv, inf_pr=float(np.abs(cval).max()) if m else 0.0, E0=E0, mu=mu))
        if callback:
            callback(hist[-1])
        if E0 <= opt.tol:
            status = OPTIMAL
            break
        if it == opt.max_iter:
            break
        Emu = _errors(p, v, lam, zL, zU, mu, g, cval, A, hasL, hasU, opt.s_max)
        while Emu <= opt.kappa_eps * mu and mu > opt.tol / 10.0:
            mu = max(opt.tol / 10.0, min(opt.kappa_mu * mu, mu ** opt.theta_mu))
            tau = max(opt.tau_min, 1.0 - mu)
            Emu = _errors(p, v, lam, zL, zU, mu, g, cval, A, hasL, hasU, opt.s_max)
        # --- Newton system (Eq. 2 with the barrier terms)
        W = p.hess_f(v) + (p.hess_c(v, lam) if m else 0.0)
        sL, sU = slackL(v), slackU(v)
        SigL = np.where(hasL, zL / sL, 0.0)
        SigU = np.where(hasU, zU / sU, 0.0)
        grad_phi = g - np.where(hasL, mu / sL, 0.0) + np.where(hasU, mu / sU, 0.0)
        rhs = -np.concatenate([grad_phi + (A.T @ lam if m else 0.0), cval])
        delta_w, delta_c = 0.0, 0.0
        first = True
        while True:
            K = np.zeros((n + m, n + m))
            K[:n, :n] = W + np.diag(SigL + SigU + delta_w)
            if m:
                K[n:, :n] = A
                K[:n, n:] = A.T
                K[n:, n:] = -delta_c * np.eye(m)
            npos, nneg, nzero = _inertia(K)
            if npos == n and nneg == m and nzero == 0:
                break
            if nzero > 0 and delta_c == 0.0 and m:
                delta_c = 1e-8 * mu ** 0.25
            if first:
                delta_w = opt.delta_w0 if delta_w_last == 0.0 else max(opt.delta_w_min, opt.kappa_w_minus * delta_w_last)
                first = False
            else:
                delta_w *= opt.kappa_w_plus_bar if delta_w_last == 0.0 else opt.kappa_w_plus
            if delta_w > opt.delta_w_max:
                break
        if delta_w > opt.delta_w_max:
            status = INERTIA_FAILED
            break
        if delta_w > 0.0:
            delta_w_last = delta_w
        sol = np.linalg.solve(K, rhs)
        dv, dl = sol[:n], sol[n:]
        dzL = np.where(hasL, mu / sL - zL - SigL * dv, 0.0)
        dzU = np.where(hasU, mu / sU - zU + SigU * dv, 0.0)
        # --- fraction to the boundary
        a_max = 1.0
        neg = hasL & (dv < 0)
        if neg.any():
            a_max = min(a_max, np.min(-tau * sL[neg] / dv[neg]))
        pos = hasU & (dv > 0)
        if pos.any():
            a_max = min(a_max, np.min(tau * sU[pos] / dv[pos]))
        a_z = 1.0
        for zz, dz, has in ((zL, dzL, hasL), (zU, dzU, hasU)):
            nz = has & (dz < 0)
            if nz.any():
                a_z = min(a_z, np.min(-tau * zz[nz] / dz[nz]))
        # --- merit function and penalty parameter
        c1 = np.abs(cval).sum() if m else 0.0
        dphi_b = grad_phi @ dv
        if m and c1 > 0:
            curv = dv @ (K[:n, :n] @ dv)
            nu_req = (dphi_b + 0.5 * max(curv, 0.0)) / (0.9 * c1)
            nu = max(nu, np.abs(lam + dl).max() + 1.0, nu_req + 1.0)
        D = dphi_b - nu * c1
        phi0 = barrier_merit(v, fv, cval, nu)
        alpha = a_max
        accepted = False
        for _ in range(opt.max_backtracks):
            vt = v + alpha * dv
            ft = p.f(vt)
            ct = p.c(vt) if m else np.zeros(0)
            phit = barrier_merit(vt, ft, ct, nu)
            if np.isfinite(phit) and phit <= phi0 + opt.eta * alpha * D:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            ls_fail += 1
            if ls_fail >= opt.max_ls_failures:
                status = LINESEARCH_FAILED
                break
        else:
            ls_fail = 0
        v = v + alpha * dv
        lam = lam + alpha * dl
        zL = zL + a_z * dzL
        zU = zU + a_z * dzU
        sL, sU = slackL(v), slackU(v)
        zL = np.where(hasL, np.maximum(np.minimum(zL, opt.kappa_sigma * mu / sL), mu / (opt.kappa_sigma * sL)), 0.0)
        zU = np.where(hasU, np.maximum(np.minimum(zU, opt.kappa_sigma * mu / sU), mu / (opt.kappa_sigma * sU)), 0.0)
        hist[-1].update(alpha=alpha, alpha_z=a_z, delta_w=delta_w, nu=nu)
    return Result(status, v, lam, zL, zU, float(p.f(v)), it, float(E0), hist)
