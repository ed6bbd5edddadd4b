"""FP64 oracle of the pseudo-arclength parameter continuation in the field
strength mu (Sec. 4, "Numerical parameter continuation").

TEST INFRASTRUCTURE ONLY: the test suite is the only caller.  The CUDA library
never imports this module; its own driver (``gl_continuation``) implements the
same steps on the device.

The paper names the method (a predictor-corrector in (psi, mu) whose corrector
is a Newton-Krylov process) and gives no formulas; the steps below are the
textbook pseudo-arclength method with a bordered Newton corrector, in the
project's reading:

* metric on (phi, nu):  ||(phi, nu)||^2 = <phi, phi>_R / |Omega| + nu^2
  (<.,.>_R of Eq. disc inner2; dividing by |Omega| makes psi = 1 have norm 1);
* the start (psi_0, mu_0) is first corrected by Newton at fixed mu_0; the first
  tangent is t = (c, 1) / ||(c, 1)|| with J c = -d GL / d mu (increasing mu);
  later tangents are secants, t = (psi_s - psi_{s-1}, mu_s - mu_{s-1}) / norm;
* predictor: (psi, mu) = (psi_s, mu_s) + ds t;
* corrector: Newton on GL(psi, mu) = 0 together with the arclength condition
  n(psi, mu) = <t_psi, psi - psi_s>_R / |Omega| + t_mu (mu - mu_s) - ds = 0.
  Each step solves J a = -GL and J c = -d GL / d mu (preconditioned MINRES, the
  preconditioner R_1(psi) set up once per step for both), then
      dmu  = (-n - <t_psi, a>_R / |Omega|) / (t_mu + <t_psi, c>_R / |Omega|),
      dpsi = a + dmu c,
  which solves the bordered system [J, dGL/dmu; t^T] (dpsi, dmu) = -(GL, n)
  (block elimination).  Converged when ||GL||_R / sqrt|Omega| <= newton_tol
  (checked before each step);
* step control: no convergence in newton_maxit steps (or a failed solve) halves
  ds and retries from the same point; after a converged step ds grows by 1.5
  (at most ds_max) if it took at most 2 Newton steps and shrinks by 0.7 (at
  least ds_min) if it took 5 or more;
* output per point: mu, the energy per unit volume F / |Omega| (Eq. discr
  energy; -1/2 for psi = 1 without field), Newton steps, the MINRES iterations
  of the last Newton step's J a = -GL solve (the quantity of Fig. 4, right),
  all MINRES iterations of the point (retries included), ||GL||_R / sqrt|Omega|,
  ds and the number of halvings.
"""
from __future__ import annotations

import numpy as np

from . import Mesh, Precond


def _defaults(**kw):
    o = dict(ds=0.05, ds_min=1e-4, ds_max=0.2, max_steps=20, mu_max=np.inf, newton_tol=1e-9, newton_maxit=8,
             linear_tol=1e-8, maxit=1000, max_coarse=512)
    o.update(kw)
    return o


def bordered_step(mesh, psi, t_psi, t_mu, ncond, r, vol_tot, **solver):
    """One corrector step: solves J a = -r and J c = -dGL/dmu with one R_1(psi)
    and eliminates the border row <t_psi, .>_R / |Omega| + t_mu (.) = -ncond.
    Returns (dpsi, dmu, info_a, info_c)."""
    ip = lambda x, y: mesh.inner_r(x, y) / vol_tot  # noqa: E731
    P = Precond(mesh, psi, **solver)
    a, ia = P.minres(-r)
    c, ic = P.minres(-mesh.residual_dmu(psi))
    dmu = (-ncond - ip(t_psi, a)) / (t_mu + ip(t_psi, c))
    return a + dmu * c, dmu, ia, ic


def _newton_fixed_mu(dim, N, edge, bhat, mu, psi, o):
    """Newton at fixed mu: returns (psi, steps, last iterations, total iterations, gnorm)."""
    steps = last = total = 0
    vol_tot = edge ** dim
    for _ in range(o["newton_maxit"] + 1):
        m = Mesh(dim, N, mu, bhat, edge=edge)
        r = m.residual(psi)
        g = np.sqrt(m.inner_r(r, r) / vol_tot)
        if g <= o["newton_tol"]:
            return psi, steps, last, total, g, True
        if steps == o["newton_maxit"]:
            break
        P = Precond(m, psi, tol=o["linear_tol"], maxit=o["maxit"], max_coarse=o["max_coarse"])
        a, info = P.minres(-r)
        if not info.converged:
            break
        psi = psi + a
        steps += 1
        last = info.iters
        total += info.iters
    return psi, steps, last, total, g, False


def continuation(dim, N, edge, psi0, mu0, bhat=(0.0, 0.0, 1.0), **kw):
    """Pseudo-arclength continuation from (psi0, mu0).  Returns (points, psi, mu)
    with one point for the corrected start and one per accepted step."""
    o = _defaults(**kw)
    vol_tot = edge ** dim
    ip = lambda m, x, y: m.inner_r(x, y) / vol_tot  # noqa: E731
    psi, mu = np.array(psi0, np.complex128), float(mu0)
    psi, steps, last, total, g, ok = _newton_fixed_mu(dim, N, edge, bhat, mu, psi, o)
    if not ok:
        raise RuntimeError("Newton at the start did not converge")
    m = Mesh(dim, N, mu, bhat, edge=edge)
    points = [dict(mu=mu, energy=m.energy(psi) / vol_tot, newton=steps, iters_last=last, iters_total=total,
                   gl_norm=g, ds=0.0, retries=0)]
    # first tangent from J c = -dGL/dmu
    P = Precond(m, psi, tol=o["linear_tol"], maxit=o["maxit"], max_coarse=o["max_coarse"])
    c, info = P.minres(-m.residual_dmu(psi))
    nrm = np.sqrt(ip(m, c, c) + 1.0)
    t_psi, t_mu = c / nrm, 1.0 / nrm
    ds = o["ds"]
    for _ in range(o["max_steps"]):
        if mu >= o["mu_max"]:
            break
        total = retries = 0
        while True:
            psi_n, mu_n = psi + ds * t_psi, mu + ds * t_mu
            steps = last = 0
            ok = False
            for it in range(o["newton_maxit"] + 1):
                mn = Mesh(dim, N, mu_n, bhat, edge=edge)
                r = mn.residual(psi_n)
                g = np.sqrt(ip(mn, r, r))
                if g <= o["newton_tol"]:
                    ok = True
                    break
                if it == o["newton_maxit"]:
                    break
                ncond = ip(mn, t_psi, psi_n - psi) + t_mu * (mu_n - mu) - ds
                dpsi, dmu, ia, ic = bordered_step(mn, psi_n, t_psi, t_mu, ncond, r, vol_tot, tol=o["linear_tol"],
                                                  maxit=o["maxit"], max_coarse=o["max_coarse"])
                total += ia.iters + ic.iters
                if not (ia.converged and ic.converged):
                    break
                psi_n = psi_n + dpsi
                mu_n = mu_n + dmu
                steps += 1
                last = ia.iters
            if ok:
                break
            ds *= 0.5
            retries += 1
            if ds < o["ds_min"]:
                return points, psi, mu
        dpsi, dmu = psi_n - psi, mu_n - mu
        nrm = np.sqrt(ip(mn, dpsi, dpsi) + dmu * dmu)
        t_psi, t_mu = dpsi / nrm, dmu / nrm
        psi, mu = psi_n, mu_n
        points.append(dict(mu=mu, energy=mn.energy(psi) / vol_tot, newton=steps, iters_last=last,
                           iters_total=total, gl_norm=g, ds=ds, retries=retries))
        if steps <= 2:
            ds = min(ds * 1.5, o["ds_max"])
        elif steps >= 5:
            ds = max(ds * 0.7, o["ds_min"])
    return points, psi, mu
