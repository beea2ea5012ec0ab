"""Density-scale characterisation by gradient (the application the paper's
differentiable use motivates: dead-layer characterisation, self-absorption).

Given measured FEPE values m_i +- sigma_i for a set of instances (energies,
sources), find the density scales s_p of the chosen groups that minimise

    chi2(s) = sum_i (FEPE_i(s) - m_i)^2 / (sigma_i^2 + sigma_sim,i^2)

by Gauss-Newton steps.  Each step runs the score-accumulating transport once
(``gadep_grad``): it returns FEPE_i(s) and the Jacobian dFEPE_i/ds_p from the
density-perturbation scores of the same histories, so no finite differences
are needed.  Every evaluation replays the same histories (same seed), so
chi2(s) is a smooth function of s up to the discreteness of the tallies.
"""
from __future__ import annotations

import numpy as np

from . import api


def fit_density_scales(bvh, mats, items, targets, target_sigma, free_groups, s0, n_group=4, iters=10,
                       tol=1e-4, max_step=0.5, opts_kw=None):
    """Fit the scales of ``free_groups``.

    items: [(energy, workloads.Source, n_hist, instance id)] simulated per call;
    targets, target_sigma: measured FEPE per item; s0: the n_group starting scales
    (groups not in free_groups stay fixed).  Returns (scales, sigma of the free
    scales from (J^T W J)^-1, list of per-step records)."""
    s = np.array(s0, dtype=np.float64)
    free = list(free_groups)
    m = np.asarray(targets, dtype=np.float64)
    sm = np.asarray(target_sigma, dtype=np.float64)
    history = []
    cov = None
    for it in range(iters):
        inst = api.make_instances([(E, src, n, iid, list(s)) for E, src, n, iid in items])
        res, _, d, ds = api.gadep_grad(bvh, mats, inst, api.make_opts(n_group=n_group, **(opts_kw or {})))
        f = np.array([r["fepe"] for r in res])
        sig = np.sqrt(sm ** 2 + np.array([r["sigma"] for r in res]) ** 2)
        J = d[:, free] / sig[:, None]
        r = (f - m) / sig
        step, *_ = np.linalg.lstsq(J, -r, rcond=None)
        step = np.clip(step, -max_step, max_step)
        cov = np.linalg.pinv(J.T @ J)
        history.append({"scales": s.copy(), "chi2": float(r @ r), "fepe": f, "step": step.copy()})
        s[free] = np.maximum(s[free] + step, 1e-3)
        if np.max(np.abs(step)) < tol:
            break
    sigma = np.sqrt(np.diag(cov)) if cov is not None else np.full(len(free), np.nan)
    return s, sigma, history
