"""Shared helpers of the GPU tests (runs the CUDA path and the oracle side by side)."""
import numpy as np

import ctqw_workloads as cw

# Tolerances stated for the hot path: max |dP(x)| against the FP64 oracle.
TOL_FP64 = 1e-11
TOL_FP32 = 2e-6
TOL_NORM_DRIFT = 1e-6


def oracle_params(w, realizations=None, eps_mean=None, J_mean=None):
    """Oracle (eps, J) per realization, J padded to N entries (wrap bond last)."""
    import oracle

    sizes = w.sizes()
    realizations = range(w.R) if realizations is None else realizations
    realizations = list(realizations)
    ue, uj = cw.uniform_draws(w.seed, realizations, [sizes[r] for r in realizations])
    out = []
    for k, r in enumerate(realizations):
        N = int(sizes[r])
        eps, J = oracle.workload_parameters(w, ue[k], uj[k], N, eps_mean, J_mean)
        Jp = np.zeros(N)
        Jp[:len(J)] = J
        out.append((eps, Jp))
    return out


def per_realization_P(psi_flat, st_off, sizes, m):
    """P_r(x) of every realization from the packed final states (host, FP64)."""
    out = []
    for r, N in enumerate(sizes):
        N = int(N)
        p = np.abs(psi_flat[st_off[r]:st_off[r + 1]].astype(np.complex128)) ** 2
        p = p.reshape((N,) * m)
        P = np.zeros(N)
        for j in range(m):
            P += p.sum(axis=tuple(a for a in range(m) if a != j))
        out.append(P / m)
    return out
