"""Shared helpers of the GPU tests (runs the CUDA path and the oracle side by side)."""
import numpy as np

import ctqw_workloads as cw

# Tolerances stated for the hot path: max |dP(x)| against the FP64 oracle.
TOL_FP64 = 1e-11
TOL_FP32 = 2e-6
TOL_NORM_DRIFT = 1e-6
U_FP32 = 2.0 ** -24       # unit roundoff of FP32

# The tensor-core one-body density (Sec. 4 builds <rho> with a single-
# precision Hermitian update): each real product from three TF32 piece
# products (the dropped and rounded pieces at most ~2^-21 of it), summed in
# FP32 in tensor memory over blocks of 256 k, then in two-word FP32 and FP64.
# The tensor cores' FP32 accumulation may round every add toward zero (a
# dense random state at N = 2048 shows a one-sided 4.6e-6 on the diagonal),
# so a block carries up to 256 ulp = 256 * 2^-23 of its sum of |terms|,
# itself at most the largest element of rho1 (Cauchy-Schwarz on the
# diagonal).
TOL_TC = 256 * 2.0 ** -23


def h_bound(w):
    """Upper bound of ||H||_2 from the workload's description (Gershgorin on
    the Kronecker sum): m (max|eps| + 2 max|J|) + |U| m (m - 1) / 2."""
    eps_max = abs(0.0) + w.eps_halfwidth
    J_max = abs(w.J0) + w.J_halfwidth
    return w.m * (eps_max + 2.0 * J_max) + abs(w.U) * w.m * (w.m - 1) / 2.0


def energy_tol(w):
    """Tolerance on an FP32 path's energy, <psi|H|psi>, against the oracle.

    E = sum_s conj(psi_s) (H psi)_s with every quantity that enters it within
    a few FP32 roundings of exact: storing the state in FP32 moves E by at
    most u ||H|| (the compensated update keeps the propagated state there),
    forming H psi and the product in FP32 adds at most 8 u ||H|| (six
    roundings in the stencil, two in the product, each relative to
    sum |psi| (|H| |psi|) <= ||H||), and the FP64 (or exact) sums add
    nothing at this scale.  16 u ||H|| leaves the remaining 7 u ||H|| for
    the state's drift over the run, which the norm bounds at ~4 u here.
    """
    return 16.0 * U_FP32 * h_bound(w)


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
