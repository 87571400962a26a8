// Exact propagation by diagonalisation, batched over realizations
// (Algorithm 1, Eq. (evolPsi)): psi(t) = W exp(-i E t) W^T psi(0) with
// H = W diag(E) W^T, in FP64, for small state dimensions D = N^m <= 64.
//
// One CTA per realization holds the dense H (built from its eps, J and U)
// and the eigenvector matrix in shared memory and diagonalises H with the
// cyclic Jacobi method in parallel form: a sweep is D-1 rounds, each round
// rotates D/2 disjoint index pairs (a round-robin schedule), first the rows
// of every pair, then the columns, so the pairs do not interfere.  The
// rotation of pair (p, q) zeroes H_pq: with tau = (H_qq - H_pp) / (2 H_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c.
// Sweeps repeat until the off-diagonal Frobenius norm is below 1e-13 of the
// whole (the FP64 rounding floor of a 64 x 64 matrix is near 1e-14), at most kMaxSweeps (a fixed bound, no open-ended wait).  An odd D
// is padded with one decoupled zero row and column.
#include <cmath>

#include "ctqw_internal.cuh"
#include "stencil.cuh"

namespace {

constexpr int kMaxD = 64;
constexpr int kMaxSweeps = 40;

__global__ void __launch_bounds__(256) exact_eigen_kernel(RealTable tab, const double *__restrict__ eps,
                                                          const double *__restrict__ J, double *evals,
                                                          double *evecs, int Dp_max, int *sweeps_out) {
    extern __shared__ double sm[];
    const int r = blockIdx.x;
    const int N = tab.N[r], m = tab.m;
    int D = 1;
    for (int j = 0; j < m; ++j) D *= N;
    const int Dp = D + (D & 1);
    double *A = sm;                 // [Dp][Dp]
    double *V = A + Dp * Dp;        // [Dp][Dp]
    double *cs = V + Dp * Dp;       // [Dp/2][2] rotation of each pair
    int *pq = reinterpret_cast<int *>(cs + Dp);   // [Dp/2][2]
    __shared__ double red[256 / 32];
    __shared__ double off_norm, all_norm;
    const int64_t po = tab.par_off[r];
    const double *e = eps + po, *jb = J + po;
    const double U = tab.U;

    // H: diagonal sum_j eps(x_j) + U #pairs; one hop -J_b between basis
    // states that differ in one coordinate by the bond b = (b, b+1 mod N)
    for (int idx = threadIdx.x; idx < Dp * Dp; idx += blockDim.x) {
        const int a = idx / Dp, b = idx % Dp;
        double v = 0.0;
        if (a < D && b < D) {
            int xa[3] = {0, 0, 0}, xb[3] = {0, 0, 0};
            int ta = a, tb = b;
            for (int j = m - 1; j >= 0; --j) {
                xa[j] = ta % N;
                ta /= N;
                xb[j] = tb % N;
                tb /= N;
            }
            int ndiff = 0, jd = -1;
            for (int j = 0; j < m; ++j)
                if (xa[j] != xb[j]) {
                    ++ndiff;
                    jd = j;
                }
            if (ndiff == 0) {
                int pairs = 0;
                for (int j = 0; j < m; ++j) {
                    v += e[xa[j]];
                    for (int l = j + 1; l < m; ++l) pairs += xa[j] == xa[l];
                }
                v += U * pairs;
            } else if (ndiff == 1) {
                const int u = xa[jd], w = xb[jd];
                // entries add: a two-site ring has both bonds between the same sites
                if ((u + 1) % N == w) v -= jb[u];
                if ((w + 1) % N == u) v -= jb[w];
            }
        }
        A[idx] = v;
        V[idx] = (a == b) ? 1.0 : 0.0;
    }
    __syncthreads();

    const int half = Dp / 2;
    int sweep = 0;
    for (; sweep < kMaxSweeps; ++sweep) {
        // convergence: off-diagonal Frobenius norm against the whole
        double so = 0.0, sa = 0.0;
        for (int idx = threadIdx.x; idx < Dp * Dp; idx += blockDim.x) {
            const double x = A[idx] * A[idx];
            sa += x;
            if (idx / Dp != idx % Dp) so += x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            so += __shfl_xor_sync(0xffffffffu, so, o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = so;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            off_norm = t;
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sa;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            all_norm = t;
        }
        __syncthreads();
        if (off_norm <= 1e-26 * all_norm || all_norm == 0.0) break;

        for (int round = 0; round < Dp - 1; ++round) {
            // pairs of this round: index Dp-1 meets `round`, the others
            // (round + k, round - k) modulo Dp-1
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int p, q;
                if (k == 0) {
                    p = Dp - 1;
                    q = round;
                } else {
                    p = (round + k) % (Dp - 1);
                    q = (round - k + (Dp - 1)) % (Dp - 1);
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                pq[2 * k] = p;
                pq[2 * k + 1] = q;
                const double apq = A[p * Dp + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double tau = (A[q * Dp + q] - A[p * Dp + p]) / (2.0 * apq);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = s;
            }
            __syncthreads();
            // rows p, q of A: A <- J^T A
            for (int idx = threadIdx.x; idx < half * Dp; idx += blockDim.x) {
                const int k = idx / Dp, col = idx % Dp;
                const int p = pq[2 * k], q = pq[2 * k + 1];
                const double c = cs[2 * k], s = cs[2 * k + 1];
                const double ap = A[p * Dp + col], aq = A[q * Dp + col];
                A[p * Dp + col] = c * ap - s * aq;
                A[q * Dp + col] = s * ap + c * aq;
            }
            __syncthreads();
            // columns p, q of A and of V: A <- A J, V <- V J
            for (int idx = threadIdx.x; idx < half * Dp; idx += blockDim.x) {
                const int k = idx / Dp, row = idx % Dp;
                const int p = pq[2 * k], q = pq[2 * k + 1];
                const double c = cs[2 * k], s = cs[2 * k + 1];
                const double ap = A[row * Dp + p], aq = A[row * Dp + q];
                A[row * Dp + p] = c * ap - s * aq;
                A[row * Dp + q] = s * ap + c * aq;
                const double vp = V[row * Dp + p], vq = V[row * Dp + q];
                V[row * Dp + p] = c * vp - s * vq;
                V[row * Dp + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    // eigenvalues and eigenvectors (columns of V) of the D real states
    double *E = evals + (int64_t)r * Dp_max;
    double *W = evecs + (int64_t)r * Dp_max * Dp_max;
    for (int i = threadIdx.x; i < D; i += blockDim.x) E[i] = A[i * Dp + i];
    for (int idx = threadIdx.x; idx < D * D; idx += blockDim.x) {
        const int row = idx / D, col = idx % D;
        W[idx] = V[row * Dp + col];
    }
    if (threadIdx.x == 0) sweeps_out[r] = sweep;
}

// psi(t) = W exp(-i E t) W^T psi(0) for one realization per block.
__global__ void __launch_bounds__(128) exact_propagate_kernel(RealTable tab, const double *evals,
                                                              const double *evecs, int Dp_max,
                                                              const double2 *__restrict__ psi0,
                                                              double2 *psi, double t) {
    __shared__ double2 cpart[kMaxD];
    const int r = blockIdx.x;
    const int N = tab.N[r];
    int D = 1;
    for (int j = 0; j < tab.m; ++j) D *= N;
    const double *E = evals + (int64_t)r * Dp_max;
    const double *W = evecs + (int64_t)r * Dp_max * Dp_max;
    const double2 *p0 = psi0 + tab.st_off[r];
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        double cr = 0.0, ci = 0.0;
        for (int a = 0; a < D; ++a) {
            cr += W[a * D + k] * p0[a].x;
            ci += W[a * D + k] * p0[a].y;
        }
        double sn, cn;
        sincos(E[k] * t, &sn, &cn);
        // exp(-i E t) (cr + i ci)
        cpart[k] = make_double2(cn * cr + sn * ci, cn * ci - sn * cr);
    }
    __syncthreads();
    double2 *out = psi + tab.st_off[r];
    for (int a = threadIdx.x; a < D; a += blockDim.x) {
        double xr = 0.0, xi = 0.0;
        for (int k = 0; k < D; ++k) {
            xr += W[a * D + k] * cpart[k].x;
            xi += W[a * D + k] * cpart[k].y;
        }
        out[a] = make_double2(xr, xi);
    }
}

}  // namespace

int exact_max_dim() { return kMaxD; }

int launch_exact_eigen(const ctqw_hamiltonian *h, double *evals, double *evecs, int *sweeps,
                       cudaStream_t s) {
    int Dmax = 1;
    for (int j = 0; j < h->m; ++j) Dmax *= h->Nmax;
    const int Dp = Dmax + (Dmax & 1);
    const size_t smem = sizeof(double) * (2 * (size_t)Dp * Dp + Dp) + sizeof(int) * Dp;
    CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)exact_eigen_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    exact_eigen_kernel<<<h->R, 256, smem, s>>>(real_table(h), h->eps64, h->J64, evals, evecs, Dp, sweeps);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_exact_propagate(const ctqw_hamiltonian *h, const double *evals, const double *evecs,
                           const void *psi0, void *psi, double t, cudaStream_t s) {
    int Dmax = 1;
    for (int j = 0; j < h->m; ++j) Dmax *= h->Nmax;
    const int Dp = Dmax + (Dmax & 1);
    exact_propagate_kernel<<<h->R, 128, 0, s>>>(real_table(h), evals, evecs, Dp, (const double2 *)psi0,
                                                (double2 *)psi, t);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}
