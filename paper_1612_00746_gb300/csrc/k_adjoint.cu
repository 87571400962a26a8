// Adjoint (reverse-mode) gradient of an ensemble loss through the Taylor
// propagation of Sec. 2.3.
//
// The forward map is n_steps applications of T = sum_{k<=K} c_k H^k with
// c_k = (-i dt)^k / k! per realization (Algorithm 3).  For the loss
// L = sum_x (Pbar(x,T) - P*(x))^2 the adjoint state starts at
// lambda_T = g * psi_T with g(s) = dL/d|psi(s)|^2, steps back with
// lambda_n = T^dagger lambda_{n+1}, and every step contributes
//   dL/dtheta += 2 Re sum_{a<K} <mu_a, dH/dtheta phi_a>,
//   phi_a = H^a psi_n,  mu_{K-1} = conj(c_K) lambda_{n+1},
//   mu_a = conj(c_{a+1}) lambda_{n+1} + H mu_{a+1},
// which is dT/dtheta = sum_k c_k sum_{a<k} H^{k-1-a} dH H^a written term by term.
// dH/deps_i counts the particles on site i; dH/dJ_b is minus the hop across
// bond b for every particle.
#include "ctqw_internal.cuh"
#include "stencil.cuh"

namespace {

// out = H in + coef * lam   (coef complex); first: out = coef * lam.
template <typename T, int M>
__global__ void __launch_bounds__(256) mu_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                 const T *__restrict__ eps,
                                                 const T *__restrict__ J,
                                                 const cplx_t<T> *__restrict__ in,
                                                 const cplx_t<T> *__restrict__ lam,
                                                 cplx_t<T> *__restrict__ out, double cre, double cim,
                                                 int first) {
    Site<M> q;
    if (!site_of<M>(tab, list, q)) return;
    const int64_t s = q.s;
    const int64_t base = tab.st_off[q.r];
    const cplx_t<T> l = lam[base + s];
    // conj(c_k) = (i dt)^k / k! is real or imaginary: the product costs two
    // multiplies in the state's own type
    const T a = (T)cre, b = (T)cim;
    T ox = a * l.x - b * l.y;
    T oy = a * l.y + b * l.x;
    if (!first) {
        const int64_t po = tab.par_off[q.r];
        const cplx_t<T> y = apply_h<T, M>(in + base, s, q.x, q.N, eps + po, J + po, (T)tab.U);
        ox += y.x;
        oy += y.y;
    }
    out[base + s] = mk<T>(ox, oy);
}

// out = H in (a plain stencil application).
template <typename T, int M>
__global__ void __launch_bounds__(256) apply_h_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                      const T *__restrict__ eps,
                                                      const T *__restrict__ J,
                                                      const cplx_t<T> *__restrict__ in,
                                                      cplx_t<T> *__restrict__ out) {
    Site<M> q;
    if (!site_of<M>(tab, list, q)) return;
    const int64_t base = tab.st_off[q.r];
    const int64_t po = tab.par_off[q.r];
    out[base + q.s] = apply_h<T, M>(in + base, q.s, q.x, q.N, eps + po, J + po, (T)tab.U);
}

// grad_eps[r][i] += 2 Re <mu, n_i phi>,  grad_J[r][b] += 2 Re <mu, dH/dJ_b phi>.
// Per-block accumulation in shared memory (FP64) when N <= kSmemN, then one
// FP64 atomic per touched entry; otherwise FP64 atomics straight to global.
// For a particle whose site is the same on every lane of a warp (the slow
// indices x_1..x_{M-1} when N is a multiple of 32) the warp sums first, so
// that a block does not serialize on one address.
constexpr int kSmemN = 1024;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int M>
__global__ void __launch_bounds__(256) grad_kernel(RealTable tab, const cplx_t<T> *__restrict__ mu,
                                                   const cplx_t<T> *__restrict__ phi,
                                                   double *grad_eps, double *grad_J) {
    __shared__ double ge[kSmemN], gj[kSmemN];
    const int r = blockIdx.y;
    const int N = tab.N[r];
    const bool use_smem = N <= kSmemN;
    if (use_smem) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) ge[i] = gj[i] = 0.0;
        __syncthreads();
    }
    int64_t D = N;
#pragma unroll
    for (int j = 1; j < M; ++j) D *= N;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t base = tab.st_off[r];
    const int64_t po = tab.par_off[r];
    const bool live = s < D;
    int x[M];
    double d = 0.0;
    cplx_t<T> u, p;
    if (live) {
        unflatten<M>(s, N, x);
        u = mu[base + s];
        p = phi[base + s];
        // Re(conj(u) p)
        d = (double)u.x * (double)p.x + (double)u.y * (double)p.y;
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) x[j] = -1;
    }
    int64_t stride = 1;
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {
        const int b = x[j];
        const bool bond = live && (tab.periodic || b < N - 1);
        double h = 0.0;
        if (bond) {
            const int64_t s2 = s + (int64_t)((b == N - 1) ? (1 - N) : 1) * stride;   // particle j on b+1
            const cplx_t<T> u2 = mu[base + s2], p2 = phi[base + s2];
            h = (double)u.x * (double)p2.x + (double)u.y * (double)p2.y + (double)u2.x * (double)p.x +
                (double)u2.y * (double)p.y;
        }
        const int b0 = __shfl_sync(0xffffffffu, b, 0);
        if (__all_sync(0xffffffffu, b == b0)) {
            // the whole warp on one site (b0 >= 0: every lane is live)
            const double de = warp_sum_d(2.0 * d), dh = warp_sum_d(-2.0 * h);
            if ((threadIdx.x & 31) == 0 && b0 >= 0) {
                if (use_smem) atomicAdd(ge + b0, de);
                else atomicAdd(grad_eps + po + b0, de);
                if (tab.periodic || b0 < N - 1) {
                    if (use_smem) atomicAdd(gj + b0, dh);
                    else atomicAdd(grad_J + po + b0, dh);
                }
            }
        } else if (live) {
            if (use_smem) atomicAdd(ge + b, 2.0 * d);
            else atomicAdd(grad_eps + po + b, 2.0 * d);
            if (bond) {
                if (use_smem) atomicAdd(gj + b, -2.0 * h);
                else atomicAdd(grad_J + po + b, -2.0 * h);
            }
        }
        stride *= N;
    }
    if (use_smem) {
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            if (ge[i] != 0.0) atomicAdd(grad_eps + po + i, ge[i]);
            if (gj[i] != 0.0) atomicAdd(grad_J + po + i, gj[i]);
        }
    }
}

// loss = sum_x (Pbar - P*)^2 over all groups; diff = Pbar - P*.  One block.
__global__ void loss_kernel(const double *__restrict__ Pbar, const double *__restrict__ target,
                            int64_t n, double *diff, double *loss) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = Pbar[i] - target[i];
        diff[i] = d;
        acc += d * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0];
}

// lambda_T(s) = g(s) psi_T(s),  g(s) = sum_j 2 diff(x_j) / (m R_g).
template <typename T, int M>
__global__ void __launch_bounds__(256) lambda_init_kernel(RealTable tab, const cplx_t<T> *__restrict__ psi,
                                                          const double *__restrict__ diff,
                                                          cplx_t<T> *__restrict__ lam) {
    const int r = blockIdx.y;
    const int N = tab.N[r];
    int64_t D = N;
#pragma unroll
    for (int j = 1; j < M; ++j) D *= N;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= D) return;
    const int g = tab.group_of[r];
    const double *dg = diff + tab.group_off[g];
    int x[M];
    unflatten<M>(s, N, x);
    double w = 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) w += dg[x[j]];
    w *= 2.0 * tab.inv_count[g] / M;
    const int64_t base = tab.st_off[r];
    const cplx_t<T> p = psi[base + s];
    lam[base + s] = mk<T>((T)(w * (double)p.x), (T)(w * (double)p.y));
}

// out[i] = sum over the group's realizations (in the fixed order of `list`)
// of grad[par_off[r] + i], i < N: the gradient with respect to parameters
// shared by the group (the means), deterministic.
__global__ void __launch_bounds__(256) group_sum_kernel(const int64_t *__restrict__ par_off,
                                                        const int32_t *__restrict__ list, int cnt, int N,
                                                        const double *__restrict__ grad,
                                                        double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = 0.0;
    for (int q = 0; q < cnt; ++q) acc += grad[par_off[list[q]] + i];
    out[i] = acc;
}

dim3 grid_for(const ctqw_hamiltonian *h) {
    int64_t D = 1;
    for (int j = 0; j < h->m; ++j) D *= h->Nmax;
    return dim3((unsigned)((D + 255) / 256), (unsigned)h->R);
}

}  // namespace

int launch_apply_h(const ctqw_hamiltonian *h, int dtype, const void *in, void *out, cudaStream_t s) {
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        if (dtype == CTQW_C64) {
            auto k = h->m == 2 ? apply_h_kernel<float, 2> : apply_h_kernel<float, 3>;
            k<<<grid, block, 0, s>>>(t, list, h->eps32, h->J32, (const float2 *)in, (float2 *)out);
        } else {
            auto k = h->m == 2 ? apply_h_kernel<double, 2> : apply_h_kernel<double, 3>;
            k<<<grid, block, 0, s>>>(t, list, h->eps64, h->J64, (const double2 *)in, (double2 *)out);
        }
    });
}

int launch_mu(const ctqw_hamiltonian *h, int dtype, const void *in, const void *lam, void *out,
              double cre, double cim, int first, cudaStream_t s) {
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        if (dtype == CTQW_C64) {
            auto k = h->m == 2 ? mu_kernel<float, 2> : mu_kernel<float, 3>;
            k<<<grid, block, 0, s>>>(t, list, h->eps32, h->J32, (const float2 *)in, (const float2 *)lam,
                                     (float2 *)out, cre, cim, first);
        } else {
            auto k = h->m == 2 ? mu_kernel<double, 2> : mu_kernel<double, 3>;
            k<<<grid, block, 0, s>>>(t, list, h->eps64, h->J64, (const double2 *)in, (const double2 *)lam,
                                     (double2 *)out, cre, cim, first);
        }
    });
}

int launch_grad(const ctqw_hamiltonian *h, int dtype, const void *mu, const void *phi,
                double *grad_eps, double *grad_J, cudaStream_t s) {
    dim3 g = grid_for(h), b(256);
    RealTable t = real_table(h);
    if (dtype == CTQW_C64) {
        auto k = h->m == 2 ? grad_kernel<float, 2> : grad_kernel<float, 3>;
        k<<<g, b, 0, s>>>(t, (const float2 *)mu, (const float2 *)phi, grad_eps, grad_J);
    } else {
        auto k = h->m == 2 ? grad_kernel<double, 2> : grad_kernel<double, 3>;
        k<<<g, b, 0, s>>>(t, (const double2 *)mu, (const double2 *)phi, grad_eps, grad_J);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_loss(const double *Pbar, const double *target, int64_t n, double *diff, double *loss,
                cudaStream_t s) {
    loss_kernel<<<1, 256, 0, s>>>(Pbar, target, n, diff, loss);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_lambda_init(const ctqw_hamiltonian *h, int dtype, const void *psi, const double *diff,
                       void *lam, cudaStream_t s) {
    dim3 g = grid_for(h), b(256);
    RealTable t = real_table(h);
    if (dtype == CTQW_C64) {
        auto k = h->m == 2 ? lambda_init_kernel<float, 2> : lambda_init_kernel<float, 3>;
        k<<<g, b, 0, s>>>(t, (const float2 *)psi, diff, (float2 *)lam);
    } else {
        auto k = h->m == 2 ? lambda_init_kernel<double, 2> : lambda_init_kernel<double, 3>;
        k<<<g, b, 0, s>>>(t, (const double2 *)psi, diff, (double2 *)lam);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_group_sum(const ctqw_hamiltonian *h, const double *grad, double *out, cudaStream_t s) {
    int off = 0;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g], cnt = h->group_count[g];
        group_sum_kernel<<<(N + 255) / 256, 256, 0, s>>>(h->par_off_d, h->by_group_d + off, cnt, N, grad,
                                                         out + h->group_off[g]);
        CTQW_CUDA_TRY(cudaGetLastError());
        off += cnt;
    }
    return CTQW_OK;
}
