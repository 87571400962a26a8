// Per-term propagation kernels: the structure of Algorithms 2 and 3 with
// one launch per Taylor term (or RK4 stage) over all realizations at once
// (the realization x node loop collapsed into one grid, Sec. 2.2).  These
// are the plain path: every term streams Phi and the running sum through HBM.
#include "ctqw_internal.cuh"
#include "stencil.cuh"

namespace {

// Phi^(j) = -(i dt/j) H Phi^(j-1);  acc = (first ? psi : acc) + Phi^(j).
template <typename T, int M>
__global__ void __launch_bounds__(256) taylor_term_kernel(RealTable tab, const T *__restrict__ eps,
                                                          const T *__restrict__ J,
                                                          const cplx_t<T> *__restrict__ in,
                                                          cplx_t<T> *__restrict__ out,
                                                          const cplx_t<T> *__restrict__ psi,
                                                          cplx_t<T> *__restrict__ acc, T coef,
                                                          int first) {
    const int r = blockIdx.y;
    const int N = tab.N[r];
    int64_t D = N;
#pragma unroll
    for (int j = 1; j < M; ++j) D *= N;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= D) return;
    const int64_t base = tab.st_off[r];
    const int64_t po = tab.par_off[r];
    int x[M];
    unflatten<M>(s, N, x);
    cplx_t<T> y = apply_h<T, M>(in + base, s, x, N, eps + po, J + po, (T)tab.U);
    cplx_t<T> phi = mk<T>(coef * y.y, -coef * y.x);   // -(i coef) y
    out[base + s] = phi;
    cplx_t<T> a = first ? psi[base + s] : acc[base + s];
    acc[base + s] = mk<T>(a.x + phi.x, a.y + phi.y);
}

// k = -i H in;  next = psi + a k (when next != null);  acc = (first ? psi : acc) + b k.
template <typename T, int M>
__global__ void __launch_bounds__(256) rk4_stage_kernel(RealTable tab, const T *__restrict__ eps,
                                                        const T *__restrict__ J,
                                                        const cplx_t<T> *__restrict__ in,
                                                        cplx_t<T> *__restrict__ next,
                                                        const cplx_t<T> *__restrict__ psi,
                                                        cplx_t<T> *__restrict__ acc, T a, T b,
                                                        int first) {
    const int r = blockIdx.y;
    const int N = tab.N[r];
    int64_t D = N;
#pragma unroll
    for (int j = 1; j < M; ++j) D *= N;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= D) return;
    const int64_t base = tab.st_off[r];
    const int64_t po = tab.par_off[r];
    int x[M];
    unflatten<M>(s, N, x);
    cplx_t<T> y = apply_h<T, M>(in + base, s, x, N, eps + po, J + po, (T)tab.U);
    cplx_t<T> k = mk<T>(y.y, -y.x);   // -i H in
    cplx_t<T> p = psi[base + s];
    if (next) next[base + s] = mk<T>(p.x + a * k.x, p.y + a * k.y);
    cplx_t<T> c = first ? p : acc[base + s];
    acc[base + s] = mk<T>(c.x + b * k.x, c.y + b * k.y);
}

dim3 grid_for(const ctqw_hamiltonian *h) {
    int64_t D = 1;
    for (int j = 0; j < h->m; ++j) D *= h->Nmax;
    return dim3((unsigned)((D + 255) / 256), (unsigned)h->R);
}

}  // namespace

int launch_taylor_term(const ctqw_hamiltonian *h, int dtype, const void *in, void *out,
                       const void *psi, void *acc, double coef, int first, cudaStream_t s) {
    dim3 grid = grid_for(h), block(256);
    RealTable t = real_table(h);
    if (dtype == CTQW_C64) {
        auto k = h->m == 2 ? taylor_term_kernel<float, 2> : taylor_term_kernel<float, 3>;
        k<<<grid, block, 0, s>>>(t, h->eps32, h->J32, (const float2 *)in, (float2 *)out,
                                 (const float2 *)psi, (float2 *)acc, (float)coef, first);
    } else {
        auto k = h->m == 2 ? taylor_term_kernel<double, 2> : taylor_term_kernel<double, 3>;
        k<<<grid, block, 0, s>>>(t, h->eps64, h->J64, (const double2 *)in, (double2 *)out,
                                 (const double2 *)psi, (double2 *)acc, coef, first);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_rk4_stage(const ctqw_hamiltonian *h, int dtype, const void *in, void *next,
                     const void *psi, void *acc, double a, double b, int first, cudaStream_t s) {
    dim3 grid = grid_for(h), block(256);
    RealTable t = real_table(h);
    if (dtype == CTQW_C64) {
        auto k = h->m == 2 ? rk4_stage_kernel<float, 2> : rk4_stage_kernel<float, 3>;
        k<<<grid, block, 0, s>>>(t, h->eps32, h->J32, (const float2 *)in, (float2 *)next,
                                 (const float2 *)psi, (float2 *)acc, (float)a, (float)b, first);
    } else {
        auto k = h->m == 2 ? rk4_stage_kernel<double, 2> : rk4_stage_kernel<double, 3>;
        k<<<grid, block, 0, s>>>(t, h->eps64, h->J64, (const double2 *)in, (double2 *)next,
                                 (const double2 *)psi, (double2 *)acc, a, b, first);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}
