// Observables of one sample (Sec. 2: <rho> = (1/R) sum_i |Psi_i><Psi_i|, of
// which only the diagonal is needed): per-realization norm and energy,
// per-size-group ensemble averages of P(x), and for m = 2 the pair
// distribution |psi(x1, x2)|^2.  All accumulation is FP64.
#include "ctqw_internal.cuh"
#include "stencil.cuh"

namespace {

constexpr int kRows = 4;      // rows (fixed x_1..x_{M-1}) per block
constexpr int kThreads = 256;

template <typename T, int M>
__global__ void __launch_bounds__(kThreads) observables_kernel(
    RealTable tab, const T *__restrict__ eps, const T *__restrict__ J,
    const cplx_t<T> *__restrict__ psi, double *P_mean, double *P_joint, double *norm,
    double *energy) {
    const int r = blockIdx.y;
    const int N = tab.N[r];
    int64_t n_rows = N;
#pragma unroll
    for (int j = 2; j < M; ++j) n_rows *= N;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    if (row0 >= n_rows) return;
    const int64_t base = tab.st_off[r];
    const int64_t po = tab.par_off[r];
    const int g = tab.group_of[r];
    const double inv_R = tab.inv_count[g];
    const double scale = inv_R / M;
    double *Pg = P_mean ? P_mean + tab.group_off[g] : nullptr;
    double *Jg = P_joint ? P_joint + tab.joint_off[g] : nullptr;
    const cplx_t<T> *a = psi + base;

    double rowpart[kRows];
#pragma unroll
    for (int q = 0; q < kRows; ++q) rowpart[q] = 0.0;
    double nrm = 0.0, en = 0.0;
    for (int col = threadIdx.x; col < N; col += blockDim.x) {
        double colacc = 0.0;
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
            const int64_t row = row0 + q;
            if (row < n_rows) {
                const int64_t s = row * N + col;
                cplx_t<T> v = a[s];
                double p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
                colacc += p;
                rowpart[q] += p;
                nrm += p;
                if (energy) {
                    int x[M];
                    unflatten<M>(s, N, x);
                    cplx_t<T> y = apply_h<T, M>(a, s, x, N, eps + po, J + po, (T)tab.U);
                    en += (double)v.x * (double)y.x + (double)v.y * (double)y.y;
                }
                if (Jg) atomicAdd(Jg + s, p * inv_R);
            }
        }
        if (Pg) atomicAdd(Pg + col, colacc * scale);
    }
    // block reductions: rows, norm, energy
    __shared__ double red[kThreads / 32][kRows + 2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kRows + 2; ++q) {
        double v = q < kRows ? rowpart[q] : (q == kRows ? nrm : en);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRows + 2) {
        const int q = threadIdx.x;
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) v += red[w][q];
        if (q < kRows) {
            const int64_t row = row0 + q;
            if (Pg && row < n_rows) {
                // coordinates x_1..x_{M-1} of this row
                int64_t t = row;
                for (int j = M - 2; j >= 0; --j) {
                    int64_t qq = t / N;
                    int xj = (int)(t - qq * N);
                    t = qq;
                    atomicAdd(Pg + xj, v * scale);
                }
            }
        } else if (q == kRows) {
            if (norm) atomicAdd(norm + r, v);
        } else {
            if (energy) atomicAdd(energy + r, v);
        }
    }
}

// psi (and lo) of realization r times 1 / sqrt(norm[r]).
template <typename T, int M>
__global__ void __launch_bounds__(256) renorm_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                     cplx_t<T> *psi, cplx_t<T> *lo,
                                                     const double *__restrict__ norm) {
    Site<M> p;
    if (!site_of<M>(tab, list, p)) return;
    const double n = norm[p.r];
    const T sc = n > 0.0 ? (T)(1.0 / sqrt(n)) : T(1);
    const int64_t i = tab.st_off[p.r] + p.s;
    cplx_t<T> v = psi[i];
    psi[i] = mk<T>(v.x * sc, v.y * sc);
    if (lo) {
        v = lo[i];
        lo[i] = mk<T>(v.x * sc, v.y * sc);
    }
}

}  // namespace

int launch_renormalize(const ctqw_hamiltonian *h, int dtype, void *psi, void *lo, cudaStream_t s) {
    CTQW_CUDA_TRY(cudaMemsetAsync(h->renorm_d, 0, sizeof(double) * h->R, s));
    CTQW_TRY(launch_observables(h, dtype, psi, nullptr, nullptr, h->renorm_d, nullptr, s));
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        if (dtype == CTQW_C64) {
            auto k = h->m == 2 ? renorm_kernel<float, 2> : renorm_kernel<float, 3>;
            k<<<grid, block, 0, s>>>(t, list, (float2 *)psi, (float2 *)lo, h->renorm_d);
        } else {
            auto k = h->m == 2 ? renorm_kernel<double, 2> : renorm_kernel<double, 3>;
            k<<<grid, block, 0, s>>>(t, list, (double2 *)psi, (double2 *)lo, h->renorm_d);
        }
    });
}

int launch_observables(const ctqw_hamiltonian *h, int dtype, const void *psi, double *P_mean,
                       double *P_joint, double *norm, double *energy, cudaStream_t s) {
    if (!P_mean && !P_joint && !norm && !energy) return CTQW_OK;
    int64_t rows = 1;
    for (int j = 1; j < h->m; ++j) rows *= h->Nmax;
    dim3 grid((unsigned)((rows + kRows - 1) / kRows), (unsigned)h->R), block(kThreads);
    RealTable t = real_table(h);
    if (dtype == CTQW_C64) {
        auto k = h->m == 2 ? observables_kernel<float, 2> : observables_kernel<float, 3>;
        k<<<grid, block, 0, s>>>(t, h->eps32, h->J32, (const float2 *)psi, P_mean, P_joint, norm,
                                 energy);
    } else {
        auto k = h->m == 2 ? observables_kernel<double, 2> : observables_kernel<double, 3>;
        k<<<grid, block, 0, s>>>(t, h->eps64, h->J64, (const double2 *)psi, P_mean, P_joint, norm,
                                 energy);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}
