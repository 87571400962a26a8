// Parameter build (Eq. (Hij): c + xi per entry) and initial states.
#include "ctqw_internal.cuh"
#include "stencil.cuh"

namespace {

// eps_{r,i} = mean_i + w (2u - 1) (optionally rounded to float32); bond N-1
// of an open chain is absent and stored as 0.  __dadd_rn / __dmul_rn keep
// the two roundings of the definition (no contraction into an FMA).
__global__ void build_params_kernel(RealTable tab, const double *__restrict__ u_eps,
                                    const double *__restrict__ u_J,
                                    const double *__restrict__ eps_mean,
                                    const double *__restrict__ J_mean, double eps_hw,
                                    double J_hw, double J0, int round_f32, float *eps32,
                                    float *J32, double *eps64, double *J64) {
    const int r = blockIdx.y;
    const int N = tab.N[r];
    const int64_t off = tab.par_off[r];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double em = eps_mean ? eps_mean[i] : 0.0;
        double jm = J_mean ? J_mean[i] : J0;
        double e = __dadd_rn(em, __dmul_rn(eps_hw, __dadd_rn(__dmul_rn(2.0, u_eps[off + i]), -1.0)));
        double j = __dadd_rn(jm, __dmul_rn(J_hw, __dadd_rn(__dmul_rn(2.0, u_J[off + i]), -1.0)));
        if (!tab.periodic && i == N - 1) j = 0.0;
        if (round_f32) {
            e = (double)__double2float_rn(e);
            j = (double)__double2float_rn(j);
        }
        eps64[off + i] = e;
        J64[off + i] = j;
        eps32[off + i] = (float)e;
        J32[off + i] = (float)j;
    }
}

// One thread per realization: sum over the m! permutations of the sites
// (signed for fermions), then normalise; the state was zeroed beforehand.
template <typename T>
__global__ void init_state_kernel(RealTable tab, const int32_t *__restrict__ sites, int stats,
                                  cplx_t<T> *psi) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= tab.R) return;
    const int m = tab.m;
    const int N = tab.N[r];
    int64_t idx[6];
    double amp[6];
    int n = 0;
    const int perms2[2][2] = {{0, 1}, {1, 0}};
    const int sign2[2] = {1, -1};
    const int perms3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int sign3[6] = {1, -1, -1, 1, 1, -1};
    const int nperm = (stats == 0) ? 1 : (m == 2 ? 2 : 6);
    for (int p = 0; p < nperm; ++p) {
        int64_t f = 0;
        for (int j = 0; j < m; ++j) {
            int src = (m == 2) ? perms2[p][j] : perms3[p][j];
            f = f * N + sites[r * m + src];
        }
        double sg = (stats == 2) ? (double)((m == 2) ? sign2[p] : sign3[p]) : 1.0;
        int k = 0;
        while (k < n && idx[k] != f) ++k;
        if (k == n) {
            idx[n] = f;
            amp[n] = 0.0;
            ++n;
        }
        amp[k] += sg;
    }
    double nrm = 0.0;
    for (int k = 0; k < n; ++k) nrm += amp[k] * amp[k];
    nrm = sqrt(nrm);
    cplx_t<T> *base = psi + tab.st_off[r];
    for (int k = 0; k < n; ++k) base[idx[k]] = mk<T>((T)(amp[k] / nrm), T(0));
}

}  // namespace

int launch_build_params(const ctqw_hamiltonian *h, const double *u_eps_d, const double *u_J_d,
                        const double *eps_mean_d, const double *J_mean_d, double eps_hw,
                        double J_hw, double J0, cudaStream_t s) {
    dim3 block(256);
    dim3 grid((unsigned)((h->Nmax + 255) / 256), (unsigned)h->R);
    build_params_kernel<<<grid, block, 0, s>>>(real_table(h), u_eps_d, u_J_d, eps_mean_d, J_mean_d,
                                               eps_hw, J_hw, J0, h->round_to_f32, h->eps32,
                                               h->J32, h->eps64, h->J64);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_init_state(const ctqw_hamiltonian *h, const int32_t *sites_d, int dtype, void *psi,
                      cudaStream_t s) {
    size_t elem = dtype == CTQW_C64 ? sizeof(float2) : sizeof(double2);
    CTQW_CUDA_TRY(cudaMemsetAsync(psi, 0, (size_t)h->total_amp * elem, s));
    dim3 block(128), grid((unsigned)((h->R + 127) / 128));
    if (dtype == CTQW_C64)
        init_state_kernel<float><<<grid, block, 0, s>>>(real_table(h), sites_d, h->statistics,
                                                        (float2 *)psi);
    else
        init_state_kernel<double><<<grid, block, 0, s>>>(real_table(h), sites_d, h->statistics,
                                                         (double2 *)psi);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}
