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

// Philox4x64-10 (Salmon et al., SC'11): ten rounds of two 64 x 64 -> 128-bit
// products with the key bumped by the Weyl constants; four output words.
struct Philox4 {
    unsigned long long w[4];
};

__device__ __forceinline__ Philox4 philox4x64(unsigned long long c0, unsigned long long c1,
                                              unsigned long long c2, unsigned long long c3,
                                              unsigned long long k0, unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    return Philox4{{c0, c1, c2, c3}};
}

__device__ __forceinline__ double unit_double(unsigned long long w) {
    return (double)(w >> 11) * 0x1.0p-53;
}

// The Hamiltonian update after step `step` (switching noise, Sec. 2): per
// site, Philox block (step, r, i, 0) under key (seed, 0); words 0, 1 decide
// and redraw eps_i, words 2, 3 the hopping of bond i (not the absent wrap
// bond of an open chain).
__global__ void switch_params_kernel(RealTable tab, unsigned long long seed, unsigned long long step,
                                     double p, const double *__restrict__ eps_mean,
                                     const double *__restrict__ J_mean, double eps_hw, double J_hw,
                                     double J0, int round_f32, float *eps32, float *J32,
                                     double *eps64, double *J64) {
    const int r = blockIdx.y;
    const int N = tab.N[r];
    const int64_t off = tab.par_off[r];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const Philox4 b = philox4x64(step, (unsigned long long)r, (unsigned long long)i, 0ull, seed, 0ull);
        if (unit_double(b.w[0]) < p) {
            const double em = eps_mean ? eps_mean[i] : 0.0;
            double e = __dadd_rn(em, __dmul_rn(eps_hw, __dadd_rn(__dmul_rn(2.0, unit_double(b.w[1])), -1.0)));
            if (round_f32) e = (double)__double2float_rn(e);
            eps64[off + i] = e;
            eps32[off + i] = (float)e;
        }
        const bool bond = tab.periodic || i < N - 1;
        if (bond && unit_double(b.w[2]) < p) {
            const double jm = J_mean ? J_mean[i] : J0;
            double j = __dadd_rn(jm, __dmul_rn(J_hw, __dadd_rn(__dmul_rn(2.0, unit_double(b.w[3])), -1.0)));
            if (round_f32) j = (double)__double2float_rn(j);
            J64[off + i] = j;
            J32[off + i] = (float)j;
        }
    }
}

__global__ void restore_params_kernel(int64_t n, const double *__restrict__ eps0, const double *__restrict__ J0,
                                      float *eps32, float *J32, double *eps64, double *J64) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        eps64[i] = eps0[i];
        J64[i] = J0[i];
        eps32[i] = (float)eps0[i];
        J32[i] = (float)J0[i];
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

int launch_switch_params(const ctqw_hamiltonian *h, uint64_t seed, uint64_t step, double p,
                         cudaStream_t s) {
    dim3 block(128), grid((unsigned)((h->Nmax + 127) / 128), (unsigned)h->R);
    switch_params_kernel<<<grid, block, 0, s>>>(real_table(h), (unsigned long long)seed,
                                                (unsigned long long)step, p, h->eps_mean_d, h->J_mean_d,
                                                h->eps_hw, h->J_hw, h->J0, h->round_to_f32, h->eps32,
                                                h->J32, h->eps64, h->J64);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int restore_params(const ctqw_hamiltonian *h, cudaStream_t s) {
    const int64_t n = h->total_par;
    restore_params_kernel<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(
        n, h->eps64_0, h->J64_0, h->eps32, h->J32, h->eps64, h->J64);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}
