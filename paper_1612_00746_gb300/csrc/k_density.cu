// One-body reduced density matrix averaged over the realizations of each
// size group (the partial trace of Sec. 2's <rho> = (1/R) sum_i |Psi_i><Psi_i|
// over all particles but one, averaged over which particle is kept):
//
//   rho1(x, x') = (1/R_g) (1/m) sum_r sum_j sum_k psi_r(x_j = x, k) conj(psi_r(x_j = x', k)),
//
// k running over the other m-1 coordinates.  For particle j the amplitude
// psi(x_j = x, k) sits at (k / K_lo) S_hi + x S_x + (k % K_lo) in the
// row-major N^m tile (x_m fastest): S_x = N^(m-1-j), K_lo = S_x,
// S_hi = N^(m-j).  One launch per particle and size group; a block owns a
// 32 x 64 tile of (x, x') and a chunk of realizations, walks k in chunks of
// 32 (16 in FP64) through shared memory, forms the products in the state's type (FP32
// for c64) per chunk and accumulates the chunks in FP64 registers, then
// adds its tile to the FP64 output with one atomic per element.
#include "ctqw_internal.cuh"
#include "stencil.cuh"

namespace {

constexpr int kTX = 64;   // x' per block
constexpr int kTY = 32;   // x per block
constexpr int kRCH = 8;   // realizations per block

// k per chunk (FP64 states: half, to stay within 48 KB of static shared memory)
template <typename T> struct Chunk { static constexpr int value = 32; };
template <> struct Chunk<double> { static constexpr int value = 16; };

template <typename T>
__global__ void __launch_bounds__(256) rho1_term_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                        int n_real, const cplx_t<T> *__restrict__ psi,
                                                        double *__restrict__ rho, int64_t rho_off, int N,
                                                        int64_t n_k, int64_t S_x, int64_t K_lo,
                                                        int64_t S_hi, double scale) {
    using C = cplx_t<T>;
    constexpr int kKC = Chunk<T>::value;
    __shared__ C A[kTY][kKC + 1];     // psi(x, k) for the block's x rows
    __shared__ C B[kKC][kTX + 1];     // psi(x', k), k-major
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    const int x0 = blockIdx.y * kTY, xp0 = blockIdx.x * kTX;
    const bool x_contig = S_x == 1;
    double accr[4][2], acci[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c) accr[q][c] = acci[q][c] = 0.0;

    const int rbeg = blockIdx.z * kRCH, rend = min(n_real, rbeg + kRCH);
    for (int rr = rbeg; rr < rend; ++rr) {
        const C *p = psi + tab.st_off[list[rr]];
        auto at = [&](int x, int64_t k) -> C {
            return p[(k / K_lo) * S_hi + (int64_t)x * S_x + (k % K_lo)];
        };
        for (int64_t k0 = 0; k0 < n_k; k0 += kKC) {
            // tiles of psi: consecutive threads along the contiguous index
            for (int e = threadIdx.x; e < kTY * kKC; e += blockDim.x) {
                const int i = x_contig ? e % kTY : e / kKC, kk = x_contig ? e / kTY : e % kKC;
                const int x = x0 + i;
                const int64_t k = k0 + kk;
                A[i][kk] = (x < N && k < n_k) ? at(x, k) : C{};
            }
            for (int e = threadIdx.x; e < kTX * kKC; e += blockDim.x) {
                const int i = x_contig ? e % kTX : e / kKC, kk = x_contig ? e / kTX : e % kKC;
                const int x = xp0 + i;
                const int64_t k = k0 + kk;
                B[kk][i] = (x < N && k < n_k) ? at(x, k) : C{};
            }
            __syncthreads();
            T sr[4][2], si[4][2];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 2; ++c) sr[q][c] = si[q][c] = T(0);
#pragma unroll 8
            for (int kk = 0; kk < kKC; ++kk) {
                const C b0 = B[kk][tx], b1 = B[kk][tx + 32];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const C a = A[ty + 8 * q][kk];
                    // a conj(b)
                    sr[q][0] += a.x * b0.x + a.y * b0.y;
                    si[q][0] += a.y * b0.x - a.x * b0.y;
                    sr[q][1] += a.x * b1.x + a.y * b1.y;
                    si[q][1] += a.y * b1.x - a.x * b1.y;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    accr[q][c] += (double)sr[q][c];
                    acci[q][c] += (double)si[q][c];
                }
            __syncthreads();
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = x0 + ty + 8 * q;
        if (x >= N) continue;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int xp = xp0 + tx + 32 * c;
            if (xp >= N) continue;
            double *o = rho + 2 * (rho_off + (int64_t)x * N + xp);
            atomicAdd(o, scale * accr[q][c]);
            atomicAdd(o + 1, scale * acci[q][c]);
        }
    }
}

}  // namespace

int launch_one_body_density(const ctqw_hamiltonian *h, int dtype, const void *psi, double *rho,
                            cudaStream_t s) {
    RealTable t = real_table(h);
    const int m = h->m;
    int off = 0;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g], cnt = h->group_count[g];
        int64_t n_k = 1;
        for (int j = 1; j < m; ++j) n_k *= N;
        const double scale = 1.0 / ((double)cnt * (double)m);
        const dim3 grid((unsigned)((N + kTX - 1) / kTX), (unsigned)((N + kTY - 1) / kTY),
                        (unsigned)((cnt + kRCH - 1) / kRCH));
        for (int j = 0; j < m; ++j) {
            int64_t S_x = 1;
            for (int l = j + 1; l < m; ++l) S_x *= N;
            const int64_t K_lo = S_x, S_hi = S_x * N;
            if (dtype == CTQW_C64)
                rho1_term_kernel<float><<<grid, 256, 0, s>>>(t, h->by_group_d + off, cnt, (const float2 *)psi,
                                                             rho, h->joint_off[g], N, n_k, S_x, K_lo, S_hi,
                                                             scale);
            else
                rho1_term_kernel<double><<<grid, 256, 0, s>>>(t, h->by_group_d + off, cnt,
                                                              (const double2 *)psi, rho, h->joint_off[g], N,
                                                              n_k, S_x, K_lo, S_hi, scale);
            CTQW_CUDA_TRY(cudaGetLastError());
        }
        off += cnt;
    }
    return CTQW_OK;
}
