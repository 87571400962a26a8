// Observables of one sample (Sec. 2: <rho> = (1/R) sum_i |Psi_i><Psi_i|, of
// which only the diagonal is needed): per-realization norm and energy
// (the norm check of Algorithms 2 and 3), per-size-group ensemble averages
// of P(x), and for m = 2 the pair distribution |psi(x1, x2)|^2.
//
// occupation_kernel (P, norm, energy): a block owns a range of rows (fixed
// x_1..x_{M-1}) of one realization and walks them in tiles of 32 columns
// (one per lane); column sums stay in registers over the block's rows, row
// sums of 8 rows at a time are reduced over the warp (one multi-value
// butterfly) into shared memory, so a block issues one atomic per column and
// per row coordinate, not one per amplitude.
// Products are formed in the state's precision.  CTQW_C128 sums in FP64.
// CTQW_C64 sums exactly: every FP32 product is turned into a 64-bit
// fixed-point integer (|psi|^2 times 2^48, energy terms times 2^44, rounded
// to nearest, one conversion instruction) and added as an integer, which
// neither rounds nor depends on the order; only block totals are converted
// to FP64.  (GB300's
// FP64 pipe runs at 1/64 of the FP32 rate; an FP64 add per product made the
// reduction slower than the propagation it samples.)  A product that is not
// finite or out of range marks the sample: norm and energy get a NaN.
// observables_kernel (everything above plus the pair distribution): one
// thread per amplitude, FP64 accumulation.
#include <algorithm>

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

// Fixed point of an FP32 value: f * 2^F rounded to the nearest 64-bit
// integer (the scaling by a power of two is exact; one conversion), exact
// when |f| >= 2^(23-F).  bad is set for Inf/NaN and for |f| >= 2^(62-F).
__device__ __forceinline__ long long fixed_of(float f, float two_F, float limit, unsigned &bad) {
    bad |= (!(fabsf(f) < limit)) ? 1u : 0u;   // also true for NaN
    return __float2ll_rn(f * two_F);
}

// Accumulator of the observables for states of element type T.
template <typename T> struct ObsSum;
template <> struct ObsSum<float> {
    using A = long long;   // exact fixed point: |psi|^2 in units of 2^-48, energy terms of 2^-44
    static __device__ __forceinline__ A p(float x, unsigned &bad) { return fixed_of(x, 0x1p48f, 0x1p14f, bad); }
    static __device__ __forceinline__ A e(float x, unsigned &bad) { return fixed_of(x, 0x1p44f, 0x1p18f, bad); }
    static __device__ __forceinline__ double dp(A a) { return (double)a * 0x1p-48; }
    static __device__ __forceinline__ double de(A a) { return (double)a * 0x1p-44; }
    // a total whose magnitude reaches 2^62 may have wrapped
    static __device__ __forceinline__ unsigned over(A a) { return (a >= (1ll << 62) || a <= -(1ll << 62)) ? 1u : 0u; }
};
template <> struct ObsSum<double> {
    using A = double;
    static __device__ __forceinline__ A p(double x, unsigned &) { return x; }
    static __device__ __forceinline__ A e(double x, unsigned &) { return x; }
    static __device__ __forceinline__ double dp(A a) { return a; }
    static __device__ __forceinline__ double de(A a) { return a; }
    static __device__ __forceinline__ unsigned over(A) { return 0u; }
};

template <typename A>
__device__ __forceinline__ A warp_total(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp totals of V values per lane at once (V a power of two <= 32): the
// first log2 V steps halve the values a lane keeps (it sends the half its
// partner keeps), the rest is a plain butterfly; lane l ends with the total
// of value (l >> (5 - log2 V)) & (V - 1).
template <int V, typename A>
__device__ __forceinline__ A warp_totals(A (&v)[V], int lane) {
#pragma unroll
    for (int o = 16, n = V; n > 1; o >>= 1, n >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < n / 2; ++q) {
            const A send = upper ? v[q] : v[q + n / 2];
            const A keep = upper ? v[q + n / 2] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    A t = v[0];
#pragma unroll
    for (int o = 16 / V; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

template <typename T>
__device__ __forceinline__ cplx_t<T> shfl_c(cplx_t<T> v, int src) {
    return mk<T>(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

constexpr int kObsWarps = 8;
constexpr int kObsRows = 8;   // rows a warp takes at once (one multi-value reduction)

// P(x), norm and energy of one sample; see the file comment.  Block
// (blockIdx.x, r - r0) owns rows_per_block rows of realization r; warp w takes
// groups of kObsRows consecutive rows (group w, w + 8, ...), lane l column
// c0 + l of each 32-column tile.  <psi|H|psi> = sum_s V(s)|psi(s)|^2 -
// 2 sum_bonds J Re(conj(psi(s)) psi(s')), every bond taken once, by the
// amplitude before it along its direction.  Dynamic shared memory:
// rows_per_block accumulators.
template <typename T, int M>
__global__ void __launch_bounds__(32 * kObsWarps) occupation_kernel(
    RealTable tab, const T *__restrict__ eps, const T *__restrict__ J,
    const cplx_t<T> *__restrict__ psi, int rows_per_block, double *P_mean, double *norm,
    double *energy, int r0) {
    using S = ObsSum<T>;
    using A = typename S::A;
    extern __shared__ __align__(16) unsigned char obs_smem[];
    A *rowacc = reinterpret_cast<A *>(obs_smem);   // [rows_per_block]
    __shared__ A colred[kObsWarps][32];
    __shared__ A red[kObsWarps][2];
    __shared__ unsigned red_bad;
    const int r = r0 + (int)blockIdx.y;
    const int N = tab.N[r];
    const int n_rows = M == 2 ? N : N * N;
    const int row0 = blockIdx.x * rows_per_block;
    if (row0 >= n_rows) return;
    const int nr = min(rows_per_block, n_rows - row0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) rowacc[i] = A(0);
    if (threadIdx.x == 0) red_bad = 0u;
    __syncthreads();
    const cplx_t<T> *a = psi + tab.st_off[r];
    const T *ep = eps + tab.par_off[r], *jp = J + tab.par_off[r];
    const T U = (T)tab.U;
    const int g = tab.group_of[r];
    const double scale = tab.inv_count[g] / M;
    double *Pg = P_mean ? P_mean + tab.group_off[g] : nullptr;
    const bool want_e = energy != nullptr;
    A en = A(0);
    unsigned bad = 0u;
    for (int c0 = 0; c0 < N; c0 += 32) {
        const int x = c0 + lane;
        const bool valid = x < N;
        const int xv = valid ? x : 0;
        const int xr = x + 1 >= N ? 0 : x + 1;          // the next column (wraps; J[N-1] = 0 when open)
        const bool load_right = lane == 31 || x + 1 >= N;
        const T ex = ep[xv], jx = valid ? jp[xv] : T(0);
        A col = A(0);
        for (int q0 = warp * kObsRows; q0 < nr; q0 += kObsWarps * kObsRows) {
            A rp[kObsRows];
#pragma unroll
            for (int u = 0; u < kObsRows; ++u) {
                const int row = row0 + q0 + u;
                const bool in = valid && q0 + u < nr;
                const int64_t rb = (int64_t)row * N;
                const cplx_t<T> c = in ? a[rb + x] : mk<T>(T(0), T(0));
                const T p = c.x * c.x + c.y * c.y;
                rp[u] = S::p(p, bad);
                col += rp[u];
                if (want_e) {
                    int xs[M - 1];
                    if (M == 2) {
                        xs[0] = row;
                    } else {
                        xs[0] = row / N;
                        xs[M - 2] = row - xs[0] * N;
                    }
                    cplx_t<T> right = shfl_c<T>(c, (lane + 1) & 31);
                    if (in && load_right) right = a[rb + xr];
                    if (in) {
                        T v = ex;
                        int pairs = 0;
#pragma unroll
                        for (int j = 0; j < M - 1; ++j) {
                            v += ep[xs[j]];
                            pairs += (xs[j] == x);
#pragma unroll
                            for (int l = j + 1; l < M - 1; ++l) pairs += (xs[j] == xs[l]);
                        }
                        v += U * T(pairs);
                        T e = p * v - T(2) * jx * (c.x * right.x + c.y * right.y);
                        // bonds along the row coordinates: the amplitude one step further along x_j
                        int64_t stride = N;
#pragma unroll
                        for (int j = M - 2; j >= 0; --j) {
                            const int xj = xs[j];
                            const int xjn = xj + 1 == N ? 0 : xj + 1;
                            const cplx_t<T> d = a[(int64_t)x + rb + (int64_t)(xjn - xj) * stride];
                            e -= T(2) * jp[xj] * (c.x * d.x + c.y * d.y);
                            stride *= N;
                        }
                        en += S::e(e, bad);
                    }
                }
            }
            // the group's row totals of this tile: lane l holds row (l >> 2) & 7
            const A rt = warp_totals<kObsRows>(rp, lane);
            if ((lane & 3) == 0 && q0 + (lane >> 2) < nr) rowacc[q0 + (lane >> 2)] += rt;
        }
        // this tile's column totals over the block's rows
        colred[warp][lane] = col;
        __syncthreads();
        if (warp == 0) {
            A t = colred[0][lane];
#pragma unroll
            for (int w = 1; w < kObsWarps; ++w) t += colred[w][lane];
            bad |= S::over(t);
            if (valid && Pg) atomicAdd(Pg + x, S::dp(t) * scale);
        }
        __syncthreads();
    }
    // row totals into P of each row coordinate, and the norm
    A nrm = A(0);
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const A t = rowacc[i];
        nrm += t;
        bad |= S::over(t);
        if (Pg) {
            const int row = row0 + i;
            if (M == 2) {
                atomicAdd(Pg + row, S::dp(t) * scale);
            } else {
                const int x1 = row / N;
                atomicAdd(Pg + x1, S::dp(t) * scale);
                atomicAdd(Pg + (row - x1 * N), S::dp(t) * scale);
            }
        }
    }
    nrm = warp_total(nrm);
    en = warp_total(en);
    if (lane == 0) {
        red[warp][0] = nrm;
        red[warp][1] = en;
    }
    if (bad) atomicOr(&red_bad, 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        A tn = red[0][0], te = red[0][1];
        for (int w = 1; w < kObsWarps; ++w) {
            tn += red[w][0];
            te += red[w][1];
        }
        const bool flag = red_bad != 0u || S::over(tn) || S::over(te);
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        if (norm) atomicAdd(norm + r, flag ? qnan : S::dp(tn));
        if (energy) atomicAdd(energy + r, flag ? qnan : S::de(te));
    }
}

// The norm check of Algorithms 2 and 3 on the sampled norms: realization r
// fails at the first sample q whose norm is not finite (reason 1) or differs
// from its first sample by more than drift_tol > 0 (reason 2).  The smallest
// key (r << 40) | (q << 8) | reason over all failures goes to the status word.
__global__ void norm_check_kernel(const double *__restrict__ norm, int64_t n_obs, int R, double drift_tol,
                                  int *status) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double n0 = norm[r];
    for (int64_t q = 0; q < n_obs; ++q) {
        const double v = norm[q * R + r];
        const unsigned reason = !isfinite(v) ? 1u : ((drift_tol > 0.0 && fabs(v - n0) > drift_tol) ? 2u : 0u);
        if (reason) {
            const unsigned long long key = ((unsigned long long)r << 40) | ((unsigned long long)q << 8) | reason;
            atomicMin(reinterpret_cast<unsigned long long *>(status + 2), key);
            atomicOr(status, 2);
            return;
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

int launch_observables_range(const ctqw_hamiltonian *h, int dtype, const void *psi, int r0, int R_run,
                             double *P_mean, double *norm, double *energy, cudaStream_t s) {
    if ((!P_mean && !norm && !energy) || R_run <= 0) return CTQW_OK;
    if (r0 < 0 || r0 + R_run > h->R) {
        ctqw_set_error("observables: realizations %d..%d outside 0..%d", r0, r0 + R_run, h->R);
        return CTQW_EINVAL;
    }
    RealTable t = real_table(h);
    // rows per block: about one wave of 8 blocks per SM over the realizations
    const int64_t rows_max = h->m == 2 ? (int64_t)h->Nmax : (int64_t)h->Nmax * h->Nmax;
    const int64_t target = 152 * 8;
    const int64_t per_r = std::max<int64_t>(1, (target + R_run - 1) / R_run);
    int64_t rpb = (rows_max + per_r - 1) / per_r;
    // a whole number of 8-row groups for every warp, at most 4096 rows
    constexpr int64_t unit = kObsWarps * kObsRows;
    rpb = std::min<int64_t>(4096, std::max<int64_t>(unit, (rpb + unit - 1) / unit * unit));
    const dim3 grid((unsigned)((rows_max + rpb - 1) / rpb), (unsigned)R_run);
    const size_t smem = (size_t)rpb * 8;
    if (dtype == CTQW_C64) {
        auto k = h->m == 2 ? occupation_kernel<float, 2> : occupation_kernel<float, 3>;
        k<<<grid, 32 * kObsWarps, smem, s>>>(t, h->eps32, h->J32, (const float2 *)psi, (int)rpb, P_mean,
                                             norm, energy, r0);
    } else {
        auto k = h->m == 2 ? occupation_kernel<double, 2> : occupation_kernel<double, 3>;
        k<<<grid, 32 * kObsWarps, smem, s>>>(t, h->eps64, h->J64, (const double2 *)psi, (int)rpb, P_mean,
                                             norm, energy, r0);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_observables(const ctqw_hamiltonian *h, int dtype, const void *psi, double *P_mean,
                       double *P_joint, double *norm, double *energy, cudaStream_t s) {
    if (!P_mean && !P_joint && !norm && !energy) return CTQW_OK;
    if (!P_joint) return launch_observables_range(h, dtype, psi, 0, h->R, P_mean, norm, energy, s);
    RealTable t = real_table(h);
    int64_t rows = 1;
    for (int j = 1; j < h->m; ++j) rows *= h->Nmax;
    dim3 grid((unsigned)((rows + kRows - 1) / kRows), (unsigned)h->R), block(kThreads);
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

int launch_norm_check(const ctqw_hamiltonian *h, const double *norm, int64_t n_obs, cudaStream_t s) {
    if (!norm || n_obs <= 0) return CTQW_OK;
    norm_check_kernel<<<(h->R + 255) / 256, 256, 0, s>>>(norm, n_obs, h->R, h->norm_drift_tol, h->status_d);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}
