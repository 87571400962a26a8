// Adjoint gradient on register tiles: two particles, complex FP32 states.
//
// The gradient of Sec. 2.3's Taylor step T = sum_{k<=K} c_k H^k,
// c_k = (-i dt)^k / k!, with respect to a parameter theta of H is
//   2 Re <lambda_{n+1}, dT/dtheta psi_n> = 2 Re sum_{a<K} <mu_a, dH/dtheta H^a psi_n>,
//   mu_a = sum_{b<K-a} conj(c_{a+b+1}) H^b lambda_{n+1}.
// In the scaled variables of the dt-weighted stencil Hh = dt H,
//   phi_a = Hh^a psi_n,   mu_a = sum_b (i^(a+b+1) / (a+b+1)!) Hh^b lambda_{n+1},
// the sum reads dt sum_a 2 Re <mu_a, dH/dtheta phi_a>, with
//   mu_{K-1} = (i^K / K!) lambda,  mu_a = (i^(a+1) / (a+1)!) lambda + Hh mu_{a+1},
// and the next adjoint state is lambda_n = T^dagger lambda_{n+1} = lambda + Hh mu_0
// (the same recurrence one level further, with coefficient i^0 / 0! = 1).
// Every term stays O(1) in FP32, where the unscaled H^a grows like |H|^a.
//
// Three kernels per step:
//  - the phi chain applies Hh on the register tiles of the forward Taylor
//    kernel (an 8W x 64 region per block, 8 rows per warp, 2 adjacent
//    columns per lane, D stages per launch with a D-deep halo) and stores
//    every level's tile;
//  - the mu chain runs the recurrence from a = K-1 down to -1 on the same
//    tiles, with lambda of the region in shared memory, stores every level
//    a >= 0 and writes lambda_n;
//  - the contraction streams mu_a and phi_a (psi_n for a = 0) for every
//    level.  dH/deps_i counts the particles on site i; dH/dJ_b is minus the
//    hop across bond b = (b, b+1): a bond collects conj(mu(x)) phi(x') from
//    both of its end points, so a point needs its own mu and phi at its four
//    neighbours.  Every point sums its terms over the levels in FP32; a warp
//    sums its rows and the block its columns, and adds them in FP64 to
//    per-tile slots (one owner per slot: no atomics, a fixed order).  A last
//    kernel sums the slots over the tiles into the per-realization
//    gradients.
// HBM per step: the chains write 2K - 1 levels and lambda_n, the contraction
// reads 2K levels: about 32 K bytes per amplitude, all of it streamed, where
// one sweep per level and term moves about 56 K with neighbour re-reads.
#include "ctqw_internal.cuh"
#include "fused_common.cuh"

namespace {

using namespace fused;

constexpr int kMaxLevels = 31;

struct ChainArgs {
    RealTable tab;
    const int32_t *list;              // the group's realizations
    const float *eps, *J;             // float32 parameters (packed per realization)
    const float2 *in;                 // input level on the region (null: the mu chain's first level)
    const float2 *q;                  // mu chain: lambda_{n+1}
    float2 *out;                      // mu chain: lambda_n (the final launch's last stage)
    float2 *lev[kMaxLevels];          // phi_a (a = 0: psi_n), written by the phi chain
    float2 *mlev[kMaxLevels];         // mu_a, written by the mu chain
    float2 co[kMaxLevels + 1];        // i^k / k!
    float dt, dtU;
    int a_in;                         // level of the launch's initial iterate
    int n_stages;                     // stencil stages of the launch
    int init;                         // mu chain: the initial iterate is (i^K / K!) lambda
    int final;                        // mu chain: the last stage is level -1 (lambda_n)
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float dotf(float2 u, float2 p) { return fmaf(u.x, p.x, u.y * p.y); }

// 32 values summed over the warp: lane l returns the total of value l
// (the FP32 counterpart of warp_sum_multi_d<32>).
__device__ __forceinline__ float warp_sum32_f(float (&v)[32], int lane) {
#pragma unroll
    for (int o = 16, n = 32; n > 1; o >>= 1, n >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < n / 2; ++q) {
            const float send = upper ? v[q] : v[q + n / 2];
            const float keep = upper ? v[q + n / 2] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// MU = false: the phi chain; MU = true: the mu chain, storing every level's
// tile for adj_contract_kernel.
template <int D, int W, bool MU>
__global__ void __launch_bounds__(32 * W, 3) adj_chain_kernel(const __grid_constant__ ChainArgs a) {
    constexpr int RS = 8 * W, T = RS - 2 * D, T2 = 64 - 2 * D, RL = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *Q = reinterpret_cast<float4 *>(smem_raw);            // mu chain: [RS][32] lambda, (row, lane) -> 2 columns
    float4 *edge = Q + (MU ? RS * 32 : 0);                        // [2 parity][W warps][2][32]
    float4 *zero = edge + 2 * W * 2 * 32;                         // [32] a row of zeros
    float4 *rowc = zero + 32;                                     // [RS + 1] (dt eps, dt eps, -dt J_up, -dt J_up)
    int *x_row = reinterpret_cast<int *>(rowc + RS + 1);          // [RS]

    const int r = a.list[blockIdx.z];
    const int N = a.tab.N[r];
    const int x1_0 = (int)blockIdx.y * T - D, x2_0 = (int)blockIdx.x * T2 - D;
    const int64_t base = a.tab.st_off[r];
    const int64_t po = a.tab.par_off[r];
    const float dt = a.dt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = warp * RL;

    for (int i = threadIdx.x; i <= RS; i += blockDim.x) {
        const int X1 = ((x1_0 + i) % N + N) % N;
        if (i < RS) x_row[i] = X1;
        const float e = i < RS ? dt * a.eps[po + X1] : 0.f;
        const float j = -dt * a.J[po + (X1 + N - 1) % N];
        rowc[i] = make_float4(e, e, j, j);
    }
    if (threadIdx.x < 32) zero[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    int X2[2];
    float2 ec[2], nJc[3];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        X2[k] = ((x2_0 + 2 * lane + k) % N + N) % N;
        const float v = dt * a.eps[po + X2[k]];
        ec[k] = make_float2(v, v);
    }
#pragma unroll
    for (int k = 0; k <= 2; ++k) {
        const int X = ((x2_0 + 2 * lane + k - 1) % N + N) % N;   // bond left of column 2 lane + k
        const float v = -dt * a.J[po + X];
        nJc[k] = make_float2(v, v);
    }
    __syncthreads();

    // the tile's points among this lane's: rows D .. D + T - 1 and columns
    // D .. D + T2 - 1 of the region that lie inside the lattice
    bool col_in[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int ck = 2 * lane + k;
        col_in[k] = ck >= D && ck < D + T2 && x2_0 + ck < N;
    }
    auto row_in = [&](int ri) { return ri >= D && ri < D + T && x1_0 + ri < N; };

    float2 P[RL][2];
    if (MU) {
        // lambda of the region into shared memory
        const float2 *gq = a.q + base;
        const uint32_t sQ = smem_u32(Q);
        for (int i = warp; i < RS; i += W) {
            const int64_t grow = (int64_t)x_row[i] * N;
#pragma unroll
            for (int k = 0; k < 2; ++k)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sQ + (uint32_t)((i * 32 + lane) * 16 + 8 * k)),
                             "l"(gq + grow + X2[k])
                             : "memory");
        }
    }
    if (!MU || !a.init) {
        const float2 *win = a.in + base;
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const int64_t grow = (int64_t)x_row[r0 + i] * N;
            P[i][0] = win[grow + X2[0]];
            P[i][1] = win[grow + X2[1]];
        }
    }
    if (MU) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
    }

    if (MU && a.init) {
        const float2 co = a.co[a.a_in + 1];
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const float4 q = Q[(r0 + i) * 32 + lane];
            P[i][0] = cmulf(co, make_float2(q.x, q.y));
            P[i][1] = cmulf(co, make_float2(q.z, q.w));
        }
        // the first level's tile
        float2 *dst = a.mlev[a.a_in] + base;
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const int ri = r0 + i;
            if (!row_in(ri)) continue;
            const int64_t grow = (int64_t)x_row[ri] * N;
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (col_in[k]) dst[grow + X2[k]] = P[i][k];
        }
    }

    const float2 dU = make_float2(a.dtU, a.dtU);
    const int from_left = (lane + 31) & 31, from_right = (lane + 1) & 31;
#pragma unroll 1
    for (int d = 1; d <= a.n_stages; ++d) {
        const int par = d & 1;
        const int lev = MU ? a.a_in - d : a.a_in + d;   // the level this stage forms
        // publish this warp's first and last rows
        float4 *eb = edge + (par * W + warp) * 2 * 32;
        eb[lane] = make_float4(P[0][0].x, P[0][0].y, P[0][1].x, P[0][1].y);
        eb[32 + lane] = make_float4(P[RL - 1][0].x, P[RL - 1][0].y, P[RL - 1][1].x, P[RL - 1][1].y);
        __syncthreads();
        const float4 u4 = warp > 0 ? edge[(par * W + warp - 1) * 2 * 32 + 32 + lane] : zero[lane];
        const float4 d4 = warp < W - 1 ? edge[(par * W + warp + 1) * 2 * 32 + lane] : zero[lane];
        float2 prev[2] = {make_float2(u4.x, u4.y), make_float2(u4.z, u4.w)};
        float4 rc = rowc[r0];
        const float2 co = MU ? a.co[lev + 1] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const float2 c0 = P[i][0], c1 = P[i][1];
            const float2 lft = shfl2(c1, from_left), rgt = shfl2(c0, from_right);
            const float2 n0 = i < RL - 1 ? P[i + 1][0] : make_float2(d4.x, d4.y);
            const float2 n1 = i < RL - 1 ? P[i + 1][1] : make_float2(d4.z, d4.w);
            const float4 rn = rowc[r0 + i + 1];
            const float2 er = make_float2(rc.x, rc.y), jup = make_float2(rc.z, rc.w), jdn = make_float2(rn.z, rn.w);
            rc = rn;
            // y = Hh P: the diagonal (column and row eps), the bonds above and
            // below, left and right, and dt U where x1 = x2
            float2 y0 = __fmul2_rn(ec[0], c0), y1 = __fmul2_rn(ec[1], c1);
            y0 = __ffma2_rn(er, c0, y0);
            y1 = __ffma2_rn(er, c1, y1);
            y0 = __ffma2_rn(jup, prev[0], y0);
            y1 = __ffma2_rn(jup, prev[1], y1);
            y0 = __ffma2_rn(jdn, n0, y0);
            y1 = __ffma2_rn(jdn, n1, y1);
            y0 = __ffma2_rn(nJc[0], lft, y0);
            y1 = __ffma2_rn(nJc[1], c0, y1);
            y0 = __ffma2_rn(nJc[1], c1, y0);
            y1 = __ffma2_rn(nJc[2], rgt, y1);
            const int X1w = x_row[r0 + i];
            if (X1w == X2[0]) y0 = __ffma2_rn(dU, c0, y0);
            if (X1w == X2[1]) y1 = __ffma2_rn(dU, c1, y1);
            prev[0] = c0;
            prev[1] = c1;
            if (MU) {
                const float4 q = Q[(r0 + i) * 32 + lane];
                // co lambda + y as four fused multiply-adds per amplitude
                P[i][0] = make_float2(fmaf(co.x, q.x, fmaf(-co.y, q.y, y0.x)), fmaf(co.x, q.y, fmaf(co.y, q.x, y0.y)));
                P[i][1] = make_float2(fmaf(co.x, q.z, fmaf(-co.y, q.w, y1.x)), fmaf(co.x, q.w, fmaf(co.y, q.z, y1.y)));
            } else {
                P[i][0] = y0;
                P[i][1] = y1;
            }
        }
        const bool last = d == a.n_stages;
        if (!MU || lev >= 0 || (a.final && last)) {
            // the phi level, lambda_n, or the stored mu level, on the tile
            float2 *dst = !MU ? a.lev[lev] + base : (lev < 0 ? a.out + base : a.mlev[lev] + base);
#pragma unroll
            for (int i = 0; i < RL; ++i) {
                const int ri = r0 + i;
                if (!row_in(ri)) continue;
                const int64_t grow = (int64_t)x_row[ri] * N;
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (col_in[k]) dst[grow + X2[k]] = P[i][k];
            }
        }
    }
}

// The per-tile slots of a size group summed over the tiles into the
// per-realization gradients: eps_x from the row and column sums at site x,
// J_b from the bond-below sum of row b and the bond-above sum of row b + 1
// (and the same along x2), scaled by 2 dt (eps) and -2 dt (J).  A bond N - 1
// exists on a ring only.
__global__ void __launch_bounds__(256) adj_tile_reduce_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                              const double *__restrict__ tg, int64_t per,
                                                              int tiles_x, int tiles_y, double dt,
                                                              double *grad_eps, double *grad_J) {
    const int z = blockIdx.y;
    const int r = list[z];
    const int N = tab.N[r];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const double *g = tg + (int64_t)z * per;
    const double *gc = g + (int64_t)tiles_x * N * 3;
    const int xp = (x + 1 == N) ? 0 : x + 1;
    double e = 0.0, j = 0.0;
    for (int t = 0; t < tiles_x; ++t) {
        e += g[((int64_t)t * N + x) * 3];
        j += g[((int64_t)t * N + x) * 3 + 1] + g[((int64_t)t * N + xp) * 3 + 2];
    }
    for (int t = 0; t < tiles_y; ++t) {
        e += gc[((int64_t)t * N + x) * 3];
        j += gc[((int64_t)t * N + x) * 3 + 1] + gc[((int64_t)t * N + xp) * 3 + 2];
    }
    const int64_t po = tab.par_off[r];
    grad_eps[po + x] += 2.0 * dt * e;
    if (tab.periodic || x < N - 1) grad_J[po + x] += -2.0 * dt * j;
}

// The contraction of every level a < K, streamed: mu_a (stored by the mu
// chain) against phi_a (stored by the phi chain; psi_n for a = 0).  A block
// owns a tile of kCtRows x kCtCols points (4 warps x 4 rows, 2 columns a
// lane); every point sums its five terms over the levels in registers, and
// at the end a warp sums its rows and the block its columns into the
// per-tile FP64 slots (one owner each).  Per level and point it reads 8 B
// of mu and 8 B of phi from HBM (the neighbour rows and the lanes' edge
// columns from L1/L2).
constexpr int kCtRows = 16, kCtCols = 64, kCtWarps = 4, kCtRL = 4;

struct ContractArgs {
    RealTable tab;
    const int32_t *list;
    const float2 *lev[kMaxLevels];    // phi_a
    const float2 *mlev[kMaxLevels];   // mu_a
    int K;
    double *tg;
    int64_t tg_per_real;
    int tiles_x;                      // column tiles (kCtCols wide)
};

__global__ void __launch_bounds__(32 * kCtWarps, 4) adj_contract_kernel(const __grid_constant__ ContractArgs a) {
    __shared__ float colsum[kCtWarps][kCtCols][3];
    const int r = a.list[blockIdx.z];
    const int N = a.tab.N[r];
    const int x1_0 = (int)blockIdx.y * kCtRows, x2_0 = (int)blockIdx.x * kCtCols;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = a.tab.st_off[r];
    auto wrap = [N](int x) { return x < 0 ? x + N : (x >= N ? x - N : x); };
    int x2[2];
    bool col_ok[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        x2[k] = x2_0 + 2 * lane + k;
        col_ok[k] = x2[k] < N;
    }
    const int xl = wrap(x2[0] - 1), xr = wrap(x2[1] + 1);
    // the neighbours along x2 come from the adjacent lane unless the lane is
    // at the warp's end or the neighbour wraps around the lattice
    const bool own_l = lane > 0 && x2[0] > 0, own_r = lane < 31 && x2[1] + 1 < N;
    int x1[kCtRL + 2];   // rows r0 - 1 .. r0 + kCtRL (wrapped)
#pragma unroll
    for (int i = 0; i < kCtRL + 2; ++i) x1[i] = wrap(x1_0 + warp * kCtRL + i - 1);
    const float2 z = make_float2(0.f, 0.f);
    float sd[kCtRL][2], sdn[kCtRL][2], sup[kCtRL][2], srt[kCtRL][2], slf[kCtRL][2];
#pragma unroll
    for (int i = 0; i < kCtRL; ++i)
#pragma unroll
        for (int k = 0; k < 2; ++k) sd[i][k] = sdn[i][k] = sup[i][k] = srt[i][k] = slf[i][k] = 0.f;
#pragma unroll 1
    for (int lv = 0; lv < a.K; ++lv) {
        const float2 *mu = a.mlev[lv] + base, *ph = a.lev[lv] + base;
        float2 u[kCtRL][2], p[kCtRL + 2][2], pl[kCtRL], pr[kCtRL];
#pragma unroll
        for (int i = 0; i < kCtRL + 2; ++i) {
            const int64_t rb = (int64_t)x1[i] * N;
#pragma unroll
            for (int k = 0; k < 2; ++k) p[i][k] = col_ok[k] ? ph[rb + x2[k]] : z;
            if (i >= 1 && i <= kCtRL) {
#pragma unroll
                for (int k = 0; k < 2; ++k) u[i - 1][k] = col_ok[k] ? mu[rb + x2[k]] : z;
                pl[i - 1] = (!own_l && col_ok[0]) ? ph[rb + xl] : z;
                pr[i - 1] = (!own_r && col_ok[1]) ? ph[rb + xr] : z;
            }
        }
#pragma unroll
        for (int i = 0; i < kCtRL; ++i) {
            const float2 l = shfl2(p[i + 1][1], (lane + 31) & 31), rr = shfl2(p[i + 1][0], (lane + 1) & 31);
            const float2 left = own_l ? l : pl[i], right = own_r ? rr : pr[i];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float2 uu = u[i][k];
                sd[i][k] += dotf(uu, p[i + 1][k]);
                sdn[i][k] += dotf(uu, p[i + 2][k]);
                sup[i][k] += dotf(uu, p[i][k]);
                srt[i][k] += dotf(uu, k ? right : p[i + 1][1]);
                slf[i][k] += dotf(uu, k ? p[i + 1][0] : left);
            }
        }
    }
    double *tg = a.tg + (int64_t)blockIdx.z * a.tg_per_real;
    // rows: 4 rows x 3 sums over the warp's 64 columns; value 4 i + q (16 of
    // the 32 slots used) ends in lane 4 i + q
    float v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = 0.f;
#pragma unroll
    for (int i = 0; i < kCtRL; ++i) {
        float e = 0.f, dn = 0.f, up = 0.f;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (col_ok[k]) {
                e += sd[i][k];
                dn += sdn[i][k];
                up += sup[i][k];
            }
        v[4 * i] = e;
        v[4 * i + 1] = dn;
        v[4 * i + 2] = up;
    }
    const float tot = warp_sum32_f(v, lane);
    {
        const int i = lane >> 2, q = lane & 3, row = x1_0 + warp * kCtRL + i;
        if (i < kCtRL && q < 3 && row < N) tg[((int64_t)blockIdx.x * N + row) * 3 + q] += (double)tot;
    }
    // columns: over the warp's rows in registers, over the warps in shared memory
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float e = 0.f, rt = 0.f, lf = 0.f;
#pragma unroll
        for (int i = 0; i < kCtRL; ++i)
            if (x1_0 + warp * kCtRL + i < N) {
                e += sd[i][k];
                rt += srt[i][k];
                lf += slf[i][k];
            }
        colsum[warp][2 * lane + k][0] = e;
        colsum[warp][2 * lane + k][1] = rt;
        colsum[warp][2 * lane + k][2] = lf;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kCtCols * 3; t += blockDim.x) {
        const int c = t / 3, q = t - 3 * (t / 3);
        if (x2_0 + c >= N) continue;
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < kCtWarps; ++w) sum += colsum[w][c][q];
        tg[(int64_t)a.tiles_x * N * 3 + ((int64_t)blockIdx.y * N + (x2_0 + c)) * 3 + q] += (double)sum;
    }
}

using ChainKernel = void (*)(ChainArgs);

struct ChainShape {
    int D, T, T2, threads;
    ChainKernel phi, mu;
    size_t smem_phi, smem_mu;
};

template <int D, int W = 8>
ChainShape chain_shape() {
    constexpr int RS = 8 * W;
    ChainShape s;
    s.D = D;
    s.T = RS - 2 * D;
    s.T2 = 64 - 2 * D;
    s.threads = 32 * W;
    s.phi = adj_chain_kernel<D, W, false>;
    s.mu = adj_chain_kernel<D, W, true>;
    s.smem_phi = sizeof(float4) * (2 * W * 2 * 32 + 32 + RS + 1) + sizeof(int) * RS;
    s.smem_mu = s.smem_phi + sizeof(float4) * RS * 32;
    return s;
}

// Depth for K levels: the fewest launches at depth <= 8, the levels split
// evenly, rounded up to a compiled depth.
ChainShape chain_shape_for(int K) {
    const int launches = (K + 7) / 8;
    const int need = (K + launches - 1) / launches;
    if (need <= 4) return chain_shape<4>();
    if (need <= 6) return chain_shape<6>();
    if (need <= 7) return chain_shape<7>();
    return chain_shape<8>();
}

ChainArgs chain_args(const ctqw_hamiltonian *h, double dt) {
    ChainArgs a;
    a.tab = real_table(h);
    a.eps = h->eps32;
    a.J = h->J32;
    a.in = nullptr;
    a.q = nullptr;
    a.out = nullptr;
    for (int i = 0; i < kMaxLevels; ++i) a.lev[i] = a.mlev[i] = nullptr;
    // i^k / k!
    double mag = 1.0;
    for (int k = 0; k <= kMaxLevels; ++k) {
        if (k > 0) mag /= k;
        const int q = k & 3;
        a.co[k] = make_float2((float)(q == 0 ? mag : (q == 2 ? -mag : 0.0)),
                              (float)(q == 1 ? mag : (q == 3 ? -mag : 0.0)));
    }
    a.dt = (float)dt;
    a.dtU = (float)(dt * h->U);
    a.a_in = 0;
    a.n_stages = 0;
    a.init = 0;
    a.final = 0;
    return a;
}

}  // namespace

bool adjoint_tiled_supported(const ctqw_hamiltonian *h, int dtype, int K) {
    return dtype == CTQW_C64 && h->m == 2 && K >= 1 && K < kMaxLevels;
}

size_t adjoint_tiled_slots(const ctqw_hamiltonian *h, int K) {
    (void)K;
    size_t n = 0;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g];
        const int tx = (N + kCtCols - 1) / kCtCols, ty = (N + kCtRows - 1) / kCtRows;
        n += (size_t)h->group_count[g] * (size_t)(tx + ty) * (size_t)N * 3;
    }
    return n;
}

// phi_a = Hh^a psi for a = 1 .. K - 1 into levels[a] (levels[0] = psi).
int launch_adjoint_phi_chain(const ctqw_hamiltonian *h, int K, double dt, void *const *levels, cudaStream_t s) {
    const ChainShape f = chain_shape_for(K);
    CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)f.phi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)f.smem_phi));
    ChainArgs a = chain_args(h, dt);
    for (int i = 0; i < K; ++i) a.lev[i] = (float2 *)levels[i];
    for (int a0 = 0; a0 < K - 1;) {
        const int n = std::min(f.D, K - 1 - a0);
        a.in = (const float2 *)levels[a0];
        a.a_in = a0;
        a.n_stages = n;
        int off = 0;
        for (size_t g = 0; g < h->group_N.size(); ++g) {
            const int N = h->group_N[g], cnt = h->group_count[g];
            a.list = h->by_group_d + off;
            const dim3 grid((unsigned)((N + f.T2 - 1) / f.T2), (unsigned)((N + f.T - 1) / f.T), (unsigned)cnt);
            f.phi<<<grid, f.threads, f.smem_phi, s>>>(a);
            CTQW_CUDA_TRY(cudaGetLastError());
            off += cnt;
        }
        a0 += n;
    }
    return CTQW_OK;
}

// The mu recurrence from level K - 1 down to -1: every level a >= 0 into
// mu_levels[a], lambda_n = T^dagger lambda into lam_out.
int launch_adjoint_mu_chain(const ctqw_hamiltonian *h, int K, double dt, const void *lam, void *const *mu_levels,
                            void *lam_out, cudaStream_t s) {
    const ChainShape f = chain_shape_for(K);
    CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)f.mu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)f.smem_mu));
    ChainArgs a = chain_args(h, dt);
    for (int i = 0; i < K; ++i) a.mlev[i] = (float2 *)mu_levels[i];
    a.q = (const float2 *)lam;
    int a_in = K - 1, remaining = K;
    bool init = true;
    while (remaining > 0) {
        const int n = std::min(f.D, remaining);
        const bool final = n == remaining;
        a.in = init ? nullptr : (const float2 *)mu_levels[a_in];
        a.out = final ? (float2 *)lam_out : nullptr;
        a.a_in = a_in;
        a.n_stages = n;
        a.init = init ? 1 : 0;
        a.final = final ? 1 : 0;
        int off = 0;
        for (size_t g = 0; g < h->group_N.size(); ++g) {
            const int N = h->group_N[g], cnt = h->group_count[g];
            const int tx = (N + f.T2 - 1) / f.T2, ty = (N + f.T - 1) / f.T;
            a.list = h->by_group_d + off;
            f.mu<<<dim3((unsigned)tx, (unsigned)ty, (unsigned)cnt), f.threads, f.smem_mu, s>>>(a);
            CTQW_CUDA_TRY(cudaGetLastError());
            off += cnt;
        }
        a_in -= n;
        init = false;
        remaining -= n;
    }
    return CTQW_OK;
}

// The contraction of mu_levels[a] with levels[a] over a < K into the tile
// slots tg.
int launch_adjoint_contract(const ctqw_hamiltonian *h, int K, void *const *levels, void *const *mu_levels,
                            double *tg, cudaStream_t s) {
    ContractArgs a;
    a.tab = real_table(h);
    for (int i = 0; i < kMaxLevels; ++i) {
        a.lev[i] = i < K ? (const float2 *)levels[i] : nullptr;
        a.mlev[i] = i < K ? (const float2 *)mu_levels[i] : nullptr;
    }
    a.K = K;
    int off = 0;
    double *tgg = tg;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g], cnt = h->group_count[g];
        const int tx = (N + kCtCols - 1) / kCtCols, ty = (N + kCtRows - 1) / kCtRows;
        a.list = h->by_group_d + off;
        a.tg = tgg;
        a.tg_per_real = (int64_t)(tx + ty) * N * 3;
        a.tiles_x = tx;
        adj_contract_kernel<<<dim3((unsigned)tx, (unsigned)ty, (unsigned)cnt), 32 * kCtWarps, 0, s>>>(a);
        CTQW_CUDA_TRY(cudaGetLastError());
        off += cnt;
        tgg += (size_t)cnt * a.tg_per_real;
    }
    return CTQW_OK;
}

// The tile slots into the per-realization gradients (added to grad_*).
int launch_adjoint_tile_reduce(const ctqw_hamiltonian *h, int K, double dt, const double *tg, double *grad_eps,
                               double *grad_J, cudaStream_t s) {
    (void)K;
    RealTable t = real_table(h);
    int off = 0;
    const double *tgg = tg;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g], cnt = h->group_count[g];
        const int tx = (N + kCtCols - 1) / kCtCols, ty = (N + kCtRows - 1) / kCtRows;
        const int64_t per = (int64_t)(tx + ty) * N * 3;
        adj_tile_reduce_kernel<<<dim3((unsigned)((N + 255) / 256), (unsigned)cnt), 256, 0, s>>>(
            t, h->by_group_d + off, tgg, per, tx, ty, dt, grad_eps, grad_J);
        CTQW_CUDA_TRY(cudaGetLastError());
        off += cnt;
        tgg += (size_t)cnt * per;
    }
    return CTQW_OK;
}
