// Temporally blocked Taylor stages for two particles in complex FP32: D
// Horner stages per launch on shared-memory tiles with halos.
//
// The order-K polynomial of Algorithm 3 (Sec. 2.3) in Horner form,
//   w_K = psi + (A/K) psi,  w_j = psi + (A/j) w_{j+1},  psi(t+dt) = psi + A w_2,
// A = -i dt H, is split into launches of D consecutive stages.  A block owns
// a T x T tile of the N x N amplitude tile of one realization.  It loads the
// launch's input iterate and psi on the tile plus D rows and columns around
// it, applies the D stages in shared memory (stage d is exact on the tile
// grown by D - d, so the halo shrinks by one per stage), and writes the
// tile of the result.  Per launch HBM carries the input iterate, psi and the
// output once (the halo reloads are L2 hits): about 24/D bytes per
// site-update against 24 for one launch per stage.  The extra arithmetic is
// the halo, sum_d (T + 2(D - d))^2 / (D T^2) - 1 of the work (20% for T = 32,
// D = 4).
//
// Coordinates outside 0..N-1 wrap around: on a ring that is the lattice, on
// an open chain the wrap bond has J[N-1] = 0, so the wrapped halo holds valid
// values of real sites and nothing crosses the open boundary.  When the
// launch ends with the final stage, the increment A w_2 is added to psi with
// its rounding error carried in a second FP32 word (lo, in place: every
// element is read and written by its own tile only), and the new psi goes to
// a separate buffer because other tiles still read the old psi as halo.
#include "ctqw_internal.cuh"
#include "fused_common.cuh"

namespace {

using namespace fused;

// One launch for every size group (register tiles): the work items
// (realization, tile row, tile column) of all groups form one 1D grid,
// groups in descending N so that the block scheduler starts the largest
// items first and the small ones fill the tail.
constexpr int kMaxFlatGroups = 32;
struct FlatGroups {
    int n;                              // groups in the launch (0: one launch per group)
    int64_t item_off[kMaxFlatGroups + 1];   // first item of each group
    int list_off[kMaxFlatGroups];       // its realizations in by_group (the launch's list)
    int tiles_y[kMaxFlatGroups], tiles_x[kMaxFlatGroups];
};

struct TiledArgs {
    RealTable tab;
    FlatGroups flat;
    const int32_t *list;     // realizations of this launch's size group (all groups when flat.n > 0)
    const float *eps, *J;    // float32 parameters (packed per realization)
    const float2 *w_in;      // input iterate (w_{j0+1}; psi itself when j0 = K)
    const float2 *psi;       // state of the step
    float2 *w_out;           // output iterate w_{j0-D+1}, or the new state when final
    float2 *lo;              // carried rounding error (final launches when compensated)
    float dt, dtU;
    int T;                   // tile side for this size group (<= the compiled maximum)
    int j0;                  // first stage of the launch (stage j maps w_{j+1} -> w_j)
    int n_stages;            // D, or fewer for the last launch of a step
    int final;               // the launch's last stage is j = 1 (state update)
    int compensated;
};


// The block's work item: its realization and tile (row, column).
struct TileItem {
    int r, ty, tx;
};

__device__ __forceinline__ TileItem tile_item(const TiledArgs &a) {
    TileItem t;
    if (a.flat.n == 0) {
        t.r = a.list[blockIdx.z];
        t.ty = blockIdx.y;
        t.tx = blockIdx.x;
        return t;
    }
    const int64_t it = blockIdx.x;
    int g = 0;
    while (g + 1 < a.flat.n && it >= a.flat.item_off[g + 1]) ++g;
    const int64_t local = it - a.flat.item_off[g];
    const int per_r = a.flat.tiles_y[g] * a.flat.tiles_x[g];
    const int q = (int)(local / per_r), rem = (int)(local - (int64_t)q * per_r);
    t.r = a.list[a.flat.list_off[g] + q];
    t.ty = rem / a.flat.tiles_x[g];
    t.tx = rem - t.ty * a.flat.tiles_x[g];
    return t;
}

// T x T output tile (T <= TMAX, chosen per size group so that the tiles
// cover N evenly), D halo, blockDim = 256 (warps over rows, lanes over
// columns).  Region rows are stored with the compiled stride RS.
template <int TMAX, int D>
__global__ void __launch_bounds__(256) taylor_tiled_kernel(const __grid_constant__ TiledArgs a) {
    constexpr int RS = TMAX + 2 * D;    // region row stride
    constexpr int RE = RS * RS;
    const int T = a.T;
    const int RC = T + 2 * D;           // region side
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *bufA = reinterpret_cast<float2 *>(smem_raw);   // [RE]
    float2 *bufB = bufA + RE;                              // [RE]
    float2 *Q = bufB + RE;                                 // [RE] psi on the region
    float *e_row = reinterpret_cast<float *>(Q + RE);      // [RS] dt eps of the region's rows
    float *e_col = e_row + RS;                             // [RS]
    float *j_row = e_col + RS;                             // [RS + 1] -dt J of the bond above row i
    float *j_col = j_row + RS + 1;                         // [RS + 1] -dt J of the bond left of column k
    int *x_row = reinterpret_cast<int *>(j_col + RS + 1);  // [RS] wrapped coordinates
    int *x_col = x_row + RS;                               // [RS]

    const int r = a.list[blockIdx.z];
    const int N = a.tab.N[r];
    const int tiles = (N + T - 1) / T;
    if ((int)blockIdx.x >= tiles || (int)blockIdx.y >= tiles) return;   // never: one grid per group
    const int x1_0 = blockIdx.y * T - D, x2_0 = blockIdx.x * T - D;
    const int64_t base = a.tab.st_off[r];
    const int64_t po = a.tab.par_off[r];
    const float dt = a.dt;

    for (int i = threadIdx.x; i < RC; i += blockDim.x) {
        const int X1 = ((x1_0 + i) % N + N) % N, X2 = ((x2_0 + i) % N + N) % N;
        x_row[i] = X1;
        x_col[i] = X2;
        e_row[i] = dt * a.eps[po + X1];
        e_col[i] = dt * a.eps[po + X2];
        j_row[i] = -dt * a.J[po + (X1 + N - 1) % N];
        j_col[i] = -dt * a.J[po + (X2 + N - 1) % N];
    }
    if (threadIdx.x == 0) {
        const int X1 = ((x1_0 + RC - 1) % N + N) % N, X2 = ((x2_0 + RC - 1) % N + N) % N;
        j_row[RC] = -dt * a.J[po + X1];
        j_col[RC] = -dt * a.J[po + X2];
    }
    __syncthreads();
    // the region of the input iterate and of psi (warps over rows, lanes over
    // columns), copied asynchronously so that every load of the block is in
    // flight at once
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
    const float2 *win = a.w_in + base, *gpsi = a.psi + base;
    const uint32_t sA = smem_u32(bufA), sQ = smem_u32(Q);
    for (int i = ty; i < RC; i += ny) {
        const int64_t grow = (int64_t)x_row[i] * N;
        for (int k = tx; k < RC; k += 32) {
            const uint32_t o = (uint32_t)(i * RS + k) * 8u;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sA + o), "l"(win + grow + x_col[k])
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sQ + o), "l"(gpsi + grow + x_col[k])
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    // every warp owns RS/8 consecutive region rows for the whole launch and
    // keeps psi of its rows and its two column passes in registers
    constexpr int CH = RS / 8;           // rows a warp (8 warps)
    static_assert(RS % 8 == 0 && RS <= 64, "region rows split over 8 warps, two column passes");
    const int r0 = ty * CH;
    float2 qv[2][CH];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
#pragma unroll
        for (int t = 0; t < CH; ++t) qv[p][t] = Q[(r0 + t) * RS + tx + 32 * p];
    }

    float2 *src = bufA, *dst = bufB;
    const float dU = a.dtU;
#pragma unroll 1
    for (int d = 1; d <= a.n_stages; ++d) {
        const int j = a.j0 - d + 1;
        const bool last_final = a.final && d == a.n_stages;   // j == 1
        const float inv_j = 1.0f / (float)j;
        // stage d is exact on the region shrunk by d; the final stage is
        // needed on the tile only
        const int lo = last_final ? D : d, hi = last_final ? D + T : RC - d;
        const int i0 = max(lo, r0), i1 = min(hi, r0 + CH);   // this warp's rows of the stage
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int k = tx + 32 * p;
            if (k < lo || k >= hi || i0 >= i1) continue;
            const float ec = e_col[k], jl = j_col[k], jr = j_col[k + 1];
            const int X2w = x_col[k];
            const bool col_in = x2_0 + k < N;
            float2 wu = src[(i0 - 1) * RS + k], wc = src[i0 * RS + k];
            float ju = j_row[i0];
#pragma unroll
            for (int t = 0; t < CH; ++t) {
                const int i = r0 + t;
                if (i < i0 || i >= i1) continue;
                const int c = i * RS + k;
                const float2 wd = src[c + RS], wl = src[c - 1], wr = src[c + 1];
                const float jd = j_row[i + 1];
                float v = e_row[i] + ec;
                if (x_row[i] == X2w) v += dU;
                // y = dt H w
                float yx = v * wc.x, yy = v * wc.y;
                yx = fmaf(ju, wu.x, yx); yy = fmaf(ju, wu.y, yy);
                yx = fmaf(jd, wd.x, yx); yy = fmaf(jd, wd.y, yy);
                yx = fmaf(jl, wl.x, yx); yy = fmaf(jl, wl.y, yy);
                yx = fmaf(jr, wr.x, yx); yy = fmaf(jr, wr.y, yy);
                const float2 q = qv[p][t];
                if (!last_final) {
                    // w_j = psi + (-i/j) y
                    dst[c] = make_float2(fmaf(inv_j, yy, q.x), fmaf(-inv_j, yx, q.y));
                } else if (col_in && x1_0 + i < N) {
                    // psi(t+dt) = psi + (-i) y, rounding error carried in lo
                    const int64_t g = base + (int64_t)x_row[i] * N + X2w;
                    float2 h = q;
                    const float2 inc = make_float2(yy, -yx);
                    if (a.compensated) {
                        float2 l = a.lo[g];
                        compensated_add(h.x, l.x, inc.x);
                        compensated_add(h.y, l.y, inc.y);
                        a.lo[g] = l;
                    } else {
                        h.x += inc.x;
                        h.y += inc.y;
                    }
                    a.w_out[g] = h;
                }
                wu = wc;
                wc = wd;
                ju = jd;
            }
        }
        __syncthreads();
        float2 *tsw = src;
        src = dst;
        dst = tsw;
    }
    if (!a.final) {
        // the tile of the launch's last iterate (exact on the tile)
        for (int i = D + ty; i < D + T; i += ny) {
            const int X1 = x1_0 + i;
            if (X1 >= N) break;
            for (int k = D + tx; k < D + T; k += 32) {
                const int X2 = x2_0 + k;
                if (X2 < N) a.w_out[base + (int64_t)X1 * N + X2] = src[i * RS + k];
            }
        }
    }
}

// The same D stages with the iterate in registers: the region is 8W rows x
// 64 columns (tile (8W - 2D) x (64 - 2D)), every warp holds 8 region rows
// and every lane the two adjacent columns 2l, 2l+1 of them.  Neighbours along x2 are in the lane or
// one 64-bit shuffle away; along x1 in registers except the warp's first
// and last rows, which pass through shared memory once per stage (one
// __syncthreads).  psi of the region stays in shared memory.  The shuffles
// wrap from column 63 to 0 and the outermost warps read zero rows: both
// only touch the halo's outer ring, which stage 1 already leaves inexact.
template <int D, int W>
__global__ void __launch_bounds__(32 * W, W == 8 ? 3 : 2) taylor_tiled_reg_kernel(const __grid_constant__ TiledArgs a) {
    constexpr int RS = 8 * W, T = RS - 2 * D, T2 = 64 - 2 * D, RL = 8;   // rows x 64 columns
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *Q = reinterpret_cast<float4 *>(smem_raw);            // [RS][32] psi, (row, lane) -> 2 columns
    float4 *edge = Q + RS * 32;                                   // [2 parity][W warps][2][32]
    float4 *zero = edge + 2 * W * 2 * 32;                         // [32] a row of zeros
    float4 *rowc = zero + 32;                                     // [RS + 1] (dt eps, dt eps, -dt J_up, -dt J_up)
    int *x_row = reinterpret_cast<int *>(rowc + RS + 1);          // [RS]

    const TileItem item = tile_item(a);
    const int r = item.r;
    const int N = a.tab.N[r];
    const int x1_0 = item.ty * T - D, x2_0 = item.tx * T2 - D;
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
    // this lane's columns and their coefficients
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
    // psi of the region (asynchronous) and the input iterate into registers
    const float2 *win = a.w_in + base, *gpsi = a.psi + base;
    const uint32_t sQ = smem_u32(Q);
    for (int i = warp; i < RS; i += W) {
        const int64_t grow = (int64_t)x_row[i] * N;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sQ + (uint32_t)((i * 32 + lane) * 16 + 8 * k)),
                         "l"(gpsi + grow + X2[k])
                         : "memory");
    }
    float2 P[RL][2];
#pragma unroll
    for (int i = 0; i < RL; ++i) {
        const int64_t grow = (int64_t)x_row[r0 + i] * N;
        P[i][0] = win[grow + X2[0]];
        P[i][1] = win[grow + X2[1]];
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    const float2 dU = make_float2(a.dtU, a.dtU);
    const int from_left = (lane + 31) & 31, from_right = (lane + 1) & 31;
#pragma unroll 1
    for (int d = 1; d <= a.n_stages; ++d) {
        const int par = d & 1;
        const int j = a.j0 - d + 1;
        const bool last_final = a.final && d == a.n_stages;   // j == 1
        const float inv_j = 1.0f / (float)j;
        // publish this warp's first and last rows
        float4 *eb = edge + (par * W + warp) * 2 * 32;
        eb[lane] = make_float4(P[0][0].x, P[0][0].y, P[0][1].x, P[0][1].y);
        eb[32 + lane] = make_float4(P[RL - 1][0].x, P[RL - 1][0].y, P[RL - 1][1].x, P[RL - 1][1].y);
        __syncthreads();
        const float4 u4 = warp > 0 ? edge[(par * W + warp - 1) * 2 * 32 + 32 + lane] : zero[lane];
        const float4 d4 = warp < W - 1 ? edge[(par * W + warp + 1) * 2 * 32 + lane] : zero[lane];
        float2 prev[2] = {make_float2(u4.x, u4.y), make_float2(u4.z, u4.w)};
        float4 rc = rowc[r0];
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const float2 c0 = P[i][0], c1 = P[i][1];
            const float2 lft = shfl2(c1, from_left), rgt = shfl2(c0, from_right);
            const float2 n0 = i < RL - 1 ? P[i + 1][0] : make_float2(d4.x, d4.y);
            const float2 n1 = i < RL - 1 ? P[i + 1][1] : make_float2(d4.z, d4.w);
            const float4 rn = rowc[r0 + i + 1];
            const float2 er = make_float2(rc.x, rc.y), jup = make_float2(rc.z, rc.w), jdn = make_float2(rn.z, rn.w);
            rc = rn;
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
            if (X1w == X2[0]) y0 = __ffma2_rn(dU, c0, y0);   // dt U on x1 = x2
            if (X1w == X2[1]) y1 = __ffma2_rn(dU, c1, y1);
            prev[0] = c0;
            prev[1] = c1;
            const float4 q = Q[(r0 + i) * 32 + lane];
            if (!last_final) {
                P[i][0] = make_float2(fmaf(inv_j, y0.y, q.x), fmaf(-inv_j, y0.x, q.y));
                P[i][1] = make_float2(fmaf(inv_j, y1.y, q.z), fmaf(-inv_j, y1.x, q.w));
            } else {
                // psi(t+dt) = psi + (-i) y on the tile, rounding error carried in lo
                const int ri = r0 + i;
                if (ri >= D && ri < D + T && x1_0 + ri < N) {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int ck = 2 * lane + k;
                        if (ck < D || ck >= D + T2 || x2_0 + ck >= N) continue;
                        const int64_t g = base + (int64_t)X1w * N + X2[k];
                        const float2 yk = k ? y1 : y0;
                        float2 h = k ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
                        const float2 inc = make_float2(yk.y, -yk.x);
                        if (a.compensated) {
                            float2 l = a.lo[g];
                            compensated_add(h.x, l.x, inc.x);
                            compensated_add(h.y, l.y, inc.y);
                            a.lo[g] = l;
                        } else {
                            h.x += inc.x;
                            h.y += inc.y;
                        }
                        a.w_out[g] = h;
                    }
                }
            }
        }
    }
    if (!a.final) {
        // the tile of the launch's last iterate
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const int ri = r0 + i;
            if (ri < D || ri >= D + T || x1_0 + ri >= N) continue;
            const int64_t grow = base + (int64_t)x_row[ri] * N;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int ck = 2 * lane + k;
                if (ck >= D && ck < D + T2 && x2_0 + ck < N) a.w_out[grow + X2[k]] = P[i][k];
            }
        }
    }
}

// The register tiles on a wider region: 64 rows x 32 CL columns (tile
// (64 - 2D) x (32 CL - 2D)), every lane owning CL adjacent columns, so a
// smaller share of the region is halo and neighbours along x2 are mostly in
// the lane.  psi rows in shared memory are lane-major (column pair k/2 of
// lane l at float4 slot (k/2)*32 + l), as in the full-row kernel.
template <int D, int CL>
__global__ void __launch_bounds__(256, 2) taylor_tiled_wide_kernel(const __grid_constant__ TiledArgs a) {
    constexpr int RR = 64, RC = 32 * CL, T1 = RR - 2 * D, T2 = RC - 2 * D, RL = 8;
    static_assert(CL % 2 == 0, "column pairs");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *Q = reinterpret_cast<float4 *>(smem_raw);            // [RR][RC / 2] lane-major pairs
    float4 *edge = Q + RR * (RC / 2);                             // [2 parity][8 warps][2][RC / 2]
    float4 *zero = edge + 2 * 8 * 2 * (RC / 2);                   // [RC / 2]
    float4 *rowc = zero + RC / 2;                                 // [RR + 1]
    int *x_row = reinterpret_cast<int *>(rowc + RR + 1);          // [RR]

    const TileItem item = tile_item(a);
    const int r = item.r;
    const int N = a.tab.N[r];
    const int x1_0 = item.ty * T1 - D, x2_0 = item.tx * T2 - D;
    const int64_t base = a.tab.st_off[r];
    const int64_t po = a.tab.par_off[r];
    const float dt = a.dt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = warp * RL;

    for (int i = threadIdx.x; i <= RR; i += blockDim.x) {
        const int X1 = ((x1_0 + i) % N + N) % N;
        if (i < RR) x_row[i] = X1;
        const float e = i < RR ? dt * a.eps[po + X1] : 0.f;
        const float j = -dt * a.J[po + (X1 + N - 1) % N];
        rowc[i] = make_float4(e, e, j, j);
    }
    for (int q = threadIdx.x; q < RC / 2; q += blockDim.x) zero[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    int X2[CL];
    float2 ec[CL], nJc[CL + 1];
#pragma unroll
    for (int k = 0; k < CL; ++k) {
        X2[k] = ((x2_0 + CL * lane + k) % N + N) % N;
        const float v = dt * a.eps[po + X2[k]];
        ec[k] = make_float2(v, v);
    }
#pragma unroll
    for (int k = 0; k <= CL; ++k) {
        const int X = ((x2_0 + CL * lane + k - 1) % N + N) % N;   // bond left of column CL lane + k
        const float v = -dt * a.J[po + X];
        nJc[k] = make_float2(v, v);
    }
    __syncthreads();
    const float2 *win = a.w_in + base, *gpsi = a.psi + base;
    const uint32_t sQ = smem_u32(Q);
    for (int i = warp; i < RR; i += 8) {
        const int64_t grow = (int64_t)x_row[i] * N;
#pragma unroll
        for (int k = 0; k < CL; ++k) {
            const uint32_t slot = (uint32_t)(i * (RC / 2) + (k / 2) * 32 + lane);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sQ + slot * 16u + 8u * (k & 1)),
                         "l"(gpsi + grow + X2[k])
                         : "memory");
        }
    }
    float2 P[RL][CL];
#pragma unroll
    for (int i = 0; i < RL; ++i) {
        const int64_t grow = (int64_t)x_row[r0 + i] * N;
#pragma unroll
        for (int k = 0; k < CL; ++k) P[i][k] = win[grow + X2[k]];
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    const float2 dU = make_float2(a.dtU, a.dtU);
    const int from_left = (lane + 31) & 31, from_right = (lane + 1) & 31;
#pragma unroll 1
    for (int d = 1; d <= a.n_stages; ++d) {
        const int par = d & 1;
        const int j = a.j0 - d + 1;
        const bool last_final = a.final && d == a.n_stages;   // j == 1
        const float inv_j = 1.0f / (float)j;
        float4 *eb = edge + (par * 8 + warp) * 2 * (RC / 2);
#pragma unroll
        for (int k = 0; k < CL; k += 2) {
            eb[(k / 2) * 32 + lane] = make_float4(P[0][k].x, P[0][k].y, P[0][k + 1].x, P[0][k + 1].y);
            eb[RC / 2 + (k / 2) * 32 + lane] =
                make_float4(P[RL - 1][k].x, P[RL - 1][k].y, P[RL - 1][k + 1].x, P[RL - 1][k + 1].y);
        }
        __syncthreads();
        const float4 *us = warp > 0 ? edge + (par * 8 + warp - 1) * 2 * (RC / 2) + RC / 2 : zero;
        const float4 *ds = warp < 7 ? edge + (par * 8 + warp + 1) * 2 * (RC / 2) : zero;
        float2 prev[CL];
#pragma unroll
        for (int k = 0; k < CL; k += 2) {
            const float4 u4 = us[(k / 2) * 32 + lane];
            prev[k] = make_float2(u4.x, u4.y);
            prev[k + 1] = make_float2(u4.z, u4.w);
        }
        float4 rc = rowc[r0];
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            float2 c[CL];
#pragma unroll
            for (int k = 0; k < CL; ++k) c[k] = P[i][k];
            const float2 lft = shfl2(c[CL - 1], from_left), rgt = shfl2(c[0], from_right);
            float2 nb[CL];
            if (i < RL - 1) {
#pragma unroll
                for (int k = 0; k < CL; ++k) nb[k] = P[i + 1][k];
            } else {
#pragma unroll
                for (int k = 0; k < CL; k += 2) {
                    const float4 d4 = ds[(k / 2) * 32 + lane];
                    nb[k] = make_float2(d4.x, d4.y);
                    nb[k + 1] = make_float2(d4.z, d4.w);
                }
            }
            const float4 rn = rowc[r0 + i + 1];
            const float2 er = make_float2(rc.x, rc.y), jup = make_float2(rc.z, rc.w), jdn = make_float2(rn.z, rn.w);
            rc = rn;
            const int X1w = x_row[r0 + i];
            float2 y[CL];
#pragma unroll
            for (int k = 0; k < CL; ++k) {
                const float2 l = (k == 0) ? lft : c[k - 1];
                const float2 rr = (k == CL - 1) ? rgt : c[k + 1];
                float2 t = __fmul2_rn(ec[k], c[k]);
                t = __ffma2_rn(er, c[k], t);
                t = __ffma2_rn(jup, prev[k], t);
                t = __ffma2_rn(jdn, nb[k], t);
                t = __ffma2_rn(nJc[k], l, t);
                t = __ffma2_rn(nJc[k + 1], rr, t);
                if (X1w == X2[k]) t = __ffma2_rn(dU, c[k], t);   // dt U on x1 = x2
                y[k] = t;
            }
#pragma unroll
            for (int k = 0; k < CL; ++k) prev[k] = c[k];
            const int ri = r0 + i;
#pragma unroll
            for (int k = 0; k < CL; k += 2) {
                const float4 q = Q[ri * (RC / 2) + (k / 2) * 32 + lane];
                if (!last_final) {
                    P[i][k] = make_float2(fmaf(inv_j, y[k].y, q.x), fmaf(-inv_j, y[k].x, q.y));
                    P[i][k + 1] = make_float2(fmaf(inv_j, y[k + 1].y, q.z), fmaf(-inv_j, y[k + 1].x, q.w));
                } else if (ri >= D && ri < D + T1 && x1_0 + ri < N) {
                    // psi(t+dt) = psi + (-i) y on the tile, rounding error carried in lo
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int ck = CL * lane + k + h2;
                        if (ck < D || ck >= D + T2 || x2_0 + ck >= N) continue;
                        const int64_t g = base + (int64_t)X1w * N + X2[k + h2];
                        const float2 yk = y[k + h2];
                        float2 hv = h2 ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
                        const float2 inc = make_float2(yk.y, -yk.x);
                        if (a.compensated) {
                            float2 l = a.lo[g];
                            compensated_add(hv.x, l.x, inc.x);
                            compensated_add(hv.y, l.y, inc.y);
                            a.lo[g] = l;
                        } else {
                            hv.x += inc.x;
                            hv.y += inc.y;
                        }
                        a.w_out[g] = hv;
                    }
                }
            }
        }
    }
    if (!a.final) {
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            const int ri = r0 + i;
            if (ri < D || ri >= D + T1 || x1_0 + ri >= N) continue;
            const int64_t grow = base + (int64_t)x_row[ri] * N;
#pragma unroll
            for (int k = 0; k < CL; ++k) {
                const int ck = CL * lane + k;
                if (ck >= D && ck < D + T2 && x2_0 + ck < N) a.w_out[grow + X2[k]] = P[i][k];
            }
        }
    }
}

using TiledKernel = void (*)(TiledArgs);

struct TiledShape {
    int TMAX, D;
    TiledKernel kern;
    size_t smem;
    bool fixed_tile;   // the register kernels: tile TMAX (rows) x TMAX2 (columns) exactly
    int TMAX2;
    int threads = 256;
};

template <int TMAX, int D>
TiledShape tiled_shape() {
    constexpr int RS = TMAX + 2 * D;
    TiledShape s;
    s.TMAX = TMAX;
    s.D = D;
    s.kern = taylor_tiled_kernel<TMAX, D>;
    s.smem = sizeof(float2) * 3 * (size_t)RS * RS + sizeof(float) * (4 * (size_t)RS + 2) +
             sizeof(int) * 2 * (size_t)RS;
    s.fixed_tile = false;
    s.TMAX2 = TMAX;
    return s;
}

template <int D, int W = 8>
TiledShape tiled_reg_shape() {
    constexpr int RS = 8 * W;
    TiledShape s;
    s.TMAX = RS - 2 * D;
    s.TMAX2 = 64 - 2 * D;
    s.D = D;
    s.kern = taylor_tiled_reg_kernel<D, W>;
    s.smem = sizeof(float4) * (RS * 32 + 2 * W * 2 * 32 + 32 + RS + 1) + sizeof(int) * RS;
    s.fixed_tile = true;
    s.threads = 32 * W;
    return s;
}

template <int D, int CL>
TiledShape tiled_wide_shape() {
    constexpr int RC = 32 * CL;
    TiledShape s;
    s.TMAX = 64 - 2 * D;
    s.TMAX2 = RC - 2 * D;
    s.D = D;
    s.kern = taylor_tiled_wide_kernel<D, CL>;
    s.smem = sizeof(float4) * (64 * (RC / 2) + 2 * 8 * 2 * (RC / 2) + RC / 2 + 65) + sizeof(int) * 64;
    s.fixed_tile = true;
    return s;
}

// regions of at most 64 x 64 (two 32-lane column passes per row); shapes
// 3..10: the iterate in registers at depths 4, 8, 2, 7, 6, 5, 3 and 1;
// 11, 12: registers on 64 x 128 regions at depths 8 and 4; 13, 14:
// registers on 96 x 64 regions (12 warps) at depths 8 and 7
constexpr int kTiledShapes = 15;

bool tiled_shape_for(int idx, TiledShape &s) {
    switch (idx) {
        case 0: s = tiled_shape<56, 4>(); return true;
        case 1: s = tiled_shape<60, 2>(); return true;
        case 2: s = tiled_shape<48, 8>(); return true;
        case 3: s = tiled_reg_shape<4>(); return true;
        case 4: s = tiled_reg_shape<8>(); return true;
        case 5: s = tiled_reg_shape<2>(); return true;
        case 6: s = tiled_reg_shape<7>(); return true;
        case 7: s = tiled_reg_shape<6>(); return true;
        case 8: s = tiled_reg_shape<5>(); return true;
        case 9: s = tiled_reg_shape<3>(); return true;
        case 10: s = tiled_reg_shape<1>(); return true;
        case 11: s = tiled_wide_shape<8, 4>(); return true;
        case 12: s = tiled_wide_shape<4, 4>(); return true;
        case 13: s = tiled_reg_shape<8, 12>(); return true;
        case 14: s = tiled_reg_shape<7, 12>(); return true;
        default: return false;
    }
}

}  // namespace

int tiled_shape_count() { return kTiledShapes; }

bool tiled_supported(const ctqw_hamiltonian *h, int dtype, int shape) {
    TiledShape s;
    return dtype == CTQW_C64 && h->m == 2 && tiled_shape_for(shape, s);
}

int tiled_depth(int shape) {
    TiledShape s;
    return tiled_shape_for(shape, s) ? s.D : 0;
}

int tiled_default_shape(int K) {
    // the fewest launches a step at depth <= 8, with the stages split evenly
    // between them (a larger tile for the same launch count)
    const int launches = (K + 7) / 8;
    const int D = (K + launches - 1) / launches;
    static const int by_depth[9] = {4, 10, 5, 9, 3, 8, 7, 6, 4};
    return by_depth[D < 1 ? 1 : (D > 8 ? 8 : D)];
}

int launch_taylor_tiled_range(const ctqw_hamiltonian *h, int shape, const void *w_in, const void *psi,
                              void *w_out, void *lo, double dt, int j0, int n_stages, int final,
                              int compensated, int r0, int R_run, cudaStream_t s) {
    const bool whole = r0 == 0 && R_run == h->R;
    if (!whole && (h->group_N.size() != 1 || r0 < 0 || R_run < 0 || r0 + R_run > h->R)) {
        ctqw_set_error("tiled path: realizations %d..%d of %d (a range needs one size group)", r0,
                       r0 + R_run, h->R);
        return CTQW_EINVAL;
    }
    if (R_run == 0) return CTQW_OK;
    TiledShape f;
    if (!tiled_shape_for(shape, f)) {
        ctqw_set_error("tiled path: unknown shape %d", shape);
        return CTQW_EUNSUPPORTED;
    }
    if (n_stages < 1 || n_stages > f.D || (final && j0 != n_stages)) {
        ctqw_set_error("tiled path: %d stages from j0=%d with depth %d", n_stages, j0, f.D);
        return CTQW_EINVAL;
    }
    TiledArgs a;
    a.tab = real_table(h);
    a.eps = h->eps32;
    a.J = h->J32;
    a.w_in = (const float2 *)w_in;
    a.psi = (const float2 *)psi;
    a.w_out = (float2 *)w_out;
    a.lo = (float2 *)lo;
    a.dt = (float)dt;
    a.dtU = (float)(dt * h->U);
    a.j0 = j0;
    a.n_stages = n_stages;
    a.final = final;
    a.compensated = compensated;
    CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)f.kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)f.smem));
    const int G = (int)h->group_N.size();
    a.flat.n = 0;
    if (f.fixed_tile && G > 1 && G <= kMaxFlatGroups) {
        // one launch over every group, largest N first (see FlatGroups)
        a.flat.n = G;
        a.list = h->by_group_d;
        int64_t items = 0;
        for (int k = 0; k < G; ++k) {
            const int g = G - 1 - k;   // groups are stored in ascending N
            int off = 0;
            for (int q = 0; q < g; ++q) off += h->group_count[q];
            const int N = h->group_N[g];
            a.flat.item_off[k] = items;
            a.flat.list_off[k] = off;
            a.flat.tiles_y[k] = (N + f.TMAX - 1) / f.TMAX;
            a.flat.tiles_x[k] = (N + f.TMAX2 - 1) / f.TMAX2;
            items += (int64_t)h->group_count[g] * a.flat.tiles_y[k] * a.flat.tiles_x[k];
        }
        a.flat.item_off[G] = items;
        a.T = f.TMAX;
        if (items > 0x7fffffffLL) {
            ctqw_set_error("tiled path: %lld tiles in one launch", (long long)items);
            return CTQW_EUNSUPPORTED;
        }
        f.kern<<<(unsigned)items, f.threads, f.smem, s>>>(a);
        CTQW_CUDA_TRY(cudaGetLastError());
        return CTQW_OK;
    }
    // one size group: a range is a slice of its (ascending) realization list
    int off = whole ? 0 : r0;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g], cnt = whole ? h->group_count[g] : R_run;
        // as few tiles per side as the compiled maximum allows, of equal size
        const int tiles = (N + f.TMAX - 1) / f.TMAX;             // along x1 (and x2 if square)
        const int tiles2 = (N + f.TMAX2 - 1) / f.TMAX2;          // along x2
        a.T = f.fixed_tile ? f.TMAX : (N + tiles - 1) / tiles;
        a.list = h->by_group_d + off;
        f.kern<<<dim3((unsigned)tiles2, (unsigned)tiles, (unsigned)cnt), f.threads, f.smem, s>>>(a);
        CTQW_CUDA_TRY(cudaGetLastError());
        off += cnt;
    }
    return CTQW_OK;
}

int launch_taylor_tiled(const ctqw_hamiltonian *h, int shape, const void *w_in, const void *psi,
                        void *w_out, void *lo, double dt, int j0, int n_stages, int final,
                        int compensated, cudaStream_t s) {
    return launch_taylor_tiled_range(h, shape, w_in, psi, w_out, lo, dt, j0, n_stages, final, compensated, 0,
                                     h->R, s);
}
