// Fused, cluster-resident Taylor propagation for two particles in complex FP32,
// full-row layout.
//
// One thread-block cluster owns one realization at a time for all steps of
// the launch (the order-K Taylor polynomial of Algorithm 3, Sec. 2.3, applied
// n_steps times).  The grid holds only as many clusters as are resident at
// once, and each takes realization after realization from a ticket counter,
// so the SMs a cluster holds stay its own until the launch ends.
// The N x N tile is split into row slabs, one per CTA; every warp owns RL
// whole rows and each lane CL = N/32 adjacent columns of them, so a warp
// covers full rows: neighbours along x2 are in the lane's registers or one
// 64-bit rotate-shuffle away (the rotation wraps from column N-1 to 0, which
// is the ring's bond and is multiplied by J[N-1] = 0 on an open chain).
// Neighbours along x1 are in registers except for the warp's first and last
// rows, which come from the adjacent warps through shared memory (one
// __syncthreads per stage) or, at the slab's edges, are pushed by the
// neighbour CTAs straight into this CTA's shared memory with st.async on an
// mbarrier (bounded waits).
//
// Arithmetic: the same polynomial in Horner form with A = -i dt H applied to
// (re, im) pairs with FFMA2:
//   w_K = psi + (A/K) psi,  w_j = psi + (A/j) w_{j+1},  psi(t+dt) = psi + A w_2,
// (forward FP32 summation would drop every term below half an ulp of the
// running sum).  The diagonal dt*(eps_x1 + eps_x2) enters as two FFMA2 with
// a per-row and a per-column pair; dt*U on x1 = x2 is added for the one lane
// of a row that owns the diagonal.  The increment A w_2 is added to the state
// with its rounding error carried in a second FP32 word (lo), so hi + lo
// holds the state to ~2^-48 relative.  lo sits in shared memory for the
// launch (lane-major like hi) and in a state-sized buffer between launches.
//
// Control flow: the diagonal offset of a warp's rows is fixed for the
// kernel, and the Horner stages of a step are K - 1 middle stages and one
// final one, so the step loop is compiled per offset with the stage mode a
// compile-time constant: no per-stage dispatch.
//
// Observables are not formed here.  At every snap_every-th step inside the
// launch the kernel stores the state to a snapshot slot (row-major, the
// layout of psi), and the host reduces the snapshots in FP64 with the
// observables kernel; a launch covers the steps between a sample and the
// sample after its last snapshot.  Keeping that work out of the kernel
// leaves the registers of the Horner loop to the stencil.
//
// Row layout in shared memory (and of the carried error in global memory):
// lane-major, the k-th column pair of lane l at float4 slot (k/2)*32 + l of
// the row, so that every 16-byte access of a warp touches 32 consecutive
// slots (a plain row-major layout puts lanes CL*8 bytes apart, a 4-way bank
// conflict for CL = 8).  Every reader uses the writer's lane mapping.
#include <algorithm>
#include <type_traits>

#include "ctqw_internal.cuh"
#include "fused_common.cuh"

namespace {

using namespace fused;

constexpr int kMaxK = 30;

struct RowsArgs {
    const double *eps;
    const double *J;
    RealTable tab;
    float2 *psi;            // state in (start of the launch) and out (end)
    float2 *lo;             // carried rounding error (lane-major rows), in and out
    float2 *snap;           // snapshot slots (states), or null
    double dt;
    float dtU;
    int K;
    long long n_steps;      // steps of this launch
    int snap_every;         // snapshot after every snap_every-th step (< n_steps), 0: none
    long long snap_stride;  // amplitudes per snapshot slot
    int compensated;
    int *status;
    unsigned long long wait_limit_ns;
    int test_timeout;
    int r0, R_run;          // realizations r0 .. r0 + R_run - 1, handed out one at a time
    int *work;              // ticket counter of the hand-out, zero at the launch
    float inv_j[kMaxK + 1];
};

enum { kHorner = 0, kFinal = 1 };

// Register state of one lane: RL rows x CL columns of the Horner iterate and
// the per-column coefficient pairs (c, c) of dt H.  The per-row pairs are the
// same for the whole warp and are read from shared memory (rowc) instead.
template <int CL, int RL>
struct Lane {
    float2 P[RL][CL];
    float2 ec[CL];        // dt eps_x2 per column
    float2 nJc[CL + 1];   // -dt J of the bond left of column k (k = CL: right of the last)
};

// One stencil application y = (dt H) P on the lane's block, then
//   kHorner: P <- Q + (-i/j) y;  kFinal: P <- -i y.
// usrc/dsrc: the rows above the first and below the last row in shared memory
// (this lane's first column), read when needed so they do not hold registers.
// Q: psi of the step in shared memory (this lane's first element, row stride N).
// OFF = (first row) mod CL, which fixes where the diagonal x1 = x2 falls.
// rowc: per slab row (dt eps_x1, dt eps_x1, -dt J above, -dt J above) for this
// warp's rows and the one below them (broadcast loads).
template <int MODE, int CL, int RL, int N, int OFF>
__device__ __forceinline__ void stage(Lane<CL, RL> &L, const float4 *__restrict__ rowc,
                                      const float2 *__restrict__ usrc,
                                      const float2 *__restrict__ dsrc, const float2 *__restrict__ Q,
                                      int lane, int x1_0, float dtU, float inv_j) {
    const int from_left = (lane + 31) & 31, from_right = (lane + 1) & 31;
    const float2 dU = make_float2(dtU, dtU);
    float4 rc = rowc[0];
    float2 prev[CL];   // old row above the current one
#pragma unroll
    for (int k = 0; k < CL; k += 2) {
        const float4 u4 = *reinterpret_cast<const float4 *>(usrc + k * 32);
        prev[k] = make_float2(u4.x, u4.y);
        prev[k + 1] = make_float2(u4.z, u4.w);
    }
#pragma unroll
    for (int i = 0; i < RL; ++i) {
        float2 c[CL];
#pragma unroll
        for (int k = 0; k < CL; ++k) c[k] = L.P[i][k];
        const float2 lft = shfl2(c[CL - 1], from_left);
        const float2 rgt = shfl2(c[0], from_right);
        float2 dn[CL];   // old row below (read from shared memory for the last row)
        if (i == RL - 1) {
#pragma unroll
            for (int k = 0; k < CL; k += 2) {
                const float4 d4 = *reinterpret_cast<const float4 *>(dsrc + k * 32);
                dn[k] = make_float2(d4.x, d4.y);
                dn[k + 1] = make_float2(d4.z, d4.w);
            }
        }
        const float4 rn = rowc[i + 1];
        const float2 er = make_float2(rc.x, rc.y), jup = make_float2(rc.z, rc.w);
        const float2 jdn = make_float2(rn.z, rn.w);
        rc = rn;
        float2 y[CL];
#pragma unroll
        for (int k = 0; k < CL; ++k) {
            const float2 nb = (i < RL - 1) ? L.P[i + 1][k] : dn[k];   // old row below
            const float2 l = (k == 0) ? lft : c[k - 1];
            const float2 r = (k == CL - 1) ? rgt : c[k + 1];
            float2 t = __fmul2_rn(L.ec[k], c[k]);
            t = __ffma2_rn(er, c[k], t);
            t = __ffma2_rn(jup, prev[k], t);
            t = __ffma2_rn(jdn, nb, t);
            t = __ffma2_rn(L.nJc[k], l, t);
            t = __ffma2_rn(L.nJc[k + 1], r, t);
            y[k] = t;
        }
        // dt U on the diagonal x2 = x1: column (OFF + i) % CL of the lane (x1_0 + i) / CL
        {
            const int kd = (OFF + i) % CL;   // a constant once the row loop is unrolled
            if (lane == (x1_0 + i) / CL) y[kd] = __ffma2_rn(dU, c[kd], y[kd]);
        }
        if (MODE == kHorner) {
#pragma unroll
            for (int k = 0; k < CL; k += 2) {
                const float4 q = *reinterpret_cast<const float4 *>(Q + i * N + k * 32);
                L.P[i][k] = make_float2(fmaf(inv_j, y[k].y, q.x), fmaf(-inv_j, y[k].x, q.y));
                L.P[i][k + 1] = make_float2(fmaf(inv_j, y[k + 1].y, q.z), fmaf(-inv_j, y[k + 1].x, q.w));
            }
        } else if (MODE == kFinal) {
#pragma unroll
            for (int k = 0; k < CL; ++k) L.P[i][k] = make_float2(y[k].y, -y[k].x);
        }
#pragma unroll
        for (int k = 0; k < CL; ++k) prev[k] = c[k];
    }
}

// CL columns per lane (N = 32 CL), RL rows per warp, W warps per CTA.
template <int CL, int RL, int W, int MINB>
__global__ void __launch_bounds__(32 * W, MINB) taylor_fused_rows_kernel(const __grid_constant__ RowsArgs a) {
    constexpr int N = 32 * CL;
    constexpr int SR = RL * W;     // slab rows
    constexpr int C = N / SR;      // CTAs per cluster
    static_assert(N % SR == 0 && C >= 1 && C <= 16 && CL % 2 == 0, "unsupported shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *hi = reinterpret_cast<float2 *>(smem_raw);      // [SR][N] psi of the step
    float2 *halo = hi + SR * N;                             // [2 parity][2: above, below][N]
    float2 *edge = halo + 2 * 2 * N;                        // [2 parity][W][2: first, last][N]
    float4 *rowc = reinterpret_cast<float4 *>(edge + 2 * W * 2 * N);  // [SR + 1] row coefficient pairs
    float2 *los = reinterpret_cast<float2 *>(rowc + SR + 1);          // [SR][N] carried error, lane-major
    __shared__ __align__(8) unsigned long long mbar[2][2];
    __shared__ __align__(8) unsigned long long mbar_never;
    __shared__ int next_r;

    const int rank = (int)cluster_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lrow0 = warp * RL;
    const int x1_0 = rank * SR + lrow0;
    const int x2_0 = lane * CL;

    Lane<CL, RL> L;
    // coefficients and state of realization r (every warp reads rowc, so the
    // caller orders this behind the previous realization's last stage)
    auto load_realization = [&](const int r) {
        const int64_t po = a.tab.par_off[r];
        const double *eps = a.eps + po, *J = a.J + po;
        const double dt = a.dt;
        for (int q = threadIdx.x; q <= SR; q += blockDim.x) {
            const int x1 = rank * SR + q;   // q = SR: only the bond below the slab is used
            const float e = q < SR ? (float)(dt * eps[x1]) : 0.f;
            const float j = (float)(-dt * J[(x1 - 1 + N) % N]);
            rowc[q] = make_float4(e, e, j, j);
        }
#pragma unroll
        for (int k = 0; k < CL; ++k) {
            const float v = (float)(dt * eps[x2_0 + k]);
            L.ec[k] = make_float2(v, v);
        }
#pragma unroll
        for (int k = 0; k <= CL; ++k) {
            const float v = (float)(-dt * J[(x2_0 + k - 1 + N) % N]);
            L.nJc[k] = make_float2(v, v);
        }
        // state in: hi = psi (shared), P = psi (registers), lo (shared, lane-major like hi)
        const float2 *glo = a.lo + a.tab.st_off[r];
#pragma unroll
        for (int i = 0; i < RL; ++i) {
#pragma unroll
            for (int k = 0; k < CL; k += 2)
                *reinterpret_cast<float4 *>(los + (lrow0 + i) * N + lane * 2 + k * 32) =
                    *reinterpret_cast<const float4 *>(glo + (size_t)(x1_0 + i) * N + lane * 2 + k * 32);
        }
#pragma unroll
        for (int i = 0; i < RL; ++i) {
#pragma unroll
            for (int k = 0; k < CL; k += 2) {
                const float4 v = *reinterpret_cast<const float4 *>(a.psi + a.tab.st_off[r] + (size_t)(x1_0 + i) * N + x2_0 + k);
                L.P[i][k] = make_float2(v.x, v.y);
                L.P[i][k + 1] = make_float2(v.z, v.w);
                *reinterpret_cast<float4 *>(hi + (lrow0 + i) * N + lane * 2 + k * 32) = v;
            }
        }
    };
    // state out (hi, and the carried error for the next launch); each thread
    // reads back only the shared words it wrote
    auto store_realization = [&](const int r) {
        float2 *glo = a.lo + a.tab.st_off[r];
#pragma unroll
        for (int i = 0; i < RL; ++i) {
#pragma unroll
            for (int k = 0; k < CL; k += 2)
                *reinterpret_cast<float4 *>(glo + (size_t)(x1_0 + i) * N + lane * 2 + k * 32) =
                    *reinterpret_cast<const float4 *>(los + (lrow0 + i) * N + lane * 2 + k * 32);
        }
#pragma unroll
        for (int i = 0; i < RL; ++i) {
#pragma unroll
            for (int k = 0; k < CL; k += 2)
                *reinterpret_cast<float4 *>(a.psi + a.tab.st_off[r] + (size_t)(x1_0 + i) * N + x2_0 + k) =
                    *reinterpret_cast<const float4 *>(hi + (lrow0 + i) * N + lane * 2 + k * 32);
        }
    };

    const int rank_up = (rank + C - 1) % C, rank_dn = (rank + 1) % C;
    const uint32_t send_up = map_rank(smem_u32(halo + N + lane * 2), rank_up);    // their "row below" slot
    const uint32_t send_up_mb = map_rank(smem_u32(&mbar[0][1]), rank_up);
    const uint32_t send_dn = map_rank(smem_u32(halo + lane * 2), rank_dn);        // their "row above" slot
    const uint32_t send_dn_mb = map_rank(smem_u32(&mbar[0][0]), rank_dn);
    bool dead = false;
    const float2 *Q = hi + lrow0 * N + lane * 2;
    const int off = x1_0 % CL;

    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q)
            for (int sd = 0; sd < 2; ++sd) mbar_init(smem_u32(&mbar[q][sd]), 1);
        mbar_init(smem_u32(&mbar_never), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_barrier();
    if (a.test_timeout && threadIdx.x == 0 && blockIdx.x == 0)
        (void)mbar_wait_bounded(smem_u32(&mbar_never), 0, 1000000ull, a.status);

    const long long n_steps = a.n_steps;
    const int K = a.K;
    // the next realization of this cluster: CTA 0 takes a ticket, the others
    // read it from CTA 0's shared memory between two cluster barriers
    auto grab = [&]() -> int {
        if (rank == 0 && threadIdx.x == 0) next_r = a.r0 + atomicAdd(a.work, 1);
        cluster_barrier();
        const int r = ld_shared_cluster_s32(map_rank(smem_u32(&next_r), 0));
        cluster_barrier();
        return r;
    };
    // the whole step loop, for this warp's (constant) diagonal offset
    auto main_loop = [&](auto off_tag) {
        constexpr int OFF = decltype(off_tag)::value;
        // the stage counter runs on across realizations: the halo slots and
        // their mbarrier phases continue without a reset, and a neighbour can
        // never be more than one stage ahead
        unsigned tc = 0;
        // realizations are handed out one at a time, so a cluster that runs
        // faster takes more of them
        for (int r = grab(); r < a.r0 + a.R_run; r = grab()) {
            __syncthreads();
            load_realization(r);
            for (long long step = 0; step < n_steps; ++step) {
                auto run_stage = [&](const int j, auto mode_tag) {
                    constexpr int MODE = decltype(mode_tag)::value;
                    const int parity = tc & 1;
                    const uint32_t phase = (tc >> 1) & 1;
                    // publish: this warp's first and last rows (shared memory; the slab
                    // edge rows also into the neighbour CTAs)
                    float2 *eb = edge + parity * (W * 2 * N) + warp * (2 * N) + lane * 2;
    #pragma unroll
                    for (int k = 0; k < CL; k += 2) {
                        const float4 t = make_float4(L.P[0][k].x, L.P[0][k].y, L.P[0][k + 1].x, L.P[0][k + 1].y);
                        const float4 b = make_float4(L.P[RL - 1][k].x, L.P[RL - 1][k].y, L.P[RL - 1][k + 1].x,
                                                     L.P[RL - 1][k + 1].y);
                        *reinterpret_cast<float4 *>(eb + k * 32) = t;
                        *reinterpret_cast<float4 *>(eb + N + k * 32) = b;
                        if (warp == 0) st_async16(send_up + parity * (2 * N * 8) + k * 256, t, send_up_mb + parity * 16);
                        if (warp == W - 1) st_async16(send_dn + parity * (2 * N * 8) + k * 256, b, send_dn_mb + parity * 16);
                    }
                    __syncthreads();
                    mbar_expect_tx2_if(smem_u32(&mbar[parity][0]), smem_u32(&mbar[parity][1]), N * 8,
                                       threadIdx.x == 0);
                    // the rows above and below this warp's block
                    const float2 *usrc, *dsrc;
                    if (warp > 0) {
                        usrc = edge + parity * (W * 2 * N) + (warp - 1) * (2 * N) + N + lane * 2;
                    } else {
                        if (!dead) dead = !mbar_wait_bounded(smem_u32(&mbar[parity][0]), phase, a.wait_limit_ns, a.status);
                        usrc = halo + parity * (2 * N) + lane * 2;
                    }
                    if (warp < W - 1) {
                        dsrc = edge + parity * (W * 2 * N) + (warp + 1) * (2 * N) + lane * 2;
                    } else {
                        if (!dead) dead = !mbar_wait_bounded(smem_u32(&mbar[parity][1]), phase, a.wait_limit_ns, a.status);
                        dsrc = halo + parity * (2 * N) + N + lane * 2;
                    }
                    stage<MODE, CL, RL, N, OFF>(L, rowc + lrow0, usrc, dsrc, Q, lane, x1_0, a.dtU, a.inv_j[j]);
                    ++tc;
                };
                for (int j = K; j >= 2; --j) run_stage(j, std::integral_constant<int, kHorner>());
                run_stage(1, std::integral_constant<int, kFinal>());
                // psi(t+dt) = psi + A w_2 (in P); rounding error carried in lo
        #pragma unroll
                for (int i = 0; i < RL; ++i) {
        #pragma unroll
                    for (int k = 0; k < CL; k += 2) {
                        float4 *hp = reinterpret_cast<float4 *>(hi + (lrow0 + i) * N + lane * 2 + k * 32);
                        float4 *lp = reinterpret_cast<float4 *>(los + (lrow0 + i) * N + lane * 2 + k * 32);
                        float4 h4 = *hp;
                        if (a.compensated) {
                            float4 l4 = *lp;
                            float2 h0 = make_float2(h4.x, h4.y), h1 = make_float2(h4.z, h4.w);
                            float2 l0 = make_float2(l4.x, l4.y), l1 = make_float2(l4.z, l4.w);
                            compensated_add2(h0, l0, L.P[i][k]);
                            compensated_add2(h1, l1, L.P[i][k + 1]);
                            h4 = make_float4(h0.x, h0.y, h1.x, h1.y);
                            *lp = make_float4(l0.x, l0.y, l1.x, l1.y);
                        } else {
                            h4.x += L.P[i][k].x;
                            h4.y += L.P[i][k].y;
                            h4.z += L.P[i][k + 1].x;
                            h4.w += L.P[i][k + 1].y;
                        }
                        *hp = h4;
                        L.P[i][k] = make_float2(h4.x, h4.y);
                        L.P[i][k + 1] = make_float2(h4.z, h4.w);
                    }
                }
                // a snapshot step: the new state (P) to its slot, row-major like psi
                if (a.snap_every > 0 && step + 1 < n_steps && (step + 1) % a.snap_every == 0) {
                    float2 *gs = a.snap + ((step + 1) / a.snap_every - 1) * a.snap_stride + a.tab.st_off[r];
        #pragma unroll
                    for (int i = 0; i < RL; ++i) {
        #pragma unroll
                        for (int k = 0; k < CL; k += 2)
                            *reinterpret_cast<float4 *>(gs + (size_t)(x1_0 + i) * N + x2_0 + k) =
                                make_float4(L.P[i][k].x, L.P[i][k].y, L.P[i][k + 1].x, L.P[i][k + 1].y);
                    }
                }
            }
            store_realization(r);
        }
    };
    // the first row's offset modulo CL: a multiple of gcd(RL, CL); only those are compiled
    constexpr int GD = RL % CL == 0 ? CL : (CL % RL == 0 ? RL : (RL % 2 == 0 && CL % 2 == 0 ? 2 : 1));
    static_assert(CL == 2 || CL == 4 || CL == 6 || CL == 8, "diagonal offsets enumerated for CL <= 8");
    switch (off) {
        case 0: main_loop(std::integral_constant<int, 0>()); break;
        case 2: if constexpr (CL > 2 && 2 % GD == 0) main_loop(std::integral_constant<int, 2 % CL>()); break;
        case 4: if constexpr (CL > 4 && 4 % GD == 0) main_loop(std::integral_constant<int, 4 % CL>()); break;
        case 6: if constexpr (CL > 6 && 6 % GD == 0) main_loop(std::integral_constant<int, 6 % CL>()); break;
        default: break;
    }
    cluster_barrier();   // no CTA leaves while a neighbour may still push into it
}

using RowsKernel = void (*)(RowsArgs);

struct RowsShape {
    int C, threads;
    size_t smem;
    RowsKernel kern;
};

template <int CL, int RL, int W, int MINB>
RowsShape rows_shape() {
    constexpr int N = 32 * CL, SR = RL * W;
    RowsShape f;
    f.C = N / SR;
    f.threads = 32 * W;
    f.smem = sizeof(float2) * ((size_t)SR * N + (size_t)2 * 2 * N + (size_t)2 * W * 2 * N) +
             sizeof(float4) * (size_t)(SR + 1) + sizeof(float2) * (size_t)SR * N;
    f.kern = taylor_fused_rows_kernel<CL, RL, W, MINB>;
    return f;
}

constexpr int kRowsShapes = 3;

bool rows_shape_for(int N, int idx, RowsShape &f) {
    RowsShape opts[kRowsShapes];
    switch (N) {
        case 64: opts[0] = rows_shape<2, 8, 8, 2>(); opts[1] = rows_shape<2, 4, 8, 2>(); opts[2] = rows_shape<2, 8, 4, 3>(); break;
        case 128: opts[0] = rows_shape<4, 8, 4, 2>(); opts[1] = rows_shape<4, 4, 8, 2>(); opts[2] = rows_shape<4, 4, 4, 3>(); break;
        case 192: opts[0] = rows_shape<6, 4, 8, 1>(); opts[1] = rows_shape<6, 4, 4, 3>(); opts[2] = rows_shape<6, 4, 4, 2>(); break;
        case 256: opts[0] = rows_shape<8, 4, 4, 2>(); opts[1] = rows_shape<8, 4, 8, 1>(); opts[2] = rows_shape<8, 4, 4, 3>(); break;
        default: return false;
    }
    if (idx < 0 || idx >= kRowsShapes) return false;
    f = opts[idx];
    return true;
}

}  // namespace

bool fused_rows_supported(const ctqw_hamiltonian *h, int dtype) {
    RowsShape f;
    return dtype == CTQW_C64 && h->m == 2 && h->uniform && rows_shape_for(h->Nmax, 0, f);
}

namespace {

int set_rows_attributes(const RowsShape &f) {
    CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)f.kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)f.smem));
    if (f.C > 8)
        CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)f.kern,
                                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return CTQW_OK;
}

int rows_clusters(const RowsShape &f, int *clusters) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)f.C);
    cfg.blockDim = dim3((unsigned)f.threads);
    cfg.dynamicSmemBytes = f.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)f.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CTQW_CUDA_TRY(cudaOccupancyMaxActiveClusters(clusters, (const void *)f.kern, &cfg));
    return CTQW_OK;
}

}  // namespace

// Tiled-to-fused throughput ratio per SM, measured on two bosons at N = 256,
// K = 16 (register tiles at depth 8 against the full-row clusters).
static constexpr double kTiledPerSmRatio = 0.25;

int fused_rows_split(const ctqw_hamiltonian *h, int shape, int K, int *R_tiled) {
    *R_tiled = 0;
    RowsShape f;
    if (!fused_rows_supported(h, CTQW_C64) || !rows_shape_for(h->Nmax, shape, f) ||
        !tiled_supported(h, CTQW_C64, tiled_default_shape(K)) || h->group_N.size() != 1)
        return CTQW_OK;
    CTQW_TRY(set_rows_attributes(f));
    int clusters = 0, per_sm = 0, n_sm = 0;
    CTQW_TRY(rows_clusters(f, &clusters));
    CTQW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)f.kern, f.threads, f.smem));
    CTQW_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device));
    if (clusters < 1 || per_sm < 1) return CTQW_OK;
    const int used = std::min(n_sm, (clusters * f.C + per_sm - 1) / per_sm);
    const int idle = n_sm - used;
    if (idle * 16 < n_sm) return CTQW_OK;   // under 1/16 of the SMs idle: not worth a second stream
    // both parts end together when each one's share of the realizations
    // matches its share of the throughput; the fused part gets whole rounds
    const double share = used / (used + kTiledPerSmRatio * idle);
    const int rounds = std::max(1, (int)std::lround(h->R * share / clusters));
    const int R_f = std::min(h->R, rounds * clusters);
    *R_tiled = h->R - R_f;
    return CTQW_OK;
}

int launch_taylor_fused_rows(const ctqw_hamiltonian *h, void *psi, void *lo, void *snap,
                             int snap_every, double dt, int K, int64_t n_steps, int compensated,
                             int shape, int test_timeout, int r0, int R_run, cudaStream_t s) {
    RowsShape f;
    if (!rows_shape_for(h->Nmax, shape, f)) {
        ctqw_set_error("fused path: unsupported size N=%d or shape %d", h->Nmax, shape);
        return CTQW_EUNSUPPORTED;
    }
    if (K > kMaxK) {
        ctqw_set_error("fused path: K=%d above %d", K, kMaxK);
        return CTQW_EUNSUPPORTED;
    }
    if (r0 < 0 || R_run < 0 || r0 + R_run > h->R) {
        ctqw_set_error("fused path: realizations %d..%d outside 0..%d", r0, r0 + R_run, h->R);
        return CTQW_EINVAL;
    }
    if (R_run == 0) return CTQW_OK;
    RowsArgs a;
    a.eps = h->eps64;
    a.J = h->J64;
    a.tab = real_table(h);
    a.psi = (float2 *)psi;
    a.lo = (float2 *)lo;
    a.snap = (float2 *)snap;
    a.snap_every = snap ? snap_every : 0;
    a.snap_stride = h->total_amp;
    a.dt = dt;
    a.dtU = (float)(dt * h->U);
    a.K = K;
    a.n_steps = n_steps;
    a.compensated = compensated;
    a.status = h->status_d;
    a.test_timeout = test_timeout;
    a.wait_limit_ns = 2000000000ull;
    a.r0 = r0;
    a.R_run = R_run;
    a.work = work_counter(h);
    a.inv_j[0] = 0.f;
    for (int j = 1; j <= kMaxK; ++j) a.inv_j[j] = (float)(1.0 / j);
    CTQW_TRY(set_rows_attributes(f));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)f.C);
    cfg.blockDim = dim3((unsigned)f.threads);
    cfg.dynamicSmemBytes = f.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)f.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    CTQW_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, (const void *)f.kern, &cfg));
    if (clusters < 1) {
        ctqw_set_error("fused path: no cluster of %d CTAs x %d threads fits", f.C, f.threads);
        return CTQW_EUNSUPPORTED;
    }
    // one cluster per resident slot, each taking realizations until none is left
    cfg.gridDim = dim3((unsigned)(std::min(R_run, clusters) * f.C));
    CTQW_CUDA_TRY(cudaMemsetAsync(a.work, 0, sizeof(int), s));
    CTQW_CUDA_TRY(cudaLaunchKernelEx(&cfg, f.kern, a));
    return CTQW_OK;
}
