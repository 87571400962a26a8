// Fused, cluster-resident Taylor propagation for two particles in complex FP32.
//
// Algorithm 3 (Sec. 2.3) applies the order-K polynomial of -i H dt to every
// state once per step.  Here one thread-block cluster owns one realization
// for the whole call: the N x N amplitude tile is split into row slabs, one
// per CTA, and each warp keeps an 8-row x 64-column block of the current
// Taylor term in registers.  Per term only edges move: the edge rows of the
// warp bands and the edge columns of the warps through this CTA's shared
// memory (behind one __syncthreads), and the slab's first and last rows
// straight into the neighbouring CTAs' shared memory with st.async, which
// completes on the receiver's mbarrier (point to point; no cluster-wide
// barrier or memory fence per term).  psi is read from HBM once and written
// once per call, so the K * n_steps stencil applications run at on-chip speed.
//
// Arithmetic: the same order-K polynomial as Algorithm 3, evaluated in
// Horner form with A = -i dt H (a real stencil applied to re and im alike):
//   w_K = psi + (A/K) psi,  w_j = psi + (A/j) w_{j+1}  (j = K-1 .. 2),
//   psi(t+dt) = psi + A w_2.
// Forward summation psi + sum_j A^j psi / j! in FP32 drops every term below
// half an ulp of the running sum (j >~ 7 at |A| ~ 0.2), which truncates the
// series per amplitude and biases the norm by ~x^8/7! per step; Horner keeps
// each term at its own scale.  The final increment A w_2 is added to the
// state with its rounding error carried in a second FP32 word (lo, in shared
// memory): hi + lo holds the state to ~2^-48 relative across all steps.
#include <type_traits>

#include "ctqw_internal.cuh"
#include "fused_common.cuh"

namespace {

using namespace fused;

constexpr int RL = 8;        // rows per warp band
constexpr int kMaxK = 30;

struct FusedArgs {
    const double *eps;       // exact parameter values (FP64 copies of the float32-rounded draws)
    const double *J;
    RealTable tab;
    float2 *psi;
    int N;
    double dt;
    double inv_dt;
    int K;
    long long n_steps;
    int obs_every;
    long long p_width;
    double *P_mean, *norm, *energy;
    int compensated;
    int *status;             // set to nonzero when a bounded wait gives up
    unsigned long long wait_limit_ns;
    int test_timeout;        // wait once on an mbarrier nothing completes (failure-path test)
    float inv_j[kMaxK + 1];  // 1 / j
};

// Modes of one stencil application y = (dt H) P on the warp's 8 x 64 block.
enum { kHorner = 0, kFinal = 1, kEnergyOnly = 2 };

// up/dn: the rows above and below the block; seam: the column beyond the
// block's left edge (used by lane 31) or right edge (used by lane 0).
//   kHorner:     P <- Q + (-i/j) y      (Q = psi of this step, read from shared memory)
//   kFinal:      P <- -i y              (the increment A w_2)
//   kEnergyOnly: P unchanged
// ENERGY adds sum Re(conj(P) y) (= dt <psi|H|psi> when P = psi) into e.
// V4: this warp's diagonal dt*(eps_x1 + eps_x2 + U delta) in shared memory as
// float4 per row pair and lane, (row 2k col 0, row 2k col 1, row 2k+1 col 0,
// row 2k+1 col 1), row-pair stride N/2 float4.  Coefficient pairs (c, c) are
// kept duplicated so every tap is one FFMA2 on the (re, im) pair.
// Rows are visited top-down (REV = false) or bottom-up (REV = true); both
// orders compute the same values (each new row only replaces a row whose old
// value is no longer needed).
template <int MODE, bool ENERGY, int N, bool REV>
__device__ __forceinline__ void stencil_term(float2 (&P)[RL][2], const float2 *__restrict__ Q,
                                             const float4 *__restrict__ V4,
                                             const float2 (&nJr)[RL + 1], const float2 (&nJc)[3],
                                             float2 up0, float2 up1, float2 dn0, float2 dn1,
                                             const float4 *__restrict__ seam4, int lane,
                                             float inv_j, double &e) {
    // "prev" is the old row already passed (above when top-down, below when bottom-up)
    float2 prev0 = REV ? dn0 : up0, prev1 = REV ? dn1 : up1;
    const int from_left = (lane + 31) & 31, from_right = (lane + 1) & 31;
    const bool l31 = lane == 31, l0 = lane == 0;
    float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f), s4 = v4;
#pragma unroll
    for (int ii = 0; ii < RL; ++ii) {
        const int i = REV ? RL - 1 - ii : ii;
        if ((ii & 1) == 0) {
            v4 = V4[(i >> 1) * (N / 2)];
            s4 = seam4[i >> 1];
        }
        const float2 c0 = P[i][0], c1 = P[i][1];
        // old neighbour rows: "nxt" is the one not yet visited
        const float2 nx0 = REV ? ((i > 0) ? P[i - 1][0] : up0) : ((i < RL - 1) ? P[i + 1][0] : dn0);
        const float2 nx1 = REV ? ((i > 0) ? P[i - 1][1] : up1) : ((i < RL - 1) ? P[i + 1][1] : dn1);
        const float2 a0 = REV ? nx0 : prev0, a1 = REV ? nx1 : prev1;   // row above (old)
        const float2 b0 = REV ? prev0 : nx0, b1 = REV ? prev1 : nx1;   // row below (old)
        const float2 sv = (i & 1) ? make_float2(s4.z, s4.w) : make_float2(s4.x, s4.y);
        const float vx = (i & 1) ? v4.z : v4.x, vy = (i & 1) ? v4.w : v4.y;
        const float2 lft = shfl2(l31 ? sv : c1, from_left);
        const float2 rgt = shfl2(l0 ? sv : c0, from_right);
        float2 y0 = make_float2(vx * c0.x, vx * c0.y);
        y0 = __ffma2_rn(nJr[i], a0, y0);
        y0 = __ffma2_rn(nJr[i + 1], b0, y0);
        y0 = __ffma2_rn(nJc[0], lft, y0);
        y0 = __ffma2_rn(nJc[1], c1, y0);
        float2 y1 = make_float2(vy * c1.x, vy * c1.y);
        y1 = __ffma2_rn(nJr[i], a1, y1);
        y1 = __ffma2_rn(nJr[i + 1], b1, y1);
        y1 = __ffma2_rn(nJc[1], c0, y1);
        y1 = __ffma2_rn(nJc[2], rgt, y1);
        if (ENERGY) e += (double)re_dot_f(c0, y0) + (double)re_dot_f(c1, y1);
        if (MODE == kHorner) {
            const float4 q = *reinterpret_cast<const float4 *>(Q + i * N);
            P[i][0] = make_float2(fmaf(inv_j, y0.y, q.x), fmaf(-inv_j, y0.x, q.y));
            P[i][1] = make_float2(fmaf(inv_j, y1.y, q.z), fmaf(-inv_j, y1.x, q.w));
        } else if (MODE == kFinal) {
            P[i][0] = make_float2(y0.y, -y0.x);
            P[i][1] = make_float2(y1.y, -y1.x);
        }
        prev0 = c0;
        prev1 = c1;
    }
}

// Store 8 float2 (one per row) to shared memory from the lanes where flag != 0
// only, as four predicated 16-byte stores (no branch).
__device__ __forceinline__ void st_shared_col8_if(uint32_t addr, int flag, const float2 (&v)[RL]) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %1, 0;\n\t"
                 "@p st.shared.v4.f32 [%0], {%2, %3, %4, %5};\n\t"
                 "@p st.shared.v4.f32 [%0+16], {%6, %7, %8, %9};\n\t"
                 "@p st.shared.v4.f32 [%0+32], {%10, %11, %12, %13};\n\t"
                 "@p st.shared.v4.f32 [%0+48], {%14, %15, %16, %17};\n\t}"
                 ::"r"(addr), "r"(flag), "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y),
                   "f"(v[2].x), "f"(v[2].y), "f"(v[3].x), "f"(v[3].y), "f"(v[4].x), "f"(v[4].y),
                   "f"(v[5].x), "f"(v[5].y), "f"(v[6].x), "f"(v[6].y), "f"(v[7].x), "f"(v[7].y)
                 : "memory");
}

// N sites, BPC warp bands per CTA (compile-time so that every offset is an
// immediate); WB = N/64 warps side by side per band, C = N/(8 BPC) CTAs per cluster.
template <int N, int BPC, int MINB>
__global__ void __launch_bounds__(32 * (N / 64) * BPC, MINB)
    taylor_fused_kernel(const __grid_constant__ FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int WB = N / 64;
    constexpr int SR = RL * BPC;      // slab rows of this CTA
    constexpr int C = N / SR;         // CTAs per cluster
    constexpr int W = WB * BPC;       // warps
    static_assert(N % 64 == 0 && N % SR == 0 && C <= 16, "unsupported fused shape");
    float2 *hi = reinterpret_cast<float2 *>(smem_raw);
    float2 *lo = hi + SR * N;
    float2 *halo = lo + SR * N;                  // [2 parity][2: row above, row below][N], filled by neighbours
    float2 *edge = halo + 2 * 2 * N;             // [2][BPC][2][N] band edges inside this CTA
    float2 *seamb = edge + 2 * BPC * 2 * N;      // [2][W][2][RL] warp edge columns
    float4 *Vs = reinterpret_cast<float4 *>(seamb + 2 * W * 2 * RL);   // [SR/2][N/2] diagonal of dt H
    double *pacc = reinterpret_cast<double *>(Vs + (SR / 2) * (N / 2));   // [N] FP64 partials
    __shared__ __align__(8) unsigned long long mbar[2][2];   // [parity][side] halo arrivals
    __shared__ __align__(8) unsigned long long mbar_never;    // failure-path test only

    const int rank = (int)cluster_rank();
    const int r = blockIdx.x / C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int band = warp / WB, wc = warp % WB;
    const int lrow0 = band * RL;                 // first local row of the warp band
    const int x1_0 = rank * SR + lrow0;          // its global row
    const int x2_0 = wc * 64 + 2 * lane;         // first of the lane's two columns

    // ---- coefficients of dt H (rounded once from FP64)
    const int64_t po = a.tab.par_off[r];
    const double *eps = a.eps + po;
    const double *J = a.J + po;
    const double dt = a.dt, U = a.tab.U;
    float2 nJr[RL + 1], nJc[3];   // (c, c) pairs of -dt J
    const float4 *V4 = Vs + (lrow0 / 2) * (N / 2) + x2_0 / 2;
#pragma unroll
    for (int k = 0; k < RL / 2; ++k) {
        float vv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int x1 = x1_0 + 2 * k + (q >> 1), x2 = x2_0 + (q & 1);
            vv[q] = (float)(dt * (eps[x1] + eps[x2] + (x1 == x2 ? U : 0.0)));
        }
        Vs[(lrow0 / 2 + k) * (N / 2) + x2_0 / 2] = make_float4(vv[0], vv[1], vv[2], vv[3]);
    }
#pragma unroll
    for (int i = 0; i <= RL; ++i) {
        const float c = (float)(-dt * J[(x1_0 + i - 1 + N) % N]);
        nJr[i] = make_float2(c, c);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float c = (float)(-dt * J[(x2_0 - 1 + q + N) % N]);
        nJc[q] = make_float2(c, c);
    }

    // ---- load the state (one HBM read per call)
    float2 *gpsi = a.psi + a.tab.st_off[r];
    float2 P[RL][2];             // current Horner iterate (psi of this step is hi in shared memory)
    const float2 *Q = hi + lrow0 * N + x2_0;
#pragma unroll
    for (int i = 0; i < RL; ++i) {
        const float4 v = *reinterpret_cast<const float4 *>(gpsi + (size_t)(x1_0 + i) * N + x2_0);
        P[i][0] = make_float2(v.x, v.y);
        P[i][1] = make_float2(v.z, v.w);
        *reinterpret_cast<float4 *>(hi + (lrow0 + i) * N + x2_0) = v;
        *reinterpret_cast<float4 *>(lo + (lrow0 + i) * N + x2_0) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int x = threadIdx.x; x < N; x += blockDim.x) pacc[x] = 0.0;

    const int rank_up = (rank + C - 1) % C, rank_dn = (rank + 1) % C;
    // band 0 sends its first row into rank_up's "row below" slot, band BPC-1
    // its last row into rank_dn's "row above" slot
    const uint32_t send_up = map_rank(smem_u32(halo + N + x2_0), rank_up);
    const uint32_t send_up_mb = map_rank(smem_u32(&mbar[0][1]), rank_up);
    const uint32_t send_dn = map_rank(smem_u32(halo + x2_0), rank_dn);
    const uint32_t send_dn_mb = map_rank(smem_u32(&mbar[0][0]), rank_dn);
    const int w_left = band * WB + (wc + WB - 1) % WB;
    const int w_right = band * WB + (wc + 1) % WB;
    const int g = a.tab.group_of[r];
    const double pscale = a.tab.inv_count[g] * 0.5;
    double *Pg = a.P_mean ? a.P_mean + a.tab.group_off[g] : nullptr;
    bool dead = false;   // a bounded wait gave up: stop waiting, finish, report

    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q)
            for (int sd = 0; sd < 2; ++sd) mbar_init(smem_u32(&mbar[q][sd]), 1);
        mbar_init(smem_u32(&mbar_never), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_barrier();   // every CTA of the cluster is running, its mbarriers initialised
    if (a.test_timeout && threadIdx.x == 0 && blockIdx.x == 0)   // exercises the give-up path; the halo protocol is untouched
        (void)mbar_wait_bounded(smem_u32(&mbar_never), 0, 1000000ull /* 1 ms */, a.status);

    unsigned tc = 0;     // terms done: slot parity tc & 1, mbarrier phase (tc >> 1) & 1
    long long obs = 0;
    const long long n_steps = a.n_steps;
    for (long long step = 0; step <= n_steps; ++step) {
        const bool sample = a.obs_every > 0 && (step % a.obs_every) == 0;
        if (sample) {
            // P(x) = (row sums + column sums) / 2, norm = sum |psi|^2 (state =
            // hi): FP32 products |psi|^2, every sum in FP64
            double colp[2] = {0.0, 0.0}, nrm = 0.0;
#pragma unroll
            for (int i = 0; i < RL; ++i) {
                const double p0 = (double)abs2_f(P[i][0]);
                const double p1 = (double)abs2_f(P[i][1]);
                colp[0] += p0;
                colp[1] += p1;
                const double rs = warp_sum_d(p0 + p1);
                nrm += rs;
                if (lane == 0 && Pg) atomicAdd(pacc + x1_0 + i, rs);
            }
            if (Pg) {
                atomicAdd(pacc + x2_0, colp[0]);
                atomicAdd(pacc + x2_0 + 1, colp[1]);
            }
            if (lane == 0 && a.norm) atomicAdd(a.norm + obs * a.tab.R + r, nrm);
            __syncthreads();
            if (Pg) {
                for (int x = threadIdx.x; x < N; x += blockDim.x) {
                    const double v = pacc[x];
                    if (v != 0.0) atomicAdd(Pg + obs * a.p_width + x, v * pscale);
                    pacc[x] = 0.0;
                }
            }
        }
        const bool last = step == n_steps;
        if (last && !(sample && a.energy)) break;

        const int K = a.K;
        // One Horner stage (or the energy-only stencil of the last sample).
        auto term = [&](auto rev_tag, const int j) {
            constexpr bool REV = decltype(rev_tag)::value;
            const int parity = tc & 1;
            const uint32_t phase = (tc >> 1) & 1;
            // publish: slab edge rows to the neighbour CTAs, band edges and
            // warp edge columns to this CTA's shared memory
            const float4 top = make_float4(P[0][0].x, P[0][0].y, P[0][1].x, P[0][1].y);
            const float4 bot = make_float4(P[RL - 1][0].x, P[RL - 1][0].y, P[RL - 1][1].x, P[RL - 1][1].y);
            if (band == 0)
                st_async16(send_up + parity * (2 * N * 8), top, send_up_mb + parity * 16);
            if (band == BPC - 1)
                st_async16(send_dn + parity * (2 * N * 8), bot, send_dn_mb + parity * 16);
            float2 *eb = edge + parity * (BPC * 2 * N) + band * (2 * N);
            *reinterpret_cast<float4 *>(eb + x2_0) = top;
            *reinterpret_cast<float4 *>(eb + N + x2_0) = bot;
            {
                float2 c0v[RL], c1v[RL];
#pragma unroll
                for (int i = 0; i < RL; ++i) {
                    c0v[i] = P[i][0];
                    c1v[i] = P[i][1];
                }
                const uint32_t sb = smem_u32(seamb + parity * (W * 2 * RL) + warp * (2 * RL));
                st_shared_col8_if(sb, lane == 0, c0v);
                st_shared_col8_if(sb + RL * 8, lane == 31, c1v);
            }
            __syncthreads();
            // this term's arrival + expected bytes on both halo slots (thread 0)
            mbar_expect_tx2_if(smem_u32(&mbar[parity][0]), smem_u32(&mbar[parity][1]), N * 8,
                               threadIdx.x == 0);
            // gather halos
            float4 u4, d4;
            if (band > 0) {
                u4 = *reinterpret_cast<const float4 *>(edge + parity * (BPC * 2 * N) + (band - 1) * (2 * N) + N + x2_0);
            } else {
                if (!dead) dead = !mbar_wait_bounded(smem_u32(&mbar[parity][0]), phase, a.wait_limit_ns, a.status);
                u4 = *reinterpret_cast<const float4 *>(halo + parity * (2 * N) + x2_0);
            }
            if (band < BPC - 1) {
                d4 = *reinterpret_cast<const float4 *>(edge + parity * (BPC * 2 * N) + (band + 1) * (2 * N) + x2_0);
            } else {
                if (!dead) dead = !mbar_wait_bounded(smem_u32(&mbar[parity][1]), phase, a.wait_limit_ns, a.status);
                d4 = *reinterpret_cast<const float4 *>(halo + parity * (2 * N) + N + x2_0);
            }
            // lane 0 reads the right neighbour warp's first column, the others
            // the left neighbour warp's last column (only lane 31 uses it)
            const float4 *seam4 = reinterpret_cast<const float4 *>(
                seamb + parity * (W * 2 * RL) + (lane == 0 ? w_right * (2 * RL) : w_left * (2 * RL) + RL));
            const float2 up0 = make_float2(u4.x, u4.y), up1 = make_float2(u4.z, u4.w);
            const float2 dn0 = make_float2(d4.x, d4.y), dn1 = make_float2(d4.z, d4.w);
            const float inv_j = a.inv_j[j];
            const bool first = j == K;
            const bool en = first && sample && a.energy;
            double e = 0.0;
            if (last) {
                stencil_term<kEnergyOnly, true, N, REV>(P, Q, V4, nJr, nJc, up0, up1, dn0, dn1, seam4, lane, inv_j, e);
            } else if (j == 1) {
                if (en)
                    stencil_term<kFinal, true, N, REV>(P, Q, V4, nJr, nJc, up0, up1, dn0, dn1, seam4, lane, inv_j, e);
                else
                    stencil_term<kFinal, false, N, REV>(P, Q, V4, nJr, nJc, up0, up1, dn0, dn1, seam4, lane, inv_j, e);
            } else if (en) {
                stencil_term<kHorner, true, N, REV>(P, Q, V4, nJr, nJc, up0, up1, dn0, dn1, seam4, lane, inv_j, e);
            } else {
                stencil_term<kHorner, false, N, REV>(P, Q, V4, nJr, nJc, up0, up1, dn0, dn1, seam4, lane, inv_j, e);
            }
            if (en || last) {
                const double es = warp_sum_d(e);
                if (lane == 0) atomicAdd(a.energy + obs * a.tab.R + r, es * a.inv_dt);
            }
            ++tc;
        };
        if (last) {
            term(std::false_type(), K);
        } else {
            for (int j = K; j >= 1; --j) term(std::false_type(), j);
        }
        if (sample) ++obs;
        if (last) break;

        // psi(t+dt) = psi + A w_2 (now in P), with the rounding error carried in lo
#pragma unroll
        for (int i = 0; i < RL; ++i) {
            float4 *hp = reinterpret_cast<float4 *>(hi + (lrow0 + i) * N + x2_0);
            float4 *lp = reinterpret_cast<float4 *>(lo + (lrow0 + i) * N + x2_0);
            float4 h4 = *hp, l4 = *lp;
            if (a.compensated) {
                compensated_add(h4.x, l4.x, P[i][0].x);
                compensated_add(h4.y, l4.y, P[i][0].y);
                compensated_add(h4.z, l4.z, P[i][1].x);
                compensated_add(h4.w, l4.w, P[i][1].y);
                *lp = l4;
            } else {
                h4.x += P[i][0].x;
                h4.y += P[i][0].y;
                h4.z += P[i][1].x;
                h4.w += P[i][1].y;
            }
            *hp = h4;
            P[i][0] = make_float2(h4.x, h4.y);
            P[i][1] = make_float2(h4.z, h4.w);
        }
    }

    // ---- write the state back (one HBM write per call)
#pragma unroll
    for (int i = 0; i < RL; ++i) {
        const float4 h4 = *reinterpret_cast<const float4 *>(hi + (lrow0 + i) * N + x2_0);
        *reinterpret_cast<float4 *>(gpsi + (size_t)(x1_0 + i) * N + x2_0) = h4;
    }
    cluster_barrier();   // no CTA leaves while a neighbour may still write its shared memory
}

using FusedKernel = void (*)(FusedArgs);

struct FusedShape {
    int BPC, C, threads;
    size_t smem;
    FusedKernel kern;
};

template <int N, int BPC, int MINB>
FusedShape make_shape() {
    FusedShape f;
    constexpr int WB = N / 64, SR = RL * BPC, W = WB * BPC;
    f.BPC = BPC;
    f.C = N / SR;
    f.threads = 32 * W;
    f.smem = sizeof(float2) * ((size_t)2 * SR * N + (size_t)2 * 2 * N + (size_t)2 * BPC * 2 * N +
                               (size_t)2 * W * 2 * RL) +
             sizeof(float) * (size_t)SR * N + sizeof(double) * (size_t)N;   // diagonal (as float4 [SR/2][N/2]) + pacc
    f.kern = taylor_fused_kernel<N, BPC, MINB>;
    return f;
}

// Shapes compiled in per N: (warp bands per CTA, CTAs per SM the registers are
// capped for).  Index 0 is the default; the others are selected with
// CTQW_FUSED_SHAPE(k) for tuning.
constexpr int kShapes = 3;

bool fused_shape(int N, int idx, FusedShape &f) {
    FusedShape opts[kShapes];
    switch (N) {
        case 64: opts[0] = make_shape<64, 8, 2>(); opts[1] = make_shape<64, 4, 2>(); opts[2] = make_shape<64, 8, 1>(); break;
        case 128: opts[0] = make_shape<128, 4, 2>(); opts[1] = make_shape<128, 2, 2>(); opts[2] = make_shape<128, 4, 1>(); break;
        case 192: opts[0] = make_shape<192, 2, 2>(); opts[1] = make_shape<192, 4, 1>(); opts[2] = make_shape<192, 2, 1>(); break;
        case 256: opts[0] = make_shape<256, 2, 2>(); opts[1] = make_shape<256, 4, 1>(); opts[2] = make_shape<256, 2, 1>(); break;
        default: return false;
    }
    if (idx < 0 || idx >= kShapes) return false;
    f = opts[idx];
    return true;
}

}  // namespace

bool fused_taylor_supported(const ctqw_hamiltonian *h, int dtype) {
    FusedShape f;
    return dtype == CTQW_C64 && h->m == 2 && h->uniform && fused_shape(h->Nmax, 0, f);
}

int launch_taylor_fused(const ctqw_hamiltonian *h, void *psi, double dt, int K, int64_t n_steps,
                        int obs_every, double *P_mean, double *norm, double *energy,
                        int compensated, int shape, int test_timeout, cudaStream_t s) {
    FusedShape f;
    if (!fused_shape(h->Nmax, shape, f)) {
        ctqw_set_error("fused path: unsupported size N=%d or shape %d", h->Nmax, shape);
        return CTQW_EUNSUPPORTED;
    }
    if (K > kMaxK) {
        ctqw_set_error("fused path: K=%d above %d", K, kMaxK);
        return CTQW_EUNSUPPORTED;
    }
    FusedArgs a;
    a.eps = h->eps64;
    a.J = h->J64;
    a.tab = real_table(h);
    a.psi = (float2 *)psi;
    a.N = h->Nmax;
    a.dt = dt;
    a.inv_dt = 1.0 / dt;
    a.K = K;
    a.n_steps = n_steps;
    a.obs_every = obs_every;
    a.p_width = h->p_width;
    a.P_mean = P_mean;
    a.norm = norm;
    a.energy = energy;
    a.compensated = compensated;
    a.status = h->status_d;
    a.test_timeout = test_timeout;
    a.wait_limit_ns = 2000000000ull;   // 2 s: halo rows normally arrive within microseconds
    a.inv_j[0] = 0.f;
    for (int j = 1; j <= kMaxK; ++j) a.inv_j[j] = (float)(1.0 / j);
    FusedKernel kern = f.kern;
    CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)f.smem));
    if (f.C > 8)
        CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)kern,
                                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(h->R * f.C));
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
    CTQW_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, (const void *)kern, &cfg));
    if (clusters < 1) {
        ctqw_set_error("fused path: no cluster of %d CTAs x %d threads fits", f.C, f.threads);
        return CTQW_EUNSUPPORTED;
    }
    CTQW_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
    return CTQW_OK;
}
