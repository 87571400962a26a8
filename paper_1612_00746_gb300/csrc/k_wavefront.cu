// Fused Taylor propagation for two particles in complex FP32 as a row
// wavefront: temporal blocking of the K stencil applications of a step.
//
// One CTA propagates one realization at a time (persistent: it loops over a
// list of realizations).  Warp s-1 is stage s of the Horner evaluation of the
// order-K polynomial of Algorithm 3 (Sec. 2.3),
//   w_K = psi + (A/K) psi,  w_j = psi + (A/j) w_{j+1},  psi(t+dt) = psi + A w_2,
// A = -i dt H, stage s producing w_{K+1-s} (stage K: the increment A w_2).
// The stages sweep the N x N tile row by row (x1), stage s two rows behind
// stage s-1: a row of w_j needs rows x1-1, x1, x1+1 of w_{j+1}, so stage s
// computes row g at tick g + 2s, once stage s-1 has finished row g+1.  One
// __syncthreads per tick orders the whole pipeline.  Each stage keeps the
// three rows it works on in registers (it reads one new row per tick) and
// passes its output to the next stage through a two-row ring in shared
// memory; psi itself streams in through a ring filled by cp.async and the
// new state goes straight back to global memory, so every step reads psi
// once and writes it once, whatever K is.
//
// Rows of consecutive steps follow each other in the same sweep (a zero row
// between steps is the open chain's boundary below the last row and above
// the first), so the pipeline fills once per launch.  Each lane owns CL = N/32
// adjacent columns of a row: neighbours along x2 are in its registers or one
// 64-bit shuffle away (the shuffle wraps from column N-1 to 0, a bond with
// J[N-1] = 0 on an open chain).
//
// The increment A w_2 is added to the state with its rounding error carried
// in a second FP32 word (workspace, one state) as in the full-row kernel.
// Row layout in shared memory and of the carried error in global memory:
// lane-major, the column pair k/2 of lane l at float4 slot (k/2)*32 + l.
#include "ctqw_internal.cuh"
#include "fused_common.cuh"

namespace {

using namespace fused;

constexpr int kWaveMaxK = 16;   // stages = warps (<= 16 warps: 128 registers a thread)
constexpr int kWaveD = 8;       // rows of psi in flight ahead of stage 1

struct WaveArgs {
    const double *eps;
    const double *J;
    RealTable tab;
    float2 *psi;          // state (hi), row-major
    float4 *lo;           // carried rounding error, lane-major rows
    const int *list;      // realizations handled by this launch
    int n_list;
    double dt;
    float dtU;
    int K;
    long long n_steps;
    int compensated;
    float inv_j[kWaveMaxK + 1];
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory");
}

template <int CL>
__device__ __forceinline__ void load_row(float2 (&v)[CL], const float2 *row, int lane) {
#pragma unroll
    for (int k = 0; k < CL; k += 2) {
        const float4 q = reinterpret_cast<const float4 *>(row)[(k / 2) * 32 + lane];
        v[k] = make_float2(q.x, q.y);
        v[k + 1] = make_float2(q.z, q.w);
    }
}

template <int CL>
__device__ __forceinline__ void zero_row(float2 (&v)[CL]) {
#pragma unroll
    for (int k = 0; k < CL; ++k) v[k] = make_float2(0.f, 0.f);
}

// Per-warp position in the sweep: row g of the pipeline (step n, row x1;
// x1 = N is the zero row between steps).
struct Cursor {
    long long g;
    int x1;
};

__device__ __forceinline__ void advance(Cursor &c, int N) {
    ++c.g;
    c.x1 = (c.x1 == N) ? 0 : c.x1 + 1;
}

// One tick of stage s for the window (wm, wc, wp) = rows (x1-1, x1, x1+1)
// after the slide: the row x1+1 is read into wp here.
template <int CL>
__device__ __forceinline__ void stage_tick(const WaveArgs &a, int s, int K, int lane, const Cursor &c,
                                           long long G, float2 (&wm)[CL], float2 (&wc)[CL],
                                           float2 (&wp)[CL], const float2 *psiring, int Rpsi,
                                           float2 *stg, const float2 *loring, int Rlo,
                                           const float4 *rowc, const float2 (&ec)[CL],
                                           const float2 (&nJc)[CL + 1], float2 *gpsi, float4 *glo,
                                           int psi_slot, int lo_slot) {
    constexpr int N = 32 * CL;
    if (c.g < -1 || c.g >= G) return;   // warp-uniform
    // the next row of the previous stage (psi for stage 1)
    const bool have_next = (c.x1 < N - 1) || (c.x1 == N && c.g + 1 < G);
    if (have_next) {
        const float2 *src = (s == 1) ? psiring + (size_t)((psi_slot + 1) % Rpsi) * N
                                     : stg + (size_t)((s - 2) * 2 + (int)((c.g + 1) & 1)) * N;
        load_row<CL>(wp, src, lane);
    } else {
        zero_row<CL>(wp);
    }
    if (c.x1 >= N) return;   // the zero row: nothing to compute

    const int x1 = c.x1;
    const float4 rc = rowc[x1], rn = rowc[x1 + 1];
    const float2 er = make_float2(rc.x, rc.y), jup = make_float2(rc.z, rc.w);
    const float2 jdn = make_float2(rn.z, rn.w);
    const float2 lft = shfl2(wc[CL - 1], (lane + 31) & 31);
    const float2 rgt = shfl2(wc[0], (lane + 1) & 31);
    float2 y[CL];
#pragma unroll
    for (int k = 0; k < CL; ++k) {
        const float2 l = (k == 0) ? lft : wc[k - 1];
        const float2 r = (k == CL - 1) ? rgt : wc[k + 1];
        float2 t = __fmul2_rn(ec[k], wc[k]);
        t = __ffma2_rn(er, wc[k], t);
        t = __ffma2_rn(jup, wm[k], t);
        t = __ffma2_rn(jdn, wp[k], t);
        t = __ffma2_rn(nJc[k], l, t);
        t = __ffma2_rn(nJc[k + 1], r, t);
        y[k] = t;
    }
    // dt U on the diagonal x2 = x1 (one lane of the row)
    if (lane == x1 / CL) {
        const int kd = x1 - lane * CL;
        const float2 dU = make_float2(a.dtU, a.dtU);
#pragma unroll
        for (int k = 0; k < CL; ++k)
            if (k == kd) y[k] = __ffma2_rn(dU, wc[k], y[k]);
    }
    if (s < K) {
        // w = psi + (-i/j) y, j = K + 1 - s
        const float inv_j = a.inv_j[K + 1 - s];
        float2 q[CL];
        if (s == 1) {
#pragma unroll
            for (int k = 0; k < CL; ++k) q[k] = wc[k];
        } else {
            load_row<CL>(q, psiring + (size_t)psi_slot * N, lane);
        }
        float4 *dst = reinterpret_cast<float4 *>(stg + (size_t)((s - 1) * 2 + (int)(c.g & 1)) * N);
#pragma unroll
        for (int k = 0; k < CL; k += 2) {
            const float4 o = make_float4(fmaf(inv_j, y[k].y, q[k].x), fmaf(-inv_j, y[k].x, q[k].y),
                                         fmaf(inv_j, y[k + 1].y, q[k + 1].x),
                                         fmaf(-inv_j, y[k + 1].x, q[k + 1].y));
            dst[(k / 2) * 32 + lane] = o;
        }
    } else {
        // psi(t+dt) = psi + (-i) y, the rounding error carried in lo
        float2 h[CL], l[CL];
        load_row<CL>(h, psiring + (size_t)psi_slot * N, lane);
        load_row<CL>(l, loring + (size_t)lo_slot * N, lane);
#pragma unroll
        for (int k = 0; k < CL; ++k) {
            const float2 inc = make_float2(y[k].y, -y[k].x);
            if (a.compensated) {
                compensated_add2(h[k], l[k], inc);
            } else {
                h[k].x += inc.x;
                h[k].y += inc.y;
            }
        }
        float4 *hrow = reinterpret_cast<float4 *>(gpsi + (size_t)x1 * N + lane * CL);
        float4 *lrow = glo + (size_t)x1 * (N / 2);
#pragma unroll
        for (int k = 0; k < CL; k += 2) {
            hrow[k / 2] = make_float4(h[k].x, h[k].y, h[k + 1].x, h[k + 1].y);
            lrow[(k / 2) * 32 + lane] = make_float4(l[k].x, l[k].y, l[k + 1].x, l[k + 1].y);
        }
    }
}

// CL columns per lane (N = 32 CL); blockDim = 32 K.
template <int CL>
__global__ void __launch_bounds__(32 * kWaveMaxK, 1) taylor_wavefront_kernel(const __grid_constant__ WaveArgs a) {
    constexpr int N = 32 * CL;
    constexpr int D = kWaveD;
    static_assert(CL % 2 == 0 && CL >= 2 && CL <= 8, "unsupported row width");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = a.K;
    const int Rpsi = 2 * K + D + 1;   // psi row g: loaded at tick g - D, last read at tick g + 2K
    const int Rlo = D + 2;            // lo row g: loaded at tick g + 2K - D - 1, read at g + 2K
    float2 *psiring = reinterpret_cast<float2 *>(smem_raw);     // [Rpsi][N]
    float2 *stg = psiring + (size_t)Rpsi * N;                    // [K-1][2][N]
    float2 *loring = stg + (size_t)(K > 1 ? K - 1 : 0) * 2 * N;  // [Rlo][N]
    float4 *rowc = reinterpret_cast<float4 *>(loring + (size_t)Rlo * N);   // [N + 1]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = warp + 1;
    const long long G = a.n_steps * (N + 1);

    for (int it = blockIdx.x; it < a.n_list; it += gridDim.x) {
        const int r = a.list[it];
        const int64_t po = a.tab.par_off[r];
        const double *eps = a.eps + po, *J = a.J + po;
        const double dt = a.dt;
        __syncthreads();   // the previous realization is done with rowc and the rings
        for (int q = threadIdx.x; q <= N; q += blockDim.x) {
            const float e = q < N ? (float)(dt * eps[q]) : 0.f;
            const float j = (float)(-dt * J[(q - 1 + N) % N]);
            rowc[q] = make_float4(e, e, j, j);
        }
        float2 ec[CL], nJc[CL + 1];
#pragma unroll
        for (int k = 0; k < CL; ++k) {
            const float v = (float)(dt * eps[lane * CL + k]);
            ec[k] = make_float2(v, v);
        }
#pragma unroll
        for (int k = 0; k <= CL; ++k) {
            const float v = (float)(-dt * J[(lane * CL + k - 1 + N) % N]);
            nJc[k] = make_float2(v, v);
        }
        float2 *gpsi = a.psi + a.tab.st_off[r];
        float4 *glo = a.lo + a.tab.st_off[r] / 2;

        // cursors at tick t = -D: stage s at row t - 2s, loader (hi) at t + D,
        // loader (lo) at t - 2K + D + 1
        Cursor cs{(long long)(-D - 2 * s), N}, ch{0, 0}, cl{(long long)(-2 * K + 1), 0};
        // x1 of negative rows is never used except cs at g = -1, where it must be N
        {
            // row -1 - 2s + ... : set x1 so that it reads N at g = -1
            const long long back = -1 - cs.g;   // ticks until g = -1
            cs.x1 = (int)(((long long)N - back % (N + 1) + (N + 1)) % (N + 1));
        }
        int psi_slot_s = (int)((((cs.g) % Rpsi) + Rpsi) % Rpsi);
        int lo_slot_s = (int)((((cs.g) % Rlo) + Rlo) % Rlo);
        int psi_slot_h = 0, lo_slot_l = (int)((((cl.g) % Rlo) + Rlo) % Rlo);
        float2 wa[CL], wb[CL], wd[CL];
        zero_row<CL>(wa);
        zero_row<CL>(wb);
        zero_row<CL>(wd);
        const uint32_t psiring_u32 = smem_u32(psiring), loring_u32 = smem_u32(loring);

        const long long T = G + 2LL * K + D;   // ticks from -D
        auto loader = [&]() {
            if (warp == 0) {
                if (ch.g < G && ch.x1 < N) {
                    const float2 *src = gpsi + (size_t)ch.x1 * N + lane * CL;
                    const uint32_t dst = psiring_u32 + (uint32_t)(psi_slot_h * N) * 8u;
#pragma unroll
                    for (int k = 0; k < CL; k += 2)
                        cp_async16(dst + (uint32_t)(((k / 2) * 32 + lane) * 16), src + k);
                }
                if (cl.g >= 0 && cl.g < G && cl.x1 < N) {
                    const float4 *src = glo + (size_t)cl.x1 * (N / 2);
                    const uint32_t dst = loring_u32 + (uint32_t)(lo_slot_l * N) * 8u;
#pragma unroll
                    for (int k = 0; k < CL; k += 2)
                        cp_async16(dst + (uint32_t)(((k / 2) * 32 + lane) * 16), src + (k / 2) * 32 + lane);
                }
                cp_async_commit();
            }
            advance(ch, N);
            psi_slot_h = (psi_slot_h + 1 == Rpsi) ? 0 : psi_slot_h + 1;
            if (cl.g >= 0) advance(cl, N); else ++cl.g;
            lo_slot_l = (lo_slot_l + 1 == Rlo) ? 0 : lo_slot_l + 1;
        };
        auto end_tick = [&]() {
            if (warp == 0) cp_async_wait<D>();
            __syncthreads();
            advance(cs, N);
            psi_slot_s = (psi_slot_s + 1 == Rpsi) ? 0 : psi_slot_s + 1;
            lo_slot_s = (lo_slot_s + 1 == Rlo) ? 0 : lo_slot_s + 1;
        };
        // three ticks per iteration so that the window rotates through wa, wb, wd
        // without register moves
        for (long long t = 0; t < T; t += 3) {
            loader();
            stage_tick<CL>(a, s, K, lane, cs, G, wa, wb, wd, psiring, Rpsi, stg, loring, Rlo, rowc, ec,
                           nJc, gpsi, glo, psi_slot_s, lo_slot_s);
            end_tick();
            loader();
            stage_tick<CL>(a, s, K, lane, cs, G, wb, wd, wa, psiring, Rpsi, stg, loring, Rlo, rowc, ec,
                           nJc, gpsi, glo, psi_slot_s, lo_slot_s);
            end_tick();
            loader();
            stage_tick<CL>(a, s, K, lane, cs, G, wd, wa, wb, psiring, Rpsi, stg, loring, Rlo, rowc, ec,
                           nJc, gpsi, glo, psi_slot_s, lo_slot_s);
            end_tick();
        }
        if (warp == 0) cp_async_wait<0>();
    }
}

using WaveKernel = void (*)(WaveArgs);

struct WaveShape {
    WaveKernel kern;
    int CL;
};

bool wave_shape_for(int N, WaveShape &f) {
    switch (N) {
        case 64: f.kern = taylor_wavefront_kernel<2>; f.CL = 2; return true;
        case 128: f.kern = taylor_wavefront_kernel<4>; f.CL = 4; return true;
        case 192: f.kern = taylor_wavefront_kernel<6>; f.CL = 6; return true;
        case 256: f.kern = taylor_wavefront_kernel<8>; f.CL = 8; return true;
        default: return false;
    }
}

size_t wave_smem(int N, int K) {
    const int D = kWaveD;
    return sizeof(float2) * (size_t)N * ((size_t)(2 * K + D + 1) + (size_t)(K > 1 ? K - 1 : 0) * 2 + (size_t)(D + 2)) +
           sizeof(float4) * (size_t)(N + 1);
}

}  // namespace

bool wavefront_supported(const ctqw_hamiltonian *h, int dtype, int K) {
    WaveShape f;
    if (dtype != CTQW_C64 || h->m != 2 || h->periodic || K < 1 || K > kWaveMaxK) return false;
    for (int N : h->group_N) {
        if (!wave_shape_for(N, f)) return false;
        // a row of step n+1 is read back D ticks before stage 1 needs it and
        // must have been written by stage K of step n by then
        if (N + 1 <= 2 * K + kWaveD) return false;
        if (wave_smem(N, K) > 227 * 1024) return false;
    }
    return true;
}

size_t wavefront_workspace_bytes(const ctqw_hamiltonian *h) {
    return sizeof(float2) * (size_t)h->total_amp;
}

int launch_taylor_wavefront(const ctqw_hamiltonian *h, void *psi, void *lo, double dt, int K,
                            int64_t n_steps, int compensated, cudaStream_t s) {
    if (n_steps <= 0) return CTQW_OK;
    int sms = 0, dev = 0;
    CTQW_CUDA_TRY(cudaGetDevice(&dev));
    CTQW_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WaveArgs a;
    a.eps = h->eps64;
    a.J = h->J64;
    a.tab = real_table(h);
    a.psi = (float2 *)psi;
    a.lo = (float4 *)lo;
    a.dt = dt;
    a.dtU = (float)(dt * h->U);
    a.K = K;
    a.n_steps = n_steps;
    a.compensated = compensated;
    a.inv_j[0] = 0.f;
    for (int j = 1; j <= kWaveMaxK; ++j) a.inv_j[j] = (float)(1.0 / j);
    // one launch per row width over that size group's realizations
    int off = 0;
    for (size_t gi = 0; gi < h->group_N.size(); ++gi) {
        const int N = h->group_N[gi], cnt = h->group_count[gi];
        WaveShape f;
        if (!wave_shape_for(N, f)) {
            ctqw_set_error("wavefront path: unsupported size N=%d", N);
            return CTQW_EUNSUPPORTED;
        }
        const size_t smem = wave_smem(N, K);
        CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)f.kern,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        a.list = h->by_group_d + off;
        a.n_list = cnt;
        const int grid = cnt < sms ? cnt : sms;
        f.kern<<<grid, 32 * K, smem, s>>>(a);
        CTQW_CUDA_TRY(cudaGetLastError());
        off += cnt;
    }
    return CTQW_OK;
}
