// One-body reduced density matrix on the tensor cores (tcgen05, TF32 with
// split operands): the dense Hermitian contraction that dominates the
// paper's post-processing (Sec. 4: cublasCher on <rho>), here for the
// partial trace over all particles but one,
//
//   rho1(x, x') = (1/R_g)(1/m) sum_r sum_j sum_k psi_r(x_j = x, k) conj(psi_r(x_j = x', k)).
//
// Per size group it is a real GEMM pair over K = R_g m N^(m-1):
//   Re rho1 = Ar Ar^T + Ai Ai^T,   Im rho1 = Ai Ar^T - Ar Ai^T
// with A[x][(r, j, k)] = psi_r(x_j = x, k).  Every FP32 operand is split
// into TF32 pieces, a = a_hi + a_lo (a_hi = a rounded to TF32, a_lo the
// rest rounded to TF32), and each product is a_hi b_hi + a_hi b_lo +
// a_lo b_hi (the dropped a_lo b_lo is ~2^-22 of it).
//
// Only the 128 x 128 tiles (x, x') with x / 128 <= x' / 128 are computed;
// the rest of rho1 is their conjugate transpose.  A CTA owns one tile and a
// range of (realization, particle) pairs, and its warps have three roles:
//  - warps 0-7 (producers) load 16 k at a time of the tile's 128 + 128 rows,
//    split them into the four TF32 arrays re_hi, re_lo, im_hi, im_lo and
//    store them into a three-stage shared-memory ring in the MMA's
//    canonical K-major layout (8-row by 16-byte core matrices);
//  - one thread of warp 8 issues 12 MMAs per 8 k (M = 128, N = 128, K = 8,
//    FP32 accumulate in TMEM: 128 columns for Re, 128 for Im) and commits
//    them to the stage's mbarrier, which hands the stage back;
//  - warps 9-12 drain: every 256 k the MMAs switch to the other of two TMEM
//    accumulators, and the drain warps add the finished FP32 partials into
//    the CTA's running totals, kept as two FP32 words (TwoSum) in a global
//    slot of its own, so the totals carry ~2^-44 of relative rounding.  A
//    block's FP32 sum in TMEM can be off by up to 256 ulp of its sum of
//    |terms| (the adds may round toward zero): at most 256 x 2^-23 of the
//    largest element of rho1.
// A second kernel sums the slots of all CTAs in FP64 and fills the lower
// triangle.  Every wait is bounded in time (status word, then the CTA stops).
#include <cstdint>

#include "ctqw_internal.cuh"

namespace {

constexpr int kM = 128;          // rows x per tile (MMA M)
constexpr int kNt = 128;         // columns x' per tile (MMA N)
constexpr int kKc = 16;          // k per shared-memory stage
constexpr int kStages = 3;       // shared-memory ring
constexpr int kProducerWarps = 8;
constexpr int kMmaWarp = kProducerWarps;           // warp 8 issues the MMAs; warps 9..12 drain TMEM
constexpr int kThreads = 32 * (kProducerWarps + 1 + 4);
constexpr int kArr = kM * kKc;   // floats per operand array of a stage
constexpr int kBlockK = 256;     // k accumulated in TMEM between two drains
constexpr uint64_t kWaitNs = 2000000000ull;   // bound of every wait (2 s)

struct TcArgs {
    RealTable tab;
    const int32_t *list;     // the group's realizations
    const float2 *psi;
    float *slots;            // per CTA: [2 (hi, lo)][2 (re, im)][kNt][kM] FP32
    int *status;
    int N, m, pairs;         // pairs = R_g m
    int tiles;               // tiles per side, ceil(N / 128)
    int pairs_per_split;
    int64_t n_k;             // N^(m-1)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory descriptor: canonical K-major layout, no swizzle
// (LBO: bytes between core matrices along K, SBO: along M/N), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, K-major, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N, bool negate_a) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (negate_a ? (1u << 13) : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of parity `parity` to complete: false after
// kWaitNs nanoseconds or once another role has raised `stop`.  Each try may
// suspend the thread for up to hint_ns (0: the hardware's default), so that
// idle roles do not spin on the barrier.
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, const volatile int *stop,
                                          uint32_t hint_ns = 0) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        if (hint_ns)
            asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n\t"
                         "selp.u32 %0, 1, 0, q;\n\t}"
                         : "=r"(done) : "r"(mb), "r"(parity), "r"(hint_ns) : "memory");
        else
            asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, q;\n\t}"
                         : "=r"(done) : "r"(mb), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 63) == 0) {
            const uint64_t t = global_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > kWaitNs || *stop) return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mb) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mb) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
}

__device__ __forceinline__ float tf32_round(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// hi + lo + v, rounded back into (hi, lo): TwoSum, then the error into lo.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// 32 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Offset (floats) of element (row, k) of a [kM x kKc] operand array in the
// canonical layout: core (row / 8, k / 4) of 8 x 4 floats, cores along K first.
__device__ __forceinline__ int canon(int row, int k) {
    return ((row >> 3) * (kKc / 4) + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

__global__ void __launch_bounds__(kThreads, 1) rho1_tc_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) float smem[];
    // stage s: A arrays at smem + s * 8 kArr + q kArr, B arrays at + 4 kArr (q = re_hi, re_lo, im_hi, im_lo)
    __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], acc_full[2], acc_empty[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ int stop;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.N, m = a.m;
    // blockIdx.x: a tile (ty <= tx) of the upper triangle, row by row; the
    // lower one is its conjugate transpose (rho1 is Hermitian)
    int ty = 0, rest = blockIdx.x;
    while (rest >= a.tiles - ty) rest -= a.tiles - ty++;
    const int x0 = ty * kM, xp0 = (ty + rest) * kNt;
    const int p0 = blockIdx.y * a.pairs_per_split;
    const int p1 = min(a.pairs, p0 + a.pairs_per_split);
    const int cta = blockIdx.y * gridDim.x + blockIdx.x;
    float *slot = a.slots + (size_t)cta * (2 * 2 * kNt * kM);

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(kProducerWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&acc_empty[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stop = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     ::"r"(smem_u32(&tmem_base)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // accumulator b (0, 1) at columns 256 b: Re at [0, 128), Im at [128, 256) of it
    const uint32_t tmem = tmem_base;

    const int64_t n_k = a.n_k;
    const int64_t chunks_per_pair = n_k / kKc;
    const int64_t n_chunks = (int64_t)(p1 - p0) * chunks_per_pair;
    const int64_t chunks_per_block = kBlockK / kKc;   // a block may span pairs
    const int64_t n_blocks = (n_chunks + chunks_per_block - 1) / chunks_per_block;
    volatile int *vstop = &stop;

    if (warp < kProducerWarps) {
        // ---- producers: global -> TF32 pieces in the stage ring --------------
        // Warps 0-3 stage the rows x, warps 4-7 the rows x'; warp w covers
        // rows 32 (w % 4) .. + 31 of its side, each thread 4 groups of 4
        // consecutive k.  Two assignments, chosen per pair by the memory
        // order of the operand, so that the global loads coalesce and every
        // quarter warp writes 128 contiguous bytes of shared memory:
        //   x contiguous (S_k = N): lane = row, group q = k / 4;
        //   k contiguous (S_k = 1): lane = 8 (k / 4) + row % 8, group q = row / 8 % 4.
        const int side = warp >> 2, row0 = 32 * (warp & 3);
        const int xA = (side ? xp0 : x0) + row0 + lane;
        int xB[4], soffA[4], soffB[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rowB = row0 + 8 * q + (lane & 7);
            xB[q] = (side ? xp0 : x0) + rowB;
            soffA[q] = side * 4 * kArr + canon(row0 + lane, 4 * q);
            soffB[q] = side * 4 * kArr + canon(rowB, 4 * (lane >> 3));
        }
        // The chunk the next load reads: amplitude (x, k0 + kk) of pair p sits
        // at base + x S_x + kk S_k.  With the partial trace over particle j,
        // S_x = N^(m-1-j); k runs over the other coordinates in order, so for
        // j < m - 1 it is contiguous within blocks of K_lo = S_x (S_k = 1; a
        // chunk of 16 never straddles two, N being a multiple of 16) and for
        // j = m - 1 it steps by N (S_k = N).
        int cp = 0;
        int64_t cc = 0, base = 0, S_x = 1, S_k = 1, K_lo = 1, S_hi = 1, rem = 0;
        auto set_pair = [&](int p) {
            cp = p;
            cc = 0;
            const int r = a.list[p / m], j = p - (p / m) * m;
            int64_t sx = 1;
            for (int l = j + 1; l < m; ++l) sx *= N;
            S_x = sx;
            K_lo = sx;
            S_hi = sx * N;
            S_k = (j == m - 1) ? N : 1;
            base = a.tab.st_off[r];
            rem = 0;
        };
        auto advance = [&]() {
            if (++cc == chunks_per_pair) {
                if (cp + 1 < p1) set_pair(cp + 1);
                return;
            }
            if (S_k != 1) {
                base += kKc * S_k;
            } else {
                base += kKc;
                rem += kKc;
                if (rem == K_lo) {
                    rem = 0;
                    base += S_hi - K_lo;
                }
            }
        };
        // the 16 amplitudes of the cursor's chunk that this thread stages;
        // v_kc: they follow the k-contiguous assignment
        auto load_chunk = [&](float2 (&v)[16], bool &v_kc) {
            v_kc = S_k == 1;
            if (v_kc) {
                // offsets are even (N a multiple of 16): two 16-byte loads per group
                const int k4 = lane >> 3;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 u0 = make_float4(0.f, 0.f, 0.f, 0.f), u1 = u0;
                    if (xB[q] < N) {
                        const float4 *src = (const float4 *)(a.psi + base + (int64_t)xB[q] * S_x + 4 * k4);
                        u0 = __ldg(src);
                        u1 = __ldg(src + 1);
                    }
                    v[4 * q] = make_float2(u0.x, u0.y);
                    v[4 * q + 1] = make_float2(u0.z, u0.w);
                    v[4 * q + 2] = make_float2(u1.x, u1.y);
                    v[4 * q + 3] = make_float2(u1.z, u1.w);
                }
            } else {
                const float2 *src = a.psi + base + xA;
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        v[4 * q + t] = xA < N ? __ldg(src + (int64_t)(4 * q + t) * S_k) : make_float2(0.f, 0.f);
            }
            advance();
        };
        // stage chunk c from v into its ring slot, then refill v with chunk
        // c + 2: two chunks of loads stay in flight per thread
        auto produce = [&](int64_t c, float2 (&v)[16], bool &v_kc) -> bool {
            const int s = (int)(c % kStages);
            const int64_t use = c / kStages;
            // the slot's previous MMAs (chunk c - kStages) must be done
            if (use > 0 && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((use - 1) & 1), vstop, 500)) {
                if (lane == 0) atomicOr(a.status, 4);
                stop = 1;
                return false;
            }
            float *st = smem + s * 8 * kArr;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 rh, rl, ih, il;
                float *ph = &rh.x, *pl = &rl.x, *qh = &ih.x, *ql = &il.x;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float2 u = v[4 * q + t];
                    ph[t] = tf32_round(u.x);
                    qh[t] = tf32_round(u.y);
                    pl[t] = tf32_round(u.x - ph[t]);
                    ql[t] = tf32_round(u.y - qh[t]);
                }
                float *dst = st + (v_kc ? soffB[q] : soffA[q]);
                *(float4 *)dst = rh;
                *(float4 *)(dst + kArr) = rl;
                *(float4 *)(dst + 2 * kArr) = ih;
                *(float4 *)(dst + 3 * kArr) = il;
            }
            // the stores, seen by the tensor cores' (async) proxy, then one arrival per warp
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&full[s]));
            if (c + 2 < n_chunks) load_chunk(v, v_kc);
            return true;
        };
        float2 va[16], vb[16];
        bool ka = false, kb = false;
        if (n_chunks > 0) {
            set_pair(p0);
            load_chunk(va, ka);
            if (n_chunks > 1) load_chunk(vb, kb);
        }
        for (int64_t c = 0; c < n_chunks; c += 2) {
            if (!produce(c, va, ka)) break;
            if (c + 1 < n_chunks && !produce(c + 1, vb, kb)) break;
        }
    } else if (warp == kMmaWarp) {
        // ---- one thread issues the MMAs -------------------------------------
        if (lane == 0) {
            constexpr uint32_t kLbo = 128, kSbo = (kKc / 4) * 128;
            const uint32_t id_pos = tf32_idesc(kM, kNt, false), id_neg = tf32_idesc(kM, kNt, true);
            int64_t blk = 0, bi = 0;
            bool ok = true;
            for (int64_t c = 0; c < n_chunks && ok; ++c) {
                const int s = (int)(c % kStages);
                const int acc = (int)(bi & 1);
                // a new block: its accumulator must have been drained (block bi - 2)
                if (blk == 0 && bi >= 2 && !mbar_wait(smem_u32(&acc_empty[acc]), (uint32_t)(((bi >> 1) - 1) & 1), vstop))
                    ok = false;
                if (ok && !mbar_wait(smem_u32(&full[s]), (uint32_t)((c / kStages) & 1), vstop)) ok = false;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(256 * acc);
                const float *st = smem + s * 8 * kArr;
                const uint32_t sa = smem_u32(st), sb = smem_u32(st + 4 * kArr);
#pragma unroll
                for (int ks = 0; ks < kKc / 8; ++ks) {
                    const uint32_t koff = (uint32_t)ks * 2 * kLbo;
                    auto A = [&](int q) { return smem_desc(sa + q * kArr * 4 + koff, kLbo, kSbo); };
                    auto B = [&](int q) { return smem_desc(sb + q * kArr * 4 + koff, kLbo, kSbo); };
                    const uint32_t first = (blk == 0 && ks == 0) ? 0u : 1u;
                    // Re += Ar Br + Ai Bi (three TF32 pieces each)
                    mma_tf32(d, A(0), B(0), id_pos, first);
                    mma_tf32(d, A(0), B(1), id_pos, 1u);
                    mma_tf32(d, A(1), B(0), id_pos, 1u);
                    mma_tf32(d, A(2), B(2), id_pos, 1u);
                    mma_tf32(d, A(2), B(3), id_pos, 1u);
                    mma_tf32(d, A(3), B(2), id_pos, 1u);
                    // Im += Ai Br - Ar Bi
                    mma_tf32(d + kNt, A(2), B(0), id_pos, first);
                    mma_tf32(d + kNt, A(2), B(1), id_pos, 1u);
                    mma_tf32(d + kNt, A(3), B(0), id_pos, 1u);
                    mma_tf32(d + kNt, A(0), B(2), id_neg, 1u);
                    mma_tf32(d + kNt, A(0), B(3), id_neg, 1u);
                    mma_tf32(d + kNt, A(1), B(2), id_neg, 1u);
                }
                mma_commit(smem_u32(&empty[s]));   // the stage is free once these are done
                if (++blk == chunks_per_block || c + 1 == n_chunks) {
                    mma_commit(smem_u32(&acc_full[acc]));   // the block's sums are ready
                    blk = 0;
                    ++bi;
                }
            }
            if (!ok) {
                atomicOr(a.status, 4);
                stop = 1;
            }
            // every MMA issued has completed before TMEM is released
            mma_commit(smem_u32(&done));
            if (!mbar_wait(smem_u32(&done), 0u, vstop) && ok) {
                atomicOr(a.status, 4);
                stop = 1;
            }
        }
        __syncwarp();
    } else {
        // ---- drain: each finished block's FP32 sums into the CTA's two-word totals
        // warp w reads TMEM lanes 32 (w % 4).. (the tile's rows), all 256 columns
        const int quarter = warp & 3, row = 32 * quarter + lane;
        for (int64_t bi = 0; bi < n_blocks; ++bi) {
            const int acc = (int)(bi & 1);
            if (!mbar_wait(smem_u32(&acc_full[acc]), (uint32_t)((bi >> 1) & 1), vstop, 2000)) {
                if (lane == 0) atomicOr(a.status, 4);
                stop = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int c0 = 0; c0 < 2 * kNt; c0 += 32) {
                float tv[32];
                tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(256 * acc + c0), tv);
                const int part = c0 / kNt;   // 0: Re, 1: Im
                float *hi = slot + (size_t)part * kNt * kM, *lo = slot + (size_t)(2 + part) * kNt * kM;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const size_t o = (size_t)(c0 - part * kNt + i) * kM + row;
                    float h = hi[o], l = lo[o];
                    two_sum_add(h, l, tv[i]);
                    hi[o] = h;
                    lo[o] = l;
                }
            }
            // this warp's reads of the accumulator are complete: hand it back
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[acc]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// rho1(x, x') = scale * sum over the splits of (hi + lo), in FP64, read
// from tile (x / 128, x' / 128) of the upper triangle, or conjugated from
// its transpose below the diagonal.
__global__ void __launch_bounds__(256) rho1_tc_reduce_kernel(const float *__restrict__ slots, int tiles, int splits,
                                                             int N, double scale, double *__restrict__ rho) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * N) return;
    int x = (int)(i / N), xp = (int)(i - (int64_t)x * N);
    const bool lower = x / kM > xp / kNt;
    if (lower) {
        const int t = x;
        x = xp;
        xp = t;
    }
    const int ty = x / kM, tx = xp / kNt, row = x - ty * kM, col = xp - tx * kNt;
    const int n_up = tiles * (tiles + 1) / 2;
    const int id = ty * tiles - ty * (ty - 1) / 2 + (tx - ty);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < splits; ++s) {
        const float *slot = slots + (size_t)(s * n_up + id) * (2 * 2 * kNt * kM);
        const size_t o = (size_t)col * kM + row;
        re += (double)slot[o] + (double)slot[2 * kNt * kM + o];
        im += (double)slot[kNt * kM + o] + (double)slot[3 * kNt * kM + o];
    }
    rho[2 * i] += scale * re;
    rho[2 * i + 1] += scale * (lower ? -im : im);
}

}  // namespace

bool one_body_density_tc_supported(const ctqw_hamiltonian *h, int dtype) {
    if (dtype != CTQW_C64 || h->m < 2) return false;
    for (int N : h->group_N)
        if (N % 16 != 0 || N > 2048) return false;
    return true;
}

int launch_one_body_density_tc(const ctqw_hamiltonian *h, const void *psi, double *rho, cudaStream_t s) {
    const size_t smem = sizeof(float) * kStages * 8 * kArr;
    CTQW_CUDA_TRY(cudaFuncSetAttribute((const void *)rho1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    int sms = 0, dev = 0;
    CTQW_CUDA_TRY(cudaGetDevice(&dev));
    CTQW_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int off = 0;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g], cnt = h->group_count[g];
        int64_t n_k = 1;
        for (int j = 1; j < h->m; ++j) n_k *= N;
        const int tiles = (N + kM - 1) / kM, n_up = tiles * (tiles + 1) / 2;
        const int pairs = cnt * h->m;
        int splits = std::max(1, sms / n_up);
        splits = std::min(splits, pairs);
        const int pps = (pairs + splits - 1) / splits;
        splits = (pairs + pps - 1) / pps;
        const size_t slot_floats = (size_t)n_up * splits * (2 * 2 * kNt * kM);
        float *slots = nullptr;
        CTQW_CUDA_TRY(ctqw_malloc_async((void **)&slots, slot_floats * sizeof(float), s));
        int st = CTQW_OK;
        const cudaError_t em = cudaMemsetAsync(slots, 0, slot_floats * sizeof(float), s);
        if (em != cudaSuccess) st = ctqw_cuda_fail(em, "memset of the rho1 slots");
        if (st == CTQW_OK) {
            TcArgs a;
            a.tab = real_table(h);
            a.list = h->by_group_d + off;
            a.psi = (const float2 *)psi;
            a.slots = slots;
            a.status = h->status_d;
            a.N = N;
            a.m = h->m;
            a.pairs = pairs;
            a.pairs_per_split = pps;
            a.n_k = n_k;
            a.tiles = tiles;
            rho1_tc_kernel<<<dim3((unsigned)n_up, (unsigned)splits), kThreads, smem, s>>>(a);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = ctqw_cuda_fail(e, "rho1 tensor-core launch");
        }
        if (st == CTQW_OK) {
            const int64_t n = (int64_t)N * N;
            rho1_tc_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
                slots, tiles, splits, N, 1.0 / ((double)cnt * h->m), rho + 2 * h->joint_off[g]);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = ctqw_cuda_fail(e, "rho1 reduction launch");
        }
        cudaFreeAsync(slots, s);
        if (st != CTQW_OK) return st;
        off += cnt;
    }
    return CTQW_OK;
}
