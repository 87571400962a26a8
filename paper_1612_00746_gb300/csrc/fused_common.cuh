// Device helpers shared by the fused propagation kernels: cluster rank and
// barrier, shared-memory addressing across the cluster, mbarrier arrivals and
// bounded waits, st.async pushes into a neighbour CTA, and the compensated
// (TwoSum / FastTwoSum) state update.
#pragma once

#include <cstdint>

#include "ctqw_internal.cuh"

namespace fused {

// (static: each translation unit keeps its own copy)

static __device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Full cluster barrier (outside the stage loop: at the start and the end of a
// kernel, and around a realization hand-out).
static __device__ __forceinline__ void cluster_barrier() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

static __device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
static __device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// 32-bit load from the shared memory of a CTA of the cluster (a map_rank address).
static __device__ __forceinline__ int ld_shared_cluster_s32(uint32_t raddr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(raddr) : "memory");
    return v;
}

static __device__ __forceinline__ void mbar_init(uint32_t mb, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
}

static __device__ __forceinline__ void mbar_expect_tx(uint32_t mb, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
                 : "memory");
}

// Arrival + expected bytes on two mbarriers, from the threads with flag != 0 only (no branch).
static __device__ __forceinline__ void mbar_expect_tx2_if(uint32_t mb0, uint32_t mb1, uint32_t bytes, int flag) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
                 "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %2;\n\t"
                 "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%1], %2;\n\t}"
                 ::"r"(mb0), "r"(mb1), "r"(bytes), "r"(flag) : "memory");
}

// 16-byte store into another CTA's shared memory, counted on its mbarrier.
static __device__ __forceinline__ void st_async16(uint32_t raddr, float4 v, uint32_t rmbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
                 ::"r"(raddr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rmbar) : "memory");
}

static __device__ __forceinline__ bool mbar_try_wait(uint32_t mb, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(mb), "r"(parity) : "memory");
    return ok != 0;
}

static __device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of parity `parity` of mbarrier `mb`, giving up after
// limit_ns of global time: then the status word is set and false returned.
static __device__ __noinline__ bool mbar_wait_slow(uint32_t mb, uint32_t parity,
                                            unsigned long long limit_ns, int *status) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(mb, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > limit_ns) {
            atomicOr(status, 1);
            return false;
        }
    }
}

static __device__ __forceinline__ bool mbar_wait_bounded(uint32_t mb, uint32_t parity,
                                                  unsigned long long limit_ns, int *status) {
    return mbar_try_wait(mb, parity) || mbar_wait_slow(mb, parity, limit_ns, status);
}

static __device__ __forceinline__ float2 ffma2(float a, float2 b, float2 c) {
    return __ffma2_rn(make_float2(a, a), b, c);
}

// (re, im) pair moved between lanes as one 64-bit value.
static __device__ __forceinline__ float2 shfl2(float2 v, int src) {
    const unsigned long long u = __shfl_sync(0xffffffffu, *reinterpret_cast<unsigned long long *>(&v), src);
    return *reinterpret_cast<const float2 *>(&u);
}

// hi + lo + s rounded back into (hi, lo): TwoSum then FastTwoSum.
static __device__ __forceinline__ void compensated_add(float &hi, float &lo, float s) {
    const float t = __fadd_rn(hi, s);
    const float bb = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(s, bb));
    const float l = __fadd_rn(err, lo);
    const float h2 = __fadd_rn(t, l);
    lo = __fsub_rn(l, __fsub_rn(h2, t));
    hi = h2;
}

// The same on an (re, im) pair with FP32x2 operations (x - y as fma(y, -1, x),
// which rounds exactly like the subtraction).
static __device__ __forceinline__ void compensated_add2(float2 &hi, float2 &lo, float2 s) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 t = __fadd2_rn(hi, s);
    const float2 bb = __ffma2_rn(hi, m1, t);
    const float2 tb = __ffma2_rn(bb, m1, t);
    const float2 err = __fadd2_rn(__ffma2_rn(tb, m1, hi), __ffma2_rn(bb, m1, s));
    const float2 l = __fadd2_rn(err, lo);
    const float2 h2 = __fadd2_rn(t, l);
    lo = __ffma2_rn(__ffma2_rn(t, m1, h2), m1, l);
    hi = h2;
}

static __device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Butterfly sum over the warp in FP64 (every lane gets the total).
static __device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the warp of V values per lane at once (V a power of two <= 32),
// in FP64: the first log2 V butterfly steps each halve the values a lane
// keeps (it sends the half its partner keeps), the remaining steps are a
// plain butterfly.  Returns, in every lane, the warp total of value
// (lane >> (5 - log2 V)) & (V - 1); that costs 2V - 1 + (5 - log2 V) adds
// per lane against 5 V for V separate butterflies.
template <int V>
static __device__ __forceinline__ double warp_sum_multi_d(double (&v)[V], int lane) {
    static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V must be a power of two <= 32");
#pragma unroll
    for (int o = 16, n = V; n > 1; o >>= 1, n >>= 1) {
        const bool upper = (lane & o) != 0;   // keeps the upper half of the values
#pragma unroll
        for (int q = 0; q < n / 2; ++q) {
            const double send = upper ? v[q] : v[q + n / 2];
            const double keep = upper ? v[q + n / 2] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    double t = v[0];
#pragma unroll
    for (int o = 16 / V; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// |c|^2 of an FP32 amplitude in FP32 (FP32 products; the sums that use it
// run in FP64).
static __device__ __forceinline__ float abs2_f(float2 c) { return fmaf(c.x, c.x, c.y * c.y); }

// Re(conj(c) y) of two FP32 amplitudes in FP32.
static __device__ __forceinline__ float re_dot_f(float2 c, float2 y) { return fmaf(c.x, y.x, c.y * y.y); }

}  // namespace fused
