// Per-term propagation kernels: the structure of Algorithms 2 and 3 with
// one launch per Taylor term (or RK4 stage) over all realizations at once
// (the realization x node loop collapsed into one grid, Sec. 2.2).  These
// are the plain path: every term streams Phi and the running sum through HBM.
#include "ctqw_internal.cuh"
#include "stencil.cuh"

namespace {

// Phi^(j) = -(i dt/j) H Phi^(j-1);  acc = (first ? psi : acc) + Phi^(j).
template <typename T, int M>
__global__ void __launch_bounds__(256) taylor_term_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                          const T *__restrict__ eps,
                                                          const T *__restrict__ J,
                                                          const cplx_t<T> *__restrict__ in,
                                                          cplx_t<T> *__restrict__ out,
                                                          const cplx_t<T> *__restrict__ psi,
                                                          cplx_t<T> *__restrict__ acc, T coef,
                                                          int first) {
    Site<M> p;
    if (!site_of<M>(tab, list, p)) return;
    const int64_t s = p.s;
    const int64_t base = tab.st_off[p.r];
    const int64_t po = tab.par_off[p.r];
    cplx_t<T> y = apply_h<T, M>(in + base, s, p.x, p.N, eps + po, J + po, (T)tab.U);
    cplx_t<T> phi = mk<T>(coef * y.y, -coef * y.x);   // -(i coef) y
    out[base + s] = phi;
    cplx_t<T> a = first ? psi[base + s] : acc[base + s];
    acc[base + s] = mk<T>(a.x + phi.x, a.y + phi.y);
}

// k = -i H in;  next = psi + a k (when next != null);  acc = (first ? psi : acc) + b k.
template <typename T, int M>
__global__ void __launch_bounds__(256) rk4_stage_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                        const T *__restrict__ eps,
                                                        const T *__restrict__ J,
                                                        const cplx_t<T> *__restrict__ in,
                                                        cplx_t<T> *__restrict__ next,
                                                        const cplx_t<T> *__restrict__ psi,
                                                        cplx_t<T> *__restrict__ acc, T a, T b,
                                                        int first) {
    Site<M> p;
    if (!site_of<M>(tab, list, p)) return;
    const int64_t s = p.s;
    const int64_t base = tab.st_off[p.r];
    const int64_t po = tab.par_off[p.r];
    cplx_t<T> y = apply_h<T, M>(in + base, s, p.x, p.N, eps + po, J + po, (T)tab.U);
    cplx_t<T> k = mk<T>(y.y, -y.x);   // -i H in
    cplx_t<T> q = psi[base + s];
    if (next) next[base + s] = mk<T>(q.x + a * k.x, q.y + a * k.y);
    cplx_t<T> c = first ? q : acc[base + s];
    acc[base + s] = mk<T>(c.x + b * k.x, c.y + b * k.y);
}

}  // namespace

int launch_taylor_term(const ctqw_hamiltonian *h, int dtype, const void *in, void *out,
                       const void *psi, void *acc, double coef, int first, cudaStream_t s) {
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        if (dtype == CTQW_C64) {
            auto k = h->m == 2 ? taylor_term_kernel<float, 2> : taylor_term_kernel<float, 3>;
            k<<<grid, block, 0, s>>>(t, list, h->eps32, h->J32, (const float2 *)in, (float2 *)out,
                                     (const float2 *)psi, (float2 *)acc, (float)coef, first);
        } else {
            auto k = h->m == 2 ? taylor_term_kernel<double, 2> : taylor_term_kernel<double, 3>;
            k<<<grid, block, 0, s>>>(t, list, h->eps64, h->J64, (const double2 *)in, (double2 *)out,
                                     (const double2 *)psi, (double2 *)acc, coef, first);
        }
    });
}

int launch_rk4_stage(const ctqw_hamiltonian *h, int dtype, const void *in, void *next,
                     const void *psi, void *acc, double a, double b, int first, cudaStream_t s) {
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        if (dtype == CTQW_C64) {
            auto k = h->m == 2 ? rk4_stage_kernel<float, 2> : rk4_stage_kernel<float, 3>;
            k<<<grid, block, 0, s>>>(t, list, h->eps32, h->J32, (const float2 *)in, (float2 *)next,
                                     (const float2 *)psi, (float2 *)acc, (float)a, (float)b, first);
        } else {
            auto k = h->m == 2 ? rk4_stage_kernel<double, 2> : rk4_stage_kernel<double, 3>;
            k<<<grid, block, 0, s>>>(t, list, h->eps64, h->J64, (const double2 *)in, (double2 *)next,
                                     (const double2 *)psi, (double2 *)acc, a, b, first);
        }
    });
}

// ---------------------------------------------------------------- FP32 per-term path
// Horner form of the same order-K polynomial (Sec. 2.3), one launch per stage:
//   w_K = psi + (A/K) psi,  w_j = psi + (A/j) w_{j+1},  psi(t+dt) = psi + A w_2,
// A = -i dt H.  In FP32 the forward sum drops every term below half an ulp
// of the running sum, which truncates the series; Horner keeps each term at
// its own scale.  The final stage adds A w_2 to the state with its rounding
// error carried in a second FP32 word (lo).
namespace {

template <int M>
__global__ void __launch_bounds__(256) horner_stage_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                           const float *__restrict__ eps,
                                                           const float *__restrict__ J,
                                                           const float2 *__restrict__ in,
                                                           const float2 *__restrict__ psi,
                                                           float2 *__restrict__ out, float coef) {
    Site<M> p;
    if (!site_of<M>(tab, list, p)) return;
    const int64_t s = p.s;
    const int64_t base = tab.st_off[p.r];
    const int64_t po = tab.par_off[p.r];
    const float2 y = apply_h<float, M>(in + base, s, p.x, p.N, eps + po, J + po, (float)tab.U);
    const float2 q = psi[base + s];
    out[base + s] = make_float2(fmaf(coef, y.y, q.x), fmaf(-coef, y.x, q.y));   // q + coef (-i) y
}

template <int M>
__global__ void __launch_bounds__(256) horner_final_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                           const float *__restrict__ eps,
                                                           const float *__restrict__ J,
                                                           const float2 *__restrict__ w2,
                                                           float2 *__restrict__ psi,
                                                           float2 *__restrict__ lo, float dt) {
    Site<M> p;
    if (!site_of<M>(tab, list, p)) return;
    const int64_t s = p.s;
    const int64_t base = tab.st_off[p.r];
    const int64_t po = tab.par_off[p.r];
    const float2 y = apply_h<float, M>(w2 + base, s, p.x, p.N, eps + po, J + po, (float)tab.U);
    const float sx = dt * y.y, sy = -dt * y.x;   // -i dt H w2
    float2 h = psi[base + s], l = lo[base + s];
    // TwoSum then FastTwoSum per component
    auto add = [](float &hi, float &lw, float v) {
        const float t = __fadd_rn(hi, v);
        const float bb = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(v, bb));
        const float e = __fadd_rn(err, lw);
        const float h2 = __fadd_rn(t, e);
        lw = __fsub_rn(e, __fsub_rn(h2, t));
        hi = h2;
    };
    add(h.x, l.x, sx);
    add(h.y, l.y, sy);
    psi[base + s] = h;
    lo[base + s] = l;
}

// The same two kernels for three particles, walking along x1: a block owns
// kRows3 slabs x1, one x2 and up to 256 x3 of one realization, and each
// thread keeps w at x1 - 1, x1, x1 + 1 of its (x2, x3) in registers (the
// next slab's value loaded one slab ahead), takes the x3 neighbours from
// the adjacent lanes and the x2 neighbours from L2: per amplitude 4 loads
// of w and psi against 8 for the one-amplitude-per-thread kernels.  The
// stencil is that of apply_h, term for term.
constexpr int kRows3 = 32;

template <bool FINAL>
__global__ void __launch_bounds__(256) horner3_rows_kernel(RealTable tab, const int32_t *__restrict__ list,
                                                           const float *__restrict__ eps,
                                                           const float *__restrict__ J,
                                                           const float2 *__restrict__ in,
                                                           const float2 *__restrict__ psi,
                                                           float2 *__restrict__ out, float2 *__restrict__ lo,
                                                           float coef, int x3_chunks) {
    const int r = list[blockIdx.z];
    const int N = tab.N[r];
    const int x3c = blockIdx.x % x3_chunks, x1c = blockIdx.x / x3_chunks;
    const int x3 = x3c * blockDim.x + threadIdx.x, x2 = blockIdx.y;
    const bool live = x3 < N;
    const int lane = threadIdx.x & 31;
    const int x1_0 = x1c * kRows3, rows = min(kRows3, N - x1_0);
    const int64_t base = tab.st_off[r];
    const int64_t po = tab.par_off[r];
    const float2 *w = in + base;
    const float2 *q_ = FINAL ? nullptr : psi + base;   // the stage's psi (not read by the final stage)
    const float *e_ = eps + po, *j_ = J + po;
    const float U = (float)tab.U;
    auto wrap = [N](int x) { return x < 0 ? x + N : (x >= N ? x - N : x); };
    const int x2l = wrap(x2 - 1), x2r = wrap(x2 + 1), x3l = wrap(x3 - 1), x3r = wrap(x3 + 1);
    const float e2 = e_[x2], jl2 = j_[x2l], jr2 = j_[x2];
    const float e3 = live ? e_[x3] : 0.f, jl3 = live ? j_[x3l] : 0.f, jr3 = live ? j_[x3] : 0.f;
    const bool own_l = lane > 0 && x3 > 0, own_r = lane < 31 && x3 + 1 < N;
    auto at = [&](int x1, int xx2, int xx3) { return ((int64_t)x1 * N + xx2) * N + xx3; };
    const float2 z = make_float2(0.f, 0.f);
    float2 w_up = z, w_c = z, w_dn = z;
    if (live) {
        w_up = w[at(wrap(x1_0 - 1), x2, x3)];
        w_c = w[at(x1_0, x2, x3)];
        w_dn = w[at(wrap(x1_0 + 1), x2, x3)];
    }
    for (int i = 0; i < rows; ++i) {
        const int x1 = x1_0 + i;
        const int64_t sidx = at(x1, x2, x3);
        float2 w_nn = z;
        if (live && i + 1 < rows) w_nn = w[at(wrap(x1 + 2), x2, x3)];
        float2 a3l = make_float2(__shfl_sync(0xffffffffu, w_c.x, (lane + 31) & 31),
                                 __shfl_sync(0xffffffffu, w_c.y, (lane + 31) & 31));
        float2 a3r = make_float2(__shfl_sync(0xffffffffu, w_c.x, (lane + 1) & 31),
                                 __shfl_sync(0xffffffffu, w_c.y, (lane + 1) & 31));
        if (live) {
            if (!own_l) a3l = w[sidx - x3 + x3l];
            if (!own_r) a3r = w[sidx - x3 + x3r];
            const float2 a2l = w[sidx + (int64_t)(x2l - x2) * N], a2r = w[sidx + (int64_t)(x2r - x2) * N];
            const int x1m = wrap(x1 - 1);
            float v = 0.f;
            v += e_[x1];
            v += e2;
            v += e3;
            v += U * (float)((x1 == x2) + (x1 == x3) + (x2 == x3));
            float yr = v * w_c.x, yi = v * w_c.y;
            yr -= jl3 * a3l.x + jr3 * a3r.x;
            yi -= jl3 * a3l.y + jr3 * a3r.y;
            yr -= jl2 * a2l.x + jr2 * a2r.x;
            yi -= jl2 * a2l.y + jr2 * a2r.y;
            const float jl1 = j_[x1m], jr1 = j_[x1];
            yr -= jl1 * w_up.x + jr1 * w_dn.x;
            yi -= jl1 * w_up.y + jr1 * w_dn.y;
            if (!FINAL) {
                const float2 q = q_[sidx];
                out[base + sidx] = make_float2(fmaf(coef, yi, q.x), fmaf(-coef, yr, q.y));   // q + coef (-i) y
            } else {
                const float sx = coef * yi, sy = -coef * yr;   // -i dt H w2
                float2 hh = out[base + sidx], l = lo[base + sidx];
                auto add = [](float &hi, float &lw, float v2) {
                    const float t = __fadd_rn(hi, v2);
                    const float bb = __fsub_rn(t, hi);
                    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(v2, bb));
                    const float e = __fadd_rn(err, lw);
                    const float h2 = __fadd_rn(t, e);
                    lw = __fsub_rn(e, __fsub_rn(h2, t));
                    hi = h2;
                };
                add(hh.x, l.x, sx);
                add(hh.y, l.y, sy);
                out[base + sidx] = hh;
                lo[base + sidx] = l;
            }
        }
        w_up = w_c;
        w_c = w_dn;
        w_dn = w_nn;
    }
}

// One launch per size group of horner3_rows_kernel: (x1 chunks x x3 chunks, x2, realizations).
template <bool FINAL>
int launch_horner3_rows(const ctqw_hamiltonian *h, const void *in, const void *psi, void *out, void *lo, double coef,
                        cudaStream_t s) {
    RealTable t = real_table(h);
    int off = 0;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g], cnt = h->group_count[g];
        const int tx = N >= 256 ? 256 : ((N + 31) / 32) * 32;
        const int x3_chunks = (N + tx - 1) / tx;
        const unsigned gx = (unsigned)(((N + kRows3 - 1) / kRows3) * x3_chunks);
        for (int done = 0; done < cnt; done += 65535) {
            const int part = cnt - done < 65535 ? cnt - done : 65535;
            horner3_rows_kernel<FINAL><<<dim3(gx, (unsigned)N, (unsigned)part), tx, 0, s>>>(
                t, h->by_group_d + off + done, h->eps32, h->J32, (const float2 *)in, (const float2 *)psi,
                (float2 *)out, (float2 *)lo, (float)coef, x3_chunks);
            CTQW_CUDA_TRY(cudaGetLastError());
        }
        off += cnt;
    }
    return CTQW_OK;
}

}  // namespace

int launch_horner_stage(const ctqw_hamiltonian *h, const void *in, const void *psi, void *out,
                        double coef, cudaStream_t s) {
    if (h->m == 3) return launch_horner3_rows<false>(h, in, psi, out, nullptr, coef, s);
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        horner_stage_kernel<2><<<grid, block, 0, s>>>(t, list, h->eps32, h->J32, (const float2 *)in,
                                                      (const float2 *)psi, (float2 *)out, (float)coef);
    });
}

int launch_horner_final(const ctqw_hamiltonian *h, const void *w2, void *psi, void *lo, double dt,
                        cudaStream_t s) {
    if (h->m == 3) return launch_horner3_rows<true>(h, w2, nullptr, psi, lo, dt, s);
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        horner_final_kernel<2><<<grid, block, 0, s>>>(t, list, h->eps32, h->J32, (const float2 *)w2,
                                                      (float2 *)psi, (float2 *)lo, (float)dt);
    });
}
