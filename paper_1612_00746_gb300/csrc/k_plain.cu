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

}  // namespace

int launch_horner_stage(const ctqw_hamiltonian *h, const void *in, const void *psi, void *out,
                        double coef, cudaStream_t s) {
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        auto k = h->m == 2 ? horner_stage_kernel<2> : horner_stage_kernel<3>;
        k<<<grid, block, 0, s>>>(t, list, h->eps32, h->J32, (const float2 *)in, (const float2 *)psi,
                                 (float2 *)out, (float)coef);
    });
}

int launch_horner_final(const ctqw_hamiltonian *h, const void *w2, void *psi, void *lo, double dt,
                        cudaStream_t s) {
    RealTable t = real_table(h);
    return for_each_group(h, [&](dim3 grid, dim3 block, const int32_t *list) {
        auto k = h->m == 2 ? horner_final_kernel<2> : horner_final_kernel<3>;
        k<<<grid, block, 0, s>>>(t, list, h->eps32, h->J32, (const float2 *)w2, (float2 *)psi,
                                 (float2 *)lo, (float)dt);
    });
}
