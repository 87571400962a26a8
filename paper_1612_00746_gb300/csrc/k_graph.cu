// Kernels of the graph path (Sec. 2: a q-dimensional lattice of N nodes, or
// a general graph where each node has its own number of links; Algorithms 2
// and 3 then read the neighbours of every row from a topology shared by all
// realizations).
//
// H = sum_j H1 acting on particle j + U * #coinciding pairs, with
// H1 = diag(eps) - sum_links J_e (|u_e><v_e| + h.c.).  The amplitude at flat
// index s (coordinates x_1..x_m, x_m fastest, strides S_j = N^(m-1-j)) gets
//   (H a)(s) = (sum_j eps[x_j] + U pairs) a(s) - sum_j sum_{k in row x_j} w_k a(s + (col_k - x_j) S_j),
// the CSR row of node x_j giving the neighbours col_k and their hoppings w_k.
// Realizations are the fastest index of every array (psi[s][r], eps[i][r],
// w[k][r], stride Rp a multiple of 4).  A thread owns four realizations of
// one amplitude in two adjacent pairs, ra = b + 2 l and rb = ra + 2 X (lane
// l of X lanes, b the first realization of the warp's group of 4X), so each
// 16-byte complex-pair load is contiguous across the warp; threadIdx.y walks
// amplitudes.  The CSR lookups and the index arithmetic of a neighbour are
// shared by four amplitudes and uniform across the warp.
#include <algorithm>

#include "graph_internal.cuh"
#include "stencil.cuh"

namespace {

constexpr int kThreads = 256;

// Four realizations (pairs ra, ra+1 and rb, rb+1) of one complex amplitude
// or one real parameter; p points at realization 0 of the row.
template <typename T> struct C4 { T re[4], im[4]; };
template <typename T> struct R4 { T v[4]; };

// The thread's two pairs: offsets ra, rb and whether the second pair exists.
struct Pairs {
    int ra, rb;
    bool vb;
};

__device__ __forceinline__ void put2(C4<float> &c, int h, float4 u) {
    c.re[2 * h] = u.x; c.im[2 * h] = u.y; c.re[2 * h + 1] = u.z; c.im[2 * h + 1] = u.w;
}
__device__ __forceinline__ C4<float> ld_c4(const float2 *__restrict__ p, const Pairs &q) {
    C4<float> c;
    put2(c, 0, __ldg(reinterpret_cast<const float4 *>(p + q.ra)));
    put2(c, 1, __ldg(reinterpret_cast<const float4 *>(p + q.rb)));
    return c;
}
__device__ __forceinline__ C4<double> ld_c4(const double2 *__restrict__ p, const Pairs &q) {
    const double2 a = __ldg(p + q.ra), b = __ldg(p + q.ra + 1), c = __ldg(p + q.rb), d = __ldg(p + q.rb + 1);
    return C4<double>{{a.x, b.x, c.x, d.x}, {a.y, b.y, c.y, d.y}};
}
// the same through the coherent path (arrays the kernel also writes)
__device__ __forceinline__ C4<float> ld_c4_rw(const float2 *p, const Pairs &q) {
    C4<float> c;
    put2(c, 0, *reinterpret_cast<const float4 *>(p + q.ra));
    put2(c, 1, *reinterpret_cast<const float4 *>(p + q.rb));
    return c;
}
__device__ __forceinline__ C4<double> ld_c4_rw(const double2 *p, const Pairs &q) {
    const double2 a = p[q.ra], b = p[q.ra + 1], c = p[q.rb], d = p[q.rb + 1];
    return C4<double>{{a.x, b.x, c.x, d.x}, {a.y, b.y, c.y, d.y}};
}
__device__ __forceinline__ void st_c4(float2 *p, const Pairs &q, const C4<float> &c) {
    *reinterpret_cast<float4 *>(p + q.ra) = make_float4(c.re[0], c.im[0], c.re[1], c.im[1]);
    if (q.vb) *reinterpret_cast<float4 *>(p + q.rb) = make_float4(c.re[2], c.im[2], c.re[3], c.im[3]);
}
__device__ __forceinline__ void st_c4(double2 *p, const Pairs &q, const C4<double> &c) {
    p[q.ra] = make_double2(c.re[0], c.im[0]);
    p[q.ra + 1] = make_double2(c.re[1], c.im[1]);
    if (q.vb) {
        p[q.rb] = make_double2(c.re[2], c.im[2]);
        p[q.rb + 1] = make_double2(c.re[3], c.im[3]);
    }
}
__device__ __forceinline__ R4<float> ld_r4(const float *__restrict__ p, const Pairs &q) {
    const float2 a = __ldg(reinterpret_cast<const float2 *>(p + q.ra)), b = __ldg(reinterpret_cast<const float2 *>(p + q.rb));
    return R4<float>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ R4<double> ld_r4(const double *__restrict__ p, const Pairs &q) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p + q.ra)), b = __ldg(reinterpret_cast<const double2 *>(p + q.rb));
    return R4<double>{{a.x, a.y, b.x, b.y}};
}

template <int M>
__device__ __forceinline__ void graph_coords(int s, int N, int (&x)[M], int (&S)[M]) {
    int stride = 1;
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {
        const int q = s / N;
        x[j] = s - q * N;
        s = q;
        S[j] = stride;
        stride *= N;
    }
}

// (H a)(s) for the thread's four realizations; Rp is the realization stride.
template <typename T, int M>
__device__ __forceinline__ C4<T> graph_apply_h4(const cplx_t<T> *a, int64_t Rp, int s, const Pairs &pr,
                                                const int (&x)[M], const int (&S)[M],
                                                const int32_t *__restrict__ row_ptr,
                                                const int32_t *__restrict__ col, const T *__restrict__ w,
                                                const T *__restrict__ eps, T U) {
    int pairs = 0;
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
        for (int l = j + 1; l < M; ++l) pairs += (x[j] == x[l]);
    R4<T> v;
#pragma unroll
    for (int q = 0; q < 4; ++q) v.v[q] = U * T(pairs);
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const R4<T> e = ld_r4(eps + (int64_t)x[j] * Rp, pr);
#pragma unroll
        for (int q = 0; q < 4; ++q) v.v[q] += e.v[q];
    }
    const C4<T> c = ld_c4(a + (int64_t)s * Rp, pr);
    C4<T> y;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        y.re[q] = v.v[q] * c.re[q];
        y.im[q] = v.v[q] * c.im[q];
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const int k0 = row_ptr[x[j]], k1 = row_ptr[x[j] + 1];
        const int64_t step = (int64_t)S[j] * Rp;                       // one node along coordinate j
        const cplx_t<T> *base = a + (int64_t)(s - x[j] * S[j]) * Rp;   // coordinate j at node 0
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const R4<T> t = ld_r4(w + (int64_t)k * Rp, pr);
            const C4<T> n = ld_c4(base + (int64_t)col[k] * step, pr);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                y.re[q] -= t.v[q] * n.re[q];
                y.im[q] -= t.v[q] * n.im[q];
            }
        }
    }
    return y;
}

// Amplitude and realization pairs of this thread, false past the ends.  A
// second pair past the end repeats the first (its loads stay in bounds) and
// is not stored.
__device__ __forceinline__ bool graph_site4(const GraphView &g, int &s, Pairs &pr) {
    s = blockIdx.x * blockDim.y + threadIdx.y;
    const int b = g.r_begin + 4 * blockIdx.y * blockDim.x;
    pr.ra = b + 2 * threadIdx.x;
    pr.rb = pr.ra + 2 * blockDim.x;
    pr.vb = pr.rb < g.r_end;
    if (!pr.vb) pr.rb = pr.ra;
    return s < g.D && pr.ra < g.r_end;
}

__device__ __forceinline__ double graph_param(double mean, double hw, double u, int round_f32) {
    double v = __dadd_rn(mean, __dmul_rn(hw, __dadd_rn(__dmul_rn(2.0, u), -1.0)));
    if (round_f32) v = (double)__double2float_rn(v);
    return v;
}

__global__ void graph_build_params_kernel(GraphView g, int E, const int32_t *__restrict__ link,
                                          const double *__restrict__ u_eps,
                                          const double *__restrict__ u_J, double eps_hw, double J_hw,
                                          double J0, int round_f32, float *eps32, double *eps64,
                                          float *w32, double *w64, double *J64) {
    const int64_t R = g.R, Rp = g.Rp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t t = t0; t < (int64_t)g.N * Rp; t += stride) {   // eps[i][r] from u_eps[r][i]
        const int64_t i = t / Rp, r = t - i * Rp;
        const double e = r < R ? graph_param(0.0, eps_hw, u_eps[r * g.N + i], round_f32) : 0.0;
        eps64[t] = e;
        eps32[t] = (float)e;
    }
    for (int64_t t = t0; t < (int64_t)E * R; t += stride)        // J[r][e] as drawn
        J64[t] = graph_param(J0, J_hw, u_J[t], round_f32);
    for (int64_t t = t0; t < (int64_t)g.nnz * Rp; t += stride) {  // w[k][r] = J[r][link[k]]
        const int64_t k = t / Rp, r = t - k * Rp;
        const double j = r < R ? graph_param(J0, J_hw, u_J[r * E + link[k]], round_f32) : 0.0;
        w64[t] = j;
        w32[t] = (float)j;
    }
}

// Localised initial state of realization r (sum over permutations of the
// occupied nodes, signed for fermions, normalised); psi zeroed beforehand.
template <typename T>
__global__ void graph_init_state_kernel(GraphView g, const int32_t *__restrict__ sites, int stats,
                                        cplx_t<T> *psi) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.R) return;
    const int m = g.m, N = g.N;
    const int perms2[2][2] = {{0, 1}, {1, 0}};
    const int sign2[2] = {1, -1};
    const int perms3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int sign3[6] = {1, -1, -1, 1, 1, -1};
    const int nperm = (stats == 0) ? 1 : (m == 2 ? 2 : 6);
    int64_t idx[6];
    double amp[6];
    int n = 0;
    for (int p = 0; p < nperm; ++p) {
        int64_t f = 0;
        for (int j = 0; j < m; ++j) f = f * N + sites[r * m + (m == 2 ? perms2[p][j] : perms3[p][j])];
        const double sg = (stats == 2) ? (double)(m == 2 ? sign2[p] : sign3[p]) : 1.0;
        int k = 0;
        while (k < n && idx[k] != f) ++k;
        if (k == n) {
            idx[n] = f;
            amp[n] = 0.0;
            ++n;
        }
        amp[k] += sg;
    }
    double nrm = 0.0;
    for (int k = 0; k < n; ++k) nrm += amp[k] * amp[k];
    nrm = sqrt(nrm);
    for (int k = 0; k < n; ++k) psi[idx[k] * g.Rp + r] = mk<T>((T)(amp[k] / nrm), T(0));
}

template <int M>
__global__ void __launch_bounds__(kThreads, 6) graph_horner_stage_kernel(GraphView g, const float *__restrict__ eps,
                                                                      const float *__restrict__ w,
                                                                      const float2 *__restrict__ in,
                                                                      const float2 *__restrict__ psi,
                                                                      float2 *__restrict__ out, float coef) {
    int s;
    Pairs pr;
    if (!graph_site4(g, s, pr)) return;
    int x[M], S[M];
    graph_coords<M>(s, g.N, x, S);
    const C4<float> y = graph_apply_h4<float, M>(in, g.Rp, s, pr, x, S, g.row_ptr, g.col, w, eps, (float)g.U);
    const int64_t i = (int64_t)s * g.Rp;
    const C4<float> q = ld_c4(psi + i, pr);
    C4<float> o;
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // q + coef (-i) y
        o.re[k] = fmaf(coef, y.im[k], q.re[k]);
        o.im[k] = fmaf(-coef, y.re[k], q.im[k]);
    }
    st_c4(out + i, pr, o);
}

template <int M>
__global__ void __launch_bounds__(kThreads, 6) graph_horner_final_kernel(GraphView g, const float *__restrict__ eps,
                                                                      const float *__restrict__ w,
                                                                      const float2 *__restrict__ w2,
                                                                      float2 *__restrict__ psi,
                                                                      float2 *__restrict__ lo, float dt) {
    int s;
    Pairs pr;
    if (!graph_site4(g, s, pr)) return;
    int x[M], S[M];
    graph_coords<M>(s, g.N, x, S);
    // TwoSum then FastTwoSum per component: the state's rounding error is
    // carried in lo from step to step
    auto add = [](float &hi, float &lw, float v) {
        const float t = __fadd_rn(hi, v);
        const float bb = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(v, bb));
        const float e = __fadd_rn(err, lw);
        const float h2 = __fadd_rn(t, e);
        lw = __fsub_rn(e, __fsub_rn(h2, t));
        hi = h2;
    };
    const C4<float> y = graph_apply_h4<float, M>(w2, g.Rp, s, pr, x, S, g.row_ptr, g.col, w, eps, (float)g.U);
    const int64_t i = (int64_t)s * g.Rp;
    C4<float> h = ld_c4_rw(psi + i, pr), l = ld_c4_rw(lo + i, pr);
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // -i dt H w2
        add(h.re[k], l.re[k], dt * y.im[k]);
        add(h.im[k], l.im[k], -dt * y.re[k]);
    }
    st_c4(psi + i, pr, h);
    st_c4(lo + i, pr, l);
}

template <typename T, int M>
__global__ void __launch_bounds__(kThreads) graph_taylor_term_kernel(GraphView g, const T *__restrict__ eps,
                                                                     const T *__restrict__ w,
                                                                     const cplx_t<T> *__restrict__ in,
                                                                     cplx_t<T> *__restrict__ out,
                                                                     const cplx_t<T> *__restrict__ psi,
                                                                     cplx_t<T> *__restrict__ acc, T coef,
                                                                     int first) {
    int s;
    Pairs pr;
    if (!graph_site4(g, s, pr)) return;
    int x[M], S[M];
    graph_coords<M>(s, g.N, x, S);
    const C4<T> y = graph_apply_h4<T, M>(in, g.Rp, s, pr, x, S, g.row_ptr, g.col, w, eps, (T)g.U);
    const int64_t i = (int64_t)s * g.Rp;
    C4<T> phi;
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // -(i coef) y
        phi.re[k] = coef * y.im[k];
        phi.im[k] = -coef * y.re[k];
    }
    st_c4(out + i, pr, phi);
    C4<T> a = first ? ld_c4_rw(psi + i, pr) : ld_c4_rw(acc + i, pr);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a.re[k] += phi.re[k];
        a.im[k] += phi.im[k];
    }
    st_c4(acc + i, pr, a);
}

template <typename T, int M>
__global__ void __launch_bounds__(kThreads) graph_rk4_stage_kernel(GraphView g, const T *__restrict__ eps,
                                                                   const T *__restrict__ w,
                                                                   const cplx_t<T> *__restrict__ in,
                                                                   cplx_t<T> *__restrict__ next,
                                                                   const cplx_t<T> *__restrict__ psi,
                                                                   cplx_t<T> *__restrict__ acc, T a, T b,
                                                                   int first) {
    int s;
    Pairs pr;
    if (!graph_site4(g, s, pr)) return;
    int x[M], S[M];
    graph_coords<M>(s, g.N, x, S);
    const C4<T> y = graph_apply_h4<T, M>(in, g.Rp, s, pr, x, S, g.row_ptr, g.col, w, eps, (T)g.U);
    const int64_t i = (int64_t)s * g.Rp;
    const C4<T> q = ld_c4_rw(psi + i, pr);
    C4<T> c = first ? q : ld_c4_rw(acc + i, pr);
    C4<T> nx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // k = -i H in
        const T kr = y.im[k], ki = -y.re[k];
        nx.re[k] = q.re[k] + a * kr;
        nx.im[k] = q.im[k] + a * ki;
        c.re[k] += b * kr;
        c.im[k] += b * ki;
    }
    if (next) st_c4(next + i, pr, nx);
    st_c4(acc + i, pr, c);
}

// Observables of one sample.  Block (32 realization quads) x (8 warps) owns
// kRows rows (fixed x_1..x_{m-1}) of the state; warp y walks the columns
// x_m = y, y + 8, ...  Column sums of P reduce over the lanes and go out with
// one atomic per column and block; row sums, norms and energies reduce over
// the warps in shared memory.  All FP64.
constexpr int kRows = 2;   // rows per block: enough blocks (R/128 x D/(2N)) to fill the GPU
constexpr int kObsWarps = 8;

template <typename T, int M>
__global__ void __launch_bounds__(32 * kObsWarps) graph_observables_kernel(GraphView g, const T *__restrict__ eps,
                                                                         const T *__restrict__ w,
                                                                         const cplx_t<T> *__restrict__ psi,
                                                                         double *P, double *norm, double *energy) {
    const int N = g.N;
    const int n_rows = g.D / N;
    const int row0 = blockIdx.x * kRows;
    const int lane = threadIdx.x, wy = threadIdx.y;
    // realization pairs as in graph_site4 (32 lanes); idle lanes load a valid pair
    Pairs pr;
    pr.ra = g.r_begin + 128 * blockIdx.y + 2 * lane;
    pr.rb = pr.ra + 64;
    const bool valid = pr.ra < g.r_end;
    pr.vb = pr.rb < g.r_end;
    if (!valid) pr.ra = g.r_begin;
    if (!pr.vb) pr.rb = pr.ra;
    const double scale = 1.0 / ((double)g.R * M);
    double rowpart[kRows];
#pragma unroll
    for (int q = 0; q < kRows; ++q) rowpart[q] = 0.0;
    double nrm[4] = {0.0, 0.0, 0.0, 0.0}, en[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = wy; c < N; c += kObsWarps) {
        double colacc = 0.0;
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
            const int row = row0 + q;
            if (row < n_rows) {
                const int s = row * N + c;
                const C4<T> v = ld_c4(psi + (int64_t)s * g.Rp, pr);
                C4<T> y;
                if (energy) {
                    int x[M], S[M];
                    graph_coords<M>(s, N, x, S);
                    y = graph_apply_h4<T, M>(psi, g.Rp, s, pr, x, S, g.row_ptr, g.col, w, eps, (T)g.U);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool vk = valid && (k < 2 || pr.vb);
                    double p = (double)v.re[k] * (double)v.re[k] + (double)v.im[k] * (double)v.im[k];
                    if (!vk) p = 0.0;
                    colacc += p;
                    rowpart[q] += p;
                    nrm[k] += p;
                    if (energy && vk) en[k] += (double)v.re[k] * (double)y.re[k] + (double)v.im[k] * (double)y.im[k];
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) colacc += __shfl_xor_sync(0xffffffffu, colacc, o);
        if (P && lane == 0) atomicAdd(P + c, colacc * scale);
    }
    __shared__ double red_row[kObsWarps][kRows];
    __shared__ double red_r[2][kObsWarps][4][32];
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
        double v = rowpart[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red_row[wy][q] = v;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        red_r[0][wy][k][lane] = nrm[k];
        red_r[1][wy][k][lane] = en[k];
    }
    __syncthreads();
    if (wy < 4) {
        // warp k < 4 reduces realization k of every lane's two pairs
        const int k = wy;
        double a = 0.0, b = 0.0;
        for (int u = 0; u < kObsWarps; ++u) {
            a += red_r[0][u][k][lane];
            b += red_r[1][u][k][lane];
        }
        const int r = (k < 2 ? pr.ra : pr.rb) + (k & 1);
        if (valid && (k < 2 || pr.vb) && r < g.R) {
            if (norm) atomicAdd(norm + r, a);
            if (energy) atomicAdd(energy + r, b);
        }
    } else if (wy == 4 && lane < kRows && P) {
        const int row = row0 + lane;
        if (row < n_rows) {
            double v = 0.0;
            for (int u = 0; u < kObsWarps; ++u) v += red_row[u][lane];
            // coordinates x_1..x_{m-1} of this row
            int t = row;
            for (int j = M - 2; j >= 0; --j) {
                const int qq = t / N;
                atomicAdd(P + (t - qq * N), v * scale);
                t = qq;
            }
        }
    }
}

struct Launch {
    dim3 grid, block;
};

// Threads: x over the chunk's realization quads (up to 32), y over amplitudes.
inline Launch graph_launch(const ctqw_graph *g, int rb, int re) {
    const int n = (re - rb + 3) / 4;
    int rx = 1;
    while (rx < 32 && rx < n) rx <<= 1;
    const int ry = kThreads / rx;
    Launch l;
    l.block = dim3((unsigned)rx, (unsigned)ry);
    l.grid = dim3((unsigned)((g->D + ry - 1) / ry), (unsigned)((n + rx - 1) / rx));
    return l;
}

}  // namespace


int launch_graph_build_params(const ctqw_graph *g, const double *u_eps_d, const double *u_J_d,
                              cudaStream_t s) {
    graph_build_params_kernel<<<1024, 256, 0, s>>>(graph_view(g, 0, g->R), g->E, g->link_d, u_eps_d, u_J_d,
                                                   g->eps_hw, g->J_hw, g->J0, g->round_to_f32, g->eps32,
                                                   g->eps64, g->w32, g->w64, g->J64);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_graph_init_state(const ctqw_graph *g, const int32_t *sites_d, int dtype, void *psi,
                            cudaStream_t s) {
    const size_t elem = dtype == CTQW_C64 ? sizeof(float2) : sizeof(double2);
    CTQW_CUDA_TRY(cudaMemsetAsync(psi, 0, (size_t)g->total_amp * elem, s));
    const dim3 grid((unsigned)((g->R + 127) / 128));
    if (dtype == CTQW_C64)
        graph_init_state_kernel<float><<<grid, 128, 0, s>>>(graph_view(g, 0, g->R), sites_d, g->statistics,
                                                            (float2 *)psi);
    else
        graph_init_state_kernel<double><<<grid, 128, 0, s>>>(graph_view(g, 0, g->R), sites_d, g->statistics,
                                                             (double2 *)psi);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_graph_horner_stage(const ctqw_graph *g, int rb, int re, const void *in, const void *psi,
                              void *out, double coef, cudaStream_t s) {
    const Launch l = graph_launch(g, rb, re);
    auto k = g->m == 2 ? graph_horner_stage_kernel<2> : graph_horner_stage_kernel<3>;
    k<<<l.grid, l.block, 0, s>>>(graph_view(g, rb, re), g->eps32, g->w32, (const float2 *)in,
                                 (const float2 *)psi, (float2 *)out, (float)coef);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_graph_horner_final(const ctqw_graph *g, int rb, int re, const void *w2, void *psi, void *lo,
                              double dt, cudaStream_t s) {
    const Launch l = graph_launch(g, rb, re);
    auto k = g->m == 2 ? graph_horner_final_kernel<2> : graph_horner_final_kernel<3>;
    k<<<l.grid, l.block, 0, s>>>(graph_view(g, rb, re), g->eps32, g->w32, (const float2 *)w2, (float2 *)psi,
                                 (float2 *)lo, (float)dt);
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_graph_taylor_term(const ctqw_graph *g, int rb, int re, int dtype, const void *in, void *out,
                             const void *psi, void *acc, double coef, int first, cudaStream_t s) {
    const Launch l = graph_launch(g, rb, re);
    if (dtype == CTQW_C64) {
        auto k = g->m == 2 ? graph_taylor_term_kernel<float, 2> : graph_taylor_term_kernel<float, 3>;
        k<<<l.grid, l.block, 0, s>>>(graph_view(g, rb, re), g->eps32, g->w32, (const float2 *)in, (float2 *)out,
                                     (const float2 *)psi, (float2 *)acc, (float)coef, first);
    } else {
        auto k = g->m == 2 ? graph_taylor_term_kernel<double, 2> : graph_taylor_term_kernel<double, 3>;
        k<<<l.grid, l.block, 0, s>>>(graph_view(g, rb, re), g->eps64, g->w64, (const double2 *)in,
                                     (double2 *)out, (const double2 *)psi, (double2 *)acc, coef, first);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_graph_rk4_stage(const ctqw_graph *g, int rb, int re, int dtype, const void *in, void *next,
                           const void *psi, void *acc, double a, double b, int first, cudaStream_t s) {
    const Launch l = graph_launch(g, rb, re);
    if (dtype == CTQW_C64) {
        auto k = g->m == 2 ? graph_rk4_stage_kernel<float, 2> : graph_rk4_stage_kernel<float, 3>;
        k<<<l.grid, l.block, 0, s>>>(graph_view(g, rb, re), g->eps32, g->w32, (const float2 *)in,
                                     (float2 *)next, (const float2 *)psi, (float2 *)acc, (float)a, (float)b, first);
    } else {
        auto k = g->m == 2 ? graph_rk4_stage_kernel<double, 2> : graph_rk4_stage_kernel<double, 3>;
        k<<<l.grid, l.block, 0, s>>>(graph_view(g, rb, re), g->eps64, g->w64, (const double2 *)in,
                                     (double2 *)next, (const double2 *)psi, (double2 *)acc, a, b, first);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}

int launch_graph_observables(const ctqw_graph *g, int rb, int re, int dtype, const void *psi,
                             double *P_mean, double *norm, double *energy, cudaStream_t s) {
    if (!P_mean && !norm && !energy) return CTQW_OK;
    const int n_rows = (int)(g->D / g->N);
    const dim3 grid((unsigned)((n_rows + kRows - 1) / kRows), (unsigned)((re - rb + 127) / 128));
    const dim3 block(32, kObsWarps);
    if (dtype == CTQW_C64) {
        auto k = g->m == 2 ? graph_observables_kernel<float, 2> : graph_observables_kernel<float, 3>;
        k<<<grid, block, 0, s>>>(graph_view(g, rb, re), g->eps32, g->w32, (const float2 *)psi, P_mean, norm,
                                 energy);
    } else {
        auto k = g->m == 2 ? graph_observables_kernel<double, 2> : graph_observables_kernel<double, 3>;
        k<<<grid, block, 0, s>>>(graph_view(g, rb, re), g->eps64, g->w64, (const double2 *)psi, P_mean, norm,
                                 energy);
    }
    CTQW_CUDA_TRY(cudaGetLastError());
    return CTQW_OK;
}
