// Structured application of the many-particle Hamiltonian (Sec. 2, Eq. (Hij)).
//
// H = sum_j H1 acting on particle j + U * #coinciding pairs, with
// H1 = diag(eps) - sum_b J_b (|b><b+1| + h.c.), bond b = (b, b+1 mod N).
// J is stored with N entries per realization; entry N-1 is the wrap bond of a
// ring and 0 on an open chain, so the stencil never branches on boundaries.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ctqw_internal.cuh"

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx<T>::type;

template <typename T>
__device__ __forceinline__ cplx_t<T> mk(T x, T y) {
    cplx_t<T> r;
    r.x = x;
    r.y = y;
    return r;
}

// Coordinates (x_1..x_M) of flat index s in an N^M tile (x_M fastest).
template <int M>
__device__ __forceinline__ void unflatten(int64_t s, int N, int (&x)[M]) {
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {
        int64_t q = s / N;
        x[j] = (int)(s - q * N);
        s = q;
    }
}

// (H a)(s) for the amplitude at flat index s with coordinates x.
template <typename T, int M>
__device__ __forceinline__ cplx_t<T> apply_h(const cplx_t<T> *__restrict__ a, int64_t s,
                                              const int (&x)[M], int N,
                                              const T *__restrict__ eps,
                                              const T *__restrict__ J, T U) {
    T v = T(0);
    int pairs = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        v += eps[x[j]];
#pragma unroll
        for (int l = j + 1; l < M; ++l) pairs += (x[j] == x[l]);
    }
    v += U * T(pairs);
    cplx_t<T> c = a[s];
    T yr = v * c.x, yi = v * c.y;
    int64_t stride = 1;
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {
        int xl = (x[j] == 0) ? N - 1 : x[j] - 1;   // left neighbour through bond xl
        int xr = (x[j] == N - 1) ? 0 : x[j] + 1;   // right neighbour through bond x[j]
        T jl = J[xl], jr = J[x[j]];
        cplx_t<T> al = a[s + (int64_t)(xl - x[j]) * stride];
        cplx_t<T> ar = a[s + (int64_t)(xr - x[j]) * stride];
        yr -= jl * al.x + jr * ar.x;
        yi -= jl * al.y + jr * ar.y;
        stride *= N;
    }
    return mk<T>(yr, yi);
}

// Grid of the per-term kernels: x = block of rows (x_1..x_{M-1} flattened;
// blockDim.y rows a block, for rows shorter than 256), y = chunk of the last
// coordinate x_M, z = realization within one size group (list: that group's
// realizations).  One launch per size group (and per 65535 realizations of
// it), so a ragged batch launches no empty blocks and no thread divides a
// 64-bit index.
template <int M>
struct Site {
    int r, N;
    int64_t s;   // flat index within the realization's state
    int x[M];
};

template <int M>
__device__ __forceinline__ bool site_of(const RealTable &tab, const int32_t *__restrict__ list, Site<M> &p) {
    p.r = list[blockIdx.z];
    p.N = tab.N[p.r];
    const int xm = blockIdx.y * blockDim.x + threadIdx.x;
    if (xm >= p.N) return false;
    const int q = blockIdx.x * blockDim.y + threadIdx.y;
    if (q >= (M == 2 ? p.N : p.N * p.N)) return false;
    if (M == 2) {
        p.x[0] = q;
    } else {
        p.x[0] = q / p.N;
        p.x[1] = q - p.x[0] * p.N;
    }
    p.x[M - 1] = xm;
    p.s = (int64_t)q * p.N + xm;
    return true;
}
