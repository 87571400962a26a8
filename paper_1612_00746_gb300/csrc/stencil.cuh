// Structured application of the many-particle Hamiltonian (Sec. 2, Eq. (Hij)).
//
// H = sum_j H1 acting on particle j + U * #coinciding pairs, with
// H1 = diag(eps) - sum_b J_b (|b><b+1| + h.c.), bond b = (b, b+1 mod N).
// J is stored with N entries per realization; entry N-1 is the wrap bond of a
// ring and 0 on an open chain, so the stencil never branches on boundaries.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

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
