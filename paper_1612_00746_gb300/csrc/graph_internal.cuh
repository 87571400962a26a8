// Internal declarations of the graph path: m particles on a q-dimensional
// lattice or a general graph (Sec. 2), one topology shared by every
// realization, noise per node and per link.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ctqw.h"

// The topology is stored once as the CSR of the one-particle graph (N + 1
// row offsets, 2E neighbour entries).  The many-particle rows of Sec. 2's
// N^m x (mk + 1) topology matrix are regenerated from it inside the
// kernels (the Kronecker sum over particles), so nothing of size N^m is
// stored besides the states.
//
// Layout: realizations are the fastest index everywhere, with the stride Rp
// = R rounded up to a multiple of 4.  The states are psi[s][r] (amplitude s
// of realization r at s Rp + r), the on-site energies eps[i][r] and the
// hoppings in CSR order w[k][r] = J_r(link of entry k); padding realizations
// carry zero parameters and zero states.  A thread owns four realizations
// of one amplitude in two pairs (16-byte loads, each contiguous across the
// warp), a warp 128, so every CSR lookup is uniform across the warp and
// every neighbour load is one coalesced row.
struct ctqw_graph {
    int m = 0, statistics = 0, N = 0, E = 0, R = 0, round_to_f32 = 1;
    double J0 = 1.0, U = 0.0, eps_hw = 0.0, J_hw = 0.0;
    int64_t D = 0;            // N^m amplitudes per realization
    int Rp = 0;               // realization stride: R rounded up to a multiple of 4
    int64_t total_amp = 0;    // Rp * D
    int nnz = 0;              // 2E
    int device = 0;
    int chunk = 0;            // realizations per pass through the steps (0: all)
    int32_t *row_ptr_d = nullptr, *col_d = nullptr, *link_d = nullptr;   // CSR of the one-particle graph
    float *eps32 = nullptr, *w32 = nullptr;                              // [N][Rp], [nnz][Rp]
    double *eps64 = nullptr, *w64 = nullptr, *J64 = nullptr;             // [N][Rp], [nnz][Rp], [R][E]
};

// Per-launch view of the topology (passed by value to kernels); a launch
// covers the realizations r_begin <= r < r_end (r_begin a multiple of 4).
struct GraphView {
    const int32_t *row_ptr;
    const int32_t *col;
    int N, m, R, Rp, nnz;
    int D;        // N^m < 2^31
    int r_begin, r_end;
    double U;
};

inline GraphView graph_view(const ctqw_graph *g, int r_begin, int r_end) {
    GraphView v;
    v.row_ptr = g->row_ptr_d;
    v.col = g->col_d;
    v.N = g->N;
    v.m = g->m;
    v.R = g->R;
    v.Rp = g->Rp;
    v.nnz = g->nnz;
    v.D = (int)g->D;
    v.r_begin = r_begin;
    v.r_end = r_end;
    v.U = g->U;
    return v;
}

// Realizations per pass through the steps: g->chunk rounded up to a
// multiple of 4 when set (at most R), else all of them.
int graph_chunk(const ctqw_graph *g);

// Parameters from the uniform draws u_eps [R][N], u_J [R][E] (device):
// eps = hw (2u - 1), J = J0 + hw_J (2u - 1), optionally rounded to float32.
int launch_graph_build_params(const ctqw_graph *g, const double *u_eps_d, const double *u_J_d,
                              cudaStream_t s);

// FP32 Horner stage out = psi + coef (-i) H in; final psi (+ lo) += -i dt H w2.
int launch_graph_horner_stage(const ctqw_graph *g, int rb, int re, const void *in, const void *psi,
                              void *out, double coef, cudaStream_t s);
int launch_graph_horner_final(const ctqw_graph *g, int rb, int re, const void *w2, void *psi, void *lo,
                              double dt, cudaStream_t s);

// Forward Taylor term: out = -(i coef) H in; acc (= psi if first) += out.
int launch_graph_taylor_term(const ctqw_graph *g, int rb, int re, int dtype, const void *in, void *out,
                             const void *psi, void *acc, double coef, int first, cudaStream_t s);

// RK4 stage: k = -i H in; next = psi + a k (if next); acc (= psi if first) += b k.
int launch_graph_rk4_stage(const ctqw_graph *g, int rb, int re, int dtype, const void *in, void *next,
                           const void *psi, void *acc, double a, double b, int first, cudaStream_t s);

// One sample: P_mean [N] += (1/(R m)) sum_r P_r(x), norm [R], energy [R]
// (outputs zeroed by the caller; any may be null).
int launch_graph_observables(const ctqw_graph *g, int rb, int re, int dtype, const void *psi,
                             double *P_mean, double *norm, double *energy, cudaStream_t s);

// Localised initial states: sites_d [R][m] (device); psi zeroed first.
int launch_graph_init_state(const ctqw_graph *g, const int32_t *sites_d, int dtype, void *psi,
                            cudaStream_t s);
