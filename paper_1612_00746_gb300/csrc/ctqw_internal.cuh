// Internal declarations shared by the translation units of libctqw.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ctqw.h"

// Library-owned description of all realizations (opaque to callers).
struct ctqw_hamiltonian {
    int m = 0, statistics = 0, periodic = 0, R = 0, round_to_f32 = 1;
    double J0 = 1.0, U = 0.0;
    int Nmax = 0;
    bool uniform = true;
    double h_norm_bound = 0.0;   // upper bound of ||H_r||_2 over all realizations (from the descriptor)
    int device = 0;
    std::vector<int32_t> sizes;                 // N_r
    std::vector<int64_t> par_off;               // [R+1] offsets of eps/J (sum N)
    std::vector<int64_t> st_off;                // [R+1] amplitude offsets (sum N^m)
    std::vector<int32_t> group_of;              // [R] size group of each realization
    std::vector<int32_t> group_N, group_count;  // [G]
    std::vector<int64_t> group_off;             // [G+1] offsets in a P_mean row
    std::vector<int64_t> joint_off;             // [G+1] offsets of the m=2 pair blocks
    int64_t total_amp = 0, total_par = 0, p_width = 0, joint_width = 0;
    // device arrays
    float *eps32 = nullptr, *J32 = nullptr;
    double *eps64 = nullptr, *J64 = nullptr;
    int32_t *sizes_d = nullptr, *group_of_d = nullptr;
    int64_t *par_off_d = nullptr, *st_off_d = nullptr, *group_off_d = nullptr,
            *joint_off_d = nullptr;
    double *inv_count_d = nullptr;  // [G] 1 / R_g
    int32_t *by_group_d = nullptr;  // [R] realization indices ordered by size group
    // switching noise: the lattice description and the parameters as built
    double eps_hw = 0.0, J_hw = 0.0;
    double *eps_mean_d = nullptr, *J_mean_d = nullptr;   // [Nmax] or null (0 / J0)
    double *eps64_0 = nullptr, *J64_0 = nullptr;         // [total_par] as built
    // status word (16 bytes): int flags at [0] (bit 0: a bounded wait gave
    // up, bit 1: the norm check failed), at byte 8 the 64-bit key of the
    // first norm failure, (realization << 40) | (sample << 8) | reason
    int *status_d = nullptr;        // 32 bytes: the status word, then at int [4] the fused kernel's ticket counter
    double *renorm_d = nullptr;     // [R] norms of the per-step renormalization
    int32_t *sites_d = nullptr;     // [R][m] initial sites (ctqw_init_state)
    double norm_drift_tol = 0.0;    // norm check: |norm - norm at step 0| above this fails (0: finiteness only)
    int density_method = 0;         // one-body density: 0 tensor cores where supported, 1 CUDA cores
    // second stream of the fused path (the realizations on the SMs that hold
    // no cluster) and the events that fork it from and join it to the caller's
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

// Per-launch view of the realization table (passed by value to kernels).
struct RealTable {
    const int32_t *N;
    const int64_t *par_off;
    const int64_t *st_off;
    const int32_t *group_of;
    const int64_t *group_off;
    const int64_t *joint_off;
    const double *inv_count;
    int R;
    int m;
    int periodic;
    double U;
};

inline int *work_counter(const ctqw_hamiltonian *h) { return h->status_d + 4; }

inline RealTable real_table(const ctqw_hamiltonian *h) {
    RealTable t;
    t.N = h->sizes_d;
    t.par_off = h->par_off_d;
    t.st_off = h->st_off_d;
    t.group_of = h->group_of_d;
    t.group_off = h->group_off_d;
    t.joint_off = h->joint_off_d;
    t.inv_count = h->inv_count_d;
    t.R = h->R;
    t.m = h->m;
    t.periodic = h->periodic;
    t.U = h->U;
    return t;
}

// Error reporting (thread-local message, see ctqw_last_error).
void ctqw_set_error(const char *fmt, ...);
int ctqw_cuda_fail(cudaError_t e, const char *what);

// Every device allocation of the library goes through these, so that a test
// can make one fail on the host (ctqw_inject_alloc_failure).
cudaError_t ctqw_malloc(void **p, size_t bytes);
cudaError_t ctqw_malloc_async(void **p, size_t bytes, cudaStream_t s);
template <typename T>
inline cudaError_t ctqw_malloc(T **p, size_t bytes) {
    return ctqw_malloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
inline cudaError_t ctqw_malloc_async(T **p, size_t bytes, cudaStream_t s) {
    return ctqw_malloc_async(reinterpret_cast<void **>(p), bytes, s);
}

// Norm check of the sampled norms ([n_obs][R]): a non-finite norm, or one
// that moved from the first sample by more than h->norm_drift_tol (> 0),
// marks the status word with the first such realization and sample.
int launch_norm_check(const ctqw_hamiltonian *h, const double *norm, int64_t n_obs, cudaStream_t s);

#define CTQW_CUDA_TRY(call)                                  \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return ctqw_cuda_fail(_e, #call); \
    } while (0)

// Propagate a nonzero status of a library call.
#define CTQW_TRY(expr)                  \
    do {                                \
        int _st = (expr);               \
        if (_st != CTQW_OK) return _st; \
    } while (0)

// One launch per size group (per 65535 of its realizations): grid (rows,
// chunks of x_M, realizations).
template <typename F>
inline int for_each_group(const ctqw_hamiltonian *h, F &&launch) {
    int off = 0;
    for (size_t g = 0; g < h->group_N.size(); ++g) {
        const int N = h->group_N[g], cnt = h->group_count[g];
        int64_t rows = 1;
        for (int j = 1; j < h->m; ++j) rows *= N;
        if (rows > 0x7fffffff) {
            ctqw_set_error("per-term path: N^(m-1) = %lld rows above the grid limit", (long long)rows);
            return CTQW_EUNSUPPORTED;
        }
        const int tx = N >= 256 ? 256 : ((N + 31) / 32) * 32;
        const int ty = 256 / tx;   // rows a block
        for (int done = 0; done < cnt; done += 65535) {
            const int part = cnt - done < 65535 ? cnt - done : 65535;
            const dim3 grid((unsigned)((rows + ty - 1) / ty), (unsigned)((N + tx - 1) / tx), (unsigned)part);
            launch(grid, dim3((unsigned)tx, (unsigned)ty), h->by_group_d + off + done);
            CTQW_CUDA_TRY(cudaGetLastError());
        }
        off += cnt;
    }
    return CTQW_OK;
}

// ---------------------------------------------------------------- launchers
// Parameter build (a1): eps/J of every realization from the uniform draws.
int launch_build_params(const ctqw_hamiltonian *h, const double *u_eps_d, const double *u_J_d,
                        const double *eps_mean_d, const double *J_mean_d, double eps_hw,
                        double J_hw, double J0, cudaStream_t s);

// Switching noise (the Hamiltonian update after step `step`): every eps and
// J of every realization redrawn with probability p (Philox4x64-10, key
// (seed, 0), counter (step, r, i, 0)); restore_params puts back the
// parameters as built.
int launch_switch_params(const ctqw_hamiltonian *h, uint64_t seed, uint64_t step, double p,
                         cudaStream_t s);
int restore_params(const ctqw_hamiltonian *h, cudaStream_t s);

// Norm correction (CTQW_FLAG_RENORMALIZE): every realization's state (and
// its carried error word lo, when not null) divided by its norm.
int launch_renormalize(const ctqw_hamiltonian *h, int dtype, void *psi, void *lo, cudaStream_t s);

// Initial state (a2).  sites_d: [R][m] int32 on the device.
int launch_init_state(const ctqw_hamiltonian *h, const int32_t *sites_d, int dtype, void *psi,
                      cudaStream_t s);

// Per-term Taylor launch (a3, plain path): out = -(i dt/j) H in; acc (= psi if first) += out.
int launch_taylor_term(const ctqw_hamiltonian *h, int dtype, const void *in, void *out,
                       const void *psi, void *acc, double coef, int first, cudaStream_t s);

// FP32 per-term path in Horner form: out = psi + coef (-i) H in;
// final: psi (+lo, carried rounding error) += -i dt H w2.
int launch_horner_stage(const ctqw_hamiltonian *h, const void *in, const void *psi, void *out,
                        double coef, cudaStream_t s);
int launch_horner_final(const ctqw_hamiltonian *h, const void *w2, void *psi, void *lo, double dt,
                        cudaStream_t s);

// RK4 stage (a4): k = -i H in; next = psi + a k (if next); acc (= psi if first) += b k.
int launch_rk4_stage(const ctqw_hamiltonian *h, int dtype, const void *in, void *next,
                     const void *psi, void *acc, double a, double b, int first, cudaStream_t s);

// Observables (a5, a6, a6b) of one sample: adds into P_mean [p_width], norm [R],
// energy [R], P_joint [joint_width]; any may be null.  Outputs must be zeroed.
int launch_observables(const ctqw_hamiltonian *h, int dtype, const void *psi, double *P_mean,
                       double *P_joint, double *norm, double *energy, cudaStream_t s);
// The same without P_joint for realizations r0 .. r0 + R_run - 1 only: their
// P terms are added into P_mean with the group's full 1/R_g weight, and
// norm/energy are indexed by the absolute realization.
int launch_observables_range(const ctqw_hamiltonian *h, int dtype, const void *psi, int r0, int R_run,
                             double *P_mean, double *norm, double *energy, cudaStream_t s);

// One-body reduced density matrix per size group (adds into rho, zeroed by
// the caller): [joint_width] complex128 at the pair-distribution offsets.
int launch_one_body_density(const ctqw_hamiltonian *h, int dtype, const void *psi, double *rho,
                            cudaStream_t s);
// The same on the tensor cores (c64, every group's N a multiple of 16 up to 2048).
bool one_body_density_tc_supported(const ctqw_hamiltonian *h, int dtype);
int launch_one_body_density_tc(const ctqw_hamiltonian *h, const void *psi, double *rho, cudaStream_t s);

// Exact propagation by diagonalisation (FP64, D = N^m <= exact_max_dim()):
// eigenpairs of every realization (evals [R][Dp], evecs [R][Dp][Dp] with Dp
// = D rounded up to even, sweeps [R] Jacobi sweeps taken), then
// psi = W exp(-i E t) W^T psi0.
int exact_max_dim();
int launch_exact_eigen(const ctqw_hamiltonian *h, double *evals, double *evecs, int *sweeps,
                       cudaStream_t s);
int launch_exact_propagate(const ctqw_hamiltonian *h, const double *evals, const double *evecs,
                           const void *psi0, void *psi, double t, cudaStream_t s);

// Adjoint pieces: out = H in; out = H in + c lam (first: c lam);
// 2 Re <mu, dH phi> into per-realization gradients; loss and lambda_T.
int launch_apply_h(const ctqw_hamiltonian *h, int dtype, const void *in, void *out, cudaStream_t s);
int launch_mu(const ctqw_hamiltonian *h, int dtype, const void *in, const void *lam, void *out,
              double cre, double cim, int first, cudaStream_t s);
// Adjoint on register tiles (c64, two particles; k_adjoint_tiled.cu): the
// phi chain phi_a = (dt H)^a psi into levels[1..K-1] (levels[0] = psi), the
// mu chain into mu_levels[0..K-1] and lambda_n into lam_out, the contraction
// of the two into per-tile FP64 slots, and the sum of the slots into the
// gradients.
bool adjoint_tiled_supported(const ctqw_hamiltonian *h, int dtype, int K);
size_t adjoint_tiled_slots(const ctqw_hamiltonian *h, int K);
int launch_adjoint_phi_chain(const ctqw_hamiltonian *h, int K, double dt, void *const *levels, cudaStream_t s);
int launch_adjoint_mu_chain(const ctqw_hamiltonian *h, int K, double dt, const void *lam, void *const *mu_levels,
                            void *lam_out, cudaStream_t s);
int launch_adjoint_contract(const ctqw_hamiltonian *h, int K, void *const *levels, void *const *mu_levels,
                            double *tg, cudaStream_t s);
int launch_adjoint_tile_reduce(const ctqw_hamiltonian *h, int K, double dt, const double *tg, double *grad_eps,
                               double *grad_J, cudaStream_t s);
int launch_grad(const ctqw_hamiltonian *h, int dtype, const void *mu, const void *phi,
                double *grad_eps, double *grad_J, cudaStream_t s);
int launch_loss(const double *Pbar, const double *target, int64_t n, double *diff, double *loss,
                cudaStream_t s);
int launch_lambda_init(const ctqw_hamiltonian *h, int dtype, const void *psi, const double *diff,
                       void *lam, cudaStream_t s);
// Per size group g: out[group_off[g] + i] = sum over the group's realizations
// r (ascending index) of grad[par_off[r] + i], i < N_g (FP64).
int launch_group_sum(const ctqw_hamiltonian *h, const double *grad, double *out, cudaStream_t s);

// Fused cluster-resident Taylor propagation (m = 2, c64), full-row layout:
// n_steps steps on chip; lo (a c64 state, lane-major rows) carries the
// rounding error in and out; when snap is not null the state after every
// snap_every-th step before the last is stored to slot q = step/snap_every - 1
// of snap (consecutive states, the layout of psi).  The launch covers
// realizations r0 .. r0 + R_run - 1 with one cluster per resident slot; the
// clusters take the realizations one at a time from the handle's ticket
// counter (work_counter), which the launch zeroes on its stream.
bool fused_rows_supported(const ctqw_hamiltonian *h, int dtype);
// How many realizations (the last ones) to run on the register tiles on the
// handle's side stream while the clusters run the rest: the SMs that hold no
// cluster (a 16-CTA cluster needs 8 SMs of one GPC) take a share matched to
// their throughput.  0 when under 1/16 of the SMs would be idle.
int fused_rows_split(const ctqw_hamiltonian *h, int shape, int K, int *R_tiled);
int launch_taylor_fused_rows(const ctqw_hamiltonian *h, void *psi, void *lo, void *snap,
                             int snap_every, double dt, int K, int64_t n_steps, int compensated,
                             int shape, int test_timeout, int r0, int R_run, cudaStream_t s);

// Fused row-wavefront Taylor propagation (m = 2, c64, open chains): every
// Taylor term of a step on chip, psi streamed once per step; lo: the carried
// rounding error (one c64 state, lane-major rows, zero before the first step).
bool wavefront_supported(const ctqw_hamiltonian *h, int dtype, int K);
size_t wavefront_workspace_bytes(const ctqw_hamiltonian *h);
int launch_taylor_wavefront(const ctqw_hamiltonian *h, void *psi, void *lo, double dt, int K,
                            int64_t n_steps, int compensated, cudaStream_t s);

// Temporally blocked Taylor stages (m = 2, c64): up to D Horner stages per
// launch on shared-memory tiles with halos; final launches add A w_2 to psi
// (compensated, lo in place) and write the new state to w_out.
int tiled_shape_count();
bool tiled_supported(const ctqw_hamiltonian *h, int dtype, int shape);
int tiled_depth(int shape);
int tiled_default_shape(int K);   // register tiles at the depth that needs the fewest launches
int launch_taylor_tiled(const ctqw_hamiltonian *h, int shape, const void *w_in, const void *psi,
                        void *w_out, void *lo, double dt, int j0, int n_stages, int final,
                        int compensated, cudaStream_t s);
// The same for realizations r0 .. r0 + R_run - 1 of a handle with one size group.
int launch_taylor_tiled_range(const ctqw_hamiltonian *h, int shape, const void *w_in, const void *psi,
                              void *w_out, void *lo, double dt, int j0, int n_stages, int final,
                              int compensated, int r0, int R_run, cudaStream_t s);

// Fused cluster-resident Taylor propagation (m = 2, c64), multi-warp bands.
bool fused_taylor_supported(const ctqw_hamiltonian *h, int dtype);
int launch_taylor_fused(const ctqw_hamiltonian *h, void *psi, double dt, int K, int64_t n_steps,
                        int obs_every, double *P_mean, double *norm, double *energy,
                        int compensated, int shape, int test_timeout, cudaStream_t s);
