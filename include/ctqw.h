/*
 * ctqw.h - C ABI of the GB300 library for many-particle continuous-time
 * quantum walks on noisy lattices (Piccinini et al., arXiv:1612.00746).
 *
 * The library propagates the state vectors of m = 2 or 3 particles on a 1D
 * tight-binding chain or ring, one noise realization per state, with the
 * truncated Taylor series of the evolution operator (Sec. 2.3, Algorithm 3)
 * or fourth-order Runge-Kutta (Sec. 2.2, Algorithm 2), and reduces the
 * diagonal of the ensemble density matrix <rho> = (1/R) sum_i |Psi_i><Psi_i|
 * (Sec. 2) to site occupations P(x) averaged over the realizations.
 *
 * Conventions (hbar = 1, sites 0-based):
 *   H1 = sum_i eps_i |i><i| - sum_b J_b (|b><b+1 mod N| + h.c.)
 *   H  = sum_j H1 acting on particle j + U * #{pairs j<l with x_j = x_l}
 *   Open chains have bonds b = 0..N-2; rings add the bond (N-1, 0).
 *   State of a realization: psi[x_1][x_2] (x_2 fastest) or psi[x_1][x_2][x_3],
 *   interleaved complex (float2 for CTQW_C64, double2 for CTQW_C128).  The
 *   states of all realizations are packed back to back; realization r starts
 *   at amplitude offset st_off[r] (see ctqw_state_size).
 *   P(x) = (1/m) sum_j sum_{states with x_j = x} |psi|^2  (normalised to the norm).
 *
 * Pointers named *_dev are device pointers, *_host host pointers.  All
 * device work is enqueued on the caller's stream (a cudaStream_t passed as
 * void*; NULL is the legacy default stream) and nothing synchronizes
 * implicitly unless stated.  Every entry point validates its arguments before
 * launching anything and returns a ctqw_status; ctqw_last_error() gives the
 * message of the last failure on the calling thread.  No entry point aborts,
 * traps or exits the process.
 */
#ifndef CTQW_H
#define CTQW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CTQW_OK 0
#define CTQW_EINVAL 1          /* bad argument (null pointer, size, range)      */
#define CTQW_ENOMEM 2          /* a device allocation failed                     */
#define CTQW_ECUDA 3           /* a CUDA runtime call or kernel launch failed    */
#define CTQW_EUNSUPPORTED 4    /* valid request the library does not implement  */
#define CTQW_ENORM 5           /* the norm check found a non-finite or drifting norm (see ctqw_check_status) */
#define CTQW_ETIMEOUT 6        /* a bounded wait inside a kernel gave up (see ctqw_check_status) */

/* Particle statistics (initial-state symmetry). */
#define CTQW_DISTINGUISHABLE 0
#define CTQW_BOSONS 1
#define CTQW_FERMIONS 2

/* Amplitude types. */
#define CTQW_C64 0             /* complex float  (float2)  */
#define CTQW_C128 1            /* complex double (double2) */

/* Propagation flags. */
#define CTQW_FLAG_PLAIN 0x1            /* force the per-term path (one launch per Taylor term) */
#define CTQW_FLAG_NO_COMPENSATION 0x2  /* c64 fused path: plain FP32 state update (no carried error term) */
#define CTQW_FLAG_RENORMALIZE 0x4      /* after every step divide each realization's state (and its carried
                                          error word) by its norm: the corrective action of the norm check of
                                          Algorithms 2 and 3 (Sec. 2.2: RK4 does not conserve the norm).  Runs
                                          on the per-term path (workspace as CTQW_FLAG_PLAIN), two extra
                                          launches per step; sampled norms are then 1 up to rounding */
#define CTQW_FLAG_TEST_WAIT_TIMEOUT 0x8 /* failure-path test: the fused kernel first waits on an mbarrier that
                                           nothing completes, gives up after 1 ms and flags the handle */
#define CTQW_FLAG_ONE_STREAM 0x10      /* fused path: run every realization on the clusters, on the caller's
                                          stream alone (see ctqw_fused_split) */
/* Fused path tuning: CTQW_FUSED_SHAPE(k) selects a compiled CTA/cluster shape
 * for the lattice size.  k = 0..2: full-row kernel (each warp owns whole rows;
 * 0 = default, the fastest measured for the size; 1 and 2 = other splits of
 * rows over warps, CTAs and clusters); k = 4..6: the banded kernel (warps
 * share rows), its shapes 0..2; k = CTQW_SHAPE_WAVEFRONT: the row-wavefront
 * kernel (one CTA per realization, one warp per Taylor term, rows streamed
 * through a pipeline; open chains, N in {64, 128, 192, 256}, also ragged,
 * K <= 16 with N + 1 > 2K + 8; needs ctqw_workspace_size bytes of workspace,
 * one c64 state, or allocates it stream-ordered when workspace_dev is NULL).
 * An index with no compiled shape returns CTQW_EUNSUPPORTED. */
#define CTQW_FUSED_SHAPE_SHIFT 8
#define CTQW_FUSED_SHAPE(k) (((uint32_t)(k) & 0xFu) << CTQW_FUSED_SHAPE_SHIFT)
#define CTQW_SHAPE_WAVEFRONT 8
/* k = CTQW_SHAPE_TILED(i), i = 0..6: the temporally blocked tiled kernel
 * (m = 2, CTQW_C64, any N, open or ring, ragged): ceil(K/D) launches per step,
 * each applying up to D Horner stages on tiles with halos.  i = 0 keeps the
 * iterate in shared memory (tile <= 56, D = 4); i = 1 keeps it in registers
 * on 64 x 128 regions (4 columns a lane), D = 8; i = 2 on 96 x 64 regions
 * (12 warps), D = 8; i = 3..6 on 64 x 64 regions (2 columns a lane),
 * D = 4, 8, 2, 7 (tile 64 - 2D).  Needs the per-term workspace (3 states). */
#define CTQW_SHAPE_TILED(i) (9 + (i))

typedef struct ctqw_hamiltonian ctqw_hamiltonian;   /* opaque, owned by the library */

/*
 * Lattice and disorder description (Eq. (Hij): every entry is a deterministic
 * part c plus a stochastic part xi, tunnelling between nearest neighbours).
 *
 * Realization r has n_sites[r] sites (or n_sites_uniform for all when n_sites
 * is NULL).  Its disorder is built from uniform draws u in [0, 1) supplied by
 * the caller, packed back to back (realization r at offset sum_{q<r} N_q):
 *   eps_{r,i} = eps_mean[i] + eps_halfwidth * (2 u_eps - 1)
 *   J_{r,b}   = J_mean[b]   + J_halfwidth   * (2 u_J   - 1)
 * with eps_mean = 0 and J_mean = J0 when the arrays are NULL.  When
 * round_to_f32 is nonzero every value is rounded to the nearest float32 so
 * that FP32 and FP64 propagation see identical Hamiltonians.
 */
typedef struct {
    int32_t n_particles;        /* m: 2 or 3                                        */
    int32_t statistics;         /* CTQW_DISTINGUISHABLE / BOSONS / FERMIONS          */
    int32_t periodic;           /* 0 open chain, 1 ring                              */
    int32_t n_realizations;     /* 1 <= R <= 65535                                  */
    const int32_t *n_sites;     /* host [R] sites per realization, or NULL           */
    int32_t n_sites_uniform;    /* used when n_sites is NULL                         */
    int32_t round_to_f32;       /* nonzero: round disorder to float32 values         */
    double J0;                  /* mean hopping when J_mean is NULL                  */
    double U;                   /* on-site interaction per coinciding pair           */
    double eps_halfwidth;       /* on-site disorder half width                       */
    double J_halfwidth;         /* hopping disorder half width                       */
    const double *eps_mean;     /* host [max N] per-site means, or NULL              */
    const double *J_mean;       /* host [max N] per-bond means, or NULL              */
    const double *u_eps_host;   /* host [sum_r N_r] uniform draws for eps            */
    const double *u_J_host;     /* host [sum_r N_r] uniform draws for J (entry N-1 of an open chain unused) */
} ctqw_lattice_desc;

/*
 * Build the stochastic Hamiltonians of all realizations (Sec. 2, Eq. (Hij)).
 * Allocates the handle and its device parameter arrays (O(sum_r N_r)), copies
 * the draws to the device and builds eps, J on the device on `stream`.  The
 * handle is usable once the stream reaches that point.  Sizes: 2 <= N <= 65536
 * for m = 2, 2 <= N <= 2048 for m = 3, and sum_r N_r^m < 2^40.
 * Errors: EINVAL for null pointers or sizes out of range, ENOMEM, ECUDA.
 */
int ctqw_build_hamiltonian(const ctqw_lattice_desc *desc, void *stream, ctqw_hamiltonian **out);

/* Free the handle and its device arrays (waits for the device first).  NULL is a no-op. */
int ctqw_destroy_hamiltonian(ctqw_hamiltonian *h);

/*
 * Plumbing: the four calls below (parameters, sizes, output layout,
 * workspace) follow no passage of the paper; they expose the library's own
 * layouts.
 *
 * Copy the built parameters back to the host (synchronizes the device).
 * eps_host and J_host are [sum_r N_r] doubles; J entry N_r-1 of an open chain
 * is 0 (the absent wrap bond).  Either pointer may be NULL.
 */
int ctqw_get_params(const ctqw_hamiltonian *h, double *eps_host, double *J_host);

/*
 * Amplitudes of all realizations, sum_r N_r^m, and optionally the per-
 * realization start offsets st_off_host [R+1] (host, int64).
 */
int ctqw_state_size(const ctqw_hamiltonian *h, int64_t *amplitudes_total, int64_t *st_off_host);

/*
 * Layout of averaged outputs.  Realizations are grouped by size (groups in
 * ascending N); P_mean rows hold the groups' averages back to back, so a row
 * has p_width = sum_g N_g doubles.  group_sizes_host [n_groups] (optional)
 * receives the N of each group, group_count_host [n_groups] (optional) the
 * number of realizations in it.
 */
int ctqw_output_layout(const ctqw_hamiltonian *h, int64_t *p_width, int32_t *n_groups,
                       int32_t *group_sizes_host, int32_t *group_count_host);

/*
 * Write the localised initial state of every realization into psi_dev
 * (zeroing everything else).  The sites are staged through a device buffer
 * of the handle (no allocation), so calls on one handle are stream-ordered.
 * sites_host is [R][m] (host, int32), the occupied sites of each
 * realization.  Bosons: normalised sum over all permutations; fermions:
 * normalised signed sum (EINVAL if two sites coincide); distinguishable:
 * |x_1..x_m>.
 */
int ctqw_init_state(const ctqw_hamiltonian *h, const int32_t *sites_host, int32_t dtype,
                    void *psi_dev, void *stream);

/*
 * Workspace bytes ctqw_propagate_taylor / ctqw_propagate_rk4 need for the
 * given dtype and flags (method 0 = Taylor, 1 = RK4): 3 states on every path
 * but the row wavefront (one state).  The fused path also accepts more (see
 * ctqw_propagate_taylor).
 */
int ctqw_workspace_size(const ctqw_hamiltonian *h, int32_t dtype, int32_t method, uint32_t flags,
                        size_t *bytes);

/*
 * Order of the truncated Taylor series (Sec. 2.3) from its remainder bound:
 * the smallest K in K_min..K_max (1 <= K_min <= K_max <= 30) with
 *   n_steps * h_dt^(K+1) / (K+1)! * exp(h_dt) <= tol / 10,
 * h_dt an upper bound of ||H dt||_2 (Lagrange remainder of exp, summed over
 * the steps; the propagator is a contraction up to that remainder).
 * *K_out gets that order and *bound_out (may be NULL) the bound it reaches.
 * When no order in range meets it: *K_out = K_max, the bound of K_max, and
 * CTQW_EUNSUPPORTED.  Pure host function: no device, no handle.
 */
int ctqw_taylor_order(double h_dt, int64_t n_steps, double tol, int32_t K_min, int32_t K_max,
                      int32_t *K_out, double *bound_out);

/*
 * ctqw_taylor_order for the handle's Hamiltonians: h_dt = |dt| times
 * m (max|eps| + 2 max|J|) + |U| m(m-1)/2, with the maxima bounded from the
 * lattice descriptor (|mean| + half width, so no device read), and tol the
 * stated tolerance of the type (2e-6 for CTQW_C64, 1e-11 for CTQW_C128).
 * Errors as ctqw_taylor_order, EINVAL for a null handle or a bad dtype.
 */
int ctqw_autotune_order(const ctqw_hamiltonian *h, int32_t dtype, double dt, int64_t n_steps,
                        int32_t K_min, int32_t K_max, int32_t *K_out);

/*
 * Advance every realization by n_steps steps of the order-K truncated Taylor
 * series of exp(-i H dt) (Sec. 2.3, Algorithm 3):
 *   Phi^(0) = Psi, Phi^(j) = -(i dt / j) H Phi^(j-1), Psi(t+dt) = sum_{j<=K} Phi^(j).
 * psi_dev (in/out) holds all states in `dtype`.  When obs_every > 0, the
 * observables are sampled at steps 0, obs_every, 2 obs_every, ... <= n_steps
 * (n_obs = n_steps / obs_every + 1 samples) into, when not NULL:
 *   P_mean_dev [n_obs][p_width] FP64: per size group, (1/R_g) sum_r P_r(x)
 *   norm_dev   [n_obs][R] FP64:  <Psi_r|Psi_r>
 *   energy_dev [n_obs][R] FP64:  <Psi_r|H_r|Psi_r>
 * The outputs are overwritten (zeroed on the stream first).  K in 1..30, or
 * 0: the order ctqw_autotune_order picks over 1..30 (host arithmetic only).
 * Observables (the norm check of Algorithms 2 and 3, and the diagonal of
 * <rho>) are formed from the state with products in its precision and
 * exact sums: FP64 for CTQW_C128; for CTQW_C64 64-bit fixed-point integer
 * sums of the FP32 products (|psi|^2 in units of 2^-48, energy terms of
 * 2^-44), converted to FP64 per block.  A sample with a non-finite or
 * out-of-range term (|psi|^2 >= 2^14) gets a NaN norm and energy.
 * Precision: CTQW_C128 propagates in FP64; CTQW_C64 propagates in FP32 and
 * carries the rounding error of every state update in a second FP32 word
 * (compensated summation).
 * Path: m = 2 chains with N a multiple of 64 up to 256 in CTQW_C64 run the
 * fused cluster kernel (every Taylor term of every step on chip; halo rows move between the CTAs
 * of a cluster point to point, see ctqw_check_status); other m = 2 handles
 * in CTQW_C64 (N > 256, ragged sizes) run the temporally blocked tiled
 * kernel with the iterate in registers, ceil(K / 8) launches a step with the
 * stages split evenly between them; everything
 * else, or CTQW_FLAG_PLAIN, runs one launch per Taylor term.  Every path
 * needs the workspace of ctqw_workspace_size (3 states).  The fused path
 * keeps the carried error in the first state and stores the state at
 * sample points into the others (S = workspace_bytes / state bytes - 1
 * slots); one launch covers S + 1 sampling intervals, so a larger
 * workspace means fewer launches.  Given no workspace, the fused path
 * allocates its 3 states stream-ordered.  With S >= 2 and enough
 * realizations, the fused path also runs the last ctqw_fused_split
 * realizations on the register tiles, on a second stream of the handle that
 * it forks from and joins back to `stream` (so the call stays ordered on
 * `stream`, also under graph capture): those tiles fill the SMs that no
 * cluster can hold.  Overlapping calls on one handle share that stream.  The
 * per-term path runs in CTQW_C128 in the order of
 * Algorithm 3 (Phi^(j) from Phi^(j-1), summed forward); in CTQW_C64 as the
 * same polynomial in Horner form (w_j = Psi + (-i dt / j) H w_{j+1}, j = K..2,
 * Psi(t+dt) = Psi - i dt H w_2) with the state update compensated, because a
 * forward FP32 sum drops every term below half an ulp of the running sum.
 * Asynchronous.
 */
int ctqw_propagate_taylor(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                          int32_t K, int64_t n_steps, int32_t obs_every, double *P_mean_dev,
                          double *norm_dev, double *energy_dev, uint32_t flags,
                          void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * How many realizations the fused path of ctqw_propagate_taylor (and of
 * ctqw_propagate_rk4, at K = 4) hands to the register tiles on the handle's
 * second stream, given a workspace of at least 3 states: the last *R_tiled
 * realizations.  A 16-CTA cluster (two particles, N = 256) needs 8 SMs of
 * one GPC, so the SMs left over in each GPC hold no cluster; the tiles get
 * the share of realizations that their throughput on those SMs can finish
 * in the time the clusters take for the rest (whole rounds of the resident
 * clusters).  0 when fewer than 1/16 of the SMs are left over, when the
 * handle has no fused path, with CTQW_FLAG_ONE_STREAM, CTQW_FLAG_PLAIN or
 * CTQW_FLAG_RENORMALIZE, or with a shape flag.  Queries the device's
 * occupancy; launches nothing.  Errors: CTQW_EINVAL for a null handle or
 * pointer or K outside 1..30.
 */
int ctqw_fused_split(const ctqw_hamiltonian *h, int32_t K, uint32_t flags, int32_t *R_tiled);

/*
 * ctqw_propagate_taylor with switching noise (Sec. 2: the stochastic terms
 * of Eq. (Hij) switch between values at random times; Algorithms 1-3 update
 * the switching times and H after every step).  Reading: after each step
 * every on-site energy and every hopping of every realization is redrawn,
 * independently with probability p_switch, from its own uniform range
 * (mean + half width * (2u - 1), rounded to float32 as at the build), and
 * otherwise keeps its value; waiting times are geometric with mean
 * 1/p_switch steps.  The draws are Philox4x64-10 (Salmon et al., SC'11)
 * under key (seed, 0), counter (step, realization, site, 0): words 0 and 1
 * decide and redraw eps of the site, words 2 and 3 the hopping of the bond
 * to its right (never the absent wrap bond of an open chain).
 * The call first restores the parameters as built, so equal arguments give
 * equal results; afterwards the handle holds the parameters after the last
 * update (ctqw_get_params).  Paths: two particles in CTQW_C64 on the
 * temporally blocked tiles, everything else (or CTQW_FLAG_PLAIN) one launch
 * per term; both need 3 states of workspace (ctqw_workspace_size with
 * CTQW_FLAG_PLAIN).  Outputs as ctqw_propagate_taylor; energies use H of
 * the sampled step.  Errors: as ctqw_propagate_taylor, EINVAL for p_switch
 * outside [0, 1] or a short workspace.  Asynchronous.
 */
int ctqw_propagate_taylor_switching(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev,
                                    double dt, int32_t K, int64_t n_steps, int32_t obs_every,
                                    double *P_mean_dev, double *norm_dev, double *energy_dev,
                                    uint32_t flags, void *workspace_dev, size_t workspace_bytes,
                                    uint64_t seed, double p_switch, void *stream);

/*
 * Exact propagation by diagonalisation (Algorithm 1, Eq. (evolPsi)), a
 * validation path for small states: every realization's dense H (D = N^m
 * <= 64) is diagonalised on the device by the cyclic Jacobi method, and
 * psi(t) = W exp(-i E t) W^T psi(0) is formed at the sampled steps
 * (t = step * dt) and at n_steps.  CTQW_C128 only.  psi_dev (in/out): the
 * initial states in, the states at n_steps * dt out.  Outputs as
 * ctqw_propagate_taylor.  sweeps_host (may be NULL): [R] Jacobi sweeps each
 * realization took (at most 40); written when the stream reaches the end of
 * the call.  Allocates its scratch stream-ordered.  Errors: EUNSUPPORTED
 * for CTQW_C64 or N^m > 64, EINVAL as ctqw_propagate_taylor.
 */
int ctqw_propagate_exact(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                         int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                         double *energy_dev, int32_t *sweeps_host, void *stream);

/*
 * Same as ctqw_propagate_taylor with the classical fourth-order Runge-Kutta
 * step of Sec. 2.2 (Algorithm 2): K^(1) = -iH Psi, K^(2) = -iH(Psi + dt/2 K^(1)),
 * K^(3) = -iH(Psi + dt/2 K^(2)), K^(4) = -iH(Psi + dt K^(3)),
 * Psi(t+dt) = Psi + dt/6 (K^(1) + 2K^(2) + 2K^(3) + K^(4)).  The norm is not
 * corrected.  This update map is the order-4 Taylor polynomial of
 * exp(-i H dt) (Sec. 2.3: order-n RK and order-n Taylor coincide for the
 * exponential); where the fused kernel applies (see ctqw_propagate_taylor)
 * it evaluates that polynomial on chip, otherwise, or with CTQW_FLAG_PLAIN,
 * one launch per stage runs the four stages above and needs the workspace
 * of ctqw_workspace_size(method = 1).
 */
int ctqw_propagate_rk4(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                       int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                       double *energy_dev, uint32_t flags, void *workspace_dev,
                       size_t workspace_bytes, void *stream);

/*
 * One-body reduced density matrix of every size group, averaged over its
 * realizations: the partial trace of Sec. 2's ensemble density matrix
 * <rho> = (1/R) sum_i |Psi_i><Psi_i| over all particles but one, averaged
 * over which particle is kept,
 *   rho1_g(x, x') = (1/R_g) (1/m) sum_r sum_j sum_{other coordinates}
 *                   psi_r(.., x_j = x, ..) conj(psi_r(.., x_j = x', ..)).
 * Hermitian, trace = the group's mean norm, diagonal = P_mean.  rho_dev:
 * device, complex128 (interleaved re, im), group g's N_g x N_g block
 * row-major starting at element sum_{g' < g} N_g'^2 (the order of
 * ctqw_output_layout's groups); overwritten (zeroed on the stream first).
 * CTQW_C64 with every group's N a multiple of 16 (up to 2048) runs on the
 * tensor cores (tcgen05, TF32): each FP32 amplitude is split into two TF32
 * pieces and every product formed from three piece products (~2^-22
 * relative), accumulated in FP32 in tensor memory over at most 256 k and
 * then in two-word FP32 totals and FP64: within 256 x 2^-23 of the largest
 * element (the tensor cores' FP32 adds may round toward zero; the CUDA-core
 * kernel sums in FP64) (see ctqw_set_density_method; it
 * allocates a scratch of 256 KB per CTA stream-ordered).  Otherwise products
 * in the state's type over chunks of 32 (16 in FP64), accumulated in FP64,
 * on CUDA cores.  m = 2 or 3.  Asynchronous.  Errors: EINVAL for null
 * pointers or a bad dtype, ENOMEM, ECUDA.  A wait of the tensor-core
 * kernel that exceeds 2 s stops it and is reported by ctqw_check_status
 * (CTQW_ETIMEOUT).
 */
int ctqw_one_body_density(const ctqw_hamiltonian *h, int32_t dtype, const void *psi_dev,
                          double *rho_dev, void *stream);

/*
 * Which units ctqw_one_body_density uses on this handle: 0 (the default)
 * the tensor cores where supported, 1 the CUDA cores always.  EINVAL for a
 * null handle or another value.
 */
int ctqw_set_density_method(ctqw_hamiltonian *h, int32_t method);

/*
 * One sample of the observables of the current states (the diagonal of
 * <rho>, Sec. 2): P_mean_dev [p_width], norm_dev [R], energy_dev [R] as in
 * ctqw_propagate_taylor, and for m = 2 optionally P_joint_dev: per size group,
 * (1/R_g) sum_r |psi_r(x1, x2)|^2 as [N_g][N_g] blocks back to back
 * (sum_g N_g^2 doubles).  Any output may be NULL; outputs are overwritten.
 */
int ctqw_ensemble_observables(const ctqw_hamiltonian *h, int32_t dtype, const void *psi_dev,
                              double *P_mean_dev, double *P_joint_dev, double *norm_dev,
                              double *energy_dev, void *stream);

/*
 * ctqw_propagate_taylor on the per-term path for callers that cannot
 * allocate device memory (the paper has no counterpart).  Such callers
 * include loops that must not call cudaMalloc because it can synchronize
 * the device, and plugins whose host program owns the device-memory budget.  Instead of a caller-provided
 * workspace, the three scratch states live in one statically sized device
 * array of 48 MiB inside this library (held on every GPU that loads it until
 * the process exits): 3 x amplitudes_total x 8 bytes (CTQW_C64) or x 16
 * bytes (CTQW_C128) must fit, else CTQW_EINVAL with a message and nothing
 * launched.  The call allocates and frees nothing.  The handle's device must
 * be the current device (else CTQW_EINVAL).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current.
 * Every call shares the one array, so calls whose work overlaps on the GPU
 * (e.g. on two streams) race and give wrong results; serialise them.
 * Arguments, outputs and results are those of ctqw_propagate_taylor with
 * CTQW_FLAG_PLAIN.  Asynchronous.
 */
int ctqw_propagate_taylor_noalloc(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev,
                                  double dt, int32_t K, int64_t n_steps, int32_t obs_every,
                                  double *P_mean_dev, double *norm_dev, double *energy_dev,
                                  void *stream);

/*
 * Workspace bytes of ctqw_adjoint_grad: (ceil(n_steps / checkpoint_every) +
 * checkpoint_every + K + 7) states plus 2 p_width + 2 sum_r N_r doubles; in
 * CTQW_C64 with two particles (the register-tile path) also K states for the
 * mu levels of a step and sum_r (ceil(N_r / 64) + ceil(N_r / 16)) N_r 3
 * doubles of per-tile gradient sums.
 */
int ctqw_adjoint_workspace_size(const ctqw_hamiltonian *h, int32_t dtype, int32_t K,
                                int64_t n_steps, int32_t checkpoint_every, size_t *bytes);

/*
 * Loss on the ensemble-averaged occupations at T = n_steps dt and its exact
 * gradient through the discrete Taylor propagation (Sec. 2.3, Algorithm 3):
 *   loss = sum_x (Pbar(x, T) - P_target(x))^2   (sum over the size groups)
 * Gradient outputs (FP64 device arrays, each may be NULL, not all four):
 *   grad_eps_dev / grad_J_dev [sum_r N_r], laid out like ctqw_get_params:
 *     dloss/deps_{r,i} and dloss/dJ_{r,b} of every realization r;
 *   grad_eps_mean_dev / grad_J_mean_dev [p_width], laid out like a P_mean
 *     row (size groups back to back, ctqw_output_layout): for group g and
 *     site (bond) i, the sum over the group's realizations of the gradients
 *     above, in ascending realization order - the gradient with respect to
 *     the means eps_mean[i], J_mean[i] the group shares (the rounding of the
 *     disorder to float32 is passed straight through).  Entry N_g - 1 of the
 *     J sums of an open chain is 0 (no wrap bond).
 * psi0_dev: initial states (not modified).  P_target_dev: [p_width] FP64.
 * loss_dev: [1] FP64.  P_final_dev: [p_width] FP64 or NULL.
 * Method: forward pass storing psi every checkpoint_every steps, then per
 * segment a replay from its checkpoint and the reverse sweep
 *   lambda_T = g psi_T,  g(s) = dloss/d|psi(s)|^2,  lambda_n = T^dagger lambda_{n+1},
 *   grad += 2 Re sum_{a<K} <mu_a, dH phi_a>,  phi_a = H^a psi_n,
 *   mu_{K-1} = conj(c_K) lambda_{n+1},  mu_a = conj(c_{a+1}) lambda_{n+1} + H mu_{a+1},
 * with c_k = (-i dt)^k / k!.  States in `dtype` (c64: FP32 states), all
 * gradient accumulation and the sums over realizations in FP64.  Needs the
 * workspace of ctqw_adjoint_workspace_size.  Errors: EINVAL for a null
 * target or loss, no gradient output, bad K / checkpoint_every or a short
 * workspace.  Asynchronous.
 */
int ctqw_adjoint_grad(const ctqw_hamiltonian *h, int32_t dtype, const void *psi0_dev, double dt,
                      int32_t K, int64_t n_steps, int32_t checkpoint_every,
                      const double *P_target_dev, double *loss_dev, double *grad_eps_dev,
                      double *grad_J_dev, double *grad_eps_mean_dev, double *grad_J_mean_dev,
                      double *P_final_dev, void *workspace_dev, size_t workspace_bytes,
                      void *stream);

/*
 * Norm check (Algorithms 2 and 3 check the norm after every step; Sec. 4 of
 * the paper asks for double checks of GPU results).  Every propagator given
 * a norm_dev output checks the norms it sampled when it finishes (one small
 * launch on the stream): a realization fails at its first sample whose norm
 * is not finite, or, when drift_tol > 0, differs from its first sample by
 * more than drift_tol.  The first failing realization and sample are kept
 * on the handle until ctqw_check_status reports them as CTQW_ENORM.
 * drift_tol = 0 (the default) checks finiteness only; the FP32 paths drift
 * by ~1e-7 over the workloads here, RK4 at large dt by much more (it does
 * not conserve the norm).  Errors: EINVAL for a null handle or a negative
 * or non-finite drift_tol.
 */
int ctqw_set_norm_check(ctqw_hamiltonian *h, double drift_tol);

/*
 * Synchronize `stream` and report a device-side failure of an earlier call
 * on this handle: CTQW_ETIMEOUT when a kernel gave up a bounded wait (the
 * fused kernel waits for halo rows from its neighbour CTAs with a 2 s limit;
 * it never spins unbounded), else CTQW_ENORM when the norm check failed, with
 * the realization, the sample and the reason in ctqw_last_error().  Each
 * event is reported once (the status is cleared); CTQW_OK otherwise.  The
 * results of a call that timed out are invalid.
 */
int ctqw_check_status(const ctqw_hamiltonian *h, void *stream);

/*
 * Failure injection for tests (the paper has no counterpart): the next
 * `after` device allocations of the library succeed and the one after them
 * fails as if the device were out of memory, so that the error path (the
 * call returns CTQW_ENOMEM and releases what it took) runs without
 * exhausting a shared GPU.  -1 switches it off.  Process-wide.  Errors:
 * EINVAL for after < -1.
 */
int ctqw_inject_alloc_failure(int32_t after);

/* ------------------------------------------------------------------------
 * q-dimensional lattices and general graphs (Sec. 2: a q-dimensional lattice
 * of N = prod_i N_i nodes, or a general graph where each node has its own
 * number of links; the topology is known in advance and holds for every
 * realization).  Conventions as above with the chain replaced by the graph:
 *   H1 = sum_i eps_i |i><i| - sum_e J_e (|u_e><v_e| + |v_e><u_e|)
 * over the links e = (u_e, v_e); repeated links add.  All realizations have
 * the same N nodes and P rows have N entries.  State layout: realizations
 * are the fastest index, amplitude s (x_m fastest, as above) of realization
 * r at s Rp + r with Rp = R rounded up to a multiple of 4 (the padding
 * realizations stay zero), so that the kernels read every neighbour as one
 * coalesced row across realizations, four realizations per thread.  The topology is stored once as the CSR of the
 * one-particle graph; the N^m x (mk + 1) many-particle topology of Sec. 2
 * is regenerated inside the kernels.
 * ------------------------------------------------------------------------ */
typedef struct ctqw_graph ctqw_graph;   /* opaque, owned by the library */

/*
 * Graph and disorder description.  Draws u in [0, 1) are supplied per
 * realization: u_eps_host [R][N] (one per node), u_J_host [R][E] (one per
 * link), and
 *   eps_{r,i} = eps_halfwidth * (2 u_eps - 1),   J_{r,e} = J0 + J_halfwidth * (2 u_J - 1),
 * each rounded to the nearest float32 when round_to_f32 is nonzero.
 */
typedef struct {
    int32_t n_particles;        /* m: 2 or 3                                         */
    int32_t statistics;         /* CTQW_DISTINGUISHABLE / BOSONS / FERMIONS           */
    int32_t n_nodes;            /* N >= 2, N^m <= 2^31 - 1                           */
    int32_t n_edges;            /* E >= 0 links                                      */
    const int32_t *edge_u;      /* host [E] first node of each link (0..N-1)         */
    const int32_t *edge_v;      /* host [E] second node, != edge_u                   */
    int32_t n_realizations;     /* 1 <= R <= 2097120, R N^m < 2^40                   */
    int32_t round_to_f32;       /* nonzero: round disorder to float32 values          */
    double J0;                  /* mean hopping                                      */
    double U;                   /* on-site interaction per coinciding pair            */
    double eps_halfwidth;       /* on-site disorder half width                        */
    double J_halfwidth;         /* hopping disorder half width                        */
    const double *u_eps_host;   /* host [R][N] uniform draws for eps                  */
    const double *u_J_host;     /* host [R][E] uniform draws for J                    */
} ctqw_graph_desc;

/*
 * Build the topology (CSR, on the host, then copied) and the parameters of
 * every realization (on the device, on `stream`, which is synchronized before
 * the call returns: the device copies of the draws are then freed).  Errors: EINVAL for null
 * pointers, sizes out of range, a link with a node out of range or with
 * u_e == v_e; ENOMEM; ECUDA.
 */
int ctqw_graph_build(const ctqw_graph_desc *desc, void *stream, ctqw_graph **out);

/* Free the handle and its device arrays (waits for the device first).  NULL is a no-op. */
int ctqw_graph_destroy(ctqw_graph *g);

/*
 * Copy the built parameters back (synchronizes the device): eps_host [R][N],
 * J_host [R][E] doubles, either may be NULL.
 */
int ctqw_graph_get_params(const ctqw_graph *g, double *eps_host, double *J_host);

/* Amplitudes of the state array, Rp N^m (Rp = R rounded up to a multiple of 4). */
int ctqw_graph_state_size(const ctqw_graph *g, int64_t *amplitudes_total);

/*
 * Localised initial states as ctqw_init_state (in the graph layout):
 * sites_host [R][m] nodes (host, int32).  EINVAL for a node out of range or
 * coinciding fermions.  Synchronizes `stream` before returning (the device
 * copy of the sites is freed after the kernel has read it).
 */
int ctqw_graph_init_state(const ctqw_graph *g, const int32_t *sites_host, int32_t dtype,
                          void *psi_dev, void *stream);

/* Workspace bytes of ctqw_graph_propagate_taylor / _rk4: 3 states of `dtype`. */
int ctqw_graph_workspace_size(const ctqw_graph *g, int32_t dtype, size_t *bytes);

/*
 * Advance every realization by n_steps order-K Taylor steps (Sec. 2.3,
 * Algorithm 3), one launch per term over all realizations.  CTQW_C128 runs
 * the terms in the order of Algorithm 3; CTQW_C64 the same polynomial in
 * Horner form with the state update compensated (the carried rounding
 * error lives in the third workspace state), as the chain's per-term path.
 * Outputs as ctqw_propagate_taylor, with P_mean_dev [n_obs][N]:
 * (1/R) sum_r P_r(x).  K in 1..30.  Errors: EINVAL for bad arguments or a
 * short workspace, ECUDA.  Asynchronous.
 */
int ctqw_graph_propagate_taylor(const ctqw_graph *g, int32_t dtype, void *psi_dev, double dt,
                                int32_t K, int64_t n_steps, int32_t obs_every, double *P_mean_dev,
                                double *norm_dev, double *energy_dev, void *workspace_dev,
                                size_t workspace_bytes, void *stream);

/*
 * Realizations per pass of ctqw_graph_propagate_taylor / _rk4 through their
 * steps.  Each pass runs every step of the call over its realizations only,
 * so that a small pass keeps its working states (psi, two iterates and the
 * error word) in L2 between launches.  0 (the default) runs all
 * realizations in one pass, which measured fastest on the 15 x 15 lattice;
 * results do not depend on it.
 */
int ctqw_graph_set_chunk(ctqw_graph *g, int32_t realizations);

/* Fourth-order Runge-Kutta on the graph (Algorithm 2); arguments as above without K. */
int ctqw_graph_propagate_rk4(const ctqw_graph *g, int32_t dtype, void *psi_dev, double dt,
                             int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                             double *energy_dev, void *workspace_dev, size_t workspace_bytes,
                             void *stream);

/*
 * One sample of the observables of the current states: P_mean_dev [N],
 * norm_dev [R], energy_dev [R] as in ctqw_graph_propagate_taylor.  Any may
 * be NULL; outputs are overwritten.  Asynchronous.
 */
int ctqw_graph_observables(const ctqw_graph *g, int32_t dtype, const void *psi_dev,
                           double *P_mean_dev, double *norm_dev, double *energy_dev, void *stream);

/* Message of the last failure on the calling thread ("" if none). */
const char *ctqw_last_error(void);

/* Library version string. */
const char *ctqw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CTQW_H */
