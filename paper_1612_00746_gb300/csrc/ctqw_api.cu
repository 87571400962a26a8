// C ABI of libctqw: argument checking, the realization table, and the host
// loops that sequence the kernels of the propagation paths.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <atomic>
#include <climits>
#include <map>

#include "ctqw_internal.cuh"

namespace {

thread_local char g_err[512] = "";
// allocations that still succeed before one is made to fail (-1: none)
std::atomic<int> g_alloc_fail_after{-1};

bool injected_alloc_failure() {
    int v = g_alloc_fail_after.load();
    while (v >= 0) {
        if (g_alloc_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

size_t elem_bytes(int dtype) { return dtype == CTQW_C64 ? sizeof(float2) : sizeof(double2); }

int64_t n_samples(int64_t n_steps, int obs_every) {
    return obs_every > 0 ? n_steps / obs_every + 1 : 0;
}

void free_device(ctqw_hamiltonian *h) {
    void *ptrs[] = {h->eps32, h->J32, h->eps64, h->J64, h->sizes_d, h->group_of_d, h->par_off_d,
                    h->st_off_d, h->group_off_d, h->joint_off_d, h->inv_count_d, h->status_d, h->renorm_d,
                    h->by_group_d, h->eps_mean_d, h->J_mean_d, h->eps64_0, h->J64_0, h->sites_d};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    h->side = nullptr;
    h->fork_ev = h->join_ev = nullptr;
}

template <typename T>
int upload(T **dst, const std::vector<T> &src, cudaStream_t s) {
    if (ctqw_malloc((void **)dst, std::max<size_t>(1, src.size()) * sizeof(T)) != cudaSuccess) {
        ctqw_set_error("cudaMalloc of %zu bytes failed", src.size() * sizeof(T));
        return CTQW_ENOMEM;
    }
    if (!src.empty())
        CTQW_CUDA_TRY(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T),
                                      cudaMemcpyHostToDevice, s));
    return CTQW_OK;
}

int zero_outputs(const ctqw_hamiltonian *h, int64_t n_obs, double *P_mean, double *norm,
                 double *energy, cudaStream_t s) {
    if (n_obs <= 0) return CTQW_OK;
    if (P_mean) CTQW_CUDA_TRY(cudaMemsetAsync(P_mean, 0, sizeof(double) * n_obs * h->p_width, s));
    if (norm) CTQW_CUDA_TRY(cudaMemsetAsync(norm, 0, sizeof(double) * n_obs * h->R, s));
    if (energy) CTQW_CUDA_TRY(cudaMemsetAsync(energy, 0, sizeof(double) * n_obs * h->R, s));
    return CTQW_OK;
}

int check_common(const ctqw_hamiltonian *h, int dtype, const void *psi, double dt,
                 int64_t n_steps, int obs_every) {
    if (!h) { ctqw_set_error("null handle"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    if (!psi) { ctqw_set_error("null psi"); return CTQW_EINVAL; }
    if (!std::isfinite(dt) || dt == 0.0) { ctqw_set_error("dt must be finite and nonzero"); return CTQW_EINVAL; }
    if (n_steps < 0) { ctqw_set_error("n_steps < 0"); return CTQW_EINVAL; }
    if (obs_every < 0) { ctqw_set_error("obs_every < 0"); return CTQW_EINVAL; }
    return CTQW_OK;
}

// out = T in with T the order-K Taylor polynomial of exp(-i H dt)
// (Algorithm 3 with one launch per term); phiA, phiB scratch states.  In
// FP32 the same polynomial in Horner form, which does not drop the terms a
// forward FP32 sum would: for two particles on the temporally blocked tiles
// (D stages per launch, the last out = in - i dt H w_2, uncompensated),
// otherwise one launch per stage.
int taylor_step_plain(const ctqw_hamiltonian *h, int dtype, const void *in, void *out, void *phiA,
                      void *phiB, double dt, int K, cudaStream_t s) {
    const int tshape = tiled_default_shape(K);
    if (dtype == CTQW_C64 && tiled_supported(h, dtype, tshape)) {
        const int D = tiled_depth(tshape);
        const void *w = in;
        void *dst = phiA;
        for (int j0 = K; j0 >= 1;) {
            const int nst = j0 < D ? j0 : D;
            const int final = (j0 - nst + 1 == 1) ? 1 : 0;
            void *o = final ? out : dst;
            int st = launch_taylor_tiled(h, tshape, w, in, o, nullptr, dt, j0, nst, final, 0, s);
            if (st != CTQW_OK) return st;
            w = o;
            dst = (dst == phiA) ? phiB : phiA;
            j0 -= nst;
        }
        return CTQW_OK;
    }
    if (dtype == CTQW_C64) {
        const void *w = in;
        void *dst = phiA;
        for (int j = K; j >= 1; --j) {
            void *o = (j == 1) ? out : dst;
            int st = launch_horner_stage(h, w, in, o, dt / j, s);
            if (st != CTQW_OK) return st;
            w = o;
            dst = (dst == phiA) ? phiB : phiA;
        }
        return CTQW_OK;
    }
    const void *src = in;
    void *dst = phiA;
    for (int j = 1; j <= K; ++j) {
        int st = launch_taylor_term(h, dtype, src, dst, in, out, dt / j, j == 1, s);
        if (st != CTQW_OK) return st;
        src = dst;
        dst = (dst == phiA) ? phiB : phiA;
    }
    return CTQW_OK;
}

struct AdjointLayout {
    int64_t n_ck = 0;
    size_t state = 0, total = 0;
    size_t off_ck = 0, off_seg = 0, off_phi = 0, off_misc = 0, off_dbl = 0, off_grad = 0, off_tg = 0, off_mu = 0;
    bool tiled = false;   // the register-tile adjoint (c64, two particles)
};

// Workspace: checkpoints every M steps, one segment of M replayed states,
// phi_1..phi_{K-1}, 8 scratch states, then Pbar and diff (FP64), the
// per-realization gradients (FP64) for calls that want only the sums, and
// on the register-tile path the per-tile gradient slots (FP64) and the K
// mu levels of a step.
AdjointLayout adjoint_layout(const ctqw_hamiltonian *h, int dtype, int K, int64_t n_steps, int M) {
    AdjointLayout L;
    L.state = (size_t)h->total_amp * elem_bytes(dtype);
    L.n_ck = n_steps > 0 ? (n_steps - 1) / M + 1 : 1;
    L.off_ck = 0;
    L.off_seg = L.off_ck + (size_t)L.n_ck * L.state;
    L.off_phi = L.off_seg + (size_t)M * L.state;
    L.off_misc = L.off_phi + (size_t)(K > 1 ? K - 1 : 0) * L.state;
    L.off_dbl = L.off_misc + 8 * L.state;
    L.off_grad = L.off_dbl + 2 * sizeof(double) * (size_t)h->p_width;
    L.off_tg = L.off_grad + 2 * sizeof(double) * (size_t)h->total_par;
    L.tiled = adjoint_tiled_supported(h, dtype, K);
    L.off_mu = L.off_tg + (L.tiled ? sizeof(double) * adjoint_tiled_slots(h, K) : 0);
    // the register-tile path keeps the K mu levels of a step
    L.off_mu = (L.off_mu + 255) / 256 * 256;
    L.total = L.off_mu + (L.tiled ? (size_t)K * L.state : 0);
    return L;
}

}  // namespace

void ctqw_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

cudaError_t ctqw_malloc(void **p, size_t bytes) {
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t ctqw_malloc_async(void **p, size_t bytes, cudaStream_t s) {
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, s);
}

int ctqw_cuda_fail(cudaError_t e, const char *what) {
    ctqw_set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CTQW_ENOMEM : CTQW_ECUDA;
}

extern "C" {

const char *ctqw_last_error(void) { return g_err; }

const char *ctqw_version(void) { return "ctqw-gb300 0.1 (sm_103a)"; }

int ctqw_build_hamiltonian(const ctqw_lattice_desc *d, void *stream, ctqw_hamiltonian **out) {
    if (!d || !out) { ctqw_set_error("null desc/out"); return CTQW_EINVAL; }
    *out = nullptr;
    if (d->n_particles != 2 && d->n_particles != 3) {
        ctqw_set_error("n_particles must be 2 or 3 (got %d)", d->n_particles);
        return CTQW_EINVAL;
    }
    if (d->statistics < 0 || d->statistics > 2) { ctqw_set_error("statistics %d", d->statistics); return CTQW_EINVAL; }
    if (d->n_realizations < 1 || d->n_realizations > 65535) {
        ctqw_set_error("n_realizations must be in 1..65535 (got %d)", d->n_realizations);
        return CTQW_EINVAL;
    }
    if (!d->u_eps_host || !d->u_J_host) { ctqw_set_error("null uniform draws"); return CTQW_EINVAL; }
    if (!std::isfinite(d->J0) || !std::isfinite(d->U) || !std::isfinite(d->eps_halfwidth) ||
        !std::isfinite(d->J_halfwidth)) {
        ctqw_set_error("non-finite lattice parameter");
        return CTQW_EINVAL;
    }
    auto *h = new ctqw_hamiltonian();
    h->m = d->n_particles;
    h->statistics = d->statistics;
    h->periodic = d->periodic ? 1 : 0;
    h->R = d->n_realizations;
    h->round_to_f32 = d->round_to_f32 ? 1 : 0;
    h->J0 = d->J0;
    h->U = d->U;
    const int nmax_allowed = h->m == 2 ? 65536 : 2048;
    h->sizes.resize(h->R);
    for (int r = 0; r < h->R; ++r) {
        int n = d->n_sites ? d->n_sites[r] : d->n_sites_uniform;
        if (n < 2 || n > nmax_allowed) {
            ctqw_set_error("realization %d: N=%d outside 2..%d", r, n, nmax_allowed);
            delete h;
            return CTQW_EINVAL;
        }
        h->sizes[r] = n;
    }
    h->Nmax = *std::max_element(h->sizes.begin(), h->sizes.end());
    {
        // ||H||_2 <= m (max|eps| + 2 max|J|) + |U| m(m-1)/2 (Gershgorin on the
        // Kronecker sum); |eps| <= |mean| + half width, the same for J, with a
        // relative margin for the rounding of the parameters to float32
        double em = 0.0, jm = std::fabs(d->J0);
        if (d->eps_mean) {
            for (int i = 0; i < h->Nmax; ++i) em = std::max(em, std::fabs(d->eps_mean[i]));
        }
        if (d->J_mean) {
            jm = 0.0;
            for (int i = 0; i < h->Nmax; ++i) jm = std::max(jm, std::fabs(d->J_mean[i]));
        }
        const double eb = (em + std::fabs(d->eps_halfwidth)) * (1.0 + 1e-6);
        const double jb = (jm + std::fabs(d->J_halfwidth)) * (1.0 + 1e-6);
        h->h_norm_bound = h->m * (eb + 2.0 * jb) + std::fabs(h->U) * h->m * (h->m - 1) / 2.0;
    }
    h->uniform = std::all_of(h->sizes.begin(), h->sizes.end(), [&](int n) { return n == h->Nmax; });
    h->par_off.assign(h->R + 1, 0);
    h->st_off.assign(h->R + 1, 0);
    for (int r = 0; r < h->R; ++r) {
        int64_t D = 1;
        for (int j = 0; j < h->m; ++j) D *= h->sizes[r];
        h->par_off[r + 1] = h->par_off[r] + h->sizes[r];
        h->st_off[r + 1] = h->st_off[r] + D;
    }
    h->total_par = h->par_off[h->R];
    h->total_amp = h->st_off[h->R];
    if (h->total_amp >= (int64_t(1) << 40)) {
        ctqw_set_error("total amplitudes %lld too large", (long long)h->total_amp);
        delete h;
        return CTQW_EINVAL;
    }
    std::map<int, int> gidx;
    for (int n : h->sizes) gidx[n] = 0;
    int G = 0;
    for (auto &kv : gidx) {
        kv.second = G++;
        h->group_N.push_back(kv.first);
    }
    h->group_count.assign(G, 0);
    h->group_of.resize(h->R);
    for (int r = 0; r < h->R; ++r) {
        h->group_of[r] = gidx[h->sizes[r]];
        h->group_count[h->group_of[r]]++;
    }
    h->group_off.assign(G + 1, 0);
    h->joint_off.assign(G + 1, 0);
    std::vector<double> inv(G);
    for (int g = 0; g < G; ++g) {
        h->group_off[g + 1] = h->group_off[g] + h->group_N[g];
        h->joint_off[g + 1] = h->joint_off[g] + (int64_t)h->group_N[g] * h->group_N[g];
        inv[g] = 1.0 / h->group_count[g];
    }
    h->p_width = h->group_off[G];
    h->joint_width = h->joint_off[G];

    cudaStream_t s = (cudaStream_t)stream;
    int st = CTQW_OK;
    double *u_eps_d = nullptr, *u_J_d = nullptr, *em_d = nullptr, *jm_d = nullptr;
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        for (void *p : {(void *)u_eps_d, (void *)u_J_d, (void *)em_d, (void *)jm_d})
            if (p) cudaFree(p);
        free_device(h);
        delete h;
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) { ctqw_set_error("no CUDA device"); return fail(CTQW_ECUDA); }
    const size_t pb = sizeof(double) * h->total_par;
    if (ctqw_malloc(&h->eps32, sizeof(float) * h->total_par) != cudaSuccess ||
        ctqw_malloc(&h->J32, sizeof(float) * h->total_par) != cudaSuccess ||
        ctqw_malloc(&h->eps64, pb) != cudaSuccess || ctqw_malloc(&h->J64, pb) != cudaSuccess ||
        ctqw_malloc(&u_eps_d, pb) != cudaSuccess || ctqw_malloc(&u_J_d, pb) != cudaSuccess ||
        ctqw_malloc((void **)&h->status_d, 32) != cudaSuccess ||
        ctqw_malloc((void **)&h->renorm_d, sizeof(double) * h->R) != cudaSuccess ||
        ctqw_malloc((void **)&h->sites_d, sizeof(int32_t) * h->R * h->m) != cudaSuccess) {
        ctqw_set_error("cudaMalloc of the parameter arrays failed");
        return fail(CTQW_ENOMEM);
    }
    if (cudaMemsetAsync(h->status_d, 0, 8, s) != cudaSuccess ||
        cudaMemsetAsync(h->status_d + 2, 0xff, 8, s) != cudaSuccess)
        return fail(CTQW_ECUDA);
    if ((st = upload(&h->sizes_d, h->sizes, s)) || (st = upload(&h->par_off_d, h->par_off, s)) ||
        (st = upload(&h->st_off_d, h->st_off, s)) || (st = upload(&h->group_of_d, h->group_of, s)) ||
        (st = upload(&h->group_off_d, h->group_off, s)) ||
        (st = upload(&h->joint_off_d, h->joint_off, s)) || (st = upload(&h->inv_count_d, inv, s)))
        return fail(st);
    {
        std::vector<int32_t> by_group;
        by_group.reserve(h->R);
        for (int g = 0; g < G; ++g)
            for (int r = 0; r < h->R; ++r)
                if (h->group_of[r] == g) by_group.push_back(r);
        if ((st = upload(&h->by_group_d, by_group, s))) return fail(st);
    }
    if (cudaMemcpyAsync(u_eps_d, d->u_eps_host, pb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(u_J_d, d->u_J_host, pb, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        ctqw_set_error("copy of the uniform draws failed");
        return fail(CTQW_ECUDA);
    }
    if (d->eps_mean) {
        if (ctqw_malloc(&em_d, sizeof(double) * h->Nmax) != cudaSuccess) return fail(CTQW_ENOMEM);
        if (cudaMemcpyAsync(em_d, d->eps_mean, sizeof(double) * h->Nmax, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(CTQW_ECUDA);
    }
    if (d->J_mean) {
        if (ctqw_malloc(&jm_d, sizeof(double) * h->Nmax) != cudaSuccess) return fail(CTQW_ENOMEM);
        if (cudaMemcpyAsync(jm_d, d->J_mean, sizeof(double) * h->Nmax, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(CTQW_ECUDA);
    }
    if ((st = launch_build_params(h, u_eps_d, u_J_d, em_d, jm_d, d->eps_halfwidth, d->J_halfwidth,
                                  d->J0, s)))
        return fail(st);
    // kept for switching noise: the means, the half widths and the parameters as built
    h->eps_hw = d->eps_halfwidth;
    h->J_hw = d->J_halfwidth;
    h->eps_mean_d = em_d;
    h->J_mean_d = jm_d;
    em_d = jm_d = nullptr;
    if (ctqw_malloc(&h->eps64_0, pb) != cudaSuccess || ctqw_malloc(&h->J64_0, pb) != cudaSuccess)
        return fail(CTQW_ENOMEM);
    if (cudaMemcpyAsync(h->eps64_0, h->eps64, pb, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->J64_0, h->J64, pb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(CTQW_ECUDA);
    if (fused_rows_supported(h, CTQW_C64)) {
        // the fused path's second stream, at the lowest priority so that the
        // clusters go first when both have work waiting
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess) {
            ctqw_cuda_fail(cudaGetLastError(), "side stream");
            return fail(CTQW_ECUDA);
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    for (void *p : {(void *)u_eps_d, (void *)u_J_d})
        if (p) cudaFree(p);
    u_eps_d = u_J_d = nullptr;
    if (e != cudaSuccess) {
        ctqw_cuda_fail(e, "parameter build");
        free_device(h);
        delete h;
        return CTQW_ECUDA;
    }
    *out = h;
    return CTQW_OK;
}

int ctqw_destroy_hamiltonian(ctqw_hamiltonian *h) {
    if (!h) return CTQW_OK;
    free_device(h);   // cudaFree waits for work still using the arrays
    delete h;
    return CTQW_OK;
}

int ctqw_get_params(const ctqw_hamiltonian *h, double *eps_host, double *J_host) {
    if (!h) { ctqw_set_error("null handle"); return CTQW_EINVAL; }
    CTQW_CUDA_TRY(cudaDeviceSynchronize());
    if (eps_host)
        CTQW_CUDA_TRY(cudaMemcpy(eps_host, h->eps64, sizeof(double) * h->total_par, cudaMemcpyDeviceToHost));
    if (J_host)
        CTQW_CUDA_TRY(cudaMemcpy(J_host, h->J64, sizeof(double) * h->total_par, cudaMemcpyDeviceToHost));
    return CTQW_OK;
}

int ctqw_state_size(const ctqw_hamiltonian *h, int64_t *amplitudes_total, int64_t *st_off_host) {
    if (!h) { ctqw_set_error("null handle"); return CTQW_EINVAL; }
    if (amplitudes_total) *amplitudes_total = h->total_amp;
    if (st_off_host) std::copy(h->st_off.begin(), h->st_off.end(), st_off_host);
    return CTQW_OK;
}

int ctqw_output_layout(const ctqw_hamiltonian *h, int64_t *p_width, int32_t *n_groups,
                       int32_t *group_sizes_host, int32_t *group_count_host) {
    if (!h) { ctqw_set_error("null handle"); return CTQW_EINVAL; }
    if (p_width) *p_width = h->p_width;
    if (n_groups) *n_groups = (int32_t)h->group_N.size();
    if (group_sizes_host) std::copy(h->group_N.begin(), h->group_N.end(), group_sizes_host);
    if (group_count_host) std::copy(h->group_count.begin(), h->group_count.end(), group_count_host);
    return CTQW_OK;
}

int ctqw_init_state(const ctqw_hamiltonian *h, const int32_t *sites_host, int32_t dtype,
                    void *psi_dev, void *stream) {
    if (!h || !sites_host || !psi_dev) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    for (int r = 0; r < h->R; ++r) {
        for (int j = 0; j < h->m; ++j) {
            int x = sites_host[r * h->m + j];
            if (x < 0 || x >= h->sizes[r]) {
                ctqw_set_error("realization %d: site %d outside 0..%d", r, x, h->sizes[r] - 1);
                return CTQW_EINVAL;
            }
            if (h->statistics == CTQW_FERMIONS)
                for (int l = 0; l < j; ++l)
                    if (sites_host[r * h->m + l] == x) {
                        ctqw_set_error("realization %d: fermions on the same site %d", r, x);
                        return CTQW_EINVAL;
                    }
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(int32_t) * h->R * h->m;
    CTQW_CUDA_TRY(cudaMemcpyAsync(h->sites_d, sites_host, bytes, cudaMemcpyHostToDevice, s));
    return launch_init_state(h, h->sites_d, dtype, psi_dev, s);
}

int ctqw_taylor_order(double h_dt, int64_t n_steps, double tol, int32_t K_min, int32_t K_max,
                      int32_t *K_out, double *bound_out) {
    if (!K_out) { ctqw_set_error("null K_out"); return CTQW_EINVAL; }
    if (!(h_dt >= 0.0) || !std::isfinite(h_dt) || n_steps < 0 || !(tol > 0.0) || K_min < 1 ||
        K_max > 30 || K_min > K_max) {
        ctqw_set_error("taylor_order: need h_dt >= 0, n_steps >= 0, tol > 0, 1 <= K_min <= K_max <= 30");
        return CTQW_EINVAL;
    }
    // remainder of the order-K series per step: h^(K+1)/(K+1)! e^h; over the
    // run n_steps times that (the propagator is a contraction up to it)
    const double steps = n_steps > 0 ? (double)n_steps : 1.0;
    double term = 1.0;   // h^k / k!
    for (int k = 1; k <= K_min; ++k) term *= h_dt / k;
    for (int K = K_min; K <= K_max; ++K) {
        const double rem = term * h_dt / (K + 1) * std::exp(h_dt) * steps;
        if (rem <= tol / 10.0) {
            *K_out = K;
            if (bound_out) *bound_out = rem;
            return CTQW_OK;
        }
        term *= h_dt / (K + 1);
    }
    *K_out = K_max;
    if (bound_out) *bound_out = term * std::exp(h_dt) * steps;
    ctqw_set_error("taylor_order: no K in %d..%d keeps the truncation within tol/10 (h dt = %g)",
                   K_min, K_max, h_dt);
    return CTQW_EUNSUPPORTED;
}

int ctqw_autotune_order(const ctqw_hamiltonian *h, int32_t dtype, double dt, int64_t n_steps,
                        int32_t K_min, int32_t K_max, int32_t *K_out) {
    if (!h) { ctqw_set_error("null handle"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    const double tol = dtype == CTQW_C64 ? 2e-6 : 1e-11;
    return ctqw_taylor_order(h->h_norm_bound * std::fabs(dt), n_steps, tol, K_min, K_max, K_out, nullptr);
}

int ctqw_workspace_size(const ctqw_hamiltonian *h, int32_t dtype, int32_t method, uint32_t flags,
                        size_t *bytes) {
    if (!h || !bytes) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    const int shape = (int)((flags >> CTQW_FUSED_SHAPE_SHIFT) & 0xF);
    if (flags & CTQW_FLAG_RENORMALIZE) flags |= CTQW_FLAG_PLAIN;   // renormalized runs are per-term
    if ((method == 0 || method == 1) && !(flags & CTQW_FLAG_PLAIN) && shape == CTQW_SHAPE_WAVEFRONT &&
        dtype == CTQW_C64) {
        *bytes = wavefront_workspace_bytes(h);
        return CTQW_OK;
    }
    *bytes = 3 * (size_t)h->total_amp * elem_bytes(dtype);
    return CTQW_OK;
}

// The row-wavefront kernel between observation points; the observables of
// each sample from the state in psi.  The carried rounding error lives in
// the workspace (allocated stream-ordered when none is given).
static int propagate_wavefront(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                               int32_t K, int64_t n_steps, int32_t obs_every, double *P_mean_dev,
                               double *norm_dev, double *energy_dev, uint32_t flags,
                               void *workspace_dev, size_t workspace_bytes, cudaStream_t s) {
    if (!wavefront_supported(h, dtype, K)) {
        ctqw_set_error("wavefront path: needs c64, m = 2, an open chain, every N in {64, 128, 192, "
                       "256} with N + 1 > 2K + 8, and K <= 16");
        return CTQW_EUNSUPPORTED;
    }
    const size_t need = wavefront_workspace_bytes(h);
    void *lo = workspace_dev;
    bool own = false;
    if (workspace_dev && workspace_bytes < need) {
        ctqw_set_error("wavefront path needs a workspace of %zu bytes (got %zu)", need, workspace_bytes);
        return CTQW_EINVAL;
    }
    if (!lo) {
        CTQW_CUDA_TRY(ctqw_malloc_async(&lo, need, s));
        own = true;
    }
    const int64_t n_obs = n_samples(n_steps, obs_every);
    int st = zero_outputs(h, n_obs, P_mean_dev, norm_dev, energy_dev, s);
    if (st == CTQW_OK && cudaMemsetAsync(lo, 0, need, s) != cudaSuccess) st = ctqw_cuda_fail(cudaGetLastError(), "memset");
    const int comp = (flags & CTQW_FLAG_NO_COMPENSATION) ? 0 : 1;
    int64_t obs = 0;
    for (int64_t step = 0; st == CTQW_OK && step <= n_steps;) {
        if (obs_every > 0 && step % obs_every == 0) {
            st = launch_observables(h, dtype, psi_dev, P_mean_dev ? P_mean_dev + obs * h->p_width : nullptr,
                                    nullptr, norm_dev ? norm_dev + obs * h->R : nullptr,
                                    energy_dev ? energy_dev + obs * h->R : nullptr, s);
            ++obs;
        }
        if (st != CTQW_OK || step == n_steps) break;
        const int64_t next = obs_every > 0 ? std::min<int64_t>(n_steps, (step / obs_every + 1) * obs_every) : n_steps;
        st = launch_taylor_wavefront(h, psi_dev, lo, dt, K, next - step, comp, s);
        step = next;
    }
    if (own) cudaFreeAsync(lo, s);
    return st;
}

// Switching noise: after every step, the Hamiltonian update (launch_switch_params).
struct SwitchSpec {
    bool on = false;
    uint64_t seed = 0;
    double p = 0.0;
    bool renorm = false;   // divide every state by its norm after each step
};

// One launch per Taylor term (c128, forward order of Algorithm 3) or per
// Horner stage (c64, compensated state update); outputs already zeroed and
// the workspace (3 states) checked by the caller.
static int propagate_per_term(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                              int32_t K, int64_t n_steps, int32_t obs_every, double *P_mean_dev,
                              double *norm_dev, double *energy_dev, void *workspace_dev,
                              cudaStream_t s, const SwitchSpec &sw) {
    const size_t sb = (size_t)h->total_amp * elem_bytes(dtype);
    char *ws = (char *)workspace_dev;
    if (dtype == CTQW_C64) {
        // FP32: Horner stages and a compensated state update (see k_plain.cu)
        void *wa = ws, *wb = ws + sb, *lo = ws + 2 * sb;
        CTQW_CUDA_TRY(cudaMemsetAsync(lo, 0, sb, s));
        int64_t obs = 0;
        for (int64_t step = 0; step <= n_steps; ++step) {
            if (obs_every > 0 && step % obs_every == 0) {
                CTQW_TRY(launch_observables(h, dtype, psi_dev, P_mean_dev ? P_mean_dev + obs * h->p_width : nullptr,
                                            nullptr, norm_dev ? norm_dev + obs * h->R : nullptr,
                                            energy_dev ? energy_dev + obs * h->R : nullptr, s));
                ++obs;
            }
            if (step == n_steps) break;
            const void *in = psi_dev;
            void *out = wa;
            if (K == 1) {
                CTQW_CUDA_TRY(cudaMemcpyAsync(wa, psi_dev, sb, cudaMemcpyDeviceToDevice, s));
                in = wa;
            }
            for (int j = K; j >= 2; --j) {
                CTQW_TRY(launch_horner_stage(h, in, psi_dev, out, dt / j, s));
                in = out;
                out = (out == wa) ? wb : wa;
            }
            CTQW_TRY(launch_horner_final(h, in, psi_dev, lo, dt, s));
            if (sw.renorm) CTQW_TRY(launch_renormalize(h, dtype, psi_dev, lo, s));
            if (sw.on) CTQW_TRY(launch_switch_params(h, sw.seed, (uint64_t)step, sw.p, s));
        }
        return CTQW_OK;
    }
    void *cur = psi_dev, *acc = ws, *phi1 = ws + sb, *phi2 = ws + 2 * sb;
    int64_t obs = 0;
    for (int64_t step = 0; step <= n_steps; ++step) {
        if (obs_every > 0 && step % obs_every == 0) {
            CTQW_TRY(launch_observables(h, dtype, cur, P_mean_dev ? P_mean_dev + obs * h->p_width : nullptr,
                                        nullptr, norm_dev ? norm_dev + obs * h->R : nullptr,
                                        energy_dev ? energy_dev + obs * h->R : nullptr, s));
            ++obs;
        }
        if (step == n_steps) break;
        const void *in = cur;
        void *out = phi1;
        for (int j = 1; j <= K; ++j) {
            CTQW_TRY(launch_taylor_term(h, dtype, in, out, cur, acc, dt / j, j == 1, s));
            in = out;
            out = (out == phi1) ? phi2 : phi1;
        }
        std::swap(cur, acc);
        if (sw.renorm) CTQW_TRY(launch_renormalize(h, dtype, cur, nullptr, s));
        if (sw.on) CTQW_TRY(launch_switch_params(h, sw.seed, (uint64_t)step, sw.p, s));
    }
    if (cur != psi_dev) CTQW_CUDA_TRY(cudaMemcpyAsync(psi_dev, cur, sb, cudaMemcpyDeviceToDevice, s));
    return CTQW_OK;
}

// The step loop of the temporally blocked tiled kernels (c64) over
// realizations r0 .. r0 + R_run - 1: ceil(K / D) launches per step.  The
// state rotates through bufs[0] (psi) and the iterate buffers bufs[1],
// bufs[2] (the new state cannot overwrite the one other tiles read as halo);
// lo carries the rounding error.  The caller zeroes the outputs and lo.
static int tiled_steps(const ctqw_hamiltonian *h, void *const bufs[3], void *lo, double dt, int32_t K,
                       int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                       double *energy_dev, int comp, int shape, const SwitchSpec &sw, int r0, int R_run,
                       cudaStream_t s) {
    const int D = tiled_depth(shape);
    int cur = 0;
    int64_t obs = 0;
    for (int64_t step = 0; step <= n_steps; ++step) {
        if (obs_every > 0 && step % obs_every == 0) {
            CTQW_TRY(launch_observables_range(h, CTQW_C64, bufs[cur], r0, R_run,
                                              P_mean_dev ? P_mean_dev + obs * h->p_width : nullptr,
                                              norm_dev ? norm_dev + obs * h->R : nullptr,
                                              energy_dev ? energy_dev + obs * h->R : nullptr, s));
            ++obs;
        }
        if (step == n_steps) break;
        const int o1 = (cur + 1) % 3, o2 = (cur + 2) % 3;
        int win = cur;
        for (int j0 = K; j0 >= 1;) {
            const int nst = j0 < D ? j0 : D;
            const int final = (j0 - nst + 1 == 1) ? 1 : 0;
            const int wout = (win == o1) ? o2 : o1;   // neither the state nor the input iterate
            CTQW_TRY(launch_taylor_tiled_range(h, shape, bufs[win], bufs[cur], bufs[wout], lo, dt, j0, nst,
                                               final, comp, r0, R_run, s));
            win = wout;
            j0 -= nst;
            if (final) cur = wout;
        }
        if (sw.on) CTQW_TRY(launch_switch_params(h, sw.seed, (uint64_t)step, sw.p, s));
    }
    if (cur != 0) {
        const size_t a0 = (size_t)h->st_off[r0] * sizeof(float2);
        const size_t a1 = (size_t)h->st_off[r0 + R_run] * sizeof(float2);
        CTQW_CUDA_TRY(cudaMemcpyAsync((char *)bufs[0] + a0, (const char *)bufs[cur] + a0, a1 - a0,
                                      cudaMemcpyDeviceToDevice, s));
    }
    return CTQW_OK;
}

// The temporally blocked tiled kernels on the whole handle, with psi and the
// two iterate buffers of the workspace; the carried rounding error stays in
// the third workspace state.
static int propagate_tiled(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                           int32_t K, int64_t n_steps, int32_t obs_every, double *P_mean_dev,
                           double *norm_dev, double *energy_dev, uint32_t flags, int shape,
                           void *workspace_dev, size_t workspace_bytes, cudaStream_t s,
                           const SwitchSpec &sw = SwitchSpec{}) {
    if (!tiled_supported(h, dtype, shape)) {
        ctqw_set_error("tiled path: needs c64 and m = 2 (shape %d)", shape);
        return CTQW_EUNSUPPORTED;
    }
    const size_t sb = (size_t)h->total_amp * elem_bytes(dtype);
    if (!workspace_dev || workspace_bytes < 3 * sb) {
        ctqw_set_error("tiled path needs a workspace of %zu bytes (got %zu)", 3 * sb, workspace_bytes);
        return CTQW_EINVAL;
    }
    const int64_t n_obs = n_samples(n_steps, obs_every);
    CTQW_TRY(zero_outputs(h, n_obs, P_mean_dev, norm_dev, energy_dev, s));
    char *ws = (char *)workspace_dev;
    void *bufs[3] = {psi_dev, ws, ws + sb};
    void *lo = ws + 2 * sb;
    CTQW_CUDA_TRY(cudaMemsetAsync(lo, 0, sb, s));
    const int comp = (flags & CTQW_FLAG_NO_COMPENSATION) ? 0 : 1;
    return tiled_steps(h, bufs, lo, dt, K, n_steps, obs_every, P_mean_dev, norm_dev, energy_dev, comp, shape,
                       sw, 0, h->R, s);
}

// The full-row fused kernel in chunks: the workspace holds the carried
// rounding error (one state) and S >= 0 snapshot slots.  A launch runs from a
// sample point over up to S + 1 sampling intervals, storing the state at the
// S sample points inside it; the observables of every sample are then taken
// in FP64 by the observables kernel (from psi at the chunk boundaries, from
// the slots inside).  Without observables it is one launch.  With no
// workspace, one of 3 states is allocated stream-ordered.
//
// A 16-CTA cluster needs 8 SMs of one GPC, so some SMs hold no cluster.
// With S >= 2 the last realizations (fused_rows_split) run meanwhile on the
// register tiles on the handle's side stream, forked from and joined to the
// caller's stream: the tiles use slots 1 and 2 of their own realizations as
// iterate buffers, the clusters' snapshots only touch theirs, and both add
// into the same zeroed P_mean rows.
static int propagate_fused_rows(const ctqw_hamiltonian *h, void *psi_dev, double dt, int32_t K,
                                int64_t n_steps, int32_t obs_every, double *P_mean_dev,
                                double *norm_dev, double *energy_dev, uint32_t flags, int shape,
                                void *workspace_dev, size_t workspace_bytes, cudaStream_t s) {
    const size_t sb = (size_t)h->total_amp * sizeof(float2);
    void *ws = workspace_dev;
    size_t wsb = workspace_bytes;
    bool own = false;
    if (!ws) {
        wsb = 3 * sb;
        CTQW_CUDA_TRY(ctqw_malloc_async(&ws, wsb, s));
        own = true;
    } else if (wsb < sb) {
        ctqw_set_error("fused path needs a workspace of at least %zu bytes (got %zu)", sb, wsb);
        return CTQW_EINVAL;
    }
    char *w = (char *)ws;
    void *lo = w;
    const int64_t slots = (int64_t)(wsb / sb) - 1;
    const int comp = (flags & CTQW_FLAG_NO_COMPENSATION) ? 0 : 1;
    int test = (flags & CTQW_FLAG_TEST_WAIT_TIMEOUT) ? 1 : 0;
    int st = CTQW_OK;
    if (cudaMemsetAsync(lo, 0, sb, s) != cudaSuccess) st = ctqw_cuda_fail(cudaGetLastError(), "memset");
    int R_t = 0;
    if (st == CTQW_OK && h->side && slots >= 2 && shape == 0 && !(flags & CTQW_FLAG_ONE_STREAM))
        st = fused_rows_split(h, shape, K, &R_t);
    const int R_f = h->R - R_t;
    cudaStream_t side = s;
    if (st == CTQW_OK && R_t > 0) {
        if (cudaEventRecord(h->fork_ev, s) != cudaSuccess || cudaStreamWaitEvent(h->side, h->fork_ev, 0) != cudaSuccess)
            st = ctqw_cuda_fail(cudaGetLastError(), "fork of the side stream");
        else
            side = h->side;
    }
    auto observe = [&](const void *state, int64_t q) {
        return launch_observables_range(h, CTQW_C64, state, 0, R_f,
                                        P_mean_dev ? P_mean_dev + q * h->p_width : nullptr,
                                        norm_dev ? norm_dev + q * h->R : nullptr,
                                        energy_dev ? energy_dev + q * h->R : nullptr, s);
    };
    for (int64_t s0 = 0; st == CTQW_OK;) {
        if (obs_every > 0 && s0 % obs_every == 0) st = observe(psi_dev, s0 / obs_every);
        if (st != CTQW_OK || s0 == n_steps) break;
        const int64_t chunk = obs_every > 0 ? std::min<int64_t>(n_steps - s0, (slots + 1) * obs_every)
                                            : n_steps - s0;
        const int64_t inside = obs_every > 0 ? (chunk - 1) / obs_every : 0;   // snapshots of this launch
        st = launch_taylor_fused_rows(h, psi_dev, lo, inside > 0 ? w + sb : nullptr, obs_every, dt, K,
                                      chunk, comp, shape, test, 0, R_f, s);
        test = 0;
        for (int64_t q = 0; st == CTQW_OK && q < inside; ++q)
            st = observe(w + (size_t)(q + 1) * sb, s0 / obs_every + q + 1);
        s0 += chunk;
    }
    if (side != s) {
        // enqueued after the clusters' work, so a full launch queue on the
        // side stream cannot hold the clusters back
        if (st == CTQW_OK) {
            void *const bufs[3] = {psi_dev, w + sb, w + 2 * sb};
            st = tiled_steps(h, bufs, lo, dt, K, n_steps, obs_every, P_mean_dev, norm_dev, energy_dev, comp,
                             tiled_default_shape(K), SwitchSpec{}, R_f, R_t, side);
        }
        // joined even after an error: nothing of this call stays behind the caller's stream
        if (cudaEventRecord(h->join_ev, side) != cudaSuccess || cudaStreamWaitEvent(s, h->join_ev, 0) != cudaSuccess)
            if (st == CTQW_OK) st = ctqw_cuda_fail(cudaGetLastError(), "join of the side stream");
    }
    if (own) cudaFreeAsync(ws, s);
    return st;
}

static int propagate_taylor_impl(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                                 int32_t K, int64_t n_steps, int32_t obs_every, double *P_mean_dev,
                                 double *norm_dev, double *energy_dev, uint32_t flags,
                                 void *workspace_dev, size_t workspace_bytes, void *stream) {
    CTQW_TRY(check_common(h, dtype, psi_dev, dt, n_steps, obs_every));
    if (K == 0) CTQW_TRY(ctqw_autotune_order(h, dtype, dt, n_steps, 1, 30, &K));
    if (K < 1 || K > 30) { ctqw_set_error("K must be in 1..30, or 0 (got %d)", K); return CTQW_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_obs = n_samples(n_steps, obs_every);
    if (flags & CTQW_FLAG_RENORMALIZE) {
        // the norm correction runs between steps: one launch per term
        const size_t need = 3 * (size_t)h->total_amp * elem_bytes(dtype);
        if (!workspace_dev || workspace_bytes < need) {
            ctqw_set_error("CTQW_FLAG_RENORMALIZE needs a workspace of %zu bytes (got %zu)", need, workspace_bytes);
            return CTQW_EINVAL;
        }
        CTQW_TRY(zero_outputs(h, n_obs, P_mean_dev, norm_dev, energy_dev, s));
        SwitchSpec sw;
        sw.renorm = true;
        return propagate_per_term(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                                  energy_dev, workspace_dev, s, sw);
    }
    const int shape = (int)((flags >> CTQW_FUSED_SHAPE_SHIFT) & 0xF);
    if (!(flags & CTQW_FLAG_PLAIN) && shape == CTQW_SHAPE_WAVEFRONT)
        return propagate_wavefront(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev,
                                   norm_dev, energy_dev, flags, workspace_dev, workspace_bytes, s);
    if (!(flags & CTQW_FLAG_PLAIN) && shape >= CTQW_SHAPE_TILED(0)) {
        // public tiled shapes 0..6 -> compiled tile kernels (see include/ctqw.h)
        static const int tiled_public[7] = {0, 11, 13, 3, 4, 5, 6};
        return propagate_tiled(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                               energy_dev, flags, tiled_public[shape - CTQW_SHAPE_TILED(0)],
                               workspace_dev, workspace_bytes, s);
    }
    const bool fused = !(flags & CTQW_FLAG_PLAIN) && fused_rows_supported(h, dtype);
    // two particles in FP32 that the cluster-resident kernel cannot hold
    // (N > 256, ragged sizes, other N): the temporally blocked tiled kernel
    // with the iterate in registers, at the depth that needs the fewest
    // launches a step (depth 8 was the fastest measured of 2, 4, 8)
    if (!fused && !(flags & CTQW_FLAG_PLAIN) && shape == 0 && tiled_supported(h, dtype, tiled_default_shape(K)))
        return propagate_tiled(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                               energy_dev, flags, tiled_default_shape(K), workspace_dev,
                               workspace_bytes, s);
    if (!fused) {
        const size_t need = 3 * (size_t)h->total_amp * elem_bytes(dtype);
        if (!workspace_dev || workspace_bytes < need) {
            ctqw_set_error("plain path needs a workspace of %zu bytes (got %zu)", need, workspace_bytes);
            return CTQW_EINVAL;
        }
    }
    CTQW_TRY(zero_outputs(h, n_obs, P_mean_dev, norm_dev, energy_dev, s));
    if (fused) {
        // shape index 0..3: full-row kernel; 4..7: the banded kernel (shape - 4)
        const int comp = (flags & CTQW_FLAG_NO_COMPENSATION) ? 0 : 1;
        const int test = (flags & CTQW_FLAG_TEST_WAIT_TIMEOUT) ? 1 : 0;
        if (shape < 4)
            return propagate_fused_rows(h, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                                        energy_dev, flags, shape, workspace_dev, workspace_bytes, s);
        return launch_taylor_fused(h, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                                   energy_dev, comp, shape - 4, test, s);
    }

    return propagate_per_term(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                              energy_dev, workspace_dev, s, SwitchSpec{});
}

static int propagate_switching_impl(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev,
                                    double dt, int32_t K, int64_t n_steps, int32_t obs_every,
                                    double *P_mean_dev, double *norm_dev, double *energy_dev,
                                    uint32_t flags, void *workspace_dev, size_t workspace_bytes,
                                    uint64_t seed, double p_switch, void *stream) {
    CTQW_TRY(check_common(h, dtype, psi_dev, dt, n_steps, obs_every));
    if (!(p_switch >= 0.0 && p_switch <= 1.0)) {
        ctqw_set_error("p_switch must be in [0, 1] (got %g)", p_switch);
        return CTQW_EINVAL;
    }
    if (K == 0) CTQW_TRY(ctqw_autotune_order(h, dtype, dt, n_steps, 1, 30, &K));
    if (K < 1 || K > 30) { ctqw_set_error("K must be in 1..30, or 0 (got %d)", K); return CTQW_EINVAL; }
    const size_t need = 3 * (size_t)h->total_amp * elem_bytes(dtype);
    if (!workspace_dev || workspace_bytes < need) {
        ctqw_set_error("switching propagation needs a workspace of %zu bytes (got %zu)", need, workspace_bytes);
        return CTQW_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CTQW_TRY(restore_params(h, s));
    SwitchSpec sw;
    sw.on = true;
    sw.seed = seed;
    sw.p = p_switch;
    const int tshape = tiled_default_shape(K);
    if (!(flags & CTQW_FLAG_PLAIN) && tiled_supported(h, dtype, tshape))
        return propagate_tiled(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                               energy_dev, flags, tshape, workspace_dev, workspace_bytes, s, sw);
    CTQW_TRY(zero_outputs(h, n_samples(n_steps, obs_every), P_mean_dev, norm_dev, energy_dev, s));
    return propagate_per_term(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                              energy_dev, workspace_dev, s, sw);
}

static int propagate_exact_impl(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                                int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                                double *energy_dev, int32_t *sweeps_host, void *stream) {
    CTQW_TRY(check_common(h, dtype, psi_dev, dt, n_steps, obs_every));
    if (dtype != CTQW_C128) { ctqw_set_error("exact propagation is FP64 (CTQW_C128)"); return CTQW_EUNSUPPORTED; }
    int64_t D = 1;
    for (int j = 0; j < h->m; ++j) D *= h->Nmax;
    if (D > exact_max_dim()) {
        ctqw_set_error("exact propagation: N^m = %lld above %d", (long long)D, exact_max_dim());
        return CTQW_EUNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t Dp = D + (D & 1);
    const size_t sb = (size_t)h->total_amp * sizeof(double2);
    double *evals = nullptr, *evecs = nullptr;
    void *psi0 = nullptr;
    int *sweeps = nullptr;
    CTQW_CUDA_TRY(ctqw_malloc_async((void **)&evals, sizeof(double) * (size_t)(h->R * Dp), s));
    CTQW_CUDA_TRY(ctqw_malloc_async((void **)&evecs, sizeof(double) * (size_t)(h->R * Dp * Dp), s));
    CTQW_CUDA_TRY(ctqw_malloc_async(&psi0, sb, s));
    CTQW_CUDA_TRY(ctqw_malloc_async((void **)&sweeps, sizeof(int) * (size_t)h->R, s));
    int st = zero_outputs(h, n_samples(n_steps, obs_every), P_mean_dev, norm_dev, energy_dev, s);
    if (st == CTQW_OK && cudaMemcpyAsync(psi0, psi_dev, sb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        st = ctqw_cuda_fail(cudaGetLastError(), "copy of psi0");
    if (st == CTQW_OK) st = launch_exact_eigen(h, evals, evecs, sweeps, s);
    int64_t obs = 0;
    for (int64_t step = 0; st == CTQW_OK && step <= n_steps; ++step) {
        const bool sample = obs_every > 0 && step % obs_every == 0;
        if (!sample && step != n_steps) continue;
        st = launch_exact_propagate(h, evals, evecs, psi0, psi_dev, dt * (double)step, s);
        if (st == CTQW_OK && sample) {
            st = launch_observables(h, dtype, psi_dev, P_mean_dev ? P_mean_dev + obs * h->p_width : nullptr,
                                    nullptr, norm_dev ? norm_dev + obs * h->R : nullptr,
                                    energy_dev ? energy_dev + obs * h->R : nullptr, s);
            ++obs;
        }
    }
    if (st == CTQW_OK && sweeps_host &&
        cudaMemcpyAsync(sweeps_host, sweeps, sizeof(int) * (size_t)h->R, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = ctqw_cuda_fail(cudaGetLastError(), "copy of the sweep counts");
    cudaFreeAsync(evals, s);
    cudaFreeAsync(evecs, s);
    cudaFreeAsync(psi0, s);
    cudaFreeAsync(sweeps, s);
    return st;
}

static int propagate_rk4_impl(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                              int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                              double *energy_dev, uint32_t flags, void *workspace_dev,
                              size_t workspace_bytes, void *stream) {
    CTQW_TRY(check_common(h, dtype, psi_dev, dt, n_steps, obs_every));
    cudaStream_t s = (cudaStream_t)stream;
    // RK4's update map is the order-4 Taylor polynomial of exp(-i H dt)
    // (Sec. 2.3): the fused kernel evaluates it directly
    if (!(flags & (CTQW_FLAG_PLAIN | CTQW_FLAG_RENORMALIZE)) && fused_rows_supported(h, dtype))
        return propagate_taylor_impl(h, dtype, psi_dev, dt, 4, n_steps, obs_every, P_mean_dev,
                                     norm_dev, energy_dev, flags, workspace_dev, workspace_bytes,
                                     stream);
    const size_t sb = (size_t)h->total_amp * elem_bytes(dtype);
    const int64_t n_obs = n_samples(n_steps, obs_every);
    CTQW_TRY(zero_outputs(h, n_obs, P_mean_dev, norm_dev, energy_dev, s));
    char *ws = (char *)workspace_dev;
    void *cur = psi_dev, *acc = ws, *t1 = ws + sb, *t2 = ws + 2 * sb;
    int64_t obs = 0;
    for (int64_t step = 0; step <= n_steps; ++step) {
        if (obs_every > 0 && step % obs_every == 0) {
            CTQW_TRY(launch_observables(h, dtype, cur, P_mean_dev ? P_mean_dev + obs * h->p_width : nullptr,
                                        nullptr, norm_dev ? norm_dev + obs * h->R : nullptr,
                                        energy_dev ? energy_dev + obs * h->R : nullptr, s));
            ++obs;
        }
        if (step == n_steps) break;
        // K1 = -iH psi: next = psi + dt/2 K1, acc = psi + dt/6 K1
        CTQW_TRY(launch_rk4_stage(h, dtype, cur, t1, cur, acc, 0.5 * dt, dt / 6.0, 1, s));
        // K2 = -iH(psi + dt/2 K1): next = psi + dt/2 K2, acc += dt/3 K2
        CTQW_TRY(launch_rk4_stage(h, dtype, t1, t2, cur, acc, 0.5 * dt, dt / 3.0, 0, s));
        // K3 = -iH(psi + dt/2 K2): next = psi + dt K3, acc += dt/3 K3
        CTQW_TRY(launch_rk4_stage(h, dtype, t2, t1, cur, acc, dt, dt / 3.0, 0, s));
        // K4 = -iH(psi + dt K3): acc += dt/6 K4
        CTQW_TRY(launch_rk4_stage(h, dtype, t1, nullptr, cur, acc, 0.0, dt / 6.0, 0, s));
        std::swap(cur, acc);
        // the corrective action of the norm check (RK4 does not conserve the norm)
        if (flags & CTQW_FLAG_RENORMALIZE) CTQW_TRY(launch_renormalize(h, dtype, cur, nullptr, s));
    }
    if (cur != psi_dev) CTQW_CUDA_TRY(cudaMemcpyAsync(psi_dev, cur, sb, cudaMemcpyDeviceToDevice, s));
    return CTQW_OK;
}

// The public propagators: the work, then the norm check of the sampled norms.
int ctqw_propagate_taylor(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                          int32_t K, int64_t n_steps, int32_t obs_every, double *P_mean_dev,
                          double *norm_dev, double *energy_dev, uint32_t flags,
                          void *workspace_dev, size_t workspace_bytes, void *stream) {
    CTQW_TRY(propagate_taylor_impl(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                                   energy_dev, flags, workspace_dev, workspace_bytes, stream));
    return launch_norm_check(h, norm_dev, n_samples(n_steps, obs_every), (cudaStream_t)stream);
}

int ctqw_fused_split(const ctqw_hamiltonian *h, int32_t K, uint32_t flags, int32_t *R_tiled) {
    if (!h || !R_tiled) { ctqw_set_error("null handle or output"); return CTQW_EINVAL; }
    if (K < 1 || K > 30) { ctqw_set_error("K must be in 1..30 (got %d)", K); return CTQW_EINVAL; }
    *R_tiled = 0;
    const int shape = (int)((flags >> CTQW_FUSED_SHAPE_SHIFT) & 0xF);
    if ((flags & (CTQW_FLAG_PLAIN | CTQW_FLAG_RENORMALIZE | CTQW_FLAG_ONE_STREAM)) || shape != 0 || !h->side)
        return CTQW_OK;
    int r = 0;
    CTQW_TRY(fused_rows_split(h, 0, K, &r));
    *R_tiled = r;
    return CTQW_OK;
}

int ctqw_propagate_taylor_switching(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev,
                                    double dt, int32_t K, int64_t n_steps, int32_t obs_every,
                                    double *P_mean_dev, double *norm_dev, double *energy_dev,
                                    uint32_t flags, void *workspace_dev, size_t workspace_bytes,
                                    uint64_t seed, double p_switch, void *stream) {
    CTQW_TRY(propagate_switching_impl(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev, norm_dev,
                                      energy_dev, flags, workspace_dev, workspace_bytes, seed, p_switch,
                                      stream));
    return launch_norm_check(h, norm_dev, n_samples(n_steps, obs_every), (cudaStream_t)stream);
}

int ctqw_propagate_exact(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                         int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                         double *energy_dev, int32_t *sweeps_host, void *stream) {
    CTQW_TRY(propagate_exact_impl(h, dtype, psi_dev, dt, n_steps, obs_every, P_mean_dev, norm_dev,
                                  energy_dev, sweeps_host, stream));
    return launch_norm_check(h, norm_dev, n_samples(n_steps, obs_every), (cudaStream_t)stream);
}

int ctqw_propagate_rk4(const ctqw_hamiltonian *h, int32_t dtype, void *psi_dev, double dt,
                       int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                       double *energy_dev, uint32_t flags, void *workspace_dev,
                       size_t workspace_bytes, void *stream) {
    CTQW_TRY(propagate_rk4_impl(h, dtype, psi_dev, dt, n_steps, obs_every, P_mean_dev, norm_dev,
                                energy_dev, flags, workspace_dev, workspace_bytes, stream));
    return launch_norm_check(h, norm_dev, n_samples(n_steps, obs_every), (cudaStream_t)stream);
}

int ctqw_set_norm_check(ctqw_hamiltonian *h, double drift_tol) {
    if (!h) { ctqw_set_error("null handle"); return CTQW_EINVAL; }
    if (!(drift_tol >= 0.0) || !std::isfinite(drift_tol)) {
        ctqw_set_error("drift_tol must be finite and >= 0 (got %g)", drift_tol);
        return CTQW_EINVAL;
    }
    h->norm_drift_tol = drift_tol;
    return CTQW_OK;
}

int ctqw_inject_alloc_failure(int32_t after) {
    if (after < -1) { ctqw_set_error("after must be >= -1 (got %d)", after); return CTQW_EINVAL; }
    g_alloc_fail_after.store(after);
    return CTQW_OK;
}

int ctqw_check_status(const ctqw_hamiltonian *h, void *stream) {
    if (!h) { ctqw_set_error("null handle"); return CTQW_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    CTQW_CUDA_TRY(cudaStreamSynchronize(s));
    struct {
        int flags, pad;
        unsigned long long key;
    } st;
    CTQW_CUDA_TRY(cudaMemcpy(&st, h->status_d, sizeof(st), cudaMemcpyDeviceToHost));
    if (st.flags == 0) return CTQW_OK;
    CTQW_CUDA_TRY(cudaMemset(h->status_d, 0, 8));
    CTQW_CUDA_TRY(cudaMemset(h->status_d + 2, 0xff, 8));
    if (st.flags & 1) {
        ctqw_set_error("a bounded wait inside a propagation kernel gave up; results of that call are invalid");
        return CTQW_ETIMEOUT;
    }
    const unsigned long long r = st.key >> 40, q = (st.key >> 8) & 0xffffffffull, why = st.key & 0xffull;
    ctqw_set_error("norm check: realization %llu, sample %llu: %s", r, q,
                   why == 1 ? "the norm is not finite" : "the norm drifted beyond the set tolerance");
    return CTQW_ENORM;
}

int ctqw_adjoint_workspace_size(const ctqw_hamiltonian *h, int32_t dtype, int32_t K,
                                int64_t n_steps, int32_t checkpoint_every, size_t *bytes) {
    if (!h || !bytes) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    if (K < 1 || K > 30 || n_steps < 0 || checkpoint_every < 1) {
        ctqw_set_error("bad K / n_steps / checkpoint_every");
        return CTQW_EINVAL;
    }
    *bytes = adjoint_layout(h, dtype, K, n_steps, checkpoint_every).total;
    return CTQW_OK;
}

int ctqw_adjoint_grad(const ctqw_hamiltonian *h, int32_t dtype, const void *psi0_dev, double dt,
                      int32_t K, int64_t n_steps, int32_t checkpoint_every,
                      const double *P_target_dev, double *loss_dev, double *grad_eps_dev,
                      double *grad_J_dev, double *grad_eps_mean_dev, double *grad_J_mean_dev,
                      double *P_final_dev, void *workspace_dev, size_t workspace_bytes,
                      void *stream) {
    CTQW_TRY(check_common(h, dtype, psi0_dev, dt, n_steps, 0));
    if (K < 1 || K > 30) { ctqw_set_error("K must be in 1..30 (got %d)", K); return CTQW_EINVAL; }
    if (checkpoint_every < 1) { ctqw_set_error("checkpoint_every must be >= 1"); return CTQW_EINVAL; }
    if (!P_target_dev || !loss_dev) {
        ctqw_set_error("null target / loss pointer");
        return CTQW_EINVAL;
    }
    if (!grad_eps_dev && !grad_J_dev && !grad_eps_mean_dev && !grad_J_mean_dev) {
        ctqw_set_error("no gradient output (all four gradient pointers are null)");
        return CTQW_EINVAL;
    }
    const int M = checkpoint_every;
    const AdjointLayout L = adjoint_layout(h, dtype, K, n_steps, M);
    if (!workspace_dev || workspace_bytes < L.total) {
        ctqw_set_error("adjoint needs a workspace of %zu bytes (got %zu)", L.total, workspace_bytes);
        return CTQW_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)workspace_dev;
    auto ck = [&](int64_t c) { return (void *)(ws + L.off_ck + (size_t)c * L.state); };
    auto seg = [&](int64_t k) { return (void *)(ws + L.off_seg + (size_t)k * L.state); };
    auto phi = [&](int a) { return (void *)(ws + L.off_phi + (size_t)(a - 1) * L.state); };
    void *misc[8];
    for (int q = 0; q < 8; ++q) misc[q] = ws + L.off_misc + (size_t)q * L.state;
    void *X = misc[0], *Y = misc[1], *tA = misc[2], *tB = misc[3];
    void *lam = misc[4], *lam2 = misc[5], *muA = misc[6], *muB = misc[7];
    double *Pbar = (double *)(ws + L.off_dbl);
    double *diff = Pbar + h->p_width;
    // per-realization gradients: the caller's arrays, or the workspace's
    if (!grad_eps_dev) grad_eps_dev = (double *)(ws + L.off_grad);
    if (!grad_J_dev) grad_J_dev = (double *)(ws + L.off_grad) + h->total_par;

    CTQW_CUDA_TRY(cudaMemsetAsync(grad_eps_dev, 0, sizeof(double) * h->total_par, s));
    CTQW_CUDA_TRY(cudaMemsetAsync(grad_J_dev, 0, sizeof(double) * h->total_par, s));
    CTQW_CUDA_TRY(cudaMemsetAsync(Pbar, 0, sizeof(double) * h->p_width, s));
    double *tg = (double *)(ws + L.off_tg);
    if (L.tiled) CTQW_CUDA_TRY(cudaMemsetAsync(tg, 0, L.off_mu - L.off_tg, s));

    // forward pass with checkpoints psi_{cM}
    CTQW_CUDA_TRY(cudaMemcpyAsync(X, psi0_dev, L.state, cudaMemcpyDeviceToDevice, s));
    void *cur = X, *nxt = Y;
    for (int64_t n = 0; n < n_steps; ++n) {
        if (n % M == 0) CTQW_CUDA_TRY(cudaMemcpyAsync(ck(n / M), cur, L.state, cudaMemcpyDeviceToDevice, s));
        CTQW_TRY(taylor_step_plain(h, dtype, cur, nxt, tA, tB, dt, K, s));
        std::swap(cur, nxt);
    }
    // loss at T and the terminal adjoint state
    CTQW_TRY(launch_observables(h, dtype, cur, Pbar, nullptr, nullptr, nullptr, s));
    CTQW_TRY(launch_loss(Pbar, P_target_dev, h->p_width, diff, loss_dev, s));
    if (P_final_dev)
        CTQW_CUDA_TRY(cudaMemcpyAsync(P_final_dev, Pbar, sizeof(double) * h->p_width,
                                      cudaMemcpyDeviceToDevice, s));
    CTQW_TRY(launch_lambda_init(h, dtype, cur, diff, lam, s));

    // conj(c_k) = (i dt)^k / k!
    double cre[31], cim[31];
    {
        double mag = 1.0;
        for (int k = 0; k <= K; ++k) {
            if (k > 0) mag *= dt / k;
            const int q = k & 3;   // i^k = 1, i, -1, -i
            cre[k] = (q == 0) ? mag : (q == 2 ? -mag : 0.0);
            cim[k] = (q == 1) ? mag : (q == 3 ? -mag : 0.0);
        }
    }
    // backward over the segments, replaying each from its checkpoint
    for (int64_t c = L.n_ck - 1; c >= 0 && n_steps > 0; --c) {
        const int64_t n0 = c * M, n1 = std::min<int64_t>(n0 + M, n_steps);
        for (int64_t k = 1; k < n1 - n0; ++k)
            CTQW_TRY(taylor_step_plain(h, dtype, k == 1 ? ck(c) : seg(k - 1), seg(k), tA, tB, dt, K, s));
        for (int64_t n = n1 - 1; n >= n0; --n) {
            const void *psi_n = (n == n0) ? ck(c) : seg(n - n0);
            if (L.tiled) {
                void *levels[32], *mu_levels[32];
                levels[0] = const_cast<void *>(psi_n);
                for (int a = 1; a < K; ++a) levels[a] = phi(a);
                for (int a = 0; a < K; ++a) mu_levels[a] = ws + L.off_mu + (size_t)a * L.state;
                CTQW_TRY(launch_adjoint_phi_chain(h, K, dt, levels, s));
                CTQW_TRY(launch_adjoint_mu_chain(h, K, dt, lam, mu_levels, lam2, s));
                CTQW_TRY(launch_adjoint_contract(h, K, levels, mu_levels, tg, s));
                std::swap(lam, lam2);
                continue;
            }
            for (int a = 1; a < K; ++a) CTQW_TRY(launch_apply_h(h, dtype, a == 1 ? psi_n : phi(a - 1), phi(a), s));
            // mu_{K-1} = conj(c_K) lambda;  mu_a = conj(c_{a+1}) lambda + H mu_{a+1}
            void *mu = muA, *mu_prev = muB;
            for (int a = K - 1; a >= 0; --a) {
                CTQW_TRY(launch_mu(h, dtype, mu_prev, lam, mu, cre[a + 1], cim[a + 1], a == K - 1, s));
                CTQW_TRY(launch_grad(h, dtype, mu, a == 0 ? psi_n : phi(a), grad_eps_dev, grad_J_dev, s));
                std::swap(mu, mu_prev);
            }
            // lambda_n = T^dagger lambda_{n+1} = sum_k conj(c_k) H^k lambda_{n+1}
            //          = lambda_{n+1} + H mu_0, mu_0 = sum_{b<K} conj(c_{b+1}) H^b lambda_{n+1}
            CTQW_TRY(launch_mu(h, dtype, mu_prev, lam, lam2, 1.0, 0.0, 0, s));
            std::swap(lam, lam2);
        }
    }
    if (L.tiled) CTQW_TRY(launch_adjoint_tile_reduce(h, K, dt, tg, grad_eps_dev, grad_J_dev, s));
    // gradients with respect to the means shared by a size group: sums over
    // its realizations, in FP64 and a fixed order
    if (grad_eps_mean_dev) CTQW_TRY(launch_group_sum(h, grad_eps_dev, grad_eps_mean_dev, s));
    if (grad_J_mean_dev) CTQW_TRY(launch_group_sum(h, grad_J_dev, grad_J_mean_dev, s));
    return CTQW_OK;
}

int ctqw_one_body_density(const ctqw_hamiltonian *h, int32_t dtype, const void *psi_dev,
                          double *rho_dev, void *stream) {
    if (!h || !psi_dev || !rho_dev) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    CTQW_CUDA_TRY(cudaMemsetAsync(rho_dev, 0, 2 * sizeof(double) * (size_t)h->joint_width, s));
    if (h->density_method == 0 && one_body_density_tc_supported(h, dtype))
        return launch_one_body_density_tc(h, psi_dev, rho_dev, s);
    return launch_one_body_density(h, dtype, psi_dev, rho_dev, s);
}

int ctqw_set_density_method(ctqw_hamiltonian *h, int32_t method) {
    if (!h) { ctqw_set_error("null handle"); return CTQW_EINVAL; }
    if (method != 0 && method != 1) { ctqw_set_error("density method must be 0 or 1 (got %d)", method); return CTQW_EINVAL; }
    h->density_method = method;
    return CTQW_OK;
}

int ctqw_ensemble_observables(const ctqw_hamiltonian *h, int32_t dtype, const void *psi_dev,
                              double *P_mean_dev, double *P_joint_dev, double *norm_dev,
                              double *energy_dev, void *stream) {
    if (!h || !psi_dev) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    if (P_joint_dev && h->m != 2) { ctqw_set_error("P_joint needs m = 2"); return CTQW_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    CTQW_TRY(zero_outputs(h, 1, P_mean_dev, norm_dev, energy_dev, s));
    if (P_joint_dev) CTQW_CUDA_TRY(cudaMemsetAsync(P_joint_dev, 0, sizeof(double) * h->joint_width, s));
    return launch_observables(h, dtype, psi_dev, P_mean_dev, P_joint_dev, norm_dev, energy_dev, s);
}

}  // extern "C"
