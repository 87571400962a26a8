// C ABI of the graph path: topology checks and CSR construction on the host,
// and the host loops that sequence the graph kernels (Algorithms 2 and 3 on a
// q-dimensional lattice or a general graph, Sec. 2).
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "ctqw_internal.cuh"
#include "graph_internal.cuh"

namespace {

size_t gelem(int dtype) { return dtype == CTQW_C64 ? sizeof(float2) : sizeof(double2); }

int64_t g_samples(int64_t n_steps, int obs_every) { return obs_every > 0 ? n_steps / obs_every + 1 : 0; }

void graph_free(ctqw_graph *g) {
    void *ptrs[] = {g->row_ptr_d, g->col_d, g->link_d, g->eps32, g->w32, g->eps64, g->w64, g->J64};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

template <typename T>
int galloc(T **dst, size_t n) {
    if (ctqw_malloc((void **)dst, std::max<size_t>(1, n) * sizeof(T)) != cudaSuccess) {
        ctqw_set_error("cudaMalloc of %zu bytes failed", n * sizeof(T));
        return CTQW_ENOMEM;
    }
    return CTQW_OK;
}

template <typename T>
int gupload(T **dst, const T *src, size_t n, cudaStream_t s) {
    CTQW_TRY(galloc(dst, n));
    if (n) CTQW_CUDA_TRY(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
    return CTQW_OK;
}

int check_graph_call(const ctqw_graph *g, int dtype, const void *psi, double dt, int64_t n_steps,
                     int obs_every, const void *ws, size_t ws_bytes) {
    if (!g) { ctqw_set_error("null graph handle"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    if (!psi) { ctqw_set_error("null psi"); return CTQW_EINVAL; }
    if (!std::isfinite(dt) || dt == 0.0) { ctqw_set_error("dt must be finite and nonzero"); return CTQW_EINVAL; }
    if (n_steps < 0) { ctqw_set_error("n_steps < 0"); return CTQW_EINVAL; }
    if (obs_every < 0) { ctqw_set_error("obs_every < 0"); return CTQW_EINVAL; }
    const size_t need = 3 * (size_t)g->total_amp * gelem(dtype);
    if (!ws || ws_bytes < need) {
        ctqw_set_error("graph propagation needs a workspace of %zu bytes (got %zu)", need, ws_bytes);
        return CTQW_EINVAL;
    }
    return CTQW_OK;
}

int zero_graph_outputs(const ctqw_graph *g, int64_t n_obs, double *P, double *norm, double *energy,
                       cudaStream_t s) {
    if (n_obs <= 0) return CTQW_OK;
    if (P) CTQW_CUDA_TRY(cudaMemsetAsync(P, 0, sizeof(double) * n_obs * g->N, s));
    if (norm) CTQW_CUDA_TRY(cudaMemsetAsync(norm, 0, sizeof(double) * n_obs * g->R, s));
    if (energy) CTQW_CUDA_TRY(cudaMemsetAsync(energy, 0, sizeof(double) * n_obs * g->R, s));
    return CTQW_OK;
}

int sample(const ctqw_graph *g, int rb, int re, int dtype, const void *psi, int64_t obs, double *P,
           double *norm, double *energy, cudaStream_t s) {
    return launch_graph_observables(g, rb, re, dtype, psi, P ? P + obs * g->N : nullptr,
                                    norm ? norm + obs * g->R : nullptr,
                                    energy ? energy + obs * g->R : nullptr, s);
}

}  // namespace

int graph_chunk(const ctqw_graph *g) { return g->chunk > 0 ? std::min((g->chunk + 3) / 4 * 4, g->R) : g->R; }

extern "C" {

int ctqw_graph_build(const ctqw_graph_desc *d, void *stream, ctqw_graph **out) {
    if (!d || !out) { ctqw_set_error("null desc/out"); return CTQW_EINVAL; }
    *out = nullptr;
    if (d->n_particles != 2 && d->n_particles != 3) {
        ctqw_set_error("n_particles must be 2 or 3 (got %d)", d->n_particles);
        return CTQW_EINVAL;
    }
    if (d->statistics < 0 || d->statistics > 2) { ctqw_set_error("statistics %d", d->statistics); return CTQW_EINVAL; }
    if (d->n_nodes < 2) { ctqw_set_error("n_nodes must be >= 2 (got %d)", d->n_nodes); return CTQW_EINVAL; }
    if (d->n_edges < 0 || d->n_edges > (1 << 29)) { ctqw_set_error("n_edges %d out of range", d->n_edges); return CTQW_EINVAL; }
    if (d->n_edges > 0 && (!d->edge_u || !d->edge_v)) { ctqw_set_error("null link list"); return CTQW_EINVAL; }
    if (d->n_realizations < 1 || d->n_realizations > 65535 * 32) {
        ctqw_set_error("n_realizations must be in 1..%d (got %d)", 65535 * 32, d->n_realizations);
        return CTQW_EINVAL;
    }
    if (!d->u_eps_host || (d->n_edges > 0 && !d->u_J_host)) { ctqw_set_error("null uniform draws"); return CTQW_EINVAL; }
    if (!std::isfinite(d->J0) || !std::isfinite(d->U) || !std::isfinite(d->eps_halfwidth) ||
        !std::isfinite(d->J_halfwidth)) {
        ctqw_set_error("non-finite graph parameter");
        return CTQW_EINVAL;
    }
    int64_t D = 1;
    for (int j = 0; j < d->n_particles; ++j) D *= d->n_nodes;
    if (D > 0x7fffffffLL) { ctqw_set_error("N^m = %lld above 2^31 - 1", (long long)D); return CTQW_EINVAL; }
    if ((double)D * d->n_realizations >= 1099511627776.0) {
        ctqw_set_error("R N^m must be below 2^40");
        return CTQW_EINVAL;
    }
    const int N = d->n_nodes, E = d->n_edges;
    // CSR of the one-particle graph: each link enters the rows of both of
    // its nodes; entries of a row are ordered by neighbour, then by link
    std::vector<int32_t> deg(N + 1, 0);
    for (int e = 0; e < E; ++e) {
        const int u = d->edge_u[e], v = d->edge_v[e];
        if (u < 0 || u >= N || v < 0 || v >= N) { ctqw_set_error("link %d joins a node out of range", e); return CTQW_EINVAL; }
        if (u == v) { ctqw_set_error("link %d joins node %d to itself", e, u); return CTQW_EINVAL; }
        ++deg[u + 1];
        ++deg[v + 1];
    }
    std::vector<int32_t> row_ptr(N + 1, 0);
    for (int i = 0; i < N; ++i) row_ptr[i + 1] = row_ptr[i] + deg[i + 1];
    const int nnz = row_ptr[N];
    std::vector<std::pair<int32_t, int32_t>> entries(nnz);   // (neighbour, link) per CSR slot
    std::vector<int32_t> fill(row_ptr.begin(), row_ptr.end() - 1);
    for (int e = 0; e < E; ++e) {
        const int u = d->edge_u[e], v = d->edge_v[e];
        entries[fill[u]++] = {v, e};
        entries[fill[v]++] = {u, e};
    }
    for (int i = 0; i < N; ++i) std::sort(entries.begin() + row_ptr[i], entries.begin() + row_ptr[i + 1]);
    std::vector<int32_t> col(nnz), link(nnz);
    for (int k = 0; k < nnz; ++k) {
        col[k] = entries[k].first;
        link[k] = entries[k].second;
    }

    auto *g = new ctqw_graph();
    g->m = d->n_particles;
    g->statistics = d->statistics;
    g->N = N;
    g->E = E;
    g->R = d->n_realizations;
    g->round_to_f32 = d->round_to_f32 ? 1 : 0;
    g->J0 = d->J0;
    g->U = d->U;
    g->eps_hw = d->eps_halfwidth;
    g->J_hw = d->J_halfwidth;
    g->D = D;
    g->Rp = (g->R + 3) / 4 * 4;
    g->total_amp = D * g->Rp;
    g->nnz = nnz;
    cudaGetDevice(&g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t RN = (size_t)g->Rp * N, RE = (size_t)g->R * E, RK = (size_t)g->Rp * nnz;
    double *u_eps_d = nullptr, *u_J_d = nullptr;
    int st = CTQW_OK;
    if (st == CTQW_OK) st = gupload(&g->row_ptr_d, row_ptr.data(), row_ptr.size(), s);
    if (st == CTQW_OK) st = gupload(&g->col_d, col.data(), col.size(), s);
    if (st == CTQW_OK) st = gupload(&g->link_d, link.data(), link.size(), s);
    if (st == CTQW_OK) st = galloc(&g->eps32, RN);
    if (st == CTQW_OK) st = galloc(&g->eps64, RN);
    if (st == CTQW_OK) st = galloc(&g->w32, RK);
    if (st == CTQW_OK) st = galloc(&g->w64, RK);
    if (st == CTQW_OK) st = galloc(&g->J64, RE);
    if (st == CTQW_OK) st = gupload(&u_eps_d, d->u_eps_host, (size_t)g->R * N, s);
    if (st == CTQW_OK) st = gupload(&u_J_d, d->u_J_host, RE, s);
    if (st == CTQW_OK) st = launch_graph_build_params(g, u_eps_d, u_J_d, s);
    // the draws are read by the build only: wait for it before freeing them
    if (st == CTQW_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        ctqw_set_error("graph parameter build failed");
        st = CTQW_ECUDA;
    }
    if (u_eps_d) cudaFree(u_eps_d);
    if (u_J_d) cudaFree(u_J_d);
    if (st != CTQW_OK) {
        graph_free(g);
        delete g;
        return st;
    }
    *out = g;
    return CTQW_OK;
}

int ctqw_graph_destroy(ctqw_graph *g) {
    if (!g) return CTQW_OK;
    cudaDeviceSynchronize();
    graph_free(g);
    delete g;
    return CTQW_OK;
}

int ctqw_graph_get_params(const ctqw_graph *g, double *eps_host, double *J_host) {
    if (!g) { ctqw_set_error("null graph handle"); return CTQW_EINVAL; }
    CTQW_CUDA_TRY(cudaDeviceSynchronize());
    if (eps_host) {
        // device eps is [N][Rp]; the caller gets [R][N]
        std::vector<double> t((size_t)g->Rp * g->N);
        CTQW_CUDA_TRY(cudaMemcpy(t.data(), g->eps64, sizeof(double) * t.size(), cudaMemcpyDeviceToHost));
        for (int i = 0; i < g->N; ++i)
            for (int r = 0; r < g->R; ++r) eps_host[(size_t)r * g->N + i] = t[(size_t)i * g->Rp + r];
    }
    if (J_host && g->E > 0)
        CTQW_CUDA_TRY(cudaMemcpy(J_host, g->J64, sizeof(double) * g->R * g->E, cudaMemcpyDeviceToHost));
    return CTQW_OK;
}

int ctqw_graph_state_size(const ctqw_graph *g, int64_t *amplitudes_total) {
    if (!g || !amplitudes_total) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    *amplitudes_total = g->total_amp;
    return CTQW_OK;
}

int ctqw_graph_init_state(const ctqw_graph *g, const int32_t *sites_host, int32_t dtype, void *psi_dev,
                          void *stream) {
    if (!g || !sites_host || !psi_dev) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    for (int r = 0; r < g->R; ++r) {
        const int32_t *x = sites_host + (size_t)r * g->m;
        for (int j = 0; j < g->m; ++j)
            if (x[j] < 0 || x[j] >= g->N) {
                ctqw_set_error("realization %d: node %d out of range", r, x[j]);
                return CTQW_EINVAL;
            }
        if (g->statistics == CTQW_FERMIONS)
            for (int j = 0; j < g->m; ++j)
                for (int l = j + 1; l < g->m; ++l)
                    if (x[j] == x[l]) {
                        ctqw_set_error("realization %d: fermions on one node", r);
                        return CTQW_EINVAL;
                    }
    }
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *sites_d = nullptr;
    CTQW_TRY(gupload(&sites_d, sites_host, (size_t)g->R * g->m, s));
    int st = launch_graph_init_state(g, sites_d, dtype, psi_dev, s);
    // sites_d is read by the kernel just enqueued: free it when the stream gets there
    if (cudaStreamSynchronize(s) != cudaSuccess && st == CTQW_OK) {
        ctqw_set_error("initial-state kernel failed");
        st = CTQW_ECUDA;
    }
    cudaFree(sites_d);
    return st;
}

int ctqw_graph_workspace_size(const ctqw_graph *g, int32_t dtype, size_t *bytes) {
    if (!g || !bytes) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    *bytes = 3 * (size_t)g->total_amp * gelem(dtype);
    return CTQW_OK;
}

int ctqw_graph_propagate_taylor(const ctqw_graph *g, int32_t dtype, void *psi_dev, double dt, int32_t K,
                                int64_t n_steps, int32_t obs_every, double *P_mean_dev, double *norm_dev,
                                double *energy_dev, void *workspace_dev, size_t workspace_bytes,
                                void *stream) {
    CTQW_TRY(check_graph_call(g, dtype, psi_dev, dt, n_steps, obs_every, workspace_dev, workspace_bytes));
    if (K < 1 || K > 30) { ctqw_set_error("K must be in 1..30 (got %d)", K); return CTQW_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t sb = (size_t)g->total_amp * gelem(dtype);
    char *ws = (char *)workspace_dev;
    CTQW_TRY(zero_graph_outputs(g, g_samples(n_steps, obs_every), P_mean_dev, norm_dev, energy_dev, s));
    const int chunk = graph_chunk(g);
    if (dtype == CTQW_C64) {
        // Horner stages w_K = psi + (A/K) psi, w_j = psi + (A/j) w_{j+1},
        // psi += A w_2 (A = -i dt H), the update compensated
        void *wa = ws, *wb = ws + sb, *lo = ws + 2 * sb;
        CTQW_CUDA_TRY(cudaMemsetAsync(lo, 0, sb, s));
        for (int rb = 0; rb < g->R; rb += chunk) {
            const int re = std::min(g->R, rb + chunk);
            int64_t obs = 0;
            for (int64_t step = 0; step <= n_steps; ++step) {
                if (obs_every > 0 && step % obs_every == 0)
                    CTQW_TRY(sample(g, rb, re, dtype, psi_dev, obs++, P_mean_dev, norm_dev, energy_dev, s));
                if (step == n_steps) break;
                const void *in = psi_dev;
                void *out = wa;
                for (int j = K; j >= 2; --j) {
                    CTQW_TRY(launch_graph_horner_stage(g, rb, re, in, psi_dev, out, dt / j, s));
                    in = out;
                    out = (out == wa) ? wb : wa;
                }
                CTQW_TRY(launch_graph_horner_final(g, rb, re, in, psi_dev, lo, dt, s));
            }
        }
        return CTQW_OK;
    }
    // FP64: Phi^(j) = -(i dt / j) H Phi^(j-1) summed forward (Algorithm 3);
    // every chunk takes the same steps, so the state ends in the same buffer
    void *fin = psi_dev;
    for (int rb = 0; rb < g->R; rb += chunk) {
        const int re = std::min(g->R, rb + chunk);
        void *cur = psi_dev, *acc = ws, *phi1 = ws + sb, *phi2 = ws + 2 * sb;
        int64_t obs = 0;
        for (int64_t step = 0; step <= n_steps; ++step) {
            if (obs_every > 0 && step % obs_every == 0)
                CTQW_TRY(sample(g, rb, re, dtype, cur, obs++, P_mean_dev, norm_dev, energy_dev, s));
            if (step == n_steps) break;
            const void *in = cur;
            void *out = phi1;
            for (int j = 1; j <= K; ++j) {
                CTQW_TRY(launch_graph_taylor_term(g, rb, re, dtype, in, out, cur, acc, dt / j, j == 1, s));
                in = out;
                out = (out == phi1) ? phi2 : phi1;
            }
            std::swap(cur, acc);
        }
        fin = cur;
    }
    if (fin != psi_dev) CTQW_CUDA_TRY(cudaMemcpyAsync(psi_dev, fin, sb, cudaMemcpyDeviceToDevice, s));
    return CTQW_OK;
}

int ctqw_graph_propagate_rk4(const ctqw_graph *g, int32_t dtype, void *psi_dev, double dt, int64_t n_steps,
                             int32_t obs_every, double *P_mean_dev, double *norm_dev, double *energy_dev,
                             void *workspace_dev, size_t workspace_bytes, void *stream) {
    CTQW_TRY(check_graph_call(g, dtype, psi_dev, dt, n_steps, obs_every, workspace_dev, workspace_bytes));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t sb = (size_t)g->total_amp * gelem(dtype);
    char *ws = (char *)workspace_dev;
    CTQW_TRY(zero_graph_outputs(g, g_samples(n_steps, obs_every), P_mean_dev, norm_dev, energy_dev, s));
    const int chunk = graph_chunk(g);
    void *fin = psi_dev;
    for (int rb = 0; rb < g->R; rb += chunk) {
        const int re = std::min(g->R, rb + chunk);
        void *cur = psi_dev, *acc = ws, *t1 = ws + sb, *t2 = ws + 2 * sb;
        int64_t obs = 0;
        for (int64_t step = 0; step <= n_steps; ++step) {
            if (obs_every > 0 && step % obs_every == 0)
                CTQW_TRY(sample(g, rb, re, dtype, cur, obs++, P_mean_dev, norm_dev, energy_dev, s));
            if (step == n_steps) break;
            // K1..K4 of Algorithm 2 (classical weights dt (1/6, 1/3, 1/3, 1/6))
            CTQW_TRY(launch_graph_rk4_stage(g, rb, re, dtype, cur, t1, cur, acc, 0.5 * dt, dt / 6.0, 1, s));
            CTQW_TRY(launch_graph_rk4_stage(g, rb, re, dtype, t1, t2, cur, acc, 0.5 * dt, dt / 3.0, 0, s));
            CTQW_TRY(launch_graph_rk4_stage(g, rb, re, dtype, t2, t1, cur, acc, dt, dt / 3.0, 0, s));
            CTQW_TRY(launch_graph_rk4_stage(g, rb, re, dtype, t1, nullptr, cur, acc, 0.0, dt / 6.0, 0, s));
            std::swap(cur, acc);
        }
        fin = cur;
    }
    if (fin != psi_dev) CTQW_CUDA_TRY(cudaMemcpyAsync(psi_dev, fin, sb, cudaMemcpyDeviceToDevice, s));
    return CTQW_OK;
}

int ctqw_graph_set_chunk(ctqw_graph *g, int32_t realizations) {
    if (!g || realizations < 0) { ctqw_set_error("null handle or negative chunk"); return CTQW_EINVAL; }
    g->chunk = realizations;
    return CTQW_OK;
}

int ctqw_graph_observables(const ctqw_graph *g, int32_t dtype, const void *psi_dev, double *P_mean_dev,
                           double *norm_dev, double *energy_dev, void *stream) {
    if (!g || !psi_dev) { ctqw_set_error("null argument"); return CTQW_EINVAL; }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) { ctqw_set_error("dtype %d", dtype); return CTQW_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    CTQW_TRY(zero_graph_outputs(g, 1, P_mean_dev, norm_dev, energy_dev, s));
    return launch_graph_observables(g, 0, g->R, dtype, psi_dev, P_mean_dev, norm_dev, energy_dev, s);
}

}  // extern "C"
