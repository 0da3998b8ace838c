// api.cu -- C ABI of libptca.so (declared in include/ptca.h): argument
// validation, the PTCA stage schedule (Sec. III.a), device state and the
// launch sequence of a sweep.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ptca.h"
#include "context.h"
#include "kernels.cuh"
#include "launch.h"

using ptca::Model;
using ptca::StageArgs;

namespace {

thread_local std::string g_err = "no error";

ptca_status fail(ptca_status s, const std::string& msg) {
    g_err = msg;
    return s;
}
ptca_status cuda_fail(cudaError_t e, const char* where) {
    return fail(e == cudaErrorMemoryAllocation ? PTCA_ERR_OOM : PTCA_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}
#define PTCA_CUDA(call)                                              \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);          \
    } while (0)
// Complete a re-solve an overlapped sweep left pending before touching the
// configuration (stream-ordered on st), or before changing how the next sweep
// runs (synchronously).
#define PTCA_SETTLE(ctx, st) PTCA_CUDA(ptca_internal_settle((ctx), (st), true))
#define PTCA_SETTLE_SYNC(ctx) PTCA_CUDA(ptca_internal_settle((ctx), nullptr, false))



// Window along one axis (same rule as the device code).
void window_axis(int L, int periodic, int Lc, int o, int c, int& start, int& ext) {
    if (L == 1) { start = 0; ext = 1; return; }
    int a = c - o, b = c - o + Lc - 1;
    if (periodic) { start = ((a % L) + L) % L; ext = Lc; return; }
    if (a < 0) a = 0;
    if (b > L - 1) b = L - 1;
    start = a; ext = b - a + 1;
}

// Window of an update site on the host (the device's make_window): start and
// extent along each axis.  Sites are indexed (z Ly + y) Lx + x.
struct HostWindow { int x0, y0, z0, ex, ey, ez; };

HostWindow host_window(const Problem& p, int site) {
    HostWindow w;
    window_axis(p.Lx, p.periodic, p.Lc, p.ox, site % p.Lx, w.x0, w.ex);
    window_axis(p.Ly, p.periodic, p.Lc, p.oy, (site / p.Lx) % p.Ly, w.y0, w.ey);
    window_axis(p.Lz, p.periodic, p.Lc, p.oz, site / (p.Lx * p.Ly), w.z0, w.ez);
    return w;
}

// Calls f(g) for every lattice site g of the window of `site`; stops and
// returns true as soon as f returns true.
template <typename F> bool any_window_site(const Problem& p, int site, F f) {
    const HostWindow w = host_window(p, site);
    for (int wz = 0; wz < w.ez; ++wz)
        for (int wy = 0; wy < w.ey; ++wy)
            for (int wx = 0; wx < w.ex; ++wx) {
                int x = w.x0 + wx, y = w.y0 + wy, z = w.z0 + wz;
                if (p.periodic) { x %= p.Lx; y %= p.Ly; z %= p.Lz; }
                if (f((z * p.Ly + y) * p.Lx + x)) return true;
            }
    return false;
}

// Stage lists.  Tiled: stage (ax, ay, az) holds (ax + s p, ay + s q, az + s r),
// row-major; block: the lattice halved along each axis of extent > 1, 2^d
// blocks (Sec. III.a: four in two dimensions, eight in three), each block one
// stage, row-major inside.
void make_schedule(const Problem& p, std::vector<int32_t>& start, std::vector<int32_t>& sites) {
    start.assign(1, 0);
    sites.clear();
    sites.reserve(p.N());
    auto idx = [&](int x, int y, int z) { return (int32_t)((z * p.Ly + y) * p.Lx + x); };
    if (p.schedule == PTCA_SCHEDULE_TILED) {
        const int s = p.stride, sy = p.Ly == 1 ? 1 : s, sz = p.Lz == 1 ? 1 : s;
        for (int az = 0; az < sz && az < p.Lz; ++az)
            for (int ay = 0; ay < sy && ay < p.Ly; ++ay)
                for (int ax = 0; ax < s && ax < p.Lx; ++ax) {
                    for (int z = az; z < p.Lz; z += sz)
                        for (int y = ay; y < p.Ly; y += sy)
                            for (int x = ax; x < p.Lx; x += s) sites.push_back(idx(x, y, z));
                    start.push_back((int32_t)sites.size());
                }
    } else {
        const int hx = (p.Lx + 1) / 2, hy = (p.Ly + 1) / 2, hz = (p.Lz + 1) / 2;
        const int nby = p.Ly == 1 ? 1 : 2, nbz = p.Lz == 1 ? 1 : 2;
        for (int bz = 0; bz < nbz; ++bz)
            for (int by = 0; by < nby; ++by)
                for (int bx = 0; bx < 2; ++bx) {
                    const int xa = bx ? hx : 0, xb = bx ? p.Lx : hx;
                    const int ya = p.Ly == 1 ? 0 : (by ? hy : 0), yb = p.Ly == 1 ? 1 : (by ? p.Ly : hy);
                    const int za = p.Lz == 1 ? 0 : (bz ? hz : 0), zb = p.Lz == 1 ? 1 : (bz ? p.Lz : hz);
                    for (int z = za; z < zb; ++z)
                        for (int y = ya; y < yb; ++y)
                            for (int x = xa; x < xb; ++x) sites.push_back(idx(x, y, z));
                    if ((int32_t)sites.size() > start.back()) start.push_back((int32_t)sites.size());
                }
    }
}

// Concurrent processing of a stage from its start configuration equals
// visiting its sites one after another iff no site of the stage lies in the
// window of a site listed after it.  Checked exactly over every window.
bool schedule_exact(const Problem& p, const std::vector<int32_t>& start, const std::vector<int32_t>& sites,
                    std::string& why) {
    const int N = p.N();
    std::vector<int32_t> stage_of(N, -1), pos(N, -1);
    for (size_t s = 0; s + 1 < start.size(); ++s)
        for (int k = start[s]; k < start[s + 1]; ++k) { stage_of[sites[k]] = (int)s; pos[sites[k]] = k; }
    for (int k = 0; k < N; ++k) {
        const int b = sites[k];
        int bad = -1;
        any_window_site(p, b, [&](int g) {
            if (g != b && stage_of[g] == stage_of[b] && pos[g] < pos[b]) { bad = g; return true; }
            return false;
        });
        if (bad >= 0) {
            char buf[160];
            snprintf(buf, sizeof buf, "site %d lies in the window of site %d of the same stage", bad, b);
            why = buf;
            return false;
        }
    }
    return true;
}

// Work order inside each stage: largest window first (ragged windows of open
// lattices), stable, so periodic lattices keep schedule order.  perm[k] for k
// in stage s's range is an index into that stage's site list.
std::vector<int32_t> window_order(const Problem& p, const std::vector<int32_t>& start,
                                  const std::vector<int32_t>& sites) {
    std::vector<int32_t> perm(sites.size());
    for (size_t stg = 0; stg + 1 < start.size(); ++stg) {
        const int a0 = start[stg], a1 = start[stg + 1];
        std::vector<std::pair<int, int>> key;
        for (int k = a0; k < a1; ++k) {
            const HostWindow w = host_window(p, sites[k]);
            key.push_back({-(w.ex * w.ey * w.ez), k - a0});
        }
        std::stable_sort(key.begin(), key.end(),
                         [](const std::pair<int, int>& u, const std::pair<int, int>& v) { return u.first < v.first; });
        for (int k = a0; k < a1; ++k) perm[k] = key[k - a0].second;
    }
    return perm;
}

// Split of every stage's work order (window_order) into the visits whose
// window holds no site of the previous stage (cyclically: stage 0 follows the
// last stage), first, and the rest; indep[s] counts the first part.
void stage_split(const Problem& p, const std::vector<int32_t>& start, const std::vector<int32_t>& sites,
                 std::vector<int32_t>& order, std::vector<int32_t>& indep) {
    const int ns = (int)start.size() - 1, N = p.N();
    const std::vector<int32_t> perm = window_order(p, start, sites);
    order.assign(sites.size(), 0);
    indep.assign(ns, 0);
    std::vector<int32_t> stage_of(N, -1);
    for (int s = 0; s < ns; ++s)
        for (int k = start[s]; k < start[s + 1]; ++k) stage_of[sites[k]] = s;
    for (int s = 0; s < ns; ++s) {
        const int q = (s + ns - 1) % ns;
        std::vector<int32_t> a, b;
        for (int k = start[s]; k < start[s + 1]; ++k) {
            const int c = perm[k], site = sites[start[s] + c];
            const bool dep = any_window_site(p, site, [&](int g) { return stage_of[g] == q; });
            (dep ? b : a).push_back(c);
        }
        indep[s] = (int32_t)a.size();
        std::copy(a.begin(), a.end(), order.begin() + start[s]);
        std::copy(b.begin(), b.end(), order.begin() + start[s] + a.size());
    }
}

ptca_status resolve(const ptca_lattice* lat, const ptca_params* par, Problem& p) {
    if (!lat || !par) return fail(PTCA_ERR_INVALID, "null lattice or params");
    p.Lx = lat->Lx; p.Ly = lat->Ly; p.periodic = lat->periodic ? 1 : 0;
    p.Lz = lat->Lz == 0 ? 1 : lat->Lz;
    if (p.Lx < 1 || p.Ly < 1 || p.Lz < 1 || (int64_t)p.Lx * p.Ly * p.Lz > (1 << 26))
        return fail(PTCA_ERR_INVALID, "lattice extents out of range");
    if (p.Lz > 1 && p.Ly == 1) return fail(PTCA_ERR_INVALID, "a cubic lattice (Lz > 1) needs Ly > 1");
    p.Lc = par->L_c;
    if (p.Lc < 2 || p.Lc > p.Lx || (p.Ly > 1 && p.Lc > p.Ly) || (p.Lz > 1 && p.Lc > p.Lz))
        return fail(PTCA_ERR_INVALID, "L_c must satisfy 2 <= L_c <= min(Lx, Ly, Lz)");
    p.schedule = par->schedule;
    if (p.schedule != PTCA_SCHEDULE_TILED && p.schedule != PTCA_SCHEDULE_BLOCK)
        return fail(PTCA_ERR_INVALID, "unknown schedule");
    int o = par->update_offset;
    if (o < 0) o = p.schedule == PTCA_SCHEDULE_TILED ? p.Lc / 2 : 0;
    if (o >= p.Lc) return fail(PTCA_ERR_INVALID, "update_offset must be < L_c");
    p.ox = o;
    p.oy = p.Ly == 1 ? 0 : o;
    p.oz = p.Lz == 1 ? 0 : o;
    p.cluster_periodic = par->cluster_periodic < 0 ? p.periodic : (par->cluster_periodic ? 1 : 0);
    p.stride = par->stride > 0 ? par->stride : p.Lc;
    if (p.schedule == PTCA_SCHEDULE_TILED && p.periodic &&
        (p.Lx % p.stride != 0 || (p.Ly > 1 && p.Ly % p.stride != 0) || (p.Lz > 1 && p.Lz % p.stride != 0)))
        return fail(PTCA_ERR_INVALID, "tiled stride must divide the lattice extents on a torus");
    p.precision = par->precision;
    if (p.precision != PTCA_FP64 && p.precision != PTCA_MIXED) return fail(PTCA_ERR_INVALID, "unknown precision");
    p.proposal = par->proposal;
    if (p.proposal != PTCA_PROPOSAL_SPHERE && p.proposal != PTCA_PROPOSAL_CONE)
        return fail(PTCA_ERR_INVALID, "unknown proposal");
    p.t = par->t; p.JH = par->J_H; p.mu = par->mu; p.T = par->T; p.cone_deg = par->cone_deg; p.seed = par->seed;
    p.model = par->model;
    p.U = par->U;
    p.m_step = par->m_step;
    p.lam = par->lam;
    p.K = par->K;
    if (p.model != PTCA_MODEL_DOUBLE_EXCHANGE && p.model != PTCA_MODEL_HUBBARD_MF && p.model != PTCA_MODEL_HOLSTEIN)
        return fail(PTCA_ERR_INVALID, "unknown model");
    if (p.model != PTCA_MODEL_DOUBLE_EXCHANGE && (!(p.m_step > 0) || !std::isfinite(p.m_step)))
        return fail(PTCA_ERR_INVALID, "the Hubbard and Holstein models need a finite m_step > 0");
    if (p.model == PTCA_MODEL_HUBBARD_MF && !std::isfinite(p.U))
        return fail(PTCA_ERR_INVALID, "Hubbard mean field needs a finite U");
    if (p.model == PTCA_MODEL_HOLSTEIN && (!std::isfinite(p.lam) || !std::isfinite(p.K)))
        return fail(PTCA_ERR_INVALID, "Holstein needs finite lambda and K");
    if (!std::isfinite(p.t) || !std::isfinite(p.JH) || !std::isfinite(p.mu) || !std::isfinite(p.T) || !(p.T > 0))
        return fail(PTCA_ERR_INVALID, "t, J_H, mu must be finite and T > 0");
    if (p.proposal == PTCA_PROPOSAL_CONE && !(p.cone_deg > 0 && p.cone_deg <= 180))
        return fail(PTCA_ERR_INVALID, "cone_deg must lie in (0, 180]");
    if (p.nmax() > ptca::cluster_max_order(p.precision == PTCA_MIXED ? 1 : 0) && p.nmax() > ptca::large_max_order())
        return fail(PTCA_ERR_INVALID, "cluster matrix order 2*N_c exceeds the supported maximum (512)");
    return PTCA_OK;
}

Model to_model(const Problem& p) {
    Model m;
    m.Lx = p.Lx; m.Ly = p.Ly; m.Lz = p.Lz; m.lattice_periodic = p.periodic;
    m.Lc = p.Lc; m.ox = p.ox; m.oy = p.oy; m.oz = p.oz; m.cluster_periodic = p.cluster_periodic;
    m.proposal = p.proposal;
    m.t = p.t; m.mu = p.mu; m.T = p.T;
    m.cone_cos = std::cos(p.cone_deg * ptca::kPi / 180.0);
    ptca::set_model_terms(m, p.model, p.JH, p.U, p.lam, p.K, p.mu, p.m_step);
    m.seed = p.seed;
    return m;
}

template <typename T> cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
}

}  // namespace


static void drop_graph(ptca_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_sweeps = -1;
}

// A launch solving `items` cluster matrices, bracketed by events on `st` when
// kernel timing is on.
template <typename F>
static cudaError_t timed_launch(ptca_ctx* ctx, int kind, int64_t items, cudaStream_t st, F launch) {
    if (!ctx->timing) return launch();
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e != cudaSuccess) {
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        return e;
    }
    ctx->tev.push_back(ev[0]);
    ctx->tev.push_back(ev[1]);
    ctx->tkind.push_back(kind);
    ctx->titems.push_back(items);
    return cudaSuccess;
}

static void drop_timing_events(ptca_ctx* c) {
    for (cudaEvent_t ev : c->tev) cudaEventDestroy(ev);
    c->tev.clear();
    c->tkind.clear();
    c->titems.clear();
}

static void free_ctx(ptca_ctx* c) {
    drop_graph(c);
    drop_timing_events(c);
    ptca_free_surrogate(c);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->side2) cudaStreamDestroy(c->side2);
    for (cudaEvent_t ev : {c->ev_fork, c->ev_join, c->ev_ind[0], c->ev_ind[1], c->ev_res[0], c->ev_res[1]})
        if (ev) cudaEventDestroy(ev);
    void* ptrs[] = {c->d_sites, c->d_S[0], c->d_S[1], c->d_S[2], c->d_S[3], c->d_split, c->d_gL, c->d_F, c->d_fill, c->d_ticket, c->d_rec_site,
                    c->d_rec_Fold, c->d_rec_Fnew, c->d_rec_lnu, c->d_rec_acc, c->d_rec_Facc, c->d_rec_fill,
                    c->d_rec_n, c->d_counters, c->d_err, c->d_obs, c->d_stage_start, c->d_perm, c->d_queue,
                    c->d_bar, c->d_sweep_ctr, c->d_flag_list, c->d_flag_count, c->d_gA,
                    c->d_chk_eig, c->d_chk_F, c->d_chk_out, c->d_sub, c->d_sub_spins};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete c;
}

// Failure reporting for the other translation units of the library.
ptca_status ptca_internal_fail(ptca_status s, const char* msg) { return fail(s, msg); }

// The device-side problem description of a context (for the other
// translation units of the library).
ptca::Model ptca_context_model(const ptca_ctx* ctx) { return to_model(ctx->p); }

extern "C" {

int32_t ptca_version(void) { return PTCA_VERSION_MAJOR * 100 + PTCA_VERSION_MINOR; }

const char* ptca_last_error(void) { return g_err.c_str(); }

ptca_status ptca_schedule(const ptca_lattice* lattice, const ptca_params* params, int32_t* stage_start,
                          int32_t* sites, int32_t* n_stages) {
    Problem p;
    ptca_status s = resolve(lattice, params, p);
    if (s != PTCA_OK) return s;
    if (!stage_start || !sites || !n_stages) return fail(PTCA_ERR_INVALID, "null output pointer");
    std::vector<int32_t> st, si;
    make_schedule(p, st, si);
    std::string why;
    if (!schedule_exact(p, st, si, why)) return fail(PTCA_ERR_INVALID, "schedule is not exact: " + why);
    std::memcpy(stage_start, st.data(), st.size() * sizeof(int32_t));
    std::memcpy(sites, si.data(), si.size() * sizeof(int32_t));
    *n_stages = (int32_t)st.size() - 1;
    return PTCA_OK;
}

ptca_status ptca_stage_split(const ptca_lattice* lattice, const ptca_params* params, int32_t* order,
                             int32_t* n_indep) {
    Problem p;
    ptca_status s = resolve(lattice, params, p);
    if (s != PTCA_OK) return s;
    if (!order || !n_indep) return fail(PTCA_ERR_INVALID, "null output pointer");
    std::vector<int32_t> st, si, ord, ind;
    make_schedule(p, st, si);
    std::string why;
    if (!schedule_exact(p, st, si, why)) return fail(PTCA_ERR_INVALID, "schedule is not exact: " + why);
    stage_split(p, st, si, ord, ind);
    std::memcpy(order, ord.data(), ord.size() * sizeof(int32_t));
    std::memcpy(n_indep, ind.data(), ind.size() * sizeof(int32_t));
    return PTCA_OK;
}

// Default re-solve margin of a PTCA_MIXED context (unless the caller set
// one): 5 to 10 times beta times the largest FP32 dF error measured for its
// reduction.  The per-matrix reductions leave up to about 2e-4 (n = 128 to
// 288), hence 1e-2; the large-cluster shared reduction, whose chases run in
// double-float, about 5e-7, hence 1e-4.
static void default_margin(ptca_ctx* c) {
    if (c->prec != 1 || c->margin_set) return;
    c->margin = (c->large && c->reduction == 2) ? 1e-4 : 1e-2;
}

ptca_status ptca_init(const ptca_lattice* lattice, const ptca_params* params, ptca_ctx** out) {
    if (!out) return fail(PTCA_ERR_INVALID, "null out");
    *out = nullptr;
    Problem p;
    ptca_status s = resolve(lattice, params, p);
    if (s != PTCA_OK) return s;
    std::vector<int32_t> st, si;
    make_schedule(p, st, si);
    std::string why;
    if (!schedule_exact(p, st, si, why)) return fail(PTCA_ERR_INVALID, "schedule is not exact: " + why);

    int dev = 0, ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return fail(PTCA_ERR_CUDA, "no CUDA device available");
    PTCA_CUDA(cudaGetDevice(&dev));
    int optin = 0;
    PTCA_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

    ptca_ctx* c = new ptca_ctx();
    c->p = p;
    c->device = dev;
    c->prec = p.precision == PTCA_MIXED ? 1 : 0;
    c->N = p.N();
    c->h_start = st;
    c->h_sites = si;
    c->nstages = (int)st.size() - 1;
    for (int k = 0; k < c->nstages; ++k) c->max_stage = std::max(c->max_stage, st[k + 1] - st[k]);
    c->nA = p.nmax();
    c->large = c->nA > ptca::cluster_max_order(c->prec);
    c->smem = c->large ? ptca::large_smem_bytes(c->prec) : ptca::cluster_smem_bytes(c->prec, c->nA);
    if (c->smem == 0 || c->smem + 256 > (size_t)optin) {
        delete c;
        return fail(PTCA_ERR_INVALID, "cluster kernels do not fit in shared memory on this device");
    }
    cudaError_t ce = ptca::configure_cluster_kernels((size_t)optin);
    if (ce == cudaSuccess && c->large) ce = ptca::configure_large_kernels((size_t)optin);
    if (ce != cudaSuccess) {
        delete c;
        return cuda_fail(ce, "ptca_init (configuring kernel shared memory)");
    }
    const int N = c->N;
    if (ce == cudaSuccess) ce = dalloc(&c->d_sites, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_S[0], 3 * (size_t)N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_S[1], 3 * (size_t)N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_F, 4 * (size_t)c->max_stage);
    if (ce == cudaSuccess) ce = dalloc(&c->d_fill, 4 * (size_t)c->max_stage);
    if (ce == cudaSuccess) ce = dalloc(&c->d_ticket, 2 * (size_t)c->max_stage);
    if (ce == cudaSuccess) ce = dalloc(&c->d_rec_site, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_rec_Fold, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_rec_Fnew, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_rec_lnu, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_rec_acc, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_rec_Facc, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_rec_fill, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_rec_n, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_counters, 4);
    if (ce == cudaSuccess) ce = dalloc(&c->d_err, 2);
    if (ce == cudaSuccess) ce = dalloc(&c->d_stage_start, c->nstages + 1);
    if (ce == cudaSuccess) ce = dalloc(&c->d_perm, N);
    if (ce == cudaSuccess) ce = dalloc(&c->d_queue, 3);
    if (ce == cudaSuccess) ce = dalloc(&c->d_flag_list, 2 * (size_t)c->max_stage);
    if (ce == cudaSuccess) ce = dalloc(&c->d_flag_count, 2);
    if (ce == cudaSuccess) ce = dalloc(&c->d_bar, 2);
    if (ce == cudaSuccess) ce = dalloc(&c->d_sweep_ctr, 1);
    if (ce == cudaSuccess) ce = dalloc(&c->d_obs, 8);
    if (ce == cudaSuccess) ce = cudaMemcpy(c->d_sites, si.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(c->d_ticket, 0, 2 * (size_t)c->max_stage * sizeof(int32_t));
    if (ce == cudaSuccess) ce = cudaMemset(c->d_err, 0, 2 * sizeof(int32_t));
    if (ce == cudaSuccess) ce = cudaMemset(c->d_queue, 0, 3 * sizeof(unsigned int));
    if (ce == cudaSuccess) ce = cudaMemset(c->d_flag_count, 0, 2 * sizeof(unsigned int));
    if (ce == cudaSuccess) ce = cudaMemset(c->d_bar, 0, 2 * sizeof(unsigned int));
    if (ce == cudaSuccess) ce = cudaMemset(c->d_sweep_ctr, 0, sizeof(unsigned long long));
    if (ce == cudaSuccess) {
        const std::vector<int32_t> perm = window_order(p, st, si);
        ce = cudaMemcpy(c->d_perm, perm.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess) ce = cudaMemcpy(c->d_stage_start, st.data(), (c->nstages + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        c->sms = sms;
        c->grid = c->large ? sms * ptca::persistent_blocks_per_sm_large(c->prec)
                           : sms * ptca::persistent_blocks_per_sm(c->prec, 8, c->nA);
        // Large clusters start on the per-stage pipeline (the persistent one
        // is slower there and is chosen explicitly).
        if (c->grid <= 0 || c->large) c->pipeline = PTCA_PIPELINE_STAGES;
        if (c->large) {
            // One global matrix slot per resident CTA of the large-cluster
            // stage kernel, three times: the overlapped pipeline runs the
            // independent visits of two consecutive stages (one set each, by
            // stage parity) and a stage's dependent visits (the third set) as
            // concurrent launches (+ 64 elements of padding, as below).
            c->large_grid = sms * std::max(1, ptca::large_blocks_per_sm(c->prec));
            if (c->prec == 1) {
                c->cl_size = ptca::cluster_stage_size(c->nA, (size_t)optin);
                c->cl_grid = c->cl_size ? ptca::cluster_stage_grid(c->cl_size, c->nA) : 0;
                if (c->cl_grid <= 0) c->cl_size = 0;
            }
            // Default: the 16-warp kernel with the matrix in global memory,
            // measured faster than the cluster kernel at orders 288 and 512
            // (the autotuner times both); in PTCA_MIXED with one reduction
            // shared by the two matrices of a visit, faster still and with a
            // far smaller dF error (its chases run in double-float).
            c->nw = 16;
            if (c->prec == 1 && ptca::large_shared_supported(c->prec, c->nA, (size_t)optin)) c->reduction = 2;
            c->gL_stride = (int64_t)c->nA * (c->nA + 1) / 2;
            const size_t es = c->prec == 1 ? sizeof(float2) : sizeof(double2);
            void* q = nullptr;
            ce = cudaMalloc(&q, (3 * (size_t)c->large_grid * (size_t)c->gL_stride + 64) * es);
            c->d_gL = q;
        }
        if (ce == cudaSuccess && c->prec == 1) {
            // Global slots for the re-solves: one per CTA of any launch
            // configuration (the narrowest CTAs give the widest persistent grid).
            c->resolve_grid = sms;
            int widest = c->grid;
            for (int nw : {4, 1})
                if (ptca::sweep_width_supported(c->prec, nw, c->nA))
                    widest = std::max(widest, sms * ptca::persistent_blocks_per_sm(c->prec, nw, c->nA));
            const int slots = std::max(std::max(widest, c->resolve_grid), c->large ? c->large_grid : 0);
            c->gA_stride = (int64_t)c->nA * (c->nA + 1) / 2;
            // + 64 elements: the fused pass may load up to 31 elements past a
            // slot (masked lanes of the diagonal chunk), also past the last.
            ce = dalloc(&c->d_gA, (size_t)slots * (size_t)c->gA_stride + 64);
            default_margin(c);
        }
    }
    if (ce == cudaSuccess) ce = cudaMemset(c->d_rec_acc, 0, N);
    if (ce == cudaSuccess) ce = cudaMemset(c->d_rec_Facc, 0, N * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemset(c->d_rec_fill, 0, N * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemset(c->d_rec_n, 0, N * sizeof(int32_t));
    const Model m = to_model(p);
    if (ce == cudaSuccess) ce = ptca::launch_init_spins(m, c->d_S[0], N, 0);
    if (ce == cudaSuccess) ce = cudaMemcpy(c->d_S[1], c->d_S[0], 3 * (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice);
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(ce, "ptca_init");
    }
    *out = c;
    return PTCA_OK;
}

ptca_status ptca_destroy(ptca_ctx* ctx) {
    if (!ctx) return PTCA_OK;
    cudaDeviceSynchronize();
    free_ctx(ctx);
    return PTCA_OK;
}

ptca_status ptca_set_T(ptca_ctx* ctx, double T) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (!(T > 0) || !std::isfinite(T)) return fail(PTCA_ERR_INVALID, "T must be finite and > 0");
    PTCA_SETTLE_SYNC(ctx);
    ctx->p.T = T;
    drop_graph(ctx);
    return PTCA_OK;
}

ptca_status ptca_set_mu(ptca_ctx* ctx, double mu) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (!std::isfinite(mu)) return fail(PTCA_ERR_INVALID, "mu must be finite");
    PTCA_SETTLE_SYNC(ctx);
    ctx->p.mu = mu;
    drop_graph(ctx);
    return PTCA_OK;
}

ptca_status ptca_get_spins(ptca_ctx* ctx, double* dst, int on_device, void* stream) {
    if (!ctx || !dst) return fail(PTCA_ERR_INVALID, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    const size_t bytes = 3 * (size_t)ctx->N * sizeof(double);
    PTCA_CUDA(cudaMemcpyAsync(dst, ctx->d_S[0], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!on_device) PTCA_CUDA(cudaStreamSynchronize(st));
    return PTCA_OK;
}

ptca_status ptca_set_spins(ptca_ctx* ctx, const double* src, int on_device, void* stream) {
    if (!ctx || !src) return fail(PTCA_ERR_INVALID, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    const size_t bytes = 3 * (size_t)ctx->N * sizeof(double);
    PTCA_CUDA(cudaMemcpyAsync(ctx->d_S[0], src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    PTCA_CUDA(cudaMemcpyAsync(ctx->d_S[1], ctx->d_S[0], bytes, cudaMemcpyDeviceToDevice, st));
    if (!on_device) PTCA_CUDA(cudaStreamSynchronize(st));
    return PTCA_OK;
}

ptca_status ptca_dims(const ptca_ctx* ctx, int32_t* nmax, int64_t* packed_stride) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (nmax) *nmax = ctx->nA;
    if (packed_stride) *packed_stride = (int64_t)ctx->nA * (ctx->nA + 1) / 2;
    return PTCA_OK;
}

ptca_status ptca_build_clusters(ptca_ctx* ctx, const int32_t* sites, int32_t m, const double* new_spins,
                                void* H_out, int64_t* offsets_out, int32_t* n_out, void* stream) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (m < 0) return fail(PTCA_ERR_INVALID, "m < 0");
    if (m == 0) return PTCA_OK;
    if (!sites || !H_out || !offsets_out || !n_out) return fail(PTCA_ERR_INVALID, "null buffer");
    const int64_t stride = (int64_t)ctx->nA * (ctx->nA + 1) / 2;
    PTCA_SETTLE(ctx, static_cast<cudaStream_t>(stream));
    PTCA_CUDA(ptca::launch_build(ctx->prec, to_model(ctx->p), ctx->d_S[0], sites, m, new_spins, H_out, stride,
                                 offsets_out, n_out, static_cast<cudaStream_t>(stream)));
    return PTCA_OK;
}

ptca_status ptca_cluster_eigvals(ptca_ctx* ctx, const void* H, const int64_t* offsets, const int32_t* n, int32_t m,
                                 double* eig_out, const int64_t* eig_offsets, void* stream) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (m < 0) return fail(PTCA_ERR_INVALID, "m < 0");
    if (m == 0) return PTCA_OK;
    if (!H || !offsets || !n || !eig_out || !eig_offsets) return fail(PTCA_ERR_INVALID, "null buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ctx->large) {
        // the matrices are reduced in the context's large-cluster slots
        PTCA_SETTLE(ctx, st);
        PTCA_CUDA(ptca::launch_eigvals_large(ctx->prec, H, offsets, n, m, ctx->nA, eig_out, eig_offsets, ctx->d_gL,
                                             ctx->gL_stride, ctx->large_grid, st));
        return PTCA_OK;
    }
    PTCA_CUDA(ptca::launch_eigvals(ctx->prec, ctx->nA, H, offsets, n, m, eig_out, eig_offsets, st));
    return PTCA_OK;
}

ptca_status ptca_free_energy(ptca_ctx* ctx, const double* eig, const int64_t* eig_offsets, const int32_t* n,
                             int32_t m, double mu, double T, double* F_out, void* stream) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (m < 0) return fail(PTCA_ERR_INVALID, "m < 0");
    if (!(T > 0) || !std::isfinite(T) || !std::isfinite(mu)) return fail(PTCA_ERR_INVALID, "bad mu or T");
    if (m == 0) return PTCA_OK;
    if (!eig || !eig_offsets || !n || !F_out) return fail(PTCA_ERR_INVALID, "null buffer");
    PTCA_CUDA(ptca::launch_free_energy(eig, eig_offsets, n, m, mu, T, F_out, static_cast<cudaStream_t>(stream)));
    return PTCA_OK;
}

static StageArgs base_args(ptca_ctx* ctx) {
    StageArgs a;
    std::memset(&a, 0, sizeof a);
    a.m = to_model(ctx->p);
    a.nA = ctx->nA;
    a.Fbuf = ctx->d_F;
    a.fillbuf = ctx->d_fill;
    a.ticket = ctx->d_ticket;
    a.rec_site = ctx->d_rec_site;
    a.rec_Fold = ctx->d_rec_Fold;
    a.rec_Fnew = ctx->d_rec_Fnew;
    a.rec_lnu = ctx->d_rec_lnu;
    a.rec_acc = ctx->d_rec_acc;
    a.rec_Facc = ctx->d_rec_Facc;
    a.rec_fill = ctx->d_rec_fill;
    a.rec_n = ctx->d_rec_n;
    a.counters = ctx->d_counters;
    a.err = ctx->d_err;
    a.margin = ctx->prec == 1 ? ctx->margin : 0.0;
    a.flag_list = ctx->d_flag_list;
    a.flag_count = ctx->d_flag_count;
    a.gA = ctx->d_gA;
    a.gA_stride = ctx->gA_stride;
    a.gL = ctx->d_gL;
    a.gL_stride = ctx->gL_stride;
    return a;
}

cudaError_t ptca_screen_stage(ptca_ctx* ctx, ptca::StageArgs& a, cudaStream_t st);
cudaError_t ptca_screen_part(ptca_ctx* ctx, ptca::StageArgs& a, int part, int row_base, int half, cudaStream_t st);

// A stage launch and a re-solve launch in the context's configuration
// (shared-memory kernels, or the large-cluster kernels).
static cudaError_t launch_stage_ctx(const ptca_ctx* ctx, const StageArgs& a, cudaStream_t st) {
    if (ctx->large && ctx->reduction == 2) return ptca::launch_stage_large_shared(a, ctx->large_grid, st);
    if (ctx->large && ctx->prec == 1 && ctx->nw == 8 && ctx->cl_size > 0)
        return ptca::launch_stage_cluster(ctx->cl_size, a, ctx->cl_grid, st);
    if (ctx->large) return ptca::launch_stage_large(ctx->prec, a, ctx->large_grid, st);
    if (ctx->reduction == 2) return ptca::launch_stage_shared(a, st);
    if (ctx->reduction == 1) return ptca::launch_stage_tiled(a, st);
    if (ctx->panel > 1) return ptca::launch_stage_panel(ctx->panel, a, st);
    return ptca::launch_stage(ctx->prec, ctx->nw, a, st);
}
static cudaError_t launch_resolve_ctx(const ptca_ctx* ctx, const StageArgs& a, cudaStream_t st) {
    if (ctx->large) return ptca::launch_resolve_large(a, ctx->resolve_grid, st);
    return ptca::launch_resolve(a, ctx->resolve_grid, st);
}

// Training-sample destination of ptca_surrogate_collect (N rows per sweep).
struct Collect {
    float* feat;
    int32_t* center;
    float* dF;
};

// Precision checker of one stage: every visit's two matrices solved with the
// FP32 reduction and in FP64 from the stage-start spins, errors max-reduced
// into the stage's row of d_chk_out.  Does not change the chain.
static cudaError_t check_stage(ptca_ctx* ctx, const StageArgs& a, int s, cudaStream_t st) {
    const int ld = ctx->nA, chunk = ctx->check_chunk;
    double* e32 = ctx->d_chk_eig;
    double* e64 = e32 + (size_t)chunk * 2 * ld;
    double* F32 = ctx->d_chk_F;
    double* F64 = F32 + 2 * (size_t)chunk;
    cudaError_t e = cudaSuccess;
    for (int c0 = 0; c0 < a.count && e == cudaSuccess; c0 += chunk) {
        const int cnt = std::min(chunk, a.count - c0);
        if (ctx->large) {
            e = ptca::launch_check_large(1, a, c0, cnt, e32, ld, F32, ctx->large_grid, st);
            if (e == cudaSuccess) e = ptca::launch_check_large(0, a, c0, cnt, e64, ld, F64, ctx->resolve_grid, st);
        } else {
            e = ptca::launch_check(1, a, c0, cnt, e32, ld, F32, 0, st);
            if (e == cudaSuccess) e = ptca::launch_check(0, a, c0, cnt, e64, ld, F64, ctx->resolve_grid, st);
        }
        if (e == cudaSuccess)
            e = ptca::launch_check_compare(a.m, a.sites + c0, cnt, e32, e64, ld, F32, F64, ctx->d_chk_out + ptca::kCheckCols * s, st);
    }
    return e;
}

// One launch per stage (Sec. III.a stage = one kernel); with the surrogate
// enabled each stage is screened first and only passing sites are solved.
static cudaError_t sweep_stages(ptca_ctx* ctx, int32_t n_sweeps, cudaStream_t st, const Collect* col = nullptr) {
    StageArgs a = base_args(ctx);
    int64_t g = 0;
    int prev_s = -1;
    cudaError_t e = cudaSuccess;
    for (int sw = 0; sw < n_sweeps && e == cudaSuccess; ++sw) {
        a.sweep = (uint64_t)(ctx->sweeps + sw);
        if (col) {
            a.sg_feat = col->feat + (size_t)sw * ctx->N * ptca::SG_IN;
            a.sg_center = col->center + (size_t)sw * ctx->N;
            a.sg_dF = col->dF + (size_t)sw * ctx->N;
        }
        for (int s = 0; s < ctx->nstages && e == cudaSuccess; ++s, ++g) {
            a.S_in = ctx->d_S[g & 1];
            a.S_out = ctx->d_S[(g + 1) & 1];
            a.sites = ctx->d_sites + ctx->h_start[s];
            a.count = ctx->h_start[s + 1] - ctx->h_start[s];
            a.rec_base = ctx->h_start[s];
            a.prev_sites = prev_s >= 0 ? ctx->d_sites + ctx->h_start[prev_s] : nullptr;
            a.prev_count = prev_s >= 0 ? ctx->h_start[prev_s + 1] - ctx->h_start[prev_s] : 0;
            a.perm = nullptr;
            a.count_dev = nullptr;
            a.sg_dFt = nullptr;
            if (ctx->checker) e = check_stage(ctx, a, s, st);
            if (e == cudaSuccess && ctx->sg.enabled && !col) e = ptca_screen_stage(ctx, a, st);
            if (e == cudaSuccess)
                e = timed_launch(ctx, 0, 2 * (int64_t)a.count, st,
                                 [&] { return launch_stage_ctx(ctx, a, st); });
            if (e == cudaSuccess && a.margin > 0.0) {
                e = timed_launch(ctx, 1, 0, st, [&] { return launch_resolve_ctx(ctx, a, st); });
                if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flag_count, 0, sizeof(unsigned int), st);
            }
            prev_s = s;
        }
    }
    if (e == cudaSuccess && g > 0)
        e = ptca::launch_copy_sites(ctx->d_S[g & 1], ctx->d_S[(g + 1) & 1], ctx->d_sites + ctx->h_start[prev_s],
                                    ctx->h_start[prev_s + 1] - ctx->h_start[prev_s], st);
    if (e == cudaSuccess) e = ptca::launch_set_u64(ctx->d_sweep_ctr, (unsigned long long)(ctx->sweeps + n_sweeps), st);
    return e;
}

// Point the per-visit scratch of `a` at half h (stage parity).
static void use_half(const ptca_ctx* ctx, StageArgs& a, int h) {
    const size_t ms = (size_t)ctx->max_stage;
    a.Fbuf = ctx->d_F + h * 2 * ms;
    a.fillbuf = ctx->d_fill + h * 2 * ms;
    a.ticket = ctx->d_ticket + h * ms;
    a.flag_list = ctx->d_flag_list + h * ms;
    a.flag_count = ctx->d_flag_count + h;
}

// Resources of the overlapped pipeline, made on first use.
static cudaError_t ensure_overlap(ptca_ctx* ctx) {
    if (ctx->side) return cudaSuccess;
    std::vector<int32_t> order;
    stage_split(ctx->p, ctx->h_start, ctx->h_sites, order, ctx->h_indep);
    cudaError_t e = cudaSuccess;
    for (int b = 2; b < 4 && e == cudaSuccess; ++b)
        if (!ctx->d_S[b]) e = dalloc(&ctx->d_S[b], 3 * (size_t)ctx->N);
    if (e == cudaSuccess && !ctx->d_split) e = dalloc(&ctx->d_split, (size_t)ctx->N);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->d_split, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    for (cudaEvent_t* ev : {&ctx->ev_fork, &ctx->ev_join, &ctx->ev_ind[0], &ctx->ev_ind[1], &ctx->ev_res[0],
                            &ctx->ev_res[1]})
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->side2) e = cudaStreamCreateWithFlags(&ctx->side2, cudaStreamNonBlocking);
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    cudaStream_t side = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) ctx->side = side;
    return e;
}

// Large clusters: the global matrix slots of set k (0, 1: independent
// visits by stage parity; 2: dependent visits).
static void *large_slots(const ptca_ctx* ctx, int k) {
    const size_t es = ctx->prec == 1 ? sizeof(float2) : sizeof(double2);
    return static_cast<char*>(ctx->d_gL) + (size_t)k * (size_t)ctx->large_grid * (size_t)ctx->gL_stride * es;
}

// StageArgs of stage gg of the overlapped pipeline's rotation (counted from
// the last time the configuration was in buffers 0 and 1): buffer gg mod 4
// in, gg+1 mod 4 out, the per-visit scratch half gg mod 2, the random stream
// of sweep `sweep`.
static StageArgs overlap_args(ptca_ctx* ctx, int64_t gg, uint64_t sweep) {
    const int s = (int)(gg % ctx->nstages);
    StageArgs a = base_args(ctx);
    use_half(ctx, a, (int)(gg & 1));
    a.sweep = sweep;
    a.S_in = ctx->d_S[gg % 4];
    a.S_out = ctx->d_S[(gg + 1) % 4];
    a.sites = ctx->d_sites + ctx->h_start[s];
    a.rec_base = ctx->h_start[s];
    if (ctx->sg.enabled) a.sg_dFt = ctx->sg.dFt + (size_t)(gg & 1) * ctx->max_stage;
    return a;
}

// Sites the dependent-visit launch of stage gg copies forward from buffer gg
// into buffer gg+1 (mod 4), which last held the configuration after stage
// gg-4: those of the min(3, ns-1) stages before stage gg, as at most two
// ranges of the flattened schedule.  (Early in a rotation some of these
// stages have not run; their sites agree in every buffer, and the copy
// changes nothing.)
static void copy_ranges(const ptca_ctx* ctx, int64_t gg, StageArgs& ad) {
    const int ns = ctx->nstages, s = (int)(gg % ns), k = std::min(3, ns - 1);
    ad.prev_sites = ad.prev2_sites = nullptr;
    ad.prev_count = ad.prev2_count = 0;
    if (k <= 0) return;
    const int q0 = ((s - k) % ns + ns) % ns, q1 = q0 + k;
    ad.prev_sites = ctx->d_sites + ctx->h_start[q0];
    ad.prev_count = ctx->h_start[std::min(q1, ns)] - ctx->h_start[q0];
    if (q1 > ns) {
        ad.prev2_sites = ctx->d_sites;
        ad.prev2_count = ctx->h_start[q1 - ns];
    }
}

// Overlapped per-stage pipeline.  Stage g (counted over the rotation) reads
// buffer g mod 4 and writes buffer g+1 mod 4, so the re-solve of stage g-1
// keeps reading its own start configuration while stage g writes.  Each
// stage is cut into the visits whose windows hold no site of stage g-1
// (I_g) and the rest (D_g).
//  - I_g reads buffer g-1 mod 4 (the configuration after stage g-2, equal
//    to that after stage g-1 on its windows) once the re-solve of stage g-2
//    (R_{g-2}) is done, alternating between the caller's stream and a
//    second stream: it runs beside the tail of I_{g-1}.  Surrogate screening
//    keeps a set of network buffers per stage parity, large clusters a set
//    of matrix slots per stage parity, so two such launches never share one.
//  - On the context's high-priority stream: R_{g-1} (once I_{g-1} is done),
//    then D_g, which also copies the sites of the three stages before g
//    forward into buffer g+1 mod 4.
// The per-visit scratch alternates halves with g, so R_{g-1} and stage g
// never share a slot (I_{g+1} shares R_{g-1}'s half and starts after it).
// Every visit reads the spins it reads in the one-stream pipeline and decides
// with the same arithmetic: the chain is the same, bit for bit.
//
// With `defer`, the call ends without the last stage's re-solve: the next
// call continues the rotation and runs it beside its own first stage's
// independent visits, as a multi-sweep call does between its sweeps.  Until
// then the configuration is in buffer (rotation) mod 4, not in buffers 0 and
// 1; every other entry point settles it first.
static cudaError_t sweep_overlap(ptca_ctx* ctx, int32_t n_sweeps, cudaStream_t st, bool defer) {
    cudaError_t e = ensure_overlap(ctx);
    if (e != cudaSuccess) return e;
    const bool screen = ctx->sg.enabled;
    cudaStream_t hs = ctx->side, s2 = ctx->side2;
    const size_t bytes = 3 * (size_t)ctx->N * sizeof(double);
    const int ns = ctx->nstages;
    const int64_t G = (int64_t)n_sweeps * ns;
    const bool cont = ctx->ov_pending;
    const int64_t g0 = cont ? ctx->ov_g : 0;
    ctx->ov_pending = false;
    StageArgs prev = base_args(ctx);  // the stage whose re-solve is pending
    int64_t gprev = -1;
    if (cont) {
        // after the previous call's work on its stream (which may differ)
        e = cudaStreamWaitEvent(st, ctx->ev_fork, 0);
        prev = overlap_args(ctx, g0 - 1, (uint64_t)(ctx->sweeps - 1));
        gprev = g0 - 1;
    } else {
        // buffers 0 and 1 agree between calls; 2 and 3 start from them too
        e = cudaMemcpyAsync(ctx->d_S[2], ctx->d_S[0], bytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_S[3], ctx->d_S[0], bytes, cudaMemcpyDeviceToDevice, st);
    }
    // the library's streams start after the caller's earlier work
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, ctx->ev_fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ctx->ev_fork, 0);
    auto resolve_prev = [&]() {
        cudaError_t r = cudaStreamWaitEvent(hs, ctx->ev_ind[gprev & 1], 0);
        if (r == cudaSuccess)
            r = timed_launch(ctx, 1, 0, hs, [&] { return launch_resolve_ctx(ctx, prev, hs); });
        if (r == cudaSuccess) r = cudaMemsetAsync(prev.flag_count, 0, sizeof(unsigned int), hs);
        if (r == cudaSuccess) r = cudaEventRecord(ctx->ev_res[gprev & 1], hs);
        return r;
    };
    for (int64_t g = 0; g < G && e == cudaSuccess; ++g) {
        const int64_t gg = g0 + g;
        const int s = (int)(gg % ns);
        StageArgs a = overlap_args(ctx, gg, (uint64_t)(ctx->sweeps + g / ns));
        const int cnt = ctx->h_start[s + 1] - ctx->h_start[s], ni = ctx->h_indep[s];
        if (gprev >= 0) e = resolve_prev();
        // I_gg: after R_{gg-2}, on the stream of this stage's parity
        cudaStream_t is = (gg & 1) ? s2 : st;
        if (e == cudaSuccess && gg >= 2) e = cudaStreamWaitEvent(is, ctx->ev_res[gg & 1], 0);
        StageArgs ai = a;
        ai.S_in = ctx->d_S[(gg + 3) % 4];
        ai.perm = ctx->d_split + ctx->h_start[s];
        ai.count = ni;
        if (ctx->large) ai.gL = large_slots(ctx, (int)(gg & 1));
        // Delayed acceptance: each part of the stage is screened on its own
        // stream just before its exact solves (network rows of the
        // independent part first, the dependent part's after them; dF~ in
        // the half of this stage's parity, which its re-solve reads later).
        if (screen && e == cudaSuccess && ni > 0) e = ptca_screen_part(ctx, ai, 0, 0, (int)(gg & 1), is);
        if (e == cudaSuccess && ni > 0)
            e = timed_launch(ctx, 0, 2 * (int64_t)ni, is, [&] { return launch_stage_ctx(ctx, ai, is); });
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_ind[gg & 1], is);
        StageArgs ad = a;
        ad.perm = ctx->d_split + ctx->h_start[s] + ni;
        ad.count = cnt - ni;
        if (ctx->large) ad.gL = large_slots(ctx, 2);  // concurrent with the independent-visit launches
        copy_ranges(ctx, gg, ad);
        if (screen && e == cudaSuccess && ad.count > 0) e = ptca_screen_part(ctx, ad, 1, 2 * ni, (int)(gg & 1), hs);
        if (e == cudaSuccess) {
            if (ad.count > 0) {
                e = timed_launch(ctx, 2, 2 * (int64_t)ad.count, hs,
                                 [&] { return launch_stage_ctx(ctx, ad, hs); });
            } else {
                e = ptca::launch_copy_sites(ad.S_in, ad.S_out, ad.prev_sites, ad.prev_count, hs);
                if (e == cudaSuccess) e = ptca::launch_copy_sites(ad.S_in, ad.S_out, ad.prev2_sites, ad.prev2_count, hs);
            }
        }
        prev = a;
        gprev = gg;
    }
    if (e == cudaSuccess && defer && G > 0) {
        ctx->ov_pending = true;
        ctx->ov_g = g0 + G;
        e = cudaEventRecord(ctx->ev_fork, st);  // the next call's stream starts after this one's
        if (e == cudaSuccess)
            e = ptca::launch_set_u64(ctx->d_sweep_ctr, (unsigned long long)(ctx->sweeps + n_sweeps), st);
        return e;
    }
    if (e == cudaSuccess && gprev >= 0) e = resolve_prev();
    // join the side stream back into the caller's stream, also after a
    // failure (every independent-visit launch precedes a re-solve there)
    cudaError_t ej = cudaEventRecord(ctx->ev_join, hs);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, ctx->ev_join, 0);
    if (ej == cudaSuccess) ej = cudaEventRecord(ctx->ev_join, s2);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, ctx->ev_join, 0);
    if (e == cudaSuccess) e = ej;
    // the configuration after the call is in buffer (g0 + G) mod 4; buffers 0 and 1 take it
    const int f = (int)((g0 + G) % 4);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        if (b != f) e = cudaMemcpyAsync(ctx->d_S[b], ctx->d_S[f], bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = ptca::launch_set_u64(ctx->d_sweep_ctr, (unsigned long long)(ctx->sweeps + n_sweeps), st);
    return e;
}

cudaError_t ptca_internal_settle(ptca_ctx* ctx, cudaStream_t st, bool have_stream) {
    if (!ctx->ov_pending) return cudaSuccess;
    ctx->ov_pending = false;
    cudaStream_t hs = ctx->side;
    const int64_t g = ctx->ov_g;
    StageArgs prev = overlap_args(ctx, g - 1, (uint64_t)(ctx->sweeps - 1));
    cudaError_t e = cudaStreamWaitEvent(hs, ctx->ev_ind[(g - 1) & 1], 0);
    if (e == cudaSuccess) e = timed_launch(ctx, 1, 0, hs, [&] { return launch_resolve_ctx(ctx, prev, hs); });
    if (e == cudaSuccess) e = cudaMemsetAsync(prev.flag_count, 0, sizeof(unsigned int), hs);
    const int f = (int)(g % 4);
    const size_t bytes = 3 * (size_t)ctx->N * sizeof(double);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        if (b != f) e = cudaMemcpyAsync(ctx->d_S[b], ctx->d_S[f], bytes, cudaMemcpyDeviceToDevice, hs);
    cudaError_t ej = cudaEventRecord(ctx->ev_join, hs);
    if (ej == cudaSuccess) ej = have_stream ? cudaStreamWaitEvent(st, ctx->ev_join, 0) : cudaStreamSynchronize(hs);
    return e == cudaSuccess ? ej : e;
}

// Everything one persistent sweep launch needs, as stream work (capturable).
static cudaError_t enqueue_persistent(ptca_ctx* ctx, int32_t n_sweeps, cudaStream_t st) {
    ptca::PersistArgs p;
    std::memset(&p, 0, sizeof p);
    p.st = base_args(ctx);
    p.st.perm = ctx->d_perm;
    p.S0 = ctx->d_S[0];
    p.S1 = ctx->d_S[1];
    p.sites = ctx->d_sites;
    p.stage_start = ctx->d_stage_start;
    p.nstages = ctx->nstages;
    p.n_sweeps = n_sweeps;
    p.sweep_ctr = ctx->d_sweep_ctr;
    p.queue = ctx->d_queue;
    p.bar = ctx->d_bar;
    p.timeout_ns = ctx->timeout_ns;
    cudaError_t e = cudaMemsetAsync(ctx->d_queue, 0, 3 * sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flag_count, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_bar, 0, 2 * sizeof(unsigned int), st);
    if (e == cudaSuccess)
        e = ctx->large ? ptca::launch_persistent_large(ctx->prec, p, ctx->grid, st)
                       : ptca::launch_persistent(ctx->prec, ctx->nw, p, ctx->grid, st);
    return e;
}

static cudaError_t sweep_graph(ptca_ctx* ctx, int32_t n_sweeps, cudaStream_t st) {
    if (ctx->graph && ctx->graph_sweeps == n_sweeps) return cudaGraphLaunch(ctx->graph, st);
    drop_graph(ctx);
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = enqueue_persistent(ctx, n_sweeps, cap);
        e = cudaStreamEndCapture(cap, &g);
        if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->graph = nullptr;
        ctx->graph_failed = true;  // fall back to direct persistent launches
        return enqueue_persistent(ctx, n_sweeps, st);
    }
    ctx->graph_sweeps = n_sweeps;
    return cudaGraphLaunch(ctx->graph, st);
}

// Stream work of n_sweeps sweeps in the context's launch configuration
// (screening and the checker need the per-stage pipeline).
static bool overlapped(const ptca_ctx* ctx) {
    return ctx->pipeline == PTCA_PIPELINE_OVERLAP && ctx->prec == 1 && ctx->margin > 0.0 && !ctx->checker;
}

static cudaError_t run_sweeps(ptca_ctx* ctx, int32_t n_sweeps, cudaStream_t st, bool defer = false) {
    const bool per_stage = ctx->pipeline == PTCA_PIPELINE_STAGES || ctx->pipeline == PTCA_PIPELINE_OVERLAP;
    if (overlapped(ctx)) return sweep_overlap(ctx, n_sweeps, st, defer);
    if (per_stage || ctx->sg.enabled || ctx->checker) return sweep_stages(ctx, n_sweeps, st);
    if (ctx->pipeline == PTCA_PIPELINE_PERSISTENT || ctx->graph_failed) return enqueue_persistent(ctx, n_sweeps, st);
    return sweep_graph(ctx, n_sweeps, st);
}

ptca_status ptca_set_pipeline(ptca_ctx* ctx, int32_t mode, double barrier_timeout_s) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (mode < PTCA_PIPELINE_STAGES || mode > PTCA_PIPELINE_OVERLAP) return fail(PTCA_ERR_INVALID, "unknown pipeline");
    const bool persistent = mode == PTCA_PIPELINE_PERSISTENT || mode == PTCA_PIPELINE_GRAPH;
    if (persistent && ctx->grid <= 0)
        return fail(PTCA_ERR_UNSUPPORTED, "persistent kernel does not fit on this device");
    if (!(barrier_timeout_s > 0) || barrier_timeout_s > 3600) return fail(PTCA_ERR_INVALID, "timeout out of range");
    PTCA_SETTLE_SYNC(ctx);
    if (mode == PTCA_PIPELINE_OVERLAP) {
        cudaError_t e = ensure_overlap(ctx);
        if (e != cudaSuccess) return cuda_fail(e, "ptca_set_pipeline (overlapped pipeline)");
    }
    ctx->pipeline = mode;
    ctx->timeout_ns = (unsigned long long)(barrier_timeout_s * 1e9);
    if (persistent) {
        // the persistent kernels run the row-chunked reduction, one per
        // matrix; the margin must then be that reduction's
        ctx->reduction = 0;
        ctx->panel = 0;
        default_margin(ctx);
    }
    drop_graph(ctx);
    return PTCA_OK;
}

ptca_status ptca_set_kernel_timing(ptca_ctx* ctx, int32_t on) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    ctx->timing = on != 0;
    if (!ctx->timing) drop_timing_events(ctx);
    return PTCA_OK;
}

ptca_status ptca_kernel_times(ptca_ctx* ctx, double* out, void* stream) {
    if (!ctx || !out) return fail(PTCA_ERR_INVALID, "null argument");
    PTCA_SETTLE(ctx, static_cast<cudaStream_t>(stream));
    PTCA_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    for (int q = 0; q < 9; ++q) out[q] = 0.0;
    std::vector<std::pair<double, double>> span;  // stage launches (kind 0), relative to the first one's start
    cudaEvent_t ref = nullptr;
    for (size_t i = 0; i < ctx->tkind.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->tev[2 * i], ctx->tev[2 * i + 1]) != cudaSuccess) {
            drop_timing_events(ctx);
            return fail(PTCA_ERR_CUDA, "kernel timing events were not recorded on this stream");
        }
        const int k = ctx->tkind[i];
        out[2 * k] += ms;
        out[2 * k + 1] += 1.0;
        if (k == 0) out[6] += (double)ctx->titems[i];
        if (k == 2) out[7] += (double)ctx->titems[i];
        if (k == 0) {
            float t0 = 0.f;
            if (!ref) ref = ctx->tev[2 * i];
            else if (cudaEventElapsedTime(&t0, ref, ctx->tev[2 * i]) != cudaSuccess) t0 = 0.f;
            span.emplace_back((double)t0, (double)t0 + ms);
        }
    }
    // union of the stage launches' intervals (look-ahead launches overlap)
    std::sort(span.begin(), span.end());
    double lo = 0.0, hi = -1.0;
    for (const auto& iv : span) {
        if (iv.first > hi) {
            if (hi > lo) out[8] += hi - lo;
            lo = iv.first;
            hi = iv.second;
        } else if (iv.second > hi) {
            hi = iv.second;
        }
    }
    if (hi > lo) out[8] += hi - lo;
    drop_timing_events(ctx);
    return PTCA_OK;
}

ptca_status ptca_get_launch_config(const ptca_ctx* ctx, ptca_launch_config* out) {
    if (!ctx || !out) return fail(PTCA_ERR_INVALID, "null argument");
    out->pipeline = ctx->pipeline;
    out->warps_per_cta = ctx->nw;
    out->ctas_per_sm = ctx->ctas_per_sm;
    out->reduction = ctx->reduction;
    out->panel_width = ctx->panel;
    return PTCA_OK;
}

ptca_status ptca_set_launch_config(ptca_ctx* ctx, const ptca_launch_config* cfg) {
    if (!ctx || !cfg) return fail(PTCA_ERR_INVALID, "null argument");
    if (cfg->pipeline < PTCA_PIPELINE_STAGES || cfg->pipeline > PTCA_PIPELINE_OVERLAP)
        return fail(PTCA_ERR_INVALID, "unknown pipeline");
    PTCA_SETTLE_SYNC(ctx);
    if (cfg->warps_per_cta != 8 && cfg->warps_per_cta != 4 && cfg->warps_per_cta != 1 && cfg->warps_per_cta != 16)
        return fail(PTCA_ERR_INVALID, "warps_per_cta must be 1, 4, 8 or 16");
    if (ctx->large && cfg->warps_per_cta != 8 && cfg->warps_per_cta != 16)
        return fail(PTCA_ERR_UNSUPPORTED,
                    "large clusters run 8-warp CTAs in thread-block clusters (PTCA_MIXED) or 16-warp CTAs with the "
                    "matrix in global memory: pass warps_per_cta = 8 or 16");
    if (!ctx->large && cfg->warps_per_cta == 16)
        return fail(PTCA_ERR_UNSUPPORTED, "16-warp CTAs serve the large-cluster orders only");
    if (!ctx->large && !ptca::sweep_width_supported(ctx->prec, cfg->warps_per_cta, ctx->nA))
        return fail(PTCA_ERR_UNSUPPORTED,
                    "narrow sweep kernels need PTCA_MIXED and matrix orders up to 128 (4 warps) or 32 (1 warp)");
    const int maxb = ctx->large ? (cfg->warps_per_cta == 16 ? ptca::persistent_blocks_per_sm_large(ctx->prec) : 0)
                                : ptca::persistent_blocks_per_sm(ctx->prec, cfg->warps_per_cta, ctx->nA);
    if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > maxb)
        return fail(PTCA_ERR_INVALID, "ctas_per_sm must be in [0, the CTAs that fit on an SM]");
    const bool persistent = cfg->pipeline == PTCA_PIPELINE_PERSISTENT || cfg->pipeline == PTCA_PIPELINE_GRAPH;
    if (persistent && maxb <= 0) return fail(PTCA_ERR_UNSUPPORTED, "persistent kernel does not fit on this device");
    if (cfg->reduction < 0 || cfg->reduction > 2) return fail(PTCA_ERR_INVALID, "reduction must be 0, 1 or 2");
    if (cfg->reduction == 2) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
        const bool ok = ctx->large ? cfg->warps_per_cta == 16 && ptca::large_shared_supported(ctx->prec, ctx->nA,
                                                                                             (size_t)optin)
                                   : cfg->warps_per_cta == 4 && ptca::shared_supported(ctx->prec, ctx->nA);
        if (!ok || persistent || cfg->panel_width > 1)
            return fail(PTCA_ERR_UNSUPPORTED,
                        "the shared reduction runs PTCA_MIXED stage kernels of 4-warp CTAs (orders up to 128) or, "
                        "for large clusters, 16-warp CTAs, in the per-stage or overlapped pipeline");
    }
    if (cfg->reduction == 1 &&
        (ctx->large || cfg->warps_per_cta != 4 || persistent || !ptca::tiled_supported(ctx->prec, ctx->nA)))
        return fail(PTCA_ERR_UNSUPPORTED,
                    "the register-tiled reduction runs PTCA_MIXED stage kernels of 4-warp CTAs, orders up to 128, "
                    "in the per-stage or overlapped pipeline");
    if (cfg->panel_width < 0 || cfg->panel_width > 8 || (cfg->panel_width > 1 && (cfg->panel_width & (cfg->panel_width - 1))))
        return fail(PTCA_ERR_INVALID, "panel_width must be 0, 1, 2, 4 or 8");
    if (cfg->panel_width > 1 &&
        (ctx->large || cfg->warps_per_cta != 8 || persistent || cfg->reduction != 0 ||
         !ptca::panel_supported(ctx->prec, ctx->nA, cfg->panel_width)))
        return fail(PTCA_ERR_UNSUPPORTED,
                    "the panel reduction runs PTCA_MIXED stage kernels of 8-warp CTAs, orders up to 128, in the "
                    "per-stage or overlapped pipeline");
    if (cfg->pipeline == PTCA_PIPELINE_OVERLAP) {
        cudaError_t e = ensure_overlap(ctx);
        if (e != cudaSuccess) return cuda_fail(e, "ptca_set_launch_config (overlapped pipeline)");
    }
    ctx->pipeline = cfg->pipeline;
    ctx->nw = cfg->warps_per_cta;
    ctx->ctas_per_sm = cfg->ctas_per_sm;
    ctx->reduction = cfg->reduction;
    ctx->panel = cfg->panel_width > 1 ? cfg->panel_width : 0;
    default_margin(ctx);
    ctx->grid = maxb > 0 ? ctx->sms * (cfg->ctas_per_sm > 0 ? cfg->ctas_per_sm : maxb) : 0;
    ctx->graph_failed = false;
    drop_graph(ctx);
    return PTCA_OK;
}

static const char* pipeline_name(int p) {
    switch (p) {
        case PTCA_PIPELINE_STAGES: return "stages";
        case PTCA_PIPELINE_PERSISTENT: return "persistent";
        case PTCA_PIPELINE_GRAPH: return "graph";
        default: return "overlap";
    }
}

ptca_status ptca_autotune(ptca_ctx* ctx, int32_t trial_sweeps, ptca_launch_config* best, char* json, int32_t json_cap,
                          void* stream) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (trial_sweeps < 1 || trial_sweeps > 100) return fail(PTCA_ERR_INVALID, "trial_sweeps in [1, 100]");
    if (ctx->checker) return fail(PTCA_ERR_INVALID, "turn the precision checker off before autotuning");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    // Candidates: CTA width x pipeline x persistent CTAs per SM.
    std::vector<ptca_launch_config> cand;
    if (ctx->large) {
        for (int nw : {16, 8}) {
            if (nw == 8 && ctx->cl_size == 0) continue;  // 8 would mean the global-slot kernel again
            cand.push_back({PTCA_PIPELINE_STAGES, nw, 0, 0});
            if (ctx->prec == 1 && ctx->margin > 0.0) cand.push_back({PTCA_PIPELINE_OVERLAP, nw, 0, 0});
        }
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
        if (ptca::large_shared_supported(ctx->prec, ctx->nA, (size_t)optin)) {
            cand.push_back({PTCA_PIPELINE_STAGES, 16, 0, 2, 0});
            if (ctx->margin > 0.0) cand.push_back({PTCA_PIPELINE_OVERLAP, 16, 0, 2, 0});
        }
        const int maxb = ptca::persistent_blocks_per_sm_large(ctx->prec);
        if (maxb > 0 && !ctx->sg.enabled)
            for (int pl : {PTCA_PIPELINE_PERSISTENT, PTCA_PIPELINE_GRAPH}) cand.push_back({pl, 16, maxb, 0});
    }
    for (int nw : {8, 4, 1}) {
        if (ctx->large || !ptca::sweep_width_supported(ctx->prec, nw, ctx->nA)) continue;
        cand.push_back({PTCA_PIPELINE_STAGES, nw, 0, 0});
        if (ctx->prec == 1 && ctx->margin > 0.0) cand.push_back({PTCA_PIPELINE_OVERLAP, nw, 0, 0});
        if (nw == 4 && ptca::tiled_supported(ctx->prec, ctx->nA)) {
            cand.push_back({PTCA_PIPELINE_STAGES, nw, 0, 1, 0});
            if (ctx->margin > 0.0) cand.push_back({PTCA_PIPELINE_OVERLAP, nw, 0, 1, 0});
        }
        // (The shared reduction, PTCA_REDUCTION_SHARED, is not a candidate:
        // its FP32 dF error is about twice the row-chunked pass's, and
        // the re-solve margin is sized for the latter.)
        if (nw == 8)
            for (int b : {2, 4, 8}) {
                if (!ptca::panel_supported(ctx->prec, ctx->nA, b)) continue;
                cand.push_back({PTCA_PIPELINE_STAGES, nw, 0, 0, b});
                if (ctx->margin > 0.0) cand.push_back({PTCA_PIPELINE_OVERLAP, nw, 0, 0, b});
            }
        const int maxb = ptca::persistent_blocks_per_sm(ctx->prec, nw, ctx->nA);
        if (maxb <= 0 || ctx->sg.enabled) continue;
        for (int pl : {PTCA_PIPELINE_PERSISTENT, PTCA_PIPELINE_GRAPH}) {
            cand.push_back({pl, nw, maxb, 0});
            if (maxb > 1) cand.push_back({pl, nw, 1, 0});
        }
    }
    // The chain state every trial starts from (both spin buffers agree
    // between sweeps) and is restored to afterwards.
    const size_t nS = 3 * (size_t)ctx->N;
    double* saved = nullptr;
    PTCA_CUDA(cudaMalloc(&saved, nS * sizeof(double)));
    PTCA_CUDA(cudaMemcpyAsync(saved, ctx->d_S[0], nS * sizeof(double), cudaMemcpyDeviceToDevice, st));
    const int64_t sweeps0 = ctx->sweeps;
    ptca_launch_config prev;
    ptca_get_launch_config(ctx, &prev);
    auto restore = [&]() {
        cudaError_t e = cudaMemcpyAsync(ctx->d_S[0], saved, nS * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_S[1], saved, nS * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = ptca::launch_set_u64(ctx->d_sweep_ctr, (unsigned long long)sweeps0, st);
        ctx->sweeps = sweeps0;
        return e;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<double> ms(cand.size(), -1.0);
    int ibest = -1;
    for (size_t i = 0; i < cand.size(); ++i) {
        if (ptca_set_launch_config(ctx, &cand[i]) != PTCA_OK) continue;
        cudaError_t e = restore();
        if (e == cudaSuccess) e = run_sweeps(ctx, 1, st);  // warm-up (and graph capture)
        if (e == cudaSuccess) e = restore();
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = run_sweeps(ctx, trial_sweeps, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        int32_t err[2] = {0, 0};
        if (e == cudaSuccess) e = cudaMemcpy(err, ctx->d_err, sizeof err, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess || err[1] != 0) {
            cudaGetLastError();
            cudaMemsetAsync(ctx->d_err, 0, 2 * sizeof(int32_t), st);
            continue;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[i] = t / trial_sweeps;
        if (ibest < 0 || ms[i] < ms[ibest]) ibest = (int)i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const ptca_launch_config chosen = ibest >= 0 ? cand[ibest] : prev;
    ptca_set_launch_config(ctx, &chosen);
    cudaError_t e = restore();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(saved);
    if (e != cudaSuccess) return cuda_fail(e, "ptca_autotune");
    if (ibest < 0) return fail(PTCA_ERR_CUDA, "no launch configuration completed a trial sweep");
    if (best) *best = chosen;
    if (json && json_cap > 0) {
        std::string js = "{\"n_max\": " + std::to_string(ctx->nA) + ", \"precision\": \"" +
                         (ctx->prec ? "mixed" : "fp64") + "\", \"sites\": " + std::to_string(ctx->N) +
                         ", \"stages\": " + std::to_string(ctx->nstages) + ", \"trial_sweeps\": " +
                         std::to_string(trial_sweeps) + ", \"candidates\": [";
        char buf[256];
        for (size_t i = 0; i < cand.size(); ++i) {
            std::snprintf(buf, sizeof buf,
                          "%s{\"pipeline\": \"%s\", \"warps_per_cta\": %d, \"ctas_per_sm\": %d, \"reduction\": %d, "
                          "\"panel_width\": %d, \"ms_per_sweep\": %s}",
                          i ? ", " : "", pipeline_name(cand[i].pipeline), cand[i].warps_per_cta, cand[i].ctas_per_sm,
                          cand[i].reduction, cand[i].panel_width, ms[i] >= 0 ? std::to_string(ms[i]).c_str() : "null");
            js += buf;
        }
        std::snprintf(buf, sizeof buf,
                      "], \"best\": {\"pipeline\": \"%s\", \"warps_per_cta\": %d, \"ctas_per_sm\": %d, "
                      "\"reduction\": %d, \"panel_width\": %d}}",
                      pipeline_name(chosen.pipeline), chosen.warps_per_cta, chosen.ctas_per_sm, chosen.reduction,
                      chosen.panel_width);
        js += buf;
        if ((int)js.size() >= json_cap) return fail(PTCA_ERR_INVALID, "json buffer too small");
        std::memcpy(json, js.c_str(), js.size() + 1);
    }
    return PTCA_OK;
}

ptca_status ptca_set_resolve_margin(ptca_ctx* ctx, double margin) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (!(margin >= 0.0) || !std::isfinite(margin)) return fail(PTCA_ERR_INVALID, "margin must be finite and >= 0");
    if (ctx->prec != 1 && margin > 0.0) return fail(PTCA_ERR_INVALID, "the re-solve margin applies to PTCA_MIXED only");
    PTCA_SETTLE_SYNC(ctx);
    ctx->margin = margin;
    ctx->margin_set = true;
    drop_graph(ctx);
    return PTCA_OK;
}

ptca_status ptca_set_checker(ptca_ctx* ctx, int32_t on) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    PTCA_SETTLE_SYNC(ctx);
    if (!on) {
        ctx->checker = false;
        return PTCA_OK;
    }
    if (ctx->prec != 1) return fail(PTCA_ERR_UNSUPPORTED, "the precision checker compares PTCA_MIXED against FP64");
    if (!ctx->d_chk_out) {
        ctx->check_chunk = std::min(ctx->max_stage, 2048);
        cudaError_t e = dalloc(&ctx->d_chk_eig, (size_t)2 * ctx->check_chunk * 2 * ctx->nA);
        if (e == cudaSuccess) e = dalloc(&ctx->d_chk_F, (size_t)2 * ctx->check_chunk * 2);
        if (e == cudaSuccess) e = dalloc(&ctx->d_chk_out, (size_t)ptca::kCheckCols * ctx->nstages);
        if (e == cudaSuccess) e = cudaMemset(ctx->d_chk_out, 0, (size_t)ptca::kCheckCols * ctx->nstages * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            cudaFree(ctx->d_chk_eig);
            cudaFree(ctx->d_chk_F);
            cudaFree(ctx->d_chk_out);
            ctx->d_chk_eig = nullptr;
            ctx->d_chk_F = nullptr;
            ctx->d_chk_out = nullptr;
            return cuda_fail(e, "ptca_set_checker");
        }
    }
    ctx->checker = true;
    return PTCA_OK;
}

ptca_status ptca_checker_read(ptca_ctx* ctx, double* out, int32_t n_rows, void* stream) {
    if (!ctx || !out) return fail(PTCA_ERR_INVALID, "null argument");
    if (n_rows < ctx->nstages) return fail(PTCA_ERR_INVALID, "out needs one row per stage");
    if (!ctx->d_chk_out) {
        for (int i = 0; i < ptca::kCheckCols * ctx->nstages; ++i) out[i] = 0.0;
        return PTCA_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<unsigned long long> bits((size_t)ptca::kCheckCols * ctx->nstages);
    PTCA_CUDA(cudaMemcpyAsync(bits.data(), ctx->d_chk_out, bits.size() * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, st));
    PTCA_CUDA(cudaMemsetAsync(ctx->d_chk_out, 0, bits.size() * sizeof(unsigned long long), st));
    PTCA_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < bits.size(); ++i) std::memcpy(&out[i], &bits[i], sizeof(double));
    return PTCA_OK;
}

ptca_status ptca_sweep(ptca_ctx* ctx, int32_t n_sweeps, ptca_sweep_stats* stats_out, void* stream) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (n_sweeps < 0) return fail(PTCA_ERR_INVALID, "n_sweeps < 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats_out) {
        PTCA_CUDA(cudaEventCreate(&ev0));
        PTCA_CUDA(cudaEventCreate(&ev1));
        PTCA_CUDA(cudaEventRecord(ev0, st));
    }
    // An overlapped sweep without statistics may continue a re-solve the
    // previous call left pending, and leave its own last one to the next
    // call; anything else settles first and completes its sweeps.
    const bool defer = overlapped(ctx) && !stats_out && n_sweeps > 0;
    if (!defer) PTCA_CUDA(ptca_internal_settle(ctx, st, true));
    PTCA_CUDA(cudaMemsetAsync(ctx->d_counters, 0, 4 * sizeof(unsigned long long), st));
    if (n_sweeps > 0) {
        cudaError_t e;
        e = run_sweeps(ctx, n_sweeps, st, defer);
        if (e != cudaSuccess) return cuda_fail(e, "ptca_sweep");
    }
    ctx->sweeps += n_sweeps;
    if (stats_out) {
        unsigned long long cnt[4];
        int32_t err[2] = {0, 0};
        PTCA_CUDA(cudaEventRecord(ev1, st));
        PTCA_CUDA(cudaMemcpyAsync(cnt, ctx->d_counters, sizeof cnt, cudaMemcpyDeviceToHost, st));
        PTCA_CUDA(cudaMemcpyAsync(err, ctx->d_err, sizeof err, cudaMemcpyDeviceToHost, st));
        PTCA_CUDA(cudaStreamSynchronize(st));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        stats_out->attempts = (int64_t)n_sweeps * ctx->N;
        stats_out->accepted = (int64_t)cnt[0];
        stats_out->eigensolves = (int64_t)cnt[1];
        stats_out->resolved = (int64_t)cnt[2];
        stats_out->screened = (int64_t)cnt[3];
        stats_out->sweeps = ctx->sweeps;
        stats_out->seconds = ms * 1e-3;
        if (err[1]) {
            cudaMemsetAsync(ctx->d_err, 0, 2 * sizeof(int32_t), st);
            return fail(PTCA_ERR_TIMEOUT, "a device-wide stage barrier timed out; the sweep is incomplete");
        }
        if (err[0]) return fail(PTCA_ERR_NUMERIC, "non-finite free-energy difference in a sweep");
    }
    return PTCA_OK;
}

// Host-side check of a caller's site list: count sites, each in [0, N), no
// repeats; with want_stage >= 0 all of stage want_stage (ctx->h_stage_of).
// Copies the list to ctx->d_sub on `st` (pageable source: staged before
// cudaMemcpyAsync returns).
static ptca_status upload_sites(ptca_ctx* ctx, const int32_t* sites, int32_t count, int* stage_out,
                                cudaStream_t st, const char* who) {
    if (count < 0 || count > ctx->N) return fail(PTCA_ERR_INVALID, std::string(who) + ": count out of range");
    if (count > 0 && !sites) return fail(PTCA_ERR_INVALID, std::string(who) + ": null site list");
    if (ctx->h_stage_of.empty()) {
        ctx->h_stage_of.assign(ctx->N, -1);
        for (int q = 0; q < ctx->nstages; ++q)
            for (int k = ctx->h_start[q]; k < ctx->h_start[q + 1]; ++k) ctx->h_stage_of[ctx->h_sites[k]] = q;
    }
    std::vector<char> seen(ctx->N, 0);
    int stage = -1;
    for (int k = 0; k < count; ++k) {
        const int32_t s = sites[k];
        if (s < 0 || s >= ctx->N) return fail(PTCA_ERR_INVALID, std::string(who) + ": site index out of range");
        if (seen[s]) return fail(PTCA_ERR_INVALID, std::string(who) + ": repeated site");
        seen[s] = 1;
        if (k == 0) stage = ctx->h_stage_of[s];
        else if (stage_out && ctx->h_stage_of[s] != stage)
            return fail(PTCA_ERR_INVALID, std::string(who) + ": the sites belong to different stages");
    }
    if (stage_out) *stage_out = stage;
    if (!ctx->d_sub) PTCA_CUDA(dalloc(&ctx->d_sub, (size_t)ctx->N));
    if (!ctx->d_sub_spins) PTCA_CUDA(dalloc(&ctx->d_sub_spins, 3 * (size_t)ctx->N));
    if (count > 0)
        PTCA_CUDA(cudaMemcpyAsync(ctx->d_sub, sites, sizeof(int32_t) * (size_t)count, cudaMemcpyHostToDevice, st));
    return PTCA_OK;
}

ptca_status ptca_stage_run(ptca_ctx* ctx, int64_t sweep_index, const int32_t* sites, int32_t count, void* stream) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    if (sweep_index < 0) return fail(PTCA_ERR_INVALID, "ptca_stage_run: sweep_index < 0");
    if (ctx->sg.enabled) return fail(PTCA_ERR_UNSUPPORTED, "ptca_stage_run: surrogate screening runs in ptca_sweep only");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    int stage = -1;
    ptca_status r = upload_sites(ctx, sites, count, &stage, st, "ptca_stage_run");
    if (r != PTCA_OK) return r;
    if (count == 0) return PTCA_OK;
    // Buffers 0 and 1 hold the same configuration between calls: the visits
    // read buffer 0 and write their decisions into buffer 1 (the stage-start
    // snapshot of Sec. III.a), then buffer 0 takes the visited sites back.
    StageArgs a = base_args(ctx);
    a.sweep = (uint64_t)sweep_index;
    a.S_in = ctx->d_S[0];
    a.S_out = ctx->d_S[1];
    a.sites = ctx->d_sub;
    a.count = count;
    a.rec_base = 0;
    PTCA_CUDA(cudaMemsetAsync(ctx->d_counters, 0, 4 * sizeof(unsigned long long), st));
    cudaError_t e = launch_stage_ctx(ctx, a, st);
    if (e == cudaSuccess && a.margin > 0.0) {
        e = launch_resolve_ctx(ctx, a, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.flag_count, 0, sizeof(unsigned int), st);
    }
    if (e == cudaSuccess) e = ptca::launch_copy_sites(ctx->d_S[1], ctx->d_S[0], ctx->d_sub, count, st);
    if (e != cudaSuccess) return cuda_fail(e, "ptca_stage_run");
    drop_graph(ctx);
    return PTCA_OK;
}

ptca_status ptca_get_sites(ptca_ctx* ctx, const int32_t* sites, int32_t count, double* out, int32_t on_device,
                           void* stream) {
    if (!ctx || (count > 0 && !out)) return fail(PTCA_ERR_INVALID, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    ptca_status r = upload_sites(ctx, sites, count, nullptr, st, "ptca_get_sites");
    if (r != PTCA_OK || count == 0) return r;
    double* dst = on_device ? out : ctx->d_sub_spins;
    PTCA_CUDA(ptca::launch_gather_sites(ctx->d_S[0], ctx->d_sub, count, dst, st));
    if (!on_device) {
        PTCA_CUDA(cudaMemcpyAsync(out, dst, 3 * sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, st));
        PTCA_CUDA(cudaStreamSynchronize(st));
    }
    return PTCA_OK;
}

ptca_status ptca_set_sites(ptca_ctx* ctx, const int32_t* sites, int32_t count, const double* spins, int32_t on_device,
                           void* stream) {
    if (!ctx || (count > 0 && !spins)) return fail(PTCA_ERR_INVALID, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    ptca_status r = upload_sites(ctx, sites, count, nullptr, st, "ptca_set_sites");
    if (r != PTCA_OK || count == 0) return r;
    const double* src = spins;
    if (!on_device) {
        PTCA_CUDA(cudaMemcpyAsync(ctx->d_sub_spins, spins, 3 * sizeof(double) * (size_t)count, cudaMemcpyHostToDevice,
                                  st));
        src = ctx->d_sub_spins;
    }
    PTCA_CUDA(ptca::launch_scatter_sites(ctx->d_sub, count, src, ctx->d_S[0], ctx->d_S[1], st));
    return PTCA_OK;
}

ptca_status ptca_surrogate_collect(ptca_ctx* ctx, int32_t n_sweeps, float* feat, int32_t* center, float* dF,
                                   void* stream) {
    if (ctx && (ctx->p.model != PTCA_MODEL_DOUBLE_EXCHANGE || ctx->p.Lz > 1 || ctx->large))
        return fail(PTCA_ERR_UNSUPPORTED, "the surrogate screen is built for the double-exchange model on square lattices");
    if (!ctx || n_sweeps < 0 || !feat || !center || !dF) return fail(PTCA_ERR_INVALID, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    PTCA_CUDA(cudaMemsetAsync(ctx->d_counters, 0, 4 * sizeof(unsigned long long), st));
    Collect col{feat, center, dF};
    cudaError_t e = sweep_stages(ctx, n_sweeps, st, &col);
    if (e != cudaSuccess) return cuda_fail(e, "ptca_surrogate_collect");
    ctx->sweeps += n_sweeps;
    return PTCA_OK;
}

ptca_status ptca_selftest_barrier_timeout(int32_t blocks, double timeout_s, void* stream) {
    if (blocks < 1 || blocks > 1024 || !(timeout_s > 0) || timeout_s > 10)
        return fail(PTCA_ERR_INVALID, "blocks in [1,1024], timeout in (0,10] s");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int* bar = nullptr;
    int32_t* err = nullptr;
    PTCA_CUDA(cudaMalloc(&bar, 2 * sizeof(unsigned int)));
    cudaError_t e = cudaMalloc(&err, 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), st);
    if (e == cudaSuccess) e = ptca::launch_barrier_selftest(blocks, bar, err, (unsigned long long)(timeout_s * 1e9), st);
    int32_t h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, err, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(bar);
    if (err) cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "ptca_selftest_barrier_timeout");
    if (h[1] == 4) return fail(PTCA_ERR_TIMEOUT, "barrier wait timed out as expected");
    return PTCA_OK;
}

ptca_status ptca_flush(ptca_ctx* ctx, void* stream) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    PTCA_SETTLE(ctx, static_cast<cudaStream_t>(stream));
    return PTCA_OK;
}

ptca_status ptca_sweep_record(ptca_ctx* ctx, int32_t* site, double* F_old, double* F_new, double* lnu,
                              uint8_t* accepted, void* stream) {
    if (!ctx) return fail(PTCA_ERR_INVALID, "null context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    const size_t N = ctx->N;
    if (site) PTCA_CUDA(cudaMemcpyAsync(site, ctx->d_rec_site, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    if (F_old) PTCA_CUDA(cudaMemcpyAsync(F_old, ctx->d_rec_Fold, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (F_new) PTCA_CUDA(cudaMemcpyAsync(F_new, ctx->d_rec_Fnew, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (lnu) PTCA_CUDA(cudaMemcpyAsync(lnu, ctx->d_rec_lnu, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (accepted) PTCA_CUDA(cudaMemcpyAsync(accepted, ctx->d_rec_acc, N, cudaMemcpyDeviceToDevice, st));
    return PTCA_OK;
}

ptca_status ptca_observables(ptca_ctx* ctx, ptca_obs* out, void* stream) {
    if (!ctx || !out) return fail(PTCA_ERR_INVALID, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PTCA_SETTLE(ctx, st);
    PTCA_CUDA(ptca::launch_observables(ctx->d_S[0], ctx->p.Lx, ctx->p.Ly, ctx->d_rec_Facc, ctx->d_rec_fill,
                                       ctx->d_rec_acc, ctx->d_rec_n, ctx->N, ctx->d_obs, st));
    double h[5];
    PTCA_CUDA(cudaMemcpyAsync(h, ctx->d_obs, sizeof h, cudaMemcpyDeviceToHost, st));
    PTCA_CUDA(cudaStreamSynchronize(st));
    out->S_00 = h[0];
    out->S_pipi = h[1];
    out->F_site = h[2];
    out->acceptance = h[3];
    out->filling = h[4];
    return PTCA_OK;
}

}  // extern "C"
