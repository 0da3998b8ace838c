// kernels_misc.cu -- small kernels (initial spins, copies, free energy of
// eigenvalue lists, observables) and the precision dispatch of the launchers.
#include "kernels.cuh"
#include "launch.h"

namespace ptca {

// Declarations of the per-precision launchers (kernels_f32.cu / kernels_f64.cu).
size_t cluster_smem_bytes_f32(int nA);
size_t cluster_smem_bytes_f64(int nA);
int cluster_max_order_f32();
int cluster_max_order_f64();
cudaError_t configure_f32(size_t);
cudaError_t configure_f64(size_t);
cudaError_t launch_build_f32(const Model&, const double*, const int32_t*, int, const double*, void*, int64_t,
                             int64_t*, int32_t*, cudaStream_t);
cudaError_t launch_build_f64(const Model&, const double*, const int32_t*, int, const double*, void*, int64_t,
                             int64_t*, int32_t*, cudaStream_t);
cudaError_t launch_eigvals_f32(int, const void*, const int64_t*, const int32_t*, int, double*, const int64_t*,
                               cudaStream_t);
cudaError_t launch_eigvals_f64(int, const void*, const int64_t*, const int32_t*, int, double*, const int64_t*,
                               cudaStream_t);
cudaError_t launch_stage_f32(const StageArgs&, cudaStream_t);
cudaError_t launch_stage_f64(const StageArgs&, cudaStream_t);
cudaError_t launch_persistent_f32(const PersistArgs&, int, cudaStream_t);
cudaError_t launch_persistent_f64(const PersistArgs&, int, cudaStream_t);
int persistent_blocks_per_sm_f32(int);
int persistent_blocks_per_sm_f64(int);
// 4-warp FP32 sweep kernels (kernels_f32w4.cu)
size_t cluster_smem_bytes_f32w4(int nA);
int cluster_max_order_f32w4();
cudaError_t configure_f32w4(size_t);
cudaError_t launch_stage_f32w4(const StageArgs&, cudaStream_t);
cudaError_t launch_persistent_f32w4(const PersistArgs&, int, cudaStream_t);
int persistent_blocks_per_sm_f32w4(int);
// one-warp FP32 sweep kernels (kernels_f32w1.cu)
size_t cluster_smem_bytes_f32w1(int nA);
int cluster_max_order_f32w1();
cudaError_t configure_f32w1(size_t);
cudaError_t launch_stage_f32w1(const StageArgs&, cudaStream_t);
cudaError_t launch_persistent_f32w1(const PersistArgs&, int, cudaStream_t);
int persistent_blocks_per_sm_f32w1(int);
cudaError_t launch_resolve_f32(const StageArgs&, int, cudaStream_t);
bool resolve_smem_fits_f32(int nA);
cudaError_t launch_check_f32(const StageArgs&, int, int, double*, int, double*, cudaStream_t);
cudaError_t launch_check_ref_f32(const StageArgs&, int, int, double*, int, double*, int, cudaStream_t);

size_t cluster_smem_bytes(int prec, int nA) { return prec ? cluster_smem_bytes_f32(nA) : cluster_smem_bytes_f64(nA); }
int cluster_max_order(int prec) { return prec ? cluster_max_order_f32() : cluster_max_order_f64(); }
cudaError_t configure_cluster_kernels(size_t smem_limit) {
    cudaError_t e = configure_f32(smem_limit);
    if (e == cudaSuccess) e = configure_f32w4(smem_limit);
    if (e == cudaSuccess) e = configure_f32w1(smem_limit);
    if (e == cudaSuccess) e = configure_tiled_kernels(smem_limit);
    if (e == cudaSuccess) e = configure_shared_kernels(smem_limit);
    if (e == cudaSuccess) e = configure_panel_kernels(smem_limit);
    if (e != cudaSuccess) return e;
    return configure_f64(smem_limit);
}
bool sweep_width_supported(int prec, int nw, int nA) {
    if (nw == 8) return nA <= cluster_max_order(prec);
    if (nw == 1) return prec == 1 && nA <= cluster_max_order_f32w1();
    return nw == 4 && prec == 1 && nA <= cluster_max_order_f32w4();
}
size_t sweep_smem_bytes(int prec, int nw, int nA) {
    if (nw == 1) return cluster_smem_bytes_f32w1(nA);
    return nw == 4 ? cluster_smem_bytes_f32w4(nA) : cluster_smem_bytes(prec, nA);
}
cudaError_t launch_build(int prec, const Model& m, const double* S, const int32_t* sites, int count,
                         const double* new_spins, void* H, int64_t stride, int64_t* offsets, int32_t* nout,
                         cudaStream_t st) {
    return prec ? launch_build_f32(m, S, sites, count, new_spins, H, stride, offsets, nout, st)
                : launch_build_f64(m, S, sites, count, new_spins, H, stride, offsets, nout, st);
}
cudaError_t launch_eigvals(int prec, int nA, const void* H, const int64_t* offsets, const int32_t* n, int count,
                           double* eig, const int64_t* eoff, cudaStream_t st) {
    return prec ? launch_eigvals_f32(nA, H, offsets, n, count, eig, eoff, st)
                : launch_eigvals_f64(nA, H, offsets, n, count, eig, eoff, st);
}
cudaError_t launch_stage(int prec, int nw, const StageArgs& a, cudaStream_t st) {
    if (nw == 4) return prec ? launch_stage_f32w4(a, st) : cudaErrorInvalidValue;
    if (nw == 1) return prec ? launch_stage_f32w1(a, st) : cudaErrorInvalidValue;
    return prec ? launch_stage_f32(a, st) : launch_stage_f64(a, st);
}
cudaError_t launch_persistent(int prec, int nw, const PersistArgs& p, int grid, cudaStream_t st) {
    if (nw == 4) return prec ? launch_persistent_f32w4(p, grid, st) : cudaErrorInvalidValue;
    if (nw == 1) return prec ? launch_persistent_f32w1(p, grid, st) : cudaErrorInvalidValue;
    return prec ? launch_persistent_f32(p, grid, st) : launch_persistent_f64(p, grid, st);
}
cudaError_t launch_resolve(const StageArgs& a, int grid, cudaStream_t st) { return launch_resolve_f32(a, grid, st); }
bool resolve_smem_fits(int nA) { return resolve_smem_fits_f32(nA); }
int persistent_blocks_per_sm(int prec, int nw, int nA) {
    if (nw == 4) return prec ? persistent_blocks_per_sm_f32w4(nA) : 0;
    if (nw == 1) return prec ? persistent_blocks_per_sm_f32w1(nA) : 0;
    return prec ? persistent_blocks_per_sm_f32(nA) : persistent_blocks_per_sm_f64(nA);
}

cudaError_t launch_check(int prec, const StageArgs& a, int c0, int count, double* eig, int ld, double* F, int grid,
                         cudaStream_t st) {
    return prec ? launch_check_f32(a, c0, count, eig, ld, F, st)
                : launch_check_ref_f32(a, c0, count, eig, ld, F, grid, st);
}

// Non-negative doubles order like their bit patterns (NaN above +inf).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(fabs(v)));
}

// Errors of the FP32-reduction spectra (e32, F32) against the FP64 ones (e64,
// F64) for `count` visits: out[0] max |d eps|, out[1] max |d dF|, out[2] max
// |d eps| / (J_H + 4|t|) (the spectral-norm bound of every cluster matrix),
// out[3] max |d dF| / max(1, |F_old|, |F_new|), out[4] max |d dF| / s with
// the free-energy-difference scale s = max(|dF|, sum_k |eps_k - mu| f_k / n)
// of the FP64 old-cluster spectrum (f the Fermi function): the typical size
// of one level's contribution to F, the scale on which dF itself lives (as
// bit patterns of non-negative doubles).
__global__ void k_check_compare(Model m, const int32_t* __restrict__ sites, int count, const double* __restrict__ e32,
                                const double* __restrict__ e64, int ld, const double* __restrict__ F32,
                                const double* __restrict__ F64, unsigned long long* out) {
    __shared__ double s_part[32];
    const int c = blockIdx.x;
    if (c >= count) return;
    const Window w = make_window(m, sites[c]);
    const int n = 2 * window_nsite(w);
    const double mu = m.mu - m.e0;  // the spectra are of the matrix without its on-site shift e0
    double de = 0.0, lev = 0.0;
    for (int var = 0; var < 2; ++var) {
        const double* a = e32 + (int64_t)(2 * c + var) * ld;
        const double* b = e64 + (int64_t)(2 * c + var) * ld;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double d = fabs(a[k] - b[k]);
            de = (d > de || d != d) ? d : de;
            if (var == 0) {
                const double x = (b[k] - mu) / m.T;
                lev += fabs(b[k] - mu) / (1.0 + exp(x));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double x = __shfl_xor_sync(0xffffffffu, de, o);
        de = (x > de || x != x) ? x : de;
        lev += __shfl_xor_sync(0xffffffffu, lev, o);
    }
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(out, de);
        atomic_max_nonneg(out + 2, de / (m.JH + 4.0 * fabs(m.t)));
        s_part[warp] = lev;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double levels = 0.0;
        for (int q = 0; q < nwarp; ++q) levels += s_part[q];
        const double d64 = F64[2 * c + 1] - F64[2 * c];
        const double d32 = F32[2 * c + 1] - F32[2 * c];
        const double ddF = fabs(d32 - d64);
        atomic_max_nonneg(out + 1, ddF);
        atomic_max_nonneg(out + 3, ddF / fmax(1.0, fmax(fabs(F64[2 * c]), fabs(F64[2 * c + 1]))));
        const double scale = fmax(fabs(d64), levels / (double)n);
        atomic_max_nonneg(out + 4, scale > 0.0 ? ddF / scale : ddF);
    }
}

cudaError_t launch_check_compare(const Model& m, const int32_t* sites, int count, const double* e32,
                                 const double* e64, int ld, const double* F32, const double* F64,
                                 unsigned long long* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_check_compare<<<count, 128, 0, st>>>(m, sites, count, e32, e64, ld, F32, F64, out);
    return cudaGetLastError();
}

__global__ void k_barrier_selftest(unsigned int* bar, int32_t* err, unsigned long long timeout_ns) {
    grid_barrier(bar, gridDim.x + 1, timeout_ns, err, nullptr);
}

cudaError_t launch_barrier_selftest(int blocks, unsigned int* bar, int32_t* err, unsigned long long timeout_ns,
                                    cudaStream_t st) {
    k_barrier_selftest<<<blocks, 32, 0, st>>>(bar, err, timeout_ns);
    return cudaGetLastError();
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

// Status word of a sweep from its device error slots: err[1] (a timed-out
// barrier) -> 4 (PTCA_ERR_TIMEOUT), else err[0] (a non-finite dF) -> 5
// (PTCA_ERR_NUMERIC), else 0.
__global__ void k_status_word(const int32_t* err, int32_t* out) { *out = err[1] ? 4 : (err[0] ? 5 : 0); }

cudaError_t launch_status_word(const int32_t* err, int32_t* out, cudaStream_t st) {
    k_status_word<<<1, 1, 0, st>>>(err, out);
    return cudaGetLastError();
}

cudaError_t launch_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st) {
    k_set_u64<<<1, 1, 0, st>>>(p, v);
    return cudaGetLastError();
}

// Initial spins: uniform on the sphere from the counter generator.
// Initial classical variables: unit vectors uniform on the sphere; for the
// Holstein model distortions x uniform in [-1, 1] in component 0.
__global__ void k_init_spins(Model m, double* __restrict__ S, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double u0, u1, s[3];
    uniform2(m.seed, 0, (uint32_t)i, RNG_INIT, u0, u1);
    if (m.model == 2) {
        s[0] = 2.0 * u0 - 1.0; s[1] = 0.0; s[2] = 0.0;
    } else {
        unit_from_uniforms(u0, u1, s);
    }
    S[3 * i] = s[0]; S[3 * i + 1] = s[1]; S[3 * i + 2] = s[2];
}

void set_model_terms(Model& m, int model, double J_H, double U, double lam, double K, double mu, double m_step) {
    m.model = model;
    m.JH = 0.0; m.e0 = 0.0; m.lam = 0.0; m.ca = 0.0; m.cb = 0.0; m.cc = 0.0; m.m_step = 0.0; m.cls_on = 0;
    if (model == 1) {
        m.JH = 0.5 * U; m.e0 = 0.5 * U; m.ca = 0.25 * U; m.cc = -0.25 * U; m.m_step = m_step; m.cls_on = 1;
    } else if (model == 2) {
        m.lam = lam; m.ca = 0.5 * K; m.cb = -lam; m.cc = mu; m.m_step = m_step; m.cls_on = 1;
    } else {
        m.JH = J_H;
    }
}

cudaError_t launch_init_spins(const Model& m, double* S, int N, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    k_init_spins<<<(N + 255) / 256, 256, 0, st>>>(m, S, N);
    return cudaGetLastError();
}

__global__ void k_copy_sites(const double* __restrict__ src, double* __restrict__ dst,
                             const int32_t* __restrict__ sites, int count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int s = sites[k];
    dst[3 * s] = src[3 * s]; dst[3 * s + 1] = src[3 * s + 1]; dst[3 * s + 2] = src[3 * s + 2];
}

cudaError_t launch_copy_sites(const double* src, double* dst, const int32_t* sites, int count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_copy_sites<<<(count + 255) / 256, 256, 0, st>>>(src, dst, sites, count);
    return cudaGetLastError();
}

// out[k] = S[sites[k]] (three components), k < count.
__global__ void k_gather_sites(const double* __restrict__ S, const int32_t* __restrict__ sites, int count,
                               double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int s = sites[k];
    out[3 * k] = S[3 * s]; out[3 * k + 1] = S[3 * s + 1]; out[3 * k + 2] = S[3 * s + 2];
}

cudaError_t launch_gather_sites(const double* S, const int32_t* sites, int count, double* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_gather_sites<<<(count + 255) / 256, 256, 0, st>>>(S, sites, count, out);
    return cudaGetLastError();
}

// S0[sites[k]] = S1[sites[k]] = in[k], k < count.
__global__ void k_scatter_sites(const int32_t* __restrict__ sites, int count, const double* __restrict__ in,
                                double* __restrict__ S0, double* __restrict__ S1) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int s = sites[k];
    for (int a = 0; a < 3; ++a) {
        const double v = in[3 * k + a];
        S0[3 * s + a] = v;
        S1[3 * s + a] = v;
    }
}

cudaError_t launch_scatter_sites(const int32_t* sites, int count, const double* in, double* S0, double* S1,
                                 cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_scatter_sites<<<(count + 255) / 256, 256, 0, st>>>(sites, count, in, S0, S1);
    return cudaGetLastError();
}

// F_i = -T sum_k softplus(-(eig_k - mu)/T), one warp per list.
__global__ void k_free_energy(const double* __restrict__ eig, const int64_t* __restrict__ eoff,
                              const int32_t* __restrict__ n, int m, double mu, double temp, double* __restrict__ F) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wid >= m) return;
    const double* e = eig + eoff[wid];
    const int nn = n[wid];
    double acc = 0.0;
    for (int k = lane; k < nn; k += 32) acc += softplus(-(e[k] - mu) / temp);
    acc = warp_sum(acc);
    if (lane == 0) F[wid] = -temp * acc;
}

cudaError_t launch_free_energy(const double* eig, const int64_t* eoff, const int32_t* n, int count, double mu,
                               double T, double* F, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int threads = 256, blocks = (count * 32 + threads - 1) / threads;
    k_free_energy<<<blocks, threads, 0, st>>>(eig, eoff, n, count, mu, T, F);
    return cudaGetLastError();
}

// Observables (single CTA): S(q) = |sum_i S_i e^{i q.r_i}|^2 / N^2 at (0,0)
// and (pi,pi) (Eq. 2 for one configuration), and the means over the last
// sweep's visits of F_acc/N_c, the acceptance and the filling.
// out: [S00, Spipi, F_site, acceptance, filling]
__global__ void k_observables(const double* __restrict__ S, int Lx, int Ly, const double* __restrict__ rec_Facc,
                              const double* __restrict__ rec_fill, const uint8_t* __restrict__ rec_acc,
                              const int32_t* __restrict__ rec_n, int N, double* __restrict__ out) {
    __shared__ double red[32];
    double m0[3] = {0, 0, 0}, mp[3] = {0, 0, 0};
    double fs = 0.0, ac = 0.0, fl = 0.0, nf = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int x = i % Lx, y = (i / Lx) % Ly, z = i / (Lx * Ly);
        const double sg = ((x + y + z) & 1) ? -1.0 : 1.0;
        for (int a = 0; a < 3; ++a) { m0[a] += S[3 * i + a]; mp[a] += sg * S[3 * i + a]; }
        if (rec_n[i] > 0) {
            ac += (double)rec_acc[i];
            if (isfinite(rec_Facc[i])) {  // proposals rejected by the surrogate screen have no F
                const double nc = 0.5 * (double)rec_n[i];
                fs += rec_Facc[i] / nc;
                fl += rec_fill[i] / nc;
                nf += 1.0;
            }
        }
    }
    double vals[10] = {m0[0], m0[1], m0[2], mp[0], mp[1], mp[2], fs, ac, fl, nf};
    double tot[10];
    for (int q = 0; q < 10; ++q) {
        tot[q] = block_sum<double>(vals[q], red);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double N2 = (double)N * (double)N;
        out[0] = (tot[0] * tot[0] + tot[1] * tot[1] + tot[2] * tot[2]) / N2;
        out[1] = (tot[3] * tot[3] + tot[4] * tot[4] + tot[5] * tot[5]) / N2;
        const double nfin = tot[9] > 0 ? tot[9] : 1.0;
        out[2] = tot[6] / nfin;
        out[3] = tot[7] / N;
        out[4] = tot[8] / nfin;
    }
}

cudaError_t launch_observables(const double* S, int Lx, int Ly, const double* rec_Facc, const double* rec_fill,
                               const uint8_t* rec_acc, const int32_t* rec_n, int N, double* out, cudaStream_t st) {
    k_observables<<<1, 1024, 0, st>>>(S, Lx, Ly, rec_Facc, rec_fill, rec_acc, rec_n, N, out);
    return cudaGetLastError();
}

}  // namespace ptca
