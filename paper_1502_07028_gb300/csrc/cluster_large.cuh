// cluster_large.cuh -- the FP32 stage kernel for large traveling clusters
// (the paper's N_c = 12^2 and 16^2, Sec. VII.a) with the cluster matrix held
// in distributed shared memory: one thread-block cluster of C CTAs per
// matrix, each CTA on its own SM.
//
// Layout.  Row i of the packed lower triangle lives in the shared memory of
// CTA i mod C, at local offset loff(i) = C q (q-1)/2 + q (r+1) with
// q = i / C, r = i mod C (the rows of one CTA are stored one after another).
// Interleaving the rows keeps every CTA's share of the shrinking trailing
// block balanced at every step.  The Householder vectors v, w, the assembled
// matrix-vector product p and the pivot column are replicated in every CTA.
//
// One reflector step (the deferred rank-2 update fused with the Hermitian
// matrix-vector product, as in householder_tridiag_large):
//   1. each CTA runs the fused pass over its own active rows: row sums of
//      A v (complete, the row is local) and per-warp column partial sums,
//      combined into the CTA's column sums;
//   2. cluster barrier; every CTA assembles p_i = (row sum of row i, from
//      its owner) + (column sums of all CTAs, in rank order) and reads the
//      pivot column from the owners -- remote shared-memory loads;
//   3. the scalar phase (w, the explicit update of the pivot column, the
//      next reflector) runs redundantly in every CTA on the replicated data,
//      so every CTA holds bitwise the same vectors;
//   4. a split cluster barrier (arrive after the remote loads of 2, wait
//      before the next pass writes) keeps a CTA's rows and partial sums
//      alive until every other CTA has read them.
// Every CTA of a cluster takes the same items in the same order, and every
// barrier is reached the same number of times by all of them.
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace ptca {

namespace cg = cooperative_groups;

constexpr int NW_CL = 8;              // warps per CTA
constexpr int CL_THREADS = 32 * NW_CL;

template <int C> __host__ __device__ __forceinline__ int cl_loff(int i) {
    const int q = i / C, r = i - q * C;
    return C * q * (q - 1) / 2 + q * (r + 1);
}

// Elements of the packed triangle of order n held by the CTA of rank r.
template <int C> __host__ __device__ inline int cl_local_elems(int n, int r) {
    if (r >= n) return 0;
    const int rows = (n - 1 - r) / C + 1;
    return cl_loff<C>(r + rows * C);
}

template <int C> __host__ __device__ inline int cl_max_local_elems(int n) {
    int mx = 0;
    for (int r = 0; r < C; ++r) mx = cl_local_elems<C>(n, r) > mx ? cl_local_elems<C>(n, r) : mx;
    return mx;
}

// Shared-memory layout of one CTA (byte offsets, 16-byte aligned).  The
// per-warp column partials are live only during the reduction, so the window
// spins of the build and the eigenvalue-stage arrays share their region.
struct ClLayout {
    size_t A, Vb, Wv, pr, cs, p, col, d, e2, pcw, sp, df, e2f, dlo, e2lo, lam, cnt, red, part, total;
};

template <int C> __host__ __device__ inline ClLayout cl_layout(int nA) {
    ClLayout L;
    const size_t nm = (size_t)((nA + 31) / 32 * 32), fc = sizeof(float2);
    size_t o = 0;
    L.A = o;    o = align16(o + (size_t)cl_max_local_elems<C>(nA) * fc + 32 * fc);  // + one warp of padding
    L.Vb = o;   o = align16(o + 2 * nm * fc);
    L.Wv = o;   o = align16(o + nm * fc);
    L.pr = o;   o = align16(o + nm * fc);
    L.cs = o;   o = align16(o + nm * fc);
    L.p = o;    o = align16(o + nm * fc);
    L.col = o;  o = align16(o + nm * fc);
    L.d = o;    o = align16(o + nm * sizeof(double));
    L.e2 = o;   o = align16(o + nm * sizeof(double));
    L.pcw = o;
    L.sp = o;                              // (nm/2) x 3 doubles = 12 nm bytes
    L.df = o + 12 * nm;                    // nm floats each
    L.e2f = o + 16 * nm;
    L.dlo = o + 20 * nm;
    L.e2lo = o + 24 * nm;
    L.lam = o + 28 * nm;                   // 2 nm floats
    L.cnt = o + 36 * nm;                   // one int per thread
    o = align16(o + max2((size_t)NW_CL * nm * fc, 36 * nm + 4 * (size_t)CL_THREADS));
    L.red = o;  o = align16(o + 8 * (size_t)NW_CL * sizeof(double));
    L.part = o; o = align16(o + 4 * sizeof(double) + 2 * fc);
    L.total = o;
    return L;
}

struct ClCarve {
    float2 *A, *Vb, *Wv, *pr, *cs, *p, *col, *pcw, *sx;
    double *d, *e2, *sp, *red, *part;
    float *df, *e2f, *dlo, *e2lo, *lam;
    int* cnt;
};

__device__ __forceinline__ ClCarve cl_carve(unsigned char* base, const ClLayout& L) {
    ClCarve c;
    c.A = reinterpret_cast<float2*>(base + L.A);
    c.Vb = reinterpret_cast<float2*>(base + L.Vb);
    c.Wv = reinterpret_cast<float2*>(base + L.Wv);
    c.pr = reinterpret_cast<float2*>(base + L.pr);
    c.cs = reinterpret_cast<float2*>(base + L.cs);
    c.p = reinterpret_cast<float2*>(base + L.p);
    c.col = reinterpret_cast<float2*>(base + L.col);
    c.pcw = reinterpret_cast<float2*>(base + L.pcw);
    c.d = reinterpret_cast<double*>(base + L.d);
    c.e2 = reinterpret_cast<double*>(base + L.e2);
    c.sp = reinterpret_cast<double*>(base + L.sp);
    c.df = reinterpret_cast<float*>(base + L.df);
    c.e2f = reinterpret_cast<float*>(base + L.e2f);
    c.dlo = reinterpret_cast<float*>(base + L.dlo);
    c.e2lo = reinterpret_cast<float*>(base + L.e2lo);
    c.lam = reinterpret_cast<float*>(base + L.lam);
    c.cnt = reinterpret_cast<int*>(base + L.cnt);
    c.red = reinterpret_cast<double*>(base + L.red);
    c.part = reinterpret_cast<double*>(base + L.part);
    c.sx = reinterpret_cast<float2*>(base + L.part + 4 * sizeof(double));
    return c;
}

// The cluster matrix of build_cluster (same elements, FP32), each CTA writing
// the elements of its own rows into its local rows.  Window spins are
// gathered by every CTA.  Caller syncs after.
template <int C>
__device__ void cl_build(const Model& m, const Window& w, const double* __restrict__ S, const double* s_new,
                         double* sp, float2* A, int rank) {
    const int nsite = window_nsite(w), n = 2 * nsite, exy = w.ex * w.ey;
    const int ea = cl_local_elems<C>(n, rank);
    for (int i = threadIdx.x; i < ea; i += blockDim.x) A[i] = make_float2(0.f, 0.f);
    const int uw = (w.uwz * w.ey + w.uwy) * w.ex + w.uwx;
    for (int s = threadIdx.x; s < nsite; s += blockDim.x) {
        const int wx = s % w.ex, wy = (s / w.ex) % w.ey, wz = s / exy;
        const int g = window_site(m, w, wx, wy, wz);
        double v0, v1, v2;
        if (s_new != nullptr && s == uw) { v0 = s_new[0]; v1 = s_new[1]; v2 = s_new[2]; }
        else { v0 = S[3 * g]; v1 = S[3 * g + 1]; v2 = S[3 * g + 2]; }
        sp[3 * s] = v0; sp[3 * s + 1] = v1; sp[3 * s + 2] = v2;
    }
    __syncthreads();
    const float t = (float)m.t, J = (float)m.JH, lam = (float)m.lam;
    auto put = [&](int r, int c, float2 v) {
        if (r % C == rank) A[cl_loff<C>(r) + c] = v;
    };
    for (int s = threadIdx.x; s < nsite; s += blockDim.x) {
        const int wx = s % w.ex, wy = (s / w.ex) % w.ey, wz = s / exy;
        const float sx = (float)sp[3 * s], sy = (float)sp[3 * s + 1], sz = (float)sp[3 * s + 2];
        const int a = 2 * s, b = 2 * s + 1;
        const float dg = lam * sx;
        put(a, a, make_float2(dg - J * sz, 0.f));
        put(b, b, make_float2(dg + J * sz, 0.f));
        put(b, a, make_float2(-J * sx, -J * sy));
        int nbs[3], mults[3];
        // +x, +y, +z bonds (same rules as build_cluster)
        nbs[0] = -1; mults[0] = 1;
        if (wx + 1 < w.ex) { nbs[0] = s + 1; if (m.cluster_periodic && w.ex == 2) mults[0] = 2; }
        else if (m.cluster_periodic && w.ex >= 3) nbs[0] = s - (w.ex - 1);
        nbs[1] = -1; mults[1] = 1;
        if (wy + 1 < w.ey) { nbs[1] = s + w.ex; if (m.cluster_periodic && w.ey == 2) mults[1] = 2; }
        else if (m.cluster_periodic && w.ey >= 3) nbs[1] = s - (w.ey - 1) * w.ex;
        nbs[2] = -1; mults[2] = 1;
        if (wz + 1 < w.ez) { nbs[2] = s + exy; if (m.cluster_periodic && w.ez == 2) mults[2] = 2; }
        else if (m.cluster_periodic && w.ez >= 3) nbs[2] = s - (w.ez - 1) * exy;
        for (int d = 0; d < 3; ++d) {
            const int nb = nbs[d];
            if (nb < 0) continue;
            const int hi = nb > s ? nb : s, lo = nb > s ? s : nb;
            for (int sg = 0; sg < 2; ++sg) put(2 * hi + sg, 2 * lo + sg, make_float2(-(float)mults[d] * t, 0.f));
        }
    }
}

// Householder reduction of the cluster-distributed matrix (order n) to real
// tridiagonal form: d[0..n-1], e2[0..n-2] in every CTA.  All CTAs of the
// cluster call it together.
template <int C>
__device__ void cl_tridiag(int n, int nm, ClCarve& c, cg::cluster_group& cl) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)cl.block_rank();
    const float2 zero = make_float2(0.f, 0.f);
    for (int i = tid; i < 2 * nm; i += CL_THREADS) c.Vb[i] = zero;
    for (int i = tid; i < nm; i += CL_THREADS) c.Wv[i] = zero;
    cl.sync();  // every CTA's rows built
    auto remote = [&](int i, int j) -> float2 {  // element (i, j <= i) from its owner
        return cl.map_shared_rank(c.A, i % C)[cl_loff<C>(i) + j];
    };
    if (n <= 2) {
        if (tid == 0) {
            c.d[0] = (double)remote(0, 0).x;
            if (n == 2) { c.d[1] = (double)remote(1, 1).x; c.e2[0] = (double)cabs2(remote(1, 0)); }
        }
        __syncthreads();
        return;
    }
    float2 vfirst;
    float tau;
    {
        // column 0: d_0, ||x||^2 and the first reflector
        float s2p = 0.f;
        for (int i = tid; i < n; i += CL_THREADS) {
            const float2 a = remote(i, 0);
            if (i == 0) c.d[0] = (double)a.x;
            if (i >= 1) s2p += cabs2(a);
            if (i >= 2) c.Vb[i] = a;
            if (i == 1) c.sx[0] = a;
        }
        const float s2 = block_sum<float>(s2p, reinterpret_cast<float*>(c.red));
        if (tid == 0) c.e2[0] = (double)s2;
        reflector_head(s2, c.sx[0], vfirst, tau);
    }
    for (int k = 0; k <= n - 3; ++k) {
        const float2* V_ = c.Vb + (k & 1) * nm;        // v_k (entry k+1 is vfirst)
        const float2* U_ = c.Vb + ((k + 1) & 1) * nm;  // v_{k-1} (zero at k = 0)
        float2* Vn = c.Vb + ((k + 1) & 1) * nm;        // v_{k+1} replaces it after the pass
        const int j0 = k + 1, m = n - j0;
        // ---- 1. fused pass over this CTA's active rows, longest first
        float2* pcw = c.pcw + warp * nm;
        for (int jr = lane; jr < m; jr += 32) pcw[jr] = zero;
        const int ilast = (n - 1) - ((n - 1 - rank) % C);
        const int R = ilast >= j0 ? (ilast - j0) / C + 1 : 0;
        for (int t = warp; t < R; t += NW_CL) {
            const int i = ilast - C * t, ri = i - j0;
            const float2 ui = U_[i], wi = c.Wv[i], vi = ri == 0 ? vfirst : V_[i];
            float2* row = c.A + cl_loff<C>(i) + j0;
            float2 racc = zero;
            constexpr int LU = 4;
            for (int jb = 0; jb <= ri; jb += 32 * LU) {
                float2 av[LU];
#pragma unroll
                for (int q = 0; q < LU; ++q) {
                    const int jr = jb + 32 * q + lane;
                    av[q] = jr <= ri ? row[jr] : zero;
                }
#pragma unroll
                for (int q = 0; q < LU; ++q) {
                    const int jr = jb + 32 * q + lane;
                    if (jr <= ri) {
                        const int j = j0 + jr;
                        const float2 vj = jr == 0 ? vfirst : V_[j];
                        float2 a = av[q];
                        a = cfms_conj_b(ui, c.Wv[j], a);
                        a = cfms_conj_b(wi, U_[j], a);
                        row[jr] = a;
                        racc = cfma(a, vj, racc);
                        if (jr < ri) pcw[jr] = cfma_conj_a(a, vi, pcw[jr]);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) racc = cadd(racc, cshfl_xor(racc, o));
            if (lane == 0) c.pr[ri] = racc;
        }
        __syncthreads();
        for (int jr = tid; jr < m; jr += CL_THREADS) {
            float2 s = c.pcw[jr];
#pragma unroll
            for (int w = 1; w < NW_CL; ++w) s = cadd(s, c.pcw[w * nm + jr]);
            c.cs[jr] = s;
        }
        // ---- 2. every CTA's row and column sums are complete: assemble p
        // and read the pivot column j0 from the owners of its rows
        cl.sync();
        for (int ri = tid; ri < m; ri += CL_THREADS) {
            const int i = j0 + ri, own = i % C;
            float2 s = cl.map_shared_rank(c.pr, own)[ri];
#pragma unroll
            for (int q = 0; q < C; ++q) s = cadd(s, cl.map_shared_rank(c.cs, q)[ri]);
            c.p[ri] = s;
            c.col[ri] = cl.map_shared_rank(c.A, own)[cl_loff<C>(i) + j0];
        }
        cl.barrier_arrive();
        __syncthreads();
        // ---- 3. scalar phase, replicated: p = tau A v, K = (tau/2) v^H p,
        // w = p - K v, the explicit update of pivot column j0 with (v_k, w_k),
        // d_j0, ||x||^2 and the next reflector
        float sp = 0.f;
        for (int ri = tid; ri < m; ri += CL_THREADS) {
            float2 p = c.p[ri];
            p.x *= tau; p.y *= tau;
            c.p[ri] = p;
            const float2 v = ri == 0 ? vfirst : V_[j0 + ri];
            sp += v.x * p.x + v.y * p.y;
        }
        const float K = 0.5f * tau * block_sum<float>(sp, reinterpret_cast<float*>(c.red));
        const float2 p0 = c.p[0];
        const float2 w0 = make_float2(p0.x - K * vfirst.x, p0.y - K * vfirst.y);
        float s2p = 0.f;
        for (int ri = tid; ri < m; ri += CL_THREADS) {
            const float2 v = ri == 0 ? vfirst : V_[j0 + ri];
            const float2 p = c.p[ri];
            const float2 w = make_float2(p.x - K * v.x, p.y - K * v.y);
            c.Wv[j0 + ri] = w;
            float2 a = c.col[ri];
            a = cfms_conj_b(v, w0, a);
            a = cfms_conj_b(w, vfirst, a);
            if (ri == 0) c.d[j0] = (double)a.x;
            if (ri >= 1) s2p += cabs2(a);
            if (ri >= 2) Vn[j0 + ri] = a;
            if (ri == 1) c.sx[0] = a;
        }
        __syncthreads();  // the first block sum's partials are read; reuse them
        const float s2 = block_sum<float>(s2p, reinterpret_cast<float*>(c.red) + NW_CL);
        if (tid == 0) c.e2[j0] = (double)s2;
        if (k + 1 <= n - 3) reflector_head(s2, c.sx[0], vfirst, tau);
        // ---- 4. the other CTAs are done reading this CTA's sums and rows
        cl.barrier_wait();
        __syncthreads();
    }
    // step n-3's update of the last diagonal entry
    if (tid == 0) {
        const float2 v = c.Vb[((n - 3) & 1) * nm + n - 1];
        const float2 w = c.Wv[n - 1];
        c.d[n - 1] = (double)(remote(n - 1, n - 1).x - 2.f * (v.x * w.x + v.y * w.y));
    }
    __syncthreads();
}

// Eigenvalues of the replicated tridiagonal below mu + 40 T: CTA r of the
// cluster takes the r-th of C equal runs of them (FP32 multisection, then one
// double-float Newton step, as tridiag_eig_F does for PTCA_MIXED) and returns
// its partial sums of softplus(-(eps-mu)/T) and of the Fermi function.
template <int C>
__device__ void cl_eig_F(int n, ClCarve& c, double mu, double temp, int rank, double& sum_sp, double& sum_fe) {
    __shared__ double s_lo, s_hi;
    __shared__ float s_pivminf;
    __shared__ int s_K;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double glo = 1e300, ghi = -1e300, ge = 0.0;
    for (int i = tid; i < n; i += CL_THREADS) {
        const double el = i > 0 ? sqrt(c.e2[i - 1]) : 0.0;
        const double er = i < n - 1 ? sqrt(c.e2[i]) : 0.0;
        glo = fmin(glo, c.d[i] - el - er);
        ghi = fmax(ghi, c.d[i] + el + er);
        const double ee = i < n - 1 ? c.e2[i] : 0.0;
        ge = fmax(ge, ee);
        c.df[i] = (float)c.d[i];
        c.e2f[i] = (float)ee;
        c.dlo[i] = (float)(c.d[i] - (double)c.df[i]);
        c.e2lo[i] = (float)(ee - (double)c.e2f[i]);
    }
    glo = warp_min(glo); ghi = warp_max(ghi); ge = warp_max(ge);
    if (lane == 0) { c.red[warp] = glo; c.red[NW_CL + warp] = ghi; c.red[2 * NW_CL + warp] = ge; }
    __syncthreads();
    if (tid == 0) {
        double lo = c.red[0], hi = c.red[NW_CL], emax2 = c.red[2 * NW_CL];
        for (int w = 1; w < NW_CL; ++w) {
            lo = fmin(lo, c.red[w]); hi = fmax(hi, c.red[NW_CL + w]); emax2 = fmax(emax2, c.red[2 * NW_CL + w]);
        }
        const double wdt = hi - lo, nrm = fmax(fabs(lo), fabs(hi));
        lo -= 1e-12 * (wdt + nrm) + 1e-300;
        hi += 1e-12 * (wdt + nrm) + 1e-300;
        s_lo = lo; s_hi = hi;
        s_pivminf = FLT_MIN * fmaxf(1.0f, (float)emax2);
        int K = n;
        const double cut = mu + kFermiCut * temp;
        if (cut < hi) K = sturm_count_f32(n, c.df, c.e2f, (float)cut, s_pivminf);
        s_K = K;
    }
    __syncthreads();
    const int K = s_K;
    const int per = (K + C - 1) / C, k_lo = rank * per, k_hi = min(K, k_lo + per), nk = max(0, k_hi - k_lo);
    const double lo = s_lo, hi = s_hi, nrm = fmax(fabs(lo), fabs(hi));
    {
        int G = 1;
        while (G < 8 && 2 * G * nk <= CL_THREADS) G *= 2;
        const int kk = tid / G, j = tid % G, k = k_lo + kk;
        const float lof = (float)lo * (lo < 0 ? 1.0000002f : 0.9999998f) - 1e-30f;
        const float hif = (float)hi * (hi > 0 ? 1.0000002f : 0.9999998f) + 1e-30f;
        const int P = CL_THREADS;
        const float h0 = (hif - lof) / (float)(P + 1);
        c.cnt[tid] = sturm_count_f32(n, c.df, c.e2f, lof + (float)(tid + 1) * h0, s_pivminf);
        __syncthreads();
        const float atolf = fmaxf(2.0f * FLT_EPSILON * (float)nrm, 1e-30f);
        const float ratio = 2.f * h0 / atolf;
        int rounds = ratio > 1.0f ? (int)ceilf(log2f(ratio) / log2f((float)(G + 1))) + 1 : 1;
        rounds = rounds < 64 ? rounds : 64;
        if ((warp * 32) / G < nk) {
            int lo_i = -1, hi_i = P;
            while (hi_i - lo_i > 1) {
                const int mid = (lo_i + hi_i) >> 1;
                if (c.cnt[mid] <= k) lo_i = mid; else hi_i = mid;
            }
            float a = lo_i < 0 ? lof : lof + (float)(lo_i + 1) * h0;
            float b = hi_i >= P ? hif : lof + (float)(hi_i + 1) * h0;
            const unsigned gmask = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
            const int gshift = (lane / G) * G;
            for (int r = 0; r < rounds; ++r) {
                const float h = (b - a) / (float)(G + 1);
                bool flag = false;
                if (kk < nk) flag = sturm_count_f32(n, c.df, c.e2f, a + (float)(j + 1) * h, s_pivminf) <= k;
                const unsigned bal = __ballot_sync(FULL_MASK, flag);
                const int J = __popc((bal >> gshift) & gmask);
                const float na = J > 0 ? a + (float)J * h : a;
                const float nb = J < G ? a + (float)(J + 1) * h : b;
                a = na; b = nb;
            }
            if (kk < nk && j == 0) { c.lam[2 * kk] = a; c.lam[2 * kk + 1] = b; }
        }
        __syncthreads();
    }
    double sp = 0.0, fe = 0.0;
    if (tid < nk) {
        const double lam = newton_polish_df(n, c.df, c.dlo, c.e2f, c.e2lo, c.lam[2 * tid], c.lam[2 * tid + 1],
                                            2.0f * FLT_EPSILON * (float)nrm, s_pivminf);
        const double x = -(lam - mu) / temp;
        sp = softplus(x);
        fe = 1.0 / (1.0 + exp(-x));
    }
    __syncthreads();
    sum_sp = block_sum<double>(sp, c.red);
    __syncthreads();
    sum_fe = block_sum<double>(fe, c.red + NW_CL);
}

// One PTCA stage of large clusters, FP32 reduction (PTCA_MIXED): cluster q of
// the grid takes items q, q + clusters, ... (item 2c: H_old of visit c, 2c+1:
// H_new), the same decisions and records as k_stage.
template <int C>
__global__ void __launch_bounds__(CL_THREADS, 1) k_stage_cluster(StageArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    __shared__ int s_last;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.prev_count + a.prev2_count;
         k += gridDim.x * blockDim.x) {
        const int s = k < a.prev_count ? a.prev_sites[k] : a.prev2_sites[k - a.prev_count];
        a.S_out[3 * s] = a.S_in[3 * s];
        a.S_out[3 * s + 1] = a.S_in[3 * s + 1];
        a.S_out[3 * s + 2] = a.S_in[3 * s + 2];
    }
    const ClLayout L = cl_layout<C>(a.nA);
    ClCarve cv = cl_carve(smem, L);
    const int nm = (a.nA + 31) / 32 * 32;
    const int nclusters = gridDim.x / C, cid = blockIdx.x / C;
    for (int item = cid; item < 2 * a.count; item += nclusters) {
        const int c = a.perm ? a.perm[item >> 1] : (item >> 1), var = item & 1;
        const int site = a.sites[c];
        const Window w = make_window(a.m, site);
        const int n = 2 * window_nsite(w);
        if (threadIdx.x == 0 && var == 1) propose(a.m, a.sweep, (uint32_t)site, a.S_in + 3 * site, s_new);
        __syncthreads();
        cl_build<C>(a.m, w, a.S_in, var ? s_new : nullptr, cv.sp, cv.A, rank);
        __syncthreads();
        const double cls = (rank == 0 && threadIdx.x == 0) ? window_classical(a.m, cv.sp, n / 2) : 0.0;
        cl_tridiag<C>(n, nm, cv, cl);
        double ssp, sfe;
        cl_eig_F<C>(n, cv, a.m.mu - a.m.e0, a.m.T, rank, ssp, sfe);
        if (threadIdx.x == 0) { cv.part[0] = ssp; cv.part[1] = sfe; }
        cl.sync();  // every CTA's partial sums are in place
        if (rank == 0) {
            if (threadIdx.x == 0) {
                double tsp = 0.0, tfe = 0.0;
                for (int q = 0; q < C; ++q) {
                    const double* pq = cl.map_shared_rank(cv.part, q);
                    tsp += pq[0];
                    tfe += pq[1];
                }
                a.Fbuf[2 * c + var] = -a.m.T * tsp + cls;
                a.fillbuf[2 * c + var] = tfe;
                __threadfence();
                s_last = (atomicAdd(&a.ticket[c], 1) == 1);
            }
            __syncthreads();
            if (s_last && threadIdx.x == 0) {
                __threadfence();
                a.ticket[c] = 0;
                const double Fo = __ldcg(&a.Fbuf[2 * c]), Fn = __ldcg(&a.Fbuf[2 * c + 1]);
                const double fo = __ldcg(&a.fillbuf[2 * c]), fn = __ldcg(&a.fillbuf[2 * c + 1]);
                double sn[3];
                const double* so = a.S_in + 3 * site;
                if (var == 1) { sn[0] = s_new[0]; sn[1] = s_new[1]; sn[2] = s_new[2]; }
                else propose(a.m, a.sweep, (uint32_t)site, so, sn);
                double u0, u1;
                uniform2(a.m.seed, a.sweep, (uint32_t)site, RNG_ACCEPT, u0, u1);
                const double lnu = log(u0);
                const double dF = Fn - Fo;
                if (!isfinite(dF)) atomicExch(a.err, 1);
                if (a.margin > 0.0 && fabs(lnu + dF / a.m.T) < a.margin) {
                    a.flag_list[atomicAdd(a.flag_count, 1u)] = c;
                    atomicAdd(&a.counters[2], 1ull);
                } else {
                    const bool acc = lnu < -dF / a.m.T;
                    double* dst = a.S_out + 3 * site;
                    if (acc) { dst[0] = sn[0]; dst[1] = sn[1]; dst[2] = sn[2]; }
                    else { dst[0] = so[0]; dst[1] = so[1]; dst[2] = so[2]; }
                    const int r = a.rec_base + c;
                    a.rec_site[r] = site;
                    a.rec_Fold[r] = Fo;
                    a.rec_Fnew[r] = Fn;
                    a.rec_lnu[r] = lnu;
                    a.rec_acc[r] = acc ? 1 : 0;
                    a.rec_Facc[r] = acc ? Fn : Fo;
                    a.rec_fill[r] = acc ? fn : fo;
                    a.rec_n[r] = n;
                    if (acc) atomicAdd(&a.counters[0], 1ull);
                    atomicAdd(&a.counters[1], 2ull);
                }
            }
        }
        cl.sync();  // rank 0 has read every CTA's partial sums; rows may be rebuilt
    }
}

}  // namespace ptca
