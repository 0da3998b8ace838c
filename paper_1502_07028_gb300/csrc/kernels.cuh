// kernels.cuh -- CUDA kernels of the PTCA hot path (templated on the
// reduction precision T and on NT = ceil(nmax/32)).
#pragma once

#include <type_traits>

#include "cluster_solve.cuh"
#include "cluster_panel.cuh"
#include "cluster_tiled.cuh"
#include "surrogate.cuh"

namespace ptca {

constexpr int NW = 8;              // warps per CTA of the cluster kernels
constexpr int CTA = 32 * NW;
constexpr double kFermiCut = 40.0; // eigenvalues above mu + 40 T change F by < T e^-40 each

// Resident CTAs per SM the launch bounds ask for (caps the registers at
// 65536 / (value * 32 * NWP)).  Shared memory holds two 8-warp or three
// 4-warp FP32 CTAs per SM for matrices up to n = 128, one CTA otherwise;
// one-warp CTAs (n <= 32) are capped at 128 registers.
template <typename T, int NT, int NWP = NW> struct MinBlocks {
    static constexpr int value = NWP == 1 ? 16 : (sizeof(T) == 4 && NT <= 4) ? (NWP == 4 ? 3 : 2) : (NWP == 4 ? 2 : 1);
};

// Shared-memory layout of one cluster CTA (byte offsets, 16-byte aligned).
// The per-warp column sums pc are live only during the reduction, so the
// window spins of the build (sp) and the eigenvalue-phase arrays -- bisection
// brackets, float copies of (d, e2), their low parts and the sampling counts
// -- share its region.
struct SmemLayout {
    size_t A, Vb, Wv, pr, pc, d, e2, df, e2f, dlo, e2lo, cnt, sp, lam, red, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline size_t max2(size_t a, size_t b) { return a > b ? a : b; }

// nA: largest matrix order stored; nmaxc = 32 * NT; cs = sizeof(complex element);
// nw: warps per CTA
__host__ __device__ inline SmemLayout smem_layout(int nA, int nmaxc, size_t cs, int nw = NW) {
    SmemLayout L;
    size_t o = 0;
    const size_t nm = (size_t)nmaxc;
    L.A = o;   o = align16(o + (size_t)nA * (nA + 1) / 2 * cs);
    L.Vb = o;  o = align16(o + 2 * nm * cs);
    L.Wv = o;  o = align16(o + nm * cs);
    L.pr = o;  o = align16(o + nm * cs);
    L.pc = o;
    L.sp = o;                       // (nm/2) x 3 doubles = 12 nm bytes
    L.lam = o;                      // 2 nm floats = 8 nm bytes
    L.df = o + 8 * nm;              // nm floats each
    L.e2f = o + 12 * nm;
    L.dlo = o + 16 * nm;
    L.e2lo = o + 20 * nm;
    L.cnt = o + 24 * nm;            // one int per thread (32 nw)
    o = align16(o + max2((size_t)nw * nm * cs, 24 * nm + 4 * 32 * (size_t)nw));
    L.d = o;   o = align16(o + nm * sizeof(double));
    L.e2 = o;  o = align16(o + nm * sizeof(double));
    L.red = o; o = align16(o + 6 * (size_t)nw * sizeof(double));
    L.total = o;
    return L;
}

// Shared-memory layout of the FP32 4-warp CTA with the register-tiled
// reduction (orders up to 128): the tiled matrix, the two reflectors, w, the
// per-warp partial vectors of p (their region shared as in smem_layout), d
// and e2 in FP32, the block-sum slots.  No row-sum vector (pr = pc).  The
// eigenvalue phase takes (d, e2) as doubles in the matrix region, free by then.
__host__ __device__ inline SmemLayout smem_layout_tiled() {
    SmemLayout L;
    size_t o = 0;
    const size_t nm = TL_NMAX, cs = sizeof(float2);
    L.A = o;   o = align16(o + (size_t)tl_elems(TL_NMAX) * cs);
    L.Vb = o;  o = align16(o + 2 * nm * cs);
    L.Wv = o;  o = align16(o + nm * cs);
    L.pc = o;
    L.pr = o;
    L.sp = o;
    L.lam = o;
    L.df = o + 8 * nm;
    L.e2f = o + 12 * nm;
    L.dlo = o + 16 * nm;
    L.e2lo = o + 20 * nm;
    L.cnt = o + 24 * nm;
    o = align16(o + max2((size_t)TL_NW * nm * cs, 24 * nm + 4 * 32 * (size_t)TL_NW));
    L.d = o;   o = align16(o + nm * sizeof(float));
    L.e2 = o;  o = align16(o + nm * sizeof(float));
    L.red = o; o = align16(o + 6 * (size_t)TL_NW * sizeof(double));
    L.total = o;
    return L;
}

template <typename T> struct Carve {
    cplx_t<T>* A; HHScratch<T> hh; double* d; double* e2; float* df; float* e2f; float* dlo; float* e2lo; int* cnt;
    double* sp; float* lam; double* red;
};

template <typename T>
__device__ __forceinline__ Carve<T> carve(unsigned char* base, const SmemLayout& L, int nw = NW) {
    Carve<T> c;
    c.A = reinterpret_cast<cplx_t<T>*>(base + L.A);
    c.hh.Vb = reinterpret_cast<cplx_t<T>*>(base + L.Vb);
    c.hh.Wv = reinterpret_cast<cplx_t<T>*>(base + L.Wv);
    c.hh.pr = reinterpret_cast<cplx_t<T>*>(base + L.pr);
    c.hh.pc = reinterpret_cast<cplx_t<T>*>(base + L.pc);
    c.red = reinterpret_cast<double*>(base + L.red);
    c.hh.redA = reinterpret_cast<T*>(base + L.red);
    c.hh.redB = reinterpret_cast<T*>(base + L.red + 2 * nw * sizeof(double));
    c.hh.sx = reinterpret_cast<cplx_t<T>*>(base + L.red + 4 * nw * sizeof(double));
    c.d = reinterpret_cast<double*>(base + L.d);
    c.e2 = reinterpret_cast<double*>(base + L.e2);
    c.df = reinterpret_cast<float*>(base + L.df);
    c.e2f = reinterpret_cast<float*>(base + L.e2f);
    c.dlo = reinterpret_cast<float*>(base + L.dlo);
    c.e2lo = reinterpret_cast<float*>(base + L.e2lo);
    c.cnt = reinterpret_cast<int*>(base + L.cnt);
    c.sp = reinterpret_cast<double*>(base + L.sp);
    c.lam = reinterpret_cast<float*>(base + L.lam);
    return c;
}

// Eigenvalues of the tridiagonal (d, e2) in shared memory.  Computes the
// eigenvalues with index < K (all when all_eigs, else those below
// mu + 40 T), one thread per eigenvalue, and returns through eig (if not
// null, global) and the block sums of softplus(-(eps-mu)/T) and of the Fermi
// function.  Every precision first brackets each eigenvalue by FP32
// multisection on the FP32-rounded (d, e2).  T == float then takes one
// double-float Newton step; T == dfl (the re-solve) confirms the widened
// bracket with double-float Sturm counts and refines it by safeguarded
// double-float Newton; T == double does the same in FP64.
template <typename T, int NWP = NW>
__device__ void tridiag_eig_F(int n, Carve<T>& c, double mu, double temp, bool all_eigs, double* eig,
                              double& sum_sp, double& sum_fermi, int& n_solved) {
    __shared__ double s_lo, s_hi, s_pivmin;
    __shared__ float s_pivminf;
    __shared__ int s_K;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Gershgorin bounds, one row per thread, and FP32 copies of (d, e2).
    double glo = 1e300, ghi = -1e300, ge = 0.0;
    if (tid < n) {
        const double el = tid > 0 ? sqrt(c.e2[tid - 1]) : 0.0;
        const double er = tid < n - 1 ? sqrt(c.e2[tid]) : 0.0;
        glo = c.d[tid] - el - er;
        ghi = c.d[tid] + el + er;
        ge = tid < n - 1 ? c.e2[tid] : 0.0;
        // Float pairs (hi + lo) holding (d, e2) exactly, for the FP32
        // multisection (hi) and the double-float refinement (hi + lo).
        c.df[tid] = (float)c.d[tid];
        c.e2f[tid] = (float)ge;
        c.dlo[tid] = (float)(c.d[tid] - (double)c.df[tid]);
        c.e2lo[tid] = (float)(ge - (double)c.e2f[tid]);
    }
    glo = warp_min(glo); ghi = warp_max(ghi); ge = warp_max(ge);
    if (lane == 0) { c.red[warp] = glo; c.red[NWP + warp] = ghi; c.red[2 * NWP + warp] = ge; }
    __syncthreads();
    if (tid == 0) {
        double lo = c.red[0], hi = c.red[NWP], emax2 = c.red[2 * NWP];
        for (int w = 1; w < NWP; ++w) {
            lo = fmin(lo, c.red[w]); hi = fmax(hi, c.red[NWP + w]); emax2 = fmax(emax2, c.red[2 * NWP + w]);
        }
        const double wdt = hi - lo, nrm = fmax(fabs(lo), fabs(hi));
        lo -= 1e-12 * (wdt + nrm) + 1e-300;
        hi += 1e-12 * (wdt + nrm) + 1e-300;
        const double pivmin = DBL_MIN * fmax(1.0, emax2);
        const float pivminf = FLT_MIN * fmaxf(1.0f, (float)emax2);
        s_lo = lo; s_hi = hi; s_pivmin = pivmin; s_pivminf = pivminf;
        int K = n;
        if (!all_eigs) {
            const double cut = mu + kFermiCut * temp;
            if (cut < hi) {
                if constexpr (sizeof(T) == 8) K = sturm_count_f64(n, c.d, c.e2, cut, pivmin);
                else K = sturm_count_f32(n, c.df, c.e2f, (float)cut, pivminf);
            }
        }
        s_K = K;
    }
    __syncthreads();
    const int K = s_K;
    const double lo = s_lo, hi = s_hi, pivmin = s_pivmin;
    const double nrm = fmax(fabs(lo), fabs(hi));
    {
        // FP32 multisection: G threads per eigenvalue evaluate G interior
        // points per round, narrowing the bracket (G+1)-fold.
        int G = 1;
        while (G < 8 && 2 * G * K <= (int)blockDim.x) G *= 2;
        const int k = tid / G, j = tid % G;
        const float lof = (float)lo * (lo < 0 ? 1.0000002f : 0.9999998f) - 1e-30f;
        const float hif = (float)hi * (hi > 0 ? 1.0000002f : 0.9999998f) + 1e-30f;
        // Sampling round: thread t counts the eigenvalues below the point
        // lof + (t + 1) h0 (P = blockDim points); eigenvalue k then starts
        // from the gap between the last point counting <= k and the next,
        // P + 1 times narrower than the Gershgorin interval.
        const int P = (int)blockDim.x;
        const float h0 = (hif - lof) / (float)(P + 1);
        int* cnt = c.cnt;
        cnt[tid] = sturm_count_f32(n, c.df, c.e2f, lof + (float)(tid + 1) * h0, s_pivminf);
        __syncthreads();
        // Bracket tolerance, floored so that a zero matrix (nrm = 0) still
        // gives a finite round count; the count is also capped (64 rounds
        // narrow any float bracket below one ulp even for G = 1).
        const float atolf = fmaxf(2.0f * FLT_EPSILON * (float)nrm, 1e-30f);
        const float ratio = 2.f * h0 / atolf;
        int rounds = ratio > 1.0f ? (int)ceilf(log2f(ratio) / log2f((float)(G + 1))) + 1 : 1;
        rounds = rounds < 64 ? rounds : 64;
        if ((warp * 32) / G < K) {
            // Last sample index with count <= k (-1: none), by binary search
            // over the non-decreasing counts.
            int lo_i = -1, hi_i = P;
            while (hi_i - lo_i > 1) {
                const int mid = (lo_i + hi_i) >> 1;
                if (cnt[mid] <= k) lo_i = mid; else hi_i = mid;
            }
            float a = lo_i < 0 ? lof : lof + (float)(lo_i + 1) * h0;
            float b = hi_i >= P ? hif : lof + (float)(hi_i + 1) * h0;
            const unsigned gmask = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
            const int gshift = (lane / G) * G;
            for (int r = 0; r < rounds; ++r) {
                const float h = (b - a) / (float)(G + 1);
                bool flag = false;
                if (k < K) flag = sturm_count_f32(n, c.df, c.e2f, a + (float)(j + 1) * h, s_pivminf) <= k;
                const unsigned bal = __ballot_sync(FULL_MASK, flag);
                const int J = __popc((bal >> gshift) & gmask);
                const float na = J > 0 ? a + (float)J * h : a;
                const float nb = J < G ? a + (float)(J + 1) * h : b;
                a = na; b = nb;
            }
            if (k < K && j == 0) { c.lam[2 * k] = a; c.lam[2 * k + 1] = b; }
        }
        __syncthreads();
    }
    double sp = 0.0, fe = 0.0;
    const int k = tid;  // dense warps for the FP64 work
    if (k < K) {
        double lam;
        if constexpr (std::is_same<T, double>::value) {
            lam = eig_f64_bracketed(n, c.d, c.e2, k, c.lam[2 * k], c.lam[2 * k + 1], 8.0 * FLT_EPSILON * nrm, lo, hi,
                                    pivmin, nrm);
        } else if constexpr (std::is_same<T, dfl>::value) {
            lam = eig_df_bracketed(n, c.df, c.dlo, c.e2f, c.e2lo, k, c.lam[2 * k], c.lam[2 * k + 1],
                                   8.0 * FLT_EPSILON * nrm, lo, hi, s_pivminf, nrm);
        } else {
            lam = newton_polish_df(n, c.df, c.dlo, c.e2f, c.e2lo, c.lam[2 * k], c.lam[2 * k + 1],
                                   2.0f * FLT_EPSILON * (float)nrm, s_pivminf);
        }
        const double x = -(lam - mu) / temp;
        sp = softplus(x);
        fe = 1.0 / (1.0 + exp(-x));
        if (eig) eig[k] = lam;
    }
    __syncthreads();
    sum_sp = block_sum<double>(sp, c.red);
    sum_fermi = block_sum<double>(fe, c.red + NWP);
    n_solved = K;
}

// ---------------------------------------------------------------------------
__global__ void k_init_spins(Model m, double* __restrict__ S, int N);
__global__ void k_copy_sites(const double* __restrict__ src, double* __restrict__ dst,
                             const int32_t* __restrict__ sites, int count);
__global__ void k_free_energy(const double* __restrict__ eig, const int64_t* __restrict__ eoff,
                              const int32_t* __restrict__ n, int m, double mu, double temp,
                              double* __restrict__ F);
__global__ void k_observables(const double* __restrict__ S, int Lx, int Ly, const double* __restrict__ rec_Facc,
                              const double* __restrict__ rec_fill, const uint8_t* __restrict__ rec_acc,
                              const int32_t* __restrict__ rec_n, int N, double* __restrict__ out);

// Build m cluster matrices straight into global memory.
template <typename T>
__global__ void __launch_bounds__(CTA) k_build(Model m, const double* __restrict__ S, const int32_t* __restrict__ sites,
                                               int count, const double* __restrict__ new_spins, cplx_t<T>* H,
                                               int64_t stride, int64_t* offsets, int32_t* nout) {
    __shared__ double sp[3 * 256];  // window spins, up to 16x16 or 6x6x6 sites
    const int c = blockIdx.x;
    if (c >= count) return;
    const int site = sites[c];
    const Window w = make_window(m, site);
    cplx_t<T>* A = H + (int64_t)c * stride;
    build_cluster<T>(m, w, S, new_spins ? new_spins + 3 * c : nullptr, sp, A, m.e0);
    if (threadIdx.x == 0) { offsets[c] = (int64_t)c * stride; nout[c] = 2 * window_nsite(w); }
}

// All eigenvalues of m packed matrices from global memory.
template <typename T, int NT>
__global__ void __launch_bounds__(CTA, MinBlocks<T, NT>::value) k_eigvals(const cplx_t<T>* __restrict__ H, const int64_t* __restrict__ offsets,
                                                 const int32_t* __restrict__ nin, int count, int nA,
                                                 double* __restrict__ eig, const int64_t* __restrict__ eoff) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(nA, 32 * NT, sizeof(cplx_t<T>));
    Carve<T> c = carve<T>(smem, L);
    const int b = blockIdx.x;
    if (b >= count) return;
    const int n = nin[b];
    double* out = eig + eoff[b];
    if (n < 1 || n > nA || n > 32 * NT) {
        for (int i = threadIdx.x; i < (n > 0 ? n : 0) && i < nA; i += blockDim.x) out[i] = nan("");
        return;
    }
    const cplx_t<T>* src = H + offsets[b];
    const int P = tri(n);
    for (int i = threadIdx.x; i < P; i += blockDim.x) c.A[i] = src[i];
    __syncthreads();
    householder_tridiag<T, NT, NW>(n, c.A, c.hh, c.d, c.e2);
    double s1, s2;
    int K;
    tridiag_eig_F<T>(n, c, 0.0, 1.0, true, out, s1, s2, K);
}

struct StageArgs;

// Precision checker: both matrices of visits c0 .. c0+count-1 of a stage
// (item 2c: H_old of visit c0+c, item 2c+1: H_new with the proposed spin),
// built from the stage-start spins and solved as a sweep solves them, except
// that all n eigenvalues are returned: eig[(2c+var)*ld + k] ascending,
// F[2c+var] = -T sum_k softplus(-(eps_k-mu)/T).  k_check: precision T, matrix
// in shared memory, one item per CTA.  k_check_ref: FP64 with the matrix in
// the CTA's global slot (as the double-float re-solve), items grid-strided.
template <typename T, int NT>
__global__ void __launch_bounds__(CTA, MinBlocks<T, NT>::value) k_check(StageArgs a, int c0, int count, double* eig,
                                                                          int ld, double* F);
template <int NT>
__global__ void __launch_bounds__(CTA, 1) k_check_ref(StageArgs a, int c0, int count, double* eig, int ld, double* F);

// One PTCA stage (Sec. III.a): block 2c holds H_old of update site c, block
// 2c+1 holds H_new with the proposed spin.  The second block to finish
// applies Metropolis (Sec. II.c steps e-f) and writes the site's spin for the
// next stage.  Reads come only from S_in (the configuration at the start of
// the stage); S_out receives this stage's decisions plus the update sites it
// does not hold yet, copied forward from S_in (the previous stage's with two
// rotating spin buffers, the two previous stages' with three), so S_out is
// the full configuration after the stage.
struct StageArgs {
    Model m;
    const double* S_in;
    double* S_out;
    const int32_t* sites;
    const int32_t* perm;           // work index -> index in the stage's site list (null: identity)
    int32_t count;
    const int32_t* prev_sites;
    int32_t prev_count;
    const int32_t* prev2_sites;    // a second copied-forward range (overlapped pipeline), may be empty
    int32_t prev2_count;
    int32_t rec_base;
    int32_t nA;
    uint64_t sweep;
    double* Fbuf;
    double* fillbuf;
    int32_t* ticket;
    int32_t* rec_site;
    double* rec_Fold;
    double* rec_Fnew;
    double* rec_lnu;
    uint8_t* rec_acc;
    double* rec_Facc;
    double* rec_fill;
    int32_t* rec_n;
    unsigned long long* counters;  // [0] accepted, [1] eigensolves, [2] re-solves
    int32_t* err;
    // PTCA_MIXED decision guard: a decision with |ln u + dF/T| < margin is
    // deferred (its stage index appended to flag_list) and re-solved in FP64
    // with the matrix in global memory (gA, one slot of gA_stride elements
    // per CTA).  margin = 0 disables it.
    double margin;
    int32_t* flag_list;
    unsigned int* flag_count;
    double2* gA;
    int64_t gA_stride;
    // Large clusters (orders above the shared-memory kernels'): one global
    // packed matrix of gL_stride elements (float2 or double2) per CTA.
    void* gL;
    int64_t gL_stride;
    // Delayed acceptance: work list (perm) length on the device, and the
    // stage-1 surrogate dF~ per stage index (stage 2 accepts iff
    // ln u < -(dF - dF~)/T).  Null when screening is off.
    const unsigned int* count_dev;
    const float* sg_dFt;
    // Training-data collection: per visit (record index) the 150 network
    // inputs [P(s_old), s_new], the patch index of the update site and dF.
    float* sg_feat;
    int32_t* sg_center;
    float* sg_dF;
};

// The fields of StageArgs that change from stage to stage, passed by value so
// that the solve can read every invariant field straight from the kernel
// parameters.
struct StageVar {
    const double* S_in;
    double* S_out;
    const int32_t* sites;
    const int32_t* perm;
    int32_t rec_base;
    uint64_t sweep;
};

__device__ __forceinline__ StageVar stage_var(const StageArgs& a) {
    StageVar v;
    v.S_in = a.S_in; v.S_out = a.S_out; v.sites = a.sites; v.perm = a.perm; v.rec_base = a.rec_base; v.sweep = a.sweep;
    return v;
}

// Decision of an update site (thread 0 of the deciding CTA): Metropolis on
// dF, or delayed-acceptance stage 2 on dF - dF~, and the training sample.
__device__ __forceinline__ double stage2_dF(const StageArgs& a, int c, double dF) {
    return a.sg_dFt ? dF - (double)a.sg_dFt[c] : dF;
}

__device__ __forceinline__ void collect_sample(const StageArgs& a, const double* S_in, const Window& w, int r,
                                               const double* sn, double dF) {
    if (!a.sg_feat) return;
    float* f = a.sg_feat + (int64_t)r * SG_IN;
    a.sg_center[r] = patch_features(a.m, w, S_in, f);
    f[147] = (float)sn[0]; f[148] = (float)sn[1]; f[149] = (float)sn[2];
    a.sg_dF[r] = (float)dF;
}

// One matrix of one update site of a stage: c indexes the stage's site list,
// var 0/1 selects H_old/H_new.  The second of the pair to finish applies
// Metropolis.  Called by all threads of the CTA; s_new and s_last are shared.
//
// kTiled (FP32, 4 warps, orders up to 128): the matrix in the tiled layout and
// the register-tiled reduction (householder_tridiag_tiled).  kPanel = B > 1
// (FP32, 8 warps, orders up to 128): the blocked reduction in panels of B
// reflectors (householder_tridiag_panel), its panel vectors past the layout.
template <typename T, int NT, int NWP, bool kLarge = false, bool kTiled = false, int kPanel = 0>
__device__ __forceinline__ void stage_item(const StageArgs& a, const StageVar v, int c, int var, unsigned char* smem,
                                           double* s_new, int* s_last) {
    static_assert(!kTiled || (std::is_same<T, float>::value && NWP == TL_NW && 32 * NT <= TL_NMAX && !kLarge),
                  "the tiled reduction is FP32, 4 warps, orders up to 128");
    static_assert(kPanel <= 1 || (std::is_same<T, float>::value && NWP == PN_NW && NT <= 4 && !kLarge && !kTiled),
                  "the panel reduction is FP32, 8 warps, orders up to 128");
    const SmemLayout L = kTiled ? smem_layout_tiled() : smem_layout(kLarge ? 0 : a.nA, 32 * NT, sizeof(cplx_t<T>), NWP);
    Carve<T> cv = carve<T>(smem, L, NWP);
    if constexpr (kLarge) cv.A = static_cast<cplx_t<T>*>(a.gL) + (int64_t)blockIdx.x * a.gL_stride;
    c = v.perm ? v.perm[c] : c;
    const int site = v.sites[c];
    int n;
    {
        const Window w = make_window(a.m, site);
        n = 2 * window_nsite(w);
        if (threadIdx.x == 0 && var == 1)
            propose(a.m, v.sweep, (uint32_t)site, v.S_in + 3 * site, s_new);
        __syncthreads();
        build_cluster<T, kTiled>(a.m, w, v.S_in, var ? s_new : nullptr, cv.sp, cv.A);
    }
    __syncthreads();
    // The window's classical energy (Hubbard mean field), parked in this
    // matrix's F slot until the eigenvalues are known.
    if (threadIdx.x == 0 && a.m.cls_on) a.Fbuf[2 * c + var] = window_classical(a.m, cv.sp, n / 2);
    if constexpr (kTiled) {
        TlScratch ts;
        ts.Vb = cv.hh.Vb; ts.Wv = cv.hh.Wv; ts.pc = cv.hh.pc;
        ts.redA = cv.hh.redA; ts.redB = cv.hh.redB; ts.sx = cv.hh.sx;
        ts.d = reinterpret_cast<float*>(smem + L.d);
        ts.e2 = reinterpret_cast<float*>(smem + L.e2);
        householder_tridiag_tiled(n, cv.A, ts);
        // (d, e2) as doubles for the eigenvalue phase, in the matrix region
        cv.d = reinterpret_cast<double*>(smem + L.A);
        cv.e2 = cv.d + TL_NMAX;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            cv.d[i] = (double)ts.d[i];
            cv.e2[i] = i < n - 1 ? (double)ts.e2[i] : 0.0;
        }
        __syncthreads();
    } else if constexpr (kLarge) {
        householder_tridiag_large<T, NWP>(n, cv.A, cv.hh, cv.d, cv.e2);
    } else if constexpr (kPanel > 1) {
        float2* PV = reinterpret_cast<float2*>(smem + L.total);
        float2* PW = PV + kPanel * 32 * NT;
        float2* dotw = PW + kPanel * 32 * NT;
        householder_tridiag_panel<NT, kPanel>(n, cv.A, cv.hh, PV, PW, dotw, cv.d, cv.e2);
    } else {
        householder_tridiag<T, NT, NWP>(n, cv.A, cv.hh, cv.d, cv.e2);
    }
    double ssp, sfe;
    int K;
    tridiag_eig_F<T, NWP>(n, cv, a.m.mu - a.m.e0, a.m.T, false, nullptr, ssp, sfe, K);
    if (threadIdx.x == 0) {
        const double F = -a.m.T * ssp + (a.m.cls_on ? a.Fbuf[2 * c + var] : 0.0);
        a.Fbuf[2 * c + var] = F;
        a.fillbuf[2 * c + var] = sfe;
        __threadfence();
        const int old = atomicAdd(&a.ticket[c], 1);
        *s_last = (old == 1);
    }
    __syncthreads();
    if (!*s_last || threadIdx.x != 0) return;
    __threadfence();
    a.ticket[c] = 0;
    const double Fo = __ldcg(&a.Fbuf[2 * c]), Fn = __ldcg(&a.Fbuf[2 * c + 1]);
    const double fo = __ldcg(&a.fillbuf[2 * c]), fn = __ldcg(&a.fillbuf[2 * c + 1]);
    double sn[3];
    const double* so = v.S_in + 3 * site;
    if (var == 1) { sn[0] = s_new[0]; sn[1] = s_new[1]; sn[2] = s_new[2]; }
    else propose(a.m, v.sweep, (uint32_t)site, so, sn);
    double u0, u1;
    uniform2(a.m.seed, v.sweep, (uint32_t)site, RNG_ACCEPT, u0, u1);
    const double lnu = log(u0);
    const double dF = Fn - Fo;
    if (!isfinite(dF)) atomicExch(a.err, 1);
    const double dFe = stage2_dF(a, c, dF);
    if (a.margin > 0.0 && fabs(lnu + dFe / a.m.T) < a.margin) {
        a.flag_list[atomicAdd(a.flag_count, 1u)] = c;
        atomicAdd(&a.counters[2], 1ull);
        return;
    }
    const bool acc = lnu < -dFe / a.m.T;
    if (a.sg_feat) collect_sample(a, v.S_in, make_window(a.m, site), v.rec_base + c, sn, dF);
    double* dst = v.S_out + 3 * site;
    if (acc) { dst[0] = sn[0]; dst[1] = sn[1]; dst[2] = sn[2]; }
    else { dst[0] = so[0]; dst[1] = so[1]; dst[2] = so[2]; }
    const int r = v.rec_base + c;
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

template <typename T, int NT, int NWP = NW, bool kTiled = false, int kPanel = 0>
__global__ void __launch_bounds__(32 * NWP, MinBlocks<T, NT, NWP>::value) k_stage(StageArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    __shared__ int s_last;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.prev_count + a.prev2_count;
         k += gridDim.x * blockDim.x) {
        const int s = k < a.prev_count ? a.prev_sites[k] : a.prev2_sites[k - a.prev_count];
        a.S_out[3 * s] = a.S_in[3 * s];
        a.S_out[3 * s + 1] = a.S_in[3 * s + 1];
        a.S_out[3 * s + 2] = a.S_in[3 * s + 2];
    }
    const int c = blockIdx.x >> 1, var = blockIdx.x & 1;
    const int count = a.count_dev ? (int)*a.count_dev : a.count;
    if (c >= count) return;
    stage_item<T, NT, NWP, false, kTiled, kPanel>(a, stage_var(a), c, var, smem, s_new, &s_last);
}

template <typename T, int NT>
__global__ void __launch_bounds__(CTA, MinBlocks<T, NT>::value) k_check(StageArgs a, int c0, int count, double* eig,
                                                                          int ld, double* F) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    const int c = blockIdx.x >> 1, var = blockIdx.x & 1;
    if (c >= count) return;
    const SmemLayout L = smem_layout(a.nA, 32 * NT, sizeof(cplx_t<T>));
    Carve<T> cv = carve<T>(smem, L);
    const int site = a.sites[c0 + c];
    const Window w = make_window(a.m, site);
    const int n = 2 * window_nsite(w);
    if (threadIdx.x == 0 && var == 1)
        propose(a.m, a.sweep, (uint32_t)site, a.S_in + 3 * site, s_new);
    __syncthreads();
    build_cluster<T>(a.m, w, a.S_in, var ? s_new : nullptr, cv.sp, cv.A);
    __syncthreads();
    const double cls = threadIdx.x == 0 ? window_classical(a.m, cv.sp, n / 2) : 0.0;
    householder_tridiag<T, NT, NW>(n, cv.A, cv.hh, cv.d, cv.e2);
    double ssp, sfe;
    int K;
    tridiag_eig_F<T>(n, cv, a.m.mu - a.m.e0, a.m.T, true, eig + (int64_t)(2 * c + var) * ld, ssp, sfe, K);
    if (threadIdx.x == 0) F[2 * c + var] = -a.m.T * ssp + cls;
}

template <int NT>
__global__ void __launch_bounds__(CTA, 1) k_check_ref(StageArgs a, int c0, int count, double* eig, int ld, double* F) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    const SmemLayout L = smem_layout(0, 32 * NT, sizeof(double2));
    for (int item = blockIdx.x; item < 2 * count; item += gridDim.x) {
        Carve<double> cv = carve<double>(smem, L);
        cv.A = a.gA + (int64_t)blockIdx.x * a.gA_stride;
        const int c = item >> 1, var = item & 1;
        const int site = a.sites[c0 + c];
        const Window w = make_window(a.m, site);
        const int n = 2 * window_nsite(w);
        if (threadIdx.x == 0 && var == 1)
            propose(a.m, a.sweep, (uint32_t)site, a.S_in + 3 * site, s_new);
        __syncthreads();
        build_cluster<double>(a.m, w, a.S_in, var ? s_new : nullptr, cv.sp, cv.A);
        __syncthreads();
        const double cls = threadIdx.x == 0 ? window_classical(a.m, cv.sp, n / 2) : 0.0;
        householder_tridiag<double, NT, NW>(n, cv.A, cv.hh, cv.d, cv.e2);
        double ssp, sfe;
        int K;
        tridiag_eig_F<double>(n, cv, a.m.mu - a.m.e0, a.m.T, true, eig + (int64_t)(2 * c + var) * ld, ssp, sfe, K);
        if (threadIdx.x == 0) F[2 * c + var] = -a.m.T * ssp + cls;
        __syncthreads();
    }
}

// Re-solve of one matrix of a deferred update site (stage index c from the
// flag list) at FP64-class precision: the matrix is built and reduced in
// double-float arithmetic (about 48 significant bits on the FP32 pipe), the
// eigenvalues of the resulting tridiagonal run in FP64, and the second of the
// pair decides (no margin test).  The matrix lives in shared memory when
// kSmemA (a.nA up to about 150 fits beside the vectors in one CTA), else in
// this CTA's global slot; the arithmetic is the same either way.  nmaxc =
// 32 * NT sizes the vectors in shared memory.
template <int NT, int NWP = NW, bool kSmemA = false, bool kLarge = false>
__device__ __noinline__ void resolve_item(const StageArgs& a, const StageVar v, int c, int var, unsigned char* smem,
                                          double* s_new, int* s_last) {
    const SmemLayout L = smem_layout(kSmemA ? a.nA : 0, 32 * NT, sizeof(dfl2), NWP);
    Carve<dfl> cv = carve<dfl>(smem, L, NWP);
    if constexpr (!kSmemA) cv.A = reinterpret_cast<dfl2*>(a.gA + (int64_t)blockIdx.x * a.gA_stride);
    const int site = v.sites[c];
    int n;
    {
        const Window w = make_window(a.m, site);
        n = 2 * window_nsite(w);
        if (threadIdx.x == 0 && var == 1)
            propose(a.m, v.sweep, (uint32_t)site, v.S_in + 3 * site, s_new);
        __syncthreads();
        build_cluster<dfl>(a.m, w, v.S_in, var ? s_new : nullptr, cv.sp, cv.A);
    }
    __syncthreads();
    if (threadIdx.x == 0 && a.m.cls_on) a.Fbuf[2 * c + var] = window_classical(a.m, cv.sp, n / 2);
    if constexpr (kLarge) householder_tridiag_large<dfl, NWP>(n, cv.A, cv.hh, cv.d, cv.e2);
    else householder_tridiag<dfl, NT, NWP>(n, cv.A, cv.hh, cv.d, cv.e2);
    double ssp, sfe;
    int K;
    tridiag_eig_F<dfl, NWP>(n, cv, a.m.mu - a.m.e0, a.m.T, false, nullptr, ssp, sfe, K);
    if (threadIdx.x == 0) {
        a.Fbuf[2 * c + var] = -a.m.T * ssp + (a.m.cls_on ? a.Fbuf[2 * c + var] : 0.0);
        a.fillbuf[2 * c + var] = sfe;
        __threadfence();
        *s_last = (atomicAdd(&a.ticket[c], 1) == 1);
    }
    __syncthreads();
    if (!*s_last || threadIdx.x != 0) return;
    __threadfence();
    a.ticket[c] = 0;
    const double Fo = __ldcg(&a.Fbuf[2 * c]), Fn = __ldcg(&a.Fbuf[2 * c + 1]);
    const double fo = __ldcg(&a.fillbuf[2 * c]), fn = __ldcg(&a.fillbuf[2 * c + 1]);
    double sn[3];
    const double* so = v.S_in + 3 * site;
    if (var == 1) { sn[0] = s_new[0]; sn[1] = s_new[1]; sn[2] = s_new[2]; }
    else propose(a.m, v.sweep, (uint32_t)site, so, sn);
    double u0, u1;
    uniform2(a.m.seed, v.sweep, (uint32_t)site, RNG_ACCEPT, u0, u1);
    const double lnu = log(u0);
    const double dF = Fn - Fo;
    if (!isfinite(dF)) atomicExch(a.err, 1);
    const bool acc = lnu < -stage2_dF(a, c, dF) / a.m.T;
    if (a.sg_feat) collect_sample(a, v.S_in, make_window(a.m, site), v.rec_base + c, sn, dF);
    double* dst = v.S_out + 3 * site;
    if (acc) { dst[0] = sn[0]; dst[1] = sn[1]; dst[2] = sn[2]; }
    else { dst[0] = so[0]; dst[1] = so[1]; dst[2] = so[2]; }
    const int r = v.rec_base + c;
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

// Re-solve the deferred update sites of one stage (per-stage pipelines), one
// CTA of RESOLVE_NW warps per matrix, the matrix in shared memory when
// kSmemA.  The same width as the persistent kernel's inline re-solve, so all
// pipelines produce bit-identical results.  16 warps were measured slower:
// the pass gains less than the scalar phases lose to the wider barriers and
// to spills at 128 registers.
constexpr int RESOLVE_NW = 8;
template <int NT, bool kSmemA>
__global__ void __launch_bounds__(32 * RESOLVE_NW, 1) k_resolve(StageArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    __shared__ int s_last;
    const int nflag = (int)*(volatile unsigned int*)a.flag_count;
    for (int item = blockIdx.x; item < 2 * nflag; item += gridDim.x) {
        const int c = a.flag_list[item >> 1];
        resolve_item<NT, RESOLVE_NW, kSmemA>(a, stage_var(a), c, item & 1, smem, s_new, &s_last);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Large traveling clusters (the paper's N_c = 12^2 and 16^2, orders up to
// 32 NW_LARGE = 512): one CTA of NW_LARGE warps per matrix, the matrix in the
// CTA's global slot (householder_tridiag_large), the vectors and the
// eigenvalue stage in shared memory.  A grid of resident CTAs strides over
// the (site, old/new) items, so that each CTA owns one slot.  Same stage
// semantics, decisions and records as k_stage.
// ---------------------------------------------------------------------------
constexpr int NW_LARGE = 16;
template <typename T>
__global__ void __launch_bounds__(32 * NW_LARGE, 1) k_stage_large(StageArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    __shared__ int s_last;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.prev_count + a.prev2_count;
         k += gridDim.x * blockDim.x) {
        const int s = k < a.prev_count ? a.prev_sites[k] : a.prev2_sites[k - a.prev_count];
        a.S_out[3 * s] = a.S_in[3 * s];
        a.S_out[3 * s + 1] = a.S_in[3 * s + 1];
        a.S_out[3 * s + 2] = a.S_in[3 * s + 2];
    }
    for (int item = blockIdx.x; item < 2 * a.count; item += gridDim.x) {
        stage_item<T, NW_LARGE, NW_LARGE, true>(a, stage_var(a), item >> 1, item & 1, smem, s_new, &s_last);
        __syncthreads();
    }
}

// Double-float re-solve of a stage's deferred large-cluster decisions (matrix
// in the CTA's global re-solve slot).
template <int NWL = NW_LARGE>
__global__ void __launch_bounds__(32 * NWL, 1) k_resolve_large(StageArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    __shared__ int s_last;
    const int nflag = (int)*(volatile unsigned int*)a.flag_count;
    for (int item = blockIdx.x; item < 2 * nflag; item += gridDim.x) {
        const int c = a.flag_list[item >> 1];
        resolve_item<NWL, NWL, false, true>(a, stage_var(a), c, item & 1, smem, s_new, &s_last);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Persistent sweep: one launch runs every stage of n_sweeps sweeps.  Each CTA
// takes (site, old/new) items of the current stage from an atomic work queue
// (sites ordered largest window first), then all CTAs meet at a device-wide
// barrier before the next stage reads the spins the stage wrote.  Every wait
// at the barrier is bounded: past the time limit the CTA records
// PTCA_ERR_TIMEOUT in err[1] and returns, so a missing participant cannot
// hang the GPU.
// ---------------------------------------------------------------------------
struct PersistArgs {
    StageArgs st;                 // model, scratch, records (per-stage fields set in the kernel)
    double* S0;
    double* S1;
    const int32_t* sites;         // flattened schedule, each stage in work order
    const int32_t* stage_start;   // nstages + 1
    int32_t nstages;
    int32_t n_sweeps;
    unsigned long long* sweep_ctr;// RNG sweep index of the next sweep (advanced by the kernel)
    unsigned int* queue;          // [0..1] work-queue counters alternating by stage, [2] re-solve queue
    unsigned int* bar;            // [0] arrivals, [1] generation
    unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Device-wide barrier over gridDim.x CTAs (all co-resident).  Returns false
// (and sets err[1] = PTCA_ERR_TIMEOUT) if the wait exceeds timeout_ns.  The
// last CTA to arrive also clears `clear_after` (a queue counter nobody uses
// until two stages later).
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int participants, unsigned long long timeout_ns,
                                             int32_t* err, unsigned int* clear_after, unsigned int* clear_after2 = nullptr) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = bar + 1;
        const unsigned int my_gen = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(bar, 1u);
        int ok = 1;
        if (arrived == participants - 1) {
            if (clear_after) *clear_after = 0u;
            if (clear_after2) *clear_after2 = 0u;
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned long long spins = 0;
            while (*gen == my_gen) {
                if (((++spins) & 63u) == 0 && (global_ns() - t0 > timeout_ns || spins > (1ull << 34))) {
                    atomicExch(err + 1, 4);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Body of the persistent kernels: shared-memory matrices (k_sweep_persistent)
// or, with kLarge, each CTA's global slot (k_sweep_persistent_large).
template <typename T, int NT, int NWP, bool kLarge>
__device__ __forceinline__ void persistent_body(const PersistArgs& p, unsigned char* smem, double* s_new, int& s_last,
                                                int& s_item) {
    const StageArgs& a = p.st;  // invariant fields, read from the kernel parameters
    const unsigned long long sweep0 = *p.sweep_ctr;
    const int G = p.nstages * p.n_sweeps;
    for (int g = 0; g < G; ++g) {
        const int s = g % p.nstages;
        const int sp = (g > 0) ? (g - 1) % p.nstages : -1;
        StageVar v;
        v.sweep = sweep0 + (unsigned long long)(g / p.nstages);
        v.S_in = (g & 1) ? p.S1 : p.S0;
        v.S_out = (g & 1) ? p.S0 : p.S1;
        v.sites = p.sites + p.stage_start[s];
        v.perm = a.perm ? a.perm + p.stage_start[s] : nullptr;
        v.rec_base = p.stage_start[s];
        const int count = p.stage_start[s + 1] - p.stage_start[s];
        if (sp >= 0) {
            const int32_t* prev = p.sites + p.stage_start[sp];
            const int pc = p.stage_start[sp + 1] - p.stage_start[sp];
            for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pc; k += gridDim.x * blockDim.x) {
                const int q = prev[k];
                v.S_out[3 * q] = v.S_in[3 * q];
                v.S_out[3 * q + 1] = v.S_in[3 * q + 1];
                v.S_out[3 * q + 2] = v.S_in[3 * q + 2];
            }
        }
        unsigned int* qc = p.queue + (g & 1);
        for (;;) {
            if (threadIdx.x == 0) s_item = (int)atomicAdd(qc, 1u);
            __syncthreads();
            const int item = s_item;
            __syncthreads();
            if (item >= 2 * count) break;
            stage_item<T, NT, NWP, kLarge>(a, v, item >> 1, item & 1, smem, s_new, &s_last);
            __syncthreads();
        }
        if (!grid_barrier(p.bar, gridDim.x, p.timeout_ns, a.err, qc)) return;
        if constexpr (sizeof(T) == 4) {
            // Deferred decisions of this stage (PTCA_MIXED margin guard).
            const int nflag = a.margin > 0.0 ? (int)*(volatile unsigned int*)a.flag_count : 0;
            if (nflag > 0) {
                for (;;) {
                    if (threadIdx.x == 0) s_item = (int)atomicAdd(p.queue + 2, 1u);
                    __syncthreads();
                    const int item = s_item;
                    __syncthreads();
                    if (item >= 2 * nflag) break;
                    resolve_item<NT, NWP, false, kLarge>(a, v, a.flag_list[item >> 1], item & 1, smem, s_new, &s_last);
                    __syncthreads();
                }
                if (!grid_barrier(p.bar, gridDim.x, p.timeout_ns, a.err, p.queue + 2, a.flag_count)) return;
            }
        }
    }
    if (G > 0) {
        // Bring the other buffer up to date with the last stage.
        const int sl = (G - 1) % p.nstages;
        const double* src = (G & 1) ? p.S1 : p.S0;
        double* dst = (G & 1) ? p.S0 : p.S1;
        const int32_t* last = p.sites + p.stage_start[sl];
        const int lc = p.stage_start[sl + 1] - p.stage_start[sl];
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < lc; k += gridDim.x * blockDim.x) {
            const int q = last[k];
            dst[3 * q] = src[3 * q]; dst[3 * q + 1] = src[3 * q + 1]; dst[3 * q + 2] = src[3 * q + 2];
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) *p.sweep_ctr = sweep0 + (unsigned long long)p.n_sweeps;
    }
}

template <typename T, int NT, int NWP = NW>
__global__ void __launch_bounds__(32 * NWP, MinBlocks<T, NT, NWP>::value)
    k_sweep_persistent(const __grid_constant__ PersistArgs p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    __shared__ int s_last, s_item;
    persistent_body<T, NT, NWP, false>(p, smem, s_new, s_last, s_item);
}

// Large clusters: the persistent pipeline with 16-warp CTAs and the matrix
// in each CTA's global slot (a.gL; re-solves in a.gA), grid <= the slots.
template <typename T>
__global__ void __launch_bounds__(32 * NW_LARGE, 1) k_sweep_persistent_large(const __grid_constant__ PersistArgs p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    __shared__ int s_last, s_item;
    persistent_body<T, NW_LARGE, NW_LARGE, true>(p, smem, s_new, s_last, s_item);
}

// Precision checker for large clusters: as k_check (T = float, the sweep's
// FP32 reduction, slots a.gL) and k_check_ref (T = double, FP64, the re-solve
// slots a.gA), one 16-warp CTA per item over a grid stride, the matrix in
// the CTA's global slot and all n eigenvalues returned.
template <typename T>
__global__ void __launch_bounds__(32 * NW_LARGE, 1) k_check_large(StageArgs a, int c0, int count, double* eig, int ld,
                                                                  double* F) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    const SmemLayout L = smem_layout(0, 32 * NW_LARGE, sizeof(cplx_t<T>), NW_LARGE);
    for (int item = blockIdx.x; item < 2 * count; item += gridDim.x) {
        Carve<T> cv = carve<T>(smem, L, NW_LARGE);
        if constexpr (sizeof(T) == 4) cv.A = static_cast<cplx_t<T>*>(a.gL) + (int64_t)blockIdx.x * a.gL_stride;
        else cv.A = a.gA + (int64_t)blockIdx.x * a.gA_stride;
        const int c = item >> 1, var = item & 1;
        const int site = a.sites[c0 + c];
        const Window w = make_window(a.m, site);
        const int n = 2 * window_nsite(w);
        if (threadIdx.x == 0 && var == 1) propose(a.m, a.sweep, (uint32_t)site, a.S_in + 3 * site, s_new);
        __syncthreads();
        build_cluster<T>(a.m, w, a.S_in, var ? s_new : nullptr, cv.sp, cv.A);
        __syncthreads();
        const double cls = threadIdx.x == 0 ? window_classical(a.m, cv.sp, n / 2) : 0.0;
        householder_tridiag_large<T, NW_LARGE>(n, cv.A, cv.hh, cv.d, cv.e2);
        double ssp, sfe;
        int K;
        tridiag_eig_F<T, NW_LARGE>(n, cv, a.m.mu - a.m.e0, a.m.T, true, eig + (int64_t)(2 * c + var) * ld, ssp, sfe,
                                   K);
        if (threadIdx.x == 0) F[2 * c + var] = -a.m.T * ssp + cls;
        __syncthreads();
    }
}

// All eigenvalues of packed matrices of large orders (up to 32 NW_LARGE), one
// 16-warp CTA per matrix over a grid stride: the matrix is copied into the
// CTA's slot (slots + blockIdx.x * stride) and reduced there.
template <typename T>
__global__ void __launch_bounds__(32 * NW_LARGE, 1) k_eigvals_large(const cplx_t<T>* __restrict__ H,
                                                                    const int64_t* __restrict__ offsets,
                                                                    const int32_t* __restrict__ nin, int count, int nA,
                                                                    double* __restrict__ eig,
                                                                    const int64_t* __restrict__ eoff, cplx_t<T>* slots,
                                                                    int64_t stride) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout(0, 32 * NW_LARGE, sizeof(cplx_t<T>), NW_LARGE);
    for (int b = blockIdx.x; b < count; b += gridDim.x) {
        Carve<T> c = carve<T>(smem, L, NW_LARGE);
        c.A = slots + (int64_t)blockIdx.x * stride;
        const int n = nin[b];
        double* out = eig + eoff[b];
        if (n < 1 || n > nA || n > 32 * NW_LARGE) {
            for (int i = threadIdx.x; i < (n > 0 ? n : 0) && i < nA; i += blockDim.x) out[i] = nan("");
            __syncthreads();
            continue;
        }
        const cplx_t<T>* src = H + offsets[b];
        const int P = tri(n);
        for (int i = threadIdx.x; i < P; i += blockDim.x) c.A[i] = src[i];
        __syncthreads();
        householder_tridiag_large<T, NW_LARGE>(n, c.A, c.hh, c.d, c.e2);
        double s1, s2;
        int K;
        tridiag_eig_F<T, NW_LARGE>(n, c, 0.0, 1.0, true, out, s1, s2, K);
        __syncthreads();
    }
}

// Barrier self-test: `blocks` CTAs wait for `blocks + 1` participants, which
// never arrive; every CTA must give up after timeout_ns and report it.
__global__ void k_barrier_selftest(unsigned int* bar, int32_t* err, unsigned long long timeout_ns);

}  // namespace ptca
