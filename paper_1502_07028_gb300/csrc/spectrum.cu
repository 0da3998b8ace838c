// spectrum.cu -- full-system spectrum of a configuration (Sec. VI): all 2N
// eigenvalues of the whole lattice's one-body Hamiltonian, where the paper
// diagonalises saved configurations with ScaLAPACK.  Everything runs in this
// library's kernels, off the sweep's hot path (step 2 in FP64 for FP64
// contexts and in double-float on the FP32 pipe for PTCA_MIXED contexts):
//   1. the dense matrix is built as its packed lower triangle (row-major:
//      element (i, j <= i) at i(i+1)/2 + j) in global memory;
//   2. a Householder reduction to real tridiagonal form spread over the whole
//      GPU: per reflector, one tiled pass applies the previous reflector's
//      deferred rank-2 update to the trailing block and accumulates the
//      Hermitian matrix-vector product with the current reflector (row and
//      column partial sums per 64 x 64 tile, in a fixed order), a reduction
//      combines the partials, and one CTA forms w, the explicit update of the
//      next pivot column and the next reflector -- the algorithm of the
//      cluster kernels (cluster_solve.cuh), with the matrix too large for one
//      SM;
//   3. one thread per eigenvalue: FP32 bisection on the FP32-rounded
//      tridiagonal, then the cluster solver's double-float Sturm counts and
//      safeguarded Newton on the exact (FP64) tridiagonal.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/ptca.h"
#include "context.h"
#include "kernels.cuh"
#include "launch.h"

namespace ptca {

__host__ __device__ __forceinline__ int64_t tri64(int64_t r) { return r * (r + 1) / 2; }

constexpr int FS_TB = 64;          // tile edge of the reduction pass
constexpr int FS_PASS_THREADS = 256;
constexpr int FS_RED_THREADS = 256;  // 8 warps; each CTA sums the partials of FS_RED_ROWS rows
constexpr int FS_RED_ROWS = 32;
constexpr int FS_SCALAR_THREADS = 1024;
constexpr int FS_EIG_THREADS = 128;

// One thread per lattice site: its on-site 2x2 block and its bonds to the
// +x, +y, +z neighbours, hopping added atomically so that an axis of extent 2
// on a torus gets both of its bonds (-2t).  H: packed lower triangle of order
// 2N, zeroed by the caller.
__global__ void k_full_hamiltonian(Model m, const double* __restrict__ S, int N, double2* __restrict__ H) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int x = i % m.Lx, y = (i / m.Lx) % m.Ly, z = i / (m.Lx * m.Ly);
    const double sx = S[3 * i], sy = S[3 * i + 1], sz = S[3 * i + 2];
    const double dg = m.e0 + m.lam * sx, J = m.JH;
    const int64_t a = 2 * (int64_t)i, b = a + 1;
    H[tri64(a) + a] = make_double2(dg - J * sz, 0.0);
    H[tri64(b) + b] = make_double2(dg + J * sz, 0.0);
    H[tri64(b) + a] = make_double2(-J * sx, -J * sy);  // element (b, a) = -J (S_x + i S_y)
    const int L[3] = {m.Lx, m.Ly, m.Lz};
    const int c[3] = {x, y, z};
    for (int d = 0; d < 3; ++d) {
        if (L[d] == 1) continue;
        int cc[3] = {c[0], c[1], c[2]};
        cc[d] += 1;
        if (cc[d] == L[d]) {
            if (!m.lattice_periodic) continue;
            cc[d] = 0;
        }
        const int j = (cc[2] * m.Ly + cc[1]) * m.Lx + cc[0];
        for (int sg = 0; sg < 2; ++sg) {
            const int64_t p = 2 * (int64_t)i + sg, q = 2 * (int64_t)j + sg;
            const int64_t hi = p > q ? p : q, lo = p > q ? q : p;
            atomicAdd(&H[tri64(hi) + lo].x, -m.t);
        }
    }
}

// The reduction runs in the real arithmetic R: double, or dfl (double-float:
// about 48 significant bits on the FP32 pipe, which runs 64 times the FP64
// rate).  A complex entry takes 16 bytes and a real one 8 in either, so the
// buffers are the same.
__device__ __forceinline__ double fs_d(double x) { return x; }
__device__ __forceinline__ double fs_d(dfl x) { return (double)x; }
template <typename R> __device__ __forceinline__ R fs_r(float x);
template <> __device__ __forceinline__ double fs_r<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ dfl fs_r<dfl>(float x) { return dfl(x, 0.f); }

// The built FP64 matrix rewritten in place as double-float pairs.
__global__ void k_fs_to_dfl(double2* A, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 x = A[i];
        reinterpret_cast<dfl2*>(A)[i] = mk(dfl(x.x), dfl(x.y));
    }
}

// Buffers of the reduction.  Reflector k acts on rows/columns k+1 .. n-1;
// its first entry is stored at index k+1 like the others.
template <typename R>
struct FsArgs {
    using C = cplx_t<R>;
    int n;
    C* A;
    const C* U;   // v_{k-1} (zero at k = 0)
    const C* V;   // v_k
    C* Vn;        // v_{k+1}, written by the scalar phase of step k
    const C* W;   // w_{k-1} (zero at k = 0)
    C* Wn;        // w_k, written by the scalar phase of step k
    C* pr;        // [T][n] row partial sums of A v_k, by tile column
    C* pc;        // [T][n] column partial sums, by tile row
    C* p;         // [n]    tau A v_k
    R* red;       // [blocks of the reduction] partial sums of Re(v^H p)
    R* tau;       // [2]    tau_k in tau[k & 1]
    double* d;    // [n]
    double* e2;   // [n]
};

// Step k's pass over the trailing block (rows and columns j0 = k+1 .. n-1),
// one 64 x 64 tile of its lower triangle per CTA: A <- A - u w^H - w u^H
// with step k-1's (u, w), then the tile's row sums of A v (into pr[tile
// column][row]) and, below the diagonal, column sums of A^H v (into
// pc[tile row][column]).  Warp q takes rows q, q+8, ...; lanes take columns
// lane and lane + 32 of the tile.  The tile's row entries of u, w and v are
// staged in shared memory, and a warp loads its next row's elements before
// it updates the current one (the pass is bound by instruction issue once
// the loads are in flight early).  Each lane's row partials go to shared
// memory and four threads per row add them up (eight each, then across the
// four), in a fixed order.
constexpr int FS_RS_LD = 33;  // row stride of the row partials (16-byte entries)
template <typename R>
__global__ void __launch_bounds__(FS_PASS_THREADS, 3) k_fs_pass(FsArgs<R> a, int k) {
    using C = cplx_t<R>;
    __shared__ C rsum[FS_TB][FS_RS_LD];
    __shared__ C csum[FS_PASS_THREADS / 32][FS_TB];
    __shared__ C svec[3][FS_TB];
    const int n = a.n, j0 = k + 1, m = n - j0;
    const int64_t b = blockIdx.x;
    int TR = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);  // corrected below
    while (tri64(TR + 1) <= b) ++TR;
    while (tri64(TR) > b) --TR;
    const int TC = (int)(b - tri64(TR));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const R r0 = fs_r<R>(0.f);
    const C zero = mk(r0, r0);
    int cr[2];
    C vc[2], uc[2], wc[2], cacc[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        cr[q] = FS_TB * TC + lane + 32 * q;
        const bool in = cr[q] < m;
        const int j = j0 + cr[q];
        vc[q] = in ? a.V[j] : zero;
        uc[q] = in ? a.U[j] : zero;
        wc[q] = in ? a.W[j] : zero;
        cacc[q] = zero;
    }
    // the tile's row entries of u, w and v, staged once
    for (int t = threadIdx.x; t < 3 * FS_TB; t += FS_PASS_THREADS) {
        const int r = t % FS_TB, ri = FS_TB * TR + r;
        const C* src = t < FS_TB ? a.U : (t < 2 * FS_TB ? a.W : a.V);
        svec[t / FS_TB][r] = ri < m ? src[j0 + ri] : zero;
    }
    __syncthreads();
    // the next row's elements are loaded before the current row is updated
    C xa[2], xb[2] = {zero, zero};
    {
        const int ri = FS_TB * TR + warp;
        const C* row = a.A + tri64(j0 + ri) + j0;
#pragma unroll
        for (int q = 0; q < 2; ++q) xa[q] = (ri < m && cr[q] <= ri) ? row[cr[q]] : zero;
    }
    for (int rr = warp; rr < FS_TB; rr += FS_PASS_THREADS / 32) {
        const int ri = FS_TB * TR + rr;
        if (ri >= m) break;
        const int rn = ri + FS_PASS_THREADS / 32;
        if (rr + FS_PASS_THREADS / 32 < FS_TB && rn < m) {
            const C* rown = a.A + tri64(j0 + rn) + j0;
#pragma unroll
            for (int q = 0; q < 2; ++q) xb[q] = cr[q] <= rn ? rown[cr[q]] : zero;
        }
        const C ui = svec[0][rr], wi = svec[1][rr], vi = svec[2][rr];
        C* row = a.A + tri64(j0 + ri) + j0;
        C racc = zero;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c = cr[q];
            if (c <= ri) {
                C x = xa[q];
                x = cfms_conj_b(ui, wc[q], x);
                x = cfms_conj_b(wi, uc[q], x);
                if (c == ri) x.y = r0;  // the diagonal stays real
                row[c] = x;
                racc = cfma(x, vc[q], racc);
                if (c < ri) cacc[q] = cfma_conj_a(x, vi, cacc[q]);
            }
            xa[q] = xb[q];
        }
        rsum[rr][lane] = racc;
    }
    csum[warp][lane] = cacc[0];
    csum[warp][lane + 32] = cacc[1];
    __syncthreads();
    {
        const int rr = threadIdx.x >> 2, part = threadIdx.x & 3, ri = FS_TB * TR + rr;
        C sum = zero;
        if (ri < m) {
            sum = rsum[rr][part];
#pragma unroll
            for (int j = 1; j < 8; ++j) sum = cadd(sum, rsum[rr][part + 4 * j]);
        }
        sum = cadd(sum, cshfl_xor(sum, 1));
        sum = cadd(sum, cshfl_xor(sum, 2));
        if (part == 0 && ri < m) a.pr[(int64_t)TC * n + ri] = sum;
    }
    if (threadIdx.x < FS_TB) {
        C sum = csum[0][threadIdx.x];
#pragma unroll
        for (int w = 1; w < FS_PASS_THREADS / 32; ++w) sum = cadd(sum, csum[w][threadIdx.x]);
        const int c = FS_TB * TC + threadIdx.x;
        if (c < m) a.pc[(int64_t)TR * n + c] = sum;
    }
}

// p = tau (A v): for row ri of band B (its tile row), the row partials of
// tiles (B, 0 .. B) plus the column partials of tiles (B .. T-1, B) (the
// diagonal tile's column sums hold the elements below the diagonal); and
// each CTA's partial sum of Re(v^H p).  A CTA takes 32 consecutive rows, one
// per lane; warp q adds the partials q, q+8, ... of that list, and warp 0
// adds the eight warps' sums, in a fixed order.
template <typename R>
__global__ void __launch_bounds__(FS_RED_THREADS) k_fs_reduce(FsArgs<R> a, int k) {
    using C = cplx_t<R>;
    __shared__ C part[FS_RED_THREADS / 32][FS_RED_ROWS];
    const int n = a.n, j0 = k + 1, m = n - j0, T = (m + FS_TB - 1) / FS_TB;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ri = blockIdx.x * FS_RED_ROWS + lane;
    const R r0 = fs_r<R>(0.f);
    C s = mk(r0, r0);
    if (ri < m) {
        const int band = ri / FS_TB;
        for (int q = warp; q <= T; q += FS_RED_THREADS / 32)
            s = cadd(s, q <= band ? a.pr[(int64_t)q * n + ri] : a.pc[(int64_t)(q - 1) * n + ri]);
    }
    part[warp][lane] = s;
    __syncthreads();
    if (warp != 0) return;
#pragma unroll
    for (int w = 1; w < FS_RED_THREADS / 32; ++w) s = cadd(s, part[w][lane]);
    R sp = r0;
    if (ri < m) {
        const R tau = a.tau[k & 1];
        s.x = s.x * tau;
        s.y = s.y * tau;
        a.p[j0 + ri] = s;
        const C v = a.V[j0 + ri];
        sp = v.x * s.x + v.y * s.y;
    }
    sp = warp_sum<R>(sp);
    if (lane == 0) a.red[blockIdx.x] = sp;
}

// Sum over the FS_SCALAR_THREADS threads of a scalar-phase CTA; every thread
// receives the same value (each warp's butterfly, then a butterfly over the
// 32 warp sums).  `red` holds 32 entries and is not read by another
// reduction until a later __syncthreads.
static_assert(FS_SCALAR_THREADS == 32 * 32, "fs_block_sum adds one value per warp in one warp");
template <typename R> __device__ __forceinline__ R fs_block_sum(R v, R* red) {
    v = warp_sum<R>(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    return warp_sum<R>(red[threadIdx.x & 31]);
}

// Column 0: d_0, ||x||^2 and the first reflector (one CTA).
template <typename R>
__global__ void __launch_bounds__(FS_SCALAR_THREADS) k_fs_setup(FsArgs<R> a) {
    using C = cplx_t<R>;
    __shared__ R red[FS_SCALAR_THREADS / 32];
    __shared__ C s_x0;
    const int n = a.n;
    R s2 = fs_r<R>(0.f);
    for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
        const C x = a.A[tri64(i)];
        s2 = s2 + cabs2(x);
        if (i >= 2) a.Vn[i] = x;
        if (i == 1) s_x0 = x;
    }
    s2 = fs_block_sum<R>(s2, red);
    if (threadIdx.x == 0) {
        a.d[0] = fs_d(a.A[0].x);
        a.e2[0] = fs_d(s2);
        C f;
        R tau;
        reflector_head<R>(s2, s_x0, f, tau);
        a.Vn[1] = f;
        a.tau[0] = tau;
    }
}

// Step k's scalar phase (one CTA): w = p - (tau/2)(v^H p) v; the explicit
// update of pivot column j0 = k+1 with (v_k, w_k); d_j0, e2_j0 and, unless
// this was the last reflector, the next reflector v_{k+1} and tau_{k+1}.
template <typename R>
__global__ void __launch_bounds__(FS_SCALAR_THREADS) k_fs_scalar(FsArgs<R> a, int k, int nred) {
    using C = cplx_t<R>;
    __shared__ R red[FS_SCALAR_THREADS / 32];
    __shared__ R s_K;
    __shared__ C s_x0;
    const int n = a.n, j0 = k + 1;
    R sp = fs_r<R>(0.f);
    for (int b = threadIdx.x; b < nred; b += blockDim.x) sp = sp + a.red[b];
    sp = fs_block_sum<R>(sp, red);
    if (threadIdx.x == 0) s_K = fs_r<R>(0.5f) * a.tau[k & 1] * sp;
    __syncthreads();
    const R K = s_K;
    const C vf = a.V[j0];
    const C p0 = a.p[j0];
    const C w0 = mk(p0.x - K * vf.x, p0.y - K * vf.y);
    R s2 = fs_r<R>(0.f);
    for (int i = j0 + threadIdx.x; i < n; i += blockDim.x) {
        const C v = a.V[i], pi = a.p[i];
        const C w = mk(pi.x - K * v.x, pi.y - K * v.y);
        a.Wn[i] = w;
        C x = a.A[tri64(i) + j0];
        x = cfms_conj_b(v, w0, x);
        x = cfms_conj_b(w, vf, x);
        if (i == j0) a.d[j0] = fs_d(x.x);
        if (i >= j0 + 1) s2 = s2 + cabs2(x);
        if (i >= j0 + 2) a.Vn[i] = x;
        if (i == j0 + 1) s_x0 = x;
    }
    s2 = fs_block_sum<R>(s2, red);
    if (threadIdx.x == 0) {
        a.e2[j0] = fs_d(s2);
        if (k + 1 <= n - 3) {
            C f;
            R tau;
            reflector_head<R>(s2, s_x0, f, tau);
            a.Vn[j0 + 1] = f;
            a.tau[(k + 1) & 1] = tau;
        }
    }
}

// The last diagonal entry: step n-3's update of A_{n-1,n-1} (V = v_{n-3},
// W = w_{n-3}).
template <typename R>
__global__ void k_fs_finish(FsArgs<R> a) {
    const int n = a.n;
    const auto v = a.V[n - 1], w = a.W[n - 1];
    a.d[n - 1] = fs_d(a.A[tri64(n - 1) + n - 1].x - fs_r<R>(2.f) * (v.x * w.x + v.y * w.y));
}

// Gershgorin bracket and Sturm-count guards of the tridiagonal (d, e2), and
// its float pairs (hi + lo = the FP64 entries exactly).  One CTA.
// prm: [0] lo, [1] hi, [2] pivmin (float), [3] nrm.
__global__ void __launch_bounds__(FS_SCALAR_THREADS) k_fs_eig_prep(int n, const double* __restrict__ d,
                                                                  const double* __restrict__ e2, float* df,
                                                                  float* dlo, float* e2f, float* e2lo, double* prm) {
    __shared__ double smin[FS_SCALAR_THREADS / 32], smax[FS_SCALAR_THREADS / 32], semax[FS_SCALAR_THREADS / 32];
    double lo = 1e300, hi = -1e300, em = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double el = i > 0 ? sqrt(e2[i - 1]) : 0.0, er = i < n - 1 ? sqrt(e2[i]) : 0.0;
        lo = fmin(lo, d[i] - el - er);
        hi = fmax(hi, d[i] + el + er);
        const double ee = i < n - 1 ? e2[i] : 0.0;
        em = fmax(em, ee);
        df[i] = (float)d[i];
        dlo[i] = (float)(d[i] - (double)df[i]);
        e2f[i] = (float)ee;
        e2lo[i] = (float)(ee - (double)e2f[i]);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    em = warp_max(em);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) { smin[warp] = lo; smax[warp] = hi; semax[warp] = em; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < nw; ++w) { lo = fmin(lo, smin[w]); hi = fmax(hi, smax[w]); em = fmax(em, semax[w]); }
        const double wdt = hi - lo, nrm = fmax(fabs(lo), fabs(hi));
        prm[0] = lo - (1e-12 * (wdt + nrm) + 1e-300);
        prm[1] = hi + (1e-12 * (wdt + nrm) + 1e-300);
        prm[2] = (double)(FLT_MIN * fmaxf(1.0f, (float)em));
        prm[3] = fmax(fabs(prm[0]), fabs(prm[1]));
    }
}

// Eigenvalue k (ascending), one thread each: FP32 bisection to a few FP32
// ulps of ||T||, then the widened bracket confirmed by double-float Sturm
// counts and finished by safeguarded double-float Newton (eig_df_bracketed).
__global__ void __launch_bounds__(FS_EIG_THREADS) k_fs_eig(int n, const float* __restrict__ df,
                                                          const float* __restrict__ dlo, const float* __restrict__ e2f,
                                                          const float* __restrict__ e2lo, const double* __restrict__ prm,
                                                          double* __restrict__ eig) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double lo = prm[0], hi = prm[1], nrm = prm[3];
    const float pivminf = (float)prm[2];
    float a = (float)lo * (lo < 0 ? 1.0000002f : 0.9999998f) - 1e-30f;
    float b = (float)hi * (hi > 0 ? 1.0000002f : 0.9999998f) + 1e-30f;
    const float atolf = fmaxf(2.0f * FLT_EPSILON * (float)nrm, 1e-30f);
    for (int it = 0; it < 96 && b - a > atolf; ++it) {
        const float mid = 0.5f * (a + b);
        if (!(mid > a && mid < b)) break;
        if (sturm_count_f32(n, df, e2f, mid, pivminf) <= k) a = mid;
        else b = mid;
    }
    eig[k] = eig_df_bracketed(n, df, dlo, e2f, e2lo, k, a, b, 8.0 * FLT_EPSILON * nrm, lo, hi, pivminf, nrm);
}

// Reduction of the packed matrix A (in R's complex form) to the real
// tridiagonal (d, e2), enqueued on st.  The buffers are those of FsArgs, as
// raw device memory; v_k sits in vb[k mod 3] and w_k in wb[k mod 2], and
// v_{-1} = vb[2] and w_{-1} = wb[1] start at zero.
template <typename R>
static cudaError_t fs_tridiagonalise(int n, void* A, void* vb_, void* wb_, void* pr, void* pc, void* p, void* red,
                                     void* tau, double* d, double* e2, cudaStream_t st) {
    using C = cplx_t<R>;
    FsArgs<R> a;
    a.n = n;
    a.A = static_cast<C*>(A);
    a.pr = static_cast<C*>(pr);
    a.pc = static_cast<C*>(pc);
    a.p = static_cast<C*>(p);
    a.red = static_cast<R*>(red);
    a.tau = static_cast<R*>(tau);
    a.d = d;
    a.e2 = e2;
    C* vb = static_cast<C*>(vb_);
    C* wb = static_cast<C*>(wb_);
    if (n == 2) {
        // d_0, d_1 and |e_0|^2 straight from the 2x2 matrix
        a.U = a.V = vb; a.Vn = vb; a.W = wb; a.Wn = wb;
        k_fs_setup<R><<<1, FS_SCALAR_THREADS, 0, st>>>(a);
        a.V = vb + n; a.W = wb;  // zero vectors: the finish reads A_11 unchanged
        k_fs_finish<R><<<1, 1, 0, st>>>(a);
        return cudaGetLastError();
    }
    a.Vn = vb;
    a.U = vb + 2 * (size_t)n;
    a.W = wb + n;
    a.V = vb;
    a.Wn = wb;
    k_fs_setup<R><<<1, FS_SCALAR_THREADS, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    for (int k = 0; k <= n - 3 && e == cudaSuccess; ++k) {
        const int mm = n - k - 1, T = (mm + FS_TB - 1) / FS_TB;
        a.U = vb + (size_t)((k + 2) % 3) * n;
        a.V = vb + (size_t)(k % 3) * n;
        a.Vn = vb + (size_t)((k + 1) % 3) * n;
        a.W = wb + (size_t)((k + 1) & 1) * n;
        a.Wn = wb + (size_t)(k & 1) * n;
        k_fs_pass<R><<<(unsigned)tri64(T), FS_PASS_THREADS, 0, st>>>(a, k);
        const int nred = (mm + FS_RED_ROWS - 1) / FS_RED_ROWS;
        k_fs_reduce<R><<<nred, FS_RED_THREADS, 0, st>>>(a, k);
        k_fs_scalar<R><<<1, FS_SCALAR_THREADS, 0, st>>>(a, k, nred);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    a.V = vb + (size_t)((n - 3) % 3) * n;
    a.W = wb + (size_t)((n - 3) & 1) * n;
    k_fs_finish<R><<<1, 1, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ptca

ptca_status ptca_internal_fail(ptca_status s, const char* msg);
ptca::Model ptca_context_model(const ptca_ctx* ctx);

extern "C" ptca_status ptca_full_spectrum(ptca_ctx* ctx, double* eig_out, void* stream) {
    using namespace ptca;
    if (!ctx || !eig_out) return ptca_internal_fail(PTCA_ERR_INVALID, "null argument");
    const int N = ctx->N;
    if (N > 16384) return ptca_internal_fail(PTCA_ERR_INVALID, "ptca_full_spectrum covers lattices of up to 16384 sites");
    const int n = 2 * N;
    const int Tmax = (n - 1 + FS_TB - 1) / FS_TB;
    cudaError_t es = ptca_internal_settle(ctx, static_cast<cudaStream_t>(stream), true);
    if (es != cudaSuccess) return ptca_internal_fail(PTCA_ERR_CUDA, cudaGetErrorString(es));
    const int red_max = (n + FS_RED_ROWS - 1) / FS_RED_ROWS;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    std::vector<void*> owned;
    auto alloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
        owned.push_back(q);
        return q;
    };
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (void* q : owned) cudaFree(q);
    };
    // + 64 elements of padding past the packed triangle
    double2* A = static_cast<double2*>(alloc(((size_t)tri64(n) + 64) * sizeof(double2)));
    double2* vb = static_cast<double2*>(alloc(3 * (size_t)n * sizeof(double2)));
    double2* wb = static_cast<double2*>(alloc(2 * (size_t)n * sizeof(double2)));
    double2* p = static_cast<double2*>(alloc((size_t)n * sizeof(double2)));
    double2* pr = static_cast<double2*>(alloc((size_t)(Tmax > 0 ? Tmax : 1) * n * sizeof(double2)));
    double2* pc = static_cast<double2*>(alloc((size_t)(Tmax > 0 ? Tmax : 1) * n * sizeof(double2)));
    double* red = static_cast<double*>(alloc((size_t)red_max * sizeof(double)));
    double* tau = static_cast<double*>(alloc(2 * sizeof(double)));
    double* d = static_cast<double*>(alloc((size_t)n * sizeof(double)));
    double* e2 = static_cast<double*>(alloc((size_t)n * sizeof(double)));
    float* f32 = static_cast<float*>(alloc(4 * (size_t)n * sizeof(float)));
    double* prm = static_cast<double*>(alloc(4 * sizeof(double)));
    for (void* q : {(void*)A, (void*)vb, (void*)wb, (void*)p, (void*)pr, (void*)pc, (void*)red, (void*)tau, (void*)d,
                    (void*)e2, (void*)f32, (void*)prm})
        if (!q) {
            release();
            return ptca_internal_fail(PTCA_ERR_OOM, "ptca_full_spectrum: not enough device memory for the matrix");
        }
    auto fail = [&](cudaError_t e, const char* where) {
        release();
        cudaGetLastError();
        return ptca_internal_fail(PTCA_ERR_CUDA, (std::string("ptca_full_spectrum: ") + where + ": " +
                                                  cudaGetErrorString(e)).c_str());
    };
    cudaError_t e = cudaMemsetAsync(A, 0, ((size_t)tri64(n) + 64) * sizeof(double2), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(vb, 0, 3 * (size_t)n * sizeof(double2), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(wb, 0, 2 * (size_t)n * sizeof(double2), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(e2, 0, (size_t)n * sizeof(double), st);
    if (e != cudaSuccess) return fail(e, "clearing the buffers");
    const Model m = ptca_context_model(ctx);
    k_full_hamiltonian<<<(N + 255) / 256, 256, 0, st>>>(m, ctx->d_S[0], N, A);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "building the matrix");

    if (ctx->prec == 1) {
        // PTCA_MIXED: the reduction in double-float
        const int64_t cnt = tri64(n) + 64;
        k_fs_to_dfl<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, 152 * 16), 256, 0, st>>>(A, cnt);
        e = fs_tridiagonalise<dfl>(n, A, vb, wb, pr, pc, p, red, tau, d, e2, st);
    } else {
        e = fs_tridiagonalise<double>(n, A, vb, wb, pr, pc, p, red, tau, d, e2, st);
    }
    if (e != cudaSuccess) return fail(e, "reducing to tridiagonal form");
    float* df = f32;
    float* dlo = f32 + n;
    float* e2f = f32 + 2 * (size_t)n;
    float* e2lo = f32 + 3 * (size_t)n;
    k_fs_eig_prep<<<1, FS_SCALAR_THREADS, 0, st>>>(n, d, e2, df, dlo, e2f, e2lo, prm);
    k_fs_eig<<<(n + FS_EIG_THREADS - 1) / FS_EIG_THREADS, FS_EIG_THREADS, 0, st>>>(n, df, dlo, e2f, e2lo, prm, eig_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "eigenvalues");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e, "synchronising");
    release();
    return PTCA_OK;
}
