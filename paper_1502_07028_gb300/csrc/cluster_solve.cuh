// cluster_solve.cuh -- per-CTA cluster eigen-solve for the traveling cluster
// approximation: window gather and cluster-matrix build (Sec. II.b-c, Fig. 1),
// Householder reduction of the Hermitian matrix to real tridiagonal form,
// tridiagonal eigenvalues by Sturm-sequence bisection, and the
// grand-canonical free energy F = -T sum_k ln(1 + exp(-(eps_k - mu)/T)).
//
// One CTA of NW warps owns one matrix.  The matrix lives in shared memory as
// its packed lower triangle (element (r,c), c <= r, at r(r+1)/2 + c).
#pragma once

#include <cfloat>
#include "device_common.cuh"

namespace ptca {

// Problem description the kernels need (copied by value into each launch).
struct Model {
    int32_t Lx, Ly, lattice_periodic;
    int32_t Lc, ox, oy, cluster_periodic;
    int32_t proposal;
    double t, JH, mu, T, cone_cos;
    uint64_t seed;
};

// Window of the traveling cluster around update site (cx, cy) along one axis:
// periodic lattice -> L_c sites starting o before the centre, wrapped;
// open lattice -> the same range clipped to the lattice.
__device__ __forceinline__ void window_axis(int L, int periodic, int Lc, int o, int c, int& start, int& ext) {
    if (L == 1) { start = 0; ext = 1; return; }
    int a = c - o, b = c - o + Lc - 1;
    if (periodic) { start = ((a % L) + L) % L; ext = Lc; return; }
    a = a < 0 ? 0 : a;
    b = b > L - 1 ? L - 1 : b;
    start = a; ext = b - a + 1;
}

struct Window { int x0, y0, ex, ey, uwx, uwy; };

__device__ __forceinline__ Window make_window(const Model& m, int site) {
    Window w;
    const int cx = site % m.Lx, cy = site / m.Lx;
    window_axis(m.Lx, m.lattice_periodic, m.Lc, m.ox, cx, w.x0, w.ex);
    window_axis(m.Ly, m.lattice_periodic, m.Lc, m.oy, cy, w.y0, w.ey);
    w.uwx = cx - w.x0; if (w.uwx < 0) w.uwx += m.Lx;
    w.uwy = cy - w.y0; if (w.uwy < 0) w.uwy += m.Ly;
    return w;
}

__device__ __forceinline__ int window_site(const Model& m, const Window& w, int wx, int wy) {
    int x = w.x0 + wx, y = w.y0 + wy;
    if (m.lattice_periodic) { if (x >= m.Lx) x -= m.Lx; if (y >= m.Ly) y -= m.Ly; }
    return y * m.Lx + x;
}

__device__ __forceinline__ int tri(int r) { return (r * (r + 1)) >> 1; }

// Gather the window spins into sp[nsite][3] (replacing the update site's spin
// by s_new when s_new != nullptr) and build the packed cluster matrix:
//   Hund block   -J_H [[S_z, S_x - i S_y], [S_x + i S_y, -S_z]] per site,
//   hopping      -t between nearest neighbours, same spin, each bond once;
// a periodic cluster wraps inside the window (an axis of extent 2 then has
// two bonds between its two sites, extent 1 none).  Caller syncs after.
template <typename T>
__device__ void build_cluster(const Model& m, const Window& w, const double* __restrict__ S,
                              const double* s_new, double* sp, cplx_t<T>* A) {
    using V = cplx_t<T>;
    const int nsite = w.ex * w.ey, n = 2 * nsite, P = tri(n);
    for (int i = threadIdx.x; i < P; i += blockDim.x) A[i] = mk(T(0), T(0));
    const int uw = w.uwy * w.ex + w.uwx;
    for (int s = threadIdx.x; s < nsite; s += blockDim.x) {
        const int wx = s % w.ex, wy = s / w.ex;
        const int g = window_site(m, w, wx, wy);
        double v0, v1, v2;
        if (s_new != nullptr && s == uw) { v0 = s_new[0]; v1 = s_new[1]; v2 = s_new[2]; }
        else { v0 = S[3 * g]; v1 = S[3 * g + 1]; v2 = S[3 * g + 2]; }
        sp[3 * s] = v0; sp[3 * s + 1] = v1; sp[3 * s + 2] = v2;
    }
    __syncthreads();
    const T t = T(m.t), J = T(m.JH);
    for (int s = threadIdx.x; s < nsite; s += blockDim.x) {
        const int wx = s % w.ex, wy = s / w.ex;
        const T sx = T(sp[3 * s]), sy = T(sp[3 * s + 1]), sz = T(sp[3 * s + 2]);
        const int a = 2 * s, b = 2 * s + 1;
        A[tri(a) + a] = mk(-J * sz, T(0));
        A[tri(b) + b] = mk(J * sz, T(0));
        A[tri(b) + a] = mk(-J * sx, -J * sy);  // element (b, a) = -J_H (S_x + i S_y)
        // +x bond
        int nb = -1, mult = 1;
        if (wx + 1 < w.ex) { nb = s + 1; if (m.cluster_periodic && w.ex == 2) mult = 2; }
        else if (m.cluster_periodic && w.ex >= 3) nb = s - (w.ex - 1);
        if (nb >= 0) {
            const int hi = nb > s ? nb : s, lo = nb > s ? s : nb;
            for (int sg = 0; sg < 2; ++sg) A[tri(2 * hi + sg) + 2 * lo + sg] = mk(-T(mult) * t, T(0));
        }
        // +y bond
        nb = -1; mult = 1;
        if (wy + 1 < w.ey) { nb = s + w.ex; if (m.cluster_periodic && w.ey == 2) mult = 2; }
        else if (m.cluster_periodic && w.ey >= 3) nb = wx;
        if (nb >= 0) {
            const int hi = nb > s ? nb : s, lo = nb > s ? s : nb;
            for (int sg = 0; sg < 2; ++sg) A[tri(2 * hi + sg) + 2 * lo + sg] = mk(-T(mult) * t, T(0));
        }
    }
}

// ---------------------------------------------------------------------------
// Householder tridiagonalisation of a Hermitian matrix (packed lower triangle
// in A, order n <= 32*NT <= 32*NW).  Step k reflects column k below the
// diagonal onto its first entry with the Hermitian unitary H = I - tau v v^H,
// v = x + (x_0/|x_0|) ||x|| e_1, tau = 1/(||x|| (||x|| + |x_0|)), and updates
// the trailing block as A <- A - v w^H - w v^H, p = tau A v,
// w = p - (tau/2)(v^H p) v.  The rank-2 update of step k is deferred and fused
// with the matrix-vector product of step k+1, so the trailing block is read
// and written once per step; the next pivot column receives its update
// explicitly first.  Output: diagonal d[0..n-1] and squared off-diagonal
// moduli e2[0..n-2] (the phases of the off-diagonal do not affect the
// eigenvalues).
//
// Work layout: row i of the trailing block belongs to warp i % NW; lane l
// handles columns j = l + 32 t (t < NT).  Each warp processes its rows in
// batches of 8; the 8 row sums are reduce-scattered across the warp.  Column
// (transposed) contributions accumulate per lane and are summed across warps
// through shared memory.
// ---------------------------------------------------------------------------
template <typename T> struct HHScratch {
    cplx_t<T>* Vb;   // 2 x NMAX   Householder vectors of consecutive steps
    cplx_t<T>* Wv;   // NMAX       w of the previous step
    cplx_t<T>* pr;   // NMAX       row sums of A v
    cplx_t<T>* pc;   // NW x NMAX  column sums of A v, per warp
    T* redA;         // NW
    T* redB;         // NW
};

template <typename V>
__device__ __forceinline__ V reduce_scatter8(const V (&v)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    V w4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        V mine = b4 ? v[q + 4] : v[q];
        V other = b4 ? v[q] : v[q + 4];
        w4[q] = cadd(mine, cshfl_xor(other, 16));
    }
    V w2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        V mine = b3 ? w4[q + 2] : w4[q];
        V other = b3 ? w4[q] : w4[q + 2];
        w2[q] = cadd(mine, cshfl_xor(other, 8));
    }
    V mine = b2 ? w2[1] : w2[0];
    V other = b2 ? w2[0] : w2[1];
    V w1 = cadd(mine, cshfl_xor(other, 4));
    w1 = cadd(w1, cshfl_xor(w1, 2));
    w1 = cadd(w1, cshfl_xor(w1, 1));
    return w1;  // row (lane >> 2) & 7 of the batch
}

template <typename T, int NT, int NW>
__device__ void householder_tridiag(int n, cplx_t<T>* A, const HHScratch<T>& sc, double* d, double* e2) {
    using V = cplx_t<T>;
    constexpr int NMAX = 32 * NT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    V* const Vb = sc.Vb;
    V* const Wv = sc.Wv;
    V* const pr = sc.pr;
    V* const pc = sc.pc;
    const V zero = mk(T(0), T(0));

    for (int i = tid; i < 2 * NMAX; i += NW * 32) Vb[i] = zero;
    for (int i = tid; i < NMAX; i += NW * 32) Wv[i] = zero;
    __syncthreads();

    if (n <= 2) {
        if (tid == 0) {
            d[0] = double(A[0].x);
            if (n == 2) { d[1] = double(A[2].x); e2[0] = double(cabs2(A[1])); }
        }
        __syncthreads();
        return;
    }

    // Column 0: d_0, ||x||^2 and the first reflector.
    T tau;
    {
        V a = zero;
        if (tid < n) a = A[tri(tid)];
        if (tid == 0) d[0] = double(a.x);
        T s2 = block_sum<T>((tid >= 1 && tid < n) ? cabs2(a) : T(0), sc.redB);
        const T sigma = sqrt(s2);
        const V x0 = A[tri(1)];
        const T ax0 = sqrt(cabs2(x0));
        if (tid == 0) e2[0] = double(s2);
        if (tid >= 1 && tid < n) {
            V v = a;
            if (tid == 1) {
                const V ph = ax0 > T(0) ? mk(x0.x / ax0, x0.y / ax0) : mk(T(1), T(0));
                v = mk(x0.x + ph.x * sigma, x0.y + ph.y * sigma);
            }
            Vb[tid] = v;
        }
        tau = sigma > T(0) ? T(1) / (sigma * (sigma + ax0)) : T(0);
        __syncthreads();
    }

    for (int k = 0; k <= n - 3; ++k) {
        const V* V_ = Vb + (k & 1) * NMAX;        // v_k
        const V* U_ = Vb + ((k + 1) & 1) * NMAX;  // v_{k-1} (zero at k = 0)
        const int j0 = k + 1;                     // first active row/column

        // ---- fused pass: A <- A - u w^H - w u^H (step k-1), accumulate A v_k
        V vc[NT], uc[NT], wc[NT], cacc[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int j = 32 * t + lane;
            vc[t] = V_[j]; uc[t] = U_[j]; wc[t] = Wv[j];
            cacc[t] = zero;
        }
        const int first = j0 + ((warp - j0) % NW + NW) % NW;
        for (int rb = first; rb < n; rb += 8 * NW) {
            V racc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) racc[r] = zero;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = rb + r * NW;
                if (i < n) {
                    const V ui = U_[i], wi = Wv[i], vi = V_[i];
                    V* row = A + tri(i);
#pragma unroll
                    for (int t = 0; t < NT; ++t) {
                        if (32 * t + 31 >= j0 && 32 * t <= i) {
                            const int j = 32 * t + lane;
                            if (j >= j0 && j <= i) {
                                V a = row[j];
                                if (k > 0) {
                                    a = cfms_conj_b(ui, wc[t], a);
                                    a = cfms_conj_b(wi, uc[t], a);
                                    if (j == i) a.y = T(0);
                                    row[j] = a;
                                }
                                racc[r] = cfma(a, vc[t], racc[r]);
                                if (j < i) cacc[t] = cfma_conj_a(a, vi, cacc[t]);
                            }
                        }
                    }
                }
            }
            const V rs = reduce_scatter8(racc, lane);
            const int ri = rb + ((lane >> 2) & 7) * NW;
            if ((lane & 3) == 0 && ri < n) pr[ri] = rs;
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int j = 32 * t + lane;
            if (j >= j0 && j < n) pc[warp * NMAX + j] = cacc[t];
        }
        __syncthreads();

        // ---- p = tau A v, s = v^H p
        V p = zero, vj = zero;
        if (tid >= j0 && tid < n) {
            p = pr[tid];
            for (int w = 0; w < NW; ++w) p = cadd(p, pc[w * NMAX + tid]);
            p.x *= tau; p.y *= tau;
            vj = V_[tid];
        }
        const T s = block_sum<T>(vj.x * p.x + vj.y * p.y, sc.redA);
        const T K = T(0.5) * tau * s;

        // ---- w = p - K v; explicit update of pivot column k+1
        V wj = mk(p.x - K * vj.x, p.y - K * vj.y);
        V pk = pr[j0];
        for (int w = 0; w < NW; ++w) pk = cadd(pk, pc[w * NMAX + j0]);
        pk.x *= tau; pk.y *= tau;
        const V vk1 = V_[j0];
        const V wk1 = mk(pk.x - K * vk1.x, pk.y - K * vk1.y);
        V a = zero;
        if (tid >= j0 && tid < n) {
            Wv[tid] = wj;
            a = A[tri(tid) + j0];
            a = cfms_conj_b(vj, wk1, a);
            a = cfms_conj_b(wj, vk1, a);
            if (tid == j0) { a.y = T(0); d[j0] = double(a.x); }
            A[tri(tid) + j0] = a;
        }
        const T s2 = block_sum<T>((tid >= j0 + 1 && tid < n) ? cabs2(a) : T(0), sc.redB);
        if (tid == 0) e2[j0] = double(s2);

        // ---- next reflector from column k+1 (none for the last column)
        if (k + 1 <= n - 3) {
            V* Vn = Vb + ((k + 1) & 1) * NMAX;
            const T sigma = sqrt(s2);
            const V x0 = A[tri(j0 + 1) + j0];
            const T ax0 = sqrt(cabs2(x0));
            if (tid >= j0 + 1 && tid < n) {
                V v = a;
                if (tid == j0 + 1) {
                    const V ph = ax0 > T(0) ? mk(x0.x / ax0, x0.y / ax0) : mk(T(1), T(0));
                    v = mk(x0.x + ph.x * sigma, x0.y + ph.y * sigma);
                }
                Vn[tid] = v;
            }
            tau = sigma > T(0) ? T(1) / (sigma * (sigma + ax0)) : T(0);
        }
        __syncthreads();
    }

    // Step n-3's update of the last diagonal entry.
    if (tid == 0) {
        const V v = Vb[((n - 3) & 1) * NMAX + n - 1];
        const V w = Wv[n - 1];
        const T ann = A[tri(n - 1) + n - 1].x - T(2) * (v.x * w.x + v.y * w.y);
        d[n - 1] = double(ann);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Tridiagonal eigenvalues.  Sturm count: number of eigenvalues below x from
// the pivots q_0 = d_0 - x, q_i = (d_i - x) - e2_{i-1}/q_{i-1}, a pivot of
// magnitude below pivmin replaced by -pivmin (Barth, Martin and Wilkinson's
// bisection with Kahan's safeguard).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int sturm_count_f64(int n, const double* d, const double* e2, double x, double pivmin) {
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    int c = q < 0.0;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        c += q < 0.0;
    }
    return c;
}

__device__ __forceinline__ int sturm_count_f32(int n, const float* d, const float* e2, float x, float pivmin) {
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    int c = q < 0.0f;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - __fdividef(e2[i - 1], q);
        if (fabsf(q) < pivmin) q = -pivmin;
        c += q < 0.0f;
    }
    return c;
}

// Gershgorin interval of the tridiagonal (computed by every thread from
// shared memory; the fixed order gives identical results in all threads).
__device__ __forceinline__ void gershgorin(int n, const double* d, const double* e2, double& lo, double& hi, double& emax2) {
    lo = 1e300; hi = -1e300; emax2 = 0.0;
    double eprev = 0.0;
    for (int i = 0; i < n; ++i) {
        const double ei = (i < n - 1) ? sqrt(e2[i]) : 0.0;
        if (i < n - 1) emax2 = fmax(emax2, e2[i]);
        lo = fmin(lo, d[i] - eprev - ei);
        hi = fmax(hi, d[i] + eprev + ei);
        eprev = ei;
    }
    const double w = hi - lo, nrm = fmax(fabs(lo), fabs(hi));
    lo -= 1e-12 * (w + nrm) + 1e-300;
    hi += 1e-12 * (w + nrm) + 1e-300;
}

// k-th smallest eigenvalue (0-based) by FP64 bisection on [lo, hi].
__device__ __forceinline__ double bisect_f64(int n, const double* d, const double* e2, int k, double lo, double hi,
                                             double pivmin, double atol) {
    for (int it = 0; it < 80; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (hi - lo <= fmax(atol, 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)))) break;
        if (sturm_count_f64(n, d, e2, mid, pivmin) <= k) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// k-th smallest eigenvalue: FP32 bisection to FP32 resolution, then one FP64
// Newton step on det(T - x) = prod q_i (the logarithmic derivative
// sum q_i'/q_i comes from the same pivot recurrence), kept only if it stays
// near the FP32 bracket.
__device__ __forceinline__ double bisect_f32_newton_f64(int n, const float* df, const float* e2f, const double* d,
                                                        const double* e2, int k, float lo, float hi, float pivminf,
                                                        float atolf, double pivmin) {
    for (int it = 0; it < 48; ++it) {
        const float mid = 0.5f * (lo + hi);
        if (hi - lo <= fmaxf(atolf, 2.0f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)))) break;
        if (sturm_count_f32(n, df, e2f, mid, pivminf) <= k) lo = mid; else hi = mid;
    }
    const double x = 0.5 * ((double)lo + (double)hi);
    double q = d[0] - x, dq = -1.0;
    if (fabs(q) < pivmin) q = -pivmin;
    double s = 0.0;
    for (int i = 1; i < n; ++i) {
        const double r = 1.0 / q;
        s = fma(dq, r, s);
        const double er = e2[i - 1] * r;
        double qn = (d[i] - x) - er;
        dq = fma(er * r, dq, -1.0);
        if (fabs(qn) < pivmin) qn = -pivmin;
        q = qn;
    }
    s = fma(dq, 1.0 / q, s);
    const double xn = x - 1.0 / s;
    const double w = fmax((double)(hi - lo), 4.0 * (double)atolf);
    if (isfinite(xn) && xn >= (double)lo - w && xn <= (double)hi + w) return xn;
    return x;
}

// softplus(x) = ln(1 + e^x), written as max(x,0) + log1p(e^-|x|).
__device__ __forceinline__ double softplus(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }

}  // namespace ptca
