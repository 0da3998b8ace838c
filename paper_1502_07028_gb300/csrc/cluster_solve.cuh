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
#include "dfloat.cuh"

namespace ptca {

// Problem description the kernels need (copied by value into each launch).
// Problem on the device.  The on-site block of site i with classical vector
// v_i is (e0 + lam v_x) 1 - JH v.sigma, and the cluster free energy adds
// ca |v|^2 + cb v_x + cc per window site when cls_on:
//   model 0 (double exchange): JH = J_H, unit spins, no classical term;
//   model 1 (Hubbard mean field, Eq. 1, <n_i> = 1): JH = e0 = U/2,
//     ca = U/4, cc = -U/4, proposals uniform in a ball of radius m_step;
//   model 2 (adiabatic Holstein): lam = lambda, v = (x, 0, 0), ca = K/2,
//     cb = -lambda, cc = mu, proposals x + m_step (2u - 1).
struct Model {
    int32_t Lx, Ly, Lz, lattice_periodic;   // Lz == 1: square lattice or chain
    int32_t Lc, ox, oy, oz, cluster_periodic;
    int32_t proposal;
    int32_t model;
    int32_t cls_on;
    double t, JH, mu, T, cone_cos;
    double e0, lam, ca, cb, cc, m_step;
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

// Window of an update site: start and extent along each axis, and the update
// site's window coordinates.  Sites are indexed (z Ly + y) Lx + x; window
// sites (wz ey + wy) ex + wx.
struct Window { int x0, y0, z0, ex, ey, ez, uwx, uwy, uwz; };

__device__ __forceinline__ Window make_window(const Model& m, int site) {
    Window w;
    const int cx = site % m.Lx, cy = (site / m.Lx) % m.Ly, cz = site / (m.Lx * m.Ly);
    window_axis(m.Lx, m.lattice_periodic, m.Lc, m.ox, cx, w.x0, w.ex);
    window_axis(m.Ly, m.lattice_periodic, m.Lc, m.oy, cy, w.y0, w.ey);
    window_axis(m.Lz, m.lattice_periodic, m.Lc, m.oz, cz, w.z0, w.ez);
    w.uwx = cx - w.x0; if (w.uwx < 0) w.uwx += m.Lx;
    w.uwy = cy - w.y0; if (w.uwy < 0) w.uwy += m.Ly;
    w.uwz = cz - w.z0; if (w.uwz < 0) w.uwz += m.Lz;
    return w;
}

__device__ __forceinline__ int window_nsite(const Window& w) { return w.ex * w.ey * w.ez; }

__device__ __forceinline__ int window_site(const Model& m, const Window& w, int wx, int wy, int wz = 0) {
    int x = w.x0 + wx, y = w.y0 + wy, z = w.z0 + wz;
    if (m.lattice_periodic) {
        if (x >= m.Lx) x -= m.Lx;
        if (y >= m.Ly) y -= m.Ly;
        if (z >= m.Lz) z -= m.Lz;
    }
    return (z * m.Ly + y) * m.Lx + x;
}

__device__ __forceinline__ int tri(int r) { return (r * (r + 1)) >> 1; }

// Storage of a cluster matrix as 4x4 complex tiles over the lower block
// triangle: tile t = tri(R) + C (C <= R) at elements 16t .. 16t+15; element
// e = 4r + c of the tile lies in its 16-byte slot e/2, and slot h is stored at
// position h ^ (t mod 8), so that lanes reading the same slot of consecutive
// tiles hit distinct shared-memory banks.  Diagonal tiles hold both triangles.
__device__ __forceinline__ int tl_pos(int t, int e) {
    return (t << 4) + ((((e >> 1) ^ (t & 7))) << 1) + (e & 1);
}
// Storage position of element (r, c), r >= c.
__device__ __forceinline__ int tl_at(int r, int c) {
    return tl_pos(tri(r >> 2) + (c >> 2), ((r & 3) << 2) + (c & 3));
}
// Complex elements of the tiled storage of an order-n matrix.
__host__ __device__ __forceinline__ int tl_elems(int n) {
    const int nb = (n + 3) >> 2;
    return ((nb * (nb + 1)) >> 1) << 4;
}
// Position of element (r, c), r >= c, in the packed lower triangle or the tiled layout.
template <bool kTiled> __device__ __forceinline__ int mat_at(int r, int c) {
    if constexpr (kTiled) return tl_at(r, c);
    else return tri(r) + c;
}

// Proposed new classical vector at `site` (Sec. II.c step c).  Double
// exchange: propose_spin (sphere or cone).  Hubbard mean field: the old field
// plus a step uniform in the ball of radius m_step -- direction from the
// proposal uniforms (as the sphere proposal), length m_step v^(1/3) with v
// the first uniform of purpose RNG_RADIUS.  Holstein: x + m_step (2u - 1).
// All are symmetric in (old, new).
__device__ __forceinline__ void propose(const Model& m, uint64_t sweep, uint32_t site, const double so[3],
                                        double sn[3]) {
    if (m.model == 2) {
        double u0, u1;
        uniform2(m.seed, sweep, site, RNG_PROPOSE, u0, u1);
        sn[0] = so[0] + m.m_step * (2.0 * u0 - 1.0);
        sn[1] = so[1];
        sn[2] = so[2];
        return;
    }
    if (m.model != 1) {
        propose_spin(m.seed, sweep, site, m.proposal, m.cone_cos, so, sn);
        return;
    }
    double u0, u1, v0, v1, dir[3];
    uniform2(m.seed, sweep, site, RNG_PROPOSE, u0, u1);
    unit_from_uniforms(u0, u1, dir);
    uniform2(m.seed, sweep, site, RNG_RADIUS, v0, v1);
    const double r = m.m_step * cbrt(v0);
    sn[0] = so[0] + r * dir[0];
    sn[1] = so[1] + r * dir[1];
    sn[2] = so[2] + r * dir[2];
}

// Classical energy of a window: ca |v|^2 + cb v_x + cc summed over its nsite
// vectors sp[nsite][3] (zero unless cls_on).  One thread.
__device__ __forceinline__ double window_classical(const Model& m, const double* sp, int nsite) {
    if (!m.cls_on) return 0.0;
    double acc = 0.0;
    for (int s = 0; s < nsite; ++s) {
        const double v0 = sp[3 * s], v1 = sp[3 * s + 1], v2 = sp[3 * s + 2];
        acc += m.ca * (v0 * v0 + v1 * v1 + v2 * v2) + m.cb * v0 + m.cc;
    }
    return acc;
}

// Gather the window spins into sp[nsite][3] (replacing the update site's spin
// by s_new when s_new != nullptr) and build the packed cluster matrix:
//   on-site block  (e0 + lam S_x) - J [[S_z, S_x - i S_y], [S_x + i S_y, -S_z]]
//                  per site (J = m.JH, lam = m.lam; e0 is the caller's
//                  diagonal shift),
//   hopping        -t between nearest neighbours (x, y and, on a cubic
//                  lattice, z), same spin, each bond once;
// a periodic cluster wraps inside the window (an axis of extent 2 then has
// two bonds between its two sites, extent 1 none).  Caller syncs after.  The
// sweep kernels pass e0 = 0 and shift mu by -m.e0 instead: a multiple of the
// identity moves every eigenvalue by exactly e0, and the reduction keeps its
// relative precision on the unshifted matrix.
//
// kTiled selects the tiled layout (tl_at): its padding is zeroed and its
// diagonal tiles receive their upper triangles too.
template <typename T, bool kTiled = false>
__device__ void build_cluster(const Model& m, const Window& w, const double* __restrict__ S,
                              const double* s_new, double* sp, cplx_t<T>* A, double e0 = 0.0) {
    using V = cplx_t<T>;
    const int nsite = window_nsite(w), n = 2 * nsite, P = kTiled ? tl_elems(n) : tri(n), exy = w.ex * w.ey;
    for (int i = threadIdx.x; i < P; i += blockDim.x) A[i] = mk(T(0), T(0));
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
    const T t = T(m.t), J = T(m.JH), d0 = T(e0), lam = T(m.lam);
    for (int s = threadIdx.x; s < nsite; s += blockDim.x) {
        const int wx = s % w.ex, wy = (s / w.ex) % w.ey, wz = s / exy;
        const T sx = T(sp[3 * s]), sy = T(sp[3 * s + 1]), sz = T(sp[3 * s + 2]);
        const int a = 2 * s, b = 2 * s + 1;
        const T dg = d0 + lam * sx;
        A[mat_at<kTiled>(a, a)] = mk(dg - J * sz, T(0));
        A[mat_at<kTiled>(b, b)] = mk(dg + J * sz, T(0));
        A[mat_at<kTiled>(b, a)] = mk(-J * sx, -J * sy);  // element (b, a) = -J_H (S_x + i S_y)
        // +x bond
        int nb = -1, mult = 1;
        if (wx + 1 < w.ex) { nb = s + 1; if (m.cluster_periodic && w.ex == 2) mult = 2; }
        else if (m.cluster_periodic && w.ex >= 3) nb = s - (w.ex - 1);
        if (nb >= 0) {
            const int hi = nb > s ? nb : s, lo = nb > s ? s : nb;
            for (int sg = 0; sg < 2; ++sg) A[mat_at<kTiled>(2 * hi + sg, 2 * lo + sg)] = mk(-T(mult) * t, T(0));
        }
        // +y bond
        nb = -1; mult = 1;
        if (wy + 1 < w.ey) { nb = s + w.ex; if (m.cluster_periodic && w.ey == 2) mult = 2; }
        else if (m.cluster_periodic && w.ey >= 3) nb = s - (w.ey - 1) * w.ex;
        if (nb >= 0) {
            const int hi = nb > s ? nb : s, lo = nb > s ? s : nb;
            for (int sg = 0; sg < 2; ++sg) A[mat_at<kTiled>(2 * hi + sg, 2 * lo + sg)] = mk(-T(mult) * t, T(0));
        }
        // +z bond
        nb = -1; mult = 1;
        if (wz + 1 < w.ez) { nb = s + exy; if (m.cluster_periodic && w.ez == 2) mult = 2; }
        else if (m.cluster_periodic && w.ez >= 3) nb = s - (w.ez - 1) * exy;
        if (nb >= 0) {
            const int hi = nb > s ? nb : s, lo = nb > s ? s : nb;
            for (int sg = 0; sg < 2; ++sg) A[mat_at<kTiled>(2 * hi + sg, 2 * lo + sg)] = mk(-T(mult) * t, T(0));
        }
    }
    if constexpr (kTiled) {
        // Upper triangles of the diagonal tiles (6 elements each).
        __syncthreads();
        const int nb = (n + 3) >> 2;
        for (int t = threadIdx.x; t < 6 * nb; t += blockDim.x) {
            const int R = t / 6, q = t % 6;
            const int r = q < 1 ? 1 : (q < 3 ? 2 : 3), c = q - (r * (r - 1)) / 2;  // (r, c), r > c
            const V x = A[tl_at(4 * R + r, 4 * R + c)];
            A[tl_pos(tri(R) + R, (c << 2) + r)] = mk(x.x, -x.y);
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
// Work layout (indices relative to the active corner j0 = k+1): relative row
// ri belongs to warp ri % NW; lane l handles relative columns l + 32 t.  Each
// warp processes its rows in batches of 8; the 8 row sums are
// reduce-scattered across the warp.  Column (transposed) contributions
// accumulate per lane and are summed across warps through shared memory.
//
// Between passes every vector entry has its own thread (relative index ri =
// threadIdx.x), so the per-step scalar work -- combining the partial sums of
// p = tau A v, the reduction v^H p, w, the explicit update of the pivot
// column, ||x||^2 and the next reflector -- is spread over the whole CTA with
// three barriers per step.  The first entry of each reflector (x_0 +
// phase(x_0) ||x||) is kept in registers by every thread; the other entries
// live in shared memory.
// ---------------------------------------------------------------------------
template <typename T> struct HHScratch {
    cplx_t<T>* Vb;   // 2 x NMAX   Householder vectors of consecutive steps
    cplx_t<T>* Wv;   // NMAX       w of the previous step
    cplx_t<T>* pr;   // NMAX       row sums of A v
    cplx_t<T>* pc;   // NW x NMAX  column sums of A v, per warp
    T* redA;         // NW
    T* redB;         // NW
    cplx_t<T>* sx;   // 3 scalars: x0 of the next reflector, its first entry, (tau, 0)
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

template <typename V>
__device__ __forceinline__ V reduce_scatter4(const V (&v)[4], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8;
    V w2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        V mine = b4 ? v[q + 2] : v[q];
        V other = b4 ? v[q] : v[q + 2];
        w2[q] = cadd(mine, cshfl_xor(other, 16));
    }
    V mine = b3 ? w2[1] : w2[0];
    V other = b3 ? w2[0] : w2[1];
    V w1 = cadd(mine, cshfl_xor(other, 8));
    w1 = cadd(w1, cshfl_xor(w1, 4));
    w1 = cadd(w1, cshfl_xor(w1, 2));
    w1 = cadd(w1, cshfl_xor(w1, 1));
    return w1;  // row (lane >> 3) & 3 of the batch
}

template <typename V>
__device__ __forceinline__ V reduce_scatter2(const V (&v)[2], int lane) {
    const bool b4 = lane & 16;
    const V mine = b4 ? v[1] : v[0];
    const V other = b4 ? v[0] : v[1];
    V w1 = cadd(mine, cshfl_xor(other, 16));
    w1 = cadd(w1, cshfl_xor(w1, 8));
    w1 = cadd(w1, cshfl_xor(w1, 4));
    w1 = cadd(w1, cshfl_xor(w1, 2));
    w1 = cadd(w1, cshfl_xor(w1, 1));
    return w1;  // row (lane >> 4) & 1 of the batch
}

// Rows per batch of the fused pass: the per-row registers of a batch are
// four complex values, so wider types take fewer rows.
template <typename T> struct PassRows { static constexpr int value = 4; };
template <> struct PassRows<float> { static constexpr int value = 8; };
template <> struct PassRows<dfl> { static constexpr int value = 2; };

// Sum over the first nact warps of a per-warp partial (the caller
// synchronises between the write and the read).
template <typename T, int NW>
__device__ __forceinline__ T sum_partials(const T* red, int nact) {
    T s = red[0];
#pragma unroll
    for (int w = 1; w < NW; ++w)
        if (w < nact) s += red[w];
    return s;
}

// Next reflector from the updated pivot column: given ||x||^2 (s2) and x_0,
// its first entry x_0 + phase(x_0) ||x|| and tau = 1 / (||x|| (||x|| + |x_0|)).
template <typename T>
__device__ __forceinline__ void reflector_head(T s2, cplx_t<T> x0, cplx_t<T>& first, T& tau) {
    const T sigma = sqroot(s2);
    const T ax0 = sqroot(cabs2(x0));
    const cplx_t<T> ph = ax0 > T(0) ? mk(x0.x / ax0, x0.y / ax0) : mk(T(1), T(0));
    first = mk(x0.x + ph.x * sigma, x0.y + ph.y * sigma);
    tau = sigma > T(0) ? T(1) / (sigma * (sigma + ax0)) : T(0);
}
// FP32: reciprocal square roots and a fast reciprocal.  Their few-ulp errors
// are far below the FP32 reduction's own, and every thread evaluates this.
template <>
__device__ __forceinline__ void reflector_head<float>(float s2, float2 x0, float2& first, float& tau) {
    const float ax2 = x0.x * x0.x + x0.y * x0.y;
    const float sigma = s2 > 0.f ? s2 * rsqrtf(s2) : 0.f;
    const float rx = ax2 > 0.f ? rsqrtf(ax2) : 0.f;
    const float ax0 = ax2 * rx;
    const float2 ph = ax2 > 0.f ? make_float2(x0.x * rx, x0.y * rx) : make_float2(1.f, 0.f);
    first = make_float2(x0.x + ph.x * sigma, x0.y + ph.y * sigma);
    tau = sigma > 0.f ? __fdividef(1.f, sigma * (sigma + ax0)) : 0.f;
}

// Shared phases of the Householder reductions below (one CTA of NW warps per
// matrix, vectors of NMAX entries in shared memory, A in shared or global
// memory).  hh_setup zeroes the vectors and forms the first reflector; it
// returns false when n <= 2 (d and e2 already written).  hh_scalar is the
// per-step scalar work after a pass (every vector entry has its own thread:
// blockDim >= n); hh_finish writes the last diagonal entry.
template <typename T, int NW, int NMAX>
__device__ __forceinline__ bool hh_setup(int n, cplx_t<T>* A, const HHScratch<T>& sc, double* d, double* e2,
                                         cplx_t<T>& vfirst, T& tau) {
    using V = cplx_t<T>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    V* const Vb = sc.Vb;
    V* const Wv = sc.Wv;
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
        return false;
    }

    // Column 0: d_0, ||x||^2 and the first reflector v_0 (entries 1 .. n-1;
    // entry 1 in registers, the rest in Vb[0 .. NMAX)).
    {
        const int ri = tid;
        const int nact = (n + 31) >> 5;  // warps holding entries
        if (warp < nact) {
            T s2p = T(0);
            if (ri < n) {
                const V a = A[tri(ri)];
                if (ri == 0) d[0] = double(a.x);
                if (ri >= 1) s2p = cabs2(a);
                if (ri >= 2) Vb[ri] = a;
                if (ri == 1) sc.sx[0] = a;
            }
            s2p = warp_sum(s2p);
            if (lane == 0) sc.redB[warp] = s2p;
        }
        __syncthreads();
        const T s2 = sum_partials<T, NW>(sc.redB, nact);
        if (tid == 0) e2[0] = double(s2);
        reflector_head(s2, sc.sx[0], vfirst, tau);
    }

    return true;
}

template <typename T, int NW, int NMAX>
__device__ __forceinline__ void hh_scalar(int k, int n, cplx_t<T>* A, const HHScratch<T>& sc, double* d,
                                          double* e2, cplx_t<T>& vfirst, T& tau) {
    using V = cplx_t<T>;
    // The scalar tail (two square roots, divisions) is recomputed by every
    // thread in FP32; in FP64 one warp computes it and shares it.
    constexpr bool kSharedTail = sizeof(T) == 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    V* const Vb = sc.Vb;
    V* const Wv = sc.Wv;
    V* const pr = sc.pr;
    V* const pc = sc.pc;
    const V zero = mk(T(0), T(0));
    const V* V_ = Vb + (k & 1) * NMAX;        // v_k (entry k+1 is vfirst)
    V* Vn = Vb + ((k + 1) & 1) * NMAX;        // v_{k+1}
    const int j0 = k + 1;
    const int m = n - j0;

    // ---- p = tau A v (thread ri combines the row and per-warp column
    // partial sums of entry ri) and the partial sums of v^H p.
    const int ri = tid;
    const bool mine = ri < m;
    const int nact = (m + 31) >> 5;  // warps holding entries
    V v = zero, p = zero;
    if (warp < nact) {
        T sp = T(0);
        if (mine) {
            p = pr[ri];
#pragma unroll
            for (int w = 0; w < NW; ++w) p = cadd(p, pc[w * NMAX + ri]);
            p.x *= tau; p.y *= tau;
            v = ri == 0 ? vfirst : V_[j0 + ri];
            pr[ri] = p;
            sp = v.x * p.x + v.y * p.y;
        }
        sp = warp_sum(sp);
        if (lane == 0) sc.redA[warp] = sp;
    }
    __syncthreads();

    // ---- w = p - (tau s / 2) v, the explicit update of pivot column
    // j0 with (v_k, w_k), d_j0, and the partial sums of ||x||^2 for the
    // next reflector, whose entries past the first go to Vn.
    if (warp < nact) {
        const T K = T(0.5) * tau * sum_partials<T, NW>(sc.redA, nact);
        const V p0 = pr[0];
        const V w0 = mk(p0.x - K * vfirst.x, p0.y - K * vfirst.y);
        T s2p = T(0);
        if (mine) {
            const V w = mk(p.x - K * v.x, p.y - K * v.y);
            Wv[j0 + ri] = w;
            V a = A[tri(j0 + ri) + j0];
            a = cfms_conj_b(v, w0, a);
            a = cfms_conj_b(w, vfirst, a);
            if (ri == 0) d[j0] = double(a.x);
            if (ri >= 1) s2p = cabs2(a);
            if (ri >= 2) Vn[j0 + ri] = a;
            if (ri == 1) sc.sx[0] = a;
        }
        s2p = warp_sum(s2p);
        if (lane == 0) sc.redB[warp] = s2p;
    }
    __syncthreads();

    // ---- ||x||^2, and the next reflector's first entry and tau.
    if constexpr (kSharedTail) {
        if (warp == 0) {
            const T s2 = sum_partials<T, NW>(sc.redB, nact);
            if (lane == 0) e2[j0] = double(s2);
            if (k + 1 <= n - 3) {
                V f;
                T tn;
                reflector_head(s2, sc.sx[0], f, tn);
                if (lane == 0) { sc.sx[1] = f; sc.sx[2] = mk(tn, T(0)); }
            }
        }
        __syncthreads();
        if (k + 1 <= n - 3) { vfirst = sc.sx[1]; tau = sc.sx[2].x; }
    } else {
        const T s2 = sum_partials<T, NW>(sc.redB, nact);
        if (tid == 0) e2[j0] = double(s2);
        if (k + 1 <= n - 3) reflector_head(s2, sc.sx[0], vfirst, tau);
    }
}

template <typename T, int NMAX>
__device__ __forceinline__ void hh_finish(int n, cplx_t<T>* A, const HHScratch<T>& sc, double* d) {
    using V = cplx_t<T>;
    // Step n-3's update of the last diagonal entry.
    if (threadIdx.x == 0) {
        const V v = sc.Vb[((n - 3) & 1) * NMAX + n - 1];
        const V w = sc.Wv[n - 1];
        const T ann = A[tri(n - 1) + n - 1].x - T(2) * (v.x * w.x + v.y * w.y);
        d[n - 1] = double(ann);
    }
    __syncthreads();
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
    V vfirst;
    T tau;
    if (!hh_setup<T, NW, NMAX>(n, A, sc, d, e2, vfirst, tau)) return;

    for (int k = 0; k <= n - 3; ++k) {
        const V* V_ = Vb + (k & 1) * NMAX;        // v_k (entry k+1 is vfirst)
        const V* U_ = Vb + ((k + 1) & 1) * NMAX;  // v_{k-1} (zero at k = 0); v_{k+1} replaces it later
        const int j0 = k + 1;                     // first active row/column

        // ---- fused pass: A <- A - u w^H - w u^H (step k-1), accumulate A v_k.
        // Indices are relative to the active corner j0.  The trailing rows
        // are cut into batches of RB consecutive rows, dealt to the warps in
        // snake order (balanced work); lane l handles relative columns
        // l + 32 t.  Per chunk t the RB elements of a lane are independent and
        // branch-free (masked loads and stores), so their loads and FMA chains
        // overlap.  At k = 0, u and w are zero and the update is a no-op.
        constexpr int RB = PassRows<T>::value;
        const int m = n - j0;
        const int nbatch = (m + RB - 1) / RB;
        V vc[NT], uc[NT], wc[NT], cacc[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int j = j0 + 32 * t + lane;
            const bool in = j < n;
            vc[t] = in ? V_[j] : zero;
            uc[t] = in ? U_[j] : zero;
            wc[t] = in ? Wv[j] : zero;
            cacc[t] = zero;
        }
        if (lane == 0) vc[0] = vfirst;
        for (int round = 0;; ++round) {
            // Heaviest batches first, snake order over the warps.
            const int slot = round * NW + ((round & 1) ? (NW - 1 - warp) : warp);
            if (slot >= nbatch) break;
            const int b = nbatch - 1 - slot;
            const int ri0 = b * RB;
            V ui[RB], wi[RB], vi[RB], racc[RB];
            int base[RB];
            const bool full_rows = ri0 + RB - 1 < m;
            if (full_rows) {
                int bi = tri(j0 + ri0) + j0;
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int i = j0 + ri0 + r;
                    ui[r] = U_[i];
                    wi[r] = Wv[i];
                    vi[r] = V_[i];
                    base[r] = bi;
                    bi += i + 1;
                    racc[r] = zero;
                }
            } else {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int ri = ri0 + r;
                    const bool ok = ri < m;
                    const int i = j0 + ri;
                    ui[r] = ok ? U_[i] : zero;
                    wi[r] = ok ? Wv[i] : zero;
                    vi[r] = ok ? V_[i] : zero;
                    base[r] = ok ? tri(i) + j0 : 0;
                    racc[r] = zero;
                }
            }
            if (ri0 == 0) vi[0] = vfirst;
            const int last = (ri0 + RB - 1 < m ? ri0 + RB - 1 : m - 1);
            const int nch = (last >> 5) + 1;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (t < nch) {
                    const int jr = 32 * t + lane;
                    if (full_rows && 32 * t + 31 < ri0) {
                        // Chunk strictly below the diagonal for every row of a
                        // full batch: no masks.
#pragma unroll
                        for (int r = 0; r < RB; ++r) {
                            V a = A[base[r] + jr];
                            a = cfms_conj_b(ui[r], wc[t], a);
                            a = cfms_conj_b(wi[r], uc[t], a);
                            A[base[r] + jr] = a;
                            racc[r] = cfma(a, vc[t], racc[r]);
                            cacc[t] = cfma_conj_a(a, vi[r], cacc[t]);
                        }
                        continue;
                    }
                    // Diagonal chunk: lane jr holds element (ri, jr) for
                    // jr <= ri.  A masked lane still loads base + jr -- at
                    // most 31 elements past the packed triangle's end, which
                    // the matrix buffers are padded for -- and its value,
                    // possibly stale or non-finite, is replaced by zero
                    // before both sums.  The diagonal's imaginary part is
                    // mathematically zero under the update and only its real
                    // part is ever read.  With s = jr - ri0, the lane holds an
                    // element of row ri0 + r iff s <= r (below the diagonal
                    // iff s < r), and rows from nr = m - ri0 on do not exist.
                    const int sl = jr - ri0, nr = m - ri0;
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const bool ok = (sl <= r) && (r < nr);
                        V a = A[base[r] + jr];
                        a = cfms_conj_b(ui[r], wc[t], a);
                        a = cfms_conj_b(wi[r], uc[t], a);
                        if (ok) A[base[r] + jr] = a;
                        a = ok ? a : zero;
                        racc[r] = cfma(a, vc[t], racc[r]);
                        const V vrow = (sl < r) ? vi[r] : zero;
                        cacc[t] = cfma_conj_a(a, vrow, cacc[t]);
                    }
                }
            }
            V out;
            if constexpr (RB == 8) {
                out = reduce_scatter8(racc, lane);
                const int ri = ri0 + ((lane >> 2) & 7);
                if ((lane & 3) == 0 && ri < m) pr[ri] = out;
            } else if constexpr (RB == 4) {
                out = reduce_scatter4(racc, lane);
                const int ri = ri0 + ((lane >> 3) & 3);
                if ((lane & 7) == 0 && ri < m) pr[ri] = out;
            } else {
                out = reduce_scatter2(racc, lane);
                const int ri = ri0 + ((lane >> 4) & 1);
                if ((lane & 15) == 0 && ri < m) pr[ri] = out;
            }
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int jr = 32 * t + lane;
            if (jr < m) pc[warp * NMAX + jr] = cacc[t];
        }
        __syncthreads();

        hh_scalar<T, NW, NMAX>(k, n, A, sc, d, e2, vfirst, tau);
    }
    hh_finish<T, NMAX>(n, A, sc, d);
}

// The same reduction for matrices too large for shared memory (n up to
// 32 NW, the paper's large traveling clusters): A lives in the CTA's global
// slot (L1/L2 resident), the vectors in shared memory.  The fused pass is the
// plain form of the one above: warp w takes rows m-1-w, m-1-w-NW, ... (the
// longest first), lane l the columns l, l+32, ... of the row; each element is
// updated with the previous step's (u, w), stored, and contributes to its
// row's sum (reduced across the warp) and, below the diagonal, to its
// column's sum in the warp's own partial row (lanes own distinct columns, so
// the order of the additions is fixed).  Between passes the scalar phases are
// those of householder_tridiag.
template <typename T, int NW>
__device__ void householder_tridiag_large(int n, cplx_t<T>* A, const HHScratch<T>& sc, double* d, double* e2) {
    using V = cplx_t<T>;
    constexpr int NMAX = 32 * NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    V* const Vb = sc.Vb;
    V* const Wv = sc.Wv;
    V* const pr = sc.pr;
    V* const pcw = sc.pc + warp * NMAX;
    const V zero = mk(T(0), T(0));
    V vfirst;
    T tau;
    if (!hh_setup<T, NW, NMAX>(n, A, sc, d, e2, vfirst, tau)) return;

    for (int k = 0; k <= n - 3; ++k) {
        const V* V_ = Vb + (k & 1) * NMAX;        // v_k (entry k+1 is vfirst)
        const V* U_ = Vb + ((k + 1) & 1) * NMAX;  // v_{k-1} (zero at k = 0)
        const int j0 = k + 1, m = n - j0;
        for (int jr = lane; jr < m; jr += 32) pcw[jr] = zero;
        for (int r = warp; r < m; r += NW) {
            const int ri = m - 1 - r, i = j0 + ri;
            const V ui = U_[i], wi = Wv[i], vi = ri == 0 ? vfirst : V_[i];
            V* row = A + tri(i) + j0;
            V racc = zero;
            // Four columns per lane at a time: their global loads are issued
            // together (the additions keep the column order).
            constexpr int LU = 4;
            for (int jb = 0; jb <= ri; jb += 32 * LU) {
                V av[LU];
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
                        const V vj = jr == 0 ? vfirst : V_[j];
                        V a = av[q];
                        a = cfms_conj_b(ui, Wv[j], a);
                        a = cfms_conj_b(wi, U_[j], a);
                        row[jr] = a;
                        racc = cfma(a, vj, racc);
                        if (jr < ri) pcw[jr] = cfma_conj_a(a, vi, pcw[jr]);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) racc = cadd(racc, cshfl_xor(racc, o));
            if (lane == 0) pr[ri] = racc;
        }
        __syncthreads();
        hh_scalar<T, NW, NMAX>(k, n, A, sc, d, e2, vfirst, tau);
    }
    hh_finish<T, NMAX>(n, A, sc, d);
}

// ---------------------------------------------------------------------------
// Tridiagonal eigenvalues.  Sturm count: number of eigenvalues below x from
// the pivots q_0 = d_0 - x, q_i = (d_i - x) - e2_{i-1}/q_{i-1}, a pivot of
// magnitude below pivmin replaced by -pivmin (Barth, Martin and Wilkinson's
// bisection with Kahan's safeguard).
// ---------------------------------------------------------------------------

// FP64 reciprocal by Newton-Raphson: an FP32 reciprocal as seed, then
// r <- r + r (1 - q r) twice (error squares each time: 2^-22 -> 2^-44 ->
// below FP64 rounding).  Outside the FP32 range the plain quotient is used.
__device__ __forceinline__ double rcp64(double q) {
    const double aq = fabs(q);
    if (aq > 1e-30 && aq < 1e30) {
        double r = (double)__fdividef(1.0f, (float)q);
        double e = __fma_rn(-q, r, 1.0);
        r = __fma_rn(r, e, r);
        e = __fma_rn(-q, r, 1.0);
        return __fma_rn(r, e, r);
    }
    return 1.0 / q;
}

__device__ __forceinline__ int sturm_count_f64(int n, const double* d, const double* e2, double x, double pivmin) {
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    int c = q < 0.0;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e2[i - 1] * rcp64(q);
        if (fabs(q) < pivmin) q = -pivmin;
        c += q < 0.0;
    }
    return c;
}

// 2^-e with e the exponent of the largest |value| among a, b, c, d: scaling a
// sequence by it is exact and keeps its entries near 1 in magnitude.
__device__ __forceinline__ float pow2_rescale(float a, float b, float c = 0.f, float d = 0.f) {
    const float m = fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(c), fabsf(d)));
    int fe = 254 - (int)((__float_as_uint(m) >> 23) & 0xffu);  // biased exponent of 2^-e
    fe = fe < 1 ? 1 : (fe > 254 ? 254 : fe);
    return __uint_as_float((unsigned)fe << 23);
}

// FP32 Sturm count, pivot form (Barth, Martin and Wilkinson's bisection with
// Kahan's pivot guard).  Run by every thread of the CTA at once in the
// multisection, it is throughput bound: its reciprocal goes to the separate
// MUFU pipe, which measured faster here than the division-free three-term
// recurrence with its extra ALU work.
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

// One FP64 pass of the pivot recurrence at x: the Sturm count and the
// logarithmic derivative s = sum_i q_i'/q_i of det(T - x) = prod_i q_i, with
// q_0' = -1 and q_i' = -1 + e2_{i-1} q_{i-1}' / q_{i-1}^2.
__device__ __forceinline__ int newton_pass_f64(int n, const double* d, const double* e2, double x, double pivmin,
                                               double& s) {
    double q = d[0] - x, dq = -1.0;
    if (fabs(q) < pivmin) q = -pivmin;
    int c = q < 0.0;
    double acc = 0.0;
    for (int i = 1; i < n; ++i) {
        const double r = rcp64(q);
        acc = __fma_rn(dq, r, acc);
        const double er = e2[i - 1] * r;
        double qn = (d[i] - x) - er;
        dq = __fma_rn(er * r, dq, -1.0);
        if (fabs(qn) < pivmin) qn = -pivmin;
        q = qn;
        c += q < 0.0;
    }
    s = __fma_rn(dq, rcp64(q), acc);
    return c;
}

// Safeguarded Newton on det(T - x) for the k-th smallest eigenvalue (0-based)
// inside [lo, hi], whose Sturm counts are clo <= k < chi, starting at x: a
// Newton step is taken while the bracket holds exactly this one eigenvalue
// and the step stays inside it and at least halves the previous width;
// otherwise the bracket is bisected.  Every pass tightens the bracket with
// its Sturm count.
__device__ __forceinline__ double eig_f64_newton(int n, const double* d, const double* e2, int k, double lo, double hi,
                                                 int clo, int chi, double x, double pivmin, double nrm) {
    const double tol = 2.0 * DBL_EPSILON * nrm;
    double width_before = hi - lo;
    for (int it = 0; it < 96 && hi - lo > tol; ++it) {
        double s;
        const int c = newton_pass_f64(n, d, e2, x, pivmin, s);
        if (c <= k) { lo = x; clo = c; } else { hi = x; chi = c; }
        double xn = 0.5 * (lo + hi);
        if (chi - clo == 1 && s != 0.0 && isfinite(s)) {
            const double cand = x - 1.0 / s;
            // A step below the tolerance means convergence: once x has
            // converged it is itself a bracket end, so the candidate can no
            // longer lie strictly inside and must not trigger a bisection.
            if (fabs(cand - x) <= tol) return fmin(fmax(cand, lo), hi);
            if (cand > lo && cand < hi && 2.0 * fabs(cand - x) <= width_before) xn = cand;
        }
        width_before = hi - lo;
        x = xn;
    }
    return x;
}

// k-th smallest eigenvalue, all FP64: bisection from the Gershgorin bracket
// down to a width of ~1e-6 ||T||, then safeguarded Newton.
__device__ __forceinline__ double eig_f64(int n, const double* d, const double* e2, int k, double lo, double hi,
                                          double pivmin, double nrm) {
    const double coarse = 1e-6 * nrm;
    int clo = 0, chi = n;
    for (int it = 0; it < 64 && hi - lo > coarse; ++it) {
        const double mid = 0.5 * (lo + hi);
        const int c = sturm_count_f64(n, d, e2, mid, pivmin);
        if (c <= k) { lo = mid; clo = c; } else { hi = mid; chi = c; }
    }
    return eig_f64_newton(n, d, e2, k, lo, hi, clo, chi, 0.5 * (lo + hi), pivmin, nrm);
}

// k-th smallest eigenvalue in FP64 from the FP32 multisection bracket
// [blo, bhi] of the FP32-rounded (d, e2).  Rounding the entries to FP32 and
// the FP32 Sturm counts move an eigenvalue by a few FP32 ulps of ||T||
// (Weyl's bound on the perturbation), so the bracket is widened by `margin`
// and confirmed with two FP64 Sturm counts before safeguarded Newton
// finishes it; if the confirmation fails the full FP64 bisection runs.
__device__ __forceinline__ double eig_f64_bracketed(int n, const double* d, const double* e2, int k, float blo,
                                                    float bhi, double margin, double lo, double hi, double pivmin,
                                                    double nrm) {
    const double a = fmax((double)blo - margin, lo), b = fmin((double)bhi + margin, hi);
    const int ca = sturm_count_f64(n, d, e2, a, pivmin);
    const int cb = sturm_count_f64(n, d, e2, b, pivmin);
    if (a < b && ca <= k && cb > k)
        return eig_f64_newton(n, d, e2, k, a, b, ca, cb, 0.5 * ((double)blo + (double)bhi), pivmin, nrm);
    return eig_f64(n, d, e2, k, lo, hi, pivmin, nrm);
}

// ---------------------------------------------------------------------------
// The same refinements in double-float arithmetic: FP64-class precision on
// the FP32 pipe.  The tridiagonal is given as float pairs (dh + dl, eh + el),
// exact copies of the FP64 entries.
// ---------------------------------------------------------------------------

// Double-float Sturm count from the leading principal minors
//   p_-1 = 1, p_0 = d_0 - x, p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2}:
// the number of sign changes along p_-1 .. p_{n-1} is the number of
// eigenvalues below x (p_i / p_{i-1} is the pivot of the LDL^T factors).  No
// division: each step is one two-product sum with a single renormalisation.
// Every 8 steps the pair is rescaled by a power of two (exact), keeping it in
// the float range; a minor that is exactly zero takes a tiny value of the
// sign opposite to its predecessor (as Kahan's guard counts a zero pivot as
// negative).
__device__ __forceinline__ int sturm_count_df(int n, const float* dh, const float* dl, const float* eh,
                                              const float* el, dfl x, float pivmin) {
    dfl p2 = dfl(1.f, 0.f), p1 = dfl(dh[0], dl[0]) - x;
    if (p1.hi == 0.f) p1 = dfl(-pivmin, 0.f);
    int c = (int)(__float_as_uint(p1.hi) >> 31);
    for (int i = 1; i < n; ++i) {
        const dfl dx = dfl(dh[i], dl[i]) - x;
        dfl p = dot2_acc(dfl(0.f, 0.f), dx, p1, -dfl(eh[i - 1], el[i - 1]), p2);
        if (p.hi == 0.f) p = dfl(-1e-30f * p1.hi, 0.f);
        c += (int)((__float_as_uint(p.hi) ^ __float_as_uint(p1.hi)) >> 31);
        p2 = p1;
        p1 = p;
        if ((i & 7) == 0) {
            const float sc = pow2_rescale(p1.hi, p2.hi);
            p1 = dfl(p1.hi * sc, p1.lo * sc);
            p2 = dfl(p2.hi * sc, p2.lo * sc);
        }
    }
    return c;
}

// Sturm count and logarithmic derivative s = p'/p of det(T - x), as
// newton_pass_f64.  The minors p_i run in double-float: near an eigenvalue
// p_{n-1} is small and must be resolved far below FP32.  Their derivatives
//   p'_i = (d_i - x) p'_{i-1} - p_{i-1} - e2_{i-1} p'_{i-2}
// run in FP32 on the leading parts: s only sets a Newton correction of size
// ~1e-6 ||T||, so its FP32 relative error moves the result by ~1e-12 ||T||.
// Minors and derivatives share the power-of-two rescaling, which leaves s
// unchanged.
__device__ __forceinline__ int newton_pass_df(int n, const float* dh, const float* dl, const float* eh,
                                              const float* el, dfl x, float pivmin, double& s) {
    dfl p2 = dfl(1.f, 0.f), p1 = dfl(dh[0], dl[0]) - x;
    float dp2 = 0.f, dp1 = -1.f;
    if (p1.hi == 0.f) p1 = dfl(-pivmin, 0.f);
    int c = (int)(__float_as_uint(p1.hi) >> 31);
    for (int i = 1; i < n; ++i) {
        const dfl dx = dfl(dh[i], dl[i]) - x;
        const float e2 = eh[i - 1];
        dfl p = dot2_acc(dfl(0.f, 0.f), dx, p1, -dfl(e2, el[i - 1]), p2);
        const float dp = __fmaf_rn(dx.hi, dp1, __fmaf_rn(-e2, dp2, -p1.hi));
        if (p.hi == 0.f) p = dfl(-1e-30f * p1.hi, 0.f);
        c += (int)((__float_as_uint(p.hi) ^ __float_as_uint(p1.hi)) >> 31);
        p2 = p1;
        p1 = p;
        dp2 = dp1;
        dp1 = dp;
        if ((i & 7) == 0) {
            const float sc = pow2_rescale(p1.hi, p2.hi, dp1, dp2);
            p1 = dfl(p1.hi * sc, p1.lo * sc);
            p2 = dfl(p2.hi * sc, p2.lo * sc);
            dp1 *= sc;
            dp2 *= sc;
        }
    }
    s = (double)dp1 / double(p1);
    return c;
}

// Safeguarded Newton as eig_f64_newton, passes in double-float; converged
// when a step falls below 1e-13 ||T|| (the double-float resolution).
__device__ __forceinline__ double eig_df_newton(int n, const float* dh, const float* dl, const float* eh,
                                                const float* el, int k, double lo, double hi, int clo, int chi,
                                                double x, float pivmin, double nrm) {
    const double tol = 1e-13 * nrm;
    double width_before = hi - lo;
    for (int it = 0; it < 96 && hi - lo > tol; ++it) {
        double s;
        const int c = newton_pass_df(n, dh, dl, eh, el, dfl(x), pivmin, s);
        if (c <= k) { lo = x; clo = c; } else { hi = x; chi = c; }
        double xn = 0.5 * (lo + hi);
        if (chi - clo == 1 && s != 0.0 && isfinite(s)) {
            const double cand = x - 1.0 / s;
            if (fabs(cand - x) <= tol) return fmin(fmax(cand, lo), hi);
            if (cand > lo && cand < hi && 2.0 * fabs(cand - x) <= width_before) xn = cand;
        }
        width_before = hi - lo;
        x = xn;
    }
    return x;
}

// k-th eigenvalue from the FP32 multisection bracket, as eig_f64_bracketed:
// widened, confirmed by two double-float Sturm counts, finished by Newton;
// the fallback bisects from the Gershgorin bracket.
__device__ __forceinline__ double eig_df_bracketed(int n, const float* dh, const float* dl, const float* eh,
                                                   const float* el, int k, float blo, float bhi, double margin,
                                                   double lo, double hi, float pivmin, double nrm) {
    double a = fmax((double)blo - margin, lo), b = fmin((double)bhi + margin, hi);
    int ca = sturm_count_df(n, dh, dl, eh, el, dfl(a), pivmin);
    int cb = sturm_count_df(n, dh, dl, eh, el, dfl(b), pivmin);
    if (!(a < b && ca <= k && cb > k)) {
        a = lo; b = hi; ca = 0; cb = n;
        for (int it = 0; it < 64 && b - a > 1e-6 * nrm; ++it) {
            const double mid = 0.5 * (a + b);
            const int c = sturm_count_df(n, dh, dl, eh, el, dfl(mid), pivmin);
            if (c <= k) { a = mid; ca = c; } else { b = mid; cb = c; }
        }
        return eig_df_newton(n, dh, dl, eh, el, k, a, b, ca, cb, 0.5 * (a + b), pivmin, nrm);
    }
    return eig_df_newton(n, dh, dl, eh, el, k, a, b, ca, cb, 0.5 * ((double)blo + (double)bhi), pivmin, nrm);
}

// One double-float Newton correction of an eigenvalue located by FP32
// multisection in [lo, hi]; kept only if it stays near that bracket.
__device__ __forceinline__ double newton_polish_df(int n, const float* dh, const float* dl, const float* eh,
                                                   const float* el, float lo, float hi, float atolf, float pivmin) {
    const double x = 0.5 * ((double)lo + (double)hi);
    double s;
    newton_pass_df(n, dh, dl, eh, el, dfl(x), pivmin, s);
    const double xn = x - 1.0 / s;
    const double w = fmax((double)(hi - lo), 4.0 * (double)atolf);
    if (isfinite(xn) && xn >= (double)lo - w && xn <= (double)hi + w) return xn;
    return x;
}

// softplus(x) = ln(1 + e^x), written as max(x,0) + log1p(e^-|x|).
__device__ __forceinline__ double softplus(double x) { return fmax(x, 0.0) + log1p(exp(-fabs(x))); }

}  // namespace ptca
