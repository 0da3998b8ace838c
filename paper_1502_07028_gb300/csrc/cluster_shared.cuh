// cluster_shared.cuh -- one Householder reduction for both matrices of a visit
// (FP32, one 4-warp CTA per update site, orders up to 128).
//
// H_new differs from H_old only in the update site's 2x2 on-site block (the
// proposal changes one classical vector, Sec. II.c step c; hopping does not
// depend on it).  In a basis where the update site's two vectors come first,
// H_new = H_old + E with E confined to the leading 2x2 block.  A block
// Householder reduction with 2-column panels that starts below that block
// never reads it: panel j's two reflectors come from rows 2j+2.. of columns
// 2j, 2j+1, and every update acts on rows and columns >= 2j+2.  So one
// reduction gives the band (bandwidth 2, 2x2 block tridiagonal) of both
// matrices, which differ only in their leading block.  Each band is then
// brought to real tridiagonal form by Givens rotations (a bulge chase) and
// solved by the eigenvalue phase of the other reductions.  The O(n^3) work of
// a visit is done once instead of twice.
//
// Reduction (panel j, rows/columns from r0 = 2j+2): the panel's QR gives
// reflectors v1 (rows r0..), v2 (rows r0+1..) with unit first entries,
// stored in place below R (R11 at (r0, 2j), R12 at (r0, 2j+1), R22 at
// (r0+1, 2j+1)).  With Q = (I - t1 v1 v1^H)(I - t2 v2 v2^H) = I - V T V^H,
// T = [[t1, -t1 t2 v1^H v2], [0, t2]], the trailing block becomes
// A - V W^H - W V^H with P = A V, Y = P T, W = Y - V (T^H V^H Y) / 2.  As in
// the one-column reductions, panel j-1's rank-4 update is deferred and fused
// with panel j's products (one read and write of the trailing triangle per
// panel), and the next panel's two columns receive their update explicitly.
//
// Storage: the packed lower triangle of rows 2..n-1 (element (i, j) at
// tri(i) + j - 3), the two w vectors, per-warp partial sums of the two
// products (each warp's row sums folded into its own partial vector), and
// the block-sum slots: 76.5 KB at n = 128, three CTAs per SM.
#pragma once

#include "kernels.cuh"

namespace ptca {

constexpr int SH_NW = 4;              // warps per CTA
constexpr int SH_NT = 4;              // 32-column chunks per lane
constexpr int SH_NMAX = 32 * SH_NT;   // largest order
constexpr int SH_RB = 4;              // rows per batch of the fused pass

__host__ __device__ __forceinline__ int sh_at(int i, int j) { return ((i * (i + 1)) >> 1) + j - 3; }

struct ShLayout { size_t M, W, pc, red, total; };
__host__ __device__ inline ShLayout sh_layout() {
    ShLayout L;
    size_t o = 0;
    L.M = o;   o = align16(o + (size_t)((SH_NMAX * (SH_NMAX + 1)) / 2 - 3) * sizeof(float2));
    L.W = o;   o = align16(o + 2 * (size_t)SH_NMAX * sizeof(float2));
    L.pc = o;  o = align16(o + 2 * (size_t)SH_NW * SH_NMAX * sizeof(float2));
    L.red = o; o = align16(o + 64 * sizeof(float));
    L.total = o;
    return L;
}

__device__ __forceinline__ float2 sh_mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) b
__device__ __forceinline__ float2 sh_cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 sh_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 sh_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Reflector with unit first entry for x (||x||^2 = s2, first entry x0):
// v = x / v0, v0 = x0 + phase(x0) ||x||, tau = |v0|^2 / (||x|| (||x|| + |x0|)),
// (I - tau v v^H) x = beta e_1, beta = -phase(x0) ||x||.  rv0 = 1 / v0; x = 0
// gives tau = 0.
__device__ __forceinline__ void sh_head(float s2, float2 x0, float2& rv0, float& tau, float2& beta) {
    const float sigma = s2 > 0.f ? sqrtf(s2) : 0.f;
    const float ax = sqrtf(x0.x * x0.x + x0.y * x0.y);
    const float2 ph = ax > 0.f ? make_float2(x0.x / ax, x0.y / ax) : make_float2(1.f, 0.f);
    const float2 v0 = make_float2(x0.x + ph.x * sigma, x0.y + ph.y * sigma);
    const float a0 = v0.x * v0.x + v0.y * v0.y;
    if (sigma > 0.f) {
        tau = a0 / (sigma * (sigma + ax));
        rv0 = make_float2(v0.x / a0, -v0.y / a0);
    } else {
        tau = 0.f;
        rv0 = make_float2(0.f, 0.f);
    }
    beta = make_float2(-ph.x * sigma, -ph.y * sigma);
}

// H_old of a visit in the basis where the update site (window index uw)
// trades places with window site 0: rows 2..n-1 of the packed lower triangle
// into M, the window's (old) vectors into sp[nsite][3].  Thread 0 receives the
// update site's on-site block for the old and the proposed vector s_new:
// t11[4 var + (0, 1, 2, 3)] = (H_00, H_11, Re H_10, Im H_10).  The entries
// are those of build_cluster (FP32).  Caller syncs after.
__device__ void build_cluster_shared(const Model& m, const Window& w, const double* __restrict__ S,
                                     const double* s_new, double* sp, float2* M, float* t11) {
    const int nsite = window_nsite(w), n = 2 * nsite, exy = w.ex * w.ey;
    const int P = ((n * (n + 1)) >> 1) - 3;
    for (int i = threadIdx.x; i < P; i += blockDim.x) M[i] = make_float2(0.f, 0.f);
    const int uw = (w.uwz * w.ey + w.uwy) * w.ex + w.uwx;
    for (int s = threadIdx.x; s < nsite; s += blockDim.x) {
        const int wx = s % w.ex, wy = (s / w.ex) % w.ey, wz = s / exy;
        const int g = window_site(m, w, wx, wy, wz);
        sp[3 * s] = S[3 * g]; sp[3 * s + 1] = S[3 * g + 1]; sp[3 * s + 2] = S[3 * g + 2];
    }
    __syncthreads();
    const float t = float(m.t), J = float(m.JH), lam = float(m.lam);
    auto phi = [uw](int s) { return s == uw ? 0 : (s == 0 ? uw : s); };
    auto bond = [&](int s, int nb, int mult) {
        const int ps = phi(s), pn = phi(nb);
        const int hi = pn > ps ? pn : ps, lo = pn > ps ? ps : pn;
        for (int sg = 0; sg < 2; ++sg) M[sh_at(2 * hi + sg, 2 * lo + sg)] = make_float2(-float(mult) * t, 0.f);
    };
    for (int s = threadIdx.x; s < nsite; s += blockDim.x) {
        const int wx = s % w.ex, wy = (s / w.ex) % w.ey, wz = s / exy;
        if (s != uw) {
            const float sx = float(sp[3 * s]), sy = float(sp[3 * s + 1]), sz = float(sp[3 * s + 2]);
            const int a = 2 * phi(s), b = a + 1;
            const float dg = lam * sx;
            M[sh_at(a, a)] = make_float2(dg - J * sz, 0.f);
            M[sh_at(b, b)] = make_float2(dg + J * sz, 0.f);
            M[sh_at(b, a)] = make_float2(-J * sx, -J * sy);
        }
        int nb = -1, mult = 1;
        if (wx + 1 < w.ex) { nb = s + 1; if (m.cluster_periodic && w.ex == 2) mult = 2; }
        else if (m.cluster_periodic && w.ex >= 3) nb = s - (w.ex - 1);
        if (nb >= 0) bond(s, nb, mult);
        nb = -1; mult = 1;
        if (wy + 1 < w.ey) { nb = s + w.ex; if (m.cluster_periodic && w.ey == 2) mult = 2; }
        else if (m.cluster_periodic && w.ey >= 3) nb = s - (w.ey - 1) * w.ex;
        if (nb >= 0) bond(s, nb, mult);
        nb = -1; mult = 1;
        if (wz + 1 < w.ez) { nb = s + exy; if (m.cluster_periodic && w.ez == 2) mult = 2; }
        else if (m.cluster_periodic && w.ez >= 3) nb = s - (w.ez - 1) * exy;
        if (nb >= 0) bond(s, nb, mult);
    }
    if (threadIdx.x == 0) {
        for (int var = 0; var < 2; ++var) {
            const double* v = var ? s_new : sp + 3 * uw;
            const float sx = float(v[0]), sy = float(v[1]), sz = float(v[2]);
            const float dg = lam * sx;
            t11[4 * var] = dg - J * sz;
            t11[4 * var + 1] = dg + J * sz;
            t11[4 * var + 2] = -J * sx;
            t11[4 * var + 3] = -J * sy;
        }
    }
}

// Panel j's fused pass over the trailing block (rows and columns from
// r0 = 2j+2): A <- A - U W^H - W U^H with panel j-1's reflectors U and w
// vectors W (skipped at j = 0), then the products A V with panel j's
// reflectors, into this warp's two partial vectors pc[2 warp + b] (row sums
// of the warp's rows plus its column sums).  Rows are dealt in batches of
// SH_RB, heaviest first, in snake order over the warps; lane l takes the
// columns l + 32 t.  Ends with a CTA barrier.
__device__ __forceinline__ void sh_pass(int n, int j, float2* M, const float2* Wv, float2* pc) {
    constexpr int NT = SH_NT, RB = SH_RB, NW_ = SH_NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = 2 * j + 2, m = n - r0, c1 = 2 * j, c2 = 2 * j + 1;
    const bool upd = j > 0;
    const float2 zero = make_float2(0.f, 0.f), one = make_float2(1.f, 0.f);
    float2* pw = pc + 2 * warp * SH_NMAX;
    for (int x = lane; x < m; x += 32) { pw[x] = zero; pw[SH_NMAX + x] = zero; }
    __syncwarp();
    float2 vc1[NT], vc2[NT], uc1[NT], uc2[NT], wc1[NT], wc2[NT], ca1[NT], ca2[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int x = 32 * t + lane, y = r0 + x;
        const bool in = x < m;
        vc1[t] = !in ? zero : (x == 0 ? one : M[sh_at(y, c1)]);
        vc2[t] = !in ? zero : (x == 0 ? zero : (x == 1 ? one : M[sh_at(y, c2)]));
        uc1[t] = in && upd ? M[sh_at(y, c1 - 2)] : zero;
        uc2[t] = in && upd ? M[sh_at(y, c2 - 2)] : zero;
        wc1[t] = in && upd ? Wv[y] : zero;
        wc2[t] = in && upd ? Wv[SH_NMAX + y] : zero;
        ca1[t] = zero;
        ca2[t] = zero;
    }
    const int nbatch = (m + RB - 1) / RB;
    for (int round = 0;; ++round) {
        const int slot = round * NW_ + ((round & 1) ? (NW_ - 1 - warp) : warp);
        if (slot >= nbatch) break;
        const int ri0 = (nbatch - 1 - slot) * RB;
        float2 ui1[RB], ui2[RB], wi1[RB], wi2[RB], vi1[RB], vi2[RB], ra[2 * RB];
        int base[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int ri = ri0 + r, y = r0 + ri;
            const bool ok = ri < m;
            ui1[r] = ok && upd ? M[sh_at(y, c1 - 2)] : zero;
            ui2[r] = ok && upd ? M[sh_at(y, c2 - 2)] : zero;
            wi1[r] = ok && upd ? Wv[y] : zero;
            wi2[r] = ok && upd ? Wv[SH_NMAX + y] : zero;
            vi1[r] = !ok ? zero : (ri == 0 ? one : M[sh_at(y, c1)]);
            vi2[r] = !ok ? zero : (ri == 0 ? zero : (ri == 1 ? one : M[sh_at(y, c2)]));
            base[r] = ok ? sh_at(y, r0) : 0;
            ra[2 * r] = zero;
            ra[2 * r + 1] = zero;
        }
        const bool full_rows = ri0 + RB - 1 < m;
        const int last = ri0 + RB - 1 < m ? ri0 + RB - 1 : m - 1;
        const int nch = (last >> 5) + 1;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (t < nch) {
                const int x = 32 * t + lane;
                if (full_rows && 32 * t + 31 < ri0) {
                    // every element of the chunk lies strictly below the diagonal
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        float2 a = M[base[r] + x];
                        if (upd) {
                            a = cfms_conj_b(ui1[r], wc1[t], a);
                            a = cfms_conj_b(wi1[r], uc1[t], a);
                            a = cfms_conj_b(ui2[r], wc2[t], a);
                            a = cfms_conj_b(wi2[r], uc2[t], a);
                            M[base[r] + x] = a;
                        }
                        ra[2 * r] = cfma(a, vc1[t], ra[2 * r]);
                        ra[2 * r + 1] = cfma(a, vc2[t], ra[2 * r + 1]);
                        ca1[t] = cfma_conj_a(a, vi1[r], ca1[t]);
                        ca2[t] = cfma_conj_a(a, vi2[r], ca2[t]);
                    }
                    continue;
                }
                // Diagonal chunk: lane x holds element (ri0 + r, x) iff
                // x - ri0 <= r (below the diagonal iff <) and the row exists.
                const int sl = x - ri0, nr = m - ri0;
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const bool ok = (sl <= r) && (r < nr);
                    float2 a = ok ? M[base[r] + x] : zero;
                    if (upd) {
                        a = cfms_conj_b(ui1[r], wc1[t], a);
                        a = cfms_conj_b(wi1[r], uc1[t], a);
                        a = cfms_conj_b(ui2[r], wc2[t], a);
                        a = cfms_conj_b(wi2[r], uc2[t], a);
                        if (ok) M[base[r] + x] = a;
                        a = ok ? a : zero;
                    }
                    ra[2 * r] = cfma(a, vc1[t], ra[2 * r]);
                    ra[2 * r + 1] = cfma(a, vc2[t], ra[2 * r + 1]);
                    const bool below = sl < r;
                    ca1[t] = cfma_conj_a(a, below ? vi1[r] : zero, ca1[t]);
                    ca2[t] = cfma_conj_a(a, below ? vi2[r] : zero, ca2[t]);
                }
            }
        }
        // value 2r + b of the batch: row ri0 + r of product b
        const float2 out = reduce_scatter8(ra, lane);
        const int q = (lane >> 2) & 7, ri = ri0 + (q >> 1);
        if ((lane & 3) == 0 && ri < m) pw[(q & 1) * SH_NMAX + ri] = out;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int x = 32 * t + lane;
        if (x < m) {
            pw[x] = cadd(pw[x], ca1[t]);
            pw[SH_NMAX + x] = cadd(pw[SH_NMAX + x], ca2[t]);
        }
    }
    __syncthreads();
}

// The block reduction of the matrix in M (order n <= SH_NMAX, rows 2..n-1):
// afterwards M holds the band of rows >= 2 (diagonal blocks and R factors in
// place).  Thread i owns row i in the vector phases.  red: 64 floats of
// block-sum slots.  Ends with a CTA barrier.
__device__ void sh_reduce(int n, float2* M, float2* Wv, float2* pc, float* red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2 zero = make_float2(0.f, 0.f), one = make_float2(1.f, 0.f);
    for (int j = 0; 2 * j + 2 < n; ++j) {
        const int r0 = 2 * j + 2, c1 = 2 * j, c2 = 2 * j + 1;
        const int i = tid;
        const bool act = i >= r0 && i < n;
        float2 x1 = act ? M[sh_at(i, c1)] : zero;
        float2 x2 = act ? M[sh_at(i, c2)] : zero;
        // first reflector: ||x1||^2 and x1's first entry
        float s = warp_sum(x1.x * x1.x + x1.y * x1.y);
        if (lane == 0) red[40 + warp] = s;
        if (i == r0) { red[44] = x1.x; red[45] = x1.y; }
        __syncthreads();
        float2 rv, beta1;
        float tau1;
        sh_head(red[40] + red[41] + red[42] + red[43], make_float2(red[44], red[45]), rv, tau1, beta1);
        const float2 v1 = i == r0 ? one : (act ? sh_mul(x1, rv) : zero);
        // x2 <- (I - tau1 v1 v1^H) x2
        float2 g = sh_cmul(v1, x2);
        g.x = warp_sum(g.x);
        g.y = warp_sum(g.y);
        if (lane == 0) { red[46 + 2 * warp] = g.x; red[47 + 2 * warp] = g.y; }
        __syncthreads();
        g = make_float2(red[46] + red[48] + red[50] + red[52], red[47] + red[49] + red[51] + red[53]);
        x2 = csub(x2, sh_mul(v1, sh_scale(g, tau1)));
        // second reflector, rows r0+1 ..
        const bool act2 = act && i > r0;
        s = warp_sum(act2 ? x2.x * x2.x + x2.y * x2.y : 0.f);
        if (lane == 0) red[54 + warp] = s;
        if (i == r0 + 1) { red[58] = x2.x; red[59] = x2.y; }
        __syncthreads();
        float2 beta2;
        float tau2;
        sh_head(red[54] + red[55] + red[56] + red[57], make_float2(red[58], red[59]), rv, tau2, beta2);
        const float2 v2 = i == r0 + 1 ? one : (act2 ? sh_mul(x2, rv) : zero);
        if (i == r0) {
            M[sh_at(i, c1)] = beta1;  // R11
            M[sh_at(i, c2)] = x2;     // R12
        } else if (act) {
            M[sh_at(i, c1)] = v1;
            M[sh_at(i, c2)] = i == r0 + 1 ? beta2 : v2;  // R22, then v2
        }
        __syncthreads();
        sh_pass(n, j, M, Wv, pc);
        // P = A V, then V^H P and v1^H v2
        float2 p1 = zero, p2 = zero;
        if (act) {
#pragma unroll
            for (int w = 0; w < SH_NW; ++w) {
                p1 = cadd(p1, pc[2 * w * SH_NMAX + i - r0]);  // the pass indexes rows from r0
                p2 = cadd(p2, pc[(2 * w + 1) * SH_NMAX + i - r0]);
            }
        }
        float q[10];
        {
            const float2 a11 = sh_cmul(v1, p1), a12 = sh_cmul(v1, p2), a21 = sh_cmul(v2, p1),
                         a22 = sh_cmul(v2, p2), d12 = sh_cmul(v1, v2);
            q[0] = a11.x; q[1] = a11.y; q[2] = a12.x; q[3] = a12.y; q[4] = a21.x;
            q[5] = a21.y; q[6] = a22.x; q[7] = a22.y; q[8] = d12.x; q[9] = d12.y;
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            q[k] = warp_sum(q[k]);
            if (lane == 0) red[10 * warp + k] = q[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 10; ++k) q[k] = red[k] + red[10 + k] + red[20 + k] + red[30 + k];
        const float2 P11 = make_float2(q[0], q[1]), P12 = make_float2(q[2], q[3]);
        const float2 P21 = make_float2(q[4], q[5]), P22 = make_float2(q[6], q[7]);
        const float2 t12 = sh_scale(make_float2(q[8], q[9]), -tau1 * tau2);
        // V^H Y = (V^H P) T, Z = T^H (V^H Y)
        const float2 Y11 = sh_scale(P11, tau1), Y21 = sh_scale(P21, tau1);
        const float2 Y12 = cadd(sh_mul(P11, t12), sh_scale(P12, tau2));
        const float2 Y22 = cadd(sh_mul(P21, t12), sh_scale(P22, tau2));
        const float2 Z11 = sh_scale(Y11, tau1), Z12 = sh_scale(Y12, tau1);
        const float2 Z21 = cadd(sh_cmul(t12, Y11), sh_scale(Y21, tau2));
        const float2 Z22 = cadd(sh_cmul(t12, Y12), sh_scale(Y22, tau2));
        const float2 y1 = sh_scale(p1, tau1);
        const float2 y2 = cadd(sh_mul(t12, p1), sh_scale(p2, tau2));
        const float2 w1 = csub(y1, sh_scale(cadd(sh_mul(v1, Z11), sh_mul(v2, Z21)), 0.5f));
        const float2 w2 = csub(y2, sh_scale(cadd(sh_mul(v1, Z12), sh_mul(v2, Z22)), 0.5f));
        if (act) { Wv[i] = w1; Wv[SH_NMAX + i] = w2; }
        __syncthreads();
        // next panel's columns r0 and r0+1 (rows >= column): A - V W^H - W V^H,
        // with V = (1, 0) at row r0 and (v1(r0+1), 1) at row r0+1
        if (act) {
            const float2 w1a = Wv[r0], w2a = Wv[SH_NMAX + r0];
            {
                float2 a = M[sh_at(i, r0)];
                a = cfms_conj_b(v1, w1a, a);
                a = cfms_conj_b(v2, w2a, a);
                a = csub(a, w1);
                if (i == r0) a.y = 0.f;
                M[sh_at(i, r0)] = a;
            }
            if (i > r0) {
                const float2 w1b = Wv[r0 + 1], w2b = Wv[SH_NMAX + r0 + 1];
                const float2 v1b = M[sh_at(r0 + 1, c1)];
                float2 a = M[sh_at(i, r0 + 1)];
                a = cfms_conj_b(v1, w1b, a);
                a = cfms_conj_b(v2, w2b, a);
                a = cfms_conj_b(w1, v1b, a);
                a = csub(a, w2);
                if (i == r0 + 1) a.y = 0.f;
                M[sh_at(i, r0 + 1)] = a;
            }
        }
        // thread i reads only its own row of these columns in the next panel
    }
    __syncthreads();
}

// Band (bandwidth 2) to real tridiagonal form by Givens rotations, one warp:
// chase k (k = 0 .. n-3) annihilates (k+2, k) with a rotation in plane
// (k+1, k+2) and chases the bulge it creates at (p+3, p) down with rotations
// in planes (p+2, p+3), ...  Chase k's step s runs in round 4k + s, so the
// rotations of one round touch disjoint rows (seven apart) and the rounds
// give the result of the sequential chases.  Lane l takes the chases k = l
// (mod 32).  dd: diagonal, e1[i] = A(i+1, i), e2c[i] = A(i+2, i), bul[i] =
// A(i+3, i) (zero).  On return dd and e1 hold the tridiagonal.
// Rotation taking (a, b) to (r, 0): c = |a| / rho, s = a conj(b) / (|a| rho),
// rho^2 = |a|^2 + |b|^2, in FP32 with correctly rounded square roots and
// quotients, then scaled to unit length to first order (c^2 + |s|^2 - 1
// formed with fused multiply-adds).  The rotations' departure from
// unitarity is not shared by the two matrices' chases and dominates the
// error of dF; the scaling halves it.
__device__ __forceinline__ void sh_rot_params(float2 a, float2 b, float aa, float bb, float& c, float2& s) {
    if (!(aa > 0.f)) {
        c = 0.f;
        s = make_float2(1.f, 0.f);
        return;
    }
    const float rho = sqrtf(aa + bb), ra = sqrtf(aa);
    c = ra / rho;
    s = sh_scale(sh_mul(a, sh_conj(b)), 1.f / (ra * rho));
    const float dlt = __fmaf_rn(c, c, __fmaf_rn(s.x, s.x, __fmaf_rn(s.y, s.y, -1.f)));
    const float f = 1.f - 0.5f * dlt;
    c *= f;
    s = sh_scale(s, f);
}

__device__ void sh_chase(int n, float* dd, float2* e1, float2* e2c, float2* bul) {
    const int lane = threadIdx.x & 31;
    if (n < 3) return;
    const float2 zero = make_float2(0.f, 0.f);
    const int rounds = 4 * (n - 3) + 1;
    for (int r = 0; r < rounds; ++r) {
        const int K = r >> 2;
        // the chases k = lane (mod 32) active in round r: st = r - 4k grows as
        // k falls while chase k's last step (n-3-k)/2 grows more slowly, so
        // the active ones are consecutive from the largest k <= r/4 down
        for (int k = K - ((K - lane) & 31); k >= 0; k -= 32) {
            const int st = r - 4 * k;
            if (k > n - 3) continue;
            if (st > (n - 3 - k) / 2) break;
            const int p = k + 1 + 2 * st, q = p + 1;
            const bool r2 = p + 2 < n, r3 = p + 3 < n;
            // every operand of the rotation first (independent loads)
            const float2 a = st == 0 ? e1[p - 1] : e2c[p - 2];
            const float2 b = st == 0 ? e2c[p - 1] : bul[p - 2];
            const float2 x1 = e1[p - 1], y1 = e2c[p - 1];
            const float dp = dd[p], dq = dd[q];
            const float2 ep = e1[p];
            const float2 x2 = r2 ? e2c[p] : zero, y2 = r2 ? e1[p + 1] : zero;
            const float2 y3 = r3 ? e2c[p + 1] : zero;
            const float aa = a.x * a.x + a.y * a.y, bb = b.x * b.x + b.y * b.y;
            if (aa + bb > 0.f) {
                float c;
                float2 sv;
                sh_rot_params(a, b, aa, bb, c, sv);
                const float2 sc = sh_conj(sv);
                const float2 r_ = cadd(sh_scale(a, c), sh_mul(sv, b));
                if (st == 0) {
                    e1[p - 1] = r_;
                    e2c[p - 1] = zero;
                } else {
                    e2c[p - 2] = r_;
                    bul[p - 2] = zero;
                    e1[p - 1] = cadd(sh_scale(x1, c), sh_mul(sv, y1));
                    e2c[p - 1] = csub(sh_scale(y1, c), sh_mul(sc, x1));
                }
                const float re = sv.x * ep.x - sv.y * ep.y;
                const float c2 = c * c, s2 = sv.x * sv.x + sv.y * sv.y;
                dd[p] = c2 * dp + 2.f * c * re + s2 * dq;
                dd[q] = s2 * dp - 2.f * c * re + c2 * dq;
                e1[p] = csub(cadd(sh_scale(sc, c * (dq - dp)), sh_scale(ep, c2)), sh_mul(sh_mul(sc, sc), sh_conj(ep)));
                if (r2) {
                    e2c[p] = cadd(sh_scale(x2, c), sh_mul(sc, y2));
                    e1[p + 1] = csub(sh_scale(y2, c), sh_mul(sv, x2));
                }
                if (r3) {
                    bul[p] = sh_mul(sc, y3);
                    e2c[p + 1] = sh_scale(y3, c);
                }
            }
        }
        __syncwarp();
    }
}

// sh_chase with the band in double-float (dfl entries, about 48 significant
// bits) and the rotations computed and applied in double-float: the chases of
// a visit's two matrices then add rounding far below the FP32 reduction's,
// which is common to both and cancels in dF.  Same rounds and windows.
__device__ void sh_chase_df(int n, dfl* dd, dfl2* e1, dfl2* e2c, dfl2* bul) {
    const int lane = threadIdx.x & 31;
    if (n < 3) return;
    const dfl z(0.f, 0.f);
    const dfl2 zero = mk(z, z);
    const int rounds = 4 * (n - 3) + 1;
    for (int r = 0; r < rounds; ++r) {
        const int K = r >> 2;
        for (int k = K - ((K - lane) & 31); k >= 0; k -= 32) {
            const int st = r - 4 * k;
            if (k > n - 3) continue;
            if (st > (n - 3 - k) / 2) break;
            const int p = k + 1 + 2 * st, q = p + 1;
            const bool r2 = p + 2 < n, r3 = p + 3 < n;
            const dfl2 a = st == 0 ? e1[p - 1] : e2c[p - 2];
            const dfl2 b = st == 0 ? e2c[p - 1] : bul[p - 2];
            const dfl2 x1 = e1[p - 1], y1 = e2c[p - 1];
            const dfl dp = dd[p], dq = dd[q];
            const dfl2 ep = e1[p];
            const dfl2 x2 = r2 ? e2c[p] : zero, y2 = r2 ? e1[p + 1] : zero;
            const dfl2 y3 = r3 ? e2c[p + 1] : zero;
            const dfl aa = cabs2(a), bb = cabs2(b);
            if (!(aa.hi > 0.f) && !(bb.hi > 0.f)) continue;
            dfl c;
            dfl2 sv;
            if (aa.hi > 0.f) {
                const dfl rr = aa + bb;
                c = sqroot(aa / rr);
                const dfl kk = dfl(1.f, 0.f) / sqroot(aa * rr);
                const dfl2 ab = cfma_conj_a(b, a, zero);  // conj(b) a
                sv = mk(ab.x * kk, ab.y * kk);
            } else {
                c = z;
                sv = mk(dfl(1.f, 0.f), z);
            }
            const dfl2 sc = mk(sv.x, -sv.y);
            auto lin = [](dfl cc, dfl2 x, dfl2 s, dfl2 y) {  // c x + s y
                return cfma(s, y, mk(x.x * cc, x.y * cc));
            };
            const dfl2 r_ = lin(c, a, sv, b);
            if (st == 0) {
                e1[p - 1] = r_;
                e2c[p - 1] = zero;
            } else {
                e2c[p - 2] = r_;
                bul[p - 2] = zero;
                e1[p - 1] = lin(c, x1, sv, y1);
                e2c[p - 1] = csub(mk(y1.x * c, y1.y * c), cfma(sc, x1, zero));
            }
            const dfl re = dot2_acc(z, sv.x, ep.x, -sv.y, ep.y);  // Re(s ep)
            const dfl c2 = c * c, s2 = cabs2(sv);
            const dfl two_c_re = (c + c) * re;
            dd[p] = c2 * dp + two_c_re + s2 * dq;
            dd[q] = s2 * dp - two_c_re + c2 * dq;
            // c conj(s) (dq - dp) + c^2 ep - conj(s)^2 conj(ep)
            const dfl cd = c * (dq - dp);
            const dfl2 sc2 = cfma(sc, sc, zero);
            e1[p] = csub(mk(sc.x * cd + ep.x * c2, sc.y * cd + ep.y * c2), cfma(sc2, mk(ep.x, -ep.y), zero));
            if (r2) {
                e2c[p] = lin(c, x2, sc, y2);
                e1[p + 1] = csub(mk(y2.x * c, y2.y * c), cfma(sv, x2, zero));
            }
            if (r3) {
                bul[p] = cfma(sc, y3, zero);
                e2c[p + 1] = mk(y3.x * c, y3.y * c);
            }
        }
        __syncwarp();
    }
}

// After the reduction: the two bands (the reduction's band with the old and
// the new leading block, t11 in thread 0's registers) into bandmem, their
// chases (warp 0: old, warp 1: new), both eigenvalue phases with their
// scratch in eigmem, and the decision (Metropolis, the guard, the record).
// nm >= n: the stride of the per-matrix arrays.  Called by all threads.
template <int NWP, bool kAccurate>
__device__ void sh_finish(const StageArgs& a, const StageVar v, int c, int site, const Window& w, int n,
                          const double* so, const double* s_new, const double* cls, const float2* M,
                          const float* t11, unsigned char* bandmem, unsigned char* eigmem, int nm) {
    // band element: float2 (FP32 chase) or dfl2 (double-float chase); per band
    // e1, e2c, bul (nm each) and the diagonal (nm reals, nm / 2 elements)
    using BE = typename std::conditional<kAccurate, dfl2, float2>::type;
    using BR = typename std::conditional<kAccurate, dfl, float>::type;
    BE* bnd = reinterpret_cast<BE*>(bandmem);
    const int BS = 3 * nm + nm / 2;
    auto be = [](float2 x) -> BE {
        if constexpr (kAccurate) return mk(dfl(x.x, 0.f), dfl(x.y, 0.f));
        else return x;
    };
    auto br = [](float x) -> BR {
        if constexpr (kAccurate) return dfl(x, 0.f);
        else return x;
    };
    const float2 zero = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 b1 = (i >= 1 && i + 1 < n) ? M[sh_at(i + 1, i)] : zero;
        const float2 b2 = i + 2 < n ? M[sh_at(i + 2, i)] : zero;
        const float b0 = i >= 2 ? M[sh_at(i, i)].x : 0.f;
        for (int var = 0; var < 2; ++var) {
            BE* e1 = bnd + var * BS;
            BR* dd = reinterpret_cast<BR*>(e1 + 3 * nm);
            if (i >= 1) e1[i] = be(b1);
            e1[nm + i] = be(b2);
            e1[2 * nm + i] = be(zero);
            if (i >= 2) dd[i] = br(b0);
            if (i == 0) {
                dd[0] = br(t11[4 * var]);
                dd[1] = br(t11[4 * var + 1]);
                e1[0] = be(make_float2(t11[4 * var + 2], t11[4 * var + 3]));
            }
        }
    }
    __syncthreads();
    // chases, then (d, e2) as doubles for the eigenvalue phase
    double* dv = reinterpret_cast<double*>(eigmem);  // [2 var][d, e2][nm]
    const int warp = threadIdx.x >> 5;
    if (warp < 2) {
        BE* e1 = bnd + warp * BS;
        BR* dd = reinterpret_cast<BR*>(e1 + 3 * nm);
        if constexpr (kAccurate) sh_chase_df(n, dd, e1, e1 + nm, e1 + 2 * nm);
        else sh_chase(n, dd, e1, e1 + nm, e1 + 2 * nm);
        double* d = dv + 2 * warp * nm;
        for (int i = threadIdx.x & 31; i < n; i += 32) {
            if constexpr (kAccurate) {
                d[i] = (double)dd[i];
                const double ex = (double)e1[i].x, ey = (double)e1[i].y;
                d[nm + i] = i < n - 1 ? ex * ex + ey * ey : 0.0;
            } else {
                d[i] = (double)dd[i];
                d[nm + i] = i < n - 1 ? (double)(e1[i].x * e1[i].x + e1[i].y * e1[i].y) : 0.0;
            }
        }
    }
    __syncthreads();
    Carve<float> cv;
    {
        unsigned char* sc = eigmem + 4 * (size_t)nm * sizeof(double);
        cv.df = reinterpret_cast<float*>(sc);
        cv.e2f = cv.df + nm;
        cv.dlo = cv.e2f + nm;
        cv.e2lo = cv.dlo + nm;
        cv.lam = cv.e2lo + nm;                                 // 2 nm floats
        cv.cnt = reinterpret_cast<int*>(cv.lam + 2 * nm);      // one per thread
        cv.red = reinterpret_cast<double*>(cv.cnt + 32 * NWP);  // 8 NWP doubles
    }
    double F[2], fill[2];
    for (int var = 0; var < 2; ++var) {
        cv.d = dv + 2 * var * nm;
        cv.e2 = cv.d + nm;
        double ssp, sfe;
        int K;
        tridiag_eig_F<float, NWP>(n, cv, a.m.mu - a.m.e0, a.m.T, false, nullptr, ssp, sfe, K);
        F[var] = -a.m.T * ssp + cls[var];
        fill[var] = sfe;
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double Fo = F[0], Fn = F[1];
    a.Fbuf[2 * c] = Fo;
    a.Fbuf[2 * c + 1] = Fn;
    a.fillbuf[2 * c] = fill[0];
    a.fillbuf[2 * c + 1] = fill[1];
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
    const double sn[3] = {s_new[0], s_new[1], s_new[2]};
    if (a.sg_feat) collect_sample(a, v.S_in, w, v.rec_base + c, sn, dF);
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
    a.rec_fill[r] = acc ? fill[1] : fill[0];
    a.rec_n[r] = n;
    if (acc) atomicAdd(&a.counters[0], 1ull);
    atomicAdd(&a.counters[1], 2ull);
}

// The window's classical energy with the old and the proposed vector
// (thread 0; zero unless the model has one).
__device__ __forceinline__ void sh_classical(const Model& m, const Window& w, int n, double* sp, const double* s_new,
                                             double* cls) {
    cls[0] = cls[1] = 0.0;
    if (threadIdx.x != 0 || !m.cls_on) return;
    const int uw = (w.uwz * w.ey + w.uwy) * w.ex + w.uwx;
    cls[0] = window_classical(m, sp, n / 2);
    const double o0 = sp[3 * uw], o1 = sp[3 * uw + 1], o2 = sp[3 * uw + 2];
    sp[3 * uw] = s_new[0]; sp[3 * uw + 1] = s_new[1]; sp[3 * uw + 2] = s_new[2];
    cls[1] = window_classical(m, sp, n / 2);
    sp[3 * uw] = o0; sp[3 * uw + 1] = o1; sp[3 * uw + 2] = o2;
}

// One update site of a stage, both matrices in this CTA (a sweep kernel's
// stage_item with the shared reduction): build, reduce once, chase and solve
// each band, decide.
__device__ __forceinline__ void stage_item_shared(const StageArgs& a, const StageVar v, int c, unsigned char* smem,
                                                  double* s_new) {
    const ShLayout L = sh_layout();
    float2* M = reinterpret_cast<float2*>(smem + L.M);
    float2* Wv = reinterpret_cast<float2*>(smem + L.W);
    float2* pc = reinterpret_cast<float2*>(smem + L.pc);
    float* red = reinterpret_cast<float*>(smem + L.red);
    c = v.perm ? v.perm[c] : c;
    const int site = v.sites[c];
    const Window w = make_window(a.m, site);
    const int n = 2 * window_nsite(w);
    const double* so = v.S_in + 3 * site;
    if (threadIdx.x == 0) propose(a.m, v.sweep, (uint32_t)site, so, s_new);
    __syncthreads();
    double* sp = reinterpret_cast<double*>(smem + L.pc);
    float t11[8];
    build_cluster_shared(a.m, w, v.S_in, s_new, sp, M, t11);
    __syncthreads();
    double cls[2];
    sh_classical(a.m, w, n, sp, s_new, cls);
    sh_reduce(n, M, Wv, pc, red);
    // the bands in the partial-sum region; (d, e2) and the eigenvalue scratch
    // in the matrix region, free once the bands are out
    sh_finish<SH_NW, false>(a, v, c, site, w, n, so, s_new, cls, M, t11, smem + L.pc, smem + L.M, SH_NMAX);
}

// One stage with the shared reduction: CTA c holds update site c.
__global__ void __launch_bounds__(32 * SH_NW, 3) k_stage_shared(StageArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.prev_count + a.prev2_count;
         k += gridDim.x * blockDim.x) {
        const int s = k < a.prev_count ? a.prev_sites[k] : a.prev2_sites[k - a.prev_count];
        a.S_out[3 * s] = a.S_in[3 * s];
        a.S_out[3 * s + 1] = a.S_in[3 * s + 1];
        a.S_out[3 * s + 2] = a.S_in[3 * s + 2];
    }
    const int c = blockIdx.x;
    const int count = a.count_dev ? (int)*a.count_dev : a.count;
    if (c >= count) return;
    stage_item_shared(a, stage_var(a), c, smem, s_new);
}


// ---------------------------------------------------------------------------
// The shared reduction for large traveling clusters (orders above the
// shared-memory kernels', up to 32 NW_LARGE): one NW_LARGE-warp CTA per update
// site, the matrix in the CTA's global slot (rows 2..n-1 of the packed
// triangle, as above), the panel's reflectors, w and the partial sums in
// shared memory.  At these orders the chases' O(n) dependent rounds are small
// beside the reduction, which is done once per visit instead of twice.
// ---------------------------------------------------------------------------

constexpr int SHL_NW = NW_LARGE;

// Shared memory of a large shared-reduction CTA for orders up to nA (nm = nA
// rounded up to 32): w, the reflectors of two consecutive panels, the row
// sums and per-warp column sums of the two products (two vectors each), the
// block-sum slots.  The window's vectors (build), the bands and the
// eigenvalue phase reuse the column-sum region.
struct ShlLayout { size_t W, Va, Vb, pr, pc, red, total; int nm; };
__host__ __device__ inline ShlLayout shl_layout(int nA) {
    ShlLayout L;
    const int nm = (nA + 31) & ~31;
    L.nm = nm;
    const size_t vv = 2 * (size_t)nm * sizeof(float2);
    size_t o = 0;
    L.W = o;   o = align16(o + vv);
    L.Va = o;  o = align16(o + vv);
    L.Vb = o;  o = align16(o + vv);
    L.pr = o;  o = align16(o + vv);
    L.pc = o;  o = align16(o + (size_t)SHL_NW * vv);
    L.red = o; o = align16(o + 256 * sizeof(float));
    L.total = o;
    return L;
}

// Panel j's fused pass (plain form of sh_pass for a matrix in global memory):
// warp w takes the trailing rows m-1-w, m-1-w-SHL_NW, ... (longest first),
// lane l the columns l, l+32, ... of the row, four global loads in flight per
// lane.  Each element gets panel j-1's rank-4 update (Vp, Wv; skipped at
// j = 0), is stored, and adds to its row's two sums (reduced across the warp
// into pr) and, below the diagonal, to its column's two sums in the warp's
// own partial vectors (lanes own distinct columns: a fixed order).  Vectors
// hold two components of stride nm, indexed by row; pr and pc by row - r0.
__device__ __forceinline__ void shl_pass(int n, int j, float2* M, const float2* Wv, const float2* Vc, const float2* Vp,
                                         float2* pr, float2* pc, int nm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = 2 * j + 2, m = n - r0;
    const bool upd = j > 0;
    const float2 zero = make_float2(0.f, 0.f);
    float2* pw = pc + 2 * warp * (size_t)nm;
    for (int x = lane; x < m; x += 32) { pw[x] = zero; pw[nm + x] = zero; }
    __syncwarp();
    for (int r = warp; r < m; r += SHL_NW) {
        const int ri = m - 1 - r, i = r0 + ri;
        const float2 ui1 = upd ? Vp[i] : zero, ui2 = upd ? Vp[nm + i] : zero;
        const float2 wi1 = upd ? Wv[i] : zero, wi2 = upd ? Wv[nm + i] : zero;
        const float2 vi1 = Vc[i], vi2 = Vc[nm + i];
        float2* row = M + sh_at(i, r0);
        float2 ra1 = zero, ra2 = zero;
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
                    const int y = r0 + jr;
                    float2 a = av[q];
                    if (upd) {
                        a = cfms_conj_b(ui1, Wv[y], a);
                        a = cfms_conj_b(wi1, Vp[y], a);
                        a = cfms_conj_b(ui2, Wv[nm + y], a);
                        a = cfms_conj_b(wi2, Vp[nm + y], a);
                        row[jr] = a;
                    }
                    ra1 = cfma(a, Vc[y], ra1);
                    ra2 = cfma(a, Vc[nm + y], ra2);
                    if (jr < ri) {
                        pw[jr] = cfma_conj_a(a, vi1, pw[jr]);
                        pw[nm + jr] = cfma_conj_a(a, vi2, pw[nm + jr]);
                    }
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ra1 = cadd(ra1, cshfl_xor(ra1, o));
            ra2 = cadd(ra2, cshfl_xor(ra2, o));
        }
        if (lane == 0) { pr[ri] = ra1; pr[nm + ri] = ra2; }
    }
    __syncthreads();
}

// The block reduction of the matrix in global memory M (order n <= 32
// SHL_NW); the algorithm and the thread-per-row vector phases of sh_reduce,
// with the reflectors kept whole in shared memory (two buffers by panel
// parity) and only R written back.  red: 256 floats.  Ends with a barrier.
__device__ void shl_reduce(int n, float2* M, float2* Wv, float2* Va, float2* Vb, float2* pr, float2* pc, float* red,
                           int nm) {
    constexpr int NWP = SHL_NW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2 zero = make_float2(0.f, 0.f), one = make_float2(1.f, 0.f);
    // block-sum slots: products 10 per warp [0, 160), ||x1||^2 [160, 176),
    // x1's first entry 176-177, v1^H x2 [178, 210), ||x2||^2 [210, 226),
    // x2's second entry 226-227
    for (int j = 0; 2 * j + 2 < n; ++j) {
        float2* Vc = (j & 1) ? Vb : Va;
        const float2* Vp = (j & 1) ? Va : Vb;
        const int r0 = 2 * j + 2, c1 = 2 * j, c2 = 2 * j + 1;
        const int i = tid;
        const bool act = i >= r0 && i < n;
        float2 x1 = act ? M[sh_at(i, c1)] : zero;
        float2 x2 = act ? M[sh_at(i, c2)] : zero;
        float s = warp_sum(x1.x * x1.x + x1.y * x1.y);
        if (lane == 0) red[160 + warp] = s;
        if (i == r0) { red[176] = x1.x; red[177] = x1.y; }
        __syncthreads();
        float s1 = 0.f;
#pragma unroll
        for (int w = 0; w < NWP; ++w) s1 += red[160 + w];
        float2 rv, beta1;
        float tau1;
        sh_head(s1, make_float2(red[176], red[177]), rv, tau1, beta1);
        const float2 v1 = i == r0 ? one : (act ? sh_mul(x1, rv) : zero);
        float2 g = sh_cmul(v1, x2);
        g.x = warp_sum(g.x);
        g.y = warp_sum(g.y);
        if (lane == 0) { red[178 + 2 * warp] = g.x; red[179 + 2 * warp] = g.y; }
        __syncthreads();
        g = zero;
#pragma unroll
        for (int w = 0; w < NWP; ++w) { g.x += red[178 + 2 * w]; g.y += red[179 + 2 * w]; }
        x2 = csub(x2, sh_mul(v1, sh_scale(g, tau1)));
        const bool act2 = act && i > r0;
        s = warp_sum(act2 ? x2.x * x2.x + x2.y * x2.y : 0.f);
        if (lane == 0) red[210 + warp] = s;
        if (i == r0 + 1) { red[226] = x2.x; red[227] = x2.y; }
        __syncthreads();
        float s2 = 0.f;
#pragma unroll
        for (int w = 0; w < NWP; ++w) s2 += red[210 + w];
        float2 beta2;
        float tau2;
        sh_head(s2, make_float2(red[226], red[227]), rv, tau2, beta2);
        const float2 v2 = i == r0 + 1 ? one : (act2 ? sh_mul(x2, rv) : zero);
        if (act) { Vc[i] = v1; Vc[nm + i] = v2; }
        if (i == r0) { M[sh_at(i, c1)] = beta1; M[sh_at(i, c2)] = x2; }
        if (i == r0 + 1) M[sh_at(i, c2)] = beta2;
        __syncthreads();
        shl_pass(n, j, M, Wv, Vc, Vp, pr, pc, nm);
        float2 p1 = zero, p2 = zero;
        if (act) {
            p1 = pr[i - r0];
            p2 = pr[nm + i - r0];
#pragma unroll
            for (int w = 0; w < NWP; ++w) {
                p1 = cadd(p1, pc[2 * w * (size_t)nm + i - r0]);
                p2 = cadd(p2, pc[(2 * w + 1) * (size_t)nm + i - r0]);
            }
        }
        float q[10];
        {
            const float2 a11 = sh_cmul(v1, p1), a12 = sh_cmul(v1, p2), a21 = sh_cmul(v2, p1),
                         a22 = sh_cmul(v2, p2), d12 = sh_cmul(v1, v2);
            q[0] = a11.x; q[1] = a11.y; q[2] = a12.x; q[3] = a12.y; q[4] = a21.x;
            q[5] = a21.y; q[6] = a22.x; q[7] = a22.y; q[8] = d12.x; q[9] = d12.y;
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            q[k] = warp_sum(q[k]);
            if (lane == 0) red[10 * warp + k] = q[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            float t = red[k];
#pragma unroll
            for (int w = 1; w < NWP; ++w) t += red[10 * w + k];
            q[k] = t;
        }
        const float2 P11 = make_float2(q[0], q[1]), P12 = make_float2(q[2], q[3]);
        const float2 P21 = make_float2(q[4], q[5]), P22 = make_float2(q[6], q[7]);
        const float2 t12 = sh_scale(make_float2(q[8], q[9]), -tau1 * tau2);
        const float2 Y11 = sh_scale(P11, tau1), Y21 = sh_scale(P21, tau1);
        const float2 Y12 = cadd(sh_mul(P11, t12), sh_scale(P12, tau2));
        const float2 Y22 = cadd(sh_mul(P21, t12), sh_scale(P22, tau2));
        const float2 Z11 = sh_scale(Y11, tau1), Z12 = sh_scale(Y12, tau1);
        const float2 Z21 = cadd(sh_cmul(t12, Y11), sh_scale(Y21, tau2));
        const float2 Z22 = cadd(sh_cmul(t12, Y12), sh_scale(Y22, tau2));
        const float2 y1 = sh_scale(p1, tau1);
        const float2 y2 = cadd(sh_mul(t12, p1), sh_scale(p2, tau2));
        const float2 w1 = csub(y1, sh_scale(cadd(sh_mul(v1, Z11), sh_mul(v2, Z21)), 0.5f));
        const float2 w2 = csub(y2, sh_scale(cadd(sh_mul(v1, Z12), sh_mul(v2, Z22)), 0.5f));
        if (act) { Wv[i] = w1; Wv[nm + i] = w2; }
        __syncthreads();
        if (act) {
            const float2 w1a = Wv[r0], w2a = Wv[nm + r0];
            {
                float2 a = M[sh_at(i, r0)];
                a = cfms_conj_b(v1, w1a, a);
                a = cfms_conj_b(v2, w2a, a);
                a = csub(a, w1);
                if (i == r0) a.y = 0.f;
                M[sh_at(i, r0)] = a;
            }
            if (i > r0) {
                const float2 w1b = Wv[r0 + 1], w2b = Wv[nm + r0 + 1];
                const float2 v1b = Vc[r0 + 1];
                float2 a = M[sh_at(i, r0 + 1)];
                a = cfms_conj_b(v1, w1b, a);
                a = cfms_conj_b(v2, w2b, a);
                a = cfms_conj_b(w1, v1b, a);
                a = csub(a, w2);
                if (i == r0 + 1) a.y = 0.f;
                M[sh_at(i, r0 + 1)] = a;
            }
        }
    }
    __syncthreads();
}

// One update site with the large shared reduction (matrix in this CTA's
// global slot).
__device__ __forceinline__ void stage_item_large_shared(const StageArgs& a, const StageVar v, int c,
                                                        unsigned char* smem, double* s_new) {
    const ShlLayout L = shl_layout(a.nA);
    const int nm = L.nm;
    float2* M = static_cast<float2*>(a.gL) + (int64_t)blockIdx.x * a.gL_stride;
    float2* Wv = reinterpret_cast<float2*>(smem + L.W);
    float2* Va = reinterpret_cast<float2*>(smem + L.Va);
    float2* Vb = reinterpret_cast<float2*>(smem + L.Vb);
    float2* pr = reinterpret_cast<float2*>(smem + L.pr);
    float2* pc = reinterpret_cast<float2*>(smem + L.pc);
    float* red = reinterpret_cast<float*>(smem + L.red);
    c = v.perm ? v.perm[c] : c;
    const int site = v.sites[c];
    const Window w = make_window(a.m, site);
    const int n = 2 * window_nsite(w);
    const double* so = v.S_in + 3 * site;
    if (threadIdx.x == 0) propose(a.m, v.sweep, (uint32_t)site, so, s_new);
    __syncthreads();
    double* sp = reinterpret_cast<double*>(smem + L.pc);
    float t11[8];
    build_cluster_shared(a.m, w, v.S_in, s_new, sp, M, t11);
    __syncthreads();
    double cls[2];
    sh_classical(a.m, w, n, sp, s_new, cls);
    shl_reduce(n, M, Wv, Va, Vb, pr, pc, red, nm);
    // bands and the eigenvalue phase in the column-sum region
    unsigned char* bandmem = smem + L.pc;
    unsigned char* eigmem = bandmem + align16((size_t)2 * (3 * nm + nm / 2) * sizeof(dfl2));
    sh_finish<SHL_NW, true>(a, v, c, site, w, n, so, s_new, cls, M, t11, bandmem, eigmem, nm);
}

// One stage of large clusters with the shared reduction: the resident CTAs
// stride over the update sites.
__global__ void __launch_bounds__(32 * SHL_NW, 1) k_stage_large_shared(StageArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_new[3];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.prev_count + a.prev2_count;
         k += gridDim.x * blockDim.x) {
        const int s = k < a.prev_count ? a.prev_sites[k] : a.prev2_sites[k - a.prev_count];
        a.S_out[3 * s] = a.S_in[3 * s];
        a.S_out[3 * s + 1] = a.S_in[3 * s + 1];
        a.S_out[3 * s + 2] = a.S_in[3 * s + 2];
    }
    const int count = a.count_dev ? (int)*a.count_dev : a.count;
    for (int c = blockIdx.x; c < count; c += gridDim.x) {
        stage_item_large_shared(a, stage_var(a), c, smem, s_new);
        __syncthreads();
    }
}

}  // namespace ptca
