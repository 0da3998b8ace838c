// cluster_panel.cuh -- blocked (panel) form of the FP32 Householder reduction
// (Sec. II.c step b: the cluster diagonalisation), for 8-warp CTAs and
// matrix orders up to 128: panels of B reflectors, the trailing block updated
// once per panel (the LAPACK LATRD scheme, written for one CTA).
//
// The reflectors are those of householder_tridiag (column k reflected onto
// its first entry below the diagonal, H = I - tau v v^H, w = p - (tau/2)
// (v^H p) v with p = tau A v); only the order of the work differs.  For
// reflector i of a panel starting at column k0 (k = k0 + i):
//   1. column k of the current matrix is formed from the stored (panel-start)
//      matrix and the panel's earlier pairs:  a_rk - sum_{t<i} (v_t,r
//      conj(w_t,k) + w_t,r conj(v_t,k));
//   2. d_k, ||x||^2 and the reflector v_i;
//   3. y = A_S v_i over the trailing block, A_S the stored matrix (a
//      read-only pass: row sums reduce-scattered per warp, column sums per
//      lane, as in the fused pass of householder_tridiag);
//   4. y -= V (W^H v_i) + W (V^H v_i) over the panel's earlier pairs, the
//      product with the current matrix;
//   5. p = tau y and w_i.
// After the panel, one pass applies A <- A - V W^H - W V^H (rank 2b) to the
// trailing block of rows and columns k0 + b ...  Every sum runs in a fixed
// order (warps, then lanes, then rows): the result does not depend on timing.
#pragma once

#include "cluster_solve.cuh"

namespace ptca {

constexpr int PN_NW = 8;  // warps per CTA of the panel reduction

// Shared memory of the panel reduction beyond smem_layout: the panel's
// vectors V and W (B each, NMAX entries) and the per-warp partial dot
// products (2B complex per warp).
__host__ __device__ inline size_t panel_extra_bytes(int B, int nmax) {
    return ((2 * (size_t)B * nmax + (size_t)PN_NW * 2 * B) * sizeof(float2) + 15) & ~size_t(15);
}

// Read-only matrix-vector product over the trailing block (rows and columns
// j0 .. n-1) of the stored matrix: row sums into pr[ri], column sums of warp
// w into pc[w * NMAX + ri] (ri relative to j0).  v: entries at absolute
// indices, zero below j0.  The layout of the work is that of the fused pass.
template <int NT, int NW>
__device__ __forceinline__ void panel_matvec(int j0, int n, const float2* __restrict__ A, const float2* v,
                                             float2* pr, float2* pc) {
    using V = float2;
    constexpr int NMAX = 32 * NT;
    constexpr int RB = 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const V zero = mk(0.f, 0.f);
    const int m = n - j0;
    const int nbatch = (m + RB - 1) / RB;
    V vc[NT], cacc[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int j = j0 + 32 * t + lane;
        vc[t] = j < n ? v[j] : zero;
        cacc[t] = zero;
    }
    for (int round = 0;; ++round) {
        const int slot = round * NW + ((round & 1) ? (NW - 1 - warp) : warp);
        if (slot >= nbatch) break;
        const int b = nbatch - 1 - slot;
        const int ri0 = b * RB;
        V vi[RB], racc[RB];
        int base[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int ri = ri0 + r;
            const bool ok = ri < m;
            const int i = j0 + ri;
            vi[r] = ok ? v[i] : zero;
            base[r] = ok ? tri(i) + j0 : 0;
            racc[r] = zero;
        }
        const bool full_rows = ri0 + RB - 1 < m;
        const int last = (ri0 + RB - 1 < m ? ri0 + RB - 1 : m - 1);
        const int nch = (last >> 5) + 1;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            if (t < nch) {
                const int jr = 32 * t + lane;
                if (full_rows && 32 * t + 31 < ri0) {
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const V a = A[base[r] + jr];
                        racc[r] = cfma(a, vc[t], racc[r]);
                        cacc[t] = cfma_conj_a(a, vi[r], cacc[t]);
                    }
                    continue;
                }
                // Diagonal chunk: as in the fused pass, a masked lane reads at
                // most 31 elements past the packed triangle (the buffers are
                // padded) and its value is replaced by zero.
                const int sl = jr - ri0, nr = m - ri0;
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const bool ok = (sl <= r) && (r < nr);
                    V a = A[base[r] + jr];
                    a = ok ? a : zero;
                    racc[r] = cfma(a, vc[t], racc[r]);
                    const V vrow = (sl < r) ? vi[r] : zero;
                    cacc[t] = cfma_conj_a(a, vrow, cacc[t]);
                }
            }
        }
        const V out = reduce_scatter8(racc, lane);
        const int ri = ri0 + ((lane >> 2) & 7);
        if ((lane & 3) == 0 && ri < m) pr[ri] = out;
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int jr = 32 * t + lane;
        if (jr < m) pc[warp * NMAX + jr] = cacc[t];
    }
}

// Trailing update after a panel: A <- A - sum_{t<nb} (v_t w_t^H + w_t v_t^H)
// on rows and columns kt .. n-1.  Lanes take columns, warps take rows; a
// lane keeps its column's 2 nb vector entries in registers.
template <int NT, int NW, int B>
__device__ __forceinline__ void panel_update(int kt, int n, int nb, float2* A, const float2* PV, const float2* PW) {
    using V = float2;
    constexpr int NMAX = 32 * NT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const V zero = mk(0.f, 0.f);
#pragma unroll 1
    for (int c = 0; kt + 32 * c < n; ++c) {
        const int j = kt + 32 * c + lane;
        V cv[B], cw[B];
#pragma unroll
        for (int t = 0; t < B; ++t) {
            const bool ok = t < nb && j < n;
            cv[t] = ok ? PV[t * NMAX + j] : zero;
            cw[t] = ok ? PW[t * NMAX + j] : zero;
        }
        // rows i >= the chunk's first column, dealt to the warps
        for (int i = kt + 32 * c + warp; i < n; i += NW) {
            if (j > i || j >= n) continue;
            V a = A[tri(i) + j];
#pragma unroll
            for (int t = 0; t < B; ++t) {
                if (t < nb) {
                    a = cfms_conj_b(PV[t * NMAX + i], cw[t], a);
                    a = cfms_conj_b(PW[t * NMAX + i], cv[t], a);
                }
            }
            A[tri(i) + j] = a;
        }
    }
}

// Householder tridiagonalisation in panels of B reflectors (order n <= 32 NT,
// 8-warp CTAs).  A: packed lower triangle (as householder_tridiag); PV, PW:
// B x 32NT panel vectors; dotw: 8 x 2B partial dot products.  Writes d and e2.
template <int NT, int B>
__device__ void householder_tridiag_panel(int n, float2* A, const HHScratch<float>& sc, float2* PV, float2* PW,
                                          float2* dotw, double* d, double* e2) {
    using V = float2;
    constexpr int NW = PN_NW;
    constexpr int NMAX = 32 * NT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const V zero = mk(0.f, 0.f);
    if (n <= 2) {
        if (tid == 0) {
            d[0] = double(A[0].x);
            if (n == 2) { d[1] = double(A[2].x); e2[0] = double(cabs2(A[1])); }
        }
        __syncthreads();
        return;
    }
    const int r = tid;  // the vector entry (matrix row) of this thread
    int k = 0;
    while (k <= n - 3) {
        const int k0 = k;
        const int nb = min(B, n - 2 - k0);  // reflectors k0 .. k0 + nb - 1
        for (int i = 0; i < nb; ++i) {
            k = k0 + i;
            const int j0 = k + 1;
            // 1-2: column k of the current matrix, d_k, ||x||^2, x_0
            V x = zero;
            if (r >= k && r < n) {
                x = A[tri(r) + k];
#pragma unroll
                for (int t = 0; t < B; ++t) {
                    if (t < i) {
                        x = cfms_conj_b(PV[t * NMAX + r], PW[t * NMAX + k], x);
                        x = cfms_conj_b(PW[t * NMAX + r], PV[t * NMAX + k], x);
                    }
                }
            }
            if (r == k) d[k] = double(x.x);
            if (r == j0) sc.sx[0] = x;
            float s2p = (r > k && r < n) ? cabs2(x) : 0.f;
            s2p = warp_sum(s2p);
            if (lane == 0) sc.redB[warp] = s2p;
            __syncthreads();
            float s2 = sc.redB[0];
#pragma unroll
            for (int w = 1; w < NW; ++w) s2 += sc.redB[w];
            if (tid == 0) e2[k] = double(s2);
            V vfirst;
            float tau;
            reflector_head(s2, sc.sx[0], vfirst, tau);
            const V v = r == j0 ? vfirst : (r > j0 && r < n ? x : zero);
            if (r < NMAX) PV[i * NMAX + r] = v;
            __syncthreads();
            // 3: y = A_S v over the trailing block
            panel_matvec<NT, NW>(j0, n, A, PV + i * NMAX, sc.pr, sc.pc);
            __syncthreads();
            // 4: y -= V (W^H v) + W (V^H v) over the earlier pairs: the dot
            // products first (per warp, then in warp order)
            const int ri = r - j0;
            const bool mine = ri >= 0 && r < n;
            V y = zero;
            if (mine) {
                y = sc.pr[ri];
#pragma unroll
                for (int w = 0; w < NW; ++w) y = cadd(y, sc.pc[w * NMAX + ri]);
            }
#pragma unroll
            for (int t = 0; t < B; ++t) {
                if (t < i) {
                    V al = zero, be = zero;  // conj(w_t,r) v_r and conj(v_t,r) v_r
                    if (mine) {
                        al = cfma_conj_a(PW[t * NMAX + r], v, al);
                        be = cfma_conj_a(PV[t * NMAX + r], v, be);
                    }
                    al.x = warp_sum(al.x); al.y = warp_sum(al.y);
                    be.x = warp_sum(be.x); be.y = warp_sum(be.y);
                    if (lane == 0) { dotw[warp * 2 * B + 2 * t] = al; dotw[warp * 2 * B + 2 * t + 1] = be; }
                }
            }
            __syncthreads();
            float sp = 0.f;
            if (mine) {
#pragma unroll
                for (int t = 0; t < B; ++t) {
                    if (t < i) {
                        V al = dotw[2 * t], be = dotw[2 * t + 1];
#pragma unroll
                        for (int w = 1; w < NW; ++w) {
                            al = cadd(al, dotw[w * 2 * B + 2 * t]);
                            be = cadd(be, dotw[w * 2 * B + 2 * t + 1]);
                        }
                        y = cfms(PV[t * NMAX + r], al, y);
                        y = cfms(PW[t * NMAX + r], be, y);
                    }
                }
                // 5: p = tau y
                y.x *= tau;
                y.y *= tau;
                sp = v.x * y.x + v.y * y.y;
            }
            sp = warp_sum(sp);
            if (lane == 0) sc.redA[warp] = sp;
            __syncthreads();
            float s = sc.redA[0];
#pragma unroll
            for (int w = 1; w < NW; ++w) s += sc.redA[w];
            const float K = 0.5f * tau * s;
            if (r < NMAX) PW[i * NMAX + r] = mine ? mk(y.x - K * v.x, y.y - K * v.y) : zero;
            __syncthreads();
        }
        // the panel's rank-2 nb update of the trailing block
        const int kt = k0 + nb;
        panel_update<NT, NW, B>(kt, n, nb, A, PV, PW);
        __syncthreads();
        k = kt;
    }
    // the last 2 x 2 block, fully updated by the last panel
    if (tid == 0) {
        d[n - 2] = double(A[tri(n - 2) + n - 2].x);
        e2[n - 2] = double(cabs2(A[tri(n - 1) + n - 2]));
        d[n - 1] = double(A[tri(n - 1) + n - 1].x);
    }
    __syncthreads();
}

}  // namespace ptca
