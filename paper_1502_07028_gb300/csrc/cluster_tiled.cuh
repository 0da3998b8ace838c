// cluster_tiled.cuh -- register-tiled form of the FP32 Householder reduction
// (Sec. II.c step b: the cluster diagonalisation), for 4-warp CTAs and
// matrix orders up to 128.
//
// The arithmetic is that of householder_tridiag (reflector k of column k,
// deferred rank-2 update of step k-1 fused with the product p = tau A v_k,
// the explicit update of the next pivot column); only the organisation of
// the fused pass differs.
//
// Storage (tl_at, tl_pos): the lower block triangle of 4x4 complex tiles,
// tile t = R(R+1)/2 + C (C <= R) at elements 16t .. 16t+15, its 16-byte slots
// swizzled by t mod 8 so that lanes reading consecutive tiles hit distinct
// banks.  Diagonal tiles hold both triangles (Hermitian); rows and columns
// past the order n, up to the next multiple of 4, are zero and stay zero.
//
// Fused pass of step k (active corner j0 = k+1 in block K = j0/4, M = NB - K
// active block rows): the off-diagonal tiles of block rows K+p and K+M-1-p
// form pair p (p tiles in the first row, M-1-p in the second: M-1 in all).
// A warp takes one pair at a time, one tile per lane: lane l holds tile
// (K+p, K+l) if l < p, else tile (K+M-1-p, K+M-2-l), so across the pairs a
// lane meets only the column blocks K+l and K+M-2-l and keeps their column
// sums (A^H v) in registers.  Each lane updates its tile in registers with
// the previous step's (u, w), stores it once, and forms its row sums (A v) and
// column sums; the row sums of the pair are reduce-scattered across the warp.
// One warp also updates the diagonal tiles, one per lane.  Vector entries
// outside the active range are kept zero in shared memory (each reflector's
// first entry stays in registers and is substituted where a lane loads the
// block holding it), so tiles that straddle the corner need no masks.  Per
// warp, the sums are added into the warp's partial vector in a fixed order
// (zero, the row sums pair by pair, the column sums, the diagonal tiles' row
// sums), and the scalar phase adds the warps' vectors in warp order: the
// result does not depend on timing.  The pass also sums v^H A v, so a
// reflector step needs two barriers (after the pass, after the scalar phase).
#pragma once

#include "cluster_solve.cuh"

namespace ptca {

constexpr int TL_NW = 4;     // warps per CTA
constexpr int TL_NMAX = 128; // largest order

// Scratch of the tiled reduction (shared memory): the two reflectors, w of the
// previous step, the per-warp partial vectors of p, the block-sum slots and
// the three scalars of the per-step tail; d and e2 in FP32 (the reduction
// produces FP32 values).
struct TlScratch {
    float2* Vb;   // 2 x TL_NMAX
    float2* Wv;   // TL_NMAX
    float2* pc;   // TL_NW x TL_NMAX
    float* redA;  // TL_NW
    float* redB;  // TL_NW
    float2* sx;   // 3
    float* d;     // TL_NMAX
    float* e2;    // TL_NMAX
};

__device__ __forceinline__ void tl_ld4(const float2* p, float2 (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 2);
    v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
}

// v_k's first entry (index j0, kept in registers, zero in shared memory) into
// the loaded block of entries 4K .. 4K+3 that holds it.
__device__ __forceinline__ void tl_put_first(float2 (&v)[4], int j0, float2 vfirst) {
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (e == (j0 & 3)) v[e] = vfirst;
}

// Tile t (16 complex elements at A + 16 t) into registers, slot h from
// position h ^ (t mod 8), and back.
__device__ __forceinline__ void tl_load_tile(const float2* A, int t, float2 (&a)[16]) {
    const float4* tp = reinterpret_cast<const float4*>(A + (t << 4));
    const int sw = t & 7;
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const float4 x = tp[h ^ sw];
        a[2 * h] = make_float2(x.x, x.y);
        a[2 * h + 1] = make_float2(x.z, x.w);
    }
}
__device__ __forceinline__ void tl_store_tile(float2* A, int t, const float2 (&a)[16]) {
    float4* tp = reinterpret_cast<float4*>(A + (t << 4));
    const int sw = t & 7;
#pragma unroll
    for (int h = 0; h < 8; ++h) tp[h ^ sw] = make_float4(a[2 * h].x, a[2 * h].y, a[2 * h + 1].x, a[2 * h + 1].y);
}

// One fused pass (step k): A <- A - u w^H - w u^H with (u, w) of step k-1,
// the per-warp partial sums of A v_k into sc.pc and each warp's share of
// v_k^H A v_k into sc.redA.  Caller syncs after.
//
// Over the pairs of a warp (p = warp, warp + 4, ...) lane l first works in
// the second row of each pair (column block K+M-2-l, while p <= l) and then
// in the first (column block K+l): its column block changes at most once,
// so its column vectors (u, w, v of the block) and the column sums of the
// current block stay in registers.
__device__ __forceinline__ void tl_pass(int k, int n, float2* A, const TlScratch& sc, float2 vfirst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = k + 1, K = j0 >> 2, NB = (n + 3) >> 2, M = NB - K;
    const float2* V_ = sc.Vb + (k & 1) * TL_NMAX;        // v_k
    const float2* U_ = sc.Vb + ((k + 1) & 1) * TL_NMAX;  // v_{k-1}
    const float2* W_ = sc.Wv;                            // w_{k-1}
    float2* pcw = sc.pc + warp * TL_NMAX - j0;           // indexed by absolute row
    const float2 zero = make_float2(0.f, 0.f);

    // Zero this warp's partial vector over the active rows (block K + lane).
    if (lane < M) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = 4 * (K + lane) + e;
            if (i >= j0 && i < n) pcw[i] = zero;
        }
    }
    __syncwarp();

    float2 cc[4], cb[4];             // column sums: current block, and block K+M-2-lane once left
    float2 uC[4], wC[4], vC[4];      // vectors of the current column block
#pragma unroll
    for (int e = 0; e < 4; ++e) { cc[e] = zero; cb[e] = zero; uC[e] = zero; wC[e] = zero; vC[e] = zero; }
    int cur = -1;                    // current segment: 0 first row (block K+l), 1 second row (block K+M-2-l)
    float vav = 0.f;                 // this lane's share of v^H A v (real: A is Hermitian)

    const int npair = M >= 2 ? (M + 1) >> 1 : 0;
    for (int p = warp; p < npair; p += TL_NW) {
        const int ra = K + p, rb = K + M - 1 - p;
        const bool mid = ra == rb;
        const int seg = lane < p ? 0 : ((!mid && lane <= M - 2) ? 1 : -1);
        if (seg >= 0 && seg != cur) {
            // entering a segment (second row -> first row at most once)
            if (cur == 1) {
#pragma unroll
                for (int e = 0; e < 4; ++e) { cb[e] = cc[e]; cc[e] = zero; }
            }
            const int C = seg ? K + M - 2 - lane : K + lane;
            tl_ld4(U_ + 4 * C, uC); tl_ld4(W_ + 4 * C, wC); tl_ld4(V_ + 4 * C, vC);
            if (C == K) tl_put_first(vC, j0, vfirst);
            cur = seg;
        }
        float2 q[4] = {zero, zero, zero, zero};
        if (seg >= 0) {
            const int R = seg ? rb : ra, C = seg ? K + M - 2 - lane : K + lane;
            const int t = tri(R) + C;
            float2 a[16];
            tl_load_tile(A, t, a);
            float2 uR[4], wR[4], vR[4];
            tl_ld4(U_ + 4 * R, uR); tl_ld4(W_ + 4 * R, wR); tl_ld4(V_ + 4 * R, vR);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 x = a[4 * i + j];
                    x = cfms_conj_b(uR[i], wC[j], x);
                    x = cfms_conj_b(wR[i], uC[j], x);
                    a[4 * i + j] = x;
                    q[i] = cfma(x, vC[j], q[i]);
                    cc[j] = cfma_conj_a(x, vR[i], cc[j]);
                }
            }
            tl_store_tile(A, t, a);
            // this tile's share of v^H A v: v_R^H q + v_C^H (A^H v_R) = 2 Re(v_R^H q)
#pragma unroll
            for (int i = 0; i < 4; ++i) vav = fmaf(2.f * vR[i].x, q[i].x, fmaf(2.f * vR[i].y, q[i].y, vav));
        }
        const bool segb = seg == 1;
        // Reduce-scatter the pair's 16 row-sum floats (row ra: 0..7, row rb:
        // 8..15; element e real/imag at 2e, 2e+1) over the 32 lanes: after
        // halving across lane bits 4, 3, 2, 1 and a final exchange across
        // bit 0, lane l holds float (l >> 1) & 15, summed over every lane.
        float x8[8];
        {
            const bool up = lane & 16;  // keeps floats 8..15
            const bool keep = up == segb;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float mx = keep ? q[e].x : 0.f, my = keep ? q[e].y : 0.f;
                const float ox = keep ? 0.f : q[e].x, oy = keep ? 0.f : q[e].y;
                x8[2 * e] = mx + __shfl_xor_sync(FULL_MASK, ox, 16);
                x8[2 * e + 1] = my + __shfl_xor_sync(FULL_MASK, oy, 16);
            }
        }
        float x4[4];
        {
            const bool up = lane & 8;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const float m = up ? x8[f + 4] : x8[f];
                const float o = up ? x8[f] : x8[f + 4];
                x4[f] = m + __shfl_xor_sync(FULL_MASK, o, 8);
            }
        }
        float x2[2];
        {
            const bool up = lane & 4;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const float m = up ? x4[f + 2] : x4[f];
                const float o = up ? x4[f] : x4[f + 2];
                x2[f] = m + __shfl_xor_sync(FULL_MASK, o, 4);
            }
        }
        float x1;
        {
            const bool up = lane & 2;
            const float m = up ? x2[1] : x2[0];
            const float o = up ? x2[0] : x2[1];
            x1 = m + __shfl_xor_sync(FULL_MASK, o, 2);
        }
        x1 += __shfl_xor_sync(FULL_MASK, x1, 1);
        if ((lane & 1) == 0) {
            const int f = (lane >> 1) & 15;
            const int s = f >> 3, e = (f >> 1) & 3;
            if (!(s && mid)) {
                const int i = 4 * (s ? rb : ra) + e;
                if (i >= j0 && i < n) reinterpret_cast<float*>(pcw + i)[f & 1] += x1;
            }
        }
        __syncwarp();
    }

    // Column sums: block K + lane, then block K + M - 2 - lane.
    if (cur == 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e) { cb[e] = cc[e]; cc[e] = zero; }
    }
    if (lane < M) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = 4 * (K + lane) + e;
            if (i >= j0 && i < n) pcw[i] = cadd(pcw[i], cc[e]);
        }
    }
    __syncwarp();
    if (lane <= M - 2) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = 4 * (K + M - 2 - lane) + e;
            if (i >= j0 && i < n) pcw[i] = cadd(pcw[i], cb[e]);
        }
    }
    __syncwarp();

    // Diagonal tiles (last warp), tile (K + lane, K + lane): the lower
    // triangle is updated and mirrored (the diagonal kept real), then the
    // full Hermitian tile multiplies v.
    if (warp == TL_NW - 1 && lane < M) {
        const int R = K + lane, t = tri(R) + R;
        float2 a[16];
        tl_load_tile(A, t, a);
        float2 u[4], w[4], v[4];
        tl_ld4(U_ + 4 * R, u); tl_ld4(W_ + 4 * R, w); tl_ld4(V_ + 4 * R, v);
        if (R == K) tl_put_first(v, j0, vfirst);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j < i; ++j) {
                float2 x = a[4 * i + j];
                x = cfms_conj_b(u[i], w[j], x);
                x = cfms_conj_b(w[i], u[j], x);
                a[4 * i + j] = x;
                a[4 * j + i] = make_float2(x.x, -x.y);
            }
            // diagonal: a_ii - 2 Re(u_i conj(w_i))
            a[5 * i] = make_float2(a[5 * i].x - 2.f * (u[i].x * w[i].x + u[i].y * w[i].y), 0.f);
        }
        tl_store_tile(A, t, a);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 sacc = zero;
#pragma unroll
            for (int j = 0; j < 4; ++j) sacc = cfma(a[4 * i + j], v[j], sacc);
            vav = fmaf(v[i].x, sacc.x, fmaf(v[i].y, sacc.y, vav));
            const int r = 4 * R + i;
            if (r >= j0 && r < n) pcw[r] = cadd(pcw[r], sacc);
        }
    }
    vav = warp_sum(vav);
    if (lane == 0) sc.redA[warp] = vav;
}

// Householder tridiagonalisation of the tiled Hermitian matrix A (order
// n <= 128), by 4-warp CTAs.  Writes d[0..n-1] and the squared off-diagonal
// moduli e2[0..n-2] (FP32).
__device__ inline void householder_tridiag_tiled(int n, float2* A, const TlScratch& sc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2 zero = make_float2(0.f, 0.f);
    float2* const Vb = sc.Vb;
    float2* const Wv = sc.Wv;
    for (int i = tid; i < 2 * TL_NMAX; i += TL_NW * 32) Vb[i] = zero;
    for (int i = tid; i < TL_NMAX; i += TL_NW * 32) Wv[i] = zero;
    __syncthreads();
    if (n <= 2) {
        if (tid == 0) {
            sc.d[0] = A[tl_at(0, 0)].x;
            if (n == 2) { sc.d[1] = A[tl_at(1, 1)].x; sc.e2[0] = cabs2(A[tl_at(1, 0)]); }
        }
        __syncthreads();
        return;
    }
    float2 vfirst;
    float tau;
    // Column 0: d_0, ||x||^2 and the first reflector (entry 1 in registers,
    // the rest in Vb).
    {
        const int ri = tid;
        float s2p = 0.f;
        if (ri < n) {
            const float2 a = A[tl_at(ri, 0)];
            if (ri == 0) sc.d[0] = a.x;
            if (ri >= 1) s2p = cabs2(a);
            if (ri >= 2) Vb[ri] = a;
            if (ri == 1) sc.sx[0] = a;
        }
        s2p = warp_sum(s2p);
        if (lane == 0) sc.redB[warp] = s2p;
        __syncthreads();
        const float s2 = sc.redB[0] + sc.redB[1] + sc.redB[2] + sc.redB[3];
        if (tid == 0) sc.e2[0] = s2;
        reflector_head(s2, sc.sx[0], vfirst, tau);
    }

    // Shared-memory vectors hold zero at and below each reflector's first
    // entry (kept in registers, vfirst); the pass substitutes it.  Per step:
    // the pass, then one phase (p, w, the pivot column, the next column's
    // norm) and its block sum: two barriers.
    for (int k = 0; k <= n - 3; ++k) {
        const int j0 = k + 1;
        const float2* V_ = Vb + (k & 1) * TL_NMAX;  // v_k
        float2* Vn = Vb + ((k + 1) & 1) * TL_NMAX;  // v_{k-1}, then v_{k+1}
        tl_pass(k, n, A, sc, vfirst);
        __syncthreads();

        // ---- p = tau A v (sum of the warps' partial vectors, in warp
        // order), K = (tau/2) v^H p = (tau^2/2) v^H A v, w = p - K v, the
        // explicit update of pivot column j0 with (v_k, w_k), d_j0, and the
        // partial sums of ||x||^2 of the next reflector, whose entries past
        // the first go to Vn (entries j0 and j0+1 of Vn and entry j0 of w
        // cleared).
        const int m = n - j0;
        const int ri = tid;
        const int nact = (m + 31) >> 5;
        if (warp < nact) {
            const float vAv = sc.redA[0] + sc.redA[1] + sc.redA[2] + sc.redA[3];
            const float Kc = 0.5f * tau * tau * vAv;
            float2 p0 = sc.pc[0];
#pragma unroll
            for (int w = 1; w < TL_NW; ++w) p0 = cadd(p0, sc.pc[w * TL_NMAX]);
            const float2 w0 = make_float2(tau * p0.x - Kc * vfirst.x, tau * p0.y - Kc * vfirst.y);
            float s2p = 0.f;
            if (ri < m) {
                float2 p = sc.pc[ri];
#pragma unroll
                for (int w = 1; w < TL_NW; ++w) p = cadd(p, sc.pc[w * TL_NMAX + ri]);
                const float2 v = ri == 0 ? vfirst : V_[j0 + ri];
                const float2 w = make_float2(tau * p.x - Kc * v.x, tau * p.y - Kc * v.y);
                Wv[j0 + ri] = ri == 0 ? zero : w;
                float2 a = A[tl_at(j0 + ri, j0)];
                a = cfms_conj_b(v, w0, a);
                a = cfms_conj_b(w, vfirst, a);
                if (ri == 0) sc.d[j0] = a.x;
                if (ri >= 1) s2p = cabs2(a);
                Vn[j0 + ri] = ri >= 2 ? a : zero;
                if (ri == 1) sc.sx[0] = a;
            }
            s2p = warp_sum(s2p);
            if (lane == 0) sc.redB[warp] = s2p;
        }
        __syncthreads();

        // ---- ||x||^2, and the next reflector's first entry and tau.
        float s2 = sc.redB[0];
#pragma unroll
        for (int w = 1; w < TL_NW; ++w)
            if (w < nact) s2 += sc.redB[w];
        if (tid == 0) sc.e2[j0] = s2;
        if (k + 1 <= n - 3) reflector_head(s2, sc.sx[0], vfirst, tau);
    }
    // Step n-3's update of the last diagonal entry.
    if (tid == 0) {
        const float2 v = Vb[((n - 3) & 1) * TL_NMAX + n - 1];
        const float2 w = Wv[n - 1];
        sc.d[n - 1] = A[tl_at(n - 1, n - 1)].x - 2.f * (v.x * w.x + v.y * w.y);
    }
    __syncthreads();
}

}  // namespace ptca
