// surrogate.cuh -- inputs of the surrogate network used for delayed-acceptance
// screening of PTCA proposals.
//
// Input of the network h (150 values): a 7x7 patch of the traveling-cluster
// window around the update site (row-major over the patch, 3 spin components
// per site), then a 3-vector.  Along an axis on which the cluster is periodic
// and at least 7 wide the patch is centred on the update site and wraps inside
// the window, so that it holds the site's neighbours in the cluster
// Hamiltonian; otherwise it is placed as centrally as the window allows.  For a
// proposal s_old -> s_new the surrogate free-energy change is
//     dF~ = scale * ( h(c[P(s_old), s_new]) - h(c[P(s_new), s_old]) ),
// where P(s) is the patch with the update site's entry set to s and c[...]
// rotates every spin of a row into the row's own frame: its update-site spin
// along +z and its last spin in the xz half-plane with x >= 0.  The cluster
// spectrum does not change under a global spin rotation, so the frame removes
// three symmetry directions from what the network has to learn; exchanging
// the two states flips the sign of dF~, which delayed acceptance needs for
// detailed balance.
#pragma once

#include "cluster_solve.cuh"

namespace ptca {

constexpr int SG_PATCH = 7;
constexpr int SG_IN = 150;       // network inputs
constexpr int SG_IN_PAD = 160;   // first-layer K (multiple of the MMA K tile)
constexpr int SG_H = 256;        // hidden width
constexpr int SG_OUT_PAD = 8;    // last-layer rows (only row 0 is used)
// Parameter vector layout: W1[H x IN_PAD] b1[H] W2[H x H] b2[H] W3[H x H] b3[H] W4[OUT_PAD x H] b4[OUT_PAD]
constexpr int SG_OFF_W1 = 0;
constexpr int SG_OFF_B1 = SG_OFF_W1 + SG_H * SG_IN_PAD;
constexpr int SG_OFF_W2 = SG_OFF_B1 + SG_H;
constexpr int SG_OFF_B2 = SG_OFF_W2 + SG_H * SG_H;
constexpr int SG_OFF_W3 = SG_OFF_B2 + SG_H;
constexpr int SG_OFF_B3 = SG_OFF_W3 + SG_H * SG_H;
constexpr int SG_OFF_W4 = SG_OFF_B3 + SG_H;
constexpr int SG_OFF_B4 = SG_OFF_W4 + SG_OUT_PAD * SG_H;
constexpr int SG_NPARAMS = SG_OFF_B4 + SG_OUT_PAD;

// Start of the patch along one axis of extent e, update site at u; wrap is
// set when the patch wraps inside a periodic window.
__device__ __forceinline__ int patch_start(int e, int u, int periodic, bool& wrap) {
    wrap = periodic && e >= SG_PATCH;
    if (wrap) return u - SG_PATCH / 2;
    const int mx = e - SG_PATCH > 0 ? e - SG_PATCH : 0;
    const int p = u - SG_PATCH / 2;
    return p < 0 ? 0 : (p > mx ? mx : p);
}

// Patch of the window around the update site from the spins S (the stage's
// starting configuration); entries outside a window smaller than 7 are 0.
// Writes 147 values to out and returns the update site's patch index.
__device__ __forceinline__ int patch_features(const Model& m, const Window& w, const double* __restrict__ S,
                                              float* out) {
    bool wrx, wry;
    const int px = patch_start(w.ex, w.uwx, m.cluster_periodic, wrx);
    const int py = patch_start(w.ey, w.uwy, m.cluster_periodic, wry);
    for (int b = 0; b < SG_PATCH; ++b)
        for (int a = 0; a < SG_PATCH; ++a) {
            int wx = px + a, wy = py + b;
            if (wrx) wx = (wx + w.ex) % w.ex;
            if (wry) wy = (wy + w.ey) % w.ey;
            const int q = 3 * (b * SG_PATCH + a);
            if (wx < w.ex && wy < w.ey) {
                const int g = window_site(m, w, wx, wy);
                out[q] = (float)S[3 * g]; out[q + 1] = (float)S[3 * g + 1]; out[q + 2] = (float)S[3 * g + 2];
            } else {
                out[q] = 0.f; out[q + 1] = 0.f; out[q + 2] = 0.f;
            }
        }
    return (w.uwy - py) * SG_PATCH + (w.uwx - px);
}

// Rows e1, e2, e3 of the rotation taking a to +z and b into the xz half-plane
// (x >= 0): e3 = a/|a|, e1 = the normalised part of b orthogonal to e3 (of x,
// then y, when b is parallel to a), e2 = e3 x e1.
__device__ __forceinline__ void spin_frame(const float* a, const float* b, double* R) {
    double e3[3] = {a[0], a[1], a[2]};
    const double na = sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
    for (int i = 0; i < 3; ++i) e3[i] /= na;
    double e1[3] = {1.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
        const double c[3] = {k == 0 ? (double)b[0] : (k == 1 ? 1.0 : 0.0),
                             k == 0 ? (double)b[1] : (k == 1 ? 0.0 : 1.0),
                             k == 0 ? (double)b[2] : 0.0};
        const double d = c[0] * e3[0] + c[1] * e3[1] + c[2] * e3[2];
        const double r[3] = {c[0] - d * e3[0], c[1] - d * e3[1], c[2] - d * e3[2]};
        const double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (nr > 1e-6) { e1[0] = r[0] / nr; e1[1] = r[1] / nr; e1[2] = r[2] / nr; break; }
    }
    R[0] = e1[0]; R[1] = e1[1]; R[2] = e1[2];
    R[3] = e3[1] * e1[2] - e3[2] * e1[1];
    R[4] = e3[2] * e1[0] - e3[0] * e1[2];
    R[5] = e3[0] * e1[1] - e3[1] * e1[0];
    R[6] = e3[0]; R[7] = e3[1]; R[8] = e3[2];
}

// The two network rows of one sample f (150 values: patch with s_old at patch
// index c, then s_new), each in its own frame, zero-padded to SG_IN_PAD:
// x1 = c[P(s_old), s_new], x2 = c[P(s_new), s_old].  Called by the whole block.
__device__ __forceinline__ void write_pair_rows(const float* f, int c, float* __restrict__ x1,
                                                float* __restrict__ x2) {
    __shared__ double R[2][9];
    if (threadIdx.x == 0) {
        spin_frame(f + 3 * c, f + 147, R[0]);
        spin_frame(f + 147, f + 3 * c, R[1]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SG_IN_PAD; k += blockDim.x) {
        if (k >= SG_IN) { x1[k] = 0.f; x2[k] = 0.f; continue; }
        const int j = k / 3, q = k - 3 * j;
        const int j2 = j == c ? 49 : (j == 49 ? c : j);
        const float* v1 = f + 3 * j;
        const float* v2 = f + 3 * j2;
        x1[k] = (float)(R[0][3 * q] * v1[0] + R[0][3 * q + 1] * v1[1] + R[0][3 * q + 2] * v1[2]);
        x2[k] = (float)(R[1][3 * q] * v2[0] + R[1][3 * q + 1] * v2[1] + R[1][3 * q + 2] * v2[2]);
    }
}

}  // namespace ptca
