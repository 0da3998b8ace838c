// device_common.cuh -- small device utilities shared by the PTCA kernels:
// complex arithmetic on float2/double2, warp and block reductions, and the
// Philox4x32-10 counter-based generator (Salmon et al., SC'11) that draws the
// initial spins, the proposals and the Metropolis uniforms.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ptca {

constexpr unsigned FULL_MASK = 0xffffffffu;

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename Cplx<T>::type;

__device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// Precision-explicit fused multiply-add and square root (no implicit
// promotion of float arguments to double).
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float sqroot(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqroot(double a) { return sqrt(a); }

// acc + a * b
template <typename V> __device__ __forceinline__ V cfma(V a, V b, V acc) {
    acc.x = fmadd(a.x, b.x, acc.x); acc.x = fmadd(-a.y, b.y, acc.x);
    acc.y = fmadd(a.x, b.y, acc.y); acc.y = fmadd(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a) * b
template <typename V> __device__ __forceinline__ V cfma_conj_a(V a, V b, V acc) {
    acc.x = fmadd(a.x, b.x, acc.x); acc.x = fmadd(a.y, b.y, acc.x);
    acc.y = fmadd(a.x, b.y, acc.y); acc.y = fmadd(-a.y, b.x, acc.y);
    return acc;
}
// acc - a * b
template <typename V> __device__ __forceinline__ V cfms(V a, V b, V acc) {
    acc.x = fmadd(-a.x, b.x, acc.x); acc.x = fmadd(a.y, b.y, acc.x);
    acc.y = fmadd(-a.x, b.y, acc.y); acc.y = fmadd(-a.y, b.x, acc.y);
    return acc;
}
// acc - a * conj(b)
template <typename V> __device__ __forceinline__ V cfms_conj_b(V a, V b, V acc) {
    acc.x = fmadd(-a.x, b.x, acc.x); acc.x = fmadd(-a.y, b.y, acc.x);
    acc.y = fmadd(-a.y, b.x, acc.y); acc.y = fmadd(a.x, b.y, acc.y);
    return acc;
}
template <typename V> __device__ __forceinline__ auto cabs2(V a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }

template <typename V> __device__ __forceinline__ V cshfl_xor(V v, int o) {
    v.x = __shfl_xor_sync(FULL_MASK, v.x, o);
    v.y = __shfl_xor_sync(FULL_MASK, v.y, o);
    return v;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}
template <typename T> __device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}

// Sum over the block; every thread receives the same value (fixed order).
// `red` must hold blockDim/32 entries and must not be read by another
// reduction until a later __syncthreads.
template <typename T> __device__ __forceinline__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = red[0];
    for (int w = 1; w < nw; ++w) s += red[w];
    return s;
}

// ---------------------------------------------------------------------------
// Philox4x32-10.  Round: multiply words 0 and 2 by the Philox multipliers,
// swap and xor the high halves with the odd words and the key; the key
// advances by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t a, b, c, d; };

__device__ __forceinline__ U4 philox10(uint32_t k0, uint32_t k1, U4 x) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * x.a, hi0 = __umulhi(0xD2511F53u, x.a);
        const uint32_t lo1 = 0xCD9E8D57u * x.c, hi1 = __umulhi(0xCD9E8D57u, x.c);
        U4 y;
        y.a = hi1 ^ x.b ^ k0;
        y.b = lo1;
        y.c = hi0 ^ x.d ^ k1;
        y.d = lo0;
        x = y;
    }
    return x;
}

enum : uint32_t {
    RNG_INIT = 0, RNG_PROPOSE = 1, RNG_ACCEPT = 2, RNG_SCREEN = 3, RNG_RADIUS = 4, RNG_BATCH = 16, RNG_PARAM = 17
};

// Two uniforms in (0,1) for (seed, sweep, site, purpose): each from 53 bits
// of one 64-bit half of the Philox output, (x + 1/2) 2^-53.
__device__ __forceinline__ void uniform2(uint64_t seed, uint64_t sweep, uint32_t site, uint32_t purpose,
                                         double& u0, double& u1) {
    U4 c{site, purpose, (uint32_t)sweep, (uint32_t)(sweep >> 32)};
    U4 r = philox10((uint32_t)seed, (uint32_t)(seed >> 32), c);
    const uint64_t a = ((uint64_t)r.b << 32) | r.a;
    const uint64_t b = ((uint64_t)r.d << 32) | r.c;
    u0 = ((double)(a >> 11) + 0.5) * 0x1p-53;
    u1 = ((double)(b >> 11) + 0.5) * 0x1p-53;
}

constexpr double kPi = 3.14159265358979323846;

// Unit vector from two uniforms: z = 2 u0 - 1, azimuth 2 pi u1.
__device__ __forceinline__ void unit_from_uniforms(double u0, double u1, double s[3]) {
    const double z = 2.0 * u0 - 1.0;
    const double r = sqrt(fmax(0.0, 1.0 - z * z));
    double sn, cs;
    sincos(2.0 * kPi * u1, &sn, &cs);
    s[0] = r * cs;
    s[1] = r * sn;
    s[2] = z;
}

// Proposal for the spin at `site` (Sec. II.c step c).  proposal 0: uniform on
// the sphere.  proposal 1: uniform on the cap of half-angle acos(cone_cos)
// around s_old, drawn about +z and turned onto s_old by the rotation that
// maps +z to s_old (rotation by pi about x when s_old is at -z).
__device__ __forceinline__ void propose_spin(uint64_t seed, uint64_t sweep, uint32_t site, int proposal,
                                             double cone_cos, const double so[3], double sn[3]) {
    double u0, u1;
    uniform2(seed, sweep, site, RNG_PROPOSE, u0, u1);
    if (proposal == 0) { unit_from_uniforms(u0, u1, sn); return; }
    const double ct = 1.0 - u0 * (1.0 - cone_cos);
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double sp, cp;
    sincos(2.0 * kPi * u1, &sp, &cp);
    const double v0 = st * cp, v1 = st * sp, v2 = ct;
    const double a = so[0], b = so[1], c = so[2];
    double r0, r1, r2;
    if (c < -1.0 + 1e-12) {
        r0 = v0; r1 = -v1; r2 = -v2;
    } else {
        const double k = 1.0 / (1.0 + c);
        r0 = (1.0 - a * a * k) * v0 + (-a * b * k) * v1 + a * v2;
        r1 = (-a * b * k) * v0 + (1.0 - b * b * k) * v1 + b * v2;
        r2 = -a * v0 - b * v1 + c * v2;
    }
    const double inv = 1.0 / sqrt(r0 * r0 + r1 * r1 + r2 * r2);
    sn[0] = r0 * inv; sn[1] = r1 * inv; sn[2] = r2 * inv;
}

}  // namespace ptca
