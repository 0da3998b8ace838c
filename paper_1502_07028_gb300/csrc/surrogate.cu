// surrogate.cu -- BF16 tensor-core kernels of the surrogate network (training
// and inference) and the delayed-acceptance screening of a PTCA stage.
//
// Matrix products: operands are rounded to bfloat16 (round to nearest even)
// when staged into shared memory and multiplied on the tensor cores,
// accumulating in FP32.  The forward products (activations times the
// transposed weights) run on tcgen05 with the accumulator in tensor memory
// (k_gemm_tc); the transposed products of the backward pass use the
// mma.sync m16n8k16 tile loop (k_gemm_bf16).  Everything else (bias, SiLU,
// loss, AdamW) runs in FP32.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "surrogate.cuh"
#include "surrogate_launch.h"

namespace ptca {

// ---------------------------------------------------------------------------
// C[M x N] = A B (+ bias[n]), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn],
// C row-major with leading dimension ldc.  CTA tile 64 x 64, K step 16,
// 4 warps in 2 x 2, each warp 32 x 32 = 2 x 4 mma tiles of 16 x 8.
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 16;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const float* __restrict__ A, long long sam,
                                                   long long sak, const float* __restrict__ B, long long sbk,
                                                   long long sbn, const float* __restrict__ bias, float* __restrict__ C,
                                                   int ldc) {
    __shared__ __nv_bfloat16 As[GBM][GBK + 8];
    __shared__ __nv_bfloat16 Bs[GBK][GBN + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    for (int k0 = 0; k0 < K; k0 += GBK) {
        __syncthreads();
        for (int e = tid; e < GBM * GBK; e += 128) {
            const int r = e / GBK, kk = e % GBK;
            const int m = m0 + r, k = k0 + kk;
            const float v = (m < M && k < K) ? A[m * sam + k * sak] : 0.f;
            As[r][kk] = __float2bfloat16_rn(v);
        }
        for (int e = tid; e < GBK * GBN; e += 128) {
            const int kk = e / GBN, c = e % GBN;
            const int k = k0 + kk, n = n0 + c;
            const float v = (k < K && n < N) ? B[k * sbk + n * sbn] : 0.f;
            Bs[kk][c] = __float2bfloat16_rn(v);
        }
        __syncthreads();
        uint32_t af[2][4], bfr[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + 16 * i + g;
            af[i][0] = pack_bf16(As[r][2 * t], As[r][2 * t + 1]);
            af[i][1] = pack_bf16(As[r + 8][2 * t], As[r + 8][2 * t + 1]);
            af[i][2] = pack_bf16(As[r][2 * t + 8], As[r][2 * t + 9]);
            af[i][3] = pack_bf16(As[r + 8][2 * t + 8], As[r + 8][2 * t + 9]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = wn + 8 * j + g;
            bfr[j][0] = pack_bf16(Bs[2 * t][c], Bs[2 * t + 1][c]);
            bfr[j][1] = pack_bf16(Bs[2 * t + 8][c], Bs[2 * t + 9][c]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float* d = acc[i][j];
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                    : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                    : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
            }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + 16 * i + g + (q >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * t + (q & 1);
                if (m < M && n < N) C[(long long)m * ldc + n] = acc[i][j][q] + (bias ? bias[n] : 0.f);
            }
}

// ---------------------------------------------------------------------------
// The forward products of the network on the 5th-generation tensor cores:
// C[M x N] = A W^T (+ bias) for A row-major (M x K, leading dimension lda)
// and W row-major (N x K, leading dimension ldw), both FP32 in global memory,
// K <= 256.  CTA (i, j) of 8 warps computes rows 128 i .. 128 i + 127 and
// columns TC_NT j .. TC_NT j + TC_NT - 1:
//   * its warps round those rows of A and of W to bfloat16 (round to nearest
//     even, as k_gemm_bf16) into shared memory in the K-major, 128-byte
//     swizzled layout of the tensor cores: 64 K-elements (128 bytes) per row
//     and K block, 8-row atoms of 1024 bytes, the 16-byte chunk c of row r at
//     chunk position c ^ (r mod 8);
//   * one thread issues tcgen05.mma (kind::f16: BF16 x BF16 -> FP32 in
//     tensor memory; M = 128, N = the tile's width rounded up to 16, K = 16
//     per instruction) and commits them to an mbarrier;
//   * warps w and w + 4 read accumulator rows 32 (w mod 4) .. + 31 (the
//     tensor-memory lanes warp w may access), each half of the columns, with
//     tcgen05.ld, and write C with the bias.
// The wait on the mbarrier is bounded: past the limit the CTA writes NaN
// into its block of C, sets *err (if given) and still frees its tensor memory.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_KB = 64, TC_NT = 64, TC_THREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading offset
// (unused with swizzling), 1024 bytes between 8-row groups, descriptor
// version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5), BF16 A
// (bits 7-9) and B (bits 10-12), both K-major, N / 8 (bits 17-22), M / 16
// (bits 24-28).
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__host__ __device__ constexpr int tc_cols(int np) { return np <= 32 ? 32 : np <= 64 ? 64 : np <= 128 ? 128 : 256; }

// Width of the N tile (the whole of a narrow N), rounded up to 16.
__host__ __device__ constexpr int tc_ntile(int N) { return N < TC_NT ? (N + 15) / 16 * 16 : TC_NT; }

__host__ __device__ constexpr size_t tc_smem_bytes(int K, int N) {
    return (size_t)((K + TC_KB - 1) / TC_KB) * (TC_M + tc_ntile(N)) * 128 + 1024 + 64;
}

// Rows [r0, r0 + rows) of X (row-major, leading dimension ld; rows >= nrows
// and columns >= K read as 0) into the swizzled bf16 layout at dst.
__device__ __forceinline__ void tc_stage(unsigned char* dst, const float* __restrict__ X, int ld, int r0, int rows,
                                         int nrows, int K, int nkb) {
    for (int e = threadIdx.x; e < nkb * rows * 8; e += blockDim.x) {
        const int c = e & 7, r = (e >> 3) % rows, kb = (e >> 3) / rows;
        const int row = r0 + r, k = kb * TC_KB + 8 * c;
        float x[8];
        if (row < nrows && k + 8 <= K && ((ld | k) & 3) == 0) {
            const float4* q = reinterpret_cast<const float4*>(X + (long long)row * ld + k);
            const float4 a = q[0], b = q[1];
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
        } else {
#pragma unroll
            for (int h = 0; h < 8; ++h) x[h] = (row < nrows && k + h < K) ? X[(long long)row * ld + k + h] : 0.f;
        }
        uint4 v;
        v.x = pack_bf16(__float2bfloat16_rn(x[0]), __float2bfloat16_rn(x[1]));
        v.y = pack_bf16(__float2bfloat16_rn(x[2]), __float2bfloat16_rn(x[3]));
        v.z = pack_bf16(__float2bfloat16_rn(x[4]), __float2bfloat16_rn(x[5]));
        v.w = pack_bf16(__float2bfloat16_rn(x[6]), __float2bfloat16_rn(x[7]));
        *reinterpret_cast<uint4*>(dst + ((size_t)kb * rows + r) * 128 + ((c ^ (r & 7)) << 4)) = v;
    }
}

__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       const float* __restrict__ W, int ldw,
                                                       const float* __restrict__ bias, float* __restrict__ C, int ldc,
                                                       int* err) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char* base = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
    const int nkb = (K + TC_KB - 1) / TC_KB, Np = tc_ntile(N), ncols = tc_cols(Np);
    unsigned char* sA = base;
    unsigned char* sW = base + (size_t)nkb * TC_M * 128;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sW + (size_t)nkb * Np * 128);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * Np;
    tc_stage(sA, A, lda, m0, TC_M, M, K, nkb);
    tc_stage(sW, W + (long long)n0 * ldw, ldw, 0, Np, N - n0, K, nkb);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the staged operands and the barrier become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t idesc = tc_idesc(Np);
        for (int s = 0; s < 4 * nkb; ++s) {
            const int kb = s >> 2, kk = s & 3;
            const uint64_t ad = tc_desc(smem_u32(sA) + (uint32_t)(kb * TC_M * 128 + kk * 32));
            const uint64_t bd = tc_desc(smem_u32(sW) + (uint32_t)(kb * Np * 128 + kk * 32));
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(s > 0 ? 1 : 0) : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(bar)) : "memory");
    }
    // bounded wait for the products (phase 0 of the barrier)
    uint32_t done = 0;
    for (long long it = 0; it < (1ll << 24) && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done) : "r"(smem_u32(bar)) : "memory");
        if (!done && (it & 255) == 255) __nanosleep(64);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int quad = warp & 3, half = warp >> 2;
    const int m = m0 + 32 * quad + lane;
    const int cw = Np / 2;  // columns per warp of the pair (a multiple of 8)
    for (int c0 = half * cw; c0 < half * cw + cw; c0 += 8) {
        uint32_t r[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m < M) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = n0 + c0 + j;
                if (n < N) C[(long long)m * ldc + n] = done ? __uint_as_float(r[j]) + (bias ? bias[n] : 0.f) : nanf("");
            }
        }
    }
    if (!done && tid == 0 && err) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols) : "memory");
}

static bool g_tc_ready = false;

cudaError_t sg_gemm(int M, int N, int K, const float* A, long long sam, long long sak, const float* B, long long sbk,
                    long long sbn, const float* bias, float* C, int ldc, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (sak == 1 && sbk == 1 && K >= 1 && K <= 256 && N <= 256 && sam < (1ll << 30) && sbn < (1ll << 30)) {
        // A row-major, W = B^T row-major: the forward products (tensor cores, tcgen05)
        if (!g_tc_ready) {
            cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)tc_smem_bytes(256, 256));
            if (e != cudaSuccess) return e;
            g_tc_ready = true;
        }
        const dim3 grid((M + TC_M - 1) / TC_M, (N + tc_ntile(N) - 1) / tc_ntile(N));
        k_gemm_tc<<<grid, TC_THREADS, tc_smem_bytes(K, N), st>>>(M, N, K, A, (int)sam, B, (int)sbn, bias, C, ldc,
                                                                nullptr);
        return cudaGetLastError();
    }
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    k_gemm_bf16<<<grid, 128, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, C, ldc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Elementwise pieces (FP32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + __expf(-z)); }

__global__ void k_silu(const float* __restrict__ Z, float* __restrict__ A, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) { const float z = Z[i]; A[i] = z * sigmoidf_(z); }
}

// dZ = dA * silu'(Z), silu'(z) = s (1 + z (1 - s)), s = sigmoid(z).
__global__ void k_silu_bwd(const float* __restrict__ dA, const float* __restrict__ Z, float* __restrict__ dZ,
                           long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) { const float z = Z[i], s = sigmoidf_(z); dZ[i] = dA[i] * s * (1.f + z * (1.f - s)); }
}

// db[n] = sum_m dZ[m][n]
__global__ void k_colsum(const float* __restrict__ dZ, int M, int N, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += dZ[(long long)m * N + n];
    db[n] = s;
}

// Batch rows from stored samples: row b = c[P(s_old), s_new], row B + b =
// c[P(s_new), s_old], zero-padded to SG_IN_PAD; sample index = idx[b].
__global__ void k_pair_rows(const float* __restrict__ feat, const int32_t* __restrict__ center,
                            const int64_t* __restrict__ idx, int Bsz, float* __restrict__ X) {
    const int b = blockIdx.x;
    if (b >= Bsz) return;
    const long long s = idx[b];
    write_pair_rows(feat + s * SG_IN, center[s], X + (long long)b * SG_IN_PAD, X + (long long)(Bsz + b) * SG_IN_PAD);
}

// Sample indices of a training step from the counter generator.
__global__ void k_batch_indices(uint64_t seed, uint64_t step, int Bsz, long long nsamples, int64_t* idx) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bsz) return;
    double u0, u1;
    uniform2(seed, step, (uint32_t)b, RNG_BATCH, u0, u1);
    long long s = (long long)(u0 * (double)nsamples);
    idx[b] = s < nsamples ? s : nsamples - 1;
}

// Loss of the pair rows and the output-layer gradient: h = Z4[:, 0],
// r = h[b] - h[B+b] - dF/scale; loss = mean r^2; dZ4 = 0 except column 0.
__global__ void k_pair_loss(const float* __restrict__ Z4, const float* __restrict__ dF, const int64_t* __restrict__ idx,
                            int Bsz, float inv_scale, float* __restrict__ dZ4, float* __restrict__ loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.f;
    if (b < Bsz) {
        const float tgt = dF[idx[b]] * inv_scale;
        r = Z4[(long long)b * SG_OUT_PAD] - Z4[(long long)(Bsz + b) * SG_OUT_PAD] - tgt;
        for (int q = 0; q < SG_OUT_PAD; ++q) {
            dZ4[(long long)b * SG_OUT_PAD + q] = q == 0 ? 2.f * r / Bsz : 0.f;
            dZ4[(long long)(Bsz + b) * SG_OUT_PAD + q] = q == 0 ? -2.f * r / Bsz : 0.f;
        }
    }
    const float s = warp_sum(r * r);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, s / Bsz);
}

// AdamW (decoupled weight decay).
__global__ void k_adamw(float* __restrict__ w, float* __restrict__ m1, float* __restrict__ m2,
                        const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float wd,
                        float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    w[i] = w[i] * (1.f - lr * wd) - lr * (a / bc1) / (sqrtf(v / bc2) + eps);
}

cudaError_t sg_elementwise(int op, const float* a, const float* b, float* c, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int th = 256;
    const unsigned blocks = (unsigned)((n + th - 1) / th);
    if (op == 0) k_silu<<<blocks, th, 0, st>>>(a, c, n);
    else k_silu_bwd<<<blocks, th, 0, st>>>(a, b, c, n);
    return cudaGetLastError();
}

cudaError_t sg_colsum(const float* dZ, int M, int N, float* db, cudaStream_t st) {
    k_colsum<<<(N + 127) / 128, 128, 0, st>>>(dZ, M, N, db);
    return cudaGetLastError();
}

cudaError_t sg_pair_rows(const float* feat, const int32_t* center, const int64_t* idx, int Bsz, float* X,
                         cudaStream_t st) {
    if (Bsz <= 0) return cudaSuccess;
    k_pair_rows<<<Bsz, 64, 0, st>>>(feat, center, idx, Bsz, X);
    return cudaGetLastError();
}

cudaError_t sg_batch_indices(uint64_t seed, uint64_t step, int Bsz, long long nsamples, int64_t* idx,
                             cudaStream_t st) {
    k_batch_indices<<<(Bsz + 255) / 256, 256, 0, st>>>(seed, step, Bsz, nsamples, idx);
    return cudaGetLastError();
}

cudaError_t sg_pair_loss(const float* Z4, const float* dF, const int64_t* idx, int Bsz, float inv_scale, float* dZ4,
                         float* loss, cudaStream_t st) {
    k_pair_loss<<<(Bsz + 255) / 256, 256, 0, st>>>(Z4, dF, idx, Bsz, inv_scale, dZ4, loss);
    return cudaGetLastError();
}

cudaError_t sg_adamw(float* w, float* m1, float* m2, const float* g, int n, float lr, float b1, float b2, float eps,
                     float wd, int step, cudaStream_t st) {
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    k_adamw<<<(n + 255) / 256, 256, 0, st>>>(w, m1, m2, g, n, lr, b1, b2, eps, wd, bc1, bc2);
    return cudaGetLastError();
}

// He-style initial parameters: weights normal with variance 2/fan_in (fan_in
// 150 for the first layer, whose padding columns stay 0), biases 0, unused
// output rows 0.  Normals by Box-Muller from the counter generator.
__global__ void k_init_params(float* theta, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= SG_NPARAMS) return;
    float v = 0.f, sd = 0.f;
    if (i < SG_OFF_B1) {
        const int k = (i - SG_OFF_W1) % SG_IN_PAD;
        sd = k < SG_IN ? sqrtf(2.f / SG_IN) : 0.f;
    } else if (i >= SG_OFF_W2 && i < SG_OFF_B2) sd = sqrtf(2.f / SG_H);
    else if (i >= SG_OFF_W3 && i < SG_OFF_B3) sd = sqrtf(2.f / SG_H);
    else if (i >= SG_OFF_W4 && i < SG_OFF_W4 + SG_H) sd = sqrtf(1.f / SG_H);
    if (sd > 0.f) {
        double u0, u1;
        uniform2(seed, 0, (uint32_t)i, RNG_PARAM, u0, u1);
        v = sd * (float)(sqrt(-2.0 * log(u0)) * cos(2.0 * kPi * u1));
    }
    theta[i] = v;
}

__global__ void k_moments(const float* __restrict__ x, long long n, double* out2) {
    double s = 0.0, q = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        s += v;
        q += v * v;
    }
    s = warp_sum(s);
    q = warp_sum(q);
    if ((threadIdx.x & 31) == 0) { atomicAdd(out2, s); atomicAdd(out2 + 1, q); }
}

__global__ void k_iota(int64_t* idx, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) idx[i] = i;
}

cudaError_t sg_init_params(float* theta, uint64_t seed, cudaStream_t st) {
    k_init_params<<<(SG_NPARAMS + 255) / 256, 256, 0, st>>>(theta, seed);
    return cudaGetLastError();
}

cudaError_t sg_moments(const float* x, long long n, double* out2, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess || n <= 0) return e;
    k_moments<<<152, 256, 0, st>>>(x, n, out2);
    return cudaGetLastError();
}

cudaError_t sg_iota(int64_t* idx, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_iota<<<(n + 255) / 256, 256, 0, st>>>(idx, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Delayed-acceptance screening of one stage.
// ---------------------------------------------------------------------------
// Rows of the stage: row c = c[P(s_old), s_new], row count + c = c[P(s_new), s_old].
// Visit c of the screened list is stage index a.perm[c] (or c without a
// list).
__global__ void k_screen_rows(StageArgs a, float* __restrict__ X) {
    const int c = blockIdx.x;
    if (c >= a.count) return;
    __shared__ float f[SG_IN];
    __shared__ double sn[3];
    __shared__ int center;
    const int site = a.sites[a.perm ? a.perm[c] : c];
    const Window w = make_window(a.m, site);
    if (threadIdx.x == 0) {
        propose(a.m, a.sweep, (uint32_t)site, a.S_in + 3 * site, sn);
        center = patch_features(a.m, w, a.S_in, f);
        f[147] = (float)sn[0]; f[148] = (float)sn[1]; f[149] = (float)sn[2];
    }
    __syncthreads();
    write_pair_rows(f, center, X + (long long)c * SG_IN_PAD, X + (long long)(a.count + c) * SG_IN_PAD);
}

// Stage 1 of delayed acceptance: dF~ = scale (h1 - h2); pass to the exact
// solve with probability min(1, exp(-dF~/T)) (uniform from its own counter
// purpose).  Passing sites are appended to the work list (as stage indices);
// rejected sites keep their spin and are recorded (free energies NaN: not
// computed).  dFt is indexed by stage index; Z4 rows by list position.
__global__ void k_screen_decide(StageArgs a, const float* __restrict__ Z4, float scale, float* __restrict__ dFt,
                                int32_t* __restrict__ work, unsigned int* __restrict__ nwork) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.count) return;
    const int c = a.perm ? a.perm[k] : k;
    const int site = a.sites[c];
    const double d = (double)scale * ((double)Z4[(long long)k * SG_OUT_PAD] - (double)Z4[(long long)(a.count + k) * SG_OUT_PAD]);
    dFt[c] = (float)d;
    double u0, u1;
    uniform2(a.m.seed, a.sweep, (uint32_t)site, RNG_SCREEN, u0, u1);
    if (log(u0) < -d / a.m.T) {
        work[atomicAdd(nwork, 1u)] = c;
        return;
    }
    const double* so = a.S_in + 3 * site;
    double* dst = a.S_out + 3 * site;
    dst[0] = so[0]; dst[1] = so[1]; dst[2] = so[2];
    const int r = a.rec_base + c;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const Window w = make_window(a.m, site);
    a.rec_site[r] = site;
    a.rec_Fold[r] = nan;
    a.rec_Fnew[r] = nan;
    a.rec_lnu[r] = nan;
    a.rec_acc[r] = 0;
    a.rec_Facc[r] = nan;
    a.rec_fill[r] = nan;
    a.rec_n[r] = 2 * window_nsite(w);
    atomicAdd(&a.counters[3], 1ull);
}

__global__ void k_pair_difference(const float* __restrict__ Z4, int n, float scale, float* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) out[b] = scale * (Z4[(long long)b * SG_OUT_PAD] - Z4[(long long)(n + b) * SG_OUT_PAD]);
}

cudaError_t sg_screen_difference(const float* Z4, int n, float scale, float* out, cudaStream_t st) {
    k_pair_difference<<<(n + 255) / 256, 256, 0, st>>>(Z4, n, scale, out);
    return cudaGetLastError();
}

cudaError_t sg_screen_rows(const StageArgs& a, float* X, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    k_screen_rows<<<a.count, 64, 0, st>>>(a, X);
    return cudaGetLastError();
}

cudaError_t sg_screen_decide(const StageArgs& a, const float* Z4, float scale, float* dFt, int32_t* work,
                             unsigned int* nwork, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    k_screen_decide<<<(a.count + 127) / 128, 128, 0, st>>>(a, Z4, scale, dFt, work, nwork);
    return cudaGetLastError();
}

}  // namespace ptca
