// surrogate_launch.h -- host launchers of the surrogate kernels (surrogate.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ptca {

struct StageArgs;

// C[M x N] = A B (+ bias), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn];
// BF16 operands on the tensor cores, FP32 accumulation.
cudaError_t sg_gemm(int M, int N, int K, const float* A, long long sam, long long sak, const float* B, long long sbk,
                    long long sbn, const float* bias, float* C, int ldc, cudaStream_t st);
// op 0: c = silu(a); op 1: c = a * silu'(b).
cudaError_t sg_elementwise(int op, const float* a, const float* b, float* c, long long n, cudaStream_t st);
cudaError_t sg_colsum(const float* dZ, int M, int N, float* db, cudaStream_t st);
cudaError_t sg_pair_rows(const float* feat, const int32_t* center, const int64_t* idx, int Bsz, float* X,
                         cudaStream_t st);
cudaError_t sg_batch_indices(uint64_t seed, uint64_t step, int Bsz, long long nsamples, int64_t* idx,
                             cudaStream_t st);
cudaError_t sg_pair_loss(const float* Z4, const float* dF, const int64_t* idx, int Bsz, float inv_scale, float* dZ4,
                         float* loss, cudaStream_t st);
cudaError_t sg_adamw(float* w, float* m1, float* m2, const float* g, int n, float lr, float b1, float b2, float eps,
                     float wd, int step, cudaStream_t st);
cudaError_t sg_screen_rows(const StageArgs& a, float* X, cudaStream_t st);
cudaError_t sg_screen_decide(const StageArgs& a, const float* Z4, float scale, float* dFt, int32_t* work,
                             unsigned int* nwork, cudaStream_t st);
// out[b] = scale (h[b] - h[n + b]) from the output layer Z4 (2n x 8).
cudaError_t sg_screen_difference(const float* Z4, int n, float scale, float* out, cudaStream_t st);
cudaError_t sg_init_params(float* theta, uint64_t seed, cudaStream_t st);
cudaError_t sg_moments(const float* x, long long n, double* out2, cudaStream_t st);
cudaError_t sg_iota(int64_t* idx, int n, cudaStream_t st);

}  // namespace ptca
