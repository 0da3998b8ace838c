// kernels_large.cu -- instantiation and launchers of the large-cluster
// kernels (orders above the shared-memory kernels' reach, up to 512): the
// FP32 and FP64 stage kernels and the double-float re-solve, all with the
// matrix in a global slot per CTA.
#include "kernels.cuh"
#include "launch.h"

namespace ptca {

namespace {

size_t large_layout(size_t cs) { return smem_layout(0, 32 * NW_LARGE, cs, NW_LARGE).total; }

template <typename K> cudaError_t allow_smem(K kernel, size_t need, size_t smem_limit) {
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, kernel);
    if (e != cudaSuccess) return e;
    if (need + attr.sharedSizeBytes > smem_limit) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
}

}  // namespace

int large_max_order() { return 32 * NW_LARGE; }

size_t large_smem_bytes(int prec) { return large_layout(prec == 1 ? sizeof(float2) : sizeof(double2)); }

cudaError_t configure_large_kernels(size_t smem_limit) {
    cudaError_t e = allow_smem(k_stage_large<float>, large_layout(sizeof(float2)), smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_stage_large<double>, large_layout(sizeof(double2)), smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_resolve_large<>, large_layout(sizeof(dfl2)), smem_limit);
    return e;
}

int large_blocks_per_sm(int prec) {
    int b = 0;
    cudaError_t e = prec == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_stage_large<float>, 32 * NW_LARGE,
                                                                              large_layout(sizeof(float2)))
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_stage_large<double>, 32 * NW_LARGE,
                                                                              large_layout(sizeof(double2)));
    return e == cudaSuccess ? b : 0;
}

cudaError_t launch_stage_large(int prec, const StageArgs& a, int grid, cudaStream_t st) {
    if (a.count <= 0 && a.prev_count + a.prev2_count <= 0) return cudaSuccess;
    if (prec == 1)
        k_stage_large<float><<<grid, 32 * NW_LARGE, large_layout(sizeof(float2)), st>>>(a);
    else
        k_stage_large<double><<<grid, 32 * NW_LARGE, large_layout(sizeof(double2)), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resolve_large(const StageArgs& a, int grid, cudaStream_t st) {
    k_resolve_large<><<<grid, 32 * NW_LARGE, large_layout(sizeof(dfl2)), st>>>(a);
    return cudaGetLastError();
}

}  // namespace ptca
