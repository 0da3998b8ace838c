// FP32 sweep kernel of 4-warp CTAs with the register-tiled Householder
// reduction (orders up to 128; per-stage and overlapped pipelines).
#include "kernels.cuh"
#include "launch.h"

namespace ptca {

size_t tiled_smem_bytes() { return smem_layout_tiled().total; }

bool tiled_supported(int prec, int nA) { return prec == 1 && nA >= 1 && nA <= TL_NMAX; }

cudaError_t configure_tiled_kernels(size_t smem_limit) {
    const size_t need = tiled_smem_bytes();
    if (need > smem_limit) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_stage<float, 4, TL_NW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)need);
}

cudaError_t launch_stage_tiled(const StageArgs& a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (a.nA > TL_NMAX) return cudaErrorInvalidValue;
    k_stage<float, 4, TL_NW, true><<<2 * a.count, 32 * TL_NW, tiled_smem_bytes(), st>>>(a);
    return cudaGetLastError();
}

}  // namespace ptca
