// FP32 stage kernel with one Householder reduction shared by the two
// matrices of a visit (launch configuration reduction = PTCA_REDUCTION_SHARED):
// 4-warp CTAs, one per update site, orders up to 128.
#include "cluster_shared.cuh"
#include "launch.h"

namespace ptca {

size_t shared_smem_bytes() { return sh_layout().total; }

bool shared_supported(int prec, int nA) { return prec == 1 && nA >= 2 && nA <= SH_NMAX; }

cudaError_t configure_shared_kernels(size_t smem_limit) {
    const size_t need = sh_layout().total;
    if (need > smem_limit) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_stage_shared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
}

cudaError_t launch_stage_shared(const StageArgs& a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    k_stage_shared<<<a.count, 32 * SH_NW, sh_layout().total, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ptca
