// FP32 stage kernels with one Householder reduction shared by the two
// matrices of a visit (launch configuration reduction = PTCA_REDUCTION_SHARED):
// 4-warp CTAs, one per update site, orders up to 128; and, for large
// clusters, NW_LARGE-warp CTAs with the matrix in a global slot.
#include "cluster_shared.cuh"
#include "launch.h"

namespace ptca {

size_t shared_smem_bytes() { return sh_layout().total; }

bool shared_supported(int prec, int nA) { return prec == 1 && nA >= 2 && nA <= SH_NMAX; }

cudaError_t configure_shared_kernels(size_t smem_limit) {
    const size_t need = sh_layout().total;
    if (need > smem_limit) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_stage_shared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    const size_t need_l = shl_layout(32 * SHL_NW).total;
    if (e == cudaSuccess && need_l + 64 <= smem_limit)
        e = cudaFuncSetAttribute(k_stage_large_shared, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_l);
    return e;
}

bool large_shared_supported(int prec, int nA, size_t smem_limit) {
    return prec == 1 && nA > 2 && nA <= 32 * SHL_NW && shl_layout(nA).total + 64 <= smem_limit;
}

cudaError_t launch_stage_large_shared(const StageArgs& a, int grid, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    const int g = a.count < grid ? a.count : grid;
    k_stage_large_shared<<<g, 32 * SHL_NW, shl_layout(a.nA).total, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stage_shared(const StageArgs& a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    k_stage_shared<<<a.count, 32 * SH_NW, sh_layout().total, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ptca
