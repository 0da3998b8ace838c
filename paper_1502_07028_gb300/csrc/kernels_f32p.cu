// FP32 sweep kernels of 8-warp CTAs with the blocked (panel) Householder
// reduction: panels of 2, 4 or 8 reflectors, orders up to 128; per-stage and
// overlapped pipelines.
#include "kernels.cuh"
#include "launch.h"

namespace ptca {

namespace {
size_t panel_smem(int B) { return smem_layout(128, 128, sizeof(float2), PN_NW).total + panel_extra_bytes(B, 128); }
template <int B> cudaError_t panel_configure(size_t smem_limit) {
    const size_t need = panel_smem(B);
    if (need > smem_limit) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_stage<float, 4, PN_NW, false, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)need);
}
}  // namespace

bool panel_supported(int prec, int nA, int B) {
    return prec == 1 && nA >= 1 && nA <= 128 && (B == 2 || B == 4 || B == 8);
}

size_t panel_smem_bytes(int B) { return panel_smem(B); }

cudaError_t configure_panel_kernels(size_t smem_limit) {
    cudaError_t e = panel_configure<2>(smem_limit);
    if (e == cudaSuccess) e = panel_configure<4>(smem_limit);
    if (e == cudaSuccess) e = panel_configure<8>(smem_limit);
    return e;
}

cudaError_t launch_stage_panel(int B, const StageArgs& a, cudaStream_t st) {
    if (a.count <= 0) return cudaSuccess;
    if (a.nA > 128) return cudaErrorInvalidValue;
    const dim3 grid(2 * a.count), block(32 * PN_NW);
    switch (B) {
        case 2: k_stage<float, 4, PN_NW, false, 2><<<grid, block, panel_smem(2), st>>>(a); break;
        case 4: k_stage<float, 4, PN_NW, false, 4><<<grid, block, panel_smem(4), st>>>(a); break;
        case 8: k_stage<float, 4, PN_NW, false, 8><<<grid, block, panel_smem(8), st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ptca
