// kernels_large.cu -- instantiation and launchers of the large-cluster
// kernels (orders above the shared-memory kernels' reach, up to 512): the
// FP32 and FP64 stage kernels and the double-float re-solve with the matrix
// in a global slot per CTA, and the FP32 stage kernel with the matrix in the
// distributed shared memory of a thread-block cluster (cluster_large.cuh).
#include "cluster_large.cuh"
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
    const size_t f = large_layout(sizeof(float2)), d = large_layout(sizeof(double2));
    cudaError_t e = allow_smem(k_stage_large<float>, f, smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_stage_large<double>, d, smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_resolve_large<>, large_layout(sizeof(dfl2)), smem_limit);
    // the FP32 persistent kernel also runs the double-float re-solve inline
    const size_t fp = f > large_layout(sizeof(dfl2)) ? f : large_layout(sizeof(dfl2));
    if (e == cudaSuccess) e = allow_smem(k_sweep_persistent_large<float>, fp, smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_sweep_persistent_large<double>, d, smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_check_large<float>, f, smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_check_large<double>, d, smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_eigvals_large<float>, f, smem_limit);
    if (e == cudaSuccess) e = allow_smem(k_eigvals_large<double>, d, smem_limit);
    return e;
}

namespace {
size_t persistent_large_smem(int prec) {
    const size_t f = large_layout(sizeof(float2)), r = large_layout(sizeof(dfl2));
    return prec == 1 ? (f > r ? f : r) : large_layout(sizeof(double2));
}
}  // namespace

// At most large_blocks_per_sm: the persistent grid then fits the stage
// kernel's slots (a.gL holds two sets of sms x large_blocks_per_sm).
int persistent_blocks_per_sm_large(int prec) {
    int b = 0;
    const size_t smem = persistent_large_smem(prec);
    cudaError_t e = prec == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_persistent_large<float>,
                                                                              32 * NW_LARGE, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_persistent_large<double>,
                                                                              32 * NW_LARGE, smem);
    if (e != cudaSuccess) return 0;
    const int s = large_blocks_per_sm(prec);
    return b < s ? b : s;
}

cudaError_t launch_persistent_large(int prec, const PersistArgs& p, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * NW_LARGE);
    cfg.dynamicSmemBytes = persistent_large_smem(prec);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return prec == 1 ? cudaLaunchKernelEx(&cfg, k_sweep_persistent_large<float>, p)
                     : cudaLaunchKernelEx(&cfg, k_sweep_persistent_large<double>, p);
}

cudaError_t launch_check_large(int prec, const StageArgs& a, int c0, int count, double* eig, int ld, double* F,
                               int grid, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (prec == 1)
        k_check_large<float><<<grid, 32 * NW_LARGE, large_layout(sizeof(float2)), st>>>(a, c0, count, eig, ld, F);
    else
        k_check_large<double><<<grid, 32 * NW_LARGE, large_layout(sizeof(double2)), st>>>(a, c0, count, eig, ld, F);
    return cudaGetLastError();
}

cudaError_t launch_eigvals_large(int prec, const void* H, const int64_t* offsets, const int32_t* n, int count, int nA,
                                 double* eig, const int64_t* eoff, void* slots, int64_t stride, int grid,
                                 cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (prec == 1)
        k_eigvals_large<float><<<grid, 32 * NW_LARGE, large_layout(sizeof(float2)), st>>>(
            static_cast<const float2*>(H), offsets, n, count, nA, eig, eoff, static_cast<float2*>(slots), stride);
    else
        k_eigvals_large<double><<<grid, 32 * NW_LARGE, large_layout(sizeof(double2)), st>>>(
            static_cast<const double2*>(H), offsets, n, count, nA, eig, eoff, static_cast<double2*>(slots), stride);
    return cudaGetLastError();
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

// ---------------------------------------------------------------------------
// Cluster kernel: the smallest cluster size (2, 4 or 8 CTAs) whose per-CTA
// share of the matrix fits in shared memory.
namespace {
template <int C> cudaError_t cl_allow(size_t smem_limit, int nA) {
    const size_t need = cl_layout<C>(nA).total;
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, k_stage_cluster<C>);
    if (e != cudaSuccess) return e;
    if (need + attr.sharedSizeBytes > smem_limit) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_stage_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
}
template <int C> cudaLaunchConfig_t cl_config(int nA, int grid, cudaStream_t st, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = cl_layout<C>(nA).total;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}
template <int C> int cl_grid(int nA) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cl_config<C>(nA, C, nullptr, attr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_stage_cluster<C>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return clusters * C;
}
}  // namespace

int cluster_stage_size(int nA, size_t smem_limit) {
    if (nA > 32 * NW_LARGE) return 0;
    if (cl_allow<2>(smem_limit, nA) == cudaSuccess) return 2;
    cudaGetLastError();
    if (cl_allow<4>(smem_limit, nA) == cudaSuccess) return 4;
    cudaGetLastError();
    if (cl_allow<8>(smem_limit, nA) == cudaSuccess) return 8;
    cudaGetLastError();
    return 0;
}

int cluster_stage_grid(int C, int nA) {
    return C == 2 ? cl_grid<2>(nA) : C == 4 ? cl_grid<4>(nA) : C == 8 ? cl_grid<8>(nA) : 0;
}

cudaError_t launch_stage_cluster(int C, const StageArgs& a, int grid, cudaStream_t st) {
    if (a.count <= 0 && a.prev_count + a.prev2_count <= 0) return cudaSuccess;
    cudaLaunchAttribute attr[1];
    switch (C) {
        case 2: { cudaLaunchConfig_t cfg = cl_config<2>(a.nA, grid, st, attr); return cudaLaunchKernelEx(&cfg, k_stage_cluster<2>, a); }
        case 4: { cudaLaunchConfig_t cfg = cl_config<4>(a.nA, grid, st, attr); return cudaLaunchKernelEx(&cfg, k_stage_cluster<4>, a); }
        case 8: { cudaLaunchConfig_t cfg = cl_config<8>(a.nA, grid, st, attr); return cudaLaunchKernelEx(&cfg, k_stage_cluster<8>, a); }
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_resolve_large(const StageArgs& a, int grid, cudaStream_t st) {
    k_resolve_large<><<<grid, 32 * NW_LARGE, large_layout(sizeof(dfl2)), st>>>(a);
    return cudaGetLastError();
}

}  // namespace ptca
