// launch.h -- host-side launchers of the PTCA kernels (called by the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ptca {

struct Model;
struct StageArgs;
struct PersistArgs;

// Dynamic shared memory of one cluster CTA for matrices up to order nA
// (0 when no kernel instantiation covers nA).  prec: 0 FP64, 1 FP32.
size_t cluster_smem_bytes(int prec, int nA);
// Largest order any instantiation covers for the precision.
int cluster_max_order(int prec);
// Opt every cluster kernel into the shared memory it may need.
cudaError_t configure_cluster_kernels(size_t smem_limit);

cudaError_t launch_init_spins(const Model& m, double* S, int N, cudaStream_t st);
// The model-dependent fields of m (coupling, on-site terms, classical energy,
// proposal step) for model 0 (double exchange), 1 (Hubbard mean field) or 2
// (Holstein).
void set_model_terms(Model& m, int model, double J_H, double U, double lam, double K, double mu, double m_step);
cudaError_t launch_copy_sites(const double* src, double* dst, const int32_t* sites, int count, cudaStream_t st);
// out[k] = S[sites[k]]; and S0[sites[k]] = S1[sites[k]] = in[k] (3 doubles each).
cudaError_t launch_gather_sites(const double* S, const int32_t* sites, int count, double* out, cudaStream_t st);
cudaError_t launch_scatter_sites(const int32_t* sites, int count, const double* in, double* S0, double* S1,
                                 cudaStream_t st);
cudaError_t launch_build(int prec, const Model& m, const double* S, const int32_t* sites, int count,
                         const double* new_spins, void* H, int64_t stride, int64_t* offsets, int32_t* nout,
                         cudaStream_t st);
cudaError_t launch_eigvals(int prec, int nA, const void* H, const int64_t* offsets, const int32_t* n, int count,
                           double* eig, const int64_t* eoff, cudaStream_t st);
cudaError_t launch_free_energy(const double* eig, const int64_t* eoff, const int32_t* n, int count, double mu,
                               double T, double* F, cudaStream_t st);
// Sweep kernels come in CTA widths nw = 8 warps (every precision and order)
// and nw = 4 warps (PTCA_MIXED, orders up to 128).
bool sweep_width_supported(int prec, int nw, int nA);
size_t sweep_smem_bytes(int prec, int nw, int nA);
cudaError_t launch_stage(int prec, int nw, const StageArgs& a, cudaStream_t st);
// The FP32 4-warp stage kernel with the register-tiled reduction (orders up
// to 128): whether it covers (prec, nA), its dynamic shared memory, its
// configuration (part of configure_cluster_kernels) and launch.
bool tiled_supported(int prec, int nA);
size_t tiled_smem_bytes();
cudaError_t configure_tiled_kernels(size_t smem_limit);
cudaError_t launch_stage_tiled(const StageArgs& a, cudaStream_t st);
// One reduction for both matrices of a visit (kernels_f32w4s.cu): FP32, 4-warp
// CTAs, one per update site, orders up to 128.
bool shared_supported(int prec, int nA);
size_t shared_smem_bytes();
cudaError_t configure_shared_kernels(size_t smem_limit);
cudaError_t launch_stage_shared(const StageArgs& a, cudaStream_t st);
// The same for large clusters: NW_LARGE-warp CTAs striding over the update
// sites, the matrix in the CTA's global slot a.gL (grid <= the slots).
bool large_shared_supported(int prec, int nA, size_t smem_limit);
cudaError_t launch_stage_large_shared(const StageArgs& a, int grid, cudaStream_t st);
// The FP32 8-warp stage kernels with the blocked (panel) reduction, panels of
// B = 2, 4 or 8 reflectors (orders up to 128).
bool panel_supported(int prec, int nA, int B);
size_t panel_smem_bytes(int B);
cudaError_t configure_panel_kernels(size_t smem_limit);
cudaError_t launch_stage_panel(int B, const StageArgs& a, cudaStream_t st);
// Persistent sweep kernel: grid CTAs (all co-resident; cooperative launch).
cudaError_t launch_persistent(int prec, int nw, const PersistArgs& p, int grid, cudaStream_t st);
// CTAs of the persistent kernel that fit on one SM for matrices up to nA.
int persistent_blocks_per_sm(int prec, int nw, int nA);
// Double-float (FP64-class) re-solve of the decisions a PTCA_MIXED stage deferred (grid CTAs).
cudaError_t launch_resolve(const StageArgs& a, int grid, cudaStream_t st);
// Whether launch_resolve keeps matrices up to order nA in shared memory (no
// global slot a.gA needed).  Valid after configure_cluster_kernels.
bool resolve_smem_fits(int nA);
// out[0] = the ptca_status a sweep's device error slots err[0..1] report.
cudaError_t launch_status_word(const int32_t* err, int32_t* out, cudaStream_t st);
// Precision checker: spectra of visits c0 .. c0+count-1 of a stage (prec 1:
// FP32 reduction as PTCA_MIXED sweeps; prec 0: FP64 on the global matrix
// slots a.gA, grid CTAs), and their FP32-vs-FP64 errors reduced into out[4].
cudaError_t launch_check(int prec, const StageArgs& a, int c0, int count, double* eig, int ld, double* F, int grid,
                         cudaStream_t st);
// Columns of a checker row (see k_check_compare).
constexpr int kCheckCols = 5;
cudaError_t launch_check_compare(const Model& m, const int32_t* sites, int count, const double* e32,
                                 const double* e64, int ld, const double* F32, const double* F64,
                                 unsigned long long* out, cudaStream_t st);
cudaError_t launch_barrier_selftest(int blocks, unsigned int* bar, int32_t* err, unsigned long long timeout_ns,
                                    cudaStream_t st);
cudaError_t launch_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st);
// Large traveling clusters (orders above cluster_max_order, up to
// large_max_order): one 16-warp CTA per matrix, the matrix in a global slot
// per CTA (a.gL, gL_stride elements of float2/double2; the re-solve uses
// a.gA), grid resident CTAs striding over the items.
int large_max_order();
size_t large_smem_bytes(int prec);
cudaError_t configure_large_kernels(size_t smem_limit);
int large_blocks_per_sm(int prec);
cudaError_t launch_stage_large(int prec, const StageArgs& a, int grid, cudaStream_t st);
cudaError_t launch_resolve_large(const StageArgs& a, int grid, cudaStream_t st);
// Persistent pipeline for large clusters (16-warp CTAs, matrix in the CTA's
// global slot a.gL, FP32 re-solves inline in a.gA): CTAs per SM that fit, and
// the cooperative launch (grid <= the slots of a.gL and a.gA).
int persistent_blocks_per_sm_large(int prec);
cudaError_t launch_persistent_large(int prec, const PersistArgs& p, int grid, cudaStream_t st);
// Precision checker for large clusters: prec 1 the FP32 reduction in the
// slots a.gL, prec 0 FP64 in the slots a.gA (grid <= the slots).
cudaError_t launch_check_large(int prec, const StageArgs& a, int c0, int count, double* eig, int ld, double* F,
                               int grid, cudaStream_t st);
// Batch eigenvalues of large orders (<= large_max_order): each CTA copies its
// matrix into slots + blockIdx.x * stride (grid <= the slots) and reduces it there.
cudaError_t launch_eigvals_large(int prec, const void* H, const int64_t* offsets, const int32_t* n, int count, int nA,
                                 double* eig, const int64_t* eoff, void* slots, int64_t stride, int grid,
                                 cudaStream_t st);
// FP32 large-cluster stage kernel with the matrix in the distributed shared
// memory of a thread-block cluster: the cluster size (2, 4 or 8 CTAs, 0 if
// none fits) for order nA (configures the kernel's shared memory), the grid
// (CTAs of the clusters that fit at once), and the launch.
int cluster_stage_size(int nA, size_t smem_limit);
int cluster_stage_grid(int C, int nA);
cudaError_t launch_stage_cluster(int C, const StageArgs& a, int grid, cudaStream_t st);
cudaError_t launch_observables(const double* S, int Lx, int Ly, const double* rec_Facc, const double* rec_fill,
                               const uint8_t* rec_acc, const int32_t* rec_n, int N, double* out, cudaStream_t st);

}  // namespace ptca
