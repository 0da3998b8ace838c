// context.h -- the library context behind the opaque ptca_ctx handle.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ptca.h"

// Resolved problem (defaults filled in).
struct Problem {
    int Lx, Ly, Lz, periodic, Lc, ox, oy, oz, cluster_periodic, schedule, stride, precision, proposal, model;
    double t, JH, mu, T, cone_deg, U, m_step, lam, K;
    uint64_t seed;
    int N() const { return Lx * Ly * Lz; }
    int nsite_max() const { return Lc * (Ly == 1 ? 1 : Lc) * (Lz == 1 ? 1 : Lc); }
    int nmax() const { return 2 * nsite_max(); }
};

namespace ptca {

// Surrogate network state (delayed-acceptance screening).
struct SurrogateState {
    bool ready = false;     // parameters initialised
    bool enabled = false;   // screen proposals in ptca_sweep
    float scale = 1.f;      // dF scale the network is trained in
    int adam_step = 0;
    float* theta = nullptr; // FP32 parameters
    float* m1 = nullptr;    // AdamW moments
    float* m2 = nullptr;
    float* grad = nullptr;
    // stage screening buffers (two sets by stage parity, 2 * max_stage rows each)
    float *X = nullptr, *Z1 = nullptr, *A1 = nullptr, *Z2 = nullptr, *A2 = nullptr, *Z3 = nullptr, *A3 = nullptr,
          *Z4 = nullptr;
    float* dFt = nullptr;
    int32_t* work = nullptr;
    unsigned int* nwork = nullptr;
    // training buffers (rows = 2 * batch)
    int batch = 0;
    float *tX = nullptr, *tZ1 = nullptr, *tA1 = nullptr, *tZ2 = nullptr, *tA2 = nullptr, *tZ3 = nullptr,
          *tA3 = nullptr, *tZ4 = nullptr, *tdZ4 = nullptr, *tdA = nullptr, *tdZ = nullptr, *tloss = nullptr;
    int64_t* tidx = nullptr;
};

}  // namespace ptca

struct ptca_ctx {
    Problem p;
    int device = 0;
    int prec = 0;  // 0 FP64, 1 FP32 reduction
    int N = 0, nstages = 0, max_stage = 0, nA = 0;
    size_t smem = 0;
    std::vector<int32_t> h_start, h_sites;
    int32_t* d_sites = nullptr;
    // Spin buffers: [0] and [1] rotate between stages and hold the same
    // configuration between calls; [2] joins the rotation in the overlapped
    // pipeline (allocated when that pipeline is first selected).
    double* d_S[4] = {nullptr, nullptr, nullptr, nullptr};
    // Per-visit scratch of a stage, in two halves (stage parity) so that a
    // stage's re-solve can run while the next stage is under way; the
    // other pipelines use half 0.
    double* d_F = nullptr;     // [2][2 max_stage]
    double* d_fill = nullptr;  // [2][2 max_stage]
    int32_t* d_ticket = nullptr;  // [2][max_stage]
    int32_t* d_rec_site = nullptr;
    double* d_rec_Fold = nullptr;
    double* d_rec_Fnew = nullptr;
    double* d_rec_lnu = nullptr;
    uint8_t* d_rec_acc = nullptr;
    double* d_rec_Facc = nullptr;
    double* d_rec_fill = nullptr;
    int32_t* d_rec_n = nullptr;
    unsigned long long* d_counters = nullptr;
    int32_t* d_err = nullptr;
    double* d_obs = nullptr;
    int64_t sweeps = 0;
    int64_t total_accepted = 0;
    // persistent pipeline
    int32_t* d_stage_start = nullptr;
    int32_t* d_perm = nullptr;
    unsigned int* d_queue = nullptr;
    unsigned int* d_bar = nullptr;
    unsigned long long* d_sweep_ctr = nullptr;
    int pipeline = PTCA_PIPELINE_GRAPH;
    int nw = 8;              // warps per CTA of the sweep kernels (8, or 4 for PTCA_MIXED, n <= 128)
    int reduction = 0;       // 1: the register-tiled FP32 reduction (4-warp stage kernels)
    int panel = 0;           // > 1: the blocked FP32 reduction in panels of this width (8-warp stage kernels)
    int ctas_per_sm = 0;     // persistent CTAs per SM (0: as many as fit)
    int sms = 0;
    unsigned long long timeout_ns = 30ull * 1000000000ull;
    int grid = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_sweeps = -1;
    cudaStream_t graph_stream = nullptr;
    bool graph_failed = false;
    // PTCA_MIXED decision guard
    double margin = 0.0;
    bool margin_set = false;              // chosen by the caller (ptca_set_resolve_margin)
    int32_t* d_flag_list = nullptr;       // [2][max_stage]
    unsigned int* d_flag_count = nullptr; // [2]
    double2* d_gA = nullptr;
    int64_t gA_stride = 0;
    int resolve_grid = 0;
    // large traveling clusters (orders above the shared-memory kernels'):
    // one global matrix slot per resident 16-warp CTA
    bool large = false;
    int large_grid = 0;
    // FP32 large clusters may instead run the cluster kernel (matrix in the
    // distributed shared memory of cl_size CTAs; 0 when it does not fit),
    // selected by warps_per_cta = 8 (16: the global-slot kernel)
    int cl_size = 0;
    int cl_grid = 0;
    void* d_gL = nullptr;
    int64_t gL_stride = 0;
    // precision checker (PTCA_MIXED): FP32-vs-FP64 spectra of every visit
    bool checker = false;
    int check_chunk = 0;
    double* d_chk_eig = nullptr;              // [2 precisions][check_chunk][2][nA]
    double* d_chk_F = nullptr;                // [2 precisions][check_chunk][2]
    unsigned long long* d_chk_out = nullptr;  // [nstages][kCheckCols], bits of non-negative doubles
    // overlapped pipeline: stage order with the visits independent of the
    // previous stage first (h_indep[s] of them), a high-priority stream for
    // the re-solves and the dependent visits, and the events ordering it
    // against the caller's stream
    int32_t* d_split = nullptr;
    std::vector<int32_t> h_indep;
    // A ptca_sweep call in the overlapped pipeline may leave its last
    // stage's re-solve to the next call (ov_pending): the rotation then
    // continues at global stage ov_g, whose predecessor's re-solve is still
    // to be enqueued on `side`; ptca_internal_settle completes it.
    bool ov_pending = false;
    int64_t ov_g = 0;
    cudaStream_t side = nullptr;
    // second stream of the independent visits (look-ahead: stage g+1's
    // independent visits beside stage g's), and per-parity events: the
    // independent visits of stage g done (ev_ind), its re-solve done (ev_res)
    cudaStream_t side2 = nullptr;
    cudaEvent_t ev_ind[2] = {nullptr, nullptr}, ev_res[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // optional per-kernel timing of the per-stage pipelines: event pairs
    // around each stage launch (kind 0), re-solve launch (kind 1) and
    // dependent-visit launch of the overlapped pipeline (kind 2), with the
    // matrices each launch solves
    bool timing = false;
    std::vector<cudaEvent_t> tev;
    std::vector<int> tkind;
    std::vector<int64_t> titems;
    // partial stages (ptca_stage_run) and site gathers/scatters
    // (ptca_get_sites / ptca_set_sites): the stage of every site, and device
    // copies of the caller's site list and of the spins moved (made on first use)
    std::vector<int32_t> h_stage_of;
    int32_t* d_sub = nullptr;         // [N]
    double* d_sub_spins = nullptr;    // [3 N]
    // surrogate network for delayed-acceptance screening
    ptca::SurrogateState sg;
};

void ptca_free_surrogate(ptca_ctx* c);
// Completes a re-solve that an overlapped sweep left pending (see ov_pending)
// and puts the configuration back into spin buffers 0 and 1: stream-ordered
// on `st`, or, when have_stream is false, before returning.
extern "C" cudaError_t ptca_internal_settle(ptca_ctx* ctx, cudaStream_t st, bool have_stream);
