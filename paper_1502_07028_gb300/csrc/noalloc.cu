// noalloc.cu -- ptca_sweep_noalloc: the PTCA sweep for callers that cannot
// allocate device memory.
//
// Some hosts own every byte of device memory through their own pool (for
// example a framework's caching allocator that has reserved the device), or
// forbid the libraries they load from allocating; others run latency-critical
// loops in which cudaMalloc/cudaFree (cudaFree synchronises the whole device)
// are not acceptable.  ptca_init allocates the context's buffers, so those
// callers cannot use ptca_sweep.  This entry point runs the same stage and
// re-solve kernels on caller-owned spins and caller-owned outputs, and keeps
// all of its own working memory in one fixed-size array in device global
// memory that the library defines at file scope.  It allocates no device
// memory: no cudaMalloc, cudaFree or allocating library routine (host-side
// argument checks and the schedule use ordinary host memory only).
//
// Properties a caller must know:
//   * The array holds kNoAllocBytes (about 2.2 MB) on every GPU on which the
//     library is loaded, until the process exits, whether or not it is used.
//   * It bounds the problem: at most kNoAllocMaxSites lattice sites.
//   * All calls share it and it keeps the last call's contents.  Calls whose
//     work overlaps on the GPU (different streams, or different host threads
//     on the same device) race on it and produce garbage; serialise them.
//     Each call clears what must start at zero before its first kernel.
//   * The first call on each device resolves the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; make that
//     first call before any stream capture.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ptca.h"
#include "kernels.cuh"
#include "launch.h"

namespace {

constexpr int kNoAllocMaxSites = 16384;  // e.g. up to a 128 x 128 lattice
constexpr int kNoAllocMaxDevices = 64;
constexpr double kNoAllocMargin = 1e-2;  // re-solve band of PTCA_MIXED, as ptca_init's default

// Byte layout of the scratch array (offsets are multiples of 256).
constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffSalt = 0;                                                          // double[3N] second spin buffer
constexpr size_t kOffF = al256(kOffSalt + 3 * sizeof(double) * kNoAllocMaxSites);       // double[2N] F per old/new matrix
constexpr size_t kOffFill = al256(kOffF + 2 * sizeof(double) * kNoAllocMaxSites);       // double[2N]
constexpr size_t kOffTicket = al256(kOffFill + 2 * sizeof(double) * kNoAllocMaxSites);  // int32[N]
constexpr size_t kOffRecSite = al256(kOffTicket + sizeof(int32_t) * kNoAllocMaxSites);  // int32[N]
constexpr size_t kOffRecFold = al256(kOffRecSite + sizeof(int32_t) * kNoAllocMaxSites); // double[N]
constexpr size_t kOffRecFnew = al256(kOffRecFold + sizeof(double) * kNoAllocMaxSites);  // double[N]
constexpr size_t kOffRecLnu = al256(kOffRecFnew + sizeof(double) * kNoAllocMaxSites);   // double[N]
constexpr size_t kOffRecFacc = al256(kOffRecLnu + sizeof(double) * kNoAllocMaxSites);   // double[N]
constexpr size_t kOffRecFill = al256(kOffRecFacc + sizeof(double) * kNoAllocMaxSites);  // double[N]
constexpr size_t kOffRecN = al256(kOffRecFill + sizeof(double) * kNoAllocMaxSites);     // int32[N]
constexpr size_t kOffRecAcc = al256(kOffRecN + sizeof(int32_t) * kNoAllocMaxSites);     // uint8[N]
constexpr size_t kOffSites = al256(kOffRecAcc + kNoAllocMaxSites);                      // int32[N] schedule
constexpr size_t kOffFlags = al256(kOffSites + sizeof(int32_t) * kNoAllocMaxSites);     // int32[N] deferred visits
constexpr size_t kOffFlagCount = al256(kOffFlags + sizeof(int32_t) * kNoAllocMaxSites); // u32[1]
constexpr size_t kOffCounters = al256(kOffFlagCount + sizeof(unsigned int));            // u64[4]
constexpr size_t kOffErr = al256(kOffCounters + 4 * sizeof(unsigned long long));        // int32[2]
constexpr size_t kNoAllocBytes = al256(kOffErr + 2 * sizeof(int32_t));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
unsigned char* g_addr[kNoAllocMaxDevices] = {};

}  // namespace

// Defined in api.cu: records the message that ptca_last_error() returns.
ptca_status ptca_internal_fail(ptca_status s, const char* msg);

extern "C" ptca_status ptca_sweep_noalloc(const ptca_lattice* lattice, const ptca_params* params, double* spins,
                                          int64_t sweep_index, double* F_out, uint8_t* accepted_out,
                                          int32_t* status_out, void* stream) {
    if (!lattice || !params || !spins)
        return ptca_internal_fail(PTCA_ERR_INVALID, "ptca_sweep_noalloc: null argument");
    if (sweep_index < 0) return ptca_internal_fail(PTCA_ERR_INVALID, "ptca_sweep_noalloc: sweep_index < 0");
    // Validate the problem and build its schedule on the host (no device memory).
    const int64_t N64 = (int64_t)lattice->Lx * (int64_t)lattice->Ly * (int64_t)(lattice->Lz > 1 ? lattice->Lz : 1);
    if (lattice->Lx < 1 || lattice->Ly < 1 || lattice->Lz < 0 || N64 > kNoAllocMaxSites)
        return ptca_internal_fail(PTCA_ERR_INVALID,
                                  ("ptca_sweep_noalloc: lattice has " + std::to_string(N64) +
                                   " sites; this entry point supports at most " + std::to_string(kNoAllocMaxSites))
                                      .c_str());
    const int N = (int)N64;
    std::vector<int32_t> stage_start(N + 1), sched(N);
    int32_t n_stages = 0;
    ptca_status st = ptca_schedule(lattice, params, stage_start.data(), sched.data(), &n_stages);
    if (st != PTCA_OK) return st;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
        return ptca_internal_fail(PTCA_ERR_CUDA, "ptca_sweep_noalloc: no usable current device");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return ptca_internal_fail(PTCA_ERR_CUDA, (std::string("ptca_sweep_noalloc: cudaGetSymbolAddress: ") +
                                                          cudaGetErrorString(e)).c_str());
            g_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_addr[dev];
    }
    int optin = 0, sms = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // Problem description (same resolution rules as ptca_init).
    const int Lc = params->L_c;
    int o = params->update_offset;
    if (o < 0) o = params->schedule == PTCA_SCHEDULE_TILED ? Lc / 2 : 0;
    ptca::Model m;
    const int Lz = lattice->Lz == 0 ? 1 : lattice->Lz;
    m.Lx = lattice->Lx; m.Ly = lattice->Ly; m.Lz = Lz; m.lattice_periodic = lattice->periodic ? 1 : 0;
    m.Lc = Lc; m.ox = o; m.oy = lattice->Ly == 1 ? 0 : o; m.oz = Lz == 1 ? 0 : o;
    m.cluster_periodic = params->cluster_periodic < 0 ? m.lattice_periodic : (params->cluster_periodic ? 1 : 0);
    m.proposal = params->proposal;
    m.t = params->t; m.mu = params->mu; m.T = params->T;
    m.cone_cos = std::cos(params->cone_deg * ptca::kPi / 180.0);
    ptca::set_model_terms(m, params->model, params->J_H, params->U, params->lam, params->K, params->mu,
                          params->m_step);
    m.seed = params->seed;
    const int prec = params->precision == PTCA_MIXED ? 1 : 0;
    const int nA = 2 * Lc * (lattice->Ly == 1 ? 1 : Lc) * (Lz == 1 ? 1 : Lc);
    const size_t smem = ptca::cluster_smem_bytes(prec, nA);
    if (smem == 0 || smem + 256 > (size_t)optin)
        return ptca_internal_fail(PTCA_ERR_INVALID, "ptca_sweep_noalloc: cluster matrix too large for this precision");
    e = ptca::configure_cluster_kernels((size_t)optin);
    if (e != cudaSuccess) return ptca_internal_fail(PTCA_ERR_CUDA, cudaGetErrorString(e));
    // PTCA_MIXED re-solves the decisions within kNoAllocMargin of the
    // threshold, as ptca_sweep does; that re-solve must keep its matrix in
    // shared memory here (the global matrix slots it uses otherwise are
    // context memory).
    if (prec == 1 && !ptca::resolve_smem_fits(nA))
        return ptca_internal_fail(PTCA_ERR_UNSUPPORTED,
                                  ("ptca_sweep_noalloc: in PTCA_MIXED the re-solve of order-" + std::to_string(nA) +
                                   " cluster matrices does not fit in shared memory; use ptca_sweep")
                                      .c_str());

    cudaStream_t stm = static_cast<cudaStream_t>(stream);
    double* S_alt = reinterpret_cast<double*>(base + kOffSalt);
    int32_t* sites = reinterpret_cast<int32_t*>(base + kOffSites);
    int32_t* ticket = reinterpret_cast<int32_t*>(base + kOffTicket);
    unsigned int* flag_count = reinterpret_cast<unsigned int*>(base + kOffFlagCount);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(base + kOffCounters);
    int32_t* err = reinterpret_cast<int32_t*>(base + kOffErr);
    // The schedule the host built and checked (pageable source: the copy is
    // staged before the call returns), cleared counters, and both spin
    // buffers equal.
    e = cudaMemcpyAsync(sites, sched.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, stm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(int32_t) * N, stm);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag_count, 0, sizeof(unsigned int), stm);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), stm);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), stm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S_alt, spins, 3 * sizeof(double) * N, cudaMemcpyDeviceToDevice, stm);
    if (e != cudaSuccess) return ptca_internal_fail(PTCA_ERR_CUDA, cudaGetErrorString(e));

    double* buf[2] = {spins, S_alt};
    ptca::StageArgs a;
    std::memset(&a, 0, sizeof a);
    a.m = m;
    a.nA = nA;
    a.sweep = (uint64_t)sweep_index;
    a.Fbuf = reinterpret_cast<double*>(base + kOffF);
    a.fillbuf = reinterpret_cast<double*>(base + kOffFill);
    a.ticket = ticket;
    a.rec_site = reinterpret_cast<int32_t*>(base + kOffRecSite);
    a.rec_Fold = reinterpret_cast<double*>(base + kOffRecFold);
    a.rec_Fnew = reinterpret_cast<double*>(base + kOffRecFnew);
    a.rec_lnu = reinterpret_cast<double*>(base + kOffRecLnu);
    a.rec_acc = reinterpret_cast<uint8_t*>(base + kOffRecAcc);
    a.rec_Facc = reinterpret_cast<double*>(base + kOffRecFacc);
    a.rec_fill = reinterpret_cast<double*>(base + kOffRecFill);
    a.rec_n = reinterpret_cast<int32_t*>(base + kOffRecN);
    a.counters = counters;
    a.err = err;
    a.margin = prec == 1 ? kNoAllocMargin : 0.0;
    a.flag_list = reinterpret_cast<int32_t*>(base + kOffFlags);
    a.flag_count = flag_count;
    for (int s = 0; s < n_stages; ++s) {
        a.S_in = buf[s & 1];
        a.S_out = buf[(s + 1) & 1];
        a.sites = sites + stage_start[s];
        a.count = stage_start[s + 1] - stage_start[s];
        a.rec_base = stage_start[s];
        a.prev_sites = s > 0 ? sites + stage_start[s - 1] : nullptr;
        a.prev_count = s > 0 ? stage_start[s] - stage_start[s - 1] : 0;
        e = ptca::launch_stage(prec, 8, a, stm);
        if (e == cudaSuccess && prec == 1) {
            // Deferred decisions of this stage: re-solved before the next
            // stage reads the spins, then the list is emptied.
            e = ptca::launch_resolve(a, sms, stm);
            if (e == cudaSuccess) e = cudaMemsetAsync(flag_count, 0, sizeof(unsigned int), stm);
        }
        if (e != cudaSuccess) return ptca_internal_fail(PTCA_ERR_CUDA, cudaGetErrorString(e));
    }
    if (n_stages > 0) {
        // Bring the other buffer up to date; the final configuration is then
        // in both, so the caller's spins hold it whatever the stage parity.
        const int last = n_stages - 1;
        e = ptca::launch_copy_sites(buf[n_stages & 1], buf[(n_stages + 1) & 1], sites + stage_start[last],
                                    stage_start[last + 1] - stage_start[last], stm);
        if (e != cudaSuccess) return ptca_internal_fail(PTCA_ERR_CUDA, cudaGetErrorString(e));
    }
    if (F_out) {
        e = cudaMemcpyAsync(F_out, a.rec_Fold, sizeof(double) * N, cudaMemcpyDeviceToDevice, stm);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(F_out + N, a.rec_Fnew, sizeof(double) * N, cudaMemcpyDeviceToDevice, stm);
        if (e != cudaSuccess) return ptca_internal_fail(PTCA_ERR_CUDA, cudaGetErrorString(e));
    }
    if (accepted_out) {
        e = cudaMemcpyAsync(accepted_out, a.rec_acc, N, cudaMemcpyDeviceToDevice, stm);
        if (e != cudaSuccess) return ptca_internal_fail(PTCA_ERR_CUDA, cudaGetErrorString(e));
    }
    if (status_out) {
        e = ptca::launch_status_word(err, status_out, stm);
        if (e != cudaSuccess) return ptca_internal_fail(PTCA_ERR_CUDA, cudaGetErrorString(e));
    }
    return PTCA_OK;
}
