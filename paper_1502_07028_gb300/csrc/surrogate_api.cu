// surrogate_api.cu -- C ABI of the surrogate network: parameters, collection
// of (patch, dF) samples from exact sweeps, training with the library's own
// forward/backward/AdamW kernels, prediction, and delayed-acceptance
// screening inside ptca_sweep.
#include <cmath>
#include <cstring>
#include <string>

#include "context.h"
#include "kernels.cuh"
#include "launch.h"
#include "surrogate_launch.h"

using ptca::SurrogateState;

ptca_status ptca_internal_fail(ptca_status s, const char* msg);

namespace {

ptca_status cfail(cudaError_t e, const char* where) {
    return ptca_internal_fail(e == cudaErrorMemoryAllocation ? PTCA_ERR_OOM : PTCA_ERR_CUDA,
                              (std::string(where) + ": " + cudaGetErrorString(e)).c_str());
}
#define SG_CUDA(call)                                        \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return cfail(_e, #call);      \
    } while (0)

template <typename T> cudaError_t dal(T** p, size_t n) { return cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T)); }

void free_train(SurrogateState& g) {
    float* fs[] = {g.tX, g.tZ1, g.tA1, g.tZ2, g.tA2, g.tZ3, g.tA3, g.tZ4, g.tdZ4, g.tdA, g.tdZ, g.tloss};
    for (float* f : fs)
        if (f) cudaFree(f);
    if (g.tidx) cudaFree(g.tidx);
    g.tX = g.tZ1 = g.tA1 = g.tZ2 = g.tA2 = g.tZ3 = g.tA3 = g.tZ4 = g.tdZ4 = g.tdA = g.tdZ = g.tloss = nullptr;
    g.tidx = nullptr;
    g.batch = 0;
}

cudaError_t ensure_train(SurrogateState& g, int B) {
    if (g.batch >= B) return cudaSuccess;
    free_train(g);
    const size_t R = 2 * (size_t)B;
    cudaError_t e = dal(&g.tX, R * ptca::SG_IN_PAD);
    float** hs[] = {&g.tZ1, &g.tA1, &g.tZ2, &g.tA2, &g.tZ3, &g.tA3, &g.tdA, &g.tdZ};
    for (float** h : hs)
        if (e == cudaSuccess) e = dal(h, R * ptca::SG_H);
    if (e == cudaSuccess) e = dal(&g.tZ4, R * ptca::SG_OUT_PAD);
    if (e == cudaSuccess) e = dal(&g.tdZ4, R * ptca::SG_OUT_PAD);
    if (e == cudaSuccess) e = dal(&g.tloss, 1);
    if (e == cudaSuccess) e = dal(&g.tidx, (size_t)B);
    if (e == cudaSuccess) g.batch = B;
    return e;
}

// h for R rows of X (R x SG_IN_PAD): Z1 A1 Z2 A2 Z3 A3 Z4 (row-major).
cudaError_t mlp_forward(const float* th, int R, const float* X, float* Z1, float* A1, float* Z2, float* A2, float* Z3,
                        float* A3, float* Z4, cudaStream_t st) {
    using namespace ptca;
    const long long H = SG_H;
    cudaError_t e = sg_gemm(R, SG_H, SG_IN_PAD, X, SG_IN_PAD, 1, th + SG_OFF_W1, 1, SG_IN_PAD, th + SG_OFF_B1, Z1, SG_H, st);
    if (e == cudaSuccess) e = sg_elementwise(0, Z1, nullptr, A1, R * H, st);
    if (e == cudaSuccess) e = sg_gemm(R, SG_H, SG_H, A1, SG_H, 1, th + SG_OFF_W2, 1, SG_H, th + SG_OFF_B2, Z2, SG_H, st);
    if (e == cudaSuccess) e = sg_elementwise(0, Z2, nullptr, A2, R * H, st);
    if (e == cudaSuccess) e = sg_gemm(R, SG_H, SG_H, A2, SG_H, 1, th + SG_OFF_W3, 1, SG_H, th + SG_OFF_B3, Z3, SG_H, st);
    if (e == cudaSuccess) e = sg_elementwise(0, Z3, nullptr, A3, R * H, st);
    if (e == cudaSuccess)
        e = sg_gemm(R, SG_OUT_PAD, SG_H, A3, SG_H, 1, th + SG_OFF_W4, 1, SG_H, th + SG_OFF_B4, Z4, SG_OUT_PAD, st);
    return e;
}

// Gradient of the batch loss (rows 0..B-1 paired with B..2B-1) into grad.
cudaError_t mlp_backward(const float* th, int R, SurrogateState& g, float* grad, cudaStream_t st) {
    using namespace ptca;
    const long long H = SG_H;
    // layer 4
    cudaError_t e = sg_gemm(SG_OUT_PAD, SG_H, R, g.tdZ4, 1, SG_OUT_PAD, g.tA3, SG_H, 1, nullptr, grad + SG_OFF_W4, SG_H, st);
    if (e == cudaSuccess) e = sg_colsum(g.tdZ4, R, SG_OUT_PAD, grad + SG_OFF_B4, st);
    if (e == cudaSuccess) e = sg_gemm(R, SG_H, SG_OUT_PAD, g.tdZ4, SG_OUT_PAD, 1, th + SG_OFF_W4, SG_H, 1, nullptr, g.tdA, SG_H, st);
    if (e == cudaSuccess) e = sg_elementwise(1, g.tdA, g.tZ3, g.tdZ, R * H, st);
    // layer 3
    if (e == cudaSuccess) e = sg_gemm(SG_H, SG_H, R, g.tdZ, 1, SG_H, g.tA2, SG_H, 1, nullptr, grad + SG_OFF_W3, SG_H, st);
    if (e == cudaSuccess) e = sg_colsum(g.tdZ, R, SG_H, grad + SG_OFF_B3, st);
    if (e == cudaSuccess) e = sg_gemm(R, SG_H, SG_H, g.tdZ, SG_H, 1, th + SG_OFF_W3, SG_H, 1, nullptr, g.tdA, SG_H, st);
    if (e == cudaSuccess) e = sg_elementwise(1, g.tdA, g.tZ2, g.tdZ, R * H, st);
    // layer 2
    if (e == cudaSuccess) e = sg_gemm(SG_H, SG_H, R, g.tdZ, 1, SG_H, g.tA1, SG_H, 1, nullptr, grad + SG_OFF_W2, SG_H, st);
    if (e == cudaSuccess) e = sg_colsum(g.tdZ, R, SG_H, grad + SG_OFF_B2, st);
    if (e == cudaSuccess) e = sg_gemm(R, SG_H, SG_H, g.tdZ, SG_H, 1, th + SG_OFF_W2, SG_H, 1, nullptr, g.tdA, SG_H, st);
    if (e == cudaSuccess) e = sg_elementwise(1, g.tdA, g.tZ1, g.tdZ, R * H, st);
    // layer 1
    if (e == cudaSuccess)
        e = sg_gemm(SG_H, SG_IN_PAD, R, g.tdZ, 1, SG_H, g.tX, SG_IN_PAD, 1, nullptr, grad + SG_OFF_W1, SG_IN_PAD, st);
    if (e == cudaSuccess) e = sg_colsum(g.tdZ, R, SG_H, grad + SG_OFF_B1, st);
    return e;
}

cudaError_t loss_grad_step(SurrogateState& g, const float* feat, const int32_t* center, const float* dF, int B,
                           float* grad, cudaStream_t st) {
    const int R = 2 * B;
    cudaError_t e = ptca::sg_pair_rows(feat, center, g.tidx, B, g.tX, st);
    if (e == cudaSuccess) e = mlp_forward(g.theta, R, g.tX, g.tZ1, g.tA1, g.tZ2, g.tA2, g.tZ3, g.tA3, g.tZ4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.tloss, 0, sizeof(float), st);
    if (e == cudaSuccess) e = ptca::sg_pair_loss(g.tZ4, dF, g.tidx, B, 1.f / g.scale, g.tdZ4, g.tloss, st);
    if (e == cudaSuccess) e = mlp_backward(g.theta, R, g, grad, st);
    return e;
}

}  // namespace

void ptca_free_surrogate(ptca_ctx* c) {
    SurrogateState& g = c->sg;
    free_train(g);
    float* fs[] = {g.theta, g.m1, g.m2, g.grad, g.X, g.Z1, g.A1, g.Z2, g.A2, g.Z3, g.A3, g.Z4, g.dFt};
    for (float* f : fs)
        if (f) cudaFree(f);
    if (g.work) cudaFree(g.work);
    if (g.nwork) cudaFree(g.nwork);
    g = SurrogateState();
}

extern "C" {

int32_t ptca_surrogate_param_count(void) { return ptca::SG_NPARAMS; }

ptca_status ptca_surrogate_init(ptca_ctx* ctx, uint64_t seed, void* stream) {
    if (!ctx) return ptca_internal_fail(PTCA_ERR_INVALID, "null context");
    if (ctx->p.model != PTCA_MODEL_DOUBLE_EXCHANGE || ctx->p.Lz > 1 || ctx->large)
        return ptca_internal_fail(PTCA_ERR_UNSUPPORTED, "the surrogate screen is built for the double-exchange model on square lattices");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SurrogateState& g = ctx->sg;
    if (!g.theta) {
        // screening rows: two sets (stage parity: the overlapped pipeline
        // screens a stage's independent visits while the previous stage's
        // are still being solved), each of 2 * max_stage rows
        const size_t P = ptca::SG_NPARAMS, R = 4 * (size_t)ctx->max_stage;
        cudaError_t e = dal(&g.theta, P);
        if (e == cudaSuccess) e = dal(&g.m1, P);
        if (e == cudaSuccess) e = dal(&g.m2, P);
        if (e == cudaSuccess) e = dal(&g.grad, P);
        if (e == cudaSuccess) e = dal(&g.X, R * ptca::SG_IN_PAD);
        float** hs[] = {&g.Z1, &g.A1, &g.Z2, &g.A2, &g.Z3, &g.A3};
        for (float** h : hs)
            if (e == cudaSuccess) e = dal(h, R * ptca::SG_H);
        if (e == cudaSuccess) e = dal(&g.Z4, R * ptca::SG_OUT_PAD);
        // dF~ per stage index in two halves (stage parity), and the work list
        // of each part of a stage (all visits, or the overlapped pipeline's
        // independent and dependent visits), per stage parity
        if (e == cudaSuccess) e = dal(&g.dFt, 2 * (size_t)ctx->max_stage);
        if (e == cudaSuccess) e = dal(&g.work, 4 * (size_t)ctx->max_stage);
        if (e == cudaSuccess) e = dal(&g.nwork, 4);
        if (e != cudaSuccess) {
            ptca_free_surrogate(ctx);
            return cfail(e, "ptca_surrogate_init");
        }
    }
    SG_CUDA(ptca::sg_init_params(g.theta, seed, st));
    SG_CUDA(cudaMemsetAsync(g.m1, 0, sizeof(float) * ptca::SG_NPARAMS, st));
    SG_CUDA(cudaMemsetAsync(g.m2, 0, sizeof(float) * ptca::SG_NPARAMS, st));
    g.adam_step = 0;
    g.scale = 1.f;
    g.ready = true;
    return PTCA_OK;
}

ptca_status ptca_surrogate_get_params(ptca_ctx* ctx, float* theta, float* scale, void* stream) {
    if (!ctx || !ctx->sg.ready) return ptca_internal_fail(PTCA_ERR_INVALID, "surrogate not initialised");
    if (theta) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        SG_CUDA(cudaMemcpyAsync(theta, ctx->sg.theta, sizeof(float) * ptca::SG_NPARAMS, cudaMemcpyDefault, st));
        SG_CUDA(cudaStreamSynchronize(st));
    }
    if (scale) *scale = ctx->sg.scale;
    return PTCA_OK;
}

ptca_status ptca_surrogate_set_params(ptca_ctx* ctx, const float* theta, float scale, void* stream) {
    if (!ctx || !theta || !(scale > 0.f)) return ptca_internal_fail(PTCA_ERR_INVALID, "bad arguments");
    if (!ctx->sg.ready) {
        ptca_status s = ptca_surrogate_init(ctx, 0, stream);
        if (s != PTCA_OK) return s;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SG_CUDA(cudaMemcpyAsync(ctx->sg.theta, theta, sizeof(float) * ptca::SG_NPARAMS, cudaMemcpyDefault, st));
    SG_CUDA(cudaStreamSynchronize(st));
    ctx->sg.scale = scale;
    return PTCA_OK;
}

ptca_status ptca_surrogate_enable(ptca_ctx* ctx, int32_t on) {
    if (!ctx) return ptca_internal_fail(PTCA_ERR_INVALID, "null context");
    if (on && !ctx->sg.ready) return ptca_internal_fail(PTCA_ERR_INVALID, "surrogate not initialised");
    SG_CUDA(ptca_internal_settle(ctx, nullptr, false));
    ctx->sg.enabled = on != 0;
    return PTCA_OK;
}

ptca_status ptca_surrogate_grad(ptca_ctx* ctx, const float* feat, const int32_t* center, const float* dF, int32_t n,
                                float* grad_out, float* loss_out, void* stream) {
    if (!ctx || !ctx->sg.ready || !feat || !center || !dF || n < 1 || n > (1 << 20))
        return ptca_internal_fail(PTCA_ERR_INVALID, "bad arguments or surrogate not initialised");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SurrogateState& g = ctx->sg;
    SG_CUDA(ensure_train(g, n));
    SG_CUDA(ptca::sg_iota(g.tidx, n, st));
    SG_CUDA(loss_grad_step(g, feat, center, dF, n, g.grad, st));
    if (grad_out) SG_CUDA(cudaMemcpyAsync(grad_out, g.grad, sizeof(float) * ptca::SG_NPARAMS, cudaMemcpyDefault, st));
    if (loss_out) SG_CUDA(cudaMemcpyAsync(loss_out, g.tloss, sizeof(float), cudaMemcpyDefault, st));
    SG_CUDA(cudaStreamSynchronize(st));
    return PTCA_OK;
}

ptca_status ptca_surrogate_train(ptca_ctx* ctx, const float* feat, const int32_t* center, const float* dF, int64_t n,
                                 int32_t steps, int32_t batch, float lr, float weight_decay, uint64_t seed,
                                 float* loss_trace, void* stream) {
    if (!ctx || !ctx->sg.ready || !feat || !center || !dF || n < 1 || steps < 0 || batch < 1 || batch > (1 << 16) ||
        !(lr > 0.f))
        return ptca_internal_fail(PTCA_ERR_INVALID, "bad arguments or surrogate not initialised");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SurrogateState& g = ctx->sg;
    SG_CUDA(ensure_train(g, batch));
    if (g.adam_step == 0) {
        // Train in units of the standard deviation of dF.
        double* mom = nullptr;
        SG_CUDA(cudaMalloc(&mom, 2 * sizeof(double)));
        double h[2] = {0, 0};
        cudaError_t e = ptca::sg_moments(dF, n, mom, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, mom, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(mom);
        if (e != cudaSuccess) return cfail(e, "ptca_surrogate_train (moments)");
        const double mean = h[0] / n, var = h[1] / n - mean * mean;
        g.scale = (float)std::sqrt(var > 1e-12 ? var : 1e-12);
    }
    for (int s = 0; s < steps; ++s) {
        SG_CUDA(ptca::sg_batch_indices(seed, (uint64_t)(g.adam_step + 1), batch, n, g.tidx, st));
        SG_CUDA(loss_grad_step(g, feat, center, dF, batch, g.grad, st));
        if (loss_trace) SG_CUDA(cudaMemcpyAsync(loss_trace + s, g.tloss, sizeof(float), cudaMemcpyDefault, st));
        ++g.adam_step;
        SG_CUDA(ptca::sg_adamw(g.theta, g.m1, g.m2, g.grad, ptca::SG_NPARAMS, lr, 0.9f, 0.999f, 1e-8f, weight_decay,
                               g.adam_step, st));
    }
    return PTCA_OK;
}

ptca_status ptca_surrogate_predict(ptca_ctx* ctx, const float* feat, const int32_t* center, int32_t n, float* dF_out,
                                   void* stream) {
    if (!ctx || !ctx->sg.ready || !feat || !center || !dF_out || n < 1 || n > (1 << 20))
        return ptca_internal_fail(PTCA_ERR_INVALID, "bad arguments or surrogate not initialised");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SurrogateState& g = ctx->sg;
    SG_CUDA(ensure_train(g, n));
    SG_CUDA(ptca::sg_iota(g.tidx, n, st));
    SG_CUDA(ptca::sg_pair_rows(feat, center, g.tidx, n, g.tX, st));
    SG_CUDA(mlp_forward(g.theta, 2 * n, g.tX, g.tZ1, g.tA1, g.tZ2, g.tA2, g.tZ3, g.tA3, g.tZ4, st));
    // dF~ = scale (h[b] - h[n + b]): reuse the pair-loss kernel with zero targets.
    SG_CUDA(ptca::sg_screen_difference(g.tZ4, n, g.scale, dF_out, st));
    return PTCA_OK;
}

}  // extern "C"

// Screening of one part of a stage inside ptca_sweep (called by api.cu):
// features of the two pair rows of each listed visit, the network, stage-1
// decisions and the work list of visits that go on to the exact solve.  The
// part's visits are a.perm[0 .. a.count) (stage indices; all of the stage
// when a.perm is null).  part 0 takes the network rows from 0, part 1 those
// after row_base (the two parts of a stage can be screened concurrently);
// dF~ goes to the half `half` (stage parity).  On return a.perm is the work
// list, a.count_dev its length and a.sg_dFt the stage's dF~.
extern "C" cudaError_t ptca_screen_part(ptca_ctx* ctx, ptca::StageArgs& a, int part, int row_base, int half,
                                        cudaStream_t st) {
    SurrogateState& g = ctx->sg;
    const int R = 2 * a.count;
    const size_t rb = (size_t)half * 2 * ctx->max_stage + (size_t)row_base;  // rows of this parity's set
    float* dFt = g.dFt + (size_t)half * ctx->max_stage;
    int32_t* work = g.work + (size_t)(2 * half + part) * ctx->max_stage;
    unsigned int* nwork = g.nwork + 2 * half + part;
    cudaError_t e = cudaMemsetAsync(nwork, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = ptca::sg_screen_rows(a, g.X + rb * ptca::SG_IN_PAD, st);
    if (e == cudaSuccess)
        e = mlp_forward(g.theta, R, g.X + rb * ptca::SG_IN_PAD, g.Z1 + rb * ptca::SG_H, g.A1 + rb * ptca::SG_H,
                        g.Z2 + rb * ptca::SG_H, g.A2 + rb * ptca::SG_H, g.Z3 + rb * ptca::SG_H, g.A3 + rb * ptca::SG_H,
                        g.Z4 + rb * ptca::SG_OUT_PAD, st);
    if (e == cudaSuccess) e = ptca::sg_screen_decide(a, g.Z4 + rb * ptca::SG_OUT_PAD, g.scale, dFt, work, nwork, st);
    a.perm = work;
    a.count_dev = nwork;
    a.sg_dFt = dFt;
    return e;
}

extern "C" cudaError_t ptca_screen_stage(ptca_ctx* ctx, ptca::StageArgs& a, cudaStream_t st) {
    return ptca_screen_part(ctx, a, 0, 0, 0, st);
}
