// spectrum.cu -- full-system spectrum of a configuration (Sec. VI): the
// one-body Hamiltonian of the whole lattice, built densely on the device by
// this library's kernel, and its eigenvalues from the CUDA toolkit's dense
// Hermitian eigensolver (FP64), where the paper uses ScaLAPACK on saved
// configurations.  Off the sweep's hot path.
#include <cusolverDn.h>

#include <string>

#include "../../include/ptca.h"
#include "context.h"
#include "kernels.cuh"
#include "launch.h"

namespace ptca {

// One thread per lattice site: its on-site 2x2 block and its bonds to the
// +x, +y, +z neighbours (both triangles), hopping added atomically so that an
// axis of extent 2 on a torus gets both of its bonds (-2t).  H is dense,
// column-major, n = 2N, zeroed by the caller.
__global__ void k_full_hamiltonian(Model m, const double* __restrict__ S, int N, double2* __restrict__ H) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t n = 2 * (int64_t)N;
    const int x = i % m.Lx, y = (i / m.Lx) % m.Ly, z = i / (m.Lx * m.Ly);
    const double sx = S[3 * i], sy = S[3 * i + 1], sz = S[3 * i + 2];
    const double dg = m.e0 + m.lam * sx, J = m.JH;
    const int64_t a = 2 * (int64_t)i, b = a + 1;
    H[a * n + a] = make_double2(dg - J * sz, 0.0);
    H[b * n + b] = make_double2(dg + J * sz, 0.0);
    H[a * n + b] = make_double2(-J * sx, -J * sy);  // column a, row b: -J (S_x + i S_y)
    H[b * n + a] = make_double2(-J * sx, J * sy);   // column b, row a: its conjugate
    const int L[3] = {m.Lx, m.Ly, m.Lz};
    const int c[3] = {x, y, z};
    for (int d = 0; d < 3; ++d) {
        if (L[d] == 1) continue;
        int cc[3] = {c[0], c[1], c[2]};
        cc[d] += 1;
        if (cc[d] == L[d]) {
            if (!m.lattice_periodic) continue;
            cc[d] = 0;
        }
        const int j = (cc[2] * m.Ly + cc[1]) * m.Lx + cc[0];
        for (int sg = 0; sg < 2; ++sg) {
            const int64_t p = 2 * (int64_t)i + sg, q = 2 * (int64_t)j + sg;
            atomicAdd(&H[p * n + q].x, -m.t);
            atomicAdd(&H[q * n + p].x, -m.t);
        }
    }
}

}  // namespace ptca

ptca_status ptca_internal_fail(ptca_status s, const char* msg);
ptca::Model ptca_context_model(const ptca_ctx* ctx);

extern "C" ptca_status ptca_full_spectrum(ptca_ctx* ctx, double* eig_out, void* stream) {
    if (!ctx || !eig_out) return ptca_internal_fail(PTCA_ERR_INVALID, "null argument");
    const int N = ctx->N;
    if (N > 16384) return ptca_internal_fail(PTCA_ERR_INVALID, "ptca_full_spectrum covers lattices of up to 16384 sites");
    const int n = 2 * N;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS)
        return ptca_internal_fail(PTCA_ERR_CUDA, "ptca_full_spectrum: cusolverDnCreate failed");
    double2* H = nullptr;
    double2* work = nullptr;
    int* info = nullptr;
    ptca_status status = PTCA_OK;
    std::string why;
    auto fail_cuda = [&](cudaError_t e, const char* where) {
        status = e == cudaErrorMemoryAllocation ? PTCA_ERR_OOM : PTCA_ERR_CUDA;
        why = std::string("ptca_full_spectrum: ") + where + ": " + cudaGetErrorString(e);
    };
    cudaError_t e = cusolverDnSetStream(h, st) == CUSOLVER_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaMalloc(&H, (size_t)n * (size_t)n * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&info, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(H, 0, (size_t)n * (size_t)n * sizeof(double2), st);
    if (e == cudaSuccess) {
        const ptca::Model m = ptca_context_model(ctx);
        ptca::k_full_hamiltonian<<<(N + 255) / 256, 256, 0, st>>>(m, ctx->d_S[0], N, H);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) fail_cuda(e, "building the matrix");
    int lwork = 0;
    if (status == PTCA_OK &&
        cusolverDnZheevd_bufferSize(h, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                    reinterpret_cast<cuDoubleComplex*>(H), n, eig_out, &lwork) !=
            CUSOLVER_STATUS_SUCCESS) {
        status = PTCA_ERR_CUDA;
        why = "ptca_full_spectrum: eigensolver workspace query failed";
    }
    if (status == PTCA_OK) {
        e = cudaMalloc(&work, (size_t)(lwork > 0 ? lwork : 1) * sizeof(double2));
        if (e != cudaSuccess) fail_cuda(e, "workspace");
    }
    if (status == PTCA_OK &&
        cusolverDnZheevd(h, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n, reinterpret_cast<cuDoubleComplex*>(H),
                         n, eig_out, reinterpret_cast<cuDoubleComplex*>(work), lwork, info) != CUSOLVER_STATUS_SUCCESS) {
        status = PTCA_ERR_CUDA;
        why = "ptca_full_spectrum: eigensolver call failed";
    }
    int hinfo = 0;
    if (status == PTCA_OK) {
        e = cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) fail_cuda(e, "synchronising");
        else if (hinfo != 0) {
            status = PTCA_ERR_NUMERIC;
            why = "ptca_full_spectrum: the eigensolver did not converge (info " + std::to_string(hinfo) + ")";
        }
    }
    cudaStreamSynchronize(st);
    cudaFree(H);
    cudaFree(work);
    cudaFree(info);
    cusolverDnDestroy(h);
    if (status != PTCA_OK) return ptca_internal_fail(status, why.c_str());
    return PTCA_OK;
}
