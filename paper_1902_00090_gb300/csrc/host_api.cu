// fdfd_solve_host: the whole path from host permittivities to host fields in
// one call (operator set-up, source, optional predicted subspace, solve), with
// the host<->device copies inside the call.
#include <vector>

#include "common.cuh"
#include "engine.cuh"

namespace ddg {

static size_t round256(size_t v) { return (v + 255) / 256 * 256; }

// Device buffer for the call's inputs and outputs, held by the context.
static ddg_status reserve_io(Context* ctx, size_t bytes, cudaStream_t st) {
    if (bytes <= ctx->io_bytes) return DDG_OK;
    if (ctx->io) {
        DDG_CHECK_CUDA(cudaStreamSynchronize(st));
        cudaFree(ctx->io);
        ctx->io = nullptr;
        ctx->io_bytes = 0;
    }
    if (cudaMalloc(&ctx->io, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->io = nullptr;
        set_error("fdfd_solve_host: cudaMalloc of %zu bytes failed", bytes);
        return DDG_ENOMEM;
    }
    ctx->io_bytes = bytes;
    return DDG_OK;
}

struct OpList {
    std::vector<ddg_op*> ops;
    ~OpList() {
        for (ddg_op* A : ops) fdfd_operator_destroy(A);
    }
};

}  // namespace ddg

using namespace ddg;

extern "C" ddg_status fdfd_solve_host(ddg_context* cptr, ddg_predictor* P, int n, const ddg_grid* grids,
                                      const double* const* eps_host, int i_src, double sigma, double j_c,
                                      const double* const* U_fixed, int k_fixed, double tol, int restart,
                                      int maxit, ddg_precision prec, double* const* x_host, ddg_info* info,
                                      void* stream) {
    if (!cptr || n < 1 || !grids || !eps_host || !x_host) {
        set_error("fdfd_solve_host: NULL context / array or n=%d", n);
        return DDG_EINVAL;
    }
    const int kp = P ? predictor_num_outputs(P) : 0;
    if (U_fixed ? (k_fixed < 1 || k_fixed + kp > kMaxAug) : k_fixed != 0) {
        set_error("fdfd_solve_host: k_fixed=%d with %d predicted vectors (need 1 <= k_fixed, k_fixed + k <= %d, "
                  "or k_fixed = 0 without U_fixed)", k_fixed, kp, kMaxAug);
        return DDG_EINVAL;
    }
    for (int s = 0; s < n; ++s) {
        if (!eps_host[s] || !x_host[s]) { set_error("fdfd_solve_host: NULL eps or x at %d", s); return DDG_EINVAL; }
        if (U_fixed && !U_fixed[s]) { set_error("fdfd_solve_host: NULL U_fixed at %d", s); return DDG_EINVAL; }
        if (grids[s].nx < 3 || grids[s].ny < 3) { set_error("fdfd_solve_host: grid %d too small", s); return DDG_EINVAL; }
        if (P && (grids[s].nx != grids[0].nx || grids[s].ny != grids[0].ny)) {
            set_error("fdfd_solve_host: with a predictor every problem needs the same grid size");
            return DDG_EINVAL;
        }
    }
    Context* ctx = reinterpret_cast<Context*>(cptr);
    cudaStream_t st = as_stream(stream);
    const int k = k_fixed + kp;
    // eps (D doubles), b and x (D complex128 each) and U (k D complex128) per problem
    std::vector<size_t> off(n + 1, 0);
    for (int s = 0; s < n; ++s) {
        const size_t D = (size_t)grids[s].nx * (size_t)grids[s].ny;
        off[s + 1] = off[s] + round256(8 * D) + 2 * round256(16 * D) + round256(16 * D * (size_t)k);
    }
    DDG_TRY(reserve_io(ctx, off[n], st));
    char* base = reinterpret_cast<char*>(ctx->io);
    std::vector<double*> eps(n), b(n), x(n), U(n);
    for (int s = 0; s < n; ++s) {
        const size_t D = (size_t)grids[s].nx * (size_t)grids[s].ny;
        char* p = base + off[s];
        eps[s] = reinterpret_cast<double*>(p);
        b[s] = reinterpret_cast<double*>(p + round256(8 * D));
        x[s] = reinterpret_cast<double*>(p + round256(8 * D) + round256(16 * D));
        U[s] = reinterpret_cast<double*>(p + round256(8 * D) + 2 * round256(16 * D));
        DDG_CHECK_CUDA(cudaMemcpyAsync(eps[s], eps_host[s], 8 * D, cudaMemcpyHostToDevice, st));
    }
    OpList ol;
    ol.ops.assign(n, nullptr);
    for (int s = 0; s < n; ++s) {
        const size_t D = (size_t)grids[s].nx * (size_t)grids[s].ny;
        DDG_TRY(fdfd_operator(&grids[s], eps[s], &ol.ops[s], stream));
        DDG_TRY(fdfd_source(ol.ops[s], i_src, sigma, j_c, b[s], stream));
        DDG_CHECK_CUDA(cudaMemsetAsync(x[s], 0, 16 * D, st));
    }
    ddg_status r;
    if (k > 0) {
        // subspace of problem s: [U_fixed[s] (k_fixed columns) | the predictor's kp vectors]
        std::vector<double*> Up(n);
        for (int s = 0; s < n; ++s) {
            const size_t D = (size_t)grids[s].nx * (size_t)grids[s].ny;
            if (k_fixed)
                DDG_CHECK_CUDA(cudaMemcpyAsync(U[s], U_fixed[s], 16 * D * k_fixed, cudaMemcpyDeviceToDevice, st));
            Up[s] = U[s] + 2 * D * k_fixed;
        }
        if (P) DDG_TRY(subspace_predict(P, n, ol.ops.data(), i_src, sigma, j_c, Up.data(), stream));
        r = augmented_gmres_solve_batched(cptr, n, ol.ops.data(), b.data(), U.data(), k, x.data(), tol, restart,
                                          maxit, prec, info, stream);
    } else {
        r = gmres_solve_batched(cptr, n, ol.ops.data(), b.data(), x.data(), tol, restart, maxit, prec, info, stream);
    }
    if (r != DDG_OK && r != DDG_ENOCONV) return r;
    for (int s = 0; s < n; ++s) {
        const size_t D = (size_t)grids[s].nx * (size_t)grids[s].ny;
        DDG_CHECK_CUDA(cudaMemcpyAsync(x_host[s], x[s], 16 * D, cudaMemcpyDeviceToHost, st));
    }
    DDG_CHECK_CUDA(cudaStreamSynchronize(st));
    return r;
}
