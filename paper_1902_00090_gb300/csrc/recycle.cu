// gmres_solve_trajectories: recycling along design trajectories.  Step t of
// every trajectory is one batched augmented solve whose subspace holds the
// predicted vectors and the trajectory's solution of step t - 1.
#include <vector>

#include "common.cuh"
#include "engine.cuh"

using namespace ddg;

extern "C" ddg_status gmres_solve_trajectories(ddg_context* cptr, int n_traj, int n_steps, const ddg_op* const* A,
                                               const double* const* b, const double* const* U, int k,
                                               double* const* x, double tol, int restart, int maxit,
                                               ddg_precision prec, ddg_info* info, void* stream) {
    if (!cptr || n_traj < 1 || n_steps < 1 || !A || !b || !x) {
        set_error("gmres_solve_trajectories: NULL argument or n_traj=%d, n_steps=%d", n_traj, n_steps);
        return DDG_EINVAL;
    }
    if (U ? (k < 0 || k + 1 > kMaxAug) : k != 0) {
        set_error("gmres_solve_trajectories: k=%d (need 0 <= k < %d, k = 0 without U)", k, kMaxAug);
        return DDG_EINVAL;
    }
    const int n = n_traj * n_steps;
    for (int s = 0; s < n; ++s) {
        if (!A[s] || !b[s] || !x[s] || (U && !U[s])) {
            set_error("gmres_solve_trajectories: NULL operator, b, x or U at %d", s);
            return DDG_EINVAL;
        }
        if (A[s]->D != A[(s / n_steps) * n_steps]->D) {
            set_error("gmres_solve_trajectories: trajectory %d changes its grid size", s / n_steps);
            return DDG_EINVAL;
        }
    }
    Context* ctx = reinterpret_cast<Context*>(cptr);
    cudaStream_t st = as_stream(stream);
    // subspace of every trajectory's current step: [U (k columns) | x_{t-1}]
    std::vector<size_t> off(n_traj + 1, 0);
    for (int r = 0; r < n_traj; ++r)
        off[r + 1] = off[r] + ((size_t)(k + 1) * (size_t)A[r * n_steps]->D * 16 + 255) / 256 * 256;
    if (n_steps > 1 && off[n_traj] > ctx->vbuf_bytes) {
        if (ctx->vbuf) {
            DDG_CHECK_CUDA(cudaStreamSynchronize(st));
            cudaFree(ctx->vbuf);
            ctx->vbuf = nullptr;
            ctx->vbuf_bytes = 0;
        }
        if (cudaMalloc(&ctx->vbuf, off[n_traj]) != cudaSuccess) {
            cudaGetLastError();
            ctx->vbuf = nullptr;
            set_error("gmres_solve_trajectories: cudaMalloc of %zu bytes failed", off[n_traj]);
            return DDG_ENOMEM;
        }
        ctx->vbuf_bytes = off[n_traj];
    }
    std::vector<const ddg_op*> As(n_traj);
    std::vector<const double*> bs(n_traj), Vs(n_traj);
    std::vector<double*> xs(n_traj);
    std::vector<ddg_info> inf(n_traj);
    bool all = true;
    for (int t = 0; t < n_steps; ++t) {
        for (int r = 0; r < n_traj; ++r) {
            const int s = r * n_steps + t;
            As[r] = A[s];
            bs[r] = b[s];
            xs[r] = x[s];
            const size_t D = (size_t)A[s]->D;
            DDG_CHECK_CUDA(cudaMemsetAsync(x[s], 0, 16 * D, st));
            if (t > 0) {
                double* V = reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->vbuf) + off[r]);
                if (k > 0) DDG_CHECK_CUDA(cudaMemcpyAsync(V, U[s], 16 * D * k, cudaMemcpyDeviceToDevice, st));
                DDG_CHECK_CUDA(cudaMemcpyAsync(V + 2 * D * k, x[s - 1], 16 * D, cudaMemcpyDeviceToDevice, st));
                Vs[r] = V;
            } else if (k > 0) {
                Vs[r] = U[s];
            }
        }
        ddg_status e;
        if (t > 0)
            e = augmented_gmres_solve_batched(cptr, n_traj, As.data(), bs.data(), Vs.data(), k + 1, xs.data(), tol,
                                              restart, maxit, prec, inf.data(), stream);
        else if (k > 0)
            e = augmented_gmres_solve_batched(cptr, n_traj, As.data(), bs.data(), Vs.data(), k, xs.data(), tol,
                                              restart, maxit, prec, inf.data(), stream);
        else
            e = gmres_solve_batched(cptr, n_traj, As.data(), bs.data(), xs.data(), tol, restart, maxit, prec,
                                    inf.data(), stream);
        if (e != DDG_OK && e != DDG_ENOCONV) return e;
        all = all && e == DDG_OK;
        if (info)
            for (int r = 0; r < n_traj; ++r) info[r * n_steps + t] = inf[r];
    }
    return all ? DDG_OK : DDG_ENOCONV;
}
