// Solve queue: many independent solves run as groups of batched solves, taken
// in order by a few lanes that work concurrently (one host thread, context and
// stream per lane), so that the last solves of one group run beside the next
// group's.  Host code only: every group is an ordinary batched solve.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "engine.cuh"

namespace ddg {

constexpr int kMaxLanes = 8;

// Everything a lane needs, shared read-only (plus the group counter and the
// first error) between the lane threads.
struct QueueJob {
    ddg_context* const* lanes;
    void* const* streams;
    int width, n, k, restart, maxit, device;
    int n_steps = 0;                  // > 0: groups of `width` trajectories of n_steps solves (recycling)
    const ddg_op* const* A;
    const double* const* b;
    const double* const* U;
    double* const* x;
    double tol;
    ddg_precision prec;
    ddg_info* info;
    std::atomic<int> next{0};         // next group to take
    std::atomic<bool> stop{false};    // a lane met an error: take no more groups
    std::atomic<bool> missed{false};  // some solve missed the tolerance
    std::mutex mu;
    ddg_status err = DDG_OK;          // first error, and its message
    std::string msg;
};

static void run_lane(QueueJob* j, int lane) {
    cudaError_t e = cudaSetDevice(j->device);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(j->mu);
        if (j->err == DDG_OK) {
            j->err = cuda_status(e, "gmres_solve_queue: cudaSetDevice");
            j->msg = ddg_last_error();
        }
        j->stop = true;
        return;
    }
    const int units = j->n_steps > 0 ? j->n / j->n_steps : j->n;   // solves, or trajectories
    const int groups = (units + j->width - 1) / j->width;
    while (!j->stop) {
        const int g = j->next.fetch_add(1);
        if (g >= groups) break;
        const int u0 = g * j->width;
        const int cnt = std::min(j->width, units - u0);
        const int s0 = j->n_steps > 0 ? u0 * j->n_steps : u0;
        ddg_info* inf = j->info ? j->info + s0 : nullptr;
        ddg_status st;
        if (j->n_steps > 0)
            st = gmres_solve_trajectories(j->lanes[lane], cnt, j->n_steps, j->A + s0, j->b + s0,
                                          j->U ? j->U + s0 : nullptr, j->k, j->x + s0, j->tol, j->restart,
                                          j->maxit, j->prec, inf, j->streams ? j->streams[lane] : nullptr);
        else if (j->U)
            st = augmented_gmres_solve_batched(j->lanes[lane], cnt, j->A + s0, j->b + s0, j->U + s0, j->k,
                                               j->x + s0, j->tol, j->restart, j->maxit, j->prec, inf,
                                               j->streams ? j->streams[lane] : nullptr);
        else
            st = gmres_solve_batched(j->lanes[lane], cnt, j->A + s0, j->b + s0, j->x + s0, j->tol, j->restart,
                                     j->maxit, j->prec, inf, j->streams ? j->streams[lane] : nullptr);
        if (st == DDG_ENOCONV) {
            j->missed = true;
        } else if (st != DDG_OK) {
            std::lock_guard<std::mutex> lk(j->mu);
            if (j->err == DDG_OK) {
                j->err = st;
                j->msg = ddg_last_error();
            }
            j->stop = true;
        }
    }
}

}  // namespace ddg

using namespace ddg;

static ddg_status run_queue(ddg_context* const* lanes, void* const* streams, int nlanes, int width, int n,
                            int n_steps, const ddg_op* const* A, const double* const* b, const double* const* U,
                            int k, double* const* x, double tol, int restart, int maxit, ddg_precision prec,
                            ddg_info* info);

extern "C" ddg_status gmres_solve_queue(ddg_context* const* lanes, void* const* streams, int nlanes, int width,
                                        int n, const ddg_op* const* A, const double* const* b,
                                        const double* const* U, int k, double* const* x, double tol, int restart,
                                        int maxit, ddg_precision prec, ddg_info* info) {
    return run_queue(lanes, streams, nlanes, width, n, 0, A, b, U, k, x, tol, restart, maxit, prec, info);
}

extern "C" ddg_status gmres_solve_queue_trajectories(ddg_context* const* lanes, void* const* streams, int nlanes,
                                                     int traj_per_group, int n_traj, int n_steps,
                                                     const ddg_op* const* A, const double* const* b,
                                                     const double* const* U, int k, double* const* x, double tol,
                                                     int restart, int maxit, ddg_precision prec, ddg_info* info) {
    if (n_traj < 1 || n_steps < 1) {
        set_error("gmres_solve_queue_trajectories: n_traj=%d, n_steps=%d", n_traj, n_steps);
        return DDG_EINVAL;
    }
    return run_queue(lanes, streams, nlanes, traj_per_group, n_traj * n_steps, n_steps, A, b, U, k, x, tol, restart,
                     maxit, prec, info);
}

static ddg_status run_queue(ddg_context* const* lanes, void* const* streams, int nlanes, int width, int n,
                            int n_steps, const ddg_op* const* A, const double* const* b, const double* const* U,
                            int k, double* const* x, double tol, int restart, int maxit, ddg_precision prec,
                            ddg_info* info) {
    if (!lanes || nlanes < 1 || nlanes > kMaxLanes) {
        set_error("gmres_solve_queue: lanes NULL or nlanes=%d outside [1,%d]", nlanes, kMaxLanes);
        return DDG_EINVAL;
    }
    if (width < 1 || n < 1 || !A || !b || !x) {
        set_error("gmres_solve_queue: width=%d, n=%d or NULL array", width, n);
        return DDG_EINVAL;
    }
    for (int l = 0; l < nlanes; ++l) {
        if (!lanes[l]) { set_error("gmres_solve_queue: lane %d has no context", l); return DDG_EINVAL; }
        for (int m = 0; m < l; ++m)
            if (lanes[m] == lanes[l] || (streams && streams[m] && streams[m] == streams[l])) {
                set_error("gmres_solve_queue: lanes %d and %d share a context or a stream", m, l);
                return DDG_EINVAL;
            }
    }
    QueueJob j;
    j.lanes = lanes;
    j.streams = streams;
    j.width = width;
    j.n = n;
    j.k = k;
    j.restart = restart;
    j.maxit = maxit;
    j.A = A;
    j.b = b;
    j.U = U;
    j.x = x;
    j.tol = tol;
    j.prec = prec;
    j.info = info;
    j.n_steps = n_steps;
    DDG_CHECK_CUDA(cudaGetDevice(&j.device));
    const int groups = ((n_steps > 0 ? n / n_steps : n) + width - 1) / width;
    const int used = std::min(nlanes, groups);
    if (used == 1) {
        run_lane(&j, 0);   // no thread for a single lane
    } else {
        std::vector<std::thread> th;
        th.reserve(used);
        try {
            for (int l = 0; l < used; ++l) th.emplace_back(run_lane, &j, l);
        } catch (...) {
            j.stop = true;
            for (auto& t : th) t.join();
            set_error("gmres_solve_queue: could not start a lane thread");
            return DDG_ENOMEM;
        }
        for (auto& t : th) t.join();
    }
    if (j.err != DDG_OK) {
        set_error("%s", j.msg.c_str());
        return j.err;
    }
    return j.missed ? DDG_ENOCONV : DDG_OK;
}
