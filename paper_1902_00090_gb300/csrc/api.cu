// Status strings, per-thread error text and the solver context (workspace owner).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <new>

#include "common.cuh"
#include "engine.cuh"

namespace ddg {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ddg_status cuda_status(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return DDG_ENOMEM;
    }
    return DDG_ECUDA;
}

ddg_status Context::reserve(size_t bytes, cudaStream_t s) {
    if (bytes <= ws_bytes) return DDG_OK;
    if (ws) {
        DDG_CHECK_CUDA(cudaStreamSynchronize(s));
        cudaFree(ws);
        ws = nullptr;
        ws_bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    if (ws_limit) {
        if (bytes > ws_limit) {
            set_error("workspace: %zu bytes needed, above the context's limit of %zu bytes "
                      "(ddg_context_set_workspace_limit)", bytes, ws_limit);
            return DDG_ENOMEM;
        }
        want = std::min(want, ws_limit);
    }
    cudaError_t e = cudaMalloc(&ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ws = nullptr;
        set_error("workspace: cudaMalloc of %zu bytes failed", want);
        return DDG_ENOMEM;
    }
    ws_bytes = want;
    return DDG_OK;
}

cudaEvent_t Context::get_event() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void Context::resolve() {
    for (auto& p : pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.cls] += t;
        else cudaGetLastError();
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.clear();
}

}  // namespace ddg

using namespace ddg;

extern "C" const char* ddg_status_str(ddg_status s) {
    switch (s) {
        case DDG_OK: return "ok";
        case DDG_EINVAL: return "invalid argument";
        case DDG_ENOMEM: return "out of device memory";
        case DDG_ECUDA: return "CUDA error";
        case DDG_ENOCONV: return "not converged within the iteration cap";
        case DDG_EBREAKDOWN: return "breakdown";
        case DDG_ETIMEOUT: return "device watchdog expired";
        case DDG_ESINGULAR: return "singular factorisation";
    }
    return "unknown status";
}

extern "C" const char* ddg_last_error(void) { return g_err; }

extern "C" int ddg_version(void) { return 100; }

extern "C" ddg_status ddg_context_create(ddg_context** out) {
    if (!out) { set_error("ddg_context_create: out is NULL"); return DDG_EINVAL; }
    Context* c = new (std::nothrow) Context();
    if (!c) return DDG_ENOMEM;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (c->sm_count <= 0) c->sm_count = 152;
    cudaError_t e = cudaMallocHost(&c->host_counts, 16 * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_bytes, DDG_K_NCLASSES * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_bytes, 0, DDG_K_NCLASSES * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        delete c;
        return cuda_status(e, "ddg_context_create: cudaMallocHost");
    }
    *out = reinterpret_cast<ddg_context*>(c);
    return DDG_OK;
}

extern "C" ddg_status ddg_context_destroy(ddg_context* ctx) {
    if (!ctx) return DDG_OK;
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaFree(c->ws);
    cudaFree(c->io);
    cudaFree(c->vbuf);
    cudaFreeHost(c->host_counts);
    if (c->ev[0]) cudaEventDestroy(c->ev[0]);
    if (c->ev[1]) cudaEventDestroy(c->ev[1]);
    cudaFree(c->d_bytes);
    c->resolve();
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    delete c;
    return DDG_OK;
}

extern "C" long long ddg_context_workspace_bytes(const ddg_context* ctx) {
    return ctx ? (long long)reinterpret_cast<const Context*>(ctx)->ws_bytes : 0;
}

extern "C" ddg_status ddg_context_set_inner_tol(ddg_context* ctx, double eta) {
    if (!ctx || !(eta > 0.0 && eta < 1.0)) { set_error("inner tol must be in (0,1)"); return DDG_EINVAL; }
    reinterpret_cast<Context*>(ctx)->inner_tol = eta;
    return DDG_OK;
}

extern "C" long long ddg_context_launches(const ddg_context* ctx) {
    return ctx ? reinterpret_cast<const Context*>(ctx)->launches : 0;
}

extern "C" ddg_status ddg_context_profile_enable(ddg_context* ctx, int enable) {
    if (!ctx) { set_error("ddg_context_profile_enable: NULL context"); return DDG_EINVAL; }
    Context* c = reinterpret_cast<Context*>(ctx);
    DDG_CHECK_CUDA(cudaDeviceSynchronize());
    c->resolve();
    for (int i = 0; i < DDG_K_NCLASSES; ++i) {
        c->ms[i] = 0.0;
        c->nlaunch[i] = 0;
    }
    DDG_CHECK_CUDA(cudaMemset(c->d_bytes, 0, DDG_K_NCLASSES * sizeof(unsigned long long)));
    c->prof = enable != 0;
    return DDG_OK;
}

extern "C" ddg_status ddg_context_profile_read(ddg_context* ctx, int cls, double* ms, double* bytes,
                                               long long* launches) {
    if (!ctx || cls < 0 || cls >= DDG_K_NCLASSES) { set_error("ddg_context_profile_read: bad argument"); return DDG_EINVAL; }
    Context* c = reinterpret_cast<Context*>(ctx);
    DDG_CHECK_CUDA(cudaDeviceSynchronize());
    c->resolve();
    unsigned long long hb[DDG_K_NCLASSES];
    DDG_CHECK_CUDA(cudaMemcpy(hb, c->d_bytes, sizeof(hb), cudaMemcpyDeviceToHost));
    if (ms) *ms = c->ms[cls];
    if (bytes) *bytes = (double)hb[cls];
    if (launches) *launches = c->nlaunch[cls];
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_orthogonalization(ddg_context* ctx, int scheme) {
    if (!ctx || (scheme != DDG_ORTH_CGS2 && scheme != DDG_ORTH_DCGS2)) {
        set_error("ddg_context_set_orthogonalization: bad context or scheme %d", scheme);
        return DDG_EINVAL;
    }
    reinterpret_cast<Context*>(ctx)->orth = scheme;
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_graphs(ddg_context* ctx, int enable) {
    if (!ctx) { set_error("ddg_context_set_graphs: NULL context"); return DDG_EINVAL; }
    reinterpret_cast<Context*>(ctx)->graphs = enable ? 1 : 0;
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_basis_storage(ddg_context* ctx, int half) {
    if (!ctx) { set_error("ddg_context_set_basis_storage: NULL context"); return DDG_EINVAL; }
    reinterpret_cast<Context*>(ctx)->half_basis = half ? 1 : 0;
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_preconditioner(ddg_context* ctx, int kind) {
    if (!ctx || kind < 0 || kind > 1) { set_error("ddg_context_set_preconditioner: bad context or kind %d", kind); return DDG_EINVAL; }
    reinterpret_cast<Context*>(ctx)->precond = kind;
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_fallback(ddg_context* ctx, double threshold) {
    if (!ctx || !(threshold > 0.0)) { set_error("ddg_context_set_fallback: threshold must be > 0"); return DDG_EINVAL; }
    reinterpret_cast<Context*>(ctx)->fallback = threshold;
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_augmented_policy(ddg_context* ctx, double wavelength, int cycles, int keep) {
    if (!ctx || !(wavelength >= 0.0) || cycles < 0 || keep < 0 || keep > kMaxAug) {
        set_error("ddg_context_set_augmented_policy: need wavelength >= 0, cycles >= 0, 0 <= keep <= %d", kMaxAug);
        return DDG_EINVAL;
    }
    Context* c = reinterpret_cast<Context*>(ctx);
    if (wavelength == 0.0) {
        c->aug_cycles = cycles;
        c->aug_keep = keep;
        return DDG_OK;
    }
    for (auto& p : c->policies)
        if (fabs(p.wavelength - wavelength) <= 1e-9 * fmax(p.wavelength, wavelength)) {
            p.cycles = cycles;
            p.keep = keep;
            return DDG_OK;
        }
    c->policies.push_back({wavelength, cycles, keep});
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_wait_limit(ddg_context* ctx, long long ns) {
    if (!ctx || ns < 0 || ns > 10000000000LL) {
        set_error("ddg_context_set_wait_limit: need 0 <= ns <= 1e10");
        return DDG_EINVAL;
    }
    reinterpret_cast<Context*>(ctx)->wait_ns = (unsigned long long)ns;
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_workspace_limit(ddg_context* ctx, long long bytes) {
    if (!ctx || bytes < 0) { set_error("ddg_context_set_workspace_limit: need bytes >= 0"); return DDG_EINVAL; }
    Context* c = reinterpret_cast<Context*>(ctx);
    c->ws_limit = (size_t)bytes;
    if (bytes && c->ws_bytes > (size_t)bytes) {
        // give back a workspace above the new limit (the next call allocates within it)
        DDG_CHECK_CUDA(cudaDeviceSynchronize());
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    return DDG_OK;
}

extern "C" ddg_status ddg_context_set_augmented_cycles(ddg_context* ctx, int cycles) {
    if (!ctx || cycles < 0) { set_error("ddg_context_set_augmented_cycles: cycles must be >= 0"); return DDG_EINVAL; }
    reinterpret_cast<Context*>(ctx)->aug_cycles = cycles;
    return DDG_OK;
}
