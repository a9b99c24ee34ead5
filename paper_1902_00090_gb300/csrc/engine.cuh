// Internal types of the batched GMRES engine.
#pragma once
#include <vector>

#include <cuda_fp16.h>

#include "common.cuh"

namespace ddg {

constexpr int kBlock = 256;          // threads per CTA of the streaming kernels
constexpr int kWarps = kBlock / 32;
constexpr int kMaxAug = 32;          // largest augmentation size k
constexpr int kMaxRestart = 1024;
constexpr unsigned long long kDefaultWaitNs = 1000000000ull;   // bounded device waits give up after 1 s

// 16-byte packs: every thread of a streaming kernel owns one pack (VEC complex
// numbers) of each work column; a CTA covers kBlock * VEC consecutive rows.
template <typename T> struct PackOf;
template <> struct PackOf<float> { using type = float4; static constexpr int VEC = 2; };
template <> struct PackOf<double> { using type = double2; static constexpr int VEC = 1; };
template <typename T> using pack_t = typename PackOf<T>::type;
template <typename T> __host__ __device__ constexpr int vec_of() { return PackOf<T>::VEC; }
template <typename T> __host__ __device__ constexpr long long chunk_rows() { return (long long)kBlock * PackOf<T>::VEC; }

__device__ __forceinline__ void unpack(const float4& p, float2 (&v)[2]) {
    v[0] = make_float2(p.x, p.y);
    v[1] = make_float2(p.z, p.w);
}
__device__ __forceinline__ void unpack(const double2& p, double2 (&v)[1]) { v[0] = p; }
__device__ __forceinline__ float4 mkpack(const float2 (&v)[2]) { return make_float4(v[0].x, v[0].y, v[1].x, v[1].y); }
__device__ __forceinline__ double2 mkpack(const double2 (&v)[1]) { return v[0]; }

// Storage of the Krylov basis [C | Q] (and nothing else): the arithmetic type,
// or, for complex64 arithmetic, IEEE half (values only: every product and sum
// stays FP32, the true residual FP64).  `round` gives the value a stored
// element will read back as, so that the columns used in dot products, updates
// and the stencil are the same numbers.
template <typename T, bool HB> struct Bstore {
    using V = c2_t<T>;
    static constexpr int VEC = PackOf<T>::VEC;
    using pack = pack_t<T>;                      // one thread's VEC elements
    static constexpr int ebytes = sizeof(V);     // bytes per complex element
    __device__ static __forceinline__ void load(const pack& p, V (&v)[VEC]) { unpack(p, v); }
    __device__ static __forceinline__ pack store(const V (&v)[VEC]) { return mkpack(v); }
    __device__ static __forceinline__ V round(V x) { return x; }
    __device__ static __forceinline__ V get(const void* base, long long i) { return reinterpret_cast<const V*>(base)[i]; }
    __device__ static __forceinline__ void set(void* base, long long i, V x) { reinterpret_cast<V*>(base)[i] = x; }
};
template <> struct Bstore<float, true> {
    using V = float2;
    static constexpr int VEC = 2;
    using pack = uint2;                          // two complex as two __half2
    static constexpr int ebytes = 4;
    __device__ static __forceinline__ float2 h2f(unsigned u) {
        __half2 h = *reinterpret_cast<const __half2*>(&u);
        return __half22float2(h);
    }
    __device__ static __forceinline__ unsigned f2h(float2 x) {
        __half2 h = __float22half2_rn(x);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    __device__ static __forceinline__ void load(const pack& p, V (&v)[2]) {
        v[0] = h2f(p.x);
        v[1] = h2f(p.y);
    }
    __device__ static __forceinline__ pack store(const V (&v)[2]) { return make_uint2(f2h(v[0]), f2h(v[1])); }
    __device__ static __forceinline__ V round(V x) { return h2f(f2h(x)); }
    __device__ static __forceinline__ V get(const void* base, long long i) {
        return h2f(reinterpret_cast<const unsigned*>(base)[i]);
    }
    __device__ static __forceinline__ void set(void* base, long long i, V x) { reinterpret_cast<unsigned*>(base)[i] = f2h(x); }
};

// Solver context: device workspace (grow-only) and tuning.
struct Context {
    int device = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int* host_counts = nullptr;      // pinned (16 ints), polled between launches
    double inner_tol = 1e-5;         // DDG_C64_REFINE inner-cycle relative tolerance
    int orth = 1;                    // 0: CGS2 (two passes per step), 1: delayed CGS2 (one reduction)
    double fallback = 0.5;           // augmented: V-only residual above this -> plain GMRES after the V step
    int aug_cycles = 1;              // augmented: restart cycles that keep all of V
    int aug_keep = 0;                // augmented: leading columns of V kept after those cycles (0: plain GMRES)
    // per-wavelength policies (cycles, keep) overriding the two above
    struct Policy { double wavelength; int cycles, keep; };
    std::vector<Policy> policies;
    int poll_every = 8;              // Arnoldi steps between host polls (host-driven loop)
    int graphs = 1;                  // delayed scheme: step loop as a CUDA graph with a device-side WHILE
    int half_basis = 0;              // complex64 solves: Krylov basis stored in IEEE half
    int precond = 0;                 // 0: none, 1: Jacobi right preconditioner (data-free baseline)
    unsigned long long wait_ns = kDefaultWaitNs;   // bounded waits of the Arnoldi kernels
    size_t ws_limit = 0;             // largest workspace the context may allocate (0: no limit)
    void* io = nullptr;              // fdfd_solve_host: device copies of the call's inputs and outputs
    size_t io_bytes = 0;
    void* vbuf = nullptr;            // gmres_solve_trajectories: each trajectory's [U | x_{t-1}]
    size_t vbuf_bytes = 0;
    int sm_count = 152;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // launch accounting and profiling
    long long launches = 0;
    bool prof = false;
    unsigned long long* d_bytes = nullptr;   // device, DDG_K_NCLASSES counters
    double ms[DDG_K_NCLASSES] = {};
    long long nlaunch[DDG_K_NCLASSES] = {};
    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    ddg_status reserve(size_t bytes, cudaStream_t s);
    cudaEvent_t get_event();
    // Brackets one kernel launch: counts it and, when profiling, records events.
    template <typename F> ddg_status launch(int cls, cudaStream_t s, F&& fn) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (prof) {
            a = get_event();
            if (a) cudaEventRecord(a, s);
        }
        fn();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e, "kernel launch");
        ++launches;
        ++nlaunch[cls];
        if (prof && a) {
            b = get_event();
            if (b) {
                cudaEventRecord(b, s);
                pending.push_back({cls, a, b});
            }
        }
        return DDG_OK;
    }
    // Adds the elapsed times of recorded launches (call after a stream sync).
    void resolve();
    // Restart policy of an augmented solve at this wavelength.
    void policy_for(double wavelength, int* cycles, int* keep) const {
        *cycles = aug_cycles;
        *keep = aug_keep;
        for (const Policy& p : policies)
            if (fabs(p.wavelength - wavelength) <= 1e-9 * fmax(p.wavelength, wavelength)) {
                *cycles = p.cycles;
                *keep = p.keep;
            }
    }
};

// Per-solve device pointers (read-only during a solve).
struct SolvePtrs {
    int nx, ny;
    long long D;
    long long ld;              // leading dimension of every D-long work column (D rounded up to a chunk)
    double kh2;
    const double* eps_d;
    const void* eps_lo;        // float* or double* (precision of the Krylov loop)
    const double2* coef_d;
    const void* coef_lo;       // float2* or double2*
    const void* dinv;          // right preconditioner M^-1 = 1 / diag(A) in the Krylov precision (ld), or null
    const double2* b;
    double2* x;
    double2* r;                // FP64 residual (ld, zero past D)
    void* M;                   // [C | Q] basis, T2, column-major, leading dimension ld
    void* V;                   // predicted vectors in T2 (ld x N), column-major
    const double2* U;          // caller's predicted vectors (FP64, D x N)
    double2* W;                // FP64 scratch for A V during set-up (ld x N, aliases M)
    void* w[2];                // T2 Arnoldi vectors (double buffered)
    double2* Rg;               // Givens-reduced Hessenberg, (m+1) x m, column-major
    double2* Hh;               // delayed scheme: H and B before rotation, in T2 (ld m+1 and kMaxAug)
    double2* tv;               // delayed scheme: [t = [C Q]^H z | s = Q^H u | alpha | gamma] (KP)
    double2* B;                // C^H A Q, kMaxAug x m
    double* cs;                // rotation cosines (m)
    double2* sn;               // rotation sines (m)
    double2* g;                // rotated right-hand side (m+1)
    double2* hsum;             // Gram-Schmidt coefficients, sum of both passes (CGS2); DCGS2: first-pass
                               // coefficients h1 of column j in buffer j & 1 (2 x KP)
    double2* hp;               // coefficients of the current pass (KP)
    double2* part;             // per-CTA partial sums, nchunks x KP
    double2* Rinv;             // R^-1 of A V = C R (N x N, column-major)
    double2* Rtmp;             // first-pass triangular factor inverse (N x N)
    double2* cr;               // C^H r at cycle start (N)
    double2* coefy;            // [z = R^-1 x_V (N) | y (k)]
    unsigned* ticket;
    int chunk0, nchunks;
    int aug_cycles;            // augmented: restart cycles that keep all of V (0: its least-squares step only)
    int aug_keep;              // augmented: leading columns of V kept after those cycles (0: plain GMRES)
};

// Per-solve mutable state.
struct SolveScal {
    int N;            // augmentation size in use (0 = plain)
    int active;       // solve still running
    int in_cycle;     // Arnoldi loop of the current cycle still running
    int pending;      // a cycle ran: back-substitute and update x
    int k;            // Arnoldi steps in the current cycle
    int iters, cycles, converged, breakdown, fallback;
    double nb, rn, beta, target, hnorm, anorm, true_res, first_res;
};

struct BatchArgs {
    unsigned long long* bytes;   // per-class algorithmic byte counters, or null
    SolvePtrs* P;
    SolveScal* S;
    const int* blk_solve;
    int* counts;       // [0] solves inside an Arnoldi loop, [1] solves still active,
                       // [4] a bounded wait gave up (kept for the whole solve call),
                       // [5] the graph-driven loop's step counter, [6..9] the graph's
                       // cycles begun, step-loop bodies, Arnoldi cycles, finished cycles
    int m;             // restart length
    int KP;            // stride of coefficient vectors (>= Nmax + m + 2)
    int nmax;          // leading dimension of B (= kMaxAug)
    double tol;
    double eta;        // inner relative tolerance (0 for complex128)
    double fallback;   // V-only relative residual above which an augmented solve continues as plain GMRES
    int maxit;
    int nsolves;       // solves in the batch (k_update2 puts one block per solve in front of its sweep)
    int* step;         // Arnoldi step of the graph-driven loop (kernels launched with i <= 0 add it)
    int low_res;       // DDG_C64_ONLY: the restart residual r = b - A x in the Krylov precision
    unsigned long long wait_ns;   // limit of the bounded waits on bulk copies into shared memory
};

// Adds `v` to the class counter once per CTA (thread 0), when profiling.
__device__ __forceinline__ void count_bytes(const BatchArgs& a, int cls, double v) {
    if (a.bytes && threadIdx.x == 0) atomicAdd(a.bytes + cls, (unsigned long long)v);
}

}  // namespace ddg
