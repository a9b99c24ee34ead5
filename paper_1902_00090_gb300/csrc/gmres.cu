// Batched restarted GMRES (Eq. 2) and data-driven GMRES (Eqs. 3-4, supplement
// S1-S7) for FDFD operators.
//
// Execution model: n independent solves advance in lock step, one kernel launch
// per phase covering every CTA of every solve still running; CTAs of finished
// solves return at once.  Each solve is cut into chunks of kBlock * VEC rows
// (one CTA per chunk, one 16-byte pack of VEC complex numbers per thread); all
// work columns use the padded leading dimension ld (a whole number of chunks,
// zero past D), so the streaming loops carry no bounds checks.  Reductions are
// deterministic: every CTA writes its partial sums, and the last CTA of a solve
// to finish (atomic ticket, no waiting) adds them in chunk order and takes the
// solve's scalar decisions (Givens rotation, convergence) in FP64.
//
// One Arnoldi step j (Eq. S2 with one reorthogonalisation, the augmentation
// block C treated as leading columns of the basis, so that the C^H A q_j block
// of Eq. S7 comes out of the same projections):
//   k_step      q_j = w_{j-1} / h_{j,j-1} (stored), w = A q_j        (stencil)
//   k_dots_w    h  = [C Q_j]^H w, and ||w||                           (pass 1)
//   k_update_w  w -= [C Q_j] h
//   k_dots_w    h' = [C Q_j]^H w                                      (pass 2)
//   k_update_w  w -= [C Q_j] h', h_{j+1,j} = ||w||, Givens rotation, |g_{j+1}|
// Cycle start: r = b - A x in FP64; (augmented) c_r = C^H r, r <- r - C c_r.
// Cycle end: y from the rotated Hessenberg, x_V = c_r - B y, z = R^-1 x_V,
// x += V z + Q y (FP64).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "bulk.cuh"
#include "engine.cuh"

namespace ddg {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ double block_sum_d(double v, double* sm) {
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kWarps; ++w) t += sm[w];
    return t;  // valid in thread 0
}

// Sum over the CTA in precision T (every thread gets the total).
template <typename T> __device__ __forceinline__ T block_sum_all(T v, T* sm) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    T t = (T)0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += sm[w];
    __syncthreads();
    return t;
}

// Returns true in every thread of the CTA that is the last of `n` CTAs to
// arrive on `ticket` (partials of all CTAs are then visible); resets the ticket.
__device__ __forceinline__ bool arrive_last(unsigned* ticket, int n) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == (unsigned)(n - 1));
        if (s_last) *ticket = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// 5-point stencil of A at cell e; ld(idx) returns the input vector at idx.
// The cell's row and column come from 32-bit division: fdfd_operator accepts
// no grid of 2^31 cells or more.
template <typename V, typename S, typename LD>
__device__ __forceinline__ V stencil(long long e, int nx, int ny, const V* __restrict__ coef, S kh2eps,
                                     const LD& ld) {
    const unsigned eu = (unsigned)e;
    const int j = (int)(eu / (unsigned)nx);
    const int i = (int)(eu - (unsigned)j * (unsigned)nx);
    const V axp = coef[i], axm = coef[nx + i];
    const V ayp = coef[2 * nx + j], aym = coef[2 * nx + ny + j];
    const long long ip = (i == nx - 1) ? e - (nx - 1) : e + 1;
    const long long im = (i == 0) ? e + (nx - 1) : e - 1;
    const long long jp = (j == ny - 1) ? e - (long long)(ny - 1) * nx : e + nx;
    const long long jm = (j == 0) ? e + (long long)(ny - 1) * nx : e - nx;
    V d = cadd(cadd(axp, axm), cadd(ayp, aym));
    d.x -= kh2eps;
    V acc = cmul(d, ld(e));
    cfms(acc, axp, ld(ip));
    cfms(acc, axm, ld(im));
    cfms(acc, ayp, ld(jp));
    cfms(acc, aym, ld(jm));
    return acc;
}

// Complex Givens rotation with real second entry b >= 0 (Golub & Van Loan 5.1.8):
// [[c, s], [-conj(s), c]] [a; b] = [r; 0], c real.
__device__ __forceinline__ void givens_d(double2 a, double b, double& c, double2& s, double2& r) {
    double aa = hypot(a.x, a.y);
    if (b == 0.0) {
        c = 1.0; s = make_double2(0.0, 0.0); r = a;
    } else if (aa == 0.0) {
        c = 0.0; s = make_double2(1.0, 0.0); r = make_double2(b, 0.0);
    } else {
        double t = hypot(aa, b);
        double2 ph = make_double2(a.x / aa, a.y / aa);
        c = aa / t;
        s = make_double2(ph.x * b / t, ph.y * b / t);
        r = make_double2(ph.x * t, ph.y * t);
    }
}

__device__ __forceinline__ void rotate(double c, double2 s, double2& u, double2& v) {
    double2 nu = cadd(cscale(u, c), cmul(s, v));
    double2 nv = csub(cscale(v, c), cmulc(s, u));
    u = nu;
    v = nv;
}

__device__ __forceinline__ double2 shfl_up_d2(double2 v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl_idx_d2(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Applies the j stored rotations to column j of the Hessenberg matrix, forms
// rotation j and updates g (one warp; col, cs, sn, out in shared memory).
// Applying rotations l = 0..j-1 in turn is the linear recurrence
//   carry_0 = col_0,  out_l = c_l carry_l + s_l col_{l+1},
//   carry_{l+1} = -conj(s_l) carry_l + c_l col_{l+1},
// evaluated as a warp prefix scan of the affine maps carry -> a carry + b:
// every lane composes the maps of its segment, the lanes scan the composites
// (5 shuffle levels) and replay their segment from its starting carry.  The
// dependent chain is O(j/32 + 5) instead of O(j): FP64 latency on this part is
// long.  Returns |g_{j+1}| (valid in every lane); out[0..j] is the rotated column.
__device__ __noinline__ double givens_column_warp(const double2* col, const double* cs, const double2* sn, int j,
                                                  double sub, double2* out, double2* g, double* cs_out,
                                                  double2* sn_out) {
    const int lane = threadIdx.x & 31;
    const int L = (j + 31) / 32;
    const int l0 = min(j, lane * L), l1 = min(j, l0 + L);
    double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
    for (int l = l0; l < l1; ++l) {
        const double2 a = make_double2(-sn[l].x, sn[l].y);  // -conj(s_l)
        const double2 b = cscale(col[l + 1], cs[l]);
        A = cmul(a, A);
        B = cadd(cmul(a, B), b);
    }
    // inclusive scan: (A, B) <- (A, B) o (A_prev, B_prev)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double2 Ap = shfl_up_d2(A, d), Bp = shfl_up_d2(B, d);
        if (lane >= d) {
            B = cadd(cmul(A, Bp), B);
            A = cmul(A, Ap);
        }
    }
    double2 Ae = shfl_up_d2(A, 1), Be = shfl_up_d2(B, 1);
    if (lane == 0) {
        Ae = make_double2(1.0, 0.0);
        Be = make_double2(0.0, 0.0);
    }
    const double2 c0 = col[0];
    double2 carry = cadd(cmul(Ae, c0), Be);
    for (int l = l0; l < l1; ++l) {
        const double2 nx = col[l + 1];
        out[l] = cadd(cscale(carry, cs[l]), cmul(sn[l], nx));
        carry = cadd(cmul(make_double2(-sn[l].x, sn[l].y), carry), cscale(nx, cs[l]));
    }
    const double2 Af = shfl_idx_d2(A, 31), Bf = shfl_idx_d2(B, 31);
    const double2 cj = cadd(cmul(Af, c0), Bf);   // column entry j after all rotations
    double est = 0.0;
    if (lane == 0) {
        double c;
        double2 snj, r;
        givens_d(cj, sub, c, snj, r);
        out[j] = r;
        out[j + 1] = make_double2(0.0, 0.0);
        *cs_out = c;
        *sn_out = snj;
        const double2 gj = g[j];
        g[j] = cscale(gj, c);
        const double2 gj1 = make_double2(-(snj.x * gj.x + snj.y * gj.y), -(snj.x * gj.y - snj.y * gj.x));
        g[j + 1] = gj1;
        est = hypot(gj1.x, gj1.y);
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, est, 0);
}

template <typename T> __device__ __forceinline__ pack_t<T> zero_pack();
template <> __device__ __forceinline__ float4 zero_pack<float>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_pack<double>() { return make_double2(0.0, 0.0); }

// Sum of 8 complex values over the 32 lanes of a warp with 9 exchanges
// (butterfly: each level halves the values a lane holds).  On return lane L
// holds the total of value ((L>>4)&1)*4 + ((L>>3)&1)*2 + ((L>>2)&1).
template <typename V> __device__ __forceinline__ V reduce8(const V (&x)[8], int lane) {
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
    V y4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        V keep = b16 ? x[i + 4] : x[i];
        V send = b16 ? x[i] : x[i + 4];
        y4[i] = cadd(keep, shfl_xor(send, 16));
    }
    V y2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        V keep = b8 ? y4[i + 2] : y4[i];
        V send = b8 ? y4[i] : y4[i + 2];
        y2[i] = cadd(keep, shfl_xor(send, 8));
    }
    V y1 = cadd(b4 ? y2[1] : y2[0], shfl_xor(b4 ? y2[0] : y2[1], 4));
    y1 = cadd(y1, shfl_xor(y1, 2));
    y1 = cadd(y1, shfl_xor(y1, 1));
    return y1;
}

// reduce8 for values a lane already holds in its butterfly order: the lane
// whose partner at level 16 / 8 / 4 keeps a given half holds that half in the
// other position, so every level keeps x[0 .. h) and sends x[h .. 2h) with no
// per-lane selects (5 of the 9 exchanges' instructions were selects).  The
// caller arranges the order: with lane bits b16, b8, b4 a lane must hold in
// x[w] (w < 4) the value that reduce8 expects at index
// (w ^ (2 b8 + b4)) + 4 b16, and in x[w + 4] the one at (w ^ (2 b8 + b4)) + 4 (1 - b16).
// On return lane L holds the same total as reduce8's.
template <typename V> __device__ __forceinline__ V reduce8_ordered(const V (&x)[8]) {
    V y4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) y4[i] = cadd(x[i], shfl_xor(x[i + 4], 16));
    V y2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) y2[i] = cadd(y4[i], shfl_xor(y4[i + 2], 8));
    V y1 = cadd(y2[0], shfl_xor(y2[1], 4));
    y1 = cadd(y1, shfl_xor(y1, 2));
    y1 = cadd(y1, shfl_xor(y1, 1));
    return y1;
}

#define SOLVE_PROLOGUE()                                  \
    const int s = a.blk_solve[blockIdx.x];                \
    SolveScal* S = a.S + s;                               \
    const SolvePtrs& P = a.P[s];                          \
    const int chunk = blockIdx.x - P.chunk0;

// ---------------------------------------------------------------- init
__global__ void k_init(BatchArgs a, int n, int nreq) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SolveScal* S = a.S + s;
    S->N = nreq;
    S->active = 1;
    S->in_cycle = 0;
    S->pending = 0;
    S->k = 0;
    S->iters = 0;
    S->cycles = 0;
    S->converged = 0;
    S->breakdown = 0;
    S->fallback = 0;
    S->nb = -1.0;
    S->rn = 0.0;
    S->beta = 0.0;
    S->target = 0.0;
    S->hnorm = 1.0;
    S->anorm = 0.0;
    S->true_res = INFINITY;
    S->first_res = NAN;
    *a.P[s].ticket = 0u;
}

// ---------------------------------------------------------------- cycle start
// r = b - A x (FP64, zero past D); ||r||, ||b||; convergence / cap decisions.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_residual(BatchArgs a) {
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    if (!S->active) return;
    const long long D = P.D;
    const long long e0 = (long long)chunk * chunk_rows<T>() + (long long)threadIdx.x * VEC;
    // x, b read and r written (16 B each), eps (8 B, or 4 B in the Krylov precision)
    count_bytes(a, DDG_K_RESIDUAL, (double)min((long long)chunk_rows<T>(), D - (long long)chunk * chunk_rows<T>()) *
                                       (a.low_res ? 52.0 : 56.0));
    __shared__ double sm[kWarps];
    const double2* __restrict__ x = P.x;
    double accr = 0.0, accb = 0.0;
    if (a.low_res) {
        // DDG_C64_ONLY: the residual in the Krylov precision, from the operator's
        // low-precision copy (no FP64 refinement)
        using V = c2_t<T>;
        const T* eps = reinterpret_cast<const T*>(P.eps_lo);
        const V* coef = reinterpret_cast<const V*>(P.coef_lo);
        const T kh2 = (T)P.kh2;
        auto ldl = [&](long long idx) { return from_d2<V>(x[idx]); };
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            const long long e = e0 + q;
            V rv = mk((T)0, (T)0);
            if (e < D) {
                const V ax = stencil(e, P.nx, P.ny, coef, kh2 * eps[e], ldl);
                const V bv = from_d2<V>(P.b[e]);
                rv = csub(bv, ax);
                accr += cabs2(rv);
                accb += cabs2(bv);
            }
            P.r[e] = to_d2(rv);
        }
    } else {
        auto ld = [&](long long idx) { return x[idx]; };
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            const long long e = e0 + q;
            double2 rv = make_double2(0.0, 0.0);
            if (e < D) {
                double2 ax = stencil(e, P.nx, P.ny, P.coef_d, P.kh2 * P.eps_d[e], ld);
                double2 bv = P.b[e];
                rv = csub(bv, ax);
                accr += cabs2(rv);
                accb += cabs2(bv);
            }
            P.r[e] = rv;
        }
    }
    double tr = block_sum_d(accr, sm);
    double tb = block_sum_d(accb, sm);
    if (threadIdx.x == 0) P.part[(long long)chunk * a.KP] = make_double2(tr, tb);
    if (!arrive_last(P.ticket, P.nchunks)) return;
    if (threadIdx.x != 0) return;
    double rn2 = 0.0, nb2 = 0.0;
    for (int c = 0; c < P.nchunks; ++c) {
        double2 t = __ldcg(P.part + (long long)c * a.KP);
        rn2 += t.x;
        nb2 += t.y;
    }
    if (S->nb < 0.0) S->nb = sqrt(nb2);
    // after a fallback (or a rank-deficient V) the solve continues as plain
    // GMRES; once the augmented cycles are done it keeps the leading aug_keep
    // columns of V (C and R of A V are triangular in the column order, so
    // those columns of C and the leading block of R^-1 are the factors of the
    // kept vectors): R^-1 is compacted to the smaller leading dimension
    if (S->fallback) {
        S->N = 0;
    } else if (S->N > 0 && S->cycles >= max(1, P.aug_cycles) && P.aug_keep < S->N) {
        const int N0 = S->N, N1 = max(0, P.aug_keep);
        for (int l = 0; l < N1; ++l)
            for (int n = 0; n < N1; ++n) P.Rinv[l * N1 + n] = P.Rinv[l * N0 + n];   // in place, forward
        S->N = N1;
    }
    const double nb = S->nb, rn = sqrt(rn2);
    S->rn = rn;
    S->pending = 0;
    S->k = 0;
    S->in_cycle = 0;
    if (nb == 0.0) {
        S->true_res = 0.0;
        S->converged = 1;
        S->active = 0;
        return;
    }
    S->true_res = rn / nb;
    if (rn <= a.tol * nb) {
        S->converged = 1;
        S->active = 0;
        return;
    }
    if (S->iters >= a.maxit || S->cycles >= a.maxit || !(rn == rn) || isinf(rn)) {
        S->active = 0;
        return;
    }
    atomicAdd(a.counts + 1, 1);
    S->cycles += 1;
    S->pending = 1;
    if (S->N == 0) {
        S->beta = rn;
        S->hnorm = rn;
        P.g[0] = make_double2(rn, 0.0);
        S->target = fmax(a.tol * nb, a.eta * rn);
        S->in_cycle = 1;
        atomicAdd(a.counts, 1);
    }
    // augmented solves: k_dots_r and k_update_r finish the cycle start
}

// c_r = C^H r (FP64 r, C in the Krylov precision), one warp reduction per column.
template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock) k_dots_r(BatchArgs a) {
    using V = c2_t<T>;
    using BS = Bstore<T, HB>;
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    const int N = S->N;
    if (!S->pending || S->in_cycle || N == 0) return;
    const long long ld = P.ld;
    const long long e0 = (long long)chunk * chunk_rows<T>() + (long long)threadIdx.x * VEC;
    count_bytes(a, DDG_K_RESIDUAL, (double)chunk_rows<T>() * ((double)N * BS::ebytes + 16.0));
    double2 rv[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) rv[q] = P.r[e0 + q];
    __shared__ double2 red[kWarps][kMaxAug];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int n = 0; n < N; ++n) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < VEC; ++q) cfmac(acc, to_d2(BS::get(P.M, (long long)n * ld + e0 + q)), rv[q]);
        acc = warp_sum(acc);
        if (lane == 0) red[wid][n] = acc;
    }
    __syncthreads();
    double2* part = P.part + (long long)chunk * a.KP;
    for (int n = threadIdx.x; n < N; n += kBlock) {
        double2 sum = make_double2(0.0, 0.0);
        for (int w = 0; w < kWarps; ++w) sum = cadd(sum, red[w][n]);
        part[n] = sum;
    }
    if (!arrive_last(P.ticket, P.nchunks)) return;
    for (int n = threadIdx.x; n < N; n += kBlock) {
        double2 sum = make_double2(0.0, 0.0);
        for (int c = 0; c < P.nchunks; ++c) sum = cadd(sum, __ldcg(P.part + (long long)c * a.KP + n));
        P.cr[n] = sum;
    }
}

// r~ = r - C c_r (FP64), beta = ||r~||: start of the Krylov loop on A~ = P_perp A.
template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock) k_update_r(BatchArgs a) {
    using V = c2_t<T>;
    using BS = Bstore<T, HB>;
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    const int N = S->N;
    if (!S->pending || S->in_cycle || N == 0) return;
    const long long ld = P.ld;
    const long long e0 = (long long)chunk * chunk_rows<T>() + (long long)threadIdx.x * VEC;
    count_bytes(a, DDG_K_RESIDUAL, (double)chunk_rows<T>() * ((double)N * BS::ebytes + 32.0));
    __shared__ double sm[kWarps];
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
        double2 v = P.r[e0 + q];
        for (int n = 0; n < N; ++n) cfms(v, to_d2(BS::get(P.M, (long long)n * ld + e0 + q)), P.cr[n]);
        P.r[e0 + q] = v;
        acc += cabs2(v);
    }
    double tot = block_sum_d(acc, sm);
    if (threadIdx.x == 0) P.part[(long long)chunk * a.KP] = make_double2(tot, 0.0);
    if (!arrive_last(P.ticket, P.nchunks)) return;
    if (threadIdx.x != 0) return;
    double n2 = 0.0;
    for (int c = 0; c < P.nchunks; ++c) n2 += __ldcg(P.part + (long long)c * a.KP).x;
    const double nrm = sqrt(n2);
    S->beta = nrm;
    if (S->cycles == 1) S->first_res = nrm / S->nb;
    S->k = 0;
    if (S->cycles == 1 && (nrm > a.fallback * S->nb || P.aug_cycles == 0)) {
        // the predicted subspace fails to cut the residual: keep its least-squares
        // step (x += V R^-1 C^H r at the cycle end) and continue as plain GMRES
        S->fallback = 1;
        return;
    }
    if (nrm <= 1e-14 * S->rn) {
        // r lies in span(A V): the V step alone solves the residual equation
        S->breakdown = 1;
        return;
    }
    S->hnorm = nrm;
    P.g[0] = make_double2(nrm, 0.0);
    S->target = fmax(a.tol * S->nb, a.eta * nrm);
    S->in_cycle = 1;
    atomicAdd(a.counts, 1);
}

// ---------------------------------------------------------------- Arnoldi step: q_j, w = A q_j
// Column j of Q is the previous (unnormalised) vector scaled by 1/h_{j,j-1}
// (for j = 0: the cycle's start vector r scaled by 1/beta); w = A q_j uses the
// same rounded values of q_j as the stored column.  Rows past D are zero.
template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock) k_step(BatchArgs a, int j) {
    using V = c2_t<T>;
    using PK = pack_t<T>;
    using BS = Bstore<T, HB>;
    using BP = typename BS::pack;
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    if (!S->in_cycle) return;
    const long long D = P.D, ld = P.ld;
    const int N = S->N;
    count_bytes(a, DDG_K_STEP, (double)chunk_rows<T>() * ((j == 0 ? 16.0 : (double)sizeof(V)) + sizeof(T) + sizeof(V) +
                                                     BS::ebytes));
    const double inv = 1.0 / S->hnorm;
    const long long p0 = (long long)chunk * kBlock + threadIdx.x;
    const long long e0 = p0 * VEC;
    BP* __restrict__ q = reinterpret_cast<BP*>(static_cast<char*>(P.M) + (long long)(N + j) * ld * BS::ebytes);
    PK* __restrict__ w = reinterpret_cast<PK*>(P.w[j & 1]);
    const T* eps = reinterpret_cast<const T*>(P.eps_lo);
    const V* coef = reinterpret_cast<const V*>(P.coef_lo);
    const T kh2 = (T)P.kh2;
    // right preconditioner: w = A M^-1 q (q itself is stored unscaled)
    const V* __restrict__ dinv = reinterpret_cast<const V*>(P.dinv);
    V qv[VEC], wv[VEC];
    if (j == 0) {
        const double2* __restrict__ src = P.r;
        // the stencil sees q_0 as it is stored
        auto ld_ = [&](long long idx) { return BS::round(from_d2<V>(cscale(src[idx], inv))); };
        auto ls_ = [&](long long idx) { return dinv ? cmul(ld_(idx), dinv[idx]) : ld_(idx); };
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            const long long e = e0 + i;
            if (e < D) {
                qv[i] = ld_(e);
                wv[i] = stencil(e, P.nx, P.ny, coef, kh2 * eps[e], ls_);
            } else {
                qv[i] = mk((T)0, (T)0);
                wv[i] = mk((T)0, (T)0);
            }
        }
    } else {
        const V* __restrict__ src = reinterpret_cast<const V*>(P.w[(j - 1) & 1]);
        const T tinv = (T)inv;
        auto ld_ = [&](long long idx) { return BS::round(cscale(src[idx], tinv)); };
        auto ls_ = [&](long long idx) { return dinv ? cmul(ld_(idx), dinv[idx]) : ld_(idx); };
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            const long long e = e0 + i;
            if (e < D) {
                qv[i] = ld_(e);
                wv[i] = stencil(e, P.nx, P.ny, coef, kh2 * eps[e], ls_);
            } else {
                qv[i] = mk((T)0, (T)0);
                wv[i] = mk((T)0, (T)0);
            }
        }
    }
    q[p0] = BS::store(qv);
    w[p0] = mkpack(wv);
}

// ---------------------------------------------------------------- Gram-Schmidt projections
// h[k] = sum_e conj(M[k ld + e]) w[e] for the columns k < K = N + j + 1 of one
// solve (mode 0: pass 1, also ||w||^2 -> anorm; mode 1: pass 2).  Columns are
// read in batches of 8 (8 independent 16-byte loads per thread in flight).
template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock) k_dots_w(BatchArgs a, int j, int mode) {
    using V = c2_t<T>;
    using PK = pack_t<T>;
    using BS = Bstore<T, HB>;
    using BP = typename BS::pack;
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    if (!S->in_cycle) return;
    const int N = S->N;
    const int K = N + j + 1;
    count_bytes(a, DDG_K_DOTS, (double)chunk_rows<T>() * ((double)K * BS::ebytes + sizeof(V)));
    const long long ldp = P.ld / VEC;
    const long long p0 = (long long)chunk * kBlock + threadIdx.x;
    const BP* __restrict__ Mp = reinterpret_cast<const BP*>(P.M);
    V v[VEC];
    unpack(reinterpret_cast<const PK*>(P.w[j & 1])[p0], v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int vidx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    __shared__ V red[kWarps][64];
    __shared__ T smt[kWarps];
    // partial sums stay in the Krylov precision (one conversion per coefficient at the end)
    V* part = reinterpret_cast<V*>(P.part) + (long long)chunk * a.KP;
    for (int k0 = 0; k0 < K; k0 += 64) {
        const int kt = min(64, K - k0);
        for (int kk = 0; kk < kt; kk += 8) {
            const int nv = min(8, kt - kk);
            const BP* col = Mp + (long long)(k0 + kk) * ldp + p0;
            BP m[8];
            if (nv == 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) m[u] = col[(long long)u * ldp];
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) m[u] = (u < nv) ? col[(long long)u * ldp] : BP{};
            }
            V acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                V mv[VEC];
                BS::load(m[u], mv);
                acc[u] = mk((T)0, (T)0);
#pragma unroll
                for (int i = 0; i < VEC; ++i) cfmac(acc[u], mv[i], v[i]);
            }
            V r = reduce8(acc, lane);
            if ((lane & 3) == 0 && vidx < nv) red[wid][kk + vidx] = r;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < kt; t += kBlock) {
            V sum = mk((T)0, (T)0);
#pragma unroll
            for (int w = 0; w < kWarps; ++w) sum = cadd(sum, red[w][t]);
            part[k0 + t] = sum;
        }
        __syncthreads();
    }
    if (mode == 0) {
        T nn = (T)0;
#pragma unroll
        for (int i = 0; i < VEC; ++i) nn += v[i].x * v[i].x + v[i].y * v[i].y;
        nn = block_sum_all(nn, smt);
        if (threadIdx.x == 0) part[K] = mk(nn, (T)0);
    }
    if (!arrive_last(P.ticket, P.nchunks)) return;
    const int Ktot = K + (mode == 0 ? 1 : 0);
    const V* pall = reinterpret_cast<const V*>(P.part);
    for (int k = threadIdx.x; k < Ktot; k += kBlock) {
        V sv_ = mk((T)0, (T)0);
        for (int c = 0; c < P.nchunks; ++c) sv_ = cadd(sv_, __ldcg(pall + (long long)c * a.KP + k));
        const double2 sum = to_d2(sv_);
        if (k < K) {
            P.hp[k] = sum;
            if (mode == 0) P.hsum[k] = sum;
            else P.hsum[k] = cadd(P.hsum[k], sum);
        } else {
            S->anorm = sqrt(sum.x);
        }
    }
}

// w -= [C Q_j] h (coefficients staged in shared memory).
//   mode 0: Arnoldi pass 1
//   mode 1: Arnoldi pass 2, then ||w||, Hessenberg column, Givens, stop test
template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock) k_update_w(BatchArgs a, int j, int mode) {
    using V = c2_t<T>;
    using PK = pack_t<T>;
    using BS = Bstore<T, HB>;
    using BP = typename BS::pack;
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    if (!S->in_cycle) return;
    const int N = S->N;
    const int K = N + j + 1;
    count_bytes(a, DDG_K_UPDATE, (double)chunk_rows<T>() * ((double)K * BS::ebytes + 2.0 * sizeof(V)));
    extern __shared__ __align__(16) unsigned char smraw[];
    V* hs = reinterpret_cast<V*>(smraw);
    for (int t = threadIdx.x; t < K; t += kBlock) hs[t] = from_d2<V>(P.hp[t]);
    __syncthreads();
    const long long ldp = P.ld / VEC;
    const long long p0 = (long long)chunk * kBlock + threadIdx.x;
    const BP* __restrict__ Mp = reinterpret_cast<const BP*>(P.M);
    PK* __restrict__ wp = reinterpret_cast<PK*>(P.w[j & 1]);
    V v[VEC];
    unpack(wp[p0], v);
    int k = 0;
    for (; k + 8 <= K; k += 8) {
        const BP* col = Mp + (long long)k * ldp + p0;
        BP m[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) m[u] = col[(long long)u * ldp];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            V mv[VEC];
            BS::load(m[u], mv);
            const V c = hs[k + u];
#pragma unroll
            for (int i = 0; i < VEC; ++i) cfms(v[i], mv[i], c);
        }
    }
    for (; k < K; ++k) {
        V mv[VEC];
        BS::load(Mp[(long long)k * ldp + p0], mv);
        const V c = hs[k];
#pragma unroll
        for (int i = 0; i < VEC; ++i) cfms(v[i], mv[i], c);
    }
    wp[p0] = mkpack(v);
    if (mode == 0) return;
    __shared__ T smt[kWarps];
    T acc = (T)0;
#pragma unroll
    for (int i = 0; i < VEC; ++i) acc += v[i].x * v[i].x + v[i].y * v[i].y;
    const T tot = block_sum_all(acc, smt);
    V* partv = reinterpret_cast<V*>(P.part);
    if (threadIdx.x == 0) partv[(long long)chunk * a.KP] = mk(tot, (T)0);
    if (!arrive_last(P.ticket, P.nchunks)) return;
    // column j of H (rows 0..j from hsum[N..N+j], row j+1 = ||w||), column j of
    // B = C^H A q_j (hsum[0..N)); Givens update of column j in shared memory.
    const int m = a.m, ldh = m + 1;
    // 16-byte arrays first, the m doubles last (keeps every double2 aligned for any m)
    double2* gcol = reinterpret_cast<double2*>(smraw);      // m + 2 entries
    double2* gsn = gcol + (m + 2);                          // m entries
    double2* gout = gsn + m;                                // m + 2 entries
    double* gcs = reinterpret_cast<double*>(gout + (m + 2)); // m entries
    for (int t = threadIdx.x; t <= j; t += kBlock) gcol[t] = P.hsum[N + t];
    for (int t = threadIdx.x; t < j; t += kBlock) {
        gcs[t] = P.cs[t];
        gsn[t] = P.sn[t];
    }
    for (int n = threadIdx.x; n < N; n += kBlock) P.B[(long long)j * a.nmax + n] = P.hsum[n];
    __shared__ double s_nrm;
    if (threadIdx.x == 0) {
        T n2 = (T)0;
        for (int c = 0; c < P.nchunks; ++c) n2 += __ldcg(reinterpret_cast<const V*>(P.part) + (long long)c * a.KP).x;
        s_nrm = sqrt((double)n2);
    }
    __syncthreads();
    const double nrm = s_nrm;
    if (threadIdx.x < 32) {
        const double est = givens_column_warp(gcol, gcs, gsn, j, nrm, gout, P.g, P.cs + j, P.sn + j);
        if (threadIdx.x != 0) goto cgs2_done;
        S->k = j + 1;
        S->iters += 1;
        S->hnorm = nrm;
        bool brk = !(nrm > 1e-14 * S->anorm);
        if (brk) S->breakdown = 1;
        if (brk || est <= S->target || S->iters >= a.maxit || j + 1 >= m) {
            S->in_cycle = 0;
            atomicSub(a.counts, 1);
        }
    }
cgs2_done:
    __syncthreads();
    for (int t = threadIdx.x; t <= j + 1; t += kBlock) P.Rg[(long long)j * ldh + t] = gout[t];
}

// ---------------------------------------------------------------- tensor-core projections (half basis)
// One half2 of the A operand of t = [C Q]^H z, s = Q^H u as a real GEMM over
// k = 2 row + (0: Re, 1: Im) of the basis columns: component c of a value v
// split into v_hi + v_lo (two halves, about 22 significant bits):
//   c = 0: (Re v_hi, Im v_hi)   -> Re(conj(q) v_hi)
//   c = 1: (Im v_hi, -Re v_hi)  -> Im(conj(q) v_hi)
//   c = 2, 3: the same for v_lo
__device__ __forceinline__ unsigned split_pair(float2 v, int c) {
    const __half hx = __float2half_rn(v.x), hy = __float2half_rn(v.y);
    const __half lx = __float2half_rn(v.x - __half2float(hx)), ly = __float2half_rn(v.y - __half2float(hy));
    __half2 r;
    switch (c) {
        case 0: r = __halves2half2(hx, hy); break;
        case 1: r = __halves2half2(hy, __hneg(hx)); break;
        case 2: r = __halves2half2(lx, ly); break;
        default: r = __halves2half2(ly, __hneg(lx)); break;
    }
    return *reinterpret_cast<const unsigned*>(&r);
}
__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr)
                 : "memory");
}
// D (16 x 8, FP32) += A (16 x 16, half, rows 8..15 zero) B (16 x 8, half)
__device__ __forceinline__ void mma16816(float& d0, float& d1, float& d2, float& d3, unsigned a0, unsigned a2,
                                         unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
        : "r"(a0), "r"(0u), "r"(a2), "r"(0u), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- column dot products of the DCGS2 reduction
// t += conj(m) z and s += conj(m) u over one thread's VEC elements of a column.
// Complex64: the two elements of a thread are paired in packed two-wide FP32
// FMAs (fma.rn.f32x2), with z and u pre-split into (x0, x1) / (y0, y1) pairs,
// then the pair halves added: 8 packed FMAs + 4 adds instead of 16 FMAs.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
template <typename T> struct DotPairs;
template <> struct DotPairs<float> {
    // each element m = (mr, mi) is used as it is stored, an aligned register
    // pair: (mr, mi) * (zr, zi) gives the terms of Re(conj(m) z) and
    // (mr, mi) * (zi, -zr) those of Im(conj(m) z)
    float2 z0, z1, zs0, zs1, u0, u1, us0, us1;
    __device__ __forceinline__ DotPairs(const float2 (&z)[2], const float2 (&u)[2])
        : z0(z[0]), z1(z[1]), zs0(make_float2(z[0].y, -z[0].x)), zs1(make_float2(z[1].y, -z[1].x)),
          u0(u[0]), u1(u[1]), us0(make_float2(u[0].y, -u[0].x)), us1(make_float2(u[1].y, -u[1].x)) {}
    __device__ __forceinline__ void dots(const float2 (&m)[2], float2& t, float2& s) const {
        const float2 zero = make_float2(0.f, 0.f);
        const float2 tr = fma2(m[1], z1, fma2(m[0], z0, zero));     // terms of Re(conj(m) z)
        const float2 ti = fma2(m[1], zs1, fma2(m[0], zs0, zero));   // terms of Im(conj(m) z)
        const float2 sr = fma2(m[1], u1, fma2(m[0], u0, zero));
        const float2 si = fma2(m[1], us1, fma2(m[0], us0, zero));
        t = make_float2(tr.x + tr.y, ti.x + ti.y);
        s = make_float2(sr.x + sr.y, si.x + si.y);
    }
};
template <> struct DotPairs<double> {
    double2 z0, u0;
    __device__ __forceinline__ DotPairs(const double2 (&z)[1], const double2 (&u)[1]) : z0(z[0]), u0(u[0]) {}
    __device__ __forceinline__ void dots(const double2 (&m)[1], double2& t, double2& s) const {
        t = make_double2(0.0, 0.0);
        s = make_double2(0.0, 0.0);
        cfmac(t, m[0], z0);
        cfmac(s, m[0], u0);
    }
};

// ---------------------------------------------------------------- delayed reorthogonalisation (DCGS2)
// Finishes Arnoldi column j = i-1 once k_dots2 has reduced s, alpha and beta
// (tv[N+i ..), tv[N+2i], tv[N+2i+2]):
//   H[0:i, j] = h1 + s,  H[i, j] = beta,  B[:, j] = h1_C   (h1: pass-1 coefficients of column j)
// then its Givens rotation, the residual estimate |g_{j+1}| and the stop test.
// With `next` (i < m; one CTA per solve launched in front of k_update2's sweep)
// warps 1.. meanwhile form h1 of column i, with A Q_i s = [C Q_{i+1}] Hs,
//   Hs = [B; H][:, 0:i] s,  h1 = (t - Hs) / beta  (rows < N+i),
//   h1_i = (gamma - s^H t_Q) / beta^2 - Hs_i / beta,
// into the other h1 buffer.  Nothing here feeds the sweep it runs beside.
// The BatchArgs fields dcgs2_finish_column reads, passed by value (a reference
// to the kernel parameter block would be copied to the stack).
struct FinishArgs {
    int m, KP, nmax, maxit;
    int* counts;
};
__device__ __forceinline__ FinishArgs finish_args(const BatchArgs& a) {
    return FinishArgs{a.m, a.KP, a.nmax, a.maxit, a.counts};
}

template <typename T>
__device__ __noinline__ void dcgs2_finish_column(FinishArgs a, SolveScal* S, const SolvePtrs& P, int i, bool next,
                                                 unsigned char* smraw) {
    using V = c2_t<T>;
    const int N = S->N;
    const int m = a.m, ldh = m + 1;
    const int j = i - 1;
    const double2* tv = P.tv;
    const double2* sv = tv + N + i;
    const double2* h1p = P.hsum + (size_t)(j & 1) * a.KP;   // h1 of column j
    double2* h1n = P.hsum + (size_t)(i & 1) * a.KP;         // h1 of column i
    // 16-byte arrays first, the m doubles last (keeps every double2 aligned for any m)
    double2* gcol = reinterpret_cast<double2*>(smraw);    // m + 2 entries
    double2* gsn = gcol + (m + 2);                        // m entries
    double2* gout = gsn + m;                              // m + 2 entries
    V* svl = reinterpret_cast<V*>(gout + (m + 2));        // s in the Krylov precision, m entries
    double* gcs = reinterpret_cast<double*>(svl + m);     // m entries (last: 8-byte items)
    V* Hl = reinterpret_cast<V*>(P.Hh);                       // Krylov-precision copy of H
    V* Bl = reinterpret_cast<V*>(P.Hh + (size_t)(m + 1) * m);  // and of B
    __shared__ double smf[kWarps];
    const double beta = tv[N + 2 * i + 2].x;
    for (int t = threadIdx.x; t < i; t += kBlock) {
        const double2 h = cadd(h1p[N + t], sv[t]);
        gcol[t] = h;
        Hl[(long long)j * ldh + t] = from_d2<V>(h);
        svl[t] = from_d2<V>(sv[t]);
    }
    if (threadIdx.x == 0) Hl[(long long)j * ldh + i] = mk((T)beta, (T)0);
    for (int n = threadIdx.x; n < N; n += kBlock) {
        Bl[(long long)j * a.nmax + n] = from_d2<V>(h1p[n]);
        P.B[(long long)j * a.nmax + n] = h1p[n];
    }
    for (int t = threadIdx.x; t < j; t += kBlock) {
        gcs[t] = P.cs[t];
        gsn[t] = P.sn[t];
    }
    double h2p = 0.0;
    for (int t = threadIdx.x; t < N + i; t += kBlock) h2p += cabs2(h1p[t]);
    const double h2 = block_sum_d(h2p, smf);   // synchronises the staging above
    __syncthreads();
    if (threadIdx.x < 32) {
        const double est = givens_column_warp(gcol, gcs, gsn, j, beta, gout, P.g, P.cs + j, P.sn + j);
        if (threadIdx.x == 0) {
            const double alpha = tv[N + 2 * i].x;
            const double anorm = sqrt(h2 + alpha);   // ||A q_{i-1}||
            S->k = i;
            S->iters += 1;
            S->hnorm = beta;
            S->anorm = anorm;
            const bool brk = !(beta > 1e-14 * anorm);
            if (brk) S->breakdown = 1;
            if (brk || est <= S->target || S->iters >= a.maxit || i >= m) {
                S->in_cycle = 0;
                atomicSub(a.counts, 1);
            }
        }
        __syncwarp();
        for (int t = threadIdx.x; t <= j + 1; t += 32) P.Rg[(long long)j * ldh + t] = gout[t];
        return;
    }
    if (!next) return;
    // Hs multiplies the reorthogonalisation coefficients s (of the order of the
    // working precision times ||u||), so it is formed in the Krylov precision T.
    const double ib = 1.0 / beta;
    const double2 gm = csub(tv[N + 2 * i + 1], tv[N + 2 * i + 3]);   // gamma - s^H t_Q
    for (int row = threadIdx.x - 32; row < N + i + 1; row += kBlock - 32) {
        // row-wise sum over columns l: loads of one column are contiguous over rows
        V hst = mk((T)0, (T)0);
        if (row < N) {
#pragma unroll 4
            for (int l = 0; l < i; ++l) cfma(hst, Bl[(long long)l * a.nmax + row], svl[l]);
        } else {
            const int qr = row - N;  // row of H; column l holds rows 0..l+1
#pragma unroll 4
            for (int l = max(0, qr - 1); l < i; ++l) cfma(hst, Hl[(long long)l * ldh + qr], svl[l]);
        }
        const double2 hs = to_d2(hst);
        h1n[row] = (row < N + i) ? cscale(csub(tv[row], hs), ib) : csub(cscale(gm, ib * ib), cscale(hs, ib));
    }
}


// Iteration i >= 1 holds u = u_i (one Gram-Schmidt pass applied, not yet
// normalised) and z = A u.  One reduction gives
//   t = [C Q_i]^H z,  s = Q_i^H u,  alpha = u^H u,  gamma = u^H z
// (at i = m only s and alpha).  The last CTA of a solve then forms
// beta = sqrt(alpha - |s|^2) (Pythagoras: q_i = (u - Q_i s) / beta) and the
// coefficients of the next sweep u_{i+1} = z / beta - [C Q_{i+1}] c without
// touching w_i = A q_i: with A q_i = (z - A Q_i s) / beta and
// A Q_i s = [C Q_{i+1}] Hs, the first-pass coefficients are
//   h1 = (t - Hs) / beta (rows < N+i),  h1_i = (gamma - s^H t_Q) / beta^2 - Hs_i / beta,
// so c = Hs / beta + h1 = t / beta and c_i = (gamma - s^H t_Q) / beta^2.
// Column i-1 (H = h1 + s, its Givens rotation, the stop test) and h1 itself are
// finished by dcgs2_finish_column.
//
// The columns stream through shared memory: a ring of stages of 16 KB, filled
// by bulk copies and completed on one mbarrier per stage.  The stages requested
// before the prologue are issued by warp 0, one column per lane (the first
// copies start sooner); in the stage loop thread 0 requests one stage,
// stages - 1 ahead (a warp-wide request there costs registers the loop needs).  A column chunk is kBlock packs of
// one thread's elements: 4 KB in the arithmetic type (4 columns a stage), 2 KB
// in half (8 columns a stage, so that the per-stage barrier and wait are paid
// per 16 KB either way).  The copies in flight per CTA set how close a launch
// comes to the HBM bandwidth: 3 stages (48 KB) at 4 CTAs per SM in the
// arithmetic type, 4 stages (64 KB) at 3 CTAs per SM in half.
constexpr int kRingBytes = 48 * 1024;
template <typename T, bool HB> struct Ring {
    static constexpr int col_bytes = kBlock * (int)sizeof(typename Bstore<T, HB>::pack);
    static constexpr int cols = 16 * 1024 / col_bytes;
    static constexpr int stages = HB ? 4 : kRingBytes / (cols * col_bytes);
    // half basis: columns 16 bytes apart beyond their length, so that the 8 rows
    // of one ldmatrix phase (one per column) fall in different banks
    static constexpr int col_stride = col_bytes + (HB ? 16 : 0);
    static constexpr int stage_bytes = cols * col_stride;
    static constexpr int ring_bytes = stages * stage_bytes;
};
static_assert(Ring<float, false>::cols == 4 && Ring<double, false>::cols == 4 && Ring<float, true>::cols == 8 &&
                  Ring<float, true>::stages == 4 && Ring<float, false>::stages == 3,
              "ring geometry");

template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock, HB ? 3 : 4) k_dots2(BatchArgs a, int i_arg) {
    using V = c2_t<T>;
    using PK = pack_t<T>;
    using BS = Bstore<T, HB>;
    using BP = typename BS::pack;
    constexpr int VEC = vec_of<T>();
    constexpr int kRing = Ring<T, HB>::stages;
    constexpr int kColBytes = Ring<T, HB>::col_bytes;
    constexpr int kRingCols = Ring<T, HB>::cols;      // columns per stage (a multiple of 4)
    constexpr int kBatchesPer32 = 32 / kRingCols;     // stages between cross-warp sums
    constexpr int kColStride = Ring<T, HB>::col_stride;
    constexpr int kStageBytes = Ring<T, HB>::stage_bytes;
    SOLVE_PROLOGUE();
    const int i = i_arg > 0 ? i_arg : *a.step - i_arg;   // graph-driven loop: device step + offset
    // in_cycle only ever drops to 0 in the preceding launch, so a 0 read before
    // the dependency wait is final and a 1 is checked again after it.  Block 0
    // always waits, so that this grid never completes before the preceding one
    // (later launches rely on that order).
    if (i > a.m || !S->in_cycle) {       // past the restart length (unrolled graph body), or stopped
        if (blockIdx.x == 0) pdl_wait();
        return;
    }
    const int N = S->N;
    const bool hz = i < a.m;           // z exists (no matvec at the last column)
    const int K = N + i;               // columns [C, q_0 .. q_{i-1}]
    const int Ktot = N + 2 * i + 2;    // [t | s | alpha | gamma]
    const long long p0 = (long long)chunk * kBlock + threadIdx.x;
    extern __shared__ __align__(128) unsigned char smraw2[];
    __shared__ __align__(8) unsigned long long full[kRing];
    const int kstart = hz ? 0 : N;     // at i = m the C columns are not needed
    const int nbat = (K - kstart + kRingCols - 1) / kRingCols;
    // this chunk's rows of column kstart, and the distance between columns
    const char* colbase = reinterpret_cast<const char*>(P.M) +
                          ((long long)kstart * P.ld + (long long)chunk * chunk_rows<T>()) * (long long)BS::ebytes;
    const long long colstride = P.ld * (long long)BS::ebytes;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // warp 0: batch b into stage b % kRing; lane 0 arms the stage's barrier,
    // lanes 0..nv-1 copy one column each
    auto issue = [&](int b) {
        const int k = b * kRingCols;
        const int nv = min(kRingCols, K - kstart - k);
        unsigned long long* bar = &full[b % kRing];
        unsigned char* dst = smraw2 + (b % kRing) * kStageBytes;
        if (lane == 0) mbar_expect_tx(bar, (unsigned)(nv * kColBytes));
        __syncwarp();
        if (lane < nv) bulk_g2s(dst + lane * kColStride, colbase + (k + lane) * colstride, kColBytes, bar);
    };
    auto issue_one = [&](int b) {      // thread 0 alone: batch b into stage b % kRing
        const int k = b * kRingCols;
        const int nv = min(kRingCols, K - kstart - k);
        unsigned long long* bar = &full[b % kRing];
        unsigned char* dst = smraw2 + (b % kRing) * kStageBytes;
        mbar_expect_tx(bar, (unsigned)(nv * kColBytes));
        for (int w = 0; w < nv; ++w) bulk_g2s(dst + w * kColStride, colbase + (k + w) * colstride, kColBytes, bar);
    };
    // All kRing stages are requested before the prologue (each later stage once
    // its slot has been read); those holding only columns older than q_{i-1}
    // (the previous launch wrote q_{i-1} and u) before the dependency wait.
    const int npre = min(kRing, nbat);   // every stage is in flight before the prologue's own loads
    int early = 0;
    while (early < npre && kstart + (early + 1) * kRingCols <= K - 1) ++early;
    if (wid == 0) {
        if (lane == 0) {
            for (int q = 0; q < kRing; ++q) mbar_init(&full[q], 1);
            mbar_init_fence();
        }
        __syncwarp();
        for (int b = 0; b < early; ++b) issue(b);
    }
    pdl_wait();
    if (!S->in_cycle) {
        // stopped by the preceding launch: let the early copies land, then leave
        if (threadIdx.x == 0)
            for (int b = 0; b < early; ++b)
                if (!mbar_wait(&full[b], 0u, a.wait_ns)) {
                    atomicExch(a.counts + 4, 1);
                    mbar_wait(&full[b], 0u);   // one more wait, at the default bound, before leaving
                }
        return;
    }
    // columns, u, and z = A u (written; reads eps) when there is a next step
    count_bytes(a, DDG_K_DOTS, (double)chunk_rows<T>() * ((double)(hz ? K : i) * BS::ebytes + 2.0 * sizeof(V) +
                                                         (hz ? (double)sizeof(T) : 0.0)));
    if (wid == 0)
        for (int b = early; b < npre; ++b) issue(b);
    V u[VEC], z[VEC];
    unpack(reinterpret_cast<const PK*>(P.w[0])[p0], u);
    if (hz) {
        // z = A u on this chunk's rows (the ring fills meanwhile); the stencil's
        // neighbours of u come from other chunks through L2
        const V* __restrict__ uu = reinterpret_cast<const V*>(P.w[0]);
        const T* eps = reinterpret_cast<const T*>(P.eps_lo);
        const V* coef = reinterpret_cast<const V*>(P.coef_lo);
        const T kh2 = (T)P.kh2;
        const long long D = P.D;
        auto sweep = [&](const auto& ld_) {
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const long long e = p0 * VEC + q;
                z[q] = e < D ? stencil(e, P.nx, P.ny, coef, kh2 * eps[e], ld_) : mk((T)0, (T)0);
            }
        };
        // right preconditioner: z = A M^-1 u (branch taken once, outside the
        // loads, so the plain stencil keeps its load batching)
        const V* __restrict__ dinv = reinterpret_cast<const V*>(P.dinv);
        if (dinv)
            sweep([&](long long idx) { return cmul(uu[idx], dinv[idx]); });
        else
            sweep([&](long long idx) { return uu[idx]; });
        reinterpret_cast<PK*>(P.w[1])[p0] = mkpack(z);
    } else {
#pragma unroll
        for (int q = 0; q < VEC; ++q) z[q] = mk((T)0, (T)0);
    }
    __shared__ T smt[kWarps];
    // this thread's terms of alpha = u^H u and gamma = u^H z, formed now so that
    // u and z need not stay live through the stage loop
    T al_p = (T)0;
    V gg_p = mk((T)0, (T)0);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
        al_p += u[q].x * u[q].x + u[q].y * u[q].y;
        cfmac(gg_p, u[q], z[q]);
    }
    // partial sums stay in the Krylov precision until the last CTA
    V* part = reinterpret_cast<V*>(P.part) + (long long)chunk * a.KP;
    bool ok = true;
    int stop = nbat;     // stages consumed before a wait gave up (nbat: all)
    if constexpr (HB) {
        // Half basis: the projections as real GEMMs on the tensor cores (mma.sync
        // m16n8k16, half in, FP32 accumulate).  A (16 x 16 per k step): rows
        // 0..7 = [Re, Im] x [hi, lo] x [z, u] of this warp's 64 rows (see
        // split_pair), rows 8..15 zero; B (16 x 8): one k step of the stage's 8
        // columns, read by ldmatrix (a column's interleaved Re/Im halves are its
        // k order); D (8 x 8 used) per warp and stage, summed across warps every
        // 32 columns.
        static_assert(VEC == 2 && kRingCols == 8 && chunk_rows<T>() == 64 * kWarps, "tensor-core tile shape");
        // split components 0 (hi) and 2 (lo) of z and u per row, once, by the
        // thread that holds the row; components 1 and 3 are their (Im, -Re) swaps
        // (zsplit shares its space with redm: the fragments are read before the
        // first barrier of the stage loop, redm is written after it)
        __shared__ __align__(16) float redm[kWarps][32][8];
        __shared__ float comb[32][8];
        static_assert(sizeof(redm) == 4 * kBlock * VEC * sizeof(unsigned), "zsplit fits redm");
        auto zsplit = reinterpret_cast<unsigned (*)[kBlock * VEC]>(&redm[0][0][0]);   // [z hi, z lo, u hi, u lo]
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            const int r = threadIdx.x * VEC + q;
            zsplit[0][r] = split_pair(z[q], 0);
            zsplit[1][r] = split_pair(z[q], 2);
            zsplit[2][r] = split_pair(u[q], 0);
            zsplit[3][r] = split_pair(u[q], 2);
        }
        __syncthreads();
        const int gq = lane >> 2, tg = lane & 3;
        // row gq of A: vector gq / 4 (z, u), part (gq / 2) & 1 (hi, lo), Re or Im row gq & 1
        const unsigned* src = zsplit[2 * (gq >> 2) + ((gq >> 1) & 1)];
        const bool swap = gq & 1;
        unsigned afr[8][2];
#pragma unroll
        for (int ks = 0; ks < 8; ++ks)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned w = src[wid * 64 + ks * 8 + tg + 4 * h];
                // (Re, Im) -> (Im, -Re): swap the halves, flip the sign of the upper one
                afr[ks][h] = swap ? (((w >> 16) | (w << 16)) ^ 0x80000000u) : w;
            }
        for (int b = 0; b < nbat; ++b) {
            const int kk = (b % kBatchesPer32) * kRingCols;
            const int nv = min(kRingCols, K - kstart - b * kRingCols);
            // stage (b - 1) % kRing has been read by every warp; a wait that gave
            // up anywhere in the block stops the loop (before any new request)
            if (__syncthreads_or(!ok)) {
                stop = b;
                break;
            }
            if (threadIdx.x == 0 && b >= 1 && b + kRing - 1 < nbat) {
                fence_proxy_async_smem();
                issue_one(b + kRing - 1);
            }
            if (!mbar_wait(&full[b % kRing], (unsigned)(b / kRing) & 1u, a.wait_ns)) ok = false;
            const unsigned sbase = smem_u32(smraw2 + (b % kRing) * kStageBytes);
            float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll
            for (int kp = 0; kp < 4; ++kp) {
                // matrix lane / 8 of the x4 load: halves k = 128 wid + 32 kp + 8 (lane / 8) .. + 7
                // of column lane % 8
                unsigned b0, b1, b2, b3;
                ldsm_x4(sbase + (unsigned)((lane & 7) * kColStride + (wid * 128 + kp * 32 + (lane >> 3) * 8) * 2),
                        b0, b1, b2, b3);
                mma16816(d0, d1, d2, d3, afr[2 * kp][0], afr[2 * kp][1], b0, b1);
                mma16816(d0, d1, d2, d3, afr[2 * kp + 1][0], afr[2 * kp + 1][1], b2, b3);
            }
            redm[wid][kk + 2 * tg][gq] = d0;       // D[gq][column 2 tg], D[gq][column 2 tg + 1]
            redm[wid][kk + 2 * tg + 1][gq] = d1;
            if ((b + 1) % kBatchesPer32 == 0 || b == nbat - 1) {
                __syncthreads();
                const int k0 = kstart + (b / kBatchesPer32) * 32;
                const int kt = min(32, K - k0);
                if (threadIdx.x < kt * 8) {
                    const int cc = threadIdx.x >> 3, mm = threadIdx.x & 7;
                    float sum = 0.f;
#pragma unroll
                    for (int w = 0; w < kWarps; ++w) sum += redm[w][cc][mm];
                    comb[cc][mm] = sum;
                }
                __syncthreads();
                if (threadIdx.x < kt) {
                    const float* c8 = comb[threadIdx.x];
                    const int k = k0 + threadIdx.x;
                    part[k] = mk(c8[0] + c8[2], c8[1] + c8[3]);                              // t_k
                    if (k >= N) part[N + i + (k - N)] = mk(c8[4] + c8[6], c8[5] + c8[7]);    // s_l
                }
            }
            (void)nv;
        }
    } else {
    // The lanes hold their partials in reduce8_ordered's order: a lane with bit
    // 16 set forms [s | t] (z and u swapped), and lanes with bits 8 / 4 set read
    // the stage's four columns in the order w ^ 2 / w ^ 1.
    const bool b16 = lane & 16;
    const int cperm = ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    V zz[VEC], uu[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
        zz[q] = b16 ? u[q] : z[q];
        uu[q] = b16 ? z[q] : u[q];
    }
    const DotPairs<T> dp(zz, uu);
    const int vidx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    __shared__ V red_t[kWarps][32];
    __shared__ V red_s[kWarps][32];
    // a stage of kRingCols columns; each 4 of them share one 8-value butterfly
    // of their t- and s-partials; cross-warp sums every 32 columns
    for (int b = 0; b < nbat; ++b) {
        const int kk = (b % kBatchesPer32) * kRingCols;
        const int nv = min(kRingCols, K - kstart - b * kRingCols);
        // stage (b - 1) % kRing has been read by every warp; a wait that gave
        // up anywhere in the block stops the loop (before any new request)
        if (__syncthreads_or(!ok)) {
            stop = b;
            break;
        }
        if (threadIdx.x == 0 && b >= 1 && b + kRing - 1 < nbat) {
            fence_proxy_async_smem();
            issue_one(b + kRing - 1);
        }
        if (!mbar_wait(&full[b % kRing], (unsigned)(b / kRing) & 1u, a.wait_ns)) ok = false;
        const BP* stg = reinterpret_cast<const BP*>(smraw2 + (b % kRing) * (kRingCols * kColBytes));
        BP m[kRingCols];
        static_assert(kRingCols == 4, "one butterfly group per stage");
#pragma unroll
        for (int w = 0; w < kRingCols; ++w) {
            const int c = w ^ cperm;   // this lane's column for butterfly position w
            m[w] = (c < nv) ? stg[c * kBlock + threadIdx.x] : BP{};
        }
#pragma unroll
        for (int g = 0; g < kRingCols / 4; ++g) {
            V acc[8];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                V mv[VEC];
                BS::load(m[4 * g + w], mv);
                dp.dots(mv, acc[w], acc[w + 4]);
            }
            const V r = reduce8_ordered(acc);
            if ((lane & 3) == 0 && 4 * g + (vidx & 3) < nv) {
                if (vidx < 4) red_t[wid][kk + 4 * g + vidx] = r;
                else red_s[wid][kk + 4 * g + vidx - 4] = r;
            }
        }
        if ((b + 1) % kBatchesPer32 == 0 || b == nbat - 1) {
            __syncthreads();
            const int k0 = kstart + (b / kBatchesPer32) * 32;
            const int kt = min(32, K - k0);
            for (int t = threadIdx.x; t < kt; t += kBlock) {
                V st = mk((T)0, (T)0), ss = mk((T)0, (T)0);
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    st = cadd(st, red_t[w][t]);
                    ss = cadd(ss, red_s[w][t]);
                }
                const int k = k0 + t;
                part[k] = st;                              // t_k
                if (k >= N) part[N + i + (k - N)] = ss;    // s_l, l = k - N
            }
        }
    }
    }
    if (__syncthreads_or(!ok) && threadIdx.x == 0) {
        // a copy did not arrive within the wait limit: report it, and give every
        // stage still in flight one more wait at the default bound (1 s), so that
        // no copy lands after this CTA has gone.  Stages [0, issued) were
        // requested; a slot is re-requested only after every thread has seen
        // its previous phase complete, so only the latest phase of each slot
        // can be outstanding.
        atomicExch(a.counts + 4, 1);
        const int issued = min(nbat, max(npre, stop + kRing - 1));
        for (int b = max(0, issued - kRing); b < issued; ++b) mbar_wait(&full[b % kRing], (unsigned)(b / kRing) & 1u);
    }
    {
        const T al = block_sum_all(al_p, smt);
        const T gr = block_sum_all(gg_p.x, smt);
        const T gi = block_sum_all(gg_p.y, smt);
        if (threadIdx.x == 0) {
            part[N + 2 * i] = mk(al, (T)0);
            part[N + 2 * i + 1] = mk(gr, gi);
        }
    }
    if (!arrive_last(P.ticket, P.nchunks)) return;
    // Last CTA of this solve: only what the next sweep needs stays here (the
    // sums over the chunks, beta and the coefficients c); the rest of column
    // i-1 (Givens rotation, stop test, Hs and h1 of column i) runs in
    // dcgs2_finish_column, in front of k_update2's sweep.
    double2* tv = P.tv;
    const V* pall = reinterpret_cast<const V*>(P.part);
    double2* tvs = reinterpret_cast<double2*>(smraw2);   // Ktot entries (the ring's space)
    const int nch = P.nchunks;
    for (int k = threadIdx.x; k < Ktot; k += kBlock) {
        // one coefficient per thread, chunks in order, 16 loads in flight
        V sum = mk((T)0, (T)0);
        if (hz || k >= N) {
            const V* pk = pall + k;
            int c = 0;
            for (; c + 16 <= nch; c += 16) {
                V v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = __ldcg(pk + (long long)(c + q) * a.KP);
#pragma unroll
                for (int q = 0; q < 16; ++q) sum = cadd(sum, v[q]);
            }
            for (; c < nch; ++c) sum = cadd(sum, __ldcg(pk + (long long)c * a.KP));
        }
        const double2 d = to_d2(sum);
        tvs[k] = d;
        tv[k] = d;
    }
    __syncthreads();
    // |s|^2 and s^H t_Q (block reductions)
    double s2p = 0.0, str = 0.0, sti = 0.0;
    for (int t = threadIdx.x; t < i; t += kBlock) {
        const double2 st_ = tvs[N + i + t];
        s2p += cabs2(st_);
        if (hz) {
            const double2 pr = cmulc(st_, tvs[N + t]);
            str += pr.x;
            sti += pr.y;
        }
    }
    __shared__ double sm[kWarps];
    __shared__ double s_beta;
    __shared__ double2 s_st;
    const double s2 = block_sum_d(s2p, sm);
    const double st_r = block_sum_d(str, sm);
    const double st_i = block_sum_d(sti, sm);
    if (threadIdx.x == 0) {
        const double alpha = tvs[N + 2 * i].x;
        const double beta = sqrt(fmax(alpha - s2, 0.0));   // Pythagoras: ||u - Q_i s||
        s_beta = beta;
        s_st = make_double2(st_r, st_i);
        tv[N + 2 * i + 2] = make_double2(beta, s2);
        tv[N + 2 * i + 3] = s_st;
    }
    __syncthreads();
    if (!hz) {
        // i = m: no next step, column m-1 is finished here
        dcgs2_finish_column<T>(finish_args(a), S, P, i, false, smraw2);
        return;
    }
    // coefficients of u_{i+1} = z / beta - [C Q_{i+1}] c:
    //   c = t / beta (rows < N+i),  c_i = (gamma - s^H t_Q) / beta^2
    const double ib = 1.0 / s_beta;
    for (int k = threadIdx.x; k < N + i; k += kBlock) P.hp[k] = cscale(tvs[k], ib);
    if (threadIdx.x == 0) P.hp[N + i] = cscale(csub(tvs[N + 2 * i + 1], s_st), ib * ib);
}

// One sweep over [C, Q_i]:  q_i = (u - Q_i s) / beta  (stored as column N+i)
// and u <- z / beta - [C, Q_i] c[0:N+i] - q_i c[N+i]  (in place).  The grid
// starts with one column-finishing block per solve (dcgs2_finish_column); a
// solve that it stops still completes this sweep, whose q_i and u are unused.
template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock, 6) k_update2(BatchArgs a, int i_arg) {
    using V = c2_t<T>;
    using PK = pack_t<T>;
    using BS = Bstore<T, HB>;
    using BP = typename BS::pack;
    constexpr int VEC = vec_of<T>();
    const int i = i_arg > 0 ? i_arg : *a.step - i_arg;   // graph-driven loop: device step + offset
    extern __shared__ __align__(16) unsigned char smraw[];
    if ((int)blockIdx.x < a.nsolves) {
        // blocks 0..nsolves-1: finish column i-1 of solve blockIdx.x (first
        // wave); they always wait, so that this grid never completes before
        // the preceding one
        pdl_wait();
        if (i >= a.m) return;             // no sweep after the last column
        SolveScal* S = a.S + blockIdx.x;
        if (!S->in_cycle) return;
        dcgs2_finish_column<T>(finish_args(a), S, a.P[blockIdx.x], i, true, smraw);
        return;
    }
    if (i >= a.m) return;
    const int bsw = blockIdx.x - a.nsolves;
    const int s = a.blk_solve[bsw];
    SolveScal* S = a.S + s;
    const SolvePtrs& P = a.P[s];
    const int chunk = bsw - P.chunk0;
    if (!S->in_cycle) return;
    const int N = S->N;
    const int K = N + i;
    const long long ldp = P.ld / VEC;
    const long long p0 = (long long)chunk * kBlock + threadIdx.x;
    const BP* __restrict__ Mp = reinterpret_cast<const BP*>(P.M);
    PK* __restrict__ up = reinterpret_cast<PK*>(P.w[0]);
    // u and the columns are not written by k_dots2: u is loaded and the first
    // 8 column chunks are pulled into L2 before the dependency wait
    V u[VEC];
    unpack(up[p0], u);
    if (threadIdx.x == 0)
        for (int w = 0; w < min(8, K); ++w)
            bulk_prefetch_l2(Mp + (long long)w * ldp + (long long)chunk * kBlock, Ring<T, HB>::col_bytes);
    pdl_wait();
    count_bytes(a, DDG_K_UPDATE, (double)chunk_rows<T>() * ((double)(K + 1) * BS::ebytes + 3.0 * sizeof(V)));
    V* cs = reinterpret_cast<V*>(smraw);      // c, N + i + 1
    V* ss = cs + (N + a.m + 1);               // s, i
    for (int t = threadIdx.x; t < K + 1; t += kBlock) cs[t] = from_d2<V>(P.hp[t]);
    for (int t = threadIdx.x; t < i; t += kBlock) ss[t] = from_d2<V>(P.tv[N + i + t]);
    __syncthreads();
    const T ib = (T)(1.0 / P.tv[N + 2 * i + 2].x);   // 1 / beta
    V nu[VEC];
    unpack(reinterpret_cast<const PK*>(P.w[1])[p0], nu);
#pragma unroll
    for (int q = 0; q < VEC; ++q) nu[q] = cscale(nu[q], ib);
    int k = 0;
    // C columns: only the new vector
    for (; k < N; ++k) {
        V mv[VEC];
        BS::load(Mp[(long long)k * ldp + p0], mv);
        const V c = cs[k];
#pragma unroll
        for (int q = 0; q < VEC; ++q) cfms(nu[q], mv[q], c);
    }
    // Q columns, 8 at a time: both vectors
    for (; k + 8 <= K; k += 8) {
        const BP* col = Mp + (long long)k * ldp + p0;
        BP m[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) m[w] = col[(long long)w * ldp];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            V mv[VEC];
            BS::load(m[w], mv);
            const V c = cs[k + w], sl = ss[k + w - N];
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                cfms(nu[q], mv[q], c);
                cfms(u[q], mv[q], sl);
            }
        }
    }
    for (; k < K; ++k) {
        V mv[VEC];
        BS::load(Mp[(long long)k * ldp + p0], mv);
        const V c = cs[k], sl = ss[k - N];
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            cfms(nu[q], mv[q], c);
            cfms(u[q], mv[q], sl);
        }
    }
    V qi[VEC];
    const V cl = cs[K];
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
        qi[q] = BS::round(cscale(u[q], ib));   // q_i as stored: later steps read it back
        cfms(nu[q], qi[q], cl);
    }
    reinterpret_cast<BP*>(static_cast<char*>(P.M) + (long long)K * P.ld * BS::ebytes)[p0] = BS::store(qi);
    up[p0] = mkpack(nu);
}

// ---------------------------------------------------------------- cycle end
// One CTA per solve: y = R_H^-1 g (back substitution, FP64), x_V = c_r - B y,
// z = R^-1 x_V; writes coefy = [z | y].
__global__ void __launch_bounds__(128) k_backsub(BatchArgs a) {
    const int s = blockIdx.x;
    SolveScal* S = a.S + s;
    if (!S->pending) return;
    const SolvePtrs& P = a.P[s];
    const int k = S->k, N = S->N, ldh = a.m + 1;
    extern __shared__ __align__(16) double2 sh[];
    double2* gg = sh;            // k
    double2* y = sh + a.m;       // k
    double2* rd = sh + 2 * a.m;  // k: 1 / R_ii
    double2* xa = sh + 3 * a.m;  // N
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        gg[i] = P.g[i];
        rd[i] = cdiv(make_double2(1.0, 0.0), P.Rg[(long long)i * ldh + i]);
    }
    __syncthreads();
    // column-oriented back substitution; every step's update is spread over
    // the whole block (FP64 issue is the limit, so all four SM quadrants work)
    for (int i = k - 1; i >= 0; --i) {
        const double2 yi = cmul(gg[i], rd[i]);
        const double2* col = P.Rg + (long long)i * ldh;
        __syncthreads();             // every thread has read gg[i]
        for (int l = threadIdx.x; l < i; l += blockDim.x) gg[l] = csub(gg[l], cmul(col[l], yi));
        if (threadIdx.x == 0) y[i] = yi;
        __syncthreads();
    }
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double2 t = P.cr[n];
        for (int i = 0; i < k; ++i) t = csub(t, cmul(P.B[(long long)i * a.nmax + n], y[i]));
        xa[n] = t;
    }
    __syncthreads();
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double2 t = make_double2(0.0, 0.0);
        for (int l = 0; l < N; ++l) t = cadd(t, cmul(P.Rinv[(long long)l * N + n], xa[l]));
        P.coefy[n] = t;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) P.coefy[N + i] = y[i];
}

// x += V z + Q y (V, Q in the Krylov precision): the correction is summed in
// blocks of 8 columns in that precision, the block sums and x in FP64.
template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock) k_update_x(BatchArgs a) {
    using V = c2_t<T>;
    using PK = pack_t<T>;
    using BS = Bstore<T, HB>;
    using BP = typename BS::pack;
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    if (!S->pending) return;
    const long long D = P.D, ldp = P.ld / VEC;
    const int N = S->N, k = S->k, nc = N + k;
    count_bytes(a, DDG_K_CYCLE_END, (double)chunk_rows<T>() * ((double)N * sizeof(V) + (double)k * BS::ebytes + 32.0));
    // coefficients [z; y] in the Krylov precision (the correction only has to
    // meet the inner tolerance; x itself is updated in FP64)
    extern __shared__ __align__(16) unsigned char smraw[];
    V* cyl = reinterpret_cast<V*>(smraw);
    for (int c = threadIdx.x; c < nc; c += kBlock) cyl[c] = from_d2<V>(P.coefy[c]);
    __syncthreads();
    const long long p0 = (long long)chunk * kBlock + threadIdx.x;
    // V (the predicted vectors, in the arithmetic type) then Q (basis storage):
    // blocks of 8 columns summed in T, the block sums in FP64
    const PK* __restrict__ Vp = reinterpret_cast<const PK*>(P.V);
    const BP* __restrict__ Qp = reinterpret_cast<const BP*>(P.M) + (long long)N * ldp;
    double2 acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = make_double2(0.0, 0.0);
    auto block = [&](const auto* base, int ncols, int coff) {
        for (int c0 = 0; c0 < ncols; c0 += 8) {
            const int nb = min(8, ncols - c0);
            V mv[8][VEC];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                if (w < nb) {
                    const auto pk = base[(long long)(c0 + w) * ldp + p0];
                    if constexpr (sizeof(pk) == sizeof(PK)) unpack(pk, mv[w]);
                    else BS::load(pk, mv[w]);
                } else {
#pragma unroll
                    for (int q = 0; q < VEC; ++q) mv[w][q] = mk((T)0, (T)0);
                }
            }
            V part[VEC];
#pragma unroll
            for (int q = 0; q < VEC; ++q) part[q] = mk((T)0, (T)0);
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                if (w >= nb) break;
                const V cw = cyl[coff + c0 + w];
#pragma unroll
                for (int q = 0; q < VEC; ++q) cfma(part[q], mv[w][q], cw);
            }
#pragma unroll
            for (int q = 0; q < VEC; ++q) acc[q] = cadd(acc[q], to_d2(part[q]));
        }
    };
    if (N > 0) block(Vp, N, 0);
    if (P.dinv) {
        // right preconditioner: x += V z + M^-1 Q y
        double2 accv[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            accv[q] = acc[q];
            acc[q] = make_double2(0.0, 0.0);
        }
        block(Qp, k, N);
        const V* dinv = reinterpret_cast<const V*>(P.dinv);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = cadd(accv[q], cmul(acc[q], to_d2(dinv[p0 * VEC + q])));
    } else {
        block(Qp, k, N);
    }
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
        const long long e = p0 * VEC + q;
        if (e < D) P.x[e] = cadd(P.x[e], acc[q]);
    }
}

// b = 0: the solution is x = 0 whatever x0 was.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_finalize(BatchArgs a) {
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    if (S->nb != 0.0) return;
    const long long e0 = (long long)chunk * chunk_rows<T>() + (long long)threadIdx.x * VEC;
#pragma unroll
    for (int q = 0; q < VEC; ++q)
        if (e0 + q < P.D) P.x[e0 + q] = make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------- augmentation set-up
// W = A U (FP64, zero past D), column by column.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_aug_av(BatchArgs a) {
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    const int N = S->N;
    const long long D = P.D, ld = P.ld;
    const long long e0 = (long long)chunk * chunk_rows<T>() + (long long)threadIdx.x * VEC;
    for (int n = 0; n < N; ++n) {
        const double2* __restrict__ u = P.U + (long long)n * D;
        auto ldu = [&](long long idx) { return u[idx]; };
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            const long long e = e0 + q;
            P.W[(long long)n * ld + e] =
                e < D ? stencil(e, P.nx, P.ny, P.coef_d, P.kh2 * P.eps_d[e], ldu) : make_double2(0.0, 0.0);
        }
    }
}

// Gram matrix G = W^H W (FP64) and, in the last CTA, its Cholesky factor
// G = R^H R and R^-1 (upper triangular).  pass 0 writes R1^-1 to Rtmp; pass 1
// writes R2^-1 to Rinv.  A non-positive or relatively tiny pivot marks the
// solve as rank deficient: it then runs as plain GMRES (N = 0, fallback = 1).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_aug_gram(BatchArgs a, int pass) {
    SOLVE_PROLOGUE();
    const int N = S->N;
    if (N == 0) return;
    const long long ld = P.ld;
    // The chunk's rows of W pass through shared memory in tiles of kTR rows;
    // each thread owns up to kSlots pairs (p <= q) of the Gram matrix and
    // accumulates them over the whole chunk (the FP64 products are the cost:
    // N(N+1)/2 complex MACs per row, with no block barrier per pair).
    constexpr int kTR = 32;
    constexpr int kSlots = (kMaxAug * (kMaxAug + 1) / 2 + kBlock - 1) / kBlock;
    __shared__ double2 tile[kTR][kMaxAug + 1];
    const int npairs = N * (N + 1) / 2;
    int pp[kSlots], qq[kSlots];
    double2 acc[kSlots];
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
        acc[k] = make_double2(0.0, 0.0);
        int idx = threadIdx.x + k * kBlock, p = 0;
        if (idx < npairs)
            while (idx >= N - p) idx -= N - p++;   // pairs in row-major order of the upper triangle
        pp[k] = p;
        qq[k] = p + idx;                          // meaningful only when the pair exists
    }
    const long long r0 = (long long)chunk * chunk_rows<T>();
    for (int rt = 0; rt < (int)chunk_rows<T>(); rt += kTR) {
        for (int idx = threadIdx.x; idx < kTR * N; idx += kBlock) {
            const int n = idx / kTR, r = idx - n * kTR;   // consecutive threads: consecutive rows of a column
            tile[r][n] = P.W[(long long)n * ld + r0 + rt + r];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSlots; ++k)
            if (threadIdx.x + k * kBlock < npairs) {
                const int p = pp[k], q = qq[k];
#pragma unroll 8
                for (int r = 0; r < kTR; ++r) cfmac(acc[k], tile[r][p], tile[r][q]);
            }
        __syncthreads();
    }
    double2* part = P.part + (long long)chunk * a.KP;
#pragma unroll
    for (int k = 0; k < kSlots; ++k)
        if (threadIdx.x + k * kBlock < npairs) part[pp[k] * N + qq[k]] = acc[k];
    if (!arrive_last(P.ticket, P.nchunks)) return;
    double2* G = P.hp;  // N x N, column-major, upper triangle used
    for (int idx = threadIdx.x; idx < N * N; idx += kBlock) {
        int p = idx / N, q = idx % N;
        if (q < p) continue;
        double2 sum = make_double2(0.0, 0.0);
        for (int c = 0; c < P.nchunks; ++c) sum = cadd(sum, __ldcg(P.part + (long long)c * a.KP + idx));
        G[q * N + p] = sum;  // G(p, q), p <= q
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // Cholesky of the Hermitian G: G = R^H R with R upper triangular, in place
    // in the upper triangle of G (column-major: R(p,q) at G[q*N + p]).
    double dmax = 0.0;
    for (int p = 0; p < N; ++p) dmax = fmax(dmax, G[p * N + p].x);
    bool ok = dmax > 0.0;
    for (int p = 0; p < N && ok; ++p) {
        double d = G[p * N + p].x;
        for (int l = 0; l < p; ++l) d -= cabs2(G[p * N + l]);
        if (!(d > 1e-13 * dmax)) { ok = false; break; }
        double rpp = sqrt(d);
        G[p * N + p] = make_double2(rpp, 0.0);
        for (int q = p + 1; q < N; ++q) {
            double2 t = G[q * N + p];
            for (int l = 0; l < p; ++l) t = csub(t, cmulc(G[p * N + l], G[q * N + l]));
            G[q * N + p] = cscale(t, 1.0 / rpp);
        }
    }
    if (!ok) {
        S->N = 0;
        S->fallback = 1;
        return;
    }
    // inverse of the upper-triangular R (column-major), column by column
    double2* Ri = pass == 0 ? P.Rtmp : P.Rinv;
    for (int q = 0; q < N; ++q) {
        for (int p = N - 1; p >= 0; --p) {
            if (p > q) { Ri[q * N + p] = make_double2(0.0, 0.0); continue; }
            double2 t = make_double2(p == q ? 1.0 : 0.0, 0.0);
            for (int l = p + 1; l <= q; ++l) t = csub(t, cmul(G[l * N + p], Ri[q * N + l]));
            Ri[q * N + p] = cdiv(t, G[p * N + p]);
        }
    }
}

// R^-1 of A V = C R with R = R2 R1: R^-1 = R1^-1 R2^-1 (one thread per solve).
__global__ void k_aug_rinv(BatchArgs a, int n) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int N = a.S[s].N;
    const SolvePtrs& P = a.P[s];
    double2* G = P.hp;
    for (int q = 0; q < N; ++q)
        for (int p = 0; p < N; ++p) {
            double2 t = make_double2(0.0, 0.0);
            for (int l = 0; l < N; ++l) t = cadd(t, cmul(P.Rtmp[l * N + p], P.Rinv[q * N + l]));
            G[q * N + p] = t;
        }
    for (int idx = 0; idx < N * N; ++idx) P.Rinv[idx] = G[idx];
}

// W <- W R_pass^-1 row by row (in place, columns from the last down).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_aug_tri(BatchArgs a, int pass) {
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    const int N = S->N;
    if (N == 0) return;
    const long long ld = P.ld;
    const double2* Ri = pass == 0 ? P.Rtmp : P.Rinv;
    const long long e0 = (long long)chunk * chunk_rows<T>() + (long long)threadIdx.x * VEC;
#pragma unroll
    for (int t = 0; t < VEC; ++t) {
        const long long e = e0 + t;
        for (int q = N - 1; q >= 0; --q) {
            double2 acc = make_double2(0.0, 0.0);
            for (int p = 0; p <= q; ++p) cfma(acc, P.W[(long long)p * ld + e], Ri[q * N + p]);
            P.W[(long long)q * ld + e] = acc;
        }
    }
}

// C in the basis storage, V in the Krylov precision (leading dimension ld, zero past D).
template <typename T, bool HB>
__global__ void __launch_bounds__(kBlock) k_aug_store(BatchArgs a) {
    using V = c2_t<T>;
    using BS = Bstore<T, HB>;
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    const int N = S->N;
    const long long D = P.D, ld = P.ld;
    V* Vl = reinterpret_cast<V*>(P.V);
    const long long e0 = (long long)chunk * chunk_rows<T>() + (long long)threadIdx.x * VEC;
    for (int n = 0; n < N; ++n)
#pragma unroll
        for (int t = 0; t < VEC; ++t) {
            const long long e = e0 + t;
            BS::set(P.M, (long long)n * ld + e, from_d2<V>(P.W[(long long)n * ld + e]));
            Vl[(long long)n * ld + e] = e < D ? from_d2<V>(P.U[(long long)n * D + e]) : mk((T)0, (T)0);
        }
}

// M^-1 = 1 / diag(A) (the stencil's centre coefficient), in the Krylov precision;
// zero past D.  The data-free baseline of the augmented method: Jacobi.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_dinv(BatchArgs a) {
    using V = c2_t<T>;
    constexpr int VEC = vec_of<T>();
    SOLVE_PROLOGUE();
    (void)S;
    const long long D = P.D;
    const int nx = P.nx, ny = P.ny;
    V* dv = reinterpret_cast<V*>(const_cast<void*>(P.dinv));
    const long long e0 = (long long)chunk * chunk_rows<T>() + (long long)threadIdx.x * VEC;
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
        const long long e = e0 + q;
        V v = mk((T)0, (T)0);
        if (e < D) {
            const int j = (int)(e / nx), i = (int)(e - (long long)j * nx);
            const double2* c = P.coef_d;
            double2 d = cadd(cadd(c[i], c[nx + i]), cadd(c[2 * nx + j], c[2 * nx + ny + j]));
            d.x -= P.kh2 * P.eps_d[e];
            v = from_d2<V>(cdiv(make_double2(1.0, 0.0), d));
        }
        dv[e] = v;
    }
}

// ---------------------------------------------------------------- host driver
static size_t align_up(size_t v, size_t al = 256) { return (v + al - 1) / al * al; }

struct Carver {
    char* base;
    size_t off = 0;
    template <typename X> X* take(size_t count) {
        off = align_up(off);
        X* p = base ? reinterpret_cast<X*>(base + off) : nullptr;
        off += count * sizeof(X);
        return p;
    }
};

// Graph-driven solve: every restart cycle of the batch runs inside one CUDA
// graph launch, under device-side WHILE and IF nodes (no host round trip
// between cycles or steps).  The graph's small kernels:
//   k_cycle_begin  clears the per-cycle counts [0..3] (what the host loop's
//                  memset does);
//   k_cycle_gate   after the cycle-start residual: continue while some solve
//                  is active and no bounded wait gave up, at most maxit + 2
//                  cycles (the host loop's bound); run the Arnoldi steps only
//                  when some solve is inside a cycle;
//   k_inner_begin  step = 1 and the step loop's first condition;
//   k_advance      advances the step by the body's `unroll` steps and keeps the
//                  step loop running while some solve is inside its Arnoldi
//                  cycle and the restart length is not exhausted (k_dots2 at
//                  step m finishes the last column; launches for steps past m
//                  return at once).
// Counts [6..9] record cycles begun, step-loop bodies, cycles with Arnoldi
// steps and cycles that ran to their end, for the launch accounting; every
// loop is bounded by a counter, never by convergence alone.
constexpr int kGraphUnroll = 8;
constexpr int kCounts = 12;          // ints of BatchArgs::counts
__global__ void k_cycle_begin(BatchArgs a) {
    a.counts[0] = 0;
    a.counts[1] = 0;
    a.counts[2] = 0;
    a.counts[3] = 0;
}
__global__ void k_cycle_gate(BatchArgs a, cudaGraphConditionalHandle outer, cudaGraphConditionalHandle arnoldi,
                             cudaGraphConditionalHandle finish) {
    const int c = a.counts[6]++;
    const bool go = a.counts[1] != 0 && a.counts[4] == 0;
    const bool ar = go && a.counts[0] > 0;
    a.counts[8] += ar ? 1 : 0;
    a.counts[9] += go ? 1 : 0;
    cudaGraphSetConditional(arnoldi, ar ? 1u : 0u);
    cudaGraphSetConditional(finish, go ? 1u : 0u);
    cudaGraphSetConditional(outer, (go && c + 1 <= a.maxit + 1) ? 1u : 0u);
}
__global__ void k_inner_begin(BatchArgs a, cudaGraphConditionalHandle loop) {
    *a.step = 1;
    cudaGraphSetConditional(loop, (a.m >= 1 && a.counts[0] > 0) ? 1u : 0u);
}
__global__ void k_advance(BatchArgs a, cudaGraphConditionalHandle loop, int unroll) {
    const int s = *a.step + unroll;
    *a.step = s;
    a.counts[7] += 1;
    cudaGraphSetConditional(loop, (s <= a.m && a.counts[0] > 0) ? 1u : 0u);
}

// Launch with programmatic stream serialisation: its blocks may start once the
// preceding kernel's blocks have exited, before that kernel's completion is
// signalled; they order themselves after it with pdl_wait() before touching
// what it writes (and prefetch what it does not).
template <typename... KArgs, typename... Args>
static void launch_overlapped(void (*kern)(KArgs...), unsigned grid, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, kern, args...);   // a failure is left for cudaGetLastError
}

// During a stream capture: the graph being captured into.
static cudaError_t capture_graph(cudaStream_t cs, cudaGraph_t* g) {
    cudaStreamCaptureStatus status;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &status, nullptr, g, nullptr, nullptr, nullptr);
    if (e == cudaSuccess && status != cudaStreamCaptureStatusActive) e = cudaErrorStreamCaptureInvalidated;
    return e;
}

// During a stream capture: appends a conditional node (IF or WHILE, one body
// graph) with handle `h` after the capture's current dependencies; later
// captured work depends on it.  `body` receives the node's body graph.
static cudaError_t append_conditional(cudaStream_t cs, cudaGraphConditionalHandle h,
                                      cudaGraphConditionalNodeType type, cudaGraph_t* body) {
    cudaStreamCaptureStatus status;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, &edges, &nd);
    if (e != cudaSuccess) return e;
    if (status != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, edges, nd, &cp);
    if (e != cudaSuccess) return e;
    *body = cp.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// The delayed scheme's whole batched solve (after the set-up) as one graph:
//   while (outer) {                                   // one restart cycle per body
//     k_cycle_begin; k_residual; [k_dots_r; k_update_r]; k_cycle_gate
//     if (arnoldi) { k_step(0); k_dots_w; k_update_w; k_inner_begin
//                    while (loop) { for u < 8: k_dots2(step + u); k_update2(step + u);  k_advance } }
//     if (finish)  { k_backsub; k_update_x }
//   }
// Bodies are captured on their own streams into the conditional nodes' body
// graphs.  The step loop's kernels read the step from device memory and add
// their offset; consecutive Arnoldi kernels keep their programmatic
// (overlapped) launch.  Each handle is created on the graph that holds its
// node and set by a kernel of that graph or of a graph nested in it.
template <typename T, bool HB>
static ddg_status build_solve_graph(const BatchArgs& args, unsigned G, int n, int Nreq, size_t dots2_smem,
                                    size_t upd_smem, size_t bs_smem, size_t ux_smem, cudaGraphExec_t* out) {
    constexpr cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaGraph_t g = nullptr, cycle_body = nullptr, arn_body = nullptr, fin_body = nullptr, step_body = nullptr;
    cudaStream_t cs[3] = {nullptr, nullptr, nullptr};
    bool capturing[3] = {false, false, false};
    cudaGraphExec_t ex = nullptr;
    cudaGraphConditionalHandle h_outer = 0, h_arn = 0, h_fin = 0, h_loop = 0;
    const char* what = "cudaGraphCreate";
    cudaError_t e = cudaGraphCreate(&g, 0);
    auto ok = [&](cudaError_t r, const char* w) {
        if (e == cudaSuccess && r != cudaSuccess) {
            e = r;
            what = w;
        }
        return e == cudaSuccess;
    };
    auto begin = [&](int i, cudaGraph_t into, const char* w) {
        if (e != cudaSuccess) return false;
        capturing[i] = ok(cudaStreamBeginCaptureToGraph(cs[i], into, nullptr, nullptr, 0, mode), w);
        return capturing[i];
    };
    auto end = [&](int i, const char* w) {
        if (!capturing[i]) return;
        cudaGraph_t body = nullptr;
        const cudaError_t el = cudaGetLastError();   // launch errors of this capture
        const cudaError_t ee = cudaStreamEndCapture(cs[i], &body);
        capturing[i] = false;
        ok(el, w);
        ok(ee, w);
    };
    if (e == cudaSuccess) ok(cudaGraphConditionalHandleCreate(&h_outer, g, 1, cudaGraphCondAssignDefault),
                             "cudaGraphConditionalHandleCreate");
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h_outer;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (ok(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp), "cudaGraphAddNode (cycle loop)"))
            cycle_body = cp.conditional.phGraph_out[0];
    }
    for (int i = 0; i < 3; ++i)
        if (e == cudaSuccess) ok(cudaStreamCreateWithFlags(&cs[i], cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
    // one restart cycle
    if (begin(0, cycle_body, "capture of the cycle")) {
        k_cycle_begin<<<1, 1, 0, cs[0]>>>(args);
        k_residual<T><<<G, kBlock, 0, cs[0]>>>(args);
        if (Nreq > 0) {
            k_dots_r<T, HB><<<G, kBlock, 0, cs[0]>>>(args);
            k_update_r<T, HB><<<G, kBlock, 0, cs[0]>>>(args);
        }
        cudaGraph_t cg = nullptr;
        if (ok(capture_graph(cs[0], &cg), "cudaStreamGetCaptureInfo") &&
            ok(cudaGraphConditionalHandleCreate(&h_arn, cg, 0, 0), "cudaGraphConditionalHandleCreate") &&
            ok(cudaGraphConditionalHandleCreate(&h_fin, cg, 0, 0), "cudaGraphConditionalHandleCreate")) {
            k_cycle_gate<<<1, 1, 0, cs[0]>>>(args, h_outer, h_arn, h_fin);
            if (ok(append_conditional(cs[0], h_arn, cudaGraphCondTypeIf, &arn_body), "Arnoldi IF node"))
                ok(append_conditional(cs[0], h_fin, cudaGraphCondTypeIf, &fin_body), "cycle-end IF node");
        }
    }
    // the cycle's Arnoldi steps: the first step, then the step loop
    if (begin(1, arn_body, "capture of the Arnoldi steps")) {
        k_step<T, HB><<<G, kBlock, 0, cs[1]>>>(args, 0);
        k_dots_w<T, HB><<<G, kBlock, 0, cs[1]>>>(args, 0, 0);
        k_update_w<T, HB><<<G, kBlock, upd_smem, cs[1]>>>(args, 0, 0);
        cudaGraph_t cg = nullptr;
        if (ok(capture_graph(cs[1], &cg), "cudaStreamGetCaptureInfo") &&
            ok(cudaGraphConditionalHandleCreate(&h_loop, cg, 0, 0), "cudaGraphConditionalHandleCreate")) {
            k_inner_begin<<<1, 1, 0, cs[1]>>>(args, h_loop);
            ok(append_conditional(cs[1], h_loop, cudaGraphCondTypeWhile, &step_body), "step WHILE node");
        }
    }
    if (begin(2, step_body, "capture of the step loop")) {
        for (int u = 0; u < kGraphUnroll; ++u) {
            if (u == 0) k_dots2<T, HB><<<G, kBlock, dots2_smem, cs[2]>>>(args, 0);
            else launch_overlapped(k_dots2<T, HB>, G, dots2_smem, cs[2], args, -u);
            launch_overlapped(k_update2<T, HB>, G + n, upd_smem, cs[2], args, -u);
        }
        k_advance<<<1, 1, 0, cs[2]>>>(args, h_loop, kGraphUnroll);
    }
    end(2, "capture of the step loop");
    end(1, "capture of the Arnoldi steps");
    // the cycle's end
    if (begin(1, fin_body, "capture of the cycle end")) {
        k_backsub<<<n, 128, bs_smem, cs[1]>>>(args);
        k_update_x<T, HB><<<G, kBlock, ux_smem, cs[1]>>>(args);
    }
    end(1, "capture of the cycle end");
    end(0, "capture of the cycle");
    if (e == cudaSuccess) ok(cudaGraphInstantiate(&ex, g, 0), "cudaGraphInstantiate");
    for (int i = 0; i < 3; ++i)
        if (cs[i]) cudaStreamDestroy(cs[i]);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        if (ex) cudaGraphExecDestroy(ex);
        cudaGetLastError();
        return cuda_status(e, what);
    }
    *out = ex;
    return DDG_OK;
}

struct GraphExecGuard {
    cudaGraphExec_t e = nullptr;
    ~GraphExecGuard() {
        if (e) cudaGraphExecDestroy(e);   // freed once any launch in flight completes
    }
};

// Dynamic shared memory of the Arnoldi kernels for restart length m and N
// augmentation vectors: the Givens staging (column, sines, result, s in the
// Krylov precision, cosines), k_dots2's column ring and, in the same space
// after it, its reduced coefficients [t | s | alpha | gamma | beta | s^H t],
// k_update's coefficient vectors.  Each kernel is opted into its size.
template <typename T, bool HB>
static ddg_status dcgs2_smem(int Nreq, int m, size_t& giv, size_t& dots2, size_t& upd) {
    using V = c2_t<T>;
    giv = 56 * (size_t)m + 128 + sizeof(V) * (size_t)m;
    dots2 = std::max({(size_t)Ring<T, HB>::ring_bytes, giv, sizeof(double2) * (size_t)(Nreq + 2 * m + 4)});
    upd = std::max(sizeof(V) * (size_t)(Nreq + 2 * m + 2), giv);
    // (the default limit covers static and dynamic shared memory together)
    DDG_CHECK_CUDA(cudaFuncSetAttribute(k_dots2<T, HB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dots2));
    DDG_CHECK_CUDA(cudaFuncSetAttribute(k_update2<T, HB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd));
    DDG_CHECK_CUDA(cudaFuncSetAttribute(k_update_w<T, HB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd));
    return DDG_OK;
}

template <typename T, bool HB>
static ddg_status run_batch(Context* ctx, int n, const ddg_op* const* A, const double* const* b, double* const* x,
                            const double* const* U, int Nreq, double tol, int m, int maxit, double eta,
                            ddg_info* info, cudaStream_t st, bool low_res = false) {
    using V = c2_t<T>;
    const long long CH = chunk_rows<T>();
    int KP = std::max(kMaxAug + 2 * m + 4, Nreq * Nreq);
    KP = (KP + 1) & ~1;
    std::vector<SolvePtrs> hp(n);
    long long total_ctas = 0;
    for (int s = 0; s < n; ++s) {
        hp[s].nchunks = (int)((A[s]->D + CH - 1) / CH);
        hp[s].chunk0 = (int)total_ctas;
        hp[s].ld = (long long)hp[s].nchunks * CH;
        total_ctas += hp[s].nchunks;
    }
    // Two passes over the same layout: size it, then carve the workspace.
    auto layout = [&](char* base) -> size_t {
        Carver c{base};
        for (int s = 0; s < n; ++s) {
            const ddg_op* op = A[s];
            SolvePtrs& P = hp[s];
            const long long ld = P.ld;
            // basis [C | Q] in its storage type; for complex64 the FP64 set-up
            // block W (A V, then C) lives in the same allocation behind C
            constexpr size_t eb = Bstore<T, HB>::ebytes;
            size_t mbytes = eb * (size_t)ld * (size_t)(Nreq + m + 1);
            size_t woff = 0;
            if (Nreq > 0 && sizeof(T) == 4) {
                woff = align_up(eb * (size_t)ld * Nreq);
                mbytes = std::max(mbytes, woff + sizeof(double2) * (size_t)ld * Nreq);
            }
            char* M = c.take<char>(mbytes);
            P.M = M;
            P.W = (Nreq > 0) ? reinterpret_cast<double2*>(M ? M + woff : nullptr) : nullptr;
            P.w[0] = c.take<V>(ld);
            P.w[1] = c.take<V>(ld);
            P.r = c.take<double2>(ld);
            P.V = (Nreq > 0) ? (void*)c.take<V>((size_t)ld * Nreq) : nullptr;
            P.Rg = c.take<double2>((size_t)(m + 1) * m);
            P.Hh = c.take<double2>((size_t)(m + 1) * m + (size_t)kMaxAug * m);   // H and B in T2
            P.tv = c.take<double2>(KP);
            P.B = c.take<double2>((size_t)kMaxAug * m);
            P.cs = c.take<double>(m);
            P.sn = c.take<double2>(m);
            P.g = c.take<double2>(m + 1);
            P.hsum = c.take<double2>(2 * (size_t)KP);
            P.hp = c.take<double2>(KP);
            P.part = c.take<double2>((size_t)P.nchunks * KP);
            P.Rinv = c.take<double2>(std::max(1, Nreq * Nreq));
            P.Rtmp = c.take<double2>(std::max(1, Nreq * Nreq));
            P.cr = c.take<double2>(std::max(1, Nreq));
            P.coefy = c.take<double2>(Nreq + m);
            P.ticket = c.take<unsigned>(1);
            P.dinv = ctx->precond ? (const void*)c.take<V>(ld) : nullptr;
            P.nx = op->nx;
            P.ny = op->ny;
            P.D = op->D;
            P.kh2 = op->kh * op->kh;
            P.eps_d = op->eps_d;
            P.coef_d = op->coef_d;
            P.eps_lo = sizeof(T) == 4 ? (const void*)op->eps_f : (const void*)op->eps_d;
            P.coef_lo = sizeof(T) == 4 ? (const void*)op->coef_f : (const void*)op->coef_d;
            P.b = reinterpret_cast<const double2*>(b[s]);
            P.x = reinterpret_cast<double2*>(x[s]);
            P.U = (Nreq > 0) ? reinterpret_cast<const double2*>(U[s]) : nullptr;
            ctx->policy_for(op->wavelength, &P.aug_cycles, &P.aug_keep);
        }
        return c.off + 4096;
    };
    size_t small_off = layout(nullptr);
    Carver tail{nullptr, small_off};
    tail.take<SolvePtrs>(n);
    tail.take<SolveScal>(n);
    tail.take<int>(total_ctas);
    tail.take<int>(kCounts);
    DDG_TRY(ctx->reserve(tail.off + 4096, st));
    char* base = reinterpret_cast<char*>(ctx->ws);
    layout(base);
    Carver t2{base, small_off};
    BatchArgs args;
    args.P = t2.take<SolvePtrs>(n);
    args.S = t2.take<SolveScal>(n);
    int* d_blk = t2.take<int>(total_ctas);
    args.blk_solve = d_blk;
    args.counts = t2.take<int>(kCounts);
    args.bytes = ctx->prof ? ctx->d_bytes : nullptr;
    args.m = m;
    args.KP = KP;
    args.nmax = kMaxAug;
    args.tol = tol;
    args.eta = eta;
    args.maxit = maxit;
    args.fallback = ctx->fallback;
    args.nsolves = n;
    args.step = args.counts + 5;
    args.low_res = low_res ? 1 : 0;
    args.wait_ns = ctx->wait_ns;
    std::vector<int> hblk(total_ctas);
    for (int s = 0; s < n; ++s)
        for (int c = 0; c < hp[s].nchunks; ++c) hblk[hp[s].chunk0 + c] = s;
    DDG_CHECK_CUDA(cudaMemcpyAsync(args.P, hp.data(), sizeof(SolvePtrs) * n, cudaMemcpyHostToDevice, st));
    DDG_CHECK_CUDA(cudaMemcpyAsync(d_blk, hblk.data(), sizeof(int) * total_ctas, cudaMemcpyHostToDevice, st));

    const unsigned G = (unsigned)total_ctas;
    size_t giv_smem, dots2_smem, upd_smem;
    DDG_TRY((dcgs2_smem<T, HB>(Nreq, m, giv_smem, dots2_smem, upd_smem)));
    const size_t ux_smem = sizeof(V) * (size_t)(Nreq + m);
    DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_init<<<(n + 127) / 128, 128, 0, st>>>(args, n, Nreq); }));
    if (ctx->precond) DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_dinv<T><<<G, kBlock, 0, st>>>(args); }));
    if (Nreq > 0) {
        DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_aug_av<T><<<G, kBlock, 0, st>>>(args); }));
        for (int pass = 0; pass < 2; ++pass) {
            DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_aug_gram<T><<<G, kBlock, 0, st>>>(args, pass); }));
            DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_aug_tri<T><<<G, kBlock, 0, st>>>(args, pass); }));
        }
        DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_aug_rinv<<<(n + 63) / 64, 64, 0, st>>>(args, n); }));
        DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_aug_store<T, HB><<<G, kBlock, 0, st>>>(args); }));
    }
    int* hc = ctx->host_counts;
    const size_t bs_smem = sizeof(double2) * (3 * (size_t)m + kMaxAug);
    DDG_CHECK_CUDA(cudaFuncSetAttribute(k_backsub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs_smem));
    DDG_CHECK_CUDA(cudaMemsetAsync(args.counts, 0, kCounts * sizeof(int), st));
    // delayed scheme: every restart cycle inside one graph launch (per-launch
    // profiling needs the host-driven loop)
    const bool use_graph = ctx->orth == 1 && ctx->graphs && !ctx->prof;
    GraphExecGuard gexec;
    if (use_graph) {
        DDG_TRY((build_solve_graph<T, HB>(args, G, n, Nreq, dots2_smem, upd_smem, bs_smem, ux_smem, &gexec.e)));
        DDG_CHECK_CUDA(cudaGraphLaunch(gexec.e, st));
        DDG_CHECK_CUDA(cudaMemcpyAsync(hc + 4, args.counts + 4, 6 * sizeof(int), cudaMemcpyDeviceToHost, st));
        DDG_CHECK_CUDA(cudaStreamSynchronize(st));
        // launches of the graph: per cycle begun k_cycle_begin, k_residual,
        // [k_dots_r, k_update_r], k_cycle_gate; per cycle with Arnoldi steps
        // k_step, k_dots_w, k_update_w, k_inner_begin; per step-loop body
        // 2 kGraphUnroll + 1; per finished cycle k_backsub, k_update_x
        const long long cycles = hc[6], bodies = hc[7], arn = hc[8], fin = hc[9];
        const long long res = 1 + (Nreq > 0 ? 2 : 0);
        ctx->launches += cycles * (res + 2) + arn * 4 + bodies * (2 * kGraphUnroll + 1) + fin * 2;
        ctx->nlaunch[DDG_K_RESIDUAL] += cycles * res;
        ctx->nlaunch[DDG_K_STEP] += cycles * 2 + arn * 2 + bodies;
        ctx->nlaunch[DDG_K_DOTS] += arn + bodies * kGraphUnroll;
        ctx->nlaunch[DDG_K_UPDATE] += arn + bodies * kGraphUnroll;
        ctx->nlaunch[DDG_K_CYCLE_END] += fin * 2;
        if (hc[4]) {
            set_error("gmres: a column copy into shared memory did not complete within its time limit");
            return DDG_ETIMEOUT;
        }
    }
    for (long long cycle = 0; !use_graph && cycle <= (long long)maxit + 1; ++cycle) {
        DDG_CHECK_CUDA(cudaMemsetAsync(args.counts, 0, 4 * sizeof(int), st));
        DDG_TRY(ctx->launch(DDG_K_RESIDUAL, st, [&] { k_residual<T><<<G, kBlock, 0, st>>>(args); }));
        if (Nreq > 0) {
            DDG_TRY(ctx->launch(DDG_K_RESIDUAL, st, [&] { k_dots_r<T, HB><<<G, kBlock, 0, st>>>(args); }));
            DDG_TRY(ctx->launch(DDG_K_RESIDUAL, st, [&] { k_update_r<T, HB><<<G, kBlock, 0, st>>>(args); }));
        }
        DDG_CHECK_CUDA(cudaMemcpyAsync(hc, args.counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        DDG_CHECK_CUDA(cudaMemcpyAsync(hc + 4, args.counts + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        DDG_CHECK_CUDA(cudaStreamSynchronize(st));
        if (hc[4]) {
            set_error("gmres: a column copy into shared memory did not complete within its time limit");
            return DDG_ETIMEOUT;
        }
        if (hc[1] == 0) break;
        if (hc[0] > 0 && ctx->orth == 1) {
            // delayed reorthogonalisation: first pass of step 0, then one
            // reduction and one sweep per step
            DDG_TRY(ctx->launch(DDG_K_STEP, st, [&] { k_step<T, HB><<<G, kBlock, 0, st>>>(args, 0); }));
            DDG_TRY(ctx->launch(DDG_K_DOTS, st, [&] { k_dots_w<T, HB><<<G, kBlock, 0, st>>>(args, 0, 0); }));
            DDG_TRY(ctx->launch(DDG_K_UPDATE, st, [&] { k_update_w<T, HB><<<G, kBlock, upd_smem, st>>>(args, 0, 0); }));
            int polled = 0;
            for (int i = 1; i <= m; ++i) {
                DDG_TRY(ctx->launch(DDG_K_DOTS, st, [&] { launch_overlapped(k_dots2<T, HB>, G, dots2_smem, st, args, i); }));
                if (i < m)
                    DDG_TRY(ctx->launch(DDG_K_UPDATE, st,
                                        [&] { launch_overlapped(k_update2<T, HB>, G + n, upd_smem, st, args, i); }));
                if (i % ctx->poll_every == 0 && i < m) {
                    const int slot = polled & 1;
                    DDG_CHECK_CUDA(cudaMemcpyAsync(hc + 2 + slot, args.counts, sizeof(int), cudaMemcpyDeviceToHost, st));
                    DDG_CHECK_CUDA(cudaEventRecord(ctx->ev[slot], st));
                    if (polled > 0) {
                        DDG_CHECK_CUDA(cudaEventSynchronize(ctx->ev[slot ^ 1]));
                        if (hc[2 + (slot ^ 1)] == 0) break;
                    }
                    ++polled;
                }
            }
        } else if (hc[0] > 0) {
            int polled = 0;
            for (int j = 0; j < m; ++j) {
                DDG_TRY(ctx->launch(DDG_K_STEP, st, [&] { k_step<T, HB><<<G, kBlock, 0, st>>>(args, j); }));
                DDG_TRY(ctx->launch(DDG_K_DOTS, st, [&] { k_dots_w<T, HB><<<G, kBlock, 0, st>>>(args, j, 0); }));
                DDG_TRY(ctx->launch(DDG_K_UPDATE, st, [&] { k_update_w<T, HB><<<G, kBlock, upd_smem, st>>>(args, j, 0); }));
                DDG_TRY(ctx->launch(DDG_K_DOTS, st, [&] { k_dots_w<T, HB><<<G, kBlock, 0, st>>>(args, j, 1); }));
                DDG_TRY(ctx->launch(DDG_K_UPDATE, st, [&] { k_update_w<T, HB><<<G, kBlock, upd_smem, st>>>(args, j, 1); }));
                if ((j + 1) % ctx->poll_every == 0 && j + 1 < m) {
                    const int slot = polled & 1;
                    DDG_CHECK_CUDA(cudaMemcpyAsync(hc + 2 + slot, args.counts, sizeof(int), cudaMemcpyDeviceToHost, st));
                    DDG_CHECK_CUDA(cudaEventRecord(ctx->ev[slot], st));
                    if (polled > 0) {
                        DDG_CHECK_CUDA(cudaEventSynchronize(ctx->ev[slot ^ 1]));
                        if (hc[2 + (slot ^ 1)] == 0) break;
                    }
                    ++polled;
                }
            }
        }
        DDG_TRY(ctx->launch(DDG_K_CYCLE_END, st, [&] { k_backsub<<<n, 128, bs_smem, st>>>(args); }));
        DDG_TRY(ctx->launch(DDG_K_CYCLE_END, st, [&] { k_update_x<T, HB><<<G, kBlock, ux_smem, st>>>(args); }));
    }
    DDG_TRY(ctx->launch(DDG_K_CYCLE_END, st, [&] { k_finalize<T><<<G, kBlock, 0, st>>>(args); }));
    std::vector<SolveScal> hs(n);
    DDG_CHECK_CUDA(cudaMemcpyAsync(hs.data(), args.S, sizeof(SolveScal) * n, cudaMemcpyDeviceToHost, st));
    DDG_CHECK_CUDA(cudaMemcpyAsync(hc + 4, args.counts + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DDG_CHECK_CUDA(cudaStreamSynchronize(st));
    ctx->resolve();
    if (hc[4]) {
        set_error("gmres: a column copy into shared memory did not complete within its time limit");
        return DDG_ETIMEOUT;
    }
    bool all = true;
    for (int s = 0; s < n; ++s) {
        all = all && hs[s].converged;
        if (info) {
            info[s].iters = hs[s].iters;
            info[s].cycles = hs[s].cycles;
            info[s].converged = hs[s].converged;
            info[s].fallback_used = hs[s].fallback;
            info[s].breakdown = hs[s].breakdown;
            info[s].true_rel_residual = hs[s].true_res;
            info[s].first_step_rel_residual = hs[s].first_res;
        }
    }
    return all ? DDG_OK : DDG_ENOCONV;
}

static ddg_status solve_entry(ddg_context* cptr, int n, const ddg_op* const* A, const double* const* b,
                              const double* const* U, int k, double* const* x, double tol, int restart,
                              int maxit, ddg_precision prec, ddg_info* info, void* stream, const char* who) {
    if (!cptr) { set_error("%s: context is NULL", who); return DDG_EINVAL; }
    if (n < 1 || !A || !b || !x) { set_error("%s: n=%d or NULL array", who, n); return DDG_EINVAL; }
    if (!(tol > 0.0 && tol < 1.0)) { set_error("%s: tol=%g outside (0,1)", who, tol); return DDG_EINVAL; }
    if (restart < 1 || restart > kMaxRestart) { set_error("%s: restart=%d outside [1,%d]", who, restart, kMaxRestart); return DDG_EINVAL; }
    if (maxit < 1) { set_error("%s: maxit=%d < 1", who, maxit); return DDG_EINVAL; }
    if (prec != DDG_C128 && prec != DDG_C64_REFINE && prec != DDG_C64_ONLY) {
        set_error("%s: unsupported precision %d", who, (int)prec);
        return DDG_EINVAL;
    }
    if (U && (k < 1 || k > kMaxAug)) { set_error("%s: k=%d outside [1,%d]", who, k, kMaxAug); return DDG_EINVAL; }
    for (int s = 0; s < n; ++s) {
        if (!A[s] || !b[s] || !x[s]) { set_error("%s: NULL operator/b/x at %d", who, s); return DDG_EINVAL; }
        if (U && !U[s]) { set_error("%s: NULL U at %d", who, s); return DDG_EINVAL; }
        if (A[s]->D > (1LL << 31) / 2) { set_error("%s: grid too large", who); return DDG_EINVAL; }
    }
    Context* ctx = reinterpret_cast<Context*>(cptr);
    cudaStream_t st = as_stream(stream);
    const int Nreq = U ? k : 0;
    if (prec == DDG_C128)
        return run_batch<double, false>(ctx, n, A, b, x, U, Nreq, tol, restart, maxit, 0.0, info, st);
    const bool lo = prec == DDG_C64_ONLY;   // cycles run to tol * ||b||; residual in FP32
    const double eta = lo ? 0.0 : ctx->inner_tol;
    if (ctx->half_basis)
        return run_batch<float, true>(ctx, n, A, b, x, U, Nreq, tol, restart, maxit, eta, info, st, lo);
    return run_batch<float, false>(ctx, n, A, b, x, U, Nreq, tol, restart, maxit, eta, info, st, lo);
}

}  // namespace ddg

using namespace ddg;

extern "C" ddg_status gmres_solve(ddg_context* ctx, const ddg_op* A, const double* b, double* x, double tol,
                                  int restart, int maxit, ddg_precision prec, ddg_info* info, void* stream) {
    return solve_entry(ctx, 1, &A, &b, nullptr, 0, &x, tol, restart, maxit, prec, info, stream, "gmres_solve");
}

extern "C" ddg_status augmented_gmres_solve(ddg_context* ctx, const ddg_op* A, const double* b, const double* U,
                                            int k, double* x, double tol, int restart, int maxit,
                                            ddg_precision prec, ddg_info* info, void* stream) {
    if (!U) { set_error("augmented_gmres_solve: U is NULL"); return DDG_EINVAL; }
    return solve_entry(ctx, 1, &A, &b, &U, k, &x, tol, restart, maxit, prec, info, stream,
                       "augmented_gmres_solve");
}

extern "C" ddg_status gmres_solve_batched(ddg_context* ctx, int n, const ddg_op* const* A, const double* const* b,
                                          double* const* x, double tol, int restart, int maxit,
                                          ddg_precision prec, ddg_info* info, void* stream) {
    return solve_entry(ctx, n, A, b, nullptr, 0, x, tol, restart, maxit, prec, info, stream,
                       "gmres_solve_batched");
}

extern "C" ddg_status augmented_gmres_solve_batched(ddg_context* ctx, int n, const ddg_op* const* A,
                                                    const double* const* b, const double* const* U, int k,
                                                    double* const* x, double tol, int restart, int maxit,
                                                    ddg_precision prec, ddg_info* info, void* stream) {
    if (!U) { set_error("augmented_gmres_solve_batched: U is NULL"); return DDG_EINVAL; }
    return solve_entry(ctx, n, A, b, U, k, x, tol, restart, maxit, prec, info, stream,
                       "augmented_gmres_solve_batched");
}

// ---------------------------------------------------------------- solve without device allocation
// gmres_solve_noalloc: one plain GMRES solve whose whole workspace lives in a
// file-scope device array, for callers that must not allocate device memory.
namespace ddg {

constexpr size_t kNoAllocBytes = (size_t)DDG_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static void* g_noalloc_base[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device.  In host code
// the array's name only stands in for it, so the address is looked up once per
// device (with that device current) and kept.
static ddg_status noalloc_base(char** out) {
    int dev = 0;
    DDG_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("gmres_solve_noalloc: device %d beyond the %d supported", dev, kNoAllocMaxDevices);
        return DDG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "gmres_solve_noalloc: cudaGetSymbolAddress");
        g_noalloc_base[dev] = p;
    }
    *out = reinterpret_cast<char*>(g_noalloc_base[dev]);
    return DDG_OK;
}

// Same kernels and order as run_batch for one solve without augmentation and
// the delayed reorthogonalisation; the workspace is carved from the static
// array; polls by synchronising the stream (no pinned buffer, no events).
template <typename T>
static ddg_status run_single_noalloc(const ddg_op* A, const double* b, double* x, double tol, int m, int maxit,
                                     double eta, ddg_info* info, cudaStream_t st) {
    using V = c2_t<T>;
    const long long CH = chunk_rows<T>();
    int KP = kMaxAug + 2 * m + 4;
    KP = (KP + 1) & ~1;
    SolvePtrs hp{};
    hp.nchunks = (int)((A->D + CH - 1) / CH);
    hp.chunk0 = 0;
    hp.ld = (long long)hp.nchunks * CH;
    const long long ld = hp.ld;
    auto layout = [&](char* base) -> size_t {
        Carver c{base};
        hp.M = c.take<char>(sizeof(V) * (size_t)ld * (size_t)(m + 1));
        hp.W = nullptr;
        hp.w[0] = c.take<V>(ld);
        hp.w[1] = c.take<V>(ld);
        hp.r = c.take<double2>(ld);
        hp.V = nullptr;
        hp.Rg = c.take<double2>((size_t)(m + 1) * m);
        hp.Hh = c.take<double2>((size_t)(m + 1) * m + (size_t)kMaxAug * m);
        hp.tv = c.take<double2>(KP);
        hp.B = c.take<double2>((size_t)kMaxAug * m);
        hp.cs = c.take<double>(m);
        hp.sn = c.take<double2>(m);
        hp.g = c.take<double2>(m + 1);
        hp.hsum = c.take<double2>(2 * (size_t)KP);
        hp.hp = c.take<double2>(KP);
        hp.part = c.take<double2>((size_t)hp.nchunks * KP);
        hp.Rinv = c.take<double2>(1);
        hp.Rtmp = c.take<double2>(1);
        hp.cr = c.take<double2>(1);
        hp.coefy = c.take<double2>(m);
        hp.ticket = c.take<unsigned>(1);
        // the same 4096-byte slack behind the last array as run_batch keeps
        return c.off + 4096;
    };
    size_t small_off = align_up(layout(nullptr));
    Carver tail{nullptr, small_off};
    tail.take<SolvePtrs>(1);
    tail.take<SolveScal>(1);
    tail.take<int>(hp.nchunks);
    tail.take<int>(8);
    const size_t need = tail.off;
    if (need > kNoAllocBytes) {
        set_error("gmres_solve_noalloc: this solve needs %zu bytes of scratch, more than the %zu-byte static "
                  "buffer (use a smaller restart or grid, or gmres_solve)", need, kNoAllocBytes);
        return DDG_EINVAL;
    }
    char* base = nullptr;
    DDG_TRY(noalloc_base(&base));
    layout(base);
    hp.nx = A->nx;
    hp.ny = A->ny;
    hp.D = A->D;
    hp.kh2 = A->kh * A->kh;
    hp.eps_d = A->eps_d;
    hp.coef_d = A->coef_d;
    hp.eps_lo = sizeof(T) == 4 ? (const void*)A->eps_f : (const void*)A->eps_d;
    hp.coef_lo = sizeof(T) == 4 ? (const void*)A->coef_f : (const void*)A->coef_d;
    hp.b = reinterpret_cast<const double2*>(b);
    hp.x = reinterpret_cast<double2*>(x);
    hp.U = nullptr;
    hp.aug_cycles = 1;
    hp.aug_keep = 0;
    Carver t2{base, small_off};
    BatchArgs args;
    args.P = t2.take<SolvePtrs>(1);
    args.S = t2.take<SolveScal>(1);
    int* d_blk = t2.take<int>(hp.nchunks);
    args.blk_solve = d_blk;
    args.counts = t2.take<int>(8);
    args.bytes = nullptr;
    args.m = m;
    args.KP = KP;
    args.nmax = kMaxAug;
    args.tol = tol;
    args.eta = eta;
    args.maxit = maxit;
    args.fallback = 1e300;
    args.nsolves = 1;
    args.step = args.counts + 5;
    args.low_res = 0;
    args.wait_ns = kDefaultWaitNs;
    // every launch reads these: the array keeps the previous call's contents
    std::vector<int> hblk(hp.nchunks, 0);
    DDG_CHECK_CUDA(cudaMemcpyAsync(args.P, &hp, sizeof(SolvePtrs), cudaMemcpyHostToDevice, st));
    DDG_CHECK_CUDA(cudaMemcpyAsync(d_blk, hblk.data(), sizeof(int) * hp.nchunks, cudaMemcpyHostToDevice, st));
    const unsigned G = (unsigned)hp.nchunks;
    size_t giv_smem, dots2_smem, upd_smem;
    DDG_TRY((dcgs2_smem<T, false>(0, m, giv_smem, dots2_smem, upd_smem)));
    const size_t ux_smem = sizeof(V) * (size_t)m;
    const size_t bs_smem = sizeof(double2) * (3 * (size_t)m + kMaxAug);
    DDG_CHECK_CUDA(cudaFuncSetAttribute(k_backsub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs_smem));
    k_init<<<1, 128, 0, st>>>(args, 1, 0);   // also zeroes the reduction ticket
    DDG_CHECK_LAUNCH("k_init");
    int hc[5] = {0, 0, 0, 0, 0};
    DDG_CHECK_CUDA(cudaMemsetAsync(args.counts, 0, 8 * sizeof(int), st));
    for (long long cycle = 0; cycle <= (long long)maxit + 1; ++cycle) {
        DDG_CHECK_CUDA(cudaMemsetAsync(args.counts, 0, 4 * sizeof(int), st));
        k_residual<T><<<G, kBlock, 0, st>>>(args);
        DDG_CHECK_LAUNCH("k_residual");
        DDG_CHECK_CUDA(cudaMemcpyAsync(hc, args.counts, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
        DDG_CHECK_CUDA(cudaStreamSynchronize(st));
        if (hc[4]) {
            set_error("gmres_solve_noalloc: a column copy into shared memory did not complete within its time limit");
            return DDG_ETIMEOUT;
        }
        if (hc[1] == 0) break;
        if (hc[0] > 0) {
            k_step<T, false><<<G, kBlock, 0, st>>>(args, 0);
            k_dots_w<T, false><<<G, kBlock, 0, st>>>(args, 0, 0);
            k_update_w<T, false><<<G, kBlock, upd_smem, st>>>(args, 0, 0);
            DDG_CHECK_LAUNCH("first Arnoldi step");
            for (int i = 1; i <= m; ++i) {
                k_dots2<T, false><<<G, kBlock, dots2_smem, st>>>(args, i);
                if (i < m) k_update2<T, false><<<G + 1, kBlock, upd_smem, st>>>(args, i);
                DDG_CHECK_LAUNCH("Arnoldi step");
                if (i % 16 == 0 && i < m) {
                    int in_cycle = 0;
                    DDG_CHECK_CUDA(cudaMemcpyAsync(&in_cycle, args.counts, sizeof(int), cudaMemcpyDeviceToHost, st));
                    DDG_CHECK_CUDA(cudaStreamSynchronize(st));
                    if (in_cycle == 0) break;
                }
            }
        }
        k_backsub<<<1, 128, bs_smem, st>>>(args);
        k_update_x<T, false><<<G, kBlock, ux_smem, st>>>(args);
        DDG_CHECK_LAUNCH("cycle end");
    }
    k_finalize<T><<<G, kBlock, 0, st>>>(args);
    DDG_CHECK_LAUNCH("k_finalize");
    SolveScal hs;
    DDG_CHECK_CUDA(cudaMemcpyAsync(&hs, args.S, sizeof(SolveScal), cudaMemcpyDeviceToHost, st));
    DDG_CHECK_CUDA(cudaMemcpyAsync(hc, args.counts, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DDG_CHECK_CUDA(cudaStreamSynchronize(st));
    if (hc[4]) {
        set_error("gmres_solve_noalloc: a column copy into shared memory did not complete within its time limit");
        return DDG_ETIMEOUT;
    }
    if (info) {
        info->iters = hs.iters;
        info->cycles = hs.cycles;
        info->converged = hs.converged;
        info->fallback_used = 0;
        info->breakdown = hs.breakdown;
        info->true_rel_residual = hs.true_res;
        info->first_step_rel_residual = hs.first_res;
    }
    return hs.converged ? DDG_OK : DDG_ENOCONV;
}

}  // namespace ddg

extern "C" ddg_status gmres_solve_noalloc(const ddg_op* A, const double* b, double* x, double tol, int restart,
                                          int maxit, ddg_precision prec, ddg_info* info, void* stream) {
    using namespace ddg;
    if (!A || !b || !x) { set_error("gmres_solve_noalloc: NULL operator, b or x"); return DDG_EINVAL; }
    if (!(tol > 0.0 && tol < 1.0)) { set_error("gmres_solve_noalloc: tol=%g outside (0,1)", tol); return DDG_EINVAL; }
    if (restart < 1 || restart > kMaxRestart) { set_error("gmres_solve_noalloc: restart=%d outside [1,%d]", restart, kMaxRestart); return DDG_EINVAL; }
    if (maxit < 1) { set_error("gmres_solve_noalloc: maxit=%d < 1", maxit); return DDG_EINVAL; }
    cudaStream_t st = as_stream(stream);
    if (prec == DDG_C128) return run_single_noalloc<double>(A, b, x, tol, restart, maxit, 0.0, info, st);
    if (prec == DDG_C64_REFINE) return run_single_noalloc<float>(A, b, x, tol, restart, maxit, 1e-5, info, st);
    set_error("gmres_solve_noalloc: unsupported precision %d", (int)prec);
    return DDG_EINVAL;
}
