// Principal components of training fields (Sec. III, "Principal component
// analysis"): the leading left singular vectors of F = [f_1 ... f_M]
// (uncentred), computed by the method of snapshots in FP64:
//   G = F^H F (M x M),  top-k eigenpairs (lambda_c, w_c) of G,
//   u_c = F w_c / sqrt(lambda_c),  sigma_c = sqrt(lambda_c).
// The eigenpairs come from block subspace iteration on G with k' = k + 16
// vectors (Cholesky QR twice after every product), followed by Rayleigh-Ritz:
// T = X^H G X is diagonalised by cyclic complex Jacobi rotations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "engine.cuh"

namespace ddg {

constexpr int kPcaMaxK = 32;
constexpr int kPcaOver = 16;
constexpr int kPcaMaxKp = kPcaMaxK + kPcaOver;
constexpr int kGT = 32;  // Gram tile

// G(i, j) = sum_e conj(F(e, i)) F(e, j) over one slice of rows (split-K);
// 32x32 output tile per CTA, 256 threads x 4 outputs.
__global__ void __launch_bounds__(256) k_pca_gram(const double2* __restrict__ F, long long D, int M,
                                                  long long rows_per_slice, double2* __restrict__ Gpart) {
    const int ti = blockIdx.x, tj = blockIdx.y, sl = blockIdx.z;
    if (tj < ti) return;  // upper tiles only (G is Hermitian)
    __shared__ double2 A[kGT][kGT + 1];
    __shared__ double2 B[kGT][kGT + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in [0, 8)
    double2 acc[4];
    for (int u = 0; u < 4; ++u) acc[u] = make_double2(0.0, 0.0);
    const long long e0 = (long long)sl * rows_per_slice;
    const long long e1 = min(D, e0 + rows_per_slice);
    for (long long eb = e0; eb < e1; eb += kGT) {
        // load rows eb..eb+31 of columns ti*32.. and tj*32..  (row index = tx: coalesced)
        for (int c = ty; c < kGT; c += 8) {
            long long e = eb + tx;
            int ci = ti * kGT + c, cj = tj * kGT + c;
            A[c][tx] = (e < e1 && ci < M) ? F[(long long)ci * D + e] : make_double2(0.0, 0.0);
            B[c][tx] = (e < e1 && cj < M) ? F[(long long)cj * D + e] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        // thread computes G(ti*32 + ty + 8u, tj*32 + tx)
        for (int r = 0; r < kGT; ++r) {
            double2 bv = B[tx][r];
#pragma unroll
            for (int u = 0; u < 4; ++u) cfmac(acc[u], A[ty + 8 * u][r], bv);
        }
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u) {
        int i = ti * kGT + ty + 8 * u, j = tj * kGT + tx;
        if (i < M && j < M) Gpart[(long long)sl * M * M + (long long)j * M + i] = acc[u];
    }
}

// Sums the split-K slices and fills the lower triangle by Hermitian symmetry.
__global__ void k_pca_gram_sum(const double2* __restrict__ Gpart, int M, int slices, double2* __restrict__ G) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)M * M) return;
    int j = (int)(idx / M), i = (int)(idx % M);
    int ii = min(i, j), jj = max(i, j);
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < slices; ++q) s = cadd(s, Gpart[(long long)q * M * M + (long long)jj * M + ii]);
    if (i > j) s.y = -s.y;  // G(i, j) = conj(G(j, i))
    if (i == j) s.y = 0.0;
    G[idx] = s;
}

// Y = G X (M x kp), one thread per output.
__global__ void k_pca_gx(const double2* __restrict__ G, const double2* __restrict__ X, int M, int kp,
                         double2* __restrict__ Y) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * kp) return;
    int c = idx / M, i = idx % M;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < M; ++l) cfma(acc, G[(long long)l * M + i], X[(long long)c * M + l]);
    Y[idx] = acc;
}

__device__ double block_sum(double v, double* sm) {
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sm[w];
    __syncthreads();
    return t;  // every thread
}

// X = Y with orthonormal columns: modified Gram-Schmidt, applied twice (one CTA).
__global__ void __launch_bounds__(256) k_pca_orth(const double2* __restrict__ Y, int M, int kp, double2* X) {
    __shared__ double sm[8];
    for (int idx = threadIdx.x; idx < M * kp; idx += blockDim.x) X[idx] = Y[idx];
    __syncthreads();
    for (int c = 0; c < kp; ++c) {
        double2* xc = X + (long long)c * M;
        for (int pass = 0; pass < 2; ++pass) {
            for (int p = 0; p < c; ++p) {
                const double2* xp = X + (long long)p * M;
                double re = 0.0, im = 0.0;
                for (int i = threadIdx.x; i < M; i += blockDim.x) {
                    double2 t = cmulc(xp[i], xc[i]);
                    re += t.x;
                    im += t.y;
                }
                re = block_sum(re, sm);
                im = block_sum(im, sm);
                double2 h = make_double2(re, im);
                for (int i = threadIdx.x; i < M; i += blockDim.x) xc[i] = csub(xc[i], cmul(xp[i], h));
                __syncthreads();
            }
        }
        double n2 = 0.0;
        for (int i = threadIdx.x; i < M; i += blockDim.x) n2 += cabs2(xc[i]);
        n2 = block_sum(n2, sm);
        double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
        for (int i = threadIdx.x; i < M; i += blockDim.x) xc[i] = cscale(xc[i], inv);
        __syncthreads();
    }
}

// Rayleigh-Ritz: T = X^H Y (Y = G X), eigen-decomposition of the Hermitian T by
// cyclic Jacobi (one CTA; one warp applies the rotations), eigenvalues sorted
// in decreasing order; W = X Z[:, :k], lambda[0..k).
__global__ void __launch_bounds__(256) k_pca_rr(const double2* __restrict__ X, const double2* __restrict__ Y, int M,
                                               int kp, int k, double2* __restrict__ W, double* __restrict__ lam) {
    extern __shared__ double2 dsm[];
    const int ld = kp + 1;
    double2* Tm = dsm;             // T(a, b) at Tm[a * ld + b]
    double2* Zm = dsm + kp * ld;   // Z(a, b) at Zm[a * ld + b]
#define T(a, b) Tm[(a) * ld + (b)]
#define Z(a, b) Zm[(a) * ld + (b)]
    __shared__ int order[kPcaMaxKp];
    for (int idx = threadIdx.x; idx < kp * kp; idx += blockDim.x) {
        int a = idx / kp, b = idx % kp;
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < M; ++i) cfmac(acc, X[(long long)a * M + i], Y[(long long)b * M + i]);
        T(a, b) = acc;
        Z(a, b) = make_double2(a == b ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    // symmetrise (T is Hermitian up to round-off)
    for (int idx = threadIdx.x; idx < kp * kp; idx += blockDim.x) {
        int a = idx / kp, b = idx % kp;
        if (a < b) {
            double2 u = T(a, b), v = T(b, a);
            double2 h = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
            T(a, b) = h;
            T(b, a) = make_double2(h.x, -h.y);
        } else if (a == b) {
            T(a, a).y = 0.0;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int sweep = 0; sweep < 60; ++sweep) {
            double off = 0.0, tot = 0.0;
            for (int idx = lane; idx < kp * kp; idx += 32) {
                int a = idx / kp, b = idx % kp;
                double v = cabs2(T(a, b));
                tot += v;
                if (a != b) off += v;
            }
            off = warp_sum_d(off);
            tot = warp_sum_d(tot);
            if (off <= 1e-30 * tot) break;
            for (int p = 0; p < kp - 1; ++p)
                for (int q = p + 1; q < kp; ++q) {
                    double2 apq = T(p, q);
                    double mag = hypot(apq.x, apq.y);
                    if (mag == 0.0) continue;
                    // phase e^{i phi} = apq / |apq|; real rotation on [[app, |apq|], [|apq|, aqq]]
                    double2 ph = make_double2(apq.x / mag, apq.y / mag);
                    double app = T(p, p).x, aqq = T(q, q).x;
                    double tau = (aqq - app) / (2.0 * mag);
                    double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                    // U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on (p, q)
                    double2 em = make_double2(ph.x, -ph.y);  // e^{-i phi}
                    double2 u10 = cscale(em, -s), u11 = cscale(em, c);
                    __syncwarp();
                    // columns: T <- T U, Z <- Z U
                    for (int r = lane; r < kp; r += 32) {
                        double2 tp = T(r, p), tq = T(r, q);
                        T(r, p) = cadd(cscale(tp, c), cmul(tq, u10));
                        T(r, q) = cadd(cscale(tp, s), cmul(tq, u11));
                        double2 zp = Z(r, p), zq = Z(r, q);
                        Z(r, p) = cadd(cscale(zp, c), cmul(zq, u10));
                        Z(r, q) = cadd(cscale(zp, s), cmul(zq, u11));
                    }
                    __syncwarp();
                    // rows: T <- U^H T
                    for (int r = lane; r < kp; r += 32) {
                        double2 tp = T(p, r), tq = T(q, r);
                        T(p, r) = cadd(cscale(tp, c), cmulc(u10, tq));
                        T(q, r) = cadd(cscale(tp, s), cmulc(u11, tq));
                    }
                    __syncwarp();
                    if (lane == 0) {
                        T(p, q) = make_double2(0.0, 0.0);
                        T(q, p) = make_double2(0.0, 0.0);
                        T(p, p).y = 0.0;
                        T(q, q).y = 0.0;
                    }
                    __syncwarp();
                }
        }
        if (lane == 0) {
            for (int a = 0; a < kp; ++a) order[a] = a;
            for (int a = 1; a < kp; ++a) {  // insertion sort, decreasing eigenvalue
                int v = order[a], b = a - 1;
                while (b >= 0 && T(order[b], order[b]).x < T(v, v).x) {
                    order[b + 1] = order[b];
                    --b;
                }
                order[b + 1] = v;
            }
            for (int c = 0; c < k; ++c) lam[c] = T(order[c], order[c]).x;
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < M * k; idx += blockDim.x) {
        int c = idx / M, i = idx % M;
        int oc = order[c];
        double2 acc = make_double2(0.0, 0.0);
        for (int a = 0; a < kp; ++a) cfma(acc, X[(long long)a * M + i], Z(a, oc));
        W[idx] = acc;
    }
}
#undef T
#undef Z

// U(e, c) = sum_m F(e, m) W(m, c) / sqrt(lambda_c); one thread per row e.
__global__ void __launch_bounds__(128) k_pca_basis(const double2* __restrict__ F, long long D, int M, int k,
                                                  const double2* __restrict__ W, const double* __restrict__ lam,
                                                  double2* __restrict__ U) {
    __shared__ double2 Ws[32][kPcaMaxK];
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double2 acc[kPcaMaxK];
#pragma unroll
    for (int c = 0; c < kPcaMaxK; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int m0 = 0; m0 < M; m0 += 32) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * k; idx += blockDim.x) {
            int mm = idx / k, c = idx % k;
            Ws[mm][c] = (m0 + mm < M) ? W[(long long)c * M + m0 + mm] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (e < D) {
            const int mt = min(32, M - m0);
            for (int mm = 0; mm < mt; ++mm) {
                double2 f = F[(long long)(m0 + mm) * D + e];
#pragma unroll
                for (int c = 0; c < kPcaMaxK; ++c)
                    if (c < k) cfma(acc[c], f, Ws[mm][c]);
            }
        }
    }
    if (e >= D) return;
#pragma unroll
    for (int c = 0; c < kPcaMaxK; ++c)
        if (c < k) {
            double l = lam[c];
            double inv = l > 0.0 ? 1.0 / sqrt(l) : 0.0;
            U[(long long)c * D + e] = cscale(acc[c], inv);
        }
}

static ddg_status pca_fit_impl(Context* ctx, const double2* F, long long D, int M, int k, double2* U,
                               double* sigma, cudaStream_t st) {
    const int kp = std::min(M, k + kPcaOver);
    const int slices = (int)std::max(1LL, std::min(64LL, D / 1024));
    const long long rps = (D + slices - 1) / slices;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    size_t off = 0;
    const size_t oGp = off; off = al(off + sizeof(double2) * (size_t)slices * M * M);
    const size_t oG = off; off = al(off + sizeof(double2) * (size_t)M * M);
    const size_t oX = off; off = al(off + sizeof(double2) * (size_t)M * kp);
    const size_t oY = off; off = al(off + sizeof(double2) * (size_t)M * kp);
    const size_t oW = off; off = al(off + sizeof(double2) * (size_t)M * k);
    const size_t oL = off; off = al(off + sizeof(double) * (size_t)k);
    DDG_TRY(ctx->reserve(off, st));
    char* base = reinterpret_cast<char*>(ctx->ws);
    double2* Gp = reinterpret_cast<double2*>(base + oGp);
    double2* G = reinterpret_cast<double2*>(base + oG);
    double2* X = reinterpret_cast<double2*>(base + oX);
    double2* Y = reinterpret_cast<double2*>(base + oY);
    double2* W = reinterpret_cast<double2*>(base + oW);
    double* lam = reinterpret_cast<double*>(base + oL);
    const int nt = (M + kGT - 1) / kGT;
    DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] {
        k_pca_gram<<<dim3(nt, nt, slices), 256, 0, st>>>(F, D, M, rps, Gp);
    }));
    DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] {
        k_pca_gram_sum<<<(unsigned)(((long long)M * M + 255) / 256), 256, 0, st>>>(Gp, M, slices, G);
    }));
    // deterministic start block: the first kp unit vectors mixed with a fixed pattern
    std::vector<double2> hx((size_t)M * kp);
    for (int c = 0; c < kp; ++c)
        for (int i = 0; i < M; ++i) {
            unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)(c * 40503u + 17u);
            h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
            hx[(size_t)c * M + i] = make_double2(((h & 0xffff) / 65535.0) - 0.5, (((h >> 16) & 0xffff) / 65535.0) - 0.5);
        }
    DDG_CHECK_CUDA(cudaMemcpyAsync(Y, hx.data(), sizeof(double2) * hx.size(), cudaMemcpyHostToDevice, st));
    DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_pca_orth<<<1, 256, 0, st>>>(Y, M, kp, X); }));
    const unsigned gx = (unsigned)((M * kp + 255) / 256);
    for (int it = 0; it < 60; ++it) {
        DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_pca_gx<<<gx, 256, 0, st>>>(G, X, M, kp, Y); }));
        DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_pca_orth<<<1, 256, 0, st>>>(Y, M, kp, X); }));
    }
    DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_pca_gx<<<gx, 256, 0, st>>>(G, X, M, kp, Y); }));
    const size_t rr_smem = sizeof(double2) * 2 * (size_t)kp * (kp + 1);
    DDG_CHECK_CUDA(cudaFuncSetAttribute(k_pca_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rr_smem));
    DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] { k_pca_rr<<<1, 256, rr_smem, st>>>(X, Y, M, kp, k, W, lam); }));
    DDG_TRY(ctx->launch(DDG_K_SETUP, st, [&] {
        k_pca_basis<<<(unsigned)((D + 127) / 128), 128, 0, st>>>(F, D, M, k, W, lam, U);
    }));
    if (sigma) {
        std::vector<double> hl(k);
        DDG_CHECK_CUDA(cudaMemcpyAsync(hl.data(), lam, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        DDG_CHECK_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < k; ++c) sigma[c] = sqrt(std::max(0.0, hl[c]));
    }
    return DDG_OK;
}

}  // namespace ddg

using namespace ddg;

extern "C" ddg_status pca_fit(ddg_context* ctx, const double* F, long long D, int M, int k, double* U,
                              double* sigma, void* stream) {
    if (!ctx || !F || !U) { set_error("pca_fit: NULL argument"); return DDG_EINVAL; }
    if (D < 1 || M < 1 || k < 1 || k > kPcaMaxK || k > M || (long long)M > D || M > 8192) {
        set_error("pca_fit: need 1 <= k <= min(%d, M), M <= D, M <= 8192 (D=%lld M=%d k=%d)", kPcaMaxK, D, M, k);
        return DDG_EINVAL;
    }
    return pca_fit_impl(reinterpret_cast<Context*>(ctx), reinterpret_cast<const double2*>(F), D, M, k,
                        reinterpret_cast<double2*>(U), sigma, as_stream(stream));
}
