// FDFD operator A(eps, omega) of Eq. 1 (Sec. II): set-up, matrix-free
// application (5-point stencil with 1D stretched-coordinate PML coefficients)
// and the line-current source.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <new>

#include "common.cuh"

namespace ddg {

// ---------------------------------------------------------------- set-up kernels
// Stretch factor s(p) = 1 - i smax (d(p)/L)^m at coordinate p (cells) of a
// periodic line of n cells; d(p) = max(L - p, p - (n - L), 0).
__device__ __forceinline__ double2 stretch_at(double p, int n, int L, double smax, double m) {
    if (L <= 0) return make_double2(1.0, 0.0);
    double d = fmax(fmax((double)L - p, p - (double)(n - L)), 0.0);
    double sg = smax * pow(d / (double)L, m);
    return make_double2(1.0, -sg);
}

// One thread per index of x (t < nx) then y (t >= nx): coefficients
// ap_t = 1/(sb_t sf_t), am_t = 1/(sb_t sf_{t-1}) in FP64 and FP32.
__global__ void k_pml_coef(int nx, int ny, int Lx, int Ly, double smx, double smy, double m,
                           double2* coef_d, float2* coef_f, double2* sb_d, float2* sb_f) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx + ny) return;
    const bool isx = t < nx;
    const int i = isx ? t : t - nx;
    const int n = isx ? nx : ny;
    const int L = isx ? Lx : Ly;
    const double sm = isx ? smx : smy;
    double2 sb = stretch_at((double)i, n, L, sm, m);
    double2 sf = stretch_at((double)i + 0.5, n, L, sm, m);
    int im = (i == 0) ? n - 1 : i - 1;
    double2 sfm = stretch_at((double)im + 0.5, n, L, sm, m);
    const double2 one = make_double2(1.0, 0.0);
    double2 ap = cdiv(one, cmul(sb, sf));
    double2 am = cdiv(one, cmul(sb, sfm));
    double2* cd = coef_d + (isx ? 0 : 2 * nx);
    float2* cf = coef_f + (isx ? 0 : 2 * nx);
    cd[i] = ap;
    cd[n + i] = am;
    cf[i] = make_float2((float)ap.x, (float)ap.y);
    cf[n + i] = make_float2((float)am.x, (float)am.y);
    sb_d[t] = sb;
    sb_f[t] = make_float2((float)sb.x, (float)sb.y);
}

// Copies eps to the operator (FP64 and FP32) and flags non-finite / non-positive values.
__global__ void k_eps_copy(const double* __restrict__ eps, long long D, double* eps_d, float* eps_f,
                           int* bad) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= D) return;
    double v = eps[e];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(bad, 1);
    eps_d[e] = v;
    eps_f[e] = (float)v;
}

// ---------------------------------------------------------------- stencil
// y = A x.  One thread per cell; coefficients of row i / column j come from the
// 1D arrays (L1-resident), eps per cell.  diag = axp+axm+ayp+aym - (k0h)^2 eps.
template <typename T>
__global__ void __launch_bounds__(256) k_apply(int nx, int ny, const T* __restrict__ eps,
                                               const c2_t<T>* __restrict__ coef, T kh2,
                                               const c2_t<T>* __restrict__ x, c2_t<T>* __restrict__ y) {
    using V = c2_t<T>;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long D = (long long)nx * ny;
    if (e >= D) return;
    int j = (int)(e / nx);
    int i = (int)(e - (long long)j * nx);
    const V axp = coef[i], axm = coef[nx + i];
    const V ayp = coef[2 * nx + j], aym = coef[2 * nx + ny + j];
    const long long ip = (i == nx - 1) ? e - (nx - 1) : e + 1;
    const long long im = (i == 0) ? e + (nx - 1) : e - 1;
    const long long jp = (j == ny - 1) ? e - (long long)(ny - 1) * nx : e + nx;
    const long long jm = (j == 0) ? e + (long long)(ny - 1) * nx : e - nx;
    V xc = x[e];
    V d = cadd(cadd(axp, axm), cadd(ayp, aym));
    d.x -= kh2 * eps[e];
    V acc = cmul(d, xc);
    cfms(acc, axp, x[ip]);
    cfms(acc, axm, x[im]);
    cfms(acc, ayp, x[jp]);
    cfms(acc, aym, x[jm]);
    y[e] = acc;
}

// y = A x in complex64 for even nx: two cells and four rows per thread with
// 16-byte loads and stores.  Thread t of row group blockIdx.y owns cells
// i0 = 2 (blockIdx.x blockDim.x + t) and i0 + 1 of rows j0 .. j0 + 3
// (j0 = 4 blockIdx.y).  Every load is issued before any arithmetic: the six
// rows j0 - 1 .. j0 + 4 of the thread's two cells (each x row is read by
// 6/4 row groups instead of 3 times, the halo rows from L2), the four eps
// pairs, and at a warp edge or a row end the neighbouring pair of each row.
// The x-neighbours i0 - 1 and i0 + 2 come from the neighbouring lanes by
// shuffles.  eps (read once) and y (written once) bypass L2 retention
// (evict-first loads, streaming stores) so that L2 keeps the x rows that the
// next row group reads again.  Rows past ny load a valid row and store
// nothing.  Same arithmetic and order as k_apply<float> per cell.
constexpr int kApplyRows = 4;
__global__ void __launch_bounds__(256) k_apply_c64_rows(int nx, int ny, const float* __restrict__ eps,
                                                        const float2* __restrict__ coef, float kh2,
                                                        const float4* __restrict__ x, float4* __restrict__ y) {
    constexpr int R = kApplyRows;
    const int j0 = blockIdx.y * R;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;   // pair index in the row
    const int nh = nx >> 1;
    const int lane = threadIdx.x & 31;
    const bool in = h < nh;
    const int hh = in ? h : nh - 1;                         // out-of-row lanes mirror the last pair
    const bool ledge = lane == 0 || hh == 0;
    const bool redge = lane == 31 || hh == nh - 1 || h + 1 >= nh;
    const int hl = hh == 0 ? nh - 1 : hh - 1, hr = hh == nh - 1 ? 0 : hh + 1;   // periodic in x
    float4 xr[R + 2];                                       // rows j0 - 1 .. j0 + R
#pragma unroll
    for (int q = 0; q < R + 2; ++q) {
        int r = j0 - 1 + q;
        if (r < 0) r += ny;                                 // periodic in y
        else if (r >= ny) r = (r == ny) ? 0 : ny - 1;       // row ny wraps; later rows feed no output
        xr[q] = __ldg(&x[(long long)r * nh + hh]);
    }
    float4 lv[R], rv[R];
    float2 ev[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int r = min(j0 + q, ny - 1);
        const long long row = (long long)r * nh;
        lv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        rv[q] = lv[q];
        if (ledge) lv[q] = __ldg(&x[row + hl]);
        if (redge) rv[q] = __ldg(&x[row + hr]);
        ev[q] = __ldcs(reinterpret_cast<const float2*>(eps) + row + hh);
    }
    const float4 axp2 = reinterpret_cast<const float4*>(coef)[hh];        // axp of cells 2hh, 2hh + 1
    const float4 axm2 = reinterpret_cast<const float4*>(coef + nx)[hh];   // axm of the same cells
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int j = j0 + q;
        const float4 c = xr[q + 1], up = xr[q + 2], dn = xr[q];
        // left neighbour of cell 2hh: the .zw of pair hh - 1; right of 2hh + 1: the .xy of pair hh + 1
        float lx = __shfl_up_sync(0xffffffffu, c.z, 1), ly = __shfl_up_sync(0xffffffffu, c.w, 1);
        float rx = __shfl_down_sync(0xffffffffu, c.x, 1), ry = __shfl_down_sync(0xffffffffu, c.y, 1);
        if (ledge) {
            lx = lv[q].z;
            ly = lv[q].w;
        }
        if (redge) {
            rx = rv[q].x;
            ry = rv[q].y;
        }
        if (!in || j >= ny) continue;                       // after the shuffles: every lane takes part
        const float2 ayp = coef[2 * nx + j], aym = coef[2 * nx + ny + j];
        float2 out[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float2 axp = s == 0 ? make_float2(axp2.x, axp2.y) : make_float2(axp2.z, axp2.w);
            const float2 axm = s == 0 ? make_float2(axm2.x, axm2.y) : make_float2(axm2.z, axm2.w);
            float2 d = cadd(cadd(axp, axm), cadd(ayp, aym));
            d.x -= kh2 * (s == 0 ? ev[q].x : ev[q].y);
            const float2 xc = s == 0 ? make_float2(c.x, c.y) : make_float2(c.z, c.w);
            const float2 xe = s == 0 ? make_float2(c.z, c.w) : make_float2(rx, ry);
            const float2 xw = s == 0 ? make_float2(lx, ly) : make_float2(c.x, c.y);
            float2 acc = cmul(d, xc);
            cfms(acc, axp, xe);
            cfms(acc, axm, xw);
            cfms(acc, ayp, s == 0 ? make_float2(up.x, up.y) : make_float2(up.z, up.w));
            cfms(acc, aym, s == 0 ? make_float2(dn.x, dn.y) : make_float2(dn.z, dn.w));
            out[s] = acc;
        }
        __stcs(&y[(long long)j * nh + h], make_float4(out[0].x, out[0].y, out[1].x, out[1].y));
    }
}

__global__ void k_source(int nx, int ny, int i_src, double sigma, double j_c, double kh,
                         double2* __restrict__ b) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long D = (long long)nx * ny;
    if (e >= D) return;
    int j = (int)(e / nx);
    int i = (int)(e - (long long)j * nx);
    double v = 0.0;
    if (i == i_src) {
        double t = ((double)j - j_c);
        v = exp(-t * t / (2.0 * sigma * sigma));
    }
    b[e] = make_double2(0.0, -kh * v);
}

ddg_status launch_apply_d(const ddg_op* A, const double2* x, double2* y, cudaStream_t s) {
    unsigned nb = (unsigned)((A->D + 255) / 256);
    k_apply<double><<<nb, 256, 0, s>>>(A->nx, A->ny, A->eps_d, A->coef_d, A->kh * A->kh, x, y);
    DDG_CHECK_LAUNCH("k_apply<double>");
    return DDG_OK;
}

ddg_status launch_apply_f(const ddg_op* A, const float2* x, float2* y, cudaStream_t s) {
    if ((A->nx & 1) == 0 && A->nx >= 4 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)y & 15) == 0) {
        const int nh = A->nx / 2;
        dim3 grid((unsigned)((nh + 255) / 256), (unsigned)((A->ny + kApplyRows - 1) / kApplyRows));
        k_apply_c64_rows<<<grid, 256, 0, s>>>(A->nx, A->ny, A->eps_f, A->coef_f, (float)(A->kh * A->kh),
                                              reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(y));
        DDG_CHECK_LAUNCH("k_apply_c64_rows");
        return DDG_OK;
    }
    unsigned nb = (unsigned)((A->D + 255) / 256);
    k_apply<float><<<nb, 256, 0, s>>>(A->nx, A->ny, A->eps_f, A->coef_f, (float)(A->kh * A->kh), x, y);
    DDG_CHECK_LAUNCH("k_apply<float>");
    return DDG_OK;
}

static void free_op(ddg_op* A) {
    if (!A) return;
    cudaFree(A->eps_d);
    cudaFree(A->eps_f);
    cudaFree(A->coef_d);
    cudaFree(A->coef_f);
    cudaFree(A->sb_d);
    cudaFree(A->sb_f);
    delete A;
}

}  // namespace ddg

using namespace ddg;

extern "C" ddg_status fdfd_operator(const ddg_grid* g, const double* eps, ddg_op** out, void* stream) {
    if (!out) { set_error("fdfd_operator: out is NULL"); return DDG_EINVAL; }
    *out = nullptr;
    if (!g || !eps) { set_error("fdfd_operator: NULL grid or eps"); return DDG_EINVAL; }
    if (g->nx < 3 || g->ny < 3 || g->npml_x < 0 || g->npml_y < 0 || 2 * g->npml_x > g->nx ||
        2 * g->npml_y > g->ny || !(g->dx > 0) || !(g->wavelength > 0) || !(g->pml_order >= 0) ||
        !(g->pml_R > 0 && g->pml_R < 1) || !std::isfinite(g->dx) || !std::isfinite(g->wavelength)) {
        set_error("fdfd_operator: invalid grid (nx=%d ny=%d npml=%d,%d dx=%g wl=%g order=%g R=%g)", g->nx,
                  g->ny, g->npml_x, g->npml_y, g->dx, g->wavelength, g->pml_order, g->pml_R);
        return DDG_EINVAL;
    }
    if ((long long)g->nx * g->ny >= (1ll << 31)) {   // the kernels index cells with 32-bit division
        set_error("fdfd_operator: nx*ny = %lld cells, at most 2^31 - 1", (long long)g->nx * g->ny);
        return DDG_EINVAL;
    }
    cudaStream_t s = as_stream(stream);
    ddg_op* A = new (std::nothrow) ddg_op();
    if (!A) return DDG_ENOMEM;
    A->nx = g->nx;
    A->ny = g->ny;
    A->D = (long long)g->nx * g->ny;
    A->dx = g->dx;
    A->wavelength = g->wavelength;
    A->kh = 2.0 * M_PI / g->wavelength * g->dx;
    A->npml_x = g->npml_x;
    A->npml_y = g->npml_y;
    A->pml_order = g->pml_order;
    A->pml_R = g->pml_R;
    cudaGetDevice(&A->device);
    int ncoef = 2 * (g->nx + g->ny);
    int* bad = nullptr;
    cudaError_t e1 = cudaMalloc(&A->eps_d, A->D * sizeof(double));
    cudaError_t e2 = cudaMalloc(&A->eps_f, A->D * sizeof(float));
    cudaError_t e3 = cudaMalloc(&A->coef_d, ncoef * sizeof(double2));
    cudaError_t e4 = cudaMalloc(&A->coef_f, ncoef * sizeof(float2));
    cudaError_t e5 = cudaMalloc(&bad, sizeof(int));
    cudaError_t e6 = cudaMalloc(&A->sb_d, (g->nx + g->ny) * sizeof(double2));
    cudaError_t e7 = cudaMalloc(&A->sb_f, (g->nx + g->ny) * sizeof(float2));
    if (e1 || e2 || e3 || e4 || e5 || e6 || e7) {
        cudaGetLastError();
        cudaFree(bad);
        free_op(A);
        set_error("fdfd_operator: cudaMalloc failed");
        return DDG_ENOMEM;
    }
    double smx = g->npml_x > 0 ? -(g->pml_order + 1.0) * std::log(g->pml_R) / (2.0 * A->kh * g->npml_x) : 0.0;
    double smy = g->npml_y > 0 ? -(g->pml_order + 1.0) * std::log(g->pml_R) / (2.0 * A->kh * g->npml_y) : 0.0;
    int h_bad = 0;
    cudaError_t ce = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (ce == cudaSuccess) {
        k_pml_coef<<<(g->nx + g->ny + 127) / 128, 128, 0, s>>>(g->nx, g->ny, g->npml_x, g->npml_y, smx, smy,
                                                             g->pml_order, A->coef_d, A->coef_f, A->sb_d, A->sb_f);
        k_eps_copy<<<(unsigned)((A->D + 255) / 256), 256, 0, s>>>(eps, A->D, A->eps_d, A->eps_f, bad);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(bad);
    if (ce != cudaSuccess) {
        free_op(A);
        return cuda_status(ce, "fdfd_operator");
    }
    if (h_bad) {
        free_op(A);
        set_error("fdfd_operator: eps has a non-finite or non-positive value");
        return DDG_EINVAL;
    }
    *out = A;
    return DDG_OK;
}

extern "C" ddg_status fdfd_operator_destroy(ddg_op* A) {
    free_op(A);
    return DDG_OK;
}

extern "C" long long fdfd_operator_size(const ddg_op* A) { return A ? A->D : 0; }

extern "C" ddg_status fdfd_apply(const ddg_op* A, const double* x, double* y, void* stream) {
    if (!A || !x || !y) { set_error("fdfd_apply: NULL argument"); return DDG_EINVAL; }
    if (x == y) { set_error("fdfd_apply: x and y overlap"); return DDG_EINVAL; }
    return launch_apply_d(A, reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(y),
                          as_stream(stream));
}

extern "C" ddg_status fdfd_apply_c64(const ddg_op* A, const float* x, float* y, void* stream) {
    if (!A || !x || !y) { set_error("fdfd_apply_c64: NULL argument"); return DDG_EINVAL; }
    if (x == y) { set_error("fdfd_apply_c64: x and y overlap"); return DDG_EINVAL; }
    return launch_apply_f(A, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y),
                          as_stream(stream));
}

extern "C" ddg_status fdfd_source(const ddg_op* A, int i_src, double sigma, double j_c, double* b,
                                  void* stream) {
    if (!A || !b) { set_error("fdfd_source: NULL argument"); return DDG_EINVAL; }
    if (i_src < 0 || i_src >= A->nx || !(sigma > 0) || !std::isfinite(j_c)) {
        set_error("fdfd_source: i_src=%d outside [0,%d) or sigma=%g <= 0", i_src, A->nx, sigma);
        return DDG_EINVAL;
    }
    k_source<<<(unsigned)((A->D + 255) / 256), 256, 0, as_stream(stream)>>>(
        A->nx, A->ny, i_src, sigma, j_c, A->kh, reinterpret_cast<double2*>(b));
    DDG_CHECK_LAUNCH("k_source");
    return DDG_OK;
}
