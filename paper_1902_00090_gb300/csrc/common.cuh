// Shared device/host helpers of the ddgmres library: complex arithmetic on
// float2/double2, status plumbing and launch checks.
#pragma once
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdint>
#include <string>

#include "../../include/ddgmres.h"

namespace ddg {

// ---------------------------------------------------------------- complex math
template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <typename T> using c2_t = typename C2<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) {
    return mk(a.x * s, a.y * s);
}
// acc += a * b
template <typename V> __host__ __device__ __forceinline__ void cfma(V& acc, V a, V b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename V> __host__ __device__ __forceinline__ void cfms(V& acc, V a, V b) {
    acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename V> __host__ __device__ __forceinline__ void cfmac(V& acc, V a, V b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
template <typename V> __host__ __device__ __forceinline__ double cabs2(V a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm (R. L. Smith, CACM 5(8), 1962) for a / b.
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.y + b.x * r;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d2(double2 a) { return a; }
template <typename V> __host__ __device__ __forceinline__ V from_d2(double2 a);
template <> __host__ __device__ __forceinline__ float2 from_d2<float2>(double2 a) {
    return make_float2((float)a.x, (float)a.y);
}
template <> __host__ __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }

template <typename V> __device__ __forceinline__ V shfl_xor(V v, int m) {
    return mk(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
template <typename V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v = cadd(v, shfl_xor(v, m));
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
ddg_status cuda_status(cudaError_t e, const char* what);

#define DDG_CHECK_CUDA(call)                                              \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return ::ddg::cuda_status(_e, #call);      \
    } while (0)
#define DDG_CHECK_LAUNCH(name)                                            \
    do {                                                                  \
        cudaError_t _e = cudaGetLastError();                              \
        if (_e != cudaSuccess) return ::ddg::cuda_status(_e, name);       \
    } while (0)
#define DDG_TRY(expr)                                                     \
    do {                                                                  \
        ddg_status _s = (expr);                                           \
        if (_s != DDG_OK) return _s;                                      \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace ddg

// ---------------------------------------------------------------- operator handle
struct ddg_op {
    int nx = 0, ny = 0;
    long long D = 0;
    double dx = 0, wavelength = 0, kh = 0;  // kh = k0 h
    int npml_x = 0, npml_y = 0;
    double pml_order = 3, pml_R = 1e-8;
    int device = 0;
    double* eps_d = nullptr;     // D doubles
    float* eps_f = nullptr;      // D floats
    // stencil coefficients: [axp(nx) | axm(nx) | ayp(ny) | aym(ny)]
    //   axp_i = 1/(sxb_i sxf_i), axm_i = 1/(sxb_i sxf_{i-1}), same along y
    double2* coef_d = nullptr;
    float2* coef_f = nullptr;
    // stretch factors at integer nodes: [sxb(nx) | syb(ny)]; diag(sxb_i syb_j) A is
    // complex symmetric, which gives A^T = S_b A S_b^-1
    double2* sb_d = nullptr;
    float2* sb_f = nullptr;
};

namespace ddg {
// Stencil launchers shared by the operator API and the solver engine.
ddg_status launch_apply_d(const ddg_op* A, const double2* x, double2* y, cudaStream_t s);
ddg_status launch_apply_f(const ddg_op* A, const float2* x, float2* y, cudaStream_t s);
}  // namespace ddg
