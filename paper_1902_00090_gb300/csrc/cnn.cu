// Subspace-predicting CNN (Sec. III, "Convolutional neural network", Fig. 3a):
// permittivity and cheap input channels -> 2k real channels = k complex
// vectors v_1..v_k spanning the predicted subspace; trained on solved fields
// with the projection loss (Eq. 5) and Adam (Methods).
//
// Architecture (the paper gives none): `levels` resolutions, two 3x3
// convolutions + ReLU per level, 2x2 average pooling between encoder levels,
// nearest 2x upsampling concatenated with the encoder output of the same level
// in the decoder, a 1x1 head to 2k channels.  NHWC tensors; weights
// [Cout][Cin][3][3] then bias per layer, in the order enc0a, enc0b, ...,
// enc{L-1}b, dec{L-2}a, dec{L-2}b, ..., dec0b, head.
//
// Precision: FP32 master weights and Adam moments; BF16 copies of the weights
// and BF16 activations in the forward pass; FP32 accumulation; FP32 gradients.
// The forward 3x3 convolutions whose channel counts are multiples of 16 run on
// the 5th-generation tensor cores (tcgen05, accumulators in tensor memory);
// the first layer, the 1x1 head and the backward pass run on CUDA cores.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "bulk.cuh"
#include "engine.cuh"

using bf16 = __nv_bfloat16;

namespace ddg {
namespace cnn {

constexpr int kMaxLevels = 8;
constexpr int TX = 32, TY = 16;   // output tile (pixels)
constexpr int COB = 16;           // output channels per CTA
constexpr int CIB = 8;            // input channels per shared-memory chunk

struct Layer {
    int co, ci, kk;
    long long w_off, b_off;
};

// ---------------------------------------------------------------- input loaders
// Forward / weight-gradient input: channels [0, c1) from x1 (half resolution
// when up1: nearest upsampling), channels [c1, c1 + c2) from x2.
struct LoadCat {
    const bf16* x1;
    int c1, up1, h1, w1;  // dimensions of x1's own grid
    const bf16* x2;
    int c2;
    __device__ __forceinline__ float operator()(int b, int y, int x, int H, int W, int c) const {
        if (c < c1) {
            if (up1) return __bfloat162float(x1[(((long long)b * h1 + (y >> 1)) * w1 + (x >> 1)) * c1 + c]);
            return __bfloat162float(x1[(((long long)b * H + y) * W + x) * c1 + c]);
        }
        return __bfloat162float(x2[(((long long)b * H + y) * W + x) * c2 + (c - c1)]);
    }
    // channels c, c + 1 (c even, c1 even) as 2 packed BF16 values
    __device__ __forceinline__ uint32_t load2(int b, int y, int x, int H, int W, int c) const {
        const bf16* src;
        if (c < c1)
            src = up1 ? x1 + ((((long long)b * h1 + (y >> 1)) * w1 + (x >> 1)) * c1 + c)
                      : x1 + ((((long long)b * H + y) * W + x) * c1 + c);
        else
            src = x2 + ((((long long)b * H + y) * W + x) * c2 + (c - c1));
        return *reinterpret_cast<const uint32_t*>(src);
    }
    // channels c .. c + 7 (c % 8 == 0, c1 % 8 == 0) as 8 packed BF16 values
    __device__ __forceinline__ uint4 load8(int b, int y, int x, int H, int W, int c) const {
        const bf16* src;
        if (c < c1)
            src = up1 ? x1 + ((((long long)b * h1 + (y >> 1)) * w1 + (x >> 1)) * c1 + c)
                      : x1 + ((((long long)b * H + y) * W + x) * c1 + c);
        else
            src = x2 + ((((long long)b * H + y) * W + x) * c2 + (c - c1));
        return *reinterpret_cast<const uint4*>(src);
    }
};

// Gradient input of the backward-data convolution: g masked by ReLU'(out).
struct LoadGrad {
    const float* g;
    const bf16* y;   // forward output after ReLU (mask = y > 0)
    int C;
    __device__ __forceinline__ float operator()(int b, int yy, int x, int H, int W, int c) const {
        const long long i = (((long long)b * H + yy) * W + x) * C + c;
        return __bfloat162float(y[i]) > 0.f ? g[i] : 0.f;
    }
    // channels c .. c + 7 (c % 8 == 0, C % 8 == 0) of the masked gradient,
    // rounded to BF16 (the tensor-core operand type), packed
    __device__ __forceinline__ uint4 load8(int b, int yy, int x, int H, int W, int c) const {
        const long long i = (((long long)b * H + yy) * W + x) * C + c;
        const float4 g0 = *reinterpret_cast<const float4*>(g + i);
        const float4 g1 = *reinterpret_cast<const float4*>(g + i + 4);
        const uint4 yv = *reinterpret_cast<const uint4*>(y + i);
        const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
        const unsigned yw[4] = {yv.x, yv.y, yv.z, yv.w};
        unsigned o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 yb = *reinterpret_cast<const __nv_bfloat162*>(&yw[q]);
            const float a = __bfloat162float(yb.x) > 0.f ? gv[2 * q] : 0.f;
            const float bq = __bfloat162float(yb.y) > 0.f ? gv[2 * q + 1] : 0.f;
            __nv_bfloat162 h = __floats2bfloat162_rn(a, bq);
            o[q] = *reinterpret_cast<unsigned*>(&h);
        }
        return make_uint4(o[0], o[1], o[2], o[3]);
    }
};

__device__ __forceinline__ void store_out(bf16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_out(float* p, float v) { *p = v; }

// ---------------------------------------------------------------- 3x3 convolution
// out[b, y, x, co] = bias[co] + sum_{ci, dy, dx} in[b, y+dy-1, x+dx-1, ci] wk[ci][3 dy + dx][co]
// (zero padding), optional ReLU.  One CTA: a 32x16 pixel tile, 16 output
// channels; each thread two neighbouring pixels of one row.  wk is BF16
// [Ci][9][Co].
template <class LD, typename TOUT>
__global__ void __launch_bounds__(256) k_conv3(LD ld, int B, int H, int W, int Ci, int Co,
                                               const bf16* __restrict__ wk, const float* __restrict__ bias,
                                               int relu, TOUT* __restrict__ out) {
    __shared__ float s_in[CIB][TY + 2][TX + 2];
    __shared__ __align__(16) float s_w[CIB][9][COB];
    const int ncob = (Co + COB - 1) / COB;
    const int b = blockIdx.z / ncob, cob = blockIdx.z % ncob;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int t = threadIdx.x, ty = t >> 4, tx2 = (t & 15) * 2;
    float acc0[COB], acc1[COB];
#pragma unroll
    for (int c = 0; c < COB; ++c) acc0[c] = acc1[c] = 0.f;
    for (int c0 = 0; c0 < Ci; c0 += CIB) {
        __syncthreads();
        for (int idx = t; idx < CIB * (TY + 2) * (TX + 2); idx += 256) {
            const int c = idx / ((TY + 2) * (TX + 2));
            const int r = (idx / (TX + 2)) % (TY + 2);
            const int q = idx % (TX + 2);
            const int yy = y0 + r - 1, xx = x0 + q - 1, ci = c0 + c;
            float v = 0.f;
            if (ci < Ci && yy >= 0 && yy < H && xx >= 0 && xx < W) v = ld(b, yy, xx, H, W, ci);
            s_in[c][r][q] = v;
        }
        for (int idx = t; idx < CIB * 9 * COB; idx += 256) {
            const int c = idx / (9 * COB), tap = (idx / COB) % 9, o = idx % COB;
            const int ci = c0 + c, co = cob * COB + o;
            s_w[c][tap][o] = (ci < Ci && co < Co) ? __bfloat162float(wk[((long long)ci * 9 + tap) * Co + co]) : 0.f;
        }
        __syncthreads();
#pragma unroll 2
        for (int c = 0; c < CIB; ++c) {
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const float v0 = s_in[c][ty + dy][tx2 + dx];
                    const float v1 = s_in[c][ty + dy][tx2 + 1 + dx];
                    const float4* wp = reinterpret_cast<const float4*>(&s_w[c][dy * 3 + dx][0]);
#pragma unroll
                    for (int q = 0; q < COB / 4; ++q) {
                        const float4 w4 = wp[q];
                        acc0[4 * q + 0] = fmaf(v0, w4.x, acc0[4 * q + 0]);
                        acc0[4 * q + 1] = fmaf(v0, w4.y, acc0[4 * q + 1]);
                        acc0[4 * q + 2] = fmaf(v0, w4.z, acc0[4 * q + 2]);
                        acc0[4 * q + 3] = fmaf(v0, w4.w, acc0[4 * q + 3]);
                        acc1[4 * q + 0] = fmaf(v1, w4.x, acc1[4 * q + 0]);
                        acc1[4 * q + 1] = fmaf(v1, w4.y, acc1[4 * q + 1]);
                        acc1[4 * q + 2] = fmaf(v1, w4.z, acc1[4 * q + 2]);
                        acc1[4 * q + 3] = fmaf(v1, w4.w, acc1[4 * q + 3]);
                    }
                }
            }
        }
    }
    const int y = y0 + ty;
    if (y >= H) return;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int x = x0 + tx2 + p;
        if (x >= W) continue;
        TOUT* o = out + (((long long)b * H + y) * W + x) * Co;
#pragma unroll
        for (int c = 0; c < COB; ++c) {
            const int co = cob * COB + c;
            if (co >= Co) break;
            float v = (p == 0 ? acc0[c] : acc1[c]) + (bias ? bias[co] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            store_out(o + co, v);
        }
    }
}

// ---------------------------------------------------------------- 3x3 convolution on tensor cores
// Implicit GEMM: D[p, co] = sum_k A[p, k] Wt[co, k], k = tap * Ci + ci (tap =
// 3 dy + dx), A[p, k] = in[b, y + dy - 1, x + dx - 1, ci] (zero outside the
// grid; the input may be the concatenation of a nearest-upsampled x1 and x2).
// One CTA: 128 consecutive pixels (M = 128) x all Co output channels (N = Co).
// K streams through two shared-memory stages of 64: all 256 threads gather the
// im2col tile and the weight tile with 16-byte loads into the K-major layout
// with 128-byte swizzle (one 128-byte row of 64 K values per pixel / output
// channel, its 16-byte chunks permuted by XOR with row % 8, 8-row atoms of
// 1024 bytes), so that the 8 threads writing one row fill one line; one
// thread issues tcgen05.mma (BF16 x BF16 -> FP32 in tensor memory, K = 16 per
// instruction, the descriptor advanced 32 bytes per step) and commits each
// stage to an mbarrier, so the gather of the next stage overlaps the MMAs of
// this one.  Epilogue: tcgen05.ld of the accumulator rows, bias, ReLU, BF16
// NHWC stores.
namespace tc {
constexpr int kM = 128;
constexpr int kKC = 64;
constexpr int kStages = 2;
constexpr int kThreads = 256;
constexpr uint32_t kRowBytes = kKC * 2;      // one swizzled row: 64 BF16 = 128 bytes
constexpr uint32_t kSBO = 8 * kRowBytes;     // adjacent 8-row atoms (1024 bytes)
constexpr uint32_t kABytes = kM * kKC * 2;
static_assert(kRowBytes == 128, "one K stage is one 128-byte swizzle row");

// stages (1024-byte aligned atoms: the dynamic base is rounded up in the kernel)
__host__ __device__ constexpr size_t smem_bytes(int co) { return (size_t)kStages * (kABytes + (size_t)co * kKC * 2) + 1024; }
// byte offset of 16-byte chunk `kg` of row `r` in a swizzled K-major tile
__device__ __forceinline__ uint32_t swz(int r, int kg) {
    return (uint32_t)(r >> 3) * kSBO + (uint32_t)(r & 7) * kRowBytes + ((uint32_t)(kg ^ (r & 7)) << 4);
}
__host__ __device__ constexpr uint32_t tmem_cols(int co) { return co <= 32 ? 32u : co <= 64 ? 64u : co <= 128 ? 128u : 256u; }

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// start address, leading byte offset (unused for this layout, 16 bytes),
// stride byte offset between 8-row atoms (1024), descriptor version 1, base
// offset 0 (atoms 1024-byte aligned), layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n (multiple of 16), M = 128.
__host__ __device__ constexpr uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
}  // namespace tc

// The gather G supplies 8 BF16 input channels per 16-byte chunk (LoadCat: the
// forward's activations; LoadGrad: the backward-data convolution's input, the
// FP32 gradient masked by ReLU' and rounded to BF16); TOUT is the output type
// (BF16 activations, or the FP32 input gradient).
template <class G, typename TOUT>
__global__ void __launch_bounds__(tc::kThreads) k_conv3_tc(G ld, int B, int H, int W, int Ci, int Co,
                                                           const bf16* __restrict__ wt, const float* __restrict__ bias,
                                                           int relu, TOUT* __restrict__ out, int* __restrict__ err) {
    using namespace tc;
    constexpr int kRowsPerThread = kM * 8 / kThreads;   // A rows gathered by one thread (fixed K group)
    extern __shared__ __align__(128) unsigned char smraw_tc[];
    __shared__ __align__(8) unsigned long long done[kStages];
    __shared__ uint32_t s_tmem;
    // swizzle atoms must start on 1024-byte boundaries
    unsigned char* smt = smraw_tc + ((1024u - (smem_u32(smraw_tc) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = B * H * W;
    const int p0 = blockIdx.x * kM;
    const int K = 9 * Ci;
    const int nch = (K + kKC - 1) / kKC;
    const uint32_t ncols = tmem_cols(Co);
    const uint32_t st_bytes = kABytes + (uint32_t)Co * kKC * 2;
    // this thread's K group and rows: row r = tid / 8 + (kThreads / 8) j
    const int kg = tid & 7, r0 = tid >> 3;
    int rb[kRowsPerThread], ryx[kRowsPerThread];   // image, and (y << 16 | x); b < 0: past the end
#pragma unroll
    for (int j = 0; j < kRowsPerThread; ++j) {
        const int p = p0 + r0 + (kThreads / 8) * j;
        if (p < P) {
            const int x = p % W, t = p / W;
            rb[j] = t / H;
            ryx[j] = ((t % H) << 16) | x;
        } else {
            rb[j] = -1;
            ryx[j] = 0;
        }
    }
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&done[q], 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
        const int s = c % kStages;
        unsigned char* As = smt + s * st_bytes;
        unsigned char* Bs = As + kABytes;
        // the MMAs that last read this stage are complete
        if (c >= kStages && !mbar_wait(&done[s], (unsigned)((c - kStages) / kStages) & 1u)) ok = false;
        const int k0 = c * kKC + kg * 8;
        const bool kin = k0 < K;
        int ci = 0, dy = 0, dx = 0;
        if (kin) {
            const int tap = k0 / Ci;
            ci = k0 - tap * Ci;
            dy = tap / 3 - 1;
            dx = tap - 3 * (tap / 3) - 1;
        }
#pragma unroll
        for (int j = 0; j < kRowsPerThread; ++j) {
            const int r = r0 + (kThreads / 8) * j;
            const int b = rb[j];
            const int yy = (ryx[j] >> 16) + dy, xx = (ryx[j] & 0xFFFF) + dx;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (kin && b >= 0 && yy >= 0 && yy < H && xx >= 0 && xx < W) v = ld.load8(b, yy, xx, H, W, ci);
            *reinterpret_cast<uint4*>(As + swz(r, kg)) = v;
        }
        for (int n = r0; n < Co; n += kThreads / 8) {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (kin) v = *reinterpret_cast<const uint4*>(wt + (long long)n * K + k0);
            *reinterpret_cast<uint4*>(Bs + swz(n, kg)) = v;
        }
        fence_proxy_async_smem();   // these shared-memory writes, before the tensor core reads them
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
            for (int ks = 0; ks < kKC / 16; ++ks)
                mma(tmem, sdesc(a0 + ks * 32), sdesc(b0 + ks * 32), idesc(Co), (c > 0 || ks > 0) ? 1u : 0u);
            commit(&done[s]);
        }
    }
    // the last commit completes once every MMA issued before it has
    const int cl = nch - 1;
    if (!mbar_wait(&done[cl % kStages], (unsigned)(cl / kStages) & 1u)) {
        ok = false;
        mbar_wait(&done[cl % kStages], (unsigned)(cl / kStages) & 1u);   // one more bounded wait before freeing
    }
    fence_after();
    // warp w reads tensor-memory lanes 32 (w % 4) .. +31 (accumulator rows),
    // columns [half, half + Co/2) with half = (w / 4) Co/2
    const int quarter = warp & 3, chalf = (warp >> 2) * (Co / 2);
    const int p = p0 + quarter * 32 + lane;
    for (int c0 = chalf; c0 < chalf + Co / 2; c0 += 8) {
        uint32_t rr[8];
        ld8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, rr);
        if (p < P) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = __uint_as_float(rr[j]) + (bias ? bias[c0 + j] : 0.f);
                if (relu) v[j] = fmaxf(v[j], 0.f);
            }
            if constexpr (sizeof(TOUT) == 4) {
                float4* o4 = reinterpret_cast<float4*>(out + (long long)p * Co + c0);
                o4[0] = make_float4(v[0], v[1], v[2], v[3]);
                o4[1] = make_float4(v[4], v[5], v[6], v[7]);
            } else {
                uint4 o;
                __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]), h1 = __floats2bfloat162_rn(v[2], v[3]);
                __nv_bfloat162 h2 = __floats2bfloat162_rn(v[4], v[5]), h3 = __floats2bfloat162_rn(v[6], v[7]);
                o.x = *reinterpret_cast<uint32_t*>(&h0);
                o.y = *reinterpret_cast<uint32_t*>(&h1);
                o.z = *reinterpret_cast<uint32_t*>(&h2);
                o.w = *reinterpret_cast<uint32_t*>(&h3);
                *reinterpret_cast<uint4*>(out + (long long)p * Co + c0) = o;
            }
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// ---------------------------------------------------------------- 3x3 convolution from TMA tiles
// The forward convolutions whose input is one plain NHWC tensor (no
// upsampled concatenation) as an implicit GEMM without any gather: one output
// tile of 16 rows x 8 columns = 128 pixels (M = 128) x all Co channels.  Its
// 18 x 10 halo tile is loaded by TMA (cp.async.bulk.tensor, 4D tensor map
// over (C, W, H, B), one copy per 8-channel chunk, zeros outside the image =
// the convolution's padding) into the layout [Ci/8][18][10][8 channels].  In
// that layout every tap (dy, dx) of the A operand is the same tile seen from
// another start address: a K-major operand without swizzle whose 8-row core
// matrices are 8 consecutive pixels of one tile row (16 bytes apart), whose
// 8-row groups (the tile's rows) are 10 pixels = 160 bytes apart (SBO) and
// whose 8-channel K groups are one chunk apart (LBO).  So the MMAs read the
// 9 taps straight from the loaded tile: 9 x Ci/16 tcgen05.mma of K = 16 per
// tile.  The weights (B, K-major [9 Ci/8][Co][8], k = tap Ci + ci) are loaded
// once per CTA by a bulk copy and stay in shared memory; each CTA walks the
// tiles blockIdx.x, + gridDim.x, ...
//
// Warp roles (no block-wide barrier between tiles): warp 0's lane 0 requests
// the tiles and issues the MMAs (two input buffers, two tensor-memory
// accumulators); warps 1-4 (tensor-memory lane quarters 1, 2, 3, 0) read an
// accumulator out (tcgen05.ld, bias, ReLU, BF16 NHWC stores) and release it.
//   full[s]    input buffer s loaded (TMA transaction count)
//   mdone[s]   the MMAs of the tile in buffer / accumulator s complete
//              (tcgen05.commit): accumulator ready, input buffer free
//   accfree[s] the 4 epilogue warps have read accumulator s out
// Every wait is bounded; one that gives up raises the error flag and the
// abort word, and the CTA waits (at the default bound) for its own copies and
// MMAs before it frees the tensor memory.
namespace tmc {
constexpr int TH = 16, TW = 8;                  // output tile: rows x columns (M = 128)
constexpr int HH = TH + 2, HWD = TW + 2;        // halo tile
constexpr uint32_t kChunkBytes = HH * HWD * 16; // one 8-channel chunk of a halo tile (2880)
constexpr uint32_t kChunkStride = 2944;         // chunks 128-byte aligned (TMA destinations)
constexpr int kBufs = 2;                        // input buffers = accumulators
constexpr int kEpiWarps = 4;
constexpr int kExpWarps = 4;                    // upsampled inputs: warps that expand the coarse tile
constexpr int kThreads = 32 * (1 + kEpiWarps);
constexpr int kThreadsUp = 32 * (1 + kEpiWarps + kExpWarps);
// upsampled input: the coarse tile under an 18 x 10 fine halo tile (fine row
// y0 - 1 + hy is coarse row y0/2 - 1 + (hy + 1)/2, the same in x)
constexpr int CH = HH / 2 + 1, CW = HWD / 2 + 1;   // 10 x 6
constexpr uint32_t kCoarseBytes = CH * CW * 16;    // one 8-channel chunk (960)
constexpr uint32_t kCoarseStride = 1024;           // 128-byte aligned (TMA destinations)
static_assert(TH * TW == tc::kM && kChunkStride >= kChunkBytes && kChunkStride % 128 == 0, "tile geometry");
static_assert(kCoarseStride >= kCoarseBytes && kCoarseStride % 128 == 0, "coarse tile geometry");
__host__ __device__ constexpr uint32_t wbytes(int ci, int co) { return 9u * (uint32_t)ci * (uint32_t)co * 2u; }
__host__ __device__ constexpr uint32_t bufbytes(int ci) { return (uint32_t)(ci / 8) * kChunkStride; }
__host__ __device__ constexpr uint32_t cbufbytes(int c1) { return (uint32_t)(c1 / 8) * kCoarseStride; }
__host__ __device__ constexpr size_t smem_bytes(int ci, int co, int c1 = 0) {
    // + the base's round-up to 128
    return (size_t)wbytes(ci, co) + (size_t)kBufs * (bufbytes(ci) + cbufbytes(c1)) + 128;
}
// Shared-memory descriptor of a K-major operand without swizzle: start
// address, leading byte offset (between 8-element K groups), stride byte
// offset (between 8-row groups), descriptor version 1, layout type 0.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// TMA load of one box of a 4D tensor map into shared memory, completing on bar.
__device__ __forceinline__ void load4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                       unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 16 consecutive accumulator columns of this warp's 32 lanes (one wait for both halves)
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
}  // namespace tmc

// c1 > 0: the input is [nearest-upsampled x1 (c1 channels, half resolution,
// tensor map tup) | x2 (Ci - c1 channels, tensor map tin)]: the x2 chunks come
// by TMA as above, the x1 chunks as a coarse 10 x 6 tile (TMA, zeros outside)
// that warps 5-8 expand into the fine halo layout (each fine pixel copies its
// coarse parent), then make visible to the tensor core (proxy fence) and
// count on the buffer's "loaded" barrier.
__global__ void __launch_bounds__(tmc::kThreadsUp) k_conv3_tma(const __grid_constant__ CUtensorMap tin,
                                                               const __grid_constant__ CUtensorMap tup, int c1, int B,
                                                               int H, int W, int Ci, int Co,
                                                               const bf16* __restrict__ wt,
                                                               const float* __restrict__ bias, int relu,
                                                               bf16* __restrict__ out, int* __restrict__ err) {
    using namespace tmc;
    extern __shared__ __align__(128) unsigned char smraw_tm[];
    __shared__ __align__(8) unsigned long long wbar, full[kBufs], mdone[kBufs], accfree[kBufs], cfull[kBufs];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    unsigned char* sm = smraw_tm + ((128u - (smem_u32(smraw_tm) & 127u)) & 127u);
    unsigned char* wsm = sm;                        // weights [9 Ci/8][Co][8]
    unsigned char* ism = sm + wbytes(Ci, Co);       // kBufs halo tiles [Ci/8][18][10][8]
    unsigned char* csm = ism + kBufs * bufbytes(Ci); // kBufs coarse tiles [c1/8][10][6][8] (c1 > 0)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = W / TW, nty = H / TH;
    const long long ntiles = (long long)B * nty * ntx;
    const int nmine = ntiles > (long long)blockIdx.x ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const uint32_t acc_cols = tc::tmem_cols(Co);
    const uint32_t ncols = kBufs * acc_cols;
    const int nchunk = Ci / 8;
    auto tile_of = [&](int it, int& b, int& y0, int& x0) {
        const long long t = (long long)blockIdx.x + (long long)it * gridDim.x;
        x0 = (int)(t % ntx) * TW;
        const long long r = t / ntx;
        y0 = (int)(r % nty) * TH;
        b = (int)(r / nty);
    };
    if (tid == 0) {
        mbar_init(&wbar, 1);
        for (int q = 0; q < kBufs; ++q) {
            mbar_init(&full[q], 1 + (c1 > 0 ? kExpWarps : 0));   // the producer, and the expanding warps
            mbar_init(&mdone[q], 1);
            mbar_init(&accfree[q], kEpiWarps);
            mbar_init(&cfull[q], 1);
        }
        mbar_init_fence();
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = s_tmem;
    auto give_up = [&]() {
        atomicExch(err, 1);
        s_abort = 1;
    };
    if (tid == 0 && nmine > 0) {
        // producer: tiles into the input buffers, MMAs into the accumulators
        auto load_tile = [&](int t) {
            int b, y0, x0;
            tile_of(t, b, y0, x0);
            const int s = t % kBufs;
            unsigned char* dst = ism + s * bufbytes(Ci);
            const int n1 = c1 / 8;     // chunks from the upsampled input (0: a plain input)
            mbar_expect_tx(&full[s], (unsigned)(nchunk - n1) * kChunkBytes);
            for (int q = n1; q < nchunk; ++q)
                load4d(dst + q * kChunkStride, &tin, 8 * (q - n1), x0 - 1, y0 - 1, b, &full[s]);
            if (n1 > 0) {
                unsigned char* cdst = csm + s * cbufbytes(c1);
                mbar_expect_tx(&cfull[s], (unsigned)n1 * kCoarseBytes);
                for (int q = 0; q < n1; ++q)
                    load4d(cdst + q * kCoarseStride, &tup, 8 * q, x0 / 2 - 1, y0 / 2 - 1, b, &cfull[s]);
            }
        };
        mbar_expect_tx(&wbar, wbytes(Ci, Co));
        bulk_g2s(wsm, wt, wbytes(Ci, Co), &wbar);
        int issued = 0, committed = 0;
        for (; issued < min(kBufs, nmine); ++issued) load_tile(issued);
        const uint32_t id = tc::idesc(Co);
        bool ok = mbar_wait(&wbar, 0u);
        for (int t = 0; ok && t < nmine && !s_abort; ++t) {
            const int s = t % kBufs;
            const unsigned par = (unsigned)(t / kBufs) & 1u;
            // tile t loaded, and accumulator s read out (tile t - 2)
            if (!mbar_wait(&full[s], par) || (t >= kBufs && !mbar_wait(&accfree[s], par ^ 1u))) {
                ok = false;
                break;
            }
            tc::fence_after();
            const uint32_t in0 = smem_u32(ism + s * bufbytes(Ci)), w0 = smem_u32(wsm);
            const uint32_t d = tmem + (uint32_t)s * acc_cols;
            int n = 0;
            for (int tap = 0; tap < 9; ++tap) {
                const uint32_t aoff = (uint32_t)((tap / 3) * HWD + tap % 3) * 16u;
                for (int q = 0; q < Ci / 16; ++q, ++n) {
                    const uint64_t ad = desc(in0 + 2u * (uint32_t)q * kChunkStride + aoff, kChunkStride, HWD * 16u);
                    const uint64_t bd = desc(w0 + (uint32_t)(tap * nchunk + 2 * q) * (uint32_t)Co * 16u,
                                             (uint32_t)Co * 16u, 128u);
                    tc::mma(d, ad, bd, id, n > 0 ? 1u : 0u);
                }
            }
            tc::commit(&mdone[s]);
            committed = t + 1;
            // tile t + 2 into buffer s once tile t's MMAs have read it
            if (issued < nmine) {
                if (!mbar_wait(&mdone[s], par)) {
                    ok = false;
                    break;
                }
                load_tile(issued++);
            }
        }
        if (!ok) {
            // let every copy and MMA this CTA started finish before leaving
            give_up();
            mbar_wait(&wbar, 0u);
            for (int t = max(0, issued - kBufs); t < issued; ++t)
                mbar_wait(&full[t % kBufs], (unsigned)(t / kBufs) & 1u);
            if (committed > 0) mbar_wait(&mdone[(committed - 1) % kBufs], (unsigned)((committed - 1) / kBufs) & 1u);
        }
    } else if (warp > kEpiWarps) {
        // expanding warps (c1 > 0 only; the launch has them only then): fine
        // halo pixel (hy, hx) of chunk q <- coarse pixel ((hy + 1)/2, (hx + 1)/2)
        const int n1 = c1 / 8;
        const int et = tid - 32 * (1 + kEpiWarps), ne = 32 * kExpWarps;
        for (int t = 0; n1 > 0 && t < nmine && !s_abort; ++t) {
            const int s = t % kBufs;
            if (!mbar_wait(&cfull[s], (unsigned)(t / kBufs) & 1u)) {
                give_up();
                break;
            }
            const unsigned char* src = csm + s * cbufbytes(c1);
            unsigned char* dst = ism + s * bufbytes(Ci);
            for (int idx = et; idx < n1 * HH * HWD; idx += ne) {
                const int q = idx / (HH * HWD), rr = idx - q * (HH * HWD);
                const int hy = rr / HWD, hx = rr - hy * HWD;
                const uint4 v = *reinterpret_cast<const uint4*>(src + q * kCoarseStride +
                                                                ((hy + 1) / 2 * CW + (hx + 1) / 2) * 16);
                *reinterpret_cast<uint4*>(dst + q * kChunkStride + rr * 16) = v;
            }
            fence_proxy_async_smem();   // these writes, before the tensor core reads them
            __syncwarp();
            if (lane == 0) arrive(&full[s]);
        }
    } else if (warp >= 1) {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;          // accumulator row = pixel (r / 8, r % 8) of the tile
        for (int t = 0; t < nmine && !s_abort; ++t) {
            const int s = t % kBufs;
            if (!mbar_wait(&mdone[s], (unsigned)(t / kBufs) & 1u)) {
                give_up();
                break;
            }
            tc::fence_after();
            int b, y0, x0;
            tile_of(t, b, y0, x0);
            bf16* o = out + (((long long)b * H + y0 + (r >> 3)) * W + x0 + (r & 7)) * Co;
            for (int c0 = 0; c0 < Co; c0 += 16) {
                uint32_t rr[16];
                ld16(tmem + (uint32_t)s * acc_cols + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, rr);
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float v0 = __uint_as_float(rr[2 * j]) + (bias ? bias[c0 + 2 * j] : 0.f);
                    float v1 = __uint_as_float(rr[2 * j + 1]) + (bias ? bias[c0 + 2 * j + 1] : 0.f);
                    if (relu) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                    pk[j] = *reinterpret_cast<uint32_t*>(&h);
                }
                *reinterpret_cast<uint4*>(o + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4*>(o + c0 + 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
            // this warp's reads of accumulator s are complete: release it
            tc::fence_before();
            __syncwarp();
            if (lane == 0) arrive(&accfree[s]);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// TMA-tile weights BF16 [co][ci][9] (ci < Ci) -> [9 Cp/8][co][8] (k = tap Cp + ci:
// K group kc = tap Cp/8 + ci/8, then the output channel, then ci % 8), the
// input channels padded with zero weights to Cp >= Ci
__global__ void k_w_tma(const bf16* __restrict__ w, int Co, int Ci, int Cp, bf16* __restrict__ wt) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Co * Cp * 9) return;
    const int co = (int)(idx / (Cp * 9)), ci = (int)((idx / 9) % Cp), tap = (int)(idx % 9);
    wt[(((long long)(tap * (Cp / 8) + ci / 8) * Co + co) << 3) + (ci & 7)] =
        ci < Ci ? w[((long long)co * Ci + ci) * 9 + tap] : __float2bfloat16_rn(0.f);
}

// ---------------------------------------------------------------- weight gradient on tensor cores
// dW[co][ci][tap] = sum over pixels p of g'[p][co] x[p + off(tap)][ci], with
// g' the output gradient masked by ReLU'(out): a GEMM D[m = co, n] = sum_p
// A[co, p] B[n, p] with n = tap * Ci + ci and K = the pixels.  One CTA: all
// output channels (M = 128, rows >= Co zero) x a tile of kWN columns n, over a
// range of pixels in K stages of 64; both operands are gathered as 8-channel
// 16-byte chunks (g' in BF16 from FP32, x through the layer's input loader)
// and scattered, one BF16 value per (row, pixel), into the K-major 128-byte
// swizzled layout of the forward kernel; one thread issues the MMAs and
// commits each stage; the FP32 accumulators are added to dW with atomics
// (the CTAs of one n tile split the pixels).  The bias gradient is summed
// separately (k_bias_grad) from the FP32 g'.
namespace tcw {
constexpr int kWN = 128;                       // columns n per CTA
}  // namespace tcw
// Four 8x8 b16 matrices from registers (lane t: row t / 4, elements 2 (t % 4),
// +1 of each) to shared memory transposed: row i of matrix q (its column i)
// goes to the 16 bytes at the address held by lane 8 q + i.
__device__ __forceinline__ void stmatrix_x4_trans(uint32_t addr, const uint32_t (&r)[4]) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3])
                 : "memory");
}
namespace tcw {
constexpr uint32_t kTileBytes = tc::kM * tc::kKC * 2;   // 128 rows x 64 K values (A and B alike)
__host__ __device__ constexpr size_t smem_bytes() { return (size_t)tc::kStages * 2 * kTileBytes + 1024; }
}  // namespace tcw

template <class LX>
__global__ void __launch_bounds__(tc::kThreads) k_wgrad_tc(LX lx, const float* __restrict__ g,
                                                           const bf16* __restrict__ yout, int B, int H, int W, int Ci,
                                                           int Co, long long pix_per_cta, float* __restrict__ dW,
                                                           int* __restrict__ err) {
    using namespace tc;
    extern __shared__ __align__(128) unsigned char smraw_wg[];
    __shared__ __align__(8) unsigned long long done[kStages];
    __shared__ uint32_t s_tmem;
    unsigned char* smt = smraw_wg + ((1024u - (smem_u32(smraw_wg) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)B * H * W;
    const int Ntot = 9 * Ci;
    const int n0 = blockIdx.x * tcw::kWN;
    const long long p_begin = (long long)blockIdx.y * pix_per_cta;
    const long long p_end = min(P, p_begin + pix_per_cta);
    const int nch = p_end > p_begin ? (int)((p_end - p_begin + kKC - 1) / kKC) : 0;
    // rows co >= Co of A never receive data: zero both stages once
    for (int q = tid; q < kStages * 2 * (int)tcw::kTileBytes / 16; q += kThreads)
        reinterpret_cast<uint4*>(smt)[q] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&done[q], 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((uint32_t)tcw::kWN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    bool ok = true;
    // this lane's B columns n = n0 + 8 (4 (warp % 4) + q) + 2 (lane % 4), q < 4,
    // the same in every stage: input channel, tap offset (-1 for n past 9 Ci)
    int bci[4], bdy[4], bdx[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int n = n0 + 8 * (4 * (warp & 3) + q) + 2 * (lane & 3);
        const int tap = n / Ci;
        bci[q] = n < Ntot ? n - tap * Ci : -1;
        bdy[q] = tap / 3 - 1;
        bdx[q] = tap % 3 - 1;
    }
    for (int c = 0; c < nch; ++c) {
        const int s = c % kStages;
        unsigned char* As = smt + s * 2 * tcw::kTileBytes;
        unsigned char* Bs = As + tcw::kTileBytes;
        if (c >= kStages && !mbar_wait(&done[s], (unsigned)((c - kStages) / kStages) & 1u)) ok = false;
        const long long pc0 = p_begin + (long long)c * kKC;
        // Both operands are K-major in the pixels while the data are
        // pixel-major: each warp stores four 8x8 blocks (8 pixels x 8 rows of
        // the operand) at a time with stmatrix .trans, which writes every
        // operand row's 8 pixels as one 16-byte chunk of the swizzled tile.
        // Block f (x4 group of 4 per warp instruction): lane t holds pixel
        // 8 pb + t / 4 and the operand rows 8 rb + 2 (t % 4), +1; lane
        // 8 q + i gives the address of row i of block q.
        const int nfa = (Co >> 3) * (kKC / 8);          // A blocks: (Co / 8) row blocks x 8 pixel blocks
        for (int fg = warp; fg < nfa / 4; fg += kThreads / 32) {
            uint32_t r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int f = fg * 4 + q, rb = f % (Co >> 3), pb = f / (Co >> 3);
                const long long p = pc0 + pb * 8 + (lane >> 2);
                const int co = rb * 8 + 2 * (lane & 3);
                uint32_t v = 0u;
                if (p < p_end) {
                    const long long i = p * Co + co;
                    const float2 gg = *reinterpret_cast<const float2*>(g + i);
                    const __nv_bfloat162 yb = *reinterpret_cast<const __nv_bfloat162*>(yout + i);
                    __nv_bfloat162 h = __floats2bfloat162_rn(__bfloat162float(yb.x) > 0.f ? gg.x : 0.f,
                                                             __bfloat162float(yb.y) > 0.f ? gg.y : 0.f);
                    v = *reinterpret_cast<uint32_t*>(&h);
                }
                r[q] = v;
            }
            const int fq = fg * 4 + (lane >> 3), rbq = fq % (Co >> 3), pbq = fq / (Co >> 3);
            stmatrix_x4_trans(smem_u32(As + swz(rbq * 8 + (lane & 7), pbq)), r);
        }
        // B blocks: 16 column blocks x 8 pixel blocks; group fg (4 blocks) has
        // the pixel block fg / 4 and the column blocks 4 (fg % 4) + q, and
        // warp w takes fg = w, w + 8, ...: its columns (bcol) are the same in
        // every group and stage, so only the pixel is decoded per group
        for (int fg = warp; fg < (tcw::kWN / 8) * (kKC / 8) / 4; fg += kThreads / 32) {
            const int pb = fg >> 2;
            const long long p = pc0 + pb * 8 + (lane >> 2);
            int b = -1, y = 0, x = 0;
            if (p < p_end) {
                const int pi = (int)p;               // pixel counts fit in 31 bits (checked at launch)
                x = pi % W;
                const int t = pi / W;
                y = t % H;
                b = t / H;
            }
            uint32_t r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t v = 0u;
                const int yy = y + bdy[q], xx = x + bdx[q];
                if (b >= 0 && bci[q] >= 0 && yy >= 0 && yy < H && xx >= 0 && xx < W)
                    v = lx.load2(b, yy, xx, H, W, bci[q]);
                r[q] = v;
            }
            const int fq = fg * 4 + (lane >> 3), nbq = fq % (tcw::kWN / 8), pbq = fq / (tcw::kWN / 8);
            stmatrix_x4_trans(smem_u32(Bs + swz(nbq * 8 + (lane & 7), pbq)), r);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
            for (int ks = 0; ks < kKC / 16; ++ks)
                mma(tmem, sdesc(a0 + ks * 32), sdesc(b0 + ks * 32), idesc(tcw::kWN), (c > 0 || ks > 0) ? 1u : 0u);
            commit(&done[s]);
        }
    }
    if (nch > 0) {
        const int cl = nch - 1;
        if (!mbar_wait(&done[cl % kStages], (unsigned)(cl / kStages) & 1u)) {
            ok = false;
            mbar_wait(&done[cl % kStages], (unsigned)(cl / kStages) & 1u);   // one more bounded wait before freeing
        }
        fence_after();
        // warp w: accumulator rows (co) 32 (w % 4) + lane, columns [half, half + kWN / 2)
        const int quarter = warp & 3, chalf = (warp >> 2) * (tcw::kWN / 2);
        const int co = quarter * 32 + lane;
        for (int c0 = chalf; c0 < chalf + tcw::kWN / 2; c0 += 8) {
            uint32_t rr[8];
            ld8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, rr);
            if (co < Co) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = n0 + c0 + j;
                    if (n < Ntot) {
                        const int tap = n / Ci, ci = n - tap * Ci;
                        atomicAdd(dW + ((long long)co * Ci + ci) * 9 + tap, __uint_as_float(rr[j]));
                    }
                }
            }
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)tcw::kWN)
                     : "memory");
    }
}

// db[co] += sum over pixels of g'[p][co] (FP32), one block per pixel slice
// Co % 4 == 0: each thread one group of 4 channels (16-byte gradient and
// 8-byte output loads), 4 pixels in flight per thread, one atomic per channel
// and block.
__global__ void __launch_bounds__(256) k_bias_grad4(const float* __restrict__ g, const bf16* __restrict__ yout,
                                                    long long P, int Co, long long pix_per_block,
                                                    float* __restrict__ db) {
    __shared__ float4 acc4[256];
    const int t = threadIdx.x;
    const int cg = Co >> 2, lanes = 256 / cg, c4 = t % cg;
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
    auto add = [&](float4 gv, uint2 yv) {
        const __nv_bfloat162 y01 = *reinterpret_cast<const __nv_bfloat162*>(&yv.x);
        const __nv_bfloat162 y23 = *reinterpret_cast<const __nv_bfloat162*>(&yv.y);
        sum.x += __bfloat162float(y01.x) > 0.f ? gv.x : 0.f;
        sum.y += __bfloat162float(y01.y) > 0.f ? gv.y : 0.f;
        sum.z += __bfloat162float(y23.x) > 0.f ? gv.z : 0.f;
        sum.w += __bfloat162float(y23.y) > 0.f ? gv.w : 0.f;
    };
    if (t < lanes * cg) {
        const long long p0 = (long long)blockIdx.x * pix_per_block;
        const long long p1 = min(P, p0 + pix_per_block);
        long long p = p0 + t / cg;
        for (; p + 3LL * lanes < p1; p += 4LL * lanes) {
            float4 gv[4];
            uint2 yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long i = (p + (long long)u * lanes) * Co + 4 * c4;
                gv[u] = *reinterpret_cast<const float4*>(g + i);
                yv[u] = *reinterpret_cast<const uint2*>(yout + i);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) add(gv[u], yv[u]);
        }
        for (; p < p1; p += lanes) {
            const long long i = p * Co + 4 * c4;
            add(*reinterpret_cast<const float4*>(g + i), *reinterpret_cast<const uint2*>(yout + i));
        }
    }
    acc4[t] = sum;
    __syncthreads();
    if (t < cg) {
        float4 tot = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < lanes; ++q) {
            const float4 v = acc4[q * cg + t];
            tot.x += v.x;
            tot.y += v.y;
            tot.z += v.z;
            tot.w += v.w;
        }
        atomicAdd(db + 4 * t, tot.x);
        atomicAdd(db + 4 * t + 1, tot.y);
        atomicAdd(db + 4 * t + 2, tot.z);
        atomicAdd(db + 4 * t + 3, tot.w);
    }
}

__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ g, const bf16* __restrict__ yout,
                                                   long long P, int Co, long long pix_per_block,
                                                   float* __restrict__ db) {
    __shared__ float acc[256];
    const int t = threadIdx.x;
    const int co = t % Co, lanes = 256 / Co;
    float sum = 0.f;
    if (t < lanes * Co) {
        const long long p0 = (long long)blockIdx.x * pix_per_block;
        const long long p1 = min(P, p0 + pix_per_block);
        for (long long p = p0 + t / Co; p < p1; p += lanes) {
            const long long i = p * Co + co;
            sum += __bfloat162float(yout[i]) > 0.f ? g[i] : 0.f;
        }
    }
    acc[t] = sum;
    __syncthreads();
    if (t < Co) {
        float tot = 0.f;
        for (int q = 0; q < lanes; ++q) tot += acc[q * Co + t];
        atomicAdd(db + t, tot);
    }
}

// backward-data weights for the tensor cores: the transposed convolution
// with flipped taps, as a forward one from Co to Ci channels:
// wt[ci][tap'][co] = w[co][ci][8 - tap'] (K-major rows, k = tap' * Co + co)
__global__ void k_w_tc_bwd(const bf16* __restrict__ w, int Co, int Ci, bf16* __restrict__ wt) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Co * Ci * 9) return;
    const int co = (int)(idx % Co);
    const int tap = (int)((idx / Co) % 9);
    const int ci = (int)(idx / ((long long)Co * 9));
    wt[idx] = w[((long long)co * Ci + ci) * 9 + (8 - tap)];
}

// tensor-core weights BF16 [co][ci][9] -> [co][9][ci] (K-major rows, k = tap * Ci + ci)
// (input channels padded with zero weights to Cp >= Ci: k = tap * Cp + ci)
__global__ void k_w_tc(const bf16* __restrict__ w, int Co, int Ci, int Cp, bf16* __restrict__ wt) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Co * Cp * 9) return;
    const int co = (int)(idx / (Cp * 9)), ci = (int)((idx / 9) % Cp), tap = (int)(idx % 9);
    wt[((long long)co * 9 + tap) * Cp + ci] = ci < Ci ? w[((long long)co * Ci + ci) * 9 + tap] : __float2bfloat16_rn(0.f);
}

// Weight gradient of a 3x3 convolution: dW[co][ci][tap] += sum_p g[p, co] in[p + tap, ci],
// db[co] += sum_p g[p, co], with g masked by ReLU'(out).  One CTA: 16 output x
// 16 input channels (one (co, ci) pair per thread, 9 taps) over a slice of
// 16x16 pixel tiles; partial sums added atomically.
template <class LX>
__global__ void __launch_bounds__(256) k_conv3_wgrad(LX lx, const float* __restrict__ g, const bf16* __restrict__ yout,
                                                     int B, int H, int W, int Ci, int Co, int tiles_per_cta,
                                                     float* __restrict__ dW, float* __restrict__ db) {
    __shared__ float s_g[256][17];
    __shared__ float s_x[16][18][19];
    const int nci = (Ci + 15) / 16;
    const int cob = blockIdx.y / nci, cib = blockIdx.y % nci;
    const int t = threadIdx.x, o = t >> 4, i = t & 15;
    const int co = cob * 16 + o, ci = cib * 16 + i;
    const int tw = (W + 15) / 16, th = (H + 15) / 16;
    const long long ntiles = (long long)B * tw * th;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    float accb = 0.f;
    for (long long tile = (long long)blockIdx.x * tiles_per_cta;
         tile < min(ntiles, (long long)(blockIdx.x + 1) * tiles_per_cta); ++tile) {
        const int b = (int)(tile / (tw * th));
        const int rem = (int)(tile % (tw * th));
        const int y0 = (rem / tw) * 16, x0 = (rem % tw) * 16;
        __syncthreads();
        for (int idx = t; idx < 256 * 16; idx += 256) {
            const int p = idx >> 4, c = idx & 15;
            const int yy = y0 + (p >> 4), xx = x0 + (p & 15), cc = cob * 16 + c;
            float v = 0.f;
            if (yy < H && xx < W && cc < Co) {
                const long long q = (((long long)b * H + yy) * W + xx) * Co + cc;
                v = __bfloat162float(yout[q]) > 0.f ? g[q] : 0.f;
            }
            s_g[p][c] = v;
        }
        for (int idx = t; idx < 16 * 18 * 18; idx += 256) {
            const int c = idx / (18 * 18), r = (idx / 18) % 18, q = idx % 18;
            const int yy = y0 + r - 1, xx = x0 + q - 1, cc = cib * 16 + c;
            float v = 0.f;
            if (cc < Ci && yy >= 0 && yy < H && xx >= 0 && xx < W) v = lx(b, yy, xx, H, W, cc);
            s_x[c][r][q] = v;
        }
        __syncthreads();
        for (int p = 0; p < 256; ++p) {
            const float gv = s_g[p][o];
            const int py = p >> 4, px = p & 15;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) acc[dy * 3 + dx] = fmaf(gv, s_x[i][py + dy][px + dx], acc[dy * 3 + dx]);
            accb += gv;
        }
    }
    if (co < Co && ci < Ci) {
#pragma unroll
        for (int k = 0; k < 9; ++k) atomicAdd(dW + ((long long)co * Ci + ci) * 9 + k, acc[k]);
    }
    if (i == 0 && cib == 0 && co < Co) atomicAdd(db + co, accb);
}

// ---------------------------------------------------------------- small kernels
// forward weights BF16 [co][ci][9] -> [ci][9][co]
__global__ void k_w_fwd(const bf16* __restrict__ w, int Co, int Ci, bf16* __restrict__ wk) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Co * Ci * 9) return;
    const int co = (int)(idx / (Ci * 9)), ci = (int)((idx / 9) % Ci), tap = (int)(idx % 9);
    wk[((long long)ci * 9 + tap) * Co + co] = w[idx];
}
// backward-data weights: input channel = co, output channel = ci, taps flipped:
// wb[co][tap'][ci] = w[co][ci][8 - tap']
__global__ void k_w_bwd(const bf16* __restrict__ w, int Co, int Ci, bf16* __restrict__ wb) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Co * Ci * 9) return;
    const int co = (int)(idx / (Ci * 9)), ci = (int)((idx / 9) % Ci), tap = (int)(idx % 9);
    wb[((long long)co * 9 + (8 - tap)) * Ci + ci] = w[idx];
}

__global__ void k_avgpool2(const bf16* __restrict__ x, int B, int H, int W, int C, bf16* __restrict__ y) {
    const long long n = (long long)B * (H / 2) * (W / 2) * C;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int c = (int)(idx % C);
    long long p = idx / C;
    const int xo = (int)(p % (W / 2));
    p /= (W / 2);
    const int yo = (int)(p % (H / 2));
    const int b = (int)(p / (H / 2));
    auto at = [&](int yy, int xx) { return __bfloat162float(x[(((long long)b * H + yy) * W + xx) * C + c]); };
    const float s = at(2 * yo, 2 * xo) + at(2 * yo, 2 * xo + 1) + at(2 * yo + 1, 2 * xo) + at(2 * yo + 1, 2 * xo + 1);
    y[idx] = __float2bfloat16_rn(0.25f * s);
}

// g_in[b, y, x, c] (+)= g_out[b, y/2, x/2, c] / 4  (backward of the average pool)
__global__ void k_avgpool2_bwd(const float* __restrict__ go, int B, int H, int W, int C, float* __restrict__ gi,
                               int accumulate) {
    const long long n = (long long)B * H * W * C;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int c = (int)(idx % C);
    long long p = idx / C;
    const int x = (int)(p % W);
    p /= W;
    const int y = (int)(p % H);
    const int b = (int)(p / H);
    const float v = 0.25f * go[(((long long)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
    gi[idx] = accumulate ? gi[idx] + v : v;
}

// Splits the gradient of a concatenated decoder input [up(h) | skip]:
// g_h[b, y', x', c] = sum of the 2x2 block (c < cu); g_skip = remaining channels.
__global__ void k_split_cat_bwd(const float* __restrict__ gx, int B, int H, int W, int cu, int cs,
                                float* __restrict__ gh, float* __restrict__ gskip) {
    const int C = cu + cs;
    const long long nlow = (long long)B * (H / 2) * (W / 2) * cu;
    const long long nsk = (long long)B * H * W * cs;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < nlow) {
        const int c = (int)(idx % cu);
        long long p = idx / cu;
        const int xo = (int)(p % (W / 2));
        p /= (W / 2);
        const int yo = (int)(p % (H / 2));
        const int b = (int)(p / (H / 2));
        float s = 0.f;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                s += gx[(((long long)b * H + 2 * yo + dy) * W + 2 * xo + dx) * C + c];
        gh[idx] = s;
    } else if (idx < nlow + nsk) {
        const long long j = idx - nlow;
        const int c = (int)(j % cs);
        const long long p = j / cs;
        gskip[j] = gx[p * C + cu + c];
    }
}

__global__ void k_add(float* __restrict__ a, const float* __restrict__ b, long long n) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) a[idx] += b[idx];
}

// 1x1 head: y[p, o] = b[o] + sum_c h[p, c] w[o][c]   (FP32 output)
__global__ void k_head_fwd(const bf16* __restrict__ h, long long P, int C, int O, const bf16* __restrict__ w,
                           const float* __restrict__ bias, float* __restrict__ y) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * O) return;
    const long long p = idx / O;
    const int o = (int)(idx % O);
    float s = bias[o];
    for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(h[p * C + c]), __bfloat162float(w[(long long)o * C + c]), s);
    y[idx] = s;
}

// The 1x1 head, one pixel per thread (C % 8 == 0, C <= 256, O <= 32): the
// weights in shared memory as [c][o] (every thread reads the same entry, a
// broadcast), the pixel's input row by 16-byte loads, all O outputs in
// registers, written as 16-byte stores when O % 4 == 0.
constexpr int kHeadMaxO = 32;
__global__ void __launch_bounds__(256) k_head_fwd_px(const bf16* __restrict__ h, long long P, int C, int O,
                                                     const bf16* __restrict__ w, const float* __restrict__ bias,
                                                     float* __restrict__ y) {
    extern __shared__ float wsh[];   // [C][O] then bias [O]
    for (int i = threadIdx.x; i < C * O; i += blockDim.x) {
        const int o = i / C, c = i - o * C;
        wsh[c * O + o] = __bfloat162float(w[i]);
    }
    for (int o = threadIdx.x; o < O; o += blockDim.x) wsh[C * O + o] = bias[o];
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float out[kHeadMaxO];
#pragma unroll
    for (int o = 0; o < kHeadMaxO; ++o) out[o] = o < O ? wsh[C * O + o] : 0.f;
    const uint4* hr = reinterpret_cast<const uint4*>(h + p * C);
    for (int c8 = 0; c8 < C / 8; ++c8) {
        const uint4 v = hr[c8];
        const unsigned wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162*>(&wv[q]);
            const float h0 = __bfloat162float(b2.x), h1 = __bfloat162float(b2.y);
            const float* w0 = wsh + (8 * c8 + 2 * q) * O;
#pragma unroll
            for (int o = 0; o < kHeadMaxO; ++o)
                if (o < O) out[o] = fmaf(h1, w0[O + o], fmaf(h0, w0[o], out[o]));
        }
    }
    float* yo = y + p * O;
    if (O % 4 == 0) {
#pragma unroll
        for (int o = 0; o < kHeadMaxO; o += 4)
            if (o < O) *reinterpret_cast<float4*>(yo + o) = make_float4(out[o], out[o + 1], out[o + 2], out[o + 3]);
    } else {
#pragma unroll
        for (int o = 0; o < kHeadMaxO; ++o)
            if (o < O) yo[o] = out[o];
    }
}

// gh[p, c] = sum_o gy[p, o] w[o][c], one pixel per thread (conditions as
// k_head_fwd_px): the gradient row in registers, 32 input channels at a time.
__global__ void __launch_bounds__(256) k_head_bwd_data_px(const float* __restrict__ gy, long long P, int C, int O,
                                                          const bf16* __restrict__ w, float* __restrict__ gh) {
    extern __shared__ float wsh[];   // [o][c]
    for (int i = threadIdx.x; i < C * O; i += blockDim.x) wsh[i] = __bfloat162float(w[i]);
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float g[kHeadMaxO];
#pragma unroll
    for (int o = 0; o < kHeadMaxO; ++o) g[o] = o < O ? gy[p * O + o] : 0.f;
    float* go = gh + p * C;
    for (int c0 = 0; c0 < C; c0 += 32) {
        float acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.f;
#pragma unroll
        for (int o = 0; o < kHeadMaxO; ++o) {
            if (o >= O) continue;
            const float* wr = wsh + o * C + c0;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (c0 + j < C) acc[j] = fmaf(g[o], wr[j], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 32; j += 4)
            if (c0 + j < C) *reinterpret_cast<float4*>(go + c0 + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
    }
}

// head backward: gh[p, c] = sum_o gy[p, o] w[o][c]; dW[o][c] += sum_p gy[p, o] h[p, c]; db[o] += sum_p gy
__global__ void k_head_bwd_data(const float* __restrict__ gy, long long P, int C, int O, const bf16* __restrict__ w,
                                float* __restrict__ gh) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * C) return;
    const long long p = idx / C;
    const int c = (int)(idx % C);
    float s = 0.f;
    for (int o = 0; o < O; ++o) s = fmaf(gy[p * O + o], __bfloat162float(w[(long long)o * C + c]), s);
    gh[idx] = s;
}
// The 1x1 head's weight and bias gradients over the pixels in parallel:
// dW[o][c] += sum_p gy[p, o] h[p, c] (c < C), db[o] += sum_p gy[p, o] (c = C).
// Each block takes a range of pixels in tiles of kHeadTile staged in shared
// memory (coalesced loads; h with a column of ones for the bias, padded to a
// multiple of 4); thread pair (o, c4) accumulates 4 consecutive c of one o;
// one atomic per output and block.
constexpr int kHeadTile = 64;
constexpr int kHeadPairs = 8;          // (o, 4 c) pairs per thread
__host__ __device__ constexpr int head_cp(int C) { return (C + 1 + 3) / 4 * 4; }
__global__ void __launch_bounds__(256) k_head_bwd_w4(const float* __restrict__ gy, const bf16* __restrict__ h,
                                                     long long P, int C, int O, long long pix_per_block,
                                                     float* __restrict__ dW, float* __restrict__ db) {
    extern __shared__ __align__(16) float hsm[];
    const int Cp = head_cp(C), nq = Cp / 4, npair = O * nq;
    float* gs = hsm;                       // [kHeadTile][O]
    float* hs = hsm + kHeadTile * O;       // [kHeadTile][Cp]
    const int t = threadIdx.x;
    float4 acc[kHeadPairs];
#pragma unroll
    for (int j = 0; j < kHeadPairs; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long p0 = (long long)blockIdx.x * pix_per_block;
    const long long p1 = min(P, p0 + pix_per_block);
    for (long long pt = p0; pt < p1; pt += kHeadTile) {
        const int np = (int)min((long long)kHeadTile, p1 - pt);
        __syncthreads();   // the previous tile is consumed
        for (int idx = t; idx < kHeadTile * O; idx += blockDim.x)
            gs[idx] = idx / O < np ? gy[pt * O + idx] : 0.f;
        for (int idx = t; idx < kHeadTile * Cp; idx += blockDim.x) {
            const int px = idx / Cp, c = idx - px * Cp;
            float v = 0.f;
            if (px < np) v = c < C ? __bfloat162float(h[(pt + px) * C + c]) : (c == C ? 1.f : 0.f);
            hs[idx] = v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kHeadPairs; ++j) {
            const int pr = t + j * 256;
            if (pr >= npair) continue;
            const int o = pr / nq, q = pr - o * nq;
            float4 a = acc[j];
            for (int px = 0; px < kHeadTile; ++px) {
                const float gv = gs[px * O + o];
                const float4 hv = *reinterpret_cast<const float4*>(hs + px * Cp + 4 * q);
                a.x += gv * hv.x;
                a.y += gv * hv.y;
                a.z += gv * hv.z;
                a.w += gv * hv.w;
            }
            acc[j] = a;
        }
    }
#pragma unroll
    for (int j = 0; j < kHeadPairs; ++j) {
        const int pr = t + j * 256;
        if (pr >= npair) continue;
        const int o = pr / nq, q = pr - o * nq;
        const float v[4] = {acc[j].x, acc[j].y, acc[j].z, acc[j].w};
        for (int u = 0; u < 4; ++u) {
            const int c = 4 * q + u;
            if (c < C) atomicAdd(dW + (long long)o * C + c, v[u]);
            else if (c == C) atomicAdd(db + o, v[u]);
        }
    }
}

__global__ void k_head_bwd_w(const float* __restrict__ gy, const bf16* __restrict__ h, long long P, int C, int O,
                             float* __restrict__ dW, float* __restrict__ db) {
    // one CTA per (o, c) pair (+ one row c == C for the bias); block reduction over pixels
    const int o = blockIdx.x / (C + 1), c = blockIdx.x % (C + 1);
    float s = 0.f;
    for (long long p = threadIdx.x; p < P; p += blockDim.x)
        s += gy[p * O + o] * (c < C ? __bfloat162float(h[p * C + c]) : 1.f);
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    __shared__ float sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) tot += sm[w2];
        if (c < C) dW[(long long)o * C + c] += tot;
        else db[o] += tot;
    }
}

// network input: (eps - 2.1)/10.15, (lambda - 1.3um)/0.25um, PML mask, source profile
struct InputDesc {
    const double* eps;
    int nx, ny, npml;
    double wavelength;
};
constexpr int kInPad = 16;   // channels of the padded input copy
__global__ void k_input(const InputDesc* __restrict__ desc, int B, int H, int W, int i_src, double sigma, double j_c,
                        const float2* __restrict__ field, int cin, bf16* __restrict__ x, bf16* __restrict__ xp) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * H * W) return;
    const int b = (int)(idx / ((long long)H * W));
    const int e = (int)(idx % ((long long)H * W));
    const int j = e / W, i = e % W;
    const InputDesc d = desc[b];
    const int L = d.npml;
    const bool inside = i >= L && i < W - L && j >= L && j < H - L;
    const double t = (double)j - j_c;
    bf16* o = x + idx * cin;
    o[0] = __float2bfloat16_rn((float)((d.eps[e] - 2.1) / 10.15));
    o[1] = __float2bfloat16_rn((float)((d.wavelength - 1.3e-6) / 0.25e-6));
    o[2] = __float2bfloat16_rn(inside ? 0.f : 1.f);
    o[3] = __float2bfloat16_rn(i == i_src ? (float)exp(-t * t / (2.0 * sigma * sigma)) : 0.f);
    if (cin == 6) {
        // an approximate field of the grid (normalised to max |f| = 1): Re, Im
        o[4] = __float2bfloat16_rn(field[e].x);
        o[5] = __float2bfloat16_rn(field[e].y);
    }
    // the same channels, zero-padded to kInPad, as two 16-byte stores
    __align__(16) bf16 pad[kInPad];
#pragma unroll
    for (int c = 0; c < kInPad; ++c) pad[c] = c < cin ? o[c] : __float2bfloat16_rn(0.f);
    uint4* q = reinterpret_cast<uint4*>(xp + idx * kInPad);
    q[0] = reinterpret_cast<const uint4*>(pad)[0];
    q[1] = reinterpret_cast<const uint4*>(pad)[1];
}

// max |f| over D values (one block), then f / max |f| in FP32
__global__ void k_field_in(const double2* __restrict__ f, long long D, float2* __restrict__ out) {
    __shared__ double sm[32];
    double m = 0.0;
    for (long long e = threadIdx.x; e < D; e += blockDim.x) m = fmax(m, hypot(f[e].x, f[e].y));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) sm[0] = m;
    }
    __syncthreads();
    const double inv = sm[0] > 0.0 ? 1.0 / sm[0] : 0.0;
    for (long long e = threadIdx.x; e < D; e += blockDim.x)
        out[e] = make_float2((float)(f[e].x * inv), (float)(f[e].y * inv));
}

// Projection loss (Eq. 5) over the pixels in parallel, three kernels:
//   k_proj_part   per sample s and block c (a range of 256-pixel tiles staged
//                 in shared memory): partial sums of a = V^H f, the upper
//                 triangle of G = V^H V and |f|^2 (FP32 per lane, FP64 across
//                 the lanes); entry e < k: a_e, then G(c, d) for c <= d in
//                 row order, last |f|^2
//   k_proj_solve  per sample: the sums over the blocks in block order (FP64),
//                 Cholesky solve G z = a (tiny ridge), l = 1 - Re(a^H z)/|f|^2;
//                 keeps z and |f|^2
//   k_proj_grad   per pixel: gy = 2 (Re, Im) of -(f - V z) z^H / (|f|^2 B)
constexpr int kLossTile = 256;
constexpr int kLossMaxEnt = 20;   // entries per warp: ceil((16 + 136 + 1) / 8) for k <= 16
__host__ __device__ constexpr int loss_entries(int k) { return k + k * (k + 1) / 2 + 1; }
__host__ __device__ constexpr size_t loss_smem(int k) {
    return sizeof(float) * (size_t)kLossTile * (2 * k + 1) + sizeof(float2) * kLossTile +
           sizeof(int2) * (size_t)loss_entries(k);
}

__global__ void __launch_bounds__(256) k_proj_part(const float* __restrict__ y, const double2* const* __restrict__ f,
                                                   int D, int k, int tiles_per_block, double2* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char lsm_raw[];
    const int s = blockIdx.y, c = blockIdx.x, nch = gridDim.x;
    const int stride = 2 * k + 1;                 // odd: lanes reading one column hit distinct banks
    float* ys = reinterpret_cast<float*>(lsm_raw);
    float2* fsm = reinterpret_cast<float2*>(ys + kLossTile * stride);
    int2* tab = reinterpret_cast<int2*>(fsm + kLossTile);   // entry -> (c, d); d < 0: a_c; c < 0: |f|^2
    const int nent = loss_entries(k);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < nent; e += blockDim.x) {
        int2 cd;
        if (e < k) cd = make_int2(e, -1);
        else if (e == nent - 1) cd = make_int2(-1, -1);
        else {
            int q = e - k, cc = 0;
            while (q >= k - cc) { q -= k - cc; ++cc; }
            cd = make_int2(cc, cc + q);
        }
        tab[e] = cd;
    }
    float ar[kLossMaxEnt], ai[kLossMaxEnt];
#pragma unroll
    for (int j = 0; j < kLossMaxEnt; ++j) ar[j] = ai[j] = 0.f;
    const float* yss = y + (long long)s * D * 2 * k;
    const double2* fs = f[s];
    const int ntiles = (D + kLossTile - 1) / kLossTile;
    for (int tt = 0; tt < tiles_per_block; ++tt) {
        const int tile = c * tiles_per_block + tt;
        if (tile >= ntiles) break;
        const int e0 = tile * kLossTile;
        const int npx = min(kLossTile, D - e0);
        __syncthreads();   // the previous tile is consumed (and the table written)
        for (int idx = threadIdx.x; idx < kLossTile * 2 * k; idx += blockDim.x) {
            const int px = idx / (2 * k), q = idx - px * 2 * k;
            ys[px * stride + q] = px < npx ? yss[(long long)(e0 + px) * 2 * k + q] : 0.f;
        }
        for (int px = threadIdx.x; px < kLossTile; px += blockDim.x) {
            const double2 fe = px < npx ? fs[e0 + px] : make_double2(0.0, 0.0);
            fsm[px] = make_float2((float)fe.x, (float)fe.y);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kLossMaxEnt; ++j) {
            const int ent = wid + 8 * j;
            if (ent >= nent) continue;
            const int2 cd = tab[ent];
            float sr = 0.f, si = 0.f;
            if (cd.y >= 0) {            // G(c, d) = v_c^H v_d
                for (int px = lane; px < kLossTile; px += 32) {
                    const float cr = ys[px * stride + 2 * cd.x], ci = ys[px * stride + 2 * cd.x + 1];
                    const float dr = ys[px * stride + 2 * cd.y], di = ys[px * stride + 2 * cd.y + 1];
                    sr += cr * dr + ci * di;
                    si += cr * di - ci * dr;
                }
            } else if (cd.x >= 0) {     // a_c = v_c^H f
                for (int px = lane; px < kLossTile; px += 32) {
                    const float vr = ys[px * stride + 2 * cd.x], vi = ys[px * stride + 2 * cd.x + 1];
                    const float2 fe = fsm[px];
                    sr += vr * fe.x + vi * fe.y;
                    si += vr * fe.y - vi * fe.x;
                }
            } else {                    // |f|^2
                for (int px = lane; px < kLossTile; px += 32) {
                    const float2 fe = fsm[px];
                    sr += fe.x * fe.x + fe.y * fe.y;
                }
            }
            ar[j] += sr;
            ai[j] += si;
        }
    }
#pragma unroll
    for (int j = 0; j < kLossMaxEnt; ++j) {
        const int ent = wid + 8 * j;
        if (ent >= nent) continue;
        double dr = ar[j], di = ai[j];
        for (int m = 16; m > 0; m >>= 1) {
            dr += __shfl_xor_sync(0xffffffffu, dr, m);
            di += __shfl_xor_sync(0xffffffffu, di, m);
        }
        if (lane == 0) part[((long long)s * nch + c) * nent + ent] = make_double2(dr, di);
    }
}

// Sums the blocks' partials (in block order), solves G z = a and writes the
// loss; zf[s] holds z_0 .. z_{k-1} and (|f|^2, 0).
__global__ void __launch_bounds__(256) k_proj_solve(const double2* __restrict__ part, int k, int nch,
                                                    double* __restrict__ loss, double2* __restrict__ zf) {
    extern __shared__ double2 sh2[];   // entries (nent), G (k*k), z (k)
    const int s = blockIdx.x;
    const int nent = loss_entries(k);
    double2* ent = sh2;
    double2* G = sh2 + nent;
    double2* z = G + k * k;
    for (int e = threadIdx.x; e < nent; e += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        const double2* pe = part + (long long)s * nch * nent + e;
        for (int c = 0; c < nch; ++c) acc = cadd(acc, pe[(long long)c * nent]);
        ent[e] = acc;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double2* a = ent;
    int q = k;
    for (int c = 0; c < k; ++c)
        for (int d = c; d < k; ++d, ++q) {
            G[d * k + c] = ent[q];                                  // G(c, d)
            G[c * k + d] = make_double2(ent[q].x, -ent[q].y);       // G(d, c)
        }
    const double sF = ent[nent - 1].x;
    // Cholesky G = R^H R (upper R in place, column-major) with a ridge of 1e-6 max diag:
    // keeps the loss finite when the predicted vectors become dependent
    double dmax = 0.0;
    for (int c = 0; c < k; ++c) dmax = fmax(dmax, G[c * k + c].x);
    for (int c = 0; c < k; ++c) G[c * k + c].x += 1e-6 * dmax + 1e-300;
    for (int p = 0; p < k; ++p) {
        double dd = G[p * k + p].x;
        for (int l = 0; l < p; ++l) dd -= cabs2(G[p * k + l]);
        const double rpp = sqrt(fmax(dd, 1e-300));
        G[p * k + p] = make_double2(rpp, 0.0);
        for (int r = p + 1; r < k; ++r) {
            double2 tq = G[r * k + p];
            for (int l = 0; l < p; ++l) tq = csub(tq, cmulc(G[p * k + l], G[r * k + l]));
            G[r * k + p] = cscale(tq, 1.0 / rpp);
        }
    }
    // R^H w = a (forward), R z = w (backward)
    for (int p = 0; p < k; ++p) {
        double2 tq = a[p];
        for (int l = 0; l < p; ++l) tq = csub(tq, cmulc(G[p * k + l], z[l]));
        z[p] = cscale(tq, 1.0 / G[p * k + p].x);
    }
    for (int p = k - 1; p >= 0; --p) {
        double2 tq = z[p];
        for (int l = p + 1; l < k; ++l) tq = csub(tq, cmul(G[l * k + p], z[l]));
        z[p] = cscale(tq, 1.0 / G[p * k + p].x);
    }
    double az = 0.0;
    for (int c = 0; c < k; ++c) az += a[c].x * z[c].x + a[c].y * z[c].y;   // Re(a^H z)
    loss[s] = 1.0 - az / sF;
    for (int c = 0; c < k; ++c) zf[(long long)s * (k + 1) + c] = z[c];
    zf[(long long)s * (k + 1) + k] = make_double2(sF, 0.0);
}

// gy[s, e] = 2 (Re, Im) of -(f - V z) conj(z_c) / (|f|^2 B), one pixel per thread.
__global__ void __launch_bounds__(256) k_proj_grad(const float* __restrict__ y, const double2* const* __restrict__ f,
                                                   int D, int k, int B, const double2* __restrict__ zf,
                                                   float* __restrict__ gy) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * D) return;
    const int s = (int)(idx / D), e = (int)(idx - (long long)s * D);
    const double2* zs = zf + (long long)s * (k + 1);
    const float scale = (float)(-2.0 / (zs[k].x * B));
    const float* ys = y + idx * 2 * k;
    float* gs = gy + idx * 2 * k;
    const double2 fe = f[s][e];
    float rr = (float)fe.x, ri = (float)fe.y;
    for (int c = 0; c < k; ++c) {
        const float vr = ys[2 * c], vi = ys[2 * c + 1];
        const float zr = (float)zs[c].x, zi = (float)zs[c].y;
        rr -= vr * zr - vi * zi;
        ri -= vr * zi + vi * zr;
    }
    for (int c = 0; c < k; ++c) {
        const float zr = (float)zs[c].x, zi = (float)zs[c].y;
        // r conj(z_c)
        gs[2 * c] = scale * (rr * zr + ri * zi);
        gs[2 * c + 1] = scale * (ri * zr - rr * zi);
    }
}

// Adam (Kingma & Ba 2015, Algorithm 1) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ thb, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float t = th[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    th[i] = t;
    thb[i] = __float2bfloat16_rn(t);
}

__global__ void k_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// network output (B, D, 2k) FP32 -> U_b (D x k complex128, column-major)
// base (D x k complex, column c at c * D) scaled, into the output layout [D][2k]
__global__ void k_base_in(const double2* __restrict__ U, long long D, int k, double scale, float* __restrict__ out) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * k) return;
    const int c = (int)(idx / D);
    const long long e = idx % D;
    const double2 u = U[idx];
    out[e * 2 * k + 2 * c] = (float)(u.x * scale);
    out[e * 2 * k + 2 * c + 1] = (float)(u.y * scale);
}
// y[b] += base[b] for every sample b with an offset (n = D * 2k values per sample)
__global__ void k_add_base(float* __restrict__ y, const float* const* __restrict__ base, long long n, int B) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * B) return;
    const float* bs = base[idx / n];
    if (bs) y[idx] += bs[idx % n];
}

__global__ void k_to_complex(const float* __restrict__ y, int D, int k, double2* const* __restrict__ U, int B) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * D * k) return;
    const int b = (int)(idx / ((long long)D * k));
    const long long r = idx % ((long long)D * k);
    const int c = (int)(r / D), e = (int)(r % D);
    const float* ye = y + ((long long)b * D + e) * 2 * k;
    U[b][(long long)c * D + e] = make_double2(ye[2 * c], ye[2 * c + 1]);
}

// ---------------------------------------------------------------- K13: orthonormal predicted vectors
// Cholesky QR applied twice, in FP64, to each problem's k predicted vectors
// (U: D x k column-major): G = U^H U = L L^H, U <- U L^-H.  The span is kept;
// after two passes U^H U = I to FP64 round-off (times the conditioning left
// by the first pass).
constexpr int kOrthRows = 2048;   // rows of one problem per block (Gram and apply)
constexpr int kOrthTile = 64;     // rows per shared-memory tile of the Gram kernel
constexpr int kOrthMaxK = 16;

__device__ __forceinline__ void orth_pair(int t, int k, int* i, int* j) {
    // t-th pair (i, j), i <= j, in row order of the upper triangle
    int r = 0;
    while (t >= k - r) { t -= k - r; ++r; }
    *i = r;
    *j = r + t;
}

// Block (c, s): partial Gram of rows [c kOrthRows, (c+1) kOrthRows) of problem
// s.  Thread groups of np = k(k+1)/2 threads share the block's rows (group g
// takes tile rows r = g mod ngroups); thread (g, p) owns pair p = (i, j) and
// sums conj(U_ri) U_rj; the groups' sums are added in a fixed order.
__global__ void __launch_bounds__(256) k_orth_gram(double2* const* __restrict__ U, int D, int k, int nch,
                                                   double2* __restrict__ part) {
    __shared__ double2 tile[kOrthTile][kOrthMaxK];
    __shared__ double2 red[256];
    const int s = blockIdx.y, c = blockIdx.x;
    const double2* u = U[s];
    const int np = k * (k + 1) / 2;
    const int ngroups = (int)blockDim.x / np;
    const int g = (int)threadIdx.x / np, p = (int)threadIdx.x % np;
    const bool active = g < ngroups;
    int pi = 0, pj = 0;
    if (active) orth_pair(p, k, &pi, &pj);
    double2 acc = make_double2(0.0, 0.0);
    const long long r0 = (long long)c * kOrthRows;
    const long long r1 = min((long long)D, r0 + kOrthRows);
    for (long long t0 = r0; t0 < r1; t0 += kOrthTile) {
        const int rows = (int)min((long long)kOrthTile, r1 - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < kOrthTile * k; e += blockDim.x) {
            const int col = e / kOrthTile, row = e % kOrthTile;
            tile[row][col] = row < rows ? u[(long long)col * D + t0 + row] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (active)
            for (int r = g; r < rows; r += ngroups) cfmac(acc, tile[r][pi], tile[r][pj]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < np) {
        double2 tot = red[threadIdx.x];
        for (int q = 1; q < ngroups; ++q) tot = cadd(tot, red[q * np + threadIdx.x]);
        part[((long long)s * nch + c) * np + threadIdx.x] = tot;
    }
}

// One block per problem: G from the partial sums (chunk order), G = L L^H by
// Cholesky, T = L^-H (upper triangular, T[p][j] at p k + j).  A pivot below
// 1e-13 of the largest diagonal entry marks a direction already spanned by
// the earlier vectors: that column of T (and row) is zero, so the vector
// comes out as zero and takes no part in the others.  dropped[s] counts them.
__global__ void k_orth_factor(const double2* __restrict__ part, int nch, int k, double2* __restrict__ T,
                              int* __restrict__ dropped) {
    __shared__ double2 G[kOrthMaxK][kOrthMaxK];
    const int s = blockIdx.x;
    const int np = k * (k + 1) / 2;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        double2 tot = make_double2(0.0, 0.0);
        for (int c = 0; c < nch; ++c) tot = cadd(tot, part[((long long)s * nch + c) * np + p]);
        int i, j;
        orth_pair(p, k, &i, &j);
        G[i][j] = tot;                                  // G_ij = sum conj(U_i) U_j, i <= j
        G[j][i] = make_double2(tot.x, -tot.y);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // one thread factors (k <= 16); its tables live in shared memory, not in
    // a per-thread stack frame
    __shared__ double L[kOrthMaxK][kOrthMaxK][2];
    __shared__ double X[kOrthMaxK][kOrthMaxK][2];
    bool keep[kOrthMaxK];
    double gmax = 0.0;
    for (int i = 0; i < k; ++i) gmax = fmax(gmax, G[i][i].x);
    int nd = 0;
    for (int j = 0; j < k; ++j) {
        double d = G[j][j].x;
        for (int q = 0; q < j; ++q) d -= L[j][q][0] * L[j][q][0] + L[j][q][1] * L[j][q][1];
        keep[j] = d > 1e-13 * gmax && gmax > 0.0;
        if (!keep[j]) {
            ++nd;
            for (int i = j; i < k; ++i) L[i][j][0] = L[i][j][1] = 0.0;
            continue;
        }
        const double ljj = sqrt(d);
        L[j][j][0] = ljj;
        L[j][j][1] = 0.0;
        for (int i = j + 1; i < k; ++i) {
            // L_ij = (G_ij - sum_q L_iq conj(L_jq)) / L_jj, with G_ij = conj(G_ji) for i > j
            double re = G[i][j].x, im = G[i][j].y;
            for (int q = 0; q < j; ++q) {
                re -= L[i][q][0] * L[j][q][0] + L[i][q][1] * L[j][q][1];
                im -= L[i][q][1] * L[j][q][0] - L[i][q][0] * L[j][q][1];
            }
            L[i][j][0] = re / ljj;
            L[i][j][1] = im / ljj;
        }
    }
    // X = L^-1 (lower) by forward substitution, dropped rows and columns zero
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < k; ++i) X[i][j][0] = X[i][j][1] = 0.0;
        if (!keep[j]) continue;
        X[j][j][0] = 1.0 / L[j][j][0];
        for (int i = j + 1; i < k; ++i) {
            if (!keep[i]) continue;
            double re = 0.0, im = 0.0;
            for (int q = j; q < i; ++q) {
                re += L[i][q][0] * X[q][j][0] - L[i][q][1] * X[q][j][1];
                im += L[i][q][0] * X[q][j][1] + L[i][q][1] * X[q][j][0];
            }
            X[i][j][0] = -re / L[i][i][0];
            X[i][j][1] = -im / L[i][i][0];
        }
    }
    double2* Ts = T + (long long)s * k * k;
    for (int p = 0; p < k; ++p)
        for (int j = 0; j < k; ++j)   // T = X^H: T_pj = conj(X_jp)
            Ts[p * k + j] = make_double2(X[j][p][0], -X[j][p][1]);
    dropped[s] = nd;
}

// U <- U T in place, one row per thread (T upper triangular).
__global__ void __launch_bounds__(256) k_orth_apply(double2* const* __restrict__ U, int D, int k,
                                                    const double2* __restrict__ T) {
    __shared__ double2 Ts[kOrthMaxK * kOrthMaxK];
    const int s = blockIdx.y;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) Ts[e] = T[(long long)s * k * k + e];
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    double2* u = U[s];
    double2 v[kOrthMaxK];
#pragma unroll
    for (int c = 0; c < kOrthMaxK; ++c)
        if (c < k) v[c] = u[(long long)c * D + r];
#pragma unroll
    for (int j = 0; j < kOrthMaxK; ++j) {
        if (j >= k) break;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int p = 0; p <= j; ++p) cfma(acc, v[p], Ts[p * k + j]);
        u[(long long)j * D + r] = acc;
    }
}

// Per-sample operator for the residual loss (FP32 coefficients).
struct FieldOpDesc {
    const float* eps;
    const float2* coef;   // [axp(nx) | axm(nx) | ayp(ny) | aym(ny)]
    const float2* sb;     // [sxb(nx) | syb(ny)]
    int nx, ny;
    float kh2;
};

// out[s][e][c] = (A f_c)[e] for the k complex columns of a [B][D][2k] tensor.
__global__ void k_fields_apply(const FieldOpDesc* __restrict__ ops, const float* __restrict__ in, int B, int D, int k,
                               float* __restrict__ out) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * D) return;
    const int s = (int)(idx / D), e = (int)(idx % D);
    const FieldOpDesc o = ops[s];
    const int nx = o.nx, ny = o.ny;
    const int j = e / nx, i = e % nx;
    const float2 axp = o.coef[i], axm = o.coef[nx + i];
    const float2 ayp = o.coef[2 * nx + j], aym = o.coef[2 * nx + ny + j];
    const int ip = (i == nx - 1) ? e - (nx - 1) : e + 1;
    const int im = (i == 0) ? e + (nx - 1) : e - 1;
    const int jp = (j == ny - 1) ? e - (ny - 1) * nx : e + nx;
    const int jm = (j == 0) ? e + (ny - 1) * nx : e - nx;
    float2 d = cadd(cadd(axp, axm), cadd(ayp, aym));
    d.x -= o.kh2 * o.eps[e];
    const float2* f = reinterpret_cast<const float2*>(in) + (long long)s * D * k;
    float2* y = reinterpret_cast<float2*>(out) + (long long)s * D * k;
    for (int c = 0; c < k; ++c) {
        float2 acc = cmul(d, f[(long long)e * k + c]);
        cfms(acc, axp, f[(long long)ip * k + c]);
        cfms(acc, axm, f[(long long)im * k + c]);
        cfms(acc, ayp, f[(long long)jp * k + c]);
        cfms(acc, aym, f[(long long)jm * k + c]);
        y[(long long)e * k + c] = acc;
    }
}

// A^H g = conj(S_b A S_b^-1 conj(g)) (A^T = S_b A S_b^-1 from the complex
// symmetry of S_b A): the two diagonal steps around k_fields_apply.
__global__ void k_adj_pre(const FieldOpDesc* __restrict__ ops, const float* __restrict__ g, int B, int D, int k,
                          float* __restrict__ u) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * D * k) return;
    const int s = (int)(idx / ((long long)D * k));
    const int e = (int)((idx / k) % D);
    const FieldOpDesc o = ops[s];
    const float2 sb = cmul(o.sb[e % o.nx], o.sb[o.nx + e / o.nx]);
    const float2 gv = reinterpret_cast<const float2*>(g)[idx];
    const float2 cg = make_float2(gv.x, -gv.y);
    // conj(g) / sb
    const float den = sb.x * sb.x + sb.y * sb.y;
    reinterpret_cast<float2*>(u)[idx] = make_float2((cg.x * sb.x + cg.y * sb.y) / den, (cg.y * sb.x - cg.x * sb.y) / den);
}
__global__ void k_adj_post(const FieldOpDesc* __restrict__ ops, float* __restrict__ v, int B, int D, int k) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * D * k) return;
    const int s = (int)(idx / ((long long)D * k));
    const int e = (int)((idx / k) % D);
    const FieldOpDesc o = ops[s];
    const float2 sb = cmul(o.sb[e % o.nx], o.sb[o.nx + e / o.nx]);
    float2* vp = reinterpret_cast<float2*>(v) + idx;
    const float2 w = cmul(sb, *vp);
    *vp = make_float2(w.x, -w.y);
}

inline unsigned nblk(long long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

struct OutputBase {
    float* dev;          // D x 2k FP32, the network's output layout
    int nx, ny;
    double wavelength;   // metres; 0 = every wavelength of this grid
};

}  // namespace cnn
}  // namespace ddg

// ---------------------------------------------------------------- predictor object
struct ddg_predictor {
    int cin = 4, levels = 0, k = 0;
    int ch[ddg::cnn::kMaxLevels] = {};
    int device = 0;
    long long nparams = 0;
    std::vector<ddg::cnn::Layer> layers;
    float* theta = nullptr;       // FP32 master
    bf16* theta_bf = nullptr;     // BF16 copy
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long step = 0;
    long long launches = 0;       // kernels launched by this predictor
    int loss_kind = 0;            // 0: projection loss (Eq. 5), 1: residual loss (Eq. 6)
    bool last_finite = true;      // the last loss was finite (else the next Adam step is skipped)
    bf16* wk = nullptr;           // per-layer re-laid-out BF16 weights (forward / backward)
    // activation workspace
    void* act = nullptr;
    size_t act_bytes = 0;
    double* d_loss = nullptr;     // per-sample losses
    float2* in_field = nullptr;   // cin = 6: the approximate field of the grid, normalised
    int field_nx = 0, field_ny = 0;
    // optional fixed output offsets (D x 2k each, the output layout), keyed by
    // grid and wavelength (wavelength 0: any wavelength of that grid)
    std::vector<ddg::cnn::OutputBase> bases;
    std::vector<const float*> base_ptrs;   // host copy of the last batch's offset pointers
    double2* orth_ws = nullptr;   // K13: Gram partial sums, factors, dropped counts
    size_t orth_bytes = 0;
    int* d_err = nullptr;         // a bounded wait in a tensor-core convolution gave up
    int tensor_cores = 5;         // bit 0: forward 3x3 convolutions on tcgen05 where the channels allow;
                                  // bit 1: the backward convolutions (data and weight gradients) too;
                                  // bit 2: forward ones with a plain input from TMA tiles (k_conv3_tma)
    int sm_count = 152;
    void* d_desc = nullptr;       // InputDesc / pointer arrays (device)
    size_t desc_bytes = 0;
};

namespace ddg {
namespace cnn {

static void** base_slots(ddg_predictor* P, int n);

static int layer_index(const ddg_predictor* P, bool dec, int level, int ab) {
    // enc l: 2l + ab ; dec l (l = L-2 .. 0): 2L + 2 (L-2-l) + ab ; head: last
    if (!dec) return 2 * level + ab;
    return 2 * P->levels + 2 * (P->levels - 2 - level) + ab;
}

struct Acts {
    // device pointers for one batch size / grid
    bf16* x0;
    bf16* x0p;     // the input with its channels zero-padded to 16 (TMA-tile first layer)
    bf16* ea[kMaxLevels];
    bf16* eb[kMaxLevels];
    bf16* pooled[kMaxLevels];
    bf16* da[kMaxLevels];
    bf16* db[kMaxLevels];
    float* y;
    float* gy;
    float* y2;     // residual loss: A V, then S_b^-1 conj(dl/dW)
    float* gy2;    // residual loss: dl/dW
    float* g1;     // scratch gradients (largest tensor)
    float* g2;
    float* g3;
    float* gskip[kMaxLevels];
    double2* lpart;   // loss partial sums (train): [B][loss blocks][entries]
    double2* lz;      // loss solutions (train): [B][k + 1]
};

// blocks per sample of the loss partial sums, and 256-pixel tiles per block
static void loss_blocks(int D, int* nch, int* tpb) {
    const int ntiles = (D + kLossTile - 1) / kLossTile;
    *nch = std::min(256, ntiles);
    *tpb = (ntiles + *nch - 1) / *nch;
}

// Activation workspace of one batch; `train` adds the gradient buffers (the
// forward-only calls, prediction and predictor_forward, need none of them).
static size_t plan_acts(const ddg_predictor* P, int B, int H, int W, char* base, Acts* A, bool train) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) / 256 * 256;
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const int L = P->levels;
    size_t maxg = 0;
    A->x0 = (bf16*)take(sizeof(bf16) * (size_t)B * H * W * P->cin);
    A->x0p = (bf16*)take(sizeof(bf16) * (size_t)B * H * W * kInPad);
    for (int l = 0; l < L; ++l) {
        const size_t px = (size_t)B * (H >> l) * (W >> l);
        if (l > 0) A->pooled[l] = (bf16*)take(sizeof(bf16) * px * P->ch[l - 1]);
        A->ea[l] = (bf16*)take(sizeof(bf16) * px * P->ch[l]);
        A->eb[l] = (bf16*)take(sizeof(bf16) * px * P->ch[l]);
        if (l < L - 1) {
            A->da[l] = (bf16*)take(sizeof(bf16) * px * P->ch[l]);
            A->db[l] = (bf16*)take(sizeof(bf16) * px * P->ch[l]);
            A->gskip[l] = train ? (float*)take(sizeof(float) * px * P->ch[l]) : nullptr;
            maxg = std::max(maxg, px * (size_t)(P->ch[l] + P->ch[l + 1]));
        }
        maxg = std::max(maxg, px * (size_t)std::max(P->ch[l], l > 0 ? P->ch[l - 1] : P->cin));
    }
    A->y = (float*)take(sizeof(float) * (size_t)B * H * W * 2 * P->k);
    if (!train) {
        A->gy = A->y2 = A->gy2 = A->g1 = A->g2 = A->g3 = nullptr;
        A->lpart = A->lz = nullptr;
        return off + 256;
    }
    A->gy = (float*)take(sizeof(float) * (size_t)B * H * W * 2 * P->k);
    A->y2 = (float*)take(sizeof(float) * (size_t)B * H * W * 2 * P->k);
    A->gy2 = (float*)take(sizeof(float) * (size_t)B * H * W * 2 * P->k);
    A->g1 = (float*)take(sizeof(float) * maxg);
    A->g2 = (float*)take(sizeof(float) * maxg);
    A->g3 = (float*)take(sizeof(float) * maxg);
    int nch = 0, tpb = 0;
    loss_blocks(H * W, &nch, &tpb);
    A->lpart = (double2*)take(sizeof(double2) * (size_t)B * nch * loss_entries(P->k));
    A->lz = (double2*)take(sizeof(double2) * (size_t)B * (P->k + 1));
    return off + 256;
}

static ddg_status ensure_acts(ddg_predictor* P, int B, int H, int W, Acts* A, bool train) {
    const size_t need = plan_acts(P, B, H, W, nullptr, A, train);
    if (need > P->act_bytes) {
        cudaFree(P->act);
        P->act = nullptr;
        P->act_bytes = 0;
        cudaError_t e = cudaMalloc(&P->act, need);
        if (e != cudaSuccess) { cudaGetLastError(); set_error("predictor: cudaMalloc of %zu bytes failed", need); return DDG_ENOMEM; }
        P->act_bytes = need;
    }
    plan_acts(P, B, H, W, reinterpret_cast<char*>(P->act), A, train);
    return DDG_OK;
}

static const bf16* wbf(const ddg_predictor* P, int li) { return P->theta_bf + P->layers[li].w_off; }
static const float* bias32(const ddg_predictor* P, int li) { return P->theta + P->layers[li].b_off; }

template <class LD, typename TOUT>
static ddg_status conv3(ddg_predictor* P, const LD& ld, int B, int H, int W, int Ci, int Co, const bf16* wk,
                        const float* bias, int relu, TOUT* out, cudaStream_t st) {
    dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY, B * ((Co + COB - 1) / COB));
    ++P->launches;
    k_conv3<LD, TOUT><<<grid, 256, 0, st>>>(ld, B, H, W, Ci, Co, wk, bias, relu, out);
    DDG_CHECK_LAUNCH("k_conv3");
    return DDG_OK;
}

// cuTensorMapEncodeTiled from the driver (looked up once; null if unavailable).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// The TMA-tile forward convolution (k_conv3_tma) when its conditions hold: a
// plain input tensor (no upsampled concatenation), Ci and Co multiples of 16
// (Co <= 256), the grid a multiple of the 16 x 8 tile, the weights and two
// halo tiles within shared memory, and a tensor map the driver accepts.
// ci_pad > 0: the input tensor holds ci_pad >= Ly.ci channels, the ones past
// Ly.ci zero (the first layer's padded input), and the weights are padded to
// match.  Returns false (nothing launched) otherwise.
static bool conv_fwd_tma(ddg_predictor* P, const LoadCat& ld, int B, int H, int W, int li, bf16* out,
                         cudaStream_t st, ddg_status* status, int ci_pad = 0) {
    const Layer& Ly = P->layers[li];
    const int Ci = ci_pad > 0 ? ci_pad : Ly.ci, Co = Ly.co;
    if (Ci < Ly.ci) return false;
    // the decoder's input: nearest-upsampled x1 (half resolution) then x2
    const bool up = ld.up1 && ld.c2 > 0;
    const int c1 = up ? ld.c1 : 0;
    const size_t smem = tmc::smem_bytes(Ci, Co, c1);
    const bool shapes = up ? (ci_pad == 0 && ld.c1 + ld.c2 == Ci && ld.c1 % 8 == 0 && ld.c2 % 8 == 0 && ld.x2 &&
                              ld.h1 * 2 == H && ld.w1 * 2 == W && (reinterpret_cast<uintptr_t>(ld.x2) & 15) == 0)
                           : (!ld.up1 && ld.c2 == 0 && ld.c1 == Ci);
    if ((P->tensor_cores & 5) != 5 || !shapes || !ld.x1 || Ci % 16 != 0 || Co % 16 != 0 || Co > 256 ||
        H % tmc::TH != 0 || W % tmc::TW != 0 || (reinterpret_cast<uintptr_t>(ld.x1) & 15) != 0 ||
        smem > 227 * 1024)
        return false;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    // 4D maps over (C, W, H, B) of an NHWC BF16 tensor, boxes of 8 channels
    auto make_map = [&](CUtensorMap* m, const bf16* base, int C, int Wd, int Hd, int bw, int bh) {
        const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)Wd, (cuuint64_t)Hd, (cuuint64_t)B};
        const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)Wd * C * 2, (cuuint64_t)Hd * Wd * C * 2};
        const cuuint32_t box[4] = {8, (cuuint32_t)bw, (cuuint32_t)bh, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap map, mapu;
    if (up) {
        if (!make_map(&map, ld.x2, ld.c2, W, H, tmc::HWD, tmc::HH) ||
            !make_map(&mapu, ld.x1, ld.c1, W / 2, H / 2, tmc::CW, tmc::CH))
            return false;
    } else {
        if (!make_map(&map, ld.x1, Ci, W, H, tmc::HWD, tmc::HH)) return false;
        mapu = map;   // unused
    }
    *status = DDG_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        *status = cuda_status(e, what);
        return true;
    };
    cudaError_t e = cudaFuncSetAttribute(k_conv3_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv3_tma, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return fail(e, "cudaFuncSetAttribute(k_conv3_tma)");
    // CTAs per SM: shared memory (228 KB an SM, 1 KB of it reserved per CTA),
    // at most 8, and the 512 tensor-memory columns (two accumulators per CTA)
    int nb = std::min(8, (int)((228 * 1024) / (smem + 1024)));
    nb = std::max(1, std::min(nb, (int)(512 / (2 * tc::tmem_cols(Co)))));
    const long long ntiles = (long long)B * (H / tmc::TH) * (W / tmc::TW);
    const unsigned grid = (unsigned)std::min<long long>(ntiles, (long long)P->sm_count * nb);
    P->launches += 2;
    k_w_tma<<<nblk((long long)Co * Ci * 9), 256, 0, st>>>(wbf(P, li), Co, Ly.ci, Ci, P->wk);
    k_conv3_tma<<<grid, up ? tmc::kThreadsUp : tmc::kThreads, smem, st>>>(map, mapu, c1, B, H, W, Ci, Co, P->wk,
                                                                         bias32(P, li), 1, out, P->d_err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e, "k_conv3_tma");
    return true;
}

// Forward 3x3 convolution of layer li: from TMA tiles when k_conv3_tma's
// conditions hold; else tensor cores with the gather when the channel counts
// allow 16-byte gathers and N = Co (multiples of 16, Co <= 256); else CUDA cores.
// ci_pad > 0: the input holds ci_pad >= Ly.ci channels, the extra ones zero
// (tensor-core paths only; the weights are padded with zeros to match).
static ddg_status conv_fwd(ddg_predictor* P, const LoadCat& ld, int B, int H, int W, int li, bf16* out,
                           cudaStream_t st, int ci_pad = 0) {
    const Layer& Ly = P->layers[li];
    ddg_status tst = DDG_OK;
    if (conv_fwd_tma(P, ld, B, H, W, li, out, st, &tst, ci_pad)) return tst;
    const int Ci = ci_pad > 0 ? ci_pad : Ly.ci;
    const bool tcok = (P->tensor_cores & 1) && Ci % 16 == 0 && Ly.co % 16 == 0 && Ly.co <= 256 &&
                      ld.c1 % 8 == 0 && ld.c2 % 8 == 0;
    ++P->launches;
    if (!tcok) {
        if (ci_pad > 0) {
            set_error("predictor: a padded input needs the tensor-core path");
            return DDG_EINVAL;
        }
        k_w_fwd<<<nblk((long long)Ly.co * Ly.ci * 9), 256, 0, st>>>(wbf(P, li), Ly.co, Ly.ci, P->wk);
        return conv3(P, ld, B, H, W, Ly.ci, Ly.co, P->wk, bias32(P, li), 1, out, st);
    }
    k_w_tc<<<nblk((long long)Ly.co * Ci * 9), 256, 0, st>>>(wbf(P, li), Ly.co, Ly.ci, Ci, P->wk);
    const size_t smem = tc::smem_bytes(Ly.co);
    DDG_CHECK_CUDA(cudaFuncSetAttribute(k_conv3_tc<LoadCat, bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    const long long npx = (long long)B * H * W;
    ++P->launches;
    k_conv3_tc<LoadCat, bf16><<<(unsigned)((npx + tc::kM - 1) / tc::kM), tc::kThreads, smem, st>>>(
        ld, B, H, W, Ci, Ly.co, P->wk, bias32(P, li), 1, out, P->d_err);
    DDG_CHECK_LAUNCH("k_conv3_tc");
    return DDG_OK;
}

// Reads and clears the tensor-core convolutions' wait flag (after a stream sync).
static ddg_status check_tc(ddg_predictor* P, cudaStream_t st) {
    int h = 0;
    DDG_CHECK_CUDA(cudaMemcpyAsync(&h, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DDG_CHECK_CUDA(cudaStreamSynchronize(st));
    if (h) {
        DDG_CHECK_CUDA(cudaMemsetAsync(P->d_err, 0, sizeof(int), st));
        set_error("predictor: a tensor-core convolution's wait did not complete within its time limit");
        return DDG_ETIMEOUT;
    }
    return DDG_OK;
}

// forward pass for B samples of one grid size; result in A->y
static ddg_status forward(ddg_predictor* P, int B, int H, int W, Acts* A, cudaStream_t st) {
    const int L = P->levels;
    const bf16* h = A->x0;
    int hc = P->cin;
    for (int l = 0; l < L; ++l) {
        const int Hl = H >> l, Wl = W >> l;
        const bf16* in = h;
        if (l > 0) {
            ++P->launches;
            k_avgpool2<<<nblk((long long)B * Hl * Wl * hc), 256, 0, st>>>(h, B, Hl * 2, Wl * 2, hc, A->pooled[l]);
            in = A->pooled[l];
        }
        for (int ab = 0; ab < 2; ++ab) {
            const int li = layer_index(P, false, l, ab);
            const Layer& Ly = P->layers[li];
            if (l == 0 && ab == 0 && Ly.ci <= kInPad && (P->tensor_cores & 1) && Ly.co % 16 == 0 &&
                Ly.co <= 256) {
                // the first layer on the tensor cores, from the input copy
                // zero-padded to 16 channels (zero weights for the padding)
                LoadCat ldp{A->x0p, kInPad, 0, Hl, Wl, nullptr, 0};
                DDG_TRY(conv_fwd(P, ldp, B, Hl, Wl, li, A->ea[0], st, kInPad));
                continue;
            }
            LoadCat ld{ab == 0 ? in : A->ea[l], Ly.ci, 0, Hl, Wl, nullptr, 0};
            DDG_TRY(conv_fwd(P, ld, B, Hl, Wl, li, ab == 0 ? A->ea[l] : A->eb[l], st));
        }
        h = A->eb[l];
        hc = P->ch[l];
    }
    for (int l = L - 2; l >= 0; --l) {
        const int Hl = H >> l, Wl = W >> l;
        for (int ab = 0; ab < 2; ++ab) {
            const int li = layer_index(P, true, l, ab);
            const Layer& Ly = P->layers[li];
            LoadCat ld = ab == 0 ? LoadCat{h, hc, 1, Hl / 2, Wl / 2, A->eb[l], P->ch[l]}
                                 : LoadCat{A->da[l], Ly.ci, 0, Hl, Wl, nullptr, 0};
            DDG_TRY(conv_fwd(P, ld, B, Hl, Wl, li, ab == 0 ? A->da[l] : A->db[l], st));
        }
        h = A->db[l];
        hc = P->ch[l];
    }
    const int lh = (int)P->layers.size() - 1;
    ++P->launches;
    if (hc % 8 == 0 && hc <= 256 && 2 * P->k <= kHeadMaxO)
        k_head_fwd_px<<<nblk((long long)B * H * W), 256, sizeof(float) * (size_t)(hc + 1) * 2 * P->k, st>>>(
            h, (long long)B * H * W, hc, 2 * P->k, wbf(P, lh), bias32(P, lh), A->y);
    else
        k_head_fwd<<<nblk((long long)B * H * W * 2 * P->k), 256, 0, st>>>(h, (long long)B * H * W, hc, 2 * P->k,
                                                                        wbf(P, lh), bias32(P, lh), A->y);
    if (!P->bases.empty()) {
        const long long n = (long long)H * W * 2 * P->k;
        ++P->launches;
        k_add_base<<<nblk(n * B), 256, 0, st>>>(A->y, reinterpret_cast<const float* const*>(base_slots(P, B)), n, B);
    }
    DDG_CHECK_LAUNCH("forward");
    return DDG_OK;
}

static unsigned wgrad_slices(long long ntiles, int blocks_yz) {
    long long want = std::max(1LL, (long long)(4 * 152) / std::max(1, blocks_yz));
    return (unsigned)std::min(ntiles, want);
}

template <class LX>
static ddg_status wgrad(ddg_predictor* P, const LX& lx, const float* g, const bf16* yout, int B, int H, int W, int li,
                        cudaStream_t st) {
    const Layer& Ly = P->layers[li];
    if ((P->tensor_cores & 2) && Ly.co % 16 == 0 && Ly.co <= 128 && Ly.ci % 16 == 0 &&
        (long long)B * H * W < (1LL << 31)) {
        // on the tensor cores (bit 2): D[co, tap Ci + ci] over the pixels
        const long long npx = (long long)B * H * W;
        const int ntn = (9 * Ly.ci + tcw::kWN - 1) / tcw::kWN;
        // three CTAs fit an SM (66.5 KB of shared memory, 128 tensor-memory columns each)
        const long long want = std::max(1LL, (long long)(3 * P->sm_count + ntn - 1) / ntn);
        long long per = (npx + want - 1) / want;
        per = std::max((long long)tc::kKC, (per + tc::kKC - 1) / tc::kKC * tc::kKC);
        const unsigned slices = (unsigned)((npx + per - 1) / per);
        const size_t smem = tcw::smem_bytes();
        DDG_CHECK_CUDA(cudaFuncSetAttribute(k_wgrad_tc<LX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ++P->launches;
        k_wgrad_tc<LX><<<dim3(ntn, slices), tc::kThreads, smem, st>>>(lx, g, yout, B, H, W, Ly.ci, Ly.co, per,
                                                                      P->grad + Ly.w_off, P->d_err);
        DDG_CHECK_LAUNCH("k_wgrad_tc");
        const long long pb = std::max(1024LL, (npx + 4 * P->sm_count - 1) / (4 * P->sm_count));
        ++P->launches;
        if (Ly.co % 4 == 0 && Ly.co <= 1024)
            k_bias_grad4<<<(unsigned)((npx + pb - 1) / pb), 256, 0, st>>>(g, yout, npx, Ly.co, pb,
                                                                          P->grad + Ly.b_off);
        else
            k_bias_grad<<<(unsigned)((npx + pb - 1) / pb), 256, 0, st>>>(g, yout, npx, Ly.co, pb,
                                                                         P->grad + Ly.b_off);
        DDG_CHECK_LAUNCH("k_bias_grad");
        return DDG_OK;
    }
    const long long ntiles = (long long)B * ((W + 15) / 16) * ((H + 15) / 16);
    const int gy = ((Ly.co + 15) / 16) * ((Ly.ci + 15) / 16);
    const unsigned sl = wgrad_slices(ntiles, gy);
    const int per = (int)((ntiles + sl - 1) / sl);
    dim3 grid(sl, gy);
    ++P->launches;
    k_conv3_wgrad<LX><<<grid, 256, 0, st>>>(lx, g, yout, B, H, W, Ly.ci, Ly.co, per, P->grad + Ly.w_off,
                                            P->grad + Ly.b_off);
    DDG_CHECK_LAUNCH("k_conv3_wgrad");
    return DDG_OK;
}

// gradient w.r.t. the input of conv layer li given the gradient g of its output (masked by ReLU'(yout))
static ddg_status bdata(ddg_predictor* P, const float* g, const bf16* yout, int B, int H, int W, int li, float* gx,
                        cudaStream_t st) {
    const Layer& Ly = P->layers[li];
    LoadGrad lg{g, yout, Ly.co};
    if ((P->tensor_cores & 2) && Ly.co % 16 == 0 && Ly.ci % 16 == 0 && Ly.ci <= 256) {
        // on the tensor cores: a forward convolution from Co to Ci channels
        // with the flipped taps; the masked gradient enters in BF16
        ++P->launches;
        k_w_tc_bwd<<<nblk((long long)Ly.co * Ly.ci * 9), 256, 0, st>>>(wbf(P, li), Ly.co, Ly.ci, P->wk);
        const size_t smem = tc::smem_bytes(Ly.ci);
        DDG_CHECK_CUDA(cudaFuncSetAttribute(k_conv3_tc<LoadGrad, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        const long long npx = (long long)B * H * W;
        ++P->launches;
        k_conv3_tc<LoadGrad, float><<<(unsigned)((npx + tc::kM - 1) / tc::kM), tc::kThreads, smem, st>>>(
            lg, B, H, W, Ly.co, Ly.ci, P->wk, nullptr, 0, gx, P->d_err);
        DDG_CHECK_LAUNCH("k_conv3_tc (backward data)");
        return DDG_OK;
    }
    ++P->launches;
    k_w_bwd<<<nblk((long long)Ly.co * Ly.ci * 9), 256, 0, st>>>(wbf(P, li), Ly.co, Ly.ci, P->wk);
    return conv3(P, lg, B, H, W, Ly.co, Ly.ci, P->wk, (const float*)nullptr, 0, gx, st);
}

// backward pass: A->gy holds d loss / d y; accumulates into P->grad
static ddg_status backward(ddg_predictor* P, int B, int H, int W, Acts* A, cudaStream_t st) {
    const int L = P->levels;
    const int lh = (int)P->layers.size() - 1;
    const long long px0 = (long long)B * H * W;
    const int O = 2 * P->k, C0 = P->ch[0];
    const bf16* hin = L > 1 ? A->db[0] : A->eb[0];   // input of the 1x1 head
    ++P->launches;
    const size_t hsm = sizeof(float) * (size_t)kHeadTile * (O + head_cp(C0));
    if (O * (head_cp(C0) / 4) <= 256 * kHeadPairs && hsm <= 48 * 1024) {
        const long long pb = std::max(1024LL, (px0 + 4 * P->sm_count - 1) / (4 * P->sm_count));
        k_head_bwd_w4<<<(unsigned)((px0 + pb - 1) / pb), 256, hsm, st>>>(A->gy, hin, px0, C0, O, pb,
                                                                          P->grad + P->layers[lh].w_off,
                                                                          P->grad + P->layers[lh].b_off);
    } else {
        k_head_bwd_w<<<O * (C0 + 1), 256, 0, st>>>(A->gy, hin, px0, C0, O, P->grad + P->layers[lh].w_off,
                                                  P->grad + P->layers[lh].b_off);
    }
    ++P->launches;
    if (C0 % 8 == 0 && C0 <= 256 && O <= kHeadMaxO)
        k_head_bwd_data_px<<<nblk(px0), 256, sizeof(float) * (size_t)C0 * O, st>>>(A->gy, px0, C0, O, wbf(P, lh),
                                                                                   A->g1);
    else
        k_head_bwd_data<<<nblk(px0 * C0), 256, 0, st>>>(A->gy, px0, C0, O, wbf(P, lh), A->g1);
    DDG_CHECK_LAUNCH("head backward");
    float* gh = A->g1;      // gradient w.r.t. the current level's output (post-ReLU)
    float* ga = A->g2;
    float* gx = A->g3;
    for (int l = 0; l <= L - 2; ++l) {
        const int Hl = H >> l, Wl = W >> l;
        const int lb = layer_index(P, true, l, 1), la = layer_index(P, true, l, 0);
        LoadCat xb{A->da[l], P->ch[l], 0, Hl, Wl, nullptr, 0};
        DDG_TRY(wgrad(P, xb, gh, A->db[l], B, Hl, Wl, lb, st));
        DDG_TRY(bdata(P, gh, A->db[l], B, Hl, Wl, lb, ga, st));
        const bf16* below = (l + 1 == L - 1) ? A->eb[L - 1] : A->db[l + 1];
        const int cu = P->ch[l + 1];
        LoadCat xa{below, cu, 1, Hl / 2, Wl / 2, A->eb[l], P->ch[l]};
        DDG_TRY(wgrad(P, xa, ga, A->da[l], B, Hl, Wl, la, st));
        DDG_TRY(bdata(P, ga, A->da[l], B, Hl, Wl, la, gx, st));
        const long long nlow = (long long)B * (Hl / 2) * (Wl / 2) * cu;
        const long long nsk = (long long)B * Hl * Wl * P->ch[l];
        ++P->launches;
        k_split_cat_bwd<<<nblk(nlow + nsk), 256, 0, st>>>(gx, B, Hl, Wl, cu, P->ch[l], gh, A->gskip[l]);
        DDG_CHECK_LAUNCH("k_split_cat_bwd");
    }
    for (int l = L - 1; l >= 0; --l) {
        const int Hl = H >> l, Wl = W >> l;
        const long long n = (long long)B * Hl * Wl * P->ch[l];
        if (l < L - 1) {
            ++P->launches;
            k_add<<<nblk(n), 256, 0, st>>>(gh, A->gskip[l], n);
        }
        const int lb = layer_index(P, false, l, 1), la = layer_index(P, false, l, 0);
        LoadCat xb{A->ea[l], P->ch[l], 0, Hl, Wl, nullptr, 0};
        DDG_TRY(wgrad(P, xb, gh, A->eb[l], B, Hl, Wl, lb, st));
        DDG_TRY(bdata(P, gh, A->eb[l], B, Hl, Wl, lb, ga, st));
        const bf16* in = l > 0 ? A->pooled[l] : A->x0;
        const int cin = l > 0 ? P->ch[l - 1] : P->cin;
        LoadCat xa{in, cin, 0, Hl, Wl, nullptr, 0};
        DDG_TRY(wgrad(P, xa, ga, A->ea[l], B, Hl, Wl, la, st));
        if (l > 0) {
            DDG_TRY(bdata(P, ga, A->ea[l], B, Hl, Wl, la, gx, st));
            const long long nin = (long long)B * (Hl * 2) * (Wl * 2) * cin;
            ++P->launches;
            k_avgpool2_bwd<<<nblk(nin), 256, 0, st>>>(gx, B, Hl * 2, Wl * 2, cin, gh, 0);
            DDG_CHECK_LAUNCH("k_avgpool2_bwd");
        }
    }
    return DDG_OK;
}

static bool same_wavelength(double a, double b) { return fabs(a - b) <= 1e-9 * fmax(fabs(a), fabs(b)); }

// The output offset of one problem: the entry of its grid and wavelength,
// else the entry of its grid for every wavelength, else none.
static const OutputBase* find_base(const ddg_predictor* P, const ddg_op* A) {
    const OutputBase* any = nullptr;
    for (const OutputBase& b : P->bases) {
        if (b.nx != A->nx || b.ny != A->ny) continue;
        if (b.wavelength == 0.0) any = &b;
        else if (same_wavelength(b.wavelength, A->wavelength)) return &b;
    }
    return any;
}

static ddg_status check_batch(const ddg_predictor* P, int n, const ddg_op* const* A, int* H, int* W) {
    if (!P || n < 1 || !A) { set_error("predictor: bad arguments"); return DDG_EINVAL; }
    for (int s = 0; s < n; ++s) {
        if (!A[s]) { set_error("predictor: NULL operator %d", s); return DDG_EINVAL; }
        if (A[s]->nx != A[0]->nx || A[s]->ny != A[0]->ny) { set_error("predictor: a batch needs one grid size"); return DDG_EINVAL; }
    }
    const int div = 1 << (P->levels - 1);
    if (A[0]->nx % div || A[0]->ny % div) {
        set_error("predictor: grid %dx%d not divisible by %d", A[0]->nx, A[0]->ny, div);
        return DDG_EINVAL;
    }
    if (!P->bases.empty())
        for (int s = 0; s < n; ++s)
            if (!find_base(P, A[s])) {
                set_error("predictor: no output base for the %dx%d grid at wavelength %g m (problem %d)", A[s]->nx,
                          A[s]->ny, A[s]->wavelength, s);
                return DDG_EINVAL;
            }
    if (P->cin == 6 && (!P->in_field || P->field_nx != A[0]->nx || P->field_ny != A[0]->ny)) {
        set_error("predictor: this network takes an input field of the %dx%d grid (predictor_set_input_field)",
                  A[0]->nx, A[0]->ny);
        return DDG_EINVAL;
    }
    *H = A[0]->ny;
    *W = A[0]->nx;
    return DDG_OK;
}

static FieldOpDesc* field_ops(ddg_predictor* P, int n);

static ddg_status build_input(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma, double j_c,
                              Acts* acts, cudaStream_t st) {
    std::vector<InputDesc> hd(n);
    std::vector<FieldOpDesc> hf(n);
    for (int s = 0; s < n; ++s) {
        hd[s] = InputDesc{A[s]->eps_d, A[s]->nx, A[s]->ny, A[s]->npml_x, A[s]->wavelength};
        hf[s] = FieldOpDesc{A[s]->eps_f, A[s]->coef_f, A[s]->sb_f, A[s]->nx, A[s]->ny, (float)(A[s]->kh * A[s]->kh)};
    }
    const size_t need = ((sizeof(InputDesc) * n + 15) / 16) * 16 + ((sizeof(FieldOpDesc) * n + 15) / 16) * 16 +
                        sizeof(void*) * 3 * n + 256;
    if (need > P->desc_bytes) {
        cudaFree(P->d_desc);
        P->d_desc = nullptr;
        P->desc_bytes = 0;
        DDG_CHECK_CUDA(cudaMalloc(&P->d_desc, need));
        P->desc_bytes = need;
    }
    DDG_CHECK_CUDA(cudaMemcpyAsync(P->d_desc, hd.data(), sizeof(InputDesc) * n, cudaMemcpyHostToDevice, st));
    DDG_CHECK_CUDA(cudaMemcpyAsync(field_ops(P, n), hf.data(), sizeof(FieldOpDesc) * n, cudaMemcpyHostToDevice, st));
    if (!P->bases.empty()) {
        // per-problem output offsets (checked to exist by check_batch); the
        // host array must outlive the asynchronous copy
        P->base_ptrs.assign(n, nullptr);
        for (int s = 0; s < n; ++s) P->base_ptrs[s] = find_base(P, A[s])->dev;
        DDG_CHECK_CUDA(cudaMemcpyAsync(base_slots(P, n), P->base_ptrs.data(), sizeof(void*) * n,
                                       cudaMemcpyHostToDevice, st));
    }
    const int H = A[0]->ny, W = A[0]->nx;
    ++P->launches;
    k_input<<<nblk((long long)n * H * W), 256, 0, st>>>(reinterpret_cast<InputDesc*>(P->d_desc), n, H, W, i_src,
                                                       sigma, j_c, P->in_field, P->cin, acts->x0, acts->x0p);
    DDG_CHECK_LAUNCH("k_input");
    return DDG_OK;
}

static FieldOpDesc* field_ops(ddg_predictor* P, int n) {
    return reinterpret_cast<FieldOpDesc*>(reinterpret_cast<char*>(P->d_desc) + ((sizeof(InputDesc) * n + 15) / 16) * 16);
}
static void** ptr_slots(ddg_predictor* P, int n) {
    return reinterpret_cast<void**>(reinterpret_cast<char*>(field_ops(P, n)) +
                                    ((sizeof(FieldOpDesc) * n + 15) / 16) * 16);
}
// n output-offset pointers behind the 2n pointer slots
static void** base_slots(ddg_predictor* P, int n) { return ptr_slots(P, n) + 2 * n; }

static void free_predictor(ddg_predictor* P) {
    if (!P) return;
    cudaFree(P->theta);
    cudaFree(P->theta_bf);
    cudaFree(P->grad);
    cudaFree(P->adam_m);
    cudaFree(P->adam_v);
    cudaFree(P->wk);
    cudaFree(P->act);
    cudaFree(P->d_loss);
    cudaFree(P->in_field);
    for (auto& b : P->bases) cudaFree(b.dev);
    cudaFree(P->orth_ws);
    cudaFree(P->d_err);
    cudaFree(P->d_desc);
    delete P;
}

}  // namespace cnn
}  // namespace ddg

using namespace ddg;
using namespace ddg::cnn;

static ddg_status create_predictor(int k, int levels, const int* channels, int cin, ddg_predictor** out) {
    if (!out) { set_error("predictor_create: out is NULL"); return DDG_EINVAL; }
    *out = nullptr;
    if (k < 1 || k > 16 || levels < 1 || levels > kMaxLevels || !channels) {
        set_error("predictor_create: need 1 <= k <= 16, 1 <= levels <= %d, channels", kMaxLevels);
        return DDG_EINVAL;
    }
    ddg_predictor* P = new (std::nothrow) ddg_predictor();
    if (!P) return DDG_ENOMEM;
    P->cin = cin;
    P->k = k;
    P->levels = levels;
    for (int l = 0; l < levels; ++l) {
        if (channels[l] < 1 || channels[l] > 1024) { delete P; set_error("predictor_create: bad channel count"); return DDG_EINVAL; }
        P->ch[l] = channels[l];
    }
    cudaGetDevice(&P->device);
    cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, P->device);
    if (P->sm_count <= 0) P->sm_count = 152;
    long long off = 0;
    size_t maxw = 0;
    auto add = [&](int co, int ci, int kk) {
        Layer Ly{co, ci, kk, off, off + (long long)co * ci * kk * kk};
        off = Ly.b_off + co;
        P->layers.push_back(Ly);
        maxw = std::max(maxw, (size_t)co * std::max(ci, kk == 3 ? kInPad : 0) * kk * kk);   // padded inputs too
    };
    for (int l = 0; l < levels; ++l) {
        add(P->ch[l], l == 0 ? P->cin : P->ch[l - 1], 3);
        add(P->ch[l], P->ch[l], 3);
    }
    for (int l = levels - 2; l >= 0; --l) {
        add(P->ch[l], P->ch[l + 1] + P->ch[l], 3);
        add(P->ch[l], P->ch[l], 3);
    }
    add(2 * k, P->ch[0], 1);
    P->nparams = off;
    const size_t n = (size_t)off;
    cudaError_t e = cudaMalloc(&P->theta, 4 * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->theta_bf, 2 * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->grad, 4 * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->adam_m, 4 * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->adam_v, 4 * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->wk, 2 * maxw);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_loss, sizeof(double) * 4096);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(P->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(P->theta, 0, 4 * n);
    if (e == cudaSuccess) e = cudaMemset(P->theta_bf, 0, 2 * n);
    if (e == cudaSuccess) e = cudaMemset(P->adam_m, 0, 4 * n);
    if (e == cudaSuccess) e = cudaMemset(P->adam_v, 0, 4 * n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_predictor(P);
        set_error("predictor_create: cudaMalloc failed");
        return DDG_ENOMEM;
    }
    *out = P;
    return DDG_OK;
}

extern "C" ddg_status predictor_create(int k, int levels, const int* channels, ddg_predictor** out) {
    return create_predictor(k, levels, channels, 4, out);
}

extern "C" ddg_status predictor_create_with_field(int k, int levels, const int* channels, ddg_predictor** out) {
    return create_predictor(k, levels, channels, 6, out);
}

extern "C" ddg_status predictor_set_input_field(ddg_predictor* P, const double* f, int nx, int ny, void* stream) {
    if (!P || !f || nx < 1 || ny < 1) { set_error("predictor_set_input_field: bad arguments"); return DDG_EINVAL; }
    if (P->cin != 6) { set_error("predictor_set_input_field: network created without an input field"); return DDG_EINVAL; }
    const long long D = (long long)nx * ny;
    cudaStream_t st = as_stream(stream);
    if (P->field_nx * (long long)P->field_ny != D) {
        cudaFree(P->in_field);
        P->in_field = nullptr;
        P->field_nx = P->field_ny = 0;
        cudaError_t e = cudaMalloc(&P->in_field, sizeof(float2) * D);
        if (e != cudaSuccess) { cudaGetLastError(); set_error("predictor_set_input_field: cudaMalloc failed"); return DDG_ENOMEM; }
    }
    P->field_nx = nx;
    P->field_ny = ny;
    ++P->launches;
    k_field_in<<<1, 1024, 0, st>>>(reinterpret_cast<const double2*>(f), D, P->in_field);
    DDG_CHECK_LAUNCH("k_field_in");
    return DDG_OK;
}

static ddg_status set_output_base(ddg_predictor* P, const double* U, int nx, int ny, double wavelength,
                                  double scale, void* stream, const char* who) {
    if (!P || nx < 1 || ny < 1 || !(wavelength >= 0.0)) { set_error("%s: bad arguments", who); return DDG_EINVAL; }
    cudaStream_t st = as_stream(stream);
    if (!U) {   // remove every offset
        DDG_CHECK_CUDA(cudaStreamSynchronize(st));
        for (auto& b : P->bases) cudaFree(b.dev);
        P->bases.clear();
        return DDG_OK;
    }
    const long long D = (long long)nx * ny;
    OutputBase* slot = nullptr;
    for (auto& b : P->bases)
        if (b.nx == nx && b.ny == ny &&
            ((wavelength == 0.0 && b.wavelength == 0.0) ||
             (wavelength > 0.0 && b.wavelength > 0.0 && same_wavelength(b.wavelength, wavelength))))
            slot = &b;
    if (!slot) {
        float* d = nullptr;
        cudaError_t e = cudaMalloc(&d, sizeof(float) * D * 2 * P->k);
        if (e != cudaSuccess) { cudaGetLastError(); set_error("%s: cudaMalloc failed", who); return DDG_ENOMEM; }
        P->bases.push_back(OutputBase{d, nx, ny, wavelength});
        slot = &P->bases.back();
    }
    ++P->launches;
    k_base_in<<<nblk(D * P->k), 256, 0, st>>>(reinterpret_cast<const double2*>(U), D, P->k, scale, slot->dev);
    DDG_CHECK_LAUNCH("k_base_in");
    return DDG_OK;
}

extern "C" ddg_status predictor_set_output_base(ddg_predictor* P, const double* U, int nx, int ny, double scale,
                                                void* stream) {
    return set_output_base(P, U, nx, ny, 0.0, scale, stream, "predictor_set_output_base");
}

extern "C" ddg_status predictor_set_output_base_wavelength(ddg_predictor* P, const double* U, int nx, int ny,
                                                           double wavelength, double scale, void* stream) {
    if (!(wavelength > 0.0)) { set_error("predictor_set_output_base_wavelength: wavelength must be > 0"); return DDG_EINVAL; }
    return set_output_base(P, U, nx, ny, wavelength, scale, stream, "predictor_set_output_base_wavelength");
}

extern "C" ddg_status predictor_destroy(ddg_predictor* P) {
    free_predictor(P);
    return DDG_OK;
}

extern "C" long long predictor_num_params(const ddg_predictor* P) { return P ? P->nparams : 0; }

extern "C" int predictor_num_outputs(const ddg_predictor* P) { return P ? P->k : 0; }

extern "C" long long predictor_launches(const ddg_predictor* P) { return P ? P->launches : 0; }

extern "C" ddg_status predictor_set_tensor_cores(ddg_predictor* P, int enable) {
    if (!P) { set_error("predictor_set_tensor_cores: NULL predictor"); return DDG_EINVAL; }
    if (enable < 0 || enable > 7) { set_error("predictor_set_tensor_cores: enable must be 0..7"); return DDG_EINVAL; }
    P->tensor_cores = enable;
    return DDG_OK;
}

extern "C" ddg_status predictor_set_params(ddg_predictor* P, const float* theta, long long n) {
    if (!P || !theta || n != P->nparams) { set_error("predictor_set_params: need %lld values", P ? P->nparams : 0LL); return DDG_EINVAL; }
    DDG_CHECK_CUDA(cudaMemcpy(P->theta, theta, 4 * (size_t)n, cudaMemcpyHostToDevice));
    ++P->launches;
    k_to_bf16<<<nblk(n), 256>>>(P->theta, P->theta_bf, n);
    DDG_CHECK_LAUNCH("k_to_bf16");
    DDG_CHECK_CUDA(cudaMemset(P->adam_m, 0, 4 * (size_t)n));
    DDG_CHECK_CUDA(cudaMemset(P->adam_v, 0, 4 * (size_t)n));
    P->step = 0;
    DDG_CHECK_CUDA(cudaDeviceSynchronize());
    return DDG_OK;
}

extern "C" ddg_status predictor_get_params(const ddg_predictor* P, float* theta, long long n) {
    if (!P || !theta || n != P->nparams) { set_error("predictor_get_params: need %lld values", P ? P->nparams : 0LL); return DDG_EINVAL; }
    DDG_CHECK_CUDA(cudaDeviceSynchronize());
    DDG_CHECK_CUDA(cudaMemcpy(theta, P->theta, 4 * (size_t)n, cudaMemcpyDeviceToHost));
    return DDG_OK;
}

extern "C" ddg_status predictor_forward(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma,
                                        double j_c, float* y, void* stream) {
    int H = 0, W = 0;
    DDG_TRY(check_batch(P, n, A, &H, &W));
    if (!y) { set_error("predictor_forward: y is NULL"); return DDG_EINVAL; }
    cudaStream_t st = as_stream(stream);
    Acts acts;
    DDG_TRY(ensure_acts(P, n, H, W, &acts, false));
    DDG_TRY(build_input(P, n, A, i_src, sigma, j_c, &acts, st));
    DDG_TRY(forward(P, n, H, W, &acts, st));
    DDG_CHECK_CUDA(cudaMemcpyAsync(y, acts.y, sizeof(float) * (size_t)n * H * W * 2 * P->k, cudaMemcpyDeviceToDevice, st));
    return check_tc(P, st);
}

extern "C" ddg_status subspace_predict(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma,
                                       double j_c, double* const* U, void* stream) {
    int H = 0, W = 0;
    DDG_TRY(check_batch(P, n, A, &H, &W));
    if (!U) { set_error("subspace_predict: U is NULL"); return DDG_EINVAL; }
    for (int s = 0; s < n; ++s)
        if (!U[s]) { set_error("subspace_predict: U[%d] is NULL", s); return DDG_EINVAL; }
    cudaStream_t st = as_stream(stream);
    Acts acts;
    DDG_TRY(ensure_acts(P, n, H, W, &acts, false));
    DDG_TRY(build_input(P, n, A, i_src, sigma, j_c, &acts, st));
    DDG_TRY(forward(P, n, H, W, &acts, st));
    void** slots = ptr_slots(P, n);
    DDG_CHECK_CUDA(cudaMemcpyAsync(slots, U, sizeof(void*) * n, cudaMemcpyHostToDevice, st));
    ++P->launches;
    k_to_complex<<<nblk((long long)n * H * W * P->k), 256, 0, st>>>(acts.y, H * W, P->k,
                                                                    reinterpret_cast<double2* const*>(slots), n);
    DDG_CHECK_LAUNCH("k_to_complex");
    // K13: Cholesky QR twice (FP64) of each problem's k vectors
    const int k = P->k, D = H * W, np = k * (k + 1) / 2;
    const int nch = (D + kOrthRows - 1) / kOrthRows;
    const size_t part_n = (size_t)n * nch * np, T_n = (size_t)n * k * k;
    const size_t need = sizeof(double2) * (part_n + T_n) + sizeof(int) * (size_t)n + 256;
    if (need > P->orth_bytes) {
        DDG_CHECK_CUDA(cudaStreamSynchronize(st));
        cudaFree(P->orth_ws);
        P->orth_ws = nullptr;
        P->orth_bytes = 0;
        cudaError_t e = cudaMalloc(&P->orth_ws, need);
        if (e != cudaSuccess) { cudaGetLastError(); set_error("subspace_predict: cudaMalloc failed"); return DDG_ENOMEM; }
        P->orth_bytes = need;
    }
    double2* part = P->orth_ws;
    double2* T = part + part_n;
    int* dropped = reinterpret_cast<int*>(T + T_n);
    double2* const* Us = reinterpret_cast<double2* const*>(slots);
    for (int pass = 0; pass < 2; ++pass) {
        P->launches += 3;
        k_orth_gram<<<dim3(nch, n), 256, 0, st>>>(Us, D, k, nch, part);
        k_orth_factor<<<n, 32, 0, st>>>(part, nch, k, T, dropped);
        k_orth_apply<<<dim3(nblk(D), n), 256, 0, st>>>(Us, D, k, T);
        DDG_CHECK_LAUNCH("orthonormalisation (K13)");
    }
    return check_tc(P, st);
}

extern "C" ddg_status predictor_loss_grad(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma,
                                          double j_c, const double* const* f, double* loss, float* grad, void* stream) {
    int H = 0, W = 0;
    DDG_TRY(check_batch(P, n, A, &H, &W));
    if (!f || n > 4096) { set_error("predictor_loss_grad: f is NULL or batch > 4096"); return DDG_EINVAL; }
    cudaStream_t st = as_stream(stream);
    Acts acts;
    DDG_TRY(ensure_acts(P, n, H, W, &acts, true));
    DDG_TRY(build_input(P, n, A, i_src, sigma, j_c, &acts, st));
    DDG_TRY(forward(P, n, H, W, &acts, st));
    void** slots = ptr_slots(P, n);
    DDG_CHECK_CUDA(cudaMemcpyAsync(slots, f, sizeof(void*) * n, cudaMemcpyHostToDevice, st));
    const int k = P->k;
    const int D = H * W;
    const double2* const* fsl = reinterpret_cast<const double2* const*>(slots);
    int nch = 0, tpb = 0;
    loss_blocks(D, &nch, &tpb);
    // Eq. 5 for V = y (projection loss) or V = A y (residual loss) and its gradient in gout
    auto proj_loss = [&](const float* yv, float* gout) {
        P->launches += 3;
        k_proj_part<<<dim3(nch, n), 256, loss_smem(k), st>>>(yv, fsl, D, k, tpb, acts.lpart);
        k_proj_solve<<<n, 256, sizeof(double2) * (size_t)(loss_entries(k) + k * k + k), st>>>(acts.lpart, k, nch,
                                                                                             P->d_loss, acts.lz);
        k_proj_grad<<<nblk((long long)n * D), 256, 0, st>>>(yv, fsl, D, k, n, acts.lz, gout);
    };
    if (P->loss_kind == 0) {
        // Eq. 5: V against the solved fields f
        proj_loss(acts.y, acts.gy);
    } else {
        // Eq. 6: W = A V against the right-hand sides b, then dl/dV = A^H dl/dW
        FieldOpDesc* fo = field_ops(P, n);
        const long long nk = (long long)n * D * k;
        ++P->launches;
        k_fields_apply<<<nblk((long long)n * D), 256, 0, st>>>(fo, acts.y, n, D, k, acts.y2);
        proj_loss(acts.y2, acts.gy2);
        ++P->launches;
        k_adj_pre<<<nblk(nk), 256, 0, st>>>(fo, acts.gy2, n, D, k, acts.y2);
        ++P->launches;
        k_fields_apply<<<nblk((long long)n * D), 256, 0, st>>>(fo, acts.y2, n, D, k, acts.gy);
        ++P->launches;
        k_adj_post<<<nblk(nk), 256, 0, st>>>(fo, acts.gy, n, D, k);
    }
    DDG_CHECK_LAUNCH("loss");

    DDG_CHECK_CUDA(cudaMemsetAsync(P->grad, 0, 4 * (size_t)P->nparams, st));
    DDG_TRY(backward(P, n, H, W, &acts, st));
    std::vector<double> hl(n);
    DDG_CHECK_CUDA(cudaMemcpyAsync(hl.data(), P->d_loss, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    if (grad) DDG_CHECK_CUDA(cudaMemcpyAsync(grad, P->grad, 4 * (size_t)P->nparams, cudaMemcpyDeviceToDevice, st));
    DDG_TRY(check_tc(P, st));
    double tot = 0.0;
    for (double v : hl) tot += v;
    if (loss) *loss = tot / n;
    P->last_finite = std::isfinite(tot);
    return DDG_OK;
}

extern "C" ddg_status predictor_adam_step(ddg_predictor* P, float lr, void* stream) {
    if (!P || !(lr > 0.f)) { set_error("predictor_adam_step: bad arguments"); return DDG_EINVAL; }
    if (!P->last_finite) return DDG_OK;   // a non-finite loss: leave weights and moments unchanged
    P->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)P->step), c2 = 1.f - powf(b2, (float)P->step);
    ++P->launches;
    k_adam<<<nblk(P->nparams), 256, 0, as_stream(stream)>>>(P->theta, P->grad, P->adam_m, P->adam_v, P->theta_bf,
                                                            P->nparams, lr, b1, b2, 1e-8f, c1, c2);
    DDG_CHECK_LAUNCH("k_adam");
    return DDG_OK;
}

extern "C" ddg_status predictor_train_step(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma,
                                           double j_c, const double* const* f, float lr, double* loss, void* stream) {
    DDG_TRY(predictor_loss_grad(P, n, A, i_src, sigma, j_c, f, loss, nullptr, stream));
    return predictor_adam_step(P, lr, stream);
}

// Checkpoint: header (magic, version, k, levels, channels, nparams, step),
// FP32 weights, Adam m and v, then an FNV-1a checksum of everything before it.
static unsigned long long fnv1a(const unsigned char* p, size_t n, unsigned long long h) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

extern "C" ddg_status predictor_save(const ddg_predictor* P, const char* path) {
    if (!P || !path) { set_error("predictor_save: bad arguments"); return DDG_EINVAL; }
    const size_t n = (size_t)P->nparams;
    std::vector<float> buf(3 * n);
    DDG_CHECK_CUDA(cudaDeviceSynchronize());
    DDG_CHECK_CUDA(cudaMemcpy(buf.data(), P->theta, 4 * n, cudaMemcpyDeviceToHost));
    DDG_CHECK_CUDA(cudaMemcpy(buf.data() + n, P->adam_m, 4 * n, cudaMemcpyDeviceToHost));
    DDG_CHECK_CUDA(cudaMemcpy(buf.data() + 2 * n, P->adam_v, 4 * n, cudaMemcpyDeviceToHost));
    long long hdr[4 + kMaxLevels] = {0x4444474d50524544LL, P->cin == 4 ? 1 : 2, P->k, P->levels};
    for (int l = 0; l < kMaxLevels; ++l) hdr[4 + l] = l < P->levels ? P->ch[l] : 0;
    long long tail[2] = {P->nparams, P->step};
    FILE* fp = fopen(path, "wb");
    if (!fp) { set_error("predictor_save: cannot open %s", path); return DDG_EINVAL; }
    unsigned long long h = 1469598103934665603ULL;
    h = fnv1a(reinterpret_cast<const unsigned char*>(hdr), sizeof(hdr), h);
    h = fnv1a(reinterpret_cast<const unsigned char*>(tail), sizeof(tail), h);
    h = fnv1a(reinterpret_cast<const unsigned char*>(buf.data()), 4 * buf.size(), h);
    bool ok = fwrite(hdr, sizeof(hdr), 1, fp) == 1 && fwrite(tail, sizeof(tail), 1, fp) == 1 &&
              fwrite(buf.data(), 4, buf.size(), fp) == buf.size() && fwrite(&h, sizeof(h), 1, fp) == 1;
    ok = (fclose(fp) == 0) && ok;
    if (!ok) { set_error("predictor_save: write to %s failed", path); return DDG_EINVAL; }
    return DDG_OK;
}

extern "C" ddg_status predictor_load(ddg_predictor* P, const char* path) {
    if (!P || !path) { set_error("predictor_load: bad arguments"); return DDG_EINVAL; }
    FILE* fp = fopen(path, "rb");
    if (!fp) { set_error("predictor_load: cannot open %s", path); return DDG_EINVAL; }
    long long hdr[4 + kMaxLevels], tail[2];
    const size_t n = (size_t)P->nparams;
    std::vector<float> buf(3 * n);
    unsigned long long hf = 0;
    bool ok = fread(hdr, sizeof(hdr), 1, fp) == 1 && fread(tail, sizeof(tail), 1, fp) == 1;
    ok = ok && hdr[0] == 0x4444474d50524544LL && hdr[1] == (P->cin == 4 ? 1 : 2) && hdr[2] == P->k && hdr[3] == P->levels &&
         tail[0] == P->nparams;
    for (int l = 0; ok && l < P->levels; ++l) ok = hdr[4 + l] == P->ch[l];
    ok = ok && fread(buf.data(), 4, buf.size(), fp) == buf.size() && fread(&hf, sizeof(hf), 1, fp) == 1;
    fclose(fp);
    if (!ok) { set_error("predictor_load: %s does not match this predictor", path); return DDG_EINVAL; }
    unsigned long long h = 1469598103934665603ULL;
    h = fnv1a(reinterpret_cast<const unsigned char*>(hdr), sizeof(hdr), h);
    h = fnv1a(reinterpret_cast<const unsigned char*>(tail), sizeof(tail), h);
    h = fnv1a(reinterpret_cast<const unsigned char*>(buf.data()), 4 * buf.size(), h);
    if (h != hf) { set_error("predictor_load: checksum mismatch in %s", path); return DDG_EINVAL; }
    DDG_CHECK_CUDA(cudaMemcpy(P->theta, buf.data(), 4 * n, cudaMemcpyHostToDevice));
    DDG_CHECK_CUDA(cudaMemcpy(P->adam_m, buf.data() + n, 4 * n, cudaMemcpyHostToDevice));
    DDG_CHECK_CUDA(cudaMemcpy(P->adam_v, buf.data() + 2 * n, 4 * n, cudaMemcpyHostToDevice));
    ++P->launches;
    k_to_bf16<<<nblk((long long)n), 256>>>(P->theta, P->theta_bf, (long long)n);
    DDG_CHECK_LAUNCH("k_to_bf16");
    P->step = tail[1];
    DDG_CHECK_CUDA(cudaDeviceSynchronize());
    return DDG_OK;
}

extern "C" ddg_status predictor_set_loss(ddg_predictor* P, int kind) {
    if (!P || (kind != 0 && kind != 1)) { set_error("predictor_set_loss: kind must be 0 (Eq. 5) or 1 (Eq. 6)"); return DDG_EINVAL; }
    P->loss_kind = kind;
    return DDG_OK;
}
