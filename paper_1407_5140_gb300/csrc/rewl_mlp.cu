// rewl_mlp.cu -- the learned warm start: a 5 -> 128 -> 128 -> 128 -> 1
// perceptron (tanh hidden units) that predicts the entropy density
// s(e) = ln g(E) / N from (model, L, q, E/N, window position).  Trained on the
// GPU with the mean squared error and Adam; the two 128 x 128 layers run on the
// tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation) in the
// forward and both backward products.  The warm start writes N * s(E) into
// every walker of an instance and starts Wang-Landau at a small ln f.
//
// Parameter vector (FP32 master copy): W1 [128x5], b1, W2 [128x128], b2,
// W3 [128x128], b3, W4 [1x128], b4; W[out][in].
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "rewl.h"
#include "rewl_device.cuh"
#include "rewl_internal.h"

namespace rewl {

enum : int {
    kH = 128,
    kIn = 5,
    kOffW1 = 0,
    kOffB1 = kOffW1 + kH * kIn,
    kOffW2 = kOffB1 + kH,
    kOffB2 = kOffW2 + kH * kH,
    kOffW3 = kOffB2 + kH,
    kOffB3 = kOffW3 + kH * kH,
    kOffW4 = kOffB3 + kH,
    kOffB4 = kOffW4 + kH,
    kNParams = kOffB4 + 1
};
static_assert(kNParams == 33921, "parameter count");

typedef __nv_bfloat16 bf16;

// Reductions over samples are split in at most kMaxParts pieces; their partial
// sums (at most kMaxParts x 128 x 128 floats) are added in a fixed order.
static constexpr int kMaxParts = 32;
static constexpr size_t kPartFloats = (size_t)kMaxParts * kH * kH;

// ---------------------------------------------------------------------------
// tensor-core GEMM: C[M x N] = A[M x K] * Bn[N x K]^T, A and Bn K-contiguous
// BF16, FP32 accumulation.  A block of 4 warps computes a 64 x 64 tile; warp
// w owns rows 16w..16w+15 and all 64 columns (8 mma n-tiles).  blockIdx.z
// splits K: the gradient epilogue stores each split's partial tile, and a
// second kernel adds the splits in a fixed order (no float atomics, so every
// gradient and training run is bitwise repeatable).
// Fragment layout of mma.m16n8k16.row.col (PTX ISA): lane = 4 g + c;
// A regs {(g, 2c..2c+1), (g+8, 2c..), (g, 2c+8..), (g+8, 2c+8..)};
// B regs {(k = 2c.., n = g), (k = 2c+8.., n = g)}; C {(g, 2c), (g, 2c+1),
// (g+8, 2c), (g+8, 2c+1)}.
// ---------------------------------------------------------------------------
enum Epi : int {
    kEpiForward = 0,   // z = acc + bias; h = tanh(z): H f32, Hb bf16 [M x N], HTb bf16 [N x M]
    kEpiBackward = 1,  // dz = acc * (1 - Hprev^2): dZ f32, dZb bf16, dZTb bf16
    kEpiGrad = 2       // G[split][m][n] = acc (partial sums, added by reduce_parts_kernel)
};

struct GemmArgs {
    const bf16 *A;
    const bf16 *Bn;
    int M, N, K, k_chunk;
    const float *bias;     // forward
    const float *Hprev;    // backward: activation of the layer whose pre-activation gradient is formed
    float *out_f;          // forward H / backward dZ / grad G
    bf16 *out_b;           // [M x N]
    bf16 *out_bt;          // [N x M]
};

__device__ __forceinline__ uint32_t ld_pair(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(GemmArgs g)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gr = lane >> 2, gc = lane & 3;
    const int m0 = blockIdx.x * 64 + warp * 16;
    const int n0 = blockIdx.y * 64;
    const int k_begin = blockIdx.z * g.k_chunk;
    const int k_end = min(g.K, k_begin + g.k_chunk);
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const bf16 *a_row0 = g.A + (size_t)(m0 + gr) * g.K;
    const bf16 *a_row1 = g.A + (size_t)(m0 + gr + 8) * g.K;
    for (int k = k_begin; k < k_end; k += 16) {
        uint32_t a[4];
        a[0] = ld_pair(a_row0 + k + 2 * gc);
        a[1] = ld_pair(a_row1 + k + 2 * gc);
        a[2] = ld_pair(a_row0 + k + 2 * gc + 8);
        a[3] = ld_pair(a_row1 + k + 2 * gc + 8);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bf16 *bp = g.Bn + (size_t)(n0 + 8 * j + gr) * g.K + k + 2 * gc;
            mma_bf16(acc[j], a, ld_pair(bp), ld_pair(bp + 8));
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int m = m0 + gr + (r >> 1) * 8;
            const int n = n0 + 8 * j + 2 * gc + (r & 1);
            const float v = acc[j][r];
            const size_t mn = (size_t)m * g.N + n, nm = (size_t)n * g.M + m;
            if (EPI == kEpiForward) {
                const float h = tanhf(v + g.bias[n]);
                g.out_f[mn] = h;
                g.out_b[mn] = __float2bfloat16_rn(h);
                g.out_bt[nm] = __float2bfloat16_rn(h);
            } else if (EPI == kEpiBackward) {
                const float hp = g.Hprev[mn];
                const float dz = v * (1.f - hp * hp);
                g.out_f[mn] = dz;
                g.out_b[mn] = __float2bfloat16_rn(dz);
                g.out_bt[nm] = __float2bfloat16_rn(dz);
            } else {
                g.out_f[(size_t)blockIdx.z * g.M * g.N + mn] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// small layers and reductions (FP32)
// ---------------------------------------------------------------------------
// h1 = tanh(W1 x + b1) for n samples; writes H1 f32, H1b, H1Tb
__global__ void layer1_kernel(const float *x, const float *p, int n, float *H, bf16 *Hb, bf16 *HTb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * kH) return;
    const int s = i / kH, u = i - s * kH;
    float z = p[kOffB1 + u];
#pragma unroll
    for (int k = 0; k < kIn; ++k) z = fmaf(p[kOffW1 + u * kIn + k], x[s * kIn + k], z);
    const float h = tanhf(z);
    H[i] = h;
    Hb[i] = __float2bfloat16_rn(h);
    HTb[(size_t)u * n + s] = __float2bfloat16_rn(h);
}

// y = W4 h3 + b4; with targets: dy = (y - t) / n and the sample's loss term
// lterm = (y - t)^2 / (2 n) (summed by sum_kernel)
__global__ void output_kernel(const float *H3, const float *p, int n, float *y, const float *t, float *dy,
                              float *lterm)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float z = p[kOffB4];
    for (int u = 0; u < kH; ++u) z = fmaf(p[kOffW4 + u], H3[(size_t)s * kH + u], z);
    if (y) y[s] = z;
    if (t) {
        const float d = z - t[s];
        dy[s] = d / (float)n;
        lterm[s] = 0.5f * d * d / (float)n;
    }
}

// dZ3 = dy W4 (1 - h3^2)
__global__ void back3_kernel(const float *dy, const float *H3, const float *p, int n, float *dZ, bf16 *dZb, bf16 *dZTb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * kH) return;
    const int s = i / kH, u = i - s * kH;
    const float h = H3[i];
    const float dz = dy[s] * p[kOffW4 + u] * (1.f - h * h);
    dZ[i] = dz;
    dZb[i] = __float2bfloat16_rn(dz);
    dZTb[(size_t)u * n + s] = __float2bfloat16_rn(dz);
}

// part[block][u] = sum over the block's rows s of w[s] X[s][u] (w = NULL:
// weights 1); one block of 128 threads per chunk of rows
__global__ void colsum_kernel(const float *X, const float *w, int n, int rows_per_block, float *part)
{
    const int u = threadIdx.x;
    const int s0 = blockIdx.x * rows_per_block, s1 = min(n, s0 + rows_per_block);
    float acc = 0.f;
    for (int s = s0; s < s1; ++s) acc += (w ? w[s] : 1.f) * X[(size_t)s * kH + u];
    part[(size_t)blockIdx.x * kH + u] = acc;
}

// part[block][u][k] = sum over the block's rows s of dZ1[s][u] x[s][k]
__global__ void dw1_kernel(const float *dZ1, const float *x, int n, int rows_per_block, float *part)
{
    const int u = threadIdx.x;
    const int s0 = blockIdx.x * rows_per_block, s1 = min(n, s0 + rows_per_block);
    float acc[kIn] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int s = s0; s < s1; ++s) {
        const float d = dZ1[(size_t)s * kH + u];
#pragma unroll
        for (int k = 0; k < kIn; ++k) acc[k] = fmaf(d, x[s * kIn + k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < kIn; ++k) part[(size_t)blockIdx.x * kH * kIn + u * kIn + k] = acc[k];
}

// out[i] = sum over p = 0, 1, ... of part[p][i], in that order
__global__ void reduce_parts_kernel(const float *part, int n_parts, int len, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float acc = 0.f;
    for (int p = 0; p < n_parts; ++p) acc += part[(size_t)p * len + i];
    out[i] = acc;
}

// BF16 copies of W2, W3 and of their transposes
__global__ void cast_weights_kernel(const float *p, bf16 *W2b, bf16 *W3b, bf16 *W2Tb, bf16 *W3Tb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kH * kH) return;
    const int r = i / kH, c = i - r * kH;
    W2b[i] = __float2bfloat16_rn(p[kOffW2 + i]);
    W3b[i] = __float2bfloat16_rn(p[kOffW3 + i]);
    W2Tb[c * kH + r] = __float2bfloat16_rn(p[kOffW2 + i]);
    W3Tb[c * kH + r] = __float2bfloat16_rn(p[kOffW3 + i]);
}

// Adam (Kingma & Ba): bias-corrected first and second moments
__global__ void adam_kernel(float *p, float *m, float *v, const float *g, int n, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from Philox (stream 3 of the seed)
__global__ void init_params_kernel(float *p, uint32_t k0, uint32_t k1)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParams) return;
    const u32x4 r = philox10((uint32_t)i, 0u, 0u, 3u, k0, k1);
    const float fan = i < kOffW2 ? (float)kIn : (i < kOffW4 ? (float)kH : (float)kH);
    const float a = rsqrtf(fan);
    p[i] = a * (2.f * ((float)(r.x >> 8) * (1.f / 16777216.f)) - 1.f);
}

// *out = sum of v[0..n) (db4, the loss): one block of 256 threads, each
// thread's strided sum, then a fixed reduction tree
__global__ void sum_kernel(const float *v, int n, float *out)
{
    __shared__ float red[256];
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// ---------------------------------------------------------------------------
// warm start: features of every (window, bin) of an instance, and the
// installation of the predicted ln g into the walkers
// ---------------------------------------------------------------------------
// x = [model, 16/L, log10 q, E/N, i/(h-1)]
__global__ void features_kernel(DevState st, int inst, int first_sample, int n, float *x)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const InstDev I = st.inst[inst];
    const int sample = first_sample + k;           // sample = window * w + local bin
    const int i = sample / I.w, b = sample - i * I.w;
    const int gb = st.lo[I.win0 + i] + b;
    const double E = (double)I.e_min + (double)gb * I.step;
    float *xs = x + (size_t)k * kIn;
    xs[0] = (float)I.model;
    xs[1] = 16.f / (float)I.L;
    xs[2] = log10f((float)I.q);
    xs[3] = (float)(E / (double)I.N);
    xs[4] = I.h > 1 ? (float)i / (float)(I.h - 1) : 0.f;
}

// ln g0 of every walker of window i: N s(E) over the realisable bins, shifted
// so that the window's smallest value is 0, rounded to the 2^-32 grid;
// the stage starts from it (lng0 = ln g, H = 0), latch reset; stage k0 (or
// frozen if k0 < 0)
__global__ void install_kernel(DevState st, int inst, const float *s_pred, int k0)
{
    const InstDev I = st.inst[inst];
    const int i = blockIdx.x;                       // window
    const int w = I.w, gwin = I.win0 + i, lo = st.lo[gwin], wi = st.ww[gwin];   // row length, window width
    __shared__ float red[256];
    float mn = 3.4e38f;
    for (int b = threadIdx.x; b < wi; b += blockDim.x)
        if (st.reach[I.reach_off + lo + b]) mn = fminf(mn, (float)I.N * s_pred[(size_t)i * w + b]);
    red[threadIdx.x] = mn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fminf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    mn = red[0];
    for (int b = threadIdx.x; b < w; b += blockDim.x) {
        const double v = (b < wi && st.reach[I.reach_off + lo + b]) ? (double)((float)I.N * s_pred[(size_t)i * w + b] - mn)
                                                                    : 0.0;
        const long long units = llrint(v * 4294967296.0);
        for (int j = 0; j < I.m; ++j) {
            const long long off = I.lng_off + (long long)(i * I.m + j) * w + b;
            st.lng[off] = units;
            st.lng0[off] = units;
            st.H[off] = 0u;
        }
    }
    if (threadIdx.x == 0) {
        for (int j = 0; j < I.m; ++j) st.latch[I.slot0 + i * I.m + j] = 0;
        st.stage[gwin] = k0 < 0 ? 0 : k0;
        st.conv[gwin] = k0 < 0 ? 2 : 0;          // 2: sampling with frozen weights
    }
}

}  // namespace rewl

using namespace rewl;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct rewl_mlp {
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    bf16 *W2b = nullptr, *W3b = nullptr, *W2Tb = nullptr, *W3Tb = nullptr;
    // activations and gradients of one batch (scratch)
    float *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *dZ = nullptr, *dZ1 = nullptr, *y = nullptr, *dy = nullptr,
          *loss = nullptr, *xbuf = nullptr, *sbuf = nullptr;
    float *lterm = nullptr;   // per-sample loss terms
    float *part = nullptr;    // partial sums of the gradient reductions (kPartFloats)
    bf16 *H1b = nullptr, *H2b = nullptr, *H1Tb = nullptr, *H2Tb = nullptr, *dZb = nullptr, *dZTb = nullptr;
    long step = 0;
    long launches = 0;
    std::string err;
};

static thread_local std::string g_mlp_error;

static rewl_status mfail(rewl_mlp *n, rewl_status s, const std::string &msg)
{
    if (n) n->err = msg;
    else g_mlp_error = msg;
    return s;
}

#define MCK(call)                                                                                       \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return mfail(net, REWL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
static cudaError_t malloc_n(T **p, size_t n)
{
    return cudaMalloc((void **)p, n * sizeof(T));
}

extern "C" void rewl_mlp_destroy(rewl_mlp *net)
{
    if (!net) return;
    if (net->stream) cudaStreamSynchronize(net->stream);
    void *bufs[] = {net->p, net->m, net->v, net->g, net->W2b, net->W3b, net->W2Tb, net->W3Tb, net->H1, net->H2, net->H3,
                    net->dZ, net->dZ1, net->y, net->dy, net->loss, net->xbuf, net->sbuf, net->H1b, net->H2b,
                    net->H1Tb, net->H2Tb, net->dZb, net->dZTb, net->lterm, net->part};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (net->own_stream && net->stream) cudaStreamDestroy(net->stream);
    delete net;
}

extern "C" rewl_status rewl_mlp_create(rewl_mlp **out, int max_batch, unsigned long long seed, void *cuda_stream)
{
    if (!out || max_batch < 64 || max_batch % 64 || max_batch > (1 << 22))
        return mfail(nullptr, REWL_EINVAL, "rewl_mlp_create: max_batch must be a multiple of 64 in [64, 2^22]");
    rewl_mlp *net = new rewl_mlp();
    *out = net;
    net->max_batch = max_batch;
    if (cuda_stream) net->stream = (cudaStream_t)cuda_stream;
    else {
        MCK(cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking));
        net->own_stream = true;
    }
    const size_t B = (size_t)max_batch, HB = B * kH;
    MCK(malloc_n(&net->p, kNParams));
    MCK(malloc_n(&net->m, kNParams));
    MCK(malloc_n(&net->v, kNParams));
    MCK(malloc_n(&net->g, kNParams));
    MCK(malloc_n(&net->W2b, kH * kH));
    MCK(malloc_n(&net->W3b, kH * kH));
    MCK(malloc_n(&net->W2Tb, kH * kH));
    MCK(malloc_n(&net->W3Tb, kH * kH));
    MCK(malloc_n(&net->H1, HB));
    MCK(malloc_n(&net->H2, HB));
    MCK(malloc_n(&net->H3, HB));
    MCK(malloc_n(&net->dZ, HB));
    MCK(malloc_n(&net->dZ1, HB));
    MCK(malloc_n(&net->y, B));
    MCK(malloc_n(&net->dy, B));
    MCK(malloc_n(&net->loss, 1));
    MCK(malloc_n(&net->xbuf, B * kIn));
    MCK(malloc_n(&net->sbuf, B));
    MCK(malloc_n(&net->lterm, B));
    MCK(malloc_n(&net->part, (size_t)kPartFloats));
    MCK(malloc_n(&net->H1b, HB));
    MCK(malloc_n(&net->H2b, HB));
    MCK(malloc_n(&net->H1Tb, HB));
    MCK(malloc_n(&net->H2Tb, HB));
    MCK(malloc_n(&net->dZb, HB));
    MCK(malloc_n(&net->dZTb, HB));
    MCK(cudaMemsetAsync(net->m, 0, kNParams * 4, net->stream));
    MCK(cudaMemsetAsync(net->v, 0, kNParams * 4, net->stream));
    init_params_kernel<<<(kNParams + 255) / 256, 256, 0, net->stream>>>(net->p, (uint32_t)seed,
                                                                        (uint32_t)(seed >> 32));
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(net->stream));
    return REWL_OK;
}

extern "C" rewl_status rewl_mlp_set_params(rewl_mlp *net, const float *host, long n)
{
    if (!net || !host || n != kNParams) return mfail(net, REWL_EINVAL, "rewl_mlp_set_params: need 33921 values");
    MCK(cudaMemcpyAsync(net->p, host, kNParams * 4, cudaMemcpyHostToDevice, net->stream));
    MCK(cudaMemsetAsync(net->m, 0, kNParams * 4, net->stream));
    MCK(cudaMemsetAsync(net->v, 0, kNParams * 4, net->stream));
    net->step = 0;
    MCK(cudaStreamSynchronize(net->stream));
    return REWL_OK;
}

extern "C" rewl_status rewl_mlp_get_params(rewl_mlp *net, float *host, long n)
{
    if (!net || !host || n != kNParams) return mfail(net, REWL_EINVAL, "rewl_mlp_get_params: need 33921 values");
    MCK(cudaStreamSynchronize(net->stream));
    MCK(cudaMemcpy(host, net->p, kNParams * 4, cudaMemcpyDeviceToHost));
    return REWL_OK;
}

static rewl_status run_gemm(rewl_mlp *net, int epi, const GemmArgs &a, int splits)
{
    dim3 grid(a.M / 64, a.N / 64, splits);
    if (epi == kEpiForward) gemm_kernel<kEpiForward><<<grid, 128, 0, net->stream>>>(a);
    else if (epi == kEpiBackward) gemm_kernel<kEpiBackward><<<grid, 128, 0, net->stream>>>(a);
    else gemm_kernel<kEpiGrad><<<grid, 128, 0, net->stream>>>(a);
    net->launches += 1;
    MCK(cudaGetLastError());
    return REWL_OK;
}

// forward pass of n samples (x device, n % 64 == 0): fills H1..H3 (+ bf16
// copies); y and, with targets, the loss and dy
static rewl_status forward(rewl_mlp *net, const float *x, int n, float *y, const float *t)
{
    rewl_status s;
    cast_weights_kernel<<<(kH * kH + 255) / 256, 256, 0, net->stream>>>(net->p, net->W2b, net->W3b, net->W2Tb,
                                                                        net->W3Tb);
    layer1_kernel<<<(n * kH + 255) / 256, 256, 0, net->stream>>>(x, net->p, n, net->H1, net->H1b, net->H1Tb);
    net->launches += 2;
    GemmArgs a{};
    a.A = net->H1b;
    a.Bn = net->W2b;
    a.M = n;
    a.N = kH;
    a.K = kH;
    a.k_chunk = kH;
    a.bias = net->p + kOffB2;
    a.out_f = net->H2;
    a.out_b = net->H2b;
    a.out_bt = net->H2Tb;
    if ((s = run_gemm(net, kEpiForward, a, 1))) return s;
    // H3: only f32 is needed downstream (output layer, back3); the bf16
    // buffers are reused as scratch here
    a.A = net->H2b;
    a.Bn = net->W3b;
    a.bias = net->p + kOffB3;
    a.out_f = net->H3;
    a.out_b = net->dZb;
    a.out_bt = net->dZTb;
    if ((s = run_gemm(net, kEpiForward, a, 1))) return s;
    output_kernel<<<(n + 127) / 128, 128, 0, net->stream>>>(net->H3, net->p, n, y, t, net->dy, net->lterm);
    net->launches += 1;
    if (t) {
        sum_kernel<<<1, 256, 0, net->stream>>>(net->lterm, n, net->loss);
        net->launches += 1;
    }
    MCK(cudaGetLastError());
    return REWL_OK;
}


// Gradient of the loss into net->g, after forward() with targets.  Buffer
// use: dZ3 in dZ/dZb/dZTb; dZ2 in dZ (f32) and in the H2 bf16 buffers (H2b,
// H2Tb are dead once dW3 is formed); dZ1 in dZ1.  Every sum over samples is
// formed as at most kMaxParts partial sums in net->part, then added in order.
static rewl_status backward(rewl_mlp *net, const float *x, int n)
{
    rewl_status s;
    const int rpb = (n + kMaxParts - 1) / kMaxParts;   // rows per colsum / dw1 block
    const int nb = (n + rpb - 1) / rpb;                 // <= kMaxParts
    const int splits = std::max(1, std::min(kMaxParts, n / 512));
    const int kc = ((n / splits + 15) / 16) * 16;
    const int ksplits = (n + kc - 1) / kc;              // <= splits
    auto reduce = [&](int parts, int len, float *out) {
        reduce_parts_kernel<<<(len + 255) / 256, 256, 0, net->stream>>>(net->part, parts, len, out);
        net->launches += 1;
    };
    // layer 4: dW4 = sum_s dy h3, db4 = sum_s dy
    colsum_kernel<<<nb, kH, 0, net->stream>>>(net->H3, net->dy, n, rpb, net->part);
    reduce(nb, kH, net->g + kOffW4);
    sum_kernel<<<1, 256, 0, net->stream>>>(net->dy, n, net->g + kOffB4);
    // dZ3 = dy W4 (1 - h3^2)
    back3_kernel<<<(n * kH + 255) / 256, 256, 0, net->stream>>>(net->dy, net->H3, net->p, n, net->dZ, net->dZb,
                                                               net->dZTb);
    net->launches += 3;
    // layer 3: dW3 = dZ3^T H2, db3 = sum dZ3
    GemmArgs a{};
    a.A = net->dZTb;
    a.Bn = net->H2Tb;
    a.M = kH;
    a.N = kH;
    a.K = n;
    a.k_chunk = kc;
    a.out_f = net->part;
    if ((s = run_gemm(net, kEpiGrad, a, ksplits))) return s;
    reduce(ksplits, kH * kH, net->g + kOffW3);
    colsum_kernel<<<nb, kH, 0, net->stream>>>(net->dZ, nullptr, n, rpb, net->part);
    reduce(nb, kH, net->g + kOffB3);
    net->launches += 1;
    // dZ2 = (dZ3 W3) (1 - h2^2)
    GemmArgs b{};
    b.A = net->dZb;
    b.Bn = net->W3Tb;
    b.M = n;
    b.N = kH;
    b.K = kH;
    b.k_chunk = kH;
    b.Hprev = net->H2;
    b.out_f = net->dZ;
    b.out_b = net->H2b;
    b.out_bt = net->H2Tb;
    if ((s = run_gemm(net, kEpiBackward, b, 1))) return s;
    // layer 2: dW2 = dZ2^T H1, db2 = sum dZ2
    a.A = net->H2Tb;
    a.Bn = net->H1Tb;
    if ((s = run_gemm(net, kEpiGrad, a, ksplits))) return s;
    reduce(ksplits, kH * kH, net->g + kOffW2);
    colsum_kernel<<<nb, kH, 0, net->stream>>>(net->dZ, nullptr, n, rpb, net->part);
    reduce(nb, kH, net->g + kOffB2);
    net->launches += 1;
    // dZ1 = (dZ2 W2) (1 - h1^2)
    b.A = net->H2b;
    b.Bn = net->W2Tb;
    b.Hprev = net->H1;
    b.out_f = net->dZ1;
    b.out_b = net->dZb;
    b.out_bt = net->dZTb;
    if ((s = run_gemm(net, kEpiBackward, b, 1))) return s;
    // layer 1: dW1 = dZ1^T x, db1 = sum dZ1
    dw1_kernel<<<nb, kH, 0, net->stream>>>(net->dZ1, x, n, rpb, net->part);
    reduce(nb, kH * kIn, net->g + kOffW1);
    colsum_kernel<<<nb, kH, 0, net->stream>>>(net->dZ1, nullptr, n, rpb, net->part);
    reduce(nb, kH, net->g + kOffB1);
    net->launches += 2;
    MCK(cudaGetLastError());
    return REWL_OK;
}

static rewl_status check_batch(rewl_mlp *net, int n)
{
    if (n < 64 || n % 64 || n > net->max_batch)
        return mfail(net, REWL_EINVAL, "batch size must be a multiple of 64 and at most max_batch");
    return REWL_OK;
}

extern "C" rewl_status rewl_mlp_forward(rewl_mlp *net, const float *x_dev, float *y_dev, int n)
{
    if (!net || !x_dev || !y_dev) return mfail(net, REWL_EINVAL, "rewl_mlp_forward: null argument");
    rewl_status s = check_batch(net, n);
    if (s) return s;
    return forward(net, x_dev, n, y_dev, nullptr);
}

extern "C" rewl_status rewl_mlp_gradient(rewl_mlp *net, const float *x_dev, const float *t_dev, int n,
                                         float *grad_host, float *loss_host)
{
    if (!net || !x_dev || !t_dev) return mfail(net, REWL_EINVAL, "rewl_mlp_gradient: null argument");
    rewl_status s = check_batch(net, n);
    if (s) return s;
    if ((s = forward(net, x_dev, n, nullptr, t_dev))) return s;
    if ((s = backward(net, x_dev, n))) return s;
    MCK(cudaStreamSynchronize(net->stream));
    if (grad_host) MCK(cudaMemcpy(grad_host, net->g, kNParams * 4, cudaMemcpyDeviceToHost));
    if (loss_host) MCK(cudaMemcpy(loss_host, net->loss, 4, cudaMemcpyDeviceToHost));
    return REWL_OK;
}

extern "C" rewl_status rewl_mlp_train_step(rewl_mlp *net, const float *x_dev, const float *t_dev, int n, float lr,
                                           float *loss_host)
{
    if (!net || !x_dev || !t_dev || !(lr > 0.f)) return mfail(net, REWL_EINVAL, "rewl_mlp_train_step: bad argument");
    rewl_status s = check_batch(net, n);
    if (s) return s;
    if ((s = forward(net, x_dev, n, nullptr, t_dev))) return s;
    if ((s = backward(net, x_dev, n))) return s;
    net->step += 1;
    // bias corrections 1 - beta^t in double: in FP32, 1 - 0.999^t loses most
    // of its digits to cancellation for small t
    const float c1 = (float)(1.0 - std::pow(0.9, (double)net->step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)net->step));
    adam_kernel<<<(kNParams + 255) / 256, 256, 0, net->stream>>>(net->p, net->m, net->v, net->g, kNParams, lr, c1, c2);
    net->launches += 1;
    MCK(cudaGetLastError());
    if (loss_host) {
        MCK(cudaStreamSynchronize(net->stream));
        MCK(cudaMemcpy(loss_host, net->loss, 4, cudaMemcpyDeviceToHost));
    }
    return REWL_OK;
}

extern "C" long rewl_mlp_launch_count(const rewl_mlp *net) { return net ? net->launches : 0; }

extern "C" const char *rewl_mlp_last_error(const rewl_mlp *net) { return net ? net->err.c_str() : g_mlp_error.c_str(); }

// ---------------------------------------------------------------------------
// warm start of one instance (called by rewl_warm_start in rewl_api.cu)
// ---------------------------------------------------------------------------
namespace rewl {

int mlp_warm_start(rewl_mlp *net, const DevState &st, int inst, int h, int w, int k0, std::string &why)
{
    const long total = (long)h * w;
    float *s_all = nullptr;
    cudaError_t e = cudaMalloc((void **)&s_all, (size_t)total * sizeof(float));
    if (e != cudaSuccess) {
        why = cudaGetErrorString(e);
        return (int)REWL_ENOMEM;
    }
    int rc = 0;
    for (long first = 0; first < total && !rc; first += net->max_batch) {
        const int n = (int)std::min<long>(net->max_batch, total - first);
        const int n_pad = (n + 63) / 64 * 64;
        features_kernel<<<(n_pad + 255) / 256, 256, 0, net->stream>>>(st, inst, (int)first, n, net->xbuf);
        // pad rows: repeat the first sample (their outputs are ignored)
        if (n_pad > n) {
            for (int r = n; r < n_pad; ++r) {
                e = cudaMemcpyAsync(net->xbuf + (size_t)r * kIn, net->xbuf, kIn * sizeof(float),
                                    cudaMemcpyDeviceToDevice, net->stream);
                if (e != cudaSuccess) break;
            }
        }
        if (e == cudaSuccess && forward(net, net->xbuf, n_pad, net->sbuf, nullptr) != REWL_OK) {
            why = net->err;
            rc = (int)REWL_ECUDA;
        }
        if (e == cudaSuccess && !rc)
            e = cudaMemcpyAsync(s_all + first, net->sbuf, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice,
                                net->stream);
        net->launches += 1;
    }
    if (!rc && e == cudaSuccess) {
        install_kernel<<<h, 256, 0, net->stream>>>(st, inst, s_all, k0);
        net->launches += 1;
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(net->stream);
    cudaFree(s_all);
    if (!rc && (e != cudaSuccess || e2 != cudaSuccess)) {
        why = cudaGetErrorString(e != cudaSuccess ? e : e2);
        rc = (int)REWL_ECUDA;
    }
    return rc;
}

}  // namespace rewl

// ---------------------------------------------------------------------------
// Forward pass without any allocation (rewl_mlp_forward_noalloc).
//
// Some callers cannot allocate device memory once they are running: their
// device memory belongs to another allocator (a framework's caching pool or a
// fixed budget fixed at start-up), or they call from a loop where cudaMalloc's
// implicit synchronisation of the whole device is not acceptable.  For them
// the activations of one forward pass live in this file-scope device array,
// loaded with the library and held by every GPU that loads it until the
// process exits.  All calls share it: two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it.  No entry of it
// needs to start at zero -- the pass writes every value before reading it --
// and it keeps whatever the last call left there.
// ---------------------------------------------------------------------------
namespace rewl {

static constexpr int kNoAllocMaxBatch = 1024;
// layout: H1, H2, H3 (FP32, n x 128 each), then BF16 H1b, H1Tb, H2b, H2Tb,
// H3b, H3Tb (n x 128 each), then BF16 W2b, W3b, W2Tb, W3Tb (128 x 128 each)
static constexpr size_t kNoAllocF32 = 3ull * kNoAllocMaxBatch * kH;
static constexpr size_t kNoAllocBf16 = 6ull * kNoAllocMaxBatch * kH + 4ull * kH * kH;
static constexpr size_t kNoAllocBytes = kNoAllocF32 * 4 + kNoAllocBf16 * 2;   // 3,276,800 bytes

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

}  // namespace rewl

extern "C" rewl_status rewl_mlp_forward_noalloc(const float *params, const float *x, float *y, int n,
                                                void *cuda_stream)
{
    // device address of the scratch array, looked up once per device with that
    // device current (the host-side name is only a stand-in for it)
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    if (!params || !x || !y) return mfail(nullptr, REWL_EINVAL, "rewl_mlp_forward_noalloc: null pointer");
    if (n < 64 || n % 64 || n > kNoAllocMaxBatch)
        return mfail(nullptr, REWL_EINVAL,
                     "rewl_mlp_forward_noalloc: n must be a multiple of 64 in [64, 1024] (static scratch limit)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mfail(nullptr, REWL_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return mfail(nullptr, REWL_EINVAL, "rewl_mlp_forward_noalloc: device index above 63");
    void *base;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!addr[dev]) {
            e = cudaGetSymbolAddress(&addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                addr[dev] = nullptr;
                return mfail(nullptr, REWL_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        base = addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t NB = (size_t)n * kH;
    float *H1 = reinterpret_cast<float *>(base);
    float *H2 = H1 + (size_t)kNoAllocMaxBatch * kH;
    float *H3 = H2 + (size_t)kNoAllocMaxBatch * kH;
    bf16 *b0 = reinterpret_cast<bf16 *>(reinterpret_cast<unsigned char *>(base) + kNoAllocF32 * 4);
    bf16 *H1b = b0, *H1Tb = b0 + NB, *H2b = b0 + 2 * NB, *H2Tb = b0 + 3 * NB, *H3b = b0 + 4 * NB,
         *H3Tb = b0 + 5 * NB;
    bf16 *W2b = b0 + 6ull * kNoAllocMaxBatch * kH, *W3b = W2b + kH * kH, *W2Tb = W3b + kH * kH,
         *W3Tb = W2Tb + kH * kH;
    cast_weights_kernel<<<(kH * kH + 255) / 256, 256, 0, s>>>(params, W2b, W3b, W2Tb, W3Tb);
    layer1_kernel<<<(n * kH + 255) / 256, 256, 0, s>>>(x, params, n, H1, H1b, H1Tb);
    GemmArgs a{};
    a.A = H1b;
    a.Bn = W2b;
    a.M = n;
    a.N = kH;
    a.K = kH;
    a.k_chunk = kH;
    a.bias = params + kOffB2;
    a.out_f = H2;
    a.out_b = H2b;
    a.out_bt = H2Tb;
    gemm_kernel<kEpiForward><<<dim3(n / 64, kH / 64, 1), 128, 0, s>>>(a);
    a.A = H2b;
    a.Bn = W3b;
    a.bias = params + kOffB3;
    a.out_f = H3;
    a.out_b = H3b;
    a.out_bt = H3Tb;
    gemm_kernel<kEpiForward><<<dim3(n / 64, kH / 64, 1), 128, 0, s>>>(a);
    output_kernel<<<(n + 127) / 128, 128, 0, s>>>(H3, params, n, y, nullptr, nullptr, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return mfail(nullptr, REWL_ECUDA, std::string("rewl_mlp_forward_noalloc: ") + cudaGetErrorString(e));
    return REWL_OK;
}
