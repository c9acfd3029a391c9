// sf_net.cu -- the learned warm start: a six-layer convolutional network that
// maps the four coarsest-level images of a quadruple (60 x 80) to the
// coarsest level's six delta fields (8 x 10 warp-grid nodes), trained on the
// GPU. The paper starts the first frame from zero flows and names a smarter
// first-frame initialisation as future work (Section 7); the prediction
// replaces that zero start at the coarsest level, the place where the
// temporal transfer of Section 5.3 enters for later frames.
//
// Layers (3x3 kernels, zero padding 1, ReLU after all but the last):
//   4 -> 32 stride 2, 32 -> 64 stride 2, 64 -> 64 stride 2, 64 -> 64,
//   64 -> 32, 32 -> 6; input I - 1/2; output [B][6][8][10].
//
// Every convolution runs as a tensor-core GEMM (sf_gemm.cu) on BF16 operands
// with FP32 accumulation:
//   forward      Z = im2col(X) W^T + b, ReLU, stored BF16 (NHWC)
//   weight grad  dW = dZ^T im2col(X)        (split-K, fixed-order reduction)
//   input grad   dX = col2im(dZ W)          (a gather, no atomics)
// im2col orders K as (ky, kx, c), padded with zeros to a multiple of 64.
// Biases, master weights, gradients and Adam moments stay FP32; every
// reduction runs in a fixed order, so training is bit-reproducible.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "sf_launch.h"

namespace sfk {

namespace {

constexpr int NT = 256;

__global__ void k_im2col_img(const float* __restrict__ img, long long img_stride, long long ch_stride, int B, int H,
                             int W, int Ho, int Wo, int stride, __nv_bfloat16* __restrict__ A, int Kp)
{
    // layer 1: four FP32 channels, normalised by -1/2; one thread per (m, k)
    const long long total = (long long)B * Ho * Wo * Kp;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t % Kp);
        const long long m = t / Kp;
        float v = 0.f;
        if (k < 36) {
            const int tap = k >> 2, c = k & 3;
            const int ky = tap / 3, kx = tap - ky * 3;
            const int ox = (int)(m % Wo);
            const long long r = m / Wo;
            const int oy = (int)(r % Ho), b = (int)(r / Ho);
            const int iy = oy * stride + ky - 1, ix = ox * stride + kx - 1;
            if (iy >= 0 && iy < H && ix >= 0 && ix < W)
                v = img[b * img_stride + c * ch_stride + (long long)iy * W + ix] - 0.5f;
        }
        A[t] = __float2bfloat16_rn(v);
    }
}

__global__ void k_im2col(const __nv_bfloat16* __restrict__ act, int B, int H, int W, int C, int Ho, int Wo, int stride,
                         __nv_bfloat16* __restrict__ A, int Kp)
{
    // C % 8 == 0: one thread per 8 consecutive K entries (one tap, 8 channels)
    const int kv = Kp / 8;
    const long long total = (long long)B * Ho * Wo * kv;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int v8 = (int)(t % kv);
        const long long m = t / kv;
        const int k = v8 * 8;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (k < 9 * C) {
            const int tap = k / C, c = k - tap * C;
            const int ky = tap / 3, kx = tap - ky * 3;
            const int ox = (int)(m % Wo);
            const long long r = m / Wo;
            const int oy = (int)(r % Ho), b = (int)(r / Ho);
            const int iy = oy * stride + ky - 1, ix = ox * stride + kx - 1;
            if (iy >= 0 && iy < H && ix >= 0 && ix < W)
                val = *reinterpret_cast<const uint4*>(act + (((long long)b * H + iy) * W + ix) * C + c);
        }
        *reinterpret_cast<uint4*>(A + m * Kp + k) = val;
    }
}

// dZ of the last layer from the squared error, and the loss partials.
__global__ void k_loss_grad(const float* __restrict__ out, const float* __restrict__ target, int B, int C, int HW,
                            float scale, float* __restrict__ dZ, float* __restrict__ part)
{
    __shared__ float sh[NT / 32];
    const int n = B * C * HW;
    float acc = 0.f;
    for (int t = blockIdx.x * NT + threadIdx.x; t < n; t += gridDim.x * NT) {
        const int px = t % HW, r = t / HW, c = r % C, b = r / C;
        const float d = out[t] - target[t];
        acc = fmaf(d, d, acc);
        dZ[((size_t)b * HW + px) * C + c] = scale * d; // NHWC, like the activations
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < NT / 32; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_sum_parts(const float* __restrict__ part, int n, float scale, float* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = (float)(s * scale);
    }
}

// Column sums of dZ [M][C] (the bias gradient), one block per column.
__global__ void k_colsum(const float* __restrict__ dZ, int M, int C, float* __restrict__ db)
{
    __shared__ float sh[NT];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (int m = threadIdx.x; m < M; m += NT) acc += dZ[(size_t)m * C + c];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = sh[0];
}

// dZ [M][C] FP32 -> BF16 row-major [M][Cp] (zero columns past C) and
// transposed [C][Mp] (zero past M), through a 32 x 32 shared tile.
__global__ void k_pack_dz(const float* __restrict__ dZ, int M, int C, int Cp, int Mp, __nv_bfloat16* __restrict__ rowm,
                          __nv_bfloat16* __restrict__ colm)
{
    __shared__ float tile[32][33];
    const int m0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int m = m0 + r, c = c0 + threadIdx.x;
        const float v = (m < M && c < C) ? dZ[(size_t)m * C + c] : 0.f;
        tile[r][threadIdx.x] = v;
        if (m < M && c < Cp) rowm[(size_t)m * Cp + c] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int c = c0 + r, m = m0 + threadIdx.x;
        if (c < C && m < Mp) colm[(size_t)c * Mp + m] = __float2bfloat16_rn(tile[threadIdx.x][r]);
    }
}

// A [M][K] BF16 -> AT [K][Mp] (zero past M).
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ A, int M, int K, int Mp,
                                 __nv_bfloat16* __restrict__ AT)
{
    __shared__ __nv_bfloat16 tile[32][34];
    const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int m = m0 + r, k = k0 + threadIdx.x;
        tile[r][threadIdx.x] = (m < M && k < K) ? A[(size_t)m * K + k] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int k = k0 + r, m = m0 + threadIdx.x;
        if (k < K && m < Mp) AT[(size_t)k * Mp + m] = tile[threadIdx.x][r];
    }
}

// Sum of split-K partials [S][n] in split order.
__global__ void k_split_reduce(const float* __restrict__ part, int S, int n, float* __restrict__ out)
{
    for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
        float s = 0.f;
        for (int k = 0; k < S; ++k) s += part[(size_t)k * n + i];
        out[i] = s;
    }
}

// Input gradient of a convolution from its column gradient (a gather over
// the up to nine output positions that read each input pixel), gated by the
// ReLU of the layer that produced the input: dZ_in = dX * [act > 0].
__global__ void k_col2im_gate(const float* __restrict__ dcol, int Kp, int B, int H, int W, int C, int Ho, int Wo,
                              int stride, const __nv_bfloat16* __restrict__ act, float* __restrict__ dZ)
{
    const long long total = (long long)B * H * W * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const long long p = t / C;
        const int ix = (int)(p % W);
        const long long r = p / W;
        const int iy = (int)(r % H), b = (int)(r / H);
        float acc = 0.f;
        for (int ky = 0; ky < 3; ++ky) {
            const int ty = iy + 1 - ky;
            if (ty < 0 || ty % stride) continue;
            const int oy = ty / stride;
            if (oy >= Ho) continue;
            for (int kx = 0; kx < 3; ++kx) {
                const int tx = ix + 1 - kx;
                if (tx < 0 || tx % stride) continue;
                const int ox = tx / stride;
                if (ox >= Wo) continue;
                acc += dcol[(((long long)b * Ho + oy) * Wo + ox) * Kp + (ky * 3 + kx) * C + c];
            }
        }
        dZ[t] = __bfloat162float(act[t]) > 0.f ? acc : 0.f;
    }
}

// Adam (Kingma and Ba) on the FP32 master copy; bc1 = 1 - beta1^t,
// bc2 = 1 - beta2^t.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// BF16 operand copies of one layer's master weights: Wb [Np][Kp] (rows past
// cout zero) and its transpose WTb [Kp][Cp] (columns past cout zero).
__global__ void k_refresh(const float* __restrict__ Wm, int cout, int Kp, int Np, int Cp, __nv_bfloat16* __restrict__ Wb,
                          __nv_bfloat16* __restrict__ WTb)
{
    const int n1 = Np * Kp, n2 = Kp * Cp;
    for (int i = blockIdx.x * NT + threadIdx.x; i < n1 + n2; i += gridDim.x * NT) {
        if (i < n1) {
            const int o = i / Kp, k = i - o * Kp;
            Wb[i] = __float2bfloat16_rn(o < cout ? Wm[(size_t)o * Kp + k] : 0.f);
        } else {
            const int j = i - n1, k = j / Cp, o = j - k * Cp;
            WTb[j] = __float2bfloat16_rn(o < cout ? Wm[(size_t)o * Kp + k] : 0.f);
        }
    }
}

// Standard layout ([cout][cin][3][3] then bias) <-> the GEMM layout
// ([cout][Kp] with k = (ky * 3 + kx) * cin + c, then bias).
__global__ void k_params_io(float* __restrict__ std_p, float* __restrict__ gemm_p, int cin, int cout, int Kp, int to_gemm)
{
    const int nw = cout * cin * 9;
    for (int i = blockIdx.x * NT + threadIdx.x; i < nw + cout; i += gridDim.x * NT) {
        if (i < nw) {
            const int tap = i % 9, r = i / 9, c = r % cin, o = r / cin;
            const size_t gi = (size_t)o * Kp + tap * cin + c;
            if (to_gemm)
                gemm_p[gi] = std_p[i];
            else
                std_p[i] = gemm_p[gi];
        } else {
            const int o = i - nw;
            if (to_gemm)
                gemm_p[(size_t)cout * Kp + o] = std_p[i];
            else
                std_p[i] = gemm_p[(size_t)cout * Kp + o];
        }
    }
}

inline int blocks_for(long long n, int cap = 152 * 8)
{
    long long b = (n + NT - 1) / NT;
    return (int)std::max<long long>(1, std::min<long long>(b, cap));
}

inline int rup(int x, int m) { return (x + m - 1) / m * m; }

struct Layer {
    int cin, cout, stride, relu;
    int H, W, Ho, Wo;
    int Kp, Np, Cp;
    size_t woff, boff;         // offsets in the internal parameter arena
    size_t soff;               // offset in the standard-layout parameter vector
    __nv_bfloat16 *Wb, *WTb;   // BF16 operand copies
    __nv_bfloat16* A;          // im2col [M][Kp]
    __nv_bfloat16* AT;         // its transpose [Kp][Mp]
    __nv_bfloat16* act;        // output [M][cout] (ReLU layers)
    float* dZ;                 // [M][cout]
    __nv_bfloat16 *dZb, *dZT;  // [M][Cp], [cout][Mp]
};

constexpr int NL = 6;
constexpr int LDEF[NL][3] = {{4, 32, 2}, {32, 64, 2}, {64, 64, 2}, {64, 64, 1}, {64, 32, 1}, {32, 6, 1}};

} // namespace

struct NetImpl {
    int max_batch = 0;
    Layer L[NL]{};
    size_t n_int = 0, n_std = 0;
    float *Wm = nullptr, *G = nullptr, *Am = nullptr, *Av = nullptr; // internal arena: params, grads, moments
    float* gstd = nullptr;      // gradients in the standard layout
    float* dcol = nullptr;      // column gradient scratch
    float* part = nullptr;      // split-K partials
    size_t part_n = 0;
    float* lpart = nullptr;     // loss partials
    float* out = nullptr;       // network output [B][6][8][10]
    float* in1 = nullptr;       // one quadruple's coarsest images [4][60][80]
    float* loss = nullptr;
    int* err = nullptr;
    int t = 0;                  // Adam steps taken
    std::vector<void*> allocs;
};

namespace {

template <typename T>
bool nalloc(NetImpl* n, T** p, size_t count)
{
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 256) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaMemset(q, 0, count * sizeof(T) + 256);
    n->allocs.push_back(q);
    *p = (T*)q;
    return true;
}

int rc_of(cudaError_t e)
{
    if (e == cudaSuccess) return SF_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA;
}

GemmArgs gemm_base(NetImpl* n)
{
    GemmArgs a{};
    a.err = n->err;
    return a;
}

int split_count(int kchunks, int& per)
{
    per = std::max(1, std::min(kchunks, 32));
    return (kchunks + per - 1) / per;
}

} // namespace

void net_free(NetImpl* n)
{
    if (!n) return;
    for (void* p : n->allocs) cudaFree(p);
    delete n;
}

NetImpl* net_create(int max_batch, int* rc)
{
    *rc = SF_ERR_ARG;
    if (max_batch < 1 || max_batch > 4096) return nullptr;
    NetImpl* n = new (std::nothrow) NetImpl();
    *rc = SF_ERR_OOM;
    if (!n) return nullptr;
    n->max_batch = max_batch;
    int H = NET_IN_H, W = NET_IN_W;
    size_t wo = 0, so = 0, dcol_max = 0, part_max = 0;
    bool ok = true;
    for (int l = 0; l < NL && ok; ++l) {
        Layer& y = n->L[l];
        y.cin = LDEF[l][0];
        y.cout = LDEF[l][1];
        y.stride = LDEF[l][2];
        y.relu = l < NL - 1;
        y.H = H;
        y.W = W;
        y.Ho = (H + y.stride - 1) / y.stride;
        y.Wo = (W + y.stride - 1) / y.stride;
        y.Kp = rup(9 * y.cin, 64);
        y.Np = rup(y.cout, 16);
        y.Cp = rup(y.cout, 64);
        y.woff = wo;
        y.boff = wo + (size_t)y.cout * y.Kp;
        wo = y.boff + y.cout;
        y.soff = so;
        so += (size_t)y.cout * y.cin * 9 + y.cout;
        const size_t M = (size_t)max_batch * y.Ho * y.Wo, Mp = rup((int)M, 64);
        ok = nalloc(n, &y.Wb, (size_t)y.Np * y.Kp) && nalloc(n, &y.WTb, (size_t)y.Kp * y.Cp) &&
             nalloc(n, &y.A, M * y.Kp) && nalloc(n, &y.AT, (size_t)y.Kp * Mp) && nalloc(n, &y.dZ, M * y.cout) &&
             nalloc(n, &y.dZb, M * y.Cp) && nalloc(n, &y.dZT, (size_t)y.cout * Mp);
        if (ok && y.relu) ok = nalloc(n, &y.act, M * y.cout);
        if (l > 0) dcol_max = std::max(dcol_max, M * y.Kp);
        int per;
        const int S = split_count((int)(Mp / 64), per);
        part_max = std::max(part_max, (size_t)S * y.cout * y.Kp);
        H = y.Ho;
        W = y.Wo;
    }
    n->n_int = wo;
    n->n_std = so;
    n->part_n = part_max;
    ok = ok && nalloc(n, &n->Wm, wo) && nalloc(n, &n->G, wo) && nalloc(n, &n->Am, wo) && nalloc(n, &n->Av, wo) &&
         nalloc(n, &n->gstd, so) && nalloc(n, &n->dcol, dcol_max) && nalloc(n, &n->part, part_max) &&
         nalloc(n, &n->lpart, 1024) && nalloc(n, &n->out, (size_t)max_batch * NET_OUT_C * NET_OUT_H * NET_OUT_W) &&
         nalloc(n, &n->loss, 1) && nalloc(n, &n->err, 1) &&
         nalloc(n, &n->in1, (size_t)4 * NET_IN_H * NET_IN_W);
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        net_free(n);
        return nullptr;
    }
    *rc = SF_OK;
    return n;
}

size_t net_param_count() { return 32 * 4 * 9 + 32 + 64 * 32 * 9 + 64 + 64 * 64 * 9 + 64 + 64 * 64 * 9 + 64 + 32 * 64 * 9 + 32 + 6 * 32 * 9 + 6; }

static void refresh_all(NetImpl* n, cudaStream_t st)
{
    for (int l = 0; l < NL; ++l) {
        Layer& y = n->L[l];
        k_refresh<<<blocks_for((long long)y.Np * y.Kp + (long long)y.Kp * y.Cp), NT, 0, st>>>(
            n->Wm + y.woff, y.cout, y.Kp, y.Np, y.Cp, y.Wb, y.WTb);
    }
}

int net_set_params(NetImpl* n, const float* p, cudaStream_t st)
{
    for (int l = 0; l < NL; ++l) {
        Layer& y = n->L[l];
        k_params_io<<<blocks_for((long long)y.cout * y.cin * 9 + y.cout), NT, 0, st>>>(
            const_cast<float*>(p) + y.soff, n->Wm + y.woff, y.cin, y.cout, y.Kp, 1);
    }
    refresh_all(n, st);
    cudaMemsetAsync(n->Am, 0, n->n_int * sizeof(float), st);
    cudaMemsetAsync(n->Av, 0, n->n_int * sizeof(float), st);
    n->t = 0;
    return rc_of(cudaGetLastError());
}

int net_get_params(NetImpl* n, float* p, cudaStream_t st)
{
    for (int l = 0; l < NL; ++l) {
        Layer& y = n->L[l];
        k_params_io<<<blocks_for((long long)y.cout * y.cin * 9 + y.cout), NT, 0, st>>>(p + y.soff, n->Wm + y.woff,
                                                                                     y.cin, y.cout, y.Kp, 0);
    }
    return rc_of(cudaGetLastError());
}

// Forward pass of `batch` images (FP32, channel c of image b at
// img + b * img_stride + c * ch_stride, rows of 80) into out [B][6][8][10].
int net_forward(NetImpl* n, const float* img, long long img_stride, long long ch_stride, int batch, float* out,
                cudaStream_t st)
{
    if (batch < 1 || batch > n->max_batch) return SF_ERR_ARG;
    for (int l = 0; l < NL; ++l) {
        Layer& y = n->L[l];
        const int M = batch * y.Ho * y.Wo;
        if (l == 0)
            k_im2col_img<<<blocks_for((long long)M * y.Kp), NT, 0, st>>>(img, img_stride, ch_stride, batch, y.H, y.W,
                                                                         y.Ho, y.Wo, y.stride, y.A, y.Kp);
        else
            k_im2col<<<blocks_for((long long)M * y.Kp / 8), NT, 0, st>>>(n->L[l - 1].act, batch, y.H, y.W, y.cin, y.Ho,
                                                                         y.Wo, y.stride, y.A, y.Kp);
        GemmArgs a = gemm_base(n);
        a.A = y.A;
        a.lda = y.Kp;
        a.B = y.Wb;
        a.ldb = y.Kp;
        a.M = M;
        a.N = y.Np;
        a.K = y.Kp;
        a.BN = y.Np;
        a.kc_per_split = y.Kp / 64;
        a.bias = n->Wm + y.boff;
        a.n_store = y.cout;
        int e;
        if (y.relu) {
            a.Cb = y.act;
            a.ldc = y.cout;
            e = GEMM_BIAS_RELU_BF16;
        } else {
            a.C = out;
            a.out_hw = y.Ho * y.Wo;
            e = GEMM_BIAS_NCHW_F32;
        }
        int rc = gemm_check(a);
        if (rc) return rc;
        rc = rc_of(launch_gemm(a, e, 1, st));
        if (rc) return rc;
    }
    return rc_of(cudaGetLastError());
}

// Forward and backward pass; gradients into the internal arena, the loss
// into n->loss.
int net_backward(NetImpl* n, const float* img, const float* target, int batch, cudaStream_t st)
{
    int rc = net_forward(n, img, (long long)4 * NET_IN_H * NET_IN_W, (long long)NET_IN_H * NET_IN_W, batch, n->out, st);
    if (rc) return rc;
    const int HW = NET_OUT_H * NET_OUT_W, nout = batch * NET_OUT_C * HW;
    const int lb = std::min(1024, (nout + NT - 1) / NT);
    Layer& last = n->L[NL - 1];
    k_loss_grad<<<lb, NT, 0, st>>>(n->out, target, batch, NET_OUT_C, HW, 2.f / (float)nout, last.dZ, n->lpart);
    k_sum_parts<<<1, 32, 0, st>>>(n->lpart, lb, 1.0f / (float)nout, n->loss);
    for (int l = NL - 1; l >= 0; --l) {
        Layer& y = n->L[l];
        const int M = batch * y.Ho * y.Wo, Mp = rup(M, 64);
        // bias gradient, and dZ in the two BF16 layouts the GEMMs read
        k_colsum<<<y.cout, NT, 0, st>>>(y.dZ, M, y.cout, n->G + y.boff);
        k_pack_dz<<<dim3((Mp + 31) / 32, (y.Cp + 31) / 32), dim3(32, 8), 0, st>>>(y.dZ, M, y.cout, y.Cp, Mp, y.dZb,
                                                                                 y.dZT);
        k_transpose_bf16<<<dim3((Mp + 31) / 32, (y.Kp + 31) / 32), dim3(32, 8), 0, st>>>(y.A, M, y.Kp, Mp, y.AT);
        // dW = dZ^T im2col(X): rows cout, columns Kp, reduction over the batch's pixels
        int per;
        const int S = split_count(Mp / 64, per);
        GemmArgs a = gemm_base(n);
        a.A = y.dZT;
        a.lda = Mp;
        a.B = y.AT;
        a.ldb = Mp;
        a.M = y.cout;
        a.N = y.Kp;
        a.K = Mp;
        a.BN = y.Kp <= 256 ? y.Kp : (y.Kp % 192 == 0 ? 192 : 160);
        a.kc_per_split = per;
        a.n_store = y.Kp;
        a.ldc = y.Kp;
        a.split_stride = (long long)y.cout * y.Kp;
        a.C = n->part;
        if ((size_t)S * y.cout * y.Kp > n->part_n) return SF_ERR_ARG;
        rc = gemm_check(a);
        if (!rc) rc = rc_of(launch_gemm(a, GEMM_F32, S, st));
        if (rc) return rc;
        k_split_reduce<<<blocks_for((long long)y.cout * y.Kp), NT, 0, st>>>(n->part, S, y.cout * y.Kp, n->G + y.woff);
        if (l == 0) break;
        // dX = col2im(dZ W), gated by the previous layer's ReLU
        GemmArgs b = gemm_base(n);
        b.A = y.dZb;
        b.lda = y.Cp;
        b.B = y.WTb;
        b.ldb = y.Cp;
        b.M = M;
        b.N = y.Kp;
        b.K = y.Cp;
        b.BN = a.BN;
        b.kc_per_split = y.Cp / 64;
        b.n_store = y.Kp;
        b.ldc = y.Kp;
        b.C = n->dcol;
        rc = gemm_check(b);
        if (!rc) rc = rc_of(launch_gemm(b, GEMM_F32, 1, st));
        if (rc) return rc;
        Layer& p = n->L[l - 1];
        k_col2im_gate<<<blocks_for((long long)batch * y.H * y.W * y.cin), NT, 0, st>>>(
            n->dcol, y.Kp, batch, y.H, y.W, y.cin, y.Ho, y.Wo, y.stride, p.act, p.dZ);
    }
    return rc_of(cudaGetLastError());
}

int net_grads_std(NetImpl* n, float* g, cudaStream_t st)
{
    for (int l = 0; l < NL; ++l) {
        Layer& y = n->L[l];
        k_params_io<<<blocks_for((long long)y.cout * y.cin * 9 + y.cout), NT, 0, st>>>(g + y.soff, n->G + y.woff, y.cin,
                                                                                     y.cout, y.Kp, 0);
    }
    return rc_of(cudaGetLastError());
}

int net_adam(NetImpl* n, float lr, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    n->t += 1;
    const float bc1 = (float)(1.0 - std::pow(0.9, n->t)), bc2 = (float)(1.0 - std::pow(0.999, n->t));
    k_adam<<<blocks_for((long long)n->n_int), NT, 0, st>>>(n->Wm, n->G, n->Am, n->Av, (int)n->n_int, lr, b1, b2, eps,
                                                          bc1, bc2);
    refresh_all(n, st);
    return rc_of(cudaGetLastError());
}

int net_error(NetImpl* n)
{
    int h = 0;
    if (cudaMemcpy(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return rc_of(cudaErrorUnknown);
    return h ? SF_ERR_TIMEOUT : SF_OK;
}

float* net_loss_ptr(NetImpl* n) { return n->loss; }
float* net_out_ptr(NetImpl* n) { return n->out; }
float* net_in_ptr(NetImpl* n) { return n->in1; }
size_t net_std_count(NetImpl* n) { return n->n_std; }

} // namespace sfk
