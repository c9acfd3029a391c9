// sf_maps.cu -- the per-level maps of Algorithm 1 (Thies et al., arXiv
// 1610.07159, Section 5.3): after a level's solve, the occlusion map (the
// triangulated warp grid rendered into the four views with a z-buffer,
// prolongated to the next finer level as its V of Eqs. 11 and 13) and the
// illumination correction map (the stereo intensity residual in the reference
// frame, low-passed by a Gaussian and box-prolongated; the next level
// subtracts it from the right images' intensities).
//
// Occlusion: one thread per (view, triangle) rasterises the triangle's pixel
// centres with edge functions and keeps the largest closeness per pixel with
// atomicMax on an order-preserving integer image of the float; one thread per
// reference pixel then compares its own closeness with the z-buffer at its
// four rounded sample positions. Illumination: one thread per pixel forms the
// two stereo residuals from bilinear texel samples; the Gaussian runs as two
// separable passes with clamped edges.
#include <math.h>

#include "sf_launch.h"
#include "sf_stages.cuh"

namespace sfk {

namespace {

constexpr int MT = 256;

// order-preserving map of floats to ints (monotone for every non-NaN value)
__device__ __forceinline__ int ord_enc(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord_dec(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// closeness of a surface point at time t: its stereo pair's horizontal
// disparity, left sample offset less right sample offset (larger = nearer)
__device__ __forceinline__ float closeness(int t, const float f[6])
{
    const int il = 2 * t, ir = il + 1;
    const float ol = sgn(il, 0) * f[0] + sgn(il, 1) * f[2] + sgn(il, 2) * f[4];
    const float orr = sgn(ir, 0) * f[0] + sgn(ir, 1) * f[2] + sgn(ir, 2) * f[4];
    return ol - orr;
}

__device__ __forceinline__ float edge_fn(float ax, float ay, float bx, float by, float px, float py)
{
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

__global__ void k_fill_int(int* __restrict__ p, int v, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void __launch_bounds__(MT) k_occ_raster(LevelGeom g, const float* __restrict__ base,
                                                   const float* __restrict__ delta, int* __restrict__ Z)
{
    const int ntri = 2 * g.ncx * g.ncy;
    const int idx = blockIdx.x * MT + threadIdx.x;
    if (idx >= 4 * ntri) return;
    const int c = idx / ntri, k = idx - c * ntri;
    const int cell = k >> 1, tri = k & 1;
    const int j = cell / g.ncx, i = cell - j * g.ncx;
    const int vi[3] = {i, i + 1, tri == 0 ? i + 1 : i};
    const int vj[3] = {j, tri == 0 ? j : j + 1, j + 1};
    float X[3], Y[3], K[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        const int n = vj[v] * g.nx + vi[v];
        float f[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) f[q] = base[q * g.G + n] + (delta ? delta[q * g.G + n] : 0.f);
        X[v] = (float)(vi[v] * g.s) + sgn(c, 0) * f[0] + sgn(c, 1) * f[2] + sgn(c, 2) * f[4];
        Y[v] = (float)(vj[v] * g.s) + sgn(c, 0) * f[1] + sgn(c, 1) * f[3] + sgn(c, 2) * f[5];
        K[v] = closeness(c >> 1, f);
    }
    const float area = edge_fn(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
    if (area == 0.f || !isfinite(area)) return;
    const float sgn_a = area < 0.f ? -1.f : 1.f, aabs = fabsf(area);
    const float xmin = fminf(X[0], fminf(X[1], X[2])), xmax = fmaxf(X[0], fmaxf(X[1], X[2]));
    const float ymin = fminf(Y[0], fminf(Y[1], Y[2])), ymax = fmaxf(Y[0], fmaxf(Y[1], Y[2]));
    const int x0 = (int)ceilf(fmaxf(xmin, 0.f)), x1 = (int)floorf(fminf(xmax, (float)(g.w - 1)));
    const int y0 = (int)ceilf(fmaxf(ymin, 0.f)), y1 = (int)floorf(fminf(ymax, (float)(g.h - 1)));
    int* Zc = Z + (size_t)c * g.w * g.h;
    for (int py = y0; py <= y1; ++py)
        for (int px = x0; px <= x1; ++px) {
            const float fx = (float)px, fy = (float)py;
            const float b0 = sgn_a * edge_fn(X[1], Y[1], X[2], Y[2], fx, fy);
            const float b1 = sgn_a * edge_fn(X[2], Y[2], X[0], Y[0], fx, fy);
            const float b2 = sgn_a * edge_fn(X[0], Y[0], X[1], Y[1], fx, fy);
            if (b0 < 0.f || b1 < 0.f || b2 < 0.f) continue;
            const float kz = (b0 * K[0] + b1 * K[1] + b2 * K[2]) / aabs;
            atomicMax(Zc + (size_t)py * g.w + px, ord_enc(kz));
        }
}

__global__ void __launch_bounds__(MT) k_occ_visible(LevelGeom g, const float* __restrict__ base,
                                                    const float* __restrict__ delta, const int* __restrict__ Z,
                                                    float tau, uint8_t* __restrict__ O)
{
    const int p = blockIdx.x * MT + threadIdx.x;
    if (p >= g.w * g.h) return;
    const int y = p / g.w, x = p - y * g.w;
    int i0, j0;
    float a, b;
    grid_cell(x, y, g.s, g.nx, g.ny, i0, j0, a, b);
    float f[6];
    pixel_fields(base, delta, nullptr, 0.f, g.G, j0 * g.nx + i0, g.nx, a, b, f);
    uint8_t vis = 1;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float px = (float)x + sgn(c, 0) * f[0] + sgn(c, 1) * f[2] + sgn(c, 2) * f[4];
        const float py = (float)y + sgn(c, 0) * f[1] + sgn(c, 1) * f[3] + sgn(c, 2) * f[5];
        const float qx = floorf(px + 0.5f), qy = floorf(py + 0.5f);
        if (!(qx >= 0.f && qx <= (float)(g.w - 1) && qy >= 0.f && qy <= (float)(g.h - 1))) {
            vis = 0;
            break;
        }
        const float z = ord_dec(Z[(size_t)c * g.w * g.h + (size_t)qy * g.w + (size_t)qx]);
        if (!(closeness(c >> 1, f) >= z - tau)) {
            vis = 0;
            break;
        }
    }
    O[p] = vis;
}

// V(x, y) = [bilinear interpolation of the coarse 0/1 map at (x/2, y/2) >= 1/2];
// the weights are multiples of 1/4, so FP32 takes the same decision as any
// wider arithmetic
__global__ void __launch_bounds__(MT) k_vis_up(int wc, int hc, const uint8_t* __restrict__ O, int w, int h,
                                               uint8_t* __restrict__ V)
{
    const int p = blockIdx.x * MT + threadIdx.x;
    if (p >= w * h) return;
    const int y = p / w, x = p - y * w;
    const float u = fminf(0.5f * x, (float)(wc - 1)), v = fminf(0.5f * y, (float)(hc - 1));
    const int i0 = min((int)floorf(u), wc - 2), j0 = min((int)floorf(v), hc - 2);
    const float a = u - (float)i0, bb = v - (float)j0;
    const uint8_t* r = O + j0 * wc + i0;
    const float top = (1.f - a) * (float)r[0] + a * (float)r[1];
    const float bot = (1.f - a) * (float)r[wc] + a * (float)r[wc + 1];
    V[p] = ((1.f - bb) * top + bb * bot) >= 0.5f ? 1 : 0;
}

// r[t][p]: the stereo intensity residual of time t at pixel p (right image
// sample less left image sample, checks d_0 and d_1 of Eqs. 1-6)
template <class TT>
__global__ void __launch_bounds__(MT) k_illum_res(LevelGeom g, const typename TT::T* __restrict__ tex,
                                                  const float* __restrict__ base, const float* __restrict__ delta,
                                                  float* __restrict__ r)
{
    const int p = blockIdx.x * MT + threadIdx.x;
    const int N = g.w * g.h;
    if (p >= N) return;
    const int y = p / g.w, x = p - y * g.w;
    int i0, j0;
    float a, b;
    grid_cell(x, y, g.s, g.nx, g.ny, i0, j0, a, b);
    float f[6];
    pixel_fields(base, delta, nullptr, 0.f, g.G, j0 * g.nx + i0, g.nx, a, b, f);
    float I[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float ox = sgn(c, 0) * f[0] + sgn(c, 1) * f[2] + sgn(c, 2) * f[4];
        const float oy = sgn(c, 0) * f[1] + sgn(c, 1) * f[3] + sgn(c, 2) * f[5];
        I[c] = tap1<TT>(tex + (size_t)c * N, g.w, g.h, x, y, ox, oy);
    }
    r[p] = I[1] - I[0];
    r[N + p] = I[3] - I[2];
}

// one separable pass of the Gaussian along x (dir 0) or y (dir 1), edges clamped, both times
__global__ void __launch_bounds__(MT) k_blur(int w, int h, GaussW gw, int dir, const float* __restrict__ src,
                                             float* __restrict__ dst)
{
    const int N = w * h;
    const int q = blockIdx.x * MT + threadIdx.x;
    if (q >= 2 * N) return;
    const int t = q / N, p = q - t * N;
    const int y = p / w, x = p - y * w;
    const float* s = src + (size_t)t * N;
    float acc = 0.f;
    for (int k = -gw.R; k <= gw.R; ++k) {
        const int xx = dir == 0 ? min(max(x + k, 0), w - 1) : x;
        const int yy = dir == 1 ? min(max(y + k, 0), h - 1) : y;
        acc = fmaf(gw.w[k + gw.R], s[yy * w + xx], acc);
    }
    dst[q] = acc;
}

// box prolongation: fine pixel (x, y) takes coarse pixel (x/2, y/2)
__global__ void __launch_bounds__(MT) k_illum_up(int wc, int hc, const float* __restrict__ R, int w, int h,
                                                 float* __restrict__ L)
{
    const int q = blockIdx.x * MT + threadIdx.x;
    const int N = w * h;
    if (q >= 2 * N) return;
    const int t = q / N, p = q - t * N;
    const int y = p / w, x = p - y * w;
    const int xc = min(x / 2, wc - 1), yc = min(y / 2, hc - 1);
    L[q] = R[(size_t)t * wc * hc + (size_t)yc * wc + xc];
}

int blocks_for(size_t n) { return (int)((n + MT - 1) / MT); }

} // namespace

GaussW gauss_weights(float sigma)
{
    GaussW g{};
    g.R = (int)ceil(3.0 * (double)sigma);
    if (g.R > GAUSS_MAX_R) g.R = GAUSS_MAX_R;
    double sum = 0.0, v[2 * GAUSS_MAX_R + 1];
    for (int k = -g.R; k <= g.R; ++k) {
        v[k + g.R] = exp(-(double)k * k / (2.0 * (double)sigma * sigma));
        sum += v[k + g.R];
    }
    for (int k = 0; k <= 2 * g.R; ++k) g.w[k] = (float)(v[k] / sum);
    return g;
}

void launch_occlusion(const LevelGeom& g, const float* base, const float* delta, float tau, int* Z, uint8_t* O,
                      cudaStream_t st)
{
    const size_t N = (size_t)g.w * g.h;
    // the z-buffer starts at -inf (its order-preserving image)
    const int neg_inf = (int)(0xff800000u ^ 0x7fffffffu);
    k_fill_int<<<blocks_for(4 * N) < 1184 ? blocks_for(4 * N) : 1184, MT, 0, st>>>(Z, neg_inf, 4 * N);
    const int ntri = 2 * g.ncx * g.ncy;
    k_occ_raster<<<blocks_for((size_t)4 * ntri), MT, 0, st>>>(g, base, delta, Z);
    k_occ_visible<<<blocks_for(N), MT, 0, st>>>(g, base, delta, Z, tau, O);
}

void launch_vis_up(int wc, int hc, const uint8_t* O, int w, int h, uint8_t* V, cudaStream_t st)
{
    k_vis_up<<<blocks_for((size_t)w * h), MT, 0, st>>>(wc, hc, O, w, h, V);
}

void launch_illum(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta,
                  const GaussW& gw, float* r, float* tmp, cudaStream_t st)
{
    const size_t N = (size_t)g.w * g.h;
    SF_TEX_DISPATCH(prec, TT, k_illum_res<TT><<<blocks_for(N), MT, 0, st>>>(
                                  g, static_cast<const typename TT::T*>(tex), base, delta, r));
    k_blur<<<blocks_for(2 * N), MT, 0, st>>>(g.w, g.h, gw, 0, r, tmp);
    k_blur<<<blocks_for(2 * N), MT, 0, st>>>(g.w, g.h, gw, 1, tmp, r);
}

void launch_illum_up(int wc, int hc, const float* R, int w, int h, float* L, cudaStream_t st)
{
    k_illum_up<<<blocks_for((size_t)2 * w * h), MT, 0, st>>>(wc, hc, R, w, h, L);
}

} // namespace sfk
