// sf_levels.cu -- streaming kernels of the solver: the mip-map pyramid with
// gradient planes (Section 5.3), level initialisation of the delta hierarchy
// with prolongation (Algorithm 1) and constant-velocity temporal transfer
// (Section 5.3), the halfway image and the feature weight w_i of the
// smoothness term (Section 4.3), and the per-level output.
#include "sf_launch.h"

namespace sfk {

namespace {

constexpr int T1D = 256;

__device__ __forceinline__ float grid_bilerp(const float* __restrict__ F, int nx, int ny, float u, float v)
{
    u = fminf(fmaxf(u, 0.f), (float)(nx - 1));
    v = fminf(fmaxf(v, 0.f), (float)(ny - 1));
    int i0 = min((int)floorf(u), nx - 2), j0 = min((int)floorf(v), ny - 2);
    float a = u - (float)i0, b = v - (float)j0;
    const float* r = F + j0 * nx + i0;
    float top = (1.f - a) * r[0] + a * r[1];
    float bot = (1.f - a) * r[nx] + a * r[nx + 1];
    return (1.f - b) * top + b * bot;
}

// Level 0 texels: intensity and central-difference gradients, edge clamped.
template <class TT>
__global__ void k_tex0(const DevArgs* __restrict__ args, const float* in0, const float* in1, const float* in2,
                       const float* in3, int w, int h, typename TT::T* __restrict__ tex)
{
    const int c = blockIdx.y;
    const float* I = args ? args->in[c] : (c == 0 ? in0 : c == 1 ? in1 : c == 2 ? in2 : in3);
    const int n = w * h;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int y = p / w, x = p - y * w;
        const int xm = max(x - 1, 0), xp = min(x + 1, w - 1), ym = max(y - 1, 0), yp = min(y + 1, h - 1);
        const float v = __ldg(I + p);
        const float gx = 0.5f * (__ldg(I + y * w + xp) - __ldg(I + y * w + xm));
        const float gy = 0.5f * (__ldg(I + yp * w + x) - __ldg(I + ym * w + x));
        tex[(size_t)c * n + p] = TT::pack(v, gx, gy);
    }
}

template <class TT>
__device__ __forceinline__ float box2(const typename TT::T* __restrict__ P, int wp, int hp, int x, int y)
{
    const int x0 = min(2 * x, wp - 1), x1 = min(2 * x + 1, wp - 1);
    const int y0 = min(2 * y, hp - 1), y1 = min(2 * y + 1, hp - 1);
    float acc = TT::ld(&P[y0 * wp + x0]).x;
    acc += TT::ld(&P[y0 * wp + x1]).x;
    acc += TT::ld(&P[y1 * wp + x0]).x;
    acc += TT::ld(&P[y1 * wp + x1]).x;
    return 0.25f * acc;
}

// Next mip level: 2x2 box of the finer intensity (edge clamped), gradients
// from the box values of the four neighbours.
template <class TT>
__global__ void k_texdown(const typename TT::T* __restrict__ texp, int wp, int hp, typename TT::T* __restrict__ tex,
                          int w, int h)
{
    const int c = blockIdx.y;
    const typename TT::T* P = texp + (size_t)c * wp * hp;
    const int n = w * h;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int y = p / w, x = p - y * w;
        const int xm = max(x - 1, 0), xp = min(x + 1, w - 1), ym = max(y - 1, 0), yp = min(y + 1, h - 1);
        const float v = box2<TT>(P, wp, hp, x, y);
        const float gx = 0.5f * (box2<TT>(P, wp, hp, xp, y) - box2<TT>(P, wp, hp, xm, y));
        const float gy = 0.5f * (box2<TT>(P, wp, hp, x, yp) - box2<TT>(P, wp, hp, x, ym));
        tex[(size_t)c * n + p] = TT::pack(v, gx, gy);
    }
}

// base = 2 Up(T_coarse) (node (i, j) reads coarse grid coordinates (i/2, j/2)),
// delta from the warm start, the temporal rule or zero.
__global__ void k_level_init(LevelGeom g, int have_coarse, int nxc, int nyc, const float* __restrict__ base_c,
                             const float* __restrict__ delta_c, float* __restrict__ base, float* __restrict__ delta,
                             const float* __restrict__ prev_delta, const float* __restrict__ prev_total,
                             const float* __restrict__ init_buf, const DevArgs* __restrict__ args, int temporal_mode,
                             int frame_direct, int use_init_direct)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.G) return;
    const int i = n % g.nx, j = n / g.nx;
    const int Gc = nxc * nyc;
    const int frame = args ? args->frame : frame_direct;
    const int use_init = args ? args->use_init : use_init_direct;
    for (int c = 0; c < 6; ++c) {
        float b = 0.f;
        if (have_coarse) {
            // T_coarse = base_c + delta_c, interpolated on the fly
            const float u = fminf(fmaxf(0.5f * i, 0.f), (float)(nxc - 1));
            const float v = fminf(fmaxf(0.5f * j, 0.f), (float)(nyc - 1));
            const int i0 = min((int)floorf(u), nxc - 2), j0 = min((int)floorf(v), nyc - 2);
            const float a = u - (float)i0, bb = v - (float)j0;
            const int m = j0 * nxc + i0;
            // delta_c == nullptr: base_c already holds the coarse totals
            const float t00 = base_c[c * Gc + m] + (delta_c ? delta_c[c * Gc + m] : 0.f);
            const float t10 = base_c[c * Gc + m + 1] + (delta_c ? delta_c[c * Gc + m + 1] : 0.f);
            const float t01 = base_c[c * Gc + m + nxc] + (delta_c ? delta_c[c * Gc + m + nxc] : 0.f);
            const float t11 = base_c[c * Gc + m + nxc + 1] + (delta_c ? delta_c[c * Gc + m + nxc + 1] : 0.f);
            const float top = (1.f - a) * t00 + a * t10, bot = (1.f - a) * t01 + a * t11;
            b = 2.f * ((1.f - bb) * top + bb * bot);
        }
        base[c * g.G + n] = b;
    }
    for (int c = 0; c < 6; ++c) {
        float d = 0.f;
        if (!have_coarse && use_init) {
            d = init_buf[c * g.G + n];
        } else if (frame > 0) {
            if (temporal_mode == SF_TEMPORAL_COPY) {
                d = prev_delta[c * g.G + n];
            } else if (temporal_mode == SF_TEMPORAL_PROPAGATE) {
                const float X = (float)(i * g.s) - 2.f * prev_total[2 * g.G + n];
                const float Y = (float)(j * g.s) - 2.f * prev_total[3 * g.G + n];
                d = grid_bilerp(prev_delta + c * g.G, g.nx, g.ny, X / (float)g.s, Y / (float)g.s);
            }
        }
        delta[c * g.G + n] = d;
    }
}

// Halfway image H(x) = mean of the four warped intensities.
template <class TT>
__global__ void k_halfway(LevelGeom g, const typename TT::T* __restrict__ tex, const float* __restrict__ base,
                          const float* __restrict__ delta, float* __restrict__ H)
{
    const int n = g.w * g.h;
    const size_t plane = (size_t)n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int y = p / g.w, x = p - y * g.w;
        int i0, j0;
        float a, b;
        grid_cell(x, y, g.s, g.nx, g.ny, i0, j0, a, b);
        float f[6];
        pixel_fields(base, delta, nullptr, 0.f, g.G, j0 * g.nx + i0, g.nx, a, b, f);
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float ox = sgn(c, 0) * f[0] + sgn(c, 1) * f[2] + sgn(c, 2) * f[4];
            const float oy = sgn(c, 0) * f[1] + sgn(c, 1) * f[3] + sgn(c, 2) * f[5];
            acc += tap1<TT>(tex + c * plane, g.w, g.h, x, y, ox, oy);
        }
        H[p] = 0.25f * acc;
    }
}

// w_i = 1 + gain exp(-lambda_min / tau), lambda_min the smaller eigenvalue of
// the structure tensor of H over the 3x3 pixels at the node.
__global__ void k_wfeat(LevelGeom g, const float* __restrict__ H, DevParams P, float* __restrict__ wf)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.G) return;
    const int i = n % g.nx, j = n / g.nx;
    float a = 0.f, b = 0.f, c = 0.f;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int qx = min(max(i * g.s + dx, 0), g.w - 1), qy = min(max(j * g.s + dy, 0), g.h - 1);
            const int xm = max(qx - 1, 0), xp = min(qx + 1, g.w - 1), ym = max(qy - 1, 0), yp = min(qy + 1, g.h - 1);
            const float hx = 0.5f * (H[qy * g.w + xp] - H[qy * g.w + xm]);
            const float hy = 0.5f * (H[yp * g.w + qx] - H[ym * g.w + qx]);
            a = fmaf(hx, hx, a);
            b = fmaf(hx, hy, b);
            c = fmaf(hy, hy, c);
        }
    float lmin = 0.5f * (a + c) - sqrtf(0.25f * (a - c) * (a - c) + b * b);
    lmin = fmaxf(lmin, 0.f);
    wf[n] = 1.f + P.wfeat_gain * expf(-lmin / P.wfeat_tau);
}

__global__ void k_fill(float* p, float v, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_add(const float* a, const float* b, float* out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

// Keeps this level's delta and total for the next frame; level 0 also
// writes the output fields.
__global__ void k_finish_level(int n6, const float* __restrict__ base, const float* __restrict__ delta,
                               float* __restrict__ prev_delta, float* __restrict__ prev_total,
                               const DevArgs* __restrict__ args, int write_out, float* __restrict__ out_direct)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n6) return;
    const float d = delta[k];
    const float T = base[k] + d;
    prev_delta[k] = d;
    prev_total[k] = T;
    if (write_out) (args ? args->out : out_direct)[k] = T;
}

template <class TT>
__global__ void k_unpack_tex(const typename TT::T* __restrict__ tex, int n, float* __restrict__ planes)
{
    const int c = blockIdx.y;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 t = TT::ld(tex + (size_t)c * n + p);
        planes[((size_t)c * 3 + 0) * n + p] = t.x;
        planes[((size_t)c * 3 + 1) * n + p] = t.y;
        planes[((size_t)c * 3 + 2) * n + p] = t.z;
    }
}

inline int grid1d(size_t n, int cap = 152 * 16)
{
    size_t b = (n + T1D - 1) / T1D;
    if (b > (size_t)cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

} // namespace

void launch_tex0(const DevArgs* args, const float* const* in_direct, int w, int h, void* tex, int prec, cudaStream_t st)
{
    dim3 grid(grid1d((size_t)w * h), 4);
    SF_TEX_DISPATCH(prec, TT, {
        auto* t = static_cast<typename TT::T*>(tex);
        if (args)
            k_tex0<TT><<<grid, T1D, 0, st>>>(args, nullptr, nullptr, nullptr, nullptr, w, h, t);
        else
            k_tex0<TT><<<grid, T1D, 0, st>>>(nullptr, in_direct[0], in_direct[1], in_direct[2], in_direct[3], w, h, t);
    });
}

void launch_texdown(const void* texp, int wp, int hp, void* tex, int w, int h, int prec, cudaStream_t st)
{
    dim3 grid(grid1d((size_t)w * h), 4);
    SF_TEX_DISPATCH(prec, TT, k_texdown<TT><<<grid, T1D, 0, st>>>(static_cast<const typename TT::T*>(texp), wp, hp,
                                                                   static_cast<typename TT::T*>(tex), w, h));
}

void launch_level_init(const LevelGeom& g, const LevelGeom* gc, const float* base_c, const float* delta_c,
                       float* base, float* delta, const float* prev_delta, const float* prev_total,
                       const float* init_buf, const DevArgs* args, int temporal_mode, int frame, int use_init,
                       cudaStream_t st)
{
    k_level_init<<<(g.G + T1D - 1) / T1D, T1D, 0, st>>>(g, gc != nullptr, gc ? gc->nx : 0, gc ? gc->ny : 0, base_c,
                                                        delta_c, base, delta, prev_delta, prev_total, init_buf,
                                                        args, temporal_mode, frame, use_init);
}

void launch_halfway(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta, float* H,
                    cudaStream_t st)
{
    SF_TEX_DISPATCH(prec, TT, k_halfway<TT><<<grid1d((size_t)g.w * g.h), T1D, 0, st>>>(
                                  g, static_cast<const typename TT::T*>(tex), base, delta, H));
}

void launch_wfeat(const LevelGeom& g, const float* H, const DevParams& P, float* wf, cudaStream_t st)
{
    k_wfeat<<<(g.G + T1D - 1) / T1D, T1D, 0, st>>>(g, H, P, wf);
}

void launch_fill(float* p, float v, size_t n, cudaStream_t st) { k_fill<<<grid1d(n), T1D, 0, st>>>(p, v, n); }

void launch_add(const float* a, const float* b, float* out, size_t n, cudaStream_t st)
{
    k_add<<<grid1d(n), T1D, 0, st>>>(a, b, out, n);
}

void launch_finish_level(const LevelGeom& g, const float* base, const float* delta, float* prev_delta,
                         float* prev_total, const DevArgs* args, int write_out, float* out, cudaStream_t st)
{
    const int n6 = 6 * g.G;
    k_finish_level<<<(n6 + T1D - 1) / T1D, T1D, 0, st>>>(n6, base, delta, prev_delta, prev_total, args, write_out,
                                                         out);
}

void launch_unpack_tex(const void* tex, int prec, int w, int h, float* planes, cudaStream_t st)
{
    dim3 grid(grid1d((size_t)w * h), 4);
    SF_TEX_DISPATCH(prec, TT, k_unpack_tex<TT><<<grid, T1D, 0, st>>>(static_cast<const typename TT::T*>(tex), w * h,
                                                                      planes));
}

} // namespace sfk
