// sf_levels.cu -- streaming kernels of the solver: the mip-map pyramid with
// gradient planes (Section 5.3), level initialisation of the delta hierarchy
// with prolongation (Algorithm 1) and constant-velocity temporal transfer
// (Section 5.3), the halfway image and the feature weight w_i of the
// smoothness term (Section 4.3), and the per-level output.
#include "sf_launch.h"
#include "sf_stages.cuh"

namespace sfk {

namespace {

constexpr int T1D = 256;

// Level 0 texels: intensity and central-difference gradients, edge clamped.
template <class TT>
__global__ void k_tex0(const DevArgs* __restrict__ args, const float* in0, const float* in1, const float* in2,
                       const float* in3, int w, int h, typename TT::T* __restrict__ tex)
{
    const int c = blockIdx.y;
    const float* I = args ? args->in[c] : (c == 0 ? in0 : c == 1 ? in1 : c == 2 ? in2 : in3);
    const int n = w * h;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        tex[(size_t)c * n + p] = tex0_texel<TT>(I, w, h, p);
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
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        tex[(size_t)c * n + p] = texdown_texel<TT>(P, wp, hp, w, h, p);
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
    const int frame = args ? args->frame : frame_direct;
    const int use_init = args ? args->use_init : use_init_direct;
    level_init_node(g, have_coarse, nxc, nyc, base_c, delta_c, base, delta, prev_delta, prev_total, init_buf,
                    temporal_mode, frame, use_init, n);
}

// Halfway image H(x) = mean of the four warped intensities.
template <class TT>
__global__ void k_halfway(LevelGeom g, const typename TT::T* __restrict__ tex, const float* __restrict__ base,
                          const float* __restrict__ delta, float* __restrict__ H)
{
    const int n = g.w * g.h;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        H[p] = halfway_pixel<TT>(g, tex, base, delta, p);
    }
}

// w_i = 1 + gain exp(-lambda_min / tau), lambda_min the smaller eigenvalue of
// the structure tensor of H over the 3x3 pixels at the node.
__global__ void k_wfeat(LevelGeom g, const float* __restrict__ H, DevParams P, float* __restrict__ wf)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.G) return;
    wf[n] = wfeat_node(g, H, P, n);
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

template <class TT>
__global__ void k_tex_intensity(const typename TT::T* __restrict__ tex, int n, float* __restrict__ out)
{
    const int c = blockIdx.y;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        out[(size_t)c * n + p] = TT::ld(tex + (size_t)c * n + p).x;
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

void launch_tex_intensity(const void* tex, int prec, int w, int h, float* out, cudaStream_t st)
{
    dim3 grid(grid1d((size_t)w * h), 4);
    SF_TEX_DISPATCH(prec, TT, k_tex_intensity<TT><<<grid, T1D, 0, st>>>(static_cast<const typename TT::T*>(tex),
                                                                         w * h, out));
}

void launch_unpack_tex(const void* tex, int prec, int w, int h, float* planes, cudaStream_t st)
{
    dim3 grid(grid1d((size_t)w * h), 4);
    SF_TEX_DISPATCH(prec, TT, k_unpack_tex<TT><<<grid, T1D, 0, st>>>(static_cast<const typename TT::T*>(tex), w * h,
                                                                      planes));
}

} // namespace sfk
