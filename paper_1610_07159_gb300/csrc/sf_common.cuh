// sf_common.cuh -- internal layouts and device helpers of the sm_103a
// halfway-domain scene-flow solver (Thies et al., arXiv 1610.07159).
//
// Data layout in device memory (one set per hierarchy level):
//   tex     [4][h][w] texels (I, dI/dx, dI/dy, 0) of the four images, so one
//           load fetches a texel with its gradient (Section 5.3 pyramid):
//           float4 (16 bytes) in FP32 mode, four FP16 or BF16 values (8 bytes)
//           in the mixed-precision modes
//   W       uint8  [h][w]: outlier weight of the current Gauss-Newton step
//   base, delta, x      float [6][G] component-major node fields
//   cell    float [CELL_VALS][ncell]: per warp-grid cell the ten symmetric 6x6
//           blocks sum_p alpha_k alpha_l H_p over its pixels and the four
//           6-vectors sum_p alpha_k b_p (Eq. 7 chain rule of Section 5.1)
//   node    float [NODE_VALS][G]: per node its own block and those coupling it
//           to the E, S, SE and SW neighbours (symmetric 6x6, 21 floats each);
//           the W, N, NW and NE couplings are the neighbours' stored blocks
//   rhs, minv, r, z, p0, p1   float [6][G] PCG vectors
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sf.h"

namespace sfk {

constexpr int NB = 21;                     // packed symmetric 6x6
constexpr int NPAIR = 10;                  // corner pairs (k <= l) of a cell
constexpr int CELL_VALS = NPAIR * NB + 24; // 234
constexpr int NODE_BLKS = 5;               // self, E, S, SE, SW
constexpr int NODE_VALS = NODE_BLKS * NB;  // 105
constexpr int ASM_THREADS = 256;
constexpr int MAX_PART = 65536;            // partial-sum slots per reduction (per-block partials of a level)

// device status bits
constexpr int DEV_TIMEOUT = 1;
constexpr int DEV_NUMERIC = 2;
constexpr int DEV_NOARGS = 4;  // a launch found no input or output buffer

struct LevelGeom {
    int w, h;     // level image size
    int nx, ny;   // grid nodes
    int G;        // nx * ny
    int ncx, ncy; // cells (nx - 1) x (ny - 1)
    int s;        // grid stride (level pixels)
    int level;
};

// Per-level parameters as the kernels use them.
struct DevParams {
    float w_reg, w_photo, w_grad, w_epi, w_smooth, w_mag;
    float wfl[3];  // w_s, w_m, w_d
    float mfl[3];  // m_s, m_m, m_d
    float eps, eps_p;
    float Fl[9];   // fundamental matrix in this level's pixels
    int robust_mode, grad_mode, wfeat_mode;
    float wfeat_gain, wfeat_tau;
};

// The maps a level's data terms take from the next coarser level (Algorithm
// 1, Section 5.3): V[h][w] the occlusion map (1 = visible; null: all
// visible) and L[2][h][w] the illumination difference of the right camera at
// times 0 and 1 in the reference frame (null: none).
struct LevelMaps {
    const uint8_t* V;
    const float* L;
};

// Control record of one Gauss-Newton step (one per level and step).
struct StepCtrl {
    double E_cur;        // energy at the linearisation point
    double E_acc;        // energy after the step (E_cur if rejected)
    double terms_cur[5]; // weighted photo, grad, smooth, epi, mag at the point
    double terms_acc[5];
    float t;             // accepted step length, 0 = rejected
    int accepted;
    int n_excluded;
    int t1_ok;           // the full step (t = 1) passed its trial (k_energy, trial mode)
    double E_t1;         // energy and weighted terms at the full step (W of the step)
    double terms_t1[5];
};

// Per-frame arguments read by the kernels of a captured graph.
struct DevArgs {
    const float* in[4];
    float* out;
    int frame;    // frames solved before this one
    int use_init; // coarsest delta from the warm-start buffer
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__host__ __device__ constexpr int sym_idx(int r, int c)
{
    return r <= c ? r * 6 - (r * (r - 1)) / 2 + (c - r) : c * 6 - (c * (c - 1)) / 2 + (r - c);
}

// Index of the corner pair (k, l) of a cell in the packed cell record.
__host__ __device__ constexpr int pair_idx(int k, int l)
{
    return k <= l ? (k == 0 ? l : (k == 1 ? 3 + l : (k == 2 ? 5 + l : 9))) : pair_idx(l, k);
}

// Signs of (s, m, d) in each image's sample position (Eqs. 1-6):
// image 0 at x-s-m+d, 1 at x+s-m-d, 2 at x-s+m-d, 3 at x+s+m+d.
__host__ __device__ constexpr float sgn(int img, int fld)
{
    return (img == 0) ? (fld == 2 ? 1.f : -1.f)
         : (img == 1) ? (fld == 0 ? 1.f : -1.f)
         : (img == 2) ? (fld == 1 ? 1.f : -1.f)
                      : 1.f;
}

// The six checks d_k = I_first - I_second of Eqs. 1-6.
__host__ __device__ constexpr int chk_first(int k) { return k == 0 ? 1 : (k == 1 ? 3 : (k == 2 ? 2 : (k == 3 ? 3 : (k == 4 ? 3 : 2)))); }
__host__ __device__ constexpr int chk_second(int k) { return k == 0 ? 0 : (k == 1 ? 2 : (k == 2 ? 0 : (k == 3 ? 1 : (k == 4 ? 0 : 1)))); }

__device__ __forceinline__ void sym_rank1(float* H, const float* J, float w)
{
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const float wr = w * J[r];
#pragma unroll
        for (int c = r; c < 6; ++c) H[sym_idx(r, c)] = fmaf(wr, J[c], H[sym_idx(r, c)]);
    }
}

__device__ __forceinline__ void sym_matvec_acc(const float* B, const float* p, float* y)
{
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        float a = y[r];
#pragma unroll
        for (int c = 0; c < 6; ++c) a = fmaf(B[sym_idx(r, c)], p[c], a);
        y[r] = a;
    }
}

// Cell and fraction along one axis of the sample position x + o (integer
// pixel x, real offset o). The fraction comes from the offset alone, so it
// keeps full FP32 precision however large x is. The position is clamped to
// [0, w-1]; the cell is min(floor(p), w-2); `clamped` marks a clamped axis
// (its derivative is 0). Offsets are limited to +-1e7 px first, which also
// keeps the integer arithmetic in range for any input.
__device__ __forceinline__ void axis_cell(int x, float o, int w, int& ix, float& f, bool& clamped)
{
    o = fminf(fmaxf(o, -1.0e7f), 1.0e7f);
    const float fo = floorf(o);
    const int pi = x + (int)fo;
    const float fr = o - fo; // exact, in [0, 1)
    if (pi < 0) {
        ix = 0;
        f = 0.f;
        clamped = true;
    } else if (pi > w - 1 || (pi == w - 1 && fr > 0.f)) {
        ix = w - 2;
        f = 1.f;
        clamped = true;
    } else if (pi == w - 1) {
        ix = w - 2;
        f = 1.f;
        clamped = false;
    } else {
        ix = pi;
        f = fr;
        clamped = false;
    }
}

// Record of the bilinear cell decisions taken by the assembly (a test aid,
// off on the solve path): every sample whose position lies within
// CELL_LOG_MARGIN px of a cell edge appends (pixel y*w + x, cell << 4 |
// clamped << 3 | image << 1 | axis). A cell is an integer decision taken in
// FP32 (reading C7); an FP64 implementation at a slightly different state can
// take the other cell there, and the analytic Jacobian of the bilinear
// interpolant jumps between cells. `n` may exceed `cap` (records past cap are
// dropped, the count still grows).
constexpr float CELL_LOG_MARGIN = 1e-3f;
struct CellLog {
    uint2* buf;
    unsigned* n;
    int cap;
};

__device__ __forceinline__ void log_cell(const CellLog* log, int pix, float o, int ix, bool clamped, int img, int axis)
{
    o = fminf(fmaxf(o, -1.0e7f), 1.0e7f);
    const float fr = o - floorf(o);
    if (fr >= CELL_LOG_MARGIN && fr <= 1.f - CELL_LOG_MARGIN) return;
    const unsigned k = atomicAdd(log->n, 1u);
    if (k < (unsigned)log->cap)
        log->buf[k] = make_uint2((unsigned)pix, ((unsigned)ix << 4) | ((clamped ? 1u : 0u) << 3) |
                                                     ((unsigned)img << 1) | (unsigned)axis);
}

// Texel storage: FP32 (float4) or 16-bit (four halves or bfloat16s in 8
// bytes). Loads convert to FP32; all arithmetic after the load is FP32.
struct TexF32 {
    using T = float4;
    __device__ __forceinline__ static float4 ld(const T* p) { return __ldg(p); }
    __device__ __forceinline__ static T pack(float a, float b, float c) { return make_float4(a, b, c, 0.f); }
};

struct TexF16 {
    using T = uint2;
    __device__ __forceinline__ static float4 ld(const T* p)
    {
        const uint2 v = __ldg(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ __forceinline__ static T pack(float a, float b, float c)
    {
        const __half2 h0 = __floats2half2_rn(a, b), h1 = __floats2half2_rn(c, 0.f);
        return make_uint2(*reinterpret_cast<const unsigned*>(&h0), *reinterpret_cast<const unsigned*>(&h1));
    }
};

struct TexBF16 {
    using T = uint2;
    __device__ __forceinline__ static float4 ld(const T* p)
    {
        const uint2 v = __ldg(p);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ __forceinline__ static T pack(float a, float b, float c)
    {
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b), h1 = __floats2bfloat162_rn(c, 0.f);
        return make_uint2(*reinterpret_cast<const unsigned*>(&h0), *reinterpret_cast<const unsigned*>(&h1));
    }
};

// Bytes per texel of a precision mode.
__host__ __device__ constexpr int texel_bytes(int prec) { return prec == SF_FP32 ? 16 : 8; }

// Host-side dispatch of a texel-typed launch on the precision mode.
#define SF_TEX_DISPATCH(prec, TT, ...)                                                                       \
    do {                                                                                                   \
        if ((prec) == SF_MIXED_FP16) {                                                                     \
            using TT = TexF16;                                                                             \
            __VA_ARGS__;                                                                                   \
        } else if ((prec) == SF_MIXED_BF16) {                                                              \
            using TT = TexBF16;                                                                            \
            __VA_ARGS__;                                                                                   \
        } else {                                                                                           \
            using TT = TexF32;                                                                             \
            __VA_ARGS__;                                                                                   \
        }                                                                                                  \
    } while (0)

// Bilinear sample of a texel plane (I, dI/dx, dI/dy) at (x + ox, y + oy)
// with the derivative of the interpolant.
struct Tap {
    float v[3], dx[3], dy[3];
};

template <class TT, bool REC = false>
__device__ __forceinline__ void tap4(const typename TT::T* __restrict__ T, int w, int h, int x, int y, float ox,
                                     float oy, Tap& o, const CellLog* log = nullptr, int img = 0)
{
    int ix, iy;
    float fx, fy;
    bool clx, cly;
    axis_cell(x, ox, w, ix, fx, clx);
    axis_cell(y, oy, h, iy, fy, cly);
    if (REC) {
        log_cell(log, y * w + x, ox, ix, clx, img, 0);
        log_cell(log, y * w + x, oy, iy, cly, img, 1);
    }
    const typename TT::T* r0 = T + (size_t)iy * w + ix;
    const float4 a = TT::ld(r0), b = TT::ld(r0 + 1), c = TT::ld(r0 + w), d = TT::ld(r0 + w + 1);
    const float av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z}, cv[3] = {c.x, c.y, c.z}, dv[3] = {d.x, d.y, d.z};
    const float gx = 1.f - fx, gy = 1.f - fy;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        float top = gx * av[p] + fx * bv[p];
        float bot = gx * cv[p] + fx * dv[p];
        o.v[p] = gy * top + fy * bot;
        o.dx[p] = clx ? 0.f : gy * (bv[p] - av[p]) + fy * (dv[p] - cv[p]);
        o.dy[p] = cly ? 0.f : bot - top;
    }
}

// Intensity only (halfway image).
template <class TT>
__device__ __forceinline__ float tap1(const typename TT::T* __restrict__ T, int w, int h, int x, int y, float ox,
                                      float oy)
{
    int ix, iy;
    float fx, fy;
    bool clx, cly;
    axis_cell(x, ox, w, ix, fx, clx);
    axis_cell(y, oy, h, iy, fy, cly);
    const typename TT::T* r0 = T + (size_t)iy * w + ix;
    float a = TT::ld(r0).x, b = TT::ld(r0 + 1).x, c = TT::ld(r0 + w).x, d = TT::ld(r0 + w + 1).x;
    float top = (1.f - fx) * a + fx * b, bot = (1.f - fx) * c + fx * d;
    return (1.f - fy) * top + fy * bot;
}

// Bilinear weights of pixel (x, y) on the warp grid (Eq. 7): cell (i0, j0)
// and fractions (a, b); pixels past the last node clamp to it.
__device__ __forceinline__ void grid_cell(int x, int y, int s, int nx, int ny, int& i0, int& j0, float& a, float& b)
{
    float u = fminf((float)x / (float)s, (float)(nx - 1));
    float v = fminf((float)y / (float)s, (float)(ny - 1));
    i0 = min((int)floorf(u), nx - 2);
    j0 = min((int)floorf(v), ny - 2);
    a = u - (float)i0;
    b = v - (float)j0;
}

// Fields of a pixel from the four nodes of its cell, F = base + delta (+ t x);
// delta and x may be null.
__device__ __forceinline__ void pixel_fields(const float* base, const float* delta, const float* x, float t, int G, int n00, int nx, float a,
                                             float b, float f[6])
{
    const int nd[4] = {n00, n00 + 1, n00 + nx, n00 + nx + 1};
    const float al[4] = {(1.f - a) * (1.f - b), a * (1.f - b), (1.f - a) * b, a * b};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float T = base[c * G + nd[k]];
            if (delta) T += delta[c * G + nd[k]];
            if (x) T = fmaf(t, x[c * G + nd[k]], T);
            acc = fmaf(al[k], T, acc);
        }
        f[c] = acc;
    }
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// float-float (unevaluated sum hi + lo) accumulation: about 44 significant
// bits from FP32 operations only. GB300's FP64 add has ~64 cycles of latency
// against ~4.5 for FP32, so reductions on a critical path avoid FP64.
// two_sum is Knuth's error-free transformation of a + b.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return ff{h, e - (h - s)};
}

__device__ __forceinline__ ff ff_from(float v) { return ff{v, 0.f}; }

__device__ __forceinline__ ff ff_shfl_xor(ff v, int m)
{
    return ff{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// Warp butterfly: every lane ends with the same total.
__device__ __forceinline__ ff ff_warp_sum(ff v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum; the result is valid in every thread. sh needs NT/32 entries.
// Within a warp the 32 values are summed in FP32 (a fixed tree), across warps
// and blocks in float-float.
template <int NT>
__device__ __forceinline__ ff ff_block_sum_fast(float x, ff* sh)
{
    const float w = warp_sum(x);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ff_from(w);
    __syncthreads();
    ff t = (threadIdx.x & 31) < NT / 32 ? sh[threadIdx.x & 31] : ff{0.f, 0.f};
    return ff_warp_sum(t);
}

// Block sum; the result is valid in every thread. sh needs NT/32 entries.
template <int NT>
__device__ __forceinline__ ff ff_block_sum(ff v, ff* sh)
{
    v = ff_warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    ff t = (threadIdx.x & 31) < NT / 32 ? sh[threadIdx.x & 31] : ff{0.f, 0.f};
    return ff_warp_sum(t);
}

// Fixed-order sum of n float-float partials written by other blocks (L2
// loads); every lane of the calling warp gets the same total.
__device__ __forceinline__ ff ff_fixed_sum(const float2* part, int n)
{
    const int lane = threadIdx.x & 31;
    ff v{0.f, 0.f};
    for (int i = lane; i < n; i += 32) {
        const float2 t = __ldcg(part + i);
        v = ff_add(v, ff{t.x, t.y});
    }
    return ff_warp_sum(v);
}

// Fixed-order sum of n float-float partials by a whole block: thread t folds
// indices t, t + NT, ... in order, then a fixed block reduction. Every thread
// of the block gets the same total.
template <int NT>
__device__ __forceinline__ ff ff_block_fixed_sum(const float2* part, int n, ff* sh)
{
    ff v{0.f, 0.f};
    for (int i = threadIdx.x; i < n; i += NT) {
        const float2 t = __ldcg(part + i);
        v = ff_add(v, ff{t.x, t.y});
    }
    return ff_block_sum<NT>(v, sh);
}

// K block sums at once: each result is bit-identical to ff_block_sum_fast
// (or ff_block_sum, ff_block_fixed_sum) of that value alone, with two CTA
// barriers in all instead of two per value. sh needs K * NT / 32 entries.
template <int NT, int K>
__device__ __forceinline__ void ff_block_sum_n(ff (&v)[K], ff* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = ff_warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh[k * (NT / 32) + warp] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = ff_warp_sum(lane < NT / 32 ? sh[k * (NT / 32) + lane] : ff{0.f, 0.f});
}

template <int NT, int K>
__device__ __forceinline__ void ff_block_sum_fast_n(const float (&x)[K], ff* sh, ff (&out)[K])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = warp_sum(x[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh[k * (NT / 32) + warp] = ff_from(w[k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = ff_warp_sum(lane < NT / 32 ? sh[k * (NT / 32) + lane] : ff{0.f, 0.f});
}

// K fixed-order sums of partial arrays (part[k] holds n[k] float-float
// partials), folded in the order of ff_block_fixed_sum with the K loads of
// one index in flight together.
template <int NT, int K>
__device__ __forceinline__ void ff_block_fixed_sum_n(const float2* const (&part)[K], const int (&n)[K], ff* sh,
                                                     ff (&out)[K])
{
    int nmax = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        out[k] = ff{0.f, 0.f};
        nmax = n[k] > nmax ? n[k] : nmax;
    }
#pragma unroll 4
    for (int i = threadIdx.x; i < nmax; i += NT) {
        float2 t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = i < n[k] ? __ldcg(part[k] + i) : make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (i < n[k]) out[k] = ff_add(out[k], ff{t[k].x, t[k].y});
    }
    ff_block_sum_n<NT, K>(out, sh);
}

// The last-block pattern of the fixed-order folds: thread 0 counts its block
// in with a release atomic (its partial-sum stores before the count), and
// the last block's threads read the partials after an acquire fence. Only
// the counting thread's own stores are ordered, so no block waits for the
// rest of its writes (a full __threadfence would).
__device__ __forceinline__ unsigned atom_add_release_gpu(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void fence_acquire_gpu_fold() { asm volatile("fence.acquire.gpu;" ::: "memory"); }

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__device__ __forceinline__ int ld_acquire_s32(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident), on a
// 64-bit arrival counter that only grows. Every launch of one kernel on one
// counter has the same number of blocks N and passes the same number of
// barriers in every block, so the counter is a multiple of N when a launch
// starts; a block reads it once (grid_barrier_base) before its first arrival,
// when at most N-1 arrivals of the first barrier can be in. Barrier k of the
// launch waits for base + k*N arrivals. Arrivals are fire-and-forget
// reductions (red.release.gpu), so N blocks do not queue behind returning
// atomics. A waiter gives up after about one second (clock64 on the SM clock),
// latches DEV_TIMEOUT and returns false; a waiter that finds an error in the
// status word (checked every 64 polls) returns false too, so the kernel
// unwinds instead of hanging. After a timeout the counter is no longer a
// multiple of N: the context resets it together with the status word. The
// limit is a parameter so that a test can run it out in a millisecond.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long grid_barrier_base(unsigned long long* ctr, unsigned nblocks)
{
    __shared__ unsigned long long base_sh;
    if (threadIdx.x == 0) base_sh = (ld_acquire_u64(ctr) / nblocks) * nblocks;
    __syncthreads();
    return base_sh;
}

__device__ __forceinline__ bool grid_barrier(unsigned long long* ctr, int* status, unsigned long long target,
                                             long long limit_cycles = 2000000000LL)
{
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        // arrive at once; the status word and the clock are read only every
        // 64 polls, so the fast path has a single reduction and the polls
        int ok = 1;
        red_release_add_u64(ctr, 1ull);
        const long long t0 = clock64();
        unsigned k = 0;
        while (ld_acquire_u64(ctr) < target) {
            if ((++k & 63u) != 0u) continue;
            if (ld_acquire_s32(status) != 0) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > limit_cycles) {
                atomicOr(status, DEV_TIMEOUT);
                ok = 0;
                break;
            }
        }
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

} // namespace sfk
