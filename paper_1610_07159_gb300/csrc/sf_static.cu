// sf_static.cu -- sf_pcg_static: the Jacobi-preconditioned conjugate-gradient
// solve of a warp-grid block system without any device allocation.
//
// Some callers cannot allocate device memory at the point where they solve:
// real-time loops that must not hit the allocator's implicit device
// synchronisation, and host applications whose memory pool or fixed device
// budget forbids a library's raw allocations after start-up. For them this entry point keeps its
// scratch in one file-scope __device__ array, fixed at build time:
// SF_STATIC_PCG_MAX_NODES nodes (z and two p buffers, 18 floats per node,
// 288 KiB, plus 32 reduction slots). Every GPU that loads the library holds
// that array until the process exits.
//
// The solve itself is the same algorithm as the context's PCG: four lanes per
// node, one thread-block cluster of up to 16 CTAs, float-float reductions.
// It reads the caller's blocks in the unpacked [G][5][6][6] layout that
// sf_probe_assemble writes.
#include <mutex>

#include "sf_launch.h"

namespace sfk {
namespace {

constexpr int ST_PT = 256;
constexpr int ST_NPB = ST_PT / 4;
constexpr int ST_MAX_CTAS = 16;
constexpr int ST_MAX_NODES = SF_STATIC_PCG_MAX_NODES;
constexpr size_t ST_VEC = (size_t)6 * ST_MAX_NODES;
// layout: z | p0 | p1 | 2 x ST_MAX_CTAS float2 partials
constexpr size_t ST_FLOATS = 3 * ST_VEC + 4 * ST_MAX_CTAS;

static __device__ __align__(256) float g_static_scratch[ST_FLOATS];

// Device address of g_static_scratch per device, looked up once with that
// device current (in host code the symbol is only a host-side stand-in). The
// cache is not refreshed after cudaDeviceReset, which unloads the module: a
// process that resets a device must not call sf_pcg_static on it afterwards.
float* g_scratch_addr[64] = {nullptr};
std::mutex g_scratch_mu;

int scratch_address(float** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return SF_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SF_ERR_CUDA;
        }
        g_scratch_addr[dev] = (float*)p;
    }
    *out = g_scratch_addr[dev];
    return SF_OK;
}

__device__ __forceinline__ float blk_entry(const float* __restrict__ blocks, int owner, int blk, int r, int c)
{
    return __ldg(blocks + ((size_t)owner * 5 + blk) * 36 + r * 6 + c);
}

__device__ __forceinline__ float st_sel6(const float* v, int c)
{
    float r = v[0];
    r = c == 1 ? v[1] : r;
    r = c == 2 ? v[2] : r;
    r = c == 3 ? v[3] : r;
    r = c == 4 ? v[4] : r;
    r = c == 5 ? v[5] : r;
    return r;
}

// Slot s of the nine-block stencil of node (i, j): 0 self, 1 E, 2 S, 3 SE,
// 4 SW (stored at the node), 5 W, 6 N, 7 NW, 8 NE (stored at the neighbour).
__device__ __forceinline__ bool st_slot(int s, int i, int j, int nx, int ny, int n, int& owner, int& blk, int& pn)
{
    int di = 0, dj = 0;
    switch (s) {
    case 1: di = 1; break;
    case 2: dj = 1; break;
    case 3: di = 1; dj = 1; break;
    case 4: di = -1; dj = 1; break;
    case 5: di = -1; break;
    case 6: dj = -1; break;
    case 7: di = -1; dj = -1; break;
    case 8: di = 1; dj = -1; break;
    default: break;
    }
    const int i2 = i + di, j2 = j + dj;
    if (i2 < 0 || i2 >= nx || j2 < 0 || j2 >= ny) return false;
    pn = n + dj * nx + di;
    owner = s >= 5 ? pn : n;
    blk = s >= 5 ? s - 4 : s;
    return true;
}

__device__ __forceinline__ ff st_allreduce(ff v, ff* sh, float2* part)
{
    __shared__ ff bc;
    const ff b = ff_block_sum<ST_PT>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = make_float2(b.hi, b.lo);
    cluster_sync_all();
    if (threadIdx.x < 32) {
        const ff t = ff_fixed_sum(part, gridDim.x);
        if (threadIdx.x == 0) bc = t;
    }
    __syncthreads();
    return bc;
}

template <int NPT>
__global__ void __launch_bounds__(ST_PT) k_pcg_static(int nx, int ny, const float* __restrict__ blocks,
                                                      const float* __restrict__ rhs, int iters, float* __restrict__ xout,
                                                      float* scratch)
{
    __shared__ ff sred[ST_PT / 32];
    const int G = nx * ny;
    float* z = scratch;
    float* p0 = scratch + ST_VEC;
    float* p1 = scratch + 2 * ST_VEC;
    float2* part = reinterpret_cast<float2*>(scratch + 3 * ST_VEC);
    float2* part_pq = part;
    float2* part_rz = part + ST_MAX_CTAS;
    const int q4 = threadIdx.x & 3;
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
    const int stride = gridDim.x * ST_NPB;
    const int slot0 = blockIdx.x * ST_NPB + (threadIdx.x >> 2);
    float xr[NPT][2], rr[NPT][2], zr[NPT][2], pr[NPT][2], mr[NPT][2], qr[NPT][2];
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = h ? c1 : c0;
            xr[k][h] = qr[k][h] = 0.f;
            if (n < G && (h == 0 || has1)) {
                const float d = blk_entry(blocks, n, 0, c, c);
                rr[k][h] = __ldg(rhs + n * 6 + c);
                mr[k][h] = d > 0.f ? 1.f / d : 1.f;
                zr[k][h] = mr[k][h] * rr[k][h];
                pr[k][h] = zr[k][h];
                z[c * G + n] = zr[k][h];
                p0[c * G + n] = zr[k][h];
                acc = fmaf(rr[k][h], zr[k][h], acc);
            } else {
                rr[k][h] = mr[k][h] = zr[k][h] = pr[k][h] = 0.f;
            }
        }
    }
    ff rz = st_allreduce(ff_from(acc), sred, part_rz);
    float beta = 0.f;
    for (int it = 0; it < iters; ++it) {
        if (!(rz.hi > 1e-30f)) break;
        const bool first = it == 0;
        const float* pprev = (it & 1) ? p0 : p1;
        float* pcur = (it & 1) ? p1 : p0;
        acc = 0.f;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int n = slot0 + k * stride;
            const bool live = n < G;
            if (live && !first) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    pr[k][h] = fmaf(beta, pr[k][h], zr[k][h]);
                    if (h == 0 || has1) pcur[(h ? c1 : c0) * G + n] = pr[k][h];
                }
            }
            float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (live) {
                const int i = n % nx, j = n / nx;
                for (int ss = 0; ss < 3; ++ss) {
                    const int s = ss == 2 ? 8 : q4 + 4 * ss;
                    if (ss == 2 && q4 != 0) continue;
                    int owner, blk, pn;
                    if (!st_slot(s, i, j, nx, ny, n, owner, blk, pn)) continue;
                    float pm[6];
#pragma unroll
                    for (int u = 0; u < 6; ++u) {
                        float v = __ldcg(z + u * G + pn);
                        if (!first) v = fmaf(beta, __ldcg(pprev + u * G + pn), v);
                        pm[u] = v;
                    }
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
                        float a = q[r];
#pragma unroll
                        for (int c = 0; c < 6; ++c) a = fmaf(blk_entry(blocks, owner, blk, r, c), pm[c], a);
                        q[r] = a;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                q[u] += __shfl_xor_sync(0xffffffffu, q[u], 1);
                q[u] += __shfl_xor_sync(0xffffffffu, q[u], 2);
            }
            if (live) {
                qr[k][0] = st_sel6(q, c0);
                qr[k][1] = has1 ? st_sel6(q, c1) : 0.f;
                acc = fmaf(pr[k][0], qr[k][0], acc);
                acc = fmaf(pr[k][1], qr[k][1], acc);
            }
        }
        const ff pq = st_allreduce(ff_from(acc), sred, part_pq);
        if (!(pq.hi > 1e-30f)) break;
        const float alpha = rz.hi / pq.hi;
        acc = 0.f;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int n = slot0 + k * stride;
            if (n >= G) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!(h == 0 || has1)) continue;
                xr[k][h] = fmaf(alpha, pr[k][h], xr[k][h]);
                rr[k][h] = fmaf(-alpha, qr[k][h], rr[k][h]);
                zr[k][h] = mr[k][h] * rr[k][h];
                z[(h ? c1 : c0) * G + n] = zr[k][h];
                acc = fmaf(rr[k][h], zr[k][h], acc);
            }
        }
        const ff rz_new = st_allreduce(ff_from(acc), sred, part_rz);
        beta = rz_new.hi / rz.hi;
        rz = rz_new;
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
        if (n >= G) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (h == 0 || has1) xout[n * 6 + (h ? c1 : c0)] = xr[k][h];
    }
}

template <int NPT>
cudaError_t launch_static(int ctas, int nx, int ny, const float* blocks, const float* rhs, int iters, float* x,
                          float* scratch, cudaStream_t st)
{
    auto kern = k_pcg_static<NPT>;
    if (ctas > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(ST_PT);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, nx, ny, blocks, rhs, iters, x, scratch);
}

} // namespace
} // namespace sfk

extern "C" int sf_pcg_static(int nx, int ny, const float* blocks, const float* rhs, int iters, float* x, void* stream)
{
    using namespace sfk;
    if (nx < 1 || ny < 1 || iters < 0 || !blocks || !rhs || !x) return SF_ERR_ARG;
    if ((long long)nx * ny > ST_MAX_NODES) return SF_ERR_ARG; // beyond the static scratch
    float* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != SF_OK) return rc;
    const int G = nx * ny;
    int npt = 1, ctas = (G + ST_NPB - 1) / ST_NPB;
    while (ctas > ST_MAX_CTAS) {
        npt *= 2;
        ctas = (G + ST_NPB * npt - 1) / (ST_NPB * npt);
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    switch (npt) {
    case 1: e = launch_static<1>(ctas, nx, ny, blocks, rhs, iters, x, scratch, st); break;
    case 2: e = launch_static<2>(ctas, nx, ny, blocks, rhs, iters, x, scratch, st); break;
    default: e = launch_static<4>(ctas, nx, ny, blocks, rhs, iters, x, scratch, st); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SF_ERR_CUDA;
    }
    return SF_OK;
}
