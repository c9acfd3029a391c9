// sf_pcg.cu -- data-parallel preconditioned conjugate gradients on the
// Gauss-Newton normal equations J^T J dx = -J^T r (Thies et al., arXiv
// 1610.07159, Section 5.1), Jacobi preconditioner.
//
// One launch runs every iteration of one solve. Four lanes serve one node:
// the node's 3x3 block stencil has nine coupling blocks (its own, E, S, SE
// and SW stored at the node, W, N, NW and NE stored at those neighbours; A is
// symmetric with symmetric 6x6 blocks), lane q applies stencil slots q and
// q + 4 (lane 0 also slot 8), and the four partial products meet in two
// shuffle rounds. The node's x, r, z, p live in the registers of its lanes,
// two components per lane (lanes 2 and 3 hold one). An iteration has two
// reductions, p.q and r.z: float-float per block, then a fixed-order sum of
// the block partials that every block computes identically, so all blocks
// take the same alpha, beta and stopping decision. A neighbour's p_k is formed
// on the fly from its z_k and p_{k-1} (double-buffered), which saves the third
// synchronisation of the textbook loop.
//
// Synchronisation: when the level fits in one thread-block cluster (up to 16
// CTAs) the launch is a single cluster and the phases meet at the hardware
// cluster barrier; larger levels use a cooperative launch over the whole GPU
// and a bounded global-memory barrier.
#include "sf_launch.h"

namespace sfk {

namespace {

constexpr int PT = 256; // threads per block
constexpr int NPB = PT / 4; // nodes per block and pass

struct ClusterSync {
    __device__ __forceinline__ bool sync(unsigned*, int*) const
    {
        cluster_sync_all();
        return true;
    }
};

struct GridSync {
    __device__ __forceinline__ bool sync(unsigned* bar, int* status) const { return grid_barrier(bar, status, gridDim.x); }
};

// Stencil slot s of node (i, j): the block (owner node, block index) and the
// node whose p it multiplies. Slots: 0 self, 1 E, 2 S, 3 SE, 4 SW (stored at
// the node), 5 W, 6 N, 7 NW, 8 NE (stored at the neighbour, which is also the
// p node). Returns false where the neighbour is off the grid.
__device__ __forceinline__ bool stencil_slot(int s, int i, int j, int nx, int ny, int n, int& owner, int& blk, int& pn)
{
    // packed per slot: di+1, dj+1 of the p node (2 bits each), block index (3 bits), stored-at-neighbour flag
    constexpr unsigned long long T = 0ull | (0x05ull << 0)   // 0: di 0 dj 0 blk 0 own   -> (1,1)
                                    | ((0x06ull | (1ull << 4)) << 8)  // 1: di 1 dj 0 blk 1
                                    | ((0x09ull | (2ull << 4)) << 16) // 2: di 0 dj 1 blk 2
                                    | ((0x0Aull | (3ull << 4)) << 24) // 3: di 1 dj 1 blk 3
                                    | ((0x08ull | (4ull << 4)) << 32) // 4: di -1 dj 1 blk 4
                                    | ((0x04ull | (1ull << 4) | 0x80ull) << 40) // 5: di -1 dj 0 blk 1 nb
                                    | ((0x01ull | (2ull << 4) | 0x80ull) << 48) // 6: di 0 dj -1 blk 2 nb
                                    | ((0x00ull | (3ull << 4) | 0x80ull) << 56); // 7: di -1 dj -1 blk 3 nb
    unsigned e;
    if (s < 8)
        e = (unsigned)(T >> (8 * s)) & 0xffu;
    else
        e = 0x02u | (4u << 4) | 0x80u; // 8: di 1 dj -1 blk 4 nb
    const int di = (int)(e & 3u) - 1, dj = (int)((e >> 2) & 3u) - 1;
    blk = (int)((e >> 4) & 7u);
    const int i2 = i + di, j2 = j + dj;
    if (i2 < 0 || i2 >= nx || j2 < 0 || j2 >= ny) return false;
    pn = n + dj * nx + di;
    owner = (e & 0x80u) ? pn : n;
    return true;
}

__device__ __forceinline__ float sel6(const float* v, int c)
{
    float r = v[0];
    r = c == 1 ? v[1] : r;
    r = c == 2 ? v[2] : r;
    r = c == 3 ? v[3] : r;
    r = c == 4 ? v[4] : r;
    r = c == 5 ? v[5] : r;
    return r;
}

template <class Sync>
__device__ __forceinline__ ff allreduce(ff v, ff* sh, float2* part, const Sync& sy, unsigned* bar, int* status, bool& ok)
{
    __shared__ ff bc;
    const ff b = ff_block_sum<PT>(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = make_float2(b.hi, b.lo);
    ok = sy.sync(bar, status) && ok;
    if (threadIdx.x < 32) {
        const ff t = ff_fixed_sum(part, gridDim.x);
        if (threadIdx.x == 0) bc = t;
    }
    __syncthreads();
    return bc;
}

template <int NPT, class Sync>
__global__ void __launch_bounds__(PT) k_pcg(LevelGeom g, const float* __restrict__ node, const float* __restrict__ rhs,
                                            const float* __restrict__ minv, float* __restrict__ xout, float* z,
                                            float* p0, float* p1, float2* part, unsigned* bar, int* status, int iters,
                                            int interleaved, Sync sy)
{
    __shared__ ff sred[PT / 32];
    const int G = g.G, nx = g.nx, ny = g.ny;
    const int q4 = threadIdx.x & 3;
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
    const int stride = gridDim.x * NPB;
    const int slot0 = blockIdx.x * NPB + (threadIdx.x >> 2);
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
                rr[k][h] = rhs[c * G + n];
                mr[k][h] = minv[c * G + n];
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
    bool ok = true;
    float2* part_pq = part;
    float2* part_rz = part + MAX_PART;
    ff rz = allreduce(ff_from(acc), sred, part_rz, sy, bar, status, ok);
    float beta = 0.f;
    for (int it = 0; it < iters && ok; ++it) {
        if (!(rz.hi > 1e-30f)) break;
        const bool first = it == 0;
        const float* pprev = (it & 1) ? p0 : p1; // p_{it-1} sits in buffer (it-1) & 1
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
#pragma unroll
                for (int ss = 0; ss < 3; ++ss) {
                    const int s = ss == 2 ? 8 : q4 + 4 * ss;
                    if (ss == 2 && q4 != 0) continue;
                    int owner, blk, pn;
                    if (!stencil_slot(s, i, j, nx, ny, n, owner, blk, pn)) continue;
                    float B[NB], pm[6];
#pragma unroll
                    for (int e = 0; e < NB; ++e) B[e] = __ldg(node + (size_t)(blk * NB + e) * G + owner);
#pragma unroll
                    for (int u = 0; u < 6; ++u) {
                        float v = __ldcg(z + u * G + pn);
                        if (!first) v = fmaf(beta, __ldcg(pprev + u * G + pn), v);
                        pm[u] = v;
                    }
                    sym_matvec_acc(B, pm, q);
                }
            }
            // the four lanes of a node are adjacent: two butterfly rounds
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                q[u] += __shfl_xor_sync(0xffffffffu, q[u], 1);
                q[u] += __shfl_xor_sync(0xffffffffu, q[u], 2);
            }
            if (live) {
                qr[k][0] = sel6(q, c0);
                qr[k][1] = has1 ? sel6(q, c1) : 0.f;
                acc = fmaf(pr[k][0], qr[k][0], acc);
                acc = fmaf(pr[k][1], qr[k][1], acc);
            }
        }
        const ff pq = allreduce(ff_from(acc), sred, part_pq, sy, bar, status, ok);
        if (!ok || !(pq.hi > 1e-30f)) break;
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
        const ff rz_new = allreduce(ff_from(acc), sred, part_rz, sy, bar, status, ok);
        beta = rz_new.hi / rz.hi;
        rz = rz_new;
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
        if (n >= G) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!(h == 0 || has1)) continue;
            const int c = h ? c1 : c0;
            if (interleaved)
                xout[n * 6 + c] = xr[k][h];
            else
                xout[c * G + n] = xr[k][h];
        }
    }
}

template <int NPT>
cudaError_t launch_cluster(int blocks, const LevelGeom& g, const float* node, const float* rhs, const float* minv,
                           float* x, float* z, float* p0, float* p1, float2* part, unsigned* bar, int* status, int iters,
                           int interleaved, cudaStream_t st)
{
    auto kern = k_pcg<NPT, ClusterSync>;
    if (blocks > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = blocks;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved,
                              ClusterSync{});
}

template <int NPT>
cudaError_t launch_grid(int blocks, const LevelGeom& g, const float* node, const float* rhs, const float* minv, float* x,
                        float* z, float* p0, float* p1, float2* part, unsigned* bar, int* status, int iters,
                        int interleaved, cudaStream_t st)
{
    LevelGeom gg = g;
    GridSync sy;
    void* args[] = {(void*)&gg, (void*)&node, (void*)&rhs, (void*)&minv, (void*)&x, (void*)&z, (void*)&p0,
                    (void*)&p1, (void*)&part, (void*)&bar, (void*)&status, (void*)&iters, (void*)&interleaved,
                    (void*)&sy};
    return cudaLaunchCooperativeKernel((const void*)k_pcg<NPT, GridSync>, dim3(blocks), dim3(PT), args, 0, st);
}

int max_coop_blocks(int sm_count)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<1, GridSync>, PT, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * sm_count;
}

int max_cluster_blocks()
{
    static int cached = -1;
    if (cached > 0) return cached;
    auto kern = k_pcg<1, ClusterSync>;
    int n = 8;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(PT);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int m = 0;
        if (cudaOccupancyMaxPotentialClusterSize(&m, kern, &cfg) == cudaSuccess && m > 0) n = m;
    }
    cudaGetLastError();
    cached = n > 16 ? 16 : n;
    return cached;
}

} // namespace

PcgPlan pcg_plan(int G, int sm_count, int mode)
{
    PcgPlan p{1, 1, 0};
    const int maxc = max_cluster_blocks();
    if (mode != SF_PCG_GRID) {
        for (int npt : {1, 2, 4}) {
            const int need = (G + NPB * npt - 1) / (NPB * npt);
            if (need <= maxc) {
                p.blocks = need < 1 ? 1 : need;
                p.npt = npt;
                p.cluster = 1;
                return p;
            }
        }
        if (mode == SF_PCG_CLUSTER) {
            p.blocks = -1;
            return p;
        }
    }
    int cap = max_coop_blocks(sm_count);
    if (cap > MAX_PART) cap = MAX_PART;
    for (int npt : {1, 2, 4}) {
        const int need = (G + NPB * npt - 1) / (NPB * npt);
        if (need <= cap) {
            p.blocks = need < 1 ? 1 : need;
            p.npt = npt;
            p.cluster = 0;
            return p;
        }
    }
    p.blocks = -1; // too large for one launch
    return p;
}

cudaError_t launch_pcg(const LevelGeom& g, const PcgPlan& plan, const float* node, const float* rhs, const float* minv,
                       float* x, float* z, float* p0, float* p1, float2* part, unsigned* bar, int* status, int iters,
                       int interleaved_out, cudaStream_t st)
{
    if (plan.cluster) {
        switch (plan.npt) {
        case 1: return launch_cluster<1>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
        case 2: return launch_cluster<2>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
        default: return launch_cluster<4>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
        }
    }
    switch (plan.npt) {
    case 1: return launch_grid<1>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
    case 2: return launch_grid<2>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
    default: return launch_grid<4>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
    }
}

} // namespace sfk
