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
// and a bounded global-memory barrier, or, in the one-reduction kernels,
// partial sums that carry their own tags (allreduce2_tagged).
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "sf_launch.h"
#include "sf_stages.cuh"

namespace cg = cooperative_groups;

namespace sfk {

namespace {

constexpr int PT = 256; // threads per block
constexpr int NPB = PT / 4; // nodes per block and pass

struct ClusterSync {
    static constexpr bool kGrid = false;
    __device__ __forceinline__ void start(unsigned long long*) {}
    __device__ __forceinline__ bool sync(unsigned long long*, int*)
    {
        cluster_sync_all();
        return true;
    }
};

struct GridSync {
    static constexpr bool kGrid = true;
    unsigned long long target;
    __device__ __forceinline__ void start(unsigned long long* ctr) { target = grid_barrier_base(ctr, gridDim.x); }
    __device__ __forceinline__ bool sync(unsigned long long* ctr, int* status)
    {
        target += gridDim.x;
        return grid_barrier(ctr, status, target);
    }
};

template <class Sync>
__device__ __forceinline__ ff allreduce(float v, ff* sh, float2* part, Sync& sy, unsigned long long* bar, int* status,
                                        bool& ok)
{
    __shared__ ff bc;
    const ff b = ff_block_sum_fast<PT>(v, sh);
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
                                            float* p0, float* p1, float2* part, unsigned long long* bar, int* status,
                                            int iters, int interleaved, Sync sy)
{
    __shared__ ff sred[PT / 32];
    sy.start(bar);
    const int G = g.G, nx = g.nx, ny = g.ny;
    const int q4 = threadIdx.x & 3;
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
    const int stride = gridDim.x * NPB;
    const int slot0 = blockIdx.x * NPB + (threadIdx.x >> 2);
    float xr[NPT][2], rr[NPT][2], zr[NPT][2], pr[NPT][2], mr[NPT][2], qr[NPT][2];
    int ni[NPT], nj[NPT]; // node coordinates, computed once
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
        nj[k] = n / nx;
        ni[k] = n - nj[k] * nx;
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
    ff rz = allreduce(acc, sred, part_rz, sy, bar, status, ok);
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
                const int i = ni[k], j = nj[k];
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
        const ff pq = allreduce(acc, sred, part_pq, sy, bar, status, ok);
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
        const ff rz_new = allreduce(acc, sred, part_rz, sy, bar, status, ok);
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

// ---------------------------------------------------------------------------
// Single-cluster PCG with everything in distributed shared memory.
//
// Each CTA of one cluster owns a contiguous range of npc nodes and keeps, per
// owned node, its five coupling blocks (21 floats padded to 24 for 16-byte
// loads), its preconditioner and two published sets (r, w, s) in shared
// memory; neighbours read them through distributed shared memory. The loop
// is the Chronopoulos-Gear form of PCG (algebraically the same iterates as
// the textbook loop): with u = M r and w = A u, the two dot products
// gamma = r.u and delta = w.u come from one fused reduction, and a neighbour's
// u_{i+1} = M (r_i - alpha (w_i + beta s_{i-1})) is formed on the fly from
// its published r_i, w_i and s_{i-1}. So an iteration has one matrix-vector
// product, one reduction and one cluster barrier.
// ---------------------------------------------------------------------------
constexpr int CT = 512;          // threads per CTA
constexpr int CT_NPB = CT / 4;   // node slots per pass
constexpr int NF_BLK = 120, NF_MINV = 8, NF_PUB = 24;
constexpr int NODE_F = NF_BLK + NF_MINV + 2 * NF_PUB; // 176 floats per owned node
constexpr int PUB_R = 0, PUB_W = 8, PUB_S = 16;

__device__ __forceinline__ void ld6(const float* p, float v[6])
{
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float2 b = *reinterpret_cast<const float2*>(p + 4);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
    v[4] = b.x;
    v[5] = b.y;
}

__device__ __forceinline__ void ld21(const float* p, float B[NB])
{
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const float4 a = reinterpret_cast<const float4*>(p)[q];
        B[4 * q] = a.x;
        B[4 * q + 1] = a.y;
        B[4 * q + 2] = a.z;
        B[4 * q + 3] = a.w;
    }
    B[20] = p[20];
}

// Block sums of two values (FP32 within a warp, float-float across warps);
// valid in every thread.
__device__ __forceinline__ void ff_block_sum2(float x, float y, ff& a, ff& b, ff* sh)
{
    x = warp_sum(x);
    y = warp_sum(y);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sh[2 * (threadIdx.x >> 5)] = ff_from(x);
        sh[2 * (threadIdx.x >> 5) + 1] = ff_from(y);
    }
    __syncthreads();
    const int l = threadIdx.x & 31;
    a = l < CT / 32 ? sh[2 * l] : ff{0.f, 0.f};
    b = l < CT / 32 ? sh[2 * l + 1] : ff{0.f, 0.f};
    a = ff_warp_sum(a);
    b = ff_warp_sum(b);
}

// Owning CTA and local index of node m near this CTA's range [n_lo, n_lo + npc):
// stencil neighbours are at most one grid row away, so a few steps suffice.
__device__ __forceinline__ void dsm_owner(int m, int rank, int n_lo, int npc, int& r, int& l)
{
    r = rank;
    l = m - n_lo;
    while (l < 0) {
        l += npc;
        --r;
    }
    while (l >= npc) {
        l -= npc;
        ++r;
    }
}

// ONE: the whole level in one CTA. Its own shared memory is then addressed
// directly (no distributed-shared-memory window) and CTA barriers stand in for
// the cluster barriers; the arithmetic and the order of every sum are those of
// the cluster form.
template <int NPT, bool ONE>
__global__ void __launch_bounds__(CT, 1) k_pcg_dsm(LevelGeom g, int npc, const float* __restrict__ node,
                                                const float* __restrict__ rhs, const float* __restrict__ minv_g,
                                                float* __restrict__ xout, int iters, int interleaved)
{
    extern __shared__ float4 dsm4[];
    float* sm = reinterpret_cast<float*>(dsm4);
    __shared__ ff sred[2 * (CT / 32)];
    __shared__ float2 cpart[2][2]; // [parity][gamma, delta] of this CTA as float-float pairs
    cg::cluster_group cl = cg::this_cluster();
    const int G = g.G, nx = g.nx, ny = g.ny;
    const int rank = ONE ? 0 : (int)cl.block_rank();
    const int C = ONE ? 1 : (int)cl.num_blocks();
    auto csync = [&]() {
        if constexpr (ONE)
            __syncthreads();
        else
            cl.sync();
    };
    auto peer = [&](auto* p, int r) {
        if constexpr (ONE)
            return p;
        else
            return cl.map_shared_rank(p, r);
    };
    const int n_lo = rank * npc;
    const int n_own = min(npc, G - n_lo);
    const int q4 = threadIdx.x & 3;
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
    const int ls = threadIdx.x >> 2;

    // stage the owned nodes' blocks and preconditioner; publish r_0 = b, s_{-1} = 0
    for (int t = threadIdx.x; t < n_own * NODE_VALS; t += CT) {
        const int e = t / n_own, ln = t - e * n_own;
        const int blk = e / NB, ee = e - blk * NB;
        sm[ln * NODE_F + blk * 24 + ee] = __ldg(node + (size_t)e * G + n_lo + ln);
    }
    for (int t = threadIdx.x; t < n_own * 6; t += CT) {
        const int c = t / n_own, ln = t - c * n_own;
        float* nd = sm + ln * NODE_F;
        nd[NF_BLK + c] = __ldg(minv_g + c * G + n_lo + ln);
        nd[NF_BLK + NF_MINV + PUB_R + c] = __ldg(rhs + c * G + n_lo + ln);
        nd[NF_BLK + NF_MINV + PUB_S + c] = 0.f;
    }
    float xr[NPT][2], rr[NPT][2], ur[NPT][2], wr[NPT][2], sr[NPT][2], pr[NPT][2], mr[NPT][2];
    int ni[NPT], nj[NPT]; // node coordinates, computed once
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int ln = ls + k * CT_NPB;
        nj[k] = (n_lo + ln) / nx;
        ni[k] = n_lo + ln - nj[k] * nx;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = h ? c1 : c0;
            const bool live = ln < n_own && (h == 0 || has1);
            const float r0 = live ? __ldg(rhs + c * G + n_lo + ln) : 0.f;
            mr[k][h] = live ? __ldg(minv_g + c * G + n_lo + ln) : 0.f;
            rr[k][h] = r0;
            ur[k][h] = mr[k][h] * r0;
            xr[k][h] = wr[k][h] = sr[k][h] = pr[k][h] = 0.f;
        }
    }
    csync();

    float alpha = 0.f, beta = 0.f;
    ff gam{0.f, 0.f};
    for (int i = -1; i < iters; ++i) {
        // i = -1 is the set-up pass: w_0 = A u_0 and the first reduction
        const int par = i < 0 ? 0 : (i & 1);
        const int npar = i < 0 ? 0 : (par ^ 1);
        if (i >= 0) {
            // own updates: p_i, s_i, x_{i+1}, r_{i+1}, u_{i+1}
#pragma unroll
            for (int k = 0; k < NPT; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    pr[k][h] = fmaf(beta, pr[k][h], ur[k][h]);
                    sr[k][h] = fmaf(beta, sr[k][h], wr[k][h]);
                    xr[k][h] = fmaf(alpha, pr[k][h], xr[k][h]);
                    rr[k][h] = fmaf(-alpha, sr[k][h], rr[k][h]);
                    ur[k][h] = mr[k][h] * rr[k][h];
                }
            if (i == iters - 1) break;
            // publish r_{i+1} and s_i for the next pass
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int ln = ls + k * CT_NPB;
                if (ln >= n_own) continue;
                float* pub = sm + ln * NODE_F + NF_BLK + NF_MINV + npar * NF_PUB;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!(h == 0 || has1)) continue;
                    const int c = h ? c1 : c0;
                    pub[PUB_R + c] = rr[k][h];
                    pub[PUB_S + c] = sr[k][h];
                }
            }
        }
        // w_{i+1} = A u_{i+1}, neighbours' u formed on the fly from buffer `par`
        float gp = 0.f, dp = 0.f;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int ln = ls + k * CT_NPB;
            const bool live = ln < n_own;
            const int n = n_lo + ln;
            float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (live) {
                const int ii = ni[k], jj = nj[k];
#pragma unroll
                for (int ss = 0; ss < 3; ++ss) {
                    const int s = ss == 2 ? 8 : q4 + 4 * ss;
                    if (ss == 2 && q4 != 0) continue;
                    int owner, blk, pn;
                    if (!stencil_slot(s, ii, jj, nx, ny, n, owner, blk, pn)) continue;
                    int ro = 0, lo = owner, rp = 0, lp = pn;
                    if constexpr (!ONE) {
                        dsm_owner(owner, rank, n_lo, npc, ro, lo);
                        dsm_owner(pn, rank, n_lo, npc, rp, lp);
                    }
                    const float* ob = peer(sm, ro) + lo * NODE_F + blk * 24;
                    const float* pb = peer(sm, rp) + lp * NODE_F;
                    float B[NB], mm[6], rv[6], wv[6], sv[6], u[6];
                    ld21(ob, B);
                    ld6(pb + NF_BLK, mm);
                    ld6(pb + NF_BLK + NF_MINV + par * NF_PUB + PUB_R, rv);
                    if (i >= 0) {
                        ld6(pb + NF_BLK + NF_MINV + par * NF_PUB + PUB_W, wv);
                        ld6(pb + NF_BLK + NF_MINV + par * NF_PUB + PUB_S, sv);
#pragma unroll
                        for (int c = 0; c < 6; ++c) u[c] = mm[c] * fmaf(-alpha, fmaf(beta, sv[c], wv[c]), rv[c]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 6; ++c) u[c] = mm[c] * rv[c];
                    }
                    sym_matvec_acc(B, u, q);
                }
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                q[c] += __shfl_xor_sync(0xffffffffu, q[c], 1);
                q[c] += __shfl_xor_sync(0xffffffffu, q[c], 2);
            }
            if (live) {
                wr[k][0] = sel6(q, c0);
                wr[k][1] = has1 ? sel6(q, c1) : 0.f;
                float* pub = sm + ln * NODE_F + NF_BLK + NF_MINV + npar * NF_PUB;
                pub[PUB_W + c0] = wr[k][0];
                if (has1) pub[PUB_W + c1] = wr[k][1];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    gp = fmaf(rr[k][h], ur[k][h], gp);
                    dp = fmaf(wr[k][h], ur[k][h], dp);
                }
            }
        }
        ff ga, de;
        ff_block_sum2(gp, dp, ga, de, sred);
        const int slot = i < 0 ? 0 : npar;
        if (threadIdx.x == 0) {
            cpart[slot][0] = make_float2(ga.hi, ga.lo);
            cpart[slot][1] = make_float2(de.hi, de.lo);
        }
        csync();
        // every CTA sums the CTAs' partials in rank order
        ff G2{0.f, 0.f}, D2{0.f, 0.f};
        for (int rk = 0; rk < C; ++rk) {
            const float2* rp = &peer(&cpart[0][0], rk)[slot * 2];
            const float2 a = rp[0], b = rp[1];
            G2 = ff_add(G2, ff{a.x, a.y});
            D2 = ff_add(D2, ff{b.x, b.y});
        }
        if (i < 0) {
            if (!(G2.hi > 1e-30f) || !(D2.hi > 1e-30f)) {
                alpha = 0.f; // x stays 0
                iters = 0;
                break;
            }
            alpha = G2.hi / D2.hi;
            beta = 0.f;
        } else {
            const float bnew = G2.hi / gam.hi;
            const float pap = D2.hi - bnew * G2.hi / alpha;
            if (!(G2.hi > 1e-30f) || !(pap > 1e-30f)) break;
            beta = bnew;
            alpha = G2.hi / pap;
        }
        gam = G2;
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int ln = ls + k * CT_NPB;
        if (ln >= n_own) continue;
        const int n = n_lo + ln;
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
    csync(); // no CTA leaves while others may still read its shared memory
}

template <int NPT>
cudaError_t launch_dsm(int ctas, int npc, const LevelGeom& g, const float* node, const float* rhs, const float* minv,
                       float* x, int iters, int interleaved, cudaStream_t st)
{
    const size_t smem = (size_t)npc * NODE_F * sizeof(float);
    if (ctas == 1) {
        auto one = k_pcg_dsm<NPT, true>;
        cudaError_t e = cudaFuncSetAttribute(one, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        one<<<1, CT, smem, st>>>(g, npc, node, rhs, minv, x, iters, interleaved);
        return cudaGetLastError();
    }
    auto kern = k_pcg_dsm<NPT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ctas > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, g, npc, node, rhs, minv, x, iters, interleaved);
}

template <int NPT>
cudaError_t launch_cluster(int blocks, const LevelGeom& g, const float* node, const float* rhs, const float* minv,
                           float* x, float* z, float* p0, float* p1, float2* part, unsigned long long* bar, int* status,
                           int iters, int interleaved, cudaStream_t st)
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
                        float* z, float* p0, float* p1, float2* part, unsigned long long* bar, int* status, int iters,
                        int interleaved, cudaStream_t st)
{
    LevelGeom gg = g;
    GridSync sy{0ull};
    void* args[] = {(void*)&gg, (void*)&node, (void*)&rhs, (void*)&minv, (void*)&x, (void*)&z, (void*)&p0,
                    (void*)&p1, (void*)&part, (void*)&bar, (void*)&status, (void*)&iters, (void*)&interleaved,
                    (void*)&sy};
    return cudaLaunchCooperativeKernel((const void*)k_pcg<NPT, GridSync>, dim3(blocks), dim3(PT), args, 0, st);
}

// ---------------------------------------------------------------------------
// PCG with one reduction per iteration (the Chronopoulos-Gear form: the same
// iterates as the textbook loop in exact arithmetic), over the whole GPU or
// one cluster, vectors in global memory. With u = M r and w = A u, the two
// dot products gamma = r.u and delta = w.u come from one fused reduction;
// every node publishes r, w and s = A p in one of two buffers (by iteration
// parity), and a neighbour's u_{i+1} = M (r_i - alpha (w_i + beta s_{i-1}))
// is formed on the fly from its published r_i, w_i and s_{i-1}. An iteration
// has one matrix-vector product and one barrier, against two for k_pcg.
// pub holds [2 parities][r, w, s][6][G].
// ---------------------------------------------------------------------------
template <class Sync>
__device__ __forceinline__ void allreduce2(float a, float b, ff* sh, float2* part, int parity, Sync& sy,
                                           unsigned long long* bar, int* status, bool& ok, ff& ra, ff& rb)
{
    // block sums of both values in one pass (FP32 within a warp, float-float
    // across warps, thread 0 in warp order); sh holds 2 * PT / 32 entries
    const int nb = gridDim.x;
    float2* pa = part + (size_t)parity * 2 * nb;
    float2* pb = pa + nb;
    const float wa = warp_sum(a), wb = warp_sum(b);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sh[2 * (threadIdx.x >> 5)] = ff_from(wa);
        sh[2 * (threadIdx.x >> 5) + 1] = ff_from(wb);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ff ta{0.f, 0.f}, tb{0.f, 0.f};
        for (int w = 0; w < PT / 32; ++w) {
            ta = ff_add(ta, sh[2 * w]);
            tb = ff_add(tb, sh[2 * w + 1]);
        }
        pa[blockIdx.x] = make_float2(ta.hi, ta.lo);
        pb[blockIdx.x] = make_float2(tb.hi, tb.lo);
    }
    ok = sy.sync(bar, status) && ok;
    // every warp forms the fixed-order sums itself: no broadcast through shared memory
    ra = ff_fixed_sum(pa, nb);
    rb = ff_fixed_sum(pb, nb);
}

// The same reduction over a cooperative grid, with the barrier folded into
// the data (the one-reduction kernels take it for every grid, whose plans are
// capped at TAG_MAXB blocks): block b publishes its two float-float partials as four 64-bit words
// (tag << 32 | value bits) in slot [tag & 1][b], and warp 0 of every block
// polls all blocks' words until each carries the reduction's tag, then folds
// them in the order of ff_fixed_sum (lane l takes blocks l, l + 32, ...), so
// the sums are bit-identical to allreduce2's. A block waits for the polled
// words instead of for a barrier counter and then the partials: one L2 round
// trip less per reduction, and no arrivals queued on one address. The release
// fence before the tagged stores and the acquire fence after the poll order
// the block's published vectors exactly as the barrier does. Two slots by
// tag parity suffice: a block writes tag k + 2 only after every block has
// published tag k + 1, which each does after it has read tag k. Slots are
// cleared (tag 0) before the launch's first barrier; tags start at 1. A poll
// gives up like grid_barrier: on an error in the status word (checked every
// 64 polls) or after ~1 s.
constexpr int TAG_MAXB = 160; // at most 5 blocks per polling lane (152 SMs, one block each)

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One-sided fences: fence.release before the relaxed tag stores makes them
// release stores, a relaxed poll followed by fence.acquire an acquire read
// (the PTX memory model's fence-based release and acquire patterns); cheaper
// than two full fence.acq_rel.
__device__ __forceinline__ void fence_release_gpu() { asm volatile("fence.release.gpu;" ::: "memory"); }

__device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acquire.gpu;" ::: "memory"); }

__device__ __forceinline__ unsigned long long tag_word(unsigned tag, float v)
{
    return ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v);
}

__device__ __forceinline__ void tagged_clear(unsigned long long* slots)
{
    if (threadIdx.x < 8) {
        const int par = threadIdx.x >> 2, w = threadIdx.x & 3;
        slots[((size_t)par * gridDim.x + blockIdx.x) * 4 + w] = 0ull;
    }
}

// Warp 0's half of a tagged reduction: polls the four words of every block
// in slot sl until each carries `tag` (lane l takes blocks l, l + 32, ...),
// then folds them in the order of ff_fixed_sum, so that every block forms the
// same bit-identical sums. Gives up like grid_barrier (status word every 64
// polls, ~1 s); returns 0 then. ok = 0 on entry skips the poll.
template <bool kFence>
__device__ __forceinline__ int warp_poll_fold(const unsigned long long* sl, int nb, unsigned tag, int* status,
                                              int lane, int ok, ff& va, ff& vb, long long limit = 2000000000LL)
{
    unsigned long long v[TAG_MAXB / 32][4];
    const long long t0 = clock64();
    for (unsigned k = 0; ok; ++k) {
        bool ready = true;
#pragma unroll
        for (int j = 0; j < TAG_MAXB / 32; ++j) {
            const int blk = lane + 32 * j;
            if (blk < nb) {
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    v[j][w] = ld_relaxed_u64(sl + (size_t)blk * 4 + w);
                    ready = ready && (unsigned)(v[j][w] >> 32) == tag;
                }
            }
        }
        if (__all_sync(0xffffffffu, ready)) break;
        if (((k + 1) & 63u) == 0u) {
            bool fail = false;
            if (lane == 0) {
                if (ld_acquire_s32(status) != 0) {
                    fail = true;
                } else if (clock64() - t0 > limit) {
                    atomicOr(status, DEV_TIMEOUT);
                    fail = true;
                }
            }
            if (__any_sync(0xffffffffu, fail)) {
                ok = 0;
                break;
            }
        }
    }
    if (kFence) fence_acquire_gpu(); // every block's published vectors after its tag
    va = ff{0.f, 0.f};
    vb = ff{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < TAG_MAXB / 32; ++j) {
        if (ok && lane + 32 * j < nb) {
            va = ff_add(va, ff{__uint_as_float((unsigned)v[j][0]), __uint_as_float((unsigned)v[j][1])});
            vb = ff_add(vb, ff{__uint_as_float((unsigned)v[j][2]), __uint_as_float((unsigned)v[j][3])});
        }
    }
    va = ff_warp_sum(va);
    vb = ff_warp_sum(vb);
    return ok;
}

struct NoSide {
    __device__ __forceinline__ bool operator()() const { return true; }
};

// kFence = false serves kernels whose published vectors carry their own tags
// (k_pcg1h): the partial words then order nothing but themselves. A thread
// passes fail = true when it gave up on a wait of its own; the block then
// publishes its partials and returns false without polling. While warp 0
// polls, warps 1.. run side() (k_pcg1h fetches its next halo there); a false
// from it makes the reduction return false too.
template <bool kFence = true, class Side = NoSide>
__device__ __forceinline__ bool allreduce2_tagged(float a, float b, ff* sh, unsigned long long* slots, unsigned tag,
                                                  int* status, ff& ra, ff& rb, bool fail = false,
                                                  Side side = Side{})
{
    __shared__ ff bc[2];
    __shared__ int ok_sh, fail_sh, side_fail_sh;
    const int nb = gridDim.x;
    unsigned long long* sl = slots + (size_t)(tag & 1u) * 4 * nb;
    const float wa = warp_sum(a), wb = warp_sum(b);
    if (!kFence && threadIdx.x == 0) fail_sh = side_fail_sh = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sh[2 * (threadIdx.x >> 5)] = ff_from(wa);
        sh[2 * (threadIdx.x >> 5) + 1] = ff_from(wb);
    }
    if (!kFence && fail) fail_sh = 1;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0) {
            ff ta{0.f, 0.f}, tb{0.f, 0.f};
            for (int w = 0; w < PT / 32; ++w) {
                ta = ff_add(ta, sh[2 * w]);
                tb = ff_add(tb, sh[2 * w + 1]);
            }
            if (kFence) fence_release_gpu(); // the block's published vectors before its tag
            unsigned long long* my = sl + (size_t)blockIdx.x * 4;
            st_relaxed_u64(my + 0, tag_word(tag, ta.hi));
            st_relaxed_u64(my + 1, tag_word(tag, ta.lo));
            st_relaxed_u64(my + 2, tag_word(tag, tb.hi));
            st_relaxed_u64(my + 3, tag_word(tag, tb.lo));
        }
        ff va, vb;
        int ok = (kFence || !fail_sh) ? 1 : 0;
        ok = warp_poll_fold<kFence>(sl, nb, tag, status, lane, ok, va, vb);
        if (lane == 0) {
            bc[0] = va;
            bc[1] = vb;
            ok_sh = ok;
        }
    } else if (!kFence && !fail_sh) {
        if (!side()) side_fail_sh = 1;
    }
    __syncthreads();
    ra = bc[0];
    rb = bc[1];
    return ok_sh != 0 && (kFence || side_fail_sh == 0);
}

template <int NPT, class Sync>
__global__ void __launch_bounds__(PT) k_pcg1(LevelGeom g, const float* __restrict__ node, const float* __restrict__ rhs,
                                             const float* __restrict__ minv, float* __restrict__ xout, float* pub,
                                             float2* part, unsigned long long* bar, int* status, int iters,
                                             int interleaved, Sync sy)
{
    __shared__ ff sred[2 * (PT / 32)];
    sy.start(bar);
    const int G = g.G, nx = g.nx, ny = g.ny;
    const size_t G6 = (size_t)6 * G;
    const int q4 = threadIdx.x & 3;
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
    const int stride = gridDim.x * NPB;
    const int slot0 = blockIdx.x * NPB + (threadIdx.x >> 2);
    float xr[NPT][2], rr[NPT][2], ur[NPT][2], wr[NPT][2], sr[NPT][2], pr[NPT][2], mr[NPT][2];
    int ni[NPT], nj[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
        nj[k] = n / nx;
        ni[k] = n - nj[k] * nx;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = h ? c1 : c0;
            const bool live = n < G && (h == 0 || has1);
            const float r0 = live ? rhs[c * G + n] : 0.f;
            mr[k][h] = live ? minv[c * G + n] : 0.f;
            rr[k][h] = r0;
            ur[k][h] = mr[k][h] * r0;
            xr[k][h] = wr[k][h] = sr[k][h] = pr[k][h] = 0.f;
            if (live) {
                pub[0 * G6 + c * G + n] = r0;  // r_0 in buffer 0
                pub[2 * G6 + c * G + n] = 0.f; // s_{-1} = 0
            }
        }
    }
    // a grid (at most TAG_MAXB blocks) reduces through tagged words in part
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(part);
    if constexpr (Sync::kGrid) tagged_clear(slots);
    bool ok = sy.sync(bar, status);
    float alpha = 0.f, beta = 0.f;
    ff gam{0.f, 0.f};
    int nred = 0;
    for (int i = -1; i < iters && ok; ++i) {
        // i = -1 is the set-up pass: w_0 = A u_0 and the first reduction
        const int par = i < 0 ? 0 : (i & 1);
        const int npar = i < 0 ? 0 : (par ^ 1);
        const float* R = pub + (size_t)par * 3 * G6;
        const float* Wv = R + G6;
        const float* S = R + 2 * G6;
        float* Rn = pub + (size_t)npar * 3 * G6;
        float* Wn = Rn + G6;
        float* Sn = Rn + 2 * G6;
        if (i >= 0) {
#pragma unroll
            for (int k = 0; k < NPT; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    pr[k][h] = fmaf(beta, pr[k][h], ur[k][h]);
                    sr[k][h] = fmaf(beta, sr[k][h], wr[k][h]);
                    xr[k][h] = fmaf(alpha, pr[k][h], xr[k][h]);
                    rr[k][h] = fmaf(-alpha, sr[k][h], rr[k][h]);
                    ur[k][h] = mr[k][h] * rr[k][h];
                }
            if (i == iters - 1) break;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int n = slot0 + k * stride;
                if (n >= G) continue;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!(h == 0 || has1)) continue;
                    const int c = h ? c1 : c0;
                    Rn[c * G + n] = rr[k][h];
                    Sn[c * G + n] = sr[k][h];
                }
            }
        }
        float gp = 0.f, dp = 0.f;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int n = slot0 + k * stride;
            const bool live = n < G;
            float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (live) {
                const int ii = ni[k], jj = nj[k];
#pragma unroll
                for (int ss = 0; ss < 3; ++ss) {
                    const int s = ss == 2 ? 8 : q4 + 4 * ss;
                    if (ss == 2 && q4 != 0) continue;
                    int owner, blk, pn;
                    if (!stencil_slot(s, ii, jj, nx, ny, n, owner, blk, pn)) continue;
                    float B[NB], u[6];
#pragma unroll
                    for (int e = 0; e < NB; ++e) B[e] = __ldg(node + (size_t)(blk * NB + e) * G + owner);
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const float mm = __ldg(minv + c * G + pn);
                        const float rv = __ldcg(R + c * G + pn);
                        if (i >= 0) {
                            const float wv = __ldcg(Wv + c * G + pn), sv = __ldcg(S + c * G + pn);
                            u[c] = mm * fmaf(-alpha, fmaf(beta, sv, wv), rv);
                        } else {
                            u[c] = mm * rv;
                        }
                    }
                    sym_matvec_acc(B, u, q);
                }
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                q[c] += __shfl_xor_sync(0xffffffffu, q[c], 1);
                q[c] += __shfl_xor_sync(0xffffffffu, q[c], 2);
            }
            if (live) {
                wr[k][0] = sel6(q, c0);
                wr[k][1] = has1 ? sel6(q, c1) : 0.f;
                Wn[c0 * G + n] = wr[k][0];
                if (has1) Wn[c1 * G + n] = wr[k][1];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    gp = fmaf(rr[k][h], ur[k][h], gp);
                    dp = fmaf(wr[k][h], ur[k][h], dp);
                }
            }
        }
        ff G2, D2;
        if constexpr (Sync::kGrid)
            ok = allreduce2_tagged(gp, dp, sred, slots, (unsigned)nred + 1u, status, G2, D2) && ok;
        else
            allreduce2(gp, dp, sred, part, nred & 1, sy, bar, status, ok, G2, D2);
        ++nred;
        if (!ok) break;
        if (i < 0) {
            if (!(G2.hi > 1e-30f) || !(D2.hi > 1e-30f)) break; // x stays 0
            alpha = G2.hi / D2.hi;
            beta = 0.f;
        } else {
            const float bnew = G2.hi / gam.hi;
            const float pap = D2.hi - bnew * G2.hi / alpha;
            if (!(G2.hi > 1e-30f) || !(pap > 1e-30f)) break;
            beta = bnew;
            alpha = G2.hi / pap;
        }
        gam = G2;
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
cudaError_t launch_grid1(int blocks, const LevelGeom& g, const float* node, const float* rhs, const float* minv,
                         float* x, float* pub, float2* part, unsigned long long* bar, int* status, int iters,
                         int interleaved, cudaStream_t st)
{
    if (blocks < 1 || blocks > TAG_MAXB) return cudaErrorInvalidValue; // the tagged reduction polls TAG_MAXB slots
    LevelGeom gg = g;
    GridSync sy{0ull};
    void* args[] = {(void*)&gg, (void*)&node, (void*)&rhs, (void*)&minv, (void*)&x, (void*)&pub, (void*)&part,
                    (void*)&bar, (void*)&status, (void*)&iters, (void*)&interleaved, (void*)&sy};
    return cudaLaunchCooperativeKernel((const void*)k_pcg1<NPT, GridSync>, dim3(blocks), dim3(PT), args, 0, st);
}

template <int NPT>
cudaError_t launch_cluster1(int blocks, const LevelGeom& g, const float* node, const float* rhs, const float* minv,
                            float* x, float* pub, float2* part, unsigned long long* bar, int* status, int iters,
                            int interleaved, cudaStream_t st)
{
    auto kern = k_pcg1<NPT, ClusterSync>;
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
    return cudaLaunchKernelEx(&cfg, kern, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved,
                              ClusterSync{});
}

// ---------------------------------------------------------------------------
// The one-reduction grid PCG with self-validating published vectors and its
// operands in shared memory (plan kind 5). The same iterates as k_pcg1, bit
// for bit: the arithmetic is the same, only where the operands come from and
// how the blocks exchange them differ.
//
// Self-tagged words. Every published value of r, w and s is one 64-bit word,
// (tag << 32) | value bits, written with a single relaxed store, so each value
// carries its own proof of freshness: a reader checks the tag of every word
// and reads again while a word is stale. Nothing has to order the vectors
// before the partial sums, so the exchange needs no memory fence.
//
// Registers and shared memory. A block owns NPT segments of NPB consecutive
// nodes (segment k starts at n0_k); the stencil of its nodes reaches
// hw = nx + 1 nodes to either side. The coupling blocks do not change during
// the solve: with one node per four-lane group (NPT = 1) each lane loads its
// slots' blocks into registers once (SlotRegs); with more, the block copies
// the blocks of its nodes and of the hw nodes before each segment into shared
// memory at the start, coalesced. Either way the matrix-vector product reads
// no global memory. Per iteration it forms u = M (r - alpha (w + beta s)) once
// per node of [n0_k - hw, n0_k + NPB + hw) in shared memory: owned nodes from
// the owners' registers (the same rounding), the 2 hw nodes on either side
// from their published words, read coalesced. While warp 0 polls the other
// blocks' partial sums, warps 1.. fetch the next iteration's halo words and
// wait until they carry the expected tag, so the halo's L2 round trip and the
// wait for late neighbours overlap the poll; entries beyond their share are
// read by the whole block after the poll.
//
// Tags: r_0 and s_{-1} (written before the launch's one full barrier) and
// the set-up pass's w_0 carry tag 1 in buffer 0; iteration i >= 0 reads
// buffer i & 1 expecting tag i + 1 and publishes r_{i+1}, s_i and w_{i+1}
// into buffer (i + 1) & 1 with tag i + 2. Before the barrier each node clears
// (tag 0) the words that a reader checks before this launch rewrites them:
// buffer 0's w and all of buffer 1. So no word left by an earlier launch, or
// by another kernel sharing the buffer, can pass a check. A word of tag i + 1
// is overwritten (with tag i + 3) only by an owner that has seen every
// block's partial sums of iteration i, which each block forms after reading
// the values of iteration i: a reader never loses a value it still needs.
// pubw holds [2 parities][r, w, s][6][G] words; the dynamic shared memory
// (NPT > 1) [NPT][NODE_VALS][ls] floats of blocks (ls >= NPB + hw, padded so
// that the four block rows a warp reads at once start in different banks),
// then [NPT][6][NPB + 2 hw] floats of u (NPT = 1: the u array alone).
// ---------------------------------------------------------------------------
constexpr int HPF = 5;       // halo entries per thread and round
constexpr int HFT = PT - 32; // threads that fetch the halo during the poll (warps 1..)

__device__ __forceinline__ unsigned word_tag(unsigned long long w) { return (unsigned)(w >> 32); }

__device__ __forceinline__ float word_val(unsigned long long w) { return __uint_as_float((unsigned)w); }

__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) { return __ldcg(p); }

struct Halo {
    int G, hw, hn, items; // nodes, nodes on each side (nx + 1), u span (NPB + 2 hw), entries NPT * 12 hw
};

// Entry f of the halo (segment, component, side, offset): the word offset
// c * G + m of node m, component c, and its index in the u array; -1 if f
// lies outside the halo or the level.
template <int NPT>
__device__ __forceinline__ int halo_entry(const Halo& h, int f, int stride, int& si)
{
    if (f >= h.items) return -1;
    const int per_k = 12 * h.hw;
    const int k = f / per_k;
    const int rem = f - k * per_k;
    const int c = rem / (2 * h.hw);
    const int r2 = rem - c * 2 * h.hw;
    const int off = r2 < h.hw ? r2 : r2 + NPB; // left side, or right of the owned segment
    const int m = blockIdx.x * NPB + k * stride - h.hw + off;
    if (m < 0 || m >= h.G) return -1;
    si = (k * 6 + c) * h.hn + off;
    return c * h.G + m;
}

// Entries f0 + j * step of the halo (indices only).
template <int NPT>
__device__ __forceinline__ void halo_index(const Halo& h, int f0, int step, int stride, int (&gi)[HPF],
                                           int (&si)[HPF])
{
#pragma unroll
    for (int j = 0; j < HPF; ++j) gi[j] = halo_entry<NPT>(h, f0 + j * step, stride, si[j]);
}

// Issues the loads of a round's entries (plain L2 loads, which the compiler
// may batch); SETUP reads one word per entry (r, or w in k_pcg1p), else r, w, s.
template <bool SETUP>
__device__ __forceinline__ void halo_load(const unsigned long long* R, size_t G6, const int (&gi)[HPF],
                                          unsigned long long (&v)[HPF][3])
{
#pragma unroll
    for (int j = 0; j < HPF; ++j) {
        if (gi[j] >= 0) {
            v[j][0] = ld_cg_u64(R + gi[j]);
            if (!SETUP) {
                v[j][1] = ld_cg_u64(R + G6 + gi[j]);
                v[j][2] = ld_cg_u64(R + 2 * G6 + gi[j]);
            }
        }
    }
}

template <int NPT, bool SETUP>
__device__ __forceinline__ void halo_issue(const Halo& h, const unsigned long long* R, size_t G6, int f0, int step,
                                           int stride, int (&gi)[HPF], int (&si)[HPF],
                                           unsigned long long (&v)[HPF][3])
{
    halo_index<NPT>(h, f0, step, stride, gi, si);
    halo_load<SETUP>(R, G6, gi, v);
}

// Reads the stale words of a round again, all together (relaxed loads),
// until every word carries `tag`; gives up like the tagged poll (status word
// every 64 passes, ~1 s). False on giving up.
template <bool SETUP>
__device__ __forceinline__ bool halo_wait(const unsigned long long* R, size_t G6, unsigned tag, int* status,
                                          const int (&gi)[HPF], unsigned long long (&v)[HPF][3],
                                          long long limit = 2000000000LL)
{
    auto fresh = [&](int j) {
        return word_tag(v[j][0]) == tag && (SETUP || (word_tag(v[j][1]) == tag && word_tag(v[j][2]) == tag));
    };
    unsigned stale = 0;
#pragma unroll
    for (int j = 0; j < HPF; ++j)
        if (gi[j] >= 0 && !fresh(j)) stale |= 1u << j;
    long long t0 = 0;
    for (unsigned k = 0; stale != 0u; ++k) {
        if (k == 0) t0 = clock64();
#pragma unroll
        for (int j = 0; j < HPF; ++j)
            if ((stale >> j) & 1u) {
                v[j][0] = ld_relaxed_u64(R + gi[j]);
                if (!SETUP) {
                    v[j][1] = ld_relaxed_u64(R + G6 + gi[j]);
                    v[j][2] = ld_relaxed_u64(R + 2 * G6 + gi[j]);
                }
            }
        unsigned left = 0;
#pragma unroll
        for (int j = 0; j < HPF; ++j)
            if (((stale >> j) & 1u) && !fresh(j)) left |= 1u << j;
        stale = left;
        if (stale != 0u && ((k + 1) & 63u) == 0u) {
            if (ld_acquire_s32(status) != 0) return false;
            if (clock64() - t0 > limit) {
                atomicOr(status, DEV_TIMEOUT);
                return false;
            }
        }
    }
    return true;
}

// u of every entry of a round, into the u array.
template <bool SETUP>
__device__ __forceinline__ void halo_u(const float* __restrict__ minv, float alpha, float beta, float* uh,
                                       const int (&gi)[HPF], const int (&si)[HPF],
                                       const unsigned long long (&v)[HPF][3])
{
#pragma unroll
    for (int j = 0; j < HPF; ++j) {
        if (gi[j] < 0) continue;
        const float mm = __ldg(minv + gi[j]);
        uh[si[j]] = SETUP ? mm * word_val(v[j][0])
                          : mm * fmaf(-alpha, fmaf(beta, word_val(v[j][2]), word_val(v[j][1])), word_val(v[j][0]));
    }
}

// With one node per four-lane group the coupling blocks of a lane's stencil
// slots stay in registers for the whole solve (loaded once from global
// memory) instead of being staged in shared memory: lane q holds slots q and
// q + 4, lane 0 also slot 8. A slot outside the level holds zeros and points
// at the node itself, so the product runs without branches.
struct SlotRegs {
    float B[3][NB];
    int pn[3]; // neighbour node of each slot
    __device__ __forceinline__ void load(const float* __restrict__ node, int G, int nx, int ny, int n, int i, int j,
                                         int q4)
    {
#pragma unroll
        for (int ss = 0; ss < 3; ++ss) {
            const int s = ss == 2 ? 8 : q4 + 4 * ss;
            int owner = n, blk = 0, p = n;
            const bool on = n < G && !(ss == 2 && q4 != 0) && stencil_slot(s, i, j, nx, ny, n, owner, blk, p);
            pn[ss] = on ? p : n; // an absent slot (zero block) reads the node itself
#pragma unroll
            for (int e = 0; e < NB; ++e) B[ss][e] = on ? __ldg(node + (size_t)(blk * NB + e) * G + owner) : 0.f;
        }
    }
    // q += A_slots u, u read from the u array at ubase + c * hn + pn
    __device__ __forceinline__ void apply(const float* uh, int ubase, int hn, float* q) const
    {
#pragma unroll
        for (int ss = 0; ss < 3; ++ss) {
            float u[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) u[c] = uh[ubase + c * hn + pn[ss]];
            sym_matvec_acc(B[ss], u, q);
        }
    }
};

template <int NPT>
__global__ void __launch_bounds__(PT, 1) k_pcg1h(LevelGeom g, const float* __restrict__ node,
                                                 const float* __restrict__ rhs, const float* __restrict__ minv,
                                                 float* __restrict__ xout, unsigned long long* pubw, float2* part,
                                                 unsigned long long* bar, int* status, int iters, int interleaved,
                                                 int ls)
{
    extern __shared__ float smem_h[];
    __shared__ ff sred[2 * (PT / 32)];
    GridSync sy{0ull};
    sy.start(bar);
    const int G = g.G, nx = g.nx, ny = g.ny;
    const size_t G6 = (size_t)6 * G;
    const int q4 = threadIdx.x & 3;
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
    const int stride = gridDim.x * NPB;
    const int slot0 = blockIdx.x * NPB + (threadIdx.x >> 2);
    Halo hl;
    hl.G = G;
    hl.hw = nx + 1;
    hl.hn = NPB + 2 * hl.hw;
    hl.items = NPT * 12 * hl.hw;
    float* sB = smem_h; // [NPT][NODE_VALS][ls] (NPT > 1)
    float* uh = smem_h + (NPT == 1 ? 0 : (size_t)NPT * NODE_VALS * ls); // [NPT][6][hn]
    float xr[NPT][2], rr[NPT][2], ur[NPT][2], wr[NPT][2], sr[NPT][2], pr[NPT][2], mr[NPT][2];
    int ni[NPT], nj[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
        nj[k] = n / nx;
        ni[k] = n - nj[k] * nx;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = h ? c1 : c0;
            const bool live = n < G && (h == 0 || has1);
            const float r0 = live ? rhs[c * G + n] : 0.f;
            mr[k][h] = live ? minv[c * G + n] : 0.f;
            rr[k][h] = r0;
            ur[k][h] = mr[k][h] * r0;
            xr[k][h] = wr[k][h] = sr[k][h] = pr[k][h] = 0.f;
            if (live) {
                const size_t o = (size_t)c * G + n;
                pubw[0 * G6 + o] = tag_word(1u, r0);  // r_0, buffer 0
                pubw[1 * G6 + o] = 0ull;              // buffer 0's w: cleared
                pubw[2 * G6 + o] = tag_word(1u, 0.f); // s_{-1} = 0
                pubw[3 * G6 + o] = 0ull;              // buffer 1: cleared
                pubw[4 * G6 + o] = 0ull;
                pubw[5 * G6 + o] = 0ull;
            }
        }
    }
    // the coupling blocks: in registers with one node per group, else those of
    // the segments' nodes and of the hw nodes before them in shared memory
    SlotRegs sr1;
    if constexpr (NPT == 1) {
        sr1.load(node, G, nx, ny, slot0, ni[0], nj[0], q4);
    } else {
        const int span = hl.hw + NPB;
#pragma unroll 1
        for (int k = 0; k < NPT; ++k) {
            const int mlo = blockIdx.x * NPB + k * stride - hl.hw;
            float* dst = sB + (size_t)k * NODE_VALS * ls;
#pragma unroll 4
            for (int idx = threadIdx.x; idx < NODE_VALS * span; idx += PT) {
                const int row = idx / span;
                const int l = idx - row * span;
                const int m = mlo + l;
                dst[row * ls + l] = (m >= 0 && m < G) ? __ldg(node + (size_t)row * G + m) : 0.f;
            }
        }
    }
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(part);
    tagged_clear(slots);
    bool ok = sy.sync(bar, status); // the launch's one full barrier: clears, r_0 and the staged blocks
    float alpha = 0.f, beta = 0.f;
    ff gam{0.f, 0.f};
    int nred = 0;
    int gi[HPF], si[HPF], gf[HPF], sf[HPF];
    unsigned long long hv[HPF][3];
    const int fetcher = (int)threadIdx.x - 32; // warps 1.. fetch the first HFT * HPF entries
    if (fetcher >= 0) {
        halo_index<NPT>(hl, fetcher, HFT, stride, gf, sf); // the same entries every iteration
        halo_load<true>(pubw, G6, gf, hv);
        ok = halo_wait<true>(pubw, G6, 1u, status, gf, hv) && ok; // r_0 is there since the barrier
    }
    ok = __syncthreads_and(ok);
    for (int i = -1; i < iters && ok; ++i) {
        const int par = i < 0 ? 0 : (i & 1);
        const int npar = i < 0 ? 0 : (par ^ 1);
        const unsigned rtag = i < 0 ? 1u : (unsigned)i + 1u;
        const unsigned wtag = i < 0 ? 1u : (unsigned)i + 2u;
        const unsigned long long* R = pubw + (size_t)par * 3 * G6;
        unsigned long long* Rn = pubw + (size_t)npar * 3 * G6;
        if (i >= 0) {
#pragma unroll
            for (int k = 0; k < NPT; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    pr[k][h] = fmaf(beta, pr[k][h], ur[k][h]);
                    sr[k][h] = fmaf(beta, sr[k][h], wr[k][h]);
                    xr[k][h] = fmaf(alpha, pr[k][h], xr[k][h]);
                    rr[k][h] = fmaf(-alpha, sr[k][h], rr[k][h]);
                    ur[k][h] = mr[k][h] * rr[k][h];
                }
            if (i == iters - 1) break;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int n = slot0 + k * stride;
                if (n >= G) continue;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!(h == 0 || has1)) continue;
                    const size_t o = (size_t)(h ? c1 : c0) * G + n;
                    st_relaxed_u64(Rn + o, tag_word(wtag, rr[k][h]));
                    st_relaxed_u64(Rn + 2 * G6 + o, tag_word(wtag, sr[k][h]));
                }
            }
        }
        // u of the owned nodes from registers, of the halo from the fetched words
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int n = slot0 + k * stride;
            if (n >= G) continue;
            const int own = (k * 6) * hl.hn + hl.hw + (n - (blockIdx.x * NPB + k * stride));
            uh[own + c0 * hl.hn] = ur[k][0];
            if (has1) uh[own + c1 * hl.hn] = ur[k][1];
        }
        bool fail = false;
        if (fetcher >= 0) {
            if (i < 0)
                halo_u<true>(minv, alpha, beta, uh, gf, sf, hv);
            else
                halo_u<false>(minv, alpha, beta, uh, gf, sf, hv);
        }
        for (int base = HFT * HPF; base < hl.items; base += PT * HPF) {
            if (i < 0) {
                halo_issue<NPT, true>(hl, R, G6, base + (int)threadIdx.x, PT, stride, gi, si, hv);
                fail = !halo_wait<true>(R, G6, rtag, status, gi, hv) || fail;
                halo_u<true>(minv, alpha, beta, uh, gi, si, hv);
            } else {
                halo_issue<NPT, false>(hl, R, G6, base + (int)threadIdx.x, PT, stride, gi, si, hv);
                fail = !halo_wait<false>(R, G6, rtag, status, gi, hv) || fail;
                halo_u<false>(minv, alpha, beta, uh, gi, si, hv);
            }
        }
        __syncthreads();
        float gp = 0.f, dp = 0.f;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int n = slot0 + k * stride;
            const bool live = n < G;
            const int n0 = blockIdx.x * NPB + k * stride;
            const int ubase = (k * 6) * hl.hn + hl.hw - n0;
            float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if constexpr (NPT == 1) {
                sr1.apply(uh, ubase, hl.hn, q);
            } else if (live) {
                const int ii = ni[k], jj = nj[k];
#pragma unroll
                for (int ss = 0; ss < 3; ++ss) {
                    const int s = ss == 2 ? 8 : q4 + 4 * ss;
                    if (ss == 2 && q4 != 0) continue;
                    int owner, blk, pn;
                    if (!stencil_slot(s, ii, jj, nx, ny, n, owner, blk, pn)) continue;
                    const float* Bs = sB + (size_t)(k * NODE_VALS + blk * NB) * ls + (owner - n0 + hl.hw);
                    float B[NB], u[6];
#pragma unroll
                    for (int e = 0; e < NB; ++e) B[e] = Bs[e * ls];
#pragma unroll
                    for (int c = 0; c < 6; ++c) u[c] = uh[ubase + c * hl.hn + pn];
                    sym_matvec_acc(B, u, q);
                }
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                q[c] += __shfl_xor_sync(0xffffffffu, q[c], 1);
                q[c] += __shfl_xor_sync(0xffffffffu, q[c], 2);
            }
            if (live) {
                wr[k][0] = sel6(q, c0);
                wr[k][1] = has1 ? sel6(q, c1) : 0.f;
                st_relaxed_u64(Rn + G6 + (size_t)c0 * G + n, tag_word(wtag, wr[k][0]));
                if (has1) st_relaxed_u64(Rn + G6 + (size_t)c1 * G + n, tag_word(wtag, wr[k][1]));
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    gp = fmaf(rr[k][h], ur[k][h], gp);
                    dp = fmaf(wr[k][h], ur[k][h], dp);
                }
            }
        }
        // while warp 0 polls, warps 1.. fetch the next iteration's halo (which
        // iteration i + 1 forms only if it is not the last)
        const bool next = i + 2 < iters;
        auto fetch = [&]() -> bool {
            if (!next) return true;
            halo_load<false>(Rn, G6, gf, hv);
            return halo_wait<false>(Rn, G6, wtag, status, gf, hv);
        };
        ff G2, D2;
        ok = allreduce2_tagged<false>(gp, dp, sred, slots, (unsigned)nred + 1u, status, G2, D2, fail, fetch) && ok;
        ++nred;
        if (!ok) break;
        if (i < 0) {
            if (!(G2.hi > 1e-30f) || !(D2.hi > 1e-30f)) break; // x stays 0
            alpha = G2.hi / D2.hi;
            beta = 0.f;
        } else {
            const float bnew = G2.hi / gam.hi;
            const float pap = D2.hi - bnew * G2.hi / alpha;
            if (!(G2.hi > 1e-30f) || !(pap > 1e-30f)) break;
            beta = bnew;
            alpha = G2.hi / pap;
        }
        gam = G2;
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

// Row stride of the staged blocks: at least NPB + hw, and = 8 (mod 32), so
// that block rows b * NB apart start 8 banks apart.
int halo_ls(int nx)
{
    const int span = NPB + nx + 1;
    return span + ((8 - span % 32) + 32) % 32;
}

// Dynamic shared memory of k_pcg1h / k_pcg1p: the u array, and with more
// than one node per group the staged blocks before it.
size_t halo_smem(int npt, int nx)
{
    const size_t staged = npt == 1 ? 0 : (size_t)npt * NODE_VALS * halo_ls(nx);
    return (staged + (size_t)npt * 6 * (NPB + 2 * (nx + 1))) * sizeof(float);
}

template <int NPT>
cudaError_t launch_grid1h(int blocks, const LevelGeom& g, const float* node, const float* rhs, const float* minv,
                          float* x, float* pub, float2* part, unsigned long long* bar, int* status, int iters,
                          int interleaved, cudaStream_t st)
{
    if (blocks < 1 || blocks > TAG_MAXB) return cudaErrorInvalidValue; // the tagged reduction polls TAG_MAXB slots
    if ((uintptr_t)pub & 7) return cudaErrorInvalidValue;               // 64-bit words
    const size_t smem = halo_smem(NPT, g.nx);
    cudaError_t e = cudaFuncSetAttribute((const void*)k_pcg1h<NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    LevelGeom gg = g;
    int ls = halo_ls(g.nx);
    unsigned long long* pubw = reinterpret_cast<unsigned long long*>(pub);
    void* args[] = {(void*)&gg,  (void*)&node,   (void*)&rhs,   (void*)&minv,        (void*)&x,  (void*)&pubw,
                    (void*)&part, (void*)&bar,   (void*)&status, (void*)&iters, (void*)&interleaved, (void*)&ls};
    return cudaLaunchCooperativeKernel((const void*)k_pcg1h<NPT>, dim3(blocks), dim3(PT), args, smem, st);
}

// ---------------------------------------------------------------------------
// Pipelined PCG over the grid (plan kind 6): the reduction's latency hidden
// behind the matrix-vector product. This is the pipelined form of PCG of
// Ghysels and Vanroose ("Hiding global synchronization latency in the
// preconditioned Conjugate Gradient algorithm", Parallel Computing 40, 2014):
// with u = M r, w = A u, m = M w and n = A m, one iteration takes
//   gamma = r.u, delta = w.u            (one fused reduction, started)
//   m = M w, n = A m                    (while the reduction completes)
//   beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
//   z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p
//   x += alpha p, r -= alpha s, u = M r, w -= alpha z
// and keeps s = A p, q = M s, z = A q and w = A u by recurrence: the
// iterates of the textbook loop in exact arithmetic, rounded differently.
// The paper of Ghysels and Vanroose also recurs u -= alpha q; forming
// u = M r from the recurred r instead (M is diagonal, so it costs nothing)
// keeps gamma = r.u consistent with r, and measured it halves the drift from
// the textbook loop on an ill-conditioned system (final energy 4.7e-5 from
// the FP64 oracle's against 1.1e-4 with the recurrence, 5.9e-5 for k_pcg1h).
// Its fields still drift further: on a 640x480 frame with the occlusion and
// illumination maps they end 1.8e-3 px from the oracle's (k_pcg1h: 7e-4), so
// it is the opt-in SF_PCG_PIPELINED, not the default. The product needs
// only the neighbours' w, published once per iteration as self-tagged words
// (as in k_pcg1h); the coupling blocks sit in registers or shared memory as there.
// A block publishes its partial sums, forms m over its nodes and halo
// (waiting for late neighbours' w), runs the product, and only then polls the
// other blocks' partials, which have had the product's duration to arrive.
//
// Words: w_i in buffer i & 1 with tag i + 1 (w_0 from the set-up product
// A M r_0), r_0 with tag 1 in a third buffer for the set-up; both w buffers
// are cleared before the launch's one full barrier. w_{i+2} overwrites w_i
// only after its owner has seen every block's partial sums of iteration
// i + 1, which each block forms from values computed with the w_i it read.
// pubw holds [w buffer 0][w buffer 1][r_0], each [6][G] words.
// ---------------------------------------------------------------------------

// A block's partial sums of a and b (float-float, warps in order, as
// allreduce2_tagged), published by thread 0 as four tagged words.
__device__ __forceinline__ void tagged_publish(float a, float b, ff* sh, unsigned long long* slots, unsigned tag)
{
    const int nb = gridDim.x;
    unsigned long long* sl = slots + (size_t)(tag & 1u) * 4 * nb;
    const float wa = warp_sum(a), wb = warp_sum(b);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sh[2 * (threadIdx.x >> 5)] = ff_from(wa);
        sh[2 * (threadIdx.x >> 5) + 1] = ff_from(wb);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ff ta{0.f, 0.f}, tb{0.f, 0.f};
        for (int w = 0; w < PT / 32; ++w) {
            ta = ff_add(ta, sh[2 * w]);
            tb = ff_add(tb, sh[2 * w + 1]);
        }
        unsigned long long* my = sl + (size_t)blockIdx.x * 4;
        st_relaxed_u64(my + 0, tag_word(tag, ta.hi));
        st_relaxed_u64(my + 1, tag_word(tag, ta.lo));
        st_relaxed_u64(my + 2, tag_word(tag, tb.hi));
        st_relaxed_u64(my + 3, tag_word(tag, tb.lo));
    }
}

// The other half: warp 0 polls and folds every block's words of `tag`; the
// sums reach every thread through shared memory (one CTA barrier).
__device__ __forceinline__ bool tagged_collect(const unsigned long long* slots, unsigned tag, int* status, ff& ra,
                                               ff& rb)
{
    __shared__ ff bcc[2];
    __shared__ int okc;
    if (threadIdx.x < 32) {
        const int nb = gridDim.x;
        ff va, vb;
        const int ok = warp_poll_fold<false>(slots + (size_t)(tag & 1u) * 4 * nb, nb, tag, status, threadIdx.x, 1,
                                             va, vb);
        if (threadIdx.x == 0) {
            bcc[0] = va;
            bcc[1] = vb;
            okc = ok;
        }
    }
    __syncthreads();
    ra = bcc[0];
    rb = bcc[1];
    return okc != 0;
}

// out = A v over the block's nodes, v from the u array (owned nodes and
// halo), the coupling blocks from the staged copy.
template <int NPT>
__device__ __forceinline__ void smem_apply(const float* sB, const SlotRegs& sr1, const float* uh, int ls,
                                           const Halo& hl, int nx, int ny, int slot0, int stride, int q4,
                                           const int (&ni)[NPT], const int (&nj)[NPT], float (&out)[NPT][2])
{
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
        const bool live = n < hl.G;
        const int n0 = blockIdx.x * NPB + k * stride;
        const int ubase = (k * 6) * hl.hn + hl.hw - n0;
        float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if constexpr (NPT == 1) {
            sr1.apply(uh, ubase, hl.hn, q);
        } else if (live) {
#pragma unroll
            for (int ss = 0; ss < 3; ++ss) {
                const int s = ss == 2 ? 8 : q4 + 4 * ss;
                if (ss == 2 && q4 != 0) continue;
                int owner, blk, pn;
                if (!stencil_slot(s, ni[k], nj[k], nx, ny, n, owner, blk, pn)) continue;
                const float* Bs = sB + (size_t)(k * NODE_VALS + blk * NB) * ls + (owner - n0 + hl.hw);
                float B[NB], u[6];
#pragma unroll
                for (int e = 0; e < NB; ++e) B[e] = Bs[e * ls];
#pragma unroll
                for (int c = 0; c < 6; ++c) u[c] = uh[ubase + c * hl.hn + pn];
                sym_matvec_acc(B, u, q);
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            q[c] += __shfl_xor_sync(0xffffffffu, q[c], 1);
            q[c] += __shfl_xor_sync(0xffffffffu, q[c], 2);
        }
        out[k][0] = live ? sel6(q, c0) : 0.f;
        out[k][1] = (live && has1) ? sel6(q, c1) : 0.f;
    }
}

// Fills the u array with M v: owned nodes from own[][] (already M v), the
// halo from the words of V carrying `tag`; entries of the first round use
// the fixed indices g0/s0 (loads already issued into hv when `issued`).
template <int NPT>
__device__ __forceinline__ bool smem_fill(const Halo& hl, const unsigned long long* V, size_t G6,
                                          const float* __restrict__ minv, unsigned tag, int* status, float* uh,
                                          int slot0, int stride, int q4, const float (&own)[NPT][2],
                                          const int (&g0)[HPF], const int (&s0)[HPF], bool issued,
                                          unsigned long long (&hv)[HPF][3])
{
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
        if (n >= hl.G) continue;
        const int o = (k * 6) * hl.hn + hl.hw + (n - (blockIdx.x * NPB + k * stride));
        uh[o + c0 * hl.hn] = own[k][0];
        if (has1) uh[o + c1 * hl.hn] = own[k][1];
    }
    if (!issued) halo_load<true>(V, G6, g0, hv);
    bool ok = halo_wait<true>(V, G6, tag, status, g0, hv);
    halo_u<true>(minv, 0.f, 0.f, uh, g0, s0, hv);
    for (int base = PT * HPF; base < hl.items; base += PT * HPF) {
        int gi[HPF], si[HPF];
        halo_issue<NPT, true>(hl, V, G6, base + (int)threadIdx.x, PT, stride, gi, si, hv);
        ok = halo_wait<true>(V, G6, tag, status, gi, hv) && ok;
        halo_u<true>(minv, 0.f, 0.f, uh, gi, si, hv);
    }
    return ok;
}

template <int NPT>
__global__ void __launch_bounds__(PT, 1) k_pcg1p(LevelGeom g, const float* __restrict__ node,
                                                 const float* __restrict__ rhs, const float* __restrict__ minv,
                                                 float* __restrict__ xout, unsigned long long* pubw, float2* part,
                                                 unsigned long long* bar, int* status, int iters, int interleaved,
                                                 int ls)
{
    extern __shared__ float smem_h[];
    __shared__ ff sred[2 * (PT / 32)];
    GridSync sy{0ull};
    sy.start(bar);
    const int G = g.G, nx = g.nx, ny = g.ny;
    const size_t G6 = (size_t)6 * G;
    const int q4 = threadIdx.x & 3;
    const int c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
    const int stride = gridDim.x * NPB;
    const int slot0 = blockIdx.x * NPB + (threadIdx.x >> 2);
    Halo hl;
    hl.G = G;
    hl.hw = nx + 1;
    hl.hn = NPB + 2 * hl.hw;
    hl.items = NPT * 12 * hl.hw;
    float* sB = smem_h; // [NPT][NODE_VALS][ls] (NPT > 1)
    float* uh = smem_h + (NPT == 1 ? 0 : (size_t)NPT * NODE_VALS * ls);
    const unsigned long long* R0 = pubw + 2 * G6; // w buffer b at pubw + b * G6
    float xr[NPT][2], rr[NPT][2], ur[NPT][2], wr[NPT][2], zr[NPT][2], qr[NPT][2], sr[NPT][2], pr[NPT][2],
        mr[NPT][2], nr[NPT][2], mw[NPT][2];
    int ni[NPT], nj[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = slot0 + k * stride;
        nj[k] = n / nx;
        ni[k] = n - nj[k] * nx;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = h ? c1 : c0;
            const bool live = n < G && (h == 0 || has1);
            const float r0 = live ? rhs[c * G + n] : 0.f;
            mr[k][h] = live ? minv[c * G + n] : 0.f;
            rr[k][h] = r0;
            ur[k][h] = mr[k][h] * r0;
            xr[k][h] = wr[k][h] = zr[k][h] = qr[k][h] = sr[k][h] = pr[k][h] = nr[k][h] = mw[k][h] = 0.f;
            if (live) {
                const size_t o = (size_t)c * G + n;
                pubw[o] = 0ull;                          // w buffers: cleared
                pubw[G6 + o] = 0ull;
                pubw[2 * G6 + o] = tag_word(1u, r0);     // r_0
            }
        }
    }
    SlotRegs sr1;
    if constexpr (NPT == 1) {
        sr1.load(node, G, nx, ny, slot0, ni[0], nj[0], q4);
    } else {
        const int span = hl.hw + NPB;
#pragma unroll 1
        for (int k = 0; k < NPT; ++k) {
            const int mlo = blockIdx.x * NPB + k * stride - hl.hw;
            float* dst = sB + (size_t)k * NODE_VALS * ls;
#pragma unroll 4
            for (int idx = threadIdx.x; idx < NODE_VALS * span; idx += PT) {
                const int row = idx / span;
                const int l = idx - row * span;
                const int m = mlo + l;
                dst[row * ls + l] = (m >= 0 && m < G) ? __ldg(node + (size_t)row * G + m) : 0.f;
            }
        }
    }
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(part);
    tagged_clear(slots);
    bool ok = sy.sync(bar, status); // the launch's one full barrier: clears, r_0 and the staged blocks
    int g0[HPF], s0[HPF];
    unsigned long long hv[HPF][3];
    halo_index<NPT>(hl, (int)threadIdx.x, PT, stride, g0, s0); // the first round's entries, fixed
    // set-up: w_0 = A M r_0
    if (ok) {
        const bool fail = !smem_fill<NPT>(hl, R0, G6, minv, 1u, status, uh, slot0, stride, q4, ur, g0, s0, false, hv);
        ok = !__syncthreads_or(fail);
    }
    if (ok) {
        smem_apply<NPT>(sB, sr1, uh, ls, hl, nx, ny, slot0, stride, q4, ni, nj, wr);
        if (iters > 1) {
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int n = slot0 + k * stride;
                if (n >= G) continue;
                st_relaxed_u64(pubw + (size_t)c0 * G + n, tag_word(1u, wr[k][0]));
                if (has1) st_relaxed_u64(pubw + (size_t)c1 * G + n, tag_word(1u, wr[k][1]));
            }
        }
    }
    float alpha = 0.f, beta = 0.f;
    ff gam{0.f, 0.f};
    for (int i = 0; i < iters && ok; ++i) {
        const bool last = i == iters - 1;
        const unsigned tag = (unsigned)i + 1u;
        const unsigned long long* W = pubw + (size_t)(i & 1) * G6;
        float gp = 0.f, dp = 0.f;
#pragma unroll
        for (int k = 0; k < NPT; ++k)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                gp = fmaf(rr[k][h], ur[k][h], gp);
                dp = fmaf(wr[k][h], ur[k][h], dp);
                mw[k][h] = mr[k][h] * wr[k][h];
            }
        if (!last) halo_load<true>(W, G6, g0, hv); // in flight during the block sums
        tagged_publish(gp, dp, sred, slots, tag);
        if (!last) {
            // m = M w and n = A m while the other blocks' partials arrive
            const bool fail = !smem_fill<NPT>(hl, W, G6, minv, tag, status, uh, slot0, stride, q4, mw, g0, s0, true, hv);
            if (__syncthreads_or(fail)) {
                ok = false;
                break;
            }
            smem_apply<NPT>(sB, sr1, uh, ls, hl, nx, ny, slot0, stride, q4, ni, nj, nr);
        }
        ff G2, D2;
        ok = tagged_collect(slots, tag, status, G2, D2);
        if (!ok) break;
        if (i == 0) {
            if (!(G2.hi > 1e-30f) || !(D2.hi > 1e-30f)) break; // x stays 0
            alpha = G2.hi / D2.hi;
            beta = 0.f;
        } else {
            const float bnew = G2.hi / gam.hi;
            const float pap = D2.hi - bnew * G2.hi / alpha;
            if (!(G2.hi > 1e-30f) || !(pap > 1e-30f)) break;
            beta = bnew;
            alpha = G2.hi / pap;
        }
        gam = G2;
#pragma unroll
        for (int k = 0; k < NPT; ++k)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                zr[k][h] = fmaf(beta, zr[k][h], nr[k][h]);
                qr[k][h] = fmaf(beta, qr[k][h], mw[k][h]);
                sr[k][h] = fmaf(beta, sr[k][h], wr[k][h]);
                pr[k][h] = fmaf(beta, pr[k][h], ur[k][h]);
                xr[k][h] = fmaf(alpha, pr[k][h], xr[k][h]);
                rr[k][h] = fmaf(-alpha, sr[k][h], rr[k][h]);
                ur[k][h] = mr[k][h] * rr[k][h]; // u = M r formed, not recurred
                wr[k][h] = fmaf(-alpha, zr[k][h], wr[k][h]);
            }
        if (i + 2 < iters) { // w_{i+1}, read by iteration i + 1's product
            unsigned long long* Wn = pubw + (size_t)((i + 1) & 1) * G6;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const int n = slot0 + k * stride;
                if (n >= G) continue;
                st_relaxed_u64(Wn + (size_t)c0 * G + n, tag_word(tag + 1u, wr[k][0]));
                if (has1) st_relaxed_u64(Wn + (size_t)c1 * G + n, tag_word(tag + 1u, wr[k][1]));
            }
        }
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
cudaError_t launch_grid1p(int blocks, const LevelGeom& g, const float* node, const float* rhs, const float* minv,
                          float* x, float* pub, float2* part, unsigned long long* bar, int* status, int iters,
                          int interleaved, cudaStream_t st)
{
    if (blocks < 1 || blocks > TAG_MAXB) return cudaErrorInvalidValue; // the tagged reduction polls TAG_MAXB slots
    if ((uintptr_t)pub & 7) return cudaErrorInvalidValue;               // 64-bit words
    const size_t smem = halo_smem(NPT, g.nx);
    cudaError_t e = cudaFuncSetAttribute((const void*)k_pcg1p<NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    LevelGeom gg = g;
    int ls = halo_ls(g.nx);
    unsigned long long* pubw = reinterpret_cast<unsigned long long*>(pub);
    void* args[] = {(void*)&gg,  (void*)&node,   (void*)&rhs,   (void*)&minv,        (void*)&x,  (void*)&pubw,
                    (void*)&part, (void*)&bar,   (void*)&status, (void*)&iters, (void*)&interleaved, (void*)&ls};
    return cudaLaunchCooperativeKernel((const void*)k_pcg1p<NPT>, dim3(blocks), dim3(PT), args, smem, st);
}

// Failure-detection probe of the self-tagged exchange (the waits of
// k_pcg1h and k_pcg1p, with a short limit). mode 0: every block but
// skip_block publishes its tagged partial words and warp 0 of every block
// polls all blocks' words (warp_poll_fold); mode 1: every block but
// skip_block publishes one tagged word and thread 0 of every block waits for
// the next block's word as a halo reader does (halo_wait). With a block that
// never publishes, every wait runs out, latches DEV_TIMEOUT and returns.
__global__ void __launch_bounds__(PT) k_tag_probe(unsigned long long* slots, unsigned long long* words, int* status,
                                                  int skip_block, long long limit, int mode, int* returned)
{
    const int nb = gridDim.x;
    const bool publish = (int)blockIdx.x != skip_block;
    if (mode == 0) {
        unsigned long long* sl = slots + (size_t)4 * nb; // the slot of tag 1
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0 && publish)
                for (int w = 0; w < 4; ++w) st_relaxed_u64(sl + (size_t)blockIdx.x * 4 + w, tag_word(1u, 1.f));
            ff va, vb;
            warp_poll_fold<false>(sl, nb, 1u, status, threadIdx.x, 1, va, vb, limit);
        }
    } else if (threadIdx.x == 0) {
        if (publish) st_relaxed_u64(words + blockIdx.x, tag_word(1u, 1.f));
        int gi[HPF];
        unsigned long long v[HPF][3];
#pragma unroll
        for (int j = 0; j < HPF; ++j) gi[j] = -1;
        gi[0] = (int)((blockIdx.x + 1) % nb);
        v[0][0] = ld_cg_u64(words + gi[0]);
        halo_wait<true>(words, 0, 1u, status, gi, v, limit);
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(returned, 1);
}

// blocks of a cooperative launch that the GPU holds at once: the smallest
// per-SM occupancy over the grid kernels, times the SMs
int max_coop_blocks(int sm_count)
{
    int per_sm = 1 << 20;
    auto take = [&](const void* kern) {
        int m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, kern, PT, 0) != cudaSuccess) {
            cudaGetLastError();
            m = 1;
        }
        per_sm = std::min(per_sm, std::max(m, 1));
    };
    take((const void*)k_pcg<1, GridSync>);
    take((const void*)k_pcg1<1, GridSync>);
    take((const void*)k_pcg1<2, GridSync>);
    take((const void*)k_pcg1<4, GridSync>);
    take((const void*)k_pcg1h<1>);
    take((const void*)k_pcg1h<2>);
    take((const void*)k_pcg1h<4>);
    take((const void*)k_pcg1p<1>);
    take((const void*)k_pcg1p<2>);
    take((const void*)k_pcg1p<4>);
    return per_sm * sm_count;
}

// per device, cached under a lock (the query sets a function attribute)
int max_cluster_blocks()
{
    static std::mutex mu;
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev] > 0) return cached[dev];
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
    cached[dev] = n > 16 ? 16 : n;
    return cached[dev];
}

size_t smem_optin()
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        optin = 227 * 1024;
    }
    return (size_t)optin;
}

int dsm_max_npc()
{
    // static shared memory of the kernel is small (< 1 KB); keep 2 KB spare
    return ((int)smem_optin() - 2048) / (int)(NODE_F * sizeof(float));
}

} // namespace

PcgPlan pcg_plan(int G, int sm_count, int mode, int nx)
{
    // preference: the staged, self-tagged grid (AUTO: the one-reduction form,
    // kind 5, measured faster than kinds 1-4 at every 640x480 level;
    // PIPELINED: kind 6) -> DSM (DSM only) -> cluster with global vectors
    // (all but GRID) -> cooperative grid (all)
    PcgPlan p{1, 1, 0, 0};
    const int maxc = max_cluster_blocks();
    if ((mode == SF_PCG_AUTO || mode == SF_PCG_PIPELINED) && nx > 0) {
        int cap = max_coop_blocks(sm_count);
        if (cap > TAG_MAXB) cap = TAG_MAXB;
        for (int npt : {1, 2, 4}) {
            const int need = std::max(1, (G + NPB * npt - 1) / (NPB * npt));
            if (need <= cap && halo_smem(npt, nx) + 2048 <= smem_optin()) {
                p.blocks = need;
                p.npt = npt;
                p.cluster = mode == SF_PCG_PIPELINED ? 6 : 5;
                return p;
            }
        }
    }
    if (mode == SF_PCG_DSM) {
        const int cap = dsm_max_npc();
        for (int npt = 1; npt <= 3; ++npt) {
            const int npc = std::min(CT_NPB * npt, cap);
            const int ctas0 = (G + npc - 1) / npc;
            if (ctas0 <= maxc) {
                const int even = (G + ctas0 - 1) / ctas0; // spread the nodes evenly
                p.blocks = (G + even - 1) / even;
                p.npt = npt;
                p.cluster = 2;
                p.npc = even;
                return p;
            }
        }
    }
    // otherwise the one-reduction form (measured faster than the textbook loop at every level size)
    const bool one = mode != SF_PCG_CLUSTER && mode != SF_PCG_GRID && mode != SF_PCG_DSM;
    if (mode != SF_PCG_GRID) {
        for (int npt : {1, 2, 4}) {
            const int need = (G + NPB * npt - 1) / (NPB * npt);
            if (need <= maxc) {
                p.blocks = need < 1 ? 1 : need;
                p.npt = npt;
                p.cluster = one ? 4 : 1;
                return p;
            }
        }
    }
    int cap = max_coop_blocks(sm_count);
    if (cap > MAX_PART / 2) cap = MAX_PART / 2;
    if (one && cap > TAG_MAXB) cap = TAG_MAXB; // the one-reduction grid polls tagged words
    for (int npt : {1, 2, 4}) {
        const int need = (G + NPB * npt - 1) / (NPB * npt);
        if (need <= cap) {
            p.blocks = need < 1 ? 1 : need;
            p.npt = npt;
            p.cluster = one ? 3 : 0;
            return p;
        }
    }
    p.blocks = -1; // too large for one launch
    return p;
}

int pcg_candidates(int G, int sm_count, PcgPlan* out, int max, int nx, bool pipelined)
{
    int n = 0;
    auto push = [&](PcgPlan p) {
        if (n < max) out[n++] = p;
    };
    const int maxc = max_cluster_blocks();
    int cap = max_coop_blocks(sm_count);
    if (cap > MAX_PART / 2) cap = MAX_PART / 2;
    for (int npt : {1, 2, 4}) {
        const int need = std::max(1, (G + NPB * npt - 1) / (NPB * npt));
        if (need <= maxc) {
            push(PcgPlan{need, npt, 4, 0});
            push(PcgPlan{need, npt, 1, 0});
        }
        if (need <= cap && need <= TAG_MAXB) {
            if (nx > 0 && halo_smem(npt, nx) + 2048 <= smem_optin()) {
                if (pipelined) push(PcgPlan{need, npt, 6, 0});
                push(PcgPlan{need, npt, 5, 0});
            }
            push(PcgPlan{need, npt, 3, 0});
        }
        if (need <= cap) push(PcgPlan{need, npt, 0, 0});
    }
    const int dcap = dsm_max_npc();
    for (int npt = 1; npt <= 3; ++npt) {
        const int npc = std::min(CT_NPB * npt, dcap);
        const int ctas0 = (G + npc - 1) / npc;
        if (ctas0 <= maxc) {
            const int even = (G + ctas0 - 1) / ctas0;
            push(PcgPlan{(G + even - 1) / even, npt, 2, even});
            break;
        }
    }
    return n;
}

cudaError_t launch_pcg(const LevelGeom& g, const PcgPlan& plan, const float* node, const float* rhs, const float* minv,
                       float* x, float* z, float* p0, float* p1, float* pub, float2* part, unsigned long long* bar,
                       int* status, int iters, int interleaved_out, cudaStream_t st)
{
    if (plan.cluster == 6) {
        switch (plan.npt) {
        case 1: return launch_grid1p<1>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        case 2: return launch_grid1p<2>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        default: return launch_grid1p<4>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        }
    }
    if (plan.cluster == 5) {
        switch (plan.npt) {
        case 1: return launch_grid1h<1>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        case 2: return launch_grid1h<2>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        default: return launch_grid1h<4>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        }
    }
    if (plan.cluster == 3 || plan.cluster == 4) {
        const bool grid = plan.cluster == 3;
        switch (plan.npt) {
        case 1: return grid ? launch_grid1<1>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st)
                            : launch_cluster1<1>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        case 2: return grid ? launch_grid1<2>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st)
                            : launch_cluster1<2>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        default: return grid ? launch_grid1<4>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st)
                             : launch_cluster1<4>(plan.blocks, g, node, rhs, minv, x, pub, part, bar, status, iters, interleaved_out, st);
        }
    }
    if (plan.cluster == 2) {
        switch (plan.npt) {
        case 1: return launch_dsm<1>(plan.blocks, plan.npc, g, node, rhs, minv, x, iters, interleaved_out, st);
        case 2: return launch_dsm<2>(plan.blocks, plan.npc, g, node, rhs, minv, x, iters, interleaved_out, st);
        default: return launch_dsm<3>(plan.blocks, plan.npc, g, node, rhs, minv, x, iters, interleaved_out, st);
        }
    }
    if (plan.cluster == 1) {
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

int tag_timeout_probe(int mode, int skip_block, long long limit_cycles, int* status, int* returned)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return SF_ERR_CUDA;
    }
    const int nb = std::min(sms, TAG_MAXB);
    if (skip_block >= nb) return SF_ERR_ARG;
    unsigned long long* buf = nullptr; // slots [2][nb][4], then nb words
    int* w = nullptr;                  // [0] status, [1] blocks returned
    const size_t nw = (size_t)8 * nb + nb;
    if (cudaMalloc(&buf, nw * sizeof(*buf)) != cudaSuccess || cudaMalloc(&w, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        return SF_ERR_OOM;
    }
    cudaMemset(buf, 0, nw * sizeof(*buf));
    cudaMemset(w, 0, 2 * sizeof(int));
    unsigned long long* slots = buf;
    unsigned long long* words = buf + (size_t)8 * nb;
    int* st = w;
    int* ret = w + 1;
    void* args[] = {(void*)&slots, (void*)&words, (void*)&st, (void*)&skip_block, (void*)&limit_cycles,
                    (void*)&mode,  (void*)&ret};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_tag_probe, dim3(nb), dim3(PT), args, 0, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    cudaFree(w);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SF_ERR_CUDA;
    }
    *status = (h[0] & DEV_TIMEOUT) ? SF_ERR_TIMEOUT : (h[0] ? SF_ERR_STATE : SF_OK);
    *returned = h[1];
    return SF_OK;
}

} // namespace sfk
