// sf_schwarz.cu -- the domain decomposition of Thies et al., arXiv 1610.07159,
// Section 5.2: the normal equations of one Gauss-Newton step solved by
// data-parallel alternating Schwarz iterations over small square subdomains,
// each subdomain's system solved by a few PCG iterations ("patch iterations")
// with all of its data in shared memory, the subdomains exchanging data
// through global memory between sweeps.
//
// Reading of the schedule (the paper names "PCG iterations with patch
// iterations each"): a sweep computes the residual r = b - A x of the current
// iterate, every subdomain (a tile of T x T nodes grown by H nodes of overlap
// on each side) solves its local system A_k e = r_k by `patch` Jacobi-PCG
// iterations from e = 0 (couplings to nodes outside the subdomain dropped:
// those nodes are held at x), and every node takes x + e from the subdomain
// whose tile holds it (restricted additive Schwarz). There are `sweeps`
// sweeps per Gauss-Newton step, from x = 0.
//
// Layout: one CTA per subdomain (CTAs loop over subdomains when there are
// more than fit on the GPU at once). Six threads serve a node, one per
// component: thread t holds component t % 6 of local node t / 6 of the
// extended domain in registers (e, r, z, p, the preconditioner), and the
// local matrix-vector product reads the node's nine coupling blocks (packed
// symmetric 6x6, staged once into shared memory when the CTA owns a single
// subdomain) and the neighbours' p from shared memory. A local iteration has
// two block reductions and no grid-wide one; sweeps meet at a bounded grid
// barrier (cooperative launch), and the iterate is double-buffered in global
// memory.
#include <algorithm>
#include <mutex>

#include "sf_launch.h"
#include "sf_stages.cuh"

namespace sfk {

namespace {

constexpr int SW_MAX_THREADS = 608; // six threads per node: extended subdomains of up to 100 nodes

struct SwGeom {
    int T, H;        // tile and overlap (nodes)
    int ntx, nty;    // tiles per row / column
    int nsub;        // ntx * nty
    int emax;        // largest extended domain (nodes)
};

__device__ __forceinline__ void sub_bounds(const LevelGeom& g, const SwGeom& s, int d, int& ti, int& tj, int& i0,
                                           int& j0, int& i1, int& j1)
{
    tj = d / s.ntx;
    ti = d - tj * s.ntx;
    i0 = max(ti * s.T - s.H, 0);
    j0 = max(tj * s.T - s.H, 0);
    i1 = min((ti + 1) * s.T + s.H, g.nx);
    j1 = min((tj + 1) * s.T + s.H, g.ny);
}

// Shared-memory layout of a subdomain (ES, a compile-time bound on its nodes):
// sA holds the five stored coupling blocks of every node as full 6x6 blocks,
// entry (row c, column cc) of block b of local node l at ((b*6 + cc)*ES + l)*6
// + c, so that the six threads of a node (one per row) read six consecutive
// words and row c of a block is six loads at fixed offsets; su holds a vector
// of the local system, component c of local node l at l*6 + c. Both layouts
// keep a warp's loads and stores free of bank conflicts.
constexpr int SW_BLK = NODE_BLKS * 36;

// Per-thread stencil of component c of local node ln: for each of the nine
// slots, the shared-memory offset of row c of the slot's block (or -1 when
// the slot's node is off the grid or outside the subdomain) and the local
// index of the slot's node; bit s of `outside` marks a slot whose node is on
// the grid but outside the subdomain.
template <int ES>
struct SlotTable {
    int aoff[9], poff[9];
    unsigned outside;

    __device__ __forceinline__ void build(const LevelGeom& g, bool live, int i, int j, int n, int ln, int c, int i0,
                                          int j0, int i1, int j1, int lx)
    {
        outside = 0u;
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            aoff[s] = -1;
            poff[s] = 0;
            int owner, blk, pn;
            if (!live || !stencil_slot(s, i, j, g.nx, g.ny, n, owner, blk, pn)) continue;
            const int pj = pn / g.nx, pi = pn - pj * g.nx;
            if (pi < i0 || pi >= i1 || pj < j0 || pj >= j1) {
                outside |= 1u << s;
                continue;
            }
            const int lp = (pj - j0) * lx + (pi - i0);
            const int lo = owner == n ? ln : lp;
            aoff[s] = (blk * 6 * ES + lo) * 6 + c;
            poff[s] = lp * 6;
        }
    }

    // row c of (A_local v)(ln), v in shared memory (l*6 + c)
    __device__ __forceinline__ float apply(const float* sA, const float* sv) const
    {
        float acc = 0.f;
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            if (aoff[s] < 0) continue;
            const float* a = sA + aoff[s];
            const float* v = sv + poff[s];
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) acc = fmaf(a[cc * ES * 6], v[cc], acc);
        }
        return acc;
    }
};

// Row c of the couplings of node n to the slots marked `outside`, times x
// from global memory (coherent loads: other CTAs wrote it before the last
// grid barrier).
__device__ __forceinline__ float outside_apply(const LevelGeom& g, const float* __restrict__ node, const float* x,
                                               unsigned outside, int i, int j, int n, int c)
{
    float acc = 0.f;
    for (int s = 0; s < 9; ++s) {
        if (!(outside & (1u << s))) continue;
        int owner, blk, pn;
        stencil_slot(s, i, j, g.nx, g.ny, n, owner, blk, pn);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc)
            acc = fmaf(__ldg(node + (size_t)(blk * NB + sym_idx(c, cc)) * g.G + owner), __ldcg(x + cc * g.G + pn), acc);
    }
    return acc;
}

// Two fixed-order block sums at once with two CTA barriers: warp sums, one
// partial per warp into spart[par] (double-buffered by the caller's
// iteration parity, so the next call's writes never meet this call's
// reads), then every warp folds the partials in warp order itself.
__device__ __forceinline__ void block_sum2(float& a, float& b, float (*spart)[32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        spart[0][warp] = a;
        spart[1][warp] = b;
    }
    __syncthreads();
    a = warp_sum(lane < nw ? spart[0][lane] : 0.f);
    b = warp_sum(lane < nw ? spart[1][lane] : 0.f);
}

template <int ES>
__global__ void __launch_bounds__(SW_MAX_THREADS) k_schwarz(LevelGeom g, SwGeom s, const float* __restrict__ node,
                                                            const float* __restrict__ rhs,
                                                            const float* __restrict__ minv, float* xout, float* xtmp,
                                                            unsigned long long* bar, int* status, int sweeps,
                                                            int patch, int interleaved)
{
    extern __shared__ float smem[];
    __shared__ float spart[2][2][32];
    float* sA = smem;              // SW_BLK * ES floats
    float* su = smem + SW_BLK * ES; // 6 * ES floats
    const bool single = (int)gridDim.x >= s.nsub; // each CTA owns at most one subdomain: blocks stay staged
    unsigned long long target = 0;
    if (gridDim.x > 1) target = grid_barrier_base(bar, gridDim.x);
    const int t = threadIdx.x;
    const int c = t % 6;
    const int ln = t / 6;
    bool ok = true;
    bool staged = false; // sA holds this CTA's subdomain (kept across sweeps when it owns only one)
    int par = 0;         // parity of the partial-sum buffer
    for (int sw = 0; sw < sweeps && ok; ++sw) {
        // sweep sw writes xw and reads the previous sweep's output; the last sweep writes xout
        float* xw = ((sweeps - 1 - sw) & 1) ? xtmp : xout;
        const float* xr = ((sweeps - sw) & 1) ? xtmp : xout;
        for (int d = blockIdx.x; d < s.nsub; d += gridDim.x) {
            int ti, tj, i0, j0, i1, j1;
            sub_bounds(g, s, d, ti, tj, i0, j0, i1, j1);
            const int lx = i1 - i0, ly = j1 - j0, En = lx * ly;
            const bool live = ln < En;
            const int i = live ? i0 + ln % lx : 0, j = live ? j0 + ln / lx : 0, n = j * g.nx + i;
            SlotTable<ES> tab;
            tab.build(g, live, i, j, n, ln, c, i0, j0, i1, j1, lx);
            __syncthreads(); // the previous subdomain's last reads of sA and su are done
            if (!(single && staged)) {
                // the coupling blocks of the extended domain, unpacked to full 6x6 blocks
                for (int k = t; k < SW_BLK * En; k += blockDim.x) {
                    const int bc = k / (6 * En), rem = k - bc * 6 * En; // bc = b*6 + cc
                    const int l = rem / 6, rr = rem - l * 6;
                    const int b = bc / 6, cc = bc - b * 6;
                    const int gi = i0 + l % lx, gj = j0 + l / lx;
                    sA[(bc * ES + l) * 6 + rr] = __ldg(node + (size_t)(b * NB + sym_idx(rr, cc)) * g.G + gj * g.nx + gi);
                }
                staged = true;
            }
            // residual of the current iterate (x = 0 in the first sweep): the subdomain's part of A x from
            // shared memory, the couplings to nodes outside it from global memory
            float r = 0.f, m = 0.f;
            if (live) {
                r = rhs[c * g.G + n];
                m = minv[c * g.G + n];
                if (sw > 0) su[ln * 6 + c] = __ldcg(xr + c * g.G + n);
            }
            __syncthreads();
            if (live && sw > 0) {
                r -= tab.apply(sA, su);
                if (tab.outside) r -= outside_apply(g, node, xr, tab.outside, i, j, n, c);
            }
            // local Jacobi-PCG from e = 0 in its one-reduction form (Chronopoulos-Gear: the iterates of the
            // textbook loop in exact arithmetic): u = M r, w = A u, gamma = r.u and delta = w.u in one sum
            float e = 0.f, u = m * r, p = 0.f, sv = 0.f, w = 0.f;
            __syncthreads(); // su free
            if (live) su[ln * 6 + c] = u;
            __syncthreads();
            if (live) w = tab.apply(sA, su);
            float gam = live ? r * u : 0.f, del = live ? w * u : 0.f;
            block_sum2(gam, del, spart[par]);
            par ^= 1;
            float gam_prev = 1.f, alpha_prev = 1.f;
            for (int it = 0; it < patch; ++it) {
                if (!(gam > 1e-30f)) break;
                const float beta = it == 0 ? 0.f : gam / gam_prev;
                const float pq = it == 0 ? del : del - beta * gam / alpha_prev; // p.A p
                if (!(pq > 1e-30f)) break;
                const float alpha = gam / pq;
                p = fmaf(beta, p, u);
                sv = fmaf(beta, sv, w); // s = A p
                e = fmaf(alpha, p, e);
                r = fmaf(-alpha, sv, r);
                if (it + 1 == patch) break; // the last update needs no new direction
                u = m * r;
                if (live) su[ln * 6 + c] = u; // su was last read before the previous sum's barrier
                __syncthreads();
                w = live ? tab.apply(sA, su) : 0.f;
                gam_prev = gam;
                alpha_prev = alpha;
                gam = live ? r * u : 0.f;
                del = live ? w * u : 0.f;
                block_sum2(gam, del, spart[par]);
                par ^= 1;
            }
            // restricted update: the tile's own nodes
            if (live && i >= ti * s.T && i < (ti + 1) * s.T && j >= tj * s.T && j < (tj + 1) * s.T) {
                const float xo = sw > 0 ? __ldcg(xr + c * g.G + n) : 0.f;
                const float xn = xo + e;
                if (sw == sweeps - 1 && interleaved)
                    xw[n * 6 + c] = xn;
                else
                    xw[c * g.G + n] = xn;
            }
        }
        if (sw + 1 < sweeps && gridDim.x > 1) {
            target += gridDim.x;
            ok = grid_barrier(bar, status, target);
        }
    }
}

constexpr int SW_STRIDES[] = {9, 16, 25, 36, 49, 64, 81, 100};

template <int ES>
const void* schwarz_kernel()
{
    return (const void*)k_schwarz<ES>;
}

const void* schwarz_kernel_for(int es)
{
    switch (es) {
    case 9: return schwarz_kernel<9>();
    case 16: return schwarz_kernel<16>();
    case 25: return schwarz_kernel<25>();
    case 36: return schwarz_kernel<36>();
    case 49: return schwarz_kernel<49>();
    case 64: return schwarz_kernel<64>();
    case 81: return schwarz_kernel<81>();
    default: return schwarz_kernel<100>();
    }
}

} // namespace

int schwarz_plan(const LevelGeom& g, int tile, int overlap, int sm_count, SchwarzPlan* out)
{
    if (tile < 1 || overlap < 0) return -1;
    const int ntx = (g.nx + tile - 1) / tile, nty = (g.ny + tile - 1) / tile;
    const int ex = std::min(tile + 2 * overlap, g.nx), ey = std::min(tile + 2 * overlap, g.ny);
    const int emax = ex * ey;
    int es = -1;
    for (int v : SW_STRIDES)
        if (emax <= v) {
            es = v;
            break;
        }
    if (es < 0) return -1; // more than 100 nodes per subdomain
    const int threads = ((6 * emax + 31) / 32) * 32;
    const size_t smem = (size_t)(SW_BLK + 6) * es * sizeof(float);
    const void* kern = schwarz_kernel_for(es);
    {
        // the dynamic shared-memory limit is a per-device function attribute
        static std::mutex mu;
        static bool attr_set[64][8] = {};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
            cudaGetLastError();
            return -1;
        }
        int k = 0;
        while (SW_STRIDES[k] != es) ++k;
        std::lock_guard<std::mutex> lk(mu);
        if (!attr_set[dev][k]) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
            attr_set[dev][k] = true;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return -1;
    }
    out->tile = tile;
    out->overlap = overlap;
    out->nsub = ntx * nty;
    out->emax = emax;
    out->es = es;
    out->threads = threads;
    out->smem = (int)smem;
    out->blocks = std::min(ntx * nty, per_sm * sm_count);
    return 0;
}

cudaError_t launch_schwarz(const LevelGeom& g, const SchwarzPlan& plan, const float* node, const float* rhs,
                           const float* minv, float* x, float* xtmp, unsigned long long* bar, int* status, int sweeps,
                           int patch, int interleaved_out, cudaStream_t st)
{
    if (sweeps < 1) {
        // no sweep: x = 0
        const size_t bytes = (size_t)6 * g.G * sizeof(float);
        return cudaMemsetAsync(x, 0, bytes, st);
    }
    SwGeom s{};
    s.T = plan.tile;
    s.H = plan.overlap;
    s.ntx = (g.nx + plan.tile - 1) / plan.tile;
    s.nty = (g.ny + plan.tile - 1) / plan.tile;
    s.nsub = plan.nsub;
    s.emax = plan.emax;
    LevelGeom gg = g;
    void* args[] = {(void*)&gg, (void*)&s, (void*)&node, (void*)&rhs, (void*)&minv, (void*)&x, (void*)&xtmp,
                    (void*)&bar, (void*)&status, (void*)&sweeps, (void*)&patch, (void*)&interleaved_out};
    return cudaLaunchCooperativeKernel(schwarz_kernel_for(plan.es), dim3(plan.blocks), dim3(plan.threads), args,
                                       (size_t)plan.smem, st);
}

} // namespace sfk
