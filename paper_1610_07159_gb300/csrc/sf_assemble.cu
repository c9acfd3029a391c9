// sf_assemble.cu -- the Gauss-Newton linearisation of the halfway-domain
// energy (Thies et al., arXiv 1610.07159, Section 5.1):
//   * per pixel: the six consistency checks of Eqs. 1-6 on bilinear samples of
//     intensity and gradient, the outlier weight W (Section 4.1), the robust
//     pseudo-Huber terms of Eqs. 11-13 and their reweighted normal-equation
//     contributions H_p, b_p;
//   * per warp-grid cell: sum_p alpha_k alpha_l H_p and sum_p alpha_k b_p
//     (the chain rule through the bilinear weights of Eq. 7), reduced in
//     shared memory; the paper precomputes these alignment blocks once per
//     step and reads them on demand (Section 5.2);
//   * per node: gather of the cell blocks plus the smoothness (Eq. 14),
//     epipolar (Eqs. 15-17) and magnitude (Eq. 18) rows, the Jacobi
//     preconditioner and the energy at the linearisation point;
//   * energies of trial steps with the backtracking decision and the update.
#include "sf_launch.h"
#include "sf_stages.cuh"

namespace sfk {

namespace {

// One CTA per cell group (assemble_group), then the block's energy partials.
// REC: also record the cell decisions of samples at a cell edge (test aid).
template <int MAXT, class TT, bool REC>
__global__ void __launch_bounds__(ETHREADS, 2) k_assemble(LevelGeom g, int cpb, const typename TT::T* __restrict__ tex,
                                                       const float* __restrict__ base, const float* __restrict__ delta,
                                                       DevParams P, LevelMaps M, uint8_t* __restrict__ Wmask,
                                                       float* __restrict__ cell, float2* __restrict__ part, CellLog log)
{
    __shared__ float sHB[ETHREADS * HB];
    __shared__ __align__(16) float sW[ETHREADS * WROW];
    __shared__ ff sred[3 * (ETHREADS / 32)];
    const int tid = threadIdx.x;
    float ep = 0.f, eg = 0.f;
    int nex = 0;
    assemble_group<MAXT, TT, REC>(g, cpb, blockIdx.x, blockIdx.y, tex, base, delta, P, M, Wmask, cell, sHB, sW, ep,
                                  eg, nex, &log);
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    const float v[3] = {ep, eg, (float)nex};
    ff t[3];
    ff_block_sum_fast_n<ETHREADS, 3>(v, sred, t);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) part[q * MAX_PART + blk] = make_float2(t[q].hi, t[q].lo);
    }
}

// Gather of the node system from the cell blocks plus the prior rows, the
// Jacobi preconditioner, and (last block) the energy at this point; four
// lanes per node.
__global__ void __launch_bounds__(ETHREADS) k_gather(LevelGeom g, const float* __restrict__ cell,
                                                     const float* __restrict__ base, const float* __restrict__ delta,
                                                     const float* __restrict__ wf, DevParams P,
                                                     float* __restrict__ node, float* __restrict__ rhs,
                                                     float* __restrict__ minv, float2* __restrict__ gpart,
                                                     const float2* __restrict__ apart, int n_asm, unsigned* counter,
                                                     StepCtrl* __restrict__ ctrl, int* status)
{
    __shared__ ff sred[6 * (ETHREADS / 32)];
    __shared__ bool last_sh;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = t >> 2;
    float es = 0.f, ee = 0.f, em = 0.f;
    gather_node4(g, n < g.G ? n : g.G - 1, t & 3, n < g.G, cell, base, delta, wf, P, node, rhs, minv, es, ee, em);
    if (!ctrl) return;
    const float v[3] = {es, ee, em};
    ff tb[3];
    ff_block_sum_fast_n<ETHREADS, 3>(v, sred, tb);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) gpart[q * MAX_PART + blockIdx.x] = make_float2(tb[q].hi, tb[q].lo);
        __threadfence();
        const unsigned done = atomicAdd(counter, 1u);
        last_sh = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_sh) return;
    __threadfence();
    {
        const float2* const parts[6] = {apart, apart + MAX_PART, apart + 2 * MAX_PART,
                                        gpart, gpart + MAX_PART, gpart + 2 * MAX_PART};
        const int nb = (int)gridDim.x;
        const int cnt[6] = {n_asm, n_asm, n_asm, nb, nb, nb};
        ff f[6];
        ff_block_fixed_sum_n<ETHREADS, 6>(parts, cnt, sred, f);
        const ff fp = f[0], fg = f[1], fx = f[2], fs = f[3], fe = f[4], fm = f[5];
        const double sp = (double)fp.hi + fp.lo, sg = (double)fg.hi + fg.lo, sx = (double)fx.hi + fx.lo;
        const double ss = (double)fs.hi + fs.lo, se = (double)fe.hi + fe.lo, sm = (double)fm.hi + fm.lo;
        if (threadIdx.x == 0) {
            StepCtrl c;
            c.terms_cur[0] = P.w_photo * sp;
            c.terms_cur[1] = P.w_grad * sg;
            c.terms_cur[2] = (double)P.w_reg * P.w_smooth * ss;
            c.terms_cur[3] = (double)P.w_reg * P.w_epi * se;
            c.terms_cur[4] = (double)P.w_reg * P.w_mag * sm;
            c.E_cur = c.terms_cur[0] + c.terms_cur[1] + c.terms_cur[2] + c.terms_cur[3] + c.terms_cur[4];
            c.E_acc = c.E_cur;
            for (int q = 0; q < 5; ++q) c.terms_acc[q] = c.terms_cur[q];
            c.t = 0.f;
            c.accepted = 0;
            c.n_excluded = (int)sx;
            c.pad = 0;
            *ctrl = c;
            if (!isfinite(c.E_cur)) atomicOr(status, DEV_NUMERIC);
            __threadfence();
            *counter = 0u;
        }
    }
}

// Energy at base + delta (+ t x): pixel blocks first, then node blocks;
// the last block to finish sums the partials in a fixed order and writes the
// record (energy, the five weighted terms, excluded pixels).
template <class TT>
__global__ void __launch_bounds__(ETHREADS) k_energy(LevelGeom g, int npixblk, const typename TT::T* __restrict__ tex,
                                                     const float* __restrict__ base, const float* __restrict__ delta,
                                                     const float* __restrict__ x, float t, const float* __restrict__ wf,
                                                     DevParams P, LevelMaps M, uint8_t* __restrict__ Wmask, int wmode,
                                                     float2* __restrict__ part, unsigned* counter,
                                                     double* __restrict__ rec, int* status)
{
    __shared__ ff sred[6 * (ETHREADS / 32)];
    __shared__ bool last_sh;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if ((int)blockIdx.x < npixblk) {
        const int N = g.w * g.h;
        for (int p = blockIdx.x * ETHREADS + threadIdx.x; p < N; p += npixblk * ETHREADS) {
            const int y = p / g.w, xx = p - y * g.w;
            int i0, j0;
            float a, bb;
            grid_cell(xx, y, g.s, g.nx, g.ny, i0, j0, a, bb);
            float f[6];
            pixel_fields(base, delta, x, t, g.G, j0 * g.nx + i0, g.nx, a, bb, f);
            int Wi;
            float Ep, Eg;
            pixel_data<false, TT>(tex, g.w, g.h, xx, y, f, P, M, wmode ? -1 : (int)Wmask[p], Wi, Ep, Eg, nullptr,
                                  nullptr);
            if (wmode) Wmask[p] = (uint8_t)Wi;
            v[0] += Ep;
            v[1] += Eg;
            v[5] += Wi ? 0.f : 1.f;
        }
    } else {
        const int n = (blockIdx.x - npixblk) * ETHREADS + threadIdx.x;
        if (n < g.G) node_prior_energy(g, P, base, delta, x, t, wf, n, v[2], v[3], v[4]);
    }
    {
        ff sq[6];
        ff_block_sum_fast_n<ETHREADS, 6>(v, sred, sq);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) part[q * MAX_PART + blockIdx.x] = make_float2(sq[q].hi, sq[q].lo);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(counter, 1u);
        last_sh = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_sh) return;
    __threadfence();
    {
        const float2* const parts[6] = {part, part + MAX_PART, part + 2 * MAX_PART,
                                        part + 3 * MAX_PART, part + 4 * MAX_PART, part + 5 * MAX_PART};
        const int nb = (int)gridDim.x;
        const int cnt[6] = {nb, nb, nb, nb, nb, nb};
        ff f[6];
        ff_block_fixed_sum_n<ETHREADS, 6>(parts, cnt, sred, f);
        double s[6];
        for (int q = 0; q < 6; ++q) s[q] = (double)f[q].hi + f[q].lo;
        if (threadIdx.x == 0) {
            double terms[5];
            terms[0] = P.w_photo * s[0];
            terms[1] = P.w_grad * s[1];
            terms[2] = (double)P.w_reg * P.w_smooth * s[2];
            terms[3] = (double)P.w_reg * P.w_epi * s[3];
            terms[4] = (double)P.w_reg * P.w_mag * s[4];
            const double E = terms[0] + terms[1] + terms[2] + terms[3] + terms[4];
            rec[0] = E;
            for (int q = 0; q < 5; ++q) rec[1 + q] = terms[q];
            rec[6] = s[5];
            if (!isfinite(E)) atomicOr(status, DEV_NUMERIC);
            __threadfence();
            *counter = 0u;
        }
    }
}

// All backtracking trials of one Gauss-Newton step and the update in one
// cooperative launch: for t = 1, 1/2, ... every block sums its share of the
// pixel and node energies at delta + t x (W of the step), a bounded grid
// barrier, then warp 0 of every block forms the fixed-order totals, so all
// blocks take the same decision; the first t whose energy does not exceed E_cur is taken
// and applied (delta += t x). Replaces max_backtracks + 1 trial launches, most
// of which found the step already taken, and the update launch.
template <class TT>
__global__ void __launch_bounds__(ETHREADS) k_trials(LevelGeom g, const typename TT::T* __restrict__ tex,
                                                     const float* base, float* delta, const float* x,
                                                     const float* __restrict__ wf, DevParams P, LevelMaps M,
                                                     const uint8_t* __restrict__ Wmask, float2* part,
                                                     unsigned long long* bar, int* status, StepCtrl* ctrl, int max_bt)
{
    __shared__ float sh[5][ETHREADS / 32];
    __shared__ double sq_sh[5];
    unsigned long long target = grid_barrier_base(bar, gridDim.x);
    const int nb = gridDim.x;
    const int tid = blockIdx.x * ETHREADS + threadIdx.x, stride = nb * ETHREADS;
    const double E_cur = ctrl->E_cur;
    const int N = g.w * g.h;
    float t = 1.f, t_acc = 0.f;
    double E_acc = E_cur, terms_acc[5];
    for (int q = 0; q < 5; ++q) terms_acc[q] = ctrl->terms_cur[q];
    bool ok = true;
    for (int j = 0; j <= max_bt && ok; ++j, t *= 0.5f) {
        float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int p = tid; p < N; p += stride) {
            const int y = p / g.w, xx = p - y * g.w;
            int i0, j0;
            float a, bb;
            grid_cell(xx, y, g.s, g.nx, g.ny, i0, j0, a, bb);
            float f[6];
            pixel_fields(base, delta, x, t, g.G, j0 * g.nx + i0, g.nx, a, bb, f);
            int Wi;
            float Ep, Eg;
            pixel_data<false, TT>(tex, g.w, g.h, xx, y, f, P, M, (int)Wmask[p], Wi, Ep, Eg, nullptr, nullptr);
            v[0] += Ep;
            v[1] += Eg;
        }
        for (int n = tid; n < g.G; n += stride) {
            float a0, a1, a2;
            node_prior_energy(g, P, base, delta, x, t, wf, n, a0, a1, a2);
            v[2] += a0;
            v[3] += a1;
            v[4] += a2;
        }
        // block sums: FP32 within a warp, float-float across warps (thread 0, warp order)
        float2* pj = part + (size_t)(j & 1) * 5 * nb;
#pragma unroll
        for (int q = 0; q < 5; ++q) v[q] = warp_sum(v[q]);
        __syncthreads();
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x >> 5] = v[q];
        __syncthreads();
        if (threadIdx.x == 0)
            for (int q = 0; q < 5; ++q) {
                ff tq{0.f, 0.f};
                for (int w = 0; w < ETHREADS / 32; ++w) tq = ff_add(tq, ff_from(sh[q][w]));
                pj[q * nb + blockIdx.x] = make_float2(tq.hi, tq.lo);
            }
        target += nb;
        ok = grid_barrier(bar, status, target);
        if (!ok) break;
        // warp 0 forms the five fixed-order totals (the fold of ff_fixed_sum,
        // the five values' loads of one index in flight together) and hands
        // them to the block; sq_sh is next written after two more CTA barriers
        if (threadIdx.x < 32) {
            ff acc[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[q] = ff{0.f, 0.f};
            for (int i = threadIdx.x; i < nb; i += 32) {
                float2 tv[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) tv[q] = __ldcg(pj + q * nb + i);
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[q] = ff_add(acc[q], ff{tv[q].x, tv[q].y});
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[q] = ff_warp_sum(acc[q]);
            if (threadIdx.x == 0)
#pragma unroll
                for (int q = 0; q < 5; ++q) sq_sh[q] = (double)acc[q].hi + acc[q].lo;
        }
        __syncthreads();
        double sq[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) sq[q] = sq_sh[q];
        double terms[5];
        terms[0] = P.w_photo * sq[0];
        terms[1] = P.w_grad * sq[1];
        terms[2] = (double)P.w_reg * P.w_smooth * sq[2];
        terms[3] = (double)P.w_reg * P.w_epi * sq[3];
        terms[4] = (double)P.w_reg * P.w_mag * sq[4];
        const double E = terms[0] + terms[1] + terms[2] + terms[3] + terms[4];
        if (E <= E_cur) {
            t_acc = t;
            E_acc = E;
            for (int q = 0; q < 5; ++q) terms_acc[q] = terms[q];
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->E_acc = E_acc;
        for (int q = 0; q < 5; ++q) ctrl->terms_acc[q] = terms_acc[q];
        ctrl->t = t_acc;
        ctrl->accepted = ok && t_acc > 0.f ? 1 : 0;
    }
    if (ok && t_acc > 0.f)
        for (int k = tid; k < 6 * g.G; k += stride) delta[k] = fmaf(t_acc, x[k], delta[k]);
}

__global__ void k_unpack_blocks(int G, const float* __restrict__ node, const float* __restrict__ rhs,
                                float* __restrict__ blocks, float* __restrict__ rhs_out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G) return;
    for (int b = 0; b < NODE_BLKS; ++b)
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 6; ++c)
                blocks[((size_t)n * NODE_BLKS + b) * 36 + r * 6 + c] = node[(size_t)(b * NB + sym_idx(r, c)) * G + n];
    for (int r = 0; r < 6; ++r) rhs_out[n * 6 + r] = rhs[r * G + n];
}

template <int MAXT>
void assemble_impl(const LevelGeom& g, int cpb, const void* tex, int prec, const float* base, const float* delta,
                   const DevParams& P, const LevelMaps& M, uint8_t* Wmask, float* cell, float2* part,
                   const CellLog* log, cudaStream_t st)
{
    dim3 grid((g.ncx + cpb - 1) / cpb, g.ncy);
    if (log) {
        SF_TEX_DISPATCH(prec, TT, k_assemble<MAXT, TT, true><<<grid, ETHREADS, 0, st>>>(
                                      g, cpb, static_cast<const typename TT::T*>(tex), base, delta, P, M, Wmask, cell,
                                      part, *log));
    } else {
        SF_TEX_DISPATCH(prec, TT, k_assemble<MAXT, TT, false><<<grid, ETHREADS, 0, st>>>(
                                      g, cpb, static_cast<const typename TT::T*>(tex), base, delta, P, M, Wmask, cell,
                                      part, CellLog{nullptr, nullptr, 0}));
    }
}

} // namespace

int assemble_blocks(const LevelGeom& g, int* cpb_out)
{
    int cpb = ETHREADS / (g.s * g.s);
    if (cpb < 1) cpb = 1;
    while (assemble_tasks_per_thread(cpb) > 4) --cpb;
    if (cpb_out) *cpb_out = cpb;
    return ((g.ncx + cpb - 1) / cpb) * g.ncy;
}

void launch_assemble(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta,
                     const DevParams& P, uint8_t* Wmask, float* cell, const Scratch& sc, cudaStream_t st,
                     const CellLog* log, const LevelMaps& M)
{
    int cpb;
    assemble_blocks(g, &cpb);
    const int need = assemble_tasks_per_thread(cpb);
    if (need <= 1)
        assemble_impl<1>(g, cpb, tex, prec, base, delta, P, M, Wmask, cell, sc.asm_part, log, st);
    else if (need <= 2)
        assemble_impl<2>(g, cpb, tex, prec, base, delta, P, M, Wmask, cell, sc.asm_part, log, st);
    else
        assemble_impl<4>(g, cpb, tex, prec, base, delta, P, M, Wmask, cell, sc.asm_part, log, st);
}

void launch_gather(const LevelGeom& g, const float* cell, const float* base, const float* delta, const float* wf,
                   const DevParams& P, float* node, float* rhs, float* minv, const Scratch& sc, StepCtrl* ctrl,
                   int n_asm_blocks, cudaStream_t st)
{
    const int blocks = (4 * g.G + ETHREADS - 1) / ETHREADS; // four lanes per node
    k_gather<<<blocks, ETHREADS, 0, st>>>(g, cell, base, delta, wf, P, node, rhs, minv, sc.gat_part, sc.asm_part,
                                          n_asm_blocks, sc.counters + 0, ctrl, sc.status);
}

void launch_energy(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta, const float* x,
                   float t, const float* wf, const DevParams& P, uint8_t* Wmask, int wmode, const Scratch& sc,
                   double* rec, cudaStream_t st, const LevelMaps& M)
{
    int npix = (g.w * g.h + ETHREADS - 1) / ETHREADS;
    if (npix > 152 * 8) npix = 152 * 8;
    const int nnode = (g.G + ETHREADS - 1) / ETHREADS;
    SF_TEX_DISPATCH(prec, TT, k_energy<TT><<<npix + nnode, ETHREADS, 0, st>>>(
                                  g, npix, static_cast<const typename TT::T*>(tex), base, delta, x, t, wf, P, M,
                                  Wmask, wmode, sc.en_part, sc.counters + 1, rec, sc.status));
}

template <class TT>
int trials_blocks_impl(int sm_count)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trials<TT>, ETHREADS, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * sm_count;
}

int trials_blocks(const LevelGeom& g, int prec, int sm_count)
{
    int cap = 0;
    SF_TEX_DISPATCH(prec, TT, cap = trials_blocks_impl<TT>(sm_count));
    // two CTAs per SM at most: room for the kernels of other levels running beside it
    if (cap > 2 * sm_count) cap = 2 * sm_count;
    const int want = (g.w * g.h + ETHREADS - 1) / ETHREADS;
    int b = want < cap ? want : cap;
    if (b > MAX_PART) b = MAX_PART;
    return b < 1 ? 1 : b;
}

cudaError_t launch_trials(const LevelGeom& g, const void* tex, int prec, const float* base, float* delta, const float* x,
                          const float* wf, const DevParams& P, const uint8_t* Wmask, const Scratch& sc,
                          unsigned long long* bar, StepCtrl* ctrl, int max_bt, int blocks, cudaStream_t st,
                          const LevelMaps& M)
{
    LevelGeom gg = g;
    DevParams pp = P;
    LevelMaps mm = M;
    float2* part = sc.en_part;
    int* status = sc.status;
    void* args[] = {(void*)&gg, nullptr, (void*)&base, (void*)&delta, (void*)&x, (void*)&wf, (void*)&pp, (void*)&mm,
                    (void*)&Wmask, (void*)&part, (void*)&bar, (void*)&status, (void*)&ctrl, (void*)&max_bt};
    cudaError_t e = cudaSuccess;
    SF_TEX_DISPATCH(prec, TT, {
        const typename TT::T* tp = static_cast<const typename TT::T*>(tex);
        args[1] = (void*)&tp;
        e = cudaLaunchCooperativeKernel((const void*)k_trials<TT>, dim3(blocks), dim3(ETHREADS), args, 0, st);
    });
    return e;
}

void launch_unpack_blocks(const LevelGeom& g, const float* node, const float* rhs, float* blocks, float* rhs_out,
                          cudaStream_t st)
{
    k_unpack_blocks<<<(g.G + 255) / 256, 256, 0, st>>>(g.G, node, rhs, blocks, rhs_out);
}

} // namespace sfk
