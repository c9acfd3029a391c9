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
//     epipolar (Eqs. 15-17) and magnitude (Eq. 18) rows (entry-parallel), the
//     right-hand side, the Jacobi preconditioner and the energy at the
//     linearisation point (component-parallel);
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

// Row and column (r <= c) of entry e of a packed symmetric 6x6 block.
__constant__ unsigned char c_sym_r[NB] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
__constant__ unsigned char c_sym_c[NB] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};

__device__ __forceinline__ float cell_entry(const float* __restrict__ cell, int ncx, int ncy, int ci, int cj, int v)
{
    if (ci < 0 || cj < 0 || ci >= ncx || cj >= ncy) return 0.f;
    return __ldg(cell + (size_t)v * ncx * ncy + cj * ncx + ci);
}

// Entry v = b * 21 + e of node n of the Gauss-Newton system (k_gather runs
// one thread per (entry, node)): the sum of its cells' pair blocks (the
// chain rule of Eq. 7), plus for the node's own block the smoothness
// (Eq. 14), epipolar (Eqs. 15-17) and magnitude (Eq. 18) rows and for the E
// and S blocks the smoothness coupling, added in the order gather_node4
// adds them, so the values are the same bit for bit. Entry-parallel: every
// thread has a few independent loads, where a node-parallel gather waits on
// long chains of them.
__device__ __forceinline__ float node_value(const LevelGeom& g, const float* __restrict__ cell,
                                            const float* __restrict__ base, const float* __restrict__ delta,
                                            const float* __restrict__ wf, const DevParams& P, int v, int n)
{
    const int b = v / NB, e = v - b * NB;
    const int i = n % g.nx, j = n / g.nx;
    const int ncx = g.ncx, ncy = g.ncy;
    const int r = c_sym_r[e], c = c_sym_c[e];
    const bool diag = r == c;
    float acc = 0.f;
    if (b == 0) {
        acc += cell_entry(cell, ncx, ncy, i - 1, j - 1, pair_idx(3, 3) * NB + e);
        acc += cell_entry(cell, ncx, ncy, i, j - 1, pair_idx(2, 2) * NB + e);
        acc += cell_entry(cell, ncx, ncy, i - 1, j, pair_idx(1, 1) * NB + e);
        acc += cell_entry(cell, ncx, ncy, i, j, pair_idx(0, 0) * NB + e);
        const float wn = wf[n];
        if (diag) {
            const int nbi[4] = {i + 1, i, i - 1, i};
            const int nbj[4] = {j, j + 1, j, j - 1};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (nbi[q] < 0 || nbj[q] < 0 || nbi[q] >= g.nx || nbj[q] >= g.ny) continue;
                const float ww = P.w_reg * P.w_smooth * (wn + wf[nbj[q] * g.nx + nbi[q]]);
                acc += ww * P.wfl[r >> 1];
            }
        }
        const float ce = P.w_reg * P.w_epi;
        if (ce != 0.f) {
            float T[6], d[6], rr[2], J[12];
            node_total(base, delta, nullptr, 0.f, g.G, n, T, d);
            epipolar(P.Fl, (float)(i * g.s), (float)(j * g.s), T, rr, J);
            acc = fmaf(ce * J[r], J[c], acc);
            acc = fmaf(ce * J[6 + r], J[6 + c], acc);
        }
        if (diag) acc += P.w_reg * P.w_mag * P.mfl[r >> 1];
    } else if (b == 1 || b == 2) {
        if (b == 1) {
            acc += cell_entry(cell, ncx, ncy, i, j - 1, pair_idx(2, 3) * NB + e);
            acc += cell_entry(cell, ncx, ncy, i, j, pair_idx(0, 1) * NB + e);
        } else {
            acc += cell_entry(cell, ncx, ncy, i - 1, j, pair_idx(1, 3) * NB + e);
            acc += cell_entry(cell, ncx, ncy, i, j, pair_idx(0, 2) * NB + e);
        }
        const int mi = b == 1 ? i + 1 : i, mj = b == 1 ? j : j + 1;
        if (diag && mi < g.nx && mj < g.ny) {
            const float ww = P.w_reg * P.w_smooth * (wf[n] + wf[mj * g.nx + mi]);
            acc -= ww * P.wfl[r >> 1];
        }
    } else if (b == 3) {
        acc += cell_entry(cell, ncx, ncy, i, j, pair_idx(0, 3) * NB + e);
    } else {
        acc += cell_entry(cell, ncx, ncy, i - 1, j, pair_idx(1, 2) * NB + e);
    }
    return acc;
}

// The node system in one launch of two kinds of blocks. The first nrhs
// blocks: the right-hand side and Jacobi preconditioner, one thread per
// (component, node) (the cells' part of b plus the prior rows, in
// gather_node4's order; the diagonal entry for the preconditioner formed by
// node_value, as the block threads form it), and the prior energies at the
// linearisation point (the thread of component 0); the last of them to
// finish forms the step's record from the assembly's and these partials in a
// fixed order. The rest: the node blocks, one thread per (entry, node).
__global__ void __launch_bounds__(ETHREADS) k_gather(LevelGeom g, int nrhs, const float* __restrict__ cell,
                                                     const float* __restrict__ base, const float* __restrict__ delta,
                                                     const float* __restrict__ wf, DevParams P,
                                                     float* __restrict__ node, float* __restrict__ rhs,
                                                     float* __restrict__ minv, float2* __restrict__ gpart,
                                                     const float2* __restrict__ apart, int n_asm, unsigned* counter,
                                                     StepCtrl* __restrict__ ctrl, int* status)
{
    __shared__ ff sred[6 * (ETHREADS / 32)];
    __shared__ bool last_sh;
    const int G = g.G;
    if ((int)blockIdx.x >= nrhs) {
        const int tb = ((int)blockIdx.x - nrhs) * ETHREADS + threadIdx.x;
        if (tb >= NODE_VALS * G) return;
        const int v = tb / G, n = tb - v * G;
        node[tb] = node_value(g, cell, base, delta, wf, P, v, n);
        return;
    }
    const int t = blockIdx.x * ETHREADS + threadIdx.x;
    float es = 0.f, ee = 0.f, em = 0.f;
    if (t < 6 * G) {
        const int u = t / G, n = t - u * G;
        const int i = n % g.nx, j = n / g.nx;
        const int ncx = g.ncx, ncy = g.ncy;
        const int rc = NPAIR * NB + u; // component u of corner k's rhs at rc + 6 k
        float bb = 0.f;
        bb += cell_entry(cell, ncx, ncy, i - 1, j - 1, rc + 6 * 3);
        bb += cell_entry(cell, ncx, ncy, i, j - 1, rc + 6 * 2);
        bb += cell_entry(cell, ncx, ncy, i - 1, j, rc + 6 * 1);
        bb += cell_entry(cell, ncx, ncy, i, j, rc + 6 * 0);
        const float du = delta[u * G + n];
        const float wn = wf[n];
        const int nbi[4] = {i + 1, i, i - 1, i};
        const int nbj[4] = {j, j + 1, j, j - 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (nbi[q] < 0 || nbj[q] < 0 || nbi[q] >= g.nx || nbj[q] >= g.ny) continue;
            const int m = nbj[q] * g.nx + nbi[q];
            const float ww = P.w_reg * P.w_smooth * (wn + wf[m]);
            const float cf = ww * P.wfl[u >> 1];
            const float df = (base[u * G + n] - base[u * G + m]) + (du - delta[u * G + m]);
            bb -= cf * df;
        }
        const float ce = P.w_reg * P.w_epi;
        if (ce != 0.f) {
            float T[6], d[6], r[2], J[12];
            node_total(base, delta, nullptr, 0.f, G, n, T, d);
            epipolar(P.Fl, (float)(i * g.s), (float)(j * g.s), T, r, J);
            bb -= ce * (r[0] * J[u] + r[1] * J[6 + u]);
        }
        bb -= P.w_reg * P.w_mag * P.mfl[u >> 1] * du;
        rhs[u * G + n] = bb;
        const float dg = node_value(g, cell, base, delta, wf, P, sym_idx(u, u), n);
        minv[u * G + n] = dg > 0.f ? 1.f / dg : 1.f;
        if (u == 0) node_prior_energy(g, P, base, delta, nullptr, 0.f, wf, n, es, ee, em);
    }
    if (!ctrl) return;
    const float v[3] = {es, ee, em};
    ff tb[3];
    ff_block_sum_fast_n<ETHREADS, 3>(v, sred, tb);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) gpart[q * MAX_PART + blockIdx.x] = make_float2(tb[q].hi, tb[q].lo);
        last_sh = atom_add_release_gpu(counter, 1u) == (unsigned)nrhs - 1;
    }
    __syncthreads();
    if (!last_sh) return;
    fence_acquire_gpu_fold();
    {
        const float2* const parts[6] = {apart, apart + MAX_PART, apart + 2 * MAX_PART,
                                        gpart, gpart + MAX_PART, gpart + 2 * MAX_PART};
        const int nb = nrhs;
        const int cnt[6] = {n_asm, n_asm, n_asm, nb, nb, nb};
        ff f[6];
        ff_block_fixed_sum_n<ETHREADS, 6>(parts, cnt, sred, f);
        const ff fp = f[0], fg = f[1], fx = f[2], fs = f[3], fe = f[4], fm = f[5];
        const double sp = (double)fp.hi + fp.lo, sg = (double)fg.hi + fg.lo, sx = (double)fx.hi + fx.lo;
        const double ss = (double)fs.hi + fs.lo, se = (double)fe.hi + fe.lo, sm = (double)fm.hi + fm.lo;
        if (threadIdx.x == 0) {
            StepCtrl cr;
            cr.terms_cur[0] = P.w_photo * sp;
            cr.terms_cur[1] = P.w_grad * sg;
            cr.terms_cur[2] = (double)P.w_reg * P.w_smooth * ss;
            cr.terms_cur[3] = (double)P.w_reg * P.w_epi * se;
            cr.terms_cur[4] = (double)P.w_reg * P.w_mag * sm;
            cr.E_cur = cr.terms_cur[0] + cr.terms_cur[1] + cr.terms_cur[2] + cr.terms_cur[3] + cr.terms_cur[4];
            cr.E_acc = cr.E_cur;
            for (int q = 0; q < 5; ++q) cr.terms_acc[q] = cr.terms_cur[q];
            cr.t = 0.f;
            cr.accepted = 0;
            cr.n_excluded = (int)sx;
            cr.t1_ok = 0;
            cr.E_t1 = cr.E_cur;
            for (int q = 0; q < 5; ++q) cr.terms_t1[q] = cr.terms_cur[q];
            *ctrl = cr;
            if (!isfinite(cr.E_cur)) atomicOr(status, DEV_NUMERIC);
            *counter = 0u; // the next launch (a later kernel) sees it
        }
    }
}

// Energy at base + delta (+ t x): pixel blocks first, then node blocks;
// the last block to finish sums the partials in a fixed order and writes the
// record (energy, the five weighted terms, excluded pixels). TRIAL: the first
// trial of a Gauss-Newton step (t = 1, W of the step): the last block writes
// the energy and terms into the step's control record instead and whether
// the step passes (E <= E_cur); a non-finite energy fails the trial, as in
// k_trials, without raising an error.
template <class TT, bool TRIAL = false>
__global__ void __launch_bounds__(ETHREADS) k_energy(LevelGeom g, int npixblk, const typename TT::T* __restrict__ tex,
                                                     const float* __restrict__ base, const float* __restrict__ delta,
                                                     const float* __restrict__ x, float t, const float* __restrict__ wf,
                                                     DevParams P, LevelMaps M, uint8_t* __restrict__ Wmask, int wmode,
                                                     float2* __restrict__ part, unsigned* counter,
                                                     double* __restrict__ rec, int* status, StepCtrl* ctrl = nullptr)
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
    if (threadIdx.x == 0) last_sh = atom_add_release_gpu(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_sh) return;
    fence_acquire_gpu_fold();
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
            if (TRIAL) {
                ctrl->E_t1 = E;
                for (int q = 0; q < 5; ++q) ctrl->terms_t1[q] = terms[q];
                ctrl->t1_ok = E <= ctrl->E_cur ? 1 : 0;
            } else {
                rec[0] = E;
                for (int q = 0; q < 5; ++q) rec[1 + q] = terms[q];
                rec[6] = s[5];
                if (!isfinite(E)) atomicOr(status, DEV_NUMERIC);
            }
            *counter = 0u; // the next launch (a later kernel) sees it
        }
    }
}

// The backtracking trials of one Gauss-Newton step and the update in one
// cooperative launch. The full step (t = 1) was tried by k_energy in trial
// mode just before (one pixel per thread over the whole GPU, its verdict in
// the control record); when it passed, every block applies it (delta += x)
// with no barrier. Otherwise, for t = 1/2, 1/4, ... every block sums its
// share of the pixel and node energies at delta + t x (W of the step), a
// bounded grid barrier, then warp 0 of every block forms the fixed-order
// totals, so all blocks take the same decision; the first t whose energy does
// not exceed E_cur is taken and applied. Replaces max_backtracks + 1 trial
// launches, most of which found the step already taken, and the update launch.
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
    float t = 0.5f, t_acc = 0.f;
    double E_acc = E_cur, terms_acc[5];
    for (int q = 0; q < 5; ++q) terms_acc[q] = ctrl->terms_cur[q];
    bool ok = true;
    if (ctrl->t1_ok) {
        t_acc = 1.f;
        E_acc = ctrl->E_t1;
        for (int q = 0; q < 5; ++q) terms_acc[q] = ctrl->terms_t1[q];
        max_bt = 0; // no backtracking
    }
    for (int j = 1; j <= max_bt && ok; ++j, t *= 0.5f) {
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
    // one launch: the right-hand side, preconditioner and energy component by component, beside the node blocks
    // entry by entry
    const int rblocks = (6 * g.G + ETHREADS - 1) / ETHREADS;
    const int bblocks = (NODE_VALS * g.G + ETHREADS - 1) / ETHREADS;
    k_gather<<<rblocks + bblocks, ETHREADS, 0, st>>>(g, rblocks, cell, base, delta, wf, P, node, rhs, minv,
                                                     sc.gat_part, sc.asm_part, n_asm_blocks, sc.counters + 0, ctrl,
                                                     sc.status);
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
    // the full step first: one pixel per thread, the verdict into the control record
    {
        // one pixel per thread while that is at most four blocks per SM of a
        // GB300; two beyond (half the partials for the last block to fold:
        // measured at 640x480 level 0 23 -> 19 us, while the small levels
        // lose at two)
        int npix = (g.w * g.h + ETHREADS - 1) / ETHREADS;
        if (npix > 152 * 4) npix = (g.w * g.h + 2 * ETHREADS - 1) / (2 * ETHREADS);
        if (npix > 152 * 8) npix = 152 * 8; // larger levels loop (the partial slots and the last block's fold)
        const int nnode = (g.G + ETHREADS - 1) / ETHREADS;
        SF_TEX_DISPATCH(prec, TT, (k_energy<TT, true><<<npix + nnode, ETHREADS, 0, st>>>(
                                      g, npix, static_cast<const typename TT::T*>(tex), base, delta, x, 1.f, wf, P, M,
                                      const_cast<uint8_t*>(Wmask), 0, sc.en_part, sc.counters + 2, nullptr,
                                      sc.status, ctrl)));
        const cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
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
