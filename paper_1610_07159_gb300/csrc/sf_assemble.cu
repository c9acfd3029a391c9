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

namespace sfk {

namespace {

constexpr int ETHREADS = 256;
constexpr int HB = NB + 6; // H_p and b_p of a pixel in shared memory (odd stride)

__constant__ int c_pair_k[NPAIR] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
__constant__ int c_pair_l[NPAIR] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};

// Data terms of one pixel at fields f (Eqs. 1-6, 11-13). Returns the
// unweighted photometric and gradient penalties; with ASSEMBLE also the
// pixel's 6x6 normal-equation block H (packed) and right-hand side b.
template <bool ASSEMBLE, class TT>
__device__ __forceinline__ void pixel_data(const typename TT::T* __restrict__ tex, int w, int h, int x, int y, const float f[6],
                                           const DevParams& P, int Wgiven, int& Wout, float& Ep, float& Eg, float* H,
                                           float* b)
{
    const size_t plane = (size_t)w * h;
    Tap tp[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float ox = sgn(c, 0) * f[0] + sgn(c, 1) * f[2] + sgn(c, 2) * f[4];
        const float oy = sgn(c, 0) * f[1] + sgn(c, 1) * f[3] + sgn(c, 2) * f[5];
        tap4<TT>(tex + c * plane, w, h, x, y, ox, oy, tp[c]);
    }
    float e[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) e[k] = tp[chk_first(k)].v[0] - tp[chk_second(k)].v[0];
    int Wi = Wgiven;
    if (Wi < 0) {
        if (P.eps_p <= 0.f) {
            Wi = 1;
        } else {
            float mx = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) mx = fmaxf(mx, fabsf(e[k]));
            Wi = mx < P.eps_p ? 1 : 0;
        }
    }
    Wout = Wi;
    Ep = 0.f;
    Eg = 0.f;
    if (ASSEMBLE) {
#pragma unroll
        for (int q = 0; q < NB; ++q) H[q] = 0.f;
#pragma unroll
        for (int q = 0; q < 6; ++q) b[q] = 0.f;
    }
    if (!Wi) return;
    const float eps2 = P.eps * P.eps;
    const bool literal = P.grad_mode == SF_GRAD_LITERAL;
    const bool irls = P.robust_mode == SF_IRLS;
    float gp[6], gg[6];
    float rho_p = 0.f, rho_g = 0.f;
    if (ASSEMBLE && !irls) {
#pragma unroll
        for (int q = 0; q < 6; ++q) gp[q] = gg[q] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int F = chk_first(k), S = chk_second(k);
        const float ph = sqrtf(fmaf(e[k], e[k], eps2));
        Ep += ph;
        const float gxk = tp[F].v[1] - tp[S].v[1], gyk = tp[F].v[2] - tp[S].v[2];
        const float q = fmaf(gxk, gxk, gyk * gyk);
        const float psi = literal ? sqrtf(fmaf(q, q, eps2)) : sqrtf(q + eps2);
        Eg += psi;
        if (ASSEMBLE) {
            float J[6];
#pragma unroll
            for (int fl = 0; fl < 3; ++fl) {
                J[2 * fl] = sgn(F, fl) * tp[F].dx[0] - sgn(S, fl) * tp[S].dx[0];
                J[2 * fl + 1] = sgn(F, fl) * tp[F].dy[0] - sgn(S, fl) * tp[S].dy[0];
            }
            // d psi / d g = coefg * g
            const float coefg = literal ? 2.f * q / psi : 1.f / psi;
            if (irls) {
                const float om = P.w_photo / (2.f * ph);
                sym_rank1(H, J, om);
#pragma unroll
                for (int r = 0; r < 6; ++r) b[r] -= om * e[k] * J[r];
            } else {
                rho_p += P.w_photo * ph;
                const float cf = P.w_photo * e[k] / ph;
#pragma unroll
                for (int r = 0; r < 6; ++r) gp[r] = fmaf(cf, J[r], gp[r]);
                rho_g += P.w_grad * psi;
            }
            const float og = 0.5f * P.w_grad * coefg;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                float Jg[6];
#pragma unroll
                for (int fl = 0; fl < 3; ++fl) {
                    Jg[2 * fl] = sgn(F, fl) * tp[F].dx[1 + a] - sgn(S, fl) * tp[S].dx[1 + a];
                    Jg[2 * fl + 1] = sgn(F, fl) * tp[F].dy[1 + a] - sgn(S, fl) * tp[S].dy[1 + a];
                }
                const float ga = a == 0 ? gxk : gyk;
                if (irls) {
                    sym_rank1(H, Jg, og);
#pragma unroll
                    for (int r = 0; r < 6; ++r) b[r] -= og * ga * Jg[r];
                } else {
                    const float cf = P.w_grad * coefg * ga;
#pragma unroll
                    for (int r = 0; r < 6; ++r) gg[r] = fmaf(cf, Jg[r], gg[r]);
                }
            }
        }
    }
    if (ASSEMBLE && !irls) {
        // one residual sqrt(rho) per pixel and term: J = grad rho / (2 sqrt rho)
#pragma unroll
        for (int r = 0; r < 6; ++r) b[r] -= 0.5f * (gp[r] + gg[r]);
        if (rho_p > 0.f) sym_rank1(H, gp, 0.25f / rho_p);
        if (rho_g > 0.f) sym_rank1(H, gg, 0.25f / rho_g);
    }
}

// Adds term(lo) .. term(hi-1) to the compensated sum (a, e): runs of SUMRUN
// terms are summed plainly and each run's sum enters with one Kahan step. A
// cell's right-hand side nearly cancels near convergence, and its blocks sum
// hundreds of pixels at the finest levels; the compensation keeps both
// accurate at a quarter of the cost of compensating every term.
constexpr int SUMRUN = 4;
template <class Term>
__device__ __forceinline__ void comp_sum(float& a, float& e, int lo, int hi, Term term)
{
    int q = lo;
    for (; q + SUMRUN <= hi; q += SUMRUN) {
        float run = term(q);
#pragma unroll
        for (int r = 1; r < SUMRUN; ++r) run += term(q + r);
        const float y = run - e;
        const float t = a + y;
        e = (t - a) - y;
        a = t;
    }
    for (; q < hi; ++q) {
        const float y = term(q) - e;
        const float t = a + y;
        e = (t - a) - y;
        a = t;
    }
}

// One CTA assembles `cpb` consecutive cells of one cell row. Pixels are
// enumerated cell-major (regular cells s x ch, the row's last cell may be
// wider), processed in chunks of ETHREADS; each thread owns up to MAXOUT of
// the cpb * CELL_VALS outputs and sums its cell's pixels of every chunk.
template <int MAXOUT, class TT>
__global__ void __launch_bounds__(ETHREADS) k_assemble(LevelGeom g, int cpb, const typename TT::T* __restrict__ tex,
                                                       const float* __restrict__ base, const float* __restrict__ delta,
                                                       DevParams P, uint8_t* __restrict__ Wmask,
                                                       float* __restrict__ cell, float2* __restrict__ part)
{
    __shared__ float sHB[ETHREADS * HB];
    __shared__ float sA[ETHREADS * 4];
    __shared__ ff sred[ETHREADS / 32];
    const int tid = threadIdx.x;
    const int s = g.s;
    const int cj = blockIdx.y, ci0 = blockIdx.x * cpb;
    const int ncell = min(cpb, g.ncx - ci0);
    const int y0 = cj * s;
    const int ch = (cj == g.ncy - 1 ? g.h : (cj + 1) * s) - y0;
    const int lastc = ci0 + ncell - 1;
    const int cw_last = (lastc == g.ncx - 1 ? g.w : (lastc + 1) * s) - lastc * s;
    const int per_reg = s * ch;
    const int total = (ncell - 1) * per_reg + cw_last * ch;
    const int nout = ncell * CELL_VALS;

    float acc[MAXOUT], cmp[MAXOUT]; // cmp: Kahan compensation of the cell sums
#pragma unroll
    for (int k = 0; k < MAXOUT; ++k) acc[k] = cmp[k] = 0.f;
    float ep = 0.f, eg = 0.f;
    int nex = 0;

    for (int c0 = 0; c0 < total; c0 += ETHREADS) {
        const int p = c0 + tid;
        float H[NB], bv[6];
        float al[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < NB; ++q) H[q] = 0.f;
#pragma unroll
        for (int q = 0; q < 6; ++q) bv[q] = 0.f;
        if (p < total) {
            const int c = min(p / per_reg, ncell - 1);
            const int q = p - c * per_reg;
            const int cw = (c == ncell - 1) ? cw_last : s;
            const int ly = q / cw, lx = q - ly * cw;
            const int x = (ci0 + c) * s + lx, y = y0 + ly;
            int i0, j0;
            float a, bb;
            grid_cell(x, y, s, g.nx, g.ny, i0, j0, a, bb);
            float f[6];
            pixel_fields(base, delta, nullptr, 0.f, g.G, j0 * g.nx + i0, g.nx, a, bb, f);
            int Wi;
            float Ep, Eg;
            pixel_data<true, TT>(tex, g.w, g.h, x, y, f, P, -1, Wi, Ep, Eg, H, bv);
            Wmask[y * g.w + x] = (uint8_t)Wi;
            ep += Ep;
            eg += Eg;
            nex += Wi ? 0 : 1;
            al[0] = (1.f - a) * (1.f - bb);
            al[1] = a * (1.f - bb);
            al[2] = (1.f - a) * bb;
            al[3] = a * bb;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) sHB[tid * HB + q] = H[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) sHB[tid * HB + NB + q] = bv[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) sA[tid * 4 + q] = al[q];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < MAXOUT; ++k) {
            const int o = tid + k * ETHREADS;
            if (o < nout) {
                const int c = o / CELL_VALS, r = o - c * CELL_VALS;
                int lo = c * per_reg, hi = (c == ncell - 1) ? total : (c + 1) * per_reg;
                lo = max(lo, c0) - c0;
                hi = min(hi, c0 + ETHREADS) - c0;
                float a = acc[k], e = cmp[k];
                if (r < NPAIR * NB) {
                    const int pr = r / NB, ee = r - pr * NB;
                    const int kk = c_pair_k[pr], ll = c_pair_l[pr];
                    comp_sum(a, e, lo, hi, [&](int q) { return sA[q * 4 + kk] * sA[q * 4 + ll] * sHB[q * HB + ee]; });
                } else {
                    const int rr = r - NPAIR * NB;
                    const int kk = rr / 6, comp = rr - kk * 6;
                    comp_sum(a, e, lo, hi, [&](int q) { return sA[q * 4 + kk] * sHB[q * HB + NB + comp]; });
                }
                cmp[k] = e;
                acc[k] = a;
            }
        }
        __syncthreads();
    }
    const int ncell_tot = g.ncx * g.ncy;
#pragma unroll
    for (int k = 0; k < MAXOUT; ++k) {
        const int o = tid + k * ETHREADS;
        if (o < nout) {
            const int c = o / CELL_VALS, r = o - c * CELL_VALS;
            cell[(size_t)r * ncell_tot + cj * g.ncx + ci0 + c] = acc[k] - cmp[k];
        }
    }
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    const ff tp = ff_block_sum_fast<ETHREADS>(ep, sred);
    const ff tg = ff_block_sum_fast<ETHREADS>(eg, sred);
    const ff tn = ff_block_sum_fast<ETHREADS>((float)nex, sred);
    if (tid == 0) {
        part[blk] = make_float2(tp.hi, tp.lo);
        part[MAX_PART + blk] = make_float2(tg.hi, tg.lo);
        part[2 * MAX_PART + blk] = make_float2(tn.hi, tn.lo);
    }
}

__device__ __forceinline__ void add_cell_pair(float* dst, const float* __restrict__ cell, int ncx, int ncy, int ci,
                                              int cj, int pr)
{
    if (ci < 0 || cj < 0 || ci >= ncx || cj >= ncy) return;
    const int nc = ncx * ncy, c = cj * ncx + ci;
#pragma unroll
    for (int e = 0; e < NB; ++e) dst[e] += __ldg(cell + (size_t)(pr * NB + e) * nc + c);
}

__device__ __forceinline__ void add_cell_rhs(float* dst, const float* __restrict__ cell, int ncx, int ncy, int ci,
                                             int cj, int corner)
{
    if (ci < 0 || cj < 0 || ci >= ncx || cj >= ncy) return;
    const int nc = ncx * ncy, c = cj * ncx + ci;
#pragma unroll
    for (int r = 0; r < 6; ++r) dst[r] += __ldg(cell + (size_t)(NPAIR * NB + corner * 6 + r) * nc + c);
}

// Epipolar residuals of one node (Eqs. 15-17) and their gradients.
__device__ __forceinline__ void epipolar(const float* Fl, float X, float Y, const float t[6], float r[2], float J[12])
{
#pragma unroll
    for (int tt = 0; tt < 2; ++tt) {
        const int il = tt == 0 ? 0 : 2, ir = tt == 0 ? 1 : 3;
        const float l0 = X + sgn(il, 0) * t[0] + sgn(il, 1) * t[2] + sgn(il, 2) * t[4];
        const float l1 = Y + sgn(il, 0) * t[1] + sgn(il, 1) * t[3] + sgn(il, 2) * t[5];
        const float r0 = X + sgn(ir, 0) * t[0] + sgn(ir, 1) * t[2] + sgn(ir, 2) * t[4];
        const float r1 = Y + sgn(ir, 0) * t[1] + sgn(ir, 1) * t[3] + sgn(ir, 2) * t[5];
        float Fr[3], Ftl[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Fr[a] = Fl[a * 3 + 0] * r0 + Fl[a * 3 + 1] * r1 + Fl[a * 3 + 2];
            Ftl[a] = Fl[0 * 3 + a] * l0 + Fl[1 * 3 + a] * l1 + Fl[2 * 3 + a];
        }
        r[tt] = l0 * Fr[0] + l1 * Fr[1] + Fr[2];
#pragma unroll
        for (int fl = 0; fl < 3; ++fl)
#pragma unroll
            for (int a = 0; a < 2; ++a) J[tt * 6 + 2 * fl + a] = sgn(il, fl) * Fr[a] + sgn(ir, fl) * Ftl[a];
    }
}

__device__ __forceinline__ void node_total(const float* __restrict__ base, const float* __restrict__ delta,
                                           const float* __restrict__ x, float t, int G, int n, float T[6], float d[6])
{
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float dd = delta[c * G + n];
        if (x) dd = fmaf(t, x[c * G + n], dd);
        d[c] = dd;
        T[c] = base[c * G + n] + dd;
    }
}

// Prior energies of one node: smoothness over its E and S edges (each
// undirected edge once, weight (w_i + w_j) w_f), epipolar, magnitude.
__device__ __forceinline__ void node_prior_energy(const LevelGeom& g, const DevParams& P, const float* __restrict__ base,
                                                  const float* __restrict__ delta, const float* __restrict__ x, float t,
                                                  const float* __restrict__ wf, int n, float& es, float& ee, float& em)
{
    const int i = n % g.nx, j = n / g.nx;
    float T[6], d[6];
    node_total(base, delta, x, t, g.G, n, T, d);
    float acc = 0.f;
    for (int nb = 0; nb < 2; ++nb) {
        const int i2 = i + (nb == 0), j2 = j + (nb == 1);
        if (i2 >= g.nx || j2 >= g.ny) continue;
        const int m = j2 * g.nx + i2;
        float Tm[6], dm[6];
        node_total(base, delta, x, t, g.G, m, Tm, dm);
        const float ww = wf[n] + wf[m];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            const float df = (base[u * g.G + n] - base[u * g.G + m]) + (d[u] - dm[u]);
            acc += ww * P.wfl[u >> 1] * df * df;
        }
    }
    es = acc;
    float r[2], J[12];
    epipolar(P.Fl, (float)(i * g.s), (float)(j * g.s), T, r, J);
    ee = r[0] * r[0] + r[1] * r[1];
    float m = 0.f;
#pragma unroll
    for (int u = 0; u < 6; ++u) m += P.mfl[u >> 1] * d[u] * d[u];
    em = m;
}

// Gather of the node system from the cell blocks plus the prior rows, the
// Jacobi preconditioner, and (last block) the energy at this point.
__global__ void __launch_bounds__(ETHREADS) k_gather(LevelGeom g, const float* __restrict__ cell,
                                                     const float* __restrict__ base, const float* __restrict__ delta,
                                                     const float* __restrict__ wf, DevParams P,
                                                     float* __restrict__ node, float* __restrict__ rhs,
                                                     float* __restrict__ minv, float2* __restrict__ gpart,
                                                     const float2* __restrict__ apart, int n_asm, unsigned* counter,
                                                     StepCtrl* __restrict__ ctrl, int* status)
{
    __shared__ ff sred[ETHREADS / 32];
    __shared__ bool last_sh;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    float es = 0.f, ee = 0.f, em = 0.f;
    if (n < g.G) {
        const int i = n % g.nx, j = n / g.nx;
        const int ncx = g.ncx, ncy = g.ncy, G = g.G;
        float Bs[NB], Be[NB], Bso[NB], Bse[NB], Bsw[NB], bb[6];
#pragma unroll
        for (int e = 0; e < NB; ++e) Bs[e] = Be[e] = Bso[e] = Bse[e] = Bsw[e] = 0.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) bb[r] = 0.f;
        // corners: 0 (ci,cj), 1 (ci+1,cj), 2 (ci,cj+1), 3 (ci+1,cj+1)
        add_cell_pair(Bs, cell, ncx, ncy, i - 1, j - 1, pair_idx(3, 3));
        add_cell_pair(Bs, cell, ncx, ncy, i, j - 1, pair_idx(2, 2));
        add_cell_pair(Bs, cell, ncx, ncy, i - 1, j, pair_idx(1, 1));
        add_cell_pair(Bs, cell, ncx, ncy, i, j, pair_idx(0, 0));
        add_cell_pair(Be, cell, ncx, ncy, i, j - 1, pair_idx(2, 3));
        add_cell_pair(Be, cell, ncx, ncy, i, j, pair_idx(0, 1));
        add_cell_pair(Bso, cell, ncx, ncy, i - 1, j, pair_idx(1, 3));
        add_cell_pair(Bso, cell, ncx, ncy, i, j, pair_idx(0, 2));
        add_cell_pair(Bse, cell, ncx, ncy, i, j, pair_idx(0, 3));
        add_cell_pair(Bsw, cell, ncx, ncy, i - 1, j, pair_idx(1, 2));
        add_cell_rhs(bb, cell, ncx, ncy, i - 1, j - 1, 3);
        add_cell_rhs(bb, cell, ncx, ncy, i, j - 1, 2);
        add_cell_rhs(bb, cell, ncx, ncy, i - 1, j, 1);
        add_cell_rhs(bb, cell, ncx, ncy, i, j, 0);

        float T[6], d[6];
        node_total(base, delta, nullptr, 0.f, G, n, T, d);
        const float wn = wf[n];
        // smoothness (Eq. 14): every 4-neighbour edge, both directed pairs
        const int nbi[4] = {i + 1, i, i - 1, i};
        const int nbj[4] = {j, j + 1, j, j - 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (nbi[q] < 0 || nbj[q] < 0 || nbi[q] >= g.nx || nbj[q] >= g.ny) continue;
            const int m = nbj[q] * g.nx + nbi[q];
            const float ww = P.w_reg * P.w_smooth * (wn + wf[m]);
            float Tm[6], dm[6];
            node_total(base, delta, nullptr, 0.f, G, m, Tm, dm);
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                const float c = ww * P.wfl[u >> 1];
                // T_n - T_m as (base difference) + (delta difference): no cancellation of the large totals
                const float df = (base[u * g.G + n] - base[u * g.G + m]) + (d[u] - dm[u]);
                Bs[sym_idx(u, u)] += c;
                bb[u] -= c * df;
                if (q == 0) Be[sym_idx(u, u)] -= c;
                if (q == 1) Bso[sym_idx(u, u)] -= c;
            }
        }
        // epipolar (Eqs. 15-17)
        {
            float r[2], J[12];
            epipolar(P.Fl, (float)(i * g.s), (float)(j * g.s), T, r, J);
            const float ce = P.w_reg * P.w_epi;
            if (ce != 0.f) {
                sym_rank1(Bs, J, ce);
                sym_rank1(Bs, J + 6, ce);
#pragma unroll
                for (int u = 0; u < 6; ++u) bb[u] -= ce * (r[0] * J[u] + r[1] * J[6 + u]);
            }
        }
        // magnitude (Eq. 18) on the delta
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            const float cm = P.w_reg * P.w_mag * P.mfl[u >> 1];
            Bs[sym_idx(u, u)] += cm;
            bb[u] -= cm * d[u];
        }
#pragma unroll
        for (int e = 0; e < NB; ++e) {
            node[(size_t)(0 * NB + e) * G + n] = Bs[e];
            node[(size_t)(1 * NB + e) * G + n] = Be[e];
            node[(size_t)(2 * NB + e) * G + n] = Bso[e];
            node[(size_t)(3 * NB + e) * G + n] = Bse[e];
            node[(size_t)(4 * NB + e) * G + n] = Bsw[e];
        }
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            rhs[u * G + n] = bb[u];
            const float dg = Bs[sym_idx(u, u)];
            minv[u * G + n] = dg > 0.f ? 1.f / dg : 1.f;
        }
        node_prior_energy(g, P, base, delta, nullptr, 0.f, wf, n, es, ee, em);
    }
    if (!ctrl) return;
    const ff ts = ff_block_sum_fast<ETHREADS>(es, sred);
    const ff te = ff_block_sum_fast<ETHREADS>(ee, sred);
    const ff tm = ff_block_sum_fast<ETHREADS>(em, sred);
    if (threadIdx.x == 0) {
        gpart[blockIdx.x] = make_float2(ts.hi, ts.lo);
        gpart[MAX_PART + blockIdx.x] = make_float2(te.hi, te.lo);
        gpart[2 * MAX_PART + blockIdx.x] = make_float2(tm.hi, tm.lo);
        __threadfence();
        const unsigned done = atomicAdd(counter, 1u);
        last_sh = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_sh) return;
    __threadfence();
    {
        const ff fp = ff_block_fixed_sum<ETHREADS>(apart, n_asm, sred);
        const ff fg = ff_block_fixed_sum<ETHREADS>(apart + MAX_PART, n_asm, sred);
        const ff fx = ff_block_fixed_sum<ETHREADS>(apart + 2 * MAX_PART, n_asm, sred);
        const ff fs = ff_block_fixed_sum<ETHREADS>(gpart, gridDim.x, sred);
        const ff fe = ff_block_fixed_sum<ETHREADS>(gpart + MAX_PART, gridDim.x, sred);
        const ff fm = ff_block_fixed_sum<ETHREADS>(gpart + 2 * MAX_PART, gridDim.x, sred);
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
// the last block to finish sums the partials in a fixed order and either
// writes the record or takes the backtracking decision.
template <class TT>
__global__ void __launch_bounds__(ETHREADS) k_energy(LevelGeom g, int npixblk, const typename TT::T* __restrict__ tex,
                                                     const float* __restrict__ base, const float* __restrict__ delta,
                                                     const float* __restrict__ x, float t, const float* __restrict__ wf,
                                                     DevParams P, uint8_t* __restrict__ Wmask, int wmode,
                                                     float2* __restrict__ part, unsigned* counter,
                                                     StepCtrl* __restrict__ ctrl, int action, int last,
                                                     double* __restrict__ rec, int* status)
{
    __shared__ ff sred[ETHREADS / 32];
    __shared__ bool last_sh;
    if (action == 1 && ld_acquire_s32(&ctrl->accepted)) return;
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
            pixel_data<false, TT>(tex, g.w, g.h, xx, y, f, P, wmode ? -1 : (int)Wmask[p], Wi, Ep, Eg, nullptr, nullptr);
            if (wmode) Wmask[p] = (uint8_t)Wi;
            v[0] += Ep;
            v[1] += Eg;
            v[5] += Wi ? 0.f : 1.f;
        }
    } else {
        const int n = (blockIdx.x - npixblk) * ETHREADS + threadIdx.x;
        if (n < g.G) node_prior_energy(g, P, base, delta, x, t, wf, n, v[2], v[3], v[4]);
    }
    for (int q = 0; q < 6; ++q) {
        const ff sq = ff_block_sum_fast<ETHREADS>(v[q], sred);
        if (threadIdx.x == 0) part[q * MAX_PART + blockIdx.x] = make_float2(sq.hi, sq.lo);
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
        double s[6];
        for (int q = 0; q < 6; ++q) {
            const ff t = ff_block_fixed_sum<ETHREADS>(part + q * MAX_PART, gridDim.x, sred);
            s[q] = (double)t.hi + t.lo;
        }
        if (threadIdx.x == 0) {
            double terms[5];
            terms[0] = P.w_photo * s[0];
            terms[1] = P.w_grad * s[1];
            terms[2] = (double)P.w_reg * P.w_smooth * s[2];
            terms[3] = (double)P.w_reg * P.w_epi * s[3];
            terms[4] = (double)P.w_reg * P.w_mag * s[4];
            const double E = terms[0] + terms[1] + terms[2] + terms[3] + terms[4];
            if (action == 0) {
                rec[0] = E;
                for (int q = 0; q < 5; ++q) rec[1 + q] = terms[q];
                rec[6] = s[5];
            } else {
                if (E <= ctrl->E_cur) {
                    ctrl->E_acc = E;
                    for (int q = 0; q < 5; ++q) ctrl->terms_acc[q] = terms[q];
                    ctrl->t = t;
                    __threadfence();
                    atomicExch(&ctrl->accepted, 1);
                } else if (last) {
                    ctrl->t = 0.f; // rejected: keep delta, E_acc stays E_cur
                }
            }
            if (!isfinite(E) && action == 0) atomicOr(status, DEV_NUMERIC);
            __threadfence();
            *counter = 0u;
        }
    }
}

__global__ void k_apply_step(int n6, float* __restrict__ delta, const float* __restrict__ x,
                             const StepCtrl* __restrict__ ctrl)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n6 || !ctrl->accepted) return;
    delta[k] = fmaf(ctrl->t, x[k], delta[k]);
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

template <int MAXOUT>
void assemble_impl(const LevelGeom& g, int cpb, const void* tex, int prec, const float* base, const float* delta,
                   const DevParams& P, uint8_t* Wmask, float* cell, float2* part, cudaStream_t st)
{
    dim3 grid((g.ncx + cpb - 1) / cpb, g.ncy);
    SF_TEX_DISPATCH(prec, TT, k_assemble<MAXOUT, TT><<<grid, ETHREADS, 0, st>>>(
                                  g, cpb, static_cast<const typename TT::T*>(tex), base, delta, P, Wmask, cell, part));
}

} // namespace

int assemble_blocks(const LevelGeom& g, int* cpb_out)
{
    int cpb = ETHREADS / (g.s * g.s);
    if (cpb < 1) cpb = 1;
    while (cpb * CELL_VALS > 16 * ETHREADS) --cpb;
    if (cpb_out) *cpb_out = cpb;
    return ((g.ncx + cpb - 1) / cpb) * g.ncy;
}

void launch_assemble(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta,
                     const DevParams& P, uint8_t* Wmask, float* cell, const Scratch& sc, cudaStream_t st)
{
    int cpb;
    assemble_blocks(g, &cpb);
    const int need = (cpb * CELL_VALS + ETHREADS - 1) / ETHREADS;
    if (need <= 1)
        assemble_impl<1>(g, cpb, tex, prec, base, delta, P, Wmask, cell, sc.asm_part, st);
    else if (need <= 2)
        assemble_impl<2>(g, cpb, tex, prec, base, delta, P, Wmask, cell, sc.asm_part, st);
    else if (need <= 4)
        assemble_impl<4>(g, cpb, tex, prec, base, delta, P, Wmask, cell, sc.asm_part, st);
    else if (need <= 8)
        assemble_impl<8>(g, cpb, tex, prec, base, delta, P, Wmask, cell, sc.asm_part, st);
    else
        assemble_impl<16>(g, cpb, tex, prec, base, delta, P, Wmask, cell, sc.asm_part, st);
}

void launch_gather(const LevelGeom& g, const float* cell, const float* base, const float* delta, const float* wf,
                   const DevParams& P, float* node, float* rhs, float* minv, const Scratch& sc, StepCtrl* ctrl,
                   int n_asm_blocks, cudaStream_t st)
{
    const int blocks = (g.G + ETHREADS - 1) / ETHREADS;
    k_gather<<<blocks, ETHREADS, 0, st>>>(g, cell, base, delta, wf, P, node, rhs, minv, sc.gat_part, sc.asm_part,
                                          n_asm_blocks, sc.counters + 0, ctrl, sc.status);
}

void launch_energy(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta, const float* x,
                   float t, const float* wf, const DevParams& P, uint8_t* Wmask, int wmode, const Scratch& sc,
                   StepCtrl* ctrl, int action, int last, double* rec, cudaStream_t st)
{
    int npix = (g.w * g.h + ETHREADS - 1) / ETHREADS;
    if (npix > 152 * 8) npix = 152 * 8;
    const int nnode = (g.G + ETHREADS - 1) / ETHREADS;
    SF_TEX_DISPATCH(prec, TT, k_energy<TT><<<npix + nnode, ETHREADS, 0, st>>>(
                                  g, npix, static_cast<const typename TT::T*>(tex), base, delta, x, t, wf, P, Wmask,
                                  wmode, sc.en_part, sc.counters + 1, ctrl, action, last, rec, sc.status));
}

void launch_apply_step(const LevelGeom& g, float* delta, const float* x, const StepCtrl* ctrl, cudaStream_t st)
{
    const int n6 = 6 * g.G;
    k_apply_step<<<(n6 + 255) / 256, 256, 0, st>>>(n6, delta, x, ctrl);
}

void launch_unpack_blocks(const LevelGeom& g, const float* node, const float* rhs, float* blocks, float* rhs_out,
                          cudaStream_t st)
{
    k_unpack_blocks<<<(g.G + 255) / 256, 256, 0, st>>>(g.G, node, rhs, blocks, rhs_out);
}

} // namespace sfk
