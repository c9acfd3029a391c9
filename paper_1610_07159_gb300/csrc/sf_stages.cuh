// sf_stages.cuh -- per-element stages of the Gauss-Newton linearisation
// (Thies et al., arXiv 1610.07159, Section 5.1), shared by the per-level
// kernels and the batched frame kernel:
//   * pixel_data: the six consistency checks of Eqs. 1-6 on bilinear samples
//     of intensity and gradient, the outlier weight W (Section 4.1), the
//     robust pseudo-Huber terms of Eqs. 11-13 and their reweighted
//     normal-equation contributions H_p, b_p;
//   * assemble_group: per warp-grid cell, sum_p alpha_k alpha_l H_p and
//     sum_p alpha_k b_p (the chain rule through the bilinear weights of
//     Eq. 7), reduced in shared memory;
//   * gather_node: the node system from the cell blocks plus the smoothness
//     (Eq. 14), epipolar (Eqs. 15-17) and magnitude (Eq. 18) rows;
//   * node_prior_energy: the prior energies of one node.
#pragma once

#include "sf_common.cuh"

namespace sfk {

namespace {

constexpr int ETHREADS = 256;
constexpr int HB = NB + 6; // H_p and b_p of a pixel in shared memory (odd stride)

__constant__ int c_pair_k[NPAIR] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
__constant__ int c_pair_l[NPAIR] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};

// Data terms of one pixel at fields f (Eqs. 1-6, 11-13). Returns the
// unweighted photometric and gradient penalties; with ASSEMBLE also the
// pixel's 6x6 normal-equation block H (packed) and right-hand side b.
template <bool ASSEMBLE, class TT, bool REC = false>
__device__ __forceinline__ void pixel_data(const typename TT::T* __restrict__ tex, int w, int h, int x, int y, const float f[6],
                                           const DevParams& P, const LevelMaps& M, int Wgiven, int& Wout, float& Ep,
                                           float& Eg, float* H, float* b, const CellLog* log = nullptr)
{
    const size_t plane = (size_t)w * h;
    Tap tp[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float ox = sgn(c, 0) * f[0] + sgn(c, 1) * f[2] + sgn(c, 2) * f[4];
        const float oy = sgn(c, 0) * f[1] + sgn(c, 1) * f[3] + sgn(c, 2) * f[5];
        tap4<TT, REC>(tex + c * plane, w, h, x, y, ox, oy, tp[c], log, c);
    }
    const int pix = y * w + x;
    if (M.L) {
        // illumination correction: the right images (1 at time 0, 3 at time 1) less the right camera's
        // difference at this pixel (a constant of the level: the Jacobian keeps)
        tp[1].v[0] -= __ldg(M.L + pix);
        tp[3].v[0] -= __ldg(M.L + plane + pix);
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
    if (M.V && !__ldg(M.V + pix)) return; // occluded in a view: V = 0 in Eqs. 11 and 13
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

// Cell reduction tasks. Per cell, 48 task kinds: kind 2e + h (e < 21) sums
// entry e of H_p against the pair weights alpha_k alpha_l of pairs
// 5h .. 5h + 4; kind 42 + c sums component c of b_p against the four corner
// weights alpha_k. A task may cover only part `p` of P contiguous parts of
// its cell's pixels; the parts meet at the end in a fixed order.
constexpr int TASK_KINDS = 48;
// per-pixel weight row in shared memory (16 floats, 16-byte aligned):
// [0..3] pairs 0-3, [4..7] pairs 5-8, [8..11] corners 0-3, [12] pair 4, [13] pair 9
constexpr int WROW = 16;

__host__ __device__ constexpr int assemble_parts(int cpb) { return cpb * TASK_KINDS >= ETHREADS ? 1 : ETHREADS / (cpb * TASK_KINDS); }
__host__ __device__ constexpr int assemble_tasks_per_thread(int cpb)
{
    return (cpb * TASK_KINDS * assemble_parts(cpb) + ETHREADS - 1) / ETHREADS;
}

// Compensated sums of n = 5 (H) or 4 (b) outputs over pixels [qa, qb):
// runs of SUMRUN pixels are summed plainly, each run enters with one Kahan
// step per output (the same scheme as comp_sum).
template <int N>
__device__ __forceinline__ void task_term(float* run, bool first, const float* sHB, int q, int hoff, const float* sW,
                                          int w4, int w1)
{
    const float h = sHB[q * HB + hoff];
    const float4 w = *reinterpret_cast<const float4*>(sW + q * WROW + w4);
    const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) run[i] = first ? wv[i] * h : fmaf(wv[i], h, run[i]);
    if (N == 5) {
        const float w5 = sW[q * WROW + w1];
        run[N - 1] = first ? w5 * h : fmaf(w5, h, run[N - 1]);
    }
}

template <int N>
__device__ __forceinline__ void kahan_add(float* a, float* e, const float* run)
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float y = run[i] - e[i];
        const float t = a[i] + y;
        e[i] = (t - a[i]) - y;
        a[i] = t;
    }
}

template <int N>
__device__ __forceinline__ void task_sum(float* a, float* e, int qa, int qb, const float* sHB, int hoff,
                                         const float* sW, int w4, int w1)
{
    float run[N];
    int q = qa;
    for (; q + SUMRUN <= qb; q += SUMRUN) {
#pragma unroll
        for (int r = 0; r < SUMRUN; ++r) task_term<N>(run, r == 0, sHB, q + r, hoff, sW, w4, w1);
        kahan_add<N>(a, e, run);
    }
    for (; q < qb; ++q) {
        task_term<N>(run, true, sHB, q, hoff, sW, w4, w1);
        kahan_add<N>(a, e, run);
    }
}

// Assembles the cells of one group: `cpb` consecutive cells of cell row
// `by`, starting at cell bx * cpb. Pixels are enumerated cell-major (regular
// cells s x ch, the row's last cell may be wider) and processed in chunks of
// ETHREADS: one pixel per thread computes H_p, b_p and its bilinear weights
// into shared memory, then each thread runs up to MAXT reduction tasks
// (above) over its cell's pixels of the chunk, five (or four) outputs at a
// time from one load of the H_p (b_p) entry and one row of weights. The
// pixel energies and the count of excluded pixels are added to the thread's
// ep, eg, nex. sHB and sW are ETHREADS * HB and ETHREADS * WROW floats of
// shared memory (sW 16-byte aligned).
template <int MAXT, class TT, bool REC = false>
__device__ __forceinline__ void assemble_group(const LevelGeom& g, int cpb, int bx, int by,
                                               const typename TT::T* __restrict__ tex, const float* base,
                                               const float* delta, const DevParams& P, const LevelMaps& M,
                                               uint8_t* Wmask, float* cell, float* sHB,
                                               float* sW, float& ep, float& eg, int& nex,
                                               const CellLog* log = nullptr)
{
    const int tid = threadIdx.x;
    const int s = g.s;
    const int cj = by, ci0 = bx * cpb;
    const int ncell = min(cpb, g.ncx - ci0);
    const int y0 = cj * s;
    const int ch = (cj == g.ncy - 1 ? g.h : (cj + 1) * s) - y0;
    const int lastc = ci0 + ncell - 1;
    const int cw_last = (lastc == g.ncx - 1 ? g.w : (lastc + 1) * s) - lastc * s;
    const int per_reg = s * ch;
    const int total = (ncell - 1) * per_reg + cw_last * ch;
    const int NP = assemble_parts(cpb);
    const int ntask = ncell * TASK_KINDS * NP;

    float acc[MAXT][5], cmp[MAXT][5]; // cmp: Kahan compensation of the cell sums
#pragma unroll
    for (int j = 0; j < MAXT; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) acc[j][i] = cmp[j][i] = 0.f;

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
            pixel_data<true, TT, REC>(tex, g.w, g.h, x, y, f, P, M, -1, Wi, Ep, Eg, H, bv, log);
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
        {
            float* wr = sW + tid * WROW;
            *reinterpret_cast<float4*>(wr) = make_float4(al[0] * al[0], al[0] * al[1], al[0] * al[2], al[0] * al[3]);
            *reinterpret_cast<float4*>(wr + 4) = make_float4(al[1] * al[2], al[1] * al[3], al[2] * al[2], al[2] * al[3]);
            *reinterpret_cast<float4*>(wr + 8) = make_float4(al[0], al[1], al[2], al[3]);
            wr[12] = al[1] * al[1];
            wr[13] = al[3] * al[3];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < MAXT; ++j) {
            const int t = tid + j * ETHREADS;
            if (t < ntask) {
                const int part = t % NP, r = t / NP, kind = r % TASK_KINDS, c = r / TASK_KINDS;
                int lo = c * per_reg, hi = (c == ncell - 1) ? total : (c + 1) * per_reg;
                lo = max(lo, c0) - c0;
                hi = min(hi, c0 + ETHREADS) - c0;
                if (hi > lo) {
                    const int qa = lo + (hi - lo) * part / NP, qb = lo + (hi - lo) * (part + 1) / NP;
                    if (kind < 2 * NB) {
                        const int half = kind & 1;
                        task_sum<5>(acc[j], cmp[j], qa, qb, sHB, kind >> 1, sW, half ? 4 : 0, half ? 13 : 12);
                    } else {
                        task_sum<4>(acc[j], cmp[j], qa, qb, sHB, NB + kind - 2 * NB, sW, 8, 0);
                    }
                }
            }
        }
        __syncthreads();
    }
    // outputs: r < 210 is entry ee of pair pr (r = pr * 21 + ee), r >= 210
    // component comp of corner k (r = 210 + k * 6 + comp)
    const int ncell_tot = g.ncx * g.ncy;
    const size_t cbase = (size_t)cj * g.ncx + ci0;
    if (NP == 1) {
#pragma unroll
        for (int j = 0; j < MAXT; ++j) {
            const int t = tid + j * ETHREADS;
            if (t < ntask) {
                const int kind = t % TASK_KINDS, c = t / TASK_KINDS;
                if (kind < 2 * NB) {
                    const int ee = kind >> 1, half = kind & 1;
#pragma unroll
                    for (int i = 0; i < 5; ++i)
                        cell[(size_t)((5 * half + i) * NB + ee) * ncell_tot + cbase + c] = acc[j][i] - cmp[j][i];
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        cell[(size_t)(NPAIR * NB + i * 6 + kind - 2 * NB) * ncell_tot + cbase + c] = acc[j][i] - cmp[j][i];
                }
            }
        }
    } else {
        // partial sums of the parts through shared memory, summed in part order
        float* sp = sHB;
#pragma unroll
        for (int j = 0; j < MAXT; ++j) {
            const int t = tid + j * ETHREADS;
            if (t < ntask)
#pragma unroll
                for (int i = 0; i < 5; ++i) sp[t * 5 + i] = acc[j][i] - cmp[j][i];
        }
        __syncthreads();
        for (int o = tid; o < ncell * CELL_VALS; o += ETHREADS) {
            const int c = o / CELL_VALS, r = o - c * CELL_VALS;
            int kind, i;
            if (r < NPAIR * NB) {
                const int pr = r / NB, ee = r - pr * NB;
                kind = 2 * ee + (pr >= 5);
                i = pr - 5 * (pr >= 5);
            } else {
                const int rr = r - NPAIR * NB;
                kind = 2 * NB + rr % 6;
                i = rr / 6;
            }
            float v = 0.f;
            for (int part = 0; part < NP; ++part) v += sp[((c * TASK_KINDS + kind) * NP + part) * 5 + i];
            cell[(size_t)r * ncell_tot + cbase + c] = v;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void add_cell_pair(float* dst, const float* cell, int ncx, int ncy, int ci,
                                              int cj, int pr)
{
    if (ci < 0 || cj < 0 || ci >= ncx || cj >= ncy) return;
    const int nc = ncx * ncy, c = cj * ncx + ci;
#pragma unroll
    for (int e = 0; e < NB; ++e) dst[e] += cell[(size_t)(pr * NB + e) * nc + c];
}

__device__ __forceinline__ void add_cell_rhs(float* dst, const float* cell, int ncx, int ncy, int ci,
                                             int cj, int corner)
{
    if (ci < 0 || cj < 0 || ci >= ncx || cj >= ncy) return;
    const int nc = ncx * ncy, c = cj * ncx + ci;
#pragma unroll
    for (int r = 0; r < 6; ++r) dst[r] += cell[(size_t)(NPAIR * NB + corner * 6 + r) * nc + c];
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

__device__ __forceinline__ void node_total(const float* base, const float* delta,
                                           const float* x, float t, int G, int n, float T[6], float d[6])
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
__device__ __forceinline__ void node_prior_energy(const LevelGeom& g, const DevParams& P, const float* base,
                                                  const float* delta, const float* x, float t,
                                                  const float* wf, int n, float& es, float& ee, float& em)
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

// Node n of the Gauss-Newton system, shared by four consecutive lanes of a
// warp (lane = lane id & 3; `live` false for the padding nodes past G, whose
// lanes still take part in the shuffle): its five coupling blocks gathered
// from the cell blocks of the (up to four) cells around it, plus the
// smoothness (Eq. 14), epipolar (Eqs. 15-17) and magnitude (Eq. 18) rows, the
// right-hand side and the Jacobi preconditioner. Lane 0 builds the node's own
// block, the prior rows and the preconditioner and adds the node's prior
// energies to es, ee, em; lane 1 the E block, lane 2 the S block, lane 3 the
// SE and SW blocks and the cells' part of the right-hand side, which it hands
// to lane 0 through a shuffle.
__device__ __forceinline__ void gather_node4(const LevelGeom& g, int n, int lane, bool live, const float* cell,
                                             const float* base, const float* delta, const float* wf,
                                             const DevParams& P, float* node, float* rhs, float* minv, float& es,
                                             float& ee, float& em)
{
    const int i = n % g.nx, j = n / g.nx;
    const int ncx = g.ncx, ncy = g.ncy, G = g.G;
    float bc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}; // cells' part of the right-hand side (lane 3)
    if (live && lane == 3) {
        float Bse[NB], Bsw[NB];
#pragma unroll
        for (int e = 0; e < NB; ++e) Bse[e] = Bsw[e] = 0.f;
        // corners: 0 (ci,cj), 1 (ci+1,cj), 2 (ci,cj+1), 3 (ci+1,cj+1)
        add_cell_pair(Bse, cell, ncx, ncy, i, j, pair_idx(0, 3));
        add_cell_pair(Bsw, cell, ncx, ncy, i - 1, j, pair_idx(1, 2));
        add_cell_rhs(bc, cell, ncx, ncy, i - 1, j - 1, 3);
        add_cell_rhs(bc, cell, ncx, ncy, i, j - 1, 2);
        add_cell_rhs(bc, cell, ncx, ncy, i - 1, j, 1);
        add_cell_rhs(bc, cell, ncx, ncy, i, j, 0);
#pragma unroll
        for (int e = 0; e < NB; ++e) {
            node[(size_t)(3 * NB + e) * G + n] = Bse[e];
            node[(size_t)(4 * NB + e) * G + n] = Bsw[e];
        }
    }
    const int src = (threadIdx.x & 31 & ~3) | 3;
#pragma unroll
    for (int u = 0; u < 6; ++u) bc[u] = __shfl_sync(0xffffffffu, bc[u], src);
    if (!live) return;
    if (lane == 1 || lane == 2) {
        // E (lane 1) or S (lane 2) block, with the smoothness edge to that neighbour
        float B[NB];
#pragma unroll
        for (int e = 0; e < NB; ++e) B[e] = 0.f;
        if (lane == 1) {
            add_cell_pair(B, cell, ncx, ncy, i, j - 1, pair_idx(2, 3));
            add_cell_pair(B, cell, ncx, ncy, i, j, pair_idx(0, 1));
        } else {
            add_cell_pair(B, cell, ncx, ncy, i - 1, j, pair_idx(1, 3));
            add_cell_pair(B, cell, ncx, ncy, i, j, pair_idx(0, 2));
        }
        const int mi = lane == 1 ? i + 1 : i, mj = lane == 1 ? j : j + 1;
        if (mi < g.nx && mj < g.ny) {
            const float ww = P.w_reg * P.w_smooth * (wf[n] + wf[mj * g.nx + mi]);
#pragma unroll
            for (int u = 0; u < 6; ++u) B[sym_idx(u, u)] -= ww * P.wfl[u >> 1];
        }
#pragma unroll
        for (int e = 0; e < NB; ++e) node[(size_t)(lane * NB + e) * G + n] = B[e];
        return;
    }
    if (lane != 0) return;
    float Bs[NB], bb[6];
#pragma unroll
    for (int e = 0; e < NB; ++e) Bs[e] = 0.f;
#pragma unroll
    for (int r = 0; r < 6; ++r) bb[r] = bc[r];
    add_cell_pair(Bs, cell, ncx, ncy, i - 1, j - 1, pair_idx(3, 3));
    add_cell_pair(Bs, cell, ncx, ncy, i, j - 1, pair_idx(2, 2));
    add_cell_pair(Bs, cell, ncx, ncy, i - 1, j, pair_idx(1, 1));
    add_cell_pair(Bs, cell, ncx, ncy, i, j, pair_idx(0, 0));

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
    for (int e = 0; e < NB; ++e) node[(size_t)e * G + n] = Bs[e];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        rhs[u * G + n] = bb[u];
        const float dg = Bs[sym_idx(u, u)];
        minv[u * G + n] = dg > 0.f ? 1.f / dg : 1.f;
    }
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    node_prior_energy(g, P, base, delta, nullptr, 0.f, wf, n, s0, s1, s2);
    es += s0;
    ee += s1;
    em += s2;
}

// ---------------------------------------------------------------------------
// pyramid and level stages
// ---------------------------------------------------------------------------

// Level-0 texel of pixel p: intensity and central-difference gradients, edge
// clamped (Section 5.3).
template <class TT>
__device__ __forceinline__ typename TT::T tex0_texel(const float* __restrict__ I, int w, int h, int p)
{
    const int y = p / w, x = p - y * w;
    const int xm = max(x - 1, 0), xp = min(x + 1, w - 1), ym = max(y - 1, 0), yp = min(y + 1, h - 1);
    const float v = __ldg(I + p);
    const float gx = 0.5f * (__ldg(I + y * w + xp) - __ldg(I + y * w + xm));
    const float gy = 0.5f * (__ldg(I + yp * w + x) - __ldg(I + ym * w + x));
    return TT::pack(v, gx, gy);
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

// Next mip level, pixel p: 2x2 box of the finer intensity (edge clamped),
// gradients from the box values of the four neighbours.
template <class TT>
__device__ __forceinline__ typename TT::T texdown_texel(const typename TT::T* __restrict__ P, int wp, int hp, int w,
                                                        int h, int p)
{
    const int y = p / w, x = p - y * w;
    const int xm = max(x - 1, 0), xp = min(x + 1, w - 1), ym = max(y - 1, 0), yp = min(y + 1, h - 1);
    const float v = box2<TT>(P, wp, hp, x, y);
    const float gx = 0.5f * (box2<TT>(P, wp, hp, xp, y) - box2<TT>(P, wp, hp, xm, y));
    const float gy = 0.5f * (box2<TT>(P, wp, hp, x, yp) - box2<TT>(P, wp, hp, x, ym));
    return TT::pack(v, gx, gy);
}

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

// Initial base and delta of node n (Algorithm 1): base = 2 Up(T_coarse), the
// coarse totals read at grid coordinates (i/2, j/2); delta from the warm
// start (coarsest level), the temporal rule of Section 5.3 or zero.
__device__ __forceinline__ void level_init_node(const LevelGeom& g, int have_coarse, int nxc, int nyc,
                                                const float* base_c, const float* delta_c,
                                                float* base, float* delta,
                                                const float* prev_delta,
                                                const float* prev_total, const float* init_buf,
                                                int temporal_mode, int frame, int use_init, int n)
{
    const int i = n % g.nx, j = n / g.nx;
    const int Gc = nxc * nyc;
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

// Halfway image H(x) at pixel p: the mean of the four warped intensities.
template <class TT>
__device__ __forceinline__ float halfway_pixel(const LevelGeom& g, const typename TT::T* __restrict__ tex,
                                               const float* base, const float* delta, int p)
{
    const size_t plane = (size_t)g.w * g.h;
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
    return 0.25f * acc;
}

// w_i = 1 + gain exp(-lambda_min / tau) of node n (Section 4.3),
// lambda_min the smaller eigenvalue of the structure tensor of H over the
// 3x3 pixels at the node.
__device__ __forceinline__ float wfeat_node(const LevelGeom& g, const float* __restrict__ H, const DevParams& P, int n)
{
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
    return 1.f + P.wfeat_gain * expf(-lmin / P.wfeat_tau);
}

// ---------------------------------------------------------------------------
// block stencil of the node system
// ---------------------------------------------------------------------------

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

} // namespace

} // namespace sfk
