// sf_batch.cu -- the frame solve of many independent stereo sequences in one
// launch (Algorithm 1 of Thies et al., arXiv 1610.07159, without the
// occlusion and illumination maps, once per sequence).
//
// One thread-block cluster serves one sequence and runs its whole frame: the
// pyramid (Section 5.3), then coarse to fine per level the initialisation of
// the delta hierarchy with the temporal transfer, the feature weights
// (Section 4.3) and the Gauss-Newton steps (Section 5.1: cell assembly, node
// gather with the priors, preconditioned CG, backtracking trials, update),
// and the hand-off to the next frame. Stages meet at the hardware cluster
// barrier, whose release/acquire semantics order the global-memory writes of
// one stage before the reads of the next; no CTA waits on another cluster, so
// clusters run in any order and need not be co-resident. Every decision that
// steers control flow (PCG stopping, step acceptance) comes from cluster sums
// that each CTA forms in the same fixed order, so all CTAs of a cluster take
// the same branches and pass the same barriers.
//
// Buffers that change during a launch (cells, node blocks, deltas, PCG
// vectors) are read with ordinary coherent loads; the non-coherent read-only
// path is used only for the input images and for texels, which are written
// once per launch before any read of them.
#include <algorithm>

#include "sf_launch.h"
#include "sf_stages.cuh"

namespace sfk {

namespace {

constexpr int BT = ETHREADS;   // threads per CTA
constexpr int BNPB = BT / 4;   // PCG node slots per CTA (four lanes per node)
constexpr int PART_Q = 8;      // values per cluster sum
constexpr int PART_STRIDE = PART_Q * BATCH_MAX_CLUSTER;

using TTB = TexF32;

struct BShared {
    float sHB[BT * HB];
    __align__(16) float sW[BT * WROW];
    ff sred[BT / 32];
    ff res[PART_Q];
    DevParams P;
};

__device__ __forceinline__ unsigned cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cl_size()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cl_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

// Cluster-wide sums of K per-thread values: a block sum per CTA, one
// float-float partial per CTA and value in global memory, the cluster
// barrier, then a fixed-order sum over the CTAs that every CTA forms
// identically. The partial buffers alternate between calls, so a fast CTA
// never overwrites partials a slow one has still to read (two barriers lie
// between a write and the next write of the same buffer).
template <int K>
__device__ __forceinline__ void cl_sum(const float (&v)[K], ff (&out)[K], float2* part, int& phase, BShared& sm,
                                       int rank, int T)
{
    static_assert(K <= PART_Q, "too many values");
    float2* pb = part + (phase & 1) * PART_STRIDE;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const ff b = ff_block_sum_fast<BT>(v[q], sm.sred);
        if (threadIdx.x == 0) pb[q * BATCH_MAX_CLUSTER + rank] = make_float2(b.hi, b.lo);
    }
    cluster_sync_all();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const ff t = ff_fixed_sum(pb + q * BATCH_MAX_CLUSTER, T);
            if (threadIdx.x == 0) sm.res[q] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) out[q] = sm.res[q];
    __syncthreads();
    ++phase;
}

__device__ __forceinline__ double ffd(ff v) { return (double)v.hi + (double)v.lo; }

// Weighted energy terms (photo, grad, smooth, epi, mag) from the raw sums.
__device__ __forceinline__ void weigh_terms(const DevParams& P, double sp, double sg, double ss, double se, double sm,
                                            double* terms)
{
    terms[0] = P.w_photo * sp;
    terms[1] = P.w_grad * sg;
    terms[2] = (double)P.w_reg * P.w_smooth * ss;
    terms[3] = (double)P.w_reg * P.w_epi * se;
    terms[4] = (double)P.w_reg * P.w_mag * sm;
}

// Jacobi-preconditioned CG on one level's block system in the one-reduction
// form of Chronopoulos and Gear, the cluster's CTAs sharing the nodes: four
// lanes per node (lane q applies stencil slots q and q + 4, lane 0 also slot
// 8; two shuffle rounds combine them). An owner keeps its iterate x and
// direction p in global memory and publishes r_k, w_k = A u_k and
// s_{k-1} = A p_{k-1} in the buffers of iteration k's parity; a neighbour's
// u_{k+1} = M (r_k - alpha_k (w_k + beta_k s_{k-1})) is formed from those, in
// the same operations as its owner forms it, so one sweep over the nodes
// (update, then w_{k+1} = A u_{k+1}) and one cluster sum of (r, u) and (w, u)
// make an iteration.
__device__ void pcg_cluster(const LevelGeom& g, const BLevel& B, int iters, float2* part, int& phase, BShared& sm,
                            int rank, int T)
{
    const int G = g.G, nx = g.nx, ny = g.ny;
    const size_t G6 = (size_t)6 * G;
    const int q4 = threadIdx.x & 3, c0 = q4, c1 = q4 + 4;
    const bool has1 = c1 < 6;
    const int grp = rank * BNPB + (threadIdx.x >> 2);
    const int stride = T * BNPB;
    // the warp's first group decides the trip count, so all 32 lanes of a
    // warp pass the shuffles together
    const int wgrp = rank * BNPB + ((threadIdx.x >> 5) << 3);
    const int nk = wgrp < G ? (G - 1 - wgrp) / stride + 1 : 0;
    float* x = B.x;
    float* pd = B.p;
    const float* node = B.node;
    const float* rhs = B.rhs;
    const float* minv = B.minv;

    float alpha = 0.f, beta = 0.f;
    ff gam{0.f, 0.f};
    for (int i = -1; i < iters; ++i) {
        // i = -1 sets up: r_0 = b, s_{-1} = 0, w_0 = A M b and the first sums
        const int par = i < 0 ? 0 : (i & 1);
        const int npar = i < 0 ? 0 : (par ^ 1);
        const float* R = B.pub + (size_t)par * 3 * G6;
        const float* Wv = R + G6;
        const float* S = R + 2 * G6;
        float* Rn = B.pub + (size_t)npar * 3 * G6;
        float* Wn = Rn + G6;
        float* Sn = Rn + 2 * G6;
        const bool last = i == iters - 1; // the update of x only
        float gp = 0.f, dp = 0.f;
        for (int k = 0; k < nk; ++k) {
            const int n = grp + k * stride;
            const bool live = n < G;
            float rn[2] = {0.f, 0.f}, un[2] = {0.f, 0.f};
            if (live) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !has1) continue;
                    const int o = (h ? c1 : c0) * G + n;
                    const float m = minv[o];
                    float r1, s;
                    if (i < 0) {
                        r1 = rhs[o];
                        s = 0.f;
                        x[o] = 0.f;
                        pd[o] = 0.f;
                    } else {
                        const float r = R[o];
                        const float p = fmaf(beta, pd[o], m * r);
                        s = fmaf(beta, S[o], Wv[o]);
                        x[o] = fmaf(alpha, p, x[o]);
                        pd[o] = p;
                        r1 = fmaf(-alpha, s, r);
                    }
                    rn[h] = r1;
                    un[h] = m * r1;
                    if (!last) {
                        Rn[o] = r1;
                        Sn[o] = s;
                    }
                }
            }
            if (last) continue;
            float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (live) {
                const int j = n / nx, ii = n - j * nx;
#pragma unroll
                for (int ss = 0; ss < 3; ++ss) {
                    const int s = ss == 2 ? 8 : q4 + 4 * ss;
                    if (ss == 2 && q4 != 0) continue;
                    int owner, blk, pnode;
                    if (!stencil_slot(s, ii, j, nx, ny, n, owner, blk, pnode)) continue;
                    float Bk[NB], u[6];
#pragma unroll
                    for (int e = 0; e < NB; ++e) Bk[e] = node[(size_t)(blk * NB + e) * G + owner];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const int o = c * G + pnode;
                        const float m = minv[o];
                        u[c] = i < 0 ? m * rhs[o] : m * fmaf(-alpha, fmaf(beta, S[o], Wv[o]), R[o]);
                    }
                    sym_matvec_acc(Bk, u, q);
                }
            }
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                q[u] += __shfl_xor_sync(0xffffffffu, q[u], 1);
                q[u] += __shfl_xor_sync(0xffffffffu, q[u], 2);
            }
            if (live) {
                const float wa = sel6(q, c0);
                Wn[c0 * G + n] = wa;
                gp = fmaf(rn[0], un[0], gp);
                dp = fmaf(wa, un[0], dp);
                if (has1) {
                    const float wb = sel6(q, c1);
                    Wn[c1 * G + n] = wb;
                    gp = fmaf(rn[1], un[1], gp);
                    dp = fmaf(wb, un[1], dp);
                }
            }
        }
        if (last) break;
        ff red[2];
        {
            const float v[2] = {gp, dp};
            cl_sum<2>(v, red, part, phase, sm, rank, T);
        }
        const ff G2 = red[0], D2 = red[1];
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
    // the last update of x has no cluster sum behind it; the trials read x
    // of every node
    cluster_sync_all();
}

template <int MAXT>
__global__ void __launch_bounds__(BT, 2) k_batch_frame(const BSeq* __restrict__ seqs,
                                                                          const int* __restrict__ order)
{
    __shared__ BShared sm;
    const int T = (int)cl_size(), rank = (int)cl_rank();
    const BSeq& S = seqs[order[cl_id()]];
    const int tid = threadIdx.x;
    const int gtid = rank * BT + tid, gstride = T * BT;
    if (S.in == nullptr || S.out == nullptr) { // every CTA of the cluster leaves before any barrier
        if (rank == 0 && tid == 0) atomicOr(S.status, DEV_NOARGS);
        return;
    }
    float2* part = S.part;
    int phase = 0;
    const int frame = *S.frames;

    // pyramid: level 0 from the inputs, then each level from the finer one
    {
        const LevelGeom g = S.lv[0].g;
        const int n = g.w * g.h;
        TTB::T* tex = (TTB::T*)S.lv[0].tex;
        for (int k = gtid; k < 4 * n; k += gstride) {
            const int c = k / n, p = k - c * n;
            tex[k] = tex0_texel<TTB>(S.in + (size_t)c * n, g.w, g.h, p);
        }
    }
    cluster_sync_all();
    for (int l = 1; l < S.L; ++l) {
        const LevelGeom gp = S.lv[l - 1].g, g = S.lv[l].g;
        const int n = g.w * g.h, np = gp.w * gp.h;
        const TTB::T* src = (const TTB::T*)S.lv[l - 1].tex;
        TTB::T* dst = (TTB::T*)S.lv[l].tex;
        for (int k = gtid; k < 4 * n; k += gstride) {
            const int c = k / n, p = k - c * n;
            dst[k] = texdown_texel<TTB>(src + (size_t)c * np, gp.w, gp.h, g.w, g.h, p);
        }
        cluster_sync_all();
    }

    for (int l = S.L - 1; l >= 0; --l) {
        const BLevel& B = S.lv[l];
        const LevelGeom g = B.g;
        if (tid == 0) sm.P = B.P;
        __syncthreads();
        const DevParams& P = sm.P;
        const bool has_c = l < S.L - 1;
        const BLevel& C = S.lv[has_c ? l + 1 : l];
        const TTB::T* tex = (const TTB::T*)B.tex;
        const int npx = g.w * g.h;

        for (int n = gtid; n < g.G; n += gstride)
            level_init_node(g, has_c, C.g.nx, C.g.ny, has_c ? C.base : nullptr, has_c ? C.delta : nullptr, B.base,
                            B.delta, B.prev_delta, B.prev_total, S.init_buf, S.temporal_mode, frame, S.use_init, n);
        cluster_sync_all();
        if (S.wfeat_mode == SF_WFEAT_EIG) {
            for (int p = gtid; p < npx; p += gstride) B.H[p] = halfway_pixel<TTB>(g, tex, B.base, B.delta, p);
            cluster_sync_all();
            for (int n = gtid; n < g.G; n += gstride) B.wf[n] = wfeat_node(g, B.H, P, n);
            cluster_sync_all();
        }

        for (int gi = 0; gi < B.gn; ++gi) {
            uint8_t* Wst = B.W + (size_t)gi * npx;
            // assembly of the cell blocks (W taken at this state)
            float ep = 0.f, eg = 0.f;
            int nex = 0;
            for (int vb = rank; vb < B.n_groups; vb += T)
                assemble_group<MAXT, TTB>(g, B.cpb, vb % B.gx, vb / B.gx, tex, B.base, B.delta, P,
                                          LevelMaps{nullptr, nullptr}, Wst, B.cell,
                                          sm.sHB, sm.sW, ep, eg, nex);
            cluster_sync_all();
            // node system with the priors; energy at the linearisation point
            float es = 0.f, ee = 0.f, em = 0.f;
            // four lanes per node; the bound is a whole number of warps, so the
            // lanes of a warp leave the loop together (gather_node4 shuffles)
            const int lanes = 4 * ((g.G + 7) & ~7);
            for (int t = gtid; t < lanes; t += gstride) {
                const int n = t >> 2;
                gather_node4(g, n < g.G ? n : g.G - 1, t & 3, n < g.G, B.cell, B.base, B.delta, B.wf, P, B.node,
                             B.rhs, B.minv, es, ee, em);
            }
            ff s6[6];
            {
                const float v[6] = {ep, eg, (float)nex, es, ee, em};
                cl_sum<6>(v, s6, part, phase, sm, rank, T);
            }
            double terms_cur[5];
            weigh_terms(P, ffd(s6[0]), ffd(s6[1]), ffd(s6[3]), ffd(s6[4]), ffd(s6[5]), terms_cur);
            const double E_cur = terms_cur[0] + terms_cur[1] + terms_cur[2] + terms_cur[3] + terms_cur[4];
            const int n_excl = (int)ffd(s6[2]);
            if (rank == 0 && tid == 0 && !isfinite(E_cur)) atomicOr(S.status, DEV_NUMERIC);

            pcg_cluster(g, B, B.pcg, part, phase, sm, rank, T);

            // backtracking on t = 1, 1/2, ...: the first trial that does not
            // raise the energy is taken (W stays that of the step)
            double E_acc = E_cur, terms_acc[5];
            for (int q = 0; q < 5; ++q) terms_acc[q] = terms_cur[q];
            float t = 1.f, t_acc = 0.f;
            for (int j = 0; j <= S.max_backtracks; ++j, t *= 0.5f) {
                float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                for (int p = gtid; p < npx; p += gstride) {
                    const int y = p / g.w, xx = p - y * g.w;
                    int i0, j0;
                    float a, bb;
                    grid_cell(xx, y, g.s, g.nx, g.ny, i0, j0, a, bb);
                    float f[6];
                    pixel_fields(B.base, B.delta, B.x, t, g.G, j0 * g.nx + i0, g.nx, a, bb, f);
                    int Wi;
                    float Ep, Eg;
                    pixel_data<false, TTB>(tex, g.w, g.h, xx, y, f, P, LevelMaps{nullptr, nullptr}, (int)Wst[p], Wi,
                                           Ep, Eg, nullptr, nullptr);
                    v[0] += Ep;
                    v[1] += Eg;
                }
                for (int n = gtid; n < g.G; n += gstride) {
                    float a0, a1, a2;
                    node_prior_energy(g, P, B.base, B.delta, B.x, t, B.wf, n, a0, a1, a2);
                    v[2] += a0;
                    v[3] += a1;
                    v[4] += a2;
                }
                ff e5[5];
                cl_sum<5>(v, e5, part, phase, sm, rank, T);
                double terms[5];
                weigh_terms(P, ffd(e5[0]), ffd(e5[1]), ffd(e5[2]), ffd(e5[3]), ffd(e5[4]), terms);
                const double E = terms[0] + terms[1] + terms[2] + terms[3] + terms[4];
                if (E <= E_cur) {
                    E_acc = E;
                    for (int q = 0; q < 5; ++q) terms_acc[q] = terms[q];
                    t_acc = t;
                    break;
                }
            }
            if (rank == 0 && tid == 0) {
                StepCtrl c;
                c.E_cur = E_cur;
                c.E_acc = E_acc;
                for (int q = 0; q < 5; ++q) {
                    c.terms_cur[q] = terms_cur[q];
                    c.terms_acc[q] = terms_acc[q];
                }
                c.t = t_acc;
                c.accepted = t_acc > 0.f;
                c.n_excluded = n_excl;
                c.t1_ok = t_acc == 1.f;
                c.E_t1 = c.t1_ok ? E_acc : E_cur;
                for (int q = 0; q < 5; ++q) c.terms_t1[q] = c.t1_ok ? terms_acc[q] : terms_cur[q];
                B.ctrl[gi] = c;
            }
            if (t_acc > 0.f)
                for (int k = gtid; k < 6 * g.G; k += gstride) B.delta[k] = fmaf(t_acc, B.x[k], B.delta[k]);
            cluster_sync_all();
        }

        // hand-off: this level's delta and total for the next frame, the
        // finest level also to the output
        for (int k = gtid; k < 6 * g.G; k += gstride) {
            const float d = B.delta[k];
            const float Tt = B.base[k] + d;
            B.prev_delta[k] = d;
            B.prev_total[k] = Tt;
            if (l == 0) S.out[k] = Tt;
        }
        cluster_sync_all();
    }
    if (rank == 0 && tid == 0) *S.frames = frame + 1;
}

__global__ void k_batch_args(BSeq* seqs, int nseq, const float* in, float* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseq) return;
    seqs[i].in = in + seqs[i].in_off;
    seqs[i].out = out + seqs[i].out_off;
}

template <int MAXT>
cudaLaunchConfig_t batch_config(int nseq, int cluster, cudaStream_t st, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(nseq * cluster), 1, 1);
    cfg.blockDim = dim3(BT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <int MAXT>
void prepare_impl()
{
    cudaFuncSetAttribute(k_batch_frame<MAXT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <int MAXT>
int active_impl(int cluster)
{
    prepare_impl<MAXT>();
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = batch_config<MAXT>(1, cluster, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_batch_frame<MAXT>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int MAXT>
cudaError_t launch_impl(const BSeq* seqs, const int* order, int nseq, int cluster, cudaStream_t st)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = batch_config<MAXT>(nseq, cluster, st, attr);
    return cudaLaunchKernelEx(&cfg, k_batch_frame<MAXT>, seqs, order);
}

} // namespace

int batch_cells_per_group(int s, int div)
{
    int cpb = ETHREADS / (s * s);
    if (cpb < 1) cpb = 1;
    while (assemble_tasks_per_thread(cpb) > 4) --cpb;
    if (div > 1) cpb = (cpb + div - 1) / div;
    return cpb < 1 ? 1 : cpb;
}

int batch_maxout(int s)
{
    // task slots per thread of the largest group any schedule uses
    int need = 1;
    for (int div = 1; div <= 4; ++div)
        need = std::max(need, assemble_tasks_per_thread(batch_cells_per_group(s, div)));
    return need <= 1 ? 1 : need <= 2 ? 2 : 4;
}

void batch_prepare(int cluster, int maxout)
{
    (void)cluster;
    if (maxout == 1)
        prepare_impl<1>();
    else if (maxout == 2)
        prepare_impl<2>();
    else
        prepare_impl<4>();
}

int batch_active_clusters(int cluster, int maxout)
{
    if (maxout == 1) return active_impl<1>(cluster);
    if (maxout == 2) return active_impl<2>(cluster);
    return active_impl<4>(cluster);
}

cudaError_t launch_batch_frame(const BSeq* seqs, const int* order, int nseq, int cluster, int maxout, cudaStream_t st)
{
    if (maxout == 1) return launch_impl<1>(seqs, order, nseq, cluster, st);
    if (maxout == 2) return launch_impl<2>(seqs, order, nseq, cluster, st);
    return launch_impl<4>(seqs, order, nseq, cluster, st);
}

void launch_batch_args(BSeq* seqs, int nseq, const float* in, float* out, cudaStream_t st)
{
    k_batch_args<<<(nseq + 127) / 128, 128, 0, st>>>(seqs, nseq, in, out);
}

} // namespace sfk
