// sf_pcg.cu -- data-parallel preconditioned conjugate gradients on the
// Gauss-Newton normal equations J^T J dx = -J^T r (Thies et al., arXiv
// 1610.07159, Section 5.1), Jacobi preconditioner.
//
// One cooperative launch runs every iteration of one solve. Each thread owns
// NPT nodes and keeps their x, r, z, p, q in registers. An iteration has two
// grid-wide reductions (p.q, then r.z), each a per-block FP64 partial, a
// bounded grid barrier, and a fixed-order sum that every block computes
// identically, so all blocks take the same alpha, beta and stopping decision.
// The direction update p = z + beta p is not a separate phase: a neighbour's
// p_k is formed on the fly from its z_k and p_{k-1} (double-buffered), which
// saves the third barrier of the textbook loop.
//
// The matrix-vector product q = A p reads, per node, its own symmetric 6x6
// block and those coupling it to its E, S, SE and SW neighbours; the W, N, NW
// and NE couplings are the neighbours' stored blocks (A is symmetric with
// symmetric blocks, so no transpose is needed).
#include "sf_launch.h"

namespace sfk {

namespace {

constexpr int PT = 128; // threads per block

__device__ __forceinline__ void load_blk(const float* __restrict__ node, int G, int blk, int n, float B[NB])
{
#pragma unroll
    for (int e = 0; e < NB; ++e) B[e] = __ldg(node + (size_t)(blk * NB + e) * G + n);
}

// p_k of node m: z_k(m) for k = 0, else z_k(m) + beta p_{k-1}(m).
__device__ __forceinline__ void p_of(const float* z, const float* pprev, int G, int m, float beta, bool first, float p[6])
{
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        float v = __ldcg(z + u * G + m);
        if (!first) v = fmaf(beta, __ldcg(pprev + u * G + m), v);
        p[u] = v;
    }
}

__device__ __forceinline__ double allreduce(double v, double* sred, double* part, int slot, unsigned* bar,
                                            int* status, bool& ok)
{
    __shared__ double bc;
    const double b = block_sum<PT>(v, sred);
    if (threadIdx.x == 0) part[slot * MAX_PART + blockIdx.x] = b;
    ok = grid_barrier(bar, status, gridDim.x);
    if (threadIdx.x < 32) {
        const double s = fixed_sum(part + slot * MAX_PART, gridDim.x);
        if (threadIdx.x == 0) bc = s;
    }
    __syncthreads();
    return bc;
}

template <int NPT>
__global__ void __launch_bounds__(PT) k_pcg(LevelGeom g, const float* __restrict__ node, const float* __restrict__ rhs,
                                            const float* __restrict__ minv, float* __restrict__ xout, float* z,
                                            float* p0, float* p1, double* part, unsigned* bar, int* status, int iters,
                                            int interleaved)
{
    __shared__ double sred[PT / 32];
    const int G = g.G, nx = g.nx, ny = g.ny;
    const int stride = gridDim.x * PT;
    const int t0 = blockIdx.x * PT + threadIdx.x;
    float xr[NPT][6], rr[NPT][6], zr[NPT][6], pr[NPT][6], qr[NPT][6], mr[NPT][6];
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = t0 + k * stride;
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            xr[k][u] = 0.f;
            qr[k][u] = 0.f;
            if (n < G) {
                rr[k][u] = rhs[u * G + n];
                mr[k][u] = minv[u * G + n];
                zr[k][u] = mr[k][u] * rr[k][u];
                pr[k][u] = zr[k][u];
                z[u * G + n] = zr[k][u];
                p0[u * G + n] = zr[k][u];
                acc += (double)rr[k][u] * zr[k][u];
            } else {
                rr[k][u] = mr[k][u] = zr[k][u] = pr[k][u] = 0.f;
            }
        }
    }
    bool ok = true;
    double rz = allreduce(acc, sred, part, 1, bar, status, ok);
    float beta = 0.f;
    for (int it = 0; it < iters && ok; ++it) {
        if (!(rz > 1e-30)) break;
        const bool first = it == 0;
        const float* pprev = (it & 1) ? p0 : p1; // p_{it-1} sits in buffer (it-1) & 1
        float* pcur = (it & 1) ? p1 : p0;
        acc = 0.0;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int n = t0 + k * stride;
            if (n >= G) continue;
            if (!first) {
#pragma unroll
                for (int u = 0; u < 6; ++u) {
                    pr[k][u] = fmaf(beta, pr[k][u], zr[k][u]);
                    pcur[u * G + n] = pr[k][u];
                }
            }
            const int i = n % nx, j = n / nx;
            float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float B[NB], pm[6];
            load_blk(node, G, 0, n, B);
            sym_matvec_acc(B, pr[k], q);
            // forward couplings stored at n
            if (i + 1 < nx) {
                load_blk(node, G, 1, n, B);
                p_of(z, pprev, G, n + 1, beta, first, pm);
                sym_matvec_acc(B, pm, q);
            }
            if (j + 1 < ny) {
                load_blk(node, G, 2, n, B);
                p_of(z, pprev, G, n + nx, beta, first, pm);
                sym_matvec_acc(B, pm, q);
                if (i + 1 < nx) {
                    load_blk(node, G, 3, n, B);
                    p_of(z, pprev, G, n + nx + 1, beta, first, pm);
                    sym_matvec_acc(B, pm, q);
                }
                if (i > 0) {
                    load_blk(node, G, 4, n, B);
                    p_of(z, pprev, G, n + nx - 1, beta, first, pm);
                    sym_matvec_acc(B, pm, q);
                }
            }
            // backward couplings stored at the neighbour
            if (i > 0) {
                load_blk(node, G, 1, n - 1, B);
                p_of(z, pprev, G, n - 1, beta, first, pm);
                sym_matvec_acc(B, pm, q);
            }
            if (j > 0) {
                load_blk(node, G, 2, n - nx, B);
                p_of(z, pprev, G, n - nx, beta, first, pm);
                sym_matvec_acc(B, pm, q);
                if (i > 0) {
                    load_blk(node, G, 3, n - nx - 1, B);
                    p_of(z, pprev, G, n - nx - 1, beta, first, pm);
                    sym_matvec_acc(B, pm, q);
                }
                if (i + 1 < nx) {
                    load_blk(node, G, 4, n - nx + 1, B);
                    p_of(z, pprev, G, n - nx + 1, beta, first, pm);
                    sym_matvec_acc(B, pm, q);
                }
            }
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                qr[k][u] = q[u];
                acc += (double)pr[k][u] * q[u];
            }
        }
        const double pq = allreduce(acc, sred, part, 0, bar, status, ok);
        if (!ok || !(pq > 1e-30)) break;
        const float alpha = (float)(rz / pq);
        acc = 0.0;
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const int n = t0 + k * stride;
            if (n >= G) continue;
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                xr[k][u] = fmaf(alpha, pr[k][u], xr[k][u]);
                rr[k][u] = fmaf(-alpha, qr[k][u], rr[k][u]);
                zr[k][u] = mr[k][u] * rr[k][u];
                z[u * G + n] = zr[k][u];
                acc += (double)rr[k][u] * zr[k][u];
            }
        }
        const double rz_new = allreduce(acc, sred, part, 1, bar, status, ok);
        beta = (float)(rz_new / rz);
        rz = rz_new;
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int n = t0 + k * stride;
        if (n >= G) continue;
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            if (interleaved)
                xout[n * 6 + u] = xr[k][u];
            else
                xout[u * G + n] = xr[k][u];
        }
    }
}

template <int NPT>
cudaError_t launch_impl(int blocks, const LevelGeom& g, const float* node, const float* rhs, const float* minv,
                        float* x, float* z, float* p0, float* p1, double* part, unsigned* bar, int* status, int iters,
                        int interleaved, cudaStream_t st)
{
    LevelGeom gg = g;
    void* args[] = {(void*)&gg, (void*)&node, (void*)&rhs, (void*)&minv, (void*)&x, (void*)&z, (void*)&p0,
                    (void*)&p1, (void*)&part, (void*)&bar, (void*)&status, (void*)&iters, (void*)&interleaved};
    return cudaLaunchCooperativeKernel((const void*)k_pcg<NPT>, dim3(blocks), dim3(PT), args, 0, st);
}

int max_coop_blocks(int npt, int sm_count)
{
    int per_sm = 0;
    cudaError_t e;
    switch (npt) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<1>, PT, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<2>, PT, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<4>, PT, 0); break;
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * sm_count;
}

} // namespace

PcgPlan pcg_plan(int G, int sm_count)
{
    PcgPlan p{1, 1};
    for (int npt : {1, 2, 4}) {
        int need = (G + PT * npt - 1) / (PT * npt);
        int cap = max_coop_blocks(npt, sm_count);
        if (cap > MAX_PART) cap = MAX_PART;
        if (need <= cap) {
            p.blocks = need < 1 ? 1 : need;
            p.npt = npt;
            return p;
        }
    }
    p.blocks = -1; // too large for one cooperative launch
    p.npt = 4;
    return p;
}

cudaError_t launch_pcg(const LevelGeom& g, const PcgPlan& plan, const float* node, const float* rhs, const float* minv,
                       float* x, float* z, float* p0, float* p1, double* part, unsigned* bar, int* status, int iters,
                       int interleaved_out, cudaStream_t st)
{
    switch (plan.npt) {
    case 1: return launch_impl<1>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
    case 2: return launch_impl<2>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
    default: return launch_impl<4>(plan.blocks, g, node, rhs, minv, x, z, p0, p1, part, bar, status, iters, interleaved_out, st);
    }
}

} // namespace sfk
