// sf_launch.h -- host-side launchers of the solver kernels (internal).
#pragma once

#include <cuda_bf16.h>

#include "sf_common.cuh"

namespace sfk {

// sf_levels.cu: image pyramid (Section 5.3), level initialisation with the
// delta hierarchy and temporal transfer, feature weights (Section 4.3).
// Texel buffers are typed by the precision mode (sf_params.precision): FP32
// float4 or 16-bit packed in 8 bytes (texel_bytes).
void launch_tex0(const DevArgs* args, const float* const* in_direct, int w, int h, void* tex, int prec, cudaStream_t st);
void launch_texdown(const void* texp, int wp, int hp, void* tex, int w, int h, int prec, cudaStream_t st);
// args == nullptr: frame and use_init are taken as given (eager launches);
// delta_c == nullptr: base_c holds the coarse totals.
void launch_level_init(const LevelGeom& g, const LevelGeom* gc, const float* base_c, const float* delta_c,
                       float* base, float* delta, const float* prev_delta, const float* prev_total,
                       const float* init_buf, const DevArgs* args, int temporal_mode, int frame, int use_init,
                       cudaStream_t st);
void launch_halfway(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta, float* H,
                    cudaStream_t st);
void launch_wfeat(const LevelGeom& g, const float* H, const DevParams& P, float* wf, cudaStream_t st);
void launch_fill(float* p, float v, size_t n, cudaStream_t st);
void launch_finish_level(const LevelGeom& g, const float* base, const float* delta, float* prev_delta,
                         float* prev_total, const DevArgs* args, int write_out, float* out, cudaStream_t st);
void launch_unpack_tex(const void* tex, int prec, int w, int h, float* planes, cudaStream_t st);
void launch_add(const float* a, const float* b, float* out, size_t n, cudaStream_t st);

// sf_assemble.cu: per-pixel data terms, cell assembly, node gather with the
// priors, trial energies with the backtracking decision, step update.
// Per-block partial sums are float-float pairs (hi, lo).
struct Scratch {
    float2* asm_part; // [3][MAX_PART]: photo, grad, excluded
    float2* gat_part; // [3][MAX_PART]: smooth, epi, mag
    float2* en_part;  // [6][MAX_PART]: photo, grad, smooth, epi, mag, excluded
    unsigned* counters; // [4]
    int* status;
};
int assemble_blocks(const LevelGeom& g, int* cpb_out);
// log: record the cell decisions of samples at a cell edge (test aid), or null
void launch_assemble(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta,
                     const DevParams& P, uint8_t* Wmask, float* cell, const Scratch& sc, cudaStream_t st,
                     const CellLog* log = nullptr, const LevelMaps& M = LevelMaps{nullptr, nullptr});
void launch_gather(const LevelGeom& g, const float* cell, const float* base, const float* delta, const float* wf,
                   const DevParams& P, float* node, float* rhs, float* minv, const Scratch& sc, StepCtrl* ctrl,
                   int n_asm_blocks, cudaStream_t st);
// Energy at base + delta (+ t x) into the record `rec` (energy, five weighted
// terms, excluded pixels). wmode: 0 = use Wmask, 1 = take W at the state and
// store it.
void launch_energy(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta, const float* x,
                   float t, const float* wf, const DevParams& P, uint8_t* Wmask, int wmode, const Scratch& sc,
                   double* rec, cudaStream_t st, const LevelMaps& M = LevelMaps{nullptr, nullptr});
// the trials of a step and its update: the full step's trial over the whole
// GPU (k_energy in trial mode), then the backtracking trials and the update
// in one cooperative launch of `blocks` CTAs (trials_blocks: all
// co-resident), on its own barrier counter
int trials_blocks(const LevelGeom& g, int prec, int sm_count);
cudaError_t launch_trials(const LevelGeom& g, const void* tex, int prec, const float* base, float* delta, const float* x,
                          const float* wf, const DevParams& P, const uint8_t* Wmask, const Scratch& sc,
                          unsigned long long* bar, StepCtrl* ctrl, int max_bt, int blocks, cudaStream_t st,
                          const LevelMaps& M = LevelMaps{nullptr, nullptr});
void launch_unpack_blocks(const LevelGeom& g, const float* node, const float* rhs, float* blocks, float* rhs_out,
                          cudaStream_t st);

// sf_pcg.cu: Jacobi-preconditioned CG on the block system, one cooperative
// launch per solve with a bounded grid barrier between phases.
struct PcgPlan {
    int blocks;  // CTAs of the launch
    int npt;     // nodes per four-lane group
    int cluster; // 2: one cluster, state in distributed shared memory;
                 // 1: one cluster, vectors in global memory; 0: cooperative grid;
                 // 3 / 4: grid / one cluster with one reduction per iteration;
                 // 5: grid, one reduction, self-tagged published vectors;
                 // 6: grid, pipelined (reduction behind the product)
    int npc;     // nodes per CTA (cluster == 2)
};
PcgPlan pcg_plan(int G, int sm_count, int mode, int nx);
// every schedule that can run a level of G nodes (for the autotuner)
// (nx > 0: also the kind-5 plans, and with `pipelined` the kind-6 plans,
// whose shared memory fits the level's rows of nx nodes)
int pcg_candidates(int G, int sm_count, PcgPlan* out, int max, int nx, bool pipelined);
// the self-tagged exchange's waits with a short limit (sf_probe_tagged_timeout)
int tag_timeout_probe(int mode, int skip_block, long long limit_cycles, int* status, int* returned);
cudaError_t launch_pcg(const LevelGeom& g, const PcgPlan& plan, const float* node, const float* rhs,
                       const float* minv, float* x, float* z, float* p0, float* p1, float* pub, float2* part,
                       unsigned long long* bar, int* status, int iters, int interleaved_out, cudaStream_t st);

// sf_maps.cu: the per-level maps of Algorithm 1 (Section 5.3).
constexpr int GAUSS_MAX_R = 16;
struct GaussW {
    int R;                        // radius ceil(3 sigma), at most GAUSS_MAX_R
    float w[2 * GAUSS_MAX_R + 1]; // normalised weights exp(-k^2 / (2 sigma^2))
};
GaussW gauss_weights(float sigma);
// occlusion map O (h*w bytes) of a level at totals base + delta (delta may be
// null); Z is a 4*h*w int scratch z-buffer
void launch_occlusion(const LevelGeom& g, const float* base, const float* delta, float tau, int* Z, uint8_t* O,
                      cudaStream_t st);
// V of the next finer level (w x h) from a coarse map O (wc x hc)
void launch_vis_up(int wc, int hc, const uint8_t* O, int w, int h, uint8_t* V, cudaStream_t st);
// the low-passed stereo residuals R[2][h][w] of a level, written to r (tmp:
// a second 2*h*w scratch)
void launch_illum(const LevelGeom& g, const void* tex, int prec, const float* base, const float* delta,
                  const GaussW& gw, float* r, float* tmp, cudaStream_t st);
// L[2][h][w] of the next finer level from R[2][hc][wc] (box prolongation)
void launch_illum_up(int wc, int hc, const float* R, int w, int h, float* L, cudaStream_t st);

// sf_schwarz.cu: the normal equations solved by restricted additive Schwarz
// sweeps over square subdomains with local PCG in shared memory (Section 5.2).
struct SchwarzPlan {
    int tile, overlap; // nodes
    int nsub;          // subdomains
    int emax;          // nodes of the largest extended subdomain
    int es;            // shared-memory stride (a compiled bound >= emax)
    int threads;       // per CTA (six per node)
    int smem;          // dynamic shared memory per CTA (bytes)
    int blocks;        // CTAs of the cooperative launch (all co-resident)
};
// 0, or -1 if the tiling cannot run (too large for one CTA)
int schwarz_plan(const LevelGeom& g, int tile, int overlap, int sm_count, SchwarzPlan* out);
// x (component-major [6][G], or interleaved [G][6] with interleaved_out) after
// `sweeps` sweeps of `patch` local iterations; xtmp is a second [6][G] buffer;
// bar a grid-barrier counter used only by this kernel
cudaError_t launch_schwarz(const LevelGeom& g, const SchwarzPlan& plan, const float* node, const float* rhs,
                           const float* minv, float* x, float* xtmp, unsigned long long* bar, int* status, int sweeps,
                           int patch, int interleaved_out, cudaStream_t st);

// sf_batch.cu: the frame solve of many independent sequences in one launch,
// one thread-block cluster per sequence. Descriptors live in device memory
// and are read-only during a launch (the per-frame input and output pointers
// are set by launch_batch_args before it).
struct BLevel {
    LevelGeom g;
    DevParams P;
    const void* tex;   // FP32 texels [4][h][w]
    uint8_t* W;        // [gn][h][w] outlier masks
    float* H;          // halfway image [h][w]
    float *base, *delta, *x, *wf, *prev_delta, *prev_total; // [6][G] (wf: [G])
    float *node, *rhs, *minv;                               // [105][G], [6][G], [6][G]
    float *p, *pub;    // PCG direction [6][G]; r, w, s of both parities [2][3][6][G]
    float* cell;       // [234][ncells]
    StepCtrl* ctrl;    // [SF_MAX_GN]
    int gn, pcg;       // Gauss-Newton steps and PCG iterations of the level
    int cpb, gx;       // cells per assembly group; groups per cell row
    int n_groups;      // gx * (ny - 1)
    int pad;
};

struct BSeq {
    int L, w0, h0;
    int temporal_mode, wfeat_mode, max_backtracks, use_init;
    int pad;
    const float* in;   // 4 planes of w0 * h0 (set per frame)
    float* out;        // 6 x G0 (set per frame)
    int* frames;       // frames solved so far; the launch increments it
    const float* init_buf;
    int* status;       // the sequence's status word
    float2* part;      // [2][8][16] cluster partial sums
    size_t in_off, out_off; // offsets of this sequence in the packed buffers
    BLevel lv[SF_MAX_LEVELS];
};

constexpr int BATCH_MAX_CLUSTER = 16;
int batch_maxout(int s);
void batch_prepare(int cluster, int maxout);
int batch_active_clusters(int cluster, int maxout);
cudaError_t launch_batch_frame(const BSeq* seqs, const int* order, int nseq, int cluster, int maxout, cudaStream_t st);
void launch_batch_args(BSeq* seqs, int nseq, const float* in, float* out, cudaStream_t st);
int batch_cells_per_group(int s, int div);

// sf_gemm.cu: C = A * B^T on the tensor cores (tcgen05), BF16 operands
// (row-major, K contiguous, K % 64 == 0, 16-byte aligned rows), FP32
// accumulation; grid (M tiles of 128, K splits, N tiles of BN).
enum { GEMM_F32 = 0, GEMM_BIAS_RELU_BF16 = 1, GEMM_BIAS_NCHW_F32 = 2 };
struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int lda, ldb;        // row strides (elements)
    int M, N, K;         // N % 16 == 0
    int BN;              // N tile (16 .. 256, % 16)
    int kc_per_split;    // 64-wide K chunks per split
    int n_store;         // columns written (<= N)
    int ldc;             // row stride of C / Cb
    int out_hw;          // GEMM_BIAS_NCHW_F32: pixels per image
    long long split_stride; // GEMM_F32: elements between split partials
    float* C;            // GEMM_F32, GEMM_BIAS_NCHW_F32
    __nv_bfloat16* Cb;   // GEMM_BIAS_RELU_BF16
    const float* bias;
    int* err;            // bit 0: an mbarrier wait timed out; bit 1: MMAs may still be in flight after it
                         // (their shared and tensor memory were released: treat the CUDA context as poisoned)
};
int gemm_check(const GemmArgs& a);
cudaError_t launch_gemm(const GemmArgs& a, int epi, int splits, cudaStream_t st);

// sf_net.cu: the warm-start network (training and inference).
constexpr int NET_IN_H = 60, NET_IN_W = 80, NET_OUT_C = 6, NET_OUT_H = 8, NET_OUT_W = 10;
struct NetImpl;
NetImpl* net_create(int max_batch, int* rc);
void net_free(NetImpl* n);
size_t net_param_count();
int net_set_params(NetImpl* n, const float* p, cudaStream_t st);
int net_get_params(NetImpl* n, float* p, cudaStream_t st);
int net_forward(NetImpl* n, const float* img, long long img_stride, long long ch_stride, int batch, float* out,
                cudaStream_t st);
int net_backward(NetImpl* n, const float* img, const float* target, int batch, cudaStream_t st);
int net_grads_std(NetImpl* n, float* g, cudaStream_t st);
int net_adam(NetImpl* n, float lr, cudaStream_t st);
int net_error(NetImpl* n);
float* net_loss_ptr(NetImpl* n);
float* net_out_ptr(NetImpl* n);
float* net_in_ptr(NetImpl* n);
void launch_tex_intensity(const void* tex, int prec, int w, int h, float* out, cudaStream_t st);

} // namespace sfk
