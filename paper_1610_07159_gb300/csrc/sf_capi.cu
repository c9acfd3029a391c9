// sf_capi.cu -- the C ABI of include/sf.h: context creation (all device
// memory up front), argument validation, the per-frame launch sequence of
// Algorithm 1 (Thies et al., arXiv 1610.07159) without the occlusion and
// illumination maps, its capture into one CUDA graph, statistics and the
// step-level probe entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sf_launch.h"

using namespace sfk;

namespace {

thread_local int g_last_error = SF_OK;

struct LevelBuf {
    void* tex = nullptr; // texels, typed by the precision mode
    uint8_t* W = nullptr;
    float* H = nullptr;
    float *base = nullptr, *delta = nullptr, *x = nullptr, *wf = nullptr;
    float *prev_delta = nullptr, *prev_total = nullptr;
    float *node = nullptr, *rhs = nullptr, *minv = nullptr;
    float *z = nullptr, *p0 = nullptr, *p1 = nullptr;
    float* pub = nullptr; // one-reduction PCG: [2][r, w, s][6][G] floats, or as many 64-bit tagged words
    float* cell = nullptr;
    uint2* cellrec = nullptr;  // [gn][cellcap] cell decisions at cell edges (record_cells)
    unsigned* celln = nullptr; // [gn] records per step
    int cellcap = 0;
    // per-level maps of Algorithm 1: the maps this level uses ([frame parity], the video pipeline
    // alternates them), and the scratch that computes this level's own for the next finer level
    uint8_t* vis[2] = {nullptr, nullptr}; // [h][w] occlusion map V used here
    float* illum[2] = {nullptr, nullptr}; // [2][h][w] illumination differences used here
    int* zbuf = nullptr;                  // [4][h][w] z-buffer
    uint8_t* occ = nullptr;               // [h][w] this level's occlusion map
    float* illr = nullptr;                // [2][h][w] stereo residuals, then low-passed
    float* illt = nullptr;                // [2][h][w] scratch of the separable blur
};

__global__ void k_set_args(DevArgs* a, const float* i0, const float* i1, const float* i2, const float* i3, float* out,
                           int frame, int use_init)
{
    a->in[0] = i0;
    a->in[1] = i1;
    a->in[2] = i2;
    a->in[3] = i3;
    a->out = out;
    a->frame = frame;
    a->use_init = use_init;
}

} // namespace

struct sf_ctx {
    int w0 = 0, h0 = 0, s = 0, L = 0;
    sf_params prm{};
    LevelGeom geo[SF_MAX_LEVELS]{};
    LevelBuf lv[SF_MAX_LEVELS];
    DevParams dp[SF_MAX_LEVELS]{};
    PcgPlan plan[SF_MAX_LEVELS]{};
    SchwarzPlan splan[SF_MAX_LEVELS]{};
    int asm_blocks[SF_MAX_LEVELS]{};
    int trial_blocks[SF_MAX_LEVELS]{};   // CTAs of the cooperative trial launch
    int sm_count = 0;
    Scratch sc[SF_MAX_LEVELS]{};              // per level, so levels can run concurrently
    float2* pcg_part[SF_MAX_LEVELS]{};
    int* status = nullptr;                    // device status word shared by all levels
    unsigned long long* bar = nullptr;        // grid-barrier arrival counters: [level] PCG, [SF_MAX_LEVELS + level]
                                              // trials, [2 * SF_MAX_LEVELS + level] Schwarz
    StepCtrl* ctrl = nullptr; // [SF_MAX_LEVELS * SF_MAX_GN + 1], the last one for probes
    double* rec = nullptr;    // [8] energy record
    DevArgs* args = nullptr;
    float* init_buf = nullptr;
    int pending_init = 0;
    float* in_buf[4] = {nullptr, nullptr, nullptr, nullptr};
    float* out_buf = nullptr;
    int frames = 0;
    GaussW gauss{};                           // weights of the illumination maps' low-pass
    cudaGraphExec_t gexec = nullptr;
    bool graph_tried = false;
    cudaStream_t cap = nullptr;
    cudaStream_t last_stream = nullptr;
    std::vector<void*> allocs;
    // profiling: event pairs around launches of the classes in profile_mask
    std::vector<cudaEvent_t> ev_begin, ev_end;
    std::vector<int> ev_class;
    int nprof = 0;
    int launches = 0; // kernel launches per frame
    // level pipeline of sf_solve_video (allocated when params.video is set)
    bool video = false;
    int ring = 0;                                        // frames in flight
    void* ring_tex[SF_MAX_LEVELS][SF_MAX_LEVELS]{};      // [ring slot][level] texels
    float* vstate_delta[SF_MAX_LEVELS][2]{};             // [level][frame parity]
    float* vstate_total[SF_MAX_LEVELS][2]{};
    float* vin[SF_MAX_LEVELS]{};                         // [ring slot] staged host inputs (4 images)
    float* vout[SF_MAX_LEVELS]{};                        // [ring slot] staged host outputs
    cudaStream_t vstream[SF_MAX_LEVELS]{};
    cudaEvent_t vev[SF_MAX_LEVELS]{};
    cudaEvent_t vfork = nullptr;
    // host outputs: level 0's fields leave through their own stream, so the
    // device-to-host copy of frame f overlaps the next frames' levels
    cudaStream_t vcopy = nullptr;
    cudaEvent_t vdone0 = nullptr;                        // level 0 of a frame done (reused per frame)
    cudaEvent_t vcopied[SF_MAX_LEVELS]{};                // [ring slot] its staged output copied out
};

namespace {

int fail(int code)
{
    g_last_error = code;
    return code;
}

template <typename T>
bool dalloc(sf_ctx* c, T** p, size_t count)
{
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaMemset(q, 0, count * sizeof(T) + 16);
    c->allocs.push_back(q);
    *p = (T*)q;
    return true;
}

void free_ctx(sf_ctx* c)
{
    if (!c) return;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (int l = 0; l < SF_MAX_LEVELS; ++l) {
        if (c->vstream[l]) cudaStreamDestroy(c->vstream[l]);
        if (c->vev[l]) cudaEventDestroy(c->vev[l]);
    }
    if (c->vfork) cudaEventDestroy(c->vfork);
    if (c->vcopy) cudaStreamDestroy(c->vcopy);
    if (c->vdone0) cudaEventDestroy(c->vdone0);
    for (cudaEvent_t e : c->vcopied)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_begin) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_end) cudaEventDestroy(e);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

DevParams make_dev_params(const sf_params& p, int level)
{
    DevParams d{};
    d.w_reg = p.w_reg;
    d.w_photo = p.w_photo;
    d.w_grad = p.w_grad;
    d.w_epi = p.w_epi;
    d.w_smooth = p.w_smooth;
    d.w_mag = p.w_mag;
    d.wfl[0] = p.w_s;
    d.wfl[1] = p.w_m;
    d.wfl[2] = p.w_d;
    d.mfl[0] = p.m_s;
    d.mfl[1] = p.m_m;
    d.mfl[2] = p.m_d;
    d.eps = p.eps;
    d.eps_p = p.eps_p;
    // F in level pixels: S F S rescaled to the Frobenius norm of F, S = diag(2^l, 2^l, 1)
    double sc[3] = {std::ldexp(1.0, level), std::ldexp(1.0, level), 1.0};
    double Fl[9], n0 = 0.0, n1 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Fl[a * 3 + b] = sc[a] * (double)p.F[a * 3 + b] * sc[b];
            n0 += (double)p.F[a * 3 + b] * p.F[a * 3 + b];
            n1 += Fl[a * 3 + b] * Fl[a * 3 + b];
        }
    for (int a = 0; a < 9; ++a) d.Fl[a] = (float)(n1 > 0.0 ? Fl[a] * std::sqrt(n0 / n1) : Fl[a]);
    d.robust_mode = p.robust_mode;
    d.grad_mode = p.grad_mode;
    d.wfeat_mode = p.wfeat_mode;
    d.wfeat_gain = p.wfeat_gain;
    d.wfeat_tau = p.wfeat_tau;
    return d;
}

bool finite_params(const sf_params& p)
{
    const float v[] = {p.w_reg, p.w_photo, p.w_grad, p.w_epi, p.w_smooth, p.w_mag, p.w_s, p.w_m, p.w_d,
                       p.m_s, p.m_m, p.m_d, p.eps, p.eps_p, p.wfeat_gain, p.wfeat_tau, p.occ_tau, p.illum_sigma};
    for (float x : v)
        if (!std::isfinite(x)) return false;
    for (float x : p.F)
        if (!std::isfinite(x)) return false;
    return true;
}

int check_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return SF_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA;
}

// Records a timing event for kernel class k if it is being profiled (inside
// a stream capture the event becomes an event-record node of the graph).
void prof_mark(sf_ctx* c, int k, bool begin, cudaStream_t st)
{
    if (!(c->prm.profile_mask & (1 << k))) return;
    if (begin) {
        if (c->nprof >= (int)c->ev_begin.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
            c->ev_begin.push_back(a);
            c->ev_end.push_back(b);
            c->ev_class.push_back(k);
        }
        c->ev_class[c->nprof] = k;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    cudaEvent_t e = begin ? c->ev_begin[c->nprof] : c->ev_end[c->nprof];
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
    if (!begin) c->nprof += 1;
}

// Inputs and outputs of one level's solve.
struct LevelIO {
    const void* tex;                                   // the level's texels
    const uint8_t* vis_in;                             // occlusion map of this level (null: none)
    const float* illum_in;                             // illumination differences of this level (null: none)
    uint8_t* vis_out;                                  // the next finer level's, made here (null: none)
    float* illum_out;
    const float* coarse_base;                          // coarse totals (base + delta, or the
    const float* coarse_delta;                         // totals alone when delta is null); null at the top
    const float* prev_delta, *prev_total;              // temporal state of the previous frame
    float* out_delta, *out_total;                      // state of this frame
    float* out_fields;                                 // finest output when args is null
    const DevArgs* args;                               // frame, warm start and output from the device
    int frame, use_init;                               // when args is null
};

void enqueue_pyramid(sf_ctx* c, const DevArgs* args, const float* const* in, void* const* tex, cudaStream_t st,
                     int& nl)
{
    const int prec = c->prm.precision;
    prof_mark(c, SF_K_PYRAMID, true, st);
    launch_tex0(args, in, c->w0, c->h0, tex[0], prec, st);
    ++nl;
    for (int l = 1; l < c->L; ++l, ++nl)
        launch_texdown(tex[l - 1], c->geo[l - 1].w, c->geo[l - 1].h, tex[l], c->geo[l].w, c->geo[l].h, prec, st);
    prof_mark(c, SF_K_PYRAMID, false, st);
}

// One level of Algorithm 1: initialisation, feature weights, the Gauss-Newton
// steps (assembly, gather, PCG, backtracking trials, update) and the hand-off.
int enqueue_level(sf_ctx* c, int l, const LevelIO& io, cudaStream_t st, int& nl)
{
    const sf_params& P = c->prm;
    const LevelGeom& g = c->geo[l];
    LevelBuf& b = c->lv[l];
    const Scratch& sc = c->sc[l];
    const bool has_c = l < c->L - 1;
    prof_mark(c, SF_K_LEVEL, true, st);
    launch_level_init(g, has_c ? &c->geo[l + 1] : nullptr, io.coarse_base, io.coarse_delta, b.base, b.delta,
                      io.prev_delta, io.prev_total, c->init_buf, io.args, P.temporal_mode, io.frame, io.use_init, st);
    ++nl;
    if (P.wfeat_mode == SF_WFEAT_EIG) {
        launch_halfway(g, io.tex, P.precision, b.base, b.delta, b.H, st);
        launch_wfeat(g, b.H, c->dp[l], b.wf, st);
        nl += 2;
    }
    prof_mark(c, SF_K_LEVEL, false, st);
    const bool finer = l < c->L - 1; // the coarsest level takes no maps
    const LevelMaps M{P.occlusion && finer ? io.vis_in : nullptr, P.illumination && finer ? io.illum_in : nullptr};
    for (int gi = 0; gi < P.gn_iters[l]; ++gi) {
        StepCtrl* ctrl = c->ctrl + l * SF_MAX_GN + gi;
        uint8_t* Wst = b.W + (size_t)gi * g.w * g.h; // this step's outlier mask, kept for inspection
        prof_mark(c, SF_K_ASSEMBLE, true, st);
        if (b.cellrec) {
            cudaMemsetAsync(b.celln + gi, 0, sizeof(unsigned), st);
            const CellLog log{b.cellrec + (size_t)gi * b.cellcap, b.celln + gi, b.cellcap};
            launch_assemble(g, io.tex, P.precision, b.base, b.delta, c->dp[l], Wst, b.cell, sc, st, &log, M);
        } else {
            launch_assemble(g, io.tex, P.precision, b.base, b.delta, c->dp[l], Wst, b.cell, sc, st, nullptr, M);
        }
        prof_mark(c, SF_K_ASSEMBLE, false, st);
        prof_mark(c, SF_K_GATHER, true, st);
        launch_gather(g, b.cell, b.base, b.delta, b.wf, c->dp[l], b.node, b.rhs, b.minv, sc, ctrl, c->asm_blocks[l],
                      st);
        prof_mark(c, SF_K_GATHER, false, st);
        prof_mark(c, SF_K_PCG, true, st);
        cudaError_t e = P.solver == SF_SOLVER_SCHWARZ
                            ? launch_schwarz(g, c->splan[l], b.node, b.rhs, b.minv, b.x, b.z,
                                             c->bar + 2 * SF_MAX_LEVELS + l, c->status, P.pcg_iters[l],
                                             P.patch_iters[l], 0, st)
                            : launch_pcg(g, c->plan[l], b.node, b.rhs, b.minv, b.x, b.z, b.p0, b.p1, b.pub,
                                         c->pcg_part[l], c->bar + l, c->status, P.pcg_iters[l], 0, st);
        prof_mark(c, SF_K_PCG, false, st);
        if (e != cudaSuccess) return check_cuda(e);
        nl += 3; // assembly, gather, the linear solve
        prof_mark(c, SF_K_ENERGY, true, st);
        e = launch_trials(g, io.tex, P.precision, b.base, b.delta, b.x, b.wf, c->dp[l], Wst, sc,
                          c->bar + SF_MAX_LEVELS + l, ctrl, P.max_backtracks, c->trial_blocks[l], st, M);
        if (e != cudaSuccess) return check_cuda(e);
        nl += 2; // the full step's trial, then the backtracking trials and the update
        prof_mark(c, SF_K_ENERGY, false, st);
    }
    prof_mark(c, SF_K_LEVEL, true, st);
    if (l == 0 && P.gn_iters[0] == 0) {
        launch_energy(g, io.tex, P.precision, b.base, b.delta, nullptr, 0.f, b.wf, c->dp[0], b.W, 1, sc, c->rec, st,
                      M);
        ++nl;
    }
    // this level's maps for the next finer level (Algorithm 1: occlusion maps, illumination maps,
    // prolongation), from its final totals base + delta
    if (l > 0 && P.occlusion && io.vis_out) {
        launch_occlusion(g, b.base, b.delta, P.occ_tau, b.zbuf, b.occ, st);
        launch_vis_up(g.w, g.h, b.occ, c->geo[l - 1].w, c->geo[l - 1].h, io.vis_out, st);
        nl += 4;
    }
    if (l > 0 && P.illumination && io.illum_out) {
        launch_illum(g, io.tex, P.precision, b.base, b.delta, c->gauss, b.illr, b.illt, st);
        launch_illum_up(g.w, g.h, b.illr, c->geo[l - 1].w, c->geo[l - 1].h, io.illum_out, st);
        nl += 4;
    }
    launch_finish_level(g, b.base, b.delta, io.out_delta, io.out_total, io.args, l == 0, io.out_fields, st);
    ++nl;
    prof_mark(c, SF_K_LEVEL, false, st);
    return check_cuda(cudaGetLastError());
}

// Enqueues one frame of Algorithm 1 on `st` (the inputs come through args).
int enqueue_frame(sf_ctx* c, cudaStream_t st)
{
    int nl = 0;
    c->nprof = 0;
    void* tex[SF_MAX_LEVELS];
    for (int l = 0; l < c->L; ++l) tex[l] = c->lv[l].tex;
    enqueue_pyramid(c, c->args, nullptr, tex, st, nl);
    for (int l = c->L - 1; l >= 0; --l) {
        const bool has_c = l < c->L - 1;
        LevelBuf& b = c->lv[l];
        LevelIO io{b.tex, b.vis[0], b.illum[0], l > 0 ? c->lv[l - 1].vis[0] : nullptr,
                   l > 0 ? c->lv[l - 1].illum[0] : nullptr, has_c ? c->lv[l + 1].base : nullptr,
                   has_c ? c->lv[l + 1].delta : nullptr, b.prev_delta, b.prev_total, b.prev_delta, b.prev_total,
                   nullptr, c->args, 0, 0};
        int rc = enqueue_level(c, l, io, st, nl);
        if (rc) return rc;
    }
    c->launches = nl + 1; // + the argument kernel of sf_solve
    return SF_OK;
}

// The level pipeline over n frames: step s runs level l on frame
// s - (L - 1 - l), levels on their own streams, with a join between steps.
// Level l of frame f needs level l + 1 of frame f (previous step) and level l
// of frame f - 1 (previous step), so the result equals the sequential order.
// host_in / host_out: stage frames from and to host memory through the ring;
// a frame's fields are copied out on the copy stream after its level 0, and
// level 0 writes a ring slot again only after that slot's copy has finished.
int enqueue_video(sf_ctx* c, const float* frames, const float* host_in, int n, float* outs, float* host_out,
                  cudaStream_t st)
{
    const int L = c->L, R = c->ring;
    const size_t N0 = (size_t)c->w0 * c->h0, G6 = (size_t)6 * c->geo[0].G;
    const int f0 = c->frames;
    int nl = 0;
    c->nprof = 0;
    if (cudaEventRecord(c->vfork, st) != cudaSuccess) return check_cuda(cudaGetLastError());
    for (int l = 0; l < L; ++l) cudaStreamWaitEvent(c->vstream[l], c->vfork, 0);
    if (host_out) cudaStreamWaitEvent(c->vcopy, c->vfork, 0);
    if (f0 > 0)
        for (int l = 0; l < L; ++l) {
            const size_t bytes = (size_t)6 * c->geo[l].G * sizeof(float);
            cudaMemcpyAsync(c->vstate_delta[l][(f0 - 1) & 1], c->lv[l].prev_delta, bytes, cudaMemcpyDeviceToDevice,
                            c->vstream[l]);
            cudaMemcpyAsync(c->vstate_total[l][(f0 - 1) & 1], c->lv[l].prev_total, bytes, cudaMemcpyDeviceToDevice,
                            c->vstream[l]);
        }
    for (int s = 0; s < n + L - 1; ++s) {
        if (s > 0) {
            for (int l = 0; l < L; ++l) cudaEventRecord(c->vev[l], c->vstream[l]);
            for (int l = 0; l < L; ++l)
                for (int m = 0; m < L; ++m)
                    if (m != l) cudaStreamWaitEvent(c->vstream[l], c->vev[m], 0);
        }
        for (int l = L - 1; l >= 0; --l) {
            const int fl = s - (L - 1 - l);
            if (fl < 0 || fl >= n) continue;
            const int fg = f0 + fl, slot = fg % R;
            cudaStream_t bs = c->vstream[l];
            if (l == L - 1) {
                const float* src = frames + (size_t)fl * 4 * N0;
                if (host_in) {
                    cudaMemcpyAsync(c->vin[slot], host_in + (size_t)fl * 4 * N0, 4 * N0 * sizeof(float),
                                    cudaMemcpyHostToDevice, bs);
                    src = c->vin[slot];
                }
                const float* in[4] = {src, src + N0, src + 2 * N0, src + 3 * N0};
                enqueue_pyramid(c, nullptr, in, c->ring_tex[slot], bs, nl);
            }
            const bool has_c = l < L - 1;
            float* out = nullptr;
            if (l == 0) out = host_out ? c->vout[slot] : outs + (size_t)fl * G6;
            // the slot's previous frame has left it (a no-op for an event not recorded yet)
            if (l == 0 && host_out) cudaStreamWaitEvent(bs, c->vcopied[slot], 0);
            // the maps of frame fg pass from level l + 1 to level l in the pipeline's previous step; the
            // next frame's are written meanwhile into the buffer of the other parity
            LevelIO io{c->ring_tex[slot][l], c->lv[l].vis[fg & 1], c->lv[l].illum[fg & 1],
                       l > 0 ? c->lv[l - 1].vis[fg & 1] : nullptr, l > 0 ? c->lv[l - 1].illum[fg & 1] : nullptr,
                       has_c ? c->vstate_total[l + 1][fg & 1] : nullptr, nullptr,
                       c->vstate_delta[l][(fg + 1) & 1], c->vstate_total[l][(fg + 1) & 1],
                       c->vstate_delta[l][fg & 1], c->vstate_total[l][fg & 1], out, nullptr, fg,
                       (l == L - 1 && fl == 0) ? c->pending_init : 0};
            int rc = enqueue_level(c, l, io, bs, nl);
            if (rc) return rc;
            if (l == 0 && host_out) {
                cudaEventRecord(c->vdone0, bs);
                cudaStreamWaitEvent(c->vcopy, c->vdone0, 0);
                cudaMemcpyAsync(host_out + (size_t)fl * G6, out, G6 * sizeof(float), cudaMemcpyDeviceToHost,
                                c->vcopy);
                cudaEventRecord(c->vcopied[slot], c->vcopy);
            }
        }
    }
    for (int l = 0; l < L; ++l) {
        cudaEventRecord(c->vev[l], c->vstream[l]);
        cudaStreamWaitEvent(st, c->vev[l], 0);
    }
    if (host_out) {
        cudaEventRecord(c->vdone0, c->vcopy);
        cudaStreamWaitEvent(st, c->vdone0, 0);
    }
    // hand the last frame's state back to the single-frame path
    const int fz = f0 + n - 1;
    for (int l = 0; l < L; ++l) {
        const size_t bytes = (size_t)6 * c->geo[l].G * sizeof(float);
        cudaMemcpyAsync(c->lv[l].prev_delta, c->vstate_delta[l][fz & 1], bytes, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(c->lv[l].prev_total, c->vstate_total[l][fz & 1], bytes, cudaMemcpyDeviceToDevice, st);
    }
    c->launches = n > 0 ? nl / n : 0;
    return check_cuda(cudaGetLastError());
}

} // namespace

// ---------------------------------------------------------------------------
// batched solve: one cluster per sequence, one launch per frame step
// ---------------------------------------------------------------------------

struct sf_batch {
    int n = 0, s = 0, maxout = 4;
    std::vector<sf_ctx*> seq;
    std::vector<BSeq> hseq;
    BSeq* dseq = nullptr;
    int* dorder = nullptr;
    int* dframes = nullptr;
    float2* dpart = nullptr;
    std::vector<size_t> in_off, out_off;
    size_t in_total = 0, out_total = 0;
    int cluster = 8, cpb_div = 1;
    const float* last_in = nullptr;
    float* last_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    cudaStream_t cap = nullptr;
    std::string key;
};

namespace {

struct BatchSchedule {
    int cluster, cpb_div;
    float ms;
};

std::mutex g_tune_mu;
std::map<std::string, BatchSchedule> g_tune_cache; // per process: shape key -> chosen schedule
std::map<std::string, PcgPlan> g_pcg_tune;          // per process: level shape -> fastest PCG schedule

void batch_free(sf_batch* b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (sf_ctx* c : b->seq) free_ctx(c);
    if (b->dseq) cudaFree(b->dseq);
    if (b->dorder) cudaFree(b->dorder);
    if (b->dframes) cudaFree(b->dframes);
    if (b->dpart) cudaFree(b->dpart);
    delete b;
}

// Descriptor of every level for the current schedule (cells per group).
int batch_fill(sf_batch* b)
{
    // the upload replaces the device descriptors, input and output pointers
    // included: the next step sets those again
    b->last_in = nullptr;
    b->last_out = nullptr;
    for (int i = 0; i < b->n; ++i) {
        sf_ctx* c = b->seq[i];
        BSeq& S = b->hseq[i];
        for (int l = 0; l < c->L; ++l) {
            BLevel& B = S.lv[l];
            const LevelGeom& g = c->geo[l];
            B.cpb = batch_cells_per_group(b->s, b->cpb_div);
            B.gx = (g.ncx + B.cpb - 1) / B.cpb;
            B.n_groups = B.gx * g.ncy;
        }
    }
    return check_cuda(cudaMemcpy(b->dseq, b->hseq.data(), sizeof(BSeq) * b->n, cudaMemcpyHostToDevice));
}

void batch_drop_graph(sf_batch* b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

int batch_enqueue(sf_batch* b, cudaStream_t st)
{
    return check_cuda(launch_batch_frame(b->dseq, b->dorder, b->n, b->cluster, b->maxout, st));
}

int batch_step(sf_batch* b, const float* in, float* out, cudaStream_t st)
{
    if (in != b->last_in || out != b->last_out) {
        launch_batch_args(b->dseq, b->n, in, out, st);
        int rc = check_cuda(cudaGetLastError());
        if (rc) return rc;
        b->last_in = in;
        b->last_out = out;
    }
    if (b->use_graph && !b->gexec) {
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        int erc = ok ? batch_enqueue(b, b->cap) : SF_ERR_CUDA;
        ok = cudaStreamEndCapture(b->cap, &graph) == cudaSuccess && ok && erc == SF_OK;
        ok = ok && cudaGraphInstantiate(&b->gexec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();
            batch_drop_graph(b);
            b->use_graph = false;
        }
    }
    int rc = b->gexec ? check_cuda(cudaGraphLaunch(b->gexec, st)) : batch_enqueue(b, st);
    if (rc) return rc;
    for (sf_ctx* c : b->seq) {
        c->frames += 1;
        c->launches = 1;
    }
    return SF_OK;
}

int batch_zero_frames(sf_batch* b)
{
    int rc = check_cuda(cudaDeviceSynchronize());
    if (!rc) rc = check_cuda(cudaMemset(b->dframes, 0, sizeof(int) * b->n));
    if (!rc) rc = check_cuda(cudaDeviceSynchronize());
    for (sf_ctx* c : b->seq) c->frames = 0;
    return rc;
}

} // namespace

struct sf_net {
    NetImpl* p = nullptr;
};

extern "C" {

int sf_params_preset(sf_params* p, int preset)
{
    if (!p) return fail(SF_ERR_ARG);
    std::memset(p, 0, sizeof(*p));
    // Table 1 (Appendix A)
    static const float tab[3][10] = {
        {1.0f, 1.0f, 2.0f, 0.0f, 5.0f, 5.0f, 0.5f, 5.0f, 100.0f, 1000.0f},
        {0.5f, 0.5f, 5.0f, 0.5f, 0.75f, 0.5f, 0.01f, 0.5f, 10.0f, 100.0f},
        {5.0f, 1.0f, 5.0f, 0.5f, 0.5f, 1.0f, 1.0f, 0.1f, 10000.0f, 10000.0f},
    };
    if (preset < 0 || preset > 2) return fail(SF_ERR_ARG);
    const float* t = tab[preset];
    p->w_reg = t[0];
    p->w_photo = t[1];
    p->w_grad = t[2];
    p->w_epi = t[3];
    p->w_s = t[4];
    p->w_m = t[5];
    p->w_d = t[6];
    p->m_s = t[7];
    p->m_m = t[8];
    p->m_d = t[9];
    p->w_smooth = 1.0f;
    p->w_mag = 1.0f;
    p->eps = 1e-3f;
    p->eps_p = 0.2f;
    const float F[9] = {0, 0, 0, 0, 0, -1, 0, 1, 0};
    std::memcpy(p->F, F, sizeof(F));
    for (int l = 0; l < SF_MAX_LEVELS; ++l) {
        p->gn_iters[l] = 3;
        p->pcg_iters[l] = 20;
    }
    p->robust_mode = SF_IRLS;
    p->grad_mode = SF_GRAD_BROX;
    p->wfeat_mode = SF_WFEAT_EIG;
    p->wfeat_gain = 9.0f;
    p->wfeat_tau = 1e-3f;
    p->temporal_mode = SF_TEMPORAL_PROPAGATE;
    p->precision = SF_FP32;
    p->max_backtracks = 4;
    p->use_graph = 1;
    p->solver = SF_SOLVER_PCG;
    for (int l = 0; l < SF_MAX_LEVELS; ++l) p->patch_iters[l] = 5;
    p->schwarz_tile = 8;
    p->schwarz_overlap = 1;
    p->occlusion = 0;
    p->occ_tau = 0.5f;
    p->illumination = 0;
    p->illum_sigma = 3.2f;
    return SF_OK;
}

sf_ctx* sf_create(int width, int height, int grid_stride, int levels, const sf_params* p)
{
    g_last_error = SF_OK;
    if (!p || width < 2 || height < 2 || grid_stride < 1 || levels < 1 || levels > SF_MAX_LEVELS ||
        width > (1 << 15) || height > (1 << 15) || grid_stride > 256 || !finite_params(*p) || !(p->eps > 0.f) ||
        p->max_backtracks < 0 || p->max_backtracks > 8 || p->robust_mode < 0 || p->robust_mode > 1 ||
        p->grad_mode < 0 || p->grad_mode > 1 || p->wfeat_mode < 0 || p->wfeat_mode > 1 || p->temporal_mode < 0 ||
        p->temporal_mode > 2 || p->precision < SF_FP32 || p->precision > SF_MIXED_FP16 || !(p->wfeat_tau > 0.f) ||
        p->pcg_mode < 0 || p->pcg_mode > SF_PCG_PIPELINED || p->solver < SF_SOLVER_PCG ||
        p->solver > SF_SOLVER_SCHWARZ || (p->solver == SF_SOLVER_SCHWARZ && (p->schwarz_tile < 1 ||
                                                                               p->schwarz_overlap < 0)) ||
        p->occlusion < 0 || p->occlusion > 1 || !(p->occ_tau >= 0.f) || p->illumination < 0 ||
        p->illumination > 1 || (p->illumination && !(p->illum_sigma > 0.f && 3.f * p->illum_sigma <= GAUSS_MAX_R))) {
        fail(SF_ERR_ARG);
        return nullptr;
    }
    for (int l = 0; l < levels; ++l)
        if (p->gn_iters[l] < 0 || p->gn_iters[l] > SF_MAX_GN || p->pcg_iters[l] < 0 || p->pcg_iters[l] > 100000 ||
            (p->solver == SF_SOLVER_SCHWARZ && (p->patch_iters[l] < 0 || p->patch_iters[l] > 100000))) {
            fail(SF_ERR_ARG);
            return nullptr;
        }
    sf_ctx* c = new (std::nothrow) sf_ctx();
    if (!c) {
        fail(SF_ERR_OOM);
        return nullptr;
    }
    c->w0 = width;
    c->h0 = height;
    c->s = grid_stride;
    c->L = levels;
    c->prm = *p;
    int w = width, h = height;
    for (int l = 0; l < levels; ++l) {
        if (l > 0) {
            w = (w + 1) / 2;
            h = (h + 1) / 2;
        }
        LevelGeom& g = c->geo[l];
        g.w = w;
        g.h = h;
        g.s = grid_stride;
        g.nx = (w + grid_stride - 1) / grid_stride;
        g.ny = (h + grid_stride - 1) / grid_stride;
        g.G = g.nx * g.ny;
        g.ncx = g.nx - 1;
        g.ncy = g.ny - 1;
        g.level = l;
        const int en_blocks = std::min((g.w * g.h + 255) / 256, 152 * 8) + (g.G + 255) / 256;
        if (w < 2 || h < 2 || g.nx < 2 || g.ny < 2 || assemble_blocks(g, nullptr) > MAX_PART || en_blocks > MAX_PART ||
            (6 * g.G + 255) / 256 > MAX_PART) {
            delete c;
            fail(SF_ERR_ARG);
            return nullptr;
        }
        c->dp[l] = make_dev_params(*p, l);
        c->asm_blocks[l] = assemble_blocks(g, nullptr);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        fail(SF_ERR_CUDA);
        return nullptr;
    }
    for (int l = 0; l < levels; ++l) {
        c->trial_blocks[l] = trials_blocks(c->geo[l], p->precision, c->sm_count);
        c->plan[l] = pcg_plan(c->geo[l].G, c->sm_count, p->pcg_mode, c->geo[l].nx);
        // a level needs the plan of the solver it runs (the global PCG has a size limit, Schwarz does not)
        if ((p->solver == SF_SOLVER_PCG && c->plan[l].blocks < 1) ||
            (p->solver == SF_SOLVER_SCHWARZ &&
             schwarz_plan(c->geo[l], p->schwarz_tile, p->schwarz_overlap, c->sm_count, &c->splan[l]) != 0)) {
            delete c;
            fail(SF_ERR_ARG);
            return nullptr;
        }
    }
    bool ok = true;
    for (int l = 0; l < levels && ok; ++l) {
        const LevelGeom& g = c->geo[l];
        LevelBuf& b = c->lv[l];
        const size_t N = (size_t)g.w * g.h, G6 = (size_t)6 * g.G;
        ok = dalloc(c, reinterpret_cast<char**>(&b.tex), 4 * N * texel_bytes(p->precision)) && dalloc(c, &b.W, N * (size_t)std::max(1, p->gn_iters[l])) && dalloc(c, &b.H, N) && dalloc(c, &b.base, G6) &&
             dalloc(c, &b.delta, G6) && dalloc(c, &b.x, G6) && dalloc(c, &b.wf, (size_t)g.G) &&
             dalloc(c, &b.prev_delta, G6) && dalloc(c, &b.prev_total, G6) &&
             dalloc(c, &b.node, (size_t)NODE_VALS * g.G) && dalloc(c, &b.rhs, G6) && dalloc(c, &b.minv, G6) &&
             dalloc(c, &b.z, G6) && dalloc(c, &b.p0, G6) && dalloc(c, &b.p1, G6) && dalloc(c, &b.pub, 12 * G6) &&
             dalloc(c, &b.cell, (size_t)CELL_VALS * (g.ncx * g.ncy));
        if (ok && (p->occlusion || p->illumination)) {
            const int nbuf = p->video ? 2 : 1;
            for (int q = 0; q < nbuf && ok; ++q) {
                if (p->occlusion) ok = dalloc(c, &b.vis[q], N);
                if (ok && p->illumination) ok = dalloc(c, &b.illum[q], 2 * N);
            }
            if (ok && p->occlusion) ok = dalloc(c, &b.zbuf, 4 * N) && dalloc(c, &b.occ, N);
            if (ok && p->illumination) ok = dalloc(c, &b.illr, 2 * N) && dalloc(c, &b.illt, 2 * N);
        }
        if (ok && p->record_cells) {
            // every sample of a pixel can sit on a cell edge (zero fields put all of them there)
            b.cellcap = (int)std::min<size_t>(8 * N, (size_t)1 << 30);
            const size_t steps = (size_t)std::max(1, p->gn_iters[l]);
            ok = dalloc(c, &b.cellrec, steps * b.cellcap) && dalloc(c, &b.celln, steps);
        }
    }
    const size_t N0 = (size_t)width * height;
    ok = ok && dalloc(c, &c->status, 4);
    for (int l = 0; l < levels && ok; ++l) {
        Scratch& sc = c->sc[l];
        ok = dalloc(c, &sc.asm_part, 3 * (size_t)MAX_PART) && dalloc(c, &sc.gat_part, 3 * (size_t)MAX_PART) &&
             dalloc(c, &sc.en_part, 6 * (size_t)MAX_PART) && dalloc(c, &sc.counters, 8) &&
             dalloc(c, &c->pcg_part[l], 2 * (size_t)MAX_PART);
        sc.status = c->status;
    }
    if (ok && p->video) {
        c->video = true;
        c->ring = levels;
        for (int r = 0; r < c->ring && ok; ++r) {
            for (int l = 0; l < levels && ok; ++l)
                ok = dalloc(c, reinterpret_cast<char**>(&c->ring_tex[r][l]),
                            4 * (size_t)c->geo[l].w * c->geo[l].h * texel_bytes(p->precision));
            ok = ok && dalloc(c, &c->vin[r], 4 * N0) && dalloc(c, &c->vout[r], (size_t)6 * c->geo[0].G);
        }
        for (int l = 0; l < levels && ok; ++l)
            for (int q = 0; q < 2 && ok; ++q)
                ok = dalloc(c, &c->vstate_delta[l][q], (size_t)6 * c->geo[l].G) &&
                     dalloc(c, &c->vstate_total[l][q], (size_t)6 * c->geo[l].G);
    }
    ok = ok && dalloc(c, &c->bar, (size_t)3 * SF_MAX_LEVELS) &&
         dalloc(c, &c->ctrl, (size_t)SF_MAX_LEVELS * SF_MAX_GN + 1) && dalloc(c, &c->rec, 8) &&
         dalloc(c, &c->args, 1) && dalloc(c, &c->init_buf, (size_t)6 * c->geo[levels - 1].G) &&
         dalloc(c, &c->in_buf[0], N0) && dalloc(c, &c->in_buf[1], N0) && dalloc(c, &c->in_buf[2], N0) &&
         dalloc(c, &c->in_buf[3], N0) && dalloc(c, &c->out_buf, (size_t)6 * c->geo[0].G);
    if (!ok) {
        free_ctx(c);
        fail(SF_ERR_OOM);
        return nullptr;
    }
    if (p->wfeat_mode == SF_WFEAT_OFF)
        for (int l = 0; l < levels; ++l) launch_fill(c->lv[l].wf, 1.f, (size_t)c->geo[l].G, 0);
    if (p->illumination) c->gauss = gauss_weights(p->illum_sigma);
    // the coarsest level sees no maps: all visible (its illumination buffers stay zero)
    for (int q = 0; q < 2; ++q)
        if (c->lv[levels - 1].vis[q])
            cudaMemset(c->lv[levels - 1].vis[q], 1, (size_t)c->geo[levels - 1].w * c->geo[levels - 1].h);
    bool sok = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (sok && c->video) {
        sok = cudaEventCreateWithFlags(&c->vfork, cudaEventDisableTiming) == cudaSuccess;
        for (int l = 0; l < levels && sok; ++l)
            sok = cudaStreamCreateWithFlags(&c->vstream[l], cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c->vev[l], cudaEventDisableTiming) == cudaSuccess;
        sok = sok && cudaStreamCreateWithFlags(&c->vcopy, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->vdone0, cudaEventDisableTiming) == cudaSuccess;
        for (int r = 0; r < c->ring && sok; ++r)
            sok = cudaEventCreateWithFlags(&c->vcopied[r], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!sok || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        fail(SF_ERR_CUDA);
        return nullptr;
    }
    return c;
}

int sf_solve(sf_ctx* c, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1, float* out_fields,
             void* stream)
{
    if (!c || !L_t || !R_t || !L_t1 || !R_t1 || !out_fields) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    k_set_args<<<1, 1, 0, st>>>(c->args, L_t, R_t, L_t1, R_t1, out_fields, c->frames, c->pending_init);
    int rc = check_cuda(cudaGetLastError());
    if (rc) return fail(rc);
    if (c->prm.use_graph && !c->graph_tried) {
        c->graph_tried = true;
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        int erc = ok ? enqueue_frame(c, c->cap) : SF_ERR_CUDA;
        ok = cudaStreamEndCapture(c->cap, &graph) == cudaSuccess && ok && erc == SF_OK;
        ok = ok && cudaGraphInstantiate(&c->gexec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();
            if (c->gexec) cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
            c->prm.use_graph = 0; // launch kernel by kernel instead
        }
    }
    if (c->gexec)
        rc = check_cuda(cudaGraphLaunch(c->gexec, st));
    else
        rc = enqueue_frame(c, st);
    if (rc) return fail(rc);
    c->frames += 1;
    c->pending_init = 0;
    return SF_OK;
}

int sf_solve_host(sf_ctx* c, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1,
                  float* out_fields, void* stream)
{
    if (!c || !L_t || !R_t || !L_t1 || !R_t1 || !out_fields) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)c->w0 * c->h0 * sizeof(float);
    const float* src[4] = {L_t, R_t, L_t1, R_t1};
    for (int k = 0; k < 4; ++k) {
        int rc = check_cuda(cudaMemcpyAsync(c->in_buf[k], src[k], bytes, cudaMemcpyHostToDevice, st));
        if (rc) return fail(rc);
    }
    int rc = sf_solve(c, c->in_buf[0], c->in_buf[1], c->in_buf[2], c->in_buf[3], c->out_buf, stream);
    if (rc) return rc;
    rc = check_cuda(cudaMemcpyAsync(out_fields, c->out_buf, (size_t)6 * c->geo[0].G * sizeof(float),
                                    cudaMemcpyDeviceToHost, st));
    if (rc) return fail(rc);
    rc = check_cuda(cudaStreamSynchronize(st));
    return rc ? fail(rc) : SF_OK;
}

int sf_solve_video(sf_ctx* c, const float* frames, int n, float* outs, void* stream)
{
    if (!c || !frames || !outs || n < 1) return fail(SF_ERR_ARG);
    if (!c->video) return fail(SF_ERR_STATE);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    int rc = enqueue_video(c, frames, nullptr, n, outs, nullptr, st);
    if (rc) return fail(rc);
    c->frames += n;
    c->pending_init = 0;
    return SF_OK;
}

int sf_solve_video_host(sf_ctx* c, const float* frames, int n, float* outs, void* stream)
{
    if (!c || !frames || !outs || n < 1) return fail(SF_ERR_ARG);
    if (!c->video) return fail(SF_ERR_STATE);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    int rc = enqueue_video(c, nullptr, frames, n, nullptr, outs, st);
    if (rc) return fail(rc);
    c->frames += n;
    c->pending_init = 0;
    rc = check_cuda(cudaStreamSynchronize(st));
    return rc ? fail(rc) : SF_OK;
}

int sf_grid_dims(const sf_ctx* c, int level, int* w, int* h, int* nx, int* ny)
{
    if (!c || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    if (w) *w = c->geo[level].w;
    if (h) *h = c->geo[level].h;
    if (nx) *nx = c->geo[level].nx;
    if (ny) *ny = c->geo[level].ny;
    return SF_OK;
}

int sf_set_init(sf_ctx* c, const float* coarsest_delta, void* stream)
{
    if (!c || !coarsest_delta) return fail(SF_ERR_ARG);
    const size_t bytes = (size_t)6 * c->geo[c->L - 1].G * sizeof(float);
    int rc = check_cuda(cudaMemcpyAsync(c->init_buf, coarsest_delta, bytes, cudaMemcpyDeviceToDevice,
                                        (cudaStream_t)stream));
    if (rc) return fail(rc);
    c->pending_init = 1;
    return SF_OK;
}

int sf_reset(sf_ctx* c)
{
    if (!c) return fail(SF_ERR_ARG);
    c->frames = 0;
    c->pending_init = 0;
    int rc = check_cuda(cudaDeviceSynchronize());
    if (!rc) rc = check_cuda(cudaMemset(c->status, 0, 4 * sizeof(int)));
    if (!rc) rc = check_cuda(cudaMemset(c->bar, 0, 3 * SF_MAX_LEVELS * sizeof(unsigned long long)));
    for (int l = 0; l < c->L && !rc; ++l) rc = check_cuda(cudaMemset(c->sc[l].counters, 0, 8 * sizeof(unsigned)));
    if (!rc) rc = check_cuda(cudaDeviceSynchronize());
    return rc ? fail(rc) : SF_OK;
}

int sf_get_stats(sf_ctx* c, sf_stats* out)
{
    if (!c || !out) return fail(SF_ERR_ARG);
    int rc = check_cuda(cudaDeviceSynchronize());
    if (rc) return fail(rc);
    std::vector<StepCtrl> h((size_t)SF_MAX_LEVELS * SF_MAX_GN + 1);
    int status = 0;
    double rec[8];
    rc = check_cuda(cudaMemcpy(h.data(), c->ctrl, h.size() * sizeof(StepCtrl), cudaMemcpyDeviceToHost));
    if (!rc) rc = check_cuda(cudaMemcpy(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (!rc) rc = check_cuda(cudaMemcpy(rec, c->rec, sizeof(rec), cudaMemcpyDeviceToHost));
    if (rc) return fail(rc);
    std::memset(out, 0, sizeof(*out));
    out->status = (status & DEV_TIMEOUT)   ? SF_ERR_TIMEOUT
                  : (status & DEV_NUMERIC) ? SF_ERR_NUMERIC
                  : (status & DEV_NOARGS)  ? SF_ERR_STATE
                                           : SF_OK;
    out->frames = c->frames;
    out->levels = c->L;
    out->launches = c->launches;
    for (int l = 0; l < c->L; ++l)
        for (int g = 0; g < c->prm.gn_iters[l] && g < SF_MAX_GN; ++g) {
            const StepCtrl& s = h[l * SF_MAX_GN + g];
            out->step_energy[l][g] = s.E_cur;
            out->step_accepted[l][g] = s.E_acc;
            out->step_t[l][g] = s.accepted ? s.t : 0.f;
            out->step_excluded[l][g] = s.n_excluded;
        }
    const int g0 = c->prm.gn_iters[0];
    if (g0 > 0) {
        const StepCtrl& s = h[g0 - 1];
        out->energy = s.E_acc;
        for (int q = 0; q < 5; ++q) out->terms[q] = s.terms_acc[q];
        out->n_excluded = s.n_excluded;
    } else {
        out->energy = rec[0];
        for (int q = 0; q < 5; ++q) out->terms[q] = rec[1 + q];
        out->n_excluded = (int)rec[6];
    }
    return out->status;
}

int sf_get_state(sf_ctx* c, int level, float* delta, float* total, void* stream)
{
    if (!c || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    const size_t bytes = (size_t)6 * c->geo[level].G * sizeof(float);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = SF_OK;
    if (delta) rc = check_cuda(cudaMemcpyAsync(delta, c->lv[level].prev_delta, bytes, cudaMemcpyDeviceToDevice, st));
    if (!rc && total)
        rc = check_cuda(cudaMemcpyAsync(total, c->lv[level].prev_total, bytes, cudaMemcpyDeviceToDevice, st));
    return rc ? fail(rc) : SF_OK;
}

int sf_kernel_times(sf_ctx* c, int klass, double* total_ms, int* launches)
{
    if (!c || klass < 0 || klass >= SF_K_COUNT || !total_ms) return fail(SF_ERR_ARG);
    if (!(c->prm.profile_mask & (1 << klass))) return fail(SF_ERR_STATE);
    int rc = check_cuda(cudaDeviceSynchronize());
    if (rc) return fail(rc);
    double tot = 0.0;
    int n = 0;
    for (int i = 0; i < c->nprof; ++i) {
        if (c->ev_class[i] != klass) continue;
        float ms = 0.f;
        rc = check_cuda(cudaEventElapsedTime(&ms, c->ev_begin[i], c->ev_end[i]));
        if (rc) return fail(rc);
        tot += ms;
        ++n;
    }
    *total_ms = tot;
    if (launches) *launches = n;
    return SF_OK;
}

void sf_destroy(sf_ctx* c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    free_ctx(c);
}

const char* sf_status_string(int s)
{
    switch (s) {
    case SF_OK: return "ok";
    case SF_ERR_ARG: return "invalid argument";
    case SF_ERR_CUDA: return "CUDA runtime error";
    case SF_ERR_OOM: return "out of memory";
    case SF_ERR_NUMERIC: return "non-finite energy";
    case SF_ERR_TIMEOUT: return "device barrier timeout";
    case SF_ERR_STATE: return "invalid state";
    default: return "unknown status";
    }
}

int sf_last_error(void) { return g_last_error; }

// ---- step-level probes ---------------------------------------------------

int sf_probe_pyramid(sf_ctx* c, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1, int level,
                     float* planes, void* stream)
{
    if (!c || !L_t || !R_t || !L_t1 || !R_t1 || !planes || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    const float* in[4] = {L_t, R_t, L_t1, R_t1};
    const int prec = c->prm.precision;
    launch_tex0(nullptr, in, c->w0, c->h0, c->lv[0].tex, prec, st);
    for (int l = 1; l < c->L; ++l)
        launch_texdown(c->lv[l - 1].tex, c->geo[l - 1].w, c->geo[l - 1].h, c->lv[l].tex, c->geo[l].w, c->geo[l].h, prec,
                       st);
    launch_unpack_tex(c->lv[level].tex, prec, c->geo[level].w, c->geo[level].h, planes, st);
    int rc = check_cuda(cudaGetLastError());
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_feature_weights(sf_ctx* c, int level, const float* T, float* wfeat, void* stream)
{
    if (!c || !T || !wfeat || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    const LevelGeom& g = c->geo[level];
    launch_halfway(g, c->lv[level].tex, c->prm.precision, T, nullptr, c->lv[level].H, st);
    launch_wfeat(g, c->lv[level].H, c->dp[level], wfeat, st);
    int rc = check_cuda(cudaGetLastError());
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_assemble(sf_ctx* c, int level, const float* base, const float* delta, const float* wfeat, float* blocks,
                      float* rhs, double* energy, unsigned char* W, void* stream)
{
    if (!c || !base || !delta || !wfeat || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    const LevelGeom& g = c->geo[level];
    LevelBuf& b = c->lv[level];
    StepCtrl* pc = c->ctrl + SF_MAX_LEVELS * SF_MAX_GN;
    launch_assemble(g, b.tex, c->prm.precision, base, delta, c->dp[level], b.W, b.cell, c->sc[level], st);
    launch_gather(g, b.cell, base, delta, wfeat, c->dp[level], b.node, b.rhs, b.minv, c->sc[level], pc, c->asm_blocks[level],
                  st);
    if (blocks && rhs) launch_unpack_blocks(g, b.node, b.rhs, blocks, rhs, st);
    int rc = SF_OK;
    if (energy) rc = check_cuda(cudaMemcpyAsync(energy, &pc->E_cur, sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (!rc && W) rc = check_cuda(cudaMemcpyAsync(W, b.W, (size_t)g.w * g.h, cudaMemcpyDeviceToDevice, st));
    if (!rc) rc = check_cuda(cudaGetLastError());
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_pcg(sf_ctx* c, int level, int iters, float* x, void* stream)
{
    if (!c || !x || level < 0 || level >= c->L || iters < 0 || c->plan[level].blocks < 1) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    const LevelGeom& g = c->geo[level];
    LevelBuf& b = c->lv[level];
    int rc = check_cuda(launch_pcg(g, c->plan[level], b.node, b.rhs, b.minv, x, b.z, b.p0, b.p1, b.pub,
                                   c->pcg_part[level], c->bar + level, c->status, iters, 1, st));
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_schwarz(sf_ctx* c, int level, int sweeps, int patch, float* x, void* stream)
{
    if (!c || !x || level < 0 || level >= c->L || sweeps < 0 || patch < 0) return fail(SF_ERR_ARG);
    SchwarzPlan plan{};
    if (schwarz_plan(c->geo[level], c->prm.schwarz_tile, c->prm.schwarz_overlap, c->sm_count, &plan) != 0)
        return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    LevelBuf& b = c->lv[level];
    int rc = check_cuda(launch_schwarz(c->geo[level], plan, b.node, b.rhs, b.minv, x, b.z,
                                       c->bar + 2 * SF_MAX_LEVELS + level, c->status, sweeps, patch, 1, st));
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_vmask(sf_ctx* c, int level, unsigned char* V, void* stream)
{
    if (!c || !V || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    if (!c->prm.occlusion) return fail(SF_ERR_STATE);
    const size_t N = (size_t)c->geo[level].w * c->geo[level].h;
    int rc = check_cuda(cudaMemcpyAsync(V, c->lv[level].vis[0], N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_occlusion(sf_ctx* c, int level, const float* T, unsigned char* O, void* stream)
{
    if (!c || !T || !O || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    if (!c->prm.occlusion) return fail(SF_ERR_STATE);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    launch_occlusion(c->geo[level], T, nullptr, c->prm.occ_tau, c->lv[level].zbuf, O, st);
    int rc = check_cuda(cudaGetLastError());
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_illum(sf_ctx* c, int level, const float* T, float* R, void* stream)
{
    if (!c || !T || !R || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    if (!c->prm.illumination) return fail(SF_ERR_STATE);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    const LevelGeom& g = c->geo[level];
    LevelBuf& b = c->lv[level];
    launch_illum(g, b.tex, c->prm.precision, T, nullptr, c->gauss, b.illr, b.illt, st);
    int rc = check_cuda(cudaMemcpyAsync(R, b.illr, (size_t)2 * g.w * g.h * sizeof(float), cudaMemcpyDeviceToDevice,
                                        st));
    if (!rc) rc = check_cuda(cudaGetLastError());
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_wmask(sf_ctx* c, int level, int step, unsigned char* W, void* stream)
{
    if (!c || !W || level < 0 || level >= c->L || step < 0 || step >= std::max(1, c->prm.gn_iters[level]))
        return fail(SF_ERR_ARG);
    const size_t N = (size_t)c->geo[level].w * c->geo[level].h;
    int rc = check_cuda(cudaMemcpyAsync(W, c->lv[level].W + (size_t)step * N, N, cudaMemcpyDeviceToDevice,
                                        (cudaStream_t)stream));
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_energy(sf_ctx* c, int level, const float* base, const float* delta, const float* wfeat,
                    const unsigned char* W, double* out6, void* stream)
{
    if (!c || !base || !delta || !wfeat || !out6 || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    c->last_stream = st;
    const LevelGeom& g = c->geo[level];
    LevelBuf& b = c->lv[level];
    int rc = SF_OK;
    if (W) rc = check_cuda(cudaMemcpyAsync(b.W, W, (size_t)g.w * g.h, cudaMemcpyDeviceToDevice, st));
    if (rc) return fail(rc);
    launch_energy(g, b.tex, c->prm.precision, base, delta, nullptr, 0.f, wfeat, c->dp[level], b.W, W ? 0 : 1,
                  c->sc[level], c->rec, st);
    rc = check_cuda(cudaMemcpyAsync(out6, c->rec, 6 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (!rc) rc = check_cuda(cudaGetLastError());
    return rc ? fail(rc) : SF_OK;
}

int sf_probe_cells(sf_ctx* c, int level, int step, unsigned* recs, int max_recs, int* n)
{
    if (!c || !n || level < 0 || level >= c->L || step < 0 || step >= std::max(1, c->prm.gn_iters[level]) ||
        max_recs < 0)
        return fail(SF_ERR_ARG);
    const LevelBuf& b = c->lv[level];
    if (!b.cellrec) return fail(SF_ERR_STATE);
    int rc = check_cuda(cudaDeviceSynchronize());
    unsigned cnt = 0;
    if (!rc) rc = check_cuda(cudaMemcpy(&cnt, b.celln + step, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (rc) return fail(rc);
    *n = (int)std::min<unsigned>(cnt, (unsigned)INT32_MAX);
    const size_t k = std::min<size_t>({(size_t)cnt, (size_t)b.cellcap, (size_t)max_recs});
    if (recs && k)
        rc = check_cuda(cudaMemcpy(recs, b.cellrec + (size_t)step * b.cellcap, k * sizeof(uint2),
                                   cudaMemcpyDeviceToHost));
    if (rc) return fail(rc);
    return cnt > (unsigned)b.cellcap ? fail(SF_ERR_STATE) : SF_OK;
}

int sf_batch_create(int n, const int* widths, const int* heights, const int* levels, int grid_stride,
                    const sf_params* p, sf_batch** out)
{
    g_last_error = SF_OK;
    if (!out) return fail(SF_ERR_ARG);
    *out = nullptr;
    if (n < 1 || n > (1 << 16) || !widths || !heights || !levels || !p || p->precision != SF_FP32 ||
        p->solver != SF_SOLVER_PCG || p->occlusion || p->illumination || p->gn_iters[0] < 1)
        return fail(SF_ERR_ARG);
    sf_batch* b = new (std::nothrow) sf_batch();
    if (!b) return fail(SF_ERR_OOM);
    b->n = n;
    b->s = grid_stride;
    b->maxout = batch_maxout(grid_stride > 0 ? grid_stride : 1);
    sf_params q = *p;
    q.use_graph = 0;
    q.video = 0;
    q.record_cells = 0;
    q.profile_mask = 0;
    std::string key = std::to_string(n) + "|" + std::to_string(grid_stride);
    for (int i = 0; i < n; ++i) {
        sf_ctx* c = sf_create(widths[i], heights[i], grid_stride, levels[i], &q);
        if (!c) {
            const int e = g_last_error;
            batch_free(b);
            return fail(e ? e : SF_ERR_ARG);
        }
        b->seq.push_back(c);
        key += "|" + std::to_string(widths[i]) + "x" + std::to_string(heights[i]) + "x" + std::to_string(levels[i]);
    }
    for (int l = 0; l < SF_MAX_LEVELS; ++l)
        key += "|" + std::to_string(p->gn_iters[l]) + ":" + std::to_string(p->pcg_iters[l]);
    key += "|" + std::to_string(p->max_backtracks) + "|" + std::to_string(p->wfeat_mode);
    b->key = key;
    bool ok = cudaMalloc(&b->dseq, sizeof(BSeq) * n) == cudaSuccess &&
              cudaMalloc(&b->dorder, sizeof(int) * n) == cudaSuccess &&
              cudaMalloc(&b->dframes, sizeof(int) * n) == cudaSuccess &&
              cudaMalloc(&b->dpart, sizeof(float2) * 2 * 8 * BATCH_MAX_CLUSTER * (size_t)n) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaMemset(b->dframes, 0, sizeof(int) * n) == cudaSuccess;
    b->hseq.resize(n);
    b->in_off.resize(n);
    b->out_off.resize(n);
    for (int i = 0; i < n && ok; ++i) {
        sf_ctx* c = b->seq[i];
        BSeq& S = b->hseq[i];
        std::memset(&S, 0, sizeof(S));
        S.L = c->L;
        S.w0 = c->w0;
        S.h0 = c->h0;
        S.temporal_mode = c->prm.temporal_mode;
        S.wfeat_mode = c->prm.wfeat_mode;
        S.max_backtracks = c->prm.max_backtracks;
        S.use_init = 0;
        S.frames = b->dframes + i;
        S.init_buf = c->init_buf;
        S.status = c->status;
        S.part = b->dpart + (size_t)i * 2 * 8 * BATCH_MAX_CLUSTER;
        S.in_off = b->in_total;
        S.out_off = b->out_total;
        b->in_off[i] = b->in_total;
        b->out_off[i] = b->out_total;
        b->in_total += (size_t)4 * c->w0 * c->h0;
        b->out_total += (size_t)6 * c->geo[0].G;
        for (int l = 0; l < c->L && ok; ++l) {
            BLevel& B = S.lv[l];
            LevelBuf& lb = c->lv[l];
            B.g = c->geo[l];
            B.P = c->dp[l];
            B.tex = lb.tex;
            B.W = lb.W;
            B.H = lb.H;
            B.base = lb.base;
            B.delta = lb.delta;
            B.x = lb.x;
            B.wf = lb.wf;
            B.prev_delta = lb.prev_delta;
            B.prev_total = lb.prev_total;
            B.node = lb.node;
            B.rhs = lb.rhs;
            B.minv = lb.minv;
            B.p = lb.p0;
            B.pub = lb.pub;
            B.cell = lb.cell;
            B.ctrl = c->ctrl + l * SF_MAX_GN;
            B.gn = c->prm.gn_iters[l];
            B.pcg = c->prm.pcg_iters[l];
        }
    }
    // longest sequences first, so the last clusters to start are short ones
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (long long)b->seq[a]->w0 * b->seq[a]->h0 > (long long)b->seq[c]->w0 * b->seq[c]->h0;
    });
    ok = ok && cudaMemcpy(b->dorder, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
        batch_prepare(BATCH_MAX_CLUSTER, b->maxout);
        // default schedule: the largest portable cluster the GPU can hold
        b->cluster = 8;
        while (b->cluster > 1 && batch_active_clusters(b->cluster, b->maxout) < 1) b->cluster /= 2;
        ok = batch_fill(b) == SF_OK && cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        return fail(SF_ERR_CUDA);
    }
    *out = b;
    return SF_OK;
}

int sf_batch_layout(const sf_batch* b, size_t* in_offsets, size_t* out_offsets, size_t* in_total, size_t* out_total)
{
    if (!b) return fail(SF_ERR_ARG);
    for (int i = 0; i < b->n; ++i) {
        if (in_offsets) in_offsets[i] = b->in_off[i];
        if (out_offsets) out_offsets[i] = b->out_off[i];
    }
    if (in_total) *in_total = b->in_total;
    if (out_total) *out_total = b->out_total;
    return SF_OK;
}

int sf_batch_solve(sf_batch* b, const float* in, float* out, void* stream)
{
    if (!b || !in || !out) return fail(SF_ERR_ARG);
    int rc = batch_step(b, in, out, (cudaStream_t)stream);
    return rc ? fail(rc) : SF_OK;
}

int sf_batch_set_schedule(sf_batch* b, int cluster, int cpb_div)
{
    if (!b || cluster < 1 || cluster > BATCH_MAX_CLUSTER || (cluster & (cluster - 1)) || cpb_div < 1 || cpb_div > 4)
        return fail(SF_ERR_ARG);
    if (batch_active_clusters(cluster, b->maxout) < 1) return fail(SF_ERR_ARG);
    int rc = check_cuda(cudaDeviceSynchronize());
    if (rc) return fail(rc);
    b->cluster = cluster;
    b->cpb_div = cpb_div;
    batch_drop_graph(b);
    rc = batch_fill(b);
    return rc ? fail(rc) : SF_OK;
}

int sf_batch_get_schedule(const sf_batch* b, int* cluster, int* cpb_div)
{
    if (!b) return fail(SF_ERR_ARG);
    if (cluster) *cluster = b->cluster;
    if (cpb_div) *cpb_div = b->cpb_div;
    return SF_OK;
}

int sf_batch_tune(sf_batch* b, const float* in, float* out, int steps, void* stream, float* best_ms)
{
    if (!b || !in || !out || steps < 1) return fail(SF_ERR_ARG);
    for (sf_ctx* c : b->seq)
        if (c->frames != 0) return fail(SF_ERR_STATE);
    cudaStream_t st = (cudaStream_t)stream;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(b->key);
        if (it != g_tune_cache.end()) {
            if (best_ms) *best_ms = it->second.ms;
            return sf_batch_set_schedule(b, it->second.cluster, it->second.cpb_div);
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(check_cuda(cudaErrorUnknown));
    BatchSchedule best{b->cluster, b->cpb_div, -1.f};
    int rc = SF_OK;
    for (int cl = 2; cl <= BATCH_MAX_CLUSTER && !rc; cl *= 2) {
        if (batch_active_clusters(cl, b->maxout) < 1) continue;
        for (int div = 1; div <= 2 && !rc; ++div) {
            rc = sf_batch_set_schedule(b, cl, div);
            if (!rc) rc = batch_zero_frames(b);
            if (!rc) rc = batch_step(b, in, out, st); // warm-up
            if (!rc) rc = check_cuda(cudaEventRecord(e0, st));
            for (int k = 0; k < steps && !rc; ++k) rc = batch_step(b, in, out, st);
            if (!rc) rc = check_cuda(cudaEventRecord(e1, st));
            if (!rc) rc = check_cuda(cudaEventSynchronize(e1));
            float ms = 0.f;
            if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1));
            ms /= steps;
            if (!rc && (best.ms < 0.f || ms < best.ms)) best = BatchSchedule{cl, div, ms};
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return fail(rc);
    rc = sf_batch_set_schedule(b, best.cluster, best.cpb_div);
    if (!rc) rc = batch_zero_frames(b);
    if (rc) return fail(rc);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[b->key] = best;
    }
    if (best_ms) *best_ms = best.ms;
    return SF_OK;
}

sf_ctx* sf_batch_sequence(sf_batch* b, int i)
{
    if (!b || i < 0 || i >= b->n) {
        fail(SF_ERR_ARG);
        return nullptr;
    }
    return b->seq[i];
}

int sf_batch_reset(sf_batch* b)
{
    if (!b) return fail(SF_ERR_ARG);
    int rc = batch_zero_frames(b);
    for (sf_ctx* c : b->seq)
        if (!rc) rc = check_cuda(cudaMemset(c->status, 0, 4 * sizeof(int)));
    if (!rc) rc = check_cuda(cudaDeviceSynchronize());
    return rc ? fail(rc) : SF_OK;
}

void sf_batch_destroy(sf_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
}

int sf_probe_gemm_bf16(const void* A, const void* B, int M, int N, int K, int BN, int splits, float* C, void* stream)
{
    if (!C || splits < 1 || BN < 16) return fail(SF_ERR_ARG);
    GemmArgs a{};
    a.A = static_cast<const __nv_bfloat16*>(A);
    a.B = static_cast<const __nv_bfloat16*>(B);
    a.lda = K;
    a.ldb = K;
    a.M = M;
    a.N = N;
    a.K = K;
    a.BN = BN;
    const int nkc = K / 64;
    a.kc_per_split = (nkc + splits - 1) / splits;
    a.n_store = N;
    a.ldc = N;
    a.split_stride = (long long)M * N;
    a.C = C;
    int* err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return fail(check_cuda(cudaErrorMemoryAllocation));
    cudaMemset(err, 0, sizeof(int));
    a.err = err;
    int rc = gemm_check(a);
    if (!rc) rc = check_cuda(launch_gemm(a, GEMM_F32, splits, (cudaStream_t)stream));
    int h = 0;
    if (!rc) rc = check_cuda(cudaStreamSynchronize((cudaStream_t)stream));
    if (!rc) rc = check_cuda(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(err);
    if (!rc && h) rc = SF_ERR_TIMEOUT;
    return rc ? fail(rc) : SF_OK;
}

int sf_net_param_count(void) { return (int)net_param_count(); }

int sf_net_create(int max_batch, sf_net** out)
{
    if (!out) return fail(SF_ERR_ARG);
    *out = nullptr;
    int rc = SF_OK;
    NetImpl* p = net_create(max_batch, &rc);
    if (!p) return fail(rc);
    sf_net* n = new (std::nothrow) sf_net();
    if (!n) {
        net_free(p);
        return fail(SF_ERR_OOM);
    }
    n->p = p;
    *out = n;
    return SF_OK;
}

int sf_net_set_params(sf_net* n, const float* params, void* stream)
{
    if (!n || !params) return fail(SF_ERR_ARG);
    int rc = net_set_params(n->p, params, (cudaStream_t)stream);
    return rc ? fail(rc) : SF_OK;
}

int sf_net_get_params(sf_net* n, float* params, void* stream)
{
    if (!n || !params) return fail(SF_ERR_ARG);
    int rc = net_get_params(n->p, params, (cudaStream_t)stream);
    return rc ? fail(rc) : SF_OK;
}

int sf_net_forward(sf_net* n, const float* imgs, int batch, float* out, void* stream)
{
    if (!n || !imgs || !out) return fail(SF_ERR_ARG);
    int rc = net_forward(n->p, imgs, (long long)4 * NET_IN_H * NET_IN_W, (long long)NET_IN_H * NET_IN_W, batch, out,
                         (cudaStream_t)stream);
    return rc ? fail(rc) : SF_OK;
}

int sf_net_gradients(sf_net* n, const float* imgs, const float* target, int batch, float* grads, float* loss,
                     void* stream)
{
    if (!n || !imgs || !target) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = net_backward(n->p, imgs, target, batch, st);
    if (!rc && grads) rc = net_grads_std(n->p, grads, st);
    if (!rc && loss) rc = check_cuda(cudaMemcpyAsync(loss, net_loss_ptr(n->p), sizeof(float), cudaMemcpyDeviceToDevice, st));
    return rc ? fail(rc) : SF_OK;
}

int sf_net_train_step(sf_net* n, const float* imgs, const float* target, int batch, float lr, float* loss,
                      void* stream)
{
    if (!n || !imgs || !target || !(lr > 0.f)) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = net_backward(n->p, imgs, target, batch, st);
    if (!rc) rc = net_adam(n->p, lr, st);
    if (!rc && loss) rc = check_cuda(cudaMemcpyAsync(loss, net_loss_ptr(n->p), sizeof(float), cudaMemcpyDeviceToDevice, st));
    return rc ? fail(rc) : SF_OK;
}

int sf_net_status(sf_net* n)
{
    if (!n) return fail(SF_ERR_ARG);
    int rc = check_cuda(cudaDeviceSynchronize());
    if (!rc) rc = net_error(n->p);
    return rc ? fail(rc) : SF_OK;
}

void sf_net_destroy(sf_net* n)
{
    if (!n) return;
    cudaDeviceSynchronize();
    net_free(n->p);
    delete n;
}

int sf_coarsest_images(sf_ctx* c, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1, float* out,
                       void* stream)
{
    if (!c || !L_t || !R_t || !L_t1 || !R_t1 || !out) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    void* tex[SF_MAX_LEVELS];
    for (int l = 0; l < c->L; ++l) tex[l] = c->lv[l].tex;
    const float* in[4] = {L_t, R_t, L_t1, R_t1};
    int nl = 0;
    const int mask = c->prm.profile_mask;
    c->prm.profile_mask = 0;
    enqueue_pyramid(c, nullptr, in, tex, st, nl);
    c->prm.profile_mask = mask;
    const LevelGeom& g = c->geo[c->L - 1];
    launch_tex_intensity(c->lv[c->L - 1].tex, c->prm.precision, g.w, g.h, out, st);
    int rc = check_cuda(cudaGetLastError());
    return rc ? fail(rc) : SF_OK;
}

int sf_warm_start(sf_net* n, sf_ctx* c, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1,
                  void* stream)
{
    if (!n || !c) return fail(SF_ERR_ARG);
    const LevelGeom& g = c->geo[c->L - 1];
    if (g.w != NET_IN_W || g.h != NET_IN_H || g.nx != NET_OUT_W || g.ny != NET_OUT_H) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    float* in = net_in_ptr(n->p);
    int rc = sf_coarsest_images(c, L_t, R_t, L_t1, R_t1, in, stream);
    if (rc) return rc;
    rc = net_forward(n->p, in, (long long)4 * NET_IN_H * NET_IN_W, (long long)NET_IN_H * NET_IN_W, 1, c->init_buf, st);
    if (rc) return fail(rc);
    c->pending_init = 1;
    return SF_OK;
}

int sf_tune_pcg(sf_ctx* c, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1, int reps,
                void* stream)
{
    if (!c || !L_t || !R_t || !L_t1 || !R_t1 || reps < 1) return fail(SF_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    // one frame leaves every level's last Gauss-Newton system in place
    float* out = c->out_buf;
    int rc = sf_solve(c, L_t, R_t, L_t1, R_t1, out, stream);
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(st));
    if (rc) return fail(rc);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(check_cuda(cudaErrorUnknown));
    for (int l = 0; l < c->L && !rc; ++l) {
        const LevelGeom& g = c->geo[l];
        LevelBuf& b = c->lv[l];
        const int iters = c->prm.pcg_iters[l];
        if (iters < 1 || c->prm.solver == SF_SOLVER_SCHWARZ) continue;
        const bool pipelined = c->prm.pcg_mode == SF_PCG_PIPELINED;
        const std::string key = std::to_string(g.nx) + "x" + std::to_string(g.ny) + "|" + std::to_string(iters) + "|" +
                                std::to_string(c->sm_count) + (pipelined ? "|p" : "");
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_pcg_tune.find(key);
            if (it != g_pcg_tune.end()) {
                c->plan[l] = it->second;
                continue;
            }
        }
        PcgPlan cand[24];
        const int nc = pcg_candidates(g.G, c->sm_count, cand, 24, g.nx, pipelined);
        float best = -1.f;
        PcgPlan pick = c->plan[l];
        for (int k = 0; k < nc && !rc; ++k) {
            // a new block count starts its barrier counter from zero
            rc = check_cuda(cudaMemsetAsync(c->bar + l, 0, sizeof(unsigned long long), st));
            if (rc) break;
            float ms = 0.f;
            for (int r = 0; r <= reps && !rc; ++r) {
                if (r == 1) cudaEventRecord(e0, st);
                rc = check_cuda(launch_pcg(g, cand[k], b.node, b.rhs, b.minv, b.x, b.z, b.p0, b.p1, b.pub,
                                           c->pcg_part[l], c->bar + l, c->status, iters, 0, st));
            }
            if (rc) break;
            cudaEventRecord(e1, st);
            rc = check_cuda(cudaEventSynchronize(e1));
            if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1));
            int status = 0;
            if (!rc) rc = check_cuda(cudaMemcpy(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost));
            if (!rc && status) rc = (status & DEV_TIMEOUT) ? SF_ERR_TIMEOUT : SF_ERR_NUMERIC;
            if (!rc && (best < 0.f || ms < best)) {
                best = ms;
                pick = cand[k];
            }
        }
        if (!rc) {
            c->plan[l] = pick;
            rc = check_cuda(cudaMemsetAsync(c->bar + l, 0, sizeof(unsigned long long), st));
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_pcg_tune[key] = pick;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st));
    // the frame graph holds the old schedules: capture again on the next solve
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->graph_tried = false;
    int rc2 = sf_reset(c);
    return rc ? fail(rc) : rc2;
}

int sf_set_pcg_schedule(sf_ctx* c, int level, int kind, int blocks, int npt)
{
    if (!c || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    PcgPlan cand[24];
    const int nc = pcg_candidates(c->geo[level].G, c->sm_count, cand, 24, c->geo[level].nx, true);
    int k = 0;
    while (k < nc && !(cand[k].cluster == kind && cand[k].blocks == blocks && cand[k].npt == npt)) ++k;
    if (k == nc) return fail(SF_ERR_ARG);
    if (check_cuda(cudaDeviceSynchronize())) return fail(SF_ERR_CUDA);
    c->plan[level] = cand[k];
    // a new block count starts its barrier counter from zero; the frame graph
    // holds the old schedule: capture again on the next solve
    if (check_cuda(cudaMemset(c->bar + level, 0, sizeof(unsigned long long)))) return fail(SF_ERR_CUDA);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->graph_tried = false;
    return SF_OK;
}

int sf_pcg_schedule(const sf_ctx* c, int level, int* kind, int* blocks, int* npt)
{
    if (!c || level < 0 || level >= c->L) return fail(SF_ERR_ARG);
    const PcgPlan& p = c->plan[level];
    if (kind) *kind = p.cluster;
    if (blocks) *blocks = p.blocks;
    if (npt) *npt = p.npt;
    return SF_OK;
}

} // extern "C"
