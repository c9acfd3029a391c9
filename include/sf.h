/*
 * sf.h -- C ABI of the GB300 (sm_103a) halfway-domain scene-flow solver.
 *
 * The solver computes, for one stereo quadruple (two rectified, pre-calibrated
 * monochrome stereo pairs at two time steps, Section 3.1 of Thies et al.,
 * "Real-time Halfway Domain Reconstruction of Motion and Geometry", arXiv
 * 1610.07159), the stereo, motion and difference flow fields s, m, d of the
 * halfway domain (Section 3.1) on a coarse bilinear warp grid (Section 3.3,
 * Eq. 7). It minimises the energy of Eqs. 8-18 (photometric and gradient
 * consistency of the six checks of Eqs. 1-6 under the pseudo-Huber penalty of
 * Eq. 12, smoothness, epipolar and magnitude priors) with robust Gauss-Newton
 * and preconditioned conjugate gradients (Section 5.1), coarse to fine on a
 * hierarchy that stores delta flows between levels (Section 5.3, Algorithm 1;
 * its occlusion and illumination maps on request).
 *
 * Every step runs in CUDA kernels of this library on one GPU; there is no CPU
 * path. All calls are plain C: pointers, sizes and status codes.
 *
 * Conventions
 *   images      float32, row-major width x height, intensities in [0, 1]
 *               (monochrome, Section 3.1). Order: L_t = I_0^0, R_t = I_1^0,
 *               L_t1 = I_0^1, R_t1 = I_1^1 (camera c, time t of I_c^t).
 *   fields      float32 [6][ny][nx] component-major: s_x, s_y, m_x, m_y, d_x,
 *               d_y of every warp-grid node, node (i, j) at level pixel
 *               (i*grid_stride, j*grid_stride); nx = ceil(w / grid_stride),
 *               ny = ceil(h / grid_stride). Values are in pixels of the level
 *               (the finest level for sf_solve's output).
 *   streams     a cudaStream_t passed as void*; NULL is the legacy default
 *               stream. Calls that take a stream only enqueue work on it.
 *   ownership   the context owns all of its device memory, allocated in
 *               sf_create; sf_solve allocates nothing. Caller buffers stay
 *               the caller's.
 *   errors      every call returns an sf_status: SF_ERR_ARG for a null or
 *               invalid argument (nothing is enqueued then), SF_ERR_CUDA for
 *               a failed runtime call. Errors raised inside kernels (a PCG
 *               barrier that gave up waiting, a non-finite energy) are
 *               latched in a device status word, reported by sf_get_stats
 *               (which waits for the work) and cleared by sf_reset.
 *   threads     one context per host thread at a time.
 */
#ifndef SF_H
#define SF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SF_API __attribute__((visibility("default")))
#else
#define SF_API
#endif

#define SF_MAX_LEVELS 8
#define SF_MAX_GN 16

typedef enum sf_status {
    SF_OK = 0,
    SF_ERR_ARG = 1,     /* invalid argument or size */
    SF_ERR_CUDA = 2,    /* a CUDA runtime call failed */
    SF_ERR_OOM = 3,     /* device or pinned allocation failed */
    SF_ERR_NUMERIC = 4, /* a non-finite energy was met on the device */
    SF_ERR_TIMEOUT = 5, /* a device-wide barrier gave up waiting */
    SF_ERR_STATE = 6    /* call not valid in the context's current state */
} sf_status;

/* Linearisation of the robust data terms (Section 5, "square root of the
 * residuals"): SF_IRLS gives each consistency check its own reweighted
 * residual (same energy, same gradient); SF_SQRT_PAPER uses one residual
 * sqrt(sum of penalties) per pixel and term, as the paper's residual count
 * M = 2N + 14G implies. */
enum { SF_IRLS = 0, SF_SQRT_PAPER = 1 };
/* Penalty of the gradient term (Eq. 13): SF_GRAD_BROX = sqrt(|g|^2 + eps^2),
 * SF_GRAD_LITERAL = sqrt(|g|^4 + eps^2) as printed. */
enum { SF_GRAD_BROX = 0, SF_GRAD_LITERAL = 1 };
/* Feature weight w_i of the smoothness term (Section 4.3). */
enum { SF_WFEAT_EIG = 0, SF_WFEAT_OFF = 1 };
/* Initialisation of frames after the first (Section 5.3). */
enum { SF_TEMPORAL_PROPAGATE = 0, SF_TEMPORAL_COPY = 1, SF_TEMPORAL_ZERO = 2 };
/* Storage precision of the image pyramid (intensity and gradient texels,
 * from which the Jacobian is formed on the fly): FP32, or 16-bit BF16 / FP16
 * (half the texel bytes). Residuals, Jacobians, normal equations, PCG and all
 * accumulation stay in FP32. */
enum { SF_FP32 = 0, SF_MIXED_BF16 = 1, SF_MIXED_FP16 = 2 };
/* Columns of Table 1 (Appendix A). */
enum { SF_PRESET_FIG2 = 0, SF_PRESET_FIG568 = 1, SF_PRESET_FIG79 = 2 };
/* Schedule of the PCG solve, per level the first that fits: a staged grid
 * (SF_PCG_AUTO and SF_PCG_PIPELINED only: a cooperative launch over the GPU
 * whose coupling blocks fit in registers or shared memory and whose
 * neighbours' vectors are exchanged as self-tagged words, without memory
 * fences; SF_PCG_AUTO runs the one-reduction form there, SF_PCG_PIPELINED
 * the pipelined form of PCG of Ghysels and Vanroose 2014, which hides the
 * grid reduction's latency behind the matrix-vector product but keeps
 * w = A u, s, q and z by recurrence (u = M r is formed), so its rounding
 * drifts further from the textbook loop: on some frames its fields end a few
 * 1e-3 px from the FP64 oracle's, where the default stays within 1e-3),
 * SF_PCG_DSM (one cluster, the whole state in distributed shared memory, one
 * barrier per iteration), then a single cluster with vectors in global
 * memory, then a cooperative launch over the GPU. SF_PCG_AUTO and
 * SF_PCG_PIPELINED start at the first and skip the second, SF_PCG_DSM starts
 * at the second, SF_PCG_CLUSTER and SF_PCG_ONE_REDUCTION at the third;
 * SF_PCG_GRID takes only the last. SF_PCG_CLUSTER and SF_PCG_GRID run the
 * textbook loop (two reductions and two barriers per iteration); the other
 * cluster and grid schedules its Chronopoulos-Gear form (one fused reduction
 * and one barrier per iteration). All are the same iterates in exact
 * arithmetic. sf_tune_pcg considers the pipelined form only under
 * SF_PCG_PIPELINED. */
enum {
    SF_PCG_AUTO = 0,
    SF_PCG_CLUSTER = 1,
    SF_PCG_GRID = 2,
    SF_PCG_DSM = 3,
    SF_PCG_ONE_REDUCTION = 4,
    SF_PCG_PIPELINED = 5
};
/* Linear solver of each Gauss-Newton step. SF_SOLVER_PCG: Jacobi-PCG on the
 * whole level (Section 5.1), pcg_iters iterations. SF_SOLVER_SCHWARZ: the
 * domain decomposition of Section 5.2, data-parallel alternating Schwarz
 * sweeps over square subdomains of schwarz_tile x schwarz_tile grid nodes
 * plus schwarz_overlap nodes of overlap on each side; every sweep solves each
 * subdomain's system by patch_iters Jacobi-PCG iterations in shared memory
 * (the paper counts outer PCG iterations of several patch iterations each:
 * pcg_iters is the number of sweeps), and the subdomains exchange the iterate through global
 * memory. Restricted additive Schwarz: each node takes the correction of the
 * subdomain whose tile holds it. */
enum { SF_SOLVER_PCG = 0, SF_SOLVER_SCHWARZ = 1 };
/* Kernel classes, for sf_params.profile_mask and sf_kernel_times. */
enum {
    SF_K_PYRAMID = 0,  /* mip-map levels with gradient planes */
    SF_K_LEVEL = 1,    /* level init, halfway image, feature weights, output */
    SF_K_ASSEMBLE = 2, /* per-pixel data terms reduced into cell blocks */
    SF_K_GATHER = 3,   /* node blocks, priors, preconditioner, energy */
    SF_K_PCG = 4,      /* the conjugate-gradient solve */
    SF_K_ENERGY = 5,   /* trial energies, backtracking, step update */
    SF_K_COUNT = 6
};

typedef struct sf_params {
    /* Table 1 (Appendix A); w_smooth = w_mag = 1 in every experiment */
    float w_reg, w_photo, w_grad, w_epi, w_smooth, w_mag;
    float w_s, w_m, w_d; /* smoothness weight per flow (Eq. 14) */
    float m_s, m_m, m_d; /* magnitude weight per flow (Eq. 18) */
    float eps;           /* pseudo-Huber epsilon, 0.001 (Eq. 12) */
    float eps_p;         /* outlier threshold of W, 0.2 (Section 4.1); <= 0 disables W */
    float F[9];          /* fundamental matrix, row-major, finest-level pixels */
    int gn_iters[SF_MAX_LEVELS];  /* Gauss-Newton steps per level, index 0 = finest */
    int pcg_iters[SF_MAX_LEVELS]; /* PCG iterations per Gauss-Newton step */
    int robust_mode;              /* SF_IRLS | SF_SQRT_PAPER */
    int grad_mode;                /* SF_GRAD_BROX | SF_GRAD_LITERAL */
    int wfeat_mode;               /* SF_WFEAT_EIG | SF_WFEAT_OFF */
    float wfeat_gain, wfeat_tau;  /* w_i = 1 + gain * exp(-lambda_min / tau) */
    int temporal_mode;            /* SF_TEMPORAL_* */
    int precision;                /* SF_FP32 | SF_MIXED_BF16 | SF_MIXED_FP16 */
    int max_backtracks;           /* step halvings tried before a step is rejected (4) */
    int use_graph;                /* 1: replay the frame as one captured CUDA graph */
    int profile_mask;             /* bit k set: time every launch of kernel class k with CUDA events */
    int pcg_mode;                 /* SF_PCG_AUTO | _CLUSTER | _GRID | _DSM | _ONE_REDUCTION | _PIPELINED */
    int video;                    /* 1: allocate the level pipeline of sf_solve_video */
    int record_cells;             /* 1: record the bilinear cell decisions at cell edges (sf_probe_cells) */
    int solver;                   /* SF_SOLVER_PCG | SF_SOLVER_SCHWARZ */
    int patch_iters[SF_MAX_LEVELS]; /* Schwarz: local PCG iterations per sweep (5) */
    int schwarz_tile;             /* Schwarz: tile side in grid nodes (8: 16 px at the paper's stride 2) */
    int schwarz_overlap;          /* Schwarz: overlap in grid nodes on each side (1: the paper's 2 px) */
    /* Per-level maps of Algorithm 1 (Section 5.3), computed after each level's
     * solve and prolongated to the next finer level; the coarsest level uses
     * none. Occlusion maps: the triangulated warp grid is rendered into each
     * of the four views with a z-buffer of closeness (the stereo pair's
     * horizontal disparity, larger = nearer); a reference pixel is visible
     * when, in every view, its rounded sample position lies in the image and
     * its closeness is at least the z-buffer's there less occ_tau; the map is
     * interpolated bilinearly to the next level and thresholded at 1/2, and
     * V = 0 removes the pixel from Eqs. 11 and 13. Illumination maps: the
     * right-minus-left intensity residual of each time's stereo pair in the
     * reference frame, low-passed by a Gaussian of illum_sigma level pixels
     * (truncated at ceil(3 sigma), at most 16; edges clamped), box-prolongated,
     * and subtracted from the right images' intensity samples of the next
     * level. Not with the batched solve. */
    int occlusion;                /* 1: occlusion maps on */
    float occ_tau;                /* closeness tolerance, level pixels of disparity (0.5) */
    int illumination;             /* 1: illumination correction maps on */
    float illum_sigma;            /* Gaussian sigma, level pixels (3.2) */
} sf_params;

typedef struct sf_stats {
    int status;                   /* latched device status (sf_status) */
    int frames;                   /* frames solved since sf_create / sf_reset */
    int levels;
    int n_excluded;               /* finest-level pixels with W = 0 in the last step */
    int launches;                 /* kernel launches per frame */
    int pad;
    double energy;                /* final energy of the last frame (Eq. 8) */
    double terms[5];              /* its weighted parts: photo, grad, smooth, epi, mag */
    /* per level and Gauss-Newton step of the last frame */
    double step_energy[SF_MAX_LEVELS][SF_MAX_GN];   /* at the linearisation point */
    double step_accepted[SF_MAX_LEVELS][SF_MAX_GN]; /* after the step */
    float step_t[SF_MAX_LEVELS][SF_MAX_GN];         /* accepted step length, 0 = rejected */
    int step_excluded[SF_MAX_LEVELS][SF_MAX_GN];    /* pixels with W = 0 */
} sf_stats;

typedef struct sf_ctx sf_ctx;

/* Fills *p with a column of Table 1 plus the defaults: eps 0.001, eps_p 0.2,
 * rectified F = [[0,0,0],[0,0,-1],[0,1,0]], 3 Gauss-Newton steps x 20 PCG
 * iterations on every level, IRLS, Brox gradient penalty, feature weight
 * gain 9 and tau 0.001, constant-velocity temporal transfer, FP32, 4
 * backtracks, graph replay on. Returns SF_ERR_ARG for an unknown preset. */
SF_API int sf_params_preset(sf_params* p, int preset);

/* Creates a solver for width x height inputs with warp-grid stride
 * grid_stride (level pixels, same on every level) and `levels` pyramid
 * levels (mip-map, factor 2, Section 5.3). Every level needs at least 2x2
 * pixels and 2x2 grid nodes. Allocates all device memory. Returns NULL on
 * error; sf_last_error() then tells why. */
SF_API sf_ctx* sf_create(int width, int height, int grid_stride, int levels, const sf_params* p);

/* Enqueues one frame of Algorithm 1 on `stream`: pyramid, coarse-to-fine
 * Gauss-Newton/PCG solve (Sections 4-5) from the previous frame's state
 * (temporal transfer, Section 5.3; zero for the first frame after
 * create/reset), and writes the finest total fields to out_fields (device,
 * float32 [6][ny][nx]). The four inputs are device pointers. SF_ERR_ARG for
 * a null pointer; returns before the work ends. */
SF_API int sf_solve(sf_ctx* ctx, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1,
             float* out_fields, void* stream);

/* The same (Algorithm 1) from host memory: copies the four images in (host
 * to device), solves, copies the fields out (device to host) and waits for
 * the stream. Host buffers should be pinned for full copy speed. */
SF_API int sf_solve_host(sf_ctx* ctx, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1,
                  float* out_fields, void* stream);

/* Solves n consecutive frames of one video, continuing from the context's
 * temporal state, and writes every frame's finest fields. frames: device
 * float32 [n][4][h][w] (each frame's L_t, R_t, L_t1, R_t1); outs: device
 * float32 [n][6][ny][nx]. The hierarchy is pipelined across frames: level l of
 * frame f needs only level l + 1 of frame f and level l of frame f - 1
 * (Algorithm 1, Section 5.3), so the levels of consecutive frames run
 * concurrently on the context's streams. The fields equal those of n
 * sf_solve calls. Needs params.video = 1 at sf_create (SF_ERR_STATE
 * otherwise). Enqueued on `stream` (the call returns before the work ends). */
SF_API int sf_solve_video(sf_ctx* ctx, const float* frames, int n, float* outs, void* stream);

/* The same (Algorithm 1, pipelined as above) from host memory (pinned for
 * full copy speed): frames are copied in and fields out through a ring of
 * device slots, overlapped with the solve; waits for the stream before
 * returning. frames: host float32 [n][4][h][w]; outs: host float32
 * [n][6][ny][nx]. SF_ERR_STATE without params.video. */
SF_API int sf_solve_video_host(sf_ctx* ctx, const float* frames, int n, float* outs, void* stream);

/* Level geometry: image size and warp-grid size of `level` (0 = finest;
 * Section 3.3, Eq. 7: node (i, j) at level pixel (i s, j s)). SF_ERR_ARG for
 * a level outside [0, levels); any output pointer may be NULL. */
SF_API int sf_grid_dims(const sf_ctx* ctx, int level, int* w, int* h, int* nx, int* ny);

/* Sets the coarsest level's initial delta for the next sf_solve (6 x G device
 * floats, the fields layout), replacing the temporal rule there once: the
 * place where Section 5.3 transfers the previous frame's flows, used by a
 * warm start of the first frame (smarter initialisation is future work in
 * Section 7). The copy is enqueued on `stream`. */
SF_API int sf_set_init(sf_ctx* ctx, const float* coarsest_delta, void* stream);

/* Forgets the temporal state (Section 5.3): the next frame starts from zero
 * flows, as the first frame does. Waits for the device and clears the
 * latched device status. */
SF_API int sf_reset(sf_ctx* ctx);

/* Waits for the context's work and copies its statistics: the energy of
 * Eq. 8 and its terms, per-step energies, step lengths and outlier counts;
 * out->status carries the latched device status (SF_ERR_TIMEOUT,
 * SF_ERR_NUMERIC), which is also returned. */
SF_API int sf_get_stats(sf_ctx* ctx, sf_stats* out);

/* Copies the final delta and total fields of `level` of the last frame (the
 * deltas and totals the hierarchy stores, Section 5.3) into device buffers
 * (6 x G floats each; either may be NULL). */
SF_API int sf_get_state(sf_ctx* ctx, int level, float* delta, float* total, void* stream);

/* PCG schedule autotuner (the linear solver of Section 5.1): solves one frame of the given quadruple (device
 * pointers), then times every PCG schedule that can run each level (one
 * cluster or the whole GPU, one or two reductions per iteration, 1-4 nodes
 * per four-lane group, distributed shared memory) on that level's last
 * Gauss-Newton system, `reps` launches each after one warm-up, and keeps the
 * fastest per level. Results are cached per process by the level's grid size,
 * iteration count and SM count. Leaves the context reset (the next solve is a
 * first frame) and captures the frame graph again on the next solve. */
SF_API int sf_tune_pcg(sf_ctx* ctx, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1, int reps,
                       void* stream);
/* The PCG schedule of a level: kind 0 grid / 1 cluster (two reductions per
 * iteration), 3 grid / 4 cluster (one reduction), 5 grid (one reduction,
 * coupling blocks staged in shared memory, published vectors as self-tagged
 * 64-bit words: no memory fences in the exchange), 6 grid (pipelined, staged
 * and self-tagged like 5), 2 distributed shared memory; CTAs; nodes per
 * four-lane group. */
SF_API int sf_pcg_schedule(const sf_ctx* ctx, int level, int* kind, int* blocks, int* npt);
/* Sets the PCG schedule of a level (kind, CTAs, nodes per group as
 * sf_pcg_schedule reports them), for a schedule kept from an earlier tuning
 * or picked by the caller's own measure. Only a schedule that sf_tune_pcg
 * would consider for the level is taken; anything else returns SF_ERR_ARG
 * and leaves the context unchanged. Waits for the device; the next solve
 * captures the frame graph again. */
SF_API int sf_set_pcg_schedule(sf_ctx* ctx, int level, int kind, int blocks, int npt);

/* Device time of kernel class `klass` in the last frame: the sum over its
 * launches (ms) and their number. Needs the class in profile_mask; waits for
 * the context's work. */
SF_API int sf_kernel_times(sf_ctx* ctx, int klass, double* total_ms, int* launches);

/* Waits for the device, then frees the context and all of its device
 * memory. NULL is ignored. */
SF_API void sf_destroy(sf_ctx* ctx);
/* A static, human-readable name of a status code. */
SF_API const char* sf_status_string(int status);
/* The status of the calling thread's last failed call (sf_create returns
 * NULL, so its reason is read here). */
SF_API int sf_last_error(void);

/* ---- step-level entry points (parity tests and profiling) --------------
 * Each runs one stage of the solve on the context's buffers for `level`,
 * with caller-given state, on `stream`. All pointers are device pointers. */

/* Builds the pyramid (the mip-map of Section 5.3, with the image gradients
 * that Eqs. 1-6 and 13 sample) from four device images and copies level
 * `level`'s planes out as float32 [4][3][h][w] (I, dI/dx, dI/dy per image). */
SF_API int sf_probe_pyramid(sf_ctx* ctx, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1,
                     int level, float* planes, void* stream);

/* Feature weights w_i (Section 4.3) at totals T (6 x G) on the current
 * pyramid: writes G floats. */
SF_API int sf_probe_feature_weights(sf_ctx* ctx, int level, const float* T, float* wfeat, void* stream);

/* Assembles the Gauss-Newton system (Section 5.1, Eqs. 19-24) at base + delta (6 x G each) with
 * feature weights wfeat (G) on the current pyramid, W taken at that state.
 * Outputs: blocks (G x 5 x 36: the node's own 6x6 block and those coupling
 * it to its E, S, SE and SW neighbours, row-major), rhs (G x 6), energy
 * (1 double: the energy at the state) and W (h*w bytes). */
SF_API int sf_probe_assemble(sf_ctx* ctx, int level, const float* base, const float* delta, const float* wfeat,
                      float* blocks, float* rhs, double* energy, unsigned char* W, void* stream);

/* Runs `iters` Jacobi-preconditioned CG iterations (Section 5.1) from zero on
 * the system last assembled for `level` (by sf_probe_assemble) and writes
 * the solution (G x 6), in the level's current PCG schedule. */
SF_API int sf_probe_pcg(sf_ctx* ctx, int level, int iters, float* x, void* stream);

/* Runs `sweeps` alternating Schwarz sweeps of `patch` local PCG iterations
 * (Section 5.2, SF_SOLVER_SCHWARZ with the context's tile and overlap) on the
 * system last assembled for `level` (by sf_probe_assemble) and writes the
 * solution (G x 6). SF_ERR_ARG if the tiling cannot run on one CTA per
 * subdomain (six threads per node of an extended subdomain, at most 640). */
SF_API int sf_probe_schwarz(sf_ctx* ctx, int level, int sweeps, int patch, float* x, void* stream);

/* The occlusion map V that `level` used in the last frame (h*w bytes, device;
 * 1 = visible): the prolongated map of level + 1, all ones at the coarsest
 * level. Needs params.occlusion = 1 (SF_ERR_STATE otherwise). Frame-by-frame
 * solves only (sf_solve). */
SF_API int sf_probe_vmask(sf_ctx* ctx, int level, unsigned char* V, void* stream);

/* The occlusion map of `level` at totals T (6 x G device floats, the fields
 * layout): O (h*w bytes, device), before prolongation. Needs
 * params.occlusion = 1. */
SF_API int sf_probe_occlusion(sf_ctx* ctx, int level, const float* T, unsigned char* O, void* stream);

/* The low-passed stereo residuals of `level` at totals T on the context's
 * current pyramid (built by sf_probe_pyramid or a solve): R (2 x h x w
 * device floats, time 0 then time 1), before prolongation. Needs
 * params.illumination = 1. */
SF_API int sf_probe_illum(sf_ctx* ctx, int level, const float* T, float* R, void* stream);

/* Copies the outlier mask W (Section 4.1) that Gauss-Newton step `step` of
 * `level` used in the last frame (h*w bytes, 1 = kept, 0 = pruned). */
SF_API int sf_probe_wmask(sf_ctx* ctx, int level, int step, unsigned char* W, void* stream);

/* Energy (Eq. 8) at base + delta with W given (h*w bytes, NULL: taken at the
 * state) and feature weights wfeat; writes 6 doubles: total, then the
 * weighted photo, grad, smooth, epi and mag parts. */
SF_API int sf_probe_energy(sf_ctx* ctx, int level, const float* base, const float* delta, const float* wfeat,
                    const unsigned char* W, double* out6, void* stream);

/* The bilinear cell decisions (reading C7: the cell of a sample at p is
 * min(floor(p), w-2), the position clamped to the image) that the assembly
 * of Gauss-Newton step `step` of `level` took in the last frame for every
 * sample lying within 1e-3 px of a cell edge. A cell is an integer decision
 * taken in FP32, and the analytic Jacobian of Section 5.1 (the derivative of
 * the bilinear interpolant) jumps between cells, so a parity check in
 * another precision replays these decisions like the outlier masks W. Needs
 * params.record_cells = 1 at sf_create (SF_ERR_STATE otherwise; recording
 * costs a few instructions per sample and an atomic per record). Waits for
 * the context's work, writes *n (the number recorded) and copies up to
 * max_recs records of two unsigned ints each, (pixel y*w + x, cell << 4 |
 * clamped << 3 | image << 1 | axis), into the HOST buffer recs (may be NULL),
 * in no particular order. SF_ERR_STATE also if more were recorded than the
 * buffer held (8 per pixel). */
SF_API int sf_probe_cells(sf_ctx* ctx, int level, int step, unsigned* recs, int max_recs, int* n);

/* Measurement aid, no counterpart in the paper: the FP32 fused
 * multiply-add rate of the current GPU (flops/s, an FMA counted as two), the
 * roofline denominator of the ALU-bound assembly of Section 5.1. Runs a
 * kernel of eight independent FMA chains per thread on every SM `reps` times
 * (1..100) on `stream`, waits, and writes the best rate. */
SF_API int sf_probe_fma_rate(int reps, double* flops_per_s, void* stream);

/* ---- failure detection, exercised without a fault ---------------------
 * The device-wide waits of this library (the grid barriers of the PCG,
 * Schwarz and trial kernels, the mbarrier waits of the tensor-core GEMM) are
 * bounded: a wait that runs out latches a status bit and returns, so a lost
 * block never hangs the GPU. These calls run the same wait code with a
 * short limit on a condition that a test controls; they have no counterpart
 * in the paper.
 *
 * sf_probe_barrier_timeout: a cooperative launch of one block per SM passes
 * one grid barrier (the library's own, limit `limit_cycles` SM clocks);
 * block `skip_block` never arrives (-1: every block arrives). Waits for the
 * launch and writes the latched status (*status: SF_OK, or SF_ERR_TIMEOUT
 * when the barrier ran out) and the number of blocks that came back from the
 * barrier (*returned). Allocates its own small device buffers. */
SF_API int sf_probe_barrier_timeout(int skip_block, long long limit_cycles, int* status, int* returned);
/* sf_probe_mbarrier_timeout: one block waits on a shared-memory mbarrier of
 * arrival count 1 (the GEMM's wait, limit `limit_cycles`); with arrive = 1
 * one thread arrives first, with arrive = 0 nothing does. *completed: 1 if
 * the wait saw the phase complete, 0 if it ran out. */
SF_API int sf_probe_mbarrier_timeout(int arrive, long long limit_cycles, int* completed);
/* sf_probe_tagged_timeout: the waits of the self-tagged PCG exchange
 * (schedule kinds 5 and 6), limit `limit_cycles` SM clocks, in a cooperative
 * launch of min(SMs, 160) blocks. mode 0: every block but `skip_block`
 * publishes its tagged partial-sum words and every block polls all blocks'
 * words; mode 1: every block but `skip_block` publishes one tagged word and
 * every block waits for the next block's word, as a halo reader does.
 * skip_block = -1: every block publishes. Waits for the launch and writes the
 * latched status (*status: SF_OK, or SF_ERR_TIMEOUT when a wait ran out) and
 * the number of blocks that came back (*returned). SF_ERR_ARG for a mode
 * other than 0 or 1, a limit outside [1, 4e9] or skip_block past the grid.
 * Allocates its own small device buffers. */
SF_API int sf_probe_tagged_timeout(int mode, int skip_block, long long limit_cycles, int* status, int* returned);

/* C[s][M][N] = A[M, K] * B[N, K]^T over split s of K (K split into `splits`
 * contiguous ranges of 64-wide chunks; the splits' partial products are
 * written separately), on the tensor cores: A and B device BF16, row-major
 * with K contiguous, K a multiple of 64, N a multiple of 16, BN the N tile
 * (16..256, a multiple of 16), C device FP32. The primitive of the
 * warm-start network's convolutions; waits for the stream. SF_ERR_TIMEOUT
 * if a tensor-core wait timed out. */
SF_API int sf_probe_gemm_bf16(const void* A, const void* B, int M, int N, int K, int BN, int splits, float* C,
                              void* stream);

/* ---- learned warm start --------------------------------------------------
 * The paper starts the first frame from zero flows and names a smarter
 * first-frame initialisation as future work (Section 7). The warm start is a
 * six-layer convolutional network (3x3 kernels, zero padding 1, ReLU after
 * all but the last layer: 4->32 stride 2, 32->64 stride 2, 64->64 stride 2,
 * 64->64, 64->32, 32->6) that maps the four coarsest-level images of a
 * quadruple (60 x 80, the coarsest level of 640 x 480 with four levels), less
 * 1/2, to the coarsest level's six delta fields on its 8 x 10 warp grid; the
 * prediction replaces the zero start of the coarsest level. Training and
 * inference run on the GPU: every convolution is a BF16 tensor-core GEMM
 * with FP32 accumulation; biases, master weights, gradients and the Adam
 * moments are FP32.
 *
 * Parameters travel as one FP32 vector in the standard layout: for each layer
 * in order its weights [out][in][3][3], then its biases [out]
 * (sf_net_param_count() floats). Images: device FP32 [B][4][60][80];
 * outputs and targets: device FP32 [B][6][8][10]. */
typedef struct sf_net sf_net;
SF_API int sf_net_param_count(void);
/* Allocates a network for batches of up to max_batch quadruples. */
SF_API int sf_net_create(int max_batch, sf_net** out);
/* Loads parameters (device FP32, standard layout) and clears the Adam state. */
SF_API int sf_net_set_params(sf_net* n, const float* params, void* stream);
SF_API int sf_net_get_params(sf_net* n, float* params, void* stream);
SF_API int sf_net_forward(sf_net* n, const float* imgs, int batch, float* out, void* stream);
/* Forward and backward pass of the mean squared error against target:
 * writes the gradient (device, standard layout; may be NULL) and the loss
 * (device float; may be NULL). */
SF_API int sf_net_gradients(sf_net* n, const float* imgs, const float* target, int batch, float* grads, float* loss,
                            void* stream);
/* One training step: forward, backward and an Adam update (beta1 0.9, beta2
 * 0.999, epsilon 1e-8, bias-corrected) with learning rate lr. */
SF_API int sf_net_train_step(sf_net* n, const float* imgs, const float* target, int batch, float lr, float* loss,
                             void* stream);
/* Waits for the device; SF_ERR_TIMEOUT if a tensor-core wait timed out. A
 * timed-out tile waits once more for its tensor-core work in flight; if that
 * also gives up, the work may still be running on memory the tile released,
 * and the CUDA context is to be treated as poisoned: the caller should stop
 * launching work on it (destroy it, or end the process). */
SF_API int sf_net_status(sf_net* n);
SF_API void sf_net_destroy(sf_net* n);
/* The coarsest-level intensities of a quadruple (device FP32 [4][h][w] of
 * the context's coarsest level), through the context's pyramid kernels. */
SF_API int sf_coarsest_images(sf_ctx* ctx, const float* L_t, const float* R_t, const float* L_t1, const float* R_t1,
                              float* out, void* stream);
/* Predicts the coarsest level's initial delta of the next sf_solve on ctx
 * from the quadruple (the context's coarsest level must be 80 x 60 with an
 * 8 x 10 grid; SF_ERR_ARG otherwise), as sf_set_init would set it. */
SF_API int sf_warm_start(sf_net* n, sf_ctx* ctx, const float* L_t, const float* R_t, const float* L_t1,
                         const float* R_t1, void* stream);

/* ---- batched solve of many sequences ----------------------------------
 * The paper solves one stereo sequence at a time (Algorithm 1). These calls
 * solve n independent sequences of any sizes together: each frame step runs
 * Algorithm 1 once for every sequence in ONE kernel launch, one thread-block
 * cluster per sequence (its stages meet at the hardware cluster barrier), the
 * launch captured once into a CUDA graph and replayed. All sequences share
 * the parameters and the grid stride; each has its own size and level count
 * and its own temporal state. FP32 texels only (params.precision must be
 * SF_FP32), and params.gn_iters[0] >= 1.
 *
 * Inputs and outputs are packed device buffers: sequence i's four images
 * (L_t, R_t, L_t1, R_t1, each w_i * h_i floats) start at float offset
 * in_offsets[i] of `in`, its finest fields (float32 [6][ny][nx]) at
 * out_offsets[i] of `out`; sf_batch_layout gives the offsets and totals
 * (sequences in the order given, each packed after the previous one). */
typedef struct sf_batch sf_batch;

/* Creates a batch of n sequences (widths[i] x heights[i], levels[i] levels,
 * each as sf_create would accept) and allocates all device memory. Writes
 * the batch to *out; returns SF_OK or an error code. */
SF_API int sf_batch_create(int n, const int* widths, const int* heights, const int* levels, int grid_stride,
                           const sf_params* p, sf_batch** out);

/* Offsets (floats) of each sequence in the packed input and output buffers
 * (arrays of n entries, either may be NULL) and the buffer sizes. */
SF_API int sf_batch_layout(const sf_batch* b, size_t* in_offsets, size_t* out_offsets, size_t* in_total,
                           size_t* out_total);

/* Enqueues one frame step of every sequence on `stream` (returns before the
 * work ends). `in` and `out` are device buffers in the packed layout. */
SF_API int sf_batch_solve(sf_batch* b, const float* in, float* out, void* stream);

/* Schedule of the launch: CTAs per sequence (`cluster`, a power of two up to
 * 16) and the divisor of the cells each CTA assembles at a time (cpb_div,
 * 1..4; 1 = as many cells as one pass of 256 threads covers). SF_ERR_ARG if
 * the GPU cannot hold one such cluster. */
SF_API int sf_batch_set_schedule(sf_batch* b, int cluster, int cpb_div);
SF_API int sf_batch_get_schedule(const sf_batch* b, int* cluster, int* cpb_div);

/* Autotuner: times `steps` frame steps on in/out (after one warm-up) for
 * every schedule the GPU can hold (clusters of 2..16 CTAs, cpb_div 1 and 2),
 * keeps the fastest and writes its time per step (ms) to best_ms (may be
 * NULL). Results are cached per process, keyed by the batch's shape (sizes,
 * levels, stride, iteration counts): a later batch of the same shape takes
 * the cached schedule without timing. Runs only before the first frame
 * (SF_ERR_STATE otherwise) and leaves every sequence at frame 0. */
SF_API int sf_batch_tune(sf_batch* b, const float* in, float* out, int steps, void* stream, float* best_ms);

/* The context of sequence i, owned by the batch (do not destroy it): for
 * sf_get_stats, sf_get_state, sf_probe_wmask and sf_grid_dims. */
SF_API sf_ctx* sf_batch_sequence(sf_batch* b, int i);

/* Forgets every sequence's temporal state and status. */
SF_API int sf_batch_reset(sf_batch* b);
SF_API void sf_batch_destroy(sf_batch* b);

/* ---- allocation-free PCG ------------------------------------------------
 * The paper has no counterpart to this call: it exists for callers that
 * cannot allocate device memory where they solve: real-time loops that must
 * not meet the allocator's implicit device synchronisation, and host
 * applications whose memory pool or fixed device budget forbids a library's
 * raw allocations after start-up.
 *
 * Runs `iters` Jacobi-preconditioned CG iterations (Section 5.1) from x = 0
 * on a block system in the layout sf_probe_assemble writes: blocks [G][5][6][6] (each
 * node's own block and those coupling it to its E, S, SE and SW neighbours,
 * row-major), rhs [G][6]; writes x [G][6]; G = nx * ny, all device memory,
 * enqueued on `stream`. Allocates nothing: its scratch is one file-scope
 * device array sized for SF_STATIC_PCG_MAX_NODES nodes (288 KiB), held by
 * every GPU that loads the library until exit; a larger G returns SF_ERR_ARG
 * without touching the GPU. The first call on a device looks the array's
 * device address up (cudaGetSymbolAddress) with that device current, so make
 * that first call before any stream capture. The looked-up address is kept
 * for the rest of the process: after cudaDeviceReset on a device, do not call
 * sf_pcg_static on that device again in the same process (the reloaded
 * library image may sit elsewhere). All calls share the array and
 * every call writes what it reads before reading it; calls that overlap on
 * the GPU (other streams, other host threads) race on it. */
#define SF_STATIC_PCG_MAX_NODES 4096
SF_API int sf_pcg_static(int nx, int ny, const float* blocks, const float* rhs, int iters, float* x, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SF_H */
