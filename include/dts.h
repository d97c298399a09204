/*
 * dts.h -- C ABI of the GB300 Domain Transform Solver library (libdts.so).
 *
 * The Domain Transform Solver (Bapat & Frahm, "The Domain Transform Solver",
 * ECCV 2018) minimises, for a target t with per-pixel confidence c under a
 * C-channel guide image I,
 *     F(z) = lambda/2 sum_i (z_i - zbar_i)^2 + sum_i c_i (z_i - t_i)^2      (Eq. 1-2)
 * where zbar = A z is the edge-aware mean (Eq. 10) computed with the domain
 * transform (§3.2): distances between neighbouring pixels (Eq. 8-9) feed a
 * recursive filter (causal then anti-causal first-order recurrence along every
 * row, then every column, for N passes with a halving sigma schedule).  The
 * solver iterates the gradient step of Eq. 3 with step 0.99 (§4) or the fixed
 * point of Eq. 4.
 *
 * Conventions for every entry point
 *  - All image pointers are DEVICE pointers owned by the caller; the library
 *    never allocates, frees or keeps them.  Scratch memory is the caller's
 *    workspace (size from dts_workspace_size), at least 256-byte aligned.
 *  - Single-channel images (target, confidence, z, gradients) are dense H x W
 *    row-major (row stride W elements).  The guide is planar C x H x W with
 *    the strides given in dts_guide.
 *  - Calls are asynchronous on `stream` (NULL = the legacy default stream).
 *    Argument errors are returned synchronously and launch nothing.  Errors
 *    detected on the device (a bounded wait that gave up) are recorded in a
 *    per-device status word that dts_last_status() returns.  No kernel traps.
 *  - Return value: a dts_status code (DTS_OK = 0).
 */
#ifndef DTS_H
#define DTS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream. */
typedef struct CUstream_st* dts_stream;

typedef enum dts_status {
    DTS_OK = 0,
    DTS_ERR_INVALID_ARG = 1, /* a size, pointer, alignment or parameter is out of range */
    DTS_ERR_UNSUPPORTED = 2, /* valid but not implemented (e.g. a line longer than the kernels hold) */
    DTS_ERR_WORKSPACE = 3,   /* workspace missing, too small or misaligned */
    DTS_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    DTS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (reported by dts_last_status) */
    DTS_ERR_NONFINITE = 6    /* reserved: non-finite values detected */
} dts_status;

typedef enum dts_dtype { DTS_F32 = 0, DTS_BF16 = 1, DTS_F16 = 2 } dts_dtype;
typedef enum dts_norm { DTS_NORM_L1 = 0, DTS_NORM_L2 = 1 } dts_norm;
typedef enum dts_update { DTS_UPDATE_GD = 0, DTS_UPDATE_JACOBI = 1, DTS_UPDATE_CG = 2 } dts_update;
typedef enum dts_conf_mode { DTS_CONF_PLAIN = 0, DTS_CONF_SUPPORT = 1 } dts_conf_mode;
typedef enum dts_filter_kernel { DTS_KERNEL_RF = 0, DTS_KERNEL_BOX = 1 } dts_filter_kernel;

/* Planar guide image I: channel k, row y, column x is element
 * k * ch_stride + y * row_stride + x of `data` (dtype F32, BF16 or F16).
 * row_stride = 0 means W; ch_stride = 0 means H * row_stride.
 * Requires C >= 1, H >= 1, W >= 1, row_stride >= W, ch_stride >= H * row_stride. */
typedef struct dts_guide {
    int C, H, W;
    int dtype;              /* dts_dtype */
    const void* data;       /* device pointer */
    long long ch_stride;    /* elements */
    long long row_stride;   /* elements */
} dts_guide;

/* Solver parameters (names follow the paper).
 *  lambda      weight of the edge-aware regulariser (Eq. 1), >= 0
 *  sigma_s     spatial standard deviation in pixels (sigma_x = sigma_y, §4), > 0
 *  sigma_r     range standard deviation in guide units (§4: colours in [0, 1]), > 0
 *  step        gradient step eta of Eq. 3 (§4 uses 0.99), > 0
 *  iterations  solver iterations K >= 0 (§4: 3000 for stereo, 10 for depth SR)
 *  passes      recursive-filter passes N per edge-aware mean, 1..16 (3 by default)
 *  norm        distance norm: DTS_NORM_L1 (1 + sigma_s/sigma_r sum_k |dI_k|) or
 *              DTS_NORM_L2 (sqrt(1 + (sigma_s/sigma_r)^2 sum_k dI_k^2), §3.2)
 *  update      DTS_UPDATE_GD (Eq. 3), DTS_UPDATE_JACOBI (Eq. 4), or DTS_UPDATE_CG:
 *              conjugate gradients (named in §5 as the way to faster convergence) on the
 *              objective of Eq. 2 itself, lambda/2 |z - A z|^2 + sum_i c_i (z_i - t_i)^2,
 *              i.e. on (lambda (I - A)^T (I - A) + 2 C) z = 2 C t from z_0 (target or z_init);
 *              `iterations` CG steps, `step` unused; DTS_KERNEL_RF, DTS_CONF_PLAIN and no
 *              checkpoints only (else DTS_ERR_UNSUPPORTED), no backward.  Each step applies
 *              A and A^T (4N passes) plus three elementwise kernels with FP64 dot products
 *  conf_mode   DTS_CONF_PLAIN (c as given) or DTS_CONF_SUPPORT (c weighted by
 *              S_flat / sum_j W_ij, §3.1 after Eq. 6)
 *  dist_dtype  storage of the distance planes: DTS_F32 or DTS_F16
 *  filter_kernel  DTS_KERNEL_RF (default): the recursive-filter kernel; DTS_KERNEL_BOX: the
 *              box kernel Eq. 10 prints, W_ij = 1 if |DT_i - DT_j| <= r with r = sigma_i sqrt(3)
 *              per pass (normalized convolution in the transformed domain); FP32 distances,
 *              DTS_CONF_PLAIN and no checkpoints only, lines up to 8192 positions, no backward
 *  charbonnier_eps  0 (default): the square (z - t)^2 on the target term.  > 0: the
 *              Charbonnier loss sqrt((z - t)^2 + eps^2) that §4 uses for stereo (eps = 0.001);
 *              DTS_UPDATE_GD: the gradient step of Eq. 3 takes c (z - t) / sqrt((z - t)^2 + eps^2)
 *              for the data term (its curvature c / eps makes the step unstable where c > eps);
 *              DTS_UPDATE_JACOBI: the fixed point of Eq. 4 with the loss's weight at the
 *              current iterate, c~ = c / sqrt((z_k - t)^2 + eps^2) in place of c (stable at any
 *              eps; its fixed points solve lambda (z - A z) + c rho'(z - t) = 0 like the gradient
 *              step's); not with DTS_UPDATE_CG.  Forward and backward
 *  save_checkpoints  0: nothing kept; 1: dts_solve keeps z_0 .. z_{K-1} in the
 *              workspace for dts_solve_backward (workspace sized with with_backward = 1),
 *              which recomputes each iteration's pass inputs from them; 2: it also keeps
 *              every pass input and the filtered iterate of every iteration (K x 2N more
 *              planes: the passes write them instead of overwriting one plane, at no extra
 *              traffic), so the backward skips the recompute */
typedef struct dts_params {
    float lambda, sigma_s, sigma_r, step;
    int iterations, passes;
    int norm, update, conf_mode;
    int dist_dtype;
    int save_checkpoints;
    int filter_kernel;
    float charbonnier_eps;
} dts_params;

/* Human-readable name of a status code (static string). */
const char* dts_status_string(int status);

/* Library version string (static). */
const char* dts_version(void);

/* Bytes of workspace that dts_filter / dts_solve (with_backward = 0) or
 * dts_solve with save_checkpoints plus dts_solve_backward (with_backward = 1)
 * need for this guide and these parameters.  0 on invalid arguments. */
size_t dts_workspace_size(const dts_guide* guide, const dts_params* params, int with_backward);

/* Domain-transform distances (§3.2, Eq. 8-9) between neighbouring pixels:
 *   dX[y][x] between (y, x-1) and (y, x), dY[y][x] between (y-1, x) and (y, x),
 *   L1: 1 + (sigma_s/sigma_r) sum_k |I_k(p) - I_k(q)|;  L2: sqrt(1 + (sigma_s/sigma_r)^2 sum_k (I_k(p) - I_k(q))^2).
 * dX[y][0] and dY[0][x] have no neighbour and are written as 1.
 * Outputs are dense H x W planes of params->dist_dtype (F32 or F16).
 * Uses params->sigma_s, sigma_r, norm, dist_dtype only. */
int dts_domain_transform(const dts_guide* guide, const dts_params* params, void* dX, void* dY, dts_stream stream);

/* Edge-aware mean dst = A src (Eq. 10 with the recursive-filter kernel of §3.2):
 * A = V(a_N) H(a_N) ... V(a_1) H(a_1), the horizontal pass first; pass i uses
 * sigma_i = sigma_s sqrt(3) 2^(N-i) / sqrt(4^N - 1) and a_i = exp(-sqrt(2)/sigma_i),
 * and each 1-D pass runs J[n] = (1 - w) x[n] + w J[n-1] with w = a_i^d forward and
 * then backward along the line.  src and dst are dense H x W FP32 and may alias. */
int dts_filter(const dts_guide* guide, const dts_params* params, const float* src, float* dst, void* ws,
               size_t ws_bytes, dts_stream stream);

/* The solver (§3.1): z_0 = z_init (or the target when z_init is NULL), then K times
 *   zbar = A z_k;  z_{k+1} = z_k - step (lambda (z_k - zbar) + c (z_k - t))       (GD, Eq. 3)
 *                  or (lambda zbar + c t) / (lambda + c)                           (Jacobi, Eq. 4)
 * target: dense H x W of target_dtype (F32, BF16 or F16); conf: dense H x W FP32
 * (c >= 0); z_out: dense H x W FP32 (may alias z_init, not target/conf).
 * With save_checkpoints = 1 the iterates z_0 .. z_{K-1} stay in the workspace.
 * With DTS_RESIDENT=1 in the environment (read on every call), a solve of at least 2^20 pixels
 * with the recursive filter, GD or Jacobi, plain confidence, FP32 distances and no checkpoints
 * runs its iterations as one cooperative kernel launch holding the iterate in shared memory (one
 * CTA per SM, so it waits for the whole GPU); dts_workspace_size must then be called with the
 * same setting.  Off by default. */
int dts_solve(const dts_guide* guide, const void* target, int target_dtype, const float* conf, const float* z_init,
              const dts_params* params, float* z_out, void* ws, size_t ws_bytes, dts_stream stream);

/* Confidence from the edge-aware variance of the target (Eq. 7, §3.1):
 *   V = DT(t^2) - DT(t)^2,   c = exp(-V / (2 sigma_c^2)),
 * with DT the edge-aware mean of Eq. 10 (the filter of dts_filter: distances and passes from
 * `params`).  The paper gives no value for sigma_c: the caller chooses it (sigma_c > 0, in the
 * units of t).  V below 0 can only come from rounding and is taken as 0, so 0 < c <= 1.
 * target: dense H x W of target_dtype (F32, BF16 or F16); conf_out: dense H x W FP32.
 * Workspace as for dts_filter (dts_workspace_size with with_backward = 0).  Argument errors
 * (including sigma_c <= 0) are DTS_ERR_INVALID_ARG, returned before any device work; the box
 * kernel (filter_kernel = DTS_KERNEL_BOX) is DTS_ERR_UNSUPPORTED here. */
int dts_confidence(const dts_guide* guide, const void* target, int target_dtype, const dts_params* params,
                   float sigma_c, float* conf_out, void* ws, size_t ws_bytes, dts_stream stream);

/* Reverse mode of dts_solve (the paper has no backward; the adjoint of each
 * recurrence is the same recurrence run in the opposite direction).  Must follow
 * a dts_solve with the same arguments, save_checkpoints = 1 and this workspace
 * (sized with with_backward = 1), which holds the checkpoints it reads.
 * grad_z: dL/dz_K (H x W FP32).  Outputs (each may be NULL, all FP32 dense):
 *   grad_target H x W (includes the z_0 = target path when z_init is NULL),
 *   grad_conf H x W, grad_guide C x H x W (through the distances; L1 uses sign(0) = 0),
 *   grad_z_init H x W (only meaningful when z_init was given).
 * Supports conf_mode = DTS_CONF_PLAIN only. */
int dts_solve_backward(const dts_guide* guide, const void* target, int target_dtype, const float* conf,
                       const float* z_init, const dts_params* params, void* ws, size_t ws_bytes, const float* grad_z,
                       float* grad_target, float* grad_conf, float* grad_guide, float* grad_z_init,
                       dts_stream stream);

/* dts_solve without a caller workspace.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory (code inside a host framework that owns every
 * device allocation, or a latency-critical loop where an allocation could block, fail or break
 * a fixed memory budget) and so cannot pass a workspace.  Arguments and results are those of
 * dts_solve with the recursive-filter kernel (filter_kernel = DTS_KERNEL_BOX returns
 * DTS_ERR_UNSUPPORTED here); inputs and outputs are still the caller's.  The scratch is a
 * 16 MiB device array inside the library (dts_noalloc_max_workspace() bytes), reserved on a
 * device when the library's module is loaded there -- with CUDA's lazy module loading, at the
 * first libdts call on that device, so make that first call (this one or any other) outside a
 * latency-critical loop -- and held until the process exits; problems whose
 * dts_workspace_size(with_backward = 0) exceeds it return DTS_ERR_WORKSPACE (16 bytes per padded
 * pixel with FP32 distances: about one megapixel), and save_checkpoints = 1 returns
 * DTS_ERR_UNSUPPORTED.  It allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * call.  The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  All calls share the
 * one array and it keeps the last call's contents (every plane a solve reads is written by that
 * solve first): calls that overlap on the GPU, on any streams, race and give wrong results. */
int dts_solve_noalloc(const dts_guide* guide, const void* target, int target_dtype, const float* conf,
                      const float* z_init, const dts_params* params, float* z_out, dts_stream stream);

/* Size in bytes of the scratch array dts_solve_noalloc uses. */
size_t dts_noalloc_max_workspace(void);

/* Workspace bytes for dts_solve_batched over these n guides (0 on invalid arguments). */
size_t dts_batched_workspace_size(int n, const dts_guide* guides, const dts_params* params);

/* n independent solves of uneven sizes (the same parameters) as ONE CUDA graph launch on `stream`,
 * the graph cached per argument set (pointers, shapes, parameters) and replayed by later calls
 * with the same arguments.  When the batch allows it -- the recursive filter, GD or Jacobi (with
 * or without the Charbonnier loss), plain confidence, iterations >= 1, at most 96 images of at
 * most 1088 x 8192 with one guide dtype -- the graph holds one persistent kernel (after a reset of
 * its control words): every image's solve is cut into stages (distances; per iteration N
 * horizontal and N vertical passes, the update fused into the first horizontal pass; the last
 * update) and the stages into jobs (groups of rows, 8-column strips), which the kernel's CTAs take
 * from one queue in stage order, each job waiting (bounded) for its image's previous stage.
 * Otherwise (or under the "batch 1" policy, see dts_autotune_batched) each image's launch sequence
 * is captured on a few internal streams forked from one origin, so small images run side by side.
 * If `stream` is being captured by the caller, the launches join the caller's graph instead.
 * guides, targets, confs and z_out are HOST arrays of n entries (device pointers, as in dts_solve;
 * target_dtype shared); z_init is the target; save_checkpoints must be 0.  The workspace holds the
 * kernel's control words, then one slice per image. */
int dts_solve_batched(int n, const dts_guide* guides, const void* const* targets, int target_dtype,
                      const float* const* confs, const dts_params* params, float* const* z_out, void* ws,
                      size_t ws_bytes, dts_stream stream);

/* Autotuner for a batch (not part of the paper's method): times dts_solve_batched on these
 * arguments with the persistent kernel and with the graph of per-image launches (2 warm-up and 3
 * timed runs each on `stream`) and keeps the faster for later batched solves ("batch 0" or
 * "batch 1" in dts_autotune_export).  A batch the persistent kernel does not take is solved once
 * and leaves the choice as it is.  Synchronises `stream`.  Arguments as for dts_solve_batched. */
int dts_autotune_batched(int n, const dts_guide* guides, const void* const* targets, int target_dtype,
                         const float* const* confs, const dts_params* params, float* const* z_out, void* ws,
                         size_t ws_bytes, dts_stream stream);

/* Autotuner (not part of the paper's method): for this guide's height and width, times each
 * candidate vertical tile shape (rows per thread x warps per CTA x cluster size, where cluster
 * size 0 is the cluster-free kernel with one CTA per 8-column strip) and horizontal
 * segment length with CUDA events on `stream`, using the workspace (sized for dts_filter) and the
 * guide's real distances, and records the fastest; later calls for the same height / width use
 * them.  Synchronises `stream`.  The results live in the process (see dts_autotune_export). */
int dts_autotune(const dts_guide* guide, const dts_params* params, void* ws, size_t ws_bytes, dts_stream stream);

/* Text of the recorded shapes: "row W items" lines (positions per thread of the horizontal
 * passes), "col H items warps cluster" lines (the vertical passes: cluster > 0 CTAs of `warps`
 * warps of `items` rows per thread; 0 the strip kernel; -1 the chained CTAs; -2 the persistent
 * TMA-fed clusters for tall columns) and "bcol H items warps cluster" lines (the vertical passes
 * of dts_solve_backward: cluster > 0, or -1 chained), and a "batch P" line (P = 0: batched solves
 * run the persistent kernel where the batch allows it; 1: the graph of per-image launches).
 * Batched solves on the graph of launches take the cluster shapes for their vertical passes.  With buf == NULL returns the bytes needed (including the terminating
 * 0); else copies and returns that count, or minus DTS_ERR_INVALID_ARG when len is too small. */
int dts_autotune_export(char* buf, size_t len);

/* Records shapes from text in the format of dts_autotune_export (shapes that are not valid
 * candidates for their size are ignored).  DTS_ERR_INVALID_ARG on malformed text. */
int dts_autotune_import(const char* text);

/* Synchronises `stream`, then returns and clears the device-side status word of
 * the current device (DTS_OK, or e.g. DTS_ERR_TIMEOUT), or DTS_ERR_CUDA if the
 * synchronisation itself failed. */
int dts_last_status(dts_stream stream);

/* ---- fault injection for tests (host-requested, one-shot; nothing faults or traps) ----
 * Each kind makes one bounded device-side wait of the next matching launch run out (about a
 * millisecond under injection instead of about a second): the kernel records DTS_ERR_TIMEOUT,
 * which dts_last_status() then returns, issues no further copies into the memory the failed wait
 * guarded, finishes (its results are invalid) and leaves the context usable.
 * DTS_INJECT_TMA_SKIP: the next vertical pass on the strip kernel (columns up to 2176 rows), when
 *   its grid covers every strip in one round, leaves out the first slab load of warp 0 of CTA 0.
 * DTS_INJECT_CHAIN_SKIP: the next chained vertical pass (taller columns) does not count the
 *   arrival of its first chunk, so the CTAs of the first strip wait for a composition that
 *   never comes.
 * DTS_INJECT_BARRIER_SKIP: the next resident solve (DTS_RESIDENT=1) leaves out CTA 0's arrival
 *   at its first grid-wide barrier.
 * DTS_INJECT_QUEUE_SKIP: the next persistent batched solve does not count its first job done, so
 *   the jobs of that image's next stage wait for it.
 * DTS_INJECT_STAGE_SKIP: the next horizontal pass on the streaming row kernel (rows over 8192
 *   columns by default) leaves out CTA 0's copies of its first row.
 * kind 0 cancels; DTS_ERR_INVALID_ARG for unknown kinds. */
#define DTS_INJECT_TMA_SKIP 1
#define DTS_INJECT_CHAIN_SKIP 2
#define DTS_INJECT_BARRIER_SKIP 3
#define DTS_INJECT_QUEUE_SKIP 4
#define DTS_INJECT_STAGE_SKIP 5
int dts_debug_inject(int kind);

/* ---- per-launch kernel timing (a tracing aid; not part of the paper's method) ----
 * mode 1: clear the record and start bracketing every kernel the library launches with two
 * CUDA events on that launch's stream; mode 2: resume without clearing; mode 0: stop.
 * Host-side only; it does not change what the kernels compute (events between kernels do
 * prevent the programmatic early launch of the next kernel; batched solves issue their launches
 * directly instead of replaying their cached graph).  DTS_ERR_INVALID_ARG for other modes. */
int dts_profile(int mode);

/* Copies up to max_records records of the launches made since dts_profile(1), in launch
 * order: kernel id (see dts_kernel_name), pixels the launch covered, flags (bit 0: FP16
 * distance planes, bit 1: 16-bit target) and the event-timed duration in milliseconds.
 * Any output pointer may be NULL.  Waits for the recorded events.  Returns the number of
 * records copied, or minus a dts_status. */
int dts_profile_read(int max_records, int* kernel, long long* pixels, int* flags, float* ms);

/* Name of a kernel id reported by dts_profile_read (static string). */
const char* dts_kernel_name(int kernel);

#ifdef __cplusplus
}
#endif

#endif /* DTS_H */
