// Internal declarations shared by the libdts translation units (not installed).
//
// Data layout inside the workspace: every plane (distances, working buffer,
// iterates) is H rows of `pitch` elements, pitch = W rounded up to 64, each
// plane starting on a 256-byte boundary.  Rows are therefore 16-byte aligned
// and the kernels load and store them with 16-byte vector accesses; the
// padding columns [W, pitch) may hold anything and are masked on load.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdlib.h>

#include "../../include/dts.h"

namespace dts {

constexpr int kPitchAlign = 64;     // elements
constexpr size_t kPlaneAlign = 256; // bytes
constexpr int kMaxPasses = 16;

// Programmatic dependent launch between consecutive kernels: every launch allows it.
inline bool pdl_enabled() { return true; }

inline long long pitch_for(int W) { return ((long long)W + kPitchAlign - 1) / kPitchAlign * kPitchAlign; }

// ---------------------------------------------------------------- device helpers
template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// Element of a dense plane of runtime dtype (target storage).
__device__ __forceinline__ float load_any(const void* p, long long i, int dtype) {
    if (dtype == DTS_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
    if (dtype == DTS_F16) return __half2float(static_cast<const __half*>(p)[i]);
    return static_cast<const float*>(p)[i];
}

// Slope of the target term's loss per unit confidence at r = z - t: r for the square of Eq. 3,
// r / sqrt(r^2 + eps^2) for the Charbonnier loss sqrt(r^2 + eps^2) of §4 (eps > 0).
__device__ __forceinline__ float target_slope(float r, float eps) {
    return eps > 0.f ? r / sqrtf(fmaf(r, r, eps * eps)) : r;
}

// One data-term update of the solver at a pixel: z = z_k, zb = zbar = A z_k, t, c (confidence,
// or the support-weighted confidence).
//   GD (Eq. 3):      z - step (lambda (z - zb) + c rho'(z - t)), with the step limited to
//                    1 / (lambda + c) when clamp is set; rho'(r) = target_slope(r, eps)
//   Jacobi (Eq. 4):  (lambda zb + c~ t) / (lambda + c~); z is kept where lambda + c~ = 0; c~ = c
//                    for the square, c / sqrt((z - t)^2 + eps^2) for the Charbonnier loss (its
//                    weight at the current iterate)
__device__ __forceinline__ float dts_update_value(float z, float zb, float t, float c, float lambda, float step,
                                                  int update, int clamp, float eps) {
    if (update == DTS_UPDATE_JACOBI) {
        float cw = c;
        if (eps > 0.f) {
            const float r = z - t;
            cw = c * rsqrtf(fmaf(r, r, eps * eps));
        }
        const float den = lambda + cw;
        return den != 0.f ? (lambda * zb + cw * t) / den : z;
    }
    float eta = step;
    if (clamp && lambda + c > 0.f) eta = fminf(eta, 1.f / (lambda + c));
    return z - eta * (lambda * (z - zb) + c * target_slope(z - t, eps));
}

// ---------------------------------------------------------------- kernel arguments
struct DistArgs {
    const void* guide;
    long long ch_stride, row_stride;
    int C, H, W, gdtype, norm;
    int dhalf;              // distance planes stored as FP16
    float k;                // sigma_s / sigma_r
    void* dX;
    void* dY;
    long long pitch;        // element pitch of dX/dY
    // optional fused copy of an H x W plane (pitch W, dtype src_dtype) into dst (pitch `pitch`, FP32)
    const void* src;
    int src_dtype;
    float* dst;
    // optional second copy of dY tiled by 8-column strips (the strip kernel's layout): element
    // (y, x) at ((x / 8) * ys_rows + y) * 8 + x % 8
    void* dYs;
    long long ys_rows;
};

// One directional pass over lines of a plane held in the workspace.
struct PassArgs {
    const void* d_tiled;    // vertical passes: the distances tiled by 8-column strips (or null)
    long long d_tiled_rows; // rows per strip of d_tiled
    const float* src;       // pass input (pitch `pitch`)
    float* dst;             // pass output (may equal src)
    long long dst_pitch;    // pitch of dst (vertical passes; horizontal passes use `pitch`)
    const void* d;          // distances along the pass direction (pitch `pitch`)
    int H, W;
    long long pitch;
    float k2;               // log2(a_i): w = exp2(k2 * d)
    // update epilogue (last vertical pass of an iteration only)
    const float* zk;        // z_k (pitch `pitch`); vertical PASS_TRANSPOSE: optional minuend
                            // (the pass then filters zk - src)
    const void* t;          // target (dense, pitch W, dtype t_dtype)
    int t_dtype;
    const float* c;         // confidence (dense pitch W) -- or chat (pitch `pitch`) when c_pitched
    int c_pitched;
    float* zout;            // z_{k+1}
    long long zout_pitch;
    float lambda, step;
    int update;             // DTS_UPDATE_GD / DTS_UPDATE_JACOBI
    int clamp_step;         // SUPPORT mode: step_i = min(step, 1 / (lambda + c_i))
    float eps;              // GD: Charbonnier loss on the target term when > 0 (else the square)
    int tc_vec;             // t and c rows may be read with 16-byte vectors (W % 4 == 0, aligned)
    // support mode: S -> chat = c * s_flat / S (written to zout)
    float s_flat;
    // device status word (bounded waits that give up write DTS_ERR_TIMEOUT here)
    int* status;
    // scratch of the chained vertical pass (col_chain_kernel): control words and chunk tuples
    unsigned* chain_ctl;
    float* chain_agg;
};

// One directional pass adjoint (see dts_backward.cu).
struct BwdArgs {
    const float* x;         // the pass input recomputed from the checkpoint (pitch `pitch`)
    const void* d;          // distances along the pass direction
    const float* gin;       // dL/d(pass output)
    const float* kout;      // the pass output (the next pass's input, or zbar for the last pass)
    float* gout;            // dL/d(pass input)
    float* dbar;            // += dL/d(distances)
    float* gz;              // dL/dz of the iterate (update variant: read then overwritten;
                            // final horizontal pass: += dL/d(pass input))
    int H, W;
    long long pitch;
    float k2;               // log2(a_i)
    float lna;              // ln(a_i)
    // data-term update adjoint (last vertical pass)
    const void* t;
    int t_dtype;
    const float* c;         // dense pitch W
    const float* zk;        // checkpoint z_k (pitch `pitch`)
    float* gt;              // += dL/dt (dense, may be null)
    float* gc;              // += dL/dc (dense, may be null)
    float lambda, step;
    int update;
    float eps;              // Charbonnier loss on the target term when > 0
    // chained vertical adjoint (columns taller than one cluster): control words, chunk tuples,
    // and the status word its bounded waits write
    unsigned* chain_ctl;
    float* chain_agg;
    int* status;
};

struct GuideGradArgs {
    const void* guide;
    long long ch_stride, row_stride;
    int C, H, W, gdtype, norm, dhalf;
    float k;                // sigma_s / sigma_r
    const void* dX;
    const void* dY;
    const float* dXb;
    const float* dYb;
    long long pitch;
    float* out;             // C x H x W dense
};

struct ColPlan {
    int items;   // rows per thread
    int warps;   // warps per CTA
    int cluster; // CTAs per cluster along the column, or one of the kernels below
};
constexpr int kColStrip = 0;   // one CTA per 8-column strip (col_strip_tma_kernel)
constexpr int kColChain = -1;  // chained CTAs (col_chain_kernel)
constexpr int kColTall = -2;   // persistent clusters fed by TMA (col_tall_kernel), ceil(H / rows) CTAs
constexpr int kColTallPair = -4;  // the same kernel, each column held by a pair of clusters (halves)
constexpr int kTallPairUnits = 64;  // most cluster pairs of one paired launch
constexpr int kColSplit = -5;  // vertical adjoint in two launches: chunk totals, then replay

struct RowPlan {
    int items;   // elements per thread
    int tpr;     // threads per row (multiple of 32)
    int rpb;     // rows per CTA
};

// PASS_TRANSPOSE: the transpose of a normalised pass (conjugate gradients on Eq. 2)
enum PassKind {
    PASS_PLAIN = 0,
    PASS_UPDATE = 1,
    PASS_SUPPORT = 2,
    PASS_SUPPORT_CONF = 3,
    PASS_UPDATE_ROW = 4,
    PASS_TRANSPOSE = 5
};

// Kernel ids reported by the per-launch timer (dts_profile / dts_kernel_name).
enum KernelId {
    KID_DISTANCES = 0,
    KID_COPY = 1,
    KID_ROW_PLAIN = 2,
    KID_ROW_SUPPORT = 3,
    KID_COL_PLAIN = 4,
    // 5: no longer used
    KID_COL_SUPPORT = 6,
    KID_ROW_BWD = 7,
    KID_ROW_BWD_FINAL = 8,
    KID_COL_BWD = 9,
    // 10: no longer used
    KID_GUIDE_GRAD = 11,
    KID_AXPY = 12,
    // 13: no longer used
    KID_ROW_UPDATE = 14,
    KID_UPDATE = 15,
    KID_UPDATE_ADJ = 16,
    KID_COL_STRIP = 17,
    KID_SQUARE = 18,
    KID_CONFIDENCE = 19,
    KID_BOX = 20,
    KID_TRANSPOSE = 21,
    KID_ROW_TRANSPOSE = 22,
    KID_COL_TRANSPOSE = 23,
    KID_CG_APPLY = 24,
    KID_CG_STEP = 25,
    KID_CG_DIRECTION = 26,
    KID_COL_STRIP_TRANSPOSE = 27,
    KID_RESIDENT = 28,
    KID_COL_CHAIN = 29,
    // 30: no longer used
    KID_COL_CHAIN_TRANSPOSE = 31,
    KID_COL_BWD_CHAIN = 32,
    KID_COL_TALL = 33,
    KID_COL_TALL_TRANSPOSE = 34,
    KID_BATCHED = 35,
    KID_ROW_STREAM = 36,
    KID_ROW_STREAM_UPDATE = 37,
    KID_COL_BWD_AGG = 38,
    KID_COL_BWD_APPLY = 39,
    KID_COL_BWD_CARRY = 40,
    KID_GUIDE_GRAD4 = 41,
};
// flags of a timing record
constexpr int kFlagDistHalf = 1;   // distance planes stored as FP16
constexpr int kFlagTarget16 = 2;   // target stored in 16 bits

// per-launch timer (dts_profile.cu): returns a handle for prof_end, or -1 when off (launches
// captured into a graph are not timed); prof_active: the timer is on
int prof_begin(int kernel, long long pixels, int flags, cudaStream_t s);
void prof_end(int handle, cudaStream_t s);
bool prof_active();

// device status word of the current device (dts_api.cu; set up by the entry points before
// their first launch)
int* status_word();
// flag value of the next chained vertical pass (never 0; dts_api.cu)
unsigned next_chain_epoch();
// SMs of the device, and resident CTAs per SM of a kernel at this block size (dts_api.cu)
int sm_count();
int blocks_per_sm(const void* kernel, int block, size_t smem);
// one-shot fault injection for tests (dts_debug_inject): true when `kind` is pending, which it
// then no longer is (dts_api.cu)
bool take_injected(int kind);
bool injection_pending();

// Bounded device-side waits: about a second at the boost clock, about a millisecond when a test
// has requested a fault injection.
constexpr long long kWaitTimeout = 2000000000LL;
constexpr long long kInjectedTimeout = 2000000LL;
inline long long default_timeout_cycles() { return kWaitTimeout; }

// Tallest column of a vertical pass, and the most chunks a chained vertical pass cuts one into
// (its CTAs of a strip must be resident together; the launch checks that twice as many fit).
constexpr int kMaxColRows = 16384;
constexpr int kChainMaxChunks = 256;
// scratch of the chained passes for an H x W plane (control words; chunk tuples of up to 9
// floats per column for both directions together, at the shortest chunk of 64 rows)
size_t chain_ctl_bytes(int W);
size_t chain_agg_bytes(int H, int W);

// launchers (dts_forward.cu); return cudaGetLastError() after the launch
cudaError_t launch_distances(const DistArgs& a, cudaStream_t s);
cudaError_t launch_copy_plane(const void* src, int src_dtype, long long src_pitch, float* dst, long long dst_pitch,
                              int H, int W, cudaStream_t s);
cudaError_t launch_row_pass(const PassArgs& a, int dist_half, int kind, const RowPlan& p, cudaStream_t s);
cudaError_t launch_col_pass(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s);
bool plan_rows(int W, RowPlan* p);
bool plan_rows_regular(int W, RowPlan* p);
// the streaming horizontal pass (dts_rows.cu): plans with an odd segment length (17 or 33)
bool row_stream_fits(int W, int items);
bool row_stream_addressable(const PassArgs& a, int dist_half, bool upd);
cudaError_t launch_row_stream(const PassArgs& a, int dist_half, int items, bool upd, cudaStream_t s);
cudaError_t prepare_row_stream_kernels();
bool row_update_fits(const RowPlan& p);
bool plan_rows_update(int W, const RowPlan& plain, RowPlan* p);
// autotuner tables (dts_forward.cu)
void set_tuned_row(int W, int items);
void set_tuned_col(int H, const ColPlan& p);
int col_candidates(int H, ColPlan* out, int max_out);
cudaError_t launch_update(const PassArgs& a, cudaStream_t s);
// box-kernel filter (dts_box.cu): lines up to kBoxMaxLine positions (FP64 sums in shared memory)
constexpr int kBoxMaxLine = 8192;
cudaError_t prepare_box_kernels();
cudaError_t launch_box_lines(const float* src, long long sp, float* dst, long long dstp, const float* d, long long dp,
                             int L, int lines, double r, cudaStream_t s);
cudaError_t launch_transpose(const float* src, long long sp, float* dst, long long dp, int H, int W, cudaStream_t s);
cudaError_t launch_square_plane(const float* src, float* dst, long long pitch, int H, int W, cudaStream_t s);
cudaError_t launch_confidence(const float* m1, const float* m2, long long pitch, int H, int W, float sigma_c,
                              float* c, cudaStream_t s);

// conjugate gradients on Eq. 2 (dts_cg.cu).  Pitched planes (row pitch `pitch`, a multiple of 4):
// z, r, p, q, u = A p, s = A^T (p - A p); c and t dense (row pitch W).  scal holds the FP64 dot
// products: slots 0 / 1 the residual norms r.r of consecutive iterations (slot_rr the current
// one), kCgSlotPq the product p.q.  partials (kCgMaxBlocks) and the ticket are the reduction's
// scratch; the ticket starts at 0 and every reduction leaves it at 0.
constexpr int kCgMaxBlocks = 2048;
constexpr int kCgSlotPq = 2;
struct CgArgs {
    int H, W;
    long long pitch;
    float* z;
    float* r;
    float* p;
    float* q;
    const float* u;
    const float* s;
    const float* c;
    const void* t;
    int t_dtype;
    bool dvec;          // c (and t) readable as aligned 16-byte vectors (W % 4 == 0)
    float lambda;
    double* scal;
    double* partials;
    unsigned* ticket;
    int slot_rr;
    float* zout;        // where the step writes z (z itself, or the caller's dense output)
    long long zout_pitch;
    bool zout_vec;      // zout rows 16-byte aligned with a pitch that is a multiple of 4
};
int cg_blocks(int H, long long pitch);
cudaError_t launch_cg_apply(const CgArgs& a, bool init, cudaStream_t s);
cudaError_t launch_cg_step(const CgArgs& a, cudaStream_t s);
cudaError_t launch_cg_direction(const CgArgs& a, cudaStream_t s);

// the batched solve as one persistent kernel over a queue of jobs (dts_batched.cu): up to
// kBatchMax images of at most kBatchMaxRows x kBatchMaxCols, recursive filter, GD or Jacobi,
// plain confidence, no checkpoints, iterations >= 1.  Control words: kBatchCtlHead words, then
// one finished-job counter per image and stage, batch_ctl_bytes in all (at the workspace start).
constexpr int kBatchMax = 96;
constexpr int kBatchCtlHead = 32;
constexpr int kBatchMaxRows = 4 * 16 * 17;  // a vertical job: 16 warps x 4 segments x 17 rows
constexpr int kBatchMaxCols = 16 * 512;     // a horizontal job: 512 threads x 16 positions
struct BatchPlanes {
    void* dX;
    void* dY;
    float* u;
    float* z;
    long long pitch;
};
struct BatchLaunch {
    int n;
    const dts_guide* guides;
    const void* const* targets;
    int tdtype;
    const float* const* confs;
    const dts_params* p;
    float* const* z_out;
    const BatchPlanes* planes;
    float k2[kMaxPasses];
    unsigned* ctl;
    int* status;
};
size_t batch_ctl_bytes(int n, const dts_params* p);
bool batch_persistent_fits(int H, int W);
cudaError_t launch_batched(const BatchLaunch& l, cudaStream_t s);

// the whole solve with the iterate resident in shared memory (dts_resident.cu): one cooperative
// CTA per tile of TH rows x 512 columns, ntx x nty tiles; scratch of ragg_floats + cagg_floats
// floats for the segment tuples and 4 unsigned words for the grid barrier
struct ResidentPlan {
    int ntx, nty, TH;
    size_t smem;
    long long ragg_floats, cagg_floats;
};
struct ResidentLaunch {
    ResidentPlan plan;
    float* zbuf;            // z_0 on entry (pitch `pitch`), then the iterates
    const float* dX;
    const float* dY;
    long long pitch;
    const void* t;
    int t_dtype;
    const float* c;
    float* zout;            // dense, pitch W
    int H, W, K, N;
    float k2[kMaxPasses];
    float lambda, step, eps;
    int update;
    float* ragg;
    float* cagg;
    unsigned* bar;
    int* status;
};
bool plan_resident(int H, int W, const dts_params* p, ResidentPlan* rp);
cudaError_t prepare_resident_kernel();
cudaError_t launch_resident(const ResidentLaunch& l, cudaStream_t s);

// Vertical plans: the strip kernel (cluster 0), the cluster kernel (cluster > 0 CTAs) or the
// chained kernel (cluster -1).  plan_cols: any pass; plan_cols_multi: the kinds the strip kernel
// does not run; plan_cols_cluster: the cluster kernel (solves that run side by side).
bool plan_cols(int H, ColPlan* p);
bool plan_cols_multi(int H, ColPlan* p);
bool plan_cols_cluster(int H, ColPlan* p);
bool chain_plan(int H, ColPlan* p);
// rows per strip of the tiled distance plane the strip kernel reads (0: columns too tall for it)
long long strip_tile_rows(int H);
cudaError_t prepare_kernels();

// backward launchers (dts_backward.cu)
bool plan_rows_bwd(int W, RowPlan* p);
bool plan_cols_bwd(int H, ColPlan* p);
bool set_tuned_bwd_col(int H, const ColPlan& p);
cudaError_t launch_row_bwd(const BwdArgs& a, int dist_half, bool final_pass, const RowPlan& p, cudaStream_t s);
cudaError_t launch_col_bwd(const BwdArgs& a, int dist_half, const ColPlan& p, cudaStream_t s);
cudaError_t launch_guide_grad(const GuideGradArgs& a, cudaStream_t s);
cudaError_t launch_update_adjoint(const BwdArgs& a, cudaStream_t s);
cudaError_t launch_axpy_plane(const float* src, long long sp, float* dst, long long dp, int H, int W, int accumulate,
                              cudaStream_t s);
cudaError_t prepare_backward_kernels();

}  // namespace dts
