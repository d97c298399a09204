// C ABI of libdts (declared in include/dts.h): argument checks, workspace layout,
// the per-pass sigma schedule and the launch sequence of each entry point.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "dts_internal.cuh"

namespace dts {

// Device-side status word (one per device that loads the library).
__device__ int g_status = 0;

namespace {

constexpr int kMaxDevices = 64;
std::atomic<int*> g_status_ptr[kMaxDevices] = {};
int g_inject = 0;  // pending fault injection (dts_debug_inject), one-shot
std::mutex g_prep_mutex;
bool g_prepared[kMaxDevices] = {};

// Once per device, with that device current: kernel attributes, and the device address of the
// status word (the bounded waits of the kernels write DTS_ERR_TIMEOUT there).  Every entry point
// calls this before its first launch, so a launch never gets a null status word.
int ensure_prepared() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DTS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_prep_mutex);
    if (!g_prepared[dev]) {
        if (prepare_kernels() != cudaSuccess || prepare_backward_kernels() != cudaSuccess ||
            prepare_box_kernels() != cudaSuccess || prepare_resident_kernel() != cudaSuccess ||
            prepare_row_stream_kernels() != cudaSuccess)
            return DTS_ERR_CUDA;
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess || p == nullptr) return DTS_ERR_CUDA;
        g_status_ptr[dev].store(static_cast<int*>(p));
        g_prepared[dev] = true;
    }
    return DTS_OK;
}

}  // namespace

// SMs of the current device (cached per process: one kind of GPU).
int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// resident CTAs per SM of a kernel (cached per kernel, block size and dynamic shared memory)
int blocks_per_sm(const void* kernel, int block, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t>, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(kernel, block, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess) n = 0;
    cache[key] = n;
    return n;
}

// Flag value of the next chained vertical pass: distinct for every launch of the process (a
// 32-bit counter that skips 0, the value a solve's cleared flags hold).
unsigned next_chain_epoch() {
    static std::atomic<unsigned> counter{0};
    unsigned e = counter.fetch_add(1u) + 1u;
    while (e == 0u) e = counter.fetch_add(1u) + 1u;
    return e;
}

// The status word of the current device, as looked up by ensure_prepared (null before).
int* status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    return g_status_ptr[dev].load();
}

bool injection_pending() {
    std::lock_guard<std::mutex> lock(g_prep_mutex);
    return g_inject != 0;
}

bool take_injected(int kind) {
    std::lock_guard<std::mutex> lock(g_prep_mutex);
    if (g_inject != kind) return false;
    g_inject = 0;
    return true;
}

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool valid_dtype(int d) { return d == DTS_F32 || d == DTS_BF16 || d == DTS_F16; }

int check_guide(const dts_guide* g) {
    if (!g || !g->data) return DTS_ERR_INVALID_ARG;
    if (g->C < 1 || g->H < 1 || g->W < 1 || !valid_dtype(g->dtype)) return DTS_ERR_INVALID_ARG;
    const long long rs = g->row_stride ? g->row_stride : g->W;
    const long long cs = g->ch_stride ? g->ch_stride : (long long)g->H * rs;
    if (rs < g->W || (g->C > 1 && cs < (long long)g->H * rs) || cs < 0) return DTS_ERR_INVALID_ARG;
    return DTS_OK;
}

int check_params(const dts_params* p) {
    if (!p) return DTS_ERR_INVALID_ARG;
    if (!(p->lambda >= 0.f) || !isfinite(p->lambda)) return DTS_ERR_INVALID_ARG;
    if (!(p->sigma_s > 0.f) || !isfinite(p->sigma_s)) return DTS_ERR_INVALID_ARG;
    if (!(p->sigma_r > 0.f) || !isfinite(p->sigma_r)) return DTS_ERR_INVALID_ARG;
    if (!(p->step > 0.f) || !isfinite(p->step)) return DTS_ERR_INVALID_ARG;
    if (p->iterations < 0 || p->passes < 1 || p->passes > kMaxPasses) return DTS_ERR_INVALID_ARG;
    if (p->norm != DTS_NORM_L1 && p->norm != DTS_NORM_L2) return DTS_ERR_INVALID_ARG;
    if (p->update != DTS_UPDATE_GD && p->update != DTS_UPDATE_JACOBI && p->update != DTS_UPDATE_CG)
        return DTS_ERR_INVALID_ARG;
    if (p->conf_mode != DTS_CONF_PLAIN && p->conf_mode != DTS_CONF_SUPPORT) return DTS_ERR_INVALID_ARG;
    if (p->dist_dtype != DTS_F32 && p->dist_dtype != DTS_F16) return DTS_ERR_INVALID_ARG;
    if (p->save_checkpoints < 0 || p->save_checkpoints > 2) return DTS_ERR_INVALID_ARG;
    if (p->filter_kernel != DTS_KERNEL_RF && p->filter_kernel != DTS_KERNEL_BOX) return DTS_ERR_INVALID_ARG;
    if (!(p->charbonnier_eps >= 0.f) || !isfinite(p->charbonnier_eps)) return DTS_ERR_INVALID_ARG;
    return DTS_OK;
}

// what conjugate gradients and the box-kernel filter support (DTS_ERR_UNSUPPORTED otherwise)
int check_box(const dts_guide* g, const dts_params* p) {
    if (p->charbonnier_eps > 0.f && p->update == DTS_UPDATE_CG) return DTS_ERR_UNSUPPORTED;
    if (p->update == DTS_UPDATE_CG &&
        (p->filter_kernel != DTS_KERNEL_RF || p->conf_mode != DTS_CONF_PLAIN || p->save_checkpoints))
        return DTS_ERR_UNSUPPORTED;
    if (p->filter_kernel != DTS_KERNEL_BOX) return DTS_OK;
    if (p->dist_dtype != DTS_F32 || p->conf_mode != DTS_CONF_PLAIN || p->save_checkpoints) return DTS_ERR_UNSUPPORTED;
    if (g->H > kBoxMaxLine || g->W > kBoxMaxLine) return DTS_ERR_UNSUPPORTED;
    return DTS_OK;
}

// bytes before the partial sums in the conjugate-gradient block: 8 FP64 scalars, the ticket
constexpr size_t kCgScalarBytes = 128;

// Workspace layout (byte offsets from the workspace base).
struct Layout {
    long long pitch;
    size_t plane_f32;   // bytes of one FP32 plane
    size_t plane_d;     // bytes of one distance plane
    size_t dX, dY, u, chat, z;  // offsets
    size_t dYs;         // dY tiled by 8-column strips (ys_rows rows per strip; 0: none)
    long long ys_rows;
    size_t chain_ctl, chain_agg;  // chained vertical passes: control words, chunk tuples
    int z_planes;       // 1 (in place) or K checkpoints
    size_t passes;      // save_checkpoints = 2: K x 2N planes, (k, 0) = zbar_k, (k, q) = input of pass q
    size_t dYt, ut;     // box kernel: transposed dY and working plane (W rows, pitch tpitch)
    size_t cg;          // conjugate gradients: planes r, p, q, then FP64 scalars, ticket, partials
    bool resident;      // the solve runs as one resident kernel (plan res), scratch at ragg, cagg, rbar
    ResidentPlan res;
    size_t ragg, cagg, rbar;
    long long tpitch;
    size_t fwd_end;     // bytes used by the forward
    // backward scratch
    size_t xin;         // 2N pass-input planes
    size_t g0, g1;      // adjoint ping-pong planes
    size_t gz;          // adjoint of the iterate
    size_t dXb, dYb;    // distance gradients
    size_t total;
};

Layout make_layout(int H, int W, const dts_params* p, int with_backward) {
    Layout L = {};
    L.pitch = pitch_for(W);
    L.plane_f32 = align_up((size_t)H * (size_t)L.pitch * 4, kPlaneAlign);
    L.plane_d = align_up((size_t)H * (size_t)L.pitch * (p->dist_dtype == DTS_F16 ? 2 : 4), kPlaneAlign);
    size_t off = 0;
    L.dX = off; off += L.plane_d;
    L.dY = off; off += L.plane_d;
    L.u = off; off += L.plane_f32;
    // dY tiled by 8-column strips for the strip kernel (columns up to its height limit)
    L.ys_rows = p->filter_kernel == DTS_KERNEL_RF ? strip_tile_rows(H) : 0;
    L.dYs = off;
    if (L.ys_rows)
        off += align_up((size_t)((W + 7) / 8) * (size_t)L.ys_rows * 8 * (p->dist_dtype == DTS_F16 ? 2 : 4), kPlaneAlign);
    L.chat = off;
    if (p->conf_mode == DTS_CONF_SUPPORT) off += L.plane_f32;
    L.chain_ctl = off;
    off += align_up(chain_ctl_bytes(W), kPlaneAlign);
    L.chain_agg = off;
    off += align_up(chain_agg_bytes(H, W), kPlaneAlign);
    L.z = off;
    const bool keep = p->save_checkpoints || with_backward;
    L.z_planes = keep ? (p->iterations > 0 ? p->iterations : 1) : 1;
    off += (size_t)L.z_planes * L.plane_f32;
    if (p->filter_kernel == DTS_KERNEL_BOX) {  // transposed dY and working plane (W rows of pitch_for(H))
        L.tpitch = pitch_for(H);
        const size_t tplane = align_up((size_t)W * (size_t)L.tpitch * 4, kPlaneAlign);
        L.dYt = off;
        off += tplane;
        L.ut = off;
        off += tplane;
    }
    L.cg = off;
    if (p->update == DTS_UPDATE_CG) off += 3 * L.plane_f32 + align_up(kCgScalarBytes + kCgMaxBlocks * sizeof(double), kPlaneAlign);
    L.resident = plan_resident(H, W, p, &L.res);
    if (L.resident) {
        L.ragg = off;
        off += align_up((size_t)L.res.ragg_floats * sizeof(float), kPlaneAlign);
        L.cagg = off;
        off += align_up((size_t)L.res.cagg_floats * sizeof(float), kPlaneAlign);
        L.rbar = off;
        off += kPlaneAlign;
    }
    L.passes = off;
    if (p->save_checkpoints == 2) off += (size_t)(p->iterations > 0 ? p->iterations : 1) * 2 * p->passes * L.plane_f32;
    L.fwd_end = off;
    if (with_backward) {
        // recompute scratch for the pass inputs (not needed when the forward kept them all)
        L.xin = off; off += (p->save_checkpoints == 2 ? 0 : (size_t)(2 * p->passes)) * L.plane_f32;
        L.g0 = off; off += L.plane_f32;
        L.g1 = off; off += L.plane_f32;
        L.gz = off; off += L.plane_f32;
        L.dXb = off; off += L.plane_f32;
        L.dYb = off; off += L.plane_f32;
    }
    L.total = off;
    return L;
}

// Per-pass feedback of the recursive filter: sigma_i = sigma_s sqrt(3) 2^(N-i) / sqrt(4^N - 1),
// a_i = exp(-sqrt(2) / sigma_i); the kernels take log2(a_i) so that w = exp2(log2(a_i) * d).
void pass_log2a(double sigma_s, int N, float* k2) {
    for (int i = 1; i <= N; ++i) {
        const double sig = sigma_s * sqrt(3.0) * ldexp(1.0, N - i) / sqrt(ldexp(1.0, 2 * N) - 1.0);
        k2[i - 1] = (float)(-sqrt(2.0) / (sig * log(2.0)));
    }
}

// Per-pass sigma_i of the same schedule (for the box kernel's radius r_i = sigma_i sqrt(3)).
void pass_sigma(double sigma_s, int N, double* sig) {
    for (int i = 1; i <= N; ++i)
        sig[i - 1] = sigma_s * sqrt(3.0) * ldexp(1.0, N - i) / sqrt(ldexp(1.0, 2 * N) - 1.0);
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DTS_OK;
    if (getenv("DTS_LOG")) fprintf(stderr, "libdts: CUDA error %s\n", cudaGetErrorString(e));
    return DTS_ERR_CUDA;
}

struct Plans {
    RowPlan rows;
    ColPlan cols;
};

int make_plans(int H, int W, Plans* pl) {
    if (!plan_rows(W, &pl->rows)) return DTS_ERR_UNSUPPORTED;
    if (!plan_cols(H, &pl->cols)) return DTS_ERR_UNSUPPORTED;
    return DTS_OK;
}

char* ws_at(void* ws, size_t off) { return static_cast<char*>(ws) + off; }

// distances into the workspace, plus an optional fused copy of `src` into plane `dst`
int run_distances(const dts_guide* g, const dts_params* p, const Layout& L, void* ws, const void* src, int src_dtype,
                  float* dst, cudaStream_t s) {
    DistArgs a = {};
    a.guide = g->data;
    a.row_stride = g->row_stride ? g->row_stride : g->W;
    a.ch_stride = g->ch_stride ? g->ch_stride : (long long)g->H * a.row_stride;
    a.C = g->C;
    a.H = g->H;
    a.W = g->W;
    a.gdtype = g->dtype;
    a.norm = p->norm;
    a.dhalf = p->dist_dtype == DTS_F16;
    a.k = p->sigma_s / p->sigma_r;
    a.dX = ws_at(ws, L.dX);
    a.dY = ws_at(ws, L.dY);
    a.pitch = L.pitch;
    a.src = src;
    a.src_dtype = src_dtype;
    a.dst = dst;
    a.ys_rows = L.ys_rows;
    a.dYs = L.ys_rows ? ws_at(ws, L.dYs) : nullptr;
    return cuda_status(launch_distances(a, s));
}

// workspace base of the pass arguments (set by the entry points before building passes)
thread_local void* t_ws = nullptr;

PassArgs base_pass(const dts_guide* g, const Layout& L) {
    PassArgs a = {};
    a.H = g->H;
    a.W = g->W;
    a.pitch = L.pitch;
    a.dst_pitch = L.pitch;
    a.status = status_word();
    if (t_ws && L.ys_rows) {  // read by the strip kernel in vertical passes (whose d is dY)
        a.d_tiled = static_cast<char*>(t_ws) + L.dYs;
        a.d_tiled_rows = L.ys_rows;
    }
    if (t_ws) {
        a.chain_ctl = reinterpret_cast<unsigned*>(static_cast<char*>(t_ws) + L.chain_ctl);
        a.chain_agg = reinterpret_cast<float*>(static_cast<char*>(t_ws) + L.chain_agg);
    }
    return a;
}

// Binds the workspace for base_pass and zeroes the chained passes' control words (every chained
// launch leaves them at zero again, so one clear per call suffices; it also clears an abort
// left by a wait that ran out in an earlier call).
int bind_workspace(void* ws, const Layout& L, int W, cudaStream_t s) {
    t_ws = ws;
    if (cudaMemsetAsync(static_cast<char*>(ws) + L.chain_ctl, 0, chain_ctl_bytes(W), s) != cudaSuccess)
        return DTS_ERR_CUDA;
    return DTS_OK;
}

// effective confidence for DTS_CONF_SUPPORT: chat = c * S_flat / S (written to L.chat)
int run_support(const dts_guide* g, const dts_params* p, const Layout& L, void* ws, const float* conf,
                const Plans& pl, cudaStream_t s) {
    const int dh = p->dist_dtype == DTS_F16;
    const double a = exp(-sqrt(2.0) / (double)p->sigma_s);
    float* u = reinterpret_cast<float*>(ws_at(ws, L.u));
    PassArgs r = base_pass(g, L);
    r.src = u;
    r.dst = u;
    r.d = ws_at(ws, L.dX);
    r.k2 = (float)log2(a);
    int st = cuda_status(launch_row_pass(r, dh, PASS_SUPPORT, pl.rows, s));
    if (st) return st;
    PassArgs c = base_pass(g, L);
    c.src = u;
    c.dst = u;
    c.d = ws_at(ws, L.dY);
    c.k2 = (float)log2(a);
    c.c = conf;
    c.zout = reinterpret_cast<float*>(ws_at(ws, L.chat));
    c.zout_pitch = L.pitch;
    c.s_flat = (float)(((1.0 + a) / (1.0 - a)) * ((1.0 + a) / (1.0 - a)));
    return cuda_status(launch_col_pass(c, dh, PASS_SUPPORT_CONF, pl.cols, s));
}

// The box-kernel filter of src (pitch L.pitch) into dst (pitch dst_pitch; may be src): per pass a
// box average along the rows, then along the columns as rows of the transposed plane.  Needs the
// distances, and dY transposed into L.dYt (prepare_box_distances).
int run_box_filter(const dts_guide* g, const dts_params* p, const Layout& L, void* ws, const float* src, float* dst,
                   long long dst_pitch, cudaStream_t s) {
    const int H = g->H, W = g->W;
    const long long P = L.pitch, TP = L.tpitch;
    float* u = reinterpret_cast<float*>(ws_at(ws, L.u));
    float* ut = reinterpret_cast<float*>(ws_at(ws, L.ut));
    const float* dX = reinterpret_cast<const float*>(ws_at(ws, L.dX));
    const float* dYt = reinterpret_cast<const float*>(ws_at(ws, L.dYt));
    double sig[kMaxPasses];
    pass_sigma(p->sigma_s, p->passes, sig);
    int st;
    for (int i = 0; i < p->passes; ++i) {
        const double r = sig[i] * sqrt(3.0);
        if ((st = cuda_status(launch_box_lines(i == 0 ? src : u, P, u, P, dX, P, W, H, r, s)))) return st;
        if ((st = cuda_status(launch_transpose(u, P, ut, TP, H, W, s)))) return st;
        if ((st = cuda_status(launch_box_lines(ut, TP, ut, TP, dYt, TP, H, W, r, s)))) return st;
        const bool last = i + 1 == p->passes;
        if ((st = cuda_status(launch_transpose(ut, TP, last ? dst : u, last ? dst_pitch : P, W, H, s)))) return st;
    }
    return DTS_OK;
}

int prepare_box_distances(const dts_guide* g, const Layout& L, void* ws, cudaStream_t s) {
    return cuda_status(launch_transpose(reinterpret_cast<const float*>(ws_at(ws, L.dY)), L.pitch,
                                        reinterpret_cast<float*>(ws_at(ws, L.dYt)), L.tpitch, g->H, g->W, s));
}

// The solve with the box kernel: z_0 = z_init or t; per iteration zbar = box filter of z_k, then
// the update of Eq. 3 / Eq. 4 in place (elementwise kernel).
int solve_box(const dts_guide* g, const void* target, int tdt, const float* conf, const float* z_init,
              const dts_params* p, float* z_out, void* ws, const Layout& L, cudaStream_t s) {
    const int K = p->iterations, H = g->H, W = g->W;
    if (K == 0) {
        if (z_init) return cuda_status(launch_copy_plane(z_init, DTS_F32, W, z_out, W, H, W, s));
        return cuda_status(launch_copy_plane(target, tdt, W, z_out, W, H, W, s));
    }
    int st;
    if ((st = bind_workspace(ws, L, g->W, s))) return st;
    float* z = reinterpret_cast<float*>(ws_at(ws, L.z));
    if (z_init) st = run_distances(g, p, L, ws, z_init, DTS_F32, z, s);
    else st = run_distances(g, p, L, ws, target, tdt, z, s);
    if (st || (st = prepare_box_distances(g, L, ws, s))) return st;
    float* zbar = reinterpret_cast<float*>(ws_at(ws, L.u));
    for (int k = 0; k < K; ++k) {
        if ((st = run_box_filter(g, p, L, ws, z, zbar, L.pitch, s))) return st;
        PassArgs a = base_pass(g, L);
        a.src = zbar;
        a.zk = z;
        a.t = target;
        a.t_dtype = tdt;
        a.c = conf;
        a.lambda = p->lambda;
        a.step = p->step;
        a.update = p->update;
        a.eps = p->charbonnier_eps;
        if (k + 1 == K) {
            a.zout = z_out;
            a.zout_pitch = W;
        } else {
            a.zout = z;
            a.zout_pitch = L.pitch;
        }
        if ((st = cuda_status(launch_update(a, s)))) return st;
    }
    return DTS_OK;
}

}  // namespace
}  // namespace dts

namespace dts {
namespace {
// Conjugate gradients on the objective of Eq. 2 (the method the paper names for faster
// convergence, §5): M z = b with M = lambda (I - A)^T (I - A) + 2 C and b = 2 C t, from z_0 =
// z_init or t, K iterations (K >= 1).  A product M x is the 2N passes of A on x into u, then the
// 2N transposed passes in reverse order (column before row) on x - u into q, the first of which
// forms x - u as it loads, then cg_apply_kernel.
int solve_cg(const dts_guide* g, const void* target, int tdt, const float* conf, const float* z_init,
             const dts_params* p, float* z_out, void* ws, const Layout& L, const Plans& pl, cudaStream_t s) {
    const int K = p->iterations, N = p->passes, W = g->W;
    ColPlan multi_shape;  // the transposed vertical pass needs the strip, chain or cluster kernel
    if (!plan_cols_multi(g->H, &multi_shape)) return DTS_ERR_UNSUPPORTED;
    int st;
    if ((st = bind_workspace(ws, L, g->W, s))) return st;
    float* z = reinterpret_cast<float*>(ws_at(ws, L.z));
    if (z_init) st = run_distances(g, p, L, ws, z_init, DTS_F32, z, s);
    else st = run_distances(g, p, L, ws, target, tdt, z, s);
    if (st) return st;
    float* u = reinterpret_cast<float*>(ws_at(ws, L.u));
    float* r = reinterpret_cast<float*>(ws_at(ws, L.cg));
    float* pd = reinterpret_cast<float*>(ws_at(ws, L.cg + L.plane_f32));
    float* q = reinterpret_cast<float*>(ws_at(ws, L.cg + 2 * L.plane_f32));
    char* sc = ws_at(ws, L.cg + 3 * L.plane_f32);
    if (cudaMemsetAsync(sc, 0, kCgScalarBytes, s) != cudaSuccess) return DTS_ERR_CUDA;
    float k2[kMaxPasses];
    pass_log2a(p->sigma_s, N, k2);
    const int dh = p->dist_dtype == DTS_F16;
    auto filter_pair = [&](const float* x) -> int {  // u = A x, q = A^T (x - A x)
        int e;
        for (int i = 0; i < N; ++i) {
            PassArgs a = base_pass(g, L);
            a.src = i == 0 ? x : u;
            a.dst = u;
            a.d = ws_at(ws, L.dX);
            a.k2 = k2[i];
            if ((e = cuda_status(launch_row_pass(a, dh, PASS_PLAIN, pl.rows, s)))) return e;
            PassArgs c = base_pass(g, L);
            c.src = u;
            c.dst = u;
            c.d = ws_at(ws, L.dY);
            c.k2 = k2[i];
            if ((e = cuda_status(launch_col_pass(c, dh, PASS_PLAIN, pl.cols, s)))) return e;
        }
        for (int i = N - 1; i >= 0; --i) {
            PassArgs c = base_pass(g, L);
            c.src = i == N - 1 ? u : q;
            c.zk = i == N - 1 ? x : nullptr;
            c.dst = q;
            c.d = ws_at(ws, L.dY);
            c.k2 = k2[i];
            if ((e = cuda_status(launch_col_pass(c, dh, PASS_TRANSPOSE, pl.cols, s)))) return e;
            PassArgs a = base_pass(g, L);
            a.src = q;
            a.dst = q;
            a.d = ws_at(ws, L.dX);
            a.k2 = k2[i];
            if ((e = cuda_status(launch_row_pass(a, dh, PASS_TRANSPOSE, pl.rows, s)))) return e;
        }
        return DTS_OK;
    };
    CgArgs a = {};
    a.H = g->H;
    a.W = W;
    a.pitch = L.pitch;
    a.z = z;
    a.r = r;
    a.p = pd;
    a.q = q;
    a.u = u;
    a.s = q;
    a.c = conf;
    a.t = target;
    a.t_dtype = tdt;
    a.dvec = W % 4 == 0 && (uintptr_t)conf % 16 == 0;
    a.lambda = p->lambda;
    a.scal = reinterpret_cast<double*>(sc);
    a.ticket = reinterpret_cast<unsigned*>(sc + 64);
    a.partials = reinterpret_cast<double*>(sc + kCgScalarBytes);
    a.zout = z;
    a.zout_pitch = L.pitch;
    a.zout_vec = true;
    // r_0 = b - M z_0, p_0 = r_0
    if ((st = filter_pair(z))) return st;
    a.slot_rr = 0;
    if ((st = cuda_status(launch_cg_apply(a, true, s)))) return st;
    for (int k = 0; k < K; ++k) {
        if ((st = filter_pair(pd))) return st;
        a.slot_rr = k & 1;
        if ((st = cuda_status(launch_cg_apply(a, false, s)))) return st;
        if (k == K - 1) {
            a.zout = z_out;
            a.zout_pitch = W;
            a.zout_vec = W % 4 == 0 && (uintptr_t)z_out % 16 == 0;
        }
        if ((st = cuda_status(launch_cg_step(a, s)))) return st;
        if (k + 1 < K && (st = cuda_status(launch_cg_direction(a, s)))) return st;
    }
    return DTS_OK;
}

// The solve as one resident kernel: distances and z_0, then every iteration in one cooperative
// launch (dts_resident.cu).
int solve_resident(const dts_guide* g, const void* target, int tdt, const float* conf, const float* z_init,
                   const dts_params* p, float* z_out, void* ws, const Layout& L, cudaStream_t s) {
    float* z = reinterpret_cast<float*>(ws_at(ws, L.z));
    int st = z_init ? run_distances(g, p, L, ws, z_init, DTS_F32, z, s) : run_distances(g, p, L, ws, target, tdt, z, s);
    if (st) return st;
    ResidentLaunch r = {};
    r.plan = L.res;
    r.zbuf = z;
    r.dX = reinterpret_cast<const float*>(ws_at(ws, L.dX));
    r.dY = reinterpret_cast<const float*>(ws_at(ws, L.dY));
    r.pitch = L.pitch;
    r.t = target;
    r.t_dtype = tdt;
    r.c = conf;
    r.zout = z_out;
    r.H = g->H;
    r.W = g->W;
    r.K = p->iterations;
    r.N = p->passes;
    pass_log2a(p->sigma_s, p->passes, r.k2);
    r.lambda = p->lambda;
    r.step = p->step;
    r.eps = p->charbonnier_eps;
    r.update = p->update;
    r.ragg = reinterpret_cast<float*>(ws_at(ws, L.ragg));
    r.cagg = reinterpret_cast<float*>(ws_at(ws, L.cagg));
    r.bar = reinterpret_cast<unsigned*>(ws_at(ws, L.rbar));
    r.status = status_word();
    return cuda_status(launch_resident(r, s));
}

int solve_forward(const dts_guide* g, const void* target, int tdt, const float* conf, const float* z_init,
                       const dts_params* p, float* z_out, void* ws, const Layout& L, const Plans& pl,
                       cudaStream_t s, bool allow_resident = false) {
    int st;
    const int K = p->iterations;
    const int W = g->W;
    if (K == 0) {
        if (z_init) return cuda_status(launch_copy_plane(z_init, DTS_F32, W, z_out, W, g->H, W, s));
        return cuda_status(launch_copy_plane(target, tdt, W, z_out, W, g->H, W, s));
    }
    if (p->update == DTS_UPDATE_CG) return solve_cg(g, target, tdt, conf, z_init, p, z_out, ws, L, pl, s);
    if ((st = bind_workspace(ws, L, g->W, s))) return st;
    if (allow_resident && L.resident) return solve_resident(g, target, tdt, conf, z_init, p, z_out, ws, L, s);
    const bool keep = L.z_planes > 1 || p->save_checkpoints;
    auto zslot = [&](int k) -> float* {
        return reinterpret_cast<float*>(ws_at(ws, L.z + (keep ? (size_t)k * L.plane_f32 : 0)));
    };
    // distances, and z_0 = z_init (or the target) into the first iterate plane
    if (z_init) st = run_distances(g, p, L, ws, z_init, DTS_F32, zslot(0), s);
    else st = run_distances(g, p, L, ws, target, tdt, zslot(0), s);
    if (st) return st;
    const bool support = p->conf_mode == DTS_CONF_SUPPORT;
    if (support && (st = run_support(g, p, L, ws, conf, pl, s))) return st;
    float k2[kMaxPasses];
    pass_log2a(p->sigma_s, p->passes, k2);
    const int dh = p->dist_dtype == DTS_F16;
    float* u = reinterpret_cast<float*>(ws_at(ws, L.u));
    const float* cplane = support ? reinterpret_cast<const float*>(ws_at(ws, L.chat)) : conf;
    // save_checkpoints = 2: every pass reads and writes its own plane of iteration k (the
    // backward then reads the pass inputs instead of recomputing them); else all passes run in
    // place on u
    const bool keep_passes = p->save_checkpoints == 2;
    const int NP = 2 * p->passes;
    auto pslot = [&](int k, int q) -> float* {
        return keep_passes ? reinterpret_cast<float*>(ws_at(ws, L.passes + ((size_t)k * NP + q) * L.plane_f32)) : u;
    };
    auto set_update = [&](PassArgs& a, const float* zk) {
        a.zk = zk;
        a.t = target;
        a.t_dtype = tdt;
        a.c = cplane;
        a.c_pitched = support;
        a.clamp_step = support;
        a.lambda = p->lambda;
        a.step = p->step;
        a.update = p->update;
        a.eps = p->charbonnier_eps;
        const int tsz = tdt == DTS_F32 ? 4 : 2;
        a.tc_vec = (W % 4 == 0) && ((uintptr_t)target % (4 * tsz) == 0) && ((uintptr_t)conf % 16 == 0);
    };
    // The data-term update of iteration k is applied by the first horizontal pass of iteration
    // k + 1 (reading z_k, zbar, t and c as vectors along rows and writing z_{k+1}); after the
    // last iteration a standalone kernel applies it.  Every row the horizontal passes take fits.
    RowPlan urows;
    if (!plan_rows_update(W, pl.rows, &urows)) return DTS_ERR_UNSUPPORTED;
    for (int k = 0; k < K; ++k) {
        float* zin = zslot(k);
        for (int i = 0; i < p->passes; ++i) {
            PassArgs r = base_pass(g, L);
            r.src = i == 0 ? zin : pslot(k, 2 * i);
            r.dst = pslot(k, 2 * i + 1);
            r.d = ws_at(ws, L.dX);
            r.k2 = k2[i];
            int rkind = PASS_PLAIN;
            if (i == 0 && k > 0) {
                rkind = PASS_UPDATE_ROW;
                r.src = pslot(k - 1, 0);  // zbar of iteration k - 1
                set_update(r, zslot(k - 1));
                r.zout = zin;  // z_k
                r.zout_pitch = L.pitch;
            }
            if ((st = cuda_status(launch_row_pass(r, dh, rkind, rkind == PASS_UPDATE_ROW ? urows : pl.rows, s)))) return st;
            PassArgs c = base_pass(g, L);
            c.src = pslot(k, 2 * i + 1);
            c.dst = pslot(k, (2 * i + 2) % NP);
            c.d = ws_at(ws, L.dY);
            c.k2 = k2[i];
            if ((st = cuda_status(launch_col_pass(c, dh, PASS_PLAIN, pl.cols, s)))) return st;
        }
    }
    {
        PassArgs a = base_pass(g, L);
        a.src = pslot(K - 1, 0);
        set_update(a, zslot(K - 1));
        a.zout = z_out;
        a.zout_pitch = W;
        if ((st = cuda_status(launch_update(a, s)))) return st;
    }
    return DTS_OK;
}

}  // namespace
}  // namespace dts

using namespace dts;

extern "C" const char* dts_status_string(int s) {
    switch (s) {
        case DTS_OK: return "DTS_OK";
        case DTS_ERR_INVALID_ARG: return "DTS_ERR_INVALID_ARG";
        case DTS_ERR_UNSUPPORTED: return "DTS_ERR_UNSUPPORTED";
        case DTS_ERR_WORKSPACE: return "DTS_ERR_WORKSPACE";
        case DTS_ERR_CUDA: return "DTS_ERR_CUDA";
        case DTS_ERR_TIMEOUT: return "DTS_ERR_TIMEOUT";
        case DTS_ERR_NONFINITE: return "DTS_ERR_NONFINITE";
        default: return "DTS_ERR_UNKNOWN";
    }
}

extern "C" const char* dts_version(void) { return "dts-gb300 0.1 (sm_103a)"; }

extern "C" size_t dts_workspace_size(const dts_guide* guide, const dts_params* params, int with_backward) {
    if (check_guide(guide) || check_params(params)) return 0;
    return make_layout(guide->H, guide->W, params, with_backward).total;
}

extern "C" int dts_domain_transform(const dts_guide* guide, const dts_params* params, void* dX, void* dY,
                                    dts_stream stream) {
    int st = check_guide(guide);
    if (!st) st = check_params(params);
    if (st) return st;
    if (!dX || !dY) return DTS_ERR_INVALID_ARG;
    DistArgs a = {};
    a.guide = guide->data;
    a.row_stride = guide->row_stride ? guide->row_stride : guide->W;
    a.ch_stride = guide->ch_stride ? guide->ch_stride : (long long)guide->H * a.row_stride;
    a.C = guide->C;
    a.H = guide->H;
    a.W = guide->W;
    a.gdtype = guide->dtype;
    a.norm = params->norm;
    a.dhalf = params->dist_dtype == DTS_F16;
    a.k = params->sigma_s / params->sigma_r;
    a.dX = dX;
    a.dY = dY;
    a.pitch = guide->W;
    return cuda_status(launch_distances(a, (cudaStream_t)stream));
}

extern "C" int dts_filter(const dts_guide* guide, const dts_params* params, const float* src, float* dst, void* ws,
                          size_t ws_bytes, dts_stream stream) {
    int st = check_guide(guide);
    if (!st) st = check_params(params);
    if (st) return st;
    if (!src || !dst) return DTS_ERR_INVALID_ARG;
    Plans pl;
    if ((st = make_plans(guide->H, guide->W, &pl))) return st;
    dts_params p = *params;
    p.conf_mode = DTS_CONF_PLAIN;
    p.save_checkpoints = 0;
    if ((st = check_box(guide, &p))) return st;
    const Layout L = make_layout(guide->H, guide->W, &p, 0);
    if (!ws || ((uintptr_t)ws % kPlaneAlign) != 0 || ws_bytes < L.fwd_end) return DTS_ERR_WORKSPACE;
    if ((st = ensure_prepared())) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = bind_workspace(ws, L, guide->W, s))) return st;
    float* u = reinterpret_cast<float*>(ws_at(ws, L.u));
    if ((st = run_distances(guide, &p, L, ws, src, DTS_F32, u, s))) return st;
    if (p.filter_kernel == DTS_KERNEL_BOX) {
        if ((st = prepare_box_distances(guide, L, ws, s))) return st;
        return run_box_filter(guide, &p, L, ws, u, dst, guide->W, s);
    }
    float k2[kMaxPasses];
    pass_log2a(p.sigma_s, p.passes, k2);
    const int dh = p.dist_dtype == DTS_F16;
    for (int i = 0; i < p.passes; ++i) {
        PassArgs r = base_pass(guide, L);
        r.src = u;
        r.dst = u;
        r.d = ws_at(ws, L.dX);
        r.k2 = k2[i];
        if ((st = cuda_status(launch_row_pass(r, dh, PASS_PLAIN, pl.rows, s)))) return st;
        PassArgs c = base_pass(guide, L);
        c.src = u;
        c.d = ws_at(ws, L.dY);
        c.k2 = k2[i];
        if (i == p.passes - 1) {
            c.dst = dst;
            c.dst_pitch = guide->W;
        } else {
            c.dst = u;
        }
        if ((st = cuda_status(launch_col_pass(c, dh, PASS_PLAIN, pl.cols, s)))) return st;
    }
    return DTS_OK;
}

extern "C" int dts_confidence(const dts_guide* guide, const void* target, int target_dtype,
                              const dts_params* params, float sigma_c, float* conf_out, void* ws, size_t ws_bytes,
                              dts_stream stream) {
    int st = check_guide(guide);
    if (!st) st = check_params(params);
    if (st) return st;
    if (!target || !conf_out || !valid_dtype(target_dtype) || !(sigma_c > 0.f) || !isfinite(sigma_c))
        return DTS_ERR_INVALID_ARG;
    Plans pl;
    if ((st = make_plans(guide->H, guide->W, &pl))) return st;
    dts_params p = *params;
    p.conf_mode = DTS_CONF_PLAIN;
    p.save_checkpoints = 0;
    if (p.filter_kernel != DTS_KERNEL_RF) return DTS_ERR_UNSUPPORTED;  // the recursive-filter mean
    const Layout L = make_layout(guide->H, guide->W, &p, 0);
    if (!ws || ((uintptr_t)ws % kPlaneAlign) != 0 || ws_bytes < L.fwd_end) return DTS_ERR_WORKSPACE;
    if ((st = ensure_prepared())) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = bind_workspace(ws, L, guide->W, s))) return st;
    const int H = guide->H, W = guide->W;
    float* m1 = reinterpret_cast<float*>(ws_at(ws, L.u));  // DT(t), filtered in place
    float* m2 = reinterpret_cast<float*>(ws_at(ws, L.z));  // DT(t^2), filtered in place
    // distances, with t copied (as FP32) into the first working plane, then t^2 into the second
    if ((st = run_distances(guide, &p, L, ws, target, target_dtype, m1, s))) return st;
    if ((st = cuda_status(launch_square_plane(m1, m2, L.pitch, H, W, s)))) return st;
    float k2[kMaxPasses];
    pass_log2a(p.sigma_s, p.passes, k2);
    const int dh = p.dist_dtype == DTS_F16;
    for (int i = 0; i < p.passes; ++i) {
        for (float* u : {m1, m2}) {  // the two planes back to back: the same distances stay in L2
            PassArgs r = base_pass(guide, L);
            r.src = u;
            r.dst = u;
            r.d = ws_at(ws, L.dX);
            r.k2 = k2[i];
            if ((st = cuda_status(launch_row_pass(r, dh, PASS_PLAIN, pl.rows, s)))) return st;
        }
        for (float* u : {m1, m2}) {
            PassArgs c = base_pass(guide, L);
            c.src = u;
            c.dst = u;
            c.d = ws_at(ws, L.dY);
            c.k2 = k2[i];
            if ((st = cuda_status(launch_col_pass(c, dh, PASS_PLAIN, pl.cols, s)))) return st;
        }
    }
    return cuda_status(launch_confidence(m1, m2, L.pitch, H, W, sigma_c, conf_out, s));
}

extern "C" int dts_solve(const dts_guide* guide, const void* target, int target_dtype, const float* conf,
                         const float* z_init, const dts_params* params, float* z_out, void* ws, size_t ws_bytes,
                         dts_stream stream) {
    int st = check_guide(guide);
    if (!st) st = check_params(params);
    if (st) return st;
    if (!target || !conf || !z_out || !valid_dtype(target_dtype)) return DTS_ERR_INVALID_ARG;
    if ((st = check_box(guide, params))) return st;
    Plans pl;
    if ((st = make_plans(guide->H, guide->W, &pl))) return st;
    const Layout L = make_layout(guide->H, guide->W, params, 0);
    if (params->iterations > 0 && (!ws || ((uintptr_t)ws % kPlaneAlign) != 0 || ws_bytes < L.fwd_end))
        return DTS_ERR_WORKSPACE;
    if ((st = ensure_prepared())) return st;
    if (params->filter_kernel == DTS_KERNEL_BOX)
        return solve_box(guide, target, target_dtype, conf, z_init, params, z_out, ws, L, (cudaStream_t)stream);
    return solve_forward(guide, target, target_dtype, conf, z_init, params, z_out, ws, L, pl, (cudaStream_t)stream,
                         true);
}


// ---------------------------------------------------------------- batched solve
// Many images of uneven sizes as one CUDA graph: the per-image launch sequences are captured on
// a few internal streams forked from one origin (so small images run side by side), the graph is
// instantiated once per argument set and replayed with a single cudaGraphLaunch.
namespace dts {
namespace {

constexpr int kBatchStreams = 8;

struct BatchResources {
    cudaStream_t capture = nullptr;
    cudaStream_t side[kBatchStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kBatchStreams] = {};
    bool ready = false;
};

struct BatchGraph {
    std::vector<unsigned long long> key;
    cudaGraphExec_t exec = nullptr;
};

std::mutex g_batch_mutex;
BatchResources g_batch_res[kMaxDevices];
std::vector<BatchGraph> g_batch_graphs[kMaxDevices];
constexpr size_t kBatchGraphCache = 8;

int batch_resources(int dev, BatchResources** out) {
    BatchResources& r = g_batch_res[dev];
    if (!r.ready) {
        if (cudaStreamCreateWithFlags(&r.capture, cudaStreamNonBlocking) != cudaSuccess) return DTS_ERR_CUDA;
        for (int j = 0; j < kBatchStreams; ++j)
            if (cudaStreamCreateWithFlags(&r.side[j], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&r.join[j], cudaEventDisableTiming) != cudaSuccess)
                return DTS_ERR_CUDA;
        if (cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming) != cudaSuccess) return DTS_ERR_CUDA;
        r.ready = true;
    }
    *out = &r;
    return DTS_OK;
}

size_t batch_slice(const dts_guide& g, const dts_params* p) {
    return align_up(make_layout(g.H, g.W, p, 0).fwd_end, kPlaneAlign);
}

// How batches run: 0, the persistent kernel where the batch allows it (else the graph of
// per-image launches); 1, the graph of per-image launches.  Set by the batched autotuner or by
// the tuner text's "batch" line.
std::atomic<int> g_batch_policy{0};

// the batch runs as the persistent kernel: recursive filter, GD or Jacobi, plain confidence, at
// least one iteration, at most kBatchMax images of one guide dtype within its size limits
bool batch_is_persistent(int n, const dts_guide* guides, const dts_params* p) {
    if (g_batch_policy.load() != 0 || n > kBatchMax || p->iterations < 1 || p->filter_kernel != DTS_KERNEL_RF ||
        p->conf_mode != DTS_CONF_PLAIN || (p->update != DTS_UPDATE_GD && p->update != DTS_UPDATE_JACOBI))
        return false;
    for (int i = 0; i < n; ++i)
        if (guides[i].dtype != guides[0].dtype || !batch_persistent_fits(guides[i].H, guides[i].W)) return false;
    return true;
}

// The batch as one persistent kernel launch (with the reset of its control words) on `origin`.
int issue_batch_persistent(int n, const dts_guide* guides, const void* const* targets, int tdt,
                           const float* const* confs, const dts_params* p, float* const* z_out, void* ws,
                           cudaStream_t origin) {
    std::vector<BatchPlanes> planes(n);
    size_t off = batch_ctl_bytes(n, p);
    for (int i = 0; i < n; ++i) {
        const Layout L = make_layout(guides[i].H, guides[i].W, p, 0);
        char* base = ws_at(ws, off);
        planes[i] = BatchPlanes{base + L.dX, base + L.dY, reinterpret_cast<float*>(base + L.u),
                                reinterpret_cast<float*>(base + L.z), L.pitch};
        off += batch_slice(guides[i], p);
    }
    BatchLaunch l = {};
    l.n = n;
    l.guides = guides;
    l.targets = targets;
    l.tdtype = tdt;
    l.confs = confs;
    l.p = p;
    l.z_out = z_out;
    l.planes = planes.data();
    pass_log2a(p->sigma_s, p->passes, l.k2);
    l.ctl = static_cast<unsigned*>(ws);
    l.status = status_word();
    return cuda_status(launch_batched(l, origin));
}

// Issues every image's solve on the side streams, forked from and joined back into `origin`.
int issue_batch(int n, const dts_guide* guides, const void* const* targets, int tdt, const float* const* confs,
                const dts_params* p, float* const* z_out, void* ws, BatchResources& r, cudaStream_t origin) {
    if (cudaEventRecord(r.fork, origin) != cudaSuccess) return DTS_ERR_CUDA;
    for (int j = 0; j < kBatchStreams; ++j)
        if (cudaStreamWaitEvent(r.side[j], r.fork, 0) != cudaSuccess) return DTS_ERR_CUDA;
    // largest images first, each onto the least loaded stream
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)guides[a].H * guides[a].W > (long long)guides[b].H * guides[b].W;
    });
    std::vector<size_t> offset(n);
    size_t off = batch_ctl_bytes(n, p);
    for (int i = 0; i < n; ++i) {
        offset[i] = off;
        off += batch_slice(guides[i], p);
    }
    long long load[kBatchStreams] = {};
    for (int i : order) {
        int j = 0;
        for (int q = 1; q < kBatchStreams; ++q)
            if (load[q] < load[j]) j = q;
        load[j] += (long long)guides[i].H * guides[i].W;
        Plans pl;
        int st = make_plans(guides[i].H, guides[i].W, &pl);
        if (st) return st;
        // solves that run side by side keep the cluster shapes for the vertical passes: their
        // smaller CTAs pack several images onto an SM (measured on the 64-image batch), and no
        // CTA of one image waits for CTAs of another to be scheduled (as a chain's might)
        if (pl.cols.cluster <= 0 && !plan_cols_cluster(guides[i].H, &pl.cols)) return DTS_ERR_UNSUPPORTED;
        const Layout L = make_layout(guides[i].H, guides[i].W, p, 0);
        st = solve_forward(&guides[i], targets[i], tdt, confs[i], nullptr, p, z_out[i], ws_at(ws, offset[i]), L, pl,
                           r.side[j]);
        if (st) return st;
    }
    for (int j = 0; j < kBatchStreams; ++j) {
        if (cudaEventRecord(r.join[j], r.side[j]) != cudaSuccess) return DTS_ERR_CUDA;
        if (cudaStreamWaitEvent(origin, r.join[j], 0) != cudaSuccess) return DTS_ERR_CUDA;
    }
    return DTS_OK;
}

}  // namespace
}  // namespace dts

extern "C" size_t dts_batched_workspace_size(int n, const dts_guide* guides, const dts_params* params) {
    if (n < 1 || !guides || check_params(params)) return 0;
    size_t total = batch_ctl_bytes(n, params);
    for (int i = 0; i < n; ++i) {
        if (check_guide(&guides[i])) return 0;
        total += batch_slice(guides[i], params);
    }
    return total;
}

extern "C" int dts_solve_batched(int n, const dts_guide* guides, const void* const* targets, int target_dtype,
                                 const float* const* confs, const dts_params* params, float* const* z_out, void* ws,
                                 size_t ws_bytes, dts_stream stream) {
    if (n < 1 || !guides || !targets || !confs || !z_out || !valid_dtype(target_dtype)) return DTS_ERR_INVALID_ARG;
    int st = check_params(params);
    if (!st && params->filter_kernel != DTS_KERNEL_RF) st = DTS_ERR_UNSUPPORTED;  // recursive-filter kernel only
    if (st) return st;
    if (params->save_checkpoints) return DTS_ERR_UNSUPPORTED;
    if (params->update == DTS_UPDATE_CG && params->conf_mode != DTS_CONF_PLAIN) return DTS_ERR_UNSUPPORTED;
    for (int i = 0; i < n; ++i) {
        if ((st = check_guide(&guides[i]))) return st;
        if (!targets[i] || !confs[i] || !z_out[i]) return DTS_ERR_INVALID_ARG;
        Plans pl;
        if ((st = make_plans(guides[i].H, guides[i].W, &pl))) return st;
        if (!plan_cols_cluster(guides[i].H, &pl.cols)) return DTS_ERR_UNSUPPORTED;  // see issue_batch
    }
    const size_t need = dts_batched_workspace_size(n, guides, params);
    if (params->iterations > 0 && (!ws || ((uintptr_t)ws % kPlaneAlign) != 0 || ws_bytes < need))
        return DTS_ERR_WORKSPACE;
    if ((st = ensure_prepared())) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DTS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    BatchResources* r = nullptr;
    if ((st = batch_resources(dev, &r))) return st;
    const bool persistent = batch_is_persistent(n, guides, params);
    auto issue = [&](cudaStream_t origin) {
        return persistent ? issue_batch_persistent(n, guides, targets, target_dtype, confs, params, z_out, ws, origin)
                          : issue_batch(n, guides, targets, target_dtype, confs, params, z_out, ws, *r, origin);
    };
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return DTS_ERR_CUDA;
    // the caller is capturing: become part of its graph; the per-launch timer is on, or a fault
    // injection is pending: launch directly (a replayed graph's kernels are not bracketed by
    // events, and an injection captured into the cached graph would recur on every replay)
    if (cap != cudaStreamCaptureStatusNone || prof_active() || injection_pending()) return issue(s);
    // key: every pointer, shape and parameter that the captured launches bake in
    std::vector<unsigned long long> key;
    key.push_back((unsigned long long)n);
    key.push_back((unsigned long long)persistent);
    key.push_back((unsigned long long)(uintptr_t)ws);
    key.push_back((unsigned long long)target_dtype);
    {
        unsigned long long pw[(sizeof(dts_params) + 7) / 8] = {};
        memcpy(pw, params, sizeof(dts_params));
        for (unsigned long long v : pw) key.push_back(v);
    }
    for (int i = 0; i < n; ++i) {
        const dts_guide& g = guides[i];
        key.insert(key.end(), {(unsigned long long)g.C, (unsigned long long)g.H, (unsigned long long)g.W,
                               (unsigned long long)g.dtype, (unsigned long long)(uintptr_t)g.data,
                               (unsigned long long)g.ch_stride, (unsigned long long)g.row_stride,
                               (unsigned long long)(uintptr_t)targets[i], (unsigned long long)(uintptr_t)confs[i],
                               (unsigned long long)(uintptr_t)z_out[i]});
    }
    auto& cache = g_batch_graphs[dev];
    for (auto& bg : cache)
        if (bg.key == key) return cudaGraphLaunch(bg.exec, s) == cudaSuccess ? DTS_OK : DTS_ERR_CUDA;
    if (cudaStreamBeginCapture(r->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DTS_ERR_CUDA;
    st = issue(r->capture);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(r->capture, &graph);
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ec != cudaSuccess || !graph) return DTS_ERR_CUDA;
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return DTS_ERR_CUDA;
    if (cache.size() >= kBatchGraphCache) {
        cudaGraphExecDestroy(cache.front().exec);
        cache.erase(cache.begin());
    }
    cache.push_back(BatchGraph{key, exec});
    return cudaGraphLaunch(exec, s) == cudaSuccess ? DTS_OK : DTS_ERR_CUDA;
}


// Times this batch both ways -- the persistent kernel and the graph of per-image launches, each
// replayed from its cached graph, 2 warm-up and 3 timed runs on `stream` -- and keeps the faster
// as the policy of later batched solves.  Batches the persistent kernel does not take leave the
// policy as it is.
extern "C" int dts_autotune_batched(int n, const dts_guide* guides, const void* const* targets, int target_dtype,
                                    const float* const* confs, const dts_params* params, float* const* z_out,
                                    void* ws, size_t ws_bytes, dts_stream stream) {
    if (n < 1 || !guides || !params) return DTS_ERR_INVALID_ARG;
    const int saved = g_batch_policy.load();
    g_batch_policy.store(0);
    const bool eligible = batch_is_persistent(n, guides, params);
    g_batch_policy.store(saved);
    int st;
    if (!eligible)  // validates the arguments all the same
        return dts_solve_batched(n, guides, targets, target_dtype, confs, params, z_out, ws, ws_bytes, stream);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return DTS_ERR_CUDA;
    float ms[2] = {0.f, 0.f};
    for (int policy = 0; policy < 2; ++policy) {
        g_batch_policy.store(policy);
        for (int r = 0; r < 5; ++r) {
            st = r == 2 && cudaEventRecord(e0, s) != cudaSuccess ? (int)DTS_ERR_CUDA : (int)DTS_OK;
            if (st || (st = dts_solve_batched(n, guides, targets, target_dtype, confs, params, z_out, ws, ws_bytes,
                                              stream))) {
                g_batch_policy.store(saved);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st;
            }
        }
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms[policy], e0, e1) != cudaSuccess) {
            g_batch_policy.store(saved);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return DTS_ERR_CUDA;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_batch_policy.store(ms[1] < ms[0] ? 1 : 0);
    return DTS_OK;
}

// ---------------------------------------------------------------- autotuner
namespace dts {
std::string tuned_export();
std::string tuned_bwd_export();
}

extern "C" int dts_autotune(const dts_guide* guide, const dts_params* params, void* ws, size_t ws_bytes,
                            dts_stream stream) {
    int st = check_guide(guide);
    if (!st) st = check_params(params);
    if (!st && params->filter_kernel != DTS_KERNEL_RF) st = DTS_ERR_UNSUPPORTED;  // recursive-filter kernel only
    if (st) return st;
    Plans pl;
    if ((st = make_plans(guide->H, guide->W, &pl))) return st;
    dts_params p = *params;
    p.conf_mode = DTS_CONF_PLAIN;
    p.save_checkpoints = 0;
    const Layout L = make_layout(guide->H, guide->W, &p, 0);
    if (!ws || ((uintptr_t)ws % kPlaneAlign) != 0 || ws_bytes < L.fwd_end) return DTS_ERR_WORKSPACE;
    if ((st = ensure_prepared())) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = bind_workspace(ws, L, guide->W, s))) return st;
    // real distances of this guide; the pass input is the iterate plane (any finite values)
    float* u = reinterpret_cast<float*>(ws_at(ws, L.u));
    if (cudaMemsetAsync(u, 0, L.plane_f32, s) != cudaSuccess) return DTS_ERR_CUDA;
    if ((st = run_distances(guide, &p, L, ws, nullptr, DTS_F32, nullptr, s))) return st;
    float k2[kMaxPasses];
    pass_log2a(p.sigma_s, 1, k2);
    const int dh = p.dist_dtype == DTS_F16;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return DTS_ERR_CUDA;
    auto time_it = [&](auto&& launch) -> float {
        for (int w = 0; w < 2; ++w)
            if (launch() != cudaSuccess) return -1.f;
        cudaEventRecord(e0, s);
        const int reps = 5;
        for (int r = 0; r < reps; ++r)
            if (launch() != cudaSuccess) return -1.f;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / reps;
    };
    // vertical shapes
    ColPlan cand[16];
    const int nc = col_candidates(guide->H, cand, 16);
    float best = 1e30f;
    ColPlan best_plan = pl.cols;
    for (int i = 0; i < nc; ++i) {
        PassArgs c = base_pass(guide, L);
        c.src = u;
        c.dst = u;
        c.d = ws_at(ws, L.dY);
        c.k2 = k2[0];
        const float t = time_it([&] { return launch_col_pass(c, dh, PASS_PLAIN, cand[i], s); });
        cudaGetLastError();
        if (t > 0.f && t < best) {
            best = t;
            best_plan = cand[i];
        }
    }
    set_tuned_col(guide->H, best_plan);
    // horizontal items per thread
    int best_items = pl.rows.items;
    best = 1e30f;
    for (int items : {8, 16, 32, 17, 33}) {
        RowPlan rp;
        rp.items = items;
        rp.tpr = ((guide->W + items - 1) / items + 31) / 32 * 32;
        if (items % 2 ? !row_stream_fits(guide->W, items) : rp.tpr > (items >= 32 ? 320 : 1024)) continue;
        rp.rpb = items % 2 || rp.tpr >= 256 ? 1 : 256 / rp.tpr;
        PassArgs r = base_pass(guide, L);
        r.src = u;
        r.dst = u;
        r.d = ws_at(ws, L.dX);
        r.k2 = k2[0];
        const float t = time_it([&] { return launch_row_pass(r, dh, PASS_PLAIN, rp, s); });
        cudaGetLastError();
        if (t > 0.f && t < best) {
            best = t;
            best_items = items;
        }
    }
    set_tuned_row(guide->W, best_items);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return DTS_OK;
}

extern "C" int dts_autotune_export(char* buf, size_t len) {
    const std::string t = tuned_export() + tuned_bwd_export() + "batch " + std::to_string(g_batch_policy.load()) + "\n";
    if (!buf) return (int)t.size() + 1;
    if (len < t.size() + 1) return -DTS_ERR_INVALID_ARG;
    memcpy(buf, t.c_str(), t.size() + 1);
    return (int)t.size() + 1;
}

extern "C" int dts_autotune_import(const char* text) {
    if (!text) return DTS_ERR_INVALID_ARG;
    const char* p = text;
    while (*p) {
        int a = 0, b = 0, c = 0, d = 0, used = 0;
        if (sscanf(p, "row %d %d %n", &a, &b, &used) == 2 && used > 0) {
            if (a >= 1 && (b == 8 || b == 16 || b == 32 || b == 17 || b == 33)) set_tuned_row(a, b);
        } else if (sscanf(p, "batch %d %n", &a, &used) == 1 && used > 0) {
            if (a == 0 || a == 1) g_batch_policy.store(a);
        } else if (sscanf(p, "bcol %d %d %d %d %n", &a, &b, &c, &d, &used) == 4 && used > 0) {
            set_tuned_bwd_col(a, ColPlan{b, c, d});
        } else if (sscanf(p, "col %d %d %d %d %n", &a, &b, &c, &d, &used) == 4 && used > 0) {
            ColPlan cp{b, c, d};
            ColPlan cand[16];
            const int nc = col_candidates(a, cand, 16);
            for (int i = 0; i < nc; ++i)
                if (cand[i].items == b && cand[i].warps == c && cand[i].cluster == d) set_tuned_col(a, cp);
        } else {
            return DTS_ERR_INVALID_ARG;
        }
        p += used;
    }
    return DTS_OK;
}

// ---------------------------------------------------------------- solve without allocation
// Callers that cannot allocate device memory (for example code running inside a host
// framework that owns every device allocation, or a latency-critical loop where an allocation
// could block, fail or exceed a fixed memory budget) cannot provide a workspace.  For them the
// solve can use this library-owned scratch array instead.  It is a file-scope device array, so
// every GPU that loads the library holds it until the process exits; all calls share it.
namespace dts {
namespace {
constexpr size_t kStaticWorkspaceBytes = (size_t)16 << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];
std::mutex g_static_mutex;
void* g_static_workspace_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code cannot use the
// array's name as a device address; it is looked up once per device, with that device current.
int static_workspace(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DTS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_workspace_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_workspace);
        if (e != cudaSuccess || ptr == nullptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        g_static_workspace_ptr[dev] = ptr;
    }
    *out = g_static_workspace_ptr[dev];
    return DTS_OK;
}
}  // namespace
}  // namespace dts

extern "C" size_t dts_noalloc_max_workspace(void) { return kStaticWorkspaceBytes; }

extern "C" int dts_solve_noalloc(const dts_guide* guide, const void* target, int target_dtype, const float* conf,
                                 const float* z_init, const dts_params* params, float* z_out, dts_stream stream) {
    int st = check_guide(guide);
    if (!st) st = check_params(params);
    if (!st && params->filter_kernel != DTS_KERNEL_RF) st = DTS_ERR_UNSUPPORTED;  // recursive-filter kernel only
    if (st) return st;
    if (!target || !conf || !z_out || !valid_dtype(target_dtype)) return DTS_ERR_INVALID_ARG;
    if (params->save_checkpoints) return DTS_ERR_UNSUPPORTED;  // checkpoints must outlive the call
    if ((st = check_box(guide, params))) return st;
    Plans pl;
    if ((st = make_plans(guide->H, guide->W, &pl))) return st;
    const Layout L = make_layout(guide->H, guide->W, params, 0);
    if (L.fwd_end > kStaticWorkspaceBytes) return DTS_ERR_WORKSPACE;
    if ((st = ensure_prepared())) return st;
    void* ws = nullptr;
    if ((st = static_workspace(&ws))) return st;
    return solve_forward(guide, target, target_dtype, conf, z_init, params, z_out, ws, L, pl, (cudaStream_t)stream);
}

extern "C" int dts_solve_backward(const dts_guide* guide, const void* target, int target_dtype, const float* conf,
                                  const float* z_init, const dts_params* params, void* ws, size_t ws_bytes,
                                  const float* grad_z, float* grad_target, float* grad_conf, float* grad_guide,
                                  float* grad_z_init, dts_stream stream) {
    int st = check_guide(guide);
    if (!st) st = check_params(params);
    if (!st && params->filter_kernel != DTS_KERNEL_RF) st = DTS_ERR_UNSUPPORTED;  // recursive-filter kernel only
    if (st) return st;
    if (!target || !conf || !grad_z || !valid_dtype(target_dtype)) return DTS_ERR_INVALID_ARG;
    if (params->conf_mode != DTS_CONF_PLAIN || params->update == DTS_UPDATE_CG) return DTS_ERR_UNSUPPORTED;
    if (params->save_checkpoints == 0) return DTS_ERR_INVALID_ARG;  // the forward kept no iterates
    Plans pl;
    if ((st = make_plans(guide->H, guide->W, &pl))) return st;
    RowPlan rb;
    ColPlan cb;
    if (!plan_rows_bwd(guide->W, &rb) || !plan_cols_bwd(guide->H, &cb)) return DTS_ERR_UNSUPPORTED;
    const Layout L = make_layout(guide->H, guide->W, params, 1);
    if (!ws || ((uintptr_t)ws % kPlaneAlign) != 0 || ws_bytes < L.total) return DTS_ERR_WORKSPACE;
    if ((st = ensure_prepared())) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = bind_workspace(ws, L, guide->W, s))) return st;
    const int H = guide->H, W = guide->W, K = params->iterations, N = params->passes;
    const long long P = L.pitch;
    const int dh = params->dist_dtype == DTS_F16;
    auto plane = [&](size_t off) { return reinterpret_cast<float*>(ws_at(ws, off)); };
    float* gz = plane(L.gz);
    float* dXb = plane(L.dXb);
    float* dYb = plane(L.dYb);
    const size_t dense = (size_t)H * W * sizeof(float);
    if (grad_target && cudaMemsetAsync(grad_target, 0, dense, s) != cudaSuccess) return DTS_ERR_CUDA;
    if (grad_conf && cudaMemsetAsync(grad_conf, 0, dense, s) != cudaSuccess) return DTS_ERR_CUDA;
    if (cudaMemsetAsync(dXb, 0, L.plane_f32, s) != cudaSuccess) return DTS_ERR_CUDA;
    if (cudaMemsetAsync(dYb, 0, L.plane_f32, s) != cudaSuccess) return DTS_ERR_CUDA;
    if ((st = cuda_status(launch_axpy_plane(grad_z, W, gz, P, H, W, 0, s)))) return st;
    float k2[kMaxPasses];
    pass_log2a(params->sigma_s, N, k2);
    float* U[2 * kMaxPasses];
    for (int p = 1; p < 2 * N; ++p) U[p] = plane(L.xin + (size_t)p * L.plane_f32);
    float* gbuf[2] = {plane(L.g0), plane(L.g1)};
    const bool kept = params->save_checkpoints == 2;
    for (int k = K - 1; k >= 0; --k) {
        U[0] = plane(L.z + (size_t)k * L.plane_f32);
        float* zbar = plane(L.xin);
        if (kept) {  // the forward kept every pass input of iteration k, and zbar_k
            for (int p = 1; p < 2 * N; ++p) U[p] = plane(L.passes + ((size_t)k * 2 * N + p) * L.plane_f32);
            zbar = plane(L.passes + (size_t)k * 2 * N * L.plane_f32);
        }
        // else recompute the inputs of passes 1 .. 2N-1 from the checkpoint z_k, and zbar (the last
        // pass's output) into the free slot 0
        for (int p = 0; p < 2 * N && !kept; ++p) {
            PassArgs a = base_pass(guide, L);
            a.src = U[p];
            a.dst = p + 1 < 2 * N ? U[p + 1] : zbar;
            a.k2 = k2[p / 2];
            if (p % 2 == 0) {
                a.d = ws_at(ws, L.dX);
                if ((st = cuda_status(launch_row_pass(a, dh, PASS_PLAIN, pl.rows, s)))) return st;
            } else {
                a.d = ws_at(ws, L.dY);
                if ((st = cuda_status(launch_col_pass(a, dh, PASS_PLAIN, pl.cols, s)))) return st;
            }
        }
        // adjoint of the data-term update: dzbar into gbuf[0], the direct part stays in gz
        {
            BwdArgs b = {};
            b.x = zbar;
            b.H = H;
            b.W = W;
            b.pitch = P;
            b.gz = gz;
            b.gout = gbuf[0];
            b.t = target;
            b.t_dtype = target_dtype;
            b.c = conf;
            b.zk = U[0];
            b.gt = grad_target;
            b.gc = grad_conf;
            b.lambda = params->lambda;
            b.step = params->step;
            b.update = params->update;
            b.eps = params->charbonnier_eps;
            if ((st = cuda_status(launch_update_adjoint(b, s)))) return st;
        }
        // adjoint passes in reverse order
        int cur = 0;
        for (int p = 2 * N - 1; p >= 0; --p) {
            BwdArgs b = {};
            b.x = U[p];
            b.H = H;
            b.W = W;
            b.pitch = P;
            b.k2 = k2[p / 2];
            b.lna = (float)((double)k2[p / 2] * log(2.0));
            b.gin = gbuf[cur];
            b.gout = gbuf[cur ^ 1];
            b.kout = p + 1 < 2 * N ? U[p + 1] : zbar;
            b.gz = gz;
            if (p % 2 == 1) {
                b.d = ws_at(ws, L.dY);
                b.dbar = dYb;
                b.chain_ctl = reinterpret_cast<unsigned*>(ws_at(ws, L.chain_ctl));
                b.chain_agg = reinterpret_cast<float*>(ws_at(ws, L.chain_agg));
                b.status = status_word();
                if ((st = cuda_status(launch_col_bwd(b, dh, cb, s)))) return st;
            } else {
                b.d = ws_at(ws, L.dX);
                b.dbar = dXb;
                if ((st = cuda_status(launch_row_bwd(b, dh, p == 0, rb, s)))) return st;
            }
            cur ^= 1;
        }
    }
    // z_0: the target itself (z_init NULL) or the caller's z_init
    if (!z_init) {
        if (grad_target && (st = cuda_status(launch_axpy_plane(gz, P, grad_target, W, H, W, 1, s)))) return st;
    } else if (grad_z_init) {
        if ((st = cuda_status(launch_axpy_plane(gz, P, grad_z_init, W, H, W, 0, s)))) return st;
    }
    if (grad_guide) {
        GuideGradArgs gg = {};
        gg.guide = guide->data;
        gg.row_stride = guide->row_stride ? guide->row_stride : W;
        gg.ch_stride = guide->ch_stride ? guide->ch_stride : (long long)H * gg.row_stride;
        gg.C = guide->C;
        gg.H = H;
        gg.W = W;
        gg.gdtype = guide->dtype;
        gg.norm = params->norm;
        gg.dhalf = dh;
        gg.k = params->sigma_s / params->sigma_r;
        gg.dX = ws_at(ws, L.dX);
        gg.dY = ws_at(ws, L.dY);
        gg.dXb = dXb;
        gg.dYb = dYb;
        gg.pitch = P;
        gg.out = grad_guide;
        if ((st = cuda_status(launch_guide_grad(gg, s)))) return st;
    }
    return DTS_OK;
}

extern "C" int dts_debug_inject(int kind) {
    if (kind < 0 || kind > DTS_INJECT_STAGE_SKIP) return DTS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_prep_mutex);
    g_inject = kind;
    return DTS_OK;
}

extern "C" int dts_last_status(dts_stream stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DTS_ERR_CUDA;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof(int)) != cudaSuccess) return DTS_ERR_CUDA;
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_status, &zero, sizeof(int)) != cudaSuccess) return DTS_ERR_CUDA;
    }
    return v;
}
