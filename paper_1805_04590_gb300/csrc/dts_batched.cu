// The batched solve as one persistent kernel (many independent images of uneven sizes, §3.1: the
// iterations of one image never read another's).
//
// Every image's solve is cut into stages -- its distances (and z_0 = t), then per iteration N
// horizontal and N vertical passes (the data-term update of the previous iteration fused into the
// first horizontal pass), then the last update -- and every stage into jobs: groups of rows for
// the distances, the horizontal passes and the update, 8-column strips over the whole height for
// the vertical passes.  The jobs of all images form one queue in round order: round r holds stage
// r of every image.  A persistent grid of CTAs takes jobs in queue order (an atomic ticket); a job
// first waits until every job of its image's previous stage has finished (a counter per stage),
// then runs, then counts itself done.  A job waits only on jobs with smaller tickets, which are
// held by CTAs that are running or finished and wait on smaller tickets still, so the queue always
// advances, whatever the number of resident CTAs.  Waits are bounded (DTS_ERR_TIMEOUT and an
// abort word that ends every later wait of the launch).
//
// The iterate and the pass buffer of an image are rewritten stage after stage by CTAs on every
// SM; the jobs read them through L2 only (an SM's L1 may hold lines of an earlier stage).
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>

#include "dts_modes.cuh"

namespace dts {

namespace {

using namespace scan;

constexpr int kBatchThreads = 512;  // 16 warps per CTA, two CTAs per SM
constexpr int kBatchRowItems = 16;  // positions per thread of the horizontal passes
constexpr int kBatchJobPixels = 16384;  // pixels a job aims at (several row groups or strips)

// one image of the batch: caller buffers, its workspace planes (row pitch `pitch`) and job shapes
struct BatchImage {
    const void* guide;
    long long ch_stride, row_stride;
    const void* t;
    const float* c;
    float* zout;
    void* dX;
    void* dY;
    float* u;
    float* z;
    long long pitch;
    int C, H, W;
    int tpr, rpb;     // horizontal passes: threads per row (a multiple of 32), rows per row group
    int gpj;          // row groups per horizontal job
    int col_items;    // rows per thread of the vertical passes (9 or 17)
    int spj;          // 8-column strips per vertical job
    int tile_rows;    // rows per distance / update job
    int row_jobs, col_jobs, tile_jobs;
    int tc_vec;       // t and c rows readable as 16-byte vectors
};

struct BatchArgs {
    int n, K, N, S;   // images, iterations, passes, stages per image (2 N K + 2)
    int gdtype, tdtype, norm, dhalf, update;
    float k;          // sigma_s / sigma_r
    float k2[kMaxPasses];
    float lambda, step, eps;
    unsigned* ctl;    // [0] ticket, [1] abort, [kBatchCtlHead + m S + s] finished jobs of stage s of image m
    long long timeout;
    int* status;
    int skip_ticket;  // fault injection: this job does not count itself done (-1: none)
    // jobs of the images before m in a round of distance / update tiles, horizontal passes, vertical passes
    int pre_tile[kBatchMax + 1], pre_row[kBatchMax + 1], pre_col[kBatchMax + 1];
    BatchImage img[kBatchMax];
};

// the image m with pre[m] <= j < pre[m + 1] (pre ascending, pre[0] = 0)
__device__ __forceinline__ int image_of(const int* pre, int n, int j) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// job t of the queue: image, stage and index of the job within the stage
struct Job {
    int m, s, j;
};
__device__ __forceinline__ Job decode(const BatchArgs& a, int t) {
    const int rt = a.pre_tile[a.n], rr = a.pre_row[a.n], rc = a.pre_col[a.n];
    Job o;
    if (t < rt) {  // round 0: distances
        o.m = image_of(a.pre_tile, a.n, t);
        o.s = 0;
        o.j = t - a.pre_tile[o.m];
        return o;
    }
    t -= rt;
    const int pairs = a.N * a.K;  // (horizontal, vertical) round pairs
    const int pair = t / (rr + rc);
    if (pair < pairs) {
        const int rem = t - pair * (rr + rc);
        if (rem < rr) {
            o.m = image_of(a.pre_row, a.n, rem);
            o.s = 1 + 2 * pair;
            o.j = rem - a.pre_row[o.m];
        } else {
            o.m = image_of(a.pre_col, a.n, rem - rr);
            o.s = 2 + 2 * pair;
            o.j = rem - rr - a.pre_col[o.m];
        }
        return o;
    }
    t -= pairs * (rr + rc);  // the last round: the update
    o.m = image_of(a.pre_tile, a.n, t);
    o.s = a.S - 1;
    o.j = t - a.pre_tile[o.m];
    return o;
}

__device__ __forceinline__ int stage_jobs(const BatchImage& im, int s, int S) {
    if (s == 0 || s == S - 1) return im.tile_jobs;
    return (s & 1) ? im.row_jobs : im.col_jobs;
}

__device__ __forceinline__ float guide_at(const void* g, long long i, int dtype) { return load_any(g, i, dtype); }

// distances dX, dY and z_0 = t for rows [r0, r0 + tile_rows) of image im (thread-strided)
__device__ void distance_job(const BatchArgs& a, const BatchImage& im, int r0) {
    const int rows = min(im.tile_rows, im.H - r0);
    const bool l2 = a.norm == DTS_NORM_L2;
    for (int i = threadIdx.x; i < rows * im.W; i += blockDim.x) {
        const int y = r0 + i / im.W;
        const int x = i - (i / im.W) * im.W;
        float sx = 0.f, sy = 0.f;
        for (int c = 0; c < im.C; ++c) {
            const long long p = (long long)c * im.ch_stride + (long long)y * im.row_stride + x;
            const float v = guide_at(im.guide, p, a.gdtype);
            const float dxv = x > 0 ? v - guide_at(im.guide, p - 1, a.gdtype) : 0.f;
            const float dyv = y > 0 ? v - guide_at(im.guide, p - im.row_stride, a.gdtype) : 0.f;
            sx += l2 ? dxv * dxv : fabsf(dxv);
            sy += l2 ? dyv * dyv : fabsf(dyv);
        }
        float dx = l2 ? sqrtf(fmaf(a.k * a.k, sx, 1.f)) : fmaf(a.k, sx, 1.f);
        float dy = l2 ? sqrtf(fmaf(a.k * a.k, sy, 1.f)) : fmaf(a.k, sy, 1.f);
        if (x == 0) dx = 1.f;
        if (y == 0) dy = 1.f;
        const long long q = (long long)y * im.pitch + x;
        if (a.dhalf) {
            static_cast<__half*>(im.dX)[q] = __float2half_rn(dx);
            static_cast<__half*>(im.dY)[q] = __float2half_rn(dy);
        } else {
            static_cast<float*>(im.dX)[q] = dx;
            static_cast<float*>(im.dY)[q] = dy;
        }
        im.z[q] = load_any(im.t, (long long)y * im.W + x, a.tdtype);
    }
}

// the last data-term update, rows [r0, r0 + tile_rows): z_K = update(z_{K-1}, zbar = u, t, c)
__device__ void update_job(const BatchArgs& a, const BatchImage& im, int r0) {
    const int rows = min(im.tile_rows, im.H - r0);
    for (int i = threadIdx.x; i < rows * im.W; i += blockDim.x) {
        const int y = r0 + i / im.W;
        const int x = i - (i / im.W) * im.W;
        const long long q = (long long)y * im.pitch + x;
        const long long di = (long long)y * im.W + x;
        im.zout[di] = dts_update_value(__ldcg(im.z + q), __ldcg(im.u + q), load_any(im.t, di, a.tdtype), im.c[di],
                                       a.lambda, a.step, a.update, 0, a.eps);
    }
}

// the pass arguments of one horizontal or vertical pass of image im
__device__ __forceinline__ PassArgs pass_args(const BatchArgs& a, const BatchImage& im, int pass) {
    PassArgs p = {};
    p.H = im.H;
    p.W = im.W;
    p.pitch = im.pitch;
    p.dst_pitch = im.pitch;
    p.k2 = a.k2[pass];
    p.status = a.status;
    return p;
}

template <bool DHALF>
__device__ void run_job(const BatchArgs& a, const Job& jb) {
    const BatchImage& im = a.img[jb.m];
    if (jb.s == 0) {
        distance_job(a, im, jb.j * im.tile_rows);
        return;
    }
    if (jb.s == a.S - 1) {
        update_job(a, im, jb.j * im.tile_rows);
        return;
    }
    const int p = jb.s - 1;                  // pass index 0 .. 2NK - 1
    const int k = p / (2 * a.N);             // iteration
    const int i = (p % (2 * a.N)) / 2;       // pass of the iteration
    PassArgs pa = pass_args(a, im, i);
    if ((p & 1) == 0) {  // horizontal
        pa.d = im.dX;
        pa.dst = im.u;
        const int g0 = jb.j * im.gpj, g1 = min(g0 + im.gpj, (im.H + im.rpb - 1) / im.rpb);
        if (i == 0 && k > 0) {
            // z_k = update(z_{k-1}, zbar_{k-1} = u, t, c), written over z_{k-1}, then filtered
            pa.src = im.u;
            pa.zk = im.z;
            pa.zout = im.z;
            pa.zout_pitch = im.pitch;
            pa.t = im.t;
            pa.t_dtype = a.tdtype;
            pa.c = im.c;
            pa.lambda = a.lambda;
            pa.step = a.step;
            pa.update = a.update;
            pa.eps = a.eps;
            pa.tc_vec = im.tc_vec;
            for (int g = g0; g < g1; ++g) {
                row_pass_body<kBatchRowItems, DHALF, PASS_UPDATE_ROW, true, true>(pa, im.tpr, im.rpb, g);
                __syncthreads();  // the body's shared arrays are reused by the next group
            }
        } else {
            pa.src = i == 0 ? im.z : im.u;
            for (int g = g0; g < g1; ++g) {
                row_pass_body<kBatchRowItems, DHALF, PASS_PLAIN, true, true>(pa, im.tpr, im.rpb, g);
                __syncthreads();
            }
        }
    } else {  // vertical, on the pass buffer in place
        pa.d = im.dY;
        pa.src = im.u;
        pa.dst = im.u;
        const int s0 = jb.j * im.spj, s1 = min(s0 + im.spj, (im.W + kStripCols - 1) / kStripCols);
        for (int st = s0; st < s1; ++st) {
            if (im.col_items == 9) strip_pass_body<9, DHALF, true>(pa, st);
            else strip_pass_body<17, DHALF, true>(pa, st);
            __syncthreads();
        }
    }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <bool DHALF>
__global__ void __launch_bounds__(kBatchThreads, 2) batched_solve_kernel(const __grid_constant__ BatchArgs a, int total) {
    __shared__ int s_ticket;
    wait_predecessor();
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&a.ctl[0], 1u);
    for (;;) {
        __syncthreads();
        const int t = s_ticket;
        __syncthreads();  // s_ticket is rewritten at the end of the job
        if (t >= total) break;
        // the next ticket is drawn now and used after this job, so its round trip overlaps the
        // job (it waits only on smaller tickets, and this CTA finishes the current job first)
        unsigned next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&a.ctl[0], 1u);
        const Job jb = decode(a, t);
        unsigned* done = a.ctl + kBatchCtlHead + (long long)jb.m * a.S;
        if (jb.s > 0 && threadIdx.x == 0) {
            // every job of the image's previous stage has finished
            const unsigned need = (unsigned)stage_jobs(a.img[jb.m], jb.s - 1, a.S);
            if (ld_acquire(done + jb.s - 1) < need && ld_acquire(a.ctl + 1) == 0u) {
                const long long t0 = clock64();
                while (ld_acquire(done + jb.s - 1) < need) {
                    if (ld_acquire(a.ctl + 1) != 0u) break;
                    if (clock64() - t0 > a.timeout) {
                        atomicExch(a.ctl + 1, 1u);
                        record_status(a.status, DTS_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        __syncthreads();
        run_job<DHALF>(a, jb);
        __syncthreads();  // every thread's writes of the job come before its count
        if (threadIdx.x == 0) {
            if (t != a.skip_ticket) {
                __threadfence();
                atomicAdd(done + jb.s, 1u);
            }
            s_ticket = (int)next;
        }
    }
}

}  // namespace

size_t batch_ctl_bytes(int n, const dts_params* p) {
    const size_t S = 2 * (size_t)p->passes * (size_t)p->iterations + 2;
    return ((kBatchCtlHead + (size_t)n * S) * sizeof(unsigned) + 255) / 256 * 256;
}

bool batch_persistent_fits(int H, int W) { return H >= 1 && H <= kBatchMaxRows && W >= 1 && W <= kBatchMaxCols; }

cudaError_t launch_batched(const BatchLaunch& l, cudaStream_t s) {
    if (l.n < 1 || l.n > kBatchMax || l.p->iterations < 1) return cudaErrorInvalidValue;
    BatchArgs a = {};
    a.n = l.n;
    a.K = l.p->iterations;
    a.N = l.p->passes;
    a.S = 2 * a.N * a.K + 2;
    a.tdtype = l.tdtype;
    a.norm = l.p->norm;
    a.dhalf = l.p->dist_dtype == DTS_F16;
    a.update = l.p->update;
    a.k = l.p->sigma_s / l.p->sigma_r;
    for (int i = 0; i < a.N; ++i) a.k2[i] = l.k2[i];
    a.lambda = l.p->lambda;
    a.step = l.p->step;
    a.eps = l.p->charbonnier_eps;
    a.ctl = l.ctl;
    a.status = l.status;
    // fault injection (tests): the first job does not count itself done, so the waits of its
    // image's next stage run out (about a millisecond)
    const bool skip = take_injected(DTS_INJECT_QUEUE_SKIP);
    a.timeout = skip ? kInjectedTimeout : kWaitTimeout;
    a.skip_ticket = skip ? 0 : -1;
    int gdtype = -1;
    a.pre_tile[0] = a.pre_row[0] = a.pre_col[0] = 0;
    for (int m = 0; m < l.n; ++m) {
        const dts_guide& g = l.guides[m];
        if (gdtype >= 0 && g.dtype != gdtype) return cudaErrorInvalidValue;  // one guide dtype per launch
        gdtype = g.dtype;
        if (!batch_persistent_fits(g.H, g.W)) return cudaErrorInvalidValue;
        BatchImage& im = a.img[m];
        im.guide = g.data;
        im.row_stride = g.row_stride ? g.row_stride : g.W;
        im.ch_stride = g.ch_stride ? g.ch_stride : (long long)g.H * im.row_stride;
        im.C = g.C;
        im.H = g.H;
        im.W = g.W;
        im.t = l.targets[m];
        im.c = l.confs[m];
        im.zout = l.z_out[m];
        im.dX = l.planes[m].dX;
        im.dY = l.planes[m].dY;
        im.u = l.planes[m].u;
        im.z = l.planes[m].z;
        im.pitch = l.planes[m].pitch;
        im.tpr = ((g.W + kBatchRowItems - 1) / kBatchRowItems + 31) / 32 * 32;
        im.rpb = kBatchThreads / im.tpr;
        im.gpj = std::max(1, kBatchJobPixels / (im.rpb * g.W));
        im.col_items = g.H <= 4 * (kBatchThreads / 32) * 9 ? 9 : 17;
        im.spj = std::max(1, kBatchJobPixels / (kStripCols * g.H));
        im.tile_rows = std::max(1, kBatchJobPixels / g.W);
        const int groups = (g.H + im.rpb - 1) / im.rpb, strips = (g.W + kStripCols - 1) / kStripCols;
        im.row_jobs = (groups + im.gpj - 1) / im.gpj;
        im.col_jobs = (strips + im.spj - 1) / im.spj;
        im.tile_jobs = (g.H + im.tile_rows - 1) / im.tile_rows;
        const int tsz = l.tdtype == DTS_F32 ? 4 : 2;
        im.tc_vec = g.W % 4 == 0 && (uintptr_t)l.targets[m] % (4 * tsz) == 0 && (uintptr_t)l.confs[m] % 16 == 0;
        a.pre_tile[m + 1] = a.pre_tile[m] + im.tile_jobs;
        a.pre_row[m + 1] = a.pre_row[m] + im.row_jobs;
        a.pre_col[m + 1] = a.pre_col[m] + im.col_jobs;
    }
    a.gdtype = gdtype;
    const long long total = 2LL * a.pre_tile[l.n] + (long long)a.N * a.K * (a.pre_row[l.n] + a.pre_col[l.n]);
    if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
    auto kernel = a.dhalf ? batched_solve_kernel<true> : batched_solve_kernel<false>;
    const int per_sm = blocks_per_sm((const void*)kernel, kBatchThreads, 0);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<long long>(total, (long long)per_sm * sm_count());
    cudaError_t e = cudaMemsetAsync(l.ctl, 0, batch_ctl_bytes(l.n, l.p), s);
    if (e != cudaSuccess) return e;
    long long pixels = 0;
    for (int m = 0; m < l.n; ++m) pixels += (long long)a.img[m].H * a.img[m].W;
    const int h = prof_begin(KID_BATCHED, pixels, (a.dhalf ? kFlagDistHalf : 0) | (l.tdtype != DTS_F32 ? kFlagTarget16 : 0), s);
    e = scan::launch_ex(kernel, dim3((unsigned)grid), dim3(kBatchThreads), 0, s, a, (int)total);
    prof_end(h, s);
    return e;
}

}  // namespace dts
