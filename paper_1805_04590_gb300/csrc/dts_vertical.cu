// Vertical pass in two cluster-free kernels (an alternative to the cluster kernel, DTS_COL_SPLIT=1).
//
// A column is cut into segments of kSeg = 32 rows.  For a segment, with c the causal value
// entering from above and k the anti-causal value entering from below,
//     c_out = A c + B,      k_start = al k + be c + ga
// (see dts_scan.cuh).  col_agg_kernel streams every segment once and stores its five numbers;
// the last CTA to finish a strip of columns (an atomic ticket, no waiting) scans the segments
// of each of its columns top-down for the carries c entering every segment and bottom-up for
// the values k entering from below.  col_apply_kernel then replays each segment from its two
// carries -- causal sweep down, anti-causal sweep up -- re-reading the segment (from L2, where
// the first kernel just left it) and writing the pass output, or the data-term update of
// Eq. 3 / Eq. 4 when it is the last pass of an iteration.  No CTA ever waits for another.
#include "dts_scan.cuh"

namespace dts {

namespace {

using namespace scan;

constexpr int kSeg = 32;        // rows per segment
constexpr int kAggWarps = 4;    // segments per aggregate CTA
constexpr int kApplyWarps = 4;  // segments per apply CTA

// ---------------------------------------------------------------- segment aggregates
// CTA = kAggWarps warps of one strip of 128 columns; warp q takes segment blockIdx.y*kAggWarps+q,
// lane l columns [4l, 4l+4) of the strip (16-byte loads along each row).  The five numbers of
// a column segment accumulate in one walk down it, each position finalised once the weight to
// its successor is known.
template <bool DHALF>
__global__ void __launch_bounds__(32 * kAggWarps) col_agg_kernel(PassArgs a) {
    __shared__ int s_last;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int c0 = (blockIdx.x * 32 + lane) * 4;
    const int s = blockIdx.y * kAggWarps + warp;
    const int r0 = s * kSeg;
    const long long P = a.pitch;
    const bool cok = c0 < a.W;

    wait_predecessor();
    float Pp[4], Q[4], r[4], be[4], ga[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Pp[i] = 1.f;
        Q[i] = 0.f;
        r[i] = 1.f;
        be[i] = ga[i] = 0.f;
    }
    if (r0 < a.H) {
#pragma unroll 4
        for (int n = 0; n <= kSeg; ++n) {
            const int row = r0 + n;
            float x[4] = {0.f, 0.f, 0.f, 0.f}, w[4] = {0.f, 0.f, 0.f, 0.f};
            if (cok && row < a.H) {
                const long long idx = (long long)row * P + c0;
                if (n < kSeg) load4_f(a.src, idx, x);
                load4_d<DHALF>(a.d, idx, w);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    w[i] = (row > 0 && c0 + i < a.W) ? ex2(a.k2 * w[i]) : 0.f;
                    if (c0 + i >= a.W) x[i] = 0.f;
                }
            }
            if (n > 0) {  // position n-1 is final now that its successor's weight is known
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float coef = fmaf(-r[i], w[i], r[i]);
                    be[i] = fmaf(coef, Pp[i], be[i]);
                    ga[i] = fmaf(coef, Q[i], ga[i]);
                    r[i] *= w[i];
                }
            }
            if (n < kSeg) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    Pp[i] *= w[i];
                    Q[i] = fmaf(w[i], Q[i] - x[i], x[i]);
                }
            }
        }
        if (cok) {
            const long long o = (long long)s * a.agg_pitch + c0;
            store4_f(a.agg + 0 * a.agg_plane, o, Pp);
            store4_f(a.agg + 1 * a.agg_plane, o, Q);
            store4_f(a.agg + 2 * a.agg_plane, o, r);
            store4_f(a.agg + 3 * a.agg_plane, o, be);
            store4_f(a.agg + 4 * a.agg_plane, o, ga);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.counters + blockIdx.x, 1u) == gridDim.y - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the strip's last CTA: carries of every segment of its 128 columns
    const int nseg = (a.H + kSeg - 1) / kSeg;
    for (int cc = threadIdx.x; cc < 128; cc += blockDim.x) {
        const int col = blockIdx.x * 128 + cc;
        if (col >= a.W) continue;
        const float* A = a.agg + 0 * a.agg_plane + col;
        const float* B = a.agg + 1 * a.agg_plane + col;
        float* cin = a.carry + col;
        float* kin = a.carry + a.agg_plane + col;
        float c = 0.f;
        for (int q = 0; q < nseg; ++q) {
            const long long o = (long long)q * a.agg_pitch;
            cin[o] = c;
            c = fmaf(__ldcg(A + o), c, __ldcg(B + o));
        }
        Coupled after = coupled_identity();
        for (int q = nseg - 1; q >= 0; --q) {
            const long long o = (long long)q * a.agg_pitch;
            const Coupled own{__ldcg(A + o), __ldcg(B + o), __ldcg(a.agg + 2 * a.agg_plane + col + o),
                              __ldcg(a.agg + 3 * a.agg_plane + col + o), __ldcg(a.agg + 4 * a.agg_plane + col + o)};
            const float c_out = fmaf(own.A, cin[o], own.B);
            kin[o] = k_entering(after, c_out);
            after = coupled_compose(own, after);
        }
    }
    if (threadIdx.x == 0) a.counters[blockIdx.x] = 0u;  // ready for the next launch
}

// ---------------------------------------------------------------- segment replay
// CTA = kApplyWarps warps = consecutive segments of one strip of 32 columns; lane = column.
template <bool DHALF, int KIND>
__global__ void __launch_bounds__(32 * kApplyWarps, 5) col_apply_kernel(PassArgs a) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int s = blockIdx.y * kApplyWarps + warp;
    const int r0 = s * kSeg;
    const long long P = a.pitch;
    const bool col_ok = col < a.W;

    wait_predecessor();
    if (!(col_ok && r0 < a.H)) return;  // no barrier below: idle lanes may leave
    const long long co = (long long)s * a.agg_pitch + col;
    const float c = a.carry[co];
    const float k = a.carry[a.agg_plane + co];
    const bool full = r0 + kSeg <= a.H;
    float x[kSeg], w[kSeg];
    const float* src = a.src + (long long)r0 * P + col;
    const long long d0 = (long long)r0 * P + col;
#pragma unroll
    for (int j = 0; j < kSeg; ++j) {
        const bool ok = full || r0 + j < a.H;
        x[j] = ok ? src[j * P] : 0.f;
        w[j] = ok ? load1_d<DHALF>(a.d, d0 + j * P) : 0.f;
    }
    const int rn = r0 + kSeg;
    const float wn = rn < a.H ? ex2(a.k2 * load1_d<DHALF>(a.d, (long long)rn * P + col)) : 0.f;
#pragma unroll
    for (int j = 0; j < kSeg; ++j) {
        const int row = r0 + j;
        w[j] = (row > 0 && row < a.H) ? ex2(a.k2 * w[j]) : 0.f;
    }
    float J = c;
#pragma unroll
    for (int j = 0; j < kSeg; ++j) {
        J = fmaf(w[j], J - x[j], x[j]);
        x[j] = J;
    }
    float K = k;
#pragma unroll
    for (int j = kSeg - 1; j >= 0; --j) {
        const float wp = (j + 1 < kSeg) ? w[j + 1] : wn;
        K = fmaf(wp, K - x[j], x[j]);
        x[j] = K;
    }
    release_successor();
#pragma unroll
    for (int j = 0; j < kSeg; ++j) {
        const int row = r0 + j;
        if (!full && row >= a.H) continue;
        if constexpr (KIND == PASS_PLAIN) {
            a.dst[(long long)row * a.dst_pitch + col] = x[j];
        } else {
            const long long idx = (long long)row * P + col;
            const long long di = (long long)row * a.W + col;
            const float zb = x[j];
            const float z = a.zk[idx];
            const float t = load_any(a.t, di, a.t_dtype);
            const float cf = a.c_pitched ? a.c[idx] : a.c[di];
            float zn;
            if (a.update == DTS_UPDATE_JACOBI) {
                const float den = a.lambda + cf;
                zn = den != 0.f ? (a.lambda * zb + cf * t) / den : z;
            } else {
                float eta = a.step;
                if (a.clamp_step && a.lambda + cf > 0.f) eta = fminf(eta, 1.f / (a.lambda + cf));
                zn = z - eta * (a.lambda * (z - zb) + cf * target_slope(z - t, a.eps));
            }
            a.zout[(long long)row * a.zout_pitch + col] = zn;
        }
    }
}

}  // namespace

// scratch of the split vertical pass: agg_pitch = W rounded up to 128 columns, nseg = ceil(H/32)
void split_col_scratch(int H, int W, long long* agg_pitch, long long* agg_plane, int* nstrips128) {
    const long long pitch = ((long long)W + 127) / 128 * 128;
    const long long nseg = ((long long)H + kSeg - 1) / kSeg;
    *agg_pitch = pitch;
    *agg_plane = pitch * nseg;
    *nstrips128 = (int)(pitch / 128);
}

cudaError_t launch_col_split(const PassArgs& a, int dist_half, int kind, cudaStream_t s) {
    const int nseg = (a.H + kSeg - 1) / kSeg;
    const int flags = (dist_half ? kFlagDistHalf : 0) | (kind == PASS_UPDATE && a.t_dtype != DTS_F32 ? kFlagTarget16 : 0);
    const long long px = (long long)a.H * a.W;
    int h = prof_begin(KID_COL_AGG, px, flags, s);
    const dim3 ga((unsigned)((a.W + 127) / 128), (unsigned)((nseg + kAggWarps - 1) / kAggWarps));
    cudaError_t e = dist_half ? launch_ex(col_agg_kernel<true>, ga, dim3(32 * kAggWarps), 0, s, a)
                              : launch_ex(col_agg_kernel<false>, ga, dim3(32 * kAggWarps), 0, s, a);
    prof_end(h, s);
    if (e != cudaSuccess) return e;
    h = prof_begin(kind == PASS_UPDATE ? KID_COL_UPDATE : KID_COL_PLAIN, px, flags, s);
    const dim3 gb((unsigned)((a.W + 31) / 32), (unsigned)((nseg + kApplyWarps - 1) / kApplyWarps));
    if (kind == PASS_UPDATE)
        e = dist_half ? launch_ex(col_apply_kernel<true, PASS_UPDATE>, gb, dim3(32 * kApplyWarps), 0, s, a)
                      : launch_ex(col_apply_kernel<false, PASS_UPDATE>, gb, dim3(32 * kApplyWarps), 0, s, a);
    else
        e = dist_half ? launch_ex(col_apply_kernel<true, PASS_PLAIN>, gb, dim3(32 * kApplyWarps), 0, s, a)
                      : launch_ex(col_apply_kernel<false, PASS_PLAIN>, gb, dim3(32 * kApplyWarps), 0, s, a);
    prof_end(h, s);
    return e;
}

}  // namespace dts
