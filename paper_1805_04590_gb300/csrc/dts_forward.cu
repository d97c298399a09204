// Forward kernels of the Domain Transform Solver for sm_103a.
//
//  distance_kernel   domain-transform distances dX, dY (§3.2, Eq. 8-9), once per solve
//  row_pass_kernel   one horizontal recursive-filter pass (causal + anti-causal, §2/§3.2)
//  col_pass_kernel   one vertical pass; the last one of an iteration also applies the
//                    data-term update of Eq. 3 (gradient step) or Eq. 4 (fixed point)
//
// Every 1-D sweep J[n] = (1 - w_n) x[n] + w_n J[n-1] (w_n = a^d_n) is an affine map of
// J[n-1].  A thread owns ITEMS consecutive elements of a line in registers, folds them
// into one affine map, the maps of all threads of the line are combined by a scan
// (warp shuffles, then shared memory, then distributed shared memory across the CTAs
// of a cluster for columns), and each thread then replays its elements from the exact
// carry-in.  A line is read once and written once per pass: 2 s_z + s_d bytes per pixel.
#include <cooperative_groups.h>

#include "dts_internal.cuh"

namespace cg = cooperative_groups;

namespace dts {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// v -> A v + B
struct Aff {
    float A, B;
};

// apply `first`, then `second`
__device__ __forceinline__ Aff compose(Aff first, Aff second) {
    return Aff{first.A * second.A, fmaf(second.A, first.B, second.B)};
}

// inclusive scan over lanes 0..lane (lane 0 applied first)
__device__ __forceinline__ Aff warp_scan_up(Aff v, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        float A = __shfl_up_sync(kFull, v.A, off);
        float B = __shfl_up_sync(kFull, v.B, off);
        if (lane >= off) v = compose(Aff{A, B}, v);
    }
    return v;
}

// inclusive scan over lanes lane..31 (lane 31 applied first)
__device__ __forceinline__ Aff warp_scan_down(Aff v, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        float A = __shfl_down_sync(kFull, v.A, off);
        float B = __shfl_down_sync(kFull, v.B, off);
        if (lane + off < 32) v = compose(Aff{A, B}, v);
    }
    return v;
}

template <bool DHALF>
__device__ __forceinline__ void load4_d(const void* base, long long idx, float* out) {
    if constexpr (DHALF) {
        uint2 v = *reinterpret_cast<const uint2*>(static_cast<const __half*>(base) + idx);
        __half2 h0 = *reinterpret_cast<__half2*>(&v.x);
        __half2 h1 = *reinterpret_cast<__half2*>(&v.y);
        float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
        out[0] = f0.x; out[1] = f0.y; out[2] = f1.x; out[3] = f1.y;
    } else {
        float4 v = *reinterpret_cast<const float4*>(static_cast<const float*>(base) + idx);
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    }
}

template <bool DHALF>
__device__ __forceinline__ float load1_d(const void* base, long long idx) {
    if constexpr (DHALF) return __half2float(static_cast<const __half*>(base)[idx]);
    else return static_cast<const float*>(base)[idx];
}

// ---------------------------------------------------------------- distances
template <typename GT, typename DT>
__global__ void __launch_bounds__(256) distance_kernel(DistArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.W) return;
    const GT* I = static_cast<const GT*>(a.guide);
    const long long p = (long long)y * a.row_stride + x;
    float sx = 0.f, sy = 0.f;
    for (int c = 0; c < a.C; ++c) {
        const GT* Ic = I + (long long)c * a.ch_stride;
        const float v = to_f32<GT>(Ic[p]);
        if (x > 0) {
            const float dv = v - to_f32<GT>(Ic[p - 1]);
            sx += a.norm == DTS_NORM_L2 ? dv * dv : fabsf(dv);
        }
        if (y > 0) {
            const float dv = v - to_f32<GT>(Ic[p - a.row_stride]);
            sy += a.norm == DTS_NORM_L2 ? dv * dv : fabsf(dv);
        }
    }
    float dx, dy;
    if (a.norm == DTS_NORM_L2) {
        dx = sqrtf(fmaf(a.k * a.k, sx, 1.f));
        dy = sqrtf(fmaf(a.k * a.k, sy, 1.f));
    } else {
        dx = fmaf(a.k, sx, 1.f);
        dy = fmaf(a.k, sy, 1.f);
    }
    const long long q = (long long)y * a.pitch + x;
    static_cast<DT*>(a.dX)[q] = from_f32<DT>(dx);
    static_cast<DT*>(a.dY)[q] = from_f32<DT>(dy);
    if (a.dst) a.dst[q] = load_any(a.src, (long long)y * a.W + x, a.src_dtype);
}

__global__ void __launch_bounds__(256) copy_plane_kernel(const void* src, int src_dtype, long long sp, float* dst,
                                                         long long dp, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    dst[(long long)y * dp + x] = load_any(src, (long long)y * sp + x, src_dtype);
}

// ---------------------------------------------------------------- horizontal pass
// CTA = rpb rows x tpr threads; thread t of a row owns elements [t*ITEMS, t*ITEMS+ITEMS).
// KIND: PASS_PLAIN (normalised causal then anti-causal on the causal result) or
//       PASS_SUPPORT (unnormalised sweeps of the constant 1: out = P + Q - 1).
template <int ITEMS, bool DHALF, int KIND>
__global__ void __launch_bounds__(1024) row_pass_kernel(PassArgs a, int tpr) {
    static_assert(ITEMS % 4 == 0, "ITEMS must be a multiple of 4");
    __shared__ Aff s_fwd[32];
    __shared__ Aff s_bwd[32];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int rloc = tid / tpr;
    const int t = tid - rloc * tpr;
    const int wpr = tpr >> 5;           // warps per row
    const int wrow = t >> 5;            // warp index within the row
    const int wbase = warp - wrow;      // first warp of this row
    const int rpb = blockDim.x / tpr;
    const int row = blockIdx.x * rpb + rloc;
    const bool row_ok = row < a.H;
    const int e0 = t * ITEMS;
    const long long P = a.pitch;
    const bool in_row = row_ok && e0 < P;

    float x[ITEMS], w[ITEMS];
    if (in_row) {
        const long long base = (long long)row * P + e0;
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            if constexpr (KIND == PASS_SUPPORT) {
                x[4 * q] = x[4 * q + 1] = x[4 * q + 2] = x[4 * q + 3] = 1.f;
            } else {
                float4 v = *reinterpret_cast<const float4*>(a.src + base + 4 * q);
                x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
            }
            load4_d<DHALF>(a.d, base + 4 * q, &w[4 * q]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) x[j] = w[j] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int e = e0 + j;
        const bool ok = row_ok && e < a.W;
        x[j] = ok ? x[j] : 0.f;
        w[j] = (ok && e > 0) ? exp2f(a.k2 * w[j]) : 0.f;
    }
    // weight between the last owned element and the next one (anti-causal needs w[e+1])
    float wn = __shfl_down_sync(kFull, w[0], 1);
    if (lane == 31) {
        const int en = e0 + ITEMS;
        wn = (row_ok && en < a.W) ? exp2f(a.k2 * load1_d<DHALF>(a.d, (long long)row * P + en)) : 0.f;
    }

    // ---- causal sweep
    Aff m{1.f, 0.f};
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if constexpr (KIND == PASS_SUPPORT) m.B = fmaf(w[j], m.B, x[j]);
        else m.B = fmaf(w[j], m.B - x[j], x[j]);
        m.A *= w[j];
    }
    Aff inc = warp_scan_up(m, lane);
    if (lane == 31) s_fwd[warp] = inc;
    float eA = __shfl_up_sync(kFull, inc.A, 1), eB = __shfl_up_sync(kFull, inc.B, 1);
    if (lane == 0) { eA = 1.f; eB = 0.f; }
    // ---- anti-causal local maps need the causal results first; for SUPPORT the
    // anti-causal sweep runs on x itself, so its reduction can start now.
    float Pv[KIND == PASS_SUPPORT ? ITEMS : 1];
    __syncthreads();
    float carry = 0.f;
    for (int q = 0; q < wrow; ++q) carry = fmaf(s_fwd[wbase + q].A, carry, s_fwd[wbase + q].B);
    carry = fmaf(eA, carry, eB);
    {
        float J = carry;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if constexpr (KIND == PASS_SUPPORT) {
                J = fmaf(w[j], J, x[j]);
                Pv[j] = J;
            } else {
                J = fmaf(w[j], J - x[j], x[j]);
                x[j] = J;
            }
        }
    }

    // ---- anti-causal sweep (right to left), w'_j = w_{j+1}
    m = Aff{1.f, 0.f};
#pragma unroll
    for (int j = ITEMS - 1; j >= 0; --j) {
        const float wp = (j == ITEMS - 1) ? wn : w[j + 1];
        if constexpr (KIND == PASS_SUPPORT) m.B = fmaf(wp, m.B, x[j]);
        else m.B = fmaf(wp, m.B - x[j], x[j]);
        m.A *= wp;
    }
    inc = warp_scan_down(m, lane);
    if (lane == 0) s_bwd[warp] = inc;
    eA = __shfl_down_sync(kFull, inc.A, 1);
    eB = __shfl_down_sync(kFull, inc.B, 1);
    if (lane == 31) { eA = 1.f; eB = 0.f; }
    __syncthreads();
    carry = 0.f;
    for (int q = wpr - 1; q > wrow; --q) carry = fmaf(s_bwd[wbase + q].A, carry, s_bwd[wbase + q].B);
    carry = fmaf(eA, carry, eB);
    {
        float K = carry;
#pragma unroll
        for (int j = ITEMS - 1; j >= 0; --j) {
            const float wp = (j == ITEMS - 1) ? wn : w[j + 1];
            if constexpr (KIND == PASS_SUPPORT) {
                K = fmaf(wp, K, x[j]);
                // P + Q - x; padding elements stay 0
                const bool ok = row_ok && (e0 + j) < a.W;
                Pv[j] = ok ? Pv[j] + K - x[j] : 0.f;
            } else {
                K = fmaf(wp, K - x[j], x[j]);
                x[j] = K;
            }
        }
    }
    if (in_row) {
        const long long base = (long long)row * P + e0;
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            float4 v;
            if constexpr (KIND == PASS_SUPPORT) v = make_float4(Pv[4 * q], Pv[4 * q + 1], Pv[4 * q + 2], Pv[4 * q + 3]);
            else v = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            *reinterpret_cast<float4*>(a.dst + base + 4 * q) = v;
        }
    }
}

// ---------------------------------------------------------------- vertical pass
// Grid (ceil(W/32), cluster, 1) with cluster dims (1, cluster, 1): one cluster per strip
// of 32 columns covering all H rows.  Lane = column (coalesced 128-byte row segments),
// warp q of CTA r owns rows [(r*NW + q)*ITEMS, +ITEMS).  Carries cross warps through
// shared memory and CTAs through distributed shared memory.
// KIND: PASS_PLAIN, PASS_UPDATE (z_{k+1} from z_k, t, c and zbar) or
//       PASS_SUPPORT_CONF (unnormalised sweeps of the row support s: S = P + Q - s,
//       then chat = c * s_flat / S).
// Largest CTA a vertical-pass shape uses (bounds the registers per thread).
template <int ITEMS>
constexpr int col_max_threads() {
    return ITEMS <= 8 ? 1024 : 512;
}

template <int ITEMS, bool DHALF, int KIND>
__global__ void __launch_bounds__(col_max_threads<ITEMS>()) col_pass_kernel(PassArgs a) {
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ Aff s_wf[32][32];
    __shared__ Aff s_wb[32][32];
    __shared__ Aff s_cf[32];
    __shared__ Aff s_cb[32];
    __shared__ float s_carry_f[32];
    __shared__ float s_carry_b[32];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const int rank = (int)cluster.block_rank();
    const int CS = (int)cluster.num_blocks();
    const int col = blockIdx.x * 32 + lane;
    const bool col_ok = col < a.W;
    const int row0 = (rank * NW + warp) * ITEMS;
    const long long P = a.pitch;

    float x[ITEMS], w[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        const bool ok = col_ok && r < a.H;
        const long long idx = (long long)r * P + col;
        x[j] = ok ? a.src[idx] : 0.f;
        w[j] = ok ? load1_d<DHALF>(a.d, idx) : 0.f;
    }
    float wn;
    {
        const int rn = row0 + ITEMS;
        wn = (col_ok && rn < a.H) ? exp2f(a.k2 * load1_d<DHALF>(a.d, (long long)rn * P + col)) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        w[j] = (col_ok && r > 0 && r < a.H) ? exp2f(a.k2 * w[j]) : 0.f;
    }

    // ---- causal (top to bottom)
    Aff m{1.f, 0.f};
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if constexpr (KIND == PASS_SUPPORT_CONF) m.B = fmaf(w[j], m.B, x[j]);
        else m.B = fmaf(w[j], m.B - x[j], x[j]);
        m.A *= w[j];
    }
    s_wf[warp][lane] = m;
    __syncthreads();
    if (warp == 0) {
        Aff tot{1.f, 0.f};
        for (int q = 0; q < NW; ++q) tot = compose(tot, s_wf[q][lane]);
        s_cf[lane] = tot;
    }
    cluster.sync();
    if (warp == 0) {
        float c = 0.f;
        for (int q = 0; q < rank; ++q) {
            const Aff o = *cluster.map_shared_rank(&s_cf[lane], q);
            c = fmaf(o.A, c, o.B);
        }
        s_carry_f[lane] = c;
    }
    __syncthreads();
    float Pv[KIND == PASS_SUPPORT_CONF ? ITEMS : 1];
    {
        float J = s_carry_f[lane];
        for (int q = 0; q < warp; ++q) J = fmaf(s_wf[q][lane].A, J, s_wf[q][lane].B);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if constexpr (KIND == PASS_SUPPORT_CONF) {
                J = fmaf(w[j], J, x[j]);
                Pv[j] = J;
            } else {
                J = fmaf(w[j], J - x[j], x[j]);
                x[j] = J;
            }
        }
    }

    // ---- anti-causal (bottom to top), w'_r = w_{r+1}
    m = Aff{1.f, 0.f};
#pragma unroll
    for (int j = ITEMS - 1; j >= 0; --j) {
        const float wp = (j == ITEMS - 1) ? wn : w[j + 1];
        if constexpr (KIND == PASS_SUPPORT_CONF) m.B = fmaf(wp, m.B, x[j]);
        else m.B = fmaf(wp, m.B - x[j], x[j]);
        m.A *= wp;
    }
    s_wb[warp][lane] = m;
    __syncthreads();
    if (warp == 0) {
        Aff tot{1.f, 0.f};
        for (int q = NW - 1; q >= 0; --q) tot = compose(tot, s_wb[q][lane]);
        s_cb[lane] = tot;
    }
    cluster.sync();
    if (warp == 0) {
        float c = 0.f;
        for (int q = CS - 1; q > rank; --q) {
            const Aff o = *cluster.map_shared_rank(&s_cb[lane], q);
            c = fmaf(o.A, c, o.B);
        }
        s_carry_b[lane] = c;
    }
    __syncthreads();
    // all remote reads of this CTA are done: peers may exit once everyone arrived
    cluster.barrier_arrive();
    {
        float K = s_carry_b[lane];
        for (int q = NW - 1; q > warp; --q) K = fmaf(s_wb[q][lane].A, K, s_wb[q][lane].B);
#pragma unroll
        for (int j = ITEMS - 1; j >= 0; --j) {
            const float wp = (j == ITEMS - 1) ? wn : w[j + 1];
            if constexpr (KIND == PASS_SUPPORT_CONF) {
                K = fmaf(wp, K, x[j]);
                Pv[j] = Pv[j] + K - x[j];
            } else {
                K = fmaf(wp, K - x[j], x[j]);
                x[j] = K;
            }
        }
    }

    // ---- epilogue
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        if (!(col_ok && r < a.H)) continue;
        const long long idx = (long long)r * P + col;
        if constexpr (KIND == PASS_PLAIN) {
            a.dst[(long long)r * a.dst_pitch + col] = x[j];
        } else if constexpr (KIND == PASS_UPDATE) {
            const long long di = (long long)r * a.W + col;
            const float zb = x[j];
            const float z = a.zk[idx];
            const float t = load_any(a.t, di, a.t_dtype);
            const float c = a.c_pitched ? a.c[idx] : a.c[di];
            float zn;
            if (a.update == DTS_UPDATE_JACOBI) {
                const float den = a.lambda + c;
                zn = den != 0.f ? (a.lambda * zb + c * t) / den : z;
            } else {
                float eta = a.step;
                if (a.clamp_step && a.lambda + c > 0.f) eta = fminf(eta, 1.f / (a.lambda + c));
                zn = z - eta * (a.lambda * (z - zb) + c * (z - t));
            }
            a.zout[(long long)r * a.zout_pitch + col] = zn;
        } else {
            const float c = a.c[(long long)r * a.W + col];
            a.zout[idx] = c * a.s_flat / Pv[j];
        }
    }
    cluster.barrier_wait();
}

template <int ITEMS, bool DHALF, int KIND>
cudaError_t launch_col_t(const PassArgs& a, const ColPlan& p, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((a.W + 31) / 32), (unsigned)p.cluster, 1);
    cfg.blockDim = dim3((unsigned)(32 * p.warps), 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = (unsigned)p.cluster;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, col_pass_kernel<ITEMS, DHALF, KIND>, a);
}

template <int ITEMS, bool DHALF>
cudaError_t launch_col_k(const PassArgs& a, int kind, const ColPlan& p, cudaStream_t s) {
    switch (kind) {
        case PASS_PLAIN: return launch_col_t<ITEMS, DHALF, PASS_PLAIN>(a, p, s);
        case PASS_UPDATE: return launch_col_t<ITEMS, DHALF, PASS_UPDATE>(a, p, s);
        case PASS_SUPPORT_CONF: return launch_col_t<ITEMS, DHALF, PASS_SUPPORT_CONF>(a, p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int ITEMS, bool DHALF>
cudaError_t launch_row_k(const PassArgs& a, int kind, const RowPlan& p, cudaStream_t s) {
    const dim3 grid((unsigned)((a.H + p.rpb - 1) / p.rpb));
    const dim3 block((unsigned)(p.tpr * p.rpb));
    if (kind == PASS_SUPPORT) row_pass_kernel<ITEMS, DHALF, PASS_SUPPORT><<<grid, block, 0, s>>>(a, p.tpr);
    else row_pass_kernel<ITEMS, DHALF, PASS_PLAIN><<<grid, block, 0, s>>>(a, p.tpr);
    return cudaGetLastError();
}

template <int ITEMS, bool DHALF>
cudaError_t allow_clusters() {
    cudaError_t e = cudaSuccess;
    const int kinds[3] = {PASS_PLAIN, PASS_UPDATE, PASS_SUPPORT_CONF};
    for (int k : kinds) {
        const void* f = nullptr;
        if (k == PASS_PLAIN) f = (const void*)col_pass_kernel<ITEMS, DHALF, PASS_PLAIN>;
        if (k == PASS_UPDATE) f = (const void*)col_pass_kernel<ITEMS, DHALF, PASS_UPDATE>;
        if (k == PASS_SUPPORT_CONF) f = (const void*)col_pass_kernel<ITEMS, DHALF, PASS_SUPPORT_CONF>;
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (r != cudaSuccess) e = r;
    }
    return e;
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_col_dispatch(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s);

cudaError_t launch_distances(const DistArgs& a, cudaStream_t s) {
    const dim3 block(256);
    const dim3 grid((unsigned)((a.W + 255) / 256), (unsigned)a.H);
    const int h = prof_begin(KID_DISTANCES, (long long)a.H * a.W, a.dhalf ? kFlagDistHalf : 0, s);
    if (a.dhalf) {
        if (a.gdtype == DTS_BF16) distance_kernel<__nv_bfloat16, __half><<<grid, block, 0, s>>>(a);
        else if (a.gdtype == DTS_F16) distance_kernel<__half, __half><<<grid, block, 0, s>>>(a);
        else distance_kernel<float, __half><<<grid, block, 0, s>>>(a);
    } else {
        if (a.gdtype == DTS_BF16) distance_kernel<__nv_bfloat16, float><<<grid, block, 0, s>>>(a);
        else if (a.gdtype == DTS_F16) distance_kernel<__half, float><<<grid, block, 0, s>>>(a);
        else distance_kernel<float, float><<<grid, block, 0, s>>>(a);
    }
    const cudaError_t e = cudaGetLastError();
    prof_end(h, s);
    return e;
}

cudaError_t launch_copy_plane(const void* src, int src_dtype, long long src_pitch, float* dst, long long dst_pitch,
                              int H, int W, cudaStream_t s) {
    const dim3 block(256);
    const dim3 grid((unsigned)((W + 255) / 256), (unsigned)H);
    const int h = prof_begin(KID_COPY, (long long)H * W, 0, s);
    copy_plane_kernel<<<grid, block, 0, s>>>(src, src_dtype, src_pitch, dst, dst_pitch, H, W);
    const cudaError_t e = cudaGetLastError();
    prof_end(h, s);
    return e;
}

cudaError_t launch_row_pass(const PassArgs& a, int dist_half, int kind, const RowPlan& p, cudaStream_t s) {
    const int h = prof_begin(kind == PASS_SUPPORT ? KID_ROW_SUPPORT : KID_ROW_PLAIN, (long long)a.H * a.W,
                             dist_half ? kFlagDistHalf : 0, s);
    cudaError_t e = cudaErrorInvalidValue;
    if (p.items == 8) e = dist_half ? launch_row_k<8, true>(a, kind, p, s) : launch_row_k<8, false>(a, kind, p, s);
    if (p.items == 16) e = dist_half ? launch_row_k<16, true>(a, kind, p, s) : launch_row_k<16, false>(a, kind, p, s);
    prof_end(h, s);
    return e;
}

cudaError_t launch_col_pass(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s) {
    const int kid = kind == PASS_UPDATE ? KID_COL_UPDATE : kind == PASS_SUPPORT_CONF ? KID_COL_SUPPORT : KID_COL_PLAIN;
    const int flags = (dist_half ? kFlagDistHalf : 0) | (kind == PASS_UPDATE && a.t_dtype != DTS_F32 ? kFlagTarget16 : 0);
    const int h = prof_begin(kid, (long long)a.H * a.W, flags, s);
    const cudaError_t e = launch_col_dispatch(a, dist_half, kind, p, s);
    prof_end(h, s);
    return e;
}

cudaError_t launch_col_dispatch(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s) {
    if (p.items == 8) return dist_half ? launch_col_k<8, true>(a, kind, p, s) : launch_col_k<8, false>(a, kind, p, s);
    if (p.items == 16) return dist_half ? launch_col_k<16, true>(a, kind, p, s) : launch_col_k<16, false>(a, kind, p, s);
    if (p.items == 32) return dist_half ? launch_col_k<32, true>(a, kind, p, s) : launch_col_k<32, false>(a, kind, p, s);
    if (p.items == 40) return dist_half ? launch_col_k<40, true>(a, kind, p, s) : launch_col_k<40, false>(a, kind, p, s);
    return cudaErrorInvalidValue;
}

// Horizontal plan: ITEMS elements per thread, one row per tpr threads (<= 1024).
bool plan_rows(int W, RowPlan* p) {
    int items;
    if (W <= 8 * 1024) items = 8;
    else if (W <= 16 * 1024) items = 16;
    else return false;
    int tpr = (W + items - 1) / items;
    tpr = (tpr + 31) / 32 * 32;
    int rpb = 256 / tpr;
    if (rpb < 1) rpb = 1;
    p->items = items;
    p->tpr = tpr;
    p->rpb = rpb;
    return true;
}

// Vertical plan: the first (items, warps) shape whose cluster holds the whole column
// with at most 8 CTAs, else at most 16 (non-portable cluster size).
bool plan_cols(int H, ColPlan* p) {
    if (H <= 256) {
        p->items = 8;
        p->warps = (H + 7) / 8;
        p->cluster = 1;
        return true;
    }
    static const int cand[][2] = {{8, 8}, {16, 8}, {16, 16}, {32, 16}, {40, 16}};
    for (int limit : {8, 16}) {
        for (const auto& c : cand) {
            const int rows = c[0] * c[1];
            const int cs = (H + rows - 1) / rows;
            if (cs <= limit) {
                p->items = c[0];
                p->warps = c[1];
                p->cluster = cs;
                return true;
            }
        }
    }
    return false;
}

cudaError_t prepare_kernels() {
    cudaError_t e = cudaSuccess, r;
    if ((r = allow_clusters<8, false>()) != cudaSuccess) e = r;
    if ((r = allow_clusters<8, true>()) != cudaSuccess) e = r;
    if ((r = allow_clusters<16, false>()) != cudaSuccess) e = r;
    if ((r = allow_clusters<16, true>()) != cudaSuccess) e = r;
    if ((r = allow_clusters<32, false>()) != cudaSuccess) e = r;
    if ((r = allow_clusters<32, true>()) != cudaSuccess) e = r;
    if ((r = allow_clusters<40, false>()) != cudaSuccess) e = r;
    if ((r = allow_clusters<40, true>()) != cudaSuccess) e = r;
    return e;
}

}  // namespace dts
