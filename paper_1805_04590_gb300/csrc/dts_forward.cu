// Forward kernels of the Domain Transform Solver for sm_103a.
//
//  distance_kernel   domain-transform distances dX, dY (§3.2, Eq. 8-9), once per solve
//  row_pass_kernel   one horizontal recursive-filter pass (causal + anti-causal, §2/§3.2)
//  col_pass_kernel   one vertical pass; the last one of an iteration also applies the
//                    data-term update of Eq. 3 (gradient step) or Eq. 4 (fixed point)
//
// A pass runs, along every line, the causal sweep J[n] = (1 - w_n) x[n] + w_n J[n-1] and then
// the anti-causal sweep K[n] = (1 - w_{n+1}) J[n] + w_{n+1} K[n+1] on its result, with
// w_n = a^(d_n) the feedback across the distance d_n between positions n-1 and n.
//
// Parallel form.  A thread owns a segment of ITEMS consecutive positions of a line in
// registers.  For the carry c entering the segment from the left and the anti-causal value k
// entering from the right, the segment satisfies
//     c_out   = A c + B                      (causal value leaving on the right)
//     k_start = al k + be c + ga             (anti-causal value at its first position)
// with A = prod w, B = causal sweep from 0, al = prod w', and
//     be = sum_n r_n (1 - w'_n) P_n,  ga = sum_n r_n (1 - w'_n) Q_n
// where P_n = prod_{m<=n} w_m, Q_n = causal sweep from 0 at n, r_n = prod_{m<n} w'_m: all of it
// accumulates in ONE forward sweep over the segment.  Adjacent groups compose associatively
// (CoupledMode::suf_compose), so a single exchange of these five numbers between the segments
// of a line -- warp shuffles, shared memory, and distributed shared memory between the CTAs of
// a cluster for columns -- gives every segment its exact carries in both directions, after
// which it replays its positions once each way.  A line is read once and written once per
// pass: 2 s_z + s_d bytes per pixel.
#include <cuda.h>  // CUtensorMap and its enums; the encoder comes from the runtime's driver entry point
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <string>
#include <mutex>
#include <tuple>

#include "dts_modes.cuh"

namespace dts {

namespace {

using namespace scan;

// ---------------------------------------------------------------- distances
// Thread = one column x and kDistRows consecutive rows; a warp covers 32 consecutive columns,
// so every guide row segment is one coalesced access and the left neighbour comes from the
// adjacent lane.
constexpr int kDistRows = 4;

template <typename GT, typename DT>
__global__ void __launch_bounds__(256) distance_kernel(DistArgs a) {
    wait_predecessor();
    const int lane = threadIdx.x & 31;
    const int x = blockIdx.x * 32 + lane;
    const int y0 = (blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kDistRows;
    const bool xok = x < a.W;
    const GT* I = static_cast<const GT*>(a.guide);
    float sx[kDistRows], sy[kDistRows];
#pragma unroll
    for (int r = 0; r < kDistRows; ++r) sx[r] = sy[r] = 0.f;
    const bool l2 = a.norm == DTS_NORM_L2;
    for (int c = 0; c < a.C; ++c) {
        const GT* Ic = I + (long long)c * a.ch_stride;
        float prev = (xok && y0 > 0 && y0 - 1 < a.H) ? to_f32<GT>(Ic[(long long)(y0 - 1) * a.row_stride + x]) : 0.f;
#pragma unroll
        for (int r = 0; r < kDistRows; ++r) {
            const int y = y0 + r;
            const bool ok = xok && y < a.H;
            const long long p = (long long)y * a.row_stride + x;
            const float v = ok ? to_f32<GT>(Ic[p]) : 0.f;
            float left = __shfl_up_sync(kFull, v, 1);
            if (lane == 0) left = (ok && x > 0) ? to_f32<GT>(Ic[p - 1]) : 0.f;
            const float dxv = v - left, dyv = v - prev;
            sx[r] += l2 ? dxv * dxv : fabsf(dxv);
            sy[r] += l2 ? dyv * dyv : fabsf(dyv);
            prev = v;
        }
    }
#pragma unroll
    for (int r = 0; r < kDistRows; ++r) {
        const int y = y0 + r;
        if (!(xok && y < a.H)) continue;
        float dx, dy;
        if (l2) {
            dx = sqrtf(fmaf(a.k * a.k, sx[r], 1.f));
            dy = sqrtf(fmaf(a.k * a.k, sy[r], 1.f));
        } else {
            dx = fmaf(a.k, sx[r], 1.f);
            dy = fmaf(a.k, sy[r], 1.f);
        }
        if (x == 0) dx = 1.f;
        if (y == 0) dy = 1.f;
        const long long q = (long long)y * a.pitch + x;
        static_cast<DT*>(a.dX)[q] = from_f32<DT>(dx);
        static_cast<DT*>(a.dY)[q] = from_f32<DT>(dy);
        if (a.dYs) static_cast<DT*>(a.dYs)[((long long)(x >> 3) * a.ys_rows + y) * 8 + (x & 7)] = from_f32<DT>(dy);
        if (a.dst) a.dst[q] = load_any(a.src, (long long)y * a.W + x, a.src_dtype);
    }
}

// Four consecutive guide values of one row (16-byte load for FP32, 8-byte for 16-bit types).
template <typename GT>
__device__ __forceinline__ void load4_guide(const GT* p, float* out) {
    if constexpr (sizeof(GT) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    } else {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        const GT* h = reinterpret_cast<const GT*>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = to_f32<GT>(h[k]);
    }
}

template <typename DT>
__device__ __forceinline__ void store4_dist(DT* p, const float* v) {
    if constexpr (sizeof(DT) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        uint2 u;
        DT* h = reinterpret_cast<DT*>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = from_f32<DT>(v[k]);
        *reinterpret_cast<uint2*>(p) = u;
    }
}

// Distances with four consecutive columns per thread (vector loads and stores), for guides whose
// rows and channels start on 4-element boundaries and W % 4 == 0.  Thread = 4 columns x
// kDistRows rows; a warp covers 128 columns.  The left neighbour of a thread's first column is
// the previous lane's last one (lane 0 loads it); the upper neighbour is the previous row held
// in registers.
template <typename GT, typename DT>
__global__ void __launch_bounds__(256) distance4_kernel(DistArgs a) {
    wait_predecessor();
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * 32 + lane) * 4;
    const int y0 = (blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kDistRows;
    const bool xok = x0 < a.W;  // W % 4 == 0: the thread's four columns are all inside or all outside
    const GT* I = static_cast<const GT*>(a.guide);
    if (a.dst && xok) {
        // the fused copy first, all rows' loads in flight at once (16-byte vectors for an FP32
        // source on 16-byte boundaries); its stores retire while the guide is read
        const bool vsrc = a.src_dtype == DTS_F32 && ((uintptr_t)a.src & 15) == 0;
        float tv[kDistRows][4];
#pragma unroll
        for (int r = 0; r < kDistRows; ++r) {
            const int y = y0 + r;
            if (y >= a.H) break;
            const long long di = (long long)y * a.W + x0;
            if (vsrc) {
                load4_f(static_cast<const float*>(a.src), di, tv[r]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) tv[r][k] = load_any(a.src, di + k, a.src_dtype);
            }
        }
#pragma unroll
        for (int r = 0; r < kDistRows; ++r) {
            const int y = y0 + r;
            if (y >= a.H) break;
            store4_f(a.dst, (long long)y * a.pitch + x0, tv[r]);
        }
    }
    float sx[kDistRows][4], sy[kDistRows][4];
#pragma unroll
    for (int r = 0; r < kDistRows; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) sx[r][k] = sy[r][k] = 0.f;
    const bool l2 = a.norm == DTS_NORM_L2;
    for (int c = 0; c < a.C; ++c) {
        const GT* Ic = I + (long long)c * a.ch_stride;
        if (xok && c + 1 < a.C) {
            // the next band's rows into L2 while this band is read (the loop waits on each band's
            // loads); measured at 16 bands: 1918 -> 1682 us, and 2252 us two bands ahead
            const GT* In = Ic + a.ch_stride + x0;
#pragma unroll
            for (int r = -1; r < kDistRows; ++r)
                if (y0 + r >= 0 && y0 + r < a.H) prefetch_l2(In + (long long)(y0 + r) * a.row_stride);
        }
        float prev[4] = {0.f, 0.f, 0.f, 0.f};
        if (xok && y0 > 0 && y0 - 1 < a.H) load4_guide<GT>(Ic + (long long)(y0 - 1) * a.row_stride + x0, prev);
#pragma unroll
        for (int r = 0; r < kDistRows; ++r) {
            const int y = y0 + r;
            const bool ok = xok && y < a.H;
            const long long p = (long long)y * a.row_stride + x0;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (ok) load4_guide<GT>(Ic + p, v);
            float left = __shfl_up_sync(kFull, v[3], 1);
            if (lane == 0) left = (ok && x0 > 0) ? to_f32<GT>(Ic[p - 1]) : 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float dxv = v[k] - (k == 0 ? left : v[k - 1]);
                const float dyv = v[k] - prev[k];
                sx[r][k] += l2 ? dxv * dxv : fabsf(dxv);
                sy[r][k] += l2 ? dyv * dyv : fabsf(dyv);
                prev[k] = v[k];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kDistRows; ++r) {
        const int y = y0 + r;
        if (!(xok && y < a.H)) continue;
        float dx[4], dy[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (l2) {
                dx[k] = sqrtf(fmaf(a.k * a.k, sx[r][k], 1.f));
                dy[k] = sqrtf(fmaf(a.k * a.k, sy[r][k], 1.f));
            } else {
                dx[k] = fmaf(a.k, sx[r][k], 1.f);
                dy[k] = fmaf(a.k, sy[r][k], 1.f);
            }
            if (y == 0) dy[k] = 1.f;
        }
        if (x0 == 0) dx[0] = 1.f;
        const long long q = (long long)y * a.pitch + x0;
        store4_dist<DT>(static_cast<DT*>(a.dX) + q, dx);
        store4_dist<DT>(static_cast<DT*>(a.dY) + q, dy);
        if (a.dYs) store4_dist<DT>(static_cast<DT*>(a.dYs) + ((long long)(x0 >> 3) * a.ys_rows + y) * 8 + (x0 & 7), dy);
    }
}

__global__ void __launch_bounds__(256) copy_plane_kernel(const void* src, int src_dtype, long long sp, float* dst,
                                                         long long dp, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    wait_predecessor();
    if (x >= W || y >= H) return;
    dst[(long long)y * dp + x] = load_any(src, (long long)y * sp + x, src_dtype);
}

// ---------------------------------------------------------------- horizontal pass
// CTA = rpb rows x tpr threads (tpr a multiple of 32, so a warp never spans two rows); thread t
// of a row owns positions [t*ITEMS, t*ITEMS + ITEMS).  The segments of a row exchange their
// aggregates through warp shuffles and one shared-memory round.
// KIND: PASS_PLAIN (CoupledMode on the plane) or PASS_SUPPORT (SupportMode on the constant 1).
// KIND PASS_UPDATE_ROW: the first pass of an iteration also applies the previous iteration's
// data-term update: it reads zbar (a.src), z_k (a.zk), t and c, writes z_{k+1} to a.zout and
// filters z_{k+1}.
// 32 positions per thread: the update pass in CTAs of up to 512 threads (rows up to 16384), the
// other passes in CTAs of up to 320 threads (rows up to 10240), two of them per SM
template <int ITEMS, int KIND>
constexpr int row_max_threads() {
    return KIND == PASS_UPDATE_ROW ? 512 : ITEMS >= 32 ? 320 : 1024;
}

// the update pass at up to 16 positions per thread is capped at 64 registers (two CTAs of 512
// threads per SM at most); 32 positions would spill
template <int ITEMS, int KIND>
constexpr int row_min_blocks() {
    return (KIND == PASS_UPDATE_ROW && ITEMS <= 16) || (KIND != PASS_UPDATE_ROW && ITEMS >= 32) ? 2 : 1;
}

template <int ITEMS, bool DHALF, int KIND, bool TWO = false>
__global__ void __launch_bounds__(row_max_threads<ITEMS, KIND>(), row_min_blocks<ITEMS, KIND>()) row_pass_kernel(PassArgs a, int tpr) {
    wait_predecessor();
    row_pass_body<ITEMS, DHALF, KIND, TWO, false>(a, tpr, blockDim.x / tpr, blockIdx.x);
}

// ---------------------------------------------------------------- vertical pass
// Lane = column (128-byte coalesced row segments); a warp owns ITEMS consecutive rows of 32
// columns.  The segments of a column are the warps of the CTAs that hold it: one shared-memory
// round inside a CTA, then one round across CTAs -- in distributed shared memory between the
// CTAs of a cluster (col_pass_kernel), or through global memory along a chain of CTAs
// (col_chain_kernel, chain_exchange).
// KIND: PASS_PLAIN (CoupledMode, store), PASS_SUPPORT_CONF (SupportMode on the row support s,
// then chat = c s_flat / S) or PASS_TRANSPOSE (TransposeMode, on zk - src when a.zk is set).  The
// data-term update is applied by the horizontal passes.
template <int KIND>
using ColMode = typename std::conditional<KIND == PASS_SUPPORT_CONF, SupportMode,
                                          typename std::conditional<KIND == PASS_TRANSPOSE, TransposeMode,
                                                                    CoupledMode>::type>::type;

// A thread's ITEMS positions of column `col` from row0 (zero outside the plane) and their
// weights w = a^d (0 outside the plane and at the column start), and wn, the weight entering
// the next segment.  The transposed pass with a minuend filters zk - src.
template <int ITEMS, bool DHALF, int KIND>
__device__ __forceinline__ void col_load(const PassArgs& a, int row0, int col, float (&x)[ITEMS], float (&w)[ITEMS],
                                         float& wn) {
    using DT = typename std::conditional<DHALF, __half, float>::type;
    const long long P = a.pitch;
    const bool col_ok = col < a.W;
    const bool full = col_ok && row0 + ITEMS <= a.H;
    {
        const float* ps = a.src + (long long)row0 * P + col;
        const DT* pd = static_cast<const DT*>(a.d) + (long long)row0 * P + col;
        if (full) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                x[j] = *ps;
                w[j] = to_f32<DT>(*pd);
                ps += P;
                pd += P;
            }
        } else {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const bool ok = col_ok && row0 + j < a.H;
                x[j] = ok ? *ps : 0.f;
                w[j] = ok ? to_f32<DT>(*pd) : 0.f;
                ps += P;
                pd += P;
            }
        }
    }
    if constexpr (KIND == PASS_TRANSPOSE) {
        if (a.zk) {  // the pass filters zk - src (the residual p - A p of conjugate gradients)
            const float* pz = a.zk + (long long)row0 * P + col;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if (col_ok && row0 + j < a.H) x[j] = *pz - x[j];
                pz += P;
            }
        }
    }
    {
        const int rn = row0 + ITEMS;
        wn = (col_ok && rn < a.H) ? ex2(a.k2 * load1_d<DHALF>(a.d, (long long)rn * P + col)) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) w[j] = ex2(a.k2 * w[j]);
    if (!full) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j)
            if (!(col_ok && row0 + j < a.H)) w[j] = 0.f;
    }
    if (row0 == 0) w[0] = 0.f;  // the column starts here
}

// The pass result x of a thread's positions: stored (plain, transposed), or the support-weighted
// confidence into zout.
template <int ITEMS, int KIND>
__device__ __forceinline__ void col_store(const PassArgs& a, int row0, int col, const float (&x)[ITEMS]) {
    const bool col_ok = col < a.W;
    if constexpr (KIND == PASS_PLAIN || KIND == PASS_TRANSPOSE) {
        float* pdst = a.dst + (long long)row0 * a.dst_pitch + col;
        if (col_ok && row0 + ITEMS <= a.H) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                *pdst = x[j];
                pdst += a.dst_pitch;
            }
        } else {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if (col_ok && row0 + j < a.H) *pdst = x[j];
                pdst += a.dst_pitch;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int r = row0 + j;
            if (!(col_ok && r < a.H)) continue;
            a.zout[(long long)r * a.pitch + col] = a.c[(long long)r * a.W + col] * a.s_flat / x[j];
        }
    }
}

// Grid (ceil(W/32), cluster) with cluster dims (1, cluster, 1): one cluster per strip of 32
// columns covering all H rows; warp q of CTA r owns rows [(r*NW + q)*ITEMS, +ITEMS).
template <int ITEMS>
constexpr int col_max_threads() {
    return ITEMS <= 8 ? 1024 : 512;
}
// resident CTAs of the largest shape the register budget must allow
template <int ITEMS, int KIND>
constexpr int col_min_blocks() {
    return ITEMS == 16 ? 2 : 1;
}

template <int ITEMS, bool DHALF, int KIND>
__global__ void __launch_bounds__(col_max_threads<ITEMS>(), col_min_blocks<ITEMS, KIND>()) col_pass_kernel(PassArgs a) {
    using M = ColMode<KIND>;
    __shared__ ColShared<M, 32> sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const int rank = (int)cg::this_cluster().block_rank();
    const int col = blockIdx.x * 32 + lane;
    const int row0 = (rank * NW + warp) * ITEMS;

    wait_predecessor();
    float x[ITEMS], w[ITEMS], wn;
    col_load<ITEMS, DHALF, KIND>(a, row0, col, x, w, wn);
    typename M::Pre own_pre, pre;
    typename M::Suf own_suf, suf;
    M::local(x, w, wn, own_pre, own_suf);
    col_exchange<M, 32>(own_pre, own_suf, lane, warp, NW, sh, pre, suf);
    release_successor();
    M::apply(x, w, wn, own_pre, pre.B, suf);
    col_store<ITEMS, KIND>(a, row0, col, x);
    cluster_exit();
}

// Chained vertical pass (columns of any height up to the chain's limit): one CTA of NW warps per
// chunk of NW x ITEMS rows of a 32-column strip, the chunks of a strip linked through global
// memory (chain_exchange); the CTA's strip and chunk come from its ticket.
template <int ITEMS, int NW>
constexpr int chain_min_blocks() {
    return ITEMS * NW <= 128 ? 4 : 2;
}

template <int ITEMS, int NW, bool DHALF, int KIND>
__global__ void __launch_bounds__(32 * NW, chain_min_blocks<ITEMS, NW>()) col_chain_kernel(PassArgs a, ChainArgs c) {
    using M = ColMode<KIND>;
    __shared__ ChainShared<M, NW> sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    wait_predecessor();
    const int ticket = chain_ticket(c);
    const int strip = ticket / c.J;
    const int chunk = ticket - strip * c.J;
    const int col = strip * 32 + lane;
    const int row0 = (chunk * NW + warp) * ITEMS;
    float x[ITEMS], w[ITEMS], wn;
    col_load<ITEMS, DHALF, KIND>(a, row0, col, x, w, wn);
    typename M::Pre own_pre, pre;
    typename M::Suf own_suf, suf;
    M::local(x, w, wn, own_pre, own_suf);
    chain_exchange<M, NW>(own_pre, own_suf, lane, warp, NW, sh, c, ticket, pre, suf);
    release_successor();
    M::apply(x, w, wn, own_pre, pre.B, suf);
    col_store<ITEMS, KIND>(a, row0, col, x);
}

// ---------------------------------------------------------------- tall columns: persistent clusters fed by TMA
// Columns over the strip kernel's height.  One cluster of CS CTAs holds a 32-column strip, CTA r
// the rows [r R, r R + R), R = kTallWarps x ITEMS (lane = column, warp q rows [q ITEMS, + ITEMS)
// of the CTA's tile); the grid is persistent (as many clusters as fit at once, each looping over
// strips s, s + gridDim.x, ...).  A CTA's tile of the pass input and of the distances arrives by
// 2-D TMA (boxes of 32 columns x kTallBox rows) into one shared-memory stage; as soon as the CTA
// holds the tile in registers it starts the next strip's loads into the stage, so they stream in
// while the strip is exchanged (shared memory in the CTA, distributed shared memory across the
// cluster), replayed and stored (128-byte rows straight from registers).  Waits on the stage's
// barrier are bounded: one that gives up records DTS_ERR_TIMEOUT, after which the CTA issues no
// more loads and waits no more (its results are invalid, the status says so; every cluster
// barrier is still passed), and before it exits it waits, bounded, for the load it gave up on.
// skip (fault injection): CTA 0 of cluster 0 leaves out its first tile load.
constexpr int kTallBox = 128;
constexpr int kTallWarps = 16;

template <int ITEMS, bool DHALF>
__host__ __device__ constexpr size_t tall_stage_bytes() {
    return (size_t)kTallWarps * ITEMS * 32 * (4 + (DHALF ? 2 : 4));
}
template <int ITEMS>
constexpr int tall_min_blocks() {
    return ITEMS <= 16 ? 2 : 1;
}

// Paired halves (pp.paired): a column of up to 32 tiles held by two clusters of CS CTAs, the
// top half (cluster 2 u) and the bottom half (cluster 2 u + 1) of the strips of unit u, which
// process the same strips in the same order.  After its cluster's exchange, the top half's last
// CTA publishes the half's causal map and the bottom half's first CTA the half's anti-causal
// composition to global slots (alternating by strip parity) under a flag stamped with the
// launch's base and the strip's round; every CTA of each half waits (bounded) for the other
// half's stamp and composes.  A half writes a slot for round r + 2 only after it has seen the
// other half's stamp for round r + 1, which that half publishes after every CTA of it passed its
// cluster barrier of round r + 1, after its reads of round r.  Both clusters of a unit are
// resident together: the grid holds only as many clusters as fit at once.
struct TallPair {
    unsigned* flags;   // per unit and parity: [top published, bottom published]
    float* slots;      // per unit and parity: causal map (2 x 32 floats), composition (5 x 32)
    unsigned base;     // this launch's stamp base (round r stamps base + r + 1)
    int paired;
};

template <int ITEMS, bool DHALF, int KIND>
__global__ void __launch_bounds__(32 * kTallWarps, tall_min_blocks<ITEMS>())
    col_tall_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_d, PassArgs a,
                    int nstrips, long long timeout, int skip, TallPair pp) {
    using M = ColMode<KIND>;
    using DT = typename std::conditional<DHALF, __half, float>::type;
    constexpr int R = kTallWarps * ITEMS;
    constexpr int kBoxes = R / kTallBox;
    static_assert(R % kTallBox == 0, "whole boxes per tile");
    constexpr uint32_t kTx = (uint32_t)tall_stage_bytes<ITEMS, DHALF>();
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ ColShared<M, kTallWarps> sh;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_failed;  // 0, or 1 + the parity of the phase a wait gave up on
    __shared__ int s_pair_failed;  // a wait for the other half gave up: no more such waits
    cg::cluster_group cluster = cg::this_cluster();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int rank = (int)cluster.block_rank();
    const int CS = (int)cluster.num_blocks();
    const int half = pp.paired ? (int)(blockIdx.x & 1) : 0;
    const int unit = pp.paired ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int units = pp.paired ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int tile_row = (half * CS + rank) * R;
    const int row0 = tile_row + warp * ITEMS;
    const long long P = a.pitch;
    float* sx = reinterpret_cast<float*>(dsm);
    const DT* sd = reinterpret_cast<const DT*>(dsm + (size_t)R * 32 * 4);

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
        s_failed = 0;
        s_pair_failed = 0;
    }
    __syncthreads();
    auto issue_d = [&](int strip) {
#pragma unroll
        for (int b = 0; b < kBoxes; ++b)
            tma_load_2d((void*)(sd + (size_t)b * kTallBox * 32), &tm_d, strip * 32, tile_row + b * kTallBox, &bar);
    };
    auto issue_x = [&](int strip) {
#pragma unroll
        for (int b = 0; b < kBoxes; ++b)
            tma_load_2d(sx + (size_t)b * kTallBox * 32, &tm_x, strip * 32, tile_row + b * kTallBox, &bar);
    };
    auto issue = [&](int strip) {
        mbar_arrive_expect_tx(&bar, kTx);
        issue_x(strip);
        issue_d(strip);
    };
    // the first tile's distances before the wait for the previous kernel (they were written at
    // the start of the solve, before the horizontal pass that precedes every vertical pass), its
    // positions after it
    const bool first = threadIdx.x == 0 && unit < nstrips && !(skip && blockIdx.x == 0 && rank == 0);
    if (first) {
        mbar_arrive_expect_tx(&bar, kTx);
        issue_d(unit);
    }
    wait_predecessor();
    if (first) issue_x(unit);
    int it = 0;
    for (int strip = unit; strip < nstrips; strip += units, ++it) {
        const int next = strip + units;
        const int col = strip * 32 + lane;
        const bool col_ok = col < a.W;
        // the distance entering the next tile: a plain load, in flight while the stage lands
        const int rn = row0 + ITEMS;
        float dnext = 0.f;
        if (warp + 1 == kTallWarps && col_ok && rn < a.H) dnext = load1_d<DHALF>(a.d, (long long)rn * P + col);
        if (!s_failed && !mbar_wait_bounded(&bar, (uint32_t)(it & 1), timeout)) {
            record_status(a.status, DTS_ERR_TIMEOUT);
            s_failed = 1 + (it & 1);
        }
        float x[ITEMS], w[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            x[j] = sx[(warp * ITEMS + j) * 32 + lane];
            w[j] = to_f32<DT>(sd[(warp * ITEMS + j) * 32 + lane]);
        }
        if (warp + 1 < kTallWarps) dnext = to_f32<DT>(sd[((warp + 1) * ITEMS) * 32 + lane]);
        // the reads above come before the next strip's TMA writes into the stage
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && next < nstrips && !s_failed) issue(next);
        const float wn = (col_ok && rn < a.H) ? ex2(a.k2 * dnext) : 0.f;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int r = row0 + j;
            const bool ok = col_ok && r < a.H;
            w[j] = (ok && r > 0) ? ex2(a.k2 * w[j]) : 0.f;
            if (!ok) x[j] = 0.f;
        }
        if constexpr (KIND == PASS_TRANSPOSE) {
            if (a.zk && col_ok) {  // the pass filters zk - src
#pragma unroll
                for (int j = 0; j < ITEMS; ++j)
                    if (row0 + j < a.H) x[j] = a.zk[(long long)(row0 + j) * P + col] - x[j];
            }
        }
        typename M::Pre own_pre, pre;
        typename M::Suf own_suf, suf;
        M::local(x, w, wn, own_pre, own_suf);
        col_exchange_iter<M, kTallWarps>(own_pre, own_suf, lane, warp, kTallWarps, sh, it == 0, pre, suf);
        if (pp.paired) {
            const int par = it & 1;
            const unsigned stamp = pp.base + (unsigned)it + 1u;
            float* slot = pp.slots + ((size_t)unit * 2 + par) * 32 * 7;
            unsigned* flag = pp.flags + ((size_t)unit * 2 + par) * 2;
            if (half == 0 && rank == CS - 1 && warp == kTallWarps - 1) {
                // the top half's causal map: everything above this last segment, then the segment
                const typename M::Pre tp = M::pre_compose(pre, own_pre);
                const float* v = reinterpret_cast<const float*>(&tp);
#pragma unroll
                for (int k = 0; k < (int)(sizeof(tp) / 4); ++k) __stcg(slot + k * 32 + lane, v[k]);
                __syncwarp();
                if (lane == 0) {
                    __threadfence();
                    st_release_u32(&flag[0], stamp);
                }
            }
            if (half == 1 && rank == 0 && warp == 0) {
                // the bottom half's composition: this first segment, then everything below it
                const typename M::Suf ts = M::suf_compose(own_suf, suf);
                const float* v = reinterpret_cast<const float*>(&ts);
#pragma unroll
                for (int k = 0; k < (int)(sizeof(ts) / 4); ++k) __stcg(slot + 64 + k * 32 + lane, v[k]);
                __syncwarp();
                if (lane == 0) {
                    __threadfence();
                    st_release_u32(&flag[1], stamp);
                }
            }
            if (threadIdx.x == 0 && !s_pair_failed && ld_acquire_u32(&flag[1 - half]) != stamp) {
                const long long t0 = clock64();
                while (ld_acquire_u32(&flag[1 - half]) != stamp) {
                    if (clock64() - t0 > timeout) {
                        record_status(a.status, DTS_ERR_TIMEOUT);
                        s_pair_failed = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __syncthreads();
            if (half == 0) {
                typename M::Suf below;
                float* v = reinterpret_cast<float*>(&below);
#pragma unroll
                for (int k = 0; k < (int)(sizeof(below) / 4); ++k) v[k] = __ldcg(slot + 64 + k * 32 + lane);
                suf = M::suf_compose(suf, below);
            } else {
                typename M::Pre above;
                float* v = reinterpret_cast<float*>(&above);
#pragma unroll
                for (int k = 0; k < (int)(sizeof(above) / 4); ++k) v[k] = __ldcg(slot + k * 32 + lane);
                pre = M::pre_compose(above, pre);
            }
        }
        if (next >= nstrips) release_successor();
        M::apply(x, w, wn, own_pre, pre.B, suf);
        col_store<ITEMS, KIND>(a, row0, col, x);
    }
    if (CS > 1 && it > 0) cluster_exit();
    // the load a wait gave up on lands before the CTA's shared memory goes to another CTA
    if (threadIdx.x == 0 && s_failed) mbar_wait_bounded(&bar, (uint32_t)(s_failed - 1), timeout);
}

// Strip kernel with plain loads (planes that tensor maps cannot describe): one CTA per strip.
template <int ITEMS, bool DHALF>
__global__ void __launch_bounds__(32 * kStripWarps) col_strip_kernel(PassArgs a) {
    wait_predecessor();
    strip_pass_body<ITEMS, DHALF, false>(a, blockIdx.x);
}

// Strip kernel fed by TMA, persistent over strips.  Warp q owns the slab of rows
// [4 q ITEMS, 4 (q + 1) ITEMS) of every strip the CTA processes: one lane loads the slab's
// positions (8 x 4 ITEMS box) and distances (one row more: the weight entering the next slab)
// into the warp's input region, completing on the warp's mbarrier (bounded waits).  As soon as
// the warp holds a strip in registers it starts the loads of its next strip into the same
// region, so they overlap the exchange and the replay.  The result goes out through a second
// region and one TMA store per warp and strip.  ITEMS is odd, so the four segments of a warp
// start on rows of different residue mod 4 (mod 8 for FP16 distances) and the column-wise
// shared-memory accesses are free of bank conflicts.
template <int ITEMS, bool DHALF>
__host__ __device__ constexpr int strip_x_bytes() {
    return 4 * ITEMS * kStripCols * 4;  // a multiple of 128 for odd ITEMS = 9, 17 (1152, 2176)
}
template <int ITEMS, bool DHALF>
__host__ __device__ constexpr int strip_d_bytes() {
    return ((4 * ITEMS + 1) * kStripCols * (DHALF ? 2 : 4) + 127) / 128 * 128;
}
// input positions, input distances, output
template <int ITEMS, bool DHALF>
__host__ __device__ constexpr int strip_slab_bytes() {
    return 2 * strip_x_bytes<ITEMS, DHALF>() + strip_d_bytes<ITEMS, DHALF>();
}

// TR: the transposed pass (TransposeMode), with the optional minuend a.zk (zk - src is filtered).
// Waits on a warp's slab barrier are bounded (timeout cycles).  A wait that gives up records
// DTS_ERR_TIMEOUT; that warp issues no further loads into its region (the late copy may still
// land there), the CTA finishes the strip at hand with what it holds (the results are invalid,
// the status says so) and leaves the strip loop, after one more bounded wait for every load of
// its own still in flight.  skip (fault injection): warp 0 of CTA 0 leaves out its first load.
template <int ITEMS, bool DHALF, bool TR = false>
__global__ void __launch_bounds__(32 * kStripWarps) col_strip_tma_kernel(const __grid_constant__ CUtensorMap tm_x,
                                                                          const __grid_constant__ CUtensorMap tm_d,
                                                                          const __grid_constant__ CUtensorMap tm_o,
                                                                          PassArgs a, int nstrips, long long timeout,
                                                                          int skip) {
    static_assert(ITEMS % 2 == 1, "odd segment length (bank-conflict-free column accesses)");
    static_assert(strip_x_bytes<ITEMS, DHALF>() % 128 == 0, "slab alignment");
    using M = typename std::conditional<TR, TransposeMode, CoupledMode>::type;
    using DT = typename std::conditional<DHALF, __half, float>::type;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ StripShared<M> sh;
    __shared__ __align__(8) uint64_t bar[kStripWarps];
    __shared__ int s_failed[kStripWarps];  // a wait of this warp gave up
    // a wait of the CTA gave up in an iteration of this parity: the CTA leaves the strip loop (a
    // slot per parity, so that a failure in the next iteration cannot change what a slower warp
    // reads for this one)
    __shared__ int s_abort[2];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const int cl = lane & (kStripCols - 1);
    const int sw = lane / kStripCols;
    const int slab_row = warp * 4 * ITEMS;
    const int row0 = slab_row + sw * ITEMS;
    unsigned char* slab = dsm + (size_t)warp * strip_slab_bytes<ITEMS, DHALF>();
    float* sx = reinterpret_cast<float*>(slab);
    const DT* sd = reinterpret_cast<const DT*>(slab + strip_x_bytes<ITEMS, DHALF>());
    float* so = reinterpret_cast<float*>(slab + strip_x_bytes<ITEMS, DHALF>() + strip_d_bytes<ITEMS, DHALF>());
    constexpr uint32_t kTx = 4 * ITEMS * kStripCols * 4 + (4 * ITEMS + 1) * kStripCols * (int)sizeof(DT);

    if (lane == 0) {
        mbar_init(&bar[warp], 1);
        mbar_init_fence();
        s_failed[warp] = 0;
    }
    if (threadIdx.x < 2) s_abort[threadIdx.x] = 0;
    __syncthreads();
    // the slab's distances: one contiguous bulk copy from the strip-tiled plane when there is one,
    // else a TMA box (full boxes count, the parts outside the plane included: they read as zero)
    constexpr uint32_t kDBytes = (4 * ITEMS + 1) * kStripCols * (int)sizeof(DT);
    const DT* dtile = static_cast<const DT*>(a.d_tiled);
    auto load_d = [&](int strip) {
        if (dtile)
            bulk_load_1d((void*)sd, dtile + ((long long)strip * a.d_tiled_rows + slab_row) * kStripCols, kDBytes,
                         &bar[warp]);
        else
            tma_load_2d((void*)sd, &tm_d, strip * kStripCols, slab_row, &bar[warp]);
    };
    auto load_slab = [&](int strip) {
        mbar_arrive_expect_tx(&bar[warp], kTx);
        tma_load_2d(sx, &tm_x, strip * kStripCols, slab_row, &bar[warp]);
        load_d(strip);
    };
    // The distances were written at the start of the solve, before the horizontal pass that
    // precedes every vertical pass (that pass waited for them before it let this launch start):
    // the first slab's distances are copied before the wait for the previous kernel, its
    // positions after it.
    const bool first = lane == 0 && (int)blockIdx.x < nstrips && !(skip && blockIdx.x == 0 && warp == 0);
    if (first) {
        mbar_arrive_expect_tx(&bar[warp], kTx);
        load_d(blockIdx.x);
    }
    wait_predecessor();
    if (first) tma_load_2d(sx, &tm_x, blockIdx.x * kStripCols, slab_row, &bar[warp]);
    int it = 0;
    for (int strip = blockIdx.x; strip < nstrips; strip += gridDim.x, ++it) {
        const int next = strip + gridDim.x;
        const int col = strip * kStripCols + cl;
        const bool col_ok = col < a.W;
        const int failed = !mbar_wait_bounded(&bar[warp], (uint32_t)(it & 1), timeout);
        if (failed) {
            record_status(a.status, DTS_ERR_TIMEOUT);
            s_failed[warp] = 1;
            s_abort[it & 1] = 1;
        }
        float x[ITEMS], w[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            x[j] = sx[(sw * ITEMS + j) * kStripCols + cl];
            w[j] = to_f32<DT>(sd[(sw * ITEMS + j) * kStripCols + cl]);
        }
        const float dn = to_f32<DT>(sd[((sw + 1) * ITEMS) * kStripCols + cl]);
        if constexpr (TR) {
            if (a.zk && col_ok) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j)
                    if (row0 + j < a.H) x[j] = a.zk[(long long)(row0 + j) * a.pitch + col] - x[j];
            }
        }
        // the reads above come before the next strip's TMA writes into the same region
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0 && next < nstrips && !s_failed[warp]) load_slab(next);
        const float wn = (col_ok && row0 + ITEMS < a.H) ? ex2(a.k2 * dn) : 0.f;
        const bool full = col_ok && row0 + ITEMS <= a.H;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) w[j] = ex2(a.k2 * w[j]);
        if (!full) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (!(col_ok && row0 + j < a.H)) w[j] = 0.f;  // positions outside the plane read as 0
        }
        if (row0 == 0) w[0] = 0.f;

        typename M::Pre own_pre, pre;
        typename M::Suf own_suf, suf;
        M::local(x, w, wn, own_pre, own_suf);
        strip_exchange<M>(own_pre, own_suf, lane, warp, NW, cl, sw, sh, pre, suf);
        const bool abort = s_abort[it & 1] != 0;  // CTA-uniform (set before the exchange's barriers)
        if (next >= nstrips) release_successor();
        M::apply(x, w, wn, own_pre, pre.B, suf);

        // the previous strip's store must have read the output region before it is rewritten
        if (lane == 0) bulk_wait_read();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) so[(sw * ITEMS + j) * kStripCols + cl] = x[j];
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            tma_store_2d(&tm_o, strip * kStripCols, slab_row, so);
            bulk_commit();
        }
        if (abort) {
            // a load still in flight (the one a wait gave up on, or the next strip's) must land
            // before the CTA's shared memory goes to another CTA
            if (lane == 0) {
                if (s_failed[warp]) mbar_wait_bounded(&bar[warp], (uint32_t)(it & 1), timeout);
                else if (next < nstrips) mbar_wait_bounded(&bar[warp], (uint32_t)((it + 1) & 1), timeout);
            }
            break;
        }
    }
    if (lane == 0) bulk_wait_read();
}

template <int ITEMS, bool DHALF, int KIND>
cudaError_t launch_col_t(const PassArgs& a, const ColPlan& p, cudaStream_t s) {
    return launch_ex(col_pass_kernel<ITEMS, DHALF, KIND>, dim3((unsigned)((a.W + 31) / 32), (unsigned)p.cluster, 1),
                     dim3((unsigned)(32 * p.warps), 1, 1), p.cluster, s, a);
}

template <int ITEMS, bool DHALF>
cudaError_t launch_col_k(const PassArgs& a, int kind, const ColPlan& p, cudaStream_t s) {
    switch (kind) {
        case PASS_PLAIN: return launch_col_t<ITEMS, DHALF, PASS_PLAIN>(a, p, s);
        case PASS_SUPPORT_CONF: return launch_col_t<ITEMS, DHALF, PASS_SUPPORT_CONF>(a, p, s);
        case PASS_TRANSPOSE: return launch_col_t<ITEMS, DHALF, PASS_TRANSPOSE>(a, p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int ITEMS, bool DHALF>
cudaError_t launch_row_k(const PassArgs& a, int kind, const RowPlan& p, cudaStream_t s) {
    const dim3 grid((unsigned)((a.H + p.rpb - 1) / p.rpb));
    const dim3 block((unsigned)(p.tpr * p.rpb));
    if (kind == PASS_SUPPORT) return launch_ex(row_pass_kernel<ITEMS, DHALF, PASS_SUPPORT>, grid, block, 0, s, a, p.tpr);
    if (kind == PASS_TRANSPOSE) return launch_ex(row_pass_kernel<ITEMS, DHALF, PASS_TRANSPOSE>, grid, block, 0, s, a, p.tpr);
    // plain and update passes: two one-direction exchanges (measured faster on the stereo and
    // depth workloads than one exchange of the coupled five numbers)
    if (kind == PASS_UPDATE_ROW)
        return launch_ex(row_pass_kernel<ITEMS, DHALF, PASS_UPDATE_ROW, true>, grid, block, 0, s, a, p.tpr);
    return launch_ex(row_pass_kernel<ITEMS, DHALF, PASS_PLAIN, true>, grid, block, 0, s, a, p.tpr);
}

template <int ITEMS, bool DHALF>
cudaError_t allow_clusters() {
    cudaError_t e = cudaSuccess;
    const void* fs[3] = {(const void*)col_pass_kernel<ITEMS, DHALF, PASS_PLAIN>,
                         (const void*)col_pass_kernel<ITEMS, DHALF, PASS_SUPPORT_CONF>,
                         (const void*)col_pass_kernel<ITEMS, DHALF, PASS_TRANSPOSE>};
    for (const void* f : fs) {
        const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (r != cudaSuccess) e = r;
    }
    return e;
}


// ---------------------------------------------------------------- host: TMA descriptors, persistent grids
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Boxes of box_cols x box_rows elements of an H x W plane with row pitch `pitch` elements; false
// when the plane breaks the tensor-map rules (16-byte aligned base and pitch) or encoding fails.
bool make_box_map(CUtensorMap* m, const void* base, bool half, int W, int H, long long pitch, int box_cols,
                  int box_rows) {
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn) return false;
    const int es = half ? 2 : 4;
    if ((uintptr_t)base % 16 != 0 || (pitch * es) % 16 != 0 || (box_cols * es) % 16 != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * es};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t elem[2] = {1, 1};
    return fn(m, half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base),
              dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tiles of 32 columns x box_rows rows of an H x W plane with row pitch `pitch` elements.
bool make_tile_map(CUtensorMap* m, const void* base, bool half, int W, int H, long long pitch, int box_rows) {
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * (half ? 2 : 4)};
    const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base),
              dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// clusters of `cs` CTAs that fit at once (cached)
int max_clusters(const void* kernel, int block, int cs, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, size_t>, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(kernel, block, cs, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, (unsigned)cs, 1);
    cfg.blockDim = dim3((unsigned)block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = (unsigned)cs;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) n = 0;
    cache[key] = n;
    return n;
}

// persistent grid over `units` work items with `slots` concurrent workers: equal rounds
int balanced_grid(int units, int slots) {
    if (slots < 1) slots = 1;
    const int rounds = (units + slots - 1) / slots;
    return (units + rounds - 1) / rounds;
}


// z_out[y][x] (pitch zout_pitch) = update(z_k, zbar = src, t, c) for every pixel
// Four consecutive pixels per thread; VEC: 16-byte accesses (W % 4 == 0, aligned planes).
template <bool VEC>
__global__ void __launch_bounds__(256) update_kernel(PassArgs a) {
    wait_predecessor();
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int y = blockIdx.y;
    if (x0 >= a.W || y >= a.H) return;
    const long long idx = (long long)y * a.pitch + x0;
    const long long di = (long long)y * a.W + x0;
    float zk[4], zb[4], t[4], c[4], z[4];
    if (VEC) {
        load4_f(a.zk, idx, zk);
        load4_f(a.src, idx, zb);
        load4_f(a.c, a.c_pitched ? idx : di, c);
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] = load_any(a.t, di + k, a.t_dtype);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = x0 + k < a.W;
            zk[k] = ok ? a.zk[idx + k] : 0.f;
            zb[k] = ok ? a.src[idx + k] : 0.f;
            c[k] = ok ? (a.c_pitched ? a.c[idx + k] : a.c[di + k]) : 0.f;
            t[k] = ok ? load_any(a.t, di + k, a.t_dtype) : 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        z[k] = dts_update_value(zk[k], zb[k], t[k], c[k], a.lambda, a.step, a.update, a.clamp_step, a.eps);
    const long long o = (long long)y * a.zout_pitch + x0;
    if (VEC) {
        store4_f(a.zout, o, z);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (x0 + k < a.W) a.zout[o + k] = z[k];
    }
}

}  // namespace

bool row_update_fits(const RowPlan& p) { return p.tpr * p.rpb <= 512; }

// Plan of the horizontal pass that also applies the data-term update (CTAs of at most 512
// threads): the plain plan when it fits, else 32 positions per thread (rows up to 16384).
bool plan_rows_update(int W, const RowPlan& plain, RowPlan* p) {
    if (row_update_fits(plain)) {
        *p = plain;
        return true;
    }
    const int tpr = ((W + 31) / 32 + 31) / 32 * 32;
    if (tpr > 512) return false;
    p->items = 32;
    p->tpr = tpr;
    p->rpb = 1;
    return true;
}

cudaError_t launch_update(const PassArgs& a, cudaStream_t s) {
    const int h = prof_begin(KID_UPDATE, (long long)a.H * a.W, a.t_dtype != DTS_F32 ? kFlagTarget16 : 0, s);
    const dim3 grid((unsigned)((a.W + 1023) / 1024), (unsigned)a.H);
    auto al16 = [](const void* p) { return (uintptr_t)p % 16 == 0; };
    const bool vec = a.W % 4 == 0 && a.pitch % 4 == 0 && a.zout_pitch % 4 == 0 && al16(a.zk) && al16(a.src) &&
                     al16(a.c) && al16(a.zout);
    const cudaError_t e = vec ? launch_ex(update_kernel<true>, grid, dim3(256), 0, s, a)
                              : launch_ex(update_kernel<false>, grid, dim3(256), 0, s, a);
    prof_end(h, s);
    return e;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_col_dispatch(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s);

cudaError_t launch_distances(const DistArgs& a, cudaStream_t s) {
    const dim3 block(256);  // 8 warps x kDistRows rows
    const int h = prof_begin(KID_DISTANCES, (long long)a.H * a.W, a.dhalf ? kFlagDistHalf : 0, s);
    cudaError_t e;
    const int gsz = a.gdtype == DTS_F32 ? 4 : 2;
    const bool vec = a.W % 4 == 0 && a.row_stride % 4 == 0 && a.ch_stride % 4 == 0 &&
                     (uintptr_t)a.guide % (4 * gsz) == 0 && a.pitch % 4 == 0;
    if (vec) {
        const dim3 grid((unsigned)((a.W + 127) / 128), (unsigned)((a.H + 8 * kDistRows - 1) / (8 * kDistRows)));
        if (a.dhalf) {
            if (a.gdtype == DTS_BF16) e = launch_ex(distance4_kernel<__nv_bfloat16, __half>, grid, block, 0, s, a);
            else if (a.gdtype == DTS_F16) e = launch_ex(distance4_kernel<__half, __half>, grid, block, 0, s, a);
            else e = launch_ex(distance4_kernel<float, __half>, grid, block, 0, s, a);
        } else {
            if (a.gdtype == DTS_BF16) e = launch_ex(distance4_kernel<__nv_bfloat16, float>, grid, block, 0, s, a);
            else if (a.gdtype == DTS_F16) e = launch_ex(distance4_kernel<__half, float>, grid, block, 0, s, a);
            else e = launch_ex(distance4_kernel<float, float>, grid, block, 0, s, a);
        }
        prof_end(h, s);
        return e;
    }
    const dim3 grid((unsigned)((a.W + 31) / 32), (unsigned)((a.H + 8 * kDistRows - 1) / (8 * kDistRows)));
    if (a.dhalf) {
        if (a.gdtype == DTS_BF16) e = launch_ex(distance_kernel<__nv_bfloat16, __half>, grid, block, 0, s, a);
        else if (a.gdtype == DTS_F16) e = launch_ex(distance_kernel<__half, __half>, grid, block, 0, s, a);
        else e = launch_ex(distance_kernel<float, __half>, grid, block, 0, s, a);
    } else {
        if (a.gdtype == DTS_BF16) e = launch_ex(distance_kernel<__nv_bfloat16, float>, grid, block, 0, s, a);
        else if (a.gdtype == DTS_F16) e = launch_ex(distance_kernel<__half, float>, grid, block, 0, s, a);
        else e = launch_ex(distance_kernel<float, float>, grid, block, 0, s, a);
    }
    prof_end(h, s);
    return e;
}

cudaError_t launch_copy_plane(const void* src, int src_dtype, long long src_pitch, float* dst, long long dst_pitch,
                              int H, int W, cudaStream_t s) {
    const dim3 block(256);
    const dim3 grid((unsigned)((W + 255) / 256), (unsigned)H);
    const int h = prof_begin(KID_COPY, (long long)H * W, 0, s);
    const cudaError_t e = launch_ex(copy_plane_kernel, grid, block, 0, s, src, src_dtype, src_pitch, dst, dst_pitch, H, W);
    prof_end(h, s);
    return e;
}

cudaError_t launch_row_pass(const PassArgs& a, int dist_half, int kind, const RowPlan& p, cudaStream_t s) {
    const int flags = (dist_half ? kFlagDistHalf : 0) | (kind == PASS_UPDATE_ROW && a.t_dtype != DTS_F32 ? kFlagTarget16 : 0);
    RowPlan q = p;
    if (p.items % 2) {
        // a streaming plan: the plain and update passes on planes the bulk copies can address,
        // else the regular kernel's plan for the row length
        const bool upd = kind == PASS_UPDATE_ROW;
        if ((kind == PASS_PLAIN || upd) && row_stream_fits(a.W, p.items) &&
            row_stream_addressable(a, dist_half, upd)) {
            const int h = prof_begin(upd ? KID_ROW_STREAM_UPDATE : KID_ROW_STREAM, (long long)a.H * a.W, flags, s);
            const cudaError_t e = launch_row_stream(a, dist_half, p.items, upd, s);
            prof_end(h, s);
            return e;
        }
        RowPlan plain;
        if (!plan_rows_regular(a.W, &plain)) return cudaErrorInvalidValue;
        if (!upd) q = plain;
        else if (!plan_rows_update(a.W, plain, &q)) return cudaErrorInvalidValue;
    }
    const int h = prof_begin(kind == PASS_SUPPORT ? KID_ROW_SUPPORT : kind == PASS_UPDATE_ROW ? KID_ROW_UPDATE
                             : kind == PASS_TRANSPOSE ? KID_ROW_TRANSPOSE : KID_ROW_PLAIN,
                             (long long)a.H * a.W, flags, s);
    cudaError_t e = cudaErrorInvalidValue;
    if (q.items == 8) e = dist_half ? launch_row_k<8, true>(a, kind, q, s) : launch_row_k<8, false>(a, kind, q, s);
    if (q.items == 16) e = dist_half ? launch_row_k<16, true>(a, kind, q, s) : launch_row_k<16, false>(a, kind, q, s);
    if (q.items == 32 && q.tpr * q.rpb <= (kind == PASS_UPDATE_ROW ? 512 : 320))
        e = dist_half ? launch_row_k<32, true>(a, kind, q, s) : launch_row_k<32, false>(a, kind, q, s);
    prof_end(h, s);
    return e;
}

cudaError_t launch_col_strip(const PassArgs& a, int dist_half, const ColPlan& p, bool tr, cudaStream_t s);
cudaError_t launch_col_chain(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s);
cudaError_t launch_col_tall(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s);

// the vertical kernel a plan names: the strip kernel (cluster 0), the cluster kernel (cluster > 0
// CTAs), the chain (-1) or the persistent TMA clusters for tall columns (-2)
cudaError_t launch_col_planned(const PassArgs& a, int dist_half, int kind, const ColPlan& q, cudaStream_t s) {
    if (q.cluster == kColStrip) return launch_col_strip(a, dist_half, q, kind == PASS_TRANSPOSE, s);
    if (q.cluster == kColChain) return launch_col_chain(a, dist_half, kind, q, s);
    if (q.cluster == kColTall || q.cluster == kColTallPair) return launch_col_tall(a, dist_half, kind, q, s);
    return launch_col_dispatch(a, dist_half, kind, q, s);
}

cudaError_t launch_col_pass(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s) {
    const bool tr = kind == PASS_TRANSPOSE;
    // the strip kernel runs plain and transposed passes; the other kinds take the plan of the
    // same height that the other kernels give
    ColPlan q = p;
    if (q.cluster == kColStrip && kind != PASS_PLAIN && !tr && !plan_cols_multi(a.H, &q)) return cudaErrorInvalidValue;
    const int kid = q.cluster == kColStrip ? (tr ? KID_COL_STRIP_TRANSPOSE : KID_COL_STRIP)
                  : kind == PASS_SUPPORT_CONF ? KID_COL_SUPPORT
                  : q.cluster == kColChain ? (tr ? KID_COL_CHAIN_TRANSPOSE : KID_COL_CHAIN)
                  : q.cluster == kColTall || q.cluster == kColTallPair ? (tr ? KID_COL_TALL_TRANSPOSE : KID_COL_TALL)
                  : tr ? KID_COL_TRANSPOSE : KID_COL_PLAIN;
    const int flags = dist_half ? kFlagDistHalf : 0;
    const int h = prof_begin(kid, (long long)a.H * a.W, flags, s);
    const cudaError_t e = launch_col_planned(a, dist_half, kind, q, s);
    prof_end(h, s);
    return e;
}

// strip kernel (no cluster): rows per segment (odd: 9, or 17 above 1152 rows) and warps of a
// strip CTA, the fewest warps whose 4 NW segments cover the column (up to kStripMaxRows rows)
constexpr int kStripMaxRows = 4 * kStripWarps * 17;

void strip_shape(int H, int* items, int* warps) {
    const int it = H <= 4 * kStripWarps * 9 ? 9 : 17;
    const int segs = (H + it - 1) / it;
    *items = it;
    *warps = (segs + 3) / 4;
}

long long strip_tile_rows(int H) {
    if (H > kStripMaxRows) return 0;
    int items, warps;
    strip_shape(H, &items, &warps);
    return 4LL * warps * items + 1;  // every row a slab box reads, the extra row of the last included
}

template <int ITEMS, bool DHALF>
cudaError_t launch_col_strip_t(const PassArgs& a, int nw, bool tr, cudaStream_t s) {
    const dim3 grid((unsigned)((a.W + kStripCols - 1) / kStripCols));
    const dim3 block((unsigned)(32 * nw));
    CUtensorMap tx, td, to;
    if (make_box_map(&tx, a.src, false, a.W, a.H, a.pitch, kStripCols, 4 * ITEMS) &&
        make_box_map(&td, a.d, DHALF, a.W, a.H, a.pitch, kStripCols, 4 * ITEMS + 1) &&
        make_box_map(&to, a.dst, false, a.W, a.H, a.dst_pitch, kStripCols, 4 * ITEMS)) {
        // shared-memory limits raised in prepare_kernels
        auto kernel = tr ? col_strip_tma_kernel<ITEMS, DHALF, true> : col_strip_tma_kernel<ITEMS, DHALF, false>;
        const size_t smem = (size_t)nw * strip_slab_bytes<ITEMS, DHALF>();
        // persistent: as many CTAs as fit at once (each loops over strips), at most one per strip
        const int nstrips = (int)grid.x;
        const int per_sm = blocks_per_sm((const void*)kernel, 32 * nw, smem);
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const int g = std::min(nstrips, per_sm * sm_count());
        // fault injection (tests): on a single-round grid, the first slab load of warp 0 of CTA 0
        // is left out, so that warp's bounded wait runs out (about a millisecond)
        const bool skip = g == nstrips && take_injected(DTS_INJECT_TMA_SKIP);
        return launch_ex_smem(kernel, dim3((unsigned)g), block, 0, smem, s, tx, td, to, a, nstrips,
                              skip ? kInjectedTimeout : default_timeout_cycles(), skip ? 1 : 0);
    }
    // planes that tensor maps cannot describe (e.g. a caller's unaligned output): plain loads, or
    // the cluster kernel for the transposed pass
    if (tr) {
        ColPlan q;
        if (!plan_cols_multi(a.H, &q) || q.cluster == kColTall || q.cluster == kColTallPair) {
            // the tall kernel loads through tensor maps too: the cluster kernel, or the chain
            if (!plan_cols_cluster(a.H, &q) && !chain_plan(a.H, &q)) return cudaErrorInvalidValue;
        }
        return launch_col_planned(a, DHALF, PASS_TRANSPOSE, q, s);
    }
    return launch_ex(col_strip_kernel<ITEMS, DHALF>, grid, block, 0, s, a);
}

cudaError_t launch_col_strip(const PassArgs& a, int dist_half, const ColPlan& p, bool tr, cudaStream_t s) {
    if (p.warps < 1 || p.warps > kStripWarps || (long long)4 * p.warps * p.items < a.H) return cudaErrorInvalidValue;
    if (p.items == 9)
        return dist_half ? launch_col_strip_t<9, true>(a, p.warps, tr, s) : launch_col_strip_t<9, false>(a, p.warps, tr, s);
    if (p.items == 17)
        return dist_half ? launch_col_strip_t<17, true>(a, p.warps, tr, s) : launch_col_strip_t<17, false>(a, p.warps, tr, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_col_dispatch(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s) {
    if (p.cluster < 1) return cudaErrorInvalidValue;
    if (p.items == 8) return dist_half ? launch_col_k<8, true>(a, kind, p, s) : launch_col_k<8, false>(a, kind, p, s);
    if (p.items == 16) return dist_half ? launch_col_k<16, true>(a, kind, p, s) : launch_col_k<16, false>(a, kind, p, s);
    if (p.items == 32) return dist_half ? launch_col_k<32, true>(a, kind, p, s) : launch_col_k<32, false>(a, kind, p, s);
    if (p.items == 40) return dist_half ? launch_col_k<40, true>(a, kind, p, s) : launch_col_k<40, false>(a, kind, p, s);
    return cudaErrorInvalidValue;
}

// chained vertical pass: one CTA per chunk of a strip, S x J CTAs; refused (invalid
// configuration) when fewer than 2 J CTAs of the kernel fit on the GPU at once
// chunks per staging block of the strip composition: the shared memory of four resident CTAs of
// 128 rows, or two of 256 rows
template <int ITEMS, int NW>
constexpr int chain_stage_cap() {
    return ITEMS * NW <= 128 ? 40 : 80;
}

template <int ITEMS, int NW, bool DHALF, int KIND>
cudaError_t allow_chain_smem() {
    return cudaFuncSetAttribute((const void*)col_chain_kernel<ITEMS, NW, DHALF, KIND>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)chain_stage_bytes<ColMode<KIND>>(chain_stage_cap<ITEMS, NW>()));
}

template <int ITEMS, int NW, bool DHALF>
cudaError_t allow_chain_smem_all() {
    cudaError_t e = cudaSuccess, r;
    if ((r = allow_chain_smem<ITEMS, NW, DHALF, PASS_PLAIN>()) != cudaSuccess) e = r;
    if ((r = allow_chain_smem<ITEMS, NW, DHALF, PASS_SUPPORT_CONF>()) != cudaSuccess) e = r;
    if ((r = allow_chain_smem<ITEMS, NW, DHALF, PASS_TRANSPOSE>()) != cudaSuccess) e = r;
    return e;
}

template <int ITEMS, int NW, bool DHALF, int KIND>
cudaError_t launch_chain_t(const PassArgs& a, cudaStream_t s) {
    auto kernel = col_chain_kernel<ITEMS, NW, DHALF, KIND>;
    ChainArgs c = {};
    c.ctl = a.chain_ctl;
    c.agg = a.chain_agg;
    c.J = (a.H + ITEMS * NW - 1) / (ITEMS * NW);
    c.S = (a.W + 31) / 32;
    c.status = a.status;
    if (!c.ctl || !c.agg || c.J > kChainMaxChunks) return cudaErrorInvalidValue;
    c.stage = std::min(c.J, chain_stage_cap<ITEMS, NW>());
    c.epoch = next_chain_epoch();
    const size_t smem = chain_stage_bytes<ColMode<KIND>>(c.stage);
    if (blocks_per_sm((const void*)kernel, 32 * NW, smem) * sm_count() < 2 * c.J) return cudaErrorInvalidConfiguration;
    const bool skip = KIND != PASS_SUPPORT_CONF && take_injected(DTS_INJECT_CHAIN_SKIP);
    c.timeout = skip ? kInjectedTimeout : default_timeout_cycles();
    c.skip_ticket = skip && c.J > 1 ? 0 : -1;
    return launch_ex_smem(kernel, dim3((unsigned)(c.S * c.J)), dim3(32 * NW), 0, smem, s, a, c);
}

template <int ITEMS, int NW, bool DHALF>
cudaError_t launch_chain_k(const PassArgs& a, int kind, cudaStream_t s) {
    switch (kind) {
        case PASS_PLAIN: return launch_chain_t<ITEMS, NW, DHALF, PASS_PLAIN>(a, s);
        case PASS_SUPPORT_CONF: return launch_chain_t<ITEMS, NW, DHALF, PASS_SUPPORT_CONF>(a, s);
        case PASS_TRANSPOSE: return launch_chain_t<ITEMS, NW, DHALF, PASS_TRANSPOSE>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_chain(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s) {
    if (p.items == 16 && p.warps == 8)
        return dist_half ? launch_chain_k<16, 8, true>(a, kind, s) : launch_chain_k<16, 8, false>(a, kind, s);
    if (p.items == 16 && p.warps == 16)
        return dist_half ? launch_chain_k<16, 16, true>(a, kind, s) : launch_chain_k<16, 16, false>(a, kind, s);
    if (p.items == 32 && p.warps == 8)
        return dist_half ? launch_chain_k<32, 8, true>(a, kind, s) : launch_chain_k<32, 8, false>(a, kind, s);
    return cudaErrorInvalidValue;
}

// persistent TMA clusters for tall columns: ceil(H / R) CTAs per cluster (at most 16), as many
// clusters as fit at once
template <int ITEMS, bool DHALF, int KIND>
cudaError_t launch_tall_t(const PassArgs& a, bool paired, cudaStream_t s) {
    auto kernel = col_tall_kernel<ITEMS, DHALF, KIND>;
    constexpr int R = kTallWarps * ITEMS;
    const int tiles = (a.H + R - 1) / R;
    if (tiles > (paired ? 32 : 16) || (paired && tiles < 2)) return cudaErrorInvalidValue;
    if (paired && (!a.chain_ctl || !a.chain_agg)) return cudaErrorInvalidValue;
    const int cs = paired ? (tiles + 1) / 2 : tiles;  // CTAs per cluster
    const size_t smem = tall_stage_bytes<ITEMS, DHALF>();
    CUtensorMap tx, td;
    if (!make_box_map(&tx, a.src, false, a.W, a.H, a.pitch, 32, kTallBox) ||
        !make_box_map(&td, a.d, DHALF, a.W, a.H, a.pitch, 32, kTallBox))
        return cudaErrorInvalidValue;
    const int nstrips = (a.W + 31) / 32;
    const int mc = max_clusters((const void*)kernel, 32 * kTallWarps, cs, smem);
    if (mc < (paired ? 2 : 1)) return cudaErrorInvalidConfiguration;
    // units: clusters, or pairs of clusters (both of a pair resident together: the grid is at
    // most the clusters that fit at once), at most kTallPairUnits pairs
    const int units = balanced_grid(nstrips, paired ? std::min(mc / 2, kTallPairUnits) : mc);
    TallPair pp = {};
    if (paired) {
        pp.flags = a.chain_ctl + chain_ctl_words(nstrips);
        pp.slots = a.chain_agg;
        pp.base = next_chain_epoch() << 12;  // rounds per launch: at most 512 strips
        pp.paired = 1;
    }
    // fault injection (tests): on a single-round grid, CTA 0 of cluster 0 leaves out its first load
    const bool skip = units == nstrips && take_injected(DTS_INJECT_TMA_SKIP);
    return launch_ex_smem(kernel, dim3((unsigned)(paired ? 2 * units : units), (unsigned)cs, 1), dim3(32 * kTallWarps),
                          cs, smem, s, tx, td, a, nstrips, skip ? kInjectedTimeout : default_timeout_cycles(),
                          skip ? 1 : 0, pp);
}

template <int ITEMS, bool DHALF>
cudaError_t launch_tall_k(const PassArgs& a, int kind, bool paired, cudaStream_t s) {
    switch (kind) {
        case PASS_PLAIN: return launch_tall_t<ITEMS, DHALF, PASS_PLAIN>(a, paired, s);
        case PASS_SUPPORT_CONF: return launch_tall_t<ITEMS, DHALF, PASS_SUPPORT_CONF>(a, paired, s);
        case PASS_TRANSPOSE: return launch_tall_t<ITEMS, DHALF, PASS_TRANSPOSE>(a, paired, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_tall(const PassArgs& a, int dist_half, int kind, const ColPlan& p, cudaStream_t s) {
    const bool pr = p.cluster == kColTallPair;
    if (p.items == 16) return dist_half ? launch_tall_k<16, true>(a, kind, pr, s) : launch_tall_k<16, false>(a, kind, pr, s);
    if (p.items == 32) return dist_half ? launch_tall_k<32, true>(a, kind, pr, s) : launch_tall_k<32, false>(a, kind, pr, s);
    if (p.items == 40) return dist_half ? launch_tall_k<40, true>(a, kind, pr, s) : launch_tall_k<40, false>(a, kind, pr, s);
    return cudaErrorInvalidValue;
}

template <int ITEMS, bool DHALF, int KIND>
cudaError_t allow_tall_t() {
    const void* f = (const void*)col_tall_kernel<ITEMS, DHALF, KIND>;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tall_stage_bytes<ITEMS, DHALF>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <int ITEMS, bool DHALF>
cudaError_t allow_tall() {
    cudaError_t e = cudaSuccess, r;
    if ((r = allow_tall_t<ITEMS, DHALF, PASS_PLAIN>()) != cudaSuccess) e = r;
    if ((r = allow_tall_t<ITEMS, DHALF, PASS_SUPPORT_CONF>()) != cudaSuccess) e = r;
    if ((r = allow_tall_t<ITEMS, DHALF, PASS_TRANSPOSE>()) != cudaSuccess) e = r;
    return e;
}

// ---------------------------------------------------------------- tuned shapes
// Shapes chosen by dts_autotune (measured per line length), consulted before the defaults.
std::mutex g_tuned_mutex;
std::map<int, int> g_tuned_row_items;      // W -> items per thread
std::map<int, ColPlan> g_tuned_col_plans;  // H -> vertical shape

void set_tuned_row(int W, int items) {
    std::lock_guard<std::mutex> lock(g_tuned_mutex);
    g_tuned_row_items[W] = items;
}
void set_tuned_col(int H, const ColPlan& p) {
    std::lock_guard<std::mutex> lock(g_tuned_mutex);
    g_tuned_col_plans[H] = p;
}
bool tuned_col(int H, ColPlan* p) {
    std::lock_guard<std::mutex> lock(g_tuned_mutex);
    auto it = g_tuned_col_plans.find(H);
    if (it == g_tuned_col_plans.end()) return false;
    *p = it->second;
    return true;
}
int tuned_row(int W) {
    std::lock_guard<std::mutex> lock(g_tuned_mutex);
    auto it = g_tuned_row_items.find(W);
    return it == g_tuned_row_items.end() ? 0 : it->second;
}
// "row W items" / "col H items warps cluster" lines
std::string tuned_export() {
    std::lock_guard<std::mutex> lock(g_tuned_mutex);
    std::string out;
    char line[96];
    for (auto& kv : g_tuned_row_items) {
        snprintf(line, sizeof(line), "row %d %d\n", kv.first, kv.second);
        out += line;
    }
    for (auto& kv : g_tuned_col_plans) {
        snprintf(line, sizeof(line), "col %d %d %d %d\n", kv.first, kv.second.items, kv.second.warps,
                 kv.second.cluster);
        out += line;
    }
    return out;
}

size_t chain_ctl_bytes(int W) {
    // + the paired tall kernel's flags: 2 per unit and strip parity
    return ((size_t)chain_ctl_words((W + 31) / 32) + 4 * kTallPairUnits) * sizeof(unsigned);
}
size_t chain_agg_bytes(int H, int W) {
    // chunks of at least 64 rows; per column and chunk up to 10 floats (the two-phase adjoint's
    // six numbers of totals and four of carries; the chain's Pre and Suf take 9 at most)
    const size_t S = (size_t)(W + 31) / 32, J = (size_t)(H + 63) / 64;
    return S * J * 32 * 10 * sizeof(float);
}

// chain shapes (rows per thread, warps per CTA), the default first
constexpr int kChainShapes[][2] = {{16, 8}, {16, 16}, {32, 8}};

bool chain_shape_fits(int H, int items, int warps) {
    const int J = (H + items * warps - 1) / (items * warps);
    return H <= kMaxColRows && J <= kChainMaxChunks;
}

// the default chain plan for columns of H rows
bool chain_plan(int H, ColPlan* p) {
    p->items = kChainShapes[0][0];
    p->warps = kChainShapes[0][1];
    p->cluster = kColChain;
    return chain_shape_fits(H, p->items, p->warps);
}

// rows per thread of the tall kernel: the most (the smallest clusters, so more of them fit at
// once) whose clusters of 16 warps hold the column in at most 10 CTAs; else the fewest whose
// clusters hold it in at most 16 (columns up to 10240 rows).  Measured on GB300 (vertical pass,
// default against this choice): 4096 x 4096 105.4 -> 74.0 us (clusters of 16 -> 7), 6000 x 3000
// 85.5 -> 72.2 us (12 -> 10), 2500 x 2500 32.5 -> 27.0 us (10 -> 4); 8192 x 1024 stays at 32
// rows (16 CTAs, 41.2 us against 46.4 us with 13 CTAs of 40 rows).
bool tall_plan(int H, ColPlan* p) {
    p->warps = kTallWarps;
    p->cluster = kColTall;
    for (int items : {40, 32, 16}) {
        if ((H + kTallWarps * items - 1) / (kTallWarps * items) <= 10) {
            p->items = items;
            return true;
        }
    }
    for (int items : {16, 32, 40}) {
        if ((H + kTallWarps * items - 1) / (kTallWarps * items) <= 16) {
            p->items = items;
            return true;
        }
    }
    return false;
}

// vertical shapes the tuner tries: the strip kernel (columns up to kStripMaxRows rows), the tall
// kernel's shapes, the chain shapes, then rows per thread x warps per CTA in clusters of at most 16
int col_candidates(int H, ColPlan* out, int max_out) {
    static const int cand[][2] = {{8, 8}, {8, 16}, {8, 32}, {16, 8}, {16, 16}, {32, 8}, {32, 16}, {40, 16}};
    int n = 0;
    if (H <= kStripMaxRows && n < max_out) {
        strip_shape(H, &out[n].items, &out[n].warps);
        out[n++].cluster = kColStrip;
    }
    for (int items : {16, 32, 40})
        if (H > 1 && (H + kTallWarps * items - 1) / (kTallWarps * items) <= 16 && n < max_out)
            out[n++] = ColPlan{items, kTallWarps, kColTall};
    for (int items : {32, 40}) {  // paired halves: columns of 3 to 32 tiles
        const int tiles = (H + kTallWarps * items - 1) / (kTallWarps * items);
        if (tiles >= 3 && tiles <= 32 && H <= kMaxColRows && n < max_out) out[n++] = ColPlan{items, kTallWarps, kColTallPair};
    }
    for (const auto& c : kChainShapes)
        if (H > 1 && chain_shape_fits(H, c[0], c[1]) && n < max_out) out[n++] = ColPlan{c[0], c[1], kColChain};
    for (const auto& c : cand) {
        const int rows = c[0] * c[1];
        const int cs = (H + rows - 1) / rows;
        if (cs > 16 || (cs > 1 && rows > 2 * H) || n >= max_out) continue;
        out[n++] = ColPlan{c[0], c[1], cs};
    }
    return n;
}

namespace {
void row_plan_of(int W, int items, RowPlan* p) {
    int tpr = (W + items - 1) / items;
    tpr = (tpr + 31) / 32 * 32;
    int rpb = items % 2 ? 1 : 256 / tpr;  // the streaming kernel takes one row per CTA
    if (rpb < 1) rpb = 1;
    p->items = items;
    p->tpr = tpr;
    p->rpb = rpb;
}
}  // namespace

// The regular horizontal kernel's plan: ITEMS positions per thread, one row per tpr threads (a
// multiple of 32): 8 up to 256 columns, 16 up to 8192 and above 10240, 32 in between (CTAs of
// at most 320 threads, two per SM, where 16 positions in CTAs of over 512 threads leave one CTA
// per SM).
bool plan_rows_regular(int W, RowPlan* p) {
    if (W > 16 * 1024) return false;
    row_plan_of(W, W <= 256 ? 8 : (W <= 8192 || W > 10240) ? 16 : 32, p);
    return true;
}

// Horizontal plan: a tuned segment length first (8, 16, 32: the regular kernel; 17, 33: the
// streaming kernel); else, for rows of at least 1024 columns, the streaming kernel at 17
// positions per thread where it takes the row (up to 8704 columns), else at 33 (up to 12672);
// else the regular plan.  Measured on GB300 (plain pass, then the pass with the update): 2048
// columns 12.4 -> 11.3 us and 25.4 -> 18.6 us (1536 rows); 2880 columns 17.7 -> 16.0 and 38.6 ->
// 35.7 us (1988 rows); 10000 columns 316 -> 222 us and 854 -> 623 us (10000 rows).
bool plan_rows(int W, RowPlan* p) {
    if (!plan_rows_regular(W, p)) return false;
    const int tuned = tuned_row(W);
    if ((tuned == 8 || tuned == 16 || tuned == 32) && ((W + tuned - 1) / tuned + 31) / 32 * 32 <= (tuned >= 32 ? 320 : 1024))
        row_plan_of(W, tuned, p);
    else if ((tuned == 17 || tuned == 33) && row_stream_fits(W, tuned))
        row_plan_of(W, tuned, p);
    else if (W >= 1024 && row_stream_fits(W, 17))
        row_plan_of(W, 17, p);
    else if (W >= 1024 && row_stream_fits(W, 33))
        row_plan_of(W, 33, p);
    return true;
}

// Vertical plan: a tuned shape first; else the strip kernel for columns up to kStripMaxRows rows
// (measured faster than clusters on the stereo, depth and 256 x 256 workloads), else the plan of
// the other kernels.
bool plan_cols(int H, ColPlan* p) {
    if (H > kMaxColRows) return false;
    if (tuned_col(H, p)) return true;
    if (H <= kStripMaxRows) {
        strip_shape(H, &p->items, &p->warps);
        p->cluster = kColStrip;
        return true;
    }
    return plan_cols_multi(H, p);
}

// Plan for the pass kinds the strip kernel does not run (and columns taller than it): a tuned
// shape of another kernel first; else the cluster kernel up to 256 rows (one CTA), the
// persistent TMA clusters up to 10240 rows, the chain above.
bool plan_cols_multi(int H, ColPlan* p) {
    if (H > kMaxColRows) return false;
    if (tuned_col(H, p) && p->cluster != kColStrip) return true;
    if (H <= 256) return plan_cols_cluster(H, p);
    if (tall_plan(H, p)) return true;
    return chain_plan(H, p);
}

// Cluster plan (solves that run side by side, whose CTAs must not wait on one another across
// streams): columns up to 256 rows in one CTA; else the first (items, warps) shape whose cluster
// holds the whole column with at most 8 CTAs, else at most 16 (non-portable size).
bool plan_cols_cluster(int H, ColPlan* p) {
    if (tuned_col(H, p) && p->cluster > 0) return true;
    if (H <= 256) {
        int nw = 1;
        while (nw * 8 < H) nw <<= 1;  // a power of two (the CTA scan works in lane groups)
        p->items = 8;
        p->warps = nw;
        p->cluster = 1;
        return true;
    }
    // measured on the 2880 x 1988 stereo workload: 16 rows x 16 warps per CTA at 64 registers
    // (two CTAs, 32 warps per SM) is fastest
    static const int cand[][2] = {{16, 16}, {32, 8}, {32, 16}, {40, 16}};
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

// dynamic shared memory of the TMA strip kernel: up to 32 slabs (208 KB at 17 rows, FP32)
template <int ITEMS, bool DHALF>
cudaError_t allow_strip_smem() {
    const cudaError_t e = cudaFuncSetAttribute((const void*)col_strip_tma_kernel<ITEMS, DHALF, false>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               kStripWarps * strip_slab_bytes<ITEMS, DHALF>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void*)col_strip_tma_kernel<ITEMS, DHALF, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kStripWarps * strip_slab_bytes<ITEMS, DHALF>());
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
    if ((r = allow_strip_smem<9, false>()) != cudaSuccess) e = r;
    if ((r = allow_strip_smem<9, true>()) != cudaSuccess) e = r;
    if ((r = allow_strip_smem<17, false>()) != cudaSuccess) e = r;
    if ((r = allow_strip_smem<17, true>()) != cudaSuccess) e = r;
    if ((r = allow_chain_smem_all<16, 8, false>()) != cudaSuccess) e = r;
    if ((r = allow_chain_smem_all<16, 8, true>()) != cudaSuccess) e = r;
    if ((r = allow_chain_smem_all<16, 16, false>()) != cudaSuccess) e = r;
    if ((r = allow_chain_smem_all<16, 16, true>()) != cudaSuccess) e = r;
    if ((r = allow_chain_smem_all<32, 8, false>()) != cudaSuccess) e = r;
    if ((r = allow_chain_smem_all<32, 8, true>()) != cudaSuccess) e = r;
    if ((r = allow_tall<16, false>()) != cudaSuccess) e = r;
    if ((r = allow_tall<16, true>()) != cudaSuccess) e = r;
    if ((r = allow_tall<32, false>()) != cudaSuccess) e = r;
    if ((r = allow_tall<32, true>()) != cudaSuccess) e = r;
    if ((r = allow_tall<40, false>()) != cudaSuccess) e = r;
    if ((r = allow_tall<40, true>()) != cudaSuccess) e = r;
    return e;
}

}  // namespace dts
