// Reverse mode of the solver for sm_103a (the paper has no backward; these kernels follow from
// the forward recurrences by the chain rule).
//
// One horizontal or vertical pass computes, along every line, J = causal(x) and K = anticausal(J)
//     J[n] = (1 - w_n) x[n] + w_n J[n-1],   K[n] = (1 - w_{n+1}) J[n] + w_{n+1} K[n+1].
// Given G = dL/dK, its adjoint is a left-to-right then right-to-left pair as well:
//     h[n]  = G[n] + w_n h[n-1]                          (total gradient of K[n])
//     gJ[n] = (1 - w_{n+1}) h[n] + w_{n+1} gJ[n+1]       (total gradient of J[n])
//     dL/dx[n] = (1 - w_n) gJ[n]
//     dL/dw_n  = gJ[n] (J[n-1] - x[n]) + h[n-1] (K[n] - J[n-1]),   dL/dd_n = ln(a) w_n dL/dw_n.
// The pass output K is read back (it is the next pass's input, or zbar for the last pass), and J
// is recomputed from the pass input with its causal map alone; the pair (h, gJ) has the same
// coupled structure as (J, K) (unnormalised on the way out).  So a pass adjoint exchanges, per
// segment, two affine maps (J and h left to right) and one coupled five-tuple (h, gJ) in one
// round.  The first horizontal pass adds the filter's adjoint into the gradient of the iterate.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>

#include "dts_scan.cuh"

namespace dts {

namespace {

using namespace scan;

struct Pre2 {
    Aff jk, hg;  // causal maps of J and of h
};

struct BackwardMode {
    using Pre = Pre2;
    using Suf = Coupled;  // (h, gJ)
    static __device__ __forceinline__ Pre pre_identity() { return Pre{aff_identity(), aff_identity()}; }
    static __device__ __forceinline__ Pre pre_compose(const Pre& f, const Pre& s) {
        return Pre{aff_compose(f.jk, s.jk), aff_compose(f.hg, s.hg)};
    }
    static __device__ __forceinline__ Suf suf_identity() { return coupled_identity(); }
    static __device__ __forceinline__ Suf suf_compose(const Suf& f, const Suf& s) { return coupled_compose(f, s); }
};

// A segment's own transforms: the causal map of J (normalised, on the pass input x), and the
// coupled transform of (h, gJ) (unnormalised, on G = dL/dK); both share the weight product.
template <int N>
__device__ __forceinline__ void adjoint_local(const float (&x)[N], const float (&w)[N], float wn, const float (&G)[N],
                                              Pre2& pre, Coupled& suf) {
    suf = coupled_local<false>(G, w, wn);
    float q = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) q = fmaf(w[j], q - x[j], x[j]);
    pre = Pre2{Aff{suf.A, q}, Aff{suf.A, suf.B}};
}

// Replays one segment given its carries: jin (J entering from the left), hin (h from the left),
// gin (gJ from the right).  In: x the pass input, G = dL/dK, K the pass output.  Out: x holds
// dL/dx and G holds ln(a) w dL/dw.  Left to right the sweep forms J and h and the two parts of
// dL/dw_n that need J[n-1] and h[n-1]: b = J[n-1] - x[n] (into x) and h[n-1] (K[n] - J[n-1])
// (into K); right to left it forms gJ and finishes both gradients.  Four arrays stay live.
template <int N>
__device__ __forceinline__ void segment_adjoint(float (&x)[N], const float (&w)[N], float wn, float (&G)[N],
                                                float (&K)[N], float jin, float hin, float gin, float lna) {
    float Jp = jin, hp = hin;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const float J = fmaf(w[j], Jp - x[j], x[j]);
        K[j] = hp * (K[j] - Jp);
        x[j] = Jp - x[j];
        hp = fmaf(w[j], hp, G[j]);
        G[j] = hp;  // h[j]
        Jp = J;
    }
    float g = gin;
#pragma unroll
    for (int j = N - 1; j >= 0; --j) {
        const float wp = (j + 1 < N) ? w[j + 1] : wn;
        g = fmaf(wp, g - G[j], G[j]);  // (1 - w') h + w' g
        G[j] = lna * w[j] * fmaf(g, x[j], K[j]);
        x[j] = fmaf(-w[j], g, g);  // (1 - w) g
    }
}

// ---------------------------------------------------------------- horizontal pass adjoint
// Same thread layout as the forward horizontal pass.  FINAL: the first pass of the filter; its
// input gradient is added into a.gz instead of written to a.gout.
// CTA limit: 1024 threads at 8 positions; 640 at 16 (rows up to 10240, registers for five arrays)
template <int ITEMS>
constexpr int row_bwd_max_threads() {
    return ITEMS <= 8 ? 1024 : 640;
}

template <int ITEMS, bool DHALF, bool FINAL>
__global__ void __launch_bounds__(row_bwd_max_threads<ITEMS>()) row_bwd_kernel(BwdArgs a, int tpr) {
    static_assert(ITEMS % 4 == 0, "ITEMS must be a multiple of 4");
    using M = BackwardMode;
    __shared__ M::Pre s_pre[32];
    __shared__ M::Suf s_suf[32];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int rloc = tid / tpr;
    const int t = tid - rloc * tpr;
    const int wpr = tpr >> 5;
    const int wrow = t >> 5;
    const int wbase = warp - wrow;
    const int rpb = blockDim.x / tpr;
    const int row = blockIdx.x * rpb + rloc;
    const bool row_ok = row < a.H;
    const int e0 = t * ITEMS;
    const long long P = a.pitch;
    const long long base = (long long)row * P + e0;
    const bool live = row_ok && e0 < P;

    wait_predecessor();
    // the distance gradient is read-modified-written at the end: bring its lines into L2 now
    if (live) prefetch_l2(a.dbar + base);
    float x[ITEMS], w[ITEMS], G[ITEMS], K[ITEMS];
    if (live) {
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            load4_f(a.x, base + 4 * q, &x[4 * q]);
            load4_f(a.gin, base + 4 * q, &G[4 * q]);
            load4_f(a.kout, base + 4 * q, &K[4 * q]);
            load4_d<DHALF>(a.d, base + 4 * q, &w[4 * q]);
        }
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) w[j] = ex2(a.k2 * w[j]);
        if (e0 + ITEMS > a.W) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (e0 + j >= a.W) x[j] = w[j] = G[j] = K[j] = 0.f;
        }
        if (e0 == 0) w[0] = 0.f;
    } else {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) x[j] = w[j] = G[j] = K[j] = 0.f;
    }
    float wn = __shfl_down_sync(kFull, w[0], 1);
    if (lane == 31) {
        const int en = e0 + ITEMS;
        wn = (row_ok && en < a.W) ? ex2(a.k2 * load1_d<DHALF>(a.d, (long long)row * P + en)) : 0.f;
    }

    M::Pre own_pre, pre;
    M::Suf own_suf, suf;
    adjoint_local(x, w, wn, G, own_pre, own_suf);
    row_exchange<M>(own_pre, own_suf, lane, warp, wrow, wbase, wpr, s_pre, s_suf, pre, suf);
    release_successor();
    const float jin = pre.jk.B;
    const float hin = pre.hg.B;
    const float gin = k_entering(suf, fmaf(own_pre.hg.A, hin, own_pre.hg.B));
    segment_adjoint(x, w, wn, G, K, jin, hin, gin, a.lna);
    const float(&db)[ITEMS] = G;

    if (live) {
        // every load before the first store (the stores could alias later loads); K is free again
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) load4_f(a.dbar, base + 4 * q, &K[4 * q]);
        float gz[FINAL ? ITEMS : 1];
        if constexpr (FINAL) {
#pragma unroll
            for (int q = 0; q < ITEMS / 4; ++q) load4_f(a.gz, base + 4 * q, &gz[4 * q]);
        }
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            float acc[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = K[4 * q + i] + ((e0 + 4 * q + i < a.W) ? db[4 * q + i] : 0.f);
            store4_f(a.dbar, base + 4 * q, acc);
            if constexpr (FINAL) {
#pragma unroll
                for (int i = 0; i < 4; ++i) gz[4 * q + i] += x[4 * q + i];
                store4_f(a.gz, base + 4 * q, &gz[4 * q]);
            } else {
                store4_f(a.gout, base + 4 * q, &x[4 * q]);
            }
        }
    }
}

// ---------------------------------------------------------------- vertical pass adjoint
// Same layout as the forward vertical pass (lane = column): one cluster per 32-column strip
// (col_bwd_kernel), or a chain of CTAs per strip linked through global memory for taller
// columns (col_bwd_chain_kernel, chain_exchange).

// the distance gradient is read-modified-written at the end: lane j brings row j of the warp's
// rows into L2 now (one 128-byte line per row of the strip)
template <int ITEMS>
__device__ __forceinline__ void col_bwd_prefetch(const BwdArgs& a, int row0, int c0, int lane) {
    if (lane < ITEMS && row0 + lane < a.H && c0 < a.W) prefetch_l2(a.dbar + (long long)(row0 + lane) * a.pitch + c0);
}

// A thread's positions of column `col` from row0: pass input x, weights w, incoming adjoint G
// and pass output K (zero outside the plane), and wn, the weight entering the next segment.
template <int ITEMS, bool DHALF>
__device__ __forceinline__ void col_bwd_load(const BwdArgs& a, int row0, int col, float (&x)[ITEMS], float (&w)[ITEMS],
                                             float (&G)[ITEMS], float (&K)[ITEMS], float& wn) {
    const long long P = a.pitch;
    const bool col_ok = col < a.W;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        const bool ok = col_ok && r < a.H;
        const long long idx = (long long)r * P + col;
        x[j] = ok ? a.x[idx] : 0.f;
        w[j] = ok ? load1_d<DHALF>(a.d, idx) : 0.f;
        G[j] = ok ? a.gin[idx] : 0.f;
        K[j] = ok ? a.kout[idx] : 0.f;
    }
    const int rn = row0 + ITEMS;
    wn = (col_ok && rn < a.H) ? ex2(a.k2 * load1_d<DHALF>(a.d, (long long)rn * P + col)) : 0.f;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        w[j] = (col_ok && r > 0 && r < a.H) ? ex2(a.k2 * w[j]) : 0.f;
    }
}

// Given the carries (pre: everything above, suf: everything below), the segment's adjoint:
// dL/dx into gout, ln(a) w dL/dw added into dbar.
template <int ITEMS>
__device__ __forceinline__ void col_bwd_finish(const BwdArgs& a, int row0, int col, float (&x)[ITEMS],
                                               const float (&w)[ITEMS], float wn, float (&G)[ITEMS], float (&K)[ITEMS],
                                               const Pre2& own_pre, const Pre2& pre, const Coupled& suf) {
    const long long P = a.pitch;
    const bool col_ok = col < a.W;
    const float jin = pre.jk.B;
    const float hin = pre.hg.B;
    const float gin = k_entering(suf, fmaf(own_pre.hg.A, hin, own_pre.hg.B));
    segment_adjoint(x, w, wn, G, K, jin, hin, gin, a.lna);
    // read every distance-gradient value before the first store (the stores could alias later
    // loads, which would otherwise wait for them one by one); K is free again
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        K[j] = (col_ok && r < a.H) ? a.dbar[(long long)r * P + col] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        if (!(col_ok && r < a.H)) continue;
        const long long idx = (long long)r * P + col;
        a.dbar[idx] = K[j] + G[j];
        a.gout[idx] = x[j];
    }
}

// one cluster per strip: warp q of CTA r owns rows [(r NW + q) ITEMS, + ITEMS)
template <int ITEMS>
constexpr int bwd_col_min_blocks() {
    return ITEMS <= 8 ? 2 : 1;  // two resident CTAs of the 8-row shape (64 registers)
}

template <int ITEMS, bool DHALF>
__global__ void __launch_bounds__(512, bwd_col_min_blocks<ITEMS>()) col_bwd_kernel(BwdArgs a) {
    using M = BackwardMode;
    __shared__ ColShared<M, 16> sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const int rank = (int)cg::this_cluster().block_rank();
    const int col = blockIdx.x * 32 + lane;
    const int row0 = (rank * NW + warp) * ITEMS;

    wait_predecessor();
    col_bwd_prefetch<ITEMS>(a, row0, blockIdx.x * 32, lane);
    float x[ITEMS], w[ITEMS], G[ITEMS], K[ITEMS], wn;
    col_bwd_load<ITEMS, DHALF>(a, row0, col, x, w, G, K, wn);
    M::Pre own_pre, pre;
    M::Suf own_suf, suf;
    adjoint_local(x, w, wn, G, own_pre, own_suf);
    col_exchange_scan<M, 16>(own_pre, own_suf, lane, warp, NW, sh, pre, suf);
    release_successor();
    col_bwd_finish<ITEMS>(a, row0, col, x, w, wn, G, K, own_pre, pre, suf);
    cluster_exit();
}

// chained: one CTA of NW warps per chunk of NW x ITEMS rows of a strip (strip and chunk from the
// CTA's ticket)
template <int ITEMS, int NW>
constexpr int bwd_chain_min_blocks() {
    return (NW >= 32 || ITEMS >= 16) ? 1 : ITEMS * NW <= 64 ? 4 : 2;
}

template <int ITEMS, int NW, bool DHALF>
__global__ void __launch_bounds__(32 * NW, bwd_chain_min_blocks<ITEMS, NW>()) col_bwd_chain_kernel(BwdArgs a, ChainArgs c) {
    using M = BackwardMode;
    __shared__ ChainShared<M, NW> sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    wait_predecessor();
    const int ticket = chain_ticket(c);
    const int strip = ticket / c.J;
    const int chunk = ticket - strip * c.J;
    const int col = strip * 32 + lane;
    const int row0 = (chunk * NW + warp) * ITEMS;
    col_bwd_prefetch<ITEMS>(a, row0, strip * 32, lane);
    float x[ITEMS], w[ITEMS], G[ITEMS], K[ITEMS], wn;
    col_bwd_load<ITEMS, DHALF>(a, row0, col, x, w, G, K, wn);
    M::Pre own_pre, pre;
    M::Suf own_suf, suf;
    adjoint_local(x, w, wn, G, own_pre, own_suf);
    chain_exchange<M, NW>(own_pre, own_suf, lane, warp, NW, sh, c, ticket, pre, suf);
    release_successor();
    col_bwd_finish<ITEMS>(a, row0, col, x, w, wn, G, K, own_pre, pre, suf);
}

// Two-phase vertical adjoint (no waits): col_bwd_agg_kernel reduces every chunk of NW x ITEMS
// rows of a 32-column strip to its totals; col_bwd_carry_kernel, one CTA per strip, turns them
// into every chunk's carries; col_bwd_apply_kernel replays every chunk from its carries.  The
// three run as consecutive launches.  They move 12 + 28 bytes per position against the chain's
// 28, but no CTA holds its chunk in registers while it waits for the rest of its column.  Chunk
// kernels: CTA b takes chunk b mod J of strip b / J.
//
// A chunk's totals need six numbers per column: the coupled (h, gJ) tuple (A, B, al, be, ga) and
// the J map's B (the J and h maps share A, and the h map is (A, B)).  Its carries need four: J
// and h entering from above (the B of the maps of everything above; their A never reaches an
// output) and be, ga of everything below (what k_entering reads).  Records (c.agg): S x J x 6 x
// 32 floats of totals, then S x J x 32 float4 carries.
constexpr int kSplitRec = 6;

__device__ __forceinline__ float4* split_carries(const ChainArgs& c) {
    return reinterpret_cast<float4*>(c.agg + (size_t)c.S * c.J * kSplitRec * 32);
}

// x, w and G of a thread's positions (col_bwd_load without the pass output)
template <int ITEMS, bool DHALF>
__device__ __forceinline__ void col_bwd_load3(const BwdArgs& a, int row0, int col, float (&x)[ITEMS],
                                              float (&w)[ITEMS], float (&G)[ITEMS], float& wn) {
    const long long P = a.pitch;
    const bool col_ok = col < a.W;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        const bool ok = col_ok && r < a.H;
        const long long idx = (long long)r * P + col;
        x[j] = ok ? a.x[idx] : 0.f;
        w[j] = ok ? load1_d<DHALF>(a.d, idx) : 0.f;
        G[j] = ok ? a.gin[idx] : 0.f;
    }
    const int rn = row0 + ITEMS;
    wn = (col_ok && rn < a.H) ? ex2(a.k2 * load1_d<DHALF>(a.d, (long long)rn * P + col)) : 0.f;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        w[j] = (col_ok && r > 0 && r < a.H) ? ex2(a.k2 * w[j]) : 0.f;
    }
}

template <int ITEMS, int NW>
constexpr int bwd_split_min_blocks() {
    return ITEMS * NW <= 64 ? 4 : ITEMS * NW <= 128 ? 2 : 1;
}

template <int ITEMS, int NW, bool DHALF>
__global__ void __launch_bounds__(32 * NW, bwd_split_min_blocks<ITEMS, NW>()) col_bwd_agg_kernel(BwdArgs a, ChainArgs c) {
    using M = BackwardMode;
    __shared__ ChainShared<M, NW> sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int strip = (int)blockIdx.x / c.J;
    const int chunk = (int)blockIdx.x - strip * c.J;
    const int col = strip * 32 + lane;
    const int row0 = (chunk * NW + warp) * ITEMS;

    wait_predecessor();
    float x[ITEMS], w[ITEMS], G[ITEMS], wn;
    col_bwd_load3<ITEMS, DHALF>(a, row0, col, x, w, G, wn);
    M::Pre own_pre;
    M::Suf own_suf;
    adjoint_local(x, w, wn, G, own_pre, own_suf);
    sh.pre[warp][lane] = own_pre;
    sh.suf[warp][lane] = own_suf;
    __syncthreads();
    release_successor();
    float* rec = c.agg + ((size_t)strip * c.J + chunk) * kSplitRec * 32 + lane;
    // the chunk's totals: its warps' J maps top down, their coupled tuples bottom up
    if (warp == NW - 1) {
        Aff t = sh.pre[0][lane].jk;
        for (int q = 1; q < NW; ++q) t = aff_compose(t, sh.pre[q][lane].jk);
        __stcg(rec + 5 * 32, t.B);
    }
    if (warp == 0) {
        Coupled t = sh.suf[NW - 1][lane];
        for (int q = NW - 2; q >= 0; --q) t = coupled_compose(sh.suf[q][lane], t);
        __stcg(rec, t.A);
        __stcg(rec + 32, t.B);
        __stcg(rec + 64, t.al);
        __stcg(rec + 96, t.be);
        __stcg(rec + 128, t.ga);
    }
}

// One CTA per strip turns the strip's chunk totals into carries.  Warps 0-7 take the prefix
// direction (top down), warps 8-15 the suffix direction (bottom up), lane = column.  The totals
// come into shared memory in blocks of kCarryStage chunks (the prefix block from the top, the
// suffix block from the bottom); each warp takes a run of consecutive chunks of the block,
// composes the run, takes the other runs' totals before it (and the carry entering the block) as
// its run's carry, and walks its run writing carries: a serial depth of about 2 kCarryStage / 8 +
// 7 compositions per block instead of kCarryStage.
constexpr int kCarryWarps = 8;
constexpr int kCarryStage = 32;

__global__ void __launch_bounds__(64 * kCarryWarps, 3) col_bwd_carry_kernel(ChainArgs c) {
    constexpr int NWC = kCarryWarps;
    constexpr int ST = kCarryStage;
    __shared__ __align__(16) float pst[ST][3][32];  // A, B (the h map's), the J map's B
    __shared__ __align__(16) float sst[ST][5][32];  // A, B, al, be, ga
    __shared__ Pre2 bp[NWC][32];
    __shared__ Coupled bs[NWC][32];
    __shared__ Pre2 runp[32];    // everything above the current prefix block
    __shared__ Coupled runs[32];  // everything below the current suffix block
    wait_predecessor();
    release_successor();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const bool prefix = warp < NWC;
    const int b = warp % NWC;
    const size_t base = (size_t)blockIdx.x * c.J;
    const float* rec = c.agg;
    float4* carry = split_carries(c);
    if (warp == 0) {
        runp[lane] = Pre2{aff_identity(), aff_identity()};
        runs[lane] = coupled_identity();
    }
    for (int b0 = 0; b0 < c.J; b0 += ST) {
        const int nb = min(ST, c.J - b0);
        const int s0 = c.J - b0 - nb;  // the suffix block: chunks [s0, s0 + nb)
        {
            // 16-byte pieces: per chunk 24 of the prefix block (fields 0-1, then field 5), then per
            // chunk 40 of the suffix block (fields 0-4); every load of a thread is issued before
            // its stores
            constexpr int NT = 64 * NWC;
            constexpr int U = (ST * 64 + NT - 1) / NT;
            const float4* r4 = reinterpret_cast<const float4*>(rec);
            const int np = nb * 24;
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = (int)threadIdx.x + u * NT;
                if (k < np) {
                    const int j = k / 24, r = k - j * 24;
                    v[u] = __ldcg(r4 + (base + b0 + j) * (kSplitRec * 8) + (r < 16 ? r : r + 24));
                } else if (k < nb * 64) {
                    const int j = (k - np) / 40, r = k - np - j * 40;
                    v[u] = __ldcg(r4 + (base + s0 + j) * (kSplitRec * 8) + r);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = (int)threadIdx.x + u * NT;
                if (k < np) reinterpret_cast<float4*>(&pst[0][0][0])[k] = v[u];
                else if (k < nb * 64) reinterpret_cast<float4*>(&sst[0][0][0])[k - np] = v[u];
            }
        }
        __syncthreads();
        const int per = (nb + NWC - 1) / NWC;
        const int j0 = min(nb, b * per);
        const int j1 = min(nb, j0 + per);
        auto pchunk = [&](int j) {
            return Pre2{Aff{pst[j][0][lane], pst[j][2][lane]}, Aff{pst[j][0][lane], pst[j][1][lane]}};
        };
        auto schunk = [&](int j) {
            return Coupled{sst[j][0][lane], sst[j][1][lane], sst[j][2][lane], sst[j][3][lane], sst[j][4][lane]};
        };
        if (prefix) {
            Pre2 t = Pre2{aff_identity(), aff_identity()};
            for (int j = j0; j < j1; ++j) t = BackwardMode::pre_compose(t, pchunk(j));
            bp[b][lane] = t;
        } else {
            Coupled t = coupled_identity();
            for (int j = j1 - 1; j >= j0; --j) t = coupled_compose(schunk(j), t);
            bs[b][lane] = t;
        }
        __syncthreads();
        Pre2 pacc;
        Coupled sacc;
        if (prefix) {
            pacc = runp[lane];
            for (int q = 0; q < b; ++q) pacc = BackwardMode::pre_compose(pacc, bp[q][lane]);
            for (int j = j0; j < j1; ++j) {
                __stcg(reinterpret_cast<float2*>(carry + (base + b0 + j) * 32 + lane), make_float2(pacc.jk.B, pacc.hg.B));
                pacc = BackwardMode::pre_compose(pacc, pchunk(j));
            }
        } else {
            sacc = runs[lane];
            for (int q = NWC - 1; q > b; --q) sacc = coupled_compose(bs[q][lane], sacc);
            for (int j = j1 - 1; j >= j0; --j) {
                __stcg(reinterpret_cast<float2*>(carry + (base + s0 + j) * 32 + lane) + 1, make_float2(sacc.be, sacc.ga));
                sacc = coupled_compose(schunk(j), sacc);
            }
        }
        __syncthreads();
        // the carries entering the next blocks: the last prefix run's and the first suffix run's
        if (prefix && b == NWC - 1) runp[lane] = pacc;
        if (!prefix && b == 0) runs[lane] = sacc;
    }
}

template <int ITEMS, int NW, bool DHALF>
__global__ void __launch_bounds__(32 * NW, bwd_split_min_blocks<ITEMS, NW>()) col_bwd_apply_kernel(BwdArgs a, ChainArgs c) {
    using M = BackwardMode;
    __shared__ ChainShared<M, NW> sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int strip = (int)blockIdx.x / c.J;
    const int chunk = (int)blockIdx.x - strip * c.J;
    const int col = strip * 32 + lane;
    const int row0 = (chunk * NW + warp) * ITEMS;

    wait_predecessor();
    col_bwd_prefetch<ITEMS>(a, row0, strip * 32, lane);
    const float4 cr = __ldcg(split_carries(c) + ((size_t)strip * c.J + chunk) * 32 + lane);
    float x[ITEMS], w[ITEMS], G[ITEMS], K[ITEMS], wn;
    col_bwd_load<ITEMS, DHALF>(a, row0, col, x, w, G, K, wn);
    M::Pre own_pre;
    M::Suf own_suf;
    adjoint_local(x, w, wn, G, own_pre, own_suf);
    sh.pre[warp][lane] = own_pre;
    sh.suf[warp][lane] = own_suf;
    __syncthreads();
    // everything above the warp's segment (only the B of the maps is used) and everything below
    M::Pre pre = Pre2{Aff{1.f, cr.x}, Aff{1.f, cr.y}};
    for (int q = 0; q < warp; ++q) pre = M::pre_compose(pre, sh.pre[q][lane]);
    M::Suf suf = M::suf_identity();
    for (int q = warp + 1; q < NW; ++q) suf = M::suf_compose(suf, sh.suf[q][lane]);
    suf = M::suf_compose(suf, Coupled{1.f, 0.f, 1.f, cr.z, cr.w});
    release_successor();
    col_bwd_finish<ITEMS>(a, row0, col, x, w, wn, G, K, own_pre, pre, suf);
}

// ---------------------------------------------------------------- guide gradient
// dL/dI_c[y][x] gathers the four distances that involve pixel (y, x):
//   L1 d = 1 + k sum |D|:          dd/dD = k sign(D)
//   L2 d = sqrt(1 + k^2 sum D^2):  dd/dD = k^2 D / d
// with D = I(p) - I(q) for the neighbour q on the left / above.
template <typename GT, bool DHALF>
__global__ void __launch_bounds__(256) guide_grad_kernel(GuideGradArgs a) {
    wait_predecessor();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.W || y >= a.H) return;
    const GT* I = static_cast<const GT*>(a.guide);
    const long long P = a.pitch;
    const long long q = (long long)y * P + x;
    const bool l2 = a.norm == DTS_NORM_L2;
    auto slope = [&](float D, long long qi, bool vertical) -> float {
        if (l2) return a.k * a.k * D / load1_d<DHALF>(vertical ? a.dY : a.dX, qi);
        return a.k * (float)((D > 0.f) - (D < 0.f));
    };
    const float gl = x > 0 ? a.dXb[q] : 0.f;
    const float gr = x + 1 < a.W ? a.dXb[q + 1] : 0.f;
    const float gu = y > 0 ? a.dYb[q] : 0.f;
    const float gd = y + 1 < a.H ? a.dYb[q + P] : 0.f;
    for (int c = 0; c < a.C; ++c) {
        const GT* Ic = I + (long long)c * a.ch_stride + (long long)y * a.row_stride + x;
        const float v = to_f32<GT>(Ic[0]);
        float g = 0.f;
        if (x > 0) g += gl * slope(v - to_f32<GT>(Ic[-1]), q, false);
        if (x + 1 < a.W) g -= gr * slope(to_f32<GT>(Ic[1]) - v, q + 1, false);
        if (y > 0) g += gu * slope(v - to_f32<GT>(Ic[-a.row_stride]), q, true);
        if (y + 1 < a.H) g -= gd * slope(to_f32<GT>(Ic[a.row_stride]) - v, q + P, true);
        a.out[((long long)c * a.H + y) * a.W + x] = g;
    }
}

// The same gradient, four consecutive pixels of a row per thread (rows of whole 16-byte units,
// aligned planes): per band one vector load each of the pixels' row and the rows above and below,
// the horizontal neighbours by warp shuffles (lanes 0 and 31 load the one past the warp), one
// vector store.  The per-pixel slopes' factors and the incoming adjoints of the four distances
// are loaded once, before the band loop.  Scalar form: 977 us at 2048 x 10000 x 16 bands, one
// round trip of 20 bytes per thread and band, 768 M warp instructions (long_scoreboard 13.7).
template <typename GT>
__device__ __forceinline__ void load4_g(const GT* p, float (&out)[4]) {
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

template <typename GT, bool DHALF>
__global__ void __launch_bounds__(256) guide_grad4_kernel(GuideGradArgs a) {
    wait_predecessor();
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int y = blockIdx.y;
    const bool xok = x0 < a.W;  // W % 4 == 0: the four pixels are all inside or all outside
    const long long P = a.pitch;
    const long long q = (long long)y * P + x0;
    const bool l2 = a.norm == DTS_NORM_L2;
    const bool hu = y > 0, hd = y + 1 < a.H;
    // incoming adjoints of the pixel's four distances (left, right, up, down) and the slopes'
    // factors: k for L1 (times the sign), k^2 / d for L2 (times the difference)
    float gl[4], gr[4], gu[4], gd[4], kl[4], kr[4], ku[4], kd[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) gl[k] = gr[k] = gu[k] = gd[k] = 0.f, kl[k] = kr[k] = ku[k] = kd[k] = a.k;
    if (xok) {
        load4_g<float>(a.dXb + q, gl);
        if (hu) load4_g<float>(a.dYb + q, gu);
        if (hd) load4_g<float>(a.dYb + q + P, gd);
    }
    // the adjoint of the right neighbour's distance: the next lane's first, past the warp by load
    float nxt = __shfl_down_sync(kFull, gl[0], 1);
    if (lane == 31) nxt = (xok && x0 + 4 < a.W) ? a.dXb[q + 4] : 0.f;
    gr[0] = gl[1];
    gr[1] = gl[2];
    gr[2] = gl[3];
    gr[3] = x0 + 4 < a.W ? nxt : 0.f;
    if (x0 == 0) gl[0] = 0.f;
    if (l2) {
        const float k2 = a.k * a.k;
        float dl[4] = {1.f, 1.f, 1.f, 1.f}, du[4] = {1.f, 1.f, 1.f, 1.f}, dd[4] = {1.f, 1.f, 1.f, 1.f};
        if (xok) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dl[k] = load1_d<DHALF>(a.dX, q + k);
                if (hu) du[k] = load1_d<DHALF>(a.dY, q + k);
                if (hd) dd[k] = load1_d<DHALF>(a.dY, q + P + k);
            }
        }
        float dn = __shfl_down_sync(kFull, dl[0], 1);
        if (lane == 31) dn = (xok && x0 + 4 < a.W) ? load1_d<DHALF>(a.dX, q + 4) : 1.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            kl[k] = k2 / dl[k];
            kr[k] = k2 / (k < 3 ? dl[k + 1] : dn);
            ku[k] = k2 / du[k];
            kd[k] = k2 / dd[k];
        }
    }
    auto slope = [&](float D, float kk) -> float { return l2 ? kk * D : kk * (float)((D > 0.f) - (D < 0.f)); };
    const GT* I = static_cast<const GT*>(a.guide) + (long long)y * a.row_stride + x0;
    float* out = a.out + (long long)y * a.W + x0;
    for (int c = 0; c < a.C; ++c) {
        const GT* Ic = I + (long long)c * a.ch_stride;
        float v[4] = {0.f, 0.f, 0.f, 0.f}, up[4] = {0.f, 0.f, 0.f, 0.f}, dn4[4] = {0.f, 0.f, 0.f, 0.f};
        if (xok) {
            load4_g<GT>(Ic, v);
            if (hu) load4_g<GT>(Ic - a.row_stride, up);
            if (hd) load4_g<GT>(Ic + a.row_stride, dn4);
        }
        float left = __shfl_up_sync(kFull, v[3], 1);
        float right = __shfl_down_sync(kFull, v[0], 1);
        if (lane == 0) left = (xok && x0 > 0) ? to_f32<GT>(Ic[-1]) : 0.f;
        if (lane == 31) right = (xok && x0 + 4 < a.W) ? to_f32<GT>(Ic[4]) : 0.f;
        if (!xok) continue;
        float g[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float l = k == 0 ? left : v[k - 1];
            const float r = k == 3 ? right : v[k + 1];
            // a missing neighbour has a zero adjoint (gl, gr, gu, gd): its term adds nothing
            g[k] = gl[k] * slope(v[k] - l, kl[k]) - gr[k] * slope(r - v[k], kr[k]) + gu[k] * slope(v[k] - up[k], ku[k]) -
                   gd[k] * slope(dn4[k] - v[k], kd[k]);
        }
        *reinterpret_cast<float4*>(out + (long long)c * a.H * a.W) = make_float4(g[0], g[1], g[2], g[3]);
    }
}

// Adjoint of the data-term update at every pixel, given g = dL/dz_{k+1} in a.gz:
//   GD      dzbar = eta lambda g,  dt += eta c rho'' g,  dc -= eta rho' g,
//           a.gz <- (1 - eta lambda - eta c rho'') g,  with rho' and rho'' at r = z_k - t: r and 1
//           for the square, r / s and eps^2 / s^3 (s = sqrt(r^2 + eps^2)) for the Charbonnier loss
//   Jacobi  dzbar = lambda g / den,  dt += c g / den,  dc += lambda (t - zbar) g / den^2,  a.gz <- 0
//           (den = lambda + c; where den = 0 the iterate was kept: a.gz <- g and nothing else)
// dzbar goes to a.gout (the input gradient of the last pass's adjoint); a.x holds zbar (Jacobi).
// Four consecutive pixels per thread; VEC: 16-byte accesses (W % 4 == 0, aligned planes), else
// element by element.  Every operand is loaded before the first store.
template <bool VEC>
__global__ void __launch_bounds__(256) update_adjoint_kernel(BwdArgs a) {
    wait_predecessor();
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int y = blockIdx.y;
    if (x0 >= a.W || y >= a.H) return;
    const long long idx = (long long)y * a.pitch + x0;
    const long long di = (long long)y * a.W + x0;
    const bool jac = a.update == DTS_UPDATE_JACOBI;
    // zz: zbar (Jacobi) or z_k (GD); zk: z_k where the Jacobi update's weight needs it
    const bool need_zk = jac && a.eps > 0.f;
    float g[4], cf[4], t[4], zz[4], zk[4] = {0.f, 0.f, 0.f, 0.f}, gt[4] = {0.f, 0.f, 0.f, 0.f},
          gc[4] = {0.f, 0.f, 0.f, 0.f};
    if (VEC) {
        load4_f(a.gz, idx, g);
        load4_f(a.c, di, cf);
        load4_f(jac ? a.x : a.zk, idx, zz);
        if (need_zk) load4_f(a.zk, idx, zk);
        if (a.gt) load4_f(a.gt, di, gt);
        if (a.gc) load4_f(a.gc, di, gc);
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] = load_any(a.t, di + k, a.t_dtype);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = x0 + k < a.W;
            g[k] = ok ? a.gz[idx + k] : 0.f;
            cf[k] = ok ? a.c[di + k] : 0.f;
            zz[k] = ok ? (jac ? a.x : a.zk)[idx + k] : 0.f;
            if (need_zk && ok) zk[k] = a.zk[idx + k];
            t[k] = ok ? load_any(a.t, di + k, a.t_dtype) : 0.f;
            if (a.gt && ok) gt[k] = a.gt[di + k];
            if (a.gc && ok) gc[k] = a.gc[di + k];
        }
    }
    float dzb[4], dz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (jac) {
            // c~ = c w, w = 1 / sqrt(r^2 + eps^2) at r = z_k - t for the Charbonnier loss (w = 1 for
            // the square); c~ reaches z_k and t through r: dc~/dr = -c r w^3
            float w = 1.f, r = 0.f;
            if (a.eps > 0.f) {
                r = zk[k] - t[k];
                w = rsqrtf(fmaf(r, r, a.eps * a.eps));
            }
            const float cw = cf[k] * w;
            const float den = a.lambda + cw;
            if (den != 0.f) {
                const float gcw = a.lambda * (t[k] - zz[k]) / (den * den) * g[k];
                const float gr = a.eps > 0.f ? -cf[k] * r * w * w * w * gcw : 0.f;
                dzb[k] = a.lambda / den * g[k];
                gt[k] += cw / den * g[k] - gr;
                gc[k] += w * gcw;
                dz[k] = gr;
            } else {
                dzb[k] = 0.f;
                dz[k] = g[k];
            }
        } else {
            const float r = zz[k] - t[k];
            float d1 = r, d2 = 1.f;
            if (a.eps > 0.f) {
                const float is = rsqrtf(fmaf(r, r, a.eps * a.eps));
                d1 = r * is;
                d2 = a.eps * a.eps * is * is * is;
            }
            dzb[k] = a.step * a.lambda * g[k];
            gt[k] += a.step * cf[k] * d2 * g[k];
            gc[k] -= a.step * d1 * g[k];
            dz[k] = (1.f - a.step * a.lambda - a.step * cf[k] * d2) * g[k];
        }
    }
    if (VEC) {
        store4_f(a.gout, idx, dzb);
        store4_f(a.gz, idx, dz);
        if (a.gt) store4_f(a.gt, di, gt);
        if (a.gc) store4_f(a.gc, di, gc);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (x0 + k >= a.W) continue;
            a.gout[idx + k] = dzb[k];
            a.gz[idx + k] = dz[k];
            if (a.gt) a.gt[di + k] = gt[k];
            if (a.gc) a.gc[di + k] = gc[k];
        }
    }
}

// dst[y][x] (pitch dp) += src[y][x] (pitch sp), or = when accumulate is 0
template <bool VEC>
__global__ void __launch_bounds__(256) axpy_plane_kernel(const float* src, long long sp, float* dst, long long dp,
                                                         int H, int W, int accumulate) {
    wait_predecessor();
    const int y = blockIdx.y;
    if constexpr (VEC) {  // four elements per thread (W, both pitches and both planes 16-byte aligned)
        const int x = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
        if (x >= W || y >= H) return;
        float4 v = *reinterpret_cast<const float4*>(src + (long long)y * sp + x);
        float4* d = reinterpret_cast<float4*>(dst + (long long)y * dp + x);
        if (accumulate) {
            const float4 o = *d;
            v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
        }
        *d = v;
    } else {
        const int x = blockIdx.x * blockDim.x + threadIdx.x;
        if (x >= W || y >= H) return;
        const float v = src[(long long)y * sp + x];
        float* d = dst + (long long)y * dp + x;
        *d = accumulate ? *d + v : v;
    }
}

template <int ITEMS, bool DHALF>
cudaError_t launch_row_bwd_t(const BwdArgs& a, bool final_pass, const RowPlan& p, cudaStream_t s) {
    const dim3 grid((unsigned)((a.H + p.rpb - 1) / p.rpb));
    const dim3 block((unsigned)(p.tpr * p.rpb));
    if (final_pass) return launch_ex(row_bwd_kernel<ITEMS, DHALF, true>, grid, block, 0, s, a, p.tpr);
    return launch_ex(row_bwd_kernel<ITEMS, DHALF, false>, grid, block, 0, s, a, p.tpr);
}

template <int ITEMS, bool DHALF>
cudaError_t launch_col_bwd_t(const BwdArgs& a, const ColPlan& p, cudaStream_t s) {
    if (p.cluster < 1 || (long long)ITEMS * p.warps * p.cluster < a.H) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((a.W + 31) / 32), (unsigned)p.cluster, 1);
    return launch_ex(col_bwd_kernel<ITEMS, DHALF>, grid, dim3((unsigned)(32 * p.warps)), p.cluster, s, a);
}

// chunks per staging block of the strip composition (two resident CTAs per SM)
constexpr int kBwdChainStage = 64;

template <int ITEMS, int NW, bool DHALF>
cudaError_t allow_bwd_chain_smem() {
    return cudaFuncSetAttribute((const void*)col_bwd_chain_kernel<ITEMS, NW, DHALF>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)chain_stage_bytes<BackwardMode>(kBwdChainStage));
}

// refused (invalid configuration) when fewer than 2 J CTAs of the kernel fit on the GPU at once
template <int ITEMS, int NW, bool DHALF>
cudaError_t launch_col_bwd_chain_t(const BwdArgs& a, cudaStream_t s) {
    auto kernel = col_bwd_chain_kernel<ITEMS, NW, DHALF>;
    ChainArgs c = {};
    c.ctl = a.chain_ctl;
    c.agg = a.chain_agg;
    c.J = (a.H + ITEMS * NW - 1) / (ITEMS * NW);
    c.S = (a.W + 31) / 32;
    c.status = a.status;
    if (!c.ctl || !c.agg || c.J > kChainMaxChunks) return cudaErrorInvalidValue;
    c.stage = std::min(c.J, kBwdChainStage);
    c.epoch = next_chain_epoch();
    const size_t smem = chain_stage_bytes<BackwardMode>(c.stage);
    if (blocks_per_sm((const void*)kernel, 32 * NW, smem) * sm_count() < 2 * c.J) return cudaErrorInvalidConfiguration;
    const bool skip = take_injected(DTS_INJECT_CHAIN_SKIP);
    c.timeout = skip ? kInjectedTimeout : default_timeout_cycles();
    c.skip_ticket = skip && c.J > 1 ? 0 : -1;
    return launch_ex_smem(kernel, dim3((unsigned)(c.S * c.J)), dim3(32 * NW), 0, smem, s, a, c);
}

template <int ITEMS, int NW, bool DHALF>
cudaError_t launch_col_bwd_split_t(const BwdArgs& a, cudaStream_t s) {
    ChainArgs c = {};
    c.ctl = a.chain_ctl;
    c.agg = a.chain_agg;
    c.J = (a.H + ITEMS * NW - 1) / (ITEMS * NW);
    c.S = (a.W + 31) / 32;
    c.status = a.status;
    if (!c.ctl || !c.agg || c.J > kChainMaxChunks) return cudaErrorInvalidValue;
    c.skip_ticket = -1;
    const dim3 grid((unsigned)(c.S * c.J));
    const long long px = (long long)a.H * a.W;
    const int fl = DHALF ? kFlagDistHalf : 0;
    int h = prof_begin(KID_COL_BWD_AGG, px, fl, s);
    cudaError_t e = launch_ex(col_bwd_agg_kernel<ITEMS, NW, DHALF>, grid, dim3(32 * NW), 0, s, a, c);
    prof_end(h, s);
    if (e != cudaSuccess) return e;
    h = prof_begin(KID_COL_BWD_CARRY, px, 0, s);
    e = launch_ex(col_bwd_carry_kernel, dim3((unsigned)c.S), dim3(64 * kCarryWarps), 0, s, c);
    prof_end(h, s);
    if (e != cudaSuccess) return e;
    h = prof_begin(KID_COL_BWD_APPLY, px, fl, s);
    e = launch_ex(col_bwd_apply_kernel<ITEMS, NW, DHALF>, grid, dim3(32 * NW), 0, s, a, c);
    prof_end(h, s);
    return e;
}

template <int ITEMS, bool DHALF>
cudaError_t allow_bwd_clusters() {
    return cudaFuncSetAttribute((const void*)col_bwd_kernel<ITEMS, DHALF>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

}  // namespace

// Backward plans: 8 positions per thread (five arrays of them live at once), 16 for rows over
// 8192 (up to 10240).
bool plan_rows_bwd(int W, RowPlan* p) {
    const int items = W <= 8192 ? 8 : 16;
    int tpr = (W + items - 1) / items;
    if (tpr > (items <= 8 ? 1024 : 640)) return false;
    tpr = (tpr + 31) / 32 * 32;
    int rpb = 256 / tpr;
    if (rpb < 1) rpb = 1;
    p->items = items;
    p->tpr = tpr;
    p->rpb = rpb;
    return true;
}

// chain shapes of the vertical adjoint (rows per thread, warps per CTA), the default first
// (measured on 10000 x 1024: 16 x 16 170 us per pass, 8 x 32 200 us, 8 x 16 229 us; the shorter
// chain of 256-row chunks waits less for the last chunk of its strip)
constexpr int kBwdChainShapes[][2] = {{16, 16}, {8, 16}, {8, 8}, {16, 8}, {8, 32}};

// shapes of the two-phase vertical adjoint (rows per thread, warps per CTA), the default first
constexpr int kBwdSplitShapes[][2] = {{8, 8}, {8, 16}, {16, 8}, {16, 16}, {8, 32}};
constexpr int kBwdClusterMaxRows = 1536;  // the default plan's cluster limit

std::mutex g_tuned_bwd_mutex;
std::map<int, ColPlan> g_tuned_bwd_cols;  // H -> vertical adjoint shape

bool valid_bwd_shape(int H, const ColPlan& p) {
    if (p.cluster == kColChain) {
        for (const auto& c : kBwdChainShapes)
            if (c[0] == p.items && c[1] == p.warps)
                return (H + p.items * p.warps - 1) / (p.items * p.warps) <= kChainMaxChunks;
        return false;
    }
    if (p.cluster == kColSplit) {
        for (const auto& c : kBwdSplitShapes)
            if (c[0] == p.items && c[1] == p.warps)
                return (H + p.items * p.warps - 1) / (p.items * p.warps) <= kChainMaxChunks;
        return false;
    }
    return (p.items == 8 || p.items == 16) && (p.warps == 8 || p.warps == 16) && p.cluster >= 1 &&
           p.cluster <= 16 && (long long)p.items * p.warps * p.cluster >= H;
}

// Backward vertical plan: a tuned shape first (set_tuned_bwd_col); else one cluster for columns
// up to 1536 rows (16 rows x 16 warps in clusters of up to 8 where they fit), the two-phase
// adjoint in 64-row chunks above.  Measured per vertical adjoint pass on GB300 (cluster or chain
// against two-phase): 1024 x 8192 84.4 / 87.5 us, 1536 x 4096 66.3 / 66.5, 1988 x 2880 66.1 /
// 62.8, 2500 x 2500 74.6 / 69.1, 4096 x 4096 218.1 / 148.3, 10000 x 10000 1516.6 (chain) / 789.6.
bool plan_cols_bwd(int H, ColPlan* p) {
    if (H > kMaxColRows) return false;
    {
        std::lock_guard<std::mutex> lock(g_tuned_bwd_mutex);
        auto it = g_tuned_bwd_cols.find(H);
        if (it != g_tuned_bwd_cols.end()) {
            *p = it->second;
            return true;
        }
    }
    static const int cand[][2] = {{16, 16}, {8, 16}, {16, 8}, {8, 8}};
    if (H > kBwdClusterMaxRows) {
        p->items = 8;
        p->warps = 8;
        p->cluster = kColSplit;
        return (H + 63) / 64 <= kChainMaxChunks;
    }
    if (H <= 128) {
        int nw = 1;
        while (nw * 8 < H) nw <<= 1;  // a power of two (the CTA scan works in lane groups)
        p->items = 8;
        p->warps = nw;
        p->cluster = 1;
        return true;
    }
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

// records a vertical adjoint shape for columns of H rows (from dts_autotune_import); false when
// it is not a valid shape for that height
bool set_tuned_bwd_col(int H, const ColPlan& p) {
    if (H < 1 || !valid_bwd_shape(H, p)) return false;
    std::lock_guard<std::mutex> lock(g_tuned_bwd_mutex);
    g_tuned_bwd_cols[H] = p;
    return true;
}

std::string tuned_bwd_export() {
    std::lock_guard<std::mutex> lock(g_tuned_bwd_mutex);
    std::string out;
    char line[96];
    for (auto& kv : g_tuned_bwd_cols) {
        snprintf(line, sizeof(line), "bcol %d %d %d %d\n", kv.first, kv.second.items, kv.second.warps, kv.second.cluster);
        out += line;
    }
    return out;
}

cudaError_t launch_row_bwd(const BwdArgs& a, int dist_half, bool final_pass, const RowPlan& p, cudaStream_t s) {
    const int h = prof_begin(final_pass ? KID_ROW_BWD_FINAL : KID_ROW_BWD, (long long)a.H * a.W,
                             dist_half ? kFlagDistHalf : 0, s);
    cudaError_t e = cudaErrorInvalidValue;
    if (p.items == 8) e = dist_half ? launch_row_bwd_t<8, true>(a, final_pass, p, s) : launch_row_bwd_t<8, false>(a, final_pass, p, s);
    if (p.items == 16)
        e = dist_half ? launch_row_bwd_t<16, true>(a, final_pass, p, s) : launch_row_bwd_t<16, false>(a, final_pass, p, s);
    prof_end(h, s);
    return e;
}

cudaError_t launch_col_bwd(const BwdArgs& a, int dist_half, const ColPlan& p, cudaStream_t s) {
    if (p.cluster == kColSplit) {  // two launches, each timed on its own
        const bool dh = dist_half != 0;
        if (p.items == 8 && p.warps == 16) return dh ? launch_col_bwd_split_t<8, 16, true>(a, s) : launch_col_bwd_split_t<8, 16, false>(a, s);
        if (p.items == 16 && p.warps == 8) return dh ? launch_col_bwd_split_t<16, 8, true>(a, s) : launch_col_bwd_split_t<16, 8, false>(a, s);
        if (p.items == 8 && p.warps == 8) return dh ? launch_col_bwd_split_t<8, 8, true>(a, s) : launch_col_bwd_split_t<8, 8, false>(a, s);
        if (p.items == 16 && p.warps == 16) return dh ? launch_col_bwd_split_t<16, 16, true>(a, s) : launch_col_bwd_split_t<16, 16, false>(a, s);
        if (p.items == 8 && p.warps == 32) return dh ? launch_col_bwd_split_t<8, 32, true>(a, s) : launch_col_bwd_split_t<8, 32, false>(a, s);
        return cudaErrorInvalidValue;
    }
    const int h = prof_begin(p.cluster < 0 ? KID_COL_BWD_CHAIN : KID_COL_BWD, (long long)a.H * a.W,
                             dist_half ? kFlagDistHalf : 0, s);
    cudaError_t e = cudaErrorInvalidValue;
    if (p.cluster < 0) {
        if (p.items == 8 && p.warps == 16)
            e = dist_half ? launch_col_bwd_chain_t<8, 16, true>(a, s) : launch_col_bwd_chain_t<8, 16, false>(a, s);
        if (p.items == 8 && p.warps == 8)
            e = dist_half ? launch_col_bwd_chain_t<8, 8, true>(a, s) : launch_col_bwd_chain_t<8, 8, false>(a, s);
        if (p.items == 16 && p.warps == 8)
            e = dist_half ? launch_col_bwd_chain_t<16, 8, true>(a, s) : launch_col_bwd_chain_t<16, 8, false>(a, s);
        if (p.items == 8 && p.warps == 32)
            e = dist_half ? launch_col_bwd_chain_t<8, 32, true>(a, s) : launch_col_bwd_chain_t<8, 32, false>(a, s);
        if (p.items == 16 && p.warps == 16)
            e = dist_half ? launch_col_bwd_chain_t<16, 16, true>(a, s) : launch_col_bwd_chain_t<16, 16, false>(a, s);
    } else {
        if (p.items == 8) e = dist_half ? launch_col_bwd_t<8, true>(a, p, s) : launch_col_bwd_t<8, false>(a, p, s);
        if (p.items == 16) e = dist_half ? launch_col_bwd_t<16, true>(a, p, s) : launch_col_bwd_t<16, false>(a, p, s);
    }
    prof_end(h, s);
    return e;
}

cudaError_t launch_guide_grad(const GuideGradArgs& a, cudaStream_t s) {
    const dim3 block(256);
    cudaError_t e;
    // four pixels per thread where every plane's rows are whole, aligned 16-byte units (8-byte
    // for a 16-bit guide)
    const size_t gsz = a.gdtype == DTS_F32 ? 4 : 2;
    auto al = [](const void* p, size_t n) { return (uintptr_t)p % n == 0; };
    const bool vec = a.W % 4 == 0 && a.pitch % 4 == 0 && a.row_stride % 4 == 0 && a.ch_stride % 4 == 0 &&
                     al(a.guide, 4 * gsz) && al(a.dXb, 16) && al(a.dYb, 16) && al(a.out, 16);
    const int h = prof_begin(vec ? KID_GUIDE_GRAD4 : KID_GUIDE_GRAD, (long long)a.H * a.W, a.dhalf ? kFlagDistHalf : 0, s);
    if (vec) {
        const dim3 grid4((unsigned)((a.W / 4 + 255) / 256), (unsigned)a.H);
        if (a.dhalf) {
            if (a.gdtype == DTS_BF16) e = launch_ex(guide_grad4_kernel<__nv_bfloat16, true>, grid4, block, 0, s, a);
            else if (a.gdtype == DTS_F16) e = launch_ex(guide_grad4_kernel<__half, true>, grid4, block, 0, s, a);
            else e = launch_ex(guide_grad4_kernel<float, true>, grid4, block, 0, s, a);
        } else {
            if (a.gdtype == DTS_BF16) e = launch_ex(guide_grad4_kernel<__nv_bfloat16, false>, grid4, block, 0, s, a);
            else if (a.gdtype == DTS_F16) e = launch_ex(guide_grad4_kernel<__half, false>, grid4, block, 0, s, a);
            else e = launch_ex(guide_grad4_kernel<float, false>, grid4, block, 0, s, a);
        }
        prof_end(h, s);
        return e;
    }
    const dim3 grid((unsigned)((a.W + 255) / 256), (unsigned)a.H);
    if (a.dhalf) {
        if (a.gdtype == DTS_BF16) e = launch_ex(guide_grad_kernel<__nv_bfloat16, true>, grid, block, 0, s, a);
        else if (a.gdtype == DTS_F16) e = launch_ex(guide_grad_kernel<__half, true>, grid, block, 0, s, a);
        else e = launch_ex(guide_grad_kernel<float, true>, grid, block, 0, s, a);
    } else {
        if (a.gdtype == DTS_BF16) e = launch_ex(guide_grad_kernel<__nv_bfloat16, false>, grid, block, 0, s, a);
        else if (a.gdtype == DTS_F16) e = launch_ex(guide_grad_kernel<__half, false>, grid, block, 0, s, a);
        else e = launch_ex(guide_grad_kernel<float, false>, grid, block, 0, s, a);
    }
    prof_end(h, s);
    return e;
}

cudaError_t launch_update_adjoint(const BwdArgs& a, cudaStream_t s) {
    const int h = prof_begin(KID_UPDATE_ADJ, (long long)a.H * a.W, a.t_dtype != DTS_F32 ? kFlagTarget16 : 0, s);
    const dim3 grid((unsigned)((a.W + 1023) / 1024), (unsigned)a.H);
    auto al16 = [](const void* p) { return (uintptr_t)p % 16 == 0; };
    const bool vec = a.W % 4 == 0 && a.pitch % 4 == 0 && al16(a.gz) && al16(a.c) && al16(a.x) && al16(a.zk) &&
                     al16(a.gout) && (!a.gt || al16(a.gt)) && (!a.gc || al16(a.gc));
    const cudaError_t e = vec ? launch_ex(update_adjoint_kernel<true>, grid, dim3(256), 0, s, a)
                              : launch_ex(update_adjoint_kernel<false>, grid, dim3(256), 0, s, a);
    prof_end(h, s);
    return e;
}

cudaError_t launch_axpy_plane(const float* src, long long sp, float* dst, long long dp, int H, int W, int accumulate,
                              cudaStream_t s) {
    const int h = prof_begin(KID_AXPY, (long long)H * W, 0, s);
    const dim3 block(256);
    auto al16 = [](const void* p) { return (uintptr_t)p % 16 == 0; };
    cudaError_t e;
    if (W % 4 == 0 && sp % 4 == 0 && dp % 4 == 0 && al16(src) && al16(dst))
        e = launch_ex(axpy_plane_kernel<true>, dim3((unsigned)((W / 4 + 255) / 256), (unsigned)H), block, 0, s, src, sp,
                      dst, dp, H, W, accumulate);
    else
        e = launch_ex(axpy_plane_kernel<false>, dim3((unsigned)((W + 255) / 256), (unsigned)H), block, 0, s, src, sp, dst,
                      dp, H, W, accumulate);
    prof_end(h, s);
    return e;
}

cudaError_t prepare_backward_kernels() {
    cudaError_t e = cudaSuccess, r;
    if ((r = allow_bwd_clusters<8, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_clusters<8, true>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_clusters<16, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_clusters<16, true>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<8, 16, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<8, 16, true>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<8, 8, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<8, 8, true>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<16, 8, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<16, 8, true>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<8, 32, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<8, 32, true>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<16, 16, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_chain_smem<16, 16, true>()) != cudaSuccess) e = r;
    return e;
}

}  // namespace dts
