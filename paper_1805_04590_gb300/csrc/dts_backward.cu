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
// Same layout as the forward vertical pass (lane = column, one cluster per 32-column strip).
// Columns taller than one cluster are cut into chunks of CS x NW x ITEMS rows, one cluster each
// (grid.y = CS x chunks).  Then the pass runs twice: chunk mode 1 writes each chunk's total
// transforms (prefix and suffix direction) to a.tot; chunk mode 2 composes the totals of the
// chunks above and below into every segment's carries and replays.  Mode 0: a single chunk.
template <int ITEMS>
constexpr int bwd_col_max_threads() {
    return 512;
}
inline int bwd_col_max_threads_host(int) { return 512; }

// two resident CTAs of the 8-row shape (64 registers)
template <int ITEMS>
constexpr int bwd_col_min_blocks() {
    return ITEMS <= 8 ? 2 : 1;
}

// chunk totals in a.tot: plane f of chunk c at (c * kTotFields + f) * tot_pitch
constexpr int kTotFields = 9;  // prefix: 2 x (A, B); suffix: (A, B, al, be, ga)

__device__ __forceinline__ void store_tot_pre(const BwdArgs& a, int chunk, int col, const Pre2& p) {
    float* t = a.tot + (long long)chunk * kTotFields * a.tot_pitch + col;
    const long long q = a.tot_pitch;
    t[0] = p.jk.A;
    t[q] = p.jk.B;
    t[2 * q] = p.hg.A;
    t[3 * q] = p.hg.B;
}
__device__ __forceinline__ void store_tot_suf(const BwdArgs& a, int chunk, int col, const Coupled& f) {
    float* t = a.tot + (long long)chunk * kTotFields * a.tot_pitch + col + 4 * a.tot_pitch;
    const long long q = a.tot_pitch;
    t[0] = f.A;
    t[q] = f.B;
    t[2 * q] = f.al;
    t[3 * q] = f.be;
    t[4 * q] = f.ga;
}
__device__ __forceinline__ Pre2 load_tot_pre(const BwdArgs& a, int chunk, int col) {
    const float* t = a.tot + (long long)chunk * kTotFields * a.tot_pitch + col;
    return Pre2{Aff{t[0], t[a.tot_pitch]}, Aff{t[2 * a.tot_pitch], t[3 * a.tot_pitch]}};
}
__device__ __forceinline__ Coupled load_tot_suf(const BwdArgs& a, int chunk, int col) {
    const float* t = a.tot + (long long)chunk * kTotFields * a.tot_pitch + col + 4 * a.tot_pitch;
    const long long q = a.tot_pitch;
    return Coupled{t[0], t[q], t[2 * q], t[3 * q], t[4 * q]};
}

template <int ITEMS, bool DHALF, bool FOLD = false, bool CHUNKED = false>
__global__ void __launch_bounds__(bwd_col_max_threads<ITEMS>(), bwd_col_min_blocks<ITEMS>()) col_bwd_kernel(BwdArgs a) {
    using M = BackwardMode;
    __shared__ ColShared<M, 16> sh;
    cg::cluster_group cluster = cg::this_cluster();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const int rank = (int)cluster.block_rank();
    const int CS = (int)cluster.num_blocks();
    const int chunk = CHUNKED ? (int)blockIdx.y / CS : 0;
    const int col = blockIdx.x * 32 + lane;
    const bool col_ok = col < a.W;
    const int row0 = ((chunk * CS + rank) * NW + warp) * ITEMS;
    const long long P = a.pitch;

    wait_predecessor();
    // the distance gradient is read-modified-written at the end: lane j brings row j of the
    // warp's rows into L2 now (one 128-byte line per row of the strip)
    if (lane < ITEMS && row0 + lane < a.H && blockIdx.x * 32 < a.W)
        prefetch_l2(a.dbar + (long long)(row0 + lane) * P + blockIdx.x * 32);
    float x[ITEMS], w[ITEMS], G[ITEMS], K[ITEMS];
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
    float wn;
    {
        const int rn = row0 + ITEMS;
        wn = (col_ok && rn < a.H) ? ex2(a.k2 * load1_d<DHALF>(a.d, (long long)rn * P + col)) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int r = row0 + j;
        w[j] = (col_ok && r > 0 && r < a.H) ? ex2(a.k2 * w[j]) : 0.f;
    }

    M::Pre own_pre, pre;
    M::Suf own_suf, suf;
    adjoint_local(x, w, wn, G, own_pre, own_suf);
    if constexpr (FOLD) col_exchange<M, 16>(own_pre, own_suf, lane, warp, NW, sh, pre, suf);
    else col_exchange_scan<M, 16>(own_pre, own_suf, lane, warp, NW, sh, pre, suf);
    release_successor();
    if (CHUNKED && a.chunk_mode == 1) {
        // this chunk's totals: the inclusive prefix at its last segment, the inclusive suffix at
        // its first
        if (col_ok && rank == CS - 1 && warp == NW - 1) store_tot_pre(a, chunk, col, M::pre_compose(pre, own_pre));
        if (col_ok && rank == 0 && warp == 0) store_tot_suf(a, chunk, col, M::suf_compose(own_suf, suf));
        cluster_exit();
        return;
    }
    if (CHUNKED && a.chunk_mode == 2 && col_ok) {
        M::Pre ep = M::pre_identity();
        for (int c = 0; c < chunk; ++c) ep = M::pre_compose(ep, load_tot_pre(a, c, col));
        M::Suf es = M::suf_identity();
        for (int c = a.nchunks - 1; c > chunk; --c) es = M::suf_compose(load_tot_suf(a, c, col), es);
        pre = M::pre_compose(ep, pre);
        suf = M::suf_compose(suf, es);
    }
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
    cluster_exit();
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
    float g[4], cf[4], t[4], zz[4], gt[4] = {0.f, 0.f, 0.f, 0.f}, gc[4] = {0.f, 0.f, 0.f, 0.f};
    if (VEC) {
        load4_f(a.gz, idx, g);
        load4_f(a.c, di, cf);
        load4_f(jac ? a.x : a.zk, idx, zz);
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
            t[k] = ok ? load_any(a.t, di + k, a.t_dtype) : 0.f;
            if (a.gt && ok) gt[k] = a.gt[di + k];
            if (a.gc && ok) gc[k] = a.gc[di + k];
        }
    }
    float dzb[4], dz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (jac) {
            const float den = a.lambda + cf[k];
            if (den != 0.f) {
                dzb[k] = a.lambda / den * g[k];
                gt[k] += cf[k] / den * g[k];
                gc[k] += a.lambda * (t[k] - zz[k]) / (den * den) * g[k];
                dz[k] = 0.f;
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
__global__ void __launch_bounds__(256) axpy_plane_kernel(const float* src, long long sp, float* dst, long long dp,
                                                         int H, int W, int accumulate) {
    wait_predecessor();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const float v = src[(long long)y * sp + x];
    float* d = dst + (long long)y * dp + x;
    *d = accumulate ? *d + v : v;
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
    const int rows = ITEMS * p.warps * p.cluster;  // one chunk
    const int nch = (a.H + rows - 1) / rows;
    const dim3 grid((unsigned)((a.W + 31) / 32), (unsigned)(p.cluster * nch), 1);
    const dim3 block((unsigned)(32 * p.warps));
    static const bool fold = getenv("DTS_BWD_FOLD") != nullptr;  // tuning aid
    if (nch == 1) {
        auto kernel = fold ? col_bwd_kernel<ITEMS, DHALF, true> : col_bwd_kernel<ITEMS, DHALF, false>;
        BwdArgs b = a;
        b.chunk_mode = 0;
        return launch_ex(kernel, grid, block, p.cluster, s, b);
    }
    if (!a.tot || a.tot_chunks < nch) return cudaErrorInvalidValue;
    auto kernel = col_bwd_kernel<ITEMS, DHALF, false, true>;
    BwdArgs b = a;
    b.nchunks = nch;
    b.chunk_mode = 1;
    cudaError_t e = launch_ex(kernel, grid, block, p.cluster, s, b);
    if (e != cudaSuccess) return e;
    b.chunk_mode = 2;
    return launch_ex(kernel, grid, block, p.cluster, s, b);
}

template <int ITEMS, bool DHALF>
cudaError_t allow_bwd_clusters() {
    cudaError_t e = cudaSuccess;
    const void* fs[3] = {(const void*)col_bwd_kernel<ITEMS, DHALF, false>, (const void*)col_bwd_kernel<ITEMS, DHALF, true>,
                         (const void*)col_bwd_kernel<ITEMS, DHALF, false, true>};
    for (const void* f : fs) {
        const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (r != cudaSuccess) e = r;
    }
    return e;
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

// Backward vertical plan (CTA at most bwd_col_max_threads): one cluster for columns up to 4096
// rows, chunks of 2048 rows above (bwd_col_chunks).
bool plan_cols_bwd(int H, ColPlan* p) {
    // DTS_BWD_COL_PLAN="items,warps" overrides the shape (tuning aid)
    static const char* env = getenv("DTS_BWD_COL_PLAN");
    if (env) {
        int it = 0, nw = 0;
        if (sscanf(env, "%d,%d", &it, &nw) == 2 && (it == 8 || it == 16) && nw >= 1 && (nw & (nw - 1)) == 0 &&
            nw * 32 <= bwd_col_max_threads_host(it)) {
            const int cs = (H + it * nw - 1) / (it * nw);
            if (cs <= 16) {
                p->items = it;
                p->warps = nw;
                p->cluster = cs;
                return true;
            }
        }
    }
    // measured on the 2880 x 1988 stereo workload: 16 rows x 16 warps (clusters of 8) is fastest
    static const int cand[][2] = {{16, 16}, {8, 16}, {16, 8}, {8, 8}};
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
    // taller columns: chunks of 2048 rows (16 x 16 x 8), two launches per pass
    if (H <= kBwdMaxRows) {
        p->items = 16;
        p->warps = 16;
        p->cluster = 8;
        return true;
    }
    return false;
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

int bwd_col_chunks(int H) {
    ColPlan p;
    if (!plan_cols_bwd(H, &p)) return 0;
    const int rows = p.items * p.warps * p.cluster;
    const int n = (H + rows - 1) / rows;
    return n > 1 ? n : 0;
}

cudaError_t launch_col_bwd(const BwdArgs& a, int dist_half, const ColPlan& p, cudaStream_t s) {
    const int h = prof_begin(KID_COL_BWD, (long long)a.H * a.W, dist_half ? kFlagDistHalf : 0, s);
    cudaError_t e = cudaErrorInvalidValue;
    if (p.items == 8) e = dist_half ? launch_col_bwd_t<8, true>(a, p, s) : launch_col_bwd_t<8, false>(a, p, s);
    if (p.items == 16) e = dist_half ? launch_col_bwd_t<16, true>(a, p, s) : launch_col_bwd_t<16, false>(a, p, s);
    prof_end(h, s);
    return e;
}

cudaError_t launch_guide_grad(const GuideGradArgs& a, cudaStream_t s) {
    const int h = prof_begin(KID_GUIDE_GRAD, (long long)a.H * a.W, a.dhalf ? kFlagDistHalf : 0, s);
    const dim3 block(256);
    const dim3 grid((unsigned)((a.W + 255) / 256), (unsigned)a.H);
    cudaError_t e;
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
    const dim3 grid((unsigned)((W + 255) / 256), (unsigned)H);
    const cudaError_t e = launch_ex(axpy_plane_kernel, grid, block, 0, s, src, sp, dst, dp, H, W, accumulate);
    prof_end(h, s);
    return e;
}

cudaError_t prepare_backward_kernels() {
    cudaError_t e = cudaSuccess, r;
    if ((r = allow_bwd_clusters<8, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_clusters<8, true>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_clusters<16, false>()) != cudaSuccess) e = r;
    if ((r = allow_bwd_clusters<16, true>()) != cudaSuccess) e = r;
    return e;
}

}  // namespace dts
