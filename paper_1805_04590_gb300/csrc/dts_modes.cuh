// The line modes of the pass kernels (what a segment of a line carries through an exchange, and
// how it replays its positions given its carries) and the exchange of the strip kernels, shared
// by the single-image pass kernels (dts_forward.cu) and the persistent batched solve
// (dts_batched.cu).
#pragma once

#include "dts_scan.cuh"

namespace dts {
namespace scan {

// ---------------------------------------------------------------- modes
// Normalised pass: causal sweep, then the anti-causal sweep on its result.
struct CoupledMode {
    using Pre = Aff;
    using Suf = Coupled;
    static __device__ __forceinline__ Pre pre_identity() { return aff_identity(); }
    static __device__ __forceinline__ Pre pre_compose(const Pre& f, const Pre& s) { return aff_compose(f, s); }
    static __device__ __forceinline__ Suf suf_identity() { return coupled_identity(); }
    static __device__ __forceinline__ Suf suf_compose(const Suf& f, const Suf& s) { return coupled_compose(f, s); }
    template <int N>
    static __device__ __forceinline__ void local(const float (&x)[N], const float (&w)[N], float wn, Pre& pre,
                                                 Suf& suf) {
        suf = coupled_local<true>(x, w, wn);
        pre = Aff{suf.A, suf.B};
    }
    // c: causal value entering on the left; after: composition of every segment to the right
    template <int N>
    static __device__ __forceinline__ void apply(float (&x)[N], const float (&w)[N], float wn, const Pre& own,
                                                 float c, const Suf& after) {
        float J = c;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            J = fmaf(w[j], J - x[j], x[j]);
            x[j] = J;
        }
        float K = k_entering(after, fmaf(own.A, c, own.B));
#pragma unroll
        for (int j = N - 1; j >= 0; --j) {
            const float wp = (j + 1 < N) ? w[j + 1] : wn;
            K = fmaf(wp, K - x[j], x[j]);
            x[j] = K;
        }
    }
};

// Transpose of a normalised pass.  The pass is (anti-causal) o (causal) with causal = L^-1 D,
// D = diag(1 - w_n), L unit lower bidiagonal with -w_n below the diagonal, and anti-causal
// = U^-1 D' with D' = diag(1 - w_{n+1}), U unit upper bidiagonal with -w_{n+1} above it.  Its
// transpose D L^-T D' U^-T is: the unnormalised causal sweep h[n] = g[n] + w_n h[n-1], then the
// normalised anti-causal sweep on h, then a factor (1 - w_n) per position.  The first two have
// the coupled five-number form with an unnormalised left-to-right recurrence.
struct TransposeMode {
    using Pre = Aff;
    using Suf = Coupled;
    static __device__ __forceinline__ Pre pre_identity() { return aff_identity(); }
    static __device__ __forceinline__ Pre pre_compose(const Pre& f, const Pre& s) { return aff_compose(f, s); }
    static __device__ __forceinline__ Suf suf_identity() { return coupled_identity(); }
    static __device__ __forceinline__ Suf suf_compose(const Suf& f, const Suf& s) { return coupled_compose(f, s); }
    template <int N>
    static __device__ __forceinline__ void local(const float (&x)[N], const float (&w)[N], float wn, Pre& pre,
                                                 Suf& suf) {
        suf = coupled_local<false>(x, w, wn);
        pre = Aff{suf.A, suf.B};
    }
    template <int N>
    static __device__ __forceinline__ void apply(float (&x)[N], const float (&w)[N], float wn, const Pre& own,
                                                 float c, const Suf& after) {
        float h = c;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            h = fmaf(w[j], h, x[j]);
            x[j] = h;
        }
        float K = k_entering(after, fmaf(own.A, c, own.B));
#pragma unroll
        for (int j = N - 1; j >= 0; --j) {
            const float wp = (j + 1 < N) ? w[j + 1] : wn;
            K = fmaf(wp, K - x[j], x[j]);
            x[j] = fmaf(-w[j], K, K);
        }
    }
};

// Support of the unnormalised kernel (confidence weighting): causal P[n] = x[n] + w_n P[n-1] and
// anti-causal Q[n] = x[n] + w'_n Q[n+1], both on x; the result is P + Q - x.  The two sweeps are
// independent: Suf carries (al, de) with Q_start = al Q_in + de.
struct SupSuf {
    float al, de;
};
struct SupportMode {
    using Pre = Aff;
    using Suf = SupSuf;
    static __device__ __forceinline__ Pre pre_identity() { return aff_identity(); }
    static __device__ __forceinline__ Pre pre_compose(const Pre& f, const Pre& s) { return aff_compose(f, s); }
    static __device__ __forceinline__ Suf suf_identity() { return Suf{1.f, 0.f}; }
    static __device__ __forceinline__ Suf suf_compose(const Suf& f, const Suf& s) {
        return Suf{f.al * s.al, fmaf(f.al, s.de, f.de)};
    }
    template <int N>
    static __device__ __forceinline__ void local(const float (&x)[N], const float (&w)[N], float wn, Pre& pre,
                                                 Suf& suf) {
        float A = 1.f, B = 0.f, r = 1.f, de = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            A *= w[j];
            B = fmaf(w[j], B, x[j]);
            de = fmaf(r, x[j], de);
            r *= (j + 1 < N) ? w[j + 1] : wn;
        }
        pre = Aff{A, B};
        suf = Suf{r, de};
    }
    template <int N>
    static __device__ __forceinline__ void apply(float (&x)[N], const float (&w)[N], float wn, const Pre& own,
                                                 float c, const Suf& after) {
        (void)own;
        float Pv[N];
        float Pc = c;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            Pc = fmaf(w[j], Pc, x[j]);
            Pv[j] = Pc;
        }
        float Qc = after.de;
#pragma unroll
        for (int j = N - 1; j >= 0; --j) {
            const float wp = (j + 1 < N) ? w[j + 1] : wn;
            Qc = fmaf(wp, Qc, x[j]);
            x[j] = Pv[j] + Qc - x[j];
        }
    }
};

// ---------------------------------------------------------------- strip vertical pass (no cluster)
// CTA = NW <= 32 warps over a strip of 8 columns and the whole column height.  Lane l of warp q
// takes column l % 8 and segment 4q + l / 8 (ITEMS rows each): 4 NW segments per column.
// Exchange: the 4 segments of a column inside a warp scan with shuffles at stride 8; the NW warp
// totals of a column scan in one warp (lane = warp); two __syncthreads, no cluster barrier.
constexpr int kStripCols = 8;
constexpr int kStripWarps = 32;

template <class M>
struct StripShared {
    typename M::Pre pre[kStripWarps][kStripCols + 1];
    typename M::Suf suf[kStripWarps][kStripCols + 1];
};

// pre / suf: the transforms of everything above / below this thread's segment in its column.
// Shared-memory writes made before the call are visible to every thread after it.
template <class M>
__device__ __forceinline__ void strip_exchange(const typename M::Pre& own_pre, const typename M::Suf& own_suf,
                                               int lane, int warp, int NW, int cl, int sw, StripShared<M>& sh,
                                               typename M::Pre& pre, typename M::Suf& suf) {
    using Pre = typename M::Pre;
    using Suf = typename M::Suf;
    constexpr int SEGS = 32 / kStripCols;
    // inside the warp: the column's segments are lanes cl, cl + 8, cl + 16, cl + 24
    Pre ip = own_pre;
    Suf is = own_suf;
#pragma unroll
    for (int off = 1; off < SEGS; off <<= 1) {
        const Pre op = shfl_up_t(ip, off * kStripCols);
        const Suf os = shfl_down_t(is, off * kStripCols);
        if (sw >= off) ip = M::pre_compose(op, ip);
        if (sw + off < SEGS) is = M::suf_compose(is, os);
    }
    Pre xp = shfl_up_t(ip, kStripCols);
    Suf xs = shfl_down_t(is, kStripCols);
    if (sw == 0) xp = M::pre_identity();
    if (sw == SEGS - 1) xs = M::suf_identity();
    if (sw == SEGS - 1) sh.pre[warp][cl] = ip;  // warp total, prefix direction
    if (sw == 0) sh.suf[warp][cl] = is;         // warp total, suffix direction
    __syncthreads();
    // across the warps: warp c < 8 (or every warp of a smaller CTA, in turn) scans column c over
    // the NW warp totals (lane = warp)
    for (int c = warp; c < kStripCols; c += NW) {
        const bool in = lane < NW;
        const Pre p = in ? sh.pre[lane][c] : M::pre_identity();
        const Suf f = in ? sh.suf[lane][c] : M::suf_identity();
        const Pre ip2 = warp_scan_pre<M>(p, lane);
        const Suf is2 = warp_scan_suf<M>(f, lane);
        Pre pe = shfl_up_t(ip2, 1);
        Suf fe = shfl_down_t(is2, 1);
        if (lane == 0) pe = M::pre_identity();
        if (lane == 31) fe = M::suf_identity();
        if (in) {
            sh.pre[lane][c] = pe;
            sh.suf[lane][c] = fe;
        }
    }
    __syncthreads();
    pre = M::pre_compose(sh.pre[warp][cl], xp);
    suf = M::suf_compose(xs, sh.suf[warp][cl]);
}

// ---------------------------------------------------------------- pass bodies
// The horizontal pass and the plain-load strip pass as device functions over one unit of work
// (a group of rows, an 8-column strip): the single-image kernels run one unit per CTA, the
// persistent batched solve runs units of every image from its work queue.
// four consecutive target / confidence values at dense index i (16-byte vectors when allowed)
__device__ __forceinline__ void load4_t(const PassArgs& a, long long i, bool vec, float* out) {
    if (vec) {
        if (a.t_dtype == DTS_F32) {
            load4_f(static_cast<const float*>(a.t), i, out);
        } else {
            const uint2 v = *reinterpret_cast<const uint2*>(static_cast<const unsigned short*>(a.t) + i);
            const unsigned short h[4] = {(unsigned short)(v.x & 0xffff), (unsigned short)(v.x >> 16),
                                         (unsigned short)(v.y & 0xffff), (unsigned short)(v.y >> 16)};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                out[k] = a.t_dtype == DTS_BF16 ? __bfloat162float(__ushort_as_bfloat16(h[k]))
                                               : __half2float(__ushort_as_half(h[k]));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = load_any(a.t, i + k, a.t_dtype);
    }
}

// TWO: the normalised pass as two one-direction exchanges of affine maps (causal, then
// anti-causal on its result) instead of one exchange of the coupled five numbers.
// The pass over the rpb rows of row group `group` (CTA thread t: row t / tpr of the group,
// positions [(t % tpr) ITEMS, + ITEMS) of it; threads beyond rpb tpr take no row).  CG: the
// planes that the same launch rewrites (the pass input, z_k) are read through L2 only, for a
// kernel whose CTAs run stage after stage (an SM's L1 may hold an earlier stage's lines).
template <int ITEMS, bool DHALF, int KIND, bool TWO, bool CG>
__device__ __forceinline__ void row_pass_body(const PassArgs& a, int tpr, int rpb, int group) {
    static_assert(ITEMS % 4 == 0, "ITEMS must be a multiple of 4");
    using M = typename std::conditional<KIND == PASS_SUPPORT, SupportMode,
                                        typename std::conditional<KIND == PASS_TRANSPOSE, TransposeMode,
                                                                  CoupledMode>::type>::type;
    __shared__ typename M::Pre s_pre[32];
    __shared__ typename M::Suf s_suf[32];
    __shared__ Aff s_two[TWO ? 32 : 1];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int rloc = tid / tpr;
    const int t = tid - rloc * tpr;
    const int wpr = tpr >> 5;       // warps per row
    const int wrow = t >> 5;        // warp index within the row
    const int wbase = warp - wrow;  // first warp of this row
    const int row = group * rpb + rloc;
    const bool row_ok = rloc < rpb && row < a.H;
    const int e0 = t * ITEMS;
    const long long P = a.pitch;
    const long long base = (long long)row * P + e0;
    const bool live = row_ok && e0 < P;

    if constexpr (KIND == PASS_UPDATE_ROW) {
        // the update operands are read group by group between stores of z_{k+1}: start bringing
        // this thread's lines into L2 now
        if (row_ok && e0 < a.W) {  // addresses inside the dense planes only
            const long long di = (long long)row * a.W + e0;
            prefetch_l2(a.zk + base);
            prefetch_l2(static_cast<const char*>(a.t) + di * (a.t_dtype == DTS_F32 ? 4 : 2));
            prefetch_l2(a.c + (a.c_pitched ? base : di));
        }
    }
    float x[ITEMS], w[ITEMS];
    if (live) {
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            if constexpr (KIND == PASS_SUPPORT) {
                x[4 * q] = x[4 * q + 1] = x[4 * q + 2] = x[4 * q + 3] = 1.f;
            } else {
                load4_p<CG>(a.src, base + 4 * q, &x[4 * q]);
            }
            load4_d<DHALF>(a.d, base + 4 * q, &w[4 * q]);
        }
        if constexpr (KIND == PASS_UPDATE_ROW) {
            // z_{k+1} from z_k, zbar (already in x), t and c; padding positions stay 0.  Every
            // operand is loaded before the first store of z_{k+1} (the stores could alias later
            // loads, which would otherwise wait for them); the update is computed in place in x.
            const long long di = (long long)row * a.W + e0;
            const bool full_seg = e0 + ITEMS <= a.W;
            // operands in groups of HALF positions (a group's loads, its update, its stores): 8 at
            // 16 positions per thread (measured: 37.0 us vs 37.5 with 4 and 40.7 with all 16 at
            // once, which costs resident rows), 16 at 32 (rows over 8192)
            constexpr int HALF = ITEMS <= 16 ? 8 : ITEMS / 2;
#pragma unroll
            for (int h0 = 0; h0 < ITEMS; h0 += HALF) {
            float zk[HALF], tt[HALF], cc[HALF];
#pragma unroll
            for (int q = h0 / 4; q < (h0 + HALF) / 4; ++q) {
                const int l = 4 * q - h0;
                load4_p<CG>(a.zk, base + 4 * q, &zk[l]);
                if (full_seg) {
                    load4_t(a, di + 4 * q, a.tc_vec, &tt[l]);
                    if (a.c_pitched) load4_f(a.c, base + 4 * q, &cc[l]);
                    else if (a.tc_vec) load4_f(a.c, di + 4 * q, &cc[l]);
                    else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) cc[l + k] = a.c[di + 4 * q + k];
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool ok = e0 + 4 * q + k < a.W;
                        tt[l + k] = ok ? load_any(a.t, di + 4 * q + k, a.t_dtype) : 0.f;
                        cc[l + k] = ok ? (a.c_pitched ? a.c[base + 4 * q + k] : a.c[di + 4 * q + k]) : 0.f;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                const float zn = dts_update_value(zk[j], x[h0 + j], tt[j], cc[j], a.lambda, a.step, a.update,
                                                  a.clamp_step, a.eps);
                x[h0 + j] = (e0 + h0 + j < a.W) ? zn : 0.f;
            }
#pragma unroll
            for (int q = h0 / 4; q < (h0 + HALF) / 4; ++q) store4_f(a.zout, base + 4 * q, &x[4 * q]);
            }
        }
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) w[j] = ex2(a.k2 * w[j]);
        if (e0 + ITEMS > a.W) {  // the segment holding the row end: clear the padding
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (e0 + j >= a.W) x[j] = w[j] = 0.f;
        }
        if (e0 == 0) w[0] = 0.f;  // the row starts here
    } else {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) x[j] = w[j] = 0.f;
    }
    // weight between this segment's last position and the next segment's first
    float wn = __shfl_down_sync(kFull, w[0], 1);
    if (lane == 31) {
        const int en = e0 + ITEMS;
        wn = (row_ok && en < a.W) ? ex2(a.k2 * load1_d<DHALF>(a.d, (long long)row * P + en)) : 0.f;
    }

    if constexpr (TWO && KIND != PASS_SUPPORT) {
        // causal sweep: segment map c -> A c + B, exclusive prefix, replay
        float A = 1.f, B = 0.f;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            A *= w[j];
            B = fmaf(w[j], B - x[j], x[j]);
        }
        const Aff pc = row_scan_aff<true>(Aff{A, B}, lane, warp, wrow, wbase, wpr, s_pre);
        float v = pc.B;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            v = fmaf(w[j], v - x[j], x[j]);
            x[j] = v;
        }
        // anti-causal sweep on the result, weights w' (the next position's)
        A = 1.f;
        B = 0.f;
#pragma unroll
        for (int j = ITEMS - 1; j >= 0; --j) {
            const float wp = (j + 1 < ITEMS) ? w[j + 1] : wn;
            A *= wp;
            B = fmaf(wp, B - x[j], x[j]);
        }
        const Aff sk = row_scan_aff<false>(Aff{A, B}, lane, warp, wrow, wbase, wpr, s_two);
        release_successor();
        v = sk.B;
#pragma unroll
        for (int j = ITEMS - 1; j >= 0; --j) {
            const float wp = (j + 1 < ITEMS) ? w[j + 1] : wn;
            v = fmaf(wp, v - x[j], x[j]);
            x[j] = v;
        }
    } else {
        typename M::Pre own_pre, pre;
        typename M::Suf own_suf, suf;
        M::local(x, w, wn, own_pre, own_suf);
        row_exchange<M>(own_pre, own_suf, lane, warp, wrow, wbase, wpr, s_pre, s_suf, pre, suf);
        release_successor();
        M::apply(x, w, wn, own_pre, pre.B, suf);
    }

    if (live) {
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) store4_f(a.dst, base + 4 * q, &x[4 * q]);
    }
}

// The strip algorithm with plain loads (each warp load covers four 32-byte row pieces) on 8-column
// strip `strip`; the CTA's NW warps hold 4 NW segments of ITEMS rows of every column.  CG: the
// pass input is read through L2 only (see row_pass_body).
template <int ITEMS, bool DHALF, bool CG>
__device__ __forceinline__ void strip_pass_body(const PassArgs& a, int strip) {
    using M = CoupledMode;
    using DT = typename std::conditional<DHALF, __half, float>::type;
    __shared__ StripShared<M> sh;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int NW = blockDim.x >> 5;
    const int cl = lane & (kStripCols - 1);  // column within the strip
    const int sw = lane / kStripCols;        // segment within the warp (0..3)
    const int col = strip * kStripCols + cl;
    const bool col_ok = col < a.W;
    const int row0 = (warp * (32 / kStripCols) + sw) * ITEMS;
    const long long P = a.pitch;

    float x[ITEMS], w[ITEMS];
    const bool full = col_ok && row0 + ITEMS <= a.H;
    {
        const float* ps = a.src + (long long)row0 * P + col;
        const DT* pd = static_cast<const DT*>(a.d) + (long long)row0 * P + col;
        if (full) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                x[j] = load1_p<CG>(ps);
                w[j] = to_f32<DT>(*pd);
                ps += P;
                pd += P;
            }
        } else {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const bool ok = col_ok && row0 + j < a.H;
                x[j] = ok ? load1_p<CG>(ps) : 0.f;
                w[j] = ok ? to_f32<DT>(*pd) : 0.f;
                ps += P;
                pd += P;
            }
        }
    }
    float wn;
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
    if (row0 == 0) w[0] = 0.f;

    typename M::Pre own_pre, pre;
    typename M::Suf own_suf, suf;
    M::local(x, w, wn, own_pre, own_suf);
    strip_exchange<M>(own_pre, own_suf, lane, warp, NW, cl, sw, sh, pre, suf);
    release_successor();
    M::apply(x, w, wn, own_pre, pre.B, suf);

    float* pdst = a.dst + (long long)row0 * a.dst_pitch + col;
    if (full) {
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
}

}  // namespace scan
}  // namespace dts
