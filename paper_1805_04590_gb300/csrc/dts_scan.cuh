// Segment algebra and line exchanges shared by the forward and backward pass kernels.
//
// A pass (forward or adjoint) runs two first-order recurrences along every line: one from left
// to right and one from right to left on the result of the first.  A thread owns a segment of
// consecutive positions.  With c the value entering the segment from the left and k the value
// entering from the right, any such pair satisfies
//     c_out   = A c + B                      (left-to-right value leaving on the right)
//     k_start = al k + be c + ga             (right-to-left value at the segment's first position)
// and these five numbers of adjacent groups compose associatively (coupled_compose).  A "mode"
// bundles what one exchange carries:
//     Pre          what the exclusive prefix needs (the left-to-right maps)
//     Suf          what the exclusive suffix needs
//     pre_identity / pre_compose, suf_identity / suf_compose   (f first, s to its right)
// row_exchange (warp shuffles + one shared-memory round) and col_exchange (shared memory + one
// distributed-shared-memory round across the CTAs of a cluster) return, for every segment, the
// composition of all segments before it (pre) and after it (suf) on its line.
#pragma once

#include <cooperative_groups.h>

#include <type_traits>
#include <utility>

#include "dts_internal.cuh"

namespace dts {
namespace scan {

namespace cg = cooperative_groups;

constexpr unsigned kFull = 0xffffffffu;

// 2^x with the SFU instruction (PTX ex2.approx.ftz.f32; relative error ~2^-22, results below
// the normal range flush to zero, which is harmless for a feedback weight).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Programmatic dependent launch: a kernel launched with the programmatic-serialization
// attribute may start while its predecessor drains; it must wait for the predecessor's
// completion (and memory) before touching global data, and it lets its own successor start
// launching once it no longer needs the SM slots it would free.  Both are no-ops otherwise.
__device__ __forceinline__ void wait_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void release_successor() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// v -> A v + B: the left-to-right map of a group of positions
struct Aff {
    float A, B;
};
__device__ __forceinline__ Aff aff_identity() { return Aff{1.f, 0.f}; }
__device__ __forceinline__ Aff aff_compose(const Aff& f, const Aff& s) { return Aff{f.A * s.A, fmaf(s.A, f.B, s.B)}; }

// the coupled five numbers of a group
struct Coupled {
    float A, B, al, be, ga;
};
__device__ __forceinline__ Coupled coupled_identity() { return Coupled{1.f, 0.f, 1.f, 0.f, 0.f}; }
// group f followed by group s:  c_mid = A_f c + B_f,  k_mid = al_s k + be_s c_mid + ga_s,
// k_start = al_f k_mid + be_f c + ga_f
__device__ __forceinline__ Coupled coupled_compose(const Coupled& f, const Coupled& s) {
    Coupled o;
    o.A = f.A * s.A;
    o.B = fmaf(s.A, f.B, s.B);
    o.al = f.al * s.al;
    o.be = fmaf(f.al * s.be, f.A, f.be);
    o.ga = fmaf(f.al, fmaf(s.be, f.B, s.ga), f.ga);
    return o;
}

// One forward walk over a segment gives its coupled numbers.  The left-to-right recurrence is
//     u[n] = w[n] u[n-1] + (NORM ? (1 - w[n]) : 1) y[n]
// and the right-to-left one, on u, is v[n] = w'[n] v[n+1] + (1 - w'[n]) u[n] with w'[n] = w[n+1]
// (wn for the last position).  P_n = prod_{m<=n} w_m is the weight of the entering value in
// u[n], Q_n the value of u[n] from a zero carry, r_n = prod_{m<n} w'_m the weight of u[n]'s
// contribution path to v at the segment start:  be = sum r_n (1-w'_n) P_n,  ga = sum r_n (1-w'_n) Q_n.
template <bool NORM, int N>
__device__ __forceinline__ Coupled coupled_local(const float (&y)[N], const float (&w)[N], float wn) {
    float P = 1.f, Q = 0.f, r = 1.f, be = 0.f, ga = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        P *= w[j];
        if constexpr (NORM) Q = fmaf(w[j], Q - y[j], y[j]);
        else Q = fmaf(w[j], Q, y[j]);
        const float wp = (j + 1 < N) ? w[j + 1] : wn;
        const float coef = fmaf(-r, wp, r);
        be = fmaf(coef, P, be);
        ga = fmaf(coef, Q, ga);
        r *= wp;
    }
    return Coupled{P, Q, r, be, ga};
}

// value entering a segment from the right, given the composition of everything after it and
// the left-to-right value leaving it
__device__ __forceinline__ float k_entering(const Coupled& after, float c_out) {
    return fmaf(after.be, c_out, after.ga);
}

template <typename T>
__device__ __forceinline__ T shfl_up_t(const T& v, int off) {
    constexpr int n = sizeof(T) / 4;
    T r;
    const float* s = reinterpret_cast<const float*>(&v);
    float* d = reinterpret_cast<float*>(&r);
#pragma unroll
    for (int i = 0; i < n; ++i) d[i] = __shfl_up_sync(kFull, s[i], off);
    return r;
}

template <typename T>
__device__ __forceinline__ T shfl_xor_t(const T& v, int mask) {
    constexpr int n = sizeof(T) / 4;
    T r;
    const float* s = reinterpret_cast<const float*>(&v);
    float* d = reinterpret_cast<float*>(&r);
#pragma unroll
    for (int i = 0; i < n; ++i) d[i] = __shfl_xor_sync(kFull, s[i], mask);
    return r;
}

template <typename T>
__device__ __forceinline__ T shfl_down_t(const T& v, int off) {
    constexpr int n = sizeof(T) / 4;
    T r;
    const float* s = reinterpret_cast<const float*>(&v);
    float* d = reinterpret_cast<float*>(&r);
#pragma unroll
    for (int i = 0; i < n; ++i) d[i] = __shfl_down_sync(kFull, s[i], off);
    return r;
}

template <typename T>
__device__ __forceinline__ T shfl_up_w(const T& v, int off, int width) {
    constexpr int n = sizeof(T) / 4;
    T r;
    const float* s = reinterpret_cast<const float*>(&v);
    float* d = reinterpret_cast<float*>(&r);
#pragma unroll
    for (int i = 0; i < n; ++i) d[i] = __shfl_up_sync(kFull, s[i], off, width);
    return r;
}

template <typename T>
__device__ __forceinline__ T shfl_down_w(const T& v, int off, int width) {
    constexpr int n = sizeof(T) / 4;
    T r;
    const float* s = reinterpret_cast<const float*>(&v);
    float* d = reinterpret_cast<float*>(&r);
#pragma unroll
    for (int i = 0; i < n; ++i) d[i] = __shfl_down_sync(kFull, s[i], off, width);
    return r;
}

// ---------------------------------------------------------------- exchanges
template <class M>
__device__ __forceinline__ typename M::Pre warp_scan_pre(typename M::Pre v, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const typename M::Pre o = shfl_up_t(v, off);
        if (lane >= off) v = M::pre_compose(o, v);
    }
    return v;
}

template <class M>
__device__ __forceinline__ typename M::Suf warp_scan_suf(typename M::Suf v, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const typename M::Suf o = shfl_down_t(v, off);
        if (lane + off < 32) v = M::suf_compose(v, o);
    }
    return v;
}

// Segments of one row are consecutive threads (a row never shares a warp with another row):
// warp `wrow` of the row's `wpr` warps, the row's first warp being CTA warp `wbase`.
// s_pre / s_suf: shared arrays of at least 32 entries.  Contains __syncthreads when wpr > 1
// (wpr must then be uniform across the CTA).
template <class M>
__device__ __forceinline__ void row_exchange(const typename M::Pre& own_pre, const typename M::Suf& own_suf,
                                             int lane, int warp, int wrow, int wbase, int wpr,
                                             typename M::Pre* s_pre, typename M::Suf* s_suf,
                                             typename M::Pre& pre, typename M::Suf& suf) {
    const typename M::Pre inc_pre = warp_scan_pre<M>(own_pre, lane);
    const typename M::Suf inc_suf = warp_scan_suf<M>(own_suf, lane);
    pre = shfl_up_t(inc_pre, 1);
    suf = shfl_down_t(inc_suf, 1);
    if (lane == 0) pre = M::pre_identity();
    if (lane == 31) suf = M::suf_identity();
    if (wpr > 1) {
        if (lane == 31) s_pre[warp] = inc_pre;
        if (lane == 0) s_suf[warp] = inc_suf;
        __syncthreads();
        typename M::Pre wpre = M::pre_identity();
        for (int q = 0; q < wrow; ++q) wpre = M::pre_compose(wpre, s_pre[wbase + q]);
        typename M::Suf wsuf = M::suf_identity();
        for (int q = wrow + 1; q < wpr; ++q) wsuf = M::suf_compose(wsuf, s_suf[wbase + q]);
        pre = M::pre_compose(wpre, pre);
        suf = M::suf_compose(suf, wsuf);
    }
}

// One-direction exchange of affine maps along a row (same thread layout as row_exchange):
// PREFIX: the map of everything left of this segment (maps compose left to right); else the map
// of everything right of it (the rightmost applies first).  s_buf: 32 entries, not shared with
// another exchange running before the same __syncthreads.  Contains __syncthreads when wpr > 1.
template <bool PREFIX>
__device__ __forceinline__ Aff row_scan_aff(Aff v, int lane, int warp, int wrow, int wbase, int wpr, Aff* s_buf) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const Aff o = PREFIX ? shfl_up_t(v, off) : shfl_down_t(v, off);
        if (PREFIX ? lane >= off : lane + off < 32) v = aff_compose(o, v);
    }
    Aff ex = PREFIX ? shfl_up_t(v, 1) : shfl_down_t(v, 1);
    if (PREFIX ? lane == 0 : lane == 31) ex = aff_identity();
    if (wpr > 1) {
        if (PREFIX ? lane == 31 : lane == 0) s_buf[warp] = v;
        __syncthreads();
        Aff w = aff_identity();
        if (PREFIX) {
            for (int q = 0; q < wrow; ++q) w = aff_compose(w, s_buf[wbase + q]);
        } else {
            for (int q = wpr - 1; q > wrow; --q) w = aff_compose(w, s_buf[wbase + q]);
        }
        ex = aff_compose(w, ex);
    }
    return ex;
}

// Shared state of a column exchange: NWMAX warps per CTA.
template <class M, int NWMAX>
struct ColShared {
    // rows padded to 33 entries: the CTA scan reads a column across the warps' rows
    typename M::Pre pre[NWMAX][33];
    typename M::Suf suf[NWMAX][33];
    typename M::Pre cta_pre[32];
    typename M::Suf cta_suf[32];
    typename M::Pre cl_pre[32];
    typename M::Suf cl_suf[32];
    typename M::Pre rem_pre[16][32];  // totals of the other CTAs of the cluster, gathered in parallel
    typename M::Suf rem_suf[16][32];
};

// Gather every peer's CTA totals (one DSMEM round, spread over the warps), then warp 0 folds
// them from local shared memory into the cluster prefix and suffix of this CTA.
template <class M, int NWMAX>
__device__ __forceinline__ void gather_cluster_totals(cg::cluster_group& cluster, int rank, int CS, int lane,
                                                      int warp, int NW, ColShared<M, NWMAX>& sh) {
    for (int q = warp; q < CS; q += NW) {
        if (q == rank) continue;
        if (q < rank) sh.rem_pre[q][lane] = *cluster.map_shared_rank(&sh.cta_pre[lane], q);
        else sh.rem_suf[q][lane] = *cluster.map_shared_rank(&sh.cta_suf[lane], q);
    }
    __syncthreads();
    if (warp == 0) {
        typename M::Pre cp = M::pre_identity();
        for (int q = 0; q < rank; ++q) cp = M::pre_compose(cp, sh.rem_pre[q][lane]);
        typename M::Suf cs = M::suf_identity();
        for (int q = rank + 1; q < CS; ++q) cs = M::suf_compose(cs, sh.rem_suf[q][lane]);
        sh.cl_pre[lane] = cp;
        sh.cl_suf[lane] = cs;
    }
}

// Segments of a column: warp q of cluster CTA r is segment r*NW + q (lane = column).  Ends with
// barrier.cluster.arrive: the caller must execute cluster_exit() before returning, after which
// no CTA of the cluster reads another's shared memory.
// Exclusive prefix / suffix over the NW warps of a CTA for each of the 32 columns, in parallel:
// with NW a power of two, warp q scans columns [q*32/NW, (q+1)*32/NW), NW lanes per column, in
// log2(NW) shuffle rounds, and writes the exclusive results back in place; the CTA totals go to
// cta_pre / cta_suf.  Ends with __syncthreads.
template <class M, int NWMAX>
__device__ __forceinline__ void cta_scan(int lane, int warp, int NW, ColShared<M, NWMAX>& sh) {
    const int q = lane & (NW - 1);         // the segment (warp) this lane stands for
    const int cw = warp * (32 / NW) + lane / NW;  // the column it scans
    typename M::Pre p = sh.pre[q][cw];
    typename M::Suf f = sh.suf[q][cw];
    for (int off = 1; off < NW; off <<= 1) {
        const typename M::Pre op = shfl_up_w(p, off, NW);
        const typename M::Suf of = shfl_down_w(f, off, NW);
        if (q >= off) p = M::pre_compose(op, p);
        if (q + off < NW) f = M::suf_compose(f, of);
    }
    if (q == NW - 1) sh.cta_pre[cw] = p;
    if (q == 0) sh.cta_suf[cw] = f;
    typename M::Pre pe = shfl_up_w(p, 1, NW);
    typename M::Suf fe = shfl_down_w(f, 1, NW);
    if (q == 0) pe = M::pre_identity();
    if (q == NW - 1) fe = M::suf_identity();
    sh.pre[q][cw] = pe;
    sh.suf[q][cw] = fe;
    __syncthreads();
}

// Segments of a column: warp q of cluster CTA r is segment r*NW + q (lane = column).  Each thread
// folds the other warps' aggregates of its column from shared memory (measured faster than the
// shuffle scan of cta_scan on the stereo workload).  Ends with barrier.cluster.arrive: the caller
// must execute cluster_exit() before returning, after which no CTA of the cluster reads another's
// shared memory.
template <class M, int NWMAX>
__device__ __forceinline__ void col_exchange(const typename M::Pre& own_pre, const typename M::Suf& own_suf,
                                             int lane, int warp, int NW, ColShared<M, NWMAX>& sh,
                                             typename M::Pre& pre, typename M::Suf& suf) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CS = (int)cluster.num_blocks();
    sh.pre[warp][lane] = own_pre;
    sh.suf[warp][lane] = own_suf;
    __syncthreads();
    typename M::Pre wpre = M::pre_identity();
    for (int q = 0; q < warp; ++q) wpre = M::pre_compose(wpre, sh.pre[q][lane]);
    typename M::Suf wsuf = M::suf_identity();
    for (int q = warp + 1; q < NW; ++q) wsuf = M::suf_compose(wsuf, sh.suf[q][lane]);
    if (CS > 1) {
        // CTA totals: the last warp holds the full prefix, the first warp the full suffix
        if (warp == NW - 1) sh.cta_pre[lane] = M::pre_compose(wpre, own_pre);
        if (warp == 0) sh.cta_suf[lane] = M::suf_compose(own_suf, wsuf);
        cluster.sync();
        gather_cluster_totals<M, NWMAX>(cluster, rank, CS, lane, warp, NW, sh);
        __syncthreads();
        wpre = M::pre_compose(sh.cl_pre[lane], wpre);
        wsuf = M::suf_compose(wsuf, sh.cl_suf[lane]);
    }
    pre = wpre;
    suf = wsuf;
    // every remote read of this CTA is done: peers may exit once all have arrived
    cluster.barrier_arrive();
}

// col_exchange with the cross-warp part done by cta_scan (log2(NW) shuffle rounds instead of a
// per-thread fold over the other warps): the better choice when the tuples are large.  NW must be
// a power of two.  Same contract as col_exchange.
template <class M, int NWMAX>
__device__ __forceinline__ void col_exchange_scan(const typename M::Pre& own_pre, const typename M::Suf& own_suf,
                                                  int lane, int warp, int NW, ColShared<M, NWMAX>& sh,
                                                  typename M::Pre& pre, typename M::Suf& suf) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CS = (int)cluster.num_blocks();
    sh.pre[warp][lane] = own_pre;
    sh.suf[warp][lane] = own_suf;
    __syncthreads();
    cta_scan<M, NWMAX>(lane, warp, NW, sh);
    typename M::Pre wpre = sh.pre[warp][lane];
    typename M::Suf wsuf = sh.suf[warp][lane];
    if (CS > 1) {
        cluster.sync();
        gather_cluster_totals<M, NWMAX>(cluster, rank, CS, lane, warp, NW, sh);
        __syncthreads();
        wpre = M::pre_compose(sh.cl_pre[lane], wpre);
        wsuf = M::suf_compose(wsuf, sh.cl_suf[lane]);
    }
    pre = wpre;
    suf = wsuf;
    cluster.barrier_arrive();
}

__device__ __forceinline__ void cluster_exit() { cg::this_cluster().barrier_wait(); }

// The same exchange for a kernel that loops over several lines per cluster (persistent grid).
// Before a CTA overwrites its totals it waits until every peer has finished reading the
// previous iteration's (the arrive at the end of that iteration); `first` skips that wait.
// After the last iteration the caller executes cluster_exit() if any iteration ran with CS > 1.
template <class M, int NWMAX>
__device__ __forceinline__ void col_exchange_iter(const typename M::Pre& own_pre, const typename M::Suf& own_suf,
                                                  int lane, int warp, int NW, ColShared<M, NWMAX>& sh, bool first,
                                                  typename M::Pre& pre, typename M::Suf& suf) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CS = (int)cluster.num_blocks();
    sh.pre[warp][lane] = own_pre;
    sh.suf[warp][lane] = own_suf;
    __syncthreads();
    typename M::Pre wpre = M::pre_identity();
    for (int q = 0; q < warp; ++q) wpre = M::pre_compose(wpre, sh.pre[q][lane]);
    typename M::Suf wsuf = M::suf_identity();
    for (int q = warp + 1; q < NW; ++q) wsuf = M::suf_compose(wsuf, sh.suf[q][lane]);
    if (CS > 1) {
        if (!first) cluster.barrier_wait();
        if (warp == NW - 1) sh.cta_pre[lane] = M::pre_compose(wpre, own_pre);
        if (warp == 0) sh.cta_suf[lane] = M::suf_compose(own_suf, wsuf);
        cluster.sync();
        gather_cluster_totals<M, NWMAX>(cluster, rank, CS, lane, warp, NW, sh);
        __syncthreads();
        wpre = M::pre_compose(sh.cl_pre[lane], wpre);
        wsuf = M::suf_compose(wsuf, sh.cl_suf[lane]);
        cluster.barrier_arrive();
    }
    pre = wpre;
    suf = wsuf;
}

// ---------------------------------------------------------------- chained column exchange
// Columns too tall for one CTA run as a chain of chunks of R rows, one CTA per chunk and no
// cluster.  A CTA draws a ticket t from an atomic counter (so tickets go out in the order CTAs
// start) and takes chunk t % J of 32-column strip t / J.  After the exchange inside the CTA it
// publishes its chunk totals (the composition of its segments in both directions, per column) to
// global memory and counts its arrival at the strip.  The CTA whose arrival completes the strip
// turns every chunk's totals, in place, into the chunk's exclusive carries (everything above it,
// everything below it), then raises the strip's flag; the other CTAs wait for the flag, read
// their carries and compose them with their own.  A pass thus reads and writes every pixel once,
// as with a cluster, but without gang scheduling: small CTAs of many strips share each SM.
//
// No deadlock when J CTAs can be resident at once: the chunks of a strip hold consecutive
// tickets and every CTA publishes before it waits, so every strip older than the newest one
// completes, and the newest one's at most J - 1 waiting CTAs leave a slot for the rest of it.
// Waits are bounded: one that runs out records DTS_ERR_TIMEOUT and raises the abort word, after
// which no CTA of the solve waits again (its results are then invalid; the kernel still ends).
//
// Control words (zeroed once per solve): ctl[0] ticket counter and ctl[32 + s] arrivals at strip
// s (every launch leaves both at zero again), ctl[1] abort, ctl[32 + S + s] flag of strip s: the
// launch's epoch (a number the host gives every launch, never 0) once its carries are in place.
struct ChainArgs {
    unsigned* ctl;
    float* agg;       // S x J x 32 Pre tuples, then S x J x 32 Suf tuples
    int J;            // chunks per strip
    int S;            // strips
    long long timeout;
    int* status;
    int skip_ticket;  // fault injection: this ticket does not count its arrival (-1: none)
    int stage;        // chunks per block of the composition's shared-memory staging (>= 1)
    unsigned epoch;   // this launch's flag value (not 0, not that of an earlier launch of the solve)
};
// dynamic shared memory of a chained exchange staging `stage` chunks of mode M's tuples
template <class M>
__host__ __device__ constexpr size_t chain_stage_bytes(int stage) {
    return (size_t)stage * 32 * (sizeof(typename M::Pre) + sizeof(typename M::Suf));
}
constexpr int kChainCtlHead = 32;
__host__ __device__ constexpr long long chain_ctl_words(int S) { return kChainCtlHead + 2LL * S; }

template <typename T>
__device__ __forceinline__ void st_cg(T* p, const T& v) {
    constexpr int n = sizeof(T) / 4;
    const float* s = reinterpret_cast<const float*>(&v);
    float* d = reinterpret_cast<float*>(p);
#pragma unroll
    for (int i = 0; i < n; ++i) __stcg(d + i, s[i]);
}
template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) {
    constexpr int n = sizeof(T) / 4;
    T v;
    const float* s = reinterpret_cast<const float*>(p);
    float* d = reinterpret_cast<float*>(&v);
#pragma unroll
    for (int i = 0; i < n; ++i) d[i] = __ldcg(s + i);
    return v;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// atomic add with acquire-release semantics at GPU scope; returns the old value
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
// records a device-side error in the status word (when there is one)
__device__ __forceinline__ void record_status(int* status, int code) {
    if (status) atomicExch(status, code);
}

// This CTA's ticket (call after wait_predecessor: the previous launch has reset the counter).
__device__ __forceinline__ int chain_ticket(const ChainArgs& c) {
    __shared__ int s_ticket;
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(&c.ctl[0], 1u);
        if (t == (unsigned)(c.S * c.J) - 1u) atomicExch(&c.ctl[0], 0u);  // every ticket is out
        s_ticket = (int)t;
    }
    __syncthreads();
    return s_ticket;
}

// Shared state of a chained exchange: NWMAX warps per CTA (rows padded to 33 entries).
template <class M, int NWMAX>
struct ChainShared {
    typename M::Pre pre[NWMAX][33];
    typename M::Suf suf[NWMAX][33];
};

// Turns the J chunk totals of `strip` (Pre tuples at gpre, Suf tuples at gsuf, chunk-major, 32
// columns each), in place, into every chunk's exclusive carries: everything above it (prefix
// direction, warp 0, top down) and everything below it (suffix direction, warp 1, bottom up).
// The tuples come into shared memory (c.stage chunks' worth, dynamic) in blocks loaded by the
// whole CTA at once: one L2 round trip per block, not one per chunk.  Every thread calls it.
template <class M>
__device__ __forceinline__ void chain_compose_strip(const ChainArgs& c, int strip, int lane, int warp,
                                                    typename M::Pre* gpre, typename M::Suf* gsuf) {
    using Pre = typename M::Pre;
    using Suf = typename M::Suf;
    extern __shared__ __align__(16) float chain_stage[];
    constexpr int NP = sizeof(Pre) / 4, NS = sizeof(Suf) / 4;
    float* stp = chain_stage;                              // c.stage x 32 Pre
    float* sts = chain_stage + (size_t)c.stage * 32 * NP;  // c.stage x 32 Suf
    Pre pacc = M::pre_identity();
    Suf sacc = M::suf_identity();
    const size_t sbase = (size_t)strip * c.J;
    for (int b0 = 0; b0 < c.J; b0 += c.stage) {
        const int nb = min(c.stage, c.J - b0);
        const int s0 = c.J - b0 - nb;  // the suffix block: chunks [s0, s0 + nb), from the bottom
        const float4* gp = reinterpret_cast<const float4*>(gpre + (sbase + b0) * 32);
        const float4* gs = reinterpret_cast<const float4*>(gsuf + (sbase + s0) * 32);
        float4* sp4 = reinterpret_cast<float4*>(stp);
        float4* ss4 = reinterpret_cast<float4*>(sts);
        for (int i = threadIdx.x; i < nb * 8 * NP; i += blockDim.x) sp4[i] = __ldcg(gp + i);
        for (int i = threadIdx.x; i < nb * 8 * NS; i += blockDim.x) ss4[i] = __ldcg(gs + i);
        __syncthreads();
        if (warp == 0) {
            const Pre* sp = reinterpret_cast<const Pre*>(stp);
            for (int j = 0; j < nb; ++j) {
                const Pre v = sp[j * 32 + lane];
                st_cg(gpre + (sbase + b0 + j) * 32 + lane, pacc);
                pacc = M::pre_compose(pacc, v);
            }
        } else if (warp == 1) {
            const Suf* ss = reinterpret_cast<const Suf*>(sts);
            for (int j = nb - 1; j >= 0; --j) {
                const Suf v = ss[j * 32 + lane];
                st_cg(gsuf + (sbase + s0 + j) * 32 + lane, sacc);
                sacc = M::suf_compose(v, sacc);
            }
        }
        __syncthreads();
    }
}

// Counts this CTA's arrival at `strip` (its chunk's totals are in place); the CTA whose arrival
// completes the strip composes the strip's carries (chain_compose_strip), resets the arrival
// count and returns true.  `count` false leaves the arrival out (fault injection).  Every thread
// of the CTA calls it.
template <class M>
__device__ __forceinline__ bool chain_arrive_compose(const ChainArgs& c, int strip, bool count, int lane, int warp,
                                                     typename M::Pre* gpre, typename M::Suf* gsuf) {
    __shared__ int s_combine;
    unsigned* arrive = c.ctl + kChainCtlHead + strip;
    if (threadIdx.x == 0) {
        // the fence publishes the CTA's tuples (ordered before it by the caller's barrier); the
        // arrival's acquire side makes the other chunks' tuples visible to the composing CTA
        __threadfence();
        s_combine = 0;
        if (count) s_combine = atom_add_acq_rel_u32(arrive, 1u) == (unsigned)c.J - 1u;
    }
    __syncthreads();
    if (!s_combine) return false;
    chain_compose_strip<M>(c, strip, lane, warp, gpre, gsuf);
    if (threadIdx.x == 0) atomicExch(arrive, 0u);
    return true;
}

// pre / suf: the transforms of everything above / below this warp's segment in its column
// (warp q of chunk r is segment r NW + q of the column; lane = column).  NW >= 2.
template <class M, int NWMAX>
__device__ __forceinline__ void chain_exchange(const typename M::Pre& own_pre, const typename M::Suf& own_suf,
                                               int lane, int warp, int NW, ChainShared<M, NWMAX>& sh,
                                               const ChainArgs& c, int ticket, typename M::Pre& pre,
                                               typename M::Suf& suf) {
    using Pre = typename M::Pre;
    using Suf = typename M::Suf;
    const int strip = ticket / c.J;
    const int chunk = ticket - strip * c.J;
    sh.pre[warp][lane] = own_pre;
    sh.suf[warp][lane] = own_suf;
    __syncthreads();
    Pre wpre = M::pre_identity();
    for (int q = 0; q < warp; ++q) wpre = M::pre_compose(wpre, sh.pre[q][lane]);
    Suf wsuf = M::suf_identity();
    for (int q = warp + 1; q < NW; ++q) wsuf = M::suf_compose(wsuf, sh.suf[q][lane]);
    if (c.J > 1) {
        Pre* gpre = reinterpret_cast<Pre*>(c.agg);
        Suf* gsuf = reinterpret_cast<Suf*>(c.agg + (size_t)c.S * c.J * 32 * (sizeof(Pre) / 4));
        const size_t mine = ((size_t)strip * c.J + chunk) * 32 + lane;
        // this chunk's totals: the last warp holds the full prefix, the first the full suffix
        if (warp == NW - 1) st_cg(gpre + mine, M::pre_compose(wpre, own_pre));
        if (warp == 0) st_cg(gsuf + mine, M::suf_compose(own_suf, wsuf));
        __syncthreads();
        unsigned* flag = c.ctl + kChainCtlHead + c.S + strip;
        if (chain_arrive_compose<M>(c, strip, ticket != c.skip_ticket, lane, warp, gpre, gsuf)) {
            if (threadIdx.x == 0) {
                __threadfence();
                st_release_u32(flag, c.epoch);
            }
        } else if (threadIdx.x == 0) {
            if (ld_acquire_u32(flag) != c.epoch && ld_acquire_u32(c.ctl + 1) == 0u) {
                const long long t0 = clock64();
                while (ld_acquire_u32(flag) != c.epoch) {
                    if (ld_acquire_u32(c.ctl + 1) != 0u) break;
                    if (clock64() - t0 > c.timeout) {
                        atomicExch(c.ctl + 1, 1u);
                        record_status(c.status, DTS_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);  // leave the L2 to the composing CTA
                }
            }
        }
        __syncthreads();
        wpre = M::pre_compose(ld_cg(gpre + mine), wpre);
        wsuf = M::suf_compose(wsuf, ld_cg(gsuf + mine));
    }
    pre = wpre;
    suf = wsuf;
}

// ---------------------------------------------------------------- TMA and mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; gives up after `limit` clock cycles (false).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// 2-D tiled TMA load of the box at (x, y) (x in elements, a multiple of 16 bytes) into shared
// memory, completing `bytes` on `bar`.  Rows or columns outside the tensor read as zero.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 1-D bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to
// shared memory, completing on `bar`
__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// 2-D tiled TMA store of the box at (x, y) from shared memory (clipped to the tensor: rows or
// columns outside it are not written), in the calling thread's bulk group.  The shared-memory
// writes it reads must be made visible to the async proxy first (fence_proxy_async_smem).
__device__ __forceinline__ void tma_store_2d(const void* tmap, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(tmap), "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the committed bulk stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------- loads
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

__device__ __forceinline__ void load4_f(const float* base, long long idx, float* out) {
    const float4 v = *reinterpret_cast<const float4*>(base + idx);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}

// four consecutive floats of a plane; CG: through L2 only (the plane is rewritten within the
// launch by other SMs, whose writes an SM's L1 would not see)
template <bool CG>
__device__ __forceinline__ void load4_p(const float* base, long long idx, float* out) {
    float4 v;
    if constexpr (CG) v = __ldcg(reinterpret_cast<const float4*>(base + idx));
    else v = *reinterpret_cast<const float4*>(base + idx);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <bool CG>
__device__ __forceinline__ float load1_p(const float* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

__device__ __forceinline__ void store4_f(float* base, long long idx, const float* v) {
    *reinterpret_cast<float4*>(base + idx) = make_float4(v[0], v[1], v[2], v[3]);
}

// ---------------------------------------------------------------- launch
// Launch with programmatic stream serialization (unless disabled) and an optional cluster shape
// (1, cluster_y, 1).
template <typename... KArgs, typename... Args>
cudaError_t launch_ex_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, int cluster_y, size_t smem,
                           cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int n = 0;
    if (cluster_y > 0) {
        attr[n].id = cudaLaunchAttributeClusterDimension;
        attr[n].val.clusterDim.x = 1;
        attr[n].val.clusterDim.y = (unsigned)cluster_y;
        attr[n].val.clusterDim.z = 1;
        ++n;
    }
    if (pdl_enabled()) {
        attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kernel)(KArgs...), dim3 grid, dim3 block, int cluster_y, cudaStream_t s,
                      Args&&... args) {
    return launch_ex_smem(kernel, grid, block, cluster_y, 0, s, std::forward<Args>(args)...);
}

}  // namespace scan
}  // namespace dts
