// Horizontal pass (§2, §3.2: causal then anti-causal recursive filter along each row) for wide
// rows, persistent and fed by bulk copies.  One CTA of NW warps takes one row at a time (rows
// blockIdx.x, blockIdx.x + gridDim.x, ...); thread t owns positions [t ITEMS, (t + 1) ITEMS).
// The row's pass input and distances arrive in shared memory by two 1-D bulk copies (one stage
// of two, completing on the stage's mbarrier), issued two rows ahead, so the copies of the next
// rows stream in while a row is scanned.  ITEMS is odd, so the threads' column-wise reads of the
// stage are free of bank conflicts.  The results go back into the stage (the same conflict-free
// pattern) and leave it as 16-byte coalesced stores of each warp's span.
// UPD: the first pass of an iteration also applies the previous iteration's data-term update
// (Eq. 3 or Eq. 4): the staged row is zbar; each warp reads z_k, t and c of its span with
// coalesced vector loads, writes z_{k+1} to a.zout and into the stage, and filters z_{k+1}.
#include "dts_internal.cuh"
#include "dts_modes.cuh"

namespace dts {
using namespace scan;

namespace {

// shared memory of a stage: the position row and the distance row of a CTA of nw warps
__host__ __device__ constexpr size_t stream_x_bytes(int nw, int items) {
    return ((size_t)nw * 32 * items * 4 + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t stream_d_bytes(int nw, int items, int dsize) {
    return ((size_t)nw * 32 * items * dsize + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t stream_stage_bytes(int nw, int items, int dsize) {
    return stream_x_bytes(nw, items) + stream_d_bytes(nw, items, dsize);
}

// Four consecutive target values from element i (i a multiple of 4, rows of 16-byte or 8-byte
// aligned vectors), storage TT fixed at compile time so that a group's loads issue together and
// their widening waits for the update: one 16-byte load for FP32, one 8-byte load for 16-bit
// storage (a BF16 value is the upper half of the FP32 one).
template <int TT>
__device__ __forceinline__ void load4_target(const void* t, long long i, float (&out)[4]) {
    if constexpr (TT == DTS_F32) {
        load4_f(static_cast<const float*>(t), i, out);
    } else {
        const uint2 v = *reinterpret_cast<const uint2*>(static_cast<const unsigned short*>(t) + i);
        if constexpr (TT == DTS_BF16) {
            out[0] = __uint_as_float(v.x << 16);
            out[1] = __uint_as_float(v.x & 0xffff0000u);
            out[2] = __uint_as_float(v.y << 16);
            out[3] = __uint_as_float(v.y & 0xffff0000u);
        } else {
            const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
            const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
            out[0] = f0.x;
            out[1] = f0.y;
            out[2] = f1.x;
            out[3] = f1.y;
        }
    }
}

// largest CTA per segment length: two stages within 227 KB of shared memory
template <int ITEMS>
constexpr int stream_max_threads() {
    return ITEMS >= 33 ? 384 : 512;
}

// RAG: rows that do not end on a whole 16-byte unit (of the positions, or of FP16 distances).
// The bulk copies then bring the whole units, the 1-3 positions (1-7 FP16 distances) after them
// come by plain loads, and the results past the last whole unit leave by plain stores.
// UPD > 0: the pass with the update, for a target stored as dtype UPD - 1 (DTS_F32, DTS_BF16,
// DTS_F16).  Waits on a stage are bounded (timeout cycles).  A wait that gives up records DTS_ERR_TIMEOUT;
// the CTA finishes the row at hand with what it holds (the results are invalid, the status says
// so), issues no further copies and leaves the row loop after one more bounded wait for each
// copy of its own still in flight.  skip (fault injection): CTA 0 leaves out its first row's copies.
template <int ITEMS, bool DHALF, int UPD, bool RAG>
__global__ void __launch_bounds__(stream_max_threads<ITEMS>()) row_stream_kernel(PassArgs a, long long timeout,
                                                                                  int skip) {
    static_assert(ITEMS % 2 == 1, "odd segment length (bank-conflict-free shared-memory reads)");
    using DT = typename std::conditional<DHALF, __half, float>::type;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ Aff s_pre[32];
    __shared__ Aff s_suf[32];
    __shared__ __align__(8) uint64_t bar[2];
    // a wait gave up in an iteration of this parity (a slot per parity, so that a failure in the
    // next iteration cannot change what a slower thread reads for this one)
    __shared__ int s_abort[2];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int NW = blockDim.x >> 5;
    const int W = a.W;
    const long long P = a.pitch;
    const size_t xb = stream_x_bytes(NW, ITEMS);
    const size_t stage = xb + stream_d_bytes(NW, ITEMS, (int)sizeof(DT));
    const int Wx = RAG ? W & ~3 : W;                     // positions the bulk copy brings
    const int Wd = RAG ? (DHALF ? W & ~7 : W & ~3) : W;  // distances the bulk copy brings
    const uint32_t kx = (uint32_t)Wx * 4u, kd = (uint32_t)Wd * (uint32_t)sizeof(DT);
    const int e0 = tid * ITEMS;
    const int span0 = warp * 32 * ITEMS;  // this warp's span of the row
    const int span1 = min(span0 + 32 * ITEMS, W);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    if (tid < 2) s_abort[tid] = 0;
    __syncthreads();
    wait_predecessor();
    auto issue = [&](int row, int st) {
        unsigned char* base = dsm + (size_t)st * stage;
        mbar_arrive_expect_tx(&bar[st], kx + kd);
        bulk_load_1d(base, a.src + (long long)row * P, kx, &bar[st]);
        bulk_load_1d(base + xb, static_cast<const DT*>(a.d) + (long long)row * P, kd, &bar[st]);
    };
    if (tid == 0) {
        if ((int)blockIdx.x < a.H && !(skip && blockIdx.x == 0)) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < a.H) issue(blockIdx.x + gridDim.x, 1);
    }
    int it = 0;
    for (int row = blockIdx.x; row < a.H; row += gridDim.x, ++it) {
        const int st = it & 1;
        float* sx = reinterpret_cast<float*>(dsm + (size_t)st * stage);
        const DT* sd = reinterpret_cast<const DT*>(dsm + (size_t)st * stage + xb);
        if (!mbar_wait_bounded(&bar[st], (uint32_t)((it >> 1) & 1), timeout)) {
            record_status(a.status, DTS_ERR_TIMEOUT);
            s_abort[it & 1] = 1;
        }
        const long long rb = (long long)row * P;
        if constexpr (UPD > 0) {
            // z_{k+1} from z_k, zbar (the stage), t and c, four positions per lane and step;
            // every operand of a group is loaded before the group's stores (z_{k+1} may alias z_k)
            const long long tb = (long long)row * W;
            constexpr int G = 5;  // float4 groups per lane and round
            for (int e1 = span0 + 4 * lane; e1 < span1; e1 += 4 * 32 * G) {
                float zk[G][4], tt[G][4], cc[G][4];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int e = e1 + 128 * g;
                    if (RAG ? e + 4 <= span1 : e < span1) {
                        load4_f(a.zk, rb + e, zk[g]);
                        if (a.tc_vec) load4_target<UPD - 1>(a.t, tb + e, tt[g]);
                        else {
#pragma unroll
                            for (int k = 0; k < 4; ++k) tt[g][k] = load_any(a.t, tb + e + k, a.t_dtype);
                        }
                        if (a.c_pitched) load4_f(a.c, rb + e, cc[g]);
                        else if (a.tc_vec) load4_f(a.c, tb + e, cc[g]);
                        else {
#pragma unroll
                            for (int k = 0; k < 4; ++k) cc[g][k] = a.c[tb + e + k];
                        }
                    }
                }
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int e = e1 + 128 * g;
                    if constexpr (RAG) {
                        if (e + 4 > span1 && e < span1) {
                            // the row's last 1-3 positions (e == Wx): one by one, zbar from the plane
                            for (int k = 0; e + k < span1; ++k) {
                                const long long i = rb + e + k;
                                const float z = dts_update_value(a.zk[i], a.src[i], load_any(a.t, tb + e + k, a.t_dtype),
                                                                 a.c_pitched ? a.c[i] : a.c[tb + e + k], a.lambda,
                                                                 a.step, a.update, a.clamp_step, a.eps);
                                a.zout[i] = z;
                                sx[e + k] = z;
                            }
                        }
                    }
                    if (RAG ? e + 4 <= span1 : e < span1) {
                        const float4 zb = *reinterpret_cast<const float4*>(sx + e);
                        const float zbv[4] = {zb.x, zb.y, zb.z, zb.w};
                        float z[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            z[k] = dts_update_value(zk[g][k], zbv[k], tt[g][k], cc[g][k], a.lambda, a.step, a.update,
                                                    a.clamp_step, a.eps);
                        store4_f(a.zout, rb + e, z);
                        *reinterpret_cast<float4*>(sx + e) = make_float4(z[0], z[1], z[2], z[3]);
                    }
                }
            }
            __syncwarp();
        }
        float x[ITEMS], w[ITEMS];
        if constexpr (RAG) {
            // the thread whose positions (or next distance) reach past the bulk copies: those
            // positions and distances into the stage from the planes (its own reads only; the
            // update pass has already written every position of the row into the stage)
            const int hi = min(e0 + ITEMS + 1, W);
            for (int e = max(e0, Wd); e < hi; ++e) {
                if (e == e0 + ITEMS) continue;  // the next thread's position: read below
                if (UPD == 0 && e >= Wx) sx[e] = a.src[rb + e];
                const_cast<DT*>(sd)[e] = static_cast<const DT*>(a.d)[rb + e];
            }
        }
        if (e0 + ITEMS <= W) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                x[j] = sx[e0 + j];
                w[j] = ex2(a.k2 * to_f32<DT>(sd[e0 + j]));
            }
        } else {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const bool ok = e0 + j < W;  // positions past the row end read as 0
                x[j] = ok ? sx[e0 + j] : 0.f;
                w[j] = ok ? ex2(a.k2 * to_f32<DT>(sd[e0 + j])) : 0.f;
            }
        }
        if (e0 == 0) w[0] = 0.f;  // the row starts here
        float dn = 0.f;  // the distance entering the next thread's positions
        if (e0 + ITEMS < W) {
            if (RAG && e0 + ITEMS >= Wd) dn = load1_d<DHALF>(a.d, rb + e0 + ITEMS);
            else dn = to_f32<DT>(sd[e0 + ITEMS]);
        }
        const float wn = e0 + ITEMS < W ? ex2(a.k2 * dn) : 0.f;

        // causal sweep: segment map c -> A c + B, exclusive prefix over the row, replay
        float A = 1.f, B = 0.f;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            A *= w[j];
            B = fmaf(w[j], B - x[j], x[j]);
        }
        const Aff pc = row_scan_aff<true>(Aff{A, B}, lane, warp, warp, 0, NW, s_pre);
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
        const Aff sk = row_scan_aff<false>(Aff{A, B}, lane, warp, warp, 0, NW, s_suf);
        if (row + (int)gridDim.x >= a.H) release_successor();
        v = sk.B;
#pragma unroll
        for (int j = ITEMS - 1; j >= 0; --j) {
            const float wp = (j + 1 < ITEMS) ? w[j + 1] : wn;
            v = fmaf(wp, v - x[j], x[j]);
            x[j] = v;
        }
        // results into the stage, then out as the warp's coalesced span
#pragma unroll
        for (int j = 0; j < ITEMS; ++j)
            if (e0 + j < W) sx[e0 + j] = x[j];
        __syncwarp();
        for (int e = span0 + 4 * lane; e < span1; e += 128) {
            if (RAG && e + 4 > span1) {
                for (int k = 0; e + k < span1; ++k) a.dst[rb + e + k] = sx[e + k];
            } else {
                const float4 o = *reinterpret_cast<const float4*>(sx + e);
                *reinterpret_cast<float4*>(a.dst + rb + e) = o;
            }
        }
        // every thread's reads and writes of the stage come before the next copy into it
        fence_proxy_async_smem();
        __syncthreads();
        const bool abort = s_abort[it & 1] != 0;  // CTA-uniform (written before the barrier)
        const int ahead = row + 2 * (int)gridDim.x;
        if (tid == 0 && !abort && ahead < a.H) issue(ahead, st);
        if constexpr (UPD > 0) {
            // the update operands of that row into L2 as well (a 128-byte line of each per lane
            // and step), so that the loads after its stage wait hit L2
            if (!abort && ahead < a.H) {
                const long long ab = (long long)ahead * P, at = (long long)ahead * W;
                constexpr int tsz = UPD - 1 == DTS_F32 ? 4 : 2;
                for (int off = span0 + lane * 32; off < span1; off += 32 * 32) {
                    prefetch_l2(a.zk + ab + off);
                    prefetch_l2(static_cast<const char*>(a.t) + (at + off) * tsz);
                    prefetch_l2(a.c + (a.c_pitched ? ab : at) + off);
                }
            }
        }
        if (abort) {
            // copies still in flight (the one a wait gave up on, the next row's) must land before
            // the CTA's shared memory goes to another CTA
            if (tid == 0) {
                mbar_wait_bounded(&bar[st], (uint32_t)((it >> 1) & 1), timeout);
                if (row + (int)gridDim.x < a.H) mbar_wait_bounded(&bar[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1), timeout);
            }
            break;
        }
    }
}

template <int ITEMS, bool DHALF, int UPD, bool RAG>
cudaError_t allow_stream_t() {
    return cudaFuncSetAttribute((const void*)row_stream_kernel<ITEMS, DHALF, UPD, RAG>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * stream_stage_bytes(stream_max_threads<ITEMS>() / 32, ITEMS, DHALF ? 2 : 4)));
}

template <int ITEMS, bool DHALF, bool RAG>
cudaError_t allow_stream_r() {
    cudaError_t e = cudaSuccess, r;
    if ((r = allow_stream_t<ITEMS, DHALF, 0, RAG>()) != cudaSuccess) e = r;
    if ((r = allow_stream_t<ITEMS, DHALF, 1 + DTS_F32, RAG>()) != cudaSuccess) e = r;
    if ((r = allow_stream_t<ITEMS, DHALF, 1 + DTS_BF16, RAG>()) != cudaSuccess) e = r;
    if ((r = allow_stream_t<ITEMS, DHALF, 1 + DTS_F16, RAG>()) != cudaSuccess) e = r;
    return e;
}

template <int ITEMS, bool DHALF>
cudaError_t allow_stream_k() {
    cudaError_t e = cudaSuccess, r;
    if ((r = allow_stream_r<ITEMS, DHALF, false>()) != cudaSuccess) e = r;
    if ((r = allow_stream_r<ITEMS, DHALF, true>()) != cudaSuccess) e = r;
    return e;
}

template <int ITEMS, bool DHALF, bool RAG>
auto stream_kernel_for(const PassArgs& a, bool upd) {
    return !upd ? row_stream_kernel<ITEMS, DHALF, 0, RAG>
           : a.t_dtype == DTS_BF16 ? row_stream_kernel<ITEMS, DHALF, 1 + DTS_BF16, RAG>
           : a.t_dtype == DTS_F16 ? row_stream_kernel<ITEMS, DHALF, 1 + DTS_F16, RAG>
                                   : row_stream_kernel<ITEMS, DHALF, 1 + DTS_F32, RAG>;
}

template <int ITEMS, bool DHALF>
cudaError_t launch_stream_t(const PassArgs& a, bool upd, cudaStream_t s) {
    const int nw = ((a.W + ITEMS - 1) / ITEMS + 31) / 32;
    const size_t smem = 2 * stream_stage_bytes(nw, ITEMS, DHALF ? 2 : 4);
    // rows that end past their last whole 16-byte unit run the kernel's ragged variant
    const bool rag = a.W % (DHALF ? 8 : 4) != 0;
    auto kernel = rag ? stream_kernel_for<ITEMS, DHALF, true>(a, upd) : stream_kernel_for<ITEMS, DHALF, false>(a, upd);
    const int per_sm = blocks_per_sm((const void*)kernel, 32 * nw, smem);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int g = std::min(a.H, per_sm * sm_count());
    // fault injection (tests): CTA 0 leaves out its first row's copies, so its wait runs out
    const bool skip = take_injected(DTS_INJECT_STAGE_SKIP);
    return launch_ex_smem(kernel, dim3((unsigned)g), dim3((unsigned)(32 * nw)), 0, smem, s, a,
                          skip ? kInjectedTimeout : default_timeout_cycles(), skip ? 1 : 0);
}

}  // namespace

// Whether the streaming kernel takes this pass with ITEMS positions per thread: rows of at
// least two warps' spans within its largest CTA, of any length (row_stream_addressable checks
// that the planes' rows start on 16-byte boundaries).
bool row_stream_fits(int W, int items) {
    if (items != 17 && items != 33) return false;
    const int nw = ((W + items - 1) / items + 31) / 32;
    const int max_nw = (items >= 33 ? 384 : 512) / 32;
    return nw >= 2 && nw <= max_nw;
}

bool row_stream_addressable(const PassArgs& a, int dist_half, bool upd) {
    auto al16 = [](const void* p) { return (uintptr_t)p % 16 == 0; };
    if (!al16(a.src) || !al16(a.d) || !al16(a.dst) || a.pitch % (dist_half ? 8 : 4) != 0) return false;
    if (upd && (!al16(a.zk) || !al16(a.zout))) return false;
    return true;
}

cudaError_t launch_row_stream(const PassArgs& a, int dist_half, int items, bool upd, cudaStream_t s) {
    if (items == 33) return dist_half ? launch_stream_t<33, true>(a, upd, s) : launch_stream_t<33, false>(a, upd, s);
    if (items == 17) return dist_half ? launch_stream_t<17, true>(a, upd, s) : launch_stream_t<17, false>(a, upd, s);
    return cudaErrorInvalidValue;
}

cudaError_t prepare_row_stream_kernels() {
    cudaError_t e = cudaSuccess, r;
    if ((r = allow_stream_k<17, false>()) != cudaSuccess) e = r;
    if ((r = allow_stream_k<17, true>()) != cudaSuccess) e = r;
    if ((r = allow_stream_k<33, false>()) != cudaSuccess) e = r;
    if ((r = allow_stream_k<33, true>()) != cudaSuccess) e = r;
    return e;
}

}  // namespace dts
