// The edge-aware mean with the box kernel that Eq. 10 prints, W_ij = 1 if |DT_i - DT_j| <= r
// (normalized convolution in the transformed domain; per pass radius r_i = sigma_i sqrt(3)).
// Along a line the domain coordinate is ct[0] = 0, ct[n] = ct[n-1] + d[n]; out[n] averages the
// x[m] with |ct[m] - ct[n]| <= r.  FP32 distances >= 1 are multiples of 2^-23, so ct is kept as
// an exact integer count of 2^-23 units (64 bits: exact for coordinates below 2^40) and window
// membership compares the exact difference ct[m] - ct[n] with R = floor(r 2^23), which is the
// same decision as |ct[m] - ct[n]| <= r in exact arithmetic: which samples a window holds is
// fixed by the inputs alone, whatever the order of the additions.  The integer comes from the
// distance's bits (for d >= 1, d 2^23 is its significand shifted by its exponent) and the sums of
// x are prefix sums held as pairs of FP32 numbers (error-free addition, Knuth's two-sum: about 48
// significant bits), so the kernel uses no FP64 arithmetic, whose rate on GB300 is a small
// fraction of FP32's.  Rows run directly; columns run as rows of the transposed plane
// (transpose_kernel).
#include <algorithm>

#include "dts_scan.cuh"

namespace dts {

namespace {

using namespace scan;

constexpr int kBoxThreads = 512;
constexpr double kBoxUnit = 8388608.0;  // 2^23: FP32 values >= 1 are whole multiples of 2^-23

// d 2^23 as an exact integer for an FP32 distance d >= 1; 0 for the unused first entry of a line
__device__ __forceinline__ long long dist_units(float d) {
    if (!(d >= 1.f)) return 0;
    const unsigned b = __float_as_uint(d);
    const int e = (int)((b >> 23) & 0xffu) - 127;
    return (long long)((b & 0x7fffffu) | 0x800000u) << e;
}

// a value as an unevaluated sum h + l of two FP32 numbers
struct Pair {
    float h, l;
};
// a + b with the rounding error of the leading part kept (two-sum), then renormalised
__device__ __forceinline__ Pair pair_add(Pair a, Pair b) {
    const float s = a.h + b.h;
    const float bv = s - a.h;
    const float err = ((a.h - (s - bv)) + (b.h - bv)) + (a.l + b.l);
    const float h = s + err;
    return Pair{h, err - (h - s)};
}
// a - b rounded to FP32
__device__ __forceinline__ float pair_diff(Pair a, Pair b) {
    const float s = a.h - b.h;
    const float bv = s - a.h;
    const float err = (a.h - (s - bv)) + (-b.h - bv);
    return s + (err + (a.l - b.l));
}
__device__ __forceinline__ Pair pair_shfl_up(Pair v, int off) {
    return Pair{__shfl_up_sync(kFull, v.h, off), __shfl_up_sync(kFull, v.l, off)};
}

// One CTA per line of length L (L <= kBoxMaxLine): stage the line in shared memory, exact prefix
// sums, then each thread averages the windows of its contiguous chunk of `per` positions.  `per`
// is odd, so the 32 threads of a warp, per positions apart, touch 32 different shared-memory
// banks in the chunk loops.  Every distance is at least 1 (2^23 units), so positions more than
// rmax = floor(r) apart never share a window: a window's ends are searched within rmax positions.
// Results go back through shared memory for coalesced stores.
__global__ void __launch_bounds__(kBoxThreads) box_line_kernel(const float* src, long long sp, float* dst,
                                                               long long dstp, const float* d, long long dp, int L,
                                                               int lines, long long R, int per, int rmax, int top) {
    extern __shared__ __align__(16) unsigned char box_smem[];
    long long* ct = reinterpret_cast<long long*>(box_smem);  // L, in 2^-23 units
    float* Sh = reinterpret_cast<float*>(ct + L);            // L + 1: S[m] = x[0] + ... + x[m-1]
    float* Sl = Sh + (L + 1);                                //        as the pair (Sh, Sl)
    float* xs = Sl + (L + 1);                                // L: the line, later the results
    float* ds = xs + L;                                      // L
    __shared__ long long w_d[kBoxThreads / 32];
    __shared__ Pair w_x[kBoxThreads / 32];
    const int line = blockIdx.x;
    if (line >= lines) return;  // uniform over the CTA
    wait_predecessor();
    const float* xl = src + (long long)line * sp;
    const float* dl = d + (long long)line * dp;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        xs[i] = xl[i];
        ds[i] = i ? dl[i] : 0.f;  // ct[0] = 0: the first distance of a line is never used
    }
    __syncthreads();
    const int b = min((int)threadIdx.x * per, L);
    const int e = min(b + per, L);
    long long sd = 0;
    Pair sx = {0.f, 0.f};
    for (int i = b; i < e; ++i) {
        sd += dist_units(ds[i]);
        sx = pair_add(sx, Pair{xs[i], 0.f});
    }
    // exclusive scan of the chunk sums over the CTA: warp shuffles, then warp 0 scans the warp totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long id = sd;
    Pair ix = sx;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long od = __shfl_up_sync(kFull, id, off);
        const Pair ox = pair_shfl_up(ix, off);
        if (lane >= off) {
            id += od;
            ix = pair_add(ox, ix);
        }
    }
    if (lane == 31) {
        w_d[warp] = id;
        w_x[warp] = ix;
    }
    long long cd = __shfl_up_sync(kFull, id, 1);
    Pair cx = pair_shfl_up(ix, 1);
    if (lane == 0) {
        cd = 0;
        cx = Pair{0.f, 0.f};
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        long long vd = lane < nw ? w_d[lane] : 0;
        Pair vx = lane < nw ? w_x[lane] : Pair{0.f, 0.f};
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long od = __shfl_up_sync(kFull, vd, off);
            const Pair ox = pair_shfl_up(vx, off);
            if (lane >= off) {
                vd += od;
                vx = pair_add(ox, vx);
            }
        }
        long long ed = __shfl_up_sync(kFull, vd, 1);
        Pair ex = pair_shfl_up(vx, 1);
        if (lane == 0) {
            ed = 0;
            ex = Pair{0.f, 0.f};
        }
        if (lane < nw) {
            w_d[lane] = ed;
            w_x[lane] = ex;
        }
    }
    __syncthreads();
    cd += w_d[warp];
    cx = pair_add(w_x[warp], cx);
    for (int i = b; i < e; ++i) {
        cd += dist_units(ds[i]);
        ct[i] = cd;
        Sh[i] = cx.h;
        Sl[i] = cx.l;
        cx = pair_add(cx, Pair{xs[i], 0.f});
    }
    if (b < e && e == L) {
        Sh[L] = cx.h;
        Sl[L] = cx.l;
    }
    __syncthreads();
    release_successor();
    // each window's ends by binary lifting with the same number of steps in every thread (top: the
    // largest power of two <= rmax), so the warps do not diverge where a window jumps an edge.
    // xs[b..e) was last read by this thread above: the results replace it.
    for (int i = b; i < e; ++i) {
        const long long ci = ct[i];
        int lo = max(0, i - rmax);  // first m with ci - ct[m] <= R (m = i qualifies)
        int up = i;                 // last m <= min(L - 1, i + rmax) with ct[m] - ci <= R
        const int hb = min(L - 1, i + rmax);
        for (int st = top; st > 0; st >>= 1) {
            const int ml = min(lo + st - 1, i);
            if (ci - ct[ml] > R) lo = ml + 1;
            const int mu = min(up + st, hb);
            if (ct[mu] - ci <= R) up = mu;
        }
        xs[i] = __fdividef(pair_diff(Pair{Sh[up + 1], Sl[up + 1]}, Pair{Sh[lo], Sl[lo]}), (float)(up - lo + 1));
    }
    __syncthreads();
    float* out = dst + (long long)line * dstp;
    for (int i = threadIdx.x; i < L; i += blockDim.x) out[i] = xs[i];
}

// dst[x][y] = src[y][x] for an H x W plane (32 x 32 tiles through shared memory; 32 x kTransposeRows
// threads, each moving 32 / kTransposeRows elements with all its loads in flight)
constexpr int kTransposeRows = 8;
__global__ void __launch_bounds__(32 * kTransposeRows) transpose_kernel(const float* src, long long sp, float* dst,
                                                                        long long dp, int H, int W) {
    __shared__ float tile[32][33];
    wait_predecessor();
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
#pragma unroll
    for (int j = threadIdx.y; j < 32; j += kTransposeRows) {
        const int y = y0 + j, x = x0 + threadIdx.x;
        if (y < H && x < W) tile[j][threadIdx.x] = src[(long long)y * sp + x];
    }
    __syncthreads();
#pragma unroll
    for (int j = threadIdx.y; j < 32; j += kTransposeRows) {
        const int x = x0 + j, y = y0 + threadIdx.x;
        if (x < W && y < H) dst[(long long)x * dp + y] = tile[threadIdx.x][j];
    }
}

}  // namespace

size_t box_line_smem(int L) { return (size_t)L * 8 + (size_t)(L + 1) * 8 + (size_t)L * 8; }  // ct, S pairs, x, d

cudaError_t prepare_box_kernels() {
    return cudaFuncSetAttribute((const void*)box_line_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)box_line_smem(kBoxMaxLine));
}

cudaError_t launch_box_lines(const float* src, long long sp, float* dst, long long dstp, const float* d, long long dp,
                             int L, int lines, double r, cudaStream_t s) {
    if (L < 1 || L > kBoxMaxLine || !(r >= 0.0)) return cudaErrorInvalidValue;
    const long long R = (long long)floor(r * kBoxUnit);  // exact: r 2^23 scales by a power of two
    const int rmax = (int)std::min(floor(r), (double)L);
    int top = rmax > 0 ? 1 : 0;  // the largest power of two <= rmax
    while (top > 0 && 2 * top <= rmax) top *= 2;
    // the fewest odd positions per thread with at most kBoxThreads threads, whole warps
    int per = (L + kBoxThreads - 1) / kBoxThreads;
    if (per % 2 == 0) ++per;
    const int threads = ((L + per - 1) / per + 31) / 32 * 32;
    const int h = prof_begin(KID_BOX, (long long)L * lines, 0, s);
    const cudaError_t e = launch_ex_smem(box_line_kernel, dim3((unsigned)lines), dim3((unsigned)threads), 0,
                                         box_line_smem(L), s, src, sp, dst, dstp, d, dp, L, lines, R, per, rmax, top);
    prof_end(h, s);
    return e;
}

cudaError_t launch_transpose(const float* src, long long sp, float* dst, long long dp, int H, int W, cudaStream_t s) {
    const int h = prof_begin(KID_TRANSPOSE, (long long)H * W, 0, s);
    const dim3 grid((unsigned)((W + 31) / 32), (unsigned)((H + 31) / 32));
    const cudaError_t e = launch_ex(transpose_kernel, grid, dim3(32, kTransposeRows), 0, s, src, sp, dst, dp, H, W);
    prof_end(h, s);
    return e;
}

}  // namespace dts
