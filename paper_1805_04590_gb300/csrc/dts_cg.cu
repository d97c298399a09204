// Elementwise and reduction steps of conjugate gradients on the objective of Eq. 2,
//     F(z) = lambda/2 |z - A z|^2 + sum_i c_i (z_i - t_i)^2,
// whose minimiser solves M z = 2 C t with M = lambda (I - A)^T (I - A) + 2 C (symmetric
// positive definite for c > 0).  The paper names conjugate gradients as the method to speed up
// its solver (§5); the pass kernels apply A and A^T, these kernels do the rest of an iteration:
//
//   cg_apply_kernel      q = M p from u = A p and s = A^T (p - A p):  q = lambda (p - u - s) + 2 c p,
//                        with the block partials of p.q (or, for the start, r = 2 c t - M z_0,
//                        p = r and the partials of r.r)
//   cg_step_kernel       alpha = r.r / p.q;  z += alpha p;  r -= alpha q;  partials of the new r.r
//   cg_direction_kernel  beta = r.r(new) / r.r(old);  p = r + beta p
//
// A thread takes four consecutive pixels of a row (one 16-byte vector of each pitched plane) in
// a grid-stride loop.  A thread adds its few products in FP32 (GB300's FP64 rate is a small
// fraction of its FP32 rate, and an FP64 operation per pixel costs more time than the memory
// traffic); the thread sums are added in FP64 across the block, every block writes its partial
// sum, and the block that finishes last adds the partials in index order, so the scalars do not
// depend on the order the blocks ran in.  The scalars stay on the device (no host round trip
// between the kernels of an iteration).
#include "dts_scan.cuh"

namespace dts {

namespace {

using namespace scan;

constexpr int kCgThreads = 256;

// four values of a dense plane (row pitch W) at dense index i, x0 = first column
__device__ __forceinline__ void load4_dense(const float* base, long long i, int x0, int W, bool vec, float* out) {
    if (vec) {
        load4_f(base, i, out);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = x0 + k < W ? base[i + k] : 0.f;
    }
}

// Sum of v over the grid: the block's sum goes to partials[blockIdx.x]; the last block to arrive
// adds the partials in index order into *out and clears the ticket for the next kernel.
__device__ __forceinline__ void grid_sum(double v, double* partials, unsigned* ticket, double* out) {
    __shared__ double s_w[kCgThreads / 32];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < kCgThreads / 32; ++i) b += s_w[i];
        partials[blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kCgThreads) acc += __ldcg(partials + i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) s_w[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < kCgThreads / 32; ++i) b += s_w[i];
        *out = b;
        *ticket = 0u;
    }
}

// INIT: p holds z_0; writes r = 2 c t - M z_0 and p = r, sums r.r.  Else writes q = M p, sums p.q.
template <bool INIT>
__global__ void __launch_bounds__(kCgThreads) cg_apply_kernel(CgArgs a) {
    wait_predecessor();
    const unsigned Qp = (unsigned)(a.pitch >> 2);
    const unsigned units = (unsigned)a.H * Qp;
    float acc = 0.f;
    for (unsigned u = blockIdx.x * kCgThreads + threadIdx.x; u < units; u += gridDim.x * kCgThreads) {
        const int y = (int)(u / Qp);
        const int x0 = (int)(u - (unsigned)y * Qp) * 4;
        if (x0 >= a.W) continue;
        const long long i = (long long)y * a.pitch + x0;
        const long long di = (long long)y * a.W + x0;
        float p[4], Ap[4], s[4], c[4], t[4];
        load4_f(INIT ? a.z : a.p, i, p);
        load4_f(a.u, i, Ap);
        load4_f(a.s, i, s);
        load4_dense(a.c, di, x0, a.W, a.dvec, c);
        if constexpr (INIT) {
#pragma unroll
            for (int k = 0; k < 4; ++k) t[k] = x0 + k < a.W ? load_any(a.t, di + k, a.t_dtype) : 0.f;
        }
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = x0 + k < a.W;
            const float mp = fmaf(a.lambda, (p[k] - Ap[k]) - s[k], 2.f * c[k] * p[k]);
            if constexpr (INIT) {
                o[k] = ok ? fmaf(2.f * c[k], t[k], -mp) : 0.f;
                acc = fmaf(o[k], o[k], acc);
            } else {
                o[k] = ok ? mp : 0.f;
                acc = fmaf(ok ? p[k] : 0.f, o[k], acc);
            }
        }
        if constexpr (INIT) {
            store4_f(a.r, i, o);
            store4_f(a.p, i, o);
        } else {
            store4_f(a.q, i, o);
        }
    }
    release_successor();
    grid_sum((double)acc, a.partials, a.ticket, a.scal + (INIT ? a.slot_rr : kCgSlotPq));
}

// alpha = rr / pq (0 once the residual or the direction vanishes: the iteration has stopped)
__global__ void __launch_bounds__(kCgThreads) cg_step_kernel(CgArgs a) {
    wait_predecessor();
    const double rr = a.scal[a.slot_rr];
    const double pq = a.scal[kCgSlotPq];
    const float alpha = (rr > 0.0 && pq > 0.0) ? (float)(rr / pq) : 0.f;
    const unsigned Qp = (unsigned)(a.pitch >> 2);
    const unsigned units = (unsigned)a.H * Qp;
    float acc = 0.f;
    for (unsigned u = blockIdx.x * kCgThreads + threadIdx.x; u < units; u += gridDim.x * kCgThreads) {
        const int y = (int)(u / Qp);
        const int x0 = (int)(u - (unsigned)y * Qp) * 4;
        if (x0 >= a.W) continue;
        const long long i = (long long)y * a.pitch + x0;
        float z[4], p[4], r[4], q[4];
        load4_f(a.z, i, z);
        load4_f(a.p, i, p);
        load4_f(a.r, i, r);
        load4_f(a.q, i, q);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            z[k] = fmaf(alpha, p[k], z[k]);
            r[k] = fmaf(-alpha, q[k], r[k]);
            if (x0 + k < a.W) acc = fmaf(r[k], r[k], acc);
        }
        store4_f(a.r, i, r);
        if (a.zout_vec) {
            store4_f(a.zout, (long long)y * a.zout_pitch + x0, z);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (x0 + k < a.W) a.zout[(long long)y * a.zout_pitch + x0 + k] = z[k];
        }
    }
    release_successor();
    grid_sum((double)acc, a.partials, a.ticket, a.scal + (a.slot_rr ^ 1));
}

__global__ void __launch_bounds__(kCgThreads) cg_direction_kernel(CgArgs a) {
    wait_predecessor();
    const double rr_old = a.scal[a.slot_rr];
    const double rr_new = a.scal[a.slot_rr ^ 1];
    const float beta = rr_old > 0.0 ? (float)(rr_new / rr_old) : 0.f;
    const unsigned Qp = (unsigned)(a.pitch >> 2);
    const unsigned units = (unsigned)a.H * Qp;
    for (unsigned u = blockIdx.x * kCgThreads + threadIdx.x; u < units; u += gridDim.x * kCgThreads) {
        const int y = (int)(u / Qp);
        const int x0 = (int)(u - (unsigned)y * Qp) * 4;
        if (x0 >= a.W) continue;
        const long long i = (long long)y * a.pitch + x0;
        float p[4], r[4];
        load4_f(a.p, i, p);
        load4_f(a.r, i, r);
#pragma unroll
        for (int k = 0; k < 4; ++k) p[k] = fmaf(beta, p[k], r[k]);
        store4_f(a.p, i, p);
    }
    release_successor();
}

int cg_sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

// blocks of the CG kernels for an H x (pitch) plane: 8 resident blocks of 256 threads per SM at
// most (the grid-stride loop covers the rest), never more than kCgMaxBlocks partials
int cg_blocks(int H, long long pitch) {
    const long long units = (long long)H * (pitch >> 2);
    long long b = (units + kCgThreads - 1) / kCgThreads;
    const long long cap = 8LL * cg_sm_count();
    if (b > cap) b = cap;
    if (b > kCgMaxBlocks) b = kCgMaxBlocks;
    return b < 1 ? 1 : (int)b;
}

cudaError_t launch_cg_apply(const CgArgs& a, bool init, cudaStream_t s) {
    const int h = prof_begin(KID_CG_APPLY, (long long)a.H * a.W, 0, s);
    const dim3 grid((unsigned)cg_blocks(a.H, a.pitch));
    const cudaError_t e = init ? launch_ex(cg_apply_kernel<true>, grid, dim3(kCgThreads), 0, s, a)
                               : launch_ex(cg_apply_kernel<false>, grid, dim3(kCgThreads), 0, s, a);
    prof_end(h, s);
    return e;
}

cudaError_t launch_cg_step(const CgArgs& a, cudaStream_t s) {
    const int h = prof_begin(KID_CG_STEP, (long long)a.H * a.W, 0, s);
    const cudaError_t e = launch_ex(cg_step_kernel, dim3((unsigned)cg_blocks(a.H, a.pitch)), dim3(kCgThreads), 0, s, a);
    prof_end(h, s);
    return e;
}

cudaError_t launch_cg_direction(const CgArgs& a, cudaStream_t s) {
    const int h = prof_begin(KID_CG_DIRECTION, (long long)a.H * a.W, 0, s);
    const cudaError_t e =
        launch_ex(cg_direction_kernel, dim3((unsigned)cg_blocks(a.H, a.pitch)), dim3(kCgThreads), 0, s, a);
    prof_end(h, s);
    return e;
}

}  // namespace dts
