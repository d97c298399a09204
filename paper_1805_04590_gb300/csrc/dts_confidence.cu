// Confidence from the edge-aware variance of the target (Eq. 7, §3.1): with DT the edge-aware
// mean of Eq. 10 (the filter of the solve), V = DT(t^2) - DT(t)^2 and c = exp(-V / (2 sigma_c^2)).
// The two filters run on the solve's pass kernels; these kernels square the target plane and
// turn the two filtered planes into the confidence.
#include "dts_scan.cuh"

namespace dts {

namespace {

using namespace scan;

// dst = src^2 over an H x W plane (both with row pitch `pitch`)
__global__ void __launch_bounds__(256) square_plane_kernel(const float* src, float* dst, long long pitch, int H,
                                                           int W) {
    wait_predecessor();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const long long i = (long long)y * pitch + x;
    const float v = src[i];
    dst[i] = v * v;
}

// c = exp(-max(m2 - m1^2, 0) * inv_2s2): m1 = DT(t), m2 = DT(t^2) (row pitch `pitch`), c dense.
// A variance below 0 can only come from rounding (DT is a non-negative average) and is taken as 0.
__global__ void __launch_bounds__(256) confidence_kernel(const float* m1, const float* m2, long long pitch, int H,
                                                         int W, float inv_2s2, float* c) {
    wait_predecessor();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const long long i = (long long)y * pitch + x;
    const float a = m1[i];
    const float v = fmaxf(fmaf(-a, a, m2[i]), 0.f);
    c[(long long)y * W + x] = expf(-v * inv_2s2);
}

}  // namespace

cudaError_t launch_square_plane(const float* src, float* dst, long long pitch, int H, int W, cudaStream_t s) {
    const int h = prof_begin(KID_SQUARE, (long long)H * W, 0, s);
    const dim3 grid((unsigned)((W + 255) / 256), (unsigned)H);
    const cudaError_t e = launch_ex(square_plane_kernel, grid, dim3(256), 0, s, src, dst, pitch, H, W);
    prof_end(h, s);
    return e;
}

cudaError_t launch_confidence(const float* m1, const float* m2, long long pitch, int H, int W, float sigma_c,
                              float* c, cudaStream_t s) {
    const int h = prof_begin(KID_CONFIDENCE, (long long)H * W, 0, s);
    const dim3 grid((unsigned)((W + 255) / 256), (unsigned)H);
    const float inv_2s2 = (float)(1.0 / (2.0 * (double)sigma_c * (double)sigma_c));
    const cudaError_t e = launch_ex(confidence_kernel, grid, dim3(256), 0, s, m1, m2, pitch, H, W, inv_2s2, c);
    prof_end(h, s);
    return e;
}

}  // namespace dts
