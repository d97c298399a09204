// Per-launch kernel timing: while enabled, every kernel libdts launches is bracketed
// by two CUDA events recorded on the launch stream.  Used by the benchmark to take
// the duration of each kernel inside the timed region.
#include <mutex>
#include <vector>

#include "dts_internal.cuh"

namespace dts {

namespace {

struct Record {
    int kernel;
    long long pixels;
    int flags;
    cudaEvent_t start, stop;
};

std::mutex g_mu;
bool g_enabled = false;
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_pool;
constexpr size_t kMaxRecords = 1 << 16;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void recycle_all() {
    for (auto& r : g_records) {
        if (r.start) g_pool.push_back(r.start);
        if (r.stop) g_pool.push_back(r.stop);
    }
    g_records.clear();
}

}  // namespace

int prof_begin(int kernel, long long pixels, int flags, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_enabled || g_records.size() >= kMaxRecords) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;  // not in graphs
    Record r = {kernel, pixels, flags, take_event(), take_event()};
    if (!r.start || !r.stop) return -1;
    cudaEventRecord(r.start, s);
    g_records.push_back(r);
    return (int)g_records.size() - 1;
}

bool prof_active() {
    std::lock_guard<std::mutex> lock(g_mu);
    return g_enabled;
}

void prof_end(int handle, cudaStream_t s) {
    if (handle < 0) return;
    std::lock_guard<std::mutex> lock(g_mu);
    if (handle < (int)g_records.size()) cudaEventRecord(g_records[handle].stop, s);
}

}  // namespace dts

using namespace dts;

extern "C" int dts_profile(int mode) {
    if (mode < 0 || mode > 2) return DTS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (mode == 1) recycle_all();
    g_enabled = mode != 0;
    return DTS_OK;
}

extern "C" int dts_profile_read(int max_records, int* kernel, long long* pixels, int* flags, float* ms) {
    std::lock_guard<std::mutex> lock(g_mu);
    const int n = (int)g_records.size() < max_records ? (int)g_records.size() : max_records;
    for (int i = 0; i < n; ++i) {
        const Record& r = g_records[i];
        if (cudaEventSynchronize(r.stop) != cudaSuccess) return -DTS_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess) return -DTS_ERR_CUDA;
        if (kernel) kernel[i] = r.kernel;
        if (pixels) pixels[i] = r.pixels;
        if (flags) flags[i] = r.flags;
        if (ms) ms[i] = t;
    }
    return n;
}

extern "C" const char* dts_kernel_name(int kernel) {
    switch (kernel) {
        case KID_DISTANCES: return "distance_kernel";
        case KID_COPY: return "copy_plane_kernel";
        case KID_ROW_PLAIN: return "row_pass_kernel";
        case KID_ROW_SUPPORT: return "row_pass_kernel<support>";
        case KID_COL_PLAIN: return "col_pass_kernel";
        case KID_COL_SUPPORT: return "col_pass_kernel<support>";
        case KID_ROW_BWD: return "row_bwd_kernel";
        case KID_ROW_BWD_FINAL: return "row_bwd_kernel<final>";
        case KID_COL_BWD: return "col_bwd_kernel";
        case KID_GUIDE_GRAD: return "guide_grad_kernel";
        case KID_AXPY: return "axpy_plane_kernel";
        case KID_ROW_UPDATE: return "row_pass_kernel<update>";
        case KID_UPDATE: return "update_kernel";
        case KID_UPDATE_ADJ: return "update_adjoint_kernel";
        case KID_COL_STRIP: return "col_strip_kernel";
        case KID_SQUARE: return "square_plane_kernel";
        case KID_CONFIDENCE: return "confidence_kernel";
        case KID_BOX: return "box_line_kernel";
        case KID_TRANSPOSE: return "transpose_kernel";
        case KID_ROW_TRANSPOSE: return "row_pass_kernel<transpose>";
        case KID_COL_TRANSPOSE: return "col_pass_kernel<transpose>";
        case KID_CG_APPLY: return "cg_apply_kernel";
        case KID_CG_STEP: return "cg_step_kernel";
        case KID_CG_DIRECTION: return "cg_direction_kernel";
        case KID_COL_STRIP_TRANSPOSE: return "col_strip_kernel<transpose>";
        case KID_RESIDENT: return "resident_solve_kernel";
        case KID_COL_CHAIN: return "col_chain_kernel";
        case KID_COL_CHAIN_TRANSPOSE: return "col_chain_kernel<transpose>";
        case KID_COL_BWD_CHAIN: return "col_bwd_chain_kernel";
        case KID_COL_TALL: return "col_tall_kernel";
        case KID_COL_TALL_TRANSPOSE: return "col_tall_kernel<transpose>";
        case KID_BATCHED: return "batched_solve_kernel";
        case KID_ROW_STREAM: return "row_stream_kernel";
        case KID_ROW_STREAM_UPDATE: return "row_stream_kernel<update>";
        case KID_COL_BWD_AGG: return "col_bwd_agg_kernel";
        case KID_COL_BWD_APPLY: return "col_bwd_apply_kernel";
        case KID_COL_BWD_CARRY: return "col_bwd_carry_kernel";
        case KID_GUIDE_GRAD4: return "guide_grad_kernel<x4>";
        default: return "unknown";
    }
}
