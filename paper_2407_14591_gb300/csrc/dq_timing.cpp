// Kernel timing hooks (dq_timing_enable / dq_timing_read): CUDA event pairs recorded on the
// caller's stream around the main kernel of every product call while timing is on.
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "dq_internal.h"

namespace dq {

namespace {
constexpr size_t kMaxTimed = 65536;
struct Timing {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> start, stop;  // event pairs, created on demand and reused
    size_t used = 0;
    long long launches = 0, kernels = 0;
    bool overflow = false;
};
Timing& timing() {
    static Timing t;
    return t;
}
}  // namespace

int timing_start(cudaStream_t st) {
    Timing& T = timing();
    std::lock_guard<std::mutex> lock(T.mu);
    if (!T.on) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
    if (T.used == kMaxTimed) {
        T.overflow = true;
        return -2;
    }
    if (T.used == T.start.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return -2;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return -2;
        }
        T.start.push_back(a);
        T.stop.push_back(b);
    }
    if (cudaEventRecord(T.start[T.used], st) != cudaSuccess) return -2;
    return (int)T.used++;
}

void timing_stop(int slot, cudaStream_t st, int kernels) {
    if (slot == -1) return;
    Timing& T = timing();
    std::lock_guard<std::mutex> lock(T.mu);
    T.launches += 1;
    T.kernels += kernels;
    if (slot >= 0) cudaEventRecord(T.stop[(size_t)slot], st);
}

}  // namespace dq

extern "C" {

int dq_timing_enable(int on) {
    dq::clear_error();
    dq::Timing& T = dq::timing();
    std::lock_guard<std::mutex> lock(T.mu);
    T.on = on != 0;
    if (T.on) {
        T.used = 0;
        T.launches = T.kernels = 0;
        T.overflow = false;
    }
    return DQ_OK;
}

int dq_timing_read(double* ms, long long* launches, long long* kernels) {
    dq::clear_error();
    dq::Timing& T = dq::timing();
    std::lock_guard<std::mutex> lock(T.mu);
    double sum = 0.0;
    for (size_t i = 0; i < T.used; ++i) {
        cudaError_t e = cudaEventSynchronize(T.stop[i]);
        float m = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&m, T.start[i], T.stop[i]);
        if (e != cudaSuccess) return dq::set_error(DQ_ECUDA, "timing events: %s", cudaGetErrorString(e));
        sum += m;
    }
    if (ms) *ms = sum;
    if (launches) *launches = T.launches;
    if (kernels) *kernels = T.kernels;
    if (T.overflow) return dq::set_error(DQ_ERANGE, "more than %zu timed launches since the last reset", dq::kMaxTimed);
    return DQ_OK;
}

}  // extern "C"
