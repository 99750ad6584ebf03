// dq_matvec_noalloc: the panel products with their scratch in a fixed, file-scope device array,
// for callers that must not allocate device memory while they run (see include/dq.h).
//
// The scratch holds the workspace header and the fixed-point copy of x that the panel kernels
// read (dq_panel.cu, dq_panel_w.cu, dq_panel_q.cu). The array is static: it is reserved when the code module that holds it
// is loaded on a GPU and stays reserved until the process exits. Under CUDA's default lazy
// module loading this file's module (it has no kernels of its own) is loaded by the first
// cudaGetSymbolAddress on each device, i.e. inside the first dq_matvec_noalloc call there, which
// is therefore the call that takes the 64 MiB from the device. Host code never dereferences the
// symbol; it asks the runtime for the array's device address once per device and passes that
// address to the kernels.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "dq_internal.h"

namespace dq {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB per GPU
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices];

// Device address of the static scratch on the current device; set up on first use.
static int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(DQ_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(DQ_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(DQ_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return DQ_OK;
}

}  // namespace dq

using namespace dq;

extern "C" int dq_matvec_noalloc(const dq_sector* s, const dq_terms* t, const void* x, void* y, int dtype,
                                 void* stream) {
    clear_error();
    if (!s || !t || !x || !y) return set_error(DQ_EINVAL, "NULL argument");
    if (t->sector != s) return set_error(DQ_EINVAL, "terms were compiled for another sector");
    if (!s->has_device) return set_error(DQ_ECUDA, "no CUDA device: the sector has host tables only");
    if (dtype != DQ_F64 && dtype != DQ_F32) return set_error(DQ_EINVAL, "dtype must be DQ_F64 or DQ_F32");
    if (!t->panel_ok && !t->pw_ok && !t->pq_ok)
        return set_error(DQ_EINVAL, "dq_matvec_noalloc serves only terms on the panel paths (dq_terms_path 1, 4 or 5)");
    // the boson panel kernel keeps x as split 64-bit words for both dtypes
    const size_t need = panel_scratch_bytes(s, t->pq_ok && !t->panel_ok && !t->pw_ok ? DQ_F64 : dtype);
    if (need > kNoAllocScratchBytes)
        return set_error(DQ_ERANGE,
                         "sector too large for the static scratch: needs %zu bytes, the limit is %zu bytes "
                         "(D <= %zu for DQ_F64, D <= %zu for DQ_F32)",
                         need, kNoAllocScratchBytes, (kNoAllocScratchBytes - 256) / 8 - 8,
                         (kNoAllocScratchBytes - 256) / 4 - 8);
    const size_t bytes = (size_t)s->D * (dtype == DQ_F64 ? 8 : 4);
    const char* xb = (const char*)x;
    char* yb = (char*)y;
    if (xb < yb + bytes && yb < xb + bytes) return set_error(DQ_EINVAL, "x and y overlap");
    void* ws = nullptr;
    int rc = noalloc_scratch(&ws);
    if (rc) return rc;
    int e = t->panel_ok ? launch_panel_matvec_ws(s, t, x, y, dtype, ws, stream)
            : t->pw_ok  ? launch_panel_w_ws(s, t, x, y, dtype, ws, stream)
                        : launch_panel_q_ws(s, t, x, y, dtype, ws, stream);
    if (e) return set_error(DQ_ECUDA, "matvec_noalloc launch: %s", cudaGetErrorString((cudaError_t)e));
    return DQ_OK;
}
