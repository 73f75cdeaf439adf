// Allocation-free variant of the batched float64 eigensolver entry point.
//
// Some callers cannot allocate device memory while they call us: hosts that
// reserve all device memory up front for their own allocator (an
// allocation here would fail, or would go around the pool that accounts
// for every byte), and latency-bound callers that cannot afford the device
// synchronisation and driver round trip a fresh allocation may cost.  For
// them mpspt_eigh_batched_noalloc keeps its working storage (the task table
// and the work copy of the input matrices) in one fixed, file-scope device
// array instead of allocating it per call.
//
// The array is 2^21 doubles (16 MiB) per device that loads the
// library and stays allocated until the process exits.  Every call shares
// it: calls whose GPU work overlaps (different streams, or several host
// threads) race on it and must be serialised by the caller.  Each call
// overwrites all of the storage it uses, so nothing carries over from the
// previous call.  The call makes `device` current for its own work and puts
// the caller's current device back before it returns, on every path.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/mpspt.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchDoubles = (size_t)1 << 21;          // 16 MiB
constexpr int kMaxBatch = 1024;
constexpr size_t kTaskDoubles = kMaxBatch * sizeof(mpspt::EigTask) / sizeof(double);

static __device__ __align__(256) double g_eigh_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_addr[64] = {};   // device address of g_eigh_scratch, per device

// Resolve the device address of the scratch array for `device` (current).
mpspt_status scratch_address(int device, double** out) {
    if (device < 0 || device >= 64) return MPSPT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_eigh_scratch) != cudaSuccess || p == nullptr) return MPSPT_ERR_CUDA;
        g_addr[device] = static_cast<double*>(p);
    }
    *out = g_addr[device];
    return MPSPT_OK;
}

// Makes `device` current for the lifetime of the guard and restores the
// device that was current before.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" mpspt_status mpspt_eigh_batched_noalloc(int device, void* stream, int batch, const int* n,
                                                   const double* A, double* V, double* w) {
    if (batch < 1 || batch > kMaxBatch || !n || !A || !V || !w) return MPSPT_ERR_INVALID;
    size_t tot = 0;
    for (int i = 0; i < batch; ++i) {
        if (n[i] < 1 || n[i] > 2048) return MPSPT_ERR_INVALID;
        tot += (size_t)n[i] * n[i];
    }
    if (tot > kScratchDoubles - kTaskDoubles) return MPSPT_ERR_INVALID;   // beyond the fixed scratch
    DeviceGuard dg(device);
    if (!dg.ok) return MPSPT_ERR_CUDA;
    double* base = nullptr;
    const mpspt_status s = scratch_address(device, &base);
    if (s != MPSPT_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mpspt::EigTask tasks[kMaxBatch];
    double* work = base + kTaskDoubles;
    size_t o = 0, ow = 0;
    for (int i = 0; i < batch; ++i) {
        tasks[i] = {work + o, V + o, w + ow, n[i], 0};
        o += (size_t)n[i] * n[i];
        ow += (size_t)n[i];
    }
    if (cudaMemcpyAsync(work, A, tot * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MPSPT_ERR_CUDA;
    if (cudaMemcpyAsync(base, tasks, batch * sizeof(mpspt::EigTask), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return MPSPT_ERR_CUDA;
    mpspt::launch_eig(reinterpret_cast<const mpspt::EigTask*>(base), batch, st);
    if (cudaGetLastError() != cudaSuccess) return MPSPT_ERR_CUDA;
    return MPSPT_OK;
}
