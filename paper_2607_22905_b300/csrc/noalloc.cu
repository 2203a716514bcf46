// Allocation-free variant of the interface solve (no counterpart in the paper).
//
// Some callers cannot allocate device memory at the moment they need a solve: code that
// runs under a caller-managed memory pool or a fixed memory budget, real-time loops that
// must not enter the allocator, and hosts that forbid cudaMalloc after start-up.  For
// them algmortar_interface_solve_noalloc keeps its temporaries in a file-scope device
// array instead of handle workspace: the right-hand side and the solution in the
// nested-dissection order, and the per-group partial products of stage 1.
#include <mutex>
#include <string>

#include "algmortar.h"
#include "kernels.h"

namespace am {

// Maximum scratch: 2 * n_lambda + (sum of separator adjacencies) doubles.
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 20;   // 8 MiB per device

// Shared by every call on a device and kept until process exit; calls whose device work
// overlaps (other streams, other host threads) race on it.
static __device__ __align__(256) double g_iface_scratch[kNoAllocScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device, looked up once per device
// (host code cannot use the symbol itself as a device pointer).
cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_iface_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}
}  // namespace

// Called from the C ABI layer with the handle's solve description.
int interface_solve_noalloc(int device, cudaStream_t st, int L, const NdSolveArgs& nd, const int32_t* d_ndpos,
                            const double* b_dev, double* eta_dev, std::string& err) {
    if (L == 0) return ALGMORTAR_OK;
    // FP64 b, eta and P; with FP32 interface inverses also their FP32 side vectors
    const bool f32 = nd.Ginv32 || nd.Cinv32;
    const int64_t fl = f32 ? ((nd.L32 + nd.nsep4 + nd.nsep + 3) / 4) * 4 : 0;
    const int64_t need = 2 * (int64_t)L + nd.np + fl / 2 + 1;
    if (need > kNoAllocScratchDoubles) {
        err = "interface_solve_noalloc: needs " + std::to_string(need) + " doubles of scratch, the static array holds " +
              std::to_string(kNoAllocScratchDoubles) + " (n_lambda too large for the allocation-free path)";
        return ALGMORTAR_TOO_LARGE;
    }
    // the handle's device is made current for the launches and the caller's current
    // device is restored before returning (on every path)
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != device) e = cudaSetDevice(device);
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{e == cudaSuccess ? prev : -1, device};
    double* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) {
        err = std::string("interface_solve_noalloc: ") + cudaGetErrorString(e);
        return ALGMORTAR_CUDA;
    }
    double* b_nd = scratch;            // every entry written by the scatter below
    double* eta_nd = scratch + L;      // written by stages 1 (interior) and 2 (separator)
    double* P = scratch + 2 * (int64_t)L;   // written by stage 1 before stage 2 reads it
    // FP32 side vectors (16-byte aligned; written before they are read, as above)
    float* fv = f32 ? reinterpret_cast<float*>(scratch + ((2 * (int64_t)L + nd.np + 1) & ~int64_t(1))) : nullptr;
    launch_scatter(L, d_ndpos, b_dev, b_nd, st);
    launch_nd_solve(nd, b_nd, eta_nd, P, fv, fl, false, ColStrides{}, 1, st);
    launch_gather(L, d_ndpos, eta_nd, eta_dev, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("interface_solve_noalloc: ") + cudaGetErrorString(e);
        return ALGMORTAR_CUDA;
    }
    return ALGMORTAR_OK;
}

}  // namespace am
