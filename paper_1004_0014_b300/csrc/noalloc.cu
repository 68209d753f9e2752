// Cost and gradient from projections without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// real-time guidance loop whose memory is all reserved at start-up (a
// cudaMalloc may synchronise the device and stall the frame), an application
// whose device memory belongs to another allocator, or code that runs where an
// allocation is not allowed at all. pr_cost_grad_static gives them the
// residual, cost and forward-mode gradient of the reconstruction (the same
// reduction kernel the solver uses) with its scratch in a fixed array that
// every GPU loading this library holds until the process exits.
#include <stdio.h>

#include <mutex>

#include "internal.h"
#include "pcarecon.h"

namespace {

// Scratch layout: block partial rows, the outputs, (a, b), the completion counter.
constexpr int kRows = 512;                       // >= the reduction's block count
constexpr size_t kPartialBytes = (size_t)kRows * pr::kMaxMom * sizeof(double);
constexpr size_t kOutOffset = kPartialBytes;            // 16 doubles
constexpr size_t kAbOffset = kOutOffset + 16 * sizeof(double);  // 2 doubles
constexpr size_t kCounterOffset = kAbOffset + 2 * sizeof(double);
constexpr size_t kScratchBytes = kCounterOffset + 256;  // 49,552 bytes in all

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices];  // device address of g_scratch, per device

__global__ void k_store_ab(double* ab, double a, double b) {
    ab[0] = a;
    ab[1] = b;
}

int err(int code, const char* msg) { return pr::set_last_error(code, msg); }

}  // namespace

extern "C" int pr_cost_grad_static(int device, void* stream, const float* p_dev, const float* q_dev,
                                   const float* y_dev, int R, int K, double a, double b, double* out_dev) {
    if (!p_dev || !q_dev || !y_dev || !out_dev) return err(PR_EINVAL, "null pointer argument");
    if (R < 1) return err(PR_EINVAL, "R must be at least 1");
    if (K < 1 || K > PR_MAX_K)
        return err(PR_EINVAL, "K must be 1..7: the static scratch holds 1 + 7 sums per block");
    if (device < 0 || device >= kMaxDevices) return err(PR_EINVAL, "device index out of range");
    if (pr::reduce_blocks() > kRows) return err(PR_EUNSUPPORTED, "reduction grid exceeds the static scratch");

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return err(PR_ECUDA, "cudaGetDevice failed");
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return err(PR_ECUDA, "cudaSetDevice failed");
    int rc = PR_OK;
    do {
        unsigned char* base = nullptr;
        {
            // One-time set-up per device, with that device current: the host-side
            // symbol is only a stand-in, the kernel needs its device address.
            std::lock_guard<std::mutex> lock(g_mutex);
            if (!g_scratch_ptr[device]) {
                void* ptr = nullptr;
                cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
                if (e != cudaSuccess || !ptr) {
                    rc = err(PR_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
                    break;
                }
                g_scratch_ptr[device] = static_cast<unsigned char*>(ptr);
            }
            base = g_scratch_ptr[device];
        }
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        double* partials = reinterpret_cast<double*>(base);
        double* out = reinterpret_cast<double*>(base + kOutOffset);
        double* ab = reinterpret_cast<double*>(base + kAbOffset);
        unsigned int* counter = reinterpret_cast<unsigned int*>(base + kCounterOffset);
        // The array keeps the previous call's contents: the completion counter
        // must start from zero.
        if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), s) != cudaSuccess) {
            rc = err(PR_ECUDA, "clearing the static counter failed");
            break;
        }
        // Launch errors come from each launch's own return code, so an
        // unrelated error the caller left pending is not taken for this call's.
        pr::Launcher L;
        L.stream = s;
        if (L(k_store_ab, dim3(1), dim3(1), 0, ab, a, b) != cudaSuccess ||
            pr::launch_cost_grad(L, p_dev, q_dev, y_dev, R, K, ab, partials, counter, out) != cudaSuccess) {
            rc = err(PR_ECUDA, "kernel launch failed");
            break;
        }
        if (cudaMemcpyAsync(out_dev, out, sizeof(double) * (1 + K), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = err(PR_ECUDA, "copy of the results failed");
            break;
        }
    } while (0);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}
