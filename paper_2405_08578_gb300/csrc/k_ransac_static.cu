// lp_ransac_static: the RANSAC stage with its scratch memory in a fixed,
// file-scope device array, for callers that cannot allocate device memory.
//
// Why: lp_ransac keeps its per-iteration scratch (hypotheses, inlier counts,
// the winning index) in workspace that the context grows with cudaMalloc,
// and creating a context allocates too.  Some callers cannot do that: a host
// application whose own caching allocator has reserved the device's memory,
// a real-time loop that must not enter the driver's allocation path (which
// may synchronise the device and take unbounded time), or a plug-in host that
// forbids device allocations after start-up.  This entry point needs no
// context and calls no allocating routine; the caller passes inputs and
// outputs, and the scratch lives in `g_ransac_scratch` below.
//
// The array is loaded with the library and stays resident on every GPU that
// loads it until the process exits.  Every call shares it (it keeps the last
// call's contents), so calls that overlap on the GPU -- on different streams,
// or from several host threads without ordering -- race on it.  The kernels
// write every scratch word before they read it, so nothing has to start at
// zero.
#include <mutex>

#include "lp_internal.cuh"

namespace {

constexpr size_t kScratchBytes = 393216;   // 384 KiB: T <= LP_RANSAC_STATIC_MAX_ITERS

static __device__ __align__(256) unsigned char g_ransac_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device (host code only sees a
// host-side stand-in under the array's name).  Looked up once per device.
int scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_ransac_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return LP_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return LP_OK;
}

}  // namespace

extern "C" LP_API int lp_ransac_static(const float* pts, int64_t M_cap, const int32_t* d_M, int iters, float thresh_px,
                                       uint64_t seed, uint32_t pair_id, double* H, uint8_t* inlier,
                                       int32_t* n_inliers, int32_t* best_t, void* stream)
{
    if (iters < 1 || iters > LP_RANSAC_STATIC_MAX_ITERS) return LP_ERR_ARG;
    if (M_cap < 0 || M_cap > (1ll << 31) - 1 || !(thresh_px > 0.f)) return LP_ERR_ARG;
    if (!H || !n_inliers || (M_cap > 0 && (!pts || !inlier))) return LP_ERR_ARG;
    if (pts && (reinterpret_cast<uintptr_t>(pts) & 15)) return LP_ERR_ALIGN;
    if (lp::ransac_workspace(M_cap, iters) > kScratchBytes) return LP_ERR_ARG;
    void* scratch = nullptr;
    const int r = scratch_address(&scratch);
    if (r != LP_OK) return r;
    const cudaError_t e = lp::launch_ransac(pts, M_cap, d_M, iters, LP_MODEL_HOMOGRAPHY, thresh_px, seed, pair_id, H,
                                            inlier, n_inliers, best_t, scratch, kScratchBytes,
                                            static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}
