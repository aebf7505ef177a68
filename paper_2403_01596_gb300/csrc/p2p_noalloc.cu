// Allocation-free leaf binning: p2p_bin_points with its scratch in a fixed
// device array instead of a caller-provided workspace.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need to bin points: real-time or embedded hosts that fix their whole
// device memory budget up front, and plug-ins whose host application owns the
// allocator and forbids device allocations from inside a callback.  For them
// p2p_bin_points_static takes the same inputs and outputs as p2p_bin_points
// but runs its sort and scan in the array below.  Like p2p_bin_points it
// synchronises the stream before returning (it reads the box count back).
//
// The array holds the scratch of P2P_BIN_STATIC_MAX_POINTS points (about
// 2 MiB).  It is a file-scope __device__ variable, so every GPU that loads
// this library keeps it until the process exits.  Host code cannot pass the
// array's name to a kernel (on the host the name is only a stand-in for the
// device symbol), so the first call on each device looks up its device
// address with cudaGetSymbolAddress while that device is current and keeps
// it; a teardown of the device's primary context (cudaDeviceReset) makes the
// kept address stale.  All calls on a device share the one array and it keeps
// the previous call's contents; the binning clears everything it needs
// zeroed.  Calls that overlap on the GPU (different streams, or different
// host threads on the same device) race on the array and must be serialised
// by the caller.
#include <mutex>

#include "p2p_internal.cuh"

namespace {

constexpr size_t kStaticBinBytes = 2162688;  // >= p2p_bin_workspace_size(P2P_BIN_STATIC_MAX_POINTS)
constexpr int kMaxDevices = 256;

static __device__ __align__(256) unsigned char g_bin_scratch[kStaticBinBytes];

std::mutex g_mutex;
void* g_scratch[kMaxDevices] = {};

// Device address of g_bin_scratch on the current device (looked up once per device).
p2p_status scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        p2p_detail::set_cuda_error(e, "p2p_bin_points_static");
        return P2P_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return P2P_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess) {
            p2p_detail::set_cuda_error(e, "p2p_bin_points_static/cudaGetSymbolAddress");
            return P2P_ERR_CUDA;
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return P2P_OK;
}

}  // namespace

extern "C" P2P_API p2p_status p2p_bin_points_static(const float* pts, int64_t n, const double lo[3], double h,
                                                    int32_t ng, int32_t* perm, int32_t* point_box, int64_t* box_keys,
                                                    int32_t* box_ptr, int32_t* num_boxes, p2p_stream_t stream) {
    if (n < 0 || n > P2P_BIN_STATIC_MAX_POINTS) {
        p2p_detail::set_message("p2p_bin_points_static: n exceeds P2P_BIN_STATIC_MAX_POINTS (65536)");
        return P2P_ERR_INVALID;
    }
    size_t need = 0;
    p2p_status st = p2p_bin_workspace_size(n, &need);
    if (st != P2P_OK) return st;
    if (need > kStaticBinBytes) return P2P_ERR_UNSUPPORTED;
    void* scratch = nullptr;
    st = scratch_for_current_device(&scratch);
    if (st != P2P_OK) return st;
    return p2p_bin_points(pts, n, lo, h, ng, perm, point_box, box_keys, box_ptr, num_boxes, scratch, kStaticBinBytes,
                          stream);
}
