// qt_launch.cuh -- host-side launch helpers of the kernels' translation units.
//
// launch_k: one kernel launch through cudaLaunchKernelEx, whose return value
// is the launch's own status.  (cudaGetLastError after a <<<>>> launch would
// also return -- and clear -- an error the caller left pending from its own
// work, and report it as ours.)
//
// DeviceOnce: a set-up step (kernel attributes, device queries) run once per
// device, thread-safe: the serving loop's workers may make their first
// launches at the same time, and a process may drive several devices.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <utility>

namespace qt {

template <class... KArgs, class... Args>
inline int launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                    Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    return int(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

class DeviceOnce {
  public:
    static constexpr int kMaxDevices = 64;
    // Runs setup(dev) for the current device unless it already succeeded
    // there; returns 0 or the first failing cudaError_t.  A failed set-up is
    // tried again by the next call.
    template <class F>
    int run(F&& setup) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return int(e);
        if (dev < 0 || dev >= kMaxDevices) return int(cudaErrorInvalidDevice);
        if (done_[dev].load(std::memory_order_acquire)) return 0;
        std::lock_guard<std::mutex> lock(mu_);
        if (done_[dev].load(std::memory_order_relaxed)) return 0;
        const int rc = setup(dev);
        if (rc == 0) done_[dev].store(true, std::memory_order_release);
        return rc;
    }

  private:
    std::mutex mu_;
    std::atomic<bool> done_[kMaxDevices] = {};
};

}  // namespace qt
