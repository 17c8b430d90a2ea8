// Library-wide host helpers: thread-local error text, launch checks, grid
// sizing.  Grids are sized to the resident capacity of the device (SM count
// times resident blocks per SM for the kernel) and the kernels stride over the
// remaining work, so one launch fills all 152 SMs of a GB300.
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>
#ifdef SLEEFCU_CHECKED
#include <cuda.h>
#endif
#include "sleefcu_common.cuh"

namespace sleefcu {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

sleefcu_status check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SLEEFCU_ECUDA;
  }
  return SLEEFCU_OK;
}

namespace {
struct OccEntry { const void *k; int dev; int blocks; };
std::mutex g_mu;
OccEntry g_occ[512];
int g_nocc = 0;
int g_sms[64];
}  // namespace

int grid_for(const void *kernel, size_t work_items) {
  int dev = 0;
  cudaGetDevice(&dev);
  int cap = 0;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    for (int i = 0; i < g_nocc; i++)
      if (g_occ[i].k == kernel && g_occ[i].dev == dev) { cap = g_occ[i].blocks; break; }
    if (cap == 0) {
      if (dev < 64 && g_sms[dev] == 0) cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
      int sms = dev < 64 ? g_sms[dev] : 152;
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBlock, 0);
      if (per < 1) per = 1;
      cap = sms * per;
      if (g_nocc < 512) g_occ[g_nocc++] = OccEntry{kernel, dev, cap};
    }
  }
  size_t need = (work_items + kBlock - 1) / kBlock;
  if (need < 1) need = 1;
  return (int)(need < (size_t)cap ? need : (size_t)cap);
}

// ---------------- checked build ----------------
namespace {
std::mutex g_chk_mu;
std::vector<sleefcu_status (*)(unsigned long long *, int)> &checked_words() {
  static std::vector<sleefcu_status (*)(unsigned long long *, int)> v;
  return v;
}
}  // namespace

void register_checked_word(sleefcu_status (*read)(unsigned long long *, int)) {
  std::lock_guard<std::mutex> lock(g_chk_mu);
  checked_words().push_back(read);
}

#ifdef SLEEFCU_CHECKED
namespace {
// cuMemGetAddressRange through the runtime's driver entry point (no link
// dependency on libcuda): the base and size of the allocation holding p
typedef CUresult (*AddrRangeFn)(CUdeviceptr *, size_t *, CUdeviceptr);
AddrRangeFn addr_range_fn() {
  static AddrRangeFn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return (AddrRangeFn)f;
  }();
  return fn;
}
}  // namespace

sleefcu_status check_dev_range(const char *name, const void *p, size_t bytes) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: pointer %p: %s (checked build)", name, p, cudaGetErrorString(e));
    return SLEEFCU_EINVAL;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
    set_error("%s: %p is not device memory (memory type %d; checked build)", name, p, (int)a.type);
    return SLEEFCU_EINVAL;
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (a.device != dev) {
    set_error("%s: %p is memory of device %d, the current device is %d (checked build)", name, p, a.device, dev);
    return SLEEFCU_EINVAL;
  }
  if (a.type == cudaMemoryTypeDevice) {
    if (AddrRangeFn fn = addr_range_fn()) {
      CUdeviceptr base = 0;
      size_t size = 0;
      if (fn(&base, &size, (CUdeviceptr)(uintptr_t)p) == CUDA_SUCCESS &&
          (uintptr_t)p + bytes > (uintptr_t)base + size) {
        set_error("%s: %zu bytes from %p run past the end of its allocation (%zu bytes from %p; checked build)",
                  name, bytes, p, size, (void *)(uintptr_t)base);
        return SLEEFCU_EINVAL;
      }
    }
  }
  return SLEEFCU_OK;
}
#endif

}  // namespace sleefcu

extern "C" int sleefcu_is_checked(void) {
#ifdef SLEEFCU_CHECKED
  return 1;
#else
  return 0;
#endif
}

extern "C" sleefcu_status sleefcu_checked_error_count(unsigned long long *count, int reset) {
#ifdef SLEEFCU_CHECKED
  if (!count) { sleefcu::set_error("sleefcu_checked_error_count: null count"); return SLEEFCU_EINVAL; }
  *count = 0;
  std::lock_guard<std::mutex> lock(sleefcu::g_chk_mu);
  for (auto read : sleefcu::checked_words()) {
    if (read(count, reset) != SLEEFCU_OK) {
      sleefcu::set_error("sleefcu_checked_error_count: %s", cudaGetErrorString(cudaGetLastError()));
      return SLEEFCU_ECUDA;
    }
  }
  return SLEEFCU_OK;
#else
  (void)count;
  (void)reset;
  sleefcu::set_error("sleefcu_checked_error_count: not a checked build (load libsleefcu_checked.so)");
  return SLEEFCU_EUNSUPPORTED;
#endif
}

extern "C" const char *sleefcu_last_error(void) { return sleefcu::g_err; }
#ifdef SLEEFCU_CHECKED
extern "C" const char *sleefcu_version(void) { return "sleefcu 0.2 (sm_103a, checked)"; }
#else
extern "C" const char *sleefcu_version(void) { return "sleefcu 0.2 (sm_103a)"; }
#endif
