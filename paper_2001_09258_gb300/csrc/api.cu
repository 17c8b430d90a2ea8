// Library-wide host helpers: thread-local error text, launch checks, grid
// sizing.  Grids are sized to the resident capacity of the device (SM count
// times resident blocks per SM for the kernel) and the kernels stride over the
// remaining work, so one launch fills all 152 SMs of a GB300.
#include <cstdarg>
#include <cstdio>
#include <mutex>
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

}  // namespace sleefcu

extern "C" const char *sleefcu_last_error(void) { return sleefcu::g_err; }
extern "C" const char *sleefcu_version(void) { return "sleefcu 0.1 (sm_103a)"; }
