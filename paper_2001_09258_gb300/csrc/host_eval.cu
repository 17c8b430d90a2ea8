// Evaluation from and to host memory: the end-to-end form of every entry
// point.  A caller whose arrays live in host memory hands the library one
// descriptor; the library streams it through device buffers it owns, in
// chunks, with copies in, kernels and copies out of up to six chunks in
// flight at once on three streams (the per-element work
// is the same entry point, so every result equals the device call's bit for
// bit).  Staging buffers and streams are created on the first call per
// device and reused; the call returns when every result is in host memory.
#include "sleefcu_common.cuh"

#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

namespace {
using namespace sleefcu;

typedef sleefcu_status (*EvalFn)(const void *x, const void *y, void *o, void *o2, size_t n, sleefcu_stream s);
struct Entry {
  const char *name;
  int esz, nin, nout;
  EvalFn f;
};

#define HE_U(NAME, T, ESZ)                                                                     \
  {#NAME, ESZ, 1, 1, [](const void *x, const void *, void *o, void *, size_t n, sleefcu_stream s) { \
     return sleefcu_##NAME((const T *)x, (T *)o, n, s); }},
#define HE_B(NAME, T, ESZ)                                                                     \
  {#NAME, ESZ, 2, 1, [](const void *x, const void *y, void *o, void *, size_t n, sleefcu_stream s) { \
     return sleefcu_##NAME((const T *)x, (const T *)y, (T *)o, n, s); }},
#define HE_SC(NAME, T, ESZ)                                                                    \
  {#NAME, ESZ, 1, 2, [](const void *x, const void *, void *o, void *o2, size_t n, sleefcu_stream s) { \
     return sleefcu_##NAME((const T *)x, (T *)o, (T *)o2, n, s); }},
const Entry kEntries[] = {
  HE_U(sin_u10_f64, double, 8)
  HE_U(sin_u35_f64, double, 8)
  HE_U(sin_u10_f32, float, 4)
  HE_U(sin_u35_f32, float, 4)
  HE_U(cos_u10_f64, double, 8)
  HE_U(cos_u35_f64, double, 8)
  HE_U(cos_u10_f32, float, 4)
  HE_U(cos_u35_f32, float, 4)
  HE_U(tan_u10_f64, double, 8)
  HE_U(tan_u35_f64, double, 8)
  HE_U(tan_u10_f32, float, 4)
  HE_U(tan_u35_f32, float, 4)
  HE_SC(sincos_u10_f64, double, 8)
  HE_SC(sincos_u35_f64, double, 8)
  HE_SC(sincos_u10_f32, float, 4)
  HE_SC(sincos_u35_f32, float, 4)
  HE_U(asin_u10_f64, double, 8)
  HE_U(asin_u35_f64, double, 8)
  HE_U(asin_u10_f32, float, 4)
  HE_U(asin_u35_f32, float, 4)
  HE_U(acos_u10_f64, double, 8)
  HE_U(acos_u35_f64, double, 8)
  HE_U(acos_u10_f32, float, 4)
  HE_U(acos_u35_f32, float, 4)
  HE_U(atan_u10_f64, double, 8)
  HE_U(atan_u35_f64, double, 8)
  HE_U(atan_u10_f32, float, 4)
  HE_U(atan_u35_f32, float, 4)
  HE_B(atan2_u10_f64, double, 8)
  HE_B(atan2_u35_f64, double, 8)
  HE_B(atan2_u10_f32, float, 4)
  HE_B(atan2_u35_f32, float, 4)
  HE_U(exp_u10_f64, double, 8)
  HE_U(exp_u35_f64, double, 8)
  HE_U(exp_u10_f32, float, 4)
  HE_U(exp_u35_f32, float, 4)
  HE_U(exp_u10_bf16, void, 2)
  HE_U(exp_u35_bf16, void, 2)
  HE_U(exp_u10_f16, void, 2)
  HE_U(exp_u35_f16, void, 2)
  HE_U(log_u10_f64, double, 8)
  HE_U(log_u35_f64, double, 8)
  HE_U(log_u10_f32, float, 4)
  HE_U(log_u35_f32, float, 4)
  HE_B(pow_u10_f64, double, 8)
  HE_B(pow_u35_f64, double, 8)
  HE_B(pow_u10_f32, float, 4)
  HE_B(pow_u35_f32, float, 4)
  HE_B(fmod_u10_f64, double, 8)
  HE_B(fmod_u35_f64, double, 8)
  HE_B(fmod_u10_f32, float, 4)
  HE_B(fmod_u35_f32, float, 4)
  HE_B(remainder_u10_f64, double, 8)
  HE_B(remainder_u35_f64, double, 8)
  HE_B(remainder_u10_f32, float, 4)
  HE_B(remainder_u35_f32, float, 4)
  HE_U(log1p_u10_f64, double, 8)
  HE_U(log1p_u35_f64, double, 8)
  HE_U(log1p_u10_f32, float, 4)
  HE_U(log1p_u35_f32, float, 4)
  HE_U(log1p_u10_bf16, void, 2)
  HE_U(log1p_u35_bf16, void, 2)
  HE_U(log1p_u10_f16, void, 2)
  HE_U(log1p_u35_f16, void, 2)
  HE_U(tanh_u10_f64, double, 8)
  HE_U(tanh_u35_f64, double, 8)
  HE_U(tanh_u10_f32, float, 4)
  HE_U(tanh_u35_f32, float, 4)
  HE_U(tanh_u10_bf16, void, 2)
  HE_U(tanh_u35_bf16, void, 2)
  HE_U(tanh_u10_f16, void, 2)
  HE_U(tanh_u35_f16, void, 2)
  HE_U(erf_u10_f64, double, 8)
  HE_U(erf_u35_f64, double, 8)
  HE_U(erf_u10_f32, float, 4)
  HE_U(erf_u35_f32, float, 4)
  HE_U(erf_u10_bf16, void, 2)
  HE_U(erf_u35_bf16, void, 2)
  HE_U(erf_u10_f16, void, 2)
  HE_U(erf_u35_f16, void, 2)
  HE_U(exp2_u10_f64, double, 8)
  HE_U(exp2_u35_f64, double, 8)
  HE_U(exp2_u10_f32, float, 4)
  HE_U(exp2_u35_f32, float, 4)
  HE_U(exp10_u10_f64, double, 8)
  HE_U(exp10_u35_f64, double, 8)
  HE_U(exp10_u10_f32, float, 4)
  HE_U(exp10_u35_f32, float, 4)
  HE_U(expm1_u10_f64, double, 8)
  HE_U(expm1_u35_f64, double, 8)
  HE_U(expm1_u10_f32, float, 4)
  HE_U(expm1_u35_f32, float, 4)
  HE_U(log2_u10_f64, double, 8)
  HE_U(log2_u35_f64, double, 8)
  HE_U(log2_u10_f32, float, 4)
  HE_U(log2_u35_f32, float, 4)
  HE_U(log10_u10_f64, double, 8)
  HE_U(log10_u35_f64, double, 8)
  HE_U(log10_u10_f32, float, 4)
  HE_U(log10_u35_f32, float, 4)
  HE_U(cbrt_u10_f64, double, 8)
  HE_U(cbrt_u35_f64, double, 8)
  HE_U(cbrt_u10_f32, float, 4)
  HE_U(cbrt_u35_f32, float, 4)
  HE_U(sinh_u10_f64, double, 8)
  HE_U(sinh_u35_f64, double, 8)
  HE_U(sinh_u10_f32, float, 4)
  HE_U(sinh_u35_f32, float, 4)
  HE_U(cosh_u10_f64, double, 8)
  HE_U(cosh_u35_f64, double, 8)
  HE_U(cosh_u10_f32, float, 4)
  HE_U(cosh_u35_f32, float, 4)
  HE_U(asinh_u10_f64, double, 8)
  HE_U(asinh_u35_f64, double, 8)
  HE_U(asinh_u10_f32, float, 4)
  HE_U(asinh_u35_f32, float, 4)
  HE_U(acosh_u10_f64, double, 8)
  HE_U(acosh_u35_f64, double, 8)
  HE_U(acosh_u10_f32, float, 4)
  HE_U(acosh_u35_f32, float, 4)
  HE_U(atanh_u10_f64, double, 8)
  HE_U(atanh_u35_f64, double, 8)
  HE_U(atanh_u10_f32, float, 4)
  HE_U(atanh_u35_f32, float, 4)
  HE_U(erfc_u10_f64, double, 8)
  HE_U(erfc_u35_f64, double, 8)
  HE_U(erfc_u10_f32, float, 4)
  HE_U(erfc_u35_f32, float, 4)
  HE_U(tgamma_u10_f64, double, 8)
  HE_U(tgamma_u35_f64, double, 8)
  HE_U(tgamma_u10_f32, float, 4)
  HE_U(tgamma_u35_f32, float, 4)
  HE_U(lgamma_u10_f64, double, 8)
  HE_U(lgamma_u35_f64, double, 8)
  HE_U(lgamma_u10_f32, float, 4)
  HE_U(lgamma_u35_f32, float, 4)
};
#undef HE_U
#undef HE_B
#undef HE_SC

const char *kFn[SLEEFCU_FN_COUNT] = {"sin",   "cos",   "tan",   "sincos", "asin",  "acos",  "atan",
                                     "atan2", "exp",   "log",   "pow",    "fmod",  "remainder",
                                     "log1p", "tanh",  "erf",   "exp2",   "exp10", "expm1", "log2",
                                     "log10", "cbrt",  "sinh",  "cosh",   "asinh", "acosh", "atanh",
                                     "erfc",  "tgamma", "lgamma"};
const char *kType[4] = {"f64", "f32", "bf16", "f16"};

const Entry *find(const sleefcu_batch_item &it) {
  if (it.fn >= SLEEFCU_FN_COUNT || it.dtype > 3 || (it.ulp != 10 && it.ulp != 35)) return nullptr;
  char name[64];
  snprintf(name, sizeof name, "%s_u%d_%s", kFn[it.fn], it.ulp, kType[it.dtype]);
  for (const Entry &e : kEntries)
    if (!strcmp(e.name, name)) return &e;
  return nullptr;
}

// chunks in flight: deep enough that the copy engines run ahead through
// items whose kernels are slow and the kernels through items whose copies
// are slow (a fast FP64 function moves its 16 bytes per element faster than
// the host link carries them, a slow one leaves the link idle)
constexpr int kDepth = 6;
constexpr int kMaxDev = 64;
struct Stage {
  bool ready = false;
  cudaStream_t in = nullptr, run = nullptr, out = nullptr;
  cudaEvent_t loaded[kDepth], done[kDepth], freed[kDepth];
  void *buf[kDepth][4] = {};                   // x, y, out, out2 per slot
  size_t bytes = 0;                            // capacity of each buffer
};
std::mutex g_mu[kMaxDev];
Stage g_stage[kMaxDev];

sleefcu_status cuda_fail(const char *what, cudaError_t e) {
  set_error("sleefcu_eval_host: %s: %s", what, cudaGetErrorString(e));
  return SLEEFCU_ECUDA;
}

sleefcu_status prepare(Stage &st, size_t bytes) {
  cudaError_t e;
  if (!st.ready) {
    if ((e = cudaStreamCreateWithFlags(&st.in, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail("stream", e);
    if ((e = cudaStreamCreateWithFlags(&st.run, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail("stream", e);
    if ((e = cudaStreamCreateWithFlags(&st.out, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail("stream", e);
    for (int b = 0; b < kDepth; b++) {
      if ((e = cudaEventCreateWithFlags(&st.loaded[b], cudaEventDisableTiming)) != cudaSuccess) return cuda_fail("event", e);
      if ((e = cudaEventCreateWithFlags(&st.done[b], cudaEventDisableTiming)) != cudaSuccess) return cuda_fail("event", e);
      if ((e = cudaEventCreateWithFlags(&st.freed[b], cudaEventDisableTiming)) != cudaSuccess) return cuda_fail("event", e);
    }
    st.ready = true;
  }
  if (bytes > st.bytes) {
    for (int b = 0; b < kDepth; b++)
      for (int k = 0; k < 4; k++) {
        if (st.buf[b][k]) cudaFree(st.buf[b][k]);
        st.buf[b][k] = nullptr;
      }
    st.bytes = 0;
    for (int b = 0; b < kDepth; b++)
      for (int k = 0; k < 4; k++)
        if ((e = cudaMalloc(&st.buf[b][k], bytes)) != cudaSuccess) {
          set_error("sleefcu_eval_host: staging buffers of %zu bytes: %s", bytes, cudaGetErrorString(e));
          return SLEEFCU_ENOMEM;
        }
    st.bytes = bytes;
  }
  return SLEEFCU_OK;
}

// every item's entry and pointers, before any work
sleefcu_status check_items(const sleefcu_batch_item *items, size_t count, const Entry **ens) {
  for (size_t i = 0; i < count; i++) {
    const sleefcu_batch_item &it = items[i];
    const Entry *en = find(it);
    if (!en) {
      set_error("sleefcu_eval_host: item %zu unsupported (fn %u, dtype %u, ulp %u)", i, it.fn, it.dtype, it.ulp);
      return SLEEFCU_EUNSUPPORTED;
    }
    if (it.n && (!it.x || !it.out || (en->nin == 2 && !it.y) || (en->nout == 2 && !it.out2))) {
      set_error("sleefcu_eval_host: item %zu: null pointer with n = %zu", i, (size_t)it.n);
      return SLEEFCU_EINVAL;
    }
    ens[i] = en;
  }
  return SLEEFCU_OK;
}

// the chunks of items[0..count) through one three-stream pipeline
sleefcu_status run_pipeline(const sleefcu_batch_item *items, const Entry *const *ens, size_t count, size_t chunk) {
  if (chunk == 0) chunk = (size_t)1 << 22;
  chunk = (chunk + 7) & ~(size_t)7;            // 16-byte aligned chunk starts for 2-byte elements
  size_t cbytes = 0;
  for (size_t i = 0; i < count; i++) {
    size_t m = items[i].n < chunk ? items[i].n : chunk;
    if (m * (size_t)ens[i]->esz > cbytes) cbytes = m * (size_t)ens[i]->esz;
  }
  if (cbytes == 0) return SLEEFCU_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDev) { set_error("sleefcu_eval_host: device %d unsupported", dev); return SLEEFCU_EUNSUPPORTED; }
  std::lock_guard<std::mutex> lock(g_mu[dev]);
  Stage &st = g_stage[dev];
  sleefcu_status rc = prepare(st, cbytes);
  if (rc != SLEEFCU_OK) return rc;
  size_t c = 0;                                // chunks issued so far, over all items
  for (size_t i = 0; i < count; i++) {
    const sleefcu_batch_item &it = items[i];
    const Entry *en = ens[i];
    const size_t n = it.n, esz = (size_t)en->esz;
    for (size_t off = 0; off < n; off += chunk, c++) {
      const int b = (int)(c % kDepth);
      const size_t m = (n - off < chunk) ? n - off : chunk, bytes = m * esz;
      if (c >= (size_t)kDepth && (e = cudaStreamWaitEvent(st.in, st.freed[b], 0)) != cudaSuccess)
        return cuda_fail("wait", e);
      if ((e = cudaMemcpyAsync(st.buf[b][0], (const char *)it.x + off * esz, bytes, cudaMemcpyHostToDevice,
                               st.in)) != cudaSuccess)
        return cuda_fail("copy in", e);
      if (en->nin == 2 && (e = cudaMemcpyAsync(st.buf[b][1], (const char *)it.y + off * esz, bytes,
                                               cudaMemcpyHostToDevice, st.in)) != cudaSuccess)
        return cuda_fail("copy in", e);
      if ((e = cudaEventRecord(st.loaded[b], st.in)) != cudaSuccess) return cuda_fail("record", e);
      if ((e = cudaStreamWaitEvent(st.run, st.loaded[b], 0)) != cudaSuccess) return cuda_fail("wait", e);
      rc = en->f(st.buf[b][0], st.buf[b][1], st.buf[b][2], st.buf[b][3], m, (sleefcu_stream)st.run);
      if (rc != SLEEFCU_OK) return rc;
      if ((e = cudaEventRecord(st.done[b], st.run)) != cudaSuccess) return cuda_fail("record", e);
      if ((e = cudaStreamWaitEvent(st.out, st.done[b], 0)) != cudaSuccess) return cuda_fail("wait", e);
      if ((e = cudaMemcpyAsync((char *)it.out + off * esz, st.buf[b][2], bytes, cudaMemcpyDeviceToHost,
                               st.out)) != cudaSuccess)
        return cuda_fail("copy out", e);
      if (en->nout == 2 && (e = cudaMemcpyAsync((char *)it.out2 + off * esz, st.buf[b][3], bytes,
                                                cudaMemcpyDeviceToHost, st.out)) != cudaSuccess)
        return cuda_fail("copy out", e);
      if ((e = cudaEventRecord(st.freed[b], st.out)) != cudaSuccess) return cuda_fail("record", e);
    }
  }
  if ((e = cudaStreamSynchronize(st.out)) != cudaSuccess) return cuda_fail("synchronize", e);
  return SLEEFCU_OK;
}
}  // namespace

extern "C" sleefcu_status sleefcu_eval_host(const sleefcu_batch_item *item, size_t chunk) {
  if (!item) { set_error("sleefcu_eval_host: null descriptor"); return SLEEFCU_EINVAL; }
  const Entry *en = nullptr;
  sleefcu_status rc = check_items(item, 1, &en);
  if (rc != SLEEFCU_OK) return rc;
  return run_pipeline(item, &en, 1, chunk);
}

extern "C" sleefcu_status sleefcu_eval_host_many(const sleefcu_batch_item *items, size_t count, size_t chunk) {
  if (count == 0) return SLEEFCU_OK;
  if (!items) { set_error("sleefcu_eval_host_many: null items with count = %zu", count); return SLEEFCU_EINVAL; }
  std::vector<const Entry *> ens(count);
  sleefcu_status rc = check_items(items, count, ens.data());
  if (rc != SLEEFCU_OK) return rc;
  return run_pipeline(items, ens.data(), count, chunk);
}
