// Shared host/device helpers for the ISDF-xTC CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../../include/isdftc.h"

namespace isdf {

// ---------------------------------------------------------------- host errors

void set_error(const char* fmt, ...);

#define ISDF_CUDA(call)                                                        \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      ::isdf::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,             \
                        cudaGetErrorString(e_));                               \
      return ISDF_E_CUDA;                                                      \
    }                                                                          \
  } while (0)

inline int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return ISDF_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return ISDF_E_CUDA;
}

#define ISDF_ARG(cond, ...)                                                    \
  do {                                                                         \
    if (!(cond)) {                                                             \
      ::isdf::set_error(__VA_ARGS__);                                          \
      return ISDF_E_ARG;                                                       \
    }                                                                          \
  } while (0)

#define ISDF_TRY(expr)                                                         \
  do {                                                                         \
    int s_ = (expr);                                                           \
    if (s_ != ISDF_OK) return s_;                                              \
  } while (0)

void count_launch();
#define ISDF_LAUNCH_CHECK()          \
  do {                               \
    ::isdf::count_launch();          \
    ISDF_CUDA(cudaGetLastError());   \
  } while (0)

// ---------------------------------------------------------------- workspace

// Bump allocator over a caller-provided workspace; 256-byte aligned slices.
struct Carve {
  char* base;
  size_t cap;
  size_t off = 0;
  bool dry;  // size query only
  Carve(void* p, size_t n) : base((char*)p), cap(n), dry(p == nullptr) {}
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* out = dry ? nullptr : (T*)(base + off);
    off += bytes;
    return out;
  }
  bool ok() const { return dry || off <= cap; }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// ---------------------------------------------------------------- device errors

// Device error word bits (OR-ed together).
enum DevErr : int {
  DEV_ERR_TIMEOUT = 1,
  DEV_ERR_NOT_PD = 2,
  DEV_ERR_NONFINITE = 4,
  DEV_ERR_ARG = 8,
};

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Default limit of every device-side spin in this library (nanoseconds), and
// the range a caller may set through isdf_options.wait_limit_ms.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr int kWaitLimitMaxMs = 60000;

// Limit the kernels launched by the calling host thread use: the default,
// or the caller's option for the duration of one call (WaitLimitScope).
inline uint64_t& wait_limit_ns() {
  static thread_local uint64_t v = kWaitLimitNs;
  return v;
}

struct WaitLimitScope {
  uint64_t saved;
  explicit WaitLimitScope(int ms) : saved(wait_limit_ns()) {
    if (ms > 0) wait_limit_ns() = (uint64_t)(ms < kWaitLimitMaxMs ? ms : kWaitLimitMaxMs) * 1000000ull;
  }
  ~WaitLimitScope() { wait_limit_ns() = saved; }
};

}  // namespace isdf
