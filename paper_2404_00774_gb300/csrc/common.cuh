// Shared helpers of the SOAR CUDA library (device side and host glue).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <atomic>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/soar.h"

namespace soar {

extern std::atomic<uint64_t> g_launches;

// Optional CUDA-event timing of named stages on the launching stream
// (enabled by soar_stage_timing; off by default, then a no-op).
void stage_mark(cudaStream_t s, const char* stage, bool begin);

// ---------------------------------------------------------------- errors

struct Error : std::runtime_error {
  soar_status status;
  Error(soar_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] inline void fail(soar_status s, const std::string& msg) { throw Error(s, msg); }

#define SOAR_REQUIRE(cond, msg)                                        \
  do {                                                                 \
    if (!(cond)) ::soar::fail(SOAR_EINVAL, std::string(__func__) + ": " + (msg)); \
  } while (0)

#define SOAR_CUDA(call)                                                             \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      ::soar::fail(e_ == cudaErrorMemoryAllocation ? SOAR_ENOMEM : SOAR_ECUDA,      \
                   std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

// Every kernel launch site of the library is followed by SOAR_LAUNCHED(),
// which checks the launch and counts it (soar_kernel_launches()).
#define SOAR_LAUNCHED()                                        \
  do {                                                         \
    SOAR_CUDA(cudaGetLastError());                             \
    ::soar::g_launches.fetch_add(1, std::memory_order_relaxed); \
  } while (0)

// ------------------------------------------------------ stream-ordered scratch

// Device scratch taken from the stream-ordered pool and returned on `stream`
// when the owner goes out of scope (after the work queued before it).
class Scratch {
 public:
  explicit Scratch(cudaStream_t s) : stream_(s) {}
  ~Scratch() {
    for (void* p : ptrs_) cudaFreeAsync(p, stream_);
  }
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    SOAR_CUDA(cudaMallocAsync(&p, bytes, stream_));
    ptrs_.push_back(p);
    return static_cast<T*>(p);
  }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;

 private:
  cudaStream_t stream_;
  std::vector<void*> ptrs_;
};

inline int num_sms() {
  static int sms = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------ device helpers

__device__ __forceinline__ float load_elem(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float load_elem(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

// Order-preserving map of an fp32 value to uint32 (larger float -> larger key).
__device__ __forceinline__ uint32_t float_key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// Composite ordering key for "score descending, id ascending": smaller key = better.
__device__ __forceinline__ uint64_t rank_key(float score, uint32_t id) {
  return ((uint64_t)(~float_key(score)) << 32) | (uint64_t)id;
}

// Exclusive scan of one value per thread across the block (all threads of
// the block call it; blockDim.x a multiple of 32); `total` gets the sum.
template <typename T>
__device__ T block_exclusive_scan(T v, T* smem_warp /*[32]*/, T& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < nw ? smem_warp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    smem_warp[lane] = s;  // inclusive scan of warp totals
  }
  __syncthreads();
  T warp_base = w > 0 ? smem_warp[w - 1] : T(0);
  total = smem_warp[nw - 1];
  __syncthreads();
  return warp_base + x - v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace soar
