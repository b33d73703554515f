// Shared device helpers for the hybrid factorization kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>

#include "hf_internal.h"

#define HF_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return hf_cuda_error(e_);        \
  } while (0)

int hf_cuda_error(cudaError_t e);       // maps to HF_ERR_OOM / HF_ERR_CUDA, keeps the message
const char* hf_last_cuda_message();

// flag slots in ctx->d_flags
enum { FLAG_DELAY_OVERFLOW = 0, FLAG_NUMERIC = 1, FLAG_SMEM = 2, FLAG_TC_TIMEOUT = 3, FLAG_COUNT = 8 };

inline cudaStream_t hf_stream(const hf_ctx* c) { return (cudaStream_t)c->opts.cuda_stream; }

int hf_ensure(DevBuf& b, size_t bytes);   // (re)allocate device memory to at least `bytes`
void hf_release(DevBuf& b);

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// |x| key for max-|diag| pivot search: NaN ranks below every number (never preferred)
template <typename T> __device__ __forceinline__ double piv_key(T x) {
  double a = fabs((double)x);
  return (a == a) ? a : -1.0;
}

// (key, id) maximum with ties broken toward the smaller id (reading R5)
__device__ __forceinline__ bool better(double ka, int ia, double kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}

// The same key and order in the factor's own type: |x| of an FP32 value is exact in FP32,
// so comparisons agree with the FP64 ones while staying off GB300's narrow FP64 pipe.
template <typename T> __device__ __forceinline__ T piv_key_t(T x) {
  const T a = fabs(x);
  return (a == a) ? a : T(-1);
}
template <typename T> __device__ __forceinline__ bool better_t(T ka, int ia, T kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}
