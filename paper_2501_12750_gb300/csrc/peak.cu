// peak.cu -- FP32 throughput microbenchmark (the denominator of the
// compute-bound rooflines).
//
// Every thread runs kChains independent multiply-add chains, so the FMA
// pipes never wait on a result; the grid fills every SM many times over.
// PAIRED issues the chains two at a time as FFMA2 (one instruction, two
// FMAs on the paired FP32 lanes); the scalar form issues one FFMA per FMA,
// so its rate also measures the warp-instruction issue rate (one FFMA warp
// instruction = 32 FMAs).  Timed with CUDA events on the caller's stream;
// clocks are whatever the GPU runs at (nothing here touches them).
#include "../../include/vtx.h"
#include "vtx_internal.h"

namespace vtx {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <bool PAIRED>
__global__ __launch_bounds__(256) void k_fma_rate(float *out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (PAIRED) {
#pragma unroll
        for (int j = 0; j < kChains; j += 2) {
          const float2 y = __ffma2_rn(make_float2(x[j], x[j + 1]), make_float2(a, a), make_float2(b, b));
          x[j] = y.x;
          x[j + 1] = y.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = __fmaf_rn(x[j], a, b);
      }
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == 1234.5f) out[0] = s;  // keeps the chains live; practically never stores
}

}  // namespace vtx

using namespace vtx;

extern "C" vtx_status vtx_measure_fp32_rate(int32_t paired, int32_t iters, void *cuda_stream, float *ms,
                                            double *flops) {
  if (!ms || !flops || iters < 1) return VTX_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int sms = sm_count();
  const int blocks = 8 * sms;  // 2,048 threads per SM, eight times over
  float *out = nullptr;
  if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return VTX_ERR_OOM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const float a = 1.0000001f, b = -1e-7f;
  // warm-up launch (clocks ramp, module loads)
  if (paired)
    k_fma_rate<true><<<blocks, 256, 0, st>>>(out, iters / 8 + 1, a, b);
  else
    k_fma_rate<false><<<blocks, 256, 0, st>>>(out, iters / 8 + 1, a, b);
  cudaEventRecord(e0, st);
  if (paired)
    k_fma_rate<true><<<blocks, 256, 0, st>>>(out, iters, a, b);
  else
    k_fma_rate<false><<<blocks, 256, 0, st>>>(out, iters, a, b);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return VTX_ERR_CUDA;
  *ms = t;
  *flops = 2.0 * (double)blocks * 256.0 * (double)kChains * (double)kUnroll * (double)iters;
  return VTX_OK;
}
