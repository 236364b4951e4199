// su2_probe_fma: this device's FP32 or FP64 fused multiply-add throughput,
// measured by a probe kernel.  It is the denominator of the rooflines of the
// kernels that are bound by arithmetic rather than memory: the FP64 heat
// bath (GB300 issues FP64 at 1/64 of the FP32 rate) and the Wilson loops.
//
// The probe: every thread runs kChains independent FMA chains (enough
// independent instructions in flight to cover the pipe's latency) for
// `iters` rounds on register operands; the grid fills every SM.  The chains'
// sums are stored so the compiler keeps the work.
#include <cuda_runtime.h>

#include "su2.h"
#include "su2_capi_util.h"
#include "su2_internal.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

template <class R>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, R a, R b, R* out) {
  R x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = R(threadIdx.x + c) * R(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

template <class R>
int probe(int iters, double* flops_per_s) {
  int per_sm = 1;
  SU2_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<R>, kProbeThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const int grid = su2::device_info().sms * per_sm;
  R* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (st) cudaStreamSynchronize(st);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
  };
  SU2_CU_CLEAN(cudaMalloc(&out, (size_t)grid * kProbeThreads * sizeof(R)), cleanup());
  SU2_CU_CLEAN(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), cleanup());
  SU2_CU_CLEAN(cudaEventCreate(&e0), cleanup());
  SU2_CU_CLEAN(cudaEventCreate(&e1), cleanup());
  const R a = R(0.999999), b = R(1e-7);
  k_fma_probe<R><<<grid, kProbeThreads, 0, st>>>(iters / 8 + 1, a, b, out);  // warm-up
  SU2_CU_CLEAN(cudaEventRecord(e0, st), cleanup());
  k_fma_probe<R><<<grid, kProbeThreads, 0, st>>>(iters, a, b, out);
  SU2_CU_CLEAN(cudaEventRecord(e1, st), cleanup());
  SU2_CU_CLEAN(cudaEventSynchronize(e1), cleanup());
  SU2_CU_CLEAN(cudaGetLastError(), cleanup());
  su2::count_launches(2);
  float ms = 0.f;
  SU2_CU_CLEAN(cudaEventElapsedTime(&ms, e0, e1), cleanup());
  cleanup();
  const double fma = (double)grid * kProbeThreads * kChains * (double)iters;
  *flops_per_s = 2.0 * fma / (ms * 1e-3);
  return SU2_OK;
}

}  // namespace

extern "C" int su2_probe_fma(int prec, int iters, double* flops_per_s) {
  su2::clear_error();
  if (!flops_per_s) return su2::fail(SU2_EINVAL, "flops_per_s is NULL");
  if (iters < 1) return su2::fail(SU2_EINVAL, "iters must be >= 1");
  if (prec == SU2_F64) return probe<double>(iters, flops_per_s);
  if (prec == SU2_F32) return probe<float>(iters, flops_per_s);
  return su2::fail(SU2_EINVAL, "prec must be SU2_F64 or SU2_F32");
}
