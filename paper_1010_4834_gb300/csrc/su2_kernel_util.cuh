// Launch-shape, reduction and dispatch helpers shared by the kernel
// translation units (internal; not installed).
#pragma once

#include "su2_internal.h"

namespace su2 {

constexpr int kThreads = 256;

// Blocks for `work` items with a grid-stride loop: every SM filled to the
// kernel's occupancy, never more blocks than items need.
template <class K>
static int grid_for(K kernel, int64_t work, int smem = 0, int block = kThreads) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t full = (int64_t)device_info().sms * per_sm;
  const int64_t need = (work + block - 1) / block;
  int64_t g = need < full ? need : full;
  return (int)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------------------
// Reduction helpers
// ---------------------------------------------------------------------------
template <class R> struct Acc;  // per-thread accumulator

// FP32: Neumaier-compensated, so a thread's many small terms keep FP32
// rounding from growing with the count.
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-sum NV doubles into partials[block*NV + k]; returns true in the last
// block to finish (all partials then visible to it).
template <int NV>
__device__ __forceinline__ bool block_partial(double (&v)[NV], double* partials,
                                              unsigned int* counter) {
  __shared__ double sh[kThreads / 32][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < kThreads / 32 ? sh[lane][k] : 0.0;
      t = warp_sum(t);
      if (lane == 0) partials[(size_t)blockIdx.x * NV + k] = t;
    }
    if (lane == 0) {
      __threadfence();
      const unsigned int ticket = atomicAdd(counter, 1u);
      last = (ticket == gridDim.x - 1);
    }
  }
  __syncthreads();
  return last;
}

// Sum of one double over a block of kThreads threads, all of which call it;
// the total is returned in thread 0.  Fixed-order trees over the lanes and
// then the warps.  Plain FP64 adds: the terms are thread or block sums, and
// their rounding (at most the term count times 2^-53 relative) stays far
// below every tolerance, while a compensated pair costs several times as
// many FP64 instructions, which GB300 issues at 1/64 of the FP32 rate: in
// the one block that finishes a reduction that was 20 us per measured sweep.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sw[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sw[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) t = warp_sum(lane < kThreads / 32 ? sw[lane] : 0.0);
  __syncthreads();  // sw is free for the next call
  return t;
}

// In the last block: tot[k] (thread 0) = sum over blocks of
// partials[b*NV + k].  Every thread adds a strided subset, then block_sum,
// so the result does not depend on timing.
template <int NV>
__device__ __forceinline__ void final_sum(const double* partials, int nblocks, double (&tot)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) a += __ldcg(partials + (size_t)b * NV + k);
    tot[k] = block_sum(a);
  }
}

// The plaquette after a measured sweep from the block sums of its three
// plaquette-summing substeps: meas[k * stride + b], k = 0, 1, 2 for
// mu = 1, 2, 3, b < nb[k].  Called by all kThreads threads of one block;
// fixed-order sums.  out = {all, spatial, space-time} means of Tr/2
// (Eq. 13), written by thread 0.
__device__ __forceinline__ void plaquette_from_block_sums(const double* meas, int stride, const int (&nb)[3],
                                                          double volume, double* out) {
  double tot[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nb[k]; b += kThreads) a += __ldcg(meas + (size_t)k * stride + b);
    tot[k] = block_sum(a);
  }
  if (threadIdx.x == 0) {
    const double S = tot[0] + tot[1], T = tot[2];
    const double n3 = 3.0 * volume;
    out[0] = (S + T) / (2.0 * n3);
    out[1] = S / n3;
    out[2] = T / n3;
  }
}

// Occupancy targets (blocks of 256 per SM) for the register-heavy kernels.
#ifndef SU2_HB_MINB
#define SU2_HB_MINB 4
#endif
template <int P> struct Occ { static constexpr int hb = SU2_HB_MINB; };
template <> struct Occ<kF64> { static constexpr int hb = 2; };

template <int P, int CP = kFlat> static Links<P, CP> links_of(void* base, int64_t vh) {
  Links<P, CP> L;
  L.set(base, vh);
  return L;
}

#define SU2_DISPATCH(prec, ...)                                  \
  switch (prec) {                                                \
    case kF64: { constexpr int P = kF64; __VA_ARGS__; break; }   \
    case kF32: { constexpr int P = kF32; __VA_ARGS__; break; }   \
    case kF16Q: { constexpr int P = kF16Q; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;                       \
  }

#define SU2_DISPATCH_MU(mu, ...)                          \
  switch (mu) {                                           \
    case 0: { constexpr int MU = 0; __VA_ARGS__; break; } \
    case 1: { constexpr int MU = 1; __VA_ARGS__; break; } \
    case 2: { constexpr int MU = 2; __VA_ARGS__; break; } \
    case 3: { constexpr int MU = 3; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;                \
  }

}  // namespace su2
