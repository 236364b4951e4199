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

struct KSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double v) {
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
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

// Neumaier pairs combine as (a.s + b.s with its rounding error) + a.c + b.c.
__device__ __forceinline__ KSum ksum_combine(KSum a, const KSum& b) {
  a.add(b.s);
  a.c += b.c;
  return a;
}

// Fixed-order tree over the lanes of a warp; lane 0 ends with the total.
__device__ __forceinline__ KSum warp_ksum(KSum a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    KSum o;
    o.s = __shfl_xor_sync(0xffffffffu, a.s, off);
    o.c = __shfl_xor_sync(0xffffffffu, a.c, off);
    a = ksum_combine(a, o);
  }
  return a;
}

// In the last block: tot[k] = sum over blocks of partials[b*NV + k].  Every
// thread adds a strided subset (compensated), then a fixed-order tree over
// lanes and warps combines them, so the result does not depend on timing and
// no thread runs a long serial FP64 chain.
template <int NV>
__device__ __forceinline__ void final_sum(const double* partials, int nblocks, double (&tot)[NV]) {
  __shared__ double ss[kThreads / 32][NV], sc[kThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    KSum a;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) a.add(__ldcg(partials + (size_t)b * NV + k));
    a = warp_ksum(a);
    if (lane == 0) {
      ss[warp][k] = a.s;
      sc[warp][k] = a.c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      KSum a;
      for (int w = 0; w < kThreads / 32; ++w) {
        KSum o;
        o.s = ss[w][k];
        o.c = sc[w][k];
        a = ksum_combine(a, o);
      }
      tot[k] = a.value();
    }
  }
}

// The plaquette after a measured sweep from the block sums of its three
// plaquette-summing substeps: meas[k * stride + b], k = 0, 1, 2 for
// mu = 1, 2, 3, b < nb[k].  Called by all kThreads threads of one block;
// fixed-order compensated sums.  out = {all, spatial, space-time} means of
// Tr/2 (Eq. 13).
__device__ __forceinline__ void plaquette_from_block_sums(const double* meas, int stride, const int (&nb)[3],
                                                          double volume, double* out) {
  __shared__ double ss[kThreads / 32][3], sc[kThreads / 32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    KSum a;
    for (int b = threadIdx.x; b < nb[k]; b += kThreads) a.add(__ldcg(meas + (size_t)k * stride + b));
    a = warp_ksum(a);
    if (lane == 0) {
      ss[warp][k] = a.s;
      sc[warp][k] = a.c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      KSum a;
      for (int w = 0; w < kThreads / 32; ++w) {
        KSum o;
        o.s = ss[w][k];
        o.c = sc[w][k];
        a = ksum_combine(a, o);
      }
      tot[k] = a.value();
    }
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

template <int P, bool CP = false> static Links<P, CP> links_of(void* base, int64_t vh) {
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
