// su2_plaquette_static: the mean plaquette of a caller-owned link store,
// computed without allocating any device memory.
//
// Who needs it: code whose device memory is handed out by someone else -- a
// framework's caching allocator that must account for every byte, a service
// running under a fixed device-memory budget, or a loop where cudaMalloc's
// implicit device synchronisation is not acceptable.  Such callers can keep
// the link store in memory they own (su2_init_external puts it at the start
// of their buffer) but cannot give the library reduction scratch.  This entry
// point takes the store directly and keeps its scratch -- one partial sum per
// block, a ticket counter and the three results -- in a fixed array in the
// library's own device memory.
//
// The array is shared by every call on a device and keeps the last call's
// contents: the counter is cleared before each launch, the partials are
// overwritten.  Two calls whose work overlaps on the GPU (different streams,
// or different threads) race on it; serialise them.  The array's device
// address is looked up once per device on the first call, with that device
// current; make that first call before any stream capture.
#include <mutex>

#include "su2.h"
#include "su2_capi_util.h"
#include "su2_internal.h"

namespace {

constexpr int kStaticThreads = 256;
// Largest grid the fixed scratch serves: 4096 blocks (two partial sums each).
constexpr int kStaticMaxBlocks = 4096;
// doubles: [0, 2 * kStaticMaxBlocks) partials, then 3 results, then the counter
constexpr int kStaticResult = 2 * kStaticMaxBlocks;
constexpr int kStaticCounter = kStaticResult + 4;
constexpr int kStaticDoubles = kStaticCounter + 4;

}  // namespace

// 64 KiB + 64 B of reduction scratch, resident on every device that loads the
// library until the process exits.
static __device__ __align__(256) double su2_static_scratch[kStaticDoubles];

namespace {

using namespace su2;

template <class R> struct SAcc;
template <> struct SAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <> struct SAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

struct SSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double v) {
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
};

__device__ __forceinline__ double sum_warp(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int P>
__device__ __forceinline__ typename Real<P>::T plaq_pair(const Links<P>& L, int q, const Quat<typename Real<P>::T>& umu,
                                                        const Quat<typename Real<P>::T>& unu, int mu, int nu,
                                                        int h_pmu, int h_pnu) {
  using R = typename Real<P>::T;
  const Quat<R> a = qmul(umu, L.ld(2 * nu + q, h_pmu));
  const Quat<R> b = qmul(unu, L.ld(2 * mu + q, h_pnu));
  return qdot(a, b);
}

// Same arithmetic as the handle-based plaquette (Section 2, Eqs. 12-13):
// per site the six (1/2) Re Tr of the plaquettes, split into spatial and
// space-time sums; per-block partials and the final fixed-order sum go to
// `scratch`, which is the fixed array above.
template <int P>
__global__ void __launch_bounds__(kStaticThreads) k_plaquette_static(Links<P> L, Geom g, double* scratch) {
  using R = typename Real<P>::T;
  __shared__ double sh[kStaticThreads / 32][2];
  __shared__ double fin[kStaticThreads][4];
  __shared__ bool last;
  SAcc<R> sp, tm;
  const int64_t V = 2 * g.vh;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < V; s += (int64_t)gridDim.x * blockDim.x) {
    const Site x = site_from_index(g, (uint32_t)s);
    const int p = parity(x), q = p ^ 1;
    const int h = (int)(s >> 1);
    const Quat<R> u0 = L.ld(0 + p, h), u1 = L.ld(2 + p, h), u2 = L.ld(4 + p, h), u3 = L.ld(6 + p, h);
    const int h0 = hidx(g, shifted<0, +1>(g, x));
    const int h1 = hidx(g, shifted<1, +1>(g, x));
    const int h2 = hidx(g, shifted<2, +1>(g, x));
    const int h3 = hidx(g, shifted<3, +1>(g, x));
    sp.add(plaq_pair<P>(L, q, u0, u1, 0, 1, h0, h1) + plaq_pair<P>(L, q, u0, u2, 0, 2, h0, h2) +
           plaq_pair<P>(L, q, u1, u2, 1, 2, h1, h2));
    tm.add(plaq_pair<P>(L, q, u0, u3, 0, 3, h0, h3) + plaq_pair<P>(L, q, u1, u3, 1, 3, h1, h3) +
           plaq_pair<P>(L, q, u2, u3, 2, 3, h2, h3));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double vs = sum_warp(sp.value()), vt = sum_warp(tm.value());
  if (lane == 0) { sh[warp][0] = vs; sh[warp][1] = vt; }
  __syncthreads();
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kStaticCounter);
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kStaticThreads / 32; ++w) { a += sh[w][0]; b += sh[w][1]; }
    scratch[2 * blockIdx.x] = a;
    scratch[2 * blockIdx.x + 1] = b;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  SSum a, b;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    a.add(__ldcg(scratch + 2 * k));
    b.add(__ldcg(scratch + 2 * k + 1));
  }
  fin[threadIdx.x][0] = a.s; fin[threadIdx.x][1] = a.c;
  fin[threadIdx.x][2] = b.s; fin[threadIdx.x][3] = b.c;
  __syncthreads();
  if (threadIdx.x == 0) {
    SSum ta, tb;
    double ca = 0.0, cb = 0.0;
    for (int t = 0; t < kStaticThreads; ++t) {
      ta.add(fin[t][0]); ca += fin[t][1];
      tb.add(fin[t][2]); cb += fin[t][3];
    }
    const double S = ta.s + ta.c + ca, T = tb.s + tb.c + cb;
    const double n3 = 3.0 * (double)V;
    scratch[kStaticResult + 0] = (S + T) / (2.0 * n3);
    scratch[kStaticResult + 1] = S / n3;
    scratch[kStaticResult + 2] = T / n3;
    *counter = 0;
  }
}

template <int P>
cudaError_t launch_static(const void* links, const Geom& g, double* scratch, int max_blocks, cudaStream_t st,
                          int* blocks_needed) {
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plaquette_static<P>, kStaticThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (2 * g.vh + kStaticThreads - 1) / kStaticThreads;
  const int64_t full = (int64_t)device_info().sms * per_sm;
  const int grid = (int)(need < full ? need : full);
  *blocks_needed = grid;
  if (grid > max_blocks) return cudaSuccess;
  Links<P> L;
  L.set(const_cast<void*>(links), g.vh);
  k_plaquette_static<P><<<grid, kStaticThreads, 0, st>>>(L, g, scratch);
  return cudaGetLastError();
}

std::mutex g_static_mu;
double* g_static_ptr[64] = {nullptr};

}  // namespace

extern "C" int su2_plaquette_static(const void* links, const int dims[4], int prec, double out[3],
                                    void* cuda_stream) {
  clear_error();
  if (!links || !out) return fail(SU2_EINVAL, "links and out must not be NULL");
  int rc = check_dims(dims);
  if (rc) return rc;
  if (prec != SU2_F64 && prec != SU2_F32 && prec != SU2_F16Q) return fail(SU2_EINVAL, "unknown precision %d", prec);
  int dev = 0;
  SU2_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SU2_EINVAL, "device ordinal %d out of range", dev);
  double* scratch = nullptr;
  {
    // once per device, with that device current: the host-side name of the
    // array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, su2_static_scratch);
      if (e != cudaSuccess) return fail(SU2_ECUDA, "cudaGetSymbolAddress(su2_static_scratch) failed: %s", cudaGetErrorString(e));
      g_static_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_static_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const Geom g = make_geom(dims);
  // the ticket counter must start at zero (an earlier call that stopped
  // early could have left it otherwise)
  SU2_CU(cudaMemsetAsync(scratch + kStaticCounter, 0, sizeof(unsigned int), st));
  int blocks = 0;
  cudaError_t e;
  switch (prec) {
    case SU2_F64: e = launch_static<kF64>(links, g, scratch, kStaticMaxBlocks, st, &blocks); break;
    case SU2_F32: e = launch_static<kF32>(links, g, scratch, kStaticMaxBlocks, st, &blocks); break;
    default: e = launch_static<kF16Q>(links, g, scratch, kStaticMaxBlocks, st, &blocks); break;
  }
  if (e != cudaSuccess) return fail(SU2_ECUDA, "plaquette launch failed: %s", cudaGetErrorString(e));
  if (blocks > kStaticMaxBlocks)
    return fail(SU2_EINVAL, "this device needs %d reduction blocks; the fixed scratch holds %d", blocks,
                kStaticMaxBlocks);
  count_launches(1);
  double res[3];
  SU2_CU(cudaMemcpyAsync(res, scratch + kStaticResult, sizeof res, cudaMemcpyDeviceToHost, st));
  SU2_CU(cudaStreamSynchronize(st));
  out[0] = res[0];
  out[1] = res[1];
  out[2] = res[2];
  return SU2_OK;
}
