// Batched lattices: many independent lattices of uneven extents and couplings
// swept together by one persistent kernel per call (captured in a CUDA graph).
//
// The heat bath of each lattice follows Section 2 (Eqs. 5-9, 11) and the
// checkerboard of Section 4 exactly as for a single lattice; lattice i uses
// Philox lattice_id = i.  All lattices advance through the same substep
// sequence: every thread of the grid takes items (one link each) from the
// concatenation of all lattices' (direction, parity) class, and a grid-wide
// barrier separates the substeps.  The barrier waits are bounded in time:
// a block that gives up raises a device error flag, every block then leaves,
// and the host reports SU2_ETIMEOUT.  The grid is launched cooperatively so
// that all blocks are co-resident.
#include <cstdlib>
#include <cstring>
#include <vector>

#include "su2.h"
#include "su2_capi_util.h"
#include "su2_internal.h"

using namespace su2;

namespace su2 {

struct BatchLattice {
  Geom g;
  void* links;
  double beta;
  int64_t item_begin;  // prefix sum of V/2 over the lattices before this one
};

struct BarrierState {
  unsigned int count;
  unsigned int gen;
  int err;            // 1: a barrier wait timed out
  unsigned int extra; // arrivals the barrier waits for beyond gridDim.x (fault injection)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a time limit.  Returns false if any block timed out.
__device__ __forceinline__ bool grid_barrier(BarrierState* bs, unsigned long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &bs->gen;
    volatile int* verr = &bs->err;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bs->count, 1u) + 1u;
    if (arrived == gridDim.x + bs->extra) {
      bs->count = 0;
      __threadfence();
      atomicExch(&bs->gen, g + 1u);
    } else {
      // bounded twice over: by the global timer and by an iteration count
      const unsigned long long t0 = global_ns();
      unsigned long long spins = 0;
      while (*vgen == g) {
        if (*verr) break;
        if (global_ns() - t0 > timeout_ns || ++spins > (1ull << 24)) {
          atomicExch(&bs->err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok = *verr == 0;
  }
  __syncthreads();
  return ok != 0;
}

template <int P>
__global__ void __launch_bounds__(256) k_batch_sweep(const BatchLattice* __restrict__ desc, int nlat,
                                                     int64_t total, int nsweeps,
                                                     const uint32_t* sweep_base,
                                                     const __grid_constant__ HBParams hp,
                                                     BarrierState* bs,
                                                     unsigned long long timeout_ns) {
  using R = typename Real<P>::T;
  const uint32_t sweep0 = *sweep_base;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int sw = 0; sw < nsweeps; ++sw) {
    for (int mu = 0; mu < 4; ++mu) {
      for (int p = 0; p < 2; ++p) {
        int l = 0;
        int64_t next = nlat > 1 ? desc[1].item_begin : total;
        for (int64_t it = tid; it < total; it += T) {
          while (it >= next) {
            ++l;
            next = l + 1 < nlat ? desc[l + 1].item_begin : total;
          }
          const BatchLattice& d = desc[l];
          Links<P> L;
          L.p = reinterpret_cast<decltype(L.p)>(d.links);
          L.vh = d.g.vh;
          const int h = (int)(it - d.item_begin);
          const Site x = site_from_half(d.g, (uint32_t)h, p);
          HBParams lp = hp;
          lp.lattice_tag = (uint32_t)l << 2;
          const uint32_t sweep = sweep0 + (uint32_t)sw;
          const R beta = (R)d.beta;
          switch (mu) {
            case 0: heatbath_site<P, 0, false>(L, d.g, x, h, p, sweep, lp, beta); break;
            case 1: heatbath_site<P, 1, false>(L, d.g, x, h, p, sweep, lp, beta); break;
            case 2: heatbath_site<P, 2, false>(L, d.g, x, h, p, sweep, lp, beta); break;
            default: heatbath_site<P, 3, false>(L, d.g, x, h, p, sweep, lp, beta); break;
          }
        }
        if (!grid_barrier(bs, timeout_ns)) return;
      }
    }
  }
}

}  // namespace su2

struct su2_batch {
  int n;
  int prec;
  uint64_t seed;
  int max_tries;
  int sampler;
  uint64_t sweep;
  int device;
  std::vector<int> dims;
  std::vector<double> betas;
  std::vector<BatchLattice> desc;
  int64_t total_items;
  void* base;
  BatchLattice* d_desc;
  BarrierState* d_bar;
  uint32_t* d_sweep;
  Scratch scratch;
  double* d_results;
  double* h_results;
  cudaStream_t stream;
  bool own_stream;
  cudaStream_t cap_stream;
  cudaGraphExec_t graph;
  int graph_n;
  int grid;
  unsigned long long timeout_ns;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int P> int occupancy_blocks() {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_sweep<P>, 256, 0);
  return per_sm;
}

int batch_grid(int prec) {
  int per_sm = prec == kF64 ? occupancy_blocks<kF64>() : prec == kF32 ? occupancy_blocks<kF32>() : occupancy_blocks<kF16Q>();
  if (per_sm < 1) per_sm = 1;
  return per_sm * device_info().sms;
}

LatticeView lview(const su2_batch* b, int i) {
  LatticeView v;
  v.links = b->desc[i].links;
  v.g = b->desc[i].g;
  v.prec = b->prec;
  return v;
}

PhiloxKey batch_key(const su2_batch* b) {
  PhiloxKey k;
  k.k0 = (uint32_t)(b->seed & 0xffffffffu);
  k.k1 = (uint32_t)(b->seed >> 32);
  return k;
}

HBParams batch_hp(const su2_batch* b) {
  HBParams hp;
  hp.beta = 0.0;  // per lattice
  hp.rk = round_keys(batch_key(b));
  hp.lattice_tag = 0;
  hp.max_tries = b->max_tries;
  hp.sampler = b->sampler;
  return hp;
}

void drop_graph(su2_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_n = 0;
}

cudaError_t enqueue_batch_sweep(su2_batch* b, int n, cudaStream_t st) {
  const HBParams hp = batch_hp(b);
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const BatchLattice* d = b->d_desc;
  const int nl = b->n;
  const int64_t tot = b->total_items;
  cudaError_t e;
  switch (b->prec) {
    case kF64: e = cudaLaunchKernelEx(&cfg, k_batch_sweep<kF64>, d, nl, tot, n, (const uint32_t*)b->d_sweep, hp, b->d_bar, b->timeout_ns); break;
    case kF32: e = cudaLaunchKernelEx(&cfg, k_batch_sweep<kF32>, d, nl, tot, n, (const uint32_t*)b->d_sweep, hp, b->d_bar, b->timeout_ns); break;
    default: e = cudaLaunchKernelEx(&cfg, k_batch_sweep<kF16Q>, d, nl, tot, n, (const uint32_t*)b->d_sweep, hp, b->d_bar, b->timeout_ns); break;
  }
  if (e != cudaSuccess) return e;
  count_launches(1);
  return launch_add_u32(b->d_sweep, (uint32_t)n, st);
}

}  // namespace

extern "C" int su2_batch_init(su2_batch** out, int n, const int* dims, const double* betas,
                              uint64_t seed, int start, int prec, void* cuda_stream) {
  clear_error();
  if (!out) return fail(SU2_EINVAL, "handle pointer is NULL");
  *out = nullptr;
  if (n < 1 || n > 1023) return fail(SU2_EINVAL, "n must be in 1..1023");
  if (!dims || !betas) return fail(SU2_EINVAL, "NULL argument");
  if (start != SU2_COLD && start != SU2_HOT) return fail(SU2_EINVAL, "start must be SU2_COLD or SU2_HOT");
  if (prec < 0 || prec > 2) return fail(SU2_EINVAL, "unknown precision %d", prec);
  for (int i = 0; i < n; ++i) {
    int rc = check_dims(dims + 4 * i);
    if (rc) return rc;
    if (!(betas[i] >= 0.0) || betas[i] != betas[i] || betas[i] > 1e300) return fail(SU2_EINVAL, "beta[%d] must be finite and >= 0", i);
  }
  su2_batch* b = new (std::nothrow) su2_batch();
  if (!b) return fail(SU2_ENOMEM, "host allocation failed");
  b->n = n;
  b->prec = prec;
  b->seed = seed;
  b->max_tries = 64;
  b->sampler = SU2_SAMPLER_KP;
  b->timeout_ns = 1000000000ull;
  b->dims.assign(dims, dims + 4 * n);
  b->betas.assign(betas, betas + n);
  cudaGetDevice(&b->device);
  // layout: per-lattice stores, descriptors, barrier, sweep counter, scratch, results
  std::vector<size_t> off(n);
  size_t o = 0;
  int64_t items = 0;
  b->desc.resize(n);
  for (int i = 0; i < n; ++i) {
    b->desc[i].g = make_geom(dims + 4 * i);
    b->desc[i].beta = betas[i];
    b->desc[i].item_begin = items;
    items += b->desc[i].g.vh;
    off[i] = o;
    o = align256(o + 8 * (size_t)b->desc[i].g.vh * link_bytes(prec));
  }
  if (items >= ((int64_t)1 << 40)) { delete b; return fail(SU2_EINVAL, "batch too large"); }
  b->total_items = items;
  const size_t o_desc = o; o = align256(o + n * sizeof(BatchLattice));
  const size_t o_bar = o; o = align256(o + sizeof(BarrierState));
  const size_t o_sweep = o; o = align256(o + 64);
  const size_t o_part = o; o = align256(o + kScratchPartials * sizeof(double));
  const size_t o_cnt = o; o = align256(o + 64 * sizeof(unsigned int));
  const size_t o_out = o; o = align256(o + kScratchOut * sizeof(double));
  const size_t o_res = o; o = align256(o + 3 * (size_t)n * sizeof(double));
  cudaError_t e = cudaMalloc(&b->base, o);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(SU2_ENOMEM, "cudaMalloc(%zu) failed: %s", o, cudaGetErrorString(e));
  }
  char* base = (char*)b->base;
  for (int i = 0; i < n; ++i) b->desc[i].links = base + off[i];
  b->d_desc = (BatchLattice*)(base + o_desc);
  b->d_bar = (BarrierState*)(base + o_bar);
  b->d_sweep = (uint32_t*)(base + o_sweep);
  b->scratch.partials = (double*)(base + o_part);
  b->scratch.counter = (unsigned int*)(base + o_cnt);
  b->scratch.out = (double*)(base + o_out);
  b->d_results = (double*)(base + o_res);
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    SU2_CU_CLEAN(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), su2_batch_destroy(b));
    b->own_stream = true;
  }
  SU2_CU_CLEAN(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), su2_batch_destroy(b));
  SU2_CU_CLEAN(cudaMallocHost(&b->h_results, 3 * (size_t)n * sizeof(double)), su2_batch_destroy(b));
  SU2_CU_CLEAN(cudaMemcpyAsync(b->d_desc, b->desc.data(), n * sizeof(BatchLattice), cudaMemcpyHostToDevice, b->stream), su2_batch_destroy(b));
  BarrierState bs;
  std::memset(&bs, 0, sizeof bs);
  // Fault injection for the timeout path, host-side switch: the barrier then
  // waits for one arrival that never comes and every wait runs out.
  const char* fault = std::getenv("SU2_FAULT");
  if (fault && std::strcmp(fault, "barrier") == 0) {
    bs.extra = 1;
    b->timeout_ns = 20000000ull;
  }
  SU2_CU_CLEAN(cudaMemcpyAsync(b->d_bar, &bs, sizeof bs, cudaMemcpyHostToDevice, b->stream), su2_batch_destroy(b));
  SU2_CU_CLEAN(cudaMemsetAsync(b->d_sweep, 0, 64, b->stream), su2_batch_destroy(b));
  SU2_CU_CLEAN(cudaMemsetAsync(b->scratch.counter, 0, 64 * sizeof(unsigned int), b->stream), su2_batch_destroy(b));
  const PhiloxKey key = batch_key(b);
  for (int i = 0; i < n; ++i)
    SU2_CU_CLEAN(launch_init(lview(b, i), start, key, (uint32_t)i << 2, b->stream), su2_batch_destroy(b));
  SU2_CU_CLEAN(cudaStreamSynchronize(b->stream), su2_batch_destroy(b));
  b->grid = batch_grid(prec);
  *out = b;
  return SU2_OK;
}

extern "C" int su2_batch_destroy(su2_batch* b) {
  clear_error();
  if (!b) return SU2_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->h_results) cudaFreeHost(b->h_results);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  if (b->base) cudaFree(b->base);
  delete b;
  return SU2_OK;
}

extern "C" int su2_batch_set_options(su2_batch* b, int max_tries, int sampler) {
  clear_error();
  if (!b) return fail(SU2_EINVAL, "handle is NULL");
  if (max_tries < 1) return fail(SU2_EINVAL, "max_tries must be >= 1");
  if (sampler != SU2_SAMPLER_KP && sampler != SU2_SAMPLER_CREUTZ) return fail(SU2_EINVAL, "unknown sampler %d", sampler);
  b->max_tries = max_tries;
  b->sampler = sampler;
  drop_graph(b);
  return SU2_OK;
}

extern "C" int su2_batch_sweep(su2_batch* b, int n) {
  clear_error();
  if (!b) return fail(SU2_EINVAL, "handle is NULL");
  if (n < 0) return fail(SU2_EINVAL, "n must be >= 0");
  if (b->sweep + (uint64_t)n >= 0xFFFFFFFFull) return fail(SU2_EINVAL, "sweep counter would reach the reserved index 2^32 - 1");
  if (n == 0) return SU2_OK;
  DeviceGuard dg(b->device);
  if (!b->graph || b->graph_n != n) {
    drop_graph(b);
    cudaGraph_t graph;
    CaptureScope no_count;
    SU2_CU(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_batch_sweep(b, n, b->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (e2 == cudaSuccess) cudaGraphDestroy(graph);
      return fail(SU2_ECUDA, "batch sweep capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return fail(SU2_ECUDA, "batch sweep graph instantiation failed: %s", cudaGetErrorString(e));
    }
    b->graph_n = n;
  }
  SU2_CU(cudaGraphLaunch(b->graph, b->stream));
  count_launches(2);
  b->sweep += (uint64_t)n;
  // The barrier flag is checked on the next synchronising call; check it
  // here too so a timed-out sweep is reported by the call that ran it.
  int err = 0;
  SU2_CU(cudaMemcpyAsync(&err, &b->d_bar->err, sizeof err, cudaMemcpyDeviceToHost, b->stream));
  SU2_CU(cudaStreamSynchronize(b->stream));
  if (err) return fail(SU2_ETIMEOUT, "a grid barrier of the batched sweep timed out; lattice contents are invalid");
  return SU2_OK;
}

static int batch_measure(su2_batch* b, int which, double* out) {
  clear_error();
  if (!b || !out) return fail(SU2_EINVAL, "NULL argument");
  DeviceGuard dg(b->device);
  const int k = which == 0 ? 3 : 1;
  for (int i = 0; i < b->n; ++i) {
    if (which == 0) SU2_CU(launch_plaquette(lview(b, i), b->scratch, b->stream));
    else SU2_CU(launch_polyakov(lview(b, i), b->scratch, b->stream));
    SU2_CU(cudaMemcpyAsync(b->d_results + (size_t)k * i, b->scratch.out, k * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
  }
  SU2_CU(cudaMemcpyAsync(b->h_results, b->d_results, (size_t)k * b->n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  SU2_CU(cudaStreamSynchronize(b->stream));
  std::memcpy(out, b->h_results, (size_t)k * b->n * sizeof(double));
  return SU2_OK;
}

extern "C" int su2_batch_plaquette(su2_batch* b, double* out) { return batch_measure(b, 0, out); }
extern "C" int su2_batch_polyakov(su2_batch* b, double* out) { return batch_measure(b, 1, out); }

static int batch_links(su2_batch* b, int i, double* host, const double* in) {
  clear_error();
  if (!b || (!host && !in)) return fail(SU2_EINVAL, "NULL argument");
  if (i < 0 || i >= b->n) return fail(SU2_EINVAL, "lattice index %d out of range", i);
  DeviceGuard dg(b->device);
  const int64_t V = 2 * b->desc[i].g.vh;
  double* stage = nullptr;
  SU2_CU(cudaMallocAsync((void**)&stage, (size_t)V * 16 * sizeof(double), b->stream));
  cudaError_t e;
  if (in) {
    e = cudaMemcpyAsync(stage, in, (size_t)V * 16 * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = launch_from_canonical(lview(b, i), stage, 0, V, b->stream);
  } else {
    e = launch_to_canonical(lview(b, i), stage, 0, V, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, stage, (size_t)V * 16 * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  }
  cudaFreeAsync(stage, b->stream);
  if (e != cudaSuccess) return fail(SU2_ECUDA, "link copy failed: %s", cudaGetErrorString(e));
  SU2_CU(cudaStreamSynchronize(b->stream));
  return SU2_OK;
}

extern "C" int su2_batch_get_links(su2_batch* b, int i, double* host) { return batch_links(b, i, host, nullptr); }
extern "C" int su2_batch_set_links(su2_batch* b, int i, const double* host) { return batch_links(b, i, nullptr, host); }
