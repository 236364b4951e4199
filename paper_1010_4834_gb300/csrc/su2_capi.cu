// C ABI of libsu2 (declared in include/su2.h): handle life cycle, device
// memory carving, CUDA-graph replay of heat-bath sweeps, measurements and
// checkpoint I/O for single lattices.  Batched lattices are in su2_batch.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "su2.h"
#include "su2_internal.h"
#include "su2_capi_util.h"

using namespace su2;

// ---------------------------------------------------------------------------
// Thread-local last error
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

namespace su2 {
int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}
void clear_error() { g_err[0] = 0; }
}  // namespace su2

extern "C" const char* su2_last_error(void) { return g_err; }
extern "C" const char* su2_version(void) { return "su2-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct su2_lattice {
  int dims[4];
  int prec;
  double beta;
  uint64_t seed;
  int max_tries;
  int sampler;
  uint64_t sweep;
  Geom g;
  int device;
  // device memory
  void* base;
  size_t bytes;
  bool own_mem;
  void* links;
  void* ape[2];
  Scratch scratch;
  uint32_t* d_sweep;
  unsigned long long* d_stats;
  double* d_hist;
  double* staging;
  int64_t staging_sites;
  double* h_out;  // pinned host results
  // streams and the cached sweep graph
  cudaStream_t stream;
  bool own_stream;
  cudaStream_t cap_stream;
  cudaGraphExec_t graph;   // kGraphSweeps plain sweeps
  cudaGraphExec_t mgraph;  // kGraphSweeps measured sweeps
  int graph_sweeps;
  int meas_nb[3];          // blocks of the three plaquette-summing substeps
  int smeared;  // 0 none, 1 in ape[0], 2 in ape[1]
  // sweep schedule and the fused pair's control block
  int schedule;            // SU2_SCHED_*
  int or_per_sweep;        // over-relaxation sweeps before each heat-bath sweep
  PairCtl* d_pair;
  unsigned int* d_done0;   // one count per time slice
  bool pair_used;          // a pair launch ran since the last error check
};

namespace {

constexpr int kGraphSweeps = 8;
constexpr int64_t kStagingSites = (int64_t)1 << 18;

struct Layout {
  size_t links, ape0, ape1, partials, counter, out, state, hist, pair, staging, total;
};


size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout_for(const int dims[4], int prec) {
  const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  const size_t lb = (size_t)link_bytes(prec);
  Layout L;
  size_t o = 0;
  L.links = o; o = align256(o + 4 * (size_t)V * lb);
  L.ape0 = o; o = align256(o + 3 * (size_t)V * lb);
  L.ape1 = o; o = align256(o + 3 * (size_t)V * lb);
  L.partials = o; o = align256(o + kScratchPartials * sizeof(double));
  L.counter = o; o = align256(o + 64 * sizeof(unsigned int));
  L.out = o; o = align256(o + kScratchOut * sizeof(double));
  L.state = o; o = align256(o + 256);
  L.hist = o; o = align256(o + (size_t)kHistRing * 4 * sizeof(double));
  L.pair = o; o = align256(o + sizeof(PairCtl) + (size_t)dims[3] * sizeof(unsigned int));
  const int64_t st = V < kStagingSites ? V : kStagingSites;
  L.staging = o; o = align256(o + (size_t)st * 16 * sizeof(double));
  L.total = o;
  return L;
}

}  // namespace

namespace su2 {
int check_dims(const int dims[4]) {
  if (!dims) return fail(SU2_EINVAL, "dims is NULL");
  int64_t V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2 || (dims[i] & 1))
      return fail(SU2_EINVAL, "extent %d = %d: every extent must be even and >= 2", i, dims[i]);
    V *= dims[i];
    if (V > ((int64_t)1 << 31) - 1) return fail(SU2_EINVAL, "lattice volume exceeds 2^31 - 1 sites");
  }
  return SU2_OK;
}
}  // namespace su2

static int check_common(double beta, int start, int prec) {
  if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(SU2_EINVAL, "beta must be finite and >= 0");
  if (start != SU2_COLD && start != SU2_HOT) return fail(SU2_EINVAL, "start must be SU2_COLD or SU2_HOT");
  if (prec != SU2_F64 && prec != SU2_F32 && prec != SU2_F16Q) return fail(SU2_EINVAL, "unknown precision %d", prec);
  return SU2_OK;
}

static LatticeView view(const su2_lattice* h) {
  LatticeView v;
  v.links = h->links;
  v.g = h->g;
  v.prec = h->prec;
  return v;
}

static PhiloxKey philox_key(uint64_t seed) {
  PhiloxKey k;
  k.k0 = (uint32_t)(seed & 0xffffffffu);
  k.k1 = (uint32_t)(seed >> 32);
  return k;
}

static HBParams hb_params(const su2_lattice* h) {
  HBParams hp;
  hp.beta = h->beta;
  hp.rk = round_keys(philox_key(h->seed));
  hp.lattice_tag = 0;
  hp.max_tries = h->max_tries;
  hp.sampler = h->sampler;
  return hp;
}

static void drop_graph(su2_lattice* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->mgraph) cudaGraphExecDestroy(h->mgraph);
  h->graph = nullptr;
  h->mgraph = nullptr;
  h->graph_sweeps = 0;
}

static int init_common(su2_lattice** out, const int dims[4], double beta, uint64_t seed, int start,
                       int prec, void* dev_buf, size_t bytes, void* stream) {
  clear_error();
  if (!out) return fail(SU2_EINVAL, "handle pointer is NULL");
  *out = nullptr;
  int rc = check_dims(dims);
  if (rc) return rc;
  if ((rc = check_common(beta, start, prec))) return rc;
  const Layout L = layout_for(dims, prec);
  su2_lattice* h = new (std::nothrow) su2_lattice();
  if (!h) return fail(SU2_ENOMEM, "host allocation failed");
  std::memcpy(h->dims, dims, sizeof h->dims);
  h->prec = prec;
  h->beta = beta;
  h->seed = seed;
  h->max_tries = 64;
  h->sampler = SU2_SAMPLER_KP;
  h->sweep = 0;
  h->g = make_geom(dims);
  cudaGetDevice(&h->device);
  if (dev_buf) {
    if (bytes < L.total) {
      delete h;
      return fail(SU2_ENOMEM, "external buffer has %zu bytes, %zu needed", bytes, L.total);
    }
    if (((uintptr_t)dev_buf & 255) != 0) {
      delete h;
      return fail(SU2_EINVAL, "external buffer must be 256-byte aligned");
    }
    h->base = dev_buf;
    h->own_mem = false;
  } else {
    cudaError_t e = cudaMalloc(&h->base, L.total);
    if (e != cudaSuccess) {
      delete h;
      cudaGetLastError();
      return fail(SU2_ENOMEM, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
    }
    h->own_mem = true;
  }
  h->bytes = L.total;
  char* b = (char*)h->base;
  h->links = b + L.links;
  h->ape[0] = b + L.ape0;
  h->ape[1] = b + L.ape1;
  h->scratch.partials = (double*)(b + L.partials);
  h->scratch.counter = (unsigned int*)(b + L.counter);
  h->scratch.out = (double*)(b + L.out);
  h->d_sweep = (uint32_t*)(b + L.state);
  h->d_stats = (unsigned long long*)(b + L.state + 64);
  h->d_hist = (double*)(b + L.hist);
  h->d_pair = (PairCtl*)(b + L.pair);
  h->d_done0 = (unsigned int*)(b + L.pair + sizeof(PairCtl));
  h->schedule = SU2_SCHED_AUTO;
  h->or_per_sweep = 0;
  h->staging = (double*)(b + L.staging);
  const int64_t V = 2 * h->g.vh;
  h->staging_sites = V < kStagingSites ? V : kStagingSites;
  if (stream) {
    h->stream = (cudaStream_t)stream;
    h->own_stream = false;
  } else {
    SU2_CU_CLEAN(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), su2_destroy(h));
    h->own_stream = true;
  }
  SU2_CU_CLEAN(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), su2_destroy(h));
  SU2_CU_CLEAN(cudaMallocHost(&h->h_out, kScratchOut * sizeof(double)), su2_destroy(h));
  SU2_CU_CLEAN(cudaMemsetAsync(b + L.counter, 0, L.out - L.counter, h->stream), su2_destroy(h));
  SU2_CU_CLEAN(cudaMemsetAsync(b + L.state, 0, 256, h->stream), su2_destroy(h));
  SU2_CU_CLEAN(cudaMemsetAsync(b + L.pair, 0, L.staging - L.pair, h->stream), su2_destroy(h));
  SU2_CU_CLEAN(launch_init(view(h), start, philox_key(h->seed), 0u, h->stream), su2_destroy(h));
  *out = h;
  return SU2_OK;
}

extern "C" int su2_required_bytes(const int dims[4], int prec, size_t* bytes) {
  clear_error();
  int rc = check_dims(dims);
  if (rc) return rc;
  if (prec < 0 || prec > 2) return fail(SU2_EINVAL, "unknown precision %d", prec);
  if (!bytes) return fail(SU2_EINVAL, "bytes is NULL");
  *bytes = layout_for(dims, prec).total;
  return SU2_OK;
}

extern "C" int su2_init(su2_lattice** h, const int dims[4], double beta, uint64_t seed, int start,
                        int prec, void* cuda_stream) {
  return init_common(h, dims, beta, seed, start, prec, nullptr, 0, cuda_stream);
}

extern "C" int su2_init_external(su2_lattice** h, const int dims[4], double beta, uint64_t seed,
                                 int start, int prec, void* dev_buf, size_t bytes,
                                 void* cuda_stream) {
  if (!dev_buf) return fail(SU2_EINVAL, "dev_buf is NULL");
  return init_common(h, dims, beta, seed, start, prec, dev_buf, bytes, cuda_stream);
}

extern "C" int su2_destroy(su2_lattice* h) {
  clear_error();
  if (!h) return SU2_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  if (h->h_out) cudaFreeHost(h->h_out);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->own_mem && h->base) cudaFree(h->base);
  delete h;
  return SU2_OK;
}

extern "C" int su2_set_stream(su2_lattice* h, void* cuda_stream) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  SU2_CU(cudaStreamSynchronize(h->stream));
  if (h->own_stream) cudaStreamDestroy(h->stream);
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
    h->own_stream = false;
  } else {
    SU2_CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  return SU2_OK;
}

extern "C" int su2_set_options(su2_lattice* h, int max_tries, int sampler) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (max_tries < 1) return fail(SU2_EINVAL, "max_tries must be >= 1");
  if (sampler != SU2_SAMPLER_KP && sampler != SU2_SAMPLER_CREUTZ) return fail(SU2_EINVAL, "unknown sampler %d", sampler);
  h->max_tries = max_tries;
  h->sampler = sampler;
  drop_graph(h);
  return SU2_OK;
}

extern "C" int su2_set_beta(su2_lattice* h, double beta) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(SU2_EINVAL, "beta must be finite and >= 0");
  h->beta = beta;
  drop_graph(h);
  return SU2_OK;
}

extern "C" int su2_set_schedule(su2_lattice* h, int schedule) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (schedule != SU2_SCHED_AUTO && schedule != SU2_SCHED_SUBSTEP && schedule != SU2_SCHED_PAIR)
    return fail(SU2_EINVAL, "unknown schedule %d", schedule);
  if (schedule == SU2_SCHED_PAIR && h->prec == SU2_F64)
    return fail(SU2_EINVAL, "the fused pair schedule runs FP32 and F16Q lattices only");
  h->schedule = schedule;
  drop_graph(h);
  return SU2_OK;
}

extern "C" int su2_set_overrelax(su2_lattice* h, int n) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (n < 0 || n > 16) return fail(SU2_EINVAL, "over-relaxation sweeps per heat-bath sweep must be in 0..16");
  h->or_per_sweep = n;
  drop_graph(h);
  return SU2_OK;
}

// Whether heat-bath sweeps run as four fused parity pairs (su2_pair.cu)
// rather than eight substeps.
// SU2_SCHED_AUTO is the substep schedule: measured on GB300 the fused pair
// is slower at every size (64^4 FP32: 495-540 us per pair against 375 us for
// its two substeps), since the substep kernel is bound by latency and issue,
// not by the HBM traffic the pair saves.
static bool use_pair(const su2_lattice* h) {
  return h->prec != SU2_F64 && h->schedule == SU2_SCHED_PAIR;
}

// Kernels one (plain or measured) sweep enqueues.
static int kernels_per_sweep(const su2_lattice* h, bool measured) {
  return 8 * h->or_per_sweep + (use_pair(h) ? 4 : 8) + (measured ? 1 : 0);
}

// The over-relaxation sweeps that precede each heat-bath sweep (Section 2,
// Eq. 10; same direction and parity order).
static cudaError_t enqueue_overrelax(su2_lattice* h, cudaStream_t st) {
  const LatticeView v = view(h);
  for (int k = 0; k < h->or_per_sweep; ++k)
    for (int mu = 0; mu < 4; ++mu)
      for (int p = 0; p < 2; ++p) {
        cudaError_t e = launch_overrelax(v, mu, p, st);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

// One sweep's eight substeps (or four fused pairs), after the handle's
// over-relaxation sweeps; sweep index = *d_sweep + off.
static cudaError_t enqueue_sweep(su2_lattice* h, uint32_t off, cudaStream_t st) {
  const LatticeView v = view(h);
  const HBParams hp = hb_params(h);
  cudaError_t e = enqueue_overrelax(h, st);
  if (e != cudaSuccess) return e;
  if (use_pair(h)) {
    h->pair_used = true;
    for (int mu = 0; mu < 4; ++mu) {
      e = launch_heatbath_pair(v, mu, h->d_sweep, off, hp, h->d_pair, h->d_done0, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (int mu = 0; mu < 4; ++mu)
    for (int p = 0; p < 2; ++p) {
      e = launch_heatbath(v, mu, p, h->d_sweep, off, hp, nullptr, st);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

// One measured sweep: the over-relaxation sweeps, the eight substeps (or
// four pairs), the odd-parity ones of mu = 1, 2, 3 also summing the
// plaquettes their links close (see k_heatbath), then the Polyakov kernel,
// whose last block turns those block sums into the plaquette, records both
// in row (*d_sweep mod kHistRing) of d_hist and advances *d_sweep.  No host
// state changes, so it replays in a graph.  Over-relaxation keeps the total
// action but not its spatial / space-time split, so it runs before the
// heat bath, whose own staples give the plaquette of the final links.
static cudaError_t enqueue_measured_sweep(su2_lattice* h, cudaStream_t st) {
  const LatticeView v = view(h);
  const HBParams hp = hb_params(h);
  cudaError_t e = enqueue_overrelax(h, st);
  if (e != cudaSuccess) return e;
  const bool pair = use_pair(h);
  if (pair) h->pair_used = true;
  for (int mu = 0; mu < 4; ++mu) {
    double* meas = mu >= 1 ? h->scratch.partials + (size_t)(mu - 1) * kMeasStride : nullptr;
    int* nb = meas ? &h->meas_nb[mu - 1] : nullptr;
    if (pair) {
      e = launch_heatbath_pair(v, mu, h->d_sweep, 0u, hp, h->d_pair, h->d_done0, st, meas, nb);
      if (e != cudaSuccess) return e;
      continue;
    }
    for (int p = 0; p < 2; ++p) {
      e = launch_heatbath(v, mu, p, h->d_sweep, 0u, hp, nullptr, st, p == 1 ? meas : nullptr,
                          p == 1 ? nb : nullptr);
      if (e != cudaSuccess) return e;
    }
  }
  SweepEpilogue ep{h->scratch.partials, {h->meas_nb[0], h->meas_nb[1], h->meas_nb[2]}, (double)(2 * v.g.vh),
                   h->d_hist, h->d_sweep};
  Scratch sp = h->scratch;
  sp.partials = h->scratch.partials + 3 * (size_t)kMeasStride;  // clear of the block sums
  return launch_polyakov(v, sp, st, &ep);
}

// SU2_ETIMEOUT if a fused-pair dependency wait gave up since the last check
// (the stream must be synchronised); the control block is then cleared.
static int check_pair(su2_lattice* h) {
  if (!h->pair_used && !use_pair(h)) return SU2_OK;
  unsigned int err = 0;
  SU2_CU(cudaMemcpyAsync(&err, &h->d_pair->err, sizeof err, cudaMemcpyDeviceToHost, h->stream));
  SU2_CU(cudaStreamSynchronize(h->stream));
  h->pair_used = false;
  if (!err) return SU2_OK;
  SU2_CU(cudaMemsetAsync(h->d_pair, 0, sizeof(PairCtl) + (size_t)h->dims[3] * sizeof(unsigned int), h->stream));
  SU2_CU(cudaStreamSynchronize(h->stream));
  return fail(SU2_ETIMEOUT, "a dependency wait of the fused heat-bath sweep timed out; the links are undefined");
}

// Capture kGraphSweeps plain (measured = false) or measured sweeps.
static int build_graph(su2_lattice* h, bool measured) {
  cudaGraphExec_t& exec = measured ? h->mgraph : h->graph;
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  cudaGraph_t graph;
  CaptureScope no_count;
  SU2_CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kGraphSweeps && e == cudaSuccess; ++i)
    e = measured ? enqueue_measured_sweep(h, h->cap_stream) : enqueue_sweep(h, (uint32_t)i, h->cap_stream);
  if (e == cudaSuccess && !measured) e = launch_add_u32(h->d_sweep, kGraphSweeps, h->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (e2 == cudaSuccess) cudaGraphDestroy(graph);
    return fail(SU2_ECUDA, "sweep graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    exec = nullptr;
    return fail(SU2_ECUDA, "sweep graph instantiation failed: %s", cudaGetErrorString(e));
  }
  h->graph_sweeps = kGraphSweeps;
  return SU2_OK;
}

extern "C" int su2_heatbath_sweep(su2_lattice* h, int n) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (n < 0) return fail(SU2_EINVAL, "n must be >= 0");
  if (h->sweep + (uint64_t)n >= 0xFFFFFFFFull) return fail(SU2_EINVAL, "sweep counter would reach the reserved index 2^32 - 1");
  DeviceGuard dg(h->device);
  if (n == 0) return SU2_OK;
  int left = n;
  if (left >= kGraphSweeps) {
    if (!h->graph) {
      int rc = build_graph(h, false);
      if (rc) return rc;
    }
    while (left >= kGraphSweeps) {
      SU2_CU(cudaGraphLaunch(h->graph, h->stream));
      count_launches(kernels_per_sweep(h, false) * kGraphSweeps + 1);
      left -= kGraphSweeps;
    }
  }
  for (int i = 0; i < left; ++i) SU2_CU(enqueue_sweep(h, (uint32_t)i, h->stream));
  if (left) SU2_CU(launch_add_u32(h->d_sweep, (uint32_t)left, h->stream));
  h->sweep += (uint64_t)n;
  h->smeared = 0;
  return SU2_OK;
}

extern "C" int su2_restart(su2_lattice* h, int start) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (start != SU2_COLD && start != SU2_HOT) return fail(SU2_EINVAL, "start must be SU2_COLD or SU2_HOT");
  DeviceGuard dg(h->device);
  SU2_CU(launch_init(view(h), start, philox_key(h->seed), 0u, h->stream));
  SU2_CU(cudaMemsetAsync(h->d_sweep, 0, sizeof(uint32_t), h->stream));
  h->sweep = 0;
  h->smeared = 0;
  return SU2_OK;
}

extern "C" int su2_sweep_measure(su2_lattice* h, int n, double* hist) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (n < 0) return fail(SU2_EINVAL, "n must be >= 0");
  if (n > 0 && !hist) return fail(SU2_EINVAL, "hist is NULL");
  if (h->sweep + (uint64_t)n >= 0xFFFFFFFFull) return fail(SU2_EINVAL, "sweep counter would reach the reserved index 2^32 - 1");
  DeviceGuard dg(h->device);
  for (int c0 = 0; c0 < n; c0 += kHistRing) {
    const int m = n - c0 < kHistRing ? n - c0 : kHistRing;
    int left = m;
    if (left >= kGraphSweeps) {
      if (!h->mgraph) {
        int rc = build_graph(h, true);
        if (rc) return rc;
      }
      while (left >= kGraphSweeps) {
        SU2_CU(cudaGraphLaunch(h->mgraph, h->stream));
        count_launches(kernels_per_sweep(h, true) * kGraphSweeps);
        left -= kGraphSweeps;
      }
    }
    for (; left > 0; --left) SU2_CU(enqueue_measured_sweep(h, h->stream));
    // sweep h->sweep + c0 + i sits in ring row (h->sweep + c0 + i) mod
    // kHistRing: at most two contiguous pieces
    const int r0 = (int)((h->sweep + (uint64_t)c0) % (uint64_t)kHistRing);
    const int first = m < kHistRing - r0 ? m : kHistRing - r0;
    SU2_CU(cudaMemcpyAsync(hist + 4 * (size_t)c0, h->d_hist + 4 * (size_t)r0, (size_t)first * 4 * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
    if (m > first)
      SU2_CU(cudaMemcpyAsync(hist + 4 * (size_t)(c0 + first), h->d_hist, (size_t)(m - first) * 4 * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
    SU2_CU(cudaStreamSynchronize(h->stream));
  }
  h->sweep += (uint64_t)n;
  if (n) h->smeared = 0;
  return check_pair(h);
}

extern "C" int su2_layout_compare(su2_lattice* h, int sweeps, double ms[3], uint64_t* mismatch) {
  clear_error();
  if (!h || !ms || !mismatch) return fail(SU2_EINVAL, "handle, ms and mismatch must not be NULL");
  if (h->prec != SU2_F32) return fail(SU2_EINVAL, "the layout comparison runs on FP32 handles only");
  if (sweeps < 1) return fail(SU2_EINVAL, "sweeps must be >= 1");
  if (h->sweep + (uint64_t)sweeps >= 0xFFFFFFFFull) return fail(SU2_EINVAL, "sweep counter would reach the reserved index 2^32 - 1");
  DeviceGuard dg(h->device);
  cudaStream_t st = h->stream;
  const LatticeView v = view(h);
  const HBParams hp = hb_params(h);
  const size_t bytes = (size_t)8 * h->g.vh * 16;
  void *start = nullptr, *first = nullptr, *other = nullptr;
  unsigned long long* d_count = nullptr;
  cudaEvent_t ev[6] = {};
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    if (start) cudaFree(start);
    if (first) cudaFree(first);
    if (other) cudaFree(other);
    if (d_count) cudaFree(d_count);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  };
  SU2_CU_CLEAN(cudaMalloc(&start, bytes), cleanup());
  SU2_CU_CLEAN(cudaMalloc(&first, bytes), cleanup());
  SU2_CU_CLEAN(cudaMalloc(&other, bytes), cleanup());
  SU2_CU_CLEAN(cudaMalloc(&d_count, sizeof(unsigned long long)), cleanup());
  for (auto& e : ev) SU2_CU_CLEAN(cudaEventCreate(&e), cleanup());
  SU2_CU_CLEAN(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st), cleanup());
  SU2_CU_CLEAN(cudaMemcpyAsync(start, h->links, bytes, cudaMemcpyDeviceToDevice, st), cleanup());
  // 1. the library's kernels
  SU2_CU_CLEAN(cudaEventRecord(ev[0], st), cleanup());
  for (int i = 0; i < sweeps; ++i) SU2_CU_CLEAN(enqueue_sweep(h, (uint32_t)i, st), cleanup());
  SU2_CU_CLEAN(cudaEventRecord(ev[1], st), cleanup());
  SU2_CU_CLEAN(cudaMemcpyAsync(first, h->links, bytes, cudaMemcpyDeviceToDevice, st), cleanup());
  // 2. the plain kernel on the library's layout
  SU2_CU_CLEAN(cudaMemcpyAsync(h->links, start, bytes, cudaMemcpyDeviceToDevice, st), cleanup());
  SU2_CU_CLEAN(cudaEventRecord(ev[2], st), cleanup());
  for (int i = 0; i < sweeps; ++i)
    for (int mu = 0; mu < 4; ++mu)
      for (int p = 0; p < 2; ++p)
        SU2_CU_CLEAN(launch_hb_plain(v, h->links, false, mu, p, h->d_sweep, (uint32_t)i, hp, st), cleanup());
  SU2_CU_CLEAN(cudaEventRecord(ev[3], st), cleanup());
  SU2_CU_CLEAN(launch_count_diff(h->links, first, bytes, d_count, st), cleanup());
  // 3. the plain kernel on the site-major single array
  SU2_CU_CLEAN(cudaMemcpyAsync(h->links, start, bytes, cudaMemcpyDeviceToDevice, st), cleanup());
  SU2_CU_CLEAN(launch_site_major(v, other, true, st), cleanup());
  SU2_CU_CLEAN(cudaEventRecord(ev[4], st), cleanup());
  for (int i = 0; i < sweeps; ++i)
    for (int mu = 0; mu < 4; ++mu)
      for (int p = 0; p < 2; ++p)
        SU2_CU_CLEAN(launch_hb_plain(v, other, true, mu, p, h->d_sweep, (uint32_t)i, hp, st), cleanup());
  SU2_CU_CLEAN(cudaEventRecord(ev[5], st), cleanup());
  SU2_CU_CLEAN(launch_site_major(v, other, false, st), cleanup());
  SU2_CU_CLEAN(launch_count_diff(h->links, first, bytes, d_count, st), cleanup());
  // the handle keeps the first run's result
  SU2_CU_CLEAN(cudaMemcpyAsync(h->links, first, bytes, cudaMemcpyDeviceToDevice, st), cleanup());
  SU2_CU_CLEAN(launch_add_u32(h->d_sweep, (uint32_t)sweeps, st), cleanup());
  unsigned long long count = 0;
  SU2_CU_CLEAN(cudaMemcpyAsync(&count, d_count, sizeof count, cudaMemcpyDeviceToHost, st), cleanup());
  SU2_CU_CLEAN(cudaStreamSynchronize(st), cleanup());
  float t[3];
  for (int k = 0; k < 3; ++k) SU2_CU_CLEAN(cudaEventElapsedTime(&t[k], ev[2 * k], ev[2 * k + 1]), cleanup());
  cleanup();
  for (int k = 0; k < 3; ++k) ms[k] = t[k];
  *mismatch = count;
  h->sweep += (uint64_t)sweeps;
  h->smeared = 0;
  return SU2_OK;
}

extern "C" int su2_kernel_launches(uint64_t* n) {
  clear_error();
  if (!n) return fail(SU2_EINVAL, "n is NULL");
  *n = launches_total();
  return SU2_OK;
}

extern "C" int su2_heatbath_substep(su2_lattice* h, int mu, int parity, uint32_t sweep) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (mu < 0 || mu > 3 || parity < 0 || parity > 1) return fail(SU2_EINVAL, "mu must be 0..3 and parity 0..1");
  DeviceGuard dg(h->device);
  SU2_CU(launch_heatbath(view(h), mu, parity, nullptr, sweep, hb_params(h), nullptr, h->stream));
  h->smeared = 0;
  return SU2_OK;
}

extern "C" int su2_heatbath_pair(su2_lattice* h, int mu, uint32_t sweep) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (mu < 0 || mu > 3) return fail(SU2_EINVAL, "mu must be 0..3");
  if (h->prec == SU2_F64) return fail(SU2_EINVAL, "the fused pair runs FP32 and F16Q lattices only");
  DeviceGuard dg(h->device);
  h->pair_used = true;
  SU2_CU(launch_heatbath_pair(view(h), mu, nullptr, sweep, hb_params(h), h->d_pair, h->d_done0, h->stream));
  h->smeared = 0;
  return SU2_OK;
}

extern "C" int su2_overrelax_sweep(su2_lattice* h, int n) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (n < 0) return fail(SU2_EINVAL, "n must be >= 0");
  DeviceGuard dg(h->device);
  for (int i = 0; i < n; ++i)
    for (int mu = 0; mu < 4; ++mu)
      for (int p = 0; p < 2; ++p) SU2_CU(launch_overrelax(view(h), mu, p, h->stream));
  if (n) h->smeared = 0;
  return SU2_OK;
}

static int fetch_out(su2_lattice* h, int count, double* dst) {
  SU2_CU(cudaMemcpyAsync(h->h_out, h->scratch.out, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  SU2_CU(cudaStreamSynchronize(h->stream));
  int rc = check_pair(h);
  if (rc) return rc;
  std::memcpy(dst, h->h_out, count * sizeof(double));
  return SU2_OK;
}

extern "C" int su2_plaquette(su2_lattice* h, double out[3]) {
  clear_error();
  if (!h || !out) return fail(SU2_EINVAL, "NULL argument");
  DeviceGuard dg(h->device);
  SU2_CU(launch_plaquette(view(h), h->scratch, h->stream));
  return fetch_out(h, 3, out);
}

extern "C" int su2_plaquette_slices(su2_lattice* h, int t_first, int t_count, double out[3]) {
  clear_error();
  if (!h || !out) return fail(SU2_EINVAL, "NULL argument");
  if (t_first < 0 || t_count < 1 || t_first + t_count > h->dims[3])
    return fail(SU2_EINVAL, "time slices [%d, %d) outside 0..%d", t_first, t_first + t_count, h->dims[3]);
  DeviceGuard dg(h->device);
  const int64_t nsig = 2 * h->g.vh / h->dims[3];
  SU2_CU(launch_plaquette(view(h), h->scratch, h->stream, nsig * t_first, nsig * t_count));
  return fetch_out(h, 3, out);
}

extern "C" int su2_time_lines(su2_lattice* h, int t_first, int t_count, double* out) {
  clear_error();
  if (!h || !out) return fail(SU2_EINVAL, "NULL argument");
  if (t_first < 0 || t_count < 1 || t_first + t_count > h->dims[3])
    return fail(SU2_EINVAL, "time slices [%d, %d) outside 0..%d", t_first, t_first + t_count, h->dims[3]);
  DeviceGuard dg(h->device);
  const int64_t nsig = 2 * h->g.vh / h->dims[3];
  const int64_t chunk = 4 * h->staging_sites;  // spatial sites whose 4 doubles fit the staging buffer
  for (int64_t x0 = 0; x0 < nsig; x0 += chunk) {
    const int64_t nx = nsig - x0 < chunk ? nsig - x0 : chunk;
    SU2_CU(launch_time_lines(view(h), t_first, t_count, x0, nx, h->staging, h->stream));
    SU2_CU(cudaMemcpyAsync(out + 4 * x0, h->staging, (size_t)nx * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
  }
  SU2_CU(cudaStreamSynchronize(h->stream));
  return check_pair(h);
}

extern "C" int su2_set_site_offset(su2_lattice* h, uint32_t site0) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  h->g.site0 = site0;
  drop_graph(h);
  return SU2_OK;
}

extern "C" int su2_polyakov(su2_lattice* h, double* L) {
  clear_error();
  if (!h || !L) return fail(SU2_EINVAL, "NULL argument");
  DeviceGuard dg(h->device);
  SU2_CU(launch_polyakov(view(h), h->scratch, h->stream));
  return fetch_out(h, 1, L);
}

extern "C" int su2_ape_smear(su2_lattice* h, double alpha, int n) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (!(alpha >= 0.0 && alpha < 1.0)) return fail(SU2_EINVAL, "alpha must be in [0, 1)");
  if (n < 0) return fail(SU2_EINVAL, "n must be >= 0");
  DeviceGuard dg(h->device);
  if (n == 0) {
    SU2_CU(launch_copy_spatial(view(h), h->ape[0], h->stream));
    h->smeared = 1;
    return SU2_OK;
  }
  LatticeView src = view(h);
  int cur = 0;
  for (int i = 0; i < n; ++i) {
    SU2_CU(launch_ape(src, h->ape[cur], alpha, h->stream));
    src.links = h->ape[cur];
    cur ^= 1;
  }
  h->smeared = (cur ^ 1) + 1;
  return SU2_OK;
}

extern "C" int su2_wilson_loops(su2_lattice* h, int Rmax, int Tmax, int use_smeared, double* out) {
  clear_error();
  if (!h || !out) return fail(SU2_EINVAL, "NULL argument");
  const int rlim = h->dims[0] < h->dims[1] ? (h->dims[0] < h->dims[2] ? h->dims[0] : h->dims[2])
                                           : (h->dims[1] < h->dims[2] ? h->dims[1] : h->dims[2]);
  if (Rmax < 1 || Rmax > rlim || Rmax > 32) return fail(SU2_EINVAL, "Rmax must be in 1..min(N0,N1,N2,32)");
  if (Tmax < 1 || Tmax > h->dims[3] || Tmax > 32) return fail(SU2_EINVAL, "Tmax must be in 1..min(N3,32)");
  if (use_smeared && !h->smeared) return fail(SU2_ESTATE, "no smeared links since the last update");
  DeviceGuard dg(h->device);
  const void* spatial = use_smeared ? h->ape[h->smeared - 1] : h->links;
  SU2_CU(launch_wilson(view(h), spatial, Rmax, Tmax, h->scratch, h->stream));
  return fetch_out(h, Rmax * Tmax, out);
}

// The device-visible address of page-locked host memory (cudaHostAlloc,
// cudaHostRegister: the conversion kernel then reads it directly over the
// host link, at the copy engine's rate), or NULL for pageable memory.
// The address a kernel on `device` reads `p` through: page-locked host memory
// (mapped), or device / managed memory of that device; nullptr for pageable
// host memory.  *other_device is set for device memory of another GPU.
static void* device_readable(const void* p, int device, bool* other_device) {
  *other_device = false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged) return a.devicePointer;
  if (a.type == cudaMemoryTypeDevice) {
    if (a.device != device) {
      *other_device = true;
      return nullptr;
    }
    return a.devicePointer;
  }
  return nullptr;
}

// Sites [first, first + count) in canonical FP64 order into host[16 * count],
// through the device staging buffer and the copy engine (kernel stores to
// host memory run at a fraction of the copy engine's rate over the host link).
static int copy_sites_out(su2_lattice* h, int64_t first, int64_t count, double* host) {
  DeviceGuard dg(h->device);
  for (int64_t k = 0; k < count; k += h->staging_sites) {
    const int64_t ns = count - k < h->staging_sites ? count - k : h->staging_sites;
    SU2_CU(launch_to_canonical(view(h), h->staging, first + k, ns, h->stream));
    SU2_CU(cudaMemcpyAsync(host + 16 * k, h->staging, (size_t)ns * 16 * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
  }
  SU2_CU(cudaStreamSynchronize(h->stream));
  return check_pair(h);
}

extern "C" int su2_get_links(su2_lattice* h, double* host) {
  clear_error();
  if (!h || !host) return fail(SU2_EINVAL, "NULL argument");
  return copy_sites_out(h, 0, 2 * h->g.vh, host);
}

extern "C" int su2_get_sites(su2_lattice* h, int64_t first, int64_t count, double* host) {
  clear_error();
  if (!h || (!host && count > 0)) return fail(SU2_EINVAL, "NULL argument");
  const int64_t V = 2 * h->g.vh;
  if (first < 0 || count < 0 || first > V || count > V - first)
    return fail(SU2_EINVAL, "sites [%lld, %lld) outside the lattice of %lld sites", (long long)first,
                (long long)(first + count), (long long)V);
  return copy_sites_out(h, first, count, host);
}

extern "C" int su2_set_links(su2_lattice* h, const double* links) {
  clear_error();
  if (!h || !links) return fail(SU2_EINVAL, "NULL argument");
  DeviceGuard dg(h->device);
  const int64_t V = 2 * h->g.vh;
  bool other = false;
  const void* d = device_readable(links, h->device, &other);
  if (other) return fail(SU2_EINVAL, "links are in the memory of another device");
  if (d) {
    SU2_CU(launch_from_canonical(view(h), static_cast<const double*>(d), 0, V, h->stream));
  } else {
    for (int64_t s0 = 0; s0 < V; s0 += h->staging_sites) {
      const int64_t ns = V - s0 < h->staging_sites ? V - s0 : h->staging_sites;
      SU2_CU(cudaMemcpyAsync(h->staging, links + 16 * s0, (size_t)ns * 16 * sizeof(double),
                             cudaMemcpyHostToDevice, h->stream));
      SU2_CU(launch_from_canonical(view(h), h->staging, s0, ns, h->stream));
    }
  }
  SU2_CU(cudaStreamSynchronize(h->stream));
  h->smeared = 0;
  return SU2_OK;
}

extern "C" int su2_sweep_count(su2_lattice* h, uint64_t* n) {
  clear_error();
  if (!h || !n) return fail(SU2_EINVAL, "NULL argument");
  *n = h->sweep;
  return SU2_OK;
}

extern "C" int su2_set_sweep_count(su2_lattice* h, uint64_t n) {
  clear_error();
  if (!h) return fail(SU2_EINVAL, "handle is NULL");
  if (n >= 0xFFFFFFFFull) return fail(SU2_EINVAL, "sweep counter must be below 2^32 - 1");
  DeviceGuard dg(h->device);
  const uint32_t v = (uint32_t)n;
  SU2_CU(cudaMemcpyAsync(h->d_sweep, &v, sizeof v, cudaMemcpyHostToDevice, h->stream));
  SU2_CU(cudaStreamSynchronize(h->stream));
  h->sweep = n;
  return SU2_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint files
// ---------------------------------------------------------------------------
namespace {
struct FileHeader {
  char magic[8];
  uint32_t version;
  int32_t dims[4];
  int32_t prec;
  double beta;
  uint64_t seed;
  uint64_t sweep;
  int32_t max_tries;
  int32_t sampler;
};
}  // namespace

extern "C" int su2_save(su2_lattice* h, const char* path) {
  clear_error();
  if (!h || !path) return fail(SU2_EINVAL, "NULL argument");
  const int64_t V = 2 * h->g.vh;
  std::vector<double> buf;
  try {
    buf.resize((size_t)V * 16);
  } catch (...) {
    return fail(SU2_ENOMEM, "host buffer for %lld sites", (long long)V);
  }
  int rc = su2_get_links(h, buf.data());
  if (rc) return rc;
  FileHeader fh;
  std::memset(&fh, 0, sizeof fh);
  std::memcpy(fh.magic, "SU2GB300", 8);
  fh.version = 1;
  for (int i = 0; i < 4; ++i) fh.dims[i] = h->dims[i];
  fh.prec = h->prec;
  fh.beta = h->beta;
  fh.seed = h->seed;
  fh.sweep = h->sweep;
  fh.max_tries = h->max_tries;
  fh.sampler = h->sampler;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(SU2_EINVAL, "cannot open %s for writing", path);
  const bool ok = std::fwrite(&fh, sizeof fh, 1, f) == 1 &&
                  std::fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  if (std::fclose(f) != 0 || !ok) return fail(SU2_EINVAL, "short write to %s", path);
  return SU2_OK;
}

extern "C" int su2_load(su2_lattice** out, const char* path, int prec, void* cuda_stream) {
  clear_error();
  if (!out || !path) return fail(SU2_EINVAL, "NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(SU2_EINVAL, "cannot open %s", path);
  FileHeader fh;
  if (std::fread(&fh, sizeof fh, 1, f) != 1 || std::memcmp(fh.magic, "SU2GB300", 8) != 0 || fh.version != 1) {
    std::fclose(f);
    return fail(SU2_EINVAL, "%s is not a version-1 SU2GB300 checkpoint", path);
  }
  int dims[4] = {fh.dims[0], fh.dims[1], fh.dims[2], fh.dims[3]};
  int rc = check_dims(dims);
  if (rc) { std::fclose(f); return rc; }
  const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  std::vector<double> buf;
  try {
    buf.resize((size_t)V * 16);
  } catch (...) {
    std::fclose(f);
    return fail(SU2_ENOMEM, "host buffer for %lld sites", (long long)V);
  }
  const bool ok = std::fread(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return fail(SU2_EINVAL, "%s is truncated", path);
  su2_lattice* h = nullptr;
  rc = su2_init(&h, dims, fh.beta, fh.seed, SU2_COLD, prec < 0 ? fh.prec : prec, cuda_stream);
  if (rc) return rc;
  if ((rc = su2_set_options(h, fh.max_tries, fh.sampler)) || (rc = su2_set_links(h, buf.data())) ||
      (rc = su2_set_sweep_count(h, fh.sweep))) {
    su2_destroy(h);
    return rc;
  }
  *out = h;
  return SU2_OK;
}
