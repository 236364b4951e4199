// Batched lattices: many independent lattices of uneven extents and couplings
// swept together by one persistent kernel per call (captured in a CUDA graph).
//
// The heat bath of each lattice follows Section 2 (Eqs. 5-9, 11) and the
// checkerboard of Section 4 exactly as for a single lattice; lattice i uses
// Philox lattice_id = i, so every link's draws are fixed by (lattice, sweep,
// site, direction) and the result does not depend on the schedule below.
//
// Schedule.  The cooperative grid is split into G groups of CTAs.  The
// lattices are dealt to the groups largest first, each to the group with the
// least work so far, and each group gets a share of the CTAs in proportion
// to its work, so that the groups finish together and small lattices do not
// leave most of a group's threads idle.  A group sweeps its lattices one
// after another, all n sweeps of one lattice before the next.  Substeps
// within a lattice are ordered by a barrier among the group's CTAs only,
// which is cheaper than a grid-wide barrier (a one-CTA group needs only the
// block barrier), and the G lattices in flight are re-read from L2 rather
// than HBM between substeps when they fit.  G defaults to one group per
// lattice; su2_batch_tune times candidate G on a scratch copy of the links.
//
// Every barrier wait is bounded twice (global timer and iteration count); a
// wait that runs out raises a device error flag, all blocks leave, and the
// host reports SU2_ETIMEOUT.  Cooperative launch guarantees that all CTAs are
// co-resident.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "su2.h"
#include "su2_capi_util.h"
#include "su2_hb_link.cuh"
#include "su2_internal.h"

using namespace su2;

namespace su2 {

struct BatchLattice {
  Geom g;
  void* links;
  double beta;
};

// One barrier per group, each on its own 128-byte line.
struct GroupBarrier {
  unsigned int count;
  unsigned int gen;
  unsigned int pad[30];
};

struct BatchCtl {
  int err;             // 1: a barrier wait timed out
  unsigned int extra;  // arrivals a barrier waits for beyond its group (fault injection)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier among the `n` CTAs of one group.  Returns false if any wait timed out.
__device__ __forceinline__ bool group_barrier(GroupBarrier* gb, unsigned int n, BatchCtl* ctl,
                                              unsigned long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  // a group of one CTA needs no more than the block barrier (unless a fault
  // is injected, which makes every barrier wait for an arrival that never comes)
  if (n == 1 && ctl->extra == 0) return true;
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &gb->gen;
    volatile int* verr = &ctl->err;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&gb->count, 1u) + 1u;
    if (arrived == n + ctl->extra) {
      gb->count = 0;
      __threadfence();
      atomicExch(&gb->gen, g + 1u);
    } else {
      // bounded twice over: by the global timer and by an iteration count
      const unsigned long long t0 = global_ns();
      unsigned long long spins = 0;
      while (*vgen == g) {
        if (*verr) break;
        if (global_ns() - t0 > timeout_ns || ++spins > (1ull << 24)) {
          atomicExch(&ctl->err, 1);
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

// Block sizes the batched kernel is built for (su2_batch_set_block_size,
// searched by su2_batch_tune); the deferral queue holds two entries a thread.
constexpr int kBatchThreads = 256;  // default
template <int BS> struct BatchQueue { static constexpr int value = 2 * BS; };

template <class R> struct BDeferred {
  Quat<R> w;
  R alpha;
  int h;
  uint32_t site;
};

// One substep (MU, p) of one lattice by the CTAs of a group: trial 1 inline,
// rejected links queued and finished by the whole block at the end.  Links
// are read with coherent loads (other CTAs of the group wrote them before the
// last barrier).
template <int P, int MU, int PAR, int BS>
__device__ __forceinline__ void batch_substep(const Links<P, kClassOff>& L, const Geom& g, int rank, int cpg,
                                              uint32_t sweep, uint32_t tag, typename Real<P>::T beta,
                                              const HBParams& hp, BDeferred<typename Real<P>::T>* queue, int* qn) {
  using R = typename Real<P>::T;
  using M = Math<R>;
  constexpr int p = PAR;
  const int vh = (int)g.vh;
  constexpr int kQ = BatchQueue<BS>::value;
  for (int base = rank * BS; base < vh; base += cpg * BS) {
    const int h = base + threadIdx.x;
    if (h >= vh) continue;
    const Site x = site_from_half(g, (uint32_t)h, p);
    const Quat<R> sig = staple<P, MU, 0xF, false>(L, g, x, h, p);
    const uint32_t site = philox_site(g, x);
    const uint4 ctr = make_uint4(site, tag, sweep, 0u);
    const R k2 = qdot(sig, sig);
    const R invk = M::rsqrt(k2);
    const R alpha = beta * k2 * invk;
    if (!(alpha >= R(1e-12))) {
      uint4 c = ctr;
      c.w = 1u;
      L.st(2 * MU + p, h, haar_from<R>(philox(c, hp.rk)));
      continue;
    }
    const R inv2a = trial_inv2a(alpha);
    const R e = trial_e(alpha, hp.sampler);
    const Quat<R> w = qscale(sig, invk);
    R a0;
    uint4 rt;
    if (trial_a0<R>(alpha, inv2a, e, ctr, 1, hp, &a0, &rt)) {
      L.st(2 * MU + p, h, compose_link<R>(a0, w, ctr, rt, hp));
    } else if (hp.max_tries > 1) {
      const int slot = atomicAdd(qn, 1);
      if (slot < kQ) {
        BDeferred<R> d;
        d.w = w;
        d.alpha = alpha;
        d.h = h;
        d.site = site;
        queue[slot] = d;
      } else if (sample_a0_from<R>(2, alpha, inv2a, e, ctr, hp, &a0, &rt)) {
        L.st(2 * MU + p, h, compose_link<R>(a0, w, ctr, rt, hp));
      }
    }
  }
  __syncthreads();
  const int n = min(*qn, kQ);
  for (int i = threadIdx.x; i < n; i += BS) {
    const BDeferred<R> d = queue[i];
    const uint4 ctr = make_uint4(d.site, tag, sweep, 0u);
    R a0;
    uint4 rt;
    if (sample_a0_from<R>(2, d.alpha, trial_inv2a(d.alpha), trial_e(d.alpha, hp.sampler), ctr, hp, &a0, &rt))
      L.st(2 * MU + p, d.h, compose_link<R>(a0, d.w, ctr, rt, hp));
  }
  __syncthreads();
  if (threadIdx.x == 0) *qn = 0;
}

// One over-relaxation substep (MU, p) of one lattice by the CTAs of a group.
template <int P, int MU, int PAR, int BS>
__device__ __forceinline__ void batch_or_substep(const Links<P, kClassOff>& L, const Geom& g, int rank, int cpg) {
  const int vh = (int)g.vh;
  for (int h = rank * BS + (int)threadIdx.x; h < vh; h += cpg * BS) or_link<P, MU, PAR, false>(L, g, h);
}

// 1024 threads per SM (64 registers a thread) for FP32 / F16Q, 512 for FP64.
template <int P, int BS>
__global__ void __launch_bounds__(BS, (P == kF64 ? 512 : 1024) / BS)
    k_batch_groups(const BatchLattice* __restrict__ desc, const int* __restrict__ order,
                   const int4* __restrict__ plan, const int* __restrict__ cta_group, int nsweeps, int nor,
                   const uint32_t* sweep_base, const __grid_constant__ HBParams hp, GroupBarrier* bars, BatchCtl* ctl,
                   unsigned long long timeout_ns) {
  using R = typename Real<P>::T;
  __shared__ BDeferred<R> queue[BatchQueue<BS>::value];
  __shared__ int qn;
  const int group = cta_group[blockIdx.x];
  if (group < 0) return;
  // plan[group] = (first lattice in `order`, lattices, first CTA, CTAs)
  const int4 pl = plan[group];
  const int cpg = pl.w;
  const int rank = (int)blockIdx.x - pl.z;
  if (threadIdx.x == 0) qn = 0;
  __syncthreads();
  const uint32_t sweep0 = *sweep_base;
  // one substep (mu, p) of lattice l by this group's CTAs
  auto substep = [&](int l, uint32_t sweep, int mu, int p) {
    const Geom g = desc[l].g;
    Links<P, kClassOff> L;
    L.set(desc[l].links, g.vh);
    const R beta = (R)desc[l].beta;
    const uint32_t tag = (uint32_t)mu | ((uint32_t)l << 2);
    switch (2 * mu + p) {
      case 0: batch_substep<P, 0, 0, BS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn); break;
      case 1: batch_substep<P, 0, 1, BS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn); break;
      case 2: batch_substep<P, 1, 0, BS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn); break;
      case 3: batch_substep<P, 1, 1, BS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn); break;
      case 4: batch_substep<P, 2, 0, BS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn); break;
      case 5: batch_substep<P, 2, 1, BS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn); break;
      case 6: batch_substep<P, 3, 0, BS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn); break;
      default: batch_substep<P, 3, 1, BS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn); break;
    }
  };
  // one lattice at a time, a barrier after each substep: the lattice's links
  // stay in L2 through its sweeps (interleaving the group's lattices between
  // barriers halves the barriers but spills the working set: 32.5 against
  // 35.5 G updates/s for the 64-lattice batch at 32 groups)
  // `nor` over-relaxation sweeps precede each heat-bath sweep
  auto or_substep = [&](int l, int mu, int p) {
    const Geom g = desc[l].g;
    Links<P, kClassOff> L;
    L.set(desc[l].links, g.vh);
    switch (2 * mu + p) {
      case 0: batch_or_substep<P, 0, 0, BS>(L, g, rank, cpg); break;
      case 1: batch_or_substep<P, 0, 1, BS>(L, g, rank, cpg); break;
      case 2: batch_or_substep<P, 1, 0, BS>(L, g, rank, cpg); break;
      case 3: batch_or_substep<P, 1, 1, BS>(L, g, rank, cpg); break;
      case 4: batch_or_substep<P, 2, 0, BS>(L, g, rank, cpg); break;
      case 5: batch_or_substep<P, 2, 1, BS>(L, g, rank, cpg); break;
      case 6: batch_or_substep<P, 3, 0, BS>(L, g, rank, cpg); break;
      default: batch_or_substep<P, 3, 1, BS>(L, g, rank, cpg); break;
    }
  };
  for (int li = 0; li < pl.y; ++li)
    for (int sw = 0; sw < nsweeps; ++sw) {
      for (int k = 0; k < nor; ++k)
        for (int mu = 0; mu < 4; ++mu)
          for (int p = 0; p < 2; ++p) {
            or_substep(order[pl.x + li], mu, p);
            if (!group_barrier(bars + group, (unsigned)cpg, ctl, timeout_ns)) return;
          }
      for (int mu = 0; mu < 4; ++mu)
        for (int p = 0; p < 2; ++p) {
          substep(order[pl.x + li], sweep0 + (uint32_t)sw, mu, p);
          if (!group_barrier(bars + group, (unsigned)cpg, ctl, timeout_ns)) return;
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
  void* base;
  size_t links_bytes;  // the lattices' stores occupy [base, base + links_bytes)
  BatchLattice* d_desc;
  int* d_order;
  int4* d_plan;
  int* d_cta_group;
  GroupBarrier* d_bars;
  BatchCtl* d_ctl;
  uint32_t* d_sweep;
  Scratch scratch;
  double* d_results;
  double* h_results;
  cudaStream_t stream;
  bool own_stream;
  cudaStream_t cap_stream;
  cudaGraphExec_t graph;
  int graph_n;
  int grid;    // co-resident CTAs
  int groups;  // current G
  int bs;      // threads per CTA (256 or 512)
  unsigned long long timeout_ns;
  int nor;                   // over-relaxation sweeps before each heat-bath sweep
  unsigned int fault_extra;  // injected missing barrier arrivals (0: none)
  bool fault_once;           // the injected fault is withdrawn after its first timeout
};

namespace {

constexpr int kMaxGroups = 1024;
constexpr int kMaxCtas = 1 << 16;  // co-resident CTAs of the persistent grid

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int P, int BS> int occupancy_blocks() {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_groups<P, BS>, BS, 0);
  return per_sm;
}

template <int BS> int batch_grid_bs(int prec) {
  int per_sm = prec == kF64 ? occupancy_blocks<kF64, BS>()
                            : prec == kF32 ? occupancy_blocks<kF32, BS>() : occupancy_blocks<kF16Q, BS>();
  if (per_sm < 1) per_sm = 1;
  return per_sm * device_info().sms;
}

int batch_grid(int prec, int bs) { return bs == 512 ? batch_grid_bs<512>(prec) : batch_grid_bs<256>(prec); }

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

// Deal the lattices to G groups, largest first, each to the group with the
// least work so far, and give every group a share of the co-resident CTAs in
// proportion to its work (at least one; remainders to the largest
// fractional shares), so that the groups finish their sweeps together and
// no group runs many idle threads on small lattices.  Writes the per-group
// plan (first lattice in `order`, lattices, first CTA, CTAs), the lattice
// order and the group of every CTA (-1: idle).
void make_plan(const su2_batch* b, int G, std::vector<int>& order, std::vector<int4>& plan,
               std::vector<int>& cta_group) {
  std::vector<int> idx(b->n);
  for (int i = 0; i < b->n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return b->desc[a].g.vh > b->desc[c].g.vh; });
  std::vector<int64_t> load(G, 0);
  std::vector<std::vector<int>> members(G);
  for (int i : idx) {
    int best = 0;
    for (int gi = 1; gi < G; ++gi)
      if (load[gi] < load[best]) best = gi;
    members[best].push_back(i);
    load[best] += b->desc[i].g.vh;
  }
  int64_t total = 0;
  for (int64_t l : load) total += l;
  const int ctas = std::max(b->grid, G);
  std::vector<int> share(G, 1);
  int used = G;
  std::vector<std::pair<double, int>> frac;
  for (int gi = 0; gi < G; ++gi) {
    const double want = (double)ctas * (double)load[gi] / (double)std::max<int64_t>(total, 1);
    const int extra = std::max(0, (int)want - 1);
    share[gi] += extra;
    used += extra;
    frac.push_back({want - (double)(int)want, gi});
  }
  std::sort(frac.begin(), frac.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& c) {
    return a.first > c.first;
  });
  for (size_t k = 0; k < frac.size() && used < ctas; ++k, ++used) share[frac[k].second] += 1;
  order.clear();
  plan.assign(G, make_int4(0, 0, 0, 0));
  cta_group.assign(b->grid, -1);
  int cta = 0;
  for (int gi = 0; gi < G; ++gi) {
    plan[gi].x = (int)order.size();
    plan[gi].y = (int)members[gi].size();
    order.insert(order.end(), members[gi].begin(), members[gi].end());
    const int take = std::min(share[gi], b->grid - cta);
    plan[gi].z = cta;
    plan[gi].w = take;
    for (int k = 0; k < take; ++k) cta_group[cta + k] = gi;
    cta += take;
  }
}

// Default G: every lattice its own group (all lattices in flight at once),
// as many as the co-resident CTAs allow.  With CTAs shared in proportion to
// work this measured fastest for the 64-lattice benchmark batch (FP32:
// 38.0 G updates/s at G = 64, 36.6 at 32, 30.0 at 16, 12.8 at 4);
// su2_batch_tune measures instead of assuming.
int default_groups(const su2_batch* b) {
  return (int)std::max(1, std::min({b->n, b->grid, kMaxGroups}));
}

int set_groups(su2_batch* b, int G) {
  std::vector<int> order, cta_group;
  std::vector<int4> plan;
  make_plan(b, G, order, plan, cta_group);
  SU2_CU(cudaMemcpyAsync(b->d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  SU2_CU(cudaMemcpyAsync(b->d_plan, plan.data(), plan.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
  SU2_CU(cudaMemcpyAsync(b->d_cta_group, cta_group.data(), cta_group.size() * sizeof(int), cudaMemcpyHostToDevice,
                         b->stream));
  SU2_CU(cudaStreamSynchronize(b->stream));
  b->groups = G;
  drop_graph(b);
  return SU2_OK;
}

cudaError_t launch_groups(const su2_batch* b, const BatchLattice* d_desc, int n, cudaStream_t st) {
  const HBParams hp = batch_hp(b);
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(b->bs);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const uint32_t* sw = b->d_sweep;
  cudaError_t e;
  auto go = [&](auto kernel) {
    return cudaLaunchKernelEx(&cfg, kernel, d_desc, (const int*)b->d_order, (const int4*)b->d_plan,
                              (const int*)b->d_cta_group, n, b->nor, sw, hp, b->d_bars, b->d_ctl, b->timeout_ns);
  };
  if (b->bs == 512) {
    e = b->prec == kF64 ? go(k_batch_groups<kF64, 512>)
                        : b->prec == kF32 ? go(k_batch_groups<kF32, 512>) : go(k_batch_groups<kF16Q, 512>);
  } else {
    e = b->prec == kF64 ? go(k_batch_groups<kF64, 256>)
                        : b->prec == kF32 ? go(k_batch_groups<kF32, 256>) : go(k_batch_groups<kF16Q, 256>);
  }
  if (e == cudaSuccess) count_launches(1);
  return e;
}

// After a batched sweep: SU2_ETIMEOUT if a barrier wait gave up.  The handle
// then recovers for the next call: the error flag and every group barrier
// are cleared and the sweep counters (host and device) go back to their
// values before the call (`sweep_before`); the links are left as the
// aborted kernel left them, which is undefined.
int check_ctl(su2_batch* b, uint64_t sweep_before) {
  int err = 0;
  SU2_CU(cudaMemcpyAsync(&err, &b->d_ctl->err, sizeof err, cudaMemcpyDeviceToHost, b->stream));
  SU2_CU(cudaStreamSynchronize(b->stream));
  if (!err) return SU2_OK;
  if (b->fault_once) {
    b->fault_extra = 0;
    b->fault_once = false;
    b->timeout_ns = 1000000000ull;
    drop_graph(b);  // the captured launch carries the short test timeout
  }
  BatchCtl ctl;
  std::memset(&ctl, 0, sizeof ctl);
  ctl.extra = b->fault_extra;
  const uint32_t sw = (uint32_t)sweep_before;
  SU2_CU(cudaMemcpyAsync(b->d_ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, b->stream));
  SU2_CU(cudaMemsetAsync(b->d_bars, 0, kMaxGroups * sizeof(GroupBarrier), b->stream));
  SU2_CU(cudaMemcpyAsync(b->d_sweep, &sw, sizeof sw, cudaMemcpyHostToDevice, b->stream));
  SU2_CU(cudaStreamSynchronize(b->stream));
  b->sweep = sweep_before;
  return fail(SU2_ETIMEOUT, "a group barrier of the batched sweep timed out; the links of every lattice are "
                            "undefined (reload them with su2_batch_set_links)");
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
    // the batched kernel addresses a lattice's links by 32-bit offsets (kClassOff)
    const int64_t v = (int64_t)dims[4 * i] * dims[4 * i + 1] * dims[4 * i + 2] * dims[4 * i + 3];
    if (4 * v >= ((int64_t)1 << 32)) return fail(SU2_EINVAL, "lattice %d: a batch member must have fewer than 2^30 sites", i);
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
  // layout: per-lattice stores, descriptors, plan, barriers, sweep counter, scratch, results
  std::vector<size_t> off(n);
  size_t o = 0;
  b->desc.resize(n);
  for (int i = 0; i < n; ++i) {
    b->desc[i].g = make_geom(dims + 4 * i);
    b->desc[i].beta = betas[i];
    off[i] = o;
    o = align256(o + 8 * (size_t)b->desc[i].g.vh * link_bytes(prec));
  }
  b->links_bytes = o;
  const size_t o_desc = o; o = align256(o + n * sizeof(BatchLattice));
  const size_t o_order = o; o = align256(o + n * sizeof(int));
  const size_t o_plan = o; o = align256(o + kMaxGroups * sizeof(int4));
  const size_t o_ctag = o; o = align256(o + kMaxCtas * sizeof(int));
  const size_t o_bars = o; o = align256(o + kMaxGroups * sizeof(GroupBarrier));
  const size_t o_ctl = o; o = align256(o + sizeof(BatchCtl));
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
  b->d_order = (int*)(base + o_order);
  b->d_plan = (int4*)(base + o_plan);
  b->d_cta_group = (int*)(base + o_ctag);
  b->d_bars = (GroupBarrier*)(base + o_bars);
  b->d_ctl = (BatchCtl*)(base + o_ctl);
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
  SU2_CU_CLEAN(cudaMemsetAsync(b->d_bars, 0, kMaxGroups * sizeof(GroupBarrier), b->stream), su2_batch_destroy(b));
  BatchCtl ctl;
  std::memset(&ctl, 0, sizeof ctl);
  // Fault injection for the timeout path, host-side switch: every barrier
  // then waits for one arrival that never comes and every wait runs out.
  // SU2_FAULT=barrier_once: the same for the first batched sweep only (the
  // recovery test).
  const char* fault = std::getenv("SU2_FAULT");
  if (fault && (std::strcmp(fault, "barrier") == 0 || std::strcmp(fault, "barrier_once") == 0)) {
    ctl.extra = b->fault_extra = 1;
    b->timeout_ns = 20000000ull;
    b->fault_once = std::strcmp(fault, "barrier_once") == 0;
  }
  SU2_CU_CLEAN(cudaMemcpyAsync(b->d_ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, b->stream), su2_batch_destroy(b));
  SU2_CU_CLEAN(cudaMemsetAsync(b->d_sweep, 0, 64, b->stream), su2_batch_destroy(b));
  SU2_CU_CLEAN(cudaMemsetAsync(b->scratch.counter, 0, 64 * sizeof(unsigned int), b->stream), su2_batch_destroy(b));
  const PhiloxKey key = batch_key(b);
  for (int i = 0; i < n; ++i)
    SU2_CU_CLEAN(launch_init(lview(b, i), start, key, (uint32_t)i << 2, b->stream), su2_batch_destroy(b));
  SU2_CU_CLEAN(cudaStreamSynchronize(b->stream), su2_batch_destroy(b));
  b->bs = kBatchThreads;
  b->grid = batch_grid(prec, b->bs);
  int rc = set_groups(b, default_groups(b));
  if (rc) {
    su2_batch_destroy(b);
    return rc;
  }
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

extern "C" int su2_batch_set_overrelax(su2_batch* b, int n) {
  clear_error();
  if (!b) return fail(SU2_EINVAL, "handle is NULL");
  if (n < 0 || n > 16) return fail(SU2_EINVAL, "over-relaxation sweeps per heat-bath sweep must be in 0..16");
  b->nor = n;
  drop_graph(b);
  return SU2_OK;
}

// Threads per CTA of the batched kernel; the co-resident grid follows it and
// the group count is kept (capped at the new grid).
static int set_block_size(su2_batch* b, int bs) {
  b->bs = bs;
  b->grid = batch_grid(b->prec, bs);
  return set_groups(b, std::min(b->groups, std::min(b->grid, b->n)));
}

extern "C" int su2_batch_set_block_size(su2_batch* b, int threads) {
  clear_error();
  if (!b) return fail(SU2_EINVAL, "handle is NULL");
  if (threads != 256 && threads != 512) return fail(SU2_EINVAL, "block size must be 256 or 512");
  DeviceGuard dg(b->device);
  return set_block_size(b, threads);
}

extern "C" int su2_batch_block_size(su2_batch* b, int* threads) {
  clear_error();
  if (!b || !threads) return fail(SU2_EINVAL, "NULL argument");
  *threads = b->bs;
  return SU2_OK;
}

extern "C" int su2_batch_set_groups(su2_batch* b, int groups) {
  clear_error();
  if (!b) return fail(SU2_EINVAL, "handle is NULL");
  if (groups < 1 || groups > b->n || groups > b->grid || groups > kMaxGroups)
    return fail(SU2_EINVAL, "groups must be in 1..min(lattices, co-resident CTAs, %d)", kMaxGroups);
  DeviceGuard dg(b->device);
  return set_groups(b, groups);
}

extern "C" int su2_batch_groups(su2_batch* b, int* groups) {
  clear_error();
  if (!b || !groups) return fail(SU2_EINVAL, "NULL argument");
  *groups = b->groups;
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
    cudaError_t e = launch_groups(b, b->d_desc, n, b->cap_stream);
    if (e == cudaSuccess) e = launch_add_u32(b->d_sweep, (uint32_t)n, b->cap_stream);
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
  const uint64_t before = b->sweep;
  SU2_CU(cudaGraphLaunch(b->graph, b->stream));
  count_launches(2);
  b->sweep += (uint64_t)n;
  // a timed-out barrier is reported by the call that ran it
  return check_ctl(b, before);
}

extern "C" int su2_batch_tune(su2_batch* b, int sweeps, int* groups) {
  clear_error();
  if (!b) return fail(SU2_EINVAL, "handle is NULL");
  if (sweeps < 1) return fail(SU2_EINVAL, "sweeps must be >= 1");
  DeviceGuard dg(b->device);
  // a scratch copy of the links, so the chain itself is not advanced
  void* copy = nullptr;
  SU2_CU(cudaMallocAsync(&copy, b->links_bytes + align256(b->n * sizeof(BatchLattice)), b->stream));
  BatchLattice* d_desc_copy = (BatchLattice*)((char*)copy + b->links_bytes);
  std::vector<BatchLattice> dc = b->desc;
  for (int i = 0; i < b->n; ++i) dc[i].links = (char*)copy + ((char*)b->desc[i].links - (char*)b->base);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(copy, b->stream);
    cudaStreamSynchronize(b->stream);
  };
  cudaError_t e = cudaMemcpyAsync(copy, b->base, b->links_bytes, cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_desc_copy, dc.data(), b->n * sizeof(BatchLattice), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cleanup();
    return fail(SU2_ECUDA, "tuning set-up failed: %s", cudaGetErrorString(e));
  }
  const int original = b->groups, original_bs = b->bs;
  int best = original, best_bs = original_bs;
  float best_ms = 1e30f;
  for (int bs : {256, 512}) {
    int rc = set_block_size(b, bs);
    if (rc) { cleanup(); set_block_size(b, original_bs); set_groups(b, original); return rc; }
    std::vector<int> cand;
    for (int G : {1, 2, 4, 8, 12, 16, 24, 32, 40, 48, 64, 96, 128}) cand.push_back(G);
    cand.push_back(default_groups(b));
    cand.push_back(b->n);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (int G : cand) {
      if (G < 1 || G > b->n || G > b->grid || G > kMaxGroups) continue;
      rc = set_groups(b, G);
      if (rc) { cleanup(); return rc; }
      e = launch_groups(b, d_desc_copy, sweeps, b->stream);  // warm the schedule
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) e = launch_groups(b, d_desc_copy, sweeps, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        cleanup();
        set_block_size(b, original_bs);
        set_groups(b, original);
        return fail(SU2_ECUDA, "tuning launch failed: %s", cudaGetErrorString(e));
      }
      int rc2 = check_ctl(b, b->sweep);
      if (rc2) { cleanup(); set_block_size(b, original_bs); set_groups(b, original); return rc2; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = G; best_bs = bs; }
    }
  }
  cleanup();
  int rc = set_block_size(b, best_bs);
  if (!rc) rc = set_groups(b, best);
  if (rc) return rc;
  if (groups) *groups = best;
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
