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
#include <type_traits>
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

// One substep (MU, p) of one lattice by the CTAs of a group, each link by
// hb_link with coherent loads (other CTAs of the group wrote the links
// before the last barrier): trial 1 inline, rejected links queued and
// finished by the whole block at the end.  MEAS (odd substeps of MU >= 1 in
// a measured sweep): plaq accumulates Tr(U_MU(x) L(x)^dagger)/2 with L the
// staple's partial sum over NU < MU, as in the single-lattice substep.
template <int P, int MU, int PAR, int BS, bool MEAS>
__device__ __forceinline__ void batch_substep(const Links<P, kClassOff>& L, const Geom& g, int rank, int cpg,
                                              uint32_t sweep, uint32_t tag, typename Real<P>::T beta,
                                              const HBParams& hp, void* queue_mem, int* qn,
                                              PlainAcc<typename Real<P>::T>& plaq) {
  using R = typename Real<P>::T;
  using Def = Deferred<R, MEAS>;
  Def* queue = static_cast<Def*>(queue_mem);
  constexpr int kQ = BatchQueue<BS>::value;
  HBCount cnt;
  const int vh = (int)g.vh;
  for (int base = rank * BS; base < vh; base += cpg * BS) {
    const int h = base + threadIdx.x;
    if (h < vh)
      hb_link<P, MU, MEAS, PAR, false, kQ, kClassOff, false>(L, g, h, tag, sweep, beta, hp, queue, qn, plaq, cnt);
  }
  __syncthreads();
  hb_drain<P, MU, MEAS, PAR, kClassOff, false>(L, queue, min(*qn, kQ), tag, sweep, hp, plaq, cnt);
  __syncthreads();
  if (threadIdx.x == 0) *qn = 0;
}

// One over-relaxation substep (MU, p) of one lattice by the CTAs of a group.
template <int P, int MU, int PAR, int BS>
__device__ __forceinline__ void batch_or_substep(const Links<P, kClassOff>& L, const Geom& g, int rank, int cpg) {
  const int vh = (int)g.vh;
  for (int h = rank * BS + (int)threadIdx.x; h < vh; h += cpg * BS) or_link<P, MU, PAR, false>(L, g, h);
}

// Measured sweeps.  The plaquette (Eq. 12) comes from the sweep's odd
// substeps of MU = 1, 2 (spatial planes) and MU = 3 (space-time planes), each
// thread's sums ps and pt; at the end of the last of them every CTA writes
// its block sums to part[4 blockIdx.x + 0, 1].  The Polyakov loop (Eqs.
// 14-15) of the sweep's final links is taken during the first substep of
// the lattice's next sweep, which changes no time link (over-relaxation or
// heat bath of MU = 0): each CTA multiplies the time links of its spatial
// sites in increasing t and writes its sum of (1/2) Tr to
// part[4 blockIdx.x + 2].  After that substep's barrier the group's first
// CTA adds the CTAs' sums (warp 0, a fixed lane assignment and tree) into
// the history; a lattice's last sweep of the call takes its Polyakov loop
// after one more barrier.  Coherent loads throughout: other CTAs of the
// group write links during the launch.
template <int BS>
__device__ __forceinline__ void block_sums_to(double v0, double v1, double* out0, double* out1) {
  __shared__ double sh[BS / 32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  if (lane == 0) {
    sh[warp][0] = v0;
    sh[warp][1] = v1;
  }
  __syncthreads();
  if (warp == 0) {
    const double t0 = warp_sum(lane < BS / 32 ? sh[lane][0] : 0.0);
    const double t1 = warp_sum(lane < BS / 32 ? sh[lane][1] : 0.0);
    if (lane == 0) {
      *out0 = t0;
      if (out1) *out1 = t1;
    }
  }
  __syncthreads();
}

template <int P, int BS>
__device__ __forceinline__ void batch_polyakov_part(const Links<P, kClassOff>& L, const Geom& g, int rank, int cpg,
                                                    double* part) {
  using R = typename Real<P>::T;
  Acc<R> pl;
  const int nsig = g.n[0] * g.n[1] * g.n[2];
  const int nt = g.n[3];
  for (int xs = rank * BS + (int)threadIdx.x; xs < nsig; xs += cpg * BS) {
    const int p0 = parity(site_from_index(g, (uint32_t)xs));   // parity of (xs, t = 0)
    const uint32_t h0 = (uint32_t)xs >> 1, hstep = (uint32_t)nsig >> 1;
    Quat<R> pr = qone<R>();
    // nt is even: the loads of two slices are issued before their products
    for (int t = 0; t < nt; t += 2) {
      const Quat<R> a = L.ldc(6 + p0, h0 + hstep * t);
      const Quat<R> b = L.ldc(6 + (p0 ^ 1), h0 + hstep * (t + 1));
      pr = qmul(qmul(pr, a), b);
    }
    pl.add(pr.w);
  }
  block_sums_to<BS>(pl.value(), 0.0, part + 4 * (size_t)blockIdx.x + 2, nullptr);
}

// The history entry of one sweep from the group's CTA sums (warp 0 of the
// group's first CTA).
__device__ __forceinline__ void batch_history(const double* part, int cta0, int cpg, const Geom& g, double* o) {
  const int lane = threadIdx.x & 31;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int r = lane; r < cpg; r += 32) {
    const double* q = part + 4 * (size_t)(cta0 + r);
    a += __ldcg(q);
    b += __ldcg(q + 1);
    c += __ldcg(q + 2);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (lane == 0) {
    const double n3 = 3.0 * (double)(2 * g.vh);
    o[0] = (a + b) / (2.0 * n3);
    o[1] = a / n3;
    o[2] = b / n3;
    o[3] = c / (double)(g.n[0] * g.n[1] * g.n[2]);
  }
}

// 1024 threads per SM (64 registers a thread) for FP32 / F16Q, 512 for FP64.
// MEAS: measured sweeps (su2_batch_sweep_measure), a separate instantiation
// so that the plain sweep's kernel carries none of the measurement.  It runs
// the same number of CTAs per SM (so the same plan) with blocks of 3/4 BS
// threads, which leaves it 85 registers a thread instead of 64: at 64 its
// bookkeeping spilled registers out of the substep loops (16 x 32^3 x 4
// FP32, 100 sweeps without any measurement work: 32.9 against the plain
// kernel's 42.0 G updates/s).
template <int BS, bool MEAS> struct BatchBlock { static constexpr int value = MEAS ? BS * 3 / 4 : BS; };

template <int P, int BS, bool MEAS>
__global__ void __launch_bounds__(BatchBlock<BS, MEAS>::value, (P == kF64 ? 512 : 1024) / BS)
    k_batch_groups(const BatchLattice* __restrict__ desc, const int* __restrict__ order,
                   const int4* __restrict__ plan, const int* __restrict__ cta_group, int nsweeps, int nor,
                   const uint32_t* sweep_base, const __grid_constant__ HBParams hp, GroupBarrier* bars, BatchCtl* ctl,
                   unsigned long long timeout_ns, double* mhist, double* mpart, int nlat) {
  using R = typename Real<P>::T;
  constexpr int kB = BatchBlock<BS, MEAS>::value;  // threads per CTA
  // the deferral queue, sized for the larger (plaquette-carrying) entries
  __shared__ __align__(16) unsigned char queue[BatchQueue<kB>::value * sizeof(Deferred<R, MEAS>)];
  __shared__ int qn;
  PlainAcc<R> ps, pt;  // measured sweep: spatial and space-time plaquette sums
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
      case 0: batch_substep<P, 0, 0, kB, false>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn, ps); break;
      case 1: batch_substep<P, 0, 1, kB, false>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn, ps); break;
      case 2: batch_substep<P, 1, 0, kB, false>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn, ps); break;
      case 3: batch_substep<P, 1, 1, kB, MEAS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn, ps); break;
      case 4: batch_substep<P, 2, 0, kB, false>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn, ps); break;
      case 5: batch_substep<P, 2, 1, kB, MEAS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn, ps); break;
      case 6: batch_substep<P, 3, 0, kB, false>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn, pt); break;
      default: batch_substep<P, 3, 1, kB, MEAS>(L, g, rank, cpg, sweep, tag, beta, hp, queue, &qn, pt); break;
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
      case 0: batch_or_substep<P, 0, 0, kB>(L, g, rank, cpg); break;
      case 1: batch_or_substep<P, 0, 1, kB>(L, g, rank, cpg); break;
      case 2: batch_or_substep<P, 1, 0, kB>(L, g, rank, cpg); break;
      case 3: batch_or_substep<P, 1, 1, kB>(L, g, rank, cpg); break;
      case 4: batch_or_substep<P, 2, 0, kB>(L, g, rank, cpg); break;
      case 5: batch_or_substep<P, 2, 1, kB>(L, g, rank, cpg); break;
      case 6: batch_or_substep<P, 3, 0, kB>(L, g, rank, cpg); break;
      default: batch_or_substep<P, 3, 1, kB>(L, g, rank, cpg); break;
    }
  };
  // measured sweeps: after the first substep of sweep sw (sw >= 1), the
  // history entry of sweep sw - 1
  auto after_first = [&](int l, int sw) {
    if constexpr (MEAS) {
      if (sw > 0 && rank == 0 && threadIdx.x < 32)
        batch_history(mpart, pl.z, cpg, desc[l].g, mhist + ((size_t)(sw - 1) * nlat + l) * 4);
    }
  };
  auto polyakov_part = [&](int l) {
    const Geom g = desc[l].g;
    Links<P, kClassOff> L;
    L.set(desc[l].links, g.vh);
    batch_polyakov_part<P, kB>(L, g, rank, cpg, mpart);
  };
  for (int li = 0; li < pl.y; ++li) {
    const int l = order[pl.x + li];
    for (int sw = 0; sw < nsweeps; ++sw) {
      bool first = true;
      for (int k = 0; k < nor; ++k)
        for (int mu = 0; mu < 4; ++mu)
          for (int p = 0; p < 2; ++p) {
            or_substep(l, mu, p);
            if constexpr (MEAS) {
              if (first && sw > 0) polyakov_part(l);
            }
            if (!group_barrier(bars + group, (unsigned)cpg, ctl, timeout_ns)) return;
            if (first) after_first(l, sw);
            first = false;
          }
      for (int mu = 0; mu < 4; ++mu)
        for (int p = 0; p < 2; ++p) {
          substep(l, sweep0 + (uint32_t)sw, mu, p);
          if constexpr (MEAS) {
            if (first && sw > 0) polyakov_part(l);
            if (mu == 3 && p == 1) {
              // the sweep's plaquette sums of this CTA
              block_sums_to<kB>(ps.value(), pt.value(), mpart + 4 * (size_t)blockIdx.x,
                                mpart + 4 * (size_t)blockIdx.x + 1);
              ps = PlainAcc<R>();
              pt = PlainAcc<R>();
            }
          }
          if (!group_barrier(bars + group, (unsigned)cpg, ctl, timeout_ns)) return;
          if (first) after_first(l, sw);
          first = false;
        }
    }
    if constexpr (MEAS) {
      // the lattice's last sweep of this call
      if (nsweeps > 0) {
        polyakov_part(l);
        if (!group_barrier(bars + group, (unsigned)cpg, ctl, timeout_ns)) return;
        after_first(l, nsweeps);
        // the next lattice's first substep overwrites these CTA sums only
        // after a barrier that warp 0 of the first CTA reaches after reading them
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
  double* d_mpart;  // measured sweeps: four partial-sum slots per CTA
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
  int per_sm_meas = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_groups<P, BS, false>, BS, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_meas, k_batch_groups<P, BS, true>,
                                                BatchBlock<BS, true>::value, 0);
  if (per_sm_meas < per_sm) per_sm = per_sm_meas;
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
  // no group gets more CTAs than its largest lattice has links for at the
  // smallest block (192 threads: the measured kernel's 3/4 of 256), so that a
  // small lattice alone does not spread its barriers over idle CTAs; CTAs
  // left over have no group and leave at once
  for (int gi = 0; gi < G; ++gi) {
    int64_t mx = 1;
    for (int i : members[gi]) mx = std::max<int64_t>(mx, b->desc[i].g.vh);
    share[gi] = (int)std::min<int64_t>(share[gi], std::max<int64_t>(1, (mx + 191) / 192));
  }
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

cudaError_t launch_groups(const su2_batch* b, const BatchLattice* d_desc, int n, cudaStream_t st,
                          double* mhist = nullptr) {
  const HBParams hp = batch_hp(b);
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(mhist ? b->bs * 3 / 4 : b->bs);   // BatchBlock
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
                              (const int*)b->d_cta_group, n, b->nor, sw, hp, b->d_bars, b->d_ctl, b->timeout_ns,
                              mhist, b->d_mpart, b->n);
  };
  auto by_bs = [&](auto meas) {
    constexpr bool M = decltype(meas)::value;
    if (b->bs == 512)
      return b->prec == kF64 ? go(k_batch_groups<kF64, 512, M>)
                             : b->prec == kF32 ? go(k_batch_groups<kF32, 512, M>) : go(k_batch_groups<kF16Q, 512, M>);
    return b->prec == kF64 ? go(k_batch_groups<kF64, 256, M>)
                           : b->prec == kF32 ? go(k_batch_groups<kF32, 256, M>) : go(k_batch_groups<kF16Q, 256, M>);
  };
  e = mhist ? by_bs(std::true_type{}) : by_bs(std::false_type{});
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
  const size_t o_mpart = o; o = align256(o + 4 * (size_t)kMaxCtas * sizeof(double));
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
  b->d_mpart = (double*)(base + o_mpart);
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

extern "C" int su2_batch_sweep_measure(su2_batch* b, int n, double* hist) {
  clear_error();
  if (!b) return fail(SU2_EINVAL, "handle is NULL");
  if (n < 1) return fail(SU2_EINVAL, "n must be >= 1");
  if (!hist) return fail(SU2_EINVAL, "hist is NULL");
  if (b->sweep + (uint64_t)n >= 0xFFFFFFFFull) return fail(SU2_EINVAL, "sweep counter would reach the reserved index 2^32 - 1");
  DeviceGuard dg(b->device);
  const size_t bytes = (size_t)n * b->n * 4 * sizeof(double);
  double* d_hist = nullptr;
  SU2_CU(cudaMallocAsync(&d_hist, bytes, b->stream));
  const uint64_t before = b->sweep;
  cudaError_t e = launch_groups(b, b->d_desc, n, b->stream, d_hist);
  if (e == cudaSuccess) e = launch_add_u32(b->d_sweep, (uint32_t)n, b->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(d_hist, b->stream);
    cudaStreamSynchronize(b->stream);
    return fail(SU2_ECUDA, "batched measured sweep launch failed: %s", cudaGetErrorString(e));
  }
  b->sweep += (uint64_t)n;
  const int rc = check_ctl(b, before);
  if (rc == SU2_OK) e = cudaMemcpyAsync(hist, d_hist, bytes, cudaMemcpyDeviceToHost, b->stream);
  cudaFreeAsync(d_hist, b->stream);
  const cudaError_t e2 = cudaStreamSynchronize(b->stream);
  if (rc != SU2_OK) return rc;
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(SU2_ECUDA, "batched measured sweep: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  return SU2_OK;
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
