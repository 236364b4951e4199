// The two checkerboard substeps of one direction (MU, parity 0) and
// (MU, parity 1) fused into one launch, scheduled as a wavefront over time
// slices so that the slices the pair touches are re-read from L2 instead of
// HBM (Section 2 Eqs. 5-9, 11; Section 4 checkerboard order).
// Paper: Cardoso & Bicudo, arXiv:1010.4834.
//
// Traffic.  A substep reads the 3.5 V distinct links its V/2 staples need and
// writes V/2: 8 link transfers per update.  The pair reads the six classes of
// the other directions and the old parity-1 MU links once (3.5 V), and
// writes both MU classes (V): 4.5 transfers per update, if the parity-0 links
// written by the first half are still in L2 when the second half reads them
// and every slice is fetched from HBM only once.
//
// Dependencies.  Time slice t of a class holds the half-sites
// [t hs, (t + 1) hs) (hs = N0 N1 N2 / 2), since the half-index runs over the
// time coordinate slowest.  A parity-0 link at slice t reads parity-1 MU
// links at slices t - 1, t, t + 1 (through the time-direction staple) and no
// link written by the pair; a parity-1 link at slice t reads parity-0 MU
// links at slices t - 1 .. t + 1, which must be final.  So P1(t) may run once
// P0(t - 1), P0(t) and P0(t + 1) have finished (periodic in t), and P0(t)
// must run before P1(t +- 1) overwrites what it reads -- which the first
// rule already implies.  Work items are chunks of one slice of one phase;
// they are handed out by a ticket counter in wave order: wave w holds the
// chunks of P0(w) (w < Nt) and then those of the L-th previous P1 slice in
// the order 1, 2, ..., Nt - 1, 0, so that every item depends only on items
// with smaller tickets and P1 trails P0 by L waves (the working set is the
// ~L + 2 slices between them).  A block that draws a P1 chunk whose
// parity-0 neighbours are not finished yet waits for them -- after it has
// finished and published everything it took before, so the block holding
// the lowest outstanding ticket never waits and the pair cannot deadlock,
// whether or not all blocks are resident.  Every wait is bounded (1 s of
// global time and an iteration cap); one that runs out raises an error flag
// in the control block, and the block stops taking work.
//
// Consistency.  Parity-0 links are published by the finishing block with a
// fence and an atomic count per slice, and read by the parity-1 half with
// loads that bypass L1 (another SM's L1 may hold a line fetched before the
// write).  The other classes are not written by the pair and stay on the
// read-only path.  The deferral queue of rejected first trials (see
// su2_hb_link.cuh) is drained at the end of every chunk, so a chunk's links
// are final when it is published.
//
// The last block to leave resets the ticket, the slice counts and the exit
// count to zero for the next launch.
#include <type_traits>

#include "su2_hb_link.cuh"
#include "su2_internal.h"
#include "su2_kernel_util.cuh"

namespace su2 {

namespace {

#ifndef SU2_PAIR_THREADS
#define SU2_PAIR_THREADS 256
#endif
constexpr int kPairThreads = SU2_PAIR_THREADS;
constexpr int kPairBlocksPerSM = 1024 / kPairThreads;

__device__ __forceinline__ unsigned long long pair_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Work item of ticket t: phase (0: parity 0, 1: parity 1), slice, chunk.
struct Item {
  int phase, slice, chunk;
};

__device__ __forceinline__ Item decode(unsigned int t, const PairShape& s) {
  Item it;
  const unsigned int cps = (unsigned int)s.cps;
  const unsigned int a = (unsigned int)s.lag * cps;              // waves 0 .. L-1: P0 only
  const unsigned int b = a + 2u * (unsigned int)(s.nt - s.lag) * cps;  // waves L .. Nt-1: P0 then P1
  int wave, r;
  bool p1;
  if (t < a) {
    wave = (int)(t / cps);
    r = (int)(t - (unsigned int)wave * cps);
    p1 = false;
  } else if (t < b) {
    const unsigned int u = t - a;
    const unsigned int k = u / (2u * cps);
    wave = s.lag + (int)k;
    r = (int)(u - k * 2u * cps);
    p1 = r >= s.cps;
    if (p1) r -= s.cps;
  } else {
    const unsigned int u = t - b;
    const unsigned int k = u / cps;
    wave = s.nt + (int)k;
    r = (int)(u - k * cps);
    p1 = true;
  }
  it.chunk = r;
  if (!p1) {
    it.phase = 0;
    it.slice = wave;
  } else {
    it.phase = 1;
    const int j = wave - s.lag;            // P1 items in the order of slices 1, 2, ..., Nt-1, 0
    it.slice = j + 1 == s.nt ? 0 : j + 1;
  }
  return it;
}

// Called by thread 0 for each item the block is about to run: if it is a
// parity-1 chunk, wait until the parity-0 slices it reads are all finished
// (slices 0 .. need, cached in *prefix).  Returns false if the wait gave up
// or another block's did.
__device__ __forceinline__ bool wait_for_item(unsigned int t, unsigned int total, const PairShape& shp,
                                              PairCtl* ctl, const unsigned int* done0, int* prefix,
                                              unsigned long long timeout_ns) {
  if (t >= total) return true;
  const Item it = decode(t, shp);
  if (it.phase == 0) return true;
  const int need = (it.slice == 0 || it.slice == shp.nt - 1) ? shp.nt - 1 : it.slice + 1;
  int pre = *prefix;
  const unsigned long long t0 = pair_ns();
  unsigned long long spins = 0;
  bool ok = true;
  while (pre < need) {
    if (ld_acquire(done0 + pre + 1) == (unsigned int)shp.cps) {
      ++pre;
      continue;
    }
    if (ld_acquire(&ctl->err) != 0u) {
      ok = false;
      break;
    }
    if (pair_ns() - t0 > timeout_ns || ++spins > (1ull << 26)) {
      atomicExch(&ctl->err, 1u);
      ok = false;
      break;
    }
    __nanosleep(64);
  }
  // the acquire loads order this thread's later loads after the producers'
  // releases; the block's barrier after this call extends that to the block
  *prefix = pre;
  return ok;
}

}  // namespace

template <int P, int MU, bool MEAS>
__global__ void __launch_bounds__(kPairThreads, kPairBlocksPerSM)
    k_heatbath_pair(Links<P, kClassPtr> L, Geom g, const uint32_t* sweep_base, uint32_t sweep_off,
                    const __grid_constant__ HBParams hp, PairCtl* ctl, unsigned int* done0, PairShape shp,
                    unsigned long long timeout_ns, double* meas) {
  using R = typename Real<P>::T;
  constexpr int BS = kPairThreads;
  // queue capacity: a chunk's links up to two per thread (at the ~5% first-
  // trial rejection of beta ~ 2.5 far more than needed; a full queue
  // finishes links inline)
  constexpr int CAP = BS * (kPairLinksPerThread < 2 ? kPairLinksPerThread : 2);
  __shared__ Deferred<R, MEAS> queue[CAP];
  __shared__ int qn;
  __shared__ unsigned int s_item;
  __shared__ int s_stop;
  __shared__ int s_prefix;   // P0 slices 0 .. s_prefix all finished (seen by this block)
  const R beta = (R)hp.beta;
  const uint32_t sweep = (sweep_base ? *sweep_base : 0u) + sweep_off;
  const uint32_t tag = (uint32_t)MU | hp.lattice_tag;
  const unsigned int total = 2u * (unsigned int)shp.nt * (unsigned int)shp.cps;
  const int chunk_links = BS * kPairLinksPerThread;
  PlainAcc<R> plaq;
  HBCount cnt;
  unsigned int next = 0;
  if (threadIdx.x == 0) {
    qn = 0;
    int pre = -1;
    const unsigned int first = atomicAdd(&ctl->ticket, 1u);
    next = atomicAdd(&ctl->ticket, 1u);
    s_stop = wait_for_item(first, total, shp, ctl, done0, &pre, timeout_ns) ? 0 : 1;
    s_prefix = pre;
    s_item = first;
  }
  __syncthreads();
  for (;;) {
    const unsigned int t = s_item;
    if (t >= total || s_stop) break;
    const Item it = decode(t, shp);
    const int h0 = it.slice * shp.hs + it.chunk * chunk_links;
    const int h1 = min(h0 + chunk_links, (it.slice + 1) * shp.hs);
    if (it.phase == 0) {
#pragma unroll
      for (int k = 0; k < kPairLinksPerThread; ++k) {
        const int h = h0 + k * BS + (int)threadIdx.x;
        if (h < h1) hb_link<P, MU, false, 0, false, CAP>(L, g, h, tag, sweep, beta, hp,
                                                         reinterpret_cast<Deferred<R, false>*>(queue), &qn, plaq, cnt);
      }
      __syncthreads();
      hb_drain<P, MU, false, 0>(L, reinterpret_cast<Deferred<R, false>*>(queue), min(qn, CAP), tag, sweep, hp, plaq,
                                cnt);
    } else {
#pragma unroll
      for (int k = 0; k < kPairLinksPerThread; ++k) {
        const int h = h0 + k * BS + (int)threadIdx.x;
        if (h < h1) hb_link<P, MU, MEAS, 1, true, CAP>(L, g, h, tag, sweep, beta, hp, queue, &qn, plaq, cnt);
      }
      __syncthreads();
      hb_drain<P, MU, MEAS, 1>(L, queue, min(qn, CAP), tag, sweep, hp, plaq, cnt);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      qn = 0;
      // publish a finished parity-0 chunk
      if (it.phase == 0) {
        __threadfence();
        atomicAdd(done0 + it.slice, 1u);
      }
      // the next item; a parity-1 chunk waits for its parity-0 neighbours
      // (this block has published everything it took before)
      const unsigned int nt_item = next;
      if (nt_item < total) next = atomicAdd(&ctl->ticket, 1u);
      int pre = s_prefix;
      if (!wait_for_item(nt_item, total, shp, ctl, done0, &pre, timeout_ns)) s_stop = 1;
      s_prefix = pre;
      s_item = nt_item;
    }
    __syncthreads();
  }
  if (MEAS) {
    __shared__ double shs[BS / 32];
    const double v = warp_sum(plaq.value());
    if ((threadIdx.x & 31) == 0) shs[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int w = 0; w < BS / 32; ++w) a += shs[w];
      meas[blockIdx.x] = a;
    }
  }
  // the last block out resets the counters for the next launch
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ctl->exits, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    for (int i = threadIdx.x; i < shp.nt; i += blockDim.x) done0[i] = 0u;
    if (threadIdx.x == 0) {
      ctl->ticket = 0u;
      ctl->exits = 0u;
    }
  }
}

int pair_grid(int prec) {
  int per_sm = 0;
  if (prec == kF32) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heatbath_pair<kF32, 0, false>, kPairThreads, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heatbath_pair<kF16Q, 0, false>, kPairThreads, 0);
  }
  if (per_sm < 1) per_sm = 1;
  return per_sm * device_info().sms;
}

PairShape pair_shape(const Geom& g) {
  PairShape s;
  s.nt = g.n[3];
  s.hs = (int)(g.vh / g.n[3]);
  const int chunk_links = kPairThreads * kPairLinksPerThread;
  s.cps = (s.hs + chunk_links - 1) / chunk_links;
  s.lag = s.nt < kPairLag ? s.nt : kPairLag;
  return s;
}

template <int P, int MU>
static void pair_launch(const LatticeView& v, int grid, const uint32_t* sweep_base, uint32_t sweep_off,
                        const HBParams& hp, PairCtl* ctl, unsigned int* done0, const PairShape& shp, cudaStream_t st,
                        double* meas) {
  const unsigned long long timeout_ns = 1000000000ull;
  const auto L = links_of<P, kClassPtr>(v.links, v.g.vh);
  if constexpr (MU >= 1) {
    if (meas) {
      k_heatbath_pair<P, MU, true><<<grid, kPairThreads, 0, st>>>(L, v.g, sweep_base, sweep_off, hp, ctl, done0, shp,
                                                                   timeout_ns, meas);
      return;
    }
  }
  k_heatbath_pair<P, MU, false><<<grid, kPairThreads, 0, st>>>(L, v.g, sweep_base, sweep_off, hp, ctl, done0, shp,
                                                                timeout_ns, meas);
}

cudaError_t launch_heatbath_pair(const LatticeView& v, int mu, const uint32_t* sweep_base, uint32_t sweep_off,
                                 const HBParams& hp, PairCtl* ctl, unsigned int* done0, cudaStream_t st,
                                 double* meas, int* meas_blocks) {
  if (v.prec != kF32 && v.prec != kF16Q) return cudaErrorInvalidValue;
  if (meas && (mu < 1 || !meas_blocks)) return cudaErrorInvalidValue;
  const PairShape shp = pair_shape(v.g);
  const int grid = pair_grid(v.prec);
  if (meas) {
    if (grid > kMeasStride) return cudaErrorInvalidConfiguration;
    *meas_blocks = grid;
  }
  if (v.prec == kF32) {
    SU2_DISPATCH_MU(mu, pair_launch<kF32, MU>(v, grid, sweep_base, sweep_off, hp, ctl, done0, shp, st, meas));
  } else {
    SU2_DISPATCH_MU(mu, pair_launch<kF16Q, MU>(v, grid, sweep_base, sweep_off, hp, ctl, done0, shp, st, meas));
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace su2
