// The checkerboard heat-bath substep for sm_103a (Section 2 Eqs. 5-9, 11;
// Section 4), with its optional plaquette sum for measured sweeps (the
// Polyakov kernel's last block turns those block sums into the plaquette).
// Paper: Cardoso & Bicudo, arXiv:1010.4834.
#include <type_traits>

#include "su2_hb_link.cuh"
#include "su2_internal.h"
#include "su2_kernel_util.cuh"

namespace su2 {

// ---------------------------------------------------------------------------
// Heat-bath substep (Section 2 Eqs. 5-9, 11; Section 4 checkerboard): one
// thread per link of direction MU on the parity-p sublattice.
//
// Most links accept their first a0 trial, but a warp would repeat the trial
// loop until its slowest lane accepts.  So every lane makes trial 1 inline;
// a link that rejects it goes to a block-wide shared-memory queue (its
// W = Sigma/k, alpha, index and site), which the whole block drains every
// DeferEvery iterations with trials 2, 3, ...  The draws and their order are
// those of the plain loop, so results are identical; only the schedule
// differs.  A full queue falls back to finishing the link inline.
//
// With MEAS (the odd-parity substeps of MU = 1, 2, 3 of a measured sweep) the
// kernel also adds up Tr(U_MU(x) L(x)^dagger)/2 over its links, with L the
// staple's partial sum over NU < MU and U the link's final value (the
// accepted draw as stored, or the kept old link), and writes one sum per
// block to `meas`.  Every plaquette of a plane (NU, MU), NU < MU, holds two
// MU-links on sites of opposite parity, so the odd-parity substep of MU counts
// each of them once; and once that substep has run, every link in directions
// <= MU has its end-of-sweep value.  The three substeps together give the
// plaquette of Eq. 12 after the sweep (planes (0,1), (0,2) and (1,2) the
// spatial part, (NU,3) the space-time part) without another pass over the
// links.
// ---------------------------------------------------------------------------
// Queue capacity: the plaquette-summing variant's entries are larger (they
// carry the partial staple), so it keeps fewer and leaves the SM's L1 share
// of the shared-memory carveout about the same.
// Block size BS: on large lattices blocks of 1024 share one deferral queue
// among more threads, which drain it less often per link (FP32 substep on
// 64^4, 55 k half-sites per SM: 202 us at 256 threads, 194 at 1024); up to
// 48^4 (17 k per SM) 256 is faster (70.9 against 72.2 us; 16^4 12.3
// against 14.0), as more, smaller blocks spread the few block iterations
// evenly over the SMs.  The switch is at SU2_HB_BIG_PER_SM half-lattice
// sites per SM.  FP64 needs 128 registers a thread, so never 1024; FP64
// lattices with fewer than two blocks of 256 per SM run blocks of 64 so
// that their few warps land on as many SMs as possible, since each SM's FP64
// pipe issues at 1/64 of the FP32 rate: on 8^4 (2048 links per substep)
// 256-thread blocks fill 8 SMs (measured sweep 344 us, 235 with blocks of
// 64).  FP32 gains nothing from it (32^3 x 4 plain sweep 32.4 -> 34.0 us).
#ifndef SU2_HB_BIG_PER_SM
#define SU2_HB_BIG_PER_SM 32768
#endif
#ifndef SU2_HB_LARGE_BS
#define SU2_HB_LARGE_BS 1024
#endif
template <int BS, bool MEAS> struct DeferCap { static constexpr int value = MEAS ? 2 * BS : 4 * BS; };
// Drain interval in block iterations: at the ~5% first-trial rejection of
// beta ~ 2.5 a queue collects about 0.05 * 1024 * interval links, which the
// capacity covers (the plaquette-summing variant's smaller queue, half as
// often); fewer drains mean fewer block-wide barriers.
template <bool MEAS> struct DeferEvery { static constexpr int value = MEAS ? 32 : 64; };

// Minimum resident blocks per SM (the register budget): 1024 threads per SM
// at 64 registers for FP32 / F16Q.
template <int P, int BS> struct HbMinBlocks {
  static constexpr int value = Occ<P>::hb * kThreads / BS > 0 ? Occ<P>::hb * kThreads / BS : 1;
};

// Programmatic dependent launch: a substep is launched with programmatic
// stream serialisation, so the launch of its grid overlaps the end of the
// previous kernel; each block first waits (griddepcontrol.wait, a hardware
// wait for the previous grid to complete and its writes to be visible) and
// reads nothing before.  No kernel triggers its dependents early (the
// implicit trigger at completion).  Sweep times, plain / measured, in us:
// 16^4 26.2 -> 25.2 / 37.9 -> 37.1, 32^3 x 4 31.0 -> 29.9 / 43.6 -> 42.6,
// 64^4 1417.6 -> 1415.3 / 1497.2 -> 1496.4.  An explicit trigger at the
// start of each block lost (64^4 sweep 1427 us, 48^4 measured sweep 512 ->
// 576 us): the next grid's blocks then hold SM slots while they wait.

template <int P, int MU, bool MEAS, int PAR, int BS>
__global__ void __launch_bounds__(BS, HbMinBlocks<P, BS>::value)
    k_heatbath(Links<P, kClassPtr> L, Geom g, const uint32_t* sweep_base, uint32_t sweep_off,
               const __grid_constant__ HBParams hp, unsigned long long* stats, double* meas) {
  constexpr int p = PAR;
  using R = typename Real<P>::T;
  using Def = Deferred<R, MEAS>;
  constexpr int kDeferCap = DeferCap<BS, MEAS>::value;
  constexpr int kHbThreads = BS;
  __shared__ Def queue[kDeferCap];
  __shared__ int qn;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const R beta = (R)hp.beta;
  const uint32_t sweep = (sweep_base ? *sweep_base : 0u) + sweep_off;
  const uint32_t tag = (uint32_t)MU | hp.lattice_tag;
  HBCount cnt;
  // MEAS: plaquettes of the planes (NU < MU, MU).  A plain sum: a thread adds
  // vh / (grid size) terms of magnitude <= 2 (about 55 on 64^4), so FP32
  // rounding stays near 1e-6 relative per thread before the FP64 block sums.
  PlainAcc<R> plaq;
  if (threadIdx.x == 0) qn = 0;
  __syncthreads();
  const int vh = (int)g.vh;
  const int stride = gridDim.x * blockDim.x;
  int it = 0;
  for (int base = blockIdx.x * blockDim.x; base < vh; base += stride, ++it) {
    const int h = base + threadIdx.x;
    if (h < vh) hb_link<P, MU, MEAS, p, false, kDeferCap>(L, g, h, tag, sweep, beta, hp, queue, &qn, plaq, cnt);
    if ((it % DeferEvery<MEAS>::value) == DeferEvery<MEAS>::value - 1 || base + stride >= vh) {
      __syncthreads();
      hb_drain<P, MU, MEAS, p>(L, queue, min(qn, kDeferCap), tag, sweep, hp, plaq, cnt);
      __syncthreads();
      if (threadIdx.x == 0) qn = 0;
      __syncthreads();
    }
  }
  if (MEAS) {
    __shared__ double shp[kHbThreads / 32];
    const double v = warp_sum(plaq.value());
    if ((threadIdx.x & 31) == 0) shp[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kHbThreads / 32; ++w) t += shp[w];
      meas[blockIdx.x] = t;
    }
  }
  if (stats) {
    __shared__ unsigned int sh[3];
    if (threadIdx.x < 3) sh[threadIdx.x] = 0;
    __syncthreads();
    if (cnt.trials) atomicAdd(&sh[0], cnt.trials);
    if (cnt.capped) atomicAdd(&sh[1], cnt.capped);
    if (cnt.haar) atomicAdd(&sh[2], cnt.haar);
    __syncthreads();
    if (threadIdx.x < 3 && sh[threadIdx.x]) atomicAdd(stats + threadIdx.x, (unsigned long long)sh[threadIdx.x]);
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_heatbath(const LatticeView& v, int mu, int parity, const uint32_t* sweep_base,
                            uint32_t sweep_off, const HBParams& hp, unsigned long long* stats,
                            cudaStream_t st, double* meas, int* meas_blocks) {
  if (meas && (mu < 1 || parity != 1 || !meas_blocks)) return cudaErrorInvalidValue;
  SU2_DISPATCH(v.prec, SU2_DISPATCH_MU(mu, {
    // direction and parity are template parameters, so every class index in
    // the kernel is a compile-time constant: per-class base pointers
    auto L = links_of<P, kClassPtr>(v.links, v.g.vh);
    const int64_t sms = device_info().sms;
    const int bs = P != kF64 ? (v.g.vh >= (int64_t)SU2_HB_BIG_PER_SM * sms ? SU2_HB_LARGE_BS : 256)
                             : (v.g.vh >= 2 * 256 * sms ? 256 : 64);
    auto launch = [&](auto kernel, int nthreads, double* m) -> cudaError_t {
      const int gr = grid_for(kernel, v.g.vh, 0, nthreads);
      if (m) {
        if (gr > kMeasStride) return cudaErrorInvalidConfiguration;
        *meas_blocks = gr;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)gr);
      cfg.blockDim = dim3((unsigned)nthreads);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, kernel, L, v.g, sweep_base, sweep_off, hp, stats, m);
    };
    // block sizes per precision: FP64 256 or 64, FP32 / F16Q 1024 or 256
    auto with_bs = [&](auto meas_c, auto par_c, double* m) -> cudaError_t {
      constexpr bool M = decltype(meas_c)::value;
      constexpr int PP = decltype(par_c)::value;
      constexpr int kSmall = P == kF64 ? 64 : 256, kLarge = P == kF64 ? 256 : SU2_HB_LARGE_BS;
      return bs == kLarge ? launch(k_heatbath<P, MU, M, PP, kLarge>, kLarge, m)
                          : launch(k_heatbath<P, MU, M, PP, kSmall>, kSmall, m);
    };
    cudaError_t e = cudaSuccess;
    if (meas) {
      if constexpr (MU >= 1) e = with_bs(std::true_type{}, std::integral_constant<int, 1>{}, meas);
    } else if (parity == 0) {
      e = with_bs(std::false_type{}, std::integral_constant<int, 0>{}, nullptr);
    } else {
      e = with_bs(std::false_type{}, std::integral_constant<int, 1>{}, nullptr);
    }
    if (e != cudaSuccess) return e;
  }));
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace su2
