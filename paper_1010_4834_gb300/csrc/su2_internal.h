// Internal host-side interface between the C ABI (su2_capi.cu) and the kernel
// translation units.  Not installed; the public interface is include/su2.h.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "su2_device.cuh"

namespace su2 {

// Device-wide constants, queried once per device.
struct DeviceInfo {
  int sms;
  int l2_bytes;
};
const DeviceInfo& device_info();

// Geometry helper (host): fills a Geom for extents n[4].
Geom make_geom(const int n[4]);

// One lattice's device view: link store base pointer (precision-typed at the
// launch), geometry, and the heat-bath parameters.
struct LatticeView {
  void* links;      // 8 classes of vh links
  Geom g;
  int prec;
};

// Reduction scratch carved from the handle's device memory.
struct Scratch {
  double* partials;      // >= kScratchPartials doubles
  unsigned int* counter; // one zero-initialised ticket counter per reduction
  double* out;           // >= kScratchOut doubles, results of the last reduction
};
constexpr size_t kScratchPartials = (size_t)1 << 20;  // 8 MiB of doubles
constexpr size_t kScratchOut = 2048;
size_t scratch_bytes();

// --- launches (all stream-ordered, return cudaGetLastError()) ------------
cudaError_t launch_init(const LatticeView& v, int start, PhiloxKey key, uint32_t lattice_tag,
                        cudaStream_t st);
// With `meas` (only for mu >= 1, parity 1) the substep also writes one
// plaquette block sum per block to meas[0, *meas_blocks) (see k_heatbath).
cudaError_t launch_heatbath(const LatticeView& v, int mu, int parity, const uint32_t* sweep_base,
                            uint32_t sweep_off, const HBParams& hp, unsigned long long* stats,
                            cudaStream_t st, double* meas = nullptr, int* meas_blocks = nullptr);
// Block sums of the three measuring substeps sit at meas + k * kMeasStride
// (k = 0, 1, 2 for mu = 1, 2, 3; nb[k] blocks each).
constexpr int kMeasStride = 8192;
// Measured sweeps record {plaquette all, spatial, space-time, Polyakov} of
// sweep s in row s mod kHistRing of a device ring, so that a run of them is
// position-independent and replays as one CUDA graph.
constexpr int kHistRing = 1024;
// What the Polyakov kernel's last block does after a measured sweep: its
// mean and the plaquette from the sweep's block sums go to row
// (*sweep mod kHistRing) of hist, then *sweep is advanced by one.
struct SweepEpilogue {
  const double* meas;  // nullptr: no epilogue (the mean goes to out[0])
  int nb[3];
  double volume;
  double* hist;
  uint32_t* sweep;
};
// The fused parity pair of direction mu (su2_pair.cu), FP32 and F16Q.  Its
// control block and per-slice counts (nt of them) must be zero before the
// first launch; every launch leaves them zero again.  `meas` as for
// launch_heatbath (mu >= 1): the parity-1 half sums the plaquettes.
struct PairCtl {
  unsigned int ticket;  // next work item
  unsigned int exits;   // blocks that have left
  unsigned int err;     // 1: a dependency wait timed out
  unsigned int pad[29];
};
struct PairShape {
  int nt;   // time slices
  int hs;   // half-sites (links of one class) per slice
  int cps;  // work chunks per slice and phase
  int lag;  // waves by which the parity-1 half trails the parity-0 half
};
#ifndef SU2_PAIR_LPT
#define SU2_PAIR_LPT 1
#endif
#ifndef SU2_PAIR_LAG
#define SU2_PAIR_LAG 3
#endif
constexpr int kPairLinksPerThread = SU2_PAIR_LPT;  // links per thread in one work chunk
constexpr int kPairLag = SU2_PAIR_LAG;
PairShape pair_shape(const Geom& g);
int pair_grid(int prec);
cudaError_t launch_heatbath_pair(const LatticeView& v, int mu, const uint32_t* sweep_base, uint32_t sweep_off,
                                 const HBParams& hp, PairCtl* ctl, unsigned int* done0, cudaStream_t st,
                                 double* meas = nullptr, int* meas_blocks = nullptr);
cudaError_t launch_overrelax(const LatticeView& v, int mu, int parity, cudaStream_t st);
// The plaquette means of sites [s0, s0 + ns) (ns < 0: every site) to s.out[0..2].
cudaError_t launch_plaquette(const LatticeView& v, const Scratch& s, cudaStream_t st, int64_t s0 = 0,
                             int64_t ns = -1);
// Products of the time links of slices [t0, t0 + nt) of spatial sites
// [x0, x0 + nx), FP64, 4 doubles per spatial site.
cudaError_t launch_time_lines(const LatticeView& v, int t0, int nt, int64_t x0, int64_t nx, double* out,
                              cudaStream_t st);
// With `ep` the reduction partials must not overlap ep->meas.
cudaError_t launch_polyakov(const LatticeView& v, const Scratch& s, cudaStream_t st,
                            const SweepEpilogue* ep = nullptr);
// APE: src has (at least) the 6 spatial classes; dst receives them.
cudaError_t launch_ape(const LatticeView& src, void* dst, double alpha, cudaStream_t st);
cudaError_t launch_copy_spatial(const LatticeView& src, void* dst, cudaStream_t st);
// Wilson loops: spatial links from `spatial` (6 classes), time links from v.
cudaError_t launch_wilson(const LatticeView& v, const void* spatial, int rmax, int tmax,
                          const Scratch& s, cudaStream_t st);
// Canonical FP64 host layout <-> device store, for sites [s0, s0 + ns).
cudaError_t launch_to_canonical(const LatticeView& v, double* canon, int64_t s0, int64_t ns,
                                cudaStream_t st);
cudaError_t launch_from_canonical(const LatticeView& v, const double* canon, int64_t s0,
                                  int64_t ns, cudaStream_t st);
cudaError_t launch_add_u32(uint32_t* p, uint32_t v, cudaStream_t st);
// Layout comparison (FP32): the plain heat-bath substep on the store `links`
// in the library's layout or in the site-major single-array layout, the
// conversion between v.links and a site-major copy, and a count of differing
// 16-byte words of two buffers (added to *count).
cudaError_t launch_hb_plain(const LatticeView& v, void* links, bool site_major, int mu, int parity,
                            const uint32_t* sweep_base, uint32_t sweep_off, const HBParams& hp, cudaStream_t st);
cudaError_t launch_site_major(const LatticeView& v, void* site_major, bool to_site_major, cudaStream_t st);
cudaError_t launch_count_diff(const void* a, const void* b, size_t bytes, unsigned long long* count,
                              cudaStream_t st);

// Process-wide count of kernels this library launched (graph replays add
// their kernel-node count through count_launches).
void count_launches(uint64_t n);
uint64_t launches_total();
// While alive on a thread, launches made by that thread (stream capture) are
// not counted; the replays of the captured graph are.
struct CaptureScope {
  CaptureScope();
  ~CaptureScope();
};

}  // namespace su2
