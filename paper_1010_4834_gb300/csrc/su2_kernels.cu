// Kernels of the SU(2) heat-bath Monte Carlo for sm_103a, except the
// heat-bath substep itself (su2_heatbath.cu): start configurations, the
// over-relaxation substep, the fused plaquette / Polyakov reductions, APE
// smearing, Wilson loops and the canonical-layout conversions.  Paper: Cardoso & Bicudo,
// arXiv:1010.4834 (Sections 2 and 4).
//
// None of this work is a dense contraction (2x2 SU(2) products in
// registers), so everything runs on the FP32/FP64 pipes; the sweep is bound
// by HBM traffic and ALU issue.  Reductions are fused into the measurement
// kernels: per-thread sums (compensated when the arithmetic is FP32), FP64
// warp shuffles, one partial per block and a last-block finisher that adds
// the partials in a fixed order, so a result is reproducible run to run.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <mutex>
#include <type_traits>

#include "su2_hb_link.cuh"
#include "su2_internal.h"
#include "su2_kernel_util.cuh"

namespace su2 {

static std::atomic<uint64_t> g_launches{0};
static thread_local int g_capturing = 0;
void count_launches(uint64_t n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }
CaptureScope::CaptureScope() { ++g_capturing; }
CaptureScope::~CaptureScope() { --g_capturing; }

// ---------------------------------------------------------------------------
// Device info and launch shapes
// ---------------------------------------------------------------------------
const DeviceInfo& device_info() {
  // filled once per device; concurrent first calls from several host
  // threads wait on the device's once_flag
  static DeviceInfo info[64];
  static std::once_flag once[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::call_once(once[dev], [dev]() {
    cudaDeviceGetAttribute(&info[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&info[dev].l2_bytes, cudaDevAttrL2CacheSize, dev);
    if (info[dev].sms <= 0) info[dev].sms = 1;
  });
  return info[dev];
}

Geom make_geom(const int n[4]) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.n[i] = n[i];
  g.n0h = n[0] / 2;
  g.vh = (int64_t)n[0] * n[1] * n[2] * n[3] / 2;
  g.st[0] = 0;
  g.st[1] = 1;
  g.st[2] = n[1];
  g.st[3] = n[1] * n[2];
  for (int d = 0; d < 4; ++d) g.wr[d] = d ? g.st[d] * (n[d] - 1) : 0;
  for (int d = 0; d < 4; ++d) {
    g.hst[d] = d ? g.n0h * g.st[d] : 0;
    g.hwr[d] = d ? g.n0h * g.wr[d] : 0;
  }
  g.f_n0h = FastDiv((uint32_t)g.n0h);
  g.f_n1 = FastDiv((uint32_t)n[1]);
  g.f_n2 = FastDiv((uint32_t)n[2]);
  g.f_n0 = FastDiv((uint32_t)n[0]);
  g.site0 = 0;
  return g;
}

size_t scratch_bytes() {
  return kScratchPartials * sizeof(double) + 256 + kScratchOut * sizeof(double) + 256;
}

// ---------------------------------------------------------------------------
// Start configurations (Section 4 kernel list: cold start U = 1, hot start a
// random element of SU(2) on every link, read here as Haar via Philox draw 0 of sweep index
// 0xFFFFFFFF).  One thread per (site, direction).
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_init(Links<P> L, Geom g, int start,
                                                   const __grid_constant__ RoundKeys rk,
                                                   uint32_t lattice_tag) {
  using R = typename Real<P>::T;
  const int64_t V = 2 * g.vh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 4 * V; w += stride) {
    const int mu = (int)(w / V);
    const uint32_t s = (uint32_t)(w - (int64_t)mu * V);
    const Site x = site_from_index(g, s);
    Quat<R> q = qone<R>();
    if (start) q = haar_from<R>(philox(make_uint4(s + g.site0, (uint32_t)mu | lattice_tag, 0xFFFFFFFFu, 0u), rk));
    L.st(2 * mu + parity(x), hidx(g, x), q);
  }
}

// ---------------------------------------------------------------------------
// Over-relaxation substep (Section 2, Eq. 10): or_link (su2_hb_link.cuh) on
// every link of direction MU and parity PAR.
// ---------------------------------------------------------------------------
template <int P, int MU, int PAR>
__global__ void __launch_bounds__(kThreads, Occ<P>::hb) k_overrelax(Links<P, kClassPtr> L, Geom g) {
  const int stride = gridDim.x * blockDim.x;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.vh; h += stride) or_link<P, MU, PAR, true>(L, g, h);
}

// ---------------------------------------------------------------------------
// Plaquette (Section 2, Eqs. 12-13): per site the six (1/2) Re Tr
// U_mu(x) U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger = (A B^dagger)_0 with
// A = U_mu(x) U_nu(x+mu), B = U_nu(x) U_mu(x+nu): the dot product A.B.
// out[0] all, out[1] spatial, out[2] space-time means.
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ typename Real<P>::T plaq(const Links<P>& L, int q, const Quat<typename Real<P>::T>& umu,
                                                   const Quat<typename Real<P>::T>& unu, int mu, int nu,
                                                   int h_pmu, int h_pnu) {
  using R = typename Real<P>::T;
  const Quat<R> a = qmul(umu, L.ld(2 * nu + q, h_pmu));
  const Quat<R> b = qmul(unu, L.ld(2 * mu + q, h_pnu));
  return qdot(a, b);
}

// The sixteen links one site's six plaquettes use: its own four and, for each
// direction mu, the three U_nu(x + mu) with nu != mu.
template <int P> struct PlaqLinks { Quat<typename Real<P>::T> u[4], n[4][3]; };

template <int P>
__device__ __forceinline__ void plaq_load(const Links<P>& L, const Geom& g, int s, PlaqLinks<P>& k, int& p) {
  const Site x = site_from_index(g, (uint32_t)s);
  p = parity(x);
  const int q = p ^ 1;
  const int h = s >> 1;
  const int hm[4] = {hidx(g, shifted<0, +1>(g, x)), hidx(g, shifted<1, +1>(g, x)), hidx(g, shifted<2, +1>(g, x)),
                     hidx(g, shifted<3, +1>(g, x))};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) k.u[mu] = L.ld(2 * mu + p, h);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int nu = j < mu ? j : j + 1;
      k.n[mu][j] = L.ld(2 * nu + q, hm[mu]);
    }
  }
}

// U_nu(x + mu) among the loaded links.
template <int P>
__device__ __forceinline__ const Quat<typename Real<P>::T>& plaq_nb(const PlaqLinks<P>& k, int mu, int nu) {
  return k.n[mu][nu < mu ? nu : nu - 1];
}

template <int P>
__device__ __forceinline__ void plaq_sums(const PlaqLinks<P>& k, typename Real<P>::T& ss, typename Real<P>::T& ts) {
  using R = typename Real<P>::T;
  ss = R(0);
  ts = R(0);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int nu = mu + 1; nu < 4; ++nu) {
      const R v = qdot(qmul(k.u[mu], plaq_nb<P>(k, mu, nu)), qmul(k.u[nu], plaq_nb<P>(k, nu, mu)));
      if (nu == 3) ts += v; else ss += v;
    }
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_plaquette(Links<P> L, Geom g, int64_t s0, int64_t V,
                                                        double* partials, unsigned int* counter, double* out) {
  using R = typename Real<P>::T;
  Acc<R> sp, tm;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the plaquettes of the V sites from s0 on (all sites: s0 = 0, V = volume);
  // 64-bit loop index: V may come within one stride of 2^31
  for (int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < s0 + V; s += stride) {
    PlaqLinks<P> k0;
    int p0;
    plaq_load<P>(L, g, (int)s, k0, p0);
    R ss0, ts0;
    plaq_sums<P>(k0, ss0, ts0);
    sp.add(ss0);
    tm.add(ts0);
  }
  double v[2] = {sp.value(), tm.value()};
  if (block_partial<2>(v, partials, counter)) {
    double tot[2];
    final_sum<2>(partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      const double n3 = 3.0 * (double)V;
      out[0] = (tot[0] + tot[1]) / (2.0 * n3);
      out[1] = tot[0] / n3;
      out[2] = tot[1] / n3;
      *counter = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Polyakov loop (Section 2, Eqs. 14-15): per spatial site the product of the
// time links in increasing t; mean of (1/2) Tr over the spatial sites.  Site
// s = xs + Nsigma t has half-index (xs >> 1) + (Nsigma/2) t.
//
// A block takes kThreads / G consecutive time lines, and each line is split
// into G consecutive segments of nt / G >= 8 links (G a power of two <= 8
// dividing nt, as large as that allows).  Warp group q loads segment q of
// every line of the block in chunks of 8 (all loads of a chunk issued
// before the products; each load instruction of a warp reads 32 consecutive
// spatial sites at one t), and the segment products are multiplied in t
// order through shared memory.  With one line per thread the kernel kept
// one chunk in flight per thread at 120 registers and ran at under half the
// copy bandwidth (ncu, 64^4: 24% warps active, long-scoreboard stalls 11 per
// issue).  After a measured sweep the last block also finishes the sweep's
// plaquette, records both in the history ring and advances the sweep
// counter (SweepEpilogue), which saves two launches per sweep.
// ---------------------------------------------------------------------------
template <int P> struct PolyMinBlocks { static constexpr int value = 4; };
template <> struct PolyMinBlocks<kF64> { static constexpr int value = 2; };

template <int P>
__global__ void __launch_bounds__(kThreads, PolyMinBlocks<P>::value)
    k_polyakov(Links<P, kClassPtr> L, Geom g, int lg, double* partials, unsigned int* counter, double* out,
               SweepEpilogue ep) {
  using R = typename Real<P>::T;
  using LT = Links<P, kClassPtr>;
  constexpr int C = 8;
  __shared__ Quat<R> seg_prod[kThreads];
  Acc<R> acc;
  const int nsig = g.n[0] * g.n[1] * g.n[2];
  const uint32_t nsig_h = (uint32_t)(nsig / 2);
  const int G = 1 << lg;
  const int lines = kThreads >> lg;  // lines per block, a multiple of 32
  const int seg = g.n[3] >> lg;
  const int q = threadIdx.x / lines;
  const int l = threadIdx.x - q * lines;
  const int t0 = q * seg;
  for (int first = blockIdx.x * lines; first < nsig; first += gridDim.x * lines) {
    const int xs = first + l;
    Quat<R> pr = qone<R>();
    if (xs < nsig) {
      const Site x = site_from_index(g, (uint32_t)xs);
      const uint32_t hh = (uint32_t)(xs >> 1);
      // the time links of x alternate between the two parity classes: b0
      // holds those at t of the parity of t0, b1 the others
      const bool swap = (parity(x) ^ (t0 & 1)) != 0;
      const typename LT::E* b0 = swap ? L.cls_base(7) : L.cls_base(6);
      const typename LT::E* b1 = swap ? L.cls_base(6) : L.cls_base(7);
      const uint32_t e0 = hh + nsig_h * (uint32_t)t0;
      int t = 0;
      for (; t + C <= seg; t += C) {
        Quat<R> u[C];
#pragma unroll
        for (int j = 0; j < C; ++j) u[j] = LT::ldp((j & 1) ? b1 : b0, e0 + nsig_h * (uint32_t)(t + j));
#pragma unroll
        for (int j = 0; j < C; ++j) pr = qmul(pr, u[j]);
      }
      for (; t < seg; ++t) pr = qmul(pr, LT::ldp((t & 1) ? b1 : b0, e0 + nsig_h * (uint32_t)t));
    }
    if (G > 1) {
      seg_prod[threadIdx.x] = pr;
      __syncthreads();
      if (q == 0) {
        for (int k = 1; k < G; ++k) pr = qmul(pr, seg_prod[k * lines + l]);
      }
      __syncthreads();
    }
    if (q == 0 && xs < nsig) acc.add(pr.w);
  }
  double v[1] = {acc.value()};
  if (block_partial<1>(v, partials, counter)) {
    double tot[1];
    final_sum<1>(partials, gridDim.x, tot);
    // every thread reads the counter here; thread 0 advances it only after
    // the barriers inside plaquette_from_block_sums
    double* row = ep.meas ? ep.hist + 4 * (size_t)(*(volatile uint32_t*)ep.sweep % (uint32_t)kHistRing) : nullptr;
    if (threadIdx.x == 0) {
      (row ? row[3] : out[0]) = tot[0] / (double)nsig;
      *counter = 0;
    }
    if (ep.meas) {
      plaquette_from_block_sums(ep.meas, kMeasStride, ep.nb, ep.volume, row);
      if (threadIdx.x == 0) *ep.sweep += 1u;
    }
  }
}

// ---------------------------------------------------------------------------
// APE smearing step (Section 2, Eq. 19), Jacobi: spatial link (x, mu) ->
// P[(1-alpha) U + (alpha/4) (four spatial staples)], P = normalisation; a sum
// with vanishing norm keeps U.
//
// One thread per site updates all three spatial links.  For a pair mu < nu
// the two forward staple terms share one product: with
// A = U_nu(x+mu) U_mu(x+nu)^dag, link mu gets U_nu(x) A^dag and link nu gets
// U_mu(x) A.  Per site that is 27 link loads and 21 products instead of 39
// and 24 for three independent link updates, and one site decode instead of
// three.  Each link's staple terms are added nu ascending, forward then
// backward.  blockIdx.y = parity.
// ---------------------------------------------------------------------------
template <int P, int MU, int NU>
__device__ __forceinline__ void ape_pair(const Links<P, kClassPtr>& L, int h, int p, const int (&dp)[3], const int (&dm)[3],
                                         const Quat<typename Real<P>::T>& umu, const Quat<typename Real<P>::T>& unu,
                                         Quat<typename Real<P>::T>& smu, Quat<typename Real<P>::T>& snu) {
  using R = typename Real<P>::T;
  const int q = p ^ 1;
  const Quat<R> a = qmul_nd(L.ld(2 * NU + q, h + dp[MU]), L.ld(2 * MU + q, h + dp[NU]));
  const int hn = h + dm[NU], hm = h + dm[MU];  // x - nu, x - mu
  // link mu, term nu: forward U_nu(x) A^dag, backward U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
  qacc_mul_nd(smu, unu, a);
  qacc_mul(smu, qmul_dn(L.ld(2 * NU + q, hn), L.ld(2 * MU + q, hn)), L.ld(2 * NU + p, hn + dp[MU]));
  // link nu, term mu: forward U_mu(x) A, backward U_mu(x-mu)^dag U_nu(x-mu) U_mu(x-mu+nu)
  qacc_mul(snu, umu, a);
  qacc_mul(snu, qmul_dn(L.ld(2 * MU + q, hm), L.ld(2 * NU + q, hm)), L.ld(2 * MU + p, hm + dp[NU]));
}

template <int P>
__device__ __forceinline__ void ape_store(const Links<P, kClassPtr>& dst, int cls, int h, const Quat<typename Real<P>::T>& u,
                                          const Quat<typename Real<P>::T>& sig, typename Real<P>::T c0,
                                          typename Real<P>::T c1) {
  using R = typename Real<P>::T;
  const Quat<R> q = qmake<R>(c0 * u.w + c1 * sig.w, c0 * u.x + c1 * sig.x, c0 * u.y + c1 * sig.y,
                             c0 * u.z + c1 * sig.z);
  const R n2 = qdot(q, q);
  dst.st(cls, h, n2 >= Math<R>::kTiny ? qscale(q, Math<R>::rsqrt(n2)) : u);
}

#ifndef SU2_APE3_MINB
#define SU2_APE3_MINB 3
#endif
// The sites of parity PAR (a template parameter, so every class index is a
// compile-time constant for the per-class base pointers).
template <int P, int PAR>
__device__ __forceinline__ void ape_sites(const Links<P, kClassPtr>& src, const Links<P, kClassPtr>& dst, const Geom& g,
                                          typename Real<P>::T c0, typename Real<P>::T c1) {
  using R = typename Real<P>::T;
  constexpr int p = PAR;
  const int vh = (int)g.vh;
  const int stride = gridDim.x * blockDim.x;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < vh; h += stride) {
    const Site x = site_from_half(g, (uint32_t)h, p);
    // half-index steps to the six spatial neighbours; the index of x + a + b
    // is h + step(a) + step(b) for steps in different directions
    const int dp[3] = {half_step<0, +1>(g, x), half_step<1, +1>(g, x), half_step<2, +1>(g, x)};
    const int dm[3] = {half_step<0, -1>(g, x), half_step<1, -1>(g, x), half_step<2, -1>(g, x)};
    const Quat<R> u0 = src.ld(0 + p, h), u1 = src.ld(2 + p, h), u2 = src.ld(4 + p, h);
    Quat<R> s0 = qmake<R>(0, 0, 0, 0), s1 = s0, s2 = s0;
    ape_pair<P, 0, 1>(src, h, p, dp, dm, u0, u1, s0, s1);
    ape_pair<P, 0, 2>(src, h, p, dp, dm, u0, u2, s0, s2);
    ape_pair<P, 1, 2>(src, h, p, dp, dm, u1, u2, s1, s2);
    ape_store<P>(dst, 0 + p, h, u0, s0, c0, c1);
    ape_store<P>(dst, 2 + p, h, u1, s1, c0, c1);
    ape_store<P>(dst, 4 + p, h, u2, s2, c0, c1);
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads, P == kF64 ? 2 : SU2_APE3_MINB)
    k_ape(Links<P, kClassPtr> src, Links<P, kClassPtr> dst, Geom g, double alpha_d) {
  using R = typename Real<P>::T;
  const R alpha = (R)alpha_d;
  const R c0 = R(1) - alpha, c1 = R(0.25) * alpha;
  if (blockIdx.y == 0) ape_sites<P, 0>(src, dst, g, c0, c1);
  else ape_sites<P, 1>(src, dst, g, c0, c1);
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_copy_spatial(Links<P> src, Links<P> dst) {
  const int64_t n = 6 * src.vh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int cls = (int)(i / src.vh);
    const int j = (int)(i - cls * src.vh);
    dst.st(cls, j, src.ld(cls, j));
  }
}

// ---------------------------------------------------------------------------
// Wilson loops (Section 2, Eq. 18), (1/2) Tr[S_R(x) T_T(x+R mu) S_R(x+T t)^dag
// T_T(x)^dag] = (A B) . (D C) with A = S_R(x), B = T_T(x+R mu), C = S_R(x+T t),
// D = T_T(x).  A thread owns one (site, spatial MU) and a chunk of TC values
// of T; it walks R = 1..rmax extending A and the TC lines C by one link each,
// rebuilds the time line B at x + R mu, and adds the TC loop values into the
// block's shared accumulators (one transposing warp reduction per R).
// blockIdx.y = 3 chunk + mu.  Per-block sums go to `partials`; a second
// kernel adds them per (R, T) in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kWilsonMaxR = 32;
constexpr int kWilsonThreads = 128;

// Walker along the time direction in half-site index space: one step adds
// the half-index stride of a time slice (wrapping at the last slice) and
// flips the parity.
struct TWalk {
  int h, par, x3;
  __device__ __forceinline__ void init(const Geom& g, const Site& y) {
    h = hidx(g, y);
    par = parity(y);
    x3 = y.x3;
  }
  __device__ __forceinline__ void step(int nt, int hts, int hwrap) {
    if (x3 + 1 == nt) { x3 = 0; h -= hwrap; } else { ++x3; h += hts; }
    par ^= 1;
  }
};

template <int P, int TC, int MU>
__device__ __forceinline__ void wilson_site(const Links<P>& Ls, const Links<P>& Lt, const Geom& g, int s,
                                            bool valid, int rmax, int t0, int nT, double* acc) {
  using R = typename Real<P>::T;
  static_assert(TC == 4 || TC == 8 || TC == 16, "T chunk must be 4, 8 or 16");
  const int lane = threadIdx.x & 31;
  const int nt = g.n[3];
  const int hts = g.n0h * g.st[3];
  const int hwrap = hts * (nt - 1);
  const Site x = site_from_index(g, (uint32_t)s);
  Quat<R> D[TC], C[TC];
  {
    TWalk w;
    w.init(g, x);
    Quat<R> pr = qone<R>();
    for (int t = 0; t < t0; ++t) { pr = qmul(pr, Lt.ld(6 + w.par, w.h)); w.step(nt, hts, hwrap); }
#pragma unroll
    for (int j = 0; j < TC; ++j) {
      if (j < nT) { pr = qmul(pr, Lt.ld(6 + w.par, w.h)); w.step(nt, hts, hwrap); }
      D[j] = pr;
      C[j] = qone<R>();
    }
  }
  Quat<R> A = qone<R>();
  Site xr = x;  // x + (r-1) mu at the top of iteration r
  Site zt = x;  // x + (r-1) mu + (t0 + 1) t
  for (int t = 0; t <= t0; ++t) zt = shifted<3, +1>(g, zt);
  for (int r = 1; r <= rmax; ++r) {
    A = qmul(A, Ls.ld(2 * MU + parity(xr), hidx(g, xr)));
    {
      TWalk z;
      z.init(g, zt);
#pragma unroll
      for (int j = 0; j < TC; ++j) {
        if (j < nT) { C[j] = qmul(C[j], Ls.ld(2 * MU + z.par, z.h)); z.step(nt, hts, hwrap); }
      }
    }
    xr = shifted<MU, +1>(g, xr);
    zt = shifted<MU, +1>(g, zt);
    TWalk w;
    w.init(g, xr);
    Quat<R> b = qone<R>();
    for (int t = 0; t < t0; ++t) { b = qmul(b, Lt.ld(6 + w.par, w.h)); w.step(nt, hts, hwrap); }
    R val[TC];
#pragma unroll
    for (int j = 0; j < TC; ++j) {
      val[j] = R(0);
      if (j < nT) {
        b = qmul(b, Lt.ld(6 + w.par, w.h));
        w.step(nt, hts, hwrap);
        if (valid) val[j] = qdot(qmul(A, b), qmul(D[j], C[j]));
      }
    }
    // Sum the TC values over the warp by a transposing butterfly: each of the
    // first log2(TC) stages trades half of a lane's values with its partner,
    // halving the count; the remaining stages finish the sum.  Afterwards the
    // lanes of each group of 32/TC hold the total of one value j = lo.
    int nv = TC;
    int lo = 0;  // this lane's values are j = lo .. lo + nv - 1
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      if (nv > 1) {
        const bool upper = (lane & off) != 0;
        const int half = nv / 2;
#pragma unroll
        for (int k = 0; k < TC / 2; ++k) {
          if (k < half) {
            const R send = upper ? val[k] : val[k + half];
            const R keep = upper ? val[k + half] : val[k];
            val[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
          }
        }
        if (upper) lo += half;
        nv = half;
      } else {
        val[0] += __shfl_xor_sync(0xffffffffu, val[0], off);
      }
    }
    if ((lane & (32 / TC - 1)) == 0 && lo < nT) atomicAdd(&acc[(r - 1) * TC + lo], (double)val[0]);
  }
}

template <int P, int TC>
__global__ void __launch_bounds__(kWilsonThreads) k_wilson(Links<P> Ls, Links<P> Lt, Geom g, int rmax,
                                                           int tmax, double* partials) {
  __shared__ double acc[kWilsonMaxR * TC];
  const int mu = blockIdx.y % 3;
  const int chunk = blockIdx.y / 3;
  const int t0 = chunk * TC;
  const int nT = min(TC, tmax - t0);
  for (int i = threadIdx.x; i < kWilsonMaxR * TC; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const int64_t V = 2 * g.vh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += stride) {
    const int64_t s = base + threadIdx.x;
    const bool valid = s < V;
    const int sv = valid ? (int)s : 0;
    if (mu == 0) wilson_site<P, TC, 0>(Ls, Lt, g, sv, valid, rmax, t0, nT, acc);
    else if (mu == 1) wilson_site<P, TC, 1>(Ls, Lt, g, sv, valid, rmax, t0, nT, acc);
    else wilson_site<P, TC, 2>(Ls, Lt, g, sv, valid, rmax, t0, nT, acc);
  }
  __syncthreads();
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  const int per = rmax * TC;
  for (int i = threadIdx.x; i < per; i += blockDim.x) partials[(size_t)bid * per + i] = acc[i];
}

// ---------------------------------------------------------------------------
// Wilson loops, time-outer form.  In the (MU, time) plane with coordinates
// (a, t), S_R(a, t) = U_MU(a, t) ... U_MU(a+R-1, t) and T_T(a, t) = U_t(a, t)
// ... U_t(a, t+T-1), the loop of Eq. 18 at (a, t) is
//   W = (1/2) Tr[S_R(a,t) T_T(a+R,t) S_R(a,t+T)^dag T_T(a,t)^dag]
//     = (F . Q),  F = S_R(a,t) T_T(a+R,t),  Q = T_T(a,t) S_R(a,t+T).
// A thread owns one site of a plane (or of a band of its time slices, when
// the whole plane does not fit) staged in shared memory and holds F for RC
// consecutive R in registers.  Stepping T by one multiplies each F by one
// time link and D = T_T(a,t) by one; Q is then rebuilt along R from D with
// one spatial link per R.  That is two quaternion products and a dot product
// per (R, T), where extending every line per (R, T) costs four to five.
// blockIdx.y = (R chunk, T chunk); chunks after the first start from prefix
// products.  Plane rows are stored with `pad` extra columns repeating the
// first ones, so the lines along MU need no periodic wrap test.  Loop values
// go through a transposing warp reduction into per-warp sums of the work
// unit (FP32 or FP64, the arithmetic's precision), which are folded into the
// block's FP64 totals after each unit in a fixed order (no atomics); per-block sums go to `partials` in a fixed layout
// for k_wilson_rt_final.
// ---------------------------------------------------------------------------
constexpr int kWrtT = 16;  // T values per chunk
// The T loop unrolled by two: W(16,16) on 64^4 FP32 21.8 -> 20.4 ms (the
// sixteen F quaternions stay in place across iterations instead of being
// moved back at the loop edge); by four 21.7 ms.
#ifndef SU2_WILSON_TUNROLL
#define SU2_WILSON_TUNROLL 2
#endif
constexpr int kWilsonTUnroll = SU2_WILSON_TUNROLL;


template <int P, int RC, int NTH>
__global__ void __launch_bounds__(NTH, 1) k_wilson_rt(Links<P> Ls, Links<P> Lt, Geom g, int rmax, int tmax,
                                                      int ntc, int pad, int tile, double* partials) {
  using R = typename Real<P>::T;
  static_assert(RC == 8 || RC == 16, "R chunk must be 8 or 16");
  constexpr int NS = RC * kWrtT;  // (R, T) slots of one chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double acc[NS];               // block totals; slot k belongs to thread k
  __shared__ R wacc[NTH / 32][NS];         // one work unit's sums per warp (in the arithmetic's precision)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rc = blockIdx.y / ntc, tc = blockIdx.y - (blockIdx.y / ntc) * ntc;
  const int r0 = rc * RC, t0 = tc * kWrtT;
  const int nR = min(RC, rmax - r0), nT = min(kWrtT, tmax - t0);
  const int nt = g.n[3];
  // a work unit is `tile` consecutive time slices of one plane.  A whole
  // plane (tile == nt) is staged once, rows read modulo nt; a band of slices
  // stages rows tstart .. tstart + nrows - 1 (mod nt), enough for every line
  // its sites start (T up to ntc * kWrtT beyond the last slice), and reads
  // them without a wrap
  const bool whole = tile >= nt;
  const int ntiles = whole ? 1 : (nt + tile - 1) / tile;
  const int nrows = whole ? nt : tile + ntc * kWrtT;
  const int wrap_at = whole ? nt : 0x7fffffff;
  for (int i = threadIdx.x; i < NS; i += NTH) acc[i] = 0.0;
  for (int i = threadIdx.x; i < (NTH / 32) * NS; i += NTH) (&wacc[0][0])[i] = R(0);
  const int ntr0 = g.n[1] * g.n[2], ntr1 = g.n[0] * g.n[2], ntr2 = g.n[0] * g.n[1];
  const int nunits = (ntr0 + ntr1 + ntr2) * ntiles;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int pl = u / ntiles, tstart = (u - pl * ntiles) * tile;
    const int mu = pl < ntr0 ? 0 : (pl < ntr0 + ntr1 ? 1 : 2);
    const int tr = pl - (mu == 0 ? 0 : (mu == 1 ? ntr0 : ntr0 + ntr1));
    const int nm = mu == 0 ? g.n[0] : (mu == 1 ? g.n[1] : g.n[2]);
    const int tn = min(tile, nt - tstart);  // slices whose sites this unit owns
    const int np = nm * tn;
    // rows of W = nm + pad columns: column c holds plane column c mod nm, so
    // every line a, a+1, ..., a + pad - 1 is read without a wrap test; row r
    // holds time slice tstart + r (mod nt), so lines along t need none either
    const int W = nm + pad;
    Quat<R>* us = reinterpret_cast<Quat<R>*>(smem_raw);   // us[c + W r] = U_mu(c mod nm, tstart + r)
    Quat<R>* ut = us + W * nrows;                         // ut[c + W r] = U_t(c mod nm, tstart + r)
    const int n1st = mu == 0 ? g.n[1] : g.n[0];
    const int c1 = tr % n1st, c2 = tr / n1st;
    __syncthreads();  // the previous unit's readers and the warp-sum fold are done
    for (int i = threadIdx.x; i < W * nrows; i += NTH) {
      const int c = i % W, r = i / W;
      const int a = c % nm;
      Site y;
      y.x0 = mu == 0 ? a : c1;
      y.x1 = mu == 0 ? c1 : (mu == 1 ? a : c2);
      y.x2 = mu == 2 ? a : c2;
      y.x3 = (tstart + r) % nt;
      y.row = y.x1 + g.n[1] * (y.x2 + g.n[2] * y.x3);
      const int h = hidx(g, y), par = parity(y);
      us[i] = Ls.ld(2 * mu + par, h);
      ut[i] = Lt.ld(6 + par, h);
    }
    __syncthreads();
    for (int base = 0; base < np; base += NTH) {
      const int i = base + threadIdx.x;
      const bool valid = i < np;
      const int a = valid ? i % nm : 0, t = valid ? i / nm : 0;   // t: local row of the site
      // F[k] = S_{r0+k+1}(a, t) T_{t0}(a+r0+k+1, t),  D = T_{t0}(a, t)
      Quat<R> F[RC];
      {
        const Quat<R>* row = us + a + W * t;
        Quat<R> sp = qone<R>();
        for (int k = 0; k < r0; ++k) sp = qmul(sp, row[k]);
#pragma unroll
        for (int k = 0; k < RC; ++k) {
          sp = qmul(sp, row[r0 + k]);
          F[k] = sp;
        }
      }
      Quat<R> D = qone<R>();
      int tt = t;                                   // row of t + T - 1 for the next T
      for (int j = 0; j < t0; ++j) {
        D = qmul(D, ut[a + W * tt]);
        const Quat<R>* row = ut + a + r0 + 1 + W * tt;
#pragma unroll
        for (int k = 0; k < RC; ++k) F[k] = qmul(F[k], row[k]);
        tt = tt + 1 == wrap_at ? 0 : tt + 1;
      }
#pragma unroll kWilsonTUnroll
      for (int j = 0; j < nT; ++j) {             // T = t0 + j + 1
        D = qmul(D, ut[a + W * tt]);
        {
          const Quat<R>* row = ut + a + r0 + 1 + W * tt;
#pragma unroll
          for (int k = 0; k < RC; ++k) F[k] = qmul(F[k], row[k]);
        }
        tt = tt + 1 == wrap_at ? 0 : tt + 1;     // row of t + T
        const Quat<R>* row = us + a + W * tt;
        Quat<R> Q = D;
        for (int k = 0; k < r0; ++k) Q = qmul(Q, row[k]);
        R val[RC];
#pragma unroll
        for (int k = 0; k < RC; ++k) {
          Q = qmul(Q, row[r0 + k]);
          val[k] = (valid && k < nR) ? qdot(F[k], Q) : R(0);
        }
        int nv = RC, lo = 0;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
          if (nv > 1) {
            const bool upper = (lane & off) != 0;
            const int half = nv / 2;
#pragma unroll
            for (int k = 0; k < RC / 2; ++k) {
              if (k < half) {
                const R send = upper ? val[k] : val[k + half];
                const R keep = upper ? val[k + half] : val[k];
                val[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
              }
            }
            if (upper) lo += half;
            nv = half;
          } else {
            val[0] += __shfl_xor_sync(0xffffffffu, val[0], off);
          }
        }
        // owner lanes hold distinct R slots: plain read-modify-write
        if ((lane & (32 / RC - 1)) == 0 && lo < nR) wacc[warp][lo * kWrtT + j] += val[0];
      }
    }
    __syncthreads();
    // fold the warps' sums into the block totals in a fixed order
    for (int k = threadIdx.x; k < NS; k += NTH) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < NTH / 32; ++w) {
        t += (double)wacc[w][k];
        wacc[w][k] = R(0);
      }
      acc[k] += t;
    }
  }
  __syncthreads();
  const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  for (int i = threadIdx.x; i < NS; i += NTH) partials[bid * NS + i] = acc[i];
}

// out[(R-1) tmax + (T-1)] from k_wilson_rt's per-block sums: one block per
// output adds the gx blocks of its (R chunk, T chunk) in a fixed order.
template <int RC>
__global__ void __launch_bounds__(kThreads) k_wilson_rt_final(const double* partials, int gx, int ntc, int tmax,
                                                              double inv, double* out) {
  const int o = blockIdx.x;
  const int r = o / tmax, t = o % tmax;
  const int y = (r / RC) * ntc + t / kWrtT;
  const int slot = (r % RC) * kWrtT + t % kWrtT;
  double a = 0.0;
  for (int bx = threadIdx.x; bx < gx; bx += blockDim.x) a += __ldcg(partials + ((size_t)y * gx + bx) * (RC * kWrtT) + slot);
  const double tot = block_sum(a);
  if (threadIdx.x == 0) out[o] = tot * inv;
}

// ---------------------------------------------------------------------------
// Wilson loops in temporal gauge.  The loop of Eq. 18 is gauge invariant, so
// it may be evaluated on any gauge transform U'_mu(x) = G(x) U_mu(x)
// G(x+mu)^dag of the links.  In the (MU, time) plane with coordinates (a, t)
// take G(a, 0) = 1 and G(a, t+1) = G(a, t) U_t(a, t) (each product
// normalised, so G stays a unit quaternion): every time line then becomes
// T_T(a, t) = G(a,t)^dag G(a,t+T), and the loop at (a, t) becomes
//   W = (1/2) Tr[S'_R(a,t) S'_R(a,t+T)^dag] = S'_R(a,t) . S'_R(a,t+T),
// with S'_R(a, r) = U'(a, r) U'(a+1, r) ... U'(a+R-1, r) the spatial line of
// the transformed links (the G between neighbouring links cancel).  A time
// line that wraps past the last slice is G(a,t)^dag P(a) G(a,t') with P(a) =
// G(a, Nt) the Polyakov line, so rows Nt + t' of an extended plane hold
// U'(a, Nt + t') = P(a) U'(a, t') P(a+1)^dag and no loop needs a wrap test.
// Per loop that is one dot product (4 FMA) where the direct form needs two
// quaternion products and a dot (36 FMA); the lines cost one product per
// (site, R), shared by all T.
//
// One block per plane at a time.  A warp owns four columns a; lane (k, c),
// k = lane % 4, c = lane / 4, owns of column 4 warp + k the RO = Nt / 8 rows
// c RO .. (c+1) RO - 1 (the rows its loops start from) and the extended
// rows Nt + 2c, Nt + 2c + 1, so every lane starts loops from RO rows and
// every row it reads beyond its own belongs to its warp: the R loop needs no
// block barrier and no lane branches off.  The time links are scanned in
// the same chunks of RO slices (products within a chunk, then a prefix over
// the chunks) and the transformed spatial links U' of the extended plane are
// staged in shared memory; then for R = 1 .. rmax every thread extends its
// RO + 2 lines by one link, publishes them, and adds the dot products with
// the lines 1 .. kTgT rows ahead into sixteen register accumulators (one per
// T), which a transposing warp reduction leaves in a per-(R, warp) slot; the
// block folds the slots into its FP64 totals in a fixed order after the
// plane.  Row strides are 2 mod 4 quaternions and the origin rows of every
// other chunk are shifted (tg_stride, tg_skew_unit), so the 16-byte shared
// accesses of eight lanes (two chunks of four columns) hit distinct banks.
// Per-block sums go to `partials` in the layout k_wilson_rt_final reads (one
// 16 x 16 chunk).
// ---------------------------------------------------------------------------
#ifndef SU2_WILSON_TG
#define SU2_WILSON_TG 1
#endif
constexpr int kTgT = 16;                 // T values in registers; also the rows added past Nt
constexpr int kTgChunks = 8;             // row chunks of a column (lanes per column)
constexpr int kTgCols = 32 / kTgChunks;  // columns of a warp
constexpr int kTgExt = kTgT / kTgChunks; // extended rows a lane owns
// block size limit (the register budget): planes of up to 64 columns in
// FP32 / F16Q, 32 in FP64
template <int P> struct TgThreads { static constexpr int value = P == kF64 ? 256 : 512; };

template <class R> __device__ __forceinline__ Quat<R> qunit(const Quat<R>& q) {
  return qscale(q, Math<R>::rsqrt(qdot(q, q)));
}

// Site (column a, slice t) of the plane (mu, c1, c2).
__device__ __forceinline__ Site plane_site(const Geom& g, int mu, int a, int c1, int c2, int t) {
  Site y;
  y.x0 = mu == 0 ? a : c1;
  y.x1 = mu == 0 ? c1 : (mu == 1 ? a : c2);
  y.x2 = mu == 2 ? a : c2;
  y.x3 = t;
  y.row = y.x1 + g.n[1] * (y.x2 + g.n[2] * y.x3);
  return y;
}

// Row layout of a staged plane, chunks of RO rows.  Eight lanes of a 16-byte
// shared access are two chunks of four columns, so rows c RO + i and
// (c+1) RO + i must start 4 mod 8 quaternions apart (16 banks), and so must
// the extended rows Nt + 2c + e and Nt + 2c + 2 + e.  The latter needs a
// row stride S = 2 mod 4; the former then holds for RO = 2 mod 4 and, with
// the origin rows of odd chunks shifted by tg_skew_unit quaternions, for RO
// = 0 mod 4 (shift 4) and RO odd (S = 2 mod 8, shift 2).  S leaves room for
// the shift after the last column.
template <int RO> __host__ __device__ constexpr int tg_skew_unit() { return RO % 4 == 0 ? 4 : (RO % 2 ? 2 : 0); }
template <int RO> __host__ __device__ __forceinline__ int tg_stride(int cols) {
  const int m = RO % 2 ? 8 : 4;
  const int lo = cols + tg_skew_unit<RO>();
  return lo + ((2 - lo % m) + m) % m;
}
template <int RO> __device__ __forceinline__ int tg_row(int r, int nt, int stride) {
  return r * stride + (r < nt ? tg_skew_unit<RO>() * ((r / RO) & 1) : 0);
}

template <int P, int RO>
__global__ void __launch_bounds__(TgThreads<P>::value, 1)
    k_wilson_tg(Links<P> Ls, Links<P> Lt, Geom g, int rmax, int tmax, double* partials) {
  using R = typename Real<P>::T;
  constexpr int NTH = TgThreads<P>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double acc64[16 * kTgT];              // block totals; slot (R-1) kTgT + T-1
  __shared__ R wsum[16][NTH / 32][kTgT];           // per R and warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nt = g.n[3], nr = nt + kTgT;           // nt = kTgChunks RO
  const int hts = g.n0h * g.st[3];
  for (int i = threadIdx.x; i < 16 * kTgT; i += blockDim.x) acc64[i] = 0.0;
  const int ntr0 = g.n[1] * g.n[2], ntr1 = g.n[0] * g.n[2], ntr2 = g.n[0] * g.n[1];
  const int nunits = ntr0 + ntr1 + ntr2;
  const int c = lane / kTgCols, r0 = c * RO;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int mu = u < ntr0 ? 0 : (u < ntr0 + ntr1 ? 1 : 2);
    const int tr = u - (mu == 0 ? 0 : (mu == 1 ? ntr0 : ntr0 + ntr1));
    const int nm = mu == 0 ? g.n[0] : (mu == 1 ? g.n[1] : g.n[2]);
    const int n1st = mu == 0 ? g.n[1] : g.n[0];
    const int c1 = tr % n1st, c2 = tr / n1st;
    const int W = nm + rmax - 1;       // columns of the staged plane (column cc is plane column cc mod nm)
    const int SU = tg_stride<RO>(W), SS = tg_stride<RO>(nm);
    Quat<R>* Ue = reinterpret_cast<Quat<R>*>(smem_raw);  // Ue[tg_row(r, SU) + cc] = U'(cc, r), r < nr
    Quat<R>* Sb = Ue + nr * SU + 4;                      // Sb[tg_row(r, SS) + a]: G(a, r), then S'_R(a, r)
    Quat<R>* Ct = Sb + nr * SS + 4;                      // Ct[k nm + a]: product of scan chunk k
    Quat<R>* Pb = Ct + kTgChunks * nm;                   // Pb[a] = P(a)
    const int a = kTgCols * warp + lane % kTgCols;
    const bool active = a < nm;
    __syncthreads();  // the previous plane's readers are done
    // (1) this lane's links, loaded together: the time and spatial links of
    // its origin rows (one site each) and the spatial links of the slices
    // 2c, 2c + 1 that its extended rows repeat; then the time links'
    // products within the chunk
    Quat<R> us[RO + kTgExt];
    if (active) {
      Quat<R> ut[RO];
      const Site y = plane_site(g, mu, a, c1, c2, r0);
      int h = hidx(g, y), par = parity(y);
#pragma unroll
      for (int i = 0; i < RO; ++i) {
        ut[i] = Lt.ld(6 + par, h);
        us[i] = Ls.ld(2 * mu + par, h);
        h += hts;
        par ^= 1;
      }
#pragma unroll
      for (int e = 0; e < kTgExt; ++e) {
        const Site ye = plane_site(g, mu, a, c1, c2, (kTgExt * c + e) % nt);
        us[RO + e] = Ls.ld(2 * mu + parity(ye), hidx(g, ye));
      }
      Quat<R> L = qone<R>();
#pragma unroll
      for (int i = 0; i < RO; ++i) {
        Sb[tg_row<RO>(r0 + i, nt, SS) + a] = L;
        L = qunit(qmul(L, ut[i]));
      }
      Ct[c * nm + a] = L;
    }
    __syncthreads();
    // (2) prefix over the chunks: G(a, r) for the thread's rows, P(a) = G(a, Nt)
    if (active) {
      Quat<R> Q = qone<R>();
      for (int k = 0; k < c; ++k) Q = qunit(qmul(Q, Ct[k * nm + a]));
      if (c > 0) {
#pragma unroll
        for (int i = 0; i < RO; ++i) {
          Quat<R>* p = Sb + tg_row<RO>(r0 + i, nt, SS) + a;
          *p = qunit(qmul(Q, *p));
        }
      }
      if (c == kTgChunks - 1) Pb[a] = qunit(qmul(Q, Ct[c * nm + a]));
    }
    __syncthreads();
    // (3) U'(a, r) = G(a, t) U_mu(a, t) G(a+1, t)^dag for the lane's rows,
    // conjugated by P on its extended rows; column a + nm (a < rmax - 1)
    // repeats column a
    if (active) {
      const int an = a + 1 == nm ? 0 : a + 1;
      const bool dup = a < rmax - 1;
#pragma unroll
      for (int i = 0; i < RO + kTgExt; ++i) {
        const bool ext = i >= RO;
        const int t = ext ? (kTgExt * c + (i - RO)) % nt : r0 + i;
        const int r = ext ? nt + kTgExt * c + (i - RO) : r0 + i;
        const int gt = tg_row<RO>(t, nt, SS);
        Quat<R> v = qmul_nd(qmul(Sb[gt + a], us[i]), Sb[gt + an]);
        if (ext) v = qmul_nd(qmul(Pb[a], v), Pb[an]);
        const int ru = tg_row<RO>(r, nt, SU);
        Ue[ru + a] = v;
        if (dup) Ue[ru + a + nm] = v;
      }
    }
    __syncthreads();  // Sb now holds lines
    // (4) R = 1 .. rmax, warp-synchronous.  The thread's rows start at
    // bu / bs (origin rows, shifted by sk) and bue / bse (extended rows).
    constexpr int unit = tg_skew_unit<RO>();
    const int sk = unit * (c & 1);
    const int bu = r0 * SU + sk + a, bs = r0 * SS + sk + a;
    const int bue = (nt + kTgExt * c) * SU + a, bse = (nt + kTgExt * c) * SS + a;
    Quat<R> own[RO];  // the origin rows' lines; the extended rows' stay in Sb
    R acc[kTgT];
#pragma unroll
    for (int k = 0; k < kTgT; ++k) acc[k] = R(0);
    for (int Rl = 1; Rl <= rmax; ++Rl) {
      if (active) {
#pragma unroll
        for (int i = 0; i < RO; ++i) {
          const Quat<R> v = Ue[bu + i * SU + Rl - 1];
          own[i] = Rl == 1 ? v : qmul(own[i], v);
          Sb[bs + i * SS] = own[i];
        }
#pragma unroll
        for (int e = 0; e < kTgExt; ++e) {
          const Quat<R> v = Ue[bue + e * SU + Rl - 1];
          Quat<R>* p = Sb + bse + e * SS;
          *p = Rl == 1 ? v : qmul(*p, v);
        }
      }
      __syncwarp();
      if (active) {
        // origin rows r0 + i, i < RO, against rows r0 + j, j = i + T; the
        // benchmark's T range (all sixteen) takes a copy without the T test
        auto dots = [&](auto full_c) {
          constexpr bool FULL = decltype(full_c)::value;
#pragma unroll
          for (int j = 1; j < RO + kTgT; ++j) {
            Quat<R> w;
            if (j < RO) {
              w = own[j < RO ? j : 0];
            } else {
              const int rr = r0 + j;  // chunk c + j / RO while below Nt
              w = Sb[rr * SS + (rr < nt ? unit * ((c + j / RO) & 1) : 0) + a];
            }
#pragma unroll
            for (int i = 0; i < RO; ++i) {
              const int T = j - i;
              if (T >= 1 && T <= kTgT && (FULL || T <= tmax))
                acc[T - 1] =
                    fma(own[i].w, w.w, fma(own[i].x, w.x, fma(own[i].y, w.y, fma(own[i].z, w.z, acc[T - 1]))));
            }
          }
        };
        if (tmax == kTgT) dots(std::true_type{});
        else dots(std::false_type{});
      }
      __syncwarp();  // the lines are read before the next R overwrites them
      // this R's sums: a transposing butterfly leaves lanes 2k and 2k+1 the
      // warp total of slot lo; the even lanes store it in this R's slot
      int lo = 0;
#pragma unroll
      for (int lev = 0; lev < 4; ++lev) {
        const int off = 16 >> lev, half = 8 >> lev;
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          if (m < half) {
            const R send = upper ? acc[m] : acc[m + half];
            const R keep = upper ? acc[m + half] : acc[m];
            acc[m] = keep + __shfl_xor_sync(0xffffffffu, send, off);
          }
        }
        if (upper) lo += half;
      }
      acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
      if ((lane & 1) == 0) wsum[Rl - 1][warp][lo] = acc[0];
#pragma unroll
      for (int k = 0; k < kTgT; ++k) acc[k] = R(0);
    }
    __syncthreads();
    // the plane's sums, warps in a fixed order
    const int nw = (int)(blockDim.x >> 5);
    for (int s = threadIdx.x; s < rmax * kTgT; s += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += (double)wsum[s / kTgT][w][s % kTgT];
      acc64[s] += t;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 16 * kTgT; i += blockDim.x) partials[(size_t)blockIdx.x * 16 * kTgT + i] = acc64[i];
}

// out[(R-1) tmax + (T-1)]: one block per output adds the per-block sums of the
// three directions and all x-blocks of T's chunk, in a fixed order.
template <int TC>
__global__ void __launch_bounds__(kThreads) k_wilson_final(const double* partials, int gx, int rmax, int tmax,
                                                           double inv, double* out) {
  const int o = blockIdx.x;
  const int r = o / tmax, t = o % tmax;
  const int c = t / TC, j = t % TC;
  const int per = rmax * TC;
  const int n = 3 * gx;
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int m = i / gx, bx = i % gx;
    a += __ldcg(partials + (size_t)((3 * c + m) * gx + bx) * per + r * TC + j);
  }
  const double tot = block_sum(a);
  if (threadIdx.x == 0) out[o] = tot * inv;
}

// ---------------------------------------------------------------------------
// Canonical FP64 host layout (site-major, direction, component) <-> store.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_to_canonical(Links<P> L, Geom g, double* c,
                                                           int64_t s0, int64_t ns) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 4 * ns; w += stride) {
    const uint32_t s = (uint32_t)(s0 + (w >> 2));
    const int mu = (int)(w & 3);
    const Site x = site_from_index(g, s);
    const auto q = L.ld(2 * mu + parity(x), hidx(g, x));
    double* o = c + 4 * w;
    o[0] = q.w; o[1] = q.x; o[2] = q.y; o[3] = q.z;
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_from_canonical(Links<P> L, Geom g, const double* c,
                                                             int64_t s0, int64_t ns) {
  using R = typename Real<P>::T;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 4 * ns; w += stride) {
    const uint32_t s = (uint32_t)(s0 + (w >> 2));
    const int mu = (int)(w & 3);
    const Site x = site_from_index(g, s);
    const double* i = c + 4 * w;
    L.st(2 * mu + parity(x), hidx(g, x), qmake<R>((R)i[0], (R)i[1], (R)i[2], (R)i[3]));
  }
}

__global__ void k_add_u32(uint32_t* p, uint32_t v) { *p += v; }

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_init(const LatticeView& v, int start, PhiloxKey key, uint32_t lattice_tag,
                        cudaStream_t st) {
  const RoundKeys rk = round_keys(key);
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_init<P>, 8 * v.g.vh);
    k_init<P><<<gr, kThreads, 0, st>>>(L, v.g, start, rk, lattice_tag);
  });
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_overrelax(const LatticeView& v, int mu, int parity, cudaStream_t st) {
  SU2_DISPATCH(v.prec, SU2_DISPATCH_MU(mu, {
    auto L = links_of<P, kClassPtr>(v.links, v.g.vh);
    if (parity == 0) {
      const int gr = grid_for(k_overrelax<P, MU, 0>, v.g.vh);
      k_overrelax<P, MU, 0><<<gr, kThreads, 0, st>>>(L, v.g);
    } else {
      const int gr = grid_for(k_overrelax<P, MU, 1>, v.g.vh);
      k_overrelax<P, MU, 1><<<gr, kThreads, 0, st>>>(L, v.g);
    }
  }));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_plaquette(const LatticeView& v, const Scratch& s, cudaStream_t st, int64_t s0, int64_t ns) {
  if (ns < 0) ns = 2 * v.g.vh;
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_plaquette<P>, ns);
    k_plaquette<P><<<gr, kThreads, 0, st>>>(L, v.g, s0, ns, s.partials, s.counter, s.out);
  });
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Time lines (for the Polyakov loop of a lattice split into time slabs,
// Section 2 Eqs. 14-15): for every spatial site xs in [x0, x0 + nx) the
// product of its time links at slices t0, t0 + 1, ..., t0 + nt - 1 in that
// order, to out[4 (xs - x0) + c] in FP64.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_time_lines(Links<P> L, Geom g, int t0, int nt, int64_t x0, int64_t nx,
                                                         double* out) {
  using R = typename Real<P>::T;
  const int64_t nsig = 2 * g.vh / g.n[3];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += stride) {
    const int64_t xs = x0 + i;
    Quat<R> pr = qone<R>();
    for (int t = t0; t < t0 + nt; ++t) {
      const Site x = site_from_index(g, (uint32_t)(xs + nsig * t));
      pr = qmul(pr, L.ld(6 + parity(x), hidx(g, x)));
    }
    double* o = out + 4 * i;
    o[0] = pr.w; o[1] = pr.x; o[2] = pr.y; o[3] = pr.z;
  }
}

cudaError_t launch_time_lines(const LatticeView& v, int t0, int nt, int64_t x0, int64_t nx, double* out,
                              cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_time_lines<P>, nx);
    k_time_lines<P><<<gr, kThreads, 0, st>>>(L, v.g, t0, nt, x0, nx, out);
  });
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_polyakov(const LatticeView& v, const Scratch& s, cudaStream_t st, const SweepEpilogue* ep) {
  SweepEpilogue e{};
  if (ep) e = *ep;
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P, kClassPtr>(v.links, v.g.vh);
    const int64_t nsig = 2 * v.g.vh / v.g.n[3];
    // segments per time line: the largest power of two <= 8 that divides nt
    // and leaves segments of at least 8 links
    int lg = 0;
    while (lg < 3 && v.g.n[3] % (2 << lg) == 0 && v.g.n[3] / (2 << lg) >= 8) ++lg;
    const int gr = grid_for(k_polyakov<P>, nsig << lg);
    k_polyakov<P><<<gr, kThreads, 0, st>>>(L, v.g, lg, s.partials, s.counter, s.out, e);
  });
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ape(const LatticeView& src, void* dst, double alpha, cudaStream_t st) {
  SU2_DISPATCH(src.prec, {
    auto S = links_of<P, kClassPtr>(src.links, src.g.vh);
    auto D = links_of<P, kClassPtr>(dst, src.g.vh);
    // two y-slices (one per parity) share the machine
    int gx = grid_for(k_ape<P>, 2 * src.g.vh) / 2;
    if (gx < 1) gx = 1;
    k_ape<P><<<dim3(gx, 2), kThreads, 0, st>>>(S, D, src.g, alpha);
  });
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_spatial(const LatticeView& src, void* dst, cudaStream_t st) {
  SU2_DISPATCH(src.prec, {
    auto S = links_of<P>(src.links, src.g.vh);
    auto D = links_of<P>(dst, src.g.vh);
    const int gr = grid_for(k_copy_spatial<P>, 6 * src.g.vh);
    k_copy_spatial<P><<<gr, kThreads, 0, st>>>(S, D);
  });
  count_launches(1);
  return cudaGetLastError();
}

template <int P> struct WilsonChunk { static constexpr int tc = 16; };
template <> struct WilsonChunk<kF64> { static constexpr int tc = 8; };

// Plane kernel shape per arithmetic precision: T chunk and block size.
#ifndef SU2_WILSON_RT
#define SU2_WILSON_RT 1
#endif
constexpr int kWilsonRtThreads = 512;
// dynamic shared memory of the time-outer kernel: 227 KB per block minus its
// static accumulators (18 KB at RC = 16)
constexpr int kWilsonRtSmemMax = 208 * 1024;

template <int P, int RC>
static cudaError_t launch_wilson_rt_rc(const LatticeView& v, const void* spatial, int rmax, int tmax, int tile,
                                       int smem, const Scratch& s, cudaStream_t st) {
  constexpr int NTH = kWilsonRtThreads;
  // the shared-memory limit is raised once per device (concurrent first
  // calls from several host threads wait on the device's once_flag)
  static std::once_flag attr_once[64];
  static cudaError_t attr_err[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64) {
    std::call_once(attr_once[dev], [dev]() {
      attr_err[dev] = cudaFuncSetAttribute(k_wilson_rt<P, RC, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kWilsonRtSmemMax);
    });
    if (attr_err[dev] != cudaSuccess) return attr_err[dev];
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wilson_rt<P, RC, NTH>, NTH, smem);
  if (per_sm < 1) per_sm = 1;
  const int nrc = (rmax + RC - 1) / RC, ntc = (tmax + kWrtT - 1) / kWrtT;
  const int nchunks = nrc * ntc;
  const int ntiles = (v.g.n[3] + tile - 1) / tile;
  const int64_t nunits = (int64_t)(v.g.n[1] * v.g.n[2] + v.g.n[0] * v.g.n[2] + v.g.n[0] * v.g.n[1]) * ntiles;
  int64_t gx = ((int64_t)device_info().sms * per_sm + nchunks - 1) / nchunks;
  if (gx > nunits) gx = nunits;
  const int64_t cap = (int64_t)kScratchPartials / (RC * kWrtT) / nchunks;
  if (gx > cap) gx = cap;
  if (gx < 1) gx = 1;
  auto Lt = links_of<P>(v.links, v.g.vh);
  auto Ls = links_of<P>(const_cast<void*>(spatial), v.g.vh);
  k_wilson_rt<P, RC, NTH><<<dim3((unsigned)gx, nchunks), NTH, smem, st>>>(Ls, Lt, v.g, rmax, tmax, ntc, nrc * RC,
                                                                         tile, s.partials);
  count_launches(1);
  const int64_t V = 2 * v.g.vh;
  k_wilson_rt_final<RC><<<rmax * tmax, kThreads, 0, st>>>(s.partials, (int)gx, ntc, tmax, 1.0 / (3.0 * (double)V),
                                                          s.out);
  count_launches(1);
  return cudaGetLastError();
}

// The time-outer kernel with as many time slices per work unit as fit in
// shared memory next to the ntc * 16 slices of line overhang (the whole
// plane when it fits); *used = false if not even one slice fits.  FP64 runs
// 8-wide R chunks (register budget).
template <int P>
static cudaError_t launch_wilson_rt(const LatticeView& v, const void* spatial, int rmax, int tmax,
                                    const Scratch& s, cudaStream_t st, bool* used) {
  using R = typename Real<P>::T;
  *used = false;
  if (!SU2_WILSON_RT) return cudaSuccess;
  const int nmax = v.g.n[0] > v.g.n[1] ? (v.g.n[0] > v.g.n[2] ? v.g.n[0] : v.g.n[2])
                                       : (v.g.n[1] > v.g.n[2] ? v.g.n[1] : v.g.n[2]);
  const int rc = (rmax <= 8 || P == kF64) ? 8 : 16;
  const int pad = (rmax + rc - 1) / rc * rc;  // columns a .. a + pad - 1 of a row
  const int overhang = (tmax + kWrtT - 1) / kWrtT * kWrtT;
  const int row_bytes = 2 * (nmax + pad) * (int)sizeof(Quat<R>);
  int tile, smem;
  if (row_bytes * v.g.n[3] <= kWilsonRtSmemMax) {
    tile = v.g.n[3];  // the whole plane, rows read modulo nt
    smem = row_bytes * tile;
  } else {
    tile = kWilsonRtSmemMax / row_bytes - overhang;
    if (tile < 1) return cudaSuccess;
    smem = row_bytes * (tile + overhang);
  }
  *used = true;
  if (rc == 8) return launch_wilson_rt_rc<P, 8>(v, spatial, rmax, tmax, tile, smem, s, st);
  if constexpr (P != kF64) return launch_wilson_rt_rc<P, 16>(v, spatial, rmax, tmax, tile, smem, s, st);
  return cudaErrorInvalidValue;
}

// The temporal-gauge kernel when R and T are at most 16, Nt is a multiple of
// 8 with Nt / 8 in {1, 2, 4, 6, 8}, one block holds four columns a warp of
// the widest plane, and the staged plane fits in shared memory; *used =
// false otherwise.
template <int P, int RO>
static cudaError_t launch_wilson_tg_rows(const LatticeView& v, const void* spatial, int rmax, int tmax,
                                         const Scratch& s, cudaStream_t st, bool* used) {
  using R = typename Real<P>::T;
  constexpr int kMaxThreads = TgThreads<P>::value;
  *used = false;
  const int nmax = std::max(v.g.n[0], std::max(v.g.n[1], v.g.n[2]));
  const int nt = v.g.n[3], nr = nt + kTgT;
  const int nth = (nmax + kTgCols - 1) / kTgCols * 32;
  if (nth > kMaxThreads) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_wilson_tg<P, RO>);
  if (e != cudaSuccess) return e;
  const int64_t smem = ((int64_t)nr * tg_stride<RO>(nmax + rmax - 1) + 4 + (int64_t)nr * tg_stride<RO>(nmax) + 4 +
                        (int64_t)kTgChunks * nmax + nmax) *
                       (int64_t)sizeof(Quat<R>);
  const int64_t dyn_max = (int64_t)optin - (int64_t)fa.sharedSizeBytes;
  if (smem > dyn_max) return cudaSuccess;
  // raised once per device, as for the time-outer kernel
  static std::once_flag attr_once[64];
  static cudaError_t attr_err[64];
  if (dev >= 0 && dev < 64) {
    const int lim = (int)dyn_max;
    std::call_once(attr_once[dev], [dev, lim]() {
      attr_err[dev] = cudaFuncSetAttribute(k_wilson_tg<P, RO>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    });
    if (attr_err[dev] != cudaSuccess) return attr_err[dev];
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wilson_tg<P, RO>, nth, (size_t)smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t nunits = (int64_t)v.g.n[1] * v.g.n[2] + (int64_t)v.g.n[0] * v.g.n[2] + (int64_t)v.g.n[0] * v.g.n[1];
  int64_t gx = (int64_t)device_info().sms * per_sm;
  if (gx > nunits) gx = nunits;
  const int64_t cap = (int64_t)kScratchPartials / (16 * kTgT);
  if (gx > cap) gx = cap;
  *used = true;
  auto Lt = links_of<P>(v.links, v.g.vh);
  auto Ls = links_of<P>(const_cast<void*>(spatial), v.g.vh);
  k_wilson_tg<P, RO><<<(unsigned)gx, nth, (size_t)smem, st>>>(Ls, Lt, v.g, rmax, tmax, s.partials);
  count_launches(1);
  const int64_t V = 2 * v.g.vh;
  k_wilson_rt_final<16><<<rmax * tmax, kThreads, 0, st>>>(s.partials, (int)gx, 1, tmax, 1.0 / (3.0 * (double)V),
                                                          s.out);
  count_launches(1);
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_wilson_tg(const LatticeView& v, const void* spatial, int rmax, int tmax,
                                    const Scratch& s, cudaStream_t st, bool* used) {
  *used = false;
  const int nt = v.g.n[3];
  if (!SU2_WILSON_TG || rmax > 16 || tmax > kTgT || nt % kTgChunks != 0) return cudaSuccess;
  switch (nt / kTgChunks) {
    case 1: return launch_wilson_tg_rows<P, 1>(v, spatial, rmax, tmax, s, st, used);
    case 2: return launch_wilson_tg_rows<P, 2>(v, spatial, rmax, tmax, s, st, used);
    case 4: return launch_wilson_tg_rows<P, 4>(v, spatial, rmax, tmax, s, st, used);
    case 6: return launch_wilson_tg_rows<P, 6>(v, spatial, rmax, tmax, s, st, used);
    case 8: return launch_wilson_tg_rows<P, 8>(v, spatial, rmax, tmax, s, st, used);
    default: return cudaSuccess;
  }
}

cudaError_t launch_wilson(const LatticeView& v, const void* spatial, int rmax, int tmax,
                          const Scratch& s, cudaStream_t st) {
  if (rmax < 1 || rmax > kWilsonMaxR || tmax < 1) return cudaErrorInvalidValue;
  {
    bool used = false;
    cudaError_t e = cudaSuccess;
    SU2_DISPATCH(v.prec, {
      e = launch_wilson_tg<P>(v, spatial, rmax, tmax, s, st, &used);
      if (e == cudaSuccess && !used) e = launch_wilson_rt<P>(v, spatial, rmax, tmax, s, st, &used);
    });
    if (e != cudaSuccess || used) return e;
  }
  // rows too long for even one time slice in shared memory: global-memory kernel
  SU2_DISPATCH(v.prec, {
    constexpr int TC = WilsonChunk<P>::tc;
    auto Lt = links_of<P>(v.links, v.g.vh);
    auto Ls = links_of<P>(const_cast<void*>(spatial), v.g.vh);
    const int nchunks = (tmax + TC - 1) / TC;
    const int64_t V = 2 * v.g.vh;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wilson<P, TC>, kWilsonThreads, 0);
    if (per_sm < 1) per_sm = 1;
    // all (chunk, direction) slices together fill the machine once
    int64_t gx = (int64_t)device_info().sms * per_sm / (3 * nchunks);
    const int64_t need = (V + kWilsonThreads - 1) / kWilsonThreads;
    if (gx > need) gx = need;
    // keep one partial set per block within the scratch buffer
    const int64_t per = (int64_t)rmax * TC;
    const int64_t cap = (int64_t)kScratchPartials / per / (3 * nchunks);
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    k_wilson<P, TC><<<dim3((unsigned)gx, 3 * nchunks), kWilsonThreads, 0, st>>>(Ls, Lt, v.g, rmax, tmax, s.partials);
    count_launches(1);
    k_wilson_final<TC><<<rmax * tmax, kThreads, 0, st>>>(s.partials, (int)gx, rmax, tmax, 1.0 / (3.0 * (double)V),
                                                         s.out);
  });
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_to_canonical(const LatticeView& v, double* canon, int64_t s0, int64_t ns,
                                cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_to_canonical<P>, 4 * ns);
    k_to_canonical<P><<<gr, kThreads, 0, st>>>(L, v.g, canon, s0, ns);
  });
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_from_canonical(const LatticeView& v, const double* canon, int64_t s0,
                                  int64_t ns, cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_from_canonical<P>, 4 * ns);
    k_from_canonical<P><<<gr, kThreads, 0, st>>>(L, v.g, canon, s0, ns);
  });
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_add_u32(uint32_t* p, uint32_t v, cudaStream_t st) {
  k_add_u32<<<1, 1, 0, st>>>(p, v);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace su2
