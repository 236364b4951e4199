// Kernels of the SU(2) heat-bath Monte Carlo for sm_103a: start
// configurations, the checkerboard heat-bath and over-relaxation substeps,
// the fused plaquette / Polyakov reductions, APE smearing, Wilson loops and
// the canonical-layout conversions.  Paper: Cardoso & Bicudo,
// arXiv:1010.4834 (Sections 2 and 4).
//
// None of these work is a dense contraction (2x2 SU(2) products in
// registers), so everything runs on the FP32/FP64 pipes; the sweep is bound
// by HBM traffic and ALU issue.  Reductions are fused into the measurement
// kernels: per-thread compensated sums, warp shuffles, one partial per block
// and a last-block finisher that adds the partials in a fixed order, so a
// result is reproducible run to run.
#include <cfloat>

#include "su2_internal.h"

namespace su2 {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Device info and launch shapes
// ---------------------------------------------------------------------------
const DeviceInfo& device_info() {
  static DeviceInfo info[64];
  static bool have[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!have[dev]) {
    cudaDeviceGetAttribute(&info[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&info[dev].l2_bytes, cudaDevAttrL2CacheSize, dev);
    if (info[dev].sms <= 0) info[dev].sms = 1;
    have[dev] = true;
  }
  return info[dev];
}

Geom make_geom(const int n[4]) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.n[i] = n[i];
  g.n0h = n[0] / 2;
  g.vh = (int64_t)n[0] * n[1] * n[2] * n[3] / 2;
  g.f_n0h = FastDiv((uint32_t)g.n0h);
  g.f_n1 = FastDiv((uint32_t)n[1]);
  g.f_n2 = FastDiv((uint32_t)n[2]);
  g.f_n0 = FastDiv((uint32_t)n[0]);
  return g;
}

size_t scratch_bytes() {
  return kScratchPartials * sizeof(double) + 256 + kScratchOut * sizeof(double) + 256;
}

// Blocks for `work` items with a grid-stride loop: enough to fill every SM
// `waves` times over at the kernel's occupancy, never more than needed.
template <class K>
static int grid_for(K kernel, int64_t work, int smem = 0) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t full = (int64_t)device_info().sms * per_sm;
  const int64_t need = (work + kThreads - 1) / kThreads;
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

// In the last block: tot[k] = sum over blocks of partials[b*NV + k], summed in
// a fixed order (strided per thread, then thread order), compensated.
template <int NV>
__device__ __forceinline__ void final_sum(const double* partials, int nblocks, double (&tot)[NV]) {
  __shared__ double ss[kThreads][NV], sc[kThreads][NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    KSum a;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) a.add(__ldcg(partials + (size_t)b * NV + k));
    ss[threadIdx.x][k] = a.s;
    sc[threadIdx.x][k] = a.c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      KSum a;
      double comp = 0.0;
      for (int t = 0; t < kThreads; ++t) { a.add(ss[t][k]); comp += sc[t][k]; }
      tot[k] = a.value() + comp;
    }
  }
}

// ---------------------------------------------------------------------------
// Start configurations (Section 4 kernel list: cold start U = 1, hot start a
// random SU(2) matrix, read here as Haar via Philox draw 0 of sweep index
// 0xFFFFFFFF).  One thread per (site, direction).
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_init(Links<P> L, Geom g, int start, PhiloxKey key,
                                                   uint32_t lattice_tag) {
  using R = typename Real<P>::T;
  const int64_t V = 2 * g.vh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 4 * V; w += stride) {
    const int mu = (int)(w / V);
    const uint32_t s = (uint32_t)(w - (int64_t)mu * V);
    int x[4];
    decode_site(g, s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    Quat<R> q = qone<R>();
    if (start) q = haar_from<R>(philox4x32_10(make_uint4(s, (uint32_t)mu | lattice_tag, 0xFFFFFFFFu, 0u), key));
    L.st(2 * mu + p, s >> 1, q);
  }
}

// ---------------------------------------------------------------------------
// Heat-bath substep (Section 2 Eqs. 5-9, 11; Section 4 checkerboard): one
// thread per link of direction mu on the parity-p sublattice.  A capped link
// (all trials rejected) is neither read nor written.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_heatbath(Links<P> L, Geom g, int mu, int p,
                                                       const uint32_t* sweep_base,
                                                       uint32_t sweep_off, HBParams hp,
                                                       unsigned long long* stats) {
  using R = typename Real<P>::T;
  const R beta = (R)hp.beta;
  const uint32_t sweep = (sweep_base ? *sweep_base : 0u) + sweep_off;
  const uint32_t tag = (uint32_t)mu | hp.lattice_tag;
  unsigned int trials = 0, capped = 0, haar = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < g.vh; h += stride) {
    int x[4];
    decode_half(g, (uint32_t)h, p, x);
    const Quat<R> sig = staple<P>(L, g, x, h, mu, p, 0xF);
    Quat<R> nl;
    const int n = heatbath_draw<R>(sig, make_uint4(site_of(g, x), tag, sweep, 0u), hp, beta, &nl);
    if (n != 0) L.st(2 * mu + p, h, nl);
    if (stats) {
      trials += n > 0 ? (unsigned)n : (n == 0 ? (unsigned)hp.max_tries : 0u);
      capped += n == 0;
      haar += n < 0;
    }
  }
  if (stats) {
    __shared__ unsigned int sh[3];
    if (threadIdx.x < 3) sh[threadIdx.x] = 0;
    __syncthreads();
    if (trials) atomicAdd(&sh[0], trials);
    if (capped) atomicAdd(&sh[1], capped);
    if (haar) atomicAdd(&sh[2], haar);
    __syncthreads();
    if (threadIdx.x < 3 && sh[threadIdx.x]) atomicAdd(stats + threadIdx.x, (unsigned long long)sh[threadIdx.x]);
  }
}

// ---------------------------------------------------------------------------
// Over-relaxation substep (Section 2, Eq. 10 with W = Sigma/|Sigma| for the
// orientation of Eq. 11): U' = W U^dagger W keeps Tr(U Sigma^dagger).
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_overrelax(Links<P> L, Geom g, int mu, int p) {
  using R = typename Real<P>::T;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < g.vh; h += stride) {
    int x[4];
    decode_half(g, (uint32_t)h, p, x);
    const Quat<R> sig = staple<P>(L, g, x, h, mu, p, 0xF);
    const R k2 = qdot(sig, sig);
    if (!(k2 >= R(P == kF64 ? 1e-300 : 1e-30))) continue;
    const Quat<R> w = qscale(sig, R(1) / sqrt_r(k2));
    const Quat<R> u = L.ld(2 * mu + p, h);
    L.st(2 * mu + p, h, qmul(qmul_nd(w, u), w));
  }
}

// ---------------------------------------------------------------------------
// Plaquette (Section 2, Eqs. 12-13): per site the six (1/2) Re Tr
// U_mu(x) U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger = (A B^dagger)_0 with
// A = U_mu(x) U_nu(x+mu), B = U_nu(x) U_mu(x+nu): the dot product A.B.
// out[0] all, out[1] spatial, out[2] space-time means.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_plaquette(Links<P> L, Geom g, double* partials,
                                                        unsigned int* counter, double* out) {
  using R = typename Real<P>::T;
  Acc<R> sp, tm;
  const int64_t V = 2 * g.vh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < V; s += stride) {
    int x[4];
    decode_site(g, (uint32_t)s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1, q = p ^ 1;
    const int64_t h = s >> 1;
    Quat<R> u[4];
    int64_t hp[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      u[mu] = L.ld(2 * mu + p, h);
      hp[mu] = hidx_shift(g, x, mu, +1);
    }
    R ssum = 0, tsum = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
      for (int nu = mu + 1; nu < 4; ++nu) {
        const Quat<R> a = qmul(u[mu], L.ld(2 * nu + q, hp[mu]));
        const Quat<R> b = qmul(u[nu], L.ld(2 * mu + q, hp[nu]));
        const R v = qdot(a, b);
        if (nu == 3) tsum += v; else ssum += v;
      }
    }
    sp.add(ssum);
    tm.add(tsum);
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
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_polyakov(Links<P> L, Geom g, double* partials,
                                                       unsigned int* counter, double* out) {
  using R = typename Real<P>::T;
  Acc<R> acc;
  const int64_t nsig = (int64_t)g.n[0] * g.n[1] * g.n[2];
  const int64_t nsig_h = nsig / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t xs = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; xs < nsig; xs += stride) {
    int x[4];
    decode_site(g, (uint32_t)xs, x);
    const int px = (x[0] + x[1] + x[2]) & 1;
    const int64_t hh = xs >> 1;
    Quat<R> pr = L.ld(6 + px, hh);
    for (int t = 1; t < g.n[3]; ++t) pr = qmul(pr, L.ld(6 + ((px + t) & 1), hh + nsig_h * t));
    acc.add(pr.w);
  }
  double v[1] = {acc.value()};
  if (block_partial<1>(v, partials, counter)) {
    double tot[1];
    final_sum<1>(partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      out[0] = tot[0] / (double)nsig;
      *counter = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// APE smearing step (Section 2, Eq. 19), Jacobi: spatial link (x, mu) ->
// P[(1-alpha) U + (alpha/4) (four spatial staples)], P = normalisation; a sum
// with vanishing norm keeps U.  blockIdx.y = mu in 0..2.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_ape(Links<P> src, Links<P> dst, Geom g,
                                                  double alpha_d) {
  using R = typename Real<P>::T;
  const int mu = blockIdx.y;
  const R alpha = (R)alpha_d;
  const R c0 = R(1) - alpha, c1 = R(0.25) * alpha;
  const int64_t V = 2 * g.vh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < V; s += stride) {
    int x[4];
    decode_site(g, (uint32_t)s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int64_t h = s >> 1;
    const Quat<R> sig = staple<P>(src, g, x, h, mu, p, 0x7);
    const Quat<R> u = src.ld(2 * mu + p, h);
    const Quat<R> q = qmake<R>(c0 * u.w + c1 * sig.w, c0 * u.x + c1 * sig.x, c0 * u.y + c1 * sig.y,
                               c0 * u.z + c1 * sig.z);
    const R n2 = qdot(q, q);
    if (n2 >= R(P == kF64 ? 1e-300 : 1e-30))
      dst.st(2 * mu + p, h, qscale(q, R(1) / sqrt_r(n2)));
    else
      dst.st(2 * mu + p, h, u);
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_copy_spatial(Links<P> src, Links<P> dst) {
  const int64_t n = 6 * src.vh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int cls = (int)(i / src.vh);
    const int64_t j = i - cls * src.vh;
    dst.st(cls, j, src.ld(cls, j));
  }
}

// ---------------------------------------------------------------------------
// Wilson loops (Section 2, Eq. 18), (1/2) Tr[S_R(x) T_T(x+R mu) S_R(x+T t)^dag
// T_T(x)^dag] = (A B) . (D C) with A = S_R(x), B = T_T(x+R mu), C = S_R(x+T t),
// D = T_T(x).  A thread owns one (site, spatial mu) and a chunk of TC values
// of T; it walks R = 1..rmax extending A and the TC lines C by one link each,
// rebuilds the time line B at x + R mu, and adds the TC loop values into the
// block's shared accumulators (warp sums first).  blockIdx.y = 3 chunk + mu.
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ Quat<typename Real<P>::T> ld_at(const Links<P>& L, const Geom& g,
                                                          const int y[4], int dir) {
  const int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  return L.ld(2 * dir + par, hidx(g, y[0], y[1], y[2], y[3]));
}

constexpr int kWilsonMaxR = 32;

template <int P, int TC>
__global__ void __launch_bounds__(kThreads) k_wilson(Links<P> Ls, Links<P> Lt, Geom g, int rmax,
                                                     int tmax, double* partials,
                                                     unsigned int* counter, double* out) {
  using R = typename Real<P>::T;
  __shared__ double acc[kWilsonMaxR * TC];
  __shared__ bool last;
  const int mu = blockIdx.y % 3;
  const int chunk = blockIdx.y / 3;
  const int t0 = chunk * TC;
  const int nT = min(TC, tmax - t0);
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kWilsonMaxR * TC; i += kThreads) acc[i] = 0.0;
  __syncthreads();
  const int64_t V = 2 * g.vh;
  const int nt = g.n[3];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += stride) {
    const int64_t s = base + threadIdx.x;
    const bool valid = s < V;
    int x[4];
    decode_site(g, (uint32_t)(valid ? s : 0), x);
    Quat<R> D[TC], C[TC];
    {
      int y[4] = {x[0], x[1], x[2], x[3]};
      Quat<R> pr = qone<R>();
      for (int t = 0; t < t0; ++t) { pr = qmul(pr, ld_at(Lt, g, y, 3)); y[3] = wrap_inc(y[3], nt); }
#pragma unroll
      for (int j = 0; j < TC; ++j) {
        if (j < nT) { pr = qmul(pr, ld_at(Lt, g, y, 3)); y[3] = wrap_inc(y[3], nt); }
        D[j] = pr;
        C[j] = qone<R>();
      }
    }
    Quat<R> A = qone<R>();
    int xr[4] = {x[0], x[1], x[2], x[3]};
    for (int r = 1; r <= rmax; ++r) {
      A = qmul(A, ld_at(Ls, g, xr, mu));
      {
        int z[4] = {xr[0], xr[1], xr[2], (xr[3] + t0 + 1) % nt};
#pragma unroll
        for (int j = 0; j < TC; ++j) {
          if (j < nT) { C[j] = qmul(C[j], ld_at(Ls, g, z, mu)); z[3] = wrap_inc(z[3], nt); }
        }
      }
      xr[mu] = wrap_inc(xr[mu], g.n[mu]);
      int w[4] = {xr[0], xr[1], xr[2], xr[3]};
      Quat<R> b = qone<R>();
      for (int t = 0; t < t0; ++t) { b = qmul(b, ld_at(Lt, g, w, 3)); w[3] = wrap_inc(w[3], nt); }
#pragma unroll
      for (int j = 0; j < TC; ++j) {
        if (j < nT) {
          b = qmul(b, ld_at(Lt, g, w, 3));
          w[3] = wrap_inc(w[3], nt);
          R val = valid ? qdot(qmul(A, b), qmul(D[j], C[j])) : R(0);
          val = warp_sum(val);
          if (lane == 0) atomicAdd(&acc[(r - 1) * TC + j], (double)val);
        }
      }
    }
  }
  __syncthreads();
  const int nb = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  const int per = rmax * TC;
  for (int i = threadIdx.x; i < per; i += kThreads) partials[(size_t)bid * per + i] = acc[i];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!last) return;
  const double inv = 1.0 / (3.0 * (double)V);
  for (int o = threadIdx.x; o < rmax * tmax; o += kThreads) {
    const int r = o / tmax, t = o % tmax;
    const int c = t / TC, j = t % TC;
    KSum a;
    for (int m = 0; m < 3; ++m)
      for (int bx = 0; bx < (int)gridDim.x; ++bx)
        a.add(__ldcg(partials + (size_t)((3 * c + m) * gridDim.x + bx) * per + r * TC + j));
    out[o] = a.value() * inv;
  }
  if (threadIdx.x == 0) *counter = 0;
}

// ---------------------------------------------------------------------------
// Canonical FP64 host layout (site-major, direction, component) <-> store.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_to_canonical(Links<P> L, Geom g, double* c,
                                                           int64_t s0, int64_t ns) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 4 * ns; w += stride) {
    const int64_t s = s0 + (w >> 2);
    const int mu = (int)(w & 3);
    int x[4];
    decode_site(g, (uint32_t)s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const auto q = L.ld(2 * mu + p, s >> 1);
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
    const int64_t s = s0 + (w >> 2);
    const int mu = (int)(w & 3);
    int x[4];
    decode_site(g, (uint32_t)s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const double* i = c + 4 * w;
    L.st(2 * mu + p, s >> 1, qmake<R>((R)i[0], (R)i[1], (R)i[2], (R)i[3]));
  }
}

__global__ void k_add_u32(uint32_t* p, uint32_t v) { *p += v; }

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <int P> static Links<P> links_of(void* base, int64_t vh) {
  Links<P> L;
  L.p = reinterpret_cast<decltype(L.p)>(base);
  L.vh = vh;
  return L;
}

#define SU2_DISPATCH(prec, ...)                                  \
  switch (prec) {                                                \
    case kF64: { constexpr int P = kF64; __VA_ARGS__; break; }   \
    case kF32: { constexpr int P = kF32; __VA_ARGS__; break; }   \
    case kF16Q: { constexpr int P = kF16Q; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;                       \
  }

cudaError_t launch_init(const LatticeView& v, int start, PhiloxKey key, uint32_t lattice_tag,
                        cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_init<P>, 8 * v.g.vh);
    k_init<P><<<gr, kThreads, 0, st>>>(L, v.g, start, key, lattice_tag);
  });
  return cudaGetLastError();
}

cudaError_t launch_heatbath(const LatticeView& v, int mu, int parity, const uint32_t* sweep_base,
                            uint32_t sweep_off, const HBParams& hp, unsigned long long* stats,
                            cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_heatbath<P>, v.g.vh);
    k_heatbath<P><<<gr, kThreads, 0, st>>>(L, v.g, mu, parity, sweep_base, sweep_off, hp, stats);
  });
  return cudaGetLastError();
}

cudaError_t launch_overrelax(const LatticeView& v, int mu, int parity, cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_overrelax<P>, v.g.vh);
    k_overrelax<P><<<gr, kThreads, 0, st>>>(L, v.g, mu, parity);
  });
  return cudaGetLastError();
}

cudaError_t launch_plaquette(const LatticeView& v, const Scratch& s, cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_plaquette<P>, 2 * v.g.vh);
    k_plaquette<P><<<gr, kThreads, 0, st>>>(L, v.g, s.partials, s.counter, s.out);
  });
  return cudaGetLastError();
}

cudaError_t launch_polyakov(const LatticeView& v, const Scratch& s, cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int64_t nsig = 2 * v.g.vh / v.g.n[3];
    const int gr = grid_for(k_polyakov<P>, nsig);
    k_polyakov<P><<<gr, kThreads, 0, st>>>(L, v.g, s.partials, s.counter, s.out);
  });
  return cudaGetLastError();
}

cudaError_t launch_ape(const LatticeView& src, void* dst, double alpha, cudaStream_t st) {
  SU2_DISPATCH(src.prec, {
    auto S = links_of<P>(src.links, src.g.vh);
    auto D = links_of<P>(dst, src.g.vh);
    // three y-slices (one per spatial direction) share the machine
    int gx = grid_for(k_ape<P>, 2 * src.g.vh) / 3;
    if (gx < 1) gx = 1;
    k_ape<P><<<dim3(gx, 3), kThreads, 0, st>>>(S, D, src.g, alpha);
  });
  return cudaGetLastError();
}

cudaError_t launch_copy_spatial(const LatticeView& src, void* dst, cudaStream_t st) {
  SU2_DISPATCH(src.prec, {
    auto S = links_of<P>(src.links, src.g.vh);
    auto D = links_of<P>(dst, src.g.vh);
    const int gr = grid_for(k_copy_spatial<P>, 6 * src.g.vh);
    k_copy_spatial<P><<<gr, kThreads, 0, st>>>(S, D);
  });
  return cudaGetLastError();
}

cudaError_t launch_wilson(const LatticeView& v, const void* spatial, int rmax, int tmax,
                          const Scratch& s, cudaStream_t st) {
  if (rmax < 1 || rmax > kWilsonMaxR || tmax < 1) return cudaErrorInvalidValue;
  SU2_DISPATCH(v.prec, {
    constexpr int TC = P == kF64 ? 4 : 8;
    auto Lt = links_of<P>(v.links, v.g.vh);
    auto Ls = links_of<P>(const_cast<void*>(spatial), v.g.vh);
    const int nchunks = (tmax + TC - 1) / TC;
    const int64_t V = 2 * v.g.vh;
    int gx = grid_for(k_wilson<P, TC>, V);
    // keep one partial set per block within the scratch buffer
    const int64_t per = (int64_t)rmax * TC;
    const int64_t max_blocks = (int64_t)kScratchPartials / per;
    const int64_t cap = max_blocks / (3 * nchunks);
    if (gx > cap) gx = (int)cap;
    if (gx < 1) return cudaErrorInvalidValue;
    k_wilson<P, TC><<<dim3(gx, 3 * nchunks), kThreads, 0, st>>>(Ls, Lt, v.g, rmax, tmax,
                                                                s.partials, s.counter, s.out);
  });
  return cudaGetLastError();
}

cudaError_t launch_to_canonical(const LatticeView& v, double* canon, int64_t s0, int64_t ns,
                                cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_to_canonical<P>, 4 * ns);
    k_to_canonical<P><<<gr, kThreads, 0, st>>>(L, v.g, canon, s0, ns);
  });
  return cudaGetLastError();
}

cudaError_t launch_from_canonical(const LatticeView& v, const double* canon, int64_t s0,
                                  int64_t ns, cudaStream_t st) {
  SU2_DISPATCH(v.prec, {
    auto L = links_of<P>(v.links, v.g.vh);
    const int gr = grid_for(k_from_canonical<P>, 4 * ns);
    k_from_canonical<P><<<gr, kThreads, 0, st>>>(L, v.g, canon, s0, ns);
  });
  return cudaGetLastError();
}

cudaError_t launch_add_u32(uint32_t* p, uint32_t v, cudaStream_t st) {
  k_add_u32<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

}  // namespace su2
