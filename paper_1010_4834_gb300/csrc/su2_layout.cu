// Link-layout comparison of Section 5.1: the paper stores all links in one
// array, site-major with the four directions of a site next to each other,
// and reports 1.4x from splitting it into one array per direction.  This
// file holds a plain heat-bath substep (one thread per link, every trial
// inline, the paper's kernel structure) written once over two index
// policies: the library's store (class = direction and parity, half-site
// index) and a single array with element 4 s + mu, s the lexicographic site
// index.  Both run the same arithmetic in the same order as k_heatbath, so all
// three leave identical links; only the memory layout differs.  FP32 only.
#include "su2_internal.h"
#include "su2_kernel_util.cuh"

namespace su2 {

struct ClassIndex {  // the library's layout
  static __device__ __forceinline__ int64_t at(const Geom& g, const Site& y, int mu) {
    return (int64_t)(2 * mu + parity(y)) * g.vh + hidx(g, y);
  }
};
struct SiteMajorIndex {  // one array, four directions per site
  static __device__ __forceinline__ int64_t at(const Geom& g, const Site& y, int mu) {
    return 4 * (int64_t)site_index(g, y) + mu;
  }
};

template <class IX>
__device__ __forceinline__ Quat<float> ld_at(const float4* p, const Geom& g, const Site& y, int mu) {
  const float4 a = __ldg(p + IX::at(g, y, mu));
  return qmake<float>(a.x, a.y, a.z, a.w);
}

// Staple of Section 2 Eq. 11, the terms in the order of staple() (NU
// ascending, forward then backward, the same products).
template <class IX, int MU>
__device__ __forceinline__ Quat<float> staple_at(const float4* p, const Geom& g, const Site& x) {
  Quat<float> s = qmake<float>(0, 0, 0, 0);
  const Site xpm = shifted<MU, +1>(g, x);
#define SU2_TERM(NU)                                                                            \
  if (MU != NU) {                                                                               \
    const Site xmn = shifted<NU, -1>(g, x);                                                     \
    const Quat<float> a = ld_at<IX>(p, g, x, NU), b = ld_at<IX>(p, g, shifted<NU, +1>(g, x), MU); \
    const Quat<float> c = ld_at<IX>(p, g, xpm, NU), d = ld_at<IX>(p, g, xmn, NU);               \
    const Quat<float> e = ld_at<IX>(p, g, xmn, MU), f = ld_at<IX>(p, g, shifted<MU, +1>(g, xmn), NU); \
    qacc_mul_nd(s, qmul(a, b), c);                                                              \
    qacc_mul(s, qmul_dn(d, e), f);                                                              \
  }
  SU2_TERM(0)
  SU2_TERM(1)
  SU2_TERM(2)
  SU2_TERM(3)
#undef SU2_TERM
  return s;
}

template <class IX, int MU>
__global__ void __launch_bounds__(kThreads, 4) k_hb_plain(float4* p, Geom g, int par, const uint32_t* sweep_base,
                                                          uint32_t sweep_off, const __grid_constant__ HBParams hp) {
  const float beta = (float)hp.beta;
  const uint32_t sweep = *sweep_base + sweep_off;
  const uint32_t tag = (uint32_t)MU | hp.lattice_tag;
  const int stride = gridDim.x * blockDim.x;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < (int)g.vh; h += stride) {
    const Site x = site_from_half(g, (uint32_t)h, par);
    const Quat<float> sig = staple_at<IX, MU>(p, g, x);
    Quat<float> nl;
    const uint4 ctr = make_uint4(philox_site(g, x), tag, sweep, 0u);
    if (heatbath_draw<float>(sig, ctr, hp, beta, &nl) != 0) {
      const int64_t i = IX::at(g, x, MU);
      p[i] = make_float4(nl.w, nl.x, nl.y, nl.z);
    }
  }
}

__global__ void k_to_site_major(Links<kF32> L, Geom g, float4* out) {
  const int64_t V = 2 * g.vh;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 4 * V; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = w >> 2;
    const int mu = (int)(w & 3);
    const Site y = site_from_index(g, (uint32_t)s);
    const Quat<float> q = L.ld(2 * mu + parity(y), hidx(g, y));
    out[w] = make_float4(q.w, q.x, q.y, q.z);
  }
}

__global__ void k_from_site_major(Links<kF32> L, Geom g, const float4* in) {
  const int64_t V = 2 * g.vh;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 4 * V; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = w >> 2;
    const int mu = (int)(w & 3);
    const Site y = site_from_index(g, (uint32_t)s);
    const float4 a = in[w];
    L.st(2 * mu + parity(y), hidx(g, y), qmake<float>(a.x, a.y, a.z, a.w));
  }
}

__global__ void k_count_diff(const uint4* a, const uint4* b, int64_t n, unsigned long long* count) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 x = a[i], y = b[i];
    c += (x.x != y.x) | (x.y != y.y) | (x.z != y.z) | (x.w != y.w);
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

cudaError_t launch_hb_plain(const LatticeView& v, void* links, bool site_major, int mu, int parity,
                            const uint32_t* sweep_base, uint32_t sweep_off, const HBParams& hp, cudaStream_t st) {
  if (v.prec != kF32) return cudaErrorInvalidValue;
  float4* p = static_cast<float4*>(links);
  SU2_DISPATCH_MU(mu, {
    if (site_major) {
      const int gr = grid_for(k_hb_plain<SiteMajorIndex, MU>, v.g.vh);
      k_hb_plain<SiteMajorIndex, MU><<<gr, kThreads, 0, st>>>(p, v.g, parity, sweep_base, sweep_off, hp);
    } else {
      const int gr = grid_for(k_hb_plain<ClassIndex, MU>, v.g.vh);
      k_hb_plain<ClassIndex, MU><<<gr, kThreads, 0, st>>>(p, v.g, parity, sweep_base, sweep_off, hp);
    }
  });
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_site_major(const LatticeView& v, void* site_major, bool to_site_major, cudaStream_t st) {
  if (v.prec != kF32) return cudaErrorInvalidValue;
  auto L = links_of<kF32>(v.links, v.g.vh);
  const int gr = grid_for(k_to_site_major, 8 * v.g.vh);
  if (to_site_major) k_to_site_major<<<gr, kThreads, 0, st>>>(L, v.g, static_cast<float4*>(site_major));
  else k_from_site_major<<<gr, kThreads, 0, st>>>(L, v.g, static_cast<const float4*>(site_major));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_count_diff(const void* a, const void* b, size_t bytes, unsigned long long* count,
                              cudaStream_t st) {
  const int64_t n = (int64_t)(bytes / 16);
  const int gr = grid_for(k_count_diff, n);
  k_count_diff<<<gr, kThreads, 0, st>>>(static_cast<const uint4*>(a), static_cast<const uint4*>(b), n, count);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace su2
