// Device building blocks for the SU(2) heat bath on sm_103a: quaternion
// algebra, the Philox4x32-10 counter-based generator, the a0 samplers, the
// structure-of-arrays link store and the checkerboard geometry.
//
// Paper: Cardoso & Bicudo, arXiv:1010.4834.  Section 2 (Eqs. 1-9, 11) defines
// the link parametrisation and the heat-bath distribution; Section 4 the
// checkerboard ("separately by direction and by even and odd sites").
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace su2 {

// ---------------------------------------------------------------------------
// Precision tags.  Arithmetic is FP64 for F64 and FP32 for F32 / F16Q.
// ---------------------------------------------------------------------------
enum Prec { kF64 = 0, kF32 = 1, kF16Q = 2 };

template <int P> struct Real { using T = float; };
template <> struct Real<kF64> { using T = double; };

// Bytes of one stored link.
__host__ __device__ constexpr int link_bytes(int p) { return p == kF64 ? 32 : (p == kF32 ? 16 : 8); }

// ---------------------------------------------------------------------------
// Quaternion q0 1 + i (q1 s1 + q2 s2 + q3 s3)  (Section 2, Eq. 1).
// Product: (ab)_0 = a0 b0 - a.b ; (ab)_v = a0 b + b0 a - a x b.
// ---------------------------------------------------------------------------
template <class R> struct Quat { R w, x, y, z; };

template <class R> __device__ __forceinline__ Quat<R> qmake(R w, R x, R y, R z) {
  Quat<R> q; q.w = w; q.x = x; q.y = y; q.z = z; return q;
}

template <class R> __device__ __forceinline__ Quat<R> qmul(const Quat<R>& a, const Quat<R>& b) {
  Quat<R> r;
  r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
  r.x = a.w * b.x + a.x * b.w - a.y * b.z + a.z * b.y;
  r.y = a.w * b.y + a.y * b.w - a.z * b.x + a.x * b.z;
  r.z = a.w * b.z + a.z * b.w - a.x * b.y + a.y * b.x;
  return r;
}

// a b^dagger
template <class R> __device__ __forceinline__ Quat<R> qmul_nd(const Quat<R>& a, const Quat<R>& b) {
  Quat<R> r;
  r.w = a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z;
  r.x = -a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
  r.y = -a.w * b.y + a.y * b.w + a.z * b.x - a.x * b.z;
  r.z = -a.w * b.z + a.z * b.w + a.x * b.y - a.y * b.x;
  return r;
}

// a^dagger b
template <class R> __device__ __forceinline__ Quat<R> qmul_dn(const Quat<R>& a, const Quat<R>& b) {
  Quat<R> r;
  r.w = a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z;
  r.x = a.w * b.x - a.x * b.w + a.y * b.z - a.z * b.y;
  r.y = a.w * b.y - a.y * b.w + a.z * b.x - a.x * b.z;
  r.z = a.w * b.z - a.z * b.w + a.x * b.y - a.y * b.x;
  return r;
}

template <class R> __device__ __forceinline__ R qdot(const Quat<R>& a, const Quat<R>& b) {
  return a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z;
}

template <class R> __device__ __forceinline__ void qacc(Quat<R>& a, const Quat<R>& b) {
  a.w += b.w; a.x += b.x; a.y += b.y; a.z += b.z;
}

template <class R> __device__ __forceinline__ Quat<R> qscale(const Quat<R>& a, R s) {
  return qmake<R>(a.w * s, a.x * s, a.y * s, a.z * s);
}

template <class R> __device__ __forceinline__ Quat<R> qone() { return qmake<R>(1, 0, 0, 0); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Each round multiplies
// counter words 0 and 2 by the round multipliers into 64-bit products, XORs
// the high halves with the odd words and the round key, and permutes; the key
// advances by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct PhiloxKey { uint32_t k0, k1; };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey key) {
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t m0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t m1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t nx = (uint32_t)(m1 >> 32) ^ c.y ^ k0;
    const uint32_t nz = (uint32_t)(m0 >> 32) ^ c.w ^ k1;
    c.y = (uint32_t)m1;
    c.w = (uint32_t)m0;
    c.x = nx;
    c.z = nz;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// uint32 -> uniform in (0,1).  FP64: (x + 1/2) 2^-32, exact.  FP32:
// ((x >> 9) + 1/2) 2^-23, exact in binary32 (23-bit resolution keeps the
// value strictly below 1).
__device__ __forceinline__ double u01d(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }
__device__ __forceinline__ float u01f(uint32_t x) { return ((float)(x >> 9) + 0.5f) * 0x1p-23f; }

template <class R> __device__ __forceinline__ R u01(uint32_t x);
template <> __device__ __forceinline__ double u01<double>(uint32_t x) { return u01d(x); }
template <> __device__ __forceinline__ float u01<float>(uint32_t x) { return u01f(x); }

// Transcendentals per precision (library calls, no hand-written math).
__device__ __forceinline__ double rlog(double v) { return log(v); }
__device__ __forceinline__ float rlog(float v) { return logf(v); }
__device__ __forceinline__ double sqrt_r(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_r(float v) { return sqrtf(v); }
__device__ __forceinline__ void rsincospi(double v, double* s, double* c) { sincospi(v, s, c); }
__device__ __forceinline__ void rsincospi(float v, float* s, float* c) { sincospif(v, s, c); }
__device__ __forceinline__ double rcospi(double v) { return cospi(v); }
__device__ __forceinline__ float rcospi(float v) { return cospif(v); }
__device__ __forceinline__ double rexp(double v) { return exp(v); }
__device__ __forceinline__ float rexp(float v) { return expf(v); }
__device__ __forceinline__ double rmax0(double v) { return fmax(v, 0.0); }
__device__ __forceinline__ float rmax0(float v) { return fmaxf(v, 0.0f); }

// Uniformly random unit quaternion (Haar measure, Section 2 Eq. 4) from four
// uniforms: two Box-Muller pairs give four normals, normalised onto S^3.
template <class R> __device__ __forceinline__ Quat<R> haar_from(uint4 r) {
  const R u0 = u01<R>(r.x), u1 = u01<R>(r.y), u2 = u01<R>(r.z), u3 = u01<R>(r.w);
  const R a = sqrt_r(R(-2) * rlog(u0));
  const R b = sqrt_r(R(-2) * rlog(u2));
  R s1, c1, s3, c3;
  rsincospi(R(2) * u1, &s1, &c1);
  rsincospi(R(2) * u3, &s3, &c3);
  Quat<R> z = qmake<R>(a * c1, a * s1, b * c3, b * s3);
  const R inv = R(1) / sqrt_r(qdot(z, z));
  return qscale(z, inv);
}

// ---------------------------------------------------------------------------
// Heat-bath parameters shared by a launch.
// ---------------------------------------------------------------------------
struct HBParams {
  double beta;
  PhiloxKey key;
  uint32_t lattice_tag;  // lattice_id << 2 (ORed with mu in counter word 1)
  int max_tries;
  int sampler;           // 0 Kennedy-Pendleton, 1 Creutz
};

// Sampled a0 (Section 2, Eq. 8) for alpha = beta k.  Trial n = 1..max_tries
// uses Philox draw n of this link.  Returns the trial that accepted, 0 if none.
//   Kennedy-Pendleton: delta = -(ln u0 + cos^2(2 pi u1) ln u2) / (2 alpha),
//                      accept if u3^2 <= 1 - delta, a0 = 1 - 2 delta.
//   Creutz:            a0 = 1 + ln(e^{-2 alpha} + (1 - e^{-2 alpha}) u0)/alpha,
//                      accept if u1^2 <= 1 - a0^2.
template <class R>
__device__ __forceinline__ int sample_a0(R alpha, uint4 ctr, PhiloxKey key, int max_tries,
                                         int sampler, R* a0) {
  const R inv2a = R(0.5) / alpha;
  const R e = sampler ? rexp(R(-2) * alpha) : R(0);
  for (int n = 1; n <= max_tries; ++n) {
    ctr.w = (uint32_t)n;
    const uint4 r = philox4x32_10(ctr, key);
    if (sampler == 0) {
      const R u0 = u01<R>(r.x), u1 = u01<R>(r.y), u2 = u01<R>(r.z), u3 = u01<R>(r.w);
      const R c = rcospi(R(2) * u1);
      const R delta = -(rlog(u0) + c * c * rlog(u2)) * inv2a;
      if (u3 * u3 <= R(1) - delta) { *a0 = R(1) - R(2) * delta; return n; }
    } else {
      const R u0 = u01<R>(r.x), u1 = u01<R>(r.y);
      const R cand = R(1) + rlog(e + (R(1) - e) * u0) / alpha;
      if (u1 * u1 <= R(1) - cand * cand) { *a0 = cand; return n; }
    }
  }
  return 0;
}

// Full heat-bath draw for one link given its staple sum (Section 2, Eqs. 5-9):
// X with x0 = a0 and uniform direction (Philox draw 0), new link X * Sigma / k.
// alpha < 1e-12: Haar link from draw 1.  `ctr` holds (site, mu | lattice_tag,
// sweep, -).  Returns trials used; 0 means every trial failed, `out` is not
// written and the caller keeps the old link; -1 marks the Haar branch.
template <class R>
__device__ __forceinline__ int heatbath_draw(const Quat<R>& sigma, uint4 ctr, const HBParams& hp,
                                             R beta, Quat<R>* out) {
  const R k2 = qdot(sigma, sigma);
  const R k = sqrt_r(k2);
  const R alpha = beta * k;
  if (!(alpha >= R(1e-12))) {
    ctr.w = 1u;
    *out = haar_from<R>(philox4x32_10(ctr, hp.key));
    return -1;
  }
  R a0;
  const int n = sample_a0<R>(alpha, ctr, hp.key, hp.max_tries, hp.sampler, &a0);
  if (n == 0) return 0;
  ctr.w = 0u;
  const uint4 r = philox4x32_10(ctr, hp.key);
  const R cos_t = R(2) * u01<R>(r.x) - R(1);
  const R sin_t = sqrt_r(rmax0(R(1) - cos_t * cos_t));
  R sp, cp;
  rsincospi(R(2) * u01<R>(r.y), &sp, &cp);
  const R rad = sqrt_r(rmax0(R(1) - a0 * a0));
  const Quat<R> x = qmake<R>(a0, rad * sin_t * cp, rad * sin_t * sp, rad * cos_t);
  const R invk = R(1) / k;
  *out = qmul(x, qscale(sigma, invk));
  return n;
}

// ---------------------------------------------------------------------------
// Link store: structure of arrays.  Class c = 2 mu + parity holds the V/2
// links of direction mu on sites of that parity, ordered by s >> 1.
// ---------------------------------------------------------------------------
template <int P> struct Links;

// ld() reads through the read-only path (valid while no thread of the same
// kernel writes the element); ldc() is a plain coherent load for kernels that
// write links other blocks read after a grid barrier.
template <> struct Links<kF64> {
  double2* p;     // 2 double2 per link
  int64_t vh;     // links per class
  __device__ __forceinline__ Quat<double> ld(int cls, int64_t i) const {
    const double2* q = p + 2 * (cls * vh + i);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    return qmake<double>(a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ Quat<double> ldc(int cls, int64_t i) const {
    const double2* q = p + 2 * (cls * vh + i);
    const double2 a = q[0], b = q[1];
    return qmake<double>(a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ void st(int cls, int64_t i, const Quat<double>& v) const {
    double2* q = p + 2 * (cls * vh + i);
    q[0] = make_double2(v.w, v.x);
    q[1] = make_double2(v.y, v.z);
  }
};

template <> struct Links<kF32> {
  float4* p;
  int64_t vh;
  __device__ __forceinline__ Quat<float> ld(int cls, int64_t i) const {
    const float4 a = __ldg(p + cls * vh + i);
    return qmake<float>(a.x, a.y, a.z, a.w);
  }
  __device__ __forceinline__ Quat<float> ldc(int cls, int64_t i) const {
    const float4 a = p[cls * vh + i];
    return qmake<float>(a.x, a.y, a.z, a.w);
  }
  __device__ __forceinline__ void st(int cls, int64_t i, const Quat<float>& v) const {
    p[cls * vh + i] = make_float4(v.w, v.x, v.y, v.z);
  }
};

// binary16 quaternion, re-normalised in FP32 on every load.
template <> struct Links<kF16Q> {
  uint2* p;
  int64_t vh;
  __device__ __forceinline__ Quat<float> ld(int cls, int64_t i) const { return unpack(__ldg(p + cls * vh + i)); }
  __device__ __forceinline__ Quat<float> ldc(int cls, int64_t i) const { return unpack(p[cls * vh + i]); }
  static __device__ __forceinline__ Quat<float> unpack(const uint2 a) {
    const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
    Quat<float> q = qmake<float>(lo.x, lo.y, hi.x, hi.y);
    const float inv = rsqrtf(qdot(q, q));
    return qscale(q, inv);
  }
  __device__ __forceinline__ void st(int cls, int64_t i, const Quat<float>& v) const {
    const __half2 lo = __floats2half2_rn(v.w, v.x);
    const __half2 hi = __floats2half2_rn(v.y, v.z);
    uint2 a;
    a.x = *reinterpret_cast<const uint32_t*>(&lo);
    a.y = *reinterpret_cast<const uint32_t*>(&hi);
    p[cls * vh + i] = a;
  }
};

// ---------------------------------------------------------------------------
// Division by a runtime-invariant divisor with one multiply-high (Granlund &
// Montgomery, "Division by invariant integers using multiplication", PLDI'94):
// for d >= 1, l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(m, n) + n) >> l for 0 <= n < 2^31.
// ---------------------------------------------------------------------------
struct FastDiv {
  uint32_t d, m, l;
  FastDiv() = default;
  __host__ explicit FastDiv(uint32_t div) : d(div) {
    l = 0;
    while ((1ull << l) < div) ++l;
    m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    return (uint32_t)(((uint64_t)__umulhi(m, n) + n) >> l);
  }
};

// Checkerboard geometry of one lattice.
struct Geom {
  int n[4];         // extents
  int n0h;          // n[0] / 2
  int64_t vh;       // V / 2
  FastDiv f_n0h, f_n1, f_n2, f_n0;
};

// Half-site index of (x0..x3): (x0 >> 1) + n0h (x1 + n1 (x2 + n2 x3)).
__device__ __forceinline__ int64_t hidx(const Geom& g, int x0, int x1, int x2, int x3) {
  return (int64_t)(x0 >> 1) + (int64_t)g.n0h * (x1 + g.n[1] * (x2 + g.n[2] * (int64_t)x3));
}

__device__ __forceinline__ int wrap_inc(int x, int n) { return x + 1 == n ? 0 : x + 1; }
__device__ __forceinline__ int wrap_dec(int x, int n) { return x == 0 ? n - 1 : x - 1; }

// Coordinates of half-site h on the parity-p sublattice.
__device__ __forceinline__ void decode_half(const Geom& g, uint32_t h, int p, int x[4]) {
  const uint32_t row = g.f_n0h.div(h);
  const int xh = (int)(h - row * (uint32_t)g.n0h);
  const uint32_t r2 = g.f_n1.div(row);
  x[1] = (int)(row - r2 * (uint32_t)g.n[1]);
  const uint32_t r3 = g.f_n2.div(r2);
  x[2] = (int)(r2 - r3 * (uint32_t)g.n[2]);
  x[3] = (int)r3;
  x[0] = 2 * xh + ((x[1] + x[2] + x[3] + p) & 1);
}

// Coordinates of full site s.
__device__ __forceinline__ void decode_site(const Geom& g, uint32_t s, int x[4]) {
  const uint32_t r1 = g.f_n0.div(s);
  x[0] = (int)(s - r1 * (uint32_t)g.n[0]);
  const uint32_t r2 = g.f_n1.div(r1);
  x[1] = (int)(r1 - r2 * (uint32_t)g.n[1]);
  const uint32_t r3 = g.f_n2.div(r2);
  x[2] = (int)(r2 - r3 * (uint32_t)g.n[2]);
  x[3] = (int)r3;
}

__device__ __forceinline__ uint32_t site_of(const Geom& g, const int x[4]) {
  return (uint32_t)(x[0] + g.n[0] * (x[1] + g.n[1] * (x[2] + g.n[2] * x[3])));
}

// Half-site index of x shifted by +-1 along d (periodic).
__device__ __forceinline__ int64_t hidx_shift(const Geom& g, const int x[4], int d, int step) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[d] = step > 0 ? wrap_inc(y[d], g.n[d]) : wrap_dec(y[d], g.n[d]);
  return hidx(g, y[0], y[1], y[2], y[3]);
}

// Half-site index of x - nu + mu.
__device__ __forceinline__ int64_t hidx_mp(const Geom& g, const int x[4], int nu, int mu) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[nu] = wrap_dec(y[nu], g.n[nu]);
  y[mu] = wrap_inc(y[mu], g.n[mu]);
  return hidx(g, y[0], y[1], y[2], y[3]);
}

// Staple sum of Section 2 Eq. 11 for link (x, mu), x of parity p with
// half-index h: for nu != mu, U_nu(x) U_mu(x+nu) U_nu(x+mu)^dagger +
// U_nu(x-nu)^dagger U_mu(x-nu) U_nu(x-nu+mu).  Classes: U_nu(x) and
// U_nu(x-nu+mu) have parity p; the four shifted links have parity 1-p.
// `nmask` selects which nu contribute (all nu != mu for the heat bath; the
// spatial ones for APE).
template <int P, bool NC = true>
__device__ __forceinline__ Quat<typename Real<P>::T> staple(const Links<P>& L, const Geom& g,
                                                           const int x[4], int64_t h, int mu,
                                                           int p, int nmask) {
  using R = typename Real<P>::T;
  Quat<R> s = qmake<R>(0, 0, 0, 0);
  const int q = p ^ 1;
  const int64_t h_pmu = hidx_shift(g, x, mu, +1);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu || !((nmask >> nu) & 1)) continue;
    const int64_t h_pnu = hidx_shift(g, x, nu, +1);
    const int64_t h_mnu = hidx_shift(g, x, nu, -1);
    const int64_t h_mp = hidx_mp(g, x, nu, mu);
    const Quat<R> a = NC ? L.ld(2 * nu + p, h) : L.ldc(2 * nu + p, h);              // U_nu(x)
    const Quat<R> b = NC ? L.ld(2 * mu + q, h_pnu) : L.ldc(2 * mu + q, h_pnu);      // U_mu(x+nu)
    const Quat<R> c = NC ? L.ld(2 * nu + q, h_pmu) : L.ldc(2 * nu + q, h_pmu);      // U_nu(x+mu)
    const Quat<R> d = NC ? L.ld(2 * nu + q, h_mnu) : L.ldc(2 * nu + q, h_mnu);      // U_nu(x-nu)
    const Quat<R> e = NC ? L.ld(2 * mu + q, h_mnu) : L.ldc(2 * mu + q, h_mnu);      // U_mu(x-nu)
    const Quat<R> f = NC ? L.ld(2 * nu + p, h_mp) : L.ldc(2 * nu + p, h_mp);        // U_nu(x-nu+mu)
    qacc(s, qmul_nd(qmul(a, b), c));
    qacc(s, qmul(qmul_dn(d, e), f));
  }
  return s;
}

}  // namespace su2
