// Device building blocks for the SU(2) heat bath on sm_103a: quaternion
// algebra, the Philox4x32-10 counter-based generator, the a0 samplers, the
// structure-of-arrays link store and the checkerboard geometry.
//
// Paper: Cardoso & Bicudo, arXiv:1010.4834.  Section 2 (Eqs. 1-9, 11) defines
// the link parametrisation and the heat-bath distribution; Section 4 the
// checkerboard order (one direction and one site parity at a time).
//
// Coordinates are kept in scalars and every lattice shift names its direction
// at compile time, so no coordinate array is ever indexed at run time (which
// would put it in local memory).
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

// s += a b^dagger and s += a b, each component one chain of fused multiply-adds.
template <class R> __device__ __forceinline__ void qacc_mul_nd(Quat<R>& s, const Quat<R>& a, const Quat<R>& b) {
  s.w = fma(a.w, b.w, fma(a.x, b.x, fma(a.y, b.y, fma(a.z, b.z, s.w))));
  s.x = fma(-a.w, b.x, fma(a.x, b.w, fma(a.y, b.z, fma(-a.z, b.y, s.x))));
  s.y = fma(-a.w, b.y, fma(a.y, b.w, fma(a.z, b.x, fma(-a.x, b.z, s.y))));
  s.z = fma(-a.w, b.z, fma(a.z, b.w, fma(a.x, b.y, fma(-a.y, b.x, s.z))));
}

template <class R> __device__ __forceinline__ void qacc_mul(Quat<R>& s, const Quat<R>& a, const Quat<R>& b) {
  s.w = fma(a.w, b.w, fma(-a.x, b.x, fma(-a.y, b.y, fma(-a.z, b.z, s.w))));
  s.x = fma(a.w, b.x, fma(a.x, b.w, fma(-a.y, b.z, fma(a.z, b.y, s.x))));
  s.y = fma(a.w, b.y, fma(a.y, b.w, fma(-a.z, b.x, fma(a.x, b.z, s.y))));
  s.z = fma(a.w, b.z, fma(a.z, b.w, fma(-a.x, b.y, fma(a.y, b.x, s.z))));
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
// advances by the Weyl increments between rounds.  The ten round keys depend
// only on the seed, so the host computes them once and the kernels read them
// from their (constant-bank) parameters.
// ---------------------------------------------------------------------------
struct PhiloxKey { uint32_t k0, k1; };

struct RoundKeys {
  uint32_t k0[10], k1[10];
};

__host__ __device__ inline RoundKeys round_keys(PhiloxKey key) {
  RoundKeys rk;
  uint32_t a = key.k0, b = key.k1;
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = a;
    rk.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return rk;
}

// The round's 32x32 -> 64-bit products as separate high and low multiplies
// (the same bits; measured 0.7% faster in the heat-bath substep than one
// widening multiply).
#ifndef SU2_PHILOX_HILO
#define SU2_PHILOX_HILO 1
#endif
__device__ __forceinline__ uint4 philox(uint4 c, const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#if SU2_PHILOX_HILO
    // the 64-bit products as separate high and low 32-bit multiplies
    const uint32_t h0 = __umulhi(0xD2511F53u, c.x), l0 = 0xD2511F53u * c.x;
    const uint32_t h1 = __umulhi(0xCD9E8D57u, c.z), l1 = 0xCD9E8D57u * c.z;
#else
    const uint64_t m0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t m1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t h0 = (uint32_t)(m0 >> 32), l0 = (uint32_t)m0;
    const uint32_t h1 = (uint32_t)(m1 >> 32), l1 = (uint32_t)m1;
#endif
    const uint32_t nx = h1 ^ c.y ^ rk.k0[r];
    const uint32_t nz = h0 ^ c.w ^ rk.k1[r];
    c.y = l1;
    c.w = l0;
    c.x = nx;
    c.z = nz;
  }
  return c;
}

// uint32 -> uniform in (0,1).  FP64: (x + 1/2) 2^-32, exact.  FP32:
// ((x >> 9) + 1/2) 2^-23, exact in binary32 (23-bit resolution keeps the
// value strictly below 1).  The FP32 value is built without an int-to-float
// conversion: the bit pattern 0x3F800000 | (x >> 9) is 1 + k 2^-23 with
// k = x >> 9, and subtracting 1 - 2^-24 (the largest float below 1) gives
// (k + 1/2) 2^-23 in one exact subtraction (the operands are within a factor
// of two of each other, and the difference needs 24 significant bits).
template <class R> __device__ __forceinline__ R u01(uint32_t x);
template <> __device__ __forceinline__ double u01<double>(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }
template <> __device__ __forceinline__ float u01<float>(uint32_t x) {
  return __uint_as_float(0x3F800000u | (x >> 9)) - 0x1.fffffep-1f;
}

// ---------------------------------------------------------------------------
// Math policy.  FP64 calls the accurate CUDA functions (the FP64 path is the
// one compared link by link with the oracle).  FP32 uses the SFU
// approximations where their error (a few 1e-7) is below the FP32 resolution
// of the result: log (max abs error 2^-21.4 on [0.5, 2], 3 ulp elsewhere),
// sin/cos of an argument reduced to [-pi, pi] by cos(2 pi u) =
// -cos(2 pi (u - 1/2)), reciprocal square root; the Box-Muller radius keeps the
// accurate logf, because there ln(u) -> 0 as u -> 1 and an absolute error
// would dominate it.
// ---------------------------------------------------------------------------
template <class R> struct Math;

template <> struct Math<double> {
  static __device__ __forceinline__ double log_fast(double v) { return log(v); }
  static __device__ __forceinline__ double log_acc(double v) { return log(v); }
  static __device__ __forceinline__ double cos2pi(double u) { return cospi(2.0 * u); }
  static __device__ __forceinline__ void sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
  static __device__ __forceinline__ double sqrt0(double v) { return sqrt(fmax(v, 0.0)); }
  static __device__ __forceinline__ double rsqrt(double v) { return 1.0 / sqrt(v); }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double exp(double v) { return ::exp(v); }
  static constexpr double kTiny = 1e-300;
};

template <> struct Math<float> {
  static __device__ __forceinline__ float log_fast(float v) { return __logf(v); }
  static __device__ __forceinline__ float log_acc(float v) { return logf(v); }
  static __device__ __forceinline__ float cos2pi(float u) {
    return -__cosf(6.28318530717958647692f * (u - 0.5f));
  }
  static __device__ __forceinline__ void sincos2pi(float u, float* s, float* c) {
    float ss, cc;
    __sincosf(6.28318530717958647692f * (u - 0.5f), &ss, &cc);
    *s = -ss;
    *c = -cc;
  }
  static __device__ __forceinline__ float sqrt0(float v) {
    v = fmaxf(v, 0.0f);
    return v * rsqrtf(fmaxf(v, 1e-30f));
  }
  static __device__ __forceinline__ float rsqrt(float v) { return rsqrtf(v); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float exp(float v) { return __expf(v); }
  static constexpr float kTiny = 1e-30f;
};

// Uniformly random unit quaternion (Haar measure, Section 2 Eq. 4) from four
// uniforms: two Box-Muller pairs give four normals, normalised onto S^3.
template <class R> __device__ __forceinline__ Quat<R> haar_from(uint4 r) {
  using M = Math<R>;
  const R u0 = u01<R>(r.x), u1 = u01<R>(r.y), u2 = u01<R>(r.z), u3 = u01<R>(r.w);
  const R a = M::sqrt0(R(-2) * M::log_acc(u0));
  const R b = M::sqrt0(R(-2) * M::log_acc(u2));
  R s1, c1, s3, c3;
  M::sincos2pi(u1, &s1, &c1);
  M::sincos2pi(u3, &s3, &c3);
  Quat<R> z = qmake<R>(a * c1, a * s1, b * c3, b * s3);
  return qscale(z, M::rsqrt(qdot(z, z)));
}

// ---------------------------------------------------------------------------
// Heat-bath parameters shared by a launch (passed as a __grid_constant__
// kernel parameter).
// ---------------------------------------------------------------------------
struct HBParams {
  double beta;
  RoundKeys rk;
  uint32_t lattice_tag;  // lattice_id << 2 (ORed with mu in counter word 1)
  int max_tries;
  int sampler;           // 0 Kennedy-Pendleton, 1 Creutz
};

// One trial n of the a0 draw (Section 2, Eq. 8) for alpha = beta k, using
// Philox draw n of this link; inv2a = 1/(2 alpha), e = exp(-2 alpha) (Creutz).
//   Kennedy-Pendleton: delta = -(ln u0 + cos^2(2 pi u1) ln u2) / (2 alpha),
//                      accept if u3^2 <= 1 - delta, a0 = 1 - 2 delta.
//   Creutz:            a0 = 1 + ln(e^{-2 alpha} + (1 - e^{-2 alpha}) u0)/alpha,
//                      accept if u1^2 <= 1 - a0^2.
// *rt receives the draw's four Philox words (compose_link reads the FP32
// direction from them).
template <class R>
__device__ __forceinline__ bool trial_a0(R alpha, R inv2a, R e, uint4 ctr, int n, const HBParams& hp, R* a0,
                                         uint4* rt) {
  using M = Math<R>;
  ctr.w = (uint32_t)n;
  const uint4 r = philox(ctr, hp.rk);
  *rt = r;
  if (hp.sampler == 0) {
    const R u0 = u01<R>(r.x), u1 = u01<R>(r.y), u2 = u01<R>(r.z), u3 = u01<R>(r.w);
    const R c = M::cos2pi(u1);
    const R delta = -(M::log_fast(u0) + c * c * M::log_fast(u2)) * inv2a;
    if (u3 * u3 <= R(1) - delta) { *a0 = R(1) - R(2) * delta; return true; }
  } else {
    const R u0 = u01<R>(r.x), u1 = u01<R>(r.y);
    const R cand = R(1) + M::div(M::log_fast(e + (R(1) - e) * u0), alpha);
    if (u1 * u1 <= R(1) - cand * cand) { *a0 = cand; return true; }
  }
  return false;
}

// The per-link constants of the trials.
template <class R> __device__ __forceinline__ R trial_inv2a(R alpha) { return Math<R>::div(R(0.5), alpha); }
template <class R> __device__ __forceinline__ R trial_e(R alpha, int sampler) {
  return sampler ? Math<R>::exp(R(-2) * alpha) : R(0);
}

// Trials first..max_tries; returns the trial that accepted, 0 if none; *rt
// holds the accepting trial's Philox words.
template <class R>
__device__ __forceinline__ int sample_a0_from(int first, R alpha, R inv2a, R e, uint4 ctr, const HBParams& hp, R* a0,
                                              uint4* rt) {
  for (int n = first; n <= hp.max_tries; ++n)
    if (trial_a0<R>(alpha, inv2a, e, ctr, n, hp, a0, rt)) return n;
  return 0;
}

// The direction of the accepted link (Section 2, Eqs. 7, 9): a uniform point
// (cos theta, phi) of the unit 2-sphere.
//   FP64: Philox draw 0 of the link, cos theta = 2 u0 - 1, phi = 2 pi u1.
//   FP32: the nine low bits of each word of the accepting trial's draw, which
//         its 23-bit uniforms leave unused: c = (x mod 2^9) 2^9 + y mod 2^9 and
//         f = (z mod 2^9) 2^9 + w mod 2^9 (18 bits each, independent of the
//         trial's uniforms), cos theta = (2c + 1) 2^-18 - 1 and
//         phi = 2 pi (f + 1/2) 2^-18; one Philox block per accepted trial
//         instead of two (the 64^4 FP32 substep 187.6 -> 179.2 us).
template <class R> __device__ __forceinline__ void link_direction(uint4 ctr, uint4 rt, const HBParams& hp, R* cos_t,
                                                                   R* sp, R* cp) {
  using M = Math<R>;
  if constexpr (sizeof(R) == 4) {
    const uint32_t c = ((rt.x & 0x1FFu) << 9) | (rt.y & 0x1FFu);
    const uint32_t f = ((rt.z & 0x1FFu) << 9) | (rt.w & 0x1FFu);
    *cos_t = fmaf((float)(2u * c + 1u), 0x1p-18f, -1.0f);   // exact: 19 significant bits
    M::sincos2pi(fmaf((float)f, 0x1p-18f, 0x1p-19f), sp, cp);
  } else {
    ctr.w = 0u;
    const uint4 r = philox(ctr, hp.rk);
    *cos_t = R(2) * u01<R>(r.x) - R(1);
    M::sincos2pi(u01<R>(r.y), sp, cp);
  }
}

// The accepted link (Section 2, Eqs. 7, 9): X with x0 = a0 and the direction
// of link_direction, times W = Sigma / k.  rt: the accepting trial's words.
template <class R>
__device__ __forceinline__ Quat<R> compose_link(R a0, const Quat<R>& w, uint4 ctr, uint4 rt, const HBParams& hp) {
  using M = Math<R>;
  R cos_t, sp, cp;
  link_direction<R>(ctr, rt, hp, &cos_t, &sp, &cp);
  const R sin_t = M::sqrt0(R(1) - cos_t * cos_t);
  const R rad = M::sqrt0(R(1) - a0 * a0);
  const Quat<R> x = qmake<R>(a0, rad * sin_t * cp, rad * sin_t * sp, rad * cos_t);
  return qmul(x, w);
}

// Full heat-bath draw for one link given its staple sum (Section 2, Eqs. 5-9).
// alpha < 1e-12: Haar link from draw 1.  `ctr` holds (site, mu | lattice_tag,
// sweep, -).  Returns trials used; 0 means every trial failed, `out` is not
// written and the caller keeps the old link; -1 marks the Haar branch.
template <class R>
__device__ __forceinline__ int heatbath_draw(const Quat<R>& sigma, uint4 ctr, const HBParams& hp,
                                             R beta, Quat<R>* out) {
  using M = Math<R>;
  const R k2 = qdot(sigma, sigma);
  const R invk = M::rsqrt(k2);
  const R alpha = beta * k2 * invk;
  if (!(alpha >= R(1e-12))) {
    ctr.w = 1u;
    *out = haar_from<R>(philox(ctr, hp.rk));
    return -1;
  }
  R a0;
  uint4 rt;
  const int n = sample_a0_from<R>(1, alpha, trial_inv2a(alpha), trial_e(alpha, hp.sampler), ctr, hp, &a0, &rt);
  if (n == 0) return 0;
  *out = compose_link<R>(a0, qscale(sigma, invk), ctr, rt, hp);
  return n;
}

// ---------------------------------------------------------------------------
// Link store: structure of arrays.  Class c = 2 mu + parity holds the V/2
// links of direction mu on sites of that parity, ordered by s >> 1.
// ld() reads through the read-only path (valid while no thread of the same
// kernel writes the element); ldc() is a plain coherent load for kernels that
// write links other blocks read after a grid barrier.
// ---------------------------------------------------------------------------
// CP selects the addressing:
//   kFlat      class cls starts at p + cls * vh;
//   kClassPtr  a class starts at its own base pointer c[cls] (kernel
//              parameters), so a load is one multiply-add of the 32-bit
//              element index onto a constant;
//   kClassOff  link i of class cls is element o[cls] + i of one base p, with
//              32-bit offsets o[cls] = cls * vh (only while 8 vh < 2^32): one
//              64-bit base in registers for all classes; 64-lattice batch
//              40.6 -> 41.9 G updates/s against kClassPtr.
// The last two are for kernels in which every class index is a compile-time
// constant (a runtime index into c[] or o[] would put the array into local
// memory).
enum AddrMode { kFlat = 0, kClassPtr = 1, kClassOff = 2 };
template <int P, int CP = kFlat> struct Links;

template <int CP> struct Links<kF64, CP> {
  using E = double2;
  double2* p;     // 2 double2 per link
  int64_t vh;     // links per class
  double2* c[8];  // start of each class (filled by set())
  uint32_t o[8];  // link offset of each class from p (kClassOff)
  // start of class cls, and link i of the class that starts at b
  __device__ __forceinline__ double2* cls_base(int cls) const {
    if constexpr (CP == kClassPtr) return c[cls];
    else return p + 2 * cls * vh;
  }
  static __device__ __forceinline__ Quat<double> ldp(const double2* b, uint32_t i) {
    const double2 a = __ldg(b + 2 * i), d = __ldg(b + 2 * i + 1);
    return qmake<double>(a.x, a.y, d.x, d.y);
  }
  __host__ __device__ void set(void* base, int64_t n) {
    p = static_cast<double2*>(base);
    vh = n;
    for (int k = 0; k < 8; ++k) {
      c[k] = p + 2 * k * n;
      o[k] = (uint32_t)(k * n);
    }
  }
  __device__ __forceinline__ double2* at(int cls, int i) const {
    if constexpr (CP == kClassOff) return p + 2 * (uint64_t)(uint32_t)(o[cls] + (uint32_t)i);
    else if constexpr (CP == kClassPtr) return c[cls] + 2 * (uint32_t)i;
    else return p + 2 * (cls * vh + (uint32_t)i);
  }
  __device__ __forceinline__ Quat<double> ld(int cls, int i) const {
    const double2* q = at(cls, i);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    return qmake<double>(a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ Quat<double> ldc(int cls, int i) const {
    const double2* q = at(cls, i);
    const double2 a = q[0], b = q[1];
    return qmake<double>(a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ Quat<double> ldcg(int cls, int i) const {
    const double2* q = at(cls, i);
    const double2 a = __ldcg(q), b = __ldcg(q + 1);
    return qmake<double>(a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ void st(int cls, int i, const Quat<double>& v) const {
    double2* q = at(cls, i);
    q[0] = make_double2(v.w, v.x);
    q[1] = make_double2(v.y, v.z);
  }
  // store v and return the value a later load of it returns
  __device__ __forceinline__ Quat<double> put(int cls, int i, const Quat<double>& v) const {
    st(cls, i, v);
    return v;
  }
};

template <int CP> struct Links<kF32, CP> {
  using E = float4;
  float4* p;
  int64_t vh;
  float4* c[8];
  uint32_t o[8];
  __device__ __forceinline__ float4* cls_base(int cls) const {
    if constexpr (CP == kClassPtr) return c[cls];
    else return p + cls * vh;
  }
  static __device__ __forceinline__ Quat<float> ldp(const float4* b, uint32_t i) {
    const float4 a = __ldg(b + i);
    return qmake<float>(a.x, a.y, a.z, a.w);
  }
  __host__ __device__ void set(void* base, int64_t n) {
    p = static_cast<float4*>(base);
    vh = n;
    for (int k = 0; k < 8; ++k) {
      c[k] = p + k * n;
      o[k] = (uint32_t)(k * n);
    }
  }
  __device__ __forceinline__ float4* at(int cls, int i) const {
    if constexpr (CP == kClassOff) return p + (uint32_t)(o[cls] + (uint32_t)i);
    else if constexpr (CP == kClassPtr) return c[cls] + (uint32_t)i;
    else return p + cls * vh + (uint32_t)i;
  }
  __device__ __forceinline__ Quat<float> ld(int cls, int i) const {
    const float4 a = __ldg(at(cls, i));
    return qmake<float>(a.x, a.y, a.z, a.w);
  }
  __device__ __forceinline__ Quat<float> ldc(int cls, int i) const {
    const float4 a = *at(cls, i);
    return qmake<float>(a.x, a.y, a.z, a.w);
  }
  __device__ __forceinline__ Quat<float> ldcg(int cls, int i) const {
    const float4 a = __ldcg(at(cls, i));
    return qmake<float>(a.x, a.y, a.z, a.w);
  }
  __device__ __forceinline__ void st(int cls, int i, const Quat<float>& v) const {
    *at(cls, i) = make_float4(v.w, v.x, v.y, v.z);
  }
  __device__ __forceinline__ Quat<float> put(int cls, int i, const Quat<float>& v) const {
    st(cls, i, v);
    return v;
  }
};

// binary16 quaternion, re-normalised in FP32 on every load.
template <int CP> struct Links<kF16Q, CP> {
  using E = uint2;
  uint2* p;
  int64_t vh;
  uint2* c[8];
  uint32_t o[8];
  __device__ __forceinline__ uint2* cls_base(int cls) const {
    if constexpr (CP == kClassPtr) return c[cls];
    else return p + cls * vh;
  }
  static __device__ __forceinline__ Quat<float> ldp(const uint2* b, uint32_t i) { return unpack(__ldg(b + i)); }
  __host__ __device__ void set(void* base, int64_t n) {
    p = static_cast<uint2*>(base);
    vh = n;
    for (int k = 0; k < 8; ++k) {
      c[k] = p + k * n;
      o[k] = (uint32_t)(k * n);
    }
  }
  __device__ __forceinline__ uint2* at(int cls, int i) const {
    if constexpr (CP == kClassOff) return p + (uint32_t)(o[cls] + (uint32_t)i);
    else if constexpr (CP == kClassPtr) return c[cls] + (uint32_t)i;
    else return p + cls * vh + (uint32_t)i;
  }
  __device__ __forceinline__ Quat<float> ld(int cls, int i) const { return unpack(__ldg(at(cls, i))); }
  __device__ __forceinline__ Quat<float> ldc(int cls, int i) const { return unpack(*at(cls, i)); }
  __device__ __forceinline__ Quat<float> ldcg(int cls, int i) const { return unpack(__ldcg(at(cls, i))); }
  // the stored binary16 components in FP32, not yet re-normalised
  static __device__ __forceinline__ Quat<float> unpack_raw(const uint2 a) {
    const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
    return qmake<float>(lo.x, lo.y, hi.x, hi.y);
  }
  static __device__ __forceinline__ Quat<float> unpack(const uint2 a) {
    const Quat<float> q = unpack_raw(a);
    return qscale(q, rsqrtf(qdot(q, q)));
  }
  __device__ __forceinline__ Quat<float> ld_raw(int cls, int i) const { return unpack_raw(__ldg(at(cls, i))); }
  __device__ __forceinline__ Quat<float> ldc_raw(int cls, int i) const { return unpack_raw(*at(cls, i)); }
  __device__ __forceinline__ Quat<float> ldcg_raw(int cls, int i) const { return unpack_raw(__ldcg(at(cls, i))); }
  static __device__ __forceinline__ uint2 pack(const Quat<float>& v) {
    const __half2 lo = __floats2half2_rn(v.w, v.x);
    const __half2 hi = __floats2half2_rn(v.y, v.z);
    uint2 a;
    a.x = *reinterpret_cast<const uint32_t*>(&lo);
    a.y = *reinterpret_cast<const uint32_t*>(&hi);
    return a;
  }
  __device__ __forceinline__ void st(int cls, int i, const Quat<float>& v) const { *at(cls, i) = pack(v); }
  // the stored value as a later load sees it: rounded to binary16, re-normalised
  __device__ __forceinline__ Quat<float> put(int cls, int i, const Quat<float>& v) const {
    const uint2 a = pack(v);
    *at(cls, i) = a;
    return unpack(a);
  }
};

template <int P, bool NC, int CP>
__device__ __forceinline__ Quat<typename Real<P>::T> ldl(const Links<P, CP>& L, int cls, int i) {
  return NC ? L.ld(cls, i) : L.ldc(cls, i);
}

// Loads of the staple's MU-direction links (the class of the other parity).
// With MCG they go through L2 only (ld.global.cg): in a kernel that writes
// that class earlier in the same launch (the fused parity pair), another
// SM's write is visible in L2 after its release, while an L1 line read
// before it could be stale.
template <int P, bool NC, bool MCG, int CP>
__device__ __forceinline__ Quat<typename Real<P>::T> ldmu(const Links<P, CP>& L, int cls, int i) {
  if constexpr (MCG) return L.ldcg(cls, i);
  else return ldl<P, NC>(L, cls, i);
}

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

// Checkerboard geometry of one lattice.  A site's "row" is
// x1 + n1 (x2 + n2 x3); its half-site index is (x0 >> 1) + n0h * row.
struct Geom {
  int n[4];         // extents
  int n0h;          // n[0] / 2
  int64_t vh;       // V / 2
  int st[4];        // row stride of a unit step in direction 1..3 (st[0] unused)
  int wr[4];        // st[d] * (n[d] - 1): row change of a wrapping step
  int hst[4];       // n0h * st[d]: half-index change of a unit step in direction d >= 1
  int hwr[4];       // n0h * wr[d]: half-index change of a wrapping step
  FastDiv f_n0h, f_n1, f_n2, f_n0;
  uint32_t site0;   // added to a site's index in its Philox counter (0 unless this
                    // lattice is one time slab of a larger one)
};

// A site: scalar coordinates and its row; only compile-time indices are used.
struct Site {
  int x0, x1, x2, x3;
  int row;
};

template <int D> __device__ __forceinline__ int& coord(Site& s) {
  return D == 0 ? s.x0 : D == 1 ? s.x1 : D == 2 ? s.x2 : s.x3;
}

// s + S * D-hat with periodic boundaries (S = +1 or -1).
template <int D, int S> __device__ __forceinline__ Site shifted(const Geom& g, Site s) {
  int& x = coord<D>(s);
  if (S > 0) {
    if (x + 1 == g.n[D]) { x = 0; if (D) s.row -= g.wr[D]; }
    else { x += 1; if (D) s.row += g.st[D]; }
  } else {
    if (x == 0) { x = g.n[D] - 1; if (D) s.row += g.wr[D]; }
    else { x -= 1; if (D) s.row -= g.st[D]; }
  }
  return s;
}

__device__ __forceinline__ int hidx(const Geom& g, const Site& s) { return (s.x0 >> 1) + g.n0h * s.row; }
__device__ __forceinline__ uint32_t site_index(const Geom& g, const Site& s) {
  return (uint32_t)(s.x0 + g.n[0] * s.row);
}
// The site word of the Philox counter: the site index, shifted by site0 for a
// slab of a larger lattice so that its draws are the larger lattice's.
__device__ __forceinline__ uint32_t philox_site(const Geom& g, const Site& s) { return site_index(g, s) + g.site0; }
__device__ __forceinline__ int parity(const Site& s) { return (s.x0 + s.x1 + s.x2 + s.x3) & 1; }

// Site with half-index h on the parity-p sublattice.
__device__ __forceinline__ Site site_from_half(const Geom& g, uint32_t h, int p) {
  Site s;
  const uint32_t row = g.f_n0h.div(h);
  const int xh = (int)(h - row * (uint32_t)g.n0h);
  const uint32_t r2 = g.f_n1.div(row);
  s.x1 = (int)(row - r2 * (uint32_t)g.n[1]);
  const uint32_t r3 = g.f_n2.div(r2);
  s.x2 = (int)(r2 - r3 * (uint32_t)g.n[2]);
  s.x3 = (int)r3;
  s.x0 = 2 * xh + ((s.x1 + s.x2 + s.x3 + p) & 1);
  s.row = (int)row;
  return s;
}

// Site with full index s.
__device__ __forceinline__ Site site_from_index(const Geom& g, uint32_t i) {
  Site s;
  const uint32_t row = g.f_n0.div(i);
  s.x0 = (int)(i - row * (uint32_t)g.n[0]);
  const uint32_t r2 = g.f_n1.div(row);
  s.x1 = (int)(row - r2 * (uint32_t)g.n[1]);
  const uint32_t r3 = g.f_n2.div(r2);
  s.x2 = (int)(r2 - r3 * (uint32_t)g.n[2]);
  s.x3 = (int)r3;
  s.row = (int)row;
  return s;
}

// Half-index change of the step x -> x + S d-hat (S = +1 or -1), periodic.
// For d >= 1 the step changes only the row; for d = 0 it changes x0 >> 1 by
// 0 or +-1 (by the parity of x0), or wraps across the row.  Steps in
// different directions change independent parts of the index, so the index of
// x + a + b is h + step(a) + step(b).
template <int D, int S> __device__ __forceinline__ int half_step(const Geom& g, const Site& x) {
  if (D == 0) {
    if (S > 0) return x.x0 + 1 == g.n[0] ? 1 - g.n0h : (x.x0 & 1);
    return x.x0 == 0 ? g.n0h - 1 : (x.x0 & 1) - 1;
  }
  const int xd = D == 1 ? x.x1 : D == 2 ? x.x2 : x.x3;
  if (S > 0) return xd + 1 == g.n[D] ? -g.hwr[D] : g.hst[D];
  return xd == 0 ? g.hwr[D] : -g.hst[D];
}

// F16Q staple loads without the per-link re-normalisation: staple_term
// scales each product of three links once instead (see there).
template <int P, bool NC, bool MCG, int CP>
__device__ __forceinline__ Quat<float> ld_raw(const Links<P, CP>& L, int cls, int i) {
  if constexpr (MCG) return L.ldcg_raw(cls, i);
  else return NC ? L.ld_raw(cls, i) : L.ldc_raw(cls, i);
}

// The two staple terms of Section 2 Eq. 11 for link (x, MU) and one NU != MU:
// U_nu(x) U_mu(x+nu) U_nu(x+mu)^dagger + U_nu(x-nu)^dagger U_mu(x-nu)
// U_nu(x-nu+mu).  U_nu(x) and U_nu(x-nu+mu) have the parity p of x; the four
// singly shifted links have parity 1-p.  Neighbour indices come from
// half-index steps (dmu = the step x -> x + MU).
template <int P, int MU, int NU, bool NC, int CP, bool MCG = false>
__device__ __forceinline__ void staple_term(const Links<P, CP>& L, const Geom& g, const Site& x, int h, int dmu,
                                            int p, Quat<typename Real<P>::T>& s) {
  using R = typename Real<P>::T;
  const int q = p ^ 1;
  const int h_mnu = h + half_step<NU, -1>(g, x);
  if constexpr (P == kF16Q) {
    // binary16 links re-normalised per term: a product of quaternions has the
    // product of their norms, so each term of three stored links is scaled
    // once by 1 / (|a| |b| |c|) (one rsqrt where per-link re-normalisation
    // takes three); equal to the staple of the re-normalised links up to
    // FP32 rounding
    const Quat<R> a = ld_raw<P, NC, false>(L, 2 * NU + p, h);
    const Quat<R> b = ld_raw<P, NC, MCG>(L, 2 * MU + q, h + half_step<NU, +1>(g, x));
    const Quat<R> c = ld_raw<P, NC, false>(L, 2 * NU + q, h + dmu);
    const Quat<R> d = ld_raw<P, NC, false>(L, 2 * NU + q, h_mnu);
    const Quat<R> e = ld_raw<P, NC, MCG>(L, 2 * MU + q, h_mnu);
    const Quat<R> f = ld_raw<P, NC, false>(L, 2 * NU + p, h_mnu + dmu);
    qacc_mul_nd(s, qscale(qmul(a, b), rsqrtf(qdot(a, a) * qdot(b, b) * qdot(c, c))), c);
    qacc_mul(s, qscale(qmul_dn(d, e), rsqrtf(qdot(d, d) * qdot(e, e) * qdot(f, f))), f);
  } else {
    const Quat<R> a = ldl<P, NC>(L, 2 * NU + p, h);                                // U_nu(x)
    const Quat<R> b = ldmu<P, NC, MCG>(L, 2 * MU + q, h + half_step<NU, +1>(g, x)); // U_mu(x+nu)
    const Quat<R> c = ldl<P, NC>(L, 2 * NU + q, h + dmu);                          // U_nu(x+mu)
    const Quat<R> d = ldl<P, NC>(L, 2 * NU + q, h_mnu);                            // U_nu(x-nu)
    const Quat<R> e = ldmu<P, NC, MCG>(L, 2 * MU + q, h_mnu);                      // U_mu(x-nu)
    const Quat<R> f = ldl<P, NC>(L, 2 * NU + p, h_mnu + dmu);                      // U_nu(x-nu+mu)
    qacc_mul_nd(s, qmul(a, b), c);
    qacc_mul(s, qmul_dn(d, e), f);
  }
}

// Staple sum for link (x, MU) over the directions NU != MU selected by NMASK
// (0xF: all, the heat bath), NU ascending.
template <int P, int MU, int NMASK, bool NC, int CP, bool MCG = false>
__device__ __forceinline__ Quat<typename Real<P>::T> staple(const Links<P, CP>& L, const Geom& g,
                                                           const Site& x, int h, int p) {
  using R = typename Real<P>::T;
  Quat<R> s = qmake<R>(0, 0, 0, 0);
  const int dmu = half_step<MU, +1>(g, x);
  if (MU != 0 && (NMASK & 1)) staple_term<P, MU, 0, NC, CP, MCG>(L, g, x, h, dmu, p, s);
  if (MU != 1 && (NMASK & 2)) staple_term<P, MU, 1, NC, CP, MCG>(L, g, x, h, dmu, p, s);
  if (MU != 2 && (NMASK & 4)) staple_term<P, MU, 2, NC, CP, MCG>(L, g, x, h, dmu, p, s);
  if (MU != 3 && (NMASK & 8)) staple_term<P, MU, 3, NC, CP, MCG>(L, g, x, h, dmu, p, s);
  return s;
}

// The staple sum of all NU != MU, accumulated in the same order as staple(),
// with `lower` set to the partial sum over NU < MU.  Tr(U_MU(x) lower^dagger)/2
// is the sum of the plaquettes in the planes (NU, MU), NU < MU, that contain
// the link (Section 2, Eq. 12).
template <int P, int MU, bool NC, int CP, bool MCG = false>
__device__ __forceinline__ Quat<typename Real<P>::T> staple_split(const Links<P, CP>& L, const Geom& g, const Site& x,
                                                                 int h, int p, Quat<typename Real<P>::T>& lower) {
  using R = typename Real<P>::T;
  Quat<R> s = qmake<R>(0, 0, 0, 0);
  const int dmu = half_step<MU, +1>(g, x);
  if (MU != 0) staple_term<P, MU, 0, NC, CP, MCG>(L, g, x, h, dmu, p, s);
  if (MU == 1) lower = s;
  if (MU != 1) staple_term<P, MU, 1, NC, CP, MCG>(L, g, x, h, dmu, p, s);
  if (MU == 2) lower = s;
  if (MU != 2) staple_term<P, MU, 2, NC, CP, MCG>(L, g, x, h, dmu, p, s);
  if (MU == 3) lower = s;
  if (MU != 3) staple_term<P, MU, 3, NC, CP, MCG>(L, g, x, h, dmu, p, s);
  if (MU == 0) lower = qmake<R>(0, 0, 0, 0);
  return s;
}

}  // namespace su2
