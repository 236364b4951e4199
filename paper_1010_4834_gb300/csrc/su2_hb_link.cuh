// One link's heat-bath update (Section 2, Eqs. 5-9, 11), shared by the
// substep kernel (su2_heatbath.cu), the fused parity-pair kernel
// (su2_pair.cu) and the batched kernel (su2_batch.cu), so all of them run
// the same arithmetic and leave the same links.
// Paper: Cardoso & Bicudo, arXiv:1010.4834.
//
// Every lane makes the link's first a0 trial inline.  A link that rejects it
// goes to a block-wide shared-memory queue (its W = Sigma/k, alpha, index and
// site), which the block later finishes with trials 2, 3, ... (hb_drain): a
// warp then does not wait on its slowest lane's trial loop.  The draws and
// their order are those of the plain loop, so only the schedule differs.  A
// full queue falls back to finishing the link inline.
//
// With MEAS the update also adds Tr(U_MU(x) L(x)^dagger)/2 to `plaq`, with L
// the staple's partial sum over NU < MU and U the link's final value (the
// accepted draw as stored, or the kept old link); see k_heatbath.
#pragma once

#include "su2_kernel_util.cuh"

namespace su2 {

template <class R> struct PlainAcc {
  R s = R(0);
  __device__ __forceinline__ void add(R v) { s += v; }
  __device__ __forceinline__ double value() const { return (double)s; }
};

// Queue entries are 16-byte aligned (FP32: 28 -> 32 bytes), so an entry
// moves in a few wide shared-memory accesses: 64^4 FP32 sweep 1412 -> 1407
// us, F16Q 1610 -> 1592 us.
template <class R, bool MEAS> struct __align__(16) Deferred {
  Quat<R> w;
  R alpha;
  int h;
  uint32_t site;
};
template <class R> struct __align__(16) Deferred<R, true> {
  Quat<R> w;
  R alpha;
  int h;
  uint32_t site;
  Quat<R> lower;
};

// Trial, capped and Haar counts of the links a thread finished.
struct HBCount {
  unsigned int trials = 0, capped = 0, haar = 0;
};

template <class R, bool MEAS>
__device__ __forceinline__ int finish_deferred(const Deferred<R, MEAS>& d, uint4 ctr, const HBParams& hp,
                                               Quat<R>* out) {
  R a0;
  uint4 rt;
  const int n =
      sample_a0_from<R>(2, d.alpha, trial_inv2a(d.alpha), trial_e(d.alpha, hp.sampler), ctr, hp, &a0, &rt);
  if (n) *out = compose_link<R>(a0, d.w, ctr, rt, hp);
  return n;
}

// Update link h of class (MU, PAR).  Rejected first trials go to queue slot
// atomicAdd(qn, 1) when it is below CAP.  MCG: the staple's loads of the
// other-parity MU class bypass L1 (the fused pair kernel writes that class
// earlier in the same launch).  NC: read-only loads; the persistent batched
// kernel, whose other CTAs write links during the launch, loads coherently.
template <int P, int MU, bool MEAS, int PAR, bool MCG, int CAP, int CP, bool NC = true>
__device__ __forceinline__ void hb_link(const Links<P, CP>& L, const Geom& g, int h, uint32_t tag, uint32_t sweep,
                                        typename Real<P>::T beta, const HBParams& hp,
                                        Deferred<typename Real<P>::T, MEAS>* queue, int* qn,
                                        PlainAcc<typename Real<P>::T>& plaq, HBCount& cnt) {
  constexpr int p = PAR;
  using R = typename Real<P>::T;
  using M = Math<R>;
  using Def = Deferred<R, MEAS>;
  const Site x = site_from_half(g, (uint32_t)h, p);
  Quat<R> lower;
  Quat<R> sig;
  if constexpr (MEAS) sig = staple_split<P, MU, NC, CP, MCG>(L, g, x, h, p, lower);
  else sig = staple<P, MU, 0xF, NC, CP, MCG>(L, g, x, h, p);
  const uint32_t site = philox_site(g, x);
  const uint4 ctr = make_uint4(site, tag, sweep, 0u);
  const R k2 = qdot(sig, sig);
  const R invk = M::rsqrt(k2);
  const R alpha = beta * k2 * invk;
  if (!(alpha >= R(1e-12))) {
    uint4 c = ctr;
    c.w = 1u;
    const Quat<R> nl = haar_from<R>(philox(c, hp.rk));
    if constexpr (MEAS) plaq.add(qdot(L.put(2 * MU + p, h, nl), lower));
    else L.st(2 * MU + p, h, nl);
    cnt.haar += 1;
    return;
  }
  const R inv2a = trial_inv2a(alpha);
  const R e = trial_e(alpha, hp.sampler);
  const Quat<R> w = qscale(sig, invk);
  R a0;
  uint4 rt;
  if (trial_a0<R>(alpha, inv2a, e, ctr, 1, hp, &a0, &rt)) {
    const Quat<R> nl = compose_link<R>(a0, w, ctr, rt, hp);
    if constexpr (MEAS) plaq.add(qdot(L.put(2 * MU + p, h, nl), lower));
    else L.st(2 * MU + p, h, nl);
    cnt.trials += 1;
  } else if (hp.max_tries > 1) {
    const int slot = atomicAdd(qn, 1);
    Def d;
    d.w = w;
    d.alpha = alpha;
    d.h = h;
    d.site = site;
    if constexpr (MEAS) d.lower = lower;
    if (slot < CAP) {
      queue[slot] = d;
    } else {
      Quat<R> nl;
      const int n = finish_deferred<R, MEAS>(d, ctr, hp, &nl);
      if constexpr (MEAS) plaq.add(qdot(n ? L.put(2 * MU + p, h, nl) : ldl<P, NC>(L, 2 * MU + p, h), lower));
      else if (n) L.st(2 * MU + p, h, nl);
      cnt.trials += n ? (unsigned)n : (unsigned)hp.max_tries;
      cnt.capped += n == 0;
    }
  } else {
    if constexpr (MEAS) plaq.add(qdot(ldl<P, NC>(L, 2 * MU + p, h), lower));
    cnt.trials += 1;
    cnt.capped += 1;
  }
}

// Finish the queue entries i = threadIdx.x, threadIdx.x + blockDim.x, ... < n.
template <int P, int MU, bool MEAS, int PAR, int CP, bool NC = true>
__device__ __forceinline__ void hb_drain(const Links<P, CP>& L, const Deferred<typename Real<P>::T, MEAS>* queue, int n,
                                         uint32_t tag, uint32_t sweep, const HBParams& hp,
                                         PlainAcc<typename Real<P>::T>& plaq, HBCount& cnt) {
  constexpr int p = PAR;
  using R = typename Real<P>::T;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const Deferred<R, MEAS> d = queue[i];
    Quat<R> nl;
    const int t = finish_deferred<R, MEAS>(d, make_uint4(d.site, tag, sweep, 0u), hp, &nl);
    if constexpr (MEAS) plaq.add(qdot(t ? L.put(2 * MU + p, d.h, nl) : ldl<P, NC>(L, 2 * MU + p, d.h), d.lower));
    else if (t) L.st(2 * MU + p, d.h, nl);
    cnt.trials += t ? (unsigned)t : (unsigned)hp.max_tries;
    cnt.capped += t == 0;
  }
}

// One over-relaxation update (Section 2, Eq. 10 with W = Sigma/|Sigma| for
// the orientation of Eq. 11): U' = W U^dagger W keeps Tr(U Sigma^dagger).
// Unlike a heat-bath link, U' is built from the old link, so rounding would
// accumulate over many over-relaxation sweeps: in FP32 each step multiplies
// |U| by |W|^2 = 1 + O(2^-22), a random walk of about 1e-5 after a thousand
// sweeps.  FP32 (and the F16Q arithmetic, whose stores are normalised again
// on load) therefore normalises U' before storing it; in FP64 the walk stays
// near 1e-15 and the update is stored as computed, like the oracle's.  NC:
// read-only loads (no other block of the launch writes these links).
template <int P, int MU, int PAR, bool NC, int CP>
__device__ __forceinline__ void or_link(const Links<P, CP>& L, const Geom& g, int h) {
  constexpr int p = PAR;
  using R = typename Real<P>::T;
  using M = Math<R>;
  const Site x = site_from_half(g, (uint32_t)h, p);
  const Quat<R> sig = staple<P, MU, 0xF, NC>(L, g, x, h, p);
  const R k2 = qdot(sig, sig);
  if (!(k2 >= M::kTiny)) return;
  const Quat<R> w = qscale(sig, M::rsqrt(k2));
  const Quat<R> u = ldl<P, NC>(L, 2 * MU + p, h);
  Quat<R> v = qmul(qmul_nd(w, u), w);
  if constexpr (P != kF64) v = qscale(v, M::rsqrt(qdot(v, v)));
  L.st(2 * MU + p, h, v);
}

}  // namespace su2
