/*
 * Plain FP64 CPU oracle for the quenched SU(2) heat-bath method of
 * Cardoso & Bicudo (arXiv:1010.4834).
 *
 * TEST INFRASTRUCTURE ONLY: called from the test suite, the package smoke
 * check and the CPU-baseline leg of the benchmark, never from the product
 * path.  Written for clarity, not speed: one link at a time, canonical site
 * order, no blocking, no reordering beyond what the paper's definitions state.
 * Shares nothing with the CUDA library.  Conventions are in su2_oracle.h.
 */
#include "su2_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads a substep uses: 1 in the serial build, the OpenMP team size in
 * the all-cores build. */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================== */
/* Random numbers                                                            */
/* ======================================================================== */

/*
 * Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of the Philox-4x32 S-box
 * (two 32x32->64 multiplications by the round multipliers, XOR of the high
 * halves with the other counter words and the round key, word permutation),
 * the key bumped by the Weyl constants between rounds.  The paper itself used
 * an LCRNG and CURAND (Section 4); a counter-based generator replaces both.
 */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t p0 = (uint64_t)mult0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)mult1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uint32 -> uniform in the open interval (0,1): (x + 1/2) 2^-32, exact in
 * FP64.  The 23-bit variant ((x >> 9) + 1/2) 2^-23 is the finest grid a
 * binary32 value in (0,1) holds exactly up to 1 - 2^-24. */
double oracle_u01(uint32_t x, int u23) {
  if (u23) return ldexp((double)(x >> 9) + 0.5, -23);
  return ldexp((double)x + 0.5, -32);
}

/* The four Philox words of draw `draw` for link (s, mu) in sweep `sweep`:
 * counter (s, mu | lattice_id << 2, sweep, draw), key = the 64-bit seed. */
void oracle_draw_words(const oracle_chain* c, long s, int mu, uint32_t sweep, uint32_t draw,
                       uint32_t r[4]) {
  uint32_t ctr[4], key[2];
  ctr[0] = (uint32_t)s;
  ctr[1] = (uint32_t)mu | (c->lattice_id << 2);
  ctr[2] = sweep;
  ctr[3] = draw;
  key[0] = (uint32_t)(c->seed & 0xffffffffu);
  key[1] = (uint32_t)(c->seed >> 32);
  oracle_philox4x32_10(ctr, key, r);
}

/* Four uniforms of draw `draw` for link (s, mu) in sweep `sweep`. */
void oracle_draw(const oracle_chain* c, long s, int mu, uint32_t sweep, uint32_t draw,
                 double u[4]) {
  uint32_t r[4];
  oracle_draw_words(c, s, mu, sweep, draw, r);
  for (int i = 0; i < 4; i++) u[i] = oracle_u01(r[i], c->u23);
}

/* ======================================================================== */
/* SU(2) algebra, Section 2 Eqs. 1-3                                         */
/* ======================================================================== */

/*
 * U = a0 1 + i a.sigma (Eq. 1).  Multiplying two such matrices and using
 * sigma_i sigma_j = delta_ij + i eps_ijk sigma_k gives
 *   (a b)_0 = a0 b0 - a.b,   (a b)_vec = a0 b + b0 a - a x b.
 */
void oracle_qmul(const double a[4], const double b[4], double out[4]) {
  double r0 = a[0] * b[0] - (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
  double cx = a[2] * b[3] - a[3] * b[2];
  double cy = a[3] * b[1] - a[1] * b[3];
  double cz = a[1] * b[2] - a[2] * b[1];
  double r1 = a[0] * b[1] + b[0] * a[1] - cx;
  double r2 = a[0] * b[2] + b[0] * a[2] - cy;
  double r3 = a[0] * b[3] + b[0] * a[3] - cz;
  out[0] = r0; out[1] = r1; out[2] = r2; out[3] = r3;
}

/* U^dagger = a0 1 - i a.sigma. */
void oracle_qdag(const double a[4], double out[4]) {
  out[0] = a[0]; out[1] = -a[1]; out[2] = -a[2]; out[3] = -a[3];
}

static void qmul3(const double a[4], const double b[4], const double c[4], double out[4]) {
  double t[4];
  oracle_qmul(a, b, t);
  oracle_qmul(t, c, out);
}

/* ======================================================================== */
/* Geometry                                                                  */
/* ======================================================================== */

long oracle_volume(int nd, const int* dims) {
  long v = 1;
  for (int i = 0; i < nd; i++) v *= dims[i];
  return v;
}

static void coords(int nd, const int* dims, long s, int* x) {
  for (int i = 0; i < nd; i++) {
    x[i] = (int)(s % dims[i]);
    s /= dims[i];
  }
}

static long site_of(int nd, const int* dims, const int* x) {
  long s = 0;
  for (int i = nd - 1; i >= 0; i--) s = s * dims[i] + x[i];
  return s;
}

static int parity_of(int nd, const int* dims, long s) {
  int x[4], p = 0;
  coords(nd, dims, s, x);
  for (int i = 0; i < nd; i++) p += x[i];
  return p & 1;
}

/* Site s + step * mu-hat with periodic boundaries (Section 2, Polyakov loop
 * paragraph: periodic in time and space). */
long oracle_shift(int nd, const int* dims, long s, int mu, int step) {
  int x[4];
  coords(nd, dims, s, x);
  int n = dims[mu];
  x[mu] = ((x[mu] + step) % n + n) % n;
  return site_of(nd, dims, x);
}

static const double* link(int nd, const double* U, long s, int mu) {
  return U + ((size_t)s * nd + mu) * 4;
}

/* ======================================================================== */
/* Start configurations                                                      */
/* ======================================================================== */

/* Cold start: U = 1 on every link (Section 4, kernel list). */
void oracle_init_cold(int nd, const int* dims, double* U) {
  long n = oracle_volume(nd, dims) * nd;
  for (long i = 0; i < n; i++) {
    U[i * 4 + 0] = 1.0;
    U[i * 4 + 1] = 0.0;
    U[i * 4 + 2] = 0.0;
    U[i * 4 + 3] = 0.0;
  }
}

/* A Haar-distributed SU(2) element from four uniforms: four independent
 * normals (Box-Muller on the pairs (u0,u1) and (u2,u3)) normalised onto S^3.
 * The normal distribution in R^4 is rotation invariant, so its direction is
 * uniform on S^3, which is the Haar measure of Eq. 4. */
static void haar_from_uniforms(const double u[4], double q[4]) {
  const double two_pi = 6.283185307179586476925286766559;
  double r01 = sqrt(-2.0 * log(u[0]));
  double r23 = sqrt(-2.0 * log(u[2]));
  double z[4];
  z[0] = r01 * cos(two_pi * u[1]);
  z[1] = r01 * sin(two_pi * u[1]);
  z[2] = r23 * cos(two_pi * u[3]);
  z[3] = r23 * sin(two_pi * u[3]);
  double n = sqrt(z[0] * z[0] + z[1] * z[1] + z[2] * z[2] + z[3] * z[3]);
  for (int i = 0; i < 4; i++) q[i] = z[i] / n;
}

/* Hot start: a random SU(2) element on every link (Section 4, kernel list),
 * read as a Haar-distributed element per link, from Philox draw 0 of the
 * reserved sweep index 0xFFFFFFFF. */
void oracle_hot_link(const oracle_chain* c, long s, int mu, double q[4]) {
  double u[4];
  oracle_draw(c, s, mu, 0xFFFFFFFFu, 0u, u);
  haar_from_uniforms(u, q);
}

void oracle_init_hot(int nd, const int* dims, const oracle_chain* c, double* U) {
  long vol = oracle_volume(nd, dims);
  for (long s = 0; s < vol; s++)
    for (int mu = 0; mu < nd; mu++) oracle_hot_link(c, s, mu, U + ((size_t)s * nd + mu) * 4);
}

/* ======================================================================== */
/* Heat bath                                                                 */
/* ======================================================================== */

/*
 * Staple sum of Section 2, Eq. 11: for every nu != mu the forward path
 * U_nu(x) U_mu(x+nu) U_nu(x+mu)^dagger and the backward path
 * U_nu(x-nu)^dagger U_mu(x-nu) U_nu(x-nu+mu).  Both run from x+mu to x, so
 * U_mu(x) Sigma^dagger closes the six plaquettes that contain U_mu(x).
 */
void oracle_staple(int nd, const int* dims, const double* U, long s, int mu, double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  long xp_mu = oracle_shift(nd, dims, s, mu, +1);
  for (int nu = 0; nu < nd; nu++) {
    if (nu == mu) continue;
    long xp_nu = oracle_shift(nd, dims, s, nu, +1);
    long xm_nu = oracle_shift(nd, dims, s, nu, -1);
    long xm_nu_p_mu = oracle_shift(nd, dims, xm_nu, mu, +1);
    double d[4], t[4];

    oracle_qdag(link(nd, U, xp_mu, nu), d);
    qmul3(link(nd, U, s, nu), link(nd, U, xp_nu, mu), d, t);
    for (int i = 0; i < 4; i++) out[i] += t[i];

    oracle_qdag(link(nd, U, xm_nu, nu), d);
    qmul3(d, link(nd, U, xm_nu, mu), link(nd, U, xm_nu_p_mu, nu), t);
    for (int i = 0; i < 4; i++) out[i] += t[i];
  }
}

/*
 * Draw a0 in [-1,1] with density sqrt(1-a0^2) exp(alpha a0), Section 2 Eq. 8
 * with alpha = beta k.  Trial n (n = 1..max_tries) uses Philox draw n.
 *
 * Kennedy-Pendleton (Phys. Lett. B 156 (1985) 393): with a0 = 1 - 2 delta the
 * density becomes sqrt(delta) exp(-2 alpha delta) * sqrt(1 - delta).  The first
 * factor is a Gamma(3/2, rate 2 alpha) density, sampled as the sum of an
 * exponential and half a squared normal:
 *   delta = -(ln u0 + cos^2(2 pi u1) ln u2) / (2 alpha);
 * the second factor is applied by accepting when u3^2 <= 1 - delta.
 *
 * Creutz (Phys. Rev. D 21 (1980) 2308, the method the paper cites): a0 with
 * density exp(alpha a0) on [-1,1] by inversion,
 *   a0 = 1 + ln(e^{-2 alpha} + (1 - e^{-2 alpha}) u0) / alpha,
 * accepted when u1^2 <= 1 - a0^2.
 *
 * Returns the accepted trial number, or 0 when every trial failed.  `margin`
 * (may be NULL) receives the smallest |lhs - rhs| of the accept tests made:
 * how close a decision came to flipping under rounding.
 */
int oracle_sample_a0(const oracle_chain* c, double alpha, long s, int mu, uint32_t sweep,
                     double* a0, double* margin) {
  const double two_pi = 6.283185307179586476925286766559;
  double best = INFINITY;
  int accepted = 0;
  for (int n = 1; n <= c->max_tries; n++) {
    double u[4];
    oracle_draw(c, s, mu, sweep, (uint32_t)n, u);
    double lhs, rhs, cand;
    if (c->sampler == ORACLE_CREUTZ) {
      double e = exp(-2.0 * alpha);
      cand = 1.0 + log(e + (1.0 - e) * u[0]) / alpha;
      lhs = u[1] * u[1];
      rhs = 1.0 - cand * cand;
    } else {
      double cs = cos(two_pi * u[1]);
      double delta = -(log(u[0]) + cs * cs * log(u[2])) / (2.0 * alpha);
      cand = 1.0 - 2.0 * delta;
      lhs = u[3] * u[3];
      rhs = 1.0 - delta;
    }
    double m = fabs(lhs - rhs);
    if (m < best) best = m;
    if (lhs <= rhs) {
      *a0 = cand;
      accepted = n;
      break;
    }
  }
  if (margin) *margin = best;
  return accepted;
}

/*
 * One heat-bath update of link (s, mu) given its staple sum Sigma
 * (Section 2, Eqs. 5-9).
 *
 * The link density is exp(beta/2 Tr(U Sigma^dagger)) (Eq. 5 with
 * V = Sigma^dagger for the orientation of Eq. 11).  Writing Sigma = k W with
 * k = sqrt(det Sigma) = |Sigma| (Eq. 6) and X = U W^dagger, Haar invariance
 * gives X the density exp(beta k x0) dX (Eq. 7), i.e. x0 = a0 from Eq. 8 and
 * the vector part uniform on the sphere of radius sqrt(1 - a0^2).  The new
 * link is U = X W (Eq. 9 with the sampled matrix in place of U).
 *
 * Direction (uniform on the 2-sphere; the paper fixes no random numbers):
 *   - 32-bit mode: Philox draw 0, cos(theta) = 2 u0 - 1, phi = 2 pi u1;
 *   - 23-bit mode (the FP32 map): the nine low bits of each word of the
 *     accepting trial's draw n, which its 23-bit uniforms do not use:
 *     c = (r0 mod 2^9) 2^9 + (r1 mod 2^9), f = (r2 mod 2^9) 2^9 + (r3 mod 2^9),
 *     cos(theta) = (2c + 1) 2^-18 - 1, phi = 2 pi (f + 1/2) 2^-18.  These bits
 *     are independent of the trial's uniforms, so the direction is still
 *     independent of a0; cos(theta) and phi are uniform on grids of 2^18
 *     midpoints.
 * Readings where the paper is silent:
 *   - all trials failing keeps the old link.  The accepted-value kernel is
 *     proportional to the target and independent of the old link, so the
 *     step is a mixture of a heat bath and the identity and still satisfies
 *     detailed balance;
 *   - alpha < 1e-12 (beta = 0 or a vanishing staple) draws the link from the
 *     Haar measure using Philox draw 1, as for the hot start.
 * Returns the accepted trial number, 0 when capped, -1 on the Haar branch.
 */
int oracle_heatbath_link(const oracle_chain* c, long s, int mu, uint32_t sweep,
                         const double sigma[4], const double old_link[4], double new_link[4],
                         double* margin) {
  const double two_pi = 6.283185307179586476925286766559;
  double k = sqrt(sigma[0] * sigma[0] + sigma[1] * sigma[1] + sigma[2] * sigma[2] +
                  sigma[3] * sigma[3]);
  double alpha = c->beta * k;
  if (!(alpha >= 1e-12)) {
    double u[4];
    oracle_draw(c, s, mu, sweep, 1u, u);
    haar_from_uniforms(u, new_link);
    if (margin) *margin = INFINITY;
    return -1;
  }
  double a0 = 0.0;
  int n = oracle_sample_a0(c, alpha, s, mu, sweep, &a0, margin);
  if (n == 0) {
    for (int i = 0; i < 4; i++) new_link[i] = old_link[i];
    return 0;
  }
  double cos_theta, phi;
  if (c->u23) {
    uint32_t r[4];
    oracle_draw_words(c, s, mu, sweep, (uint32_t)n, r);
    uint32_t cb = ((r[0] & 0x1FFu) << 9) | (r[1] & 0x1FFu);
    uint32_t fb = ((r[2] & 0x1FFu) << 9) | (r[3] & 0x1FFu);
    cos_theta = ldexp(2.0 * cb + 1.0, -18) - 1.0;
    phi = two_pi * ldexp(fb + 0.5, -18);
  } else {
    double u[4];
    oracle_draw(c, s, mu, sweep, 0u, u);
    cos_theta = 2.0 * u[0] - 1.0;
    phi = two_pi * u[1];
  }
  double sin_theta = sqrt(fmax(0.0, 1.0 - cos_theta * cos_theta));
  double r = sqrt(fmax(0.0, 1.0 - a0 * a0));
  double x[4], w[4];
  x[0] = a0;
  x[1] = r * sin_theta * cos(phi);
  x[2] = r * sin_theta * sin(phi);
  x[3] = r * cos_theta;
  for (int i = 0; i < 4; i++) w[i] = sigma[i] / k;
  oracle_qmul(x, w, new_link);
  return n;
}

/*
 * One checkerboard substep: every link of direction mu on sites of parity
 * `parity` (the checkerboard order of Section 4: one direction and one site
 * parity at a time).
 * The links of one (mu, parity) class do not enter each other's staples, so
 * the order of the loop does not matter; canonical order is used.  For the
 * same reason the sites may be shared among threads: built with OpenMP (the
 * all-cores CPU baseline), the loop runs on every host core and leaves the
 * same links and counts as the serial build, which ignores the pragma.
 * `margin` (may be NULL) receives, per updated link at index s*nd+mu, the
 * decision margin of oracle_sample_a0.
 */
void oracle_substep(int nd, const int* dims, double* U, const oracle_chain* c, uint32_t sweep,
                    int mu, int parity, oracle_stats* st, double* margin) {
  long vol = oracle_volume(nd, dims);
  uint64_t updates = 0, trials = 0, capped = 0, haar = 0;
#pragma omp parallel for schedule(static) reduction(+ : updates, trials, capped, haar)
  for (long s = 0; s < vol; s++) {
    if (parity_of(nd, dims, s) != parity) continue;
    double sigma[4], nl[4], m = INFINITY;
    oracle_staple(nd, dims, U, s, mu, sigma);
    double* l = U + ((size_t)s * nd + mu) * 4;
    int n = oracle_heatbath_link(c, s, mu, sweep, sigma, l, nl, &m);
    for (int i = 0; i < 4; i++) l[i] = nl[i];
    if (margin) margin[(size_t)s * nd + mu] = m;
    updates++;
    if (n > 0) trials += (uint64_t)n;
    if (n == 0) { capped++; trials += (uint64_t)c->max_tries; }
    if (n < 0) haar++;
  }
  if (st) {
    st->updates += updates;
    st->trials += trials;
    st->capped += capped;
    st->haar += haar;
  }
}

/* One sweep: direction outer, parity inner (even first). */
void oracle_sweep(int nd, const int* dims, double* U, const oracle_chain* c, uint32_t sweep,
                  oracle_stats* st) {
  for (int mu = 0; mu < nd; mu++)
    for (int p = 0; p < 2; p++) oracle_substep(nd, dims, U, c, sweep, mu, p, st, NULL);
}

/*
 * Over-relaxation, Section 2 Eq. 10, read with W = Sigma/|Sigma| for the
 * staple orientation of Eq. 11: U' = W U^dagger W, which keeps
 * Tr(U Sigma^dagger) and hence the action unchanged.  Links with a vanishing
 * staple are left as they are.
 */
void oracle_overrelax_substep(int nd, const int* dims, double* U, int mu, int parity) {
  long vol = oracle_volume(nd, dims);
  for (long s = 0; s < vol; s++) {
    if (parity_of(nd, dims, s) != parity) continue;
    double sigma[4];
    oracle_staple(nd, dims, U, s, mu, sigma);
    double k = sqrt(sigma[0] * sigma[0] + sigma[1] * sigma[1] + sigma[2] * sigma[2] +
                    sigma[3] * sigma[3]);
    if (!(k >= 1e-300)) continue;
    double w[4], d[4], t[4];
    for (int i = 0; i < 4; i++) w[i] = sigma[i] / k;
    double* l = U + ((size_t)s * nd + mu) * 4;
    oracle_qdag(l, d);
    qmul3(w, d, w, t);
    for (int i = 0; i < 4; i++) l[i] = t[i];
  }
}

/* ======================================================================== */
/* Measurements                                                              */
/* ======================================================================== */

/* Neumaier's compensated summation (Z. Angew. Math. Mech. 54 (1974) 39). */
typedef struct { double sum, comp; } ksum;

static void ksum_add(ksum* k, double v) {
  double t = k->sum + v;
  if (fabs(k->sum) >= fabs(v))
    k->comp += (k->sum - t) + v;
  else
    k->comp += (v - t) + k->sum;
  k->sum = t;
}

static double ksum_value(const ksum* k) { return k->sum + k->comp; }

/*
 * Mean plaquette, Section 2 Eqs. 12-13.  Returned as the mean of
 * (1/2) Re Tr[U_mu(s) U_nu(s+mu) U_mu(s+nu)^dagger U_nu(s)^dagger] over all
 * sites and planes mu < nu (1 on the cold start; the paper's P_mu_nu is one
 * minus this).  out[0]: all planes; out[1]: planes without the time
 * direction; out[2]: planes containing it.  With nd = 2 there is no purely
 * spatial plane and out[1] is 0.
 */
void oracle_plaquette(int nd, const int* dims, const double* U, double out[3]) {
  long vol = oracle_volume(nd, dims);
  int t = nd - 1;
  ksum all = {0, 0}, spat = {0, 0}, temp = {0, 0};
  long n_all = 0, n_spat = 0, n_temp = 0;
  for (long s = 0; s < vol; s++) {
    for (int mu = 0; mu < nd; mu++) {
      for (int nu = mu + 1; nu < nd; nu++) {
        long xp_mu = oracle_shift(nd, dims, s, mu, +1);
        long xp_nu = oracle_shift(nd, dims, s, nu, +1);
        double a[4], b[4], d1[4], d2[4];
        oracle_qdag(link(nd, U, xp_nu, mu), d1);
        oracle_qdag(link(nd, U, s, nu), d2);
        oracle_qmul(link(nd, U, s, mu), link(nd, U, xp_mu, nu), a);
        oracle_qmul(a, d1, b);
        oracle_qmul(b, d2, a);
        double v = a[0];
        ksum_add(&all, v);
        n_all++;
        if (nu == t) {
          ksum_add(&temp, v);
          n_temp++;
        } else {
          ksum_add(&spat, v);
          n_spat++;
        }
      }
    }
  }
  out[0] = ksum_value(&all) / (double)n_all;
  out[1] = n_spat ? ksum_value(&spat) / (double)n_spat : 0.0;
  out[2] = n_temp ? ksum_value(&temp) / (double)n_temp : 0.0;
}

/*
 * Polyakov loop, Section 2 Eqs. 14-15: for each spatial site the product of
 * the time-direction links in increasing t, one half of its trace, averaged
 * over the N_sigma spatial sites.  Signed (the modulus is the caller's).
 */
double oracle_polyakov(int nd, const int* dims, const double* U) {
  int t = nd - 1;
  long vol = oracle_volume(nd, dims);
  long nsig = vol / dims[t];
  ksum acc = {0, 0};
  for (long xs = 0; xs < nsig; xs++) {
    double p[4] = {1.0, 0.0, 0.0, 0.0}, q[4];
    for (int tt = 0; tt < dims[t]; tt++) {
      long s = xs + nsig * tt;
      oracle_qmul(p, link(nd, U, s, t), q);
      memcpy(p, q, sizeof p);
    }
    ksum_add(&acc, p[0]);
  }
  return ksum_value(&acc) / (double)nsig;
}

/* Ordered product of n links of direction mu starting at s. */
static void line(int nd, const int* dims, const double* U, long s, int mu, int n, double out[4]) {
  double p[4] = {1.0, 0.0, 0.0, 0.0}, q[4];
  for (int i = 0; i < n; i++) {
    oracle_qmul(p, link(nd, U, s, mu), q);
    memcpy(p, q, sizeof p);
    s = oracle_shift(nd, dims, s, mu, +1);
  }
  memcpy(out, p, sizeof p);
}

/*
 * Wilson loops, Section 2 Eq. 18: the R x T rectangle with a spatial side of
 * R links in direction mu and a temporal side of T links,
 *   (1/2) Tr[S_R(x) T_T(x + R mu) S_R(x + T t)^dagger T_T(x)^dagger],
 * S_R and T_T the ordered line products.  Read with the factor 1/2 (so that
 * W(1,1) is the space-time plaquette) and averaged over all sites and the
 * nd-1 spatial directions.  out[(R-1)*tmax + (T-1)], 1 <= R <= rmax,
 * 1 <= T <= tmax.
 */
void oracle_wilson_loops(int nd, const int* dims, const double* U, int rmax, int tmax,
                         double* out) {
  int t = nd - 1;
  long vol = oracle_volume(nd, dims);
  for (int R = 1; R <= rmax; R++) {
    for (int T = 1; T <= tmax; T++) {
      ksum acc = {0, 0};
      for (long s = 0; s < vol; s++) {
        for (int mu = 0; mu < t; mu++) {
          double sr[4], tt[4], sr2[4], tt0[4], d1[4], d2[4], a[4], b[4];
          line(nd, dims, U, s, mu, R, sr);
          line(nd, dims, U, oracle_shift(nd, dims, s, mu, R), t, T, tt);
          line(nd, dims, U, oracle_shift(nd, dims, s, t, T), mu, R, sr2);
          line(nd, dims, U, s, t, T, tt0);
          oracle_qdag(sr2, d1);
          oracle_qdag(tt0, d2);
          oracle_qmul(sr, tt, a);
          oracle_qmul(a, d1, b);
          oracle_qmul(b, d2, a);
          ksum_add(&acc, a[0]);
        }
      }
      out[(R - 1) * tmax + (T - 1)] = ksum_value(&acc) / ((double)vol * (double)t);
    }
  }
}

/*
 * One APE smearing step, Section 2 Eq. 19, spatial links only.  Read as a
 * Jacobi update (every new link from the old field) with
 *   U'_mu(x) = P[(1 - alpha) U_mu(x) + (alpha/4) Sum],
 * Sum = the forward and backward staples of Eq. 11 over the two spatial
 * nu != mu (four staples).  For SU(2) the projection P is division by the
 * norm, so the paper's prefactor 1/(1+6w) drops out and only the weight ratio
 * matters: w = alpha / (4 (1 - alpha)).  Temporal links are copied.  A sum
 * with norm below 1e-300 keeps the old link.
 */
void oracle_ape_step(int nd, const int* dims, const double* Uin, double* Uout, double alpha) {
  int t = nd - 1;
  long vol = oracle_volume(nd, dims);
  for (long s = 0; s < vol; s++) {
    for (int mu = 0; mu < nd; mu++) {
      const double* l = link(nd, Uin, s, mu);
      double* o = Uout + ((size_t)s * nd + mu) * 4;
      if (mu == t) {
        memcpy(o, l, 4 * sizeof(double));
        continue;
      }
      double sum[4] = {0, 0, 0, 0};
      long xp_mu = oracle_shift(nd, dims, s, mu, +1);
      for (int nu = 0; nu < t; nu++) {
        if (nu == mu) continue;
        long xp_nu = oracle_shift(nd, dims, s, nu, +1);
        long xm_nu = oracle_shift(nd, dims, s, nu, -1);
        long xm_nu_p_mu = oracle_shift(nd, dims, xm_nu, mu, +1);
        double d[4], st[4];
        oracle_qdag(link(nd, Uin, xp_mu, nu), d);
        qmul3(link(nd, Uin, s, nu), link(nd, Uin, xp_nu, mu), d, st);
        for (int i = 0; i < 4; i++) sum[i] += st[i];
        oracle_qdag(link(nd, Uin, xm_nu, nu), d);
        qmul3(d, link(nd, Uin, xm_nu, mu), link(nd, Uin, xm_nu_p_mu, nu), st);
        for (int i = 0; i < 4; i++) sum[i] += st[i];
      }
      double q[4];
      for (int i = 0; i < 4; i++) q[i] = (1.0 - alpha) * l[i] + 0.25 * alpha * sum[i];
      double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      if (!(n >= 1e-300)) {
        memcpy(o, l, 4 * sizeof(double));
        continue;
      }
      for (int i = 0; i < 4; i++) o[i] = q[i] / n;
    }
  }
}
