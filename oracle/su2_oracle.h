/*
 * Plain FP64 CPU oracle for the quenched SU(2) heat-bath method of
 * Cardoso & Bicudo, "SU(2) Lattice Gauge Theory Simulations on Fermi GPUs"
 * (arXiv:1010.4834).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no source, header, table or helper with the
 * CUDA library; both sides are written independently from the paper.
 *
 * Conventions (fixed here and checked by the tests under tests/):
 *   nd      number of dimensions, 2..4; the last dimension is time.
 *   dims    extents (N0, N1, ..., N_{nd-1}), each even and >= 2.
 *   site    s = x0 + N0*(x1 + N1*(x2 + N2*x3)); parity p(s) = (sum x_i) mod 2.
 *   links   canonical FP64 array U[(s*nd + mu)*4 + c], c = 0..3, the
 *           quaternion (q0,q1,q2,q3) <-> q0*1 + i(q1 s1 + q2 s2 + q3 s3)
 *           (Section 2, Eq. 1).
 *   Philox  key = (seed & 0xffffffff, seed >> 32);
 *           ctr = (s, mu | lattice_id << 2, sweep, draw).
 *           Hot start uses sweep = 0xFFFFFFFF, draw 0.  Heat-bath trial n
 *           uses draw n; the direction draw 0 (32-bit map) or the accepting
 *           trial's low bits (23-bit map, the FP32 comparison).
 *
 * Every function below names the passage of the paper it follows.  Where the
 * paper is silent the reading taken is stated at the function.
 */
#ifndef SU2_ORACLE_H
#define SU2_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sampler choice for the a0 draw of Section 2, Eq. 8. */
enum { ORACLE_KP = 0, ORACLE_CREUTZ = 1 };

typedef struct {
  double beta;          /* Section 2, Eq. 5: beta = 4/g0^2                   */
  uint64_t seed;        /* Philox key                                        */
  uint32_t lattice_id;  /* batch member, 0 for a single lattice              */
  int max_tries;        /* cap on sampler trials, >= 1                       */
  int sampler;          /* ORACLE_KP or ORACLE_CREUTZ                        */
  int u23;              /* 0: uniforms with 32-bit resolution, direction    */
                        /* from draw 0; 1 (the FP32 map): 23-bit uniforms,  */
                        /* direction from the accepting trial's low bits    */
} oracle_chain;

/* Counts collected by a substep or sweep. */
typedef struct {
  uint64_t updates;     /* links visited                                     */
  uint64_t trials;      /* sampler trials evaluated                          */
  uint64_t capped;      /* links whose trials all failed (old link kept)     */
  uint64_t haar;        /* links drawn from the Haar measure (alpha ~ 0)     */
} oracle_stats;

/* Threads the substep loop runs on (1 unless built with OpenMP). */
int oracle_threads(void);

/* --- random numbers ---------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double oracle_u01(uint32_t x, int u23);
void oracle_draw_words(const oracle_chain* c, long s, int mu, uint32_t sweep, uint32_t draw,
                       uint32_t r[4]);
void oracle_draw(const oracle_chain* c, long s, int mu, uint32_t sweep, uint32_t draw,
                 double u[4]);

/* --- SU(2) algebra (Section 2, Eqs. 1-3) -------------------------------- */
void oracle_qmul(const double a[4], const double b[4], double out[4]);
void oracle_qdag(const double a[4], double out[4]);

/* --- lattice geometry --------------------------------------------------- */
long oracle_volume(int nd, const int* dims);
long oracle_shift(int nd, const int* dims, long s, int mu, int step);

/* --- start configurations (Section 4, kernel list: cold / hot start) ---- */
void oracle_init_cold(int nd, const int* dims, double* U);
void oracle_init_hot(int nd, const int* dims, const oracle_chain* c, double* U);
/* the hot-start value of the single link (s, mu) */
void oracle_hot_link(const oracle_chain* c, long s, int mu, double q[4]);

/* --- heat bath (Section 2, Eqs. 5-9 and 11) ----------------------------- */
void oracle_staple(int nd, const int* dims, const double* U, long s, int mu, double out[4]);
int oracle_sample_a0(const oracle_chain* c, double alpha, long s, int mu, uint32_t sweep,
                     double* a0, double* margin);
int oracle_heatbath_link(const oracle_chain* c, long s, int mu, uint32_t sweep,
                         const double sigma[4], const double old_link[4], double new_link[4],
                         double* margin);
void oracle_substep(int nd, const int* dims, double* U, const oracle_chain* c, uint32_t sweep,
                    int mu, int parity, oracle_stats* st, double* margin);
void oracle_sweep(int nd, const int* dims, double* U, const oracle_chain* c, uint32_t sweep,
                  oracle_stats* st);

/* --- over-relaxation (Section 2, Eq. 10) -------------------------------- */
void oracle_overrelax_substep(int nd, const int* dims, double* U, int mu, int parity);

/* --- measurements (Section 2, Eqs. 12-15, 18, 19) ----------------------- */
void oracle_plaquette(int nd, const int* dims, const double* U, double out[3]);
double oracle_polyakov(int nd, const int* dims, const double* U);
void oracle_wilson_loops(int nd, const int* dims, const double* U, int rmax, int tmax,
                         double* out);
void oracle_ape_step(int nd, const int* dims, const double* Uin, double* Uout, double alpha);

#ifdef __cplusplus
}
#endif
#endif
