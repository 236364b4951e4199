/*
 * su2.h -- C ABI of libsu2, a GB300 (sm_103a) implementation of the quenched
 * SU(2) lattice gauge theory Monte Carlo of Cardoso & Bicudo, "SU(2) Lattice
 * Gauge Theory Simulations on Fermi GPUs" (arXiv:1010.4834).
 *
 * The calls follow the paper's statement of the problem: start configurations
 * (Section 4, kernel list: cold start, hot start, read a configuration), the
 * checkerboard heat-bath update (Section 2, Eqs. 5-9 and 11; Section 4, one
 * direction and one site parity at a time), over-relaxation
 * (Section 2, Eq. 10) and the measurements: plaquette (Eqs. 12-13), Polyakov
 * loop (Eqs. 14-15), Wilson loops (Eq. 18) and APE smearing (Eq. 19).
 *
 * Conventions
 *   dims     (N0, N1, N2, N3) = (Nx, Ny, Nz, Nt); direction 3 is time.
 *            Every extent is even and >= 2 (the checkerboard needs even
 *            periodic extents); otherwise SU2_EINVAL.
 *   site     s = x0 + N0*(x1 + N1*(x2 + N2*x3)); parity (x0+x1+x2+x3) mod 2.
 *   link     quaternion (q0,q1,q2,q3) <-> q0*1 + i(q1 s1 + q2 s2 + q3 s3)
 *            (Section 2, Eq. 1).
 *   host     "canonical" host arrays are double[V][4][4]: site-major,
 *            direction, quaternion component -- 16 doubles per site.
 *   RNG      Philox4x32-10 keyed by (seed_lo, seed_hi); counter
 *            (site, mu | lattice_id << 2, sweep, draw).  The hot start uses
 *            sweep index 0xFFFFFFFF.  Heat-bath sweep i (counted from 0 since
 *            the start) uses sweep index i, so a resumed chain replays the
 *            same stream.  Trial n of a link uses draw n; its direction on
 *            the sphere comes from draw 0 (F64) or from the nine low bits of
 *            each word of the accepting trial's draw (F32, F16Q: the bits
 *            their 23-bit uniforms leave unused).
 *   device   links live on the device in a structure of arrays: for each
 *            direction mu and parity p, a contiguous array of the V/2 links
 *            of that class, ordered by s >> 1.  Element: 2 x double2 (F64),
 *            float4 (F32) or 4 x binary16 (F16Q, normalised in FP32 on load).
 *
 * Errors: every call returns an int status (SU2_OK = 0 on success).  No
 * exception crosses the ABI.  su2_last_error() gives a message for the last
 * failing call on the calling thread.  A failed call leaves the handle usable
 * unless it returned SU2_ECUDA, in which case the CUDA context may be lost.
 *
 * Streams: each handle carries one CUDA stream (NULL -> a stream the library
 * creates).  All device work of a call is enqueued on it in order.  Calls
 * that return host values (measurements, get_links, sweep_count with device
 * state) synchronise that stream before returning.
 *
 * Ownership: handles are owned by the library until su2_destroy /
 * su2_batch_destroy.  Host arrays passed in are owned by the caller and only
 * read or written during the call.  With su2_init_external the device buffer
 * belongs to the caller and must outlive the handle.
 *
 * Threading: a handle must not be used from two threads at once.
 */
#ifndef SU2_H
#define SU2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SU2_OK 0
#define SU2_EINVAL 1   /* an argument is out of range                         */
#define SU2_ENOMEM 2   /* device or host allocation failed / buffer too small */
#define SU2_ECUDA 3    /* a CUDA call failed; see su2_last_error()            */
#define SU2_ETIMEOUT 4 /* a bounded device-side wait gave up                  */
#define SU2_ESTATE 5   /* call not valid in the handle's current state        */

/* start configurations (Section 4, kernel list) */
#define SU2_COLD 0 /* every link = 1                                          */
#define SU2_HOT 1  /* every link Haar-random (Section 2, Eq. 4)               */

/* link storage precision */
#define SU2_F64 0  /* FP64 links, FP64 arithmetic                             */
#define SU2_F32 1  /* FP32 links, FP32 arithmetic, FP64 reductions            */
#define SU2_F16Q 2 /* binary16 quaternion storage, normalised on load, FP32   */

/* a0 sampler for Section 2, Eq. 8 */
#define SU2_SAMPLER_KP 0     /* Kennedy-Pendleton (default)                   */
#define SU2_SAMPLER_CREUTZ 1 /* Creutz, the method the paper cites            */

/* heat-bath sweep schedule (su2_set_schedule) */
#define SU2_SCHED_AUTO 0    /* the library's choice: substeps (the faster on GB300)         */
#define SU2_SCHED_SUBSTEP 1 /* eight substep launches per sweep                           */
#define SU2_SCHED_PAIR 2    /* four fused parity-pair launches per sweep (FP32, F16Q)     */

typedef struct su2_lattice su2_lattice;
typedef struct su2_batch su2_batch;

/* Thread-local message describing the last failure on this thread ("" if none). */
const char* su2_last_error(void);

/* Library version string. */
const char* su2_version(void);

/*
 * Device bytes a lattice of these extents and precision needs: the link store,
 * the two APE buffers (spatial links only) and reduction scratch.  For
 * su2_init_external.  Returns SU2_EINVAL for bad extents or precision.
 */
int su2_required_bytes(const int dims[4], int prec, size_t* bytes);

/*
 * Create a lattice and initialise it (Section 4: cold or hot start).
 * beta >= 0 (Section 2, Eq. 5: beta = 4/g0^2).  `cuda_stream` is a
 * cudaStream_t or NULL (the library then creates its own stream).  The
 * library allocates su2_required_bytes() of device memory.
 */
int su2_init(su2_lattice** h, const int dims[4], double beta, uint64_t seed, int start, int prec,
             void* cuda_stream);

/*
 * As su2_init, but all device memory comes from the caller: `dev_buf` is a
 * device pointer to `bytes` >= su2_required_bytes() bytes, 256-byte aligned,
 * which the caller keeps alive until su2_destroy.  SU2_ENOMEM if too small,
 * SU2_EINVAL if NULL or not 256-byte aligned.
 */
int su2_init_external(su2_lattice** h, const int dims[4], double beta, uint64_t seed, int start,
                      int prec, void* dev_buf, size_t bytes, void* cuda_stream);

/* Release the handle and any memory the library allocated for it.  NULL is a no-op. */
int su2_destroy(su2_lattice* h);

/* Replace the handle's stream (NULL -> the library's own stream). */
int su2_set_stream(su2_lattice* h, void* cuda_stream);

/*
 * Sampler options.  max_tries >= 1 (default 64): trials of the a0 sampler per
 * link before the old link is kept (an exact step: the accepted-value kernel is
 * proportional to the target and independent of the old link).  max_tries = 1
 * reproduces the single-trial setting of the paper's benchmarks (Section 5.1).
 * sampler: SU2_SAMPLER_KP or SU2_SAMPLER_CREUTZ.
 */
int su2_set_options(su2_lattice* h, int max_tries, int sampler);

/* Change beta (>= 0) for subsequent sweeps. */
int su2_set_beta(su2_lattice* h, double beta);

/*
 * How heat-bath sweeps are launched; the links they leave are the same
 * either way (every draw is keyed by sweep, site and direction, and the
 * links of one (direction, parity) class are independent).
 * SU2_SCHED_SUBSTEP: eight launches per sweep, one per (direction, parity)
 * substep (Section 4's order).  SU2_SCHED_PAIR: four launches, each running
 * the two parities of one direction as a wavefront over time slices so that
 * the links the pair shares are re-read from L2 instead of device memory
 * (parity 1 of slice t starts once parity 0 of slices t-1, t, t+1 is final);
 * FP32 and F16Q only (SU2_EINVAL for FP64).  SU2_SCHED_AUTO (the default)
 * runs substeps: measured on GB300 the pair is slower at every lattice size
 * (64^4 FP32: about 500 us per pair launch against 375 us for its two
 * substeps), because the substep kernel is bound by memory latency and
 * instruction issue rather than by the traffic the pair saves.
 * The pair's dependency waits are bounded; if one gives up, the next call
 * that synchronises returns SU2_ETIMEOUT and the links are undefined.
 * Drops the cached sweep graphs.
 */
int su2_set_schedule(su2_lattice* h, int schedule);

/*
 * n in 0..16 over-relaxation sweeps (Section 2, Eq. 10; as
 * su2_overrelax_sweep) before every heat-bath sweep of su2_heatbath_sweep
 * and su2_sweep_measure, the usual way to shorten autocorrelation times.
 * They come first because over-relaxation keeps the total action but not
 * its spatial / space-time split, which su2_sweep_measure takes from the
 * heat bath's own staples.  Default 0.  Drops the cached sweep graphs.
 */
int su2_set_overrelax(su2_lattice* h, int n);

/*
 * n >= 0 heat-bath sweeps.  One sweep = for mu = 0..3, for parity = 0, 1:
 * update every link of direction mu on sites of that parity from its staple
 * sum (Section 2, Eqs. 5-9, 11; Section 4).  Advances the sweep counter by n
 * and invalidates the APE-smeared copy.  Stream-ordered, does not synchronise.
 */
int su2_heatbath_sweep(su2_lattice* h, int n);

/*
 * Re-run the start configuration in place (Section 4: cold or hot start with
 * the handle's seed), reset the sweep counter to 0 and drop the smeared copy.
 * Stream-ordered, does not synchronise.
 */
int su2_restart(su2_lattice* h, int start);

/*
 * The Monte Carlo production loop: n >= 0 times (one heat-bath sweep, then
 * su2_plaquette and su2_polyakov of the new configuration).  hist[4*i + k]
 * receives, for sweep i of this call, the three plaquette means (k = 0..2)
 * and the Polyakov loop (k = 3).  Results stay on the device until the end
 * of the call (one synchronisation per 1024 sweeps).  Advances the sweep
 * counter by n.  The plaquette is summed inside the sweep (in the
 * odd-parity substeps of mu = 1, 2, 3, from their staples), so it equals
 * su2_plaquette of the new configuration up to the order of summation (a
 * link whose first a0 trial was rejected adds its term in whichever thread
 * finishes it, which can change from run to run, so the plaquette can vary
 * in its last bits, about 1e-11 on 64^4 FP32, while the links do not); the
 * Polyakov loop equals su2_polyakov; the links are the same as after
 * su2_heatbath_sweep.  A measured sweep is nine launches (eight substeps and
 * the Polyakov kernel, which also finishes the plaquette and advances the
 * device sweep counter); runs of eight replay from a cached CUDA graph that
 * su2_set_beta and su2_set_options drop.  hist is caller-owned host memory
 * of 4 n doubles; n < 0, or hist NULL with n > 0, returns SU2_EINVAL.
 */
int su2_sweep_measure(su2_lattice* h, int n, double* hist);

/*
 * The link-layout comparison of Section 5.1 (one array holding all links,
 * the four directions of a site next to each other, against one array per
 * direction), run on this GPU.  FP32 handles only (SU2_EINVAL otherwise);
 * sweeps >= 1.  From the current configuration the call runs `sweeps`
 * heat-bath sweeps three times: with the library's own kernels (ms[0]), with
 * a plain one-thread-per-link kernel on the library's layout (ms[1]), and
 * with the same plain kernel on a site-major single array, element
 * 4 s + mu (ms[2]); ms[] are CUDA-event times on the handle's stream,
 * conversions excluded.  *mismatch receives the number of 16-byte links in
 * which the second and third results differ from the first (0 expected: the
 * three run the same arithmetic).  The handle ends in the state of the first
 * run (sweep counter advanced by `sweeps`).  Allocates and frees two link
 * stores of device memory; synchronises.
 */
int su2_layout_compare(su2_lattice* h, int sweeps, double ms[3], uint64_t* mismatch);

/*
 * One checkerboard substep (direction mu in 0..3, parity in 0..1) of the heat
 * bath with Philox sweep index `sweep`.  Does not change the sweep counter.
 * Exposed for parity tests and custom schedules.
 */
int su2_heatbath_substep(su2_lattice* h, int mu, int parity, uint32_t sweep);

/*
 * Both substeps of direction mu (parity 0, then parity 1) with Philox sweep
 * index `sweep`, as one fused launch (see su2_set_schedule); leaves the links
 * that su2_heatbath_substep(mu, 0, sweep) then (mu, 1, sweep) leave.  FP32
 * and F16Q only (SU2_EINVAL for FP64).  Does not change the sweep counter.
 * Exposed for parity tests and custom schedules.
 */
int su2_heatbath_pair(su2_lattice* h, int mu, uint32_t sweep);

/*
 * n >= 0 over-relaxation sweeps, U -> W U^dagger W with W = Sigma/|Sigma|
 * (Section 2, Eq. 10, read for the staple orientation of Eq. 11).  Same
 * direction/parity order as the heat bath.  Deterministic; the sweep counter
 * is unchanged.
 */
int su2_overrelax_sweep(su2_lattice* h, int n);

/*
 * Mean plaquette (Section 2, Eqs. 12-13), as the mean of (1/2) Re Tr of the
 * plaquette: out[0] over all 6V plaquettes, out[1] over the 3V spatial ones,
 * out[2] over the 3V space-time ones.  1 on the cold start; the paper's
 * <P> per plaquette is 1 - out[0].  Per-thread sums (compensated in FP32),
 * then FP64 block and final sums in a fixed order.
 * Synchronises.
 */
int su2_plaquette(su2_lattice* h, double out[3]);

/*
 * The paper has no counterpart to this entry point: it is su2_plaquette for
 * callers that cannot allocate device memory -- a framework whose caching
 * allocator must own every device byte, a service with a fixed memory
 * budget, or a loop that cannot accept cudaMalloc's implicit device
 * synchronisation.  It needs no handle: `links` is a device pointer to a link
 * store in the layout described above (for a handle made with
 * su2_init_external it is the start of the caller's buffer), `dims` and
 * `prec` describe it, out[3] (host) receives what su2_plaquette returns.  The
 * reduction scratch is a fixed 64 KiB array in the library's device memory
 * (one partial per block, at most 4096 blocks; SU2_EINVAL if a device would
 * need more).  The call allocates nothing.  The first call on each device
 * looks the array's address up with that device current; make it before any
 * stream capture.  The address is kept for the life of the process: after a
 * cudaDeviceReset of that device it is stale, and the entry point must not
 * be called on that device again.  All calls share the array: calls that
 * overlap on the GPU race, so serialise them.  `cuda_stream` NULL is the
 * legacy default stream.  Synchronises the stream.
 */
int su2_plaquette_static(const void* links, const int dims[4], int prec, double out[3], void* cuda_stream);

/*
 * Support for splitting one lattice into time slabs over several GPUs
 * (Section 4's multi-GPU decomposition; the driver is
 * paper_1010_4834_gb300/tslab.py).  A slab is a lattice of its own whose
 * first and last time slices are copies of the neighbouring slabs' boundary
 * slices (ghosts).
 *
 * su2_set_site_offset: the Philox counter of local site s uses site word
 * s + site0 (mod 2^32) in every later draw (heat bath, hot start), so that a
 * slab draws the numbers of the whole lattice: site0 = (global time of local
 * slice 0) x N0 N1 N2.  Default 0.  Drops the cached sweep graphs.
 *
 * su2_plaquette_slices: as su2_plaquette, over the plaquettes whose base site
 * lies in time slices [t_first, t_first + t_count) only (means over those
 * 6 N0 N1 N2 t_count plaquettes).  SU2_EINVAL for a range outside the
 * lattice.  Synchronises.
 *
 * su2_time_lines: for every spatial site xs (index x0 + N0 (x1 + N1 x2)) the
 * product U_3(xs, t_first) U_3(xs, t_first + 1) ... of the time links of
 * slices [t_first, t_first + t_count), in FP64, to out[4 xs .. 4 xs + 3]
 * (caller-owned host memory of 4 N0 N1 N2 doubles); the slabs' lines,
 * multiplied in time order, give the Polyakov loop (Eqs. 14-15).
 * SU2_EINVAL for a range outside the lattice.  Synchronises.
 */
int su2_set_site_offset(su2_lattice* h, uint32_t site0);
int su2_plaquette_slices(su2_lattice* h, int t_first, int t_count, double out[3]);
int su2_time_lines(su2_lattice* h, int t_first, int t_count, double* out);

/*
 * Signed Polyakov loop (Section 2, Eqs. 14-15): mean over the N0 N1 N2
 * spatial sites of (1/2) Tr of the product of time links in increasing t.
 * Synchronises.
 */
int su2_polyakov(su2_lattice* h, double* L);

/*
 * n >= 0 APE smearing steps with 0 <= alpha < 1 (Section 2, Eq. 19):
 * U'_mu = P[(1-alpha) U_mu + (alpha/4) (sum of the four spatial staples)],
 * spatial mu only, Jacobi update, P = normalisation.  The paper's w relates by
 * w = alpha / (4 (1 - alpha)).  Writes the smeared copy; the Markov chain is
 * untouched.  n = 0 makes the smeared copy equal to the current links.
 */
int su2_ape_smear(su2_lattice* h, double alpha, int n);

/*
 * Wilson loops (Section 2, Eq. 18): out[(R-1)*Tmax + (T-1)] for 1 <= R <= Rmax,
 * 1 <= T <= Tmax, the mean over all sites and the three spatial directions of
 * (1/2) Tr of the R x T loop.  1 <= Rmax <= min(N0,N1,N2), 1 <= Tmax <= N3,
 * Rmax, Tmax <= 32.  use_smeared = 1 takes the spatial links from the last
 * su2_ape_smear (SU2_ESTATE if there is none since the last sweep or
 * set_links); temporal links are always the chain's.  For Rmax, Tmax <= 16
 * and N3 / 8 in {1, 2, 4, 6, 8} the loops are evaluated in temporal gauge
 * (the loop is gauge invariant: after the transform each is one dot
 * product of two spatial lines), which equals the direct product up to
 * rounding; other shapes multiply the loops out.  Synchronises.
 */
int su2_wilson_loops(su2_lattice* h, int Rmax, int Tmax, int use_smeared, double* out);

/*
 * Copy links to / from caller-owned host memory in the canonical FP64 layout
 * (4V quaternions, 16 doubles per site).  set_links converts to the handle's
 * precision (F16Q rounds to binary16), invalidates the smeared copy and keeps
 * the sweep counter.  Both synchronise.  set_links from page-locked host
 * memory (cudaHostAlloc, cudaHostRegister) lets the conversion kernel read
 * the host buffer directly; set_links also takes device (or managed) memory
 * of the handle's device in the same layout, which the conversion kernel
 * reads on the handle's stream (the caller makes sure it is ready there,
 * e.g. filled by an earlier copy on that stream or after an event wait);
 * pageable host memory goes through a device staging buffer in chunks.
 */
int su2_get_links(su2_lattice* h, double* host);
int su2_set_links(su2_lattice* h, const double* links);

/*
 * The links of sites [first, first + count) (lexicographic site index, as in
 * the canonical layout) into host[16 * count], for lattices too large to
 * copy whole.  SU2_EINVAL if the range leaves the lattice.  Synchronises.
 */
int su2_get_sites(su2_lattice* h, int64_t first, int64_t count, double* host);

/*
 * Number of CUDA kernels this library has launched in this process (all
 * handles; a replayed sweep graph counts each of its kernels).
 */
int su2_kernel_launches(uint64_t* n);

/*
 * The paper has no counterpart to this entry point: a measurement helper.
 * *flops_per_s receives this device's fused multiply-add throughput in
 * prec SU2_F64 or SU2_F32 (2 flops per FMA), from a probe kernel of `iters`
 * >= 1 rounds of eight independent FMA chains per thread over a grid that
 * fills every SM, timed with CUDA events after a warm-up launch.  It is the
 * denominator of the rooflines of arithmetic-bound kernels (the FP64 heat
 * bath, the Wilson loops).  Allocates and frees a small output buffer and a
 * stream; synchronises.  SU2_EINVAL for other precisions or iters < 1.
 */
int su2_probe_fma(int prec, int iters, double* flops_per_s);

/* Sweep counter: heat-bath sweeps done since the start (or as set by set_sweep_count / load). */
int su2_sweep_count(su2_lattice* h, uint64_t* n);
int su2_set_sweep_count(su2_lattice* h, uint64_t n);

/*
 * Checkpoint (Section 4 lists reading a configuration from a file): a binary
 * file with a header (magic "SU2GB300", version, dims, beta, seed, sweep
 * counter, precision, sampler options) followed by the canonical FP64 links.
 * su2_load creates a new handle with precision `prec` (-1: as saved).
 */
int su2_save(su2_lattice* h, const char* path);
int su2_load(su2_lattice** h, const char* path, int prec, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched lattices: n independent lattices with their own extents and beta,
 * swept together.  Lattice i uses Philox lattice_id = i.
 * ------------------------------------------------------------------------- */

/*
 * dims: n x 4 extents (each lattice obeys the su2_init rules and has fewer
 * than 2^30 sites, since the batched kernel addresses a lattice's links by
 * 32-bit offsets; SU2_EINVAL otherwise), betas: n couplings >= 0,
 * 1 <= n <= 1023.  Cold or hot start per lattice.  prec: SU2_F32 or SU2_F64
 * or SU2_F16Q.
 */
int su2_batch_init(su2_batch** b, int n, const int* dims, const double* betas, uint64_t seed,
                   int start, int prec, void* cuda_stream);
int su2_batch_destroy(su2_batch* b);
int su2_batch_set_options(su2_batch* b, int max_tries, int sampler);

/*
 * n heat-bath sweeps of every lattice, in one persistent cooperative kernel
 * launch per call (replayed from a CUDA graph).  The lattices are dealt to G
 * groups (largest first, each to the group with the least work), and every
 * group gets a share of the grid's CTAs in proportion to its work; a group
 * sweeps its lattices one lattice at a time, the eight substeps of a
 * lattice ordered by bounded barriers among the group's CTAs (a group of
 * one CTA needs only the block barrier).  Results do not depend on G (every draw is keyed by
 * lattice, sweep, site and direction).  SU2_ETIMEOUT if a barrier wait gave
 * up (bounded by a 1 s timer): the links of every lattice are then undefined,
 * while the handle itself recovers -- its barriers and error flag are cleared
 * and its sweep counter is back at its value before the call -- so the caller
 * can reload the lattices with su2_batch_set_links and sweep again.
 */
int su2_batch_sweep(su2_batch* b, int n);

/*
 * n in 0..16 over-relaxation sweeps (Section 2, Eq. 10) of every lattice
 * before each of its heat-bath sweeps, inside the same persistent launch
 * (as su2_set_overrelax for one lattice).  Default 0.
 */
int su2_batch_set_overrelax(su2_batch* b, int n);

/*
 * The schedule's group count G (1 <= G <= min(lattices, co-resident CTAs)),
 * i.e. the number of lattices swept at the same time.  The default is one
 * group per lattice (all in flight), capped at the co-resident CTAs.
 * su2_batch_set_block_size: threads per CTA of the batched kernel, 256 (the
 * default) or 512 (SU2_EINVAL otherwise); the co-resident grid follows and the
 * group count is kept, capped at the new grid.
 * su2_batch_tune times `sweeps` sweeps for every candidate pair (block size,
 * G) on a scratch copy of the links (the chain is not advanced; it allocates
 * and frees that copy), keeps the fastest and returns its G in *groups (may
 * be NULL; su2_batch_block_size gives the block size).
 */
int su2_batch_set_groups(su2_batch* b, int groups);
int su2_batch_groups(su2_batch* b, int* groups);
int su2_batch_set_block_size(su2_batch* b, int threads);
int su2_batch_block_size(su2_batch* b, int* threads);
int su2_batch_tune(su2_batch* b, int sweeps, int* groups);

/*
 * n measured sweeps (n >= 1): the chain of su2_batch_sweep(b, n), and after
 * each sweep s of this call and each lattice i the lattice's plaquette
 * (all, spatial, space-time; Section 2, Eq. 12) and Polyakov loop
 * (Eqs. 14-15) as su2_sweep_measure gives them, in
 * hist[(s * n_lattices + i) * 4 + k] (host, n * n_lattices * 4 doubles,
 * owned by the caller).  One persistent cooperative launch: after the eight
 * substeps of a lattice's sweep its group adds the plaquettes at, and the
 * time-ordered products of time links through, its share of the sites, and
 * the group's first CTA adds the CTAs' sums in a fixed order (the values
 * depend on the group count only through that order).  Allocates and frees
 * a device buffer of the history's size; synchronises.  SU2_ETIMEOUT as for
 * su2_batch_sweep (hist is then not written).
 */
int su2_batch_sweep_measure(su2_batch* b, int n, double* hist);

/* out[3*i + k]: su2_plaquette of lattice i.  Synchronises. */
int su2_batch_plaquette(su2_batch* b, double* out);
/* out[i]: su2_polyakov of lattice i.  Synchronises. */
int su2_batch_polyakov(su2_batch* b, double* out);
/* Canonical FP64 links of lattice i (V_i * 16 doubles).  Synchronises. */
int su2_batch_get_links(su2_batch* b, int i, double* host);
int su2_batch_set_links(su2_batch* b, int i, const double* host);

#ifdef __cplusplus
}
#endif
#endif /* SU2_H */
