/*
 * ising.h — C ABI of the GB300-native Ising-film Monte Carlo library.
 *
 * The library runs the checkerboard single-spin-flip Metropolis sweep of the
 * nearest-neighbour Ising model on an Lx x Ly x Lz simple-cubic film (Block,
 * Kim, Virnau & Binder, arXiv:1411.5588) and the integer observable sums that
 * feed the paper's thermodynamic integrations, entirely in CUDA kernels for
 * sm_103a.  Nothing here takes a framework type: arguments are plain values,
 * host pointers (marked "host") or device pointers (marked "device").
 *
 * Model (Eq. 1, Sec. II A):
 *   E = -J sum_<ij> S_i S_j - H sum_i S_i - H1 sum_{kx=1} S_i - Hn sum_{kx=Lx} S_i,
 *   Hn = -H1, S_i = +-1, sites (kx,ky,kz) with 1-based indices.
 *   x: free surfaces at kx = 1 and kx = Lx (ISING_X_PBC is a test geometry).
 *   z: periodic.
 *   y: ISING_Y_GAPBC, the generalized antiperiodic rule of Eq. 11,
 *      S(kx, ky +- Ly, kz) = -S(Lx+1-kx, ky, kz); ISING_Y_PBC and ISING_Y_APBC
 *      are the plain periodic / antiperiodic films of Sec. II C (Eq. 20).
 *
 * Dynamics (Appendix: checkerboard update; the rule itself is Metropolis):
 *   one sweep = four phases, colour c = (kx+ky+kz) mod 2:
 *   {c=0, ky<Ly}, {c=0, ky=Ly}, {c=1, ky<Ly}, {c=1, ky=Ly}.
 *   A site flips iff dE <= 0 or u < floor(exp(-dE/T) * 2^32), with
 *   dE = 2 s (J sigma + h) in binary64 (h = H, += H1 on kx=1, += Hn on kx=Lx)
 *   and u word (z0>>1)&3 of Philox4x32-10 with counter
 *   (row = (kx-1)*Ly + (ky-1), z0>>3, sweep, z0&1), z0 = kz-1, key
 *   (lo32(seed) ^ hi32(seed), replica).  Sweeps are numbered from 0 and must
 *   stay below 0xFFFFFFFF.  Initial states draw from counter
 *   (row, z0>>3, 0xFFFFFFFF, 2 | (z0&1)).
 *
 * Records (Eqs. 1, 7, 9, 17, 19): one record is 5 + Lx int64,
 *   {sweeps completed, B, M, M1, Mn, m(1), ..., m(Lx)}, where
 *   B = sum over bonds of sigma_b S_i S_j (sigma_b = -1 on the antiperiodic
 *   wrap bonds; a pair joined through two neighbour slots, e.g. Lz = 2,
 *   counts twice), M = sum S, M1 = m(1), Mn = m(Lx) and m(kx) is the sum of
 *   layer kx.  The energy is E = -J B - H M - H1 M1 - Hn Mn.
 *
 * Memory: the library owns every device buffer it allocates; callers own
 * every pointer they pass.  Spins are bit-packed on the device (1 bit per
 * site).  Host spin arrays use the canonical int8 order
 * ((kx-1)*Ly + (ky-1))*Lz + (kz-1), values +1 / -1.
 *
 * Errors: every call returns an ISING_* status; nothing aborts, and no
 * kernel traps.  ising_last_error() gives a one-line message for the calling
 * thread.  A call that fails with ISING_ECUDA or ISING_ENOMEM has consumed
 * the CUDA runtime's pending error, so the failure does not resurface in a
 * later call (a sticky error, which leaves the context unusable, persists).
 * Device waits inside the library are bounded and report ISING_ETIMEOUT.  A
 * handle may be used from one host thread at a time.
 */
#ifndef ISING_GB300_H
#define ISING_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ISING_OK = 0,
    ISING_EINVAL = 1,   /* bad argument or unsupported size */
    ISING_ENOMEM = 2,   /* device or host allocation failed / budget exceeded */
    ISING_ECUDA = 3,    /* a CUDA runtime call failed */
    ISING_ETIMEOUT = 4, /* a bounded wait ran out */
    ISING_EBUSY = 5,    /* the object is in use (e.g. jobs still running) */
    ISING_ENOTFOUND = 6 /* unknown ticket / job */
};

enum { ISING_Y_GAPBC = 0, ISING_Y_PBC = 1, ISING_Y_APBC = 2 };
enum { ISING_X_FREE = 0, ISING_X_PBC = 1 };
enum { ISING_INIT_RANDOM = 0, ISING_INIT_SLAB_Y = 1, ISING_INIT_ALL_UP = 2 };
/* Launch shapes of the sweep (identical chains and records for every one):
 * RESIDENT  one block keeps the whole film in shared memory for a whole
 *           ising_sweep call (films of at most 65536 spins whose packed
 *           planes fit in 48 KiB);
 * GRID_1    two grid launches per sweep, one 32-site word per thread: the
 *           shortest launch latency.  A recorded sweep's second launch also
 *           sums the record, and a small kernel writes it;
 * GRID_2    the same with two words per thread, which overlaps one word's
 *           loads with the other's arithmetic;
 * GRID_Q    the same with four threads per word, each drawing two of its
 *           eight Philox calls: four times the threads for the same work,
 *           for films too small to fill the GPU otherwise.
 * CLUSTER   a thread-block cluster of C CTAs keeps a film in distributed
 *           shared memory for all sweeps of an ising_sweep or
 *           ising_batch_sweep call, CTA r holding layers [r Lx / C,
 *           (r+1) Lx / C) of both parity planes, a cluster barrier between
 *           half-sweeps; then it takes its next film.  A single film runs on
 *           one cluster of the largest C <= 8 it qualifies for (see
 *           ising_batch_set_shape).  In a batch each lane runs
 *           n_SM / (C lanes) clusters, one CTA per SM, and its films go to
 *           them largest first, each to the cluster with the least work so
 *           far.  Films never wait for one another and no launch boundary
 *           falls between half-sweeps (the Appendix's many independent
 *           films, each on its own few SMs).
 * AUTO      the autotuner's measurement for this film shape and record
 *           interval if there is one, else RESIDENT up to 32768 spins and
 *           GRID_1 above. */
enum { ISING_SHAPE_AUTO = 0, ISING_SHAPE_RESIDENT = 1, ISING_SHAPE_GRID_1 = 2, ISING_SHAPE_GRID_2 = 3,
       ISING_SHAPE_GRID_Q = 4, ISING_SHAPE_CLUSTER = 5 };

typedef struct ising ising;

/* ------------------------------------------------------------ one film */

/* Create a film on the current CUDA device (Eq. 1, Sec. II A).
 * Lx >= 1, Ly >= 2, Lz >= 2 and even, T > 0 (T = +inf means beta = 0).
 * Starts all spins +1, y = GAPBC, x free, H = 0, replica 0, sweep 0.
 * *out receives the handle (host pointer).  EINVAL / ENOMEM / ECUDA. */
int ising_create(int Lx, int Ly, int Lz, double J, double H1, double T, uint64_t seed, ising **out);

/* Boundary modes, bulk field H and RNG replica index (key word 1).
 * x_mode = ISING_X_PBC needs Lx even.  Resets nothing else.  EINVAL. */
int ising_set_options(ising *h, int y_mode, int x_mode, double H, uint32_t replica);

/* Change the temperature (T > 0 or +inf) and the surface field H1 of Eq. 1;
 * rebuilds the acceptance thresholds.  EINVAL. */
int ising_set_params(ising *h, double J, double H1, double T);

/* Stream used for every launch and copy of this handle (a cudaStream_t
 * passed as void*; NULL = the library's own stream).  The caller keeps the
 * stream alive while the handle uses it. */
int ising_set_stream(ising *h, void *cuda_stream);

/* Initial state, drawn on the device: RANDOM (S = +1 iff u < 2^31), SLAB_Y
 * (S = +1 for ky <= Ly/2 else -1, then each spin reversed iff
 * u < floor(flip_p 2^32), 0 <= flip_p <= 1) or ALL_UP.  Sets sweep = 0 and
 * drops pending records. */
int ising_init(ising *h, int kind, double flip_p);

/* Copy spins from host memory s (Lx*Ly*Lz int8, canonical order, values +-1;
 * any value > 0 reads as +1).  Stream-ordered; returns after the copy. */
int ising_set_spins(ising *h, const int8_t *s);

/* Copy spins to host memory s (Lx*Ly*Lz int8, canonical order). Synchronises. */
int ising_get_spins(ising *h, int8_t *s);

/* Device-pointer variants: s is device memory of Lx*Ly*Lz int8. Async. */
int ising_set_spins_device(ising *h, const int8_t *s);
int ising_get_spins_device(ising *h, int8_t *s);

/* Packed state exchange (device pointers): the library's own layout, of
 * ising_packed_words() uint32 words.  Async.  For checkpoints. */
size_t ising_packed_words(const ising *h);
int ising_get_packed_device(ising *h, uint32_t *dst);
int ising_set_packed_device(ising *h, const uint32_t *src);

/* Sweep counter (sweeps completed).  Setting it (with the spins) resumes a
 * chain bit-exactly; it must stay below 0xFFFFFFFF. */
int ising_get_sweep(const ising *h, uint64_t *sweep);
int ising_set_sweep(ising *h, uint64_t sweep);

/* Make room for n_records more pending records, so that later ising_sweep
 * calls do not grow the series (growth is a device allocation, a copy of the
 * pending records and a synchronisation).  ENOMEM when the series would pass
 * 2^32 - 16 records or the device cannot hold it; a refused or failed growth
 * leaves the series and the pending records as they were. */
int ising_reserve_records(ising *h, uint64_t n_records);

/* Pin the launch shape of this handle's ising_sweep calls (ISING_SHAPE_*;
 * AUTO unpins).  RESIDENT or CLUSTER on a film that does not qualify is
 * EINVAL. */
int ising_set_shape(ising *h, int shape);

/* The shape an ising_sweep(h, n, measure_every) call would use now. */
int ising_get_shape(ising *h, uint32_t measure_every, int *shape);

/* Autotuner: times every launch shape that fits the film (a few ms per
 * shape) on a scratch film of the same shape and parameters, with a record
 * every measure_every sweeps, so this handle's chain is not touched.  The
 * fastest goes into a process-wide table keyed by (Lx, Ly, Lz, boundary
 * modes, table variant, record interval up to 16) that every AUTO handle of
 * that key then uses; *shape (may be NULL) receives it.  Shapes are tried
 * in the order RESIDENT, GRID_1, GRID_2, GRID_Q, CLUSTER, and a later one must be at least 2%
 * faster to win.  Synchronises. */
int ising_autotune(ising *h, uint32_t measure_every, int *shape);

/* Enqueue n_sweeps sweeps on the handle's stream (asynchronous).  After every
 * sweep whose count of completed sweeps is a multiple of measure_every (> 0)
 * one record is appended to the handle's device-side series; 0 = no records.
 * EINVAL if the counter would reach 0xFFFFFFFF, ENOMEM if the series cannot
 * grow. */
int ising_sweep(ising *h, uint64_t n_sweeps, uint32_t measure_every);

/* Measure the current state: synchronises, then fills *out.  m_x (host,
 * caller-owned, Lx int64) receives the layer sums m(kx) when non-NULL. */
typedef struct {
    uint64_t sweep;
    int64_t bond_sum; /* B */
    int64_t M, M1, Mn;
    int64_t *m_x;
} ising_obs;
int ising_measure(ising *h, ising_obs *out);

/* Asynchronous drain: enqueue the copy of up to cap pending records (oldest
 * first, 5 + Lx int64 each) into host memory buf on cuda_stream (a
 * cudaStream_t as void*; NULL = a copy stream of the handle), ordered after
 * all work enqueued on the handle so far, so that it overlaps the sweeps
 * enqueued next.  buf should be pinned (page-locked) for the copy to be
 * asynchronous; it must stay valid until the copy completes, which it has
 * once that stream reaches this point (synchronise it, or the handle with
 * ising_synchronize after ising_read_series).  *n_records receives the count;
 * those records count as read.  Later sweeps never overwrite ring slots
 * still being copied, and growing the ring waits for the copy. */
int ising_read_series_async(ising *h, int64_t *buf, size_t cap, size_t *n_records, void *cuda_stream);

/* Drain up to cap pending records (5 + Lx int64 each, oldest first) into
 * host memory buf; *n_records receives the number copied.  Synchronises. */
int ising_read_series(ising *h, int64_t *buf, size_t cap, size_t *n_records);

/* Number of records waiting in the series. */
int ising_pending_records(const ising *h, size_t *n_records);

/* Block until all work of the handle is done (bounded by timeout_s;
 * ETIMEOUT otherwise). */
int ising_synchronize(ising *h, double timeout_s);

int ising_destroy(ising *h);

/* ------------------------------------------------- batches of replicas */

/* One job = one independent film with its own parameters and RNG key
 * (the many-H1/T integration points of Sec. II C, Eqs. 9, 19, 22). */
typedef struct {
    int32_t Lx, Ly, Lz;
    int32_t y_mode, x_mode;
    int32_t init_kind;     /* ISING_INIT_* */
    double J, H, H1, T;
    double flip_p;         /* SLAB_Y flips */
    uint64_t seed;
    uint32_t replica;
    uint32_t measure_every; /* 0 = no records */
    uint64_t n_sweeps;      /* used by the server; ignored by ising_batch_sweep */
} ising_job;

typedef struct ising_batch ising_batch;

#define ISING_MAX_LANES 16

/* Allocate and initialise n films updated together.  The films are spread
 * over `lanes` lanes (the largest film first, each to the lane with the
 * fewest sites so far); a lane's launches cover all of its films, and the
 * lanes run concurrently on their own streams, so that one lane's launch
 * boundaries overlap another's work.  Every film's chain, records and spins
 * are the same whatever the lanes.  lanes = 0: two lanes when n >= 2, else
 * one; more lanes than films are cut to n.  jobs: host array of n.
 * EINVAL (lanes > ISING_MAX_LANES) / ENOMEM. */
int ising_batch_create_lanes(const ising_job *jobs, size_t n, uint32_t lanes, ising_batch **out);
/* ising_batch_create_lanes with lanes = 0. */
int ising_batch_create(const ising_job *jobs, size_t n, ising_batch **out);
int ising_batch_get_lanes(const ising_batch *b, uint32_t *lanes);
/* The batch's stream (lane 0's; NULL: a stream of the library's own).  Each
 * ising_batch_sweep forks from it to the other lanes and joins back, so work
 * queued on it after the call sees every film swept. */
int ising_batch_set_stream(ising_batch *b, void *cuda_stream);

/* Enqueue n_sweeps sweeps of every film (asynchronous).  Records follow each
 * job's measure_every.  use_graph != 0 captures each lane's sweep chunk in a
 * CUDA graph once and replays it. */
int ising_batch_sweep(ising_batch *b, uint64_t n_sweeps, int use_graph);

/* Room for n_records more pending records of every film that records (see
 * ising_reserve_records).  ENOMEM, with every film's series as it was (lanes
 * grown before the refusal keep their larger rings). */
int ising_batch_reserve_records(ising_batch *b, uint64_t n_records);

/* Launch shape of the batch: GRID_1, GRID_2, GRID_Q, CLUSTER, or AUTO (the
 * autotuner's choice once ising_batch_autotune has run, else GRID_1).
 * CLUSTER takes the pinned cluster size (ising_batch_set_cluster_size), else
 * the largest C <= 8 for which every film qualifies and the n films' n C CTAs
 * fit on the GPU's SMs (C = 1 when the films outnumber the SMs); a film
 * qualifies for C when Lx >= C and a CTA's slab of ceil(Lx / C) layers (two
 * planes of Ly W 32-bit words each, W = ceil(Lz / 64)) plus 24 Lx bytes of
 * tables fits in 200 KiB of shared memory and the GPU can hold such a
 * cluster (cudaOccupancyMaxActiveClusters > 0).  EINVAL when none qualifies.
 * RESIDENT is EINVAL for a batch.  Changing it drops the captured graphs. */
int ising_batch_set_shape(ising_batch *b, int shape);
int ising_batch_get_shape(ising_batch *b, int *shape);
/* CTAs per film of the CLUSTER shape: 1..8, or 0 for the automatic choice
 * above.  EINVAL if > 8 or some film does not qualify (nothing changes).
 * Takes effect at once when the batch runs on the cluster path (CLUSTER
 * set, or AUTO after the autotuner chose it; 0 then restores the automatic
 * or the autotuner's size).  get: the size the batch runs with now, 0 when
 * it is on a grid shape. */
int ising_batch_set_cluster_size(ising_batch *b, uint32_t cluster_size);
int ising_batch_get_cluster_size(const ising_batch *b, uint32_t *cluster_size);

/* Autotuner: times GRID_1, GRID_2, GRID_Q and CLUSTER at every cluster size
 * for which all films qualify, on a
 * scratch batch of the same jobs in the same lanes (from their initial
 * states; the kernels' work does not depend on the spins), all lanes
 * running, graph replay and records included, and adopts the fastest for
 * every lane unless a shape is pinned; *shape (may be NULL) receives it.
 * Synchronises. */
int ising_batch_autotune(ising_batch *b, int *shape);

/* Per-film accessors (index i < n).  Host buffers; synchronise. */
int ising_batch_get_spins(ising_batch *b, size_t i, int8_t *s);
int ising_batch_read_series(ising_batch *b, size_t i, int64_t *buf, size_t cap, size_t *n_records);
/* Records of film i enqueued so far and not yet read (host counter; does not
 * synchronise). */
int ising_batch_pending_records(const ising_batch *b, size_t i, size_t *n);
/* Wait for every lane (bounded by timeout_s; ETIMEOUT otherwise). */
int ising_batch_synchronize(ising_batch *b, double timeout_s);
int ising_batch_destroy(ising_batch *b);

/* ------------------------------------------- continuous-batching server */

typedef struct ising_server ising_server;
typedef uint64_t ising_ticket;

/* A server owns a device pool of at most hbm_budget_bytes and a host thread
 * that runs chunks of chunk_sweeps sweeps over every admitted job, admits
 * queued jobs whenever their packed lattice and record series fit in the
 * pool, and retires finished jobs.  A job's result is identical whether it
 * runs alone or among others (its RNG stream depends only on its own key). */
int ising_server_create(size_t hbm_budget_bytes, uint32_t chunk_sweeps, ising_server **out);

/* Queue jobs (host array of n); *first receives the ticket of jobs[0], the
 * others follow consecutively.  EINVAL if a job can never fit the budget. */
int ising_batch_submit(ising_server *s, const ising_job *jobs, size_t n, ising_ticket *first);

/* *done = 1 once the job's sweeps are finished and its result is ready. */
int ising_batch_poll(ising_server *s, ising_ticket t, int *done);

/* Wait for one job (bounded; ETIMEOUT otherwise). */
int ising_batch_wait(ising_server *s, ising_ticket t, double timeout_s);

/* Result of a finished job: its records (host buf, cap records of 5 + Lx
 * int64) and its final spins (host, may be NULL).  Timing in seconds since
 * the server started: submit, admit and finish.  first_chunk / last_chunk:
 * the indices (from 0, in launch order) of the first and last chunk that ran
 * sweeps of the job; two jobs whose ranges intersect shared launches on the
 * device.  Frees the job's slot. */
typedef struct {
    double t_submit, t_admit, t_finish;
    uint64_t n_records;
    uint64_t first_chunk, last_chunk;
} ising_job_info;
int ising_batch_result(ising_server *s, ising_ticket t, int64_t *buf, size_t cap, int8_t *spins,
                       ising_job_info *info);

/* Pool statistics: bytes in use, jobs queued / running / finished, chunks run. */
typedef struct {
    size_t bytes_in_use, bytes_budget;
    uint64_t queued, running, finished, chunks;
    uint64_t attempts; /* spin-flip attempts done so far */
} ising_server_stats;
int ising_server_get_stats(ising_server *s, ising_server_stats *st);
int ising_server_destroy(ising_server *s);

/* ------------------------------------------- host FP64 integration */

/* Gauss-Legendre nodes and weights on [a, b] (n >= 1), Newton iteration on
 * P_n.  x, w: host arrays of n. */
int ising_gauss_legendre(int n, double a, double b, double *x, double *w);

/* Mean of records[k*stride + col] over k = first..n-1 (exact integer sum,
 * then one division).  records: host. */
int ising_series_mean(const int64_t *records, size_t n, size_t stride, size_t col, size_t first,
                      double *mean);

/* Eq. 1 from a record series (5 + Lx int64 per record): E[k] = -J B - H M
 * - H1 M1 - Hn Mn with Hn = -H1, in binary64 from each record's integers (E
 * may be NULL, else n doubles), and *mean (may be NULL) = the same
 * combination of the column means over records first..n-1, each mean an
 * exact integer sum and one division.  At least one output.  host. */
int ising_series_energy(const int64_t *records, size_t n, int Lx, double J, double H, double H1, double *E,
                        size_t first, double *mean);

/* The film's own integral over its surface field: with Hn = -H1 written
 * into Eq. 1, dF/dH1 = -(M1 - Mn), so F(H1) - F(0) = -integral_0^{H1}
 * (m_1 - m_n) dH1' per wall site, from n Gauss-Legendre nodes on [0, H1];
 * m1[i], mn[i] are the per-site layer magnetisations of layers 1 and Lx at
 * node i.  In a uniform (+) film (periodic y) this is the wall term
 * gamma+(|H1|) + gamma+(-|H1|) - 2 gamma+(0) of Eq. 21 (Eq. 7 for each
 * wall); in a film with an interface, summed over the wall sites
 * (M1, Mn totals), it is the F_int(H1) - F_int(0) of Eq. 21.  The Young
 * difference of Eq. 9 is ising_ti_young_difference.  host. */
int ising_ti_surface_field(int n, double H1, const double *m1, const double *mn, double *delta_f1);

/* Eq. 9: delta_f1(H1) = -integral_0^{H1} (m_1 + m_n) dH1' from n
 * Gauss-Legendre nodes on [0, H1], m1[i], mn[i] as above, measured in a
 * uniform film with periodic y.  By Eqs. 4 and 7 this is
 * f1(+)(H1) - f1(-)(H1), the difference of the two phases' surface free
 * energies at the wall with field H1 that enters Eqs. 8 and 16 (at T = 0 it
 * is -2 H1).  host. */
int ising_ti_young_difference(int n, double H1, const double *m1, const double *mn, double *delta_f1);

/* Eq. 19: beta F(beta_b) - beta F(beta_a) = integral U dbeta by the
 * trapezoid rule over n points (beta[i], U[i]), beta ascending or
 * descending.  host. */
int ising_ti_beta_trapezoid(int n, const double *beta, const double *U, double *out);

/* Eq. 19 written over T: integral U dbeta = -integral U / T^2 dT, trapezoid
 * in T over n points (T[i], U[i]).  host. */
int ising_ti_temperature_trapezoid(int n, const double *T, const double *U, double *out);

/* ----------------------------------------------- interfacial analysis
 * Host FP64 post-processing of Secs. II B - IV.  Every pointer is host
 * memory owned by the caller; nothing is kept.  Status ISING_EINVAL for
 * null pointers, sizes below the stated minimum or fits whose abscissae are
 * all equal. */

/* Eq. 17: mbar[kx-1] = per-site magnetisation of layer kx averaged over
 * records first..n-1 of a (5 + Lx)-int64 record series (as ising_read_series
 * writes it): exact integer sum of the m(kx) column, then one division by
 * (n - first) Ly Lz. */
int ising_layer_profile(const int64_t *records, size_t n, int Lx, int Ly, int Lz, size_t first, double *mbar);

/* Eq. 12: m_minus[kx-1] = -m_plus[Lx-kx], the (-) profile from the (+) one.
 * The arrays must not be the same. */
int ising_mirror_profile(int Lx, const double *m_plus, double *m_minus);

/* Eq. 18 with y+ + y- = Ly: y_plus[kx-1] = Ly (mbar - m-) / (m+ - m-) per
 * layer (Lx values; m+ = m- in a layer is EINVAL).  A straight-line fit of
 * y_plus over layers k_lo..k_hi (1 <= k_lo < k_hi <= Lx) gives the dividing
 * plane; theta = atan(1 / |slope|), the acute angle between the plane and
 * the walls, in (0, pi/2] (pi/2 for a plane perpendicular to the walls). */
int ising_contact_angle(int Lx, int Ly, const double *mbar, const double *m_plus, const double *m_minus, int k_lo,
                        int k_hi, double *y_plus, double *theta);

/* Eq. 8: theta = acos(|delta_f1| / gamma_pi2), the acute Young angle.
 * gamma_pi2 > 0; |delta_f1| > gamma_pi2 (a wet wall) is EINVAL. */
int ising_young_angle(double delta_f1, double gamma_pi2, double *theta);

/* Eq. 16 integrated from gamma(theta[0]) = gamma0 over n points: with
 * g = gamma / sin(theta), dg/dtheta = -delta_f1 / sin^2(theta), trapezoid
 * rule between consecutive points; gamma[i] = g_i sin(theta[i]).  theta in
 * (0, pi), in the order the points were measured (normally from pi/2 at
 * H1 = 0 downwards); delta_f1 in the sign of Eq. 16, where an isotropic
 * tension gives cos(theta) = delta_f1 / gamma (so |delta_f1| of Eq. 9 for
 * the acute angle). */
int ising_gamma_of_theta(int n, const double *theta, const double *delta_f1, double gamma0, double *gamma);

/* Eq. 19 along a path beta[0], beta[1], ... (beta > 0): beta_i F_i =
 * beta_0 F0 + integral_{beta_0}^{beta_i} U dbeta by the trapezoid rule,
 * F[0] = F0.  With U = U_APBC - U_PBC and beta_0 = 0.2 < beta_c, F0 = 0
 * gives the Delta F of Eq. 20; a low-temperature start uses F0 = U0 (the
 * ground-state energy). */
int ising_ti_free_energy_beta(int n, const double *beta, const double *U, double F0, double *F);

/* Eq. 20: least-squares line dF / (Lz Lx) = gamma_pi2 + (2 / Lx) tau0 over
 * n >= 2 films of sizes (Lx[i], Lz[i]). */
int ising_fit_gamma_tau(int n, const double *Lx, const double *Lz, const double *dF, double *gamma_pi2, double *tau0);

/* Eq. 21 solved for its line term: R = 2 Lz [tau(H1, theta) - tau(0, pi/2)]
 *   = dF_film - Lx Lz [gamma_theta / sin(theta) - gamma_pi2]
 *     - Lz Ly s_wall - Lz Lx delta_f1 / tan(theta),
 * dF_film = F_int(H1) - F_int(0) of the film with the interface (Eq. 22's
 * integral over H1), s_wall the per-site wall term of a uniform film
 * (ising_ti_surface_field), delta_f1 the Young difference (Eq. 9). */
int ising_line_tension_residual(double dF_film, double Lx, double Ly, double Lz, double theta, double gamma_theta,
                                double gamma_pi2, double s_wall, double delta_f1, double *R);

/* Sec. II C's size scan: films with Lx Lz and Ly Lz held fixed differ only
 * by 2 Lz dtau; least-squares line R = intercept + 2 dtau Lz over n >= 2
 * films. */
int ising_line_tension_lz_scan(int n, const double *Lz, const double *R, double *dtau, double *intercept);

/* Eqs. 23-24: c from the least-squares fit gamma / gamma_pi2 - 1 =
 * c (pi/2 - theta)^2 through the origin, kappa = gamma_pi2 (1 + 2c). */
int ising_stiffness(int n, const double *theta, const double *gamma, double gamma_pi2, double *c, double *kappa);

/* Eq. 25: C from the fit 1 - 2 kappa / (pi T) = C ((T - T_R) / T_c)^(1/2)
 * through the origin; every T[i] > T_R. */
int ising_roughening_kappa_fit(int n, const double *T, const double *kappa, double T_R, double T_c, double *C);

/* Eq. 26 below roughening: least-squares line gamma = gamma_flat +
 * f_s |pi/2 - theta| over n >= 2 angles near pi/2. */
int ising_step_free_energy(int n, const double *theta, const double *gamma, double *f_s, double *gamma_flat);

/* Eq. 27 with f_s proportional to 1 / xi_R: least-squares line
 * ln f_s = log_amp - A (1 - T / T_R)^(-1/2) over n >= 2 points, T < T_R,
 * f_s > 0. */
int ising_roughening_fs_fit(int n, const double *T, const double *f_s, double T_R, double *A, double *log_amp);

/* Sec. III C: the critical field H1* below which the contact angle stays at
 * pi/2, from a scan (H1[i] strictly increasing, theta[i]), n >= 2: the
 * first point whose tilt pi/2 - theta exceeds tol, and the crossing of
 * tol on the line through it and the point before.  f_s = 2 H1* +
 * T ln(Lx) / Lz (Eq. 32 solved for f_s; the paper's f_s = 2 H1* as
 * Lz -> infinity).  EINVAL when the tilt does not cross tol inside the scan
 * (or already at its first point). */
int ising_critical_field(int n, const double *H1, const double *theta, double tol, double T, double Lx, double Lz,
                         double *h1_star, double *f_s);

/* Eqs. 28-32, the single-step model: phi = <pi/2 - theta> =
 * (W+1 - W-1) / (Lx Z) with W0 = 1, W+-1 = Lx exp(-f_s Lz / T)
 * exp(+-2 H1 Lz / T), evaluated relative to the largest weight (no
 * overflow); h1_star = f_s / 2 - T ln(Lx) / (2 Lz).  T, Lx, Lz > 0. */
int ising_step_model(double H1, double f_s, double T, double Lx, double Lz, double *phi, double *h1_star);

/* ------------------------------------------------- the procedures
 * Secs. II B - IV as whole calls over the record series of a film set
 * (each series as ising_read_series / ising_batch_read_series writes it).
 * Records first..n-1 of every series are averaged (exact integer sums, one
 * division).  Host memory, owned by the caller; EINVAL for null pointers,
 * films without records past `first`, or films of one group that differ in
 * size. */
typedef struct {
    const int64_t *records; /* n x (5 + Lx) int64 */
    size_t n;
    int Lx, Ly, Lz;
    double J, H, H1;        /* the film's Eq. 1 couplings (for its energy) */
} ising_series;

/* Contact angle and gamma(theta) (Secs. II B, III A), for k fields H1[j]:
 *   inter[j]  the film with the Eq. 11 boundary at H1[j];
 *   plus[j]   a periodic-y film started all up (the (+) plateaus);
 *   node[j * n_gl + i]  periodic-y films at the n_gl Gauss-Legendre nodes
 *             of [0, H1[j]] (ising_gauss_legendre).
 * inter and plus share one size.  Per field: the Eq. 17 profiles, the (-)
 * plateaus by Eq. 12 and the dividing plane of Eq. 18 over all layers give
 * theta[j] (and y_plus[j * Lx ...], may be NULL); the walls of the node films
 * (per-site layer-1 and layer-Lx means) give the Young difference
 * delta_f1[j] (Eq. 9) and Young's angle theta_young[j] (Eq. 8; NaN where
 * |delta_f1| > gamma_pi2).  gamma[j]: Eq. 16 integrated from theta = pi/2,
 * gamma = gamma_pi2 at H1 = 0 through the measured angles in order, with
 * |delta_f1| (the acute angle). */
int ising_procedure_contact_angle(int k, const double *H1, int n_gl, const ising_series *inter,
                                  const ising_series *plus, const ising_series *node, size_t first, double gamma_pi2,
                                  double *theta, double *theta_young, double *delta_f1, double *gamma,
                                  double *y_plus);

/* gamma(pi/2) and tau(0, pi/2) by integration over beta (Sec. II C): for
 * n_sizes sizes Lx = Lz = L[s] and n_beta inverse temperatures beta[b]
 * (from beta[0] < beta_c), the antiperiodic film apbc[s * n_beta + b] and
 * the periodic film pbc[s * n_beta + b].  dF[s] = F_APBC - F_PBC at the last
 * beta by Eq. 19 over U = <E_APBC> - <E_PBC> (Eq. 1 means), from 0 at
 * beta[0]; then the Eq. 20 fit. */
int ising_procedure_interface_tension(int n_sizes, const double *L, int n_beta, const double *beta,
                                      const ising_series *apbc, const ising_series *pbc, size_t first, double *dF,
                                      double *gamma_pi2, double *tau0);

/* The line tension (Sec. IV, Eqs. 21-22) over a constant-area set of
 * n_sizes sizes: inter[s * n_gl + i] the film with the Eq. 11 boundary and
 * plus[s * n_gl + i] the periodic-y film at node i of [0, H1].  Per size:
 * dF_film = the interface film's own integral over H1 (wall totals),
 * s_wall = the (+) film's per-site integral, delta_f1 = its Young difference,
 * and R[s] = ising_line_tension_residual with the given theta, gamma_theta
 * and gamma_pi2; then dtau and the intercept from the scan in Lz.
 * dF_film, s_wall, delta_f1 may be NULL. */
int ising_procedure_line_tension(int n_sizes, int n_gl, double H1, const ising_series *inter,
                                 const ising_series *plus, size_t first, double theta, double gamma_theta,
                                 double gamma_pi2, double *R, double *dF_film, double *s_wall, double *delta_f1,
                                 double *dtau, double *intercept);

/* Stiffness and steps (Secs. III B, III C) from k measured angles and
 * tensions: c and kappa (Eqs. 23-24), f_s and gamma_flat from Eq. 26 over
 * the flat point (pi/2, gamma_pi2) and the k points, then the single-step
 * model at that f_s for each of n_h fields H1[i]: phi[i], and h1_star
 * (Eqs. 28-32). */
int ising_procedure_stiffness_steps(int k, const double *theta, const double *gamma, double gamma_pi2, double T,
                                    double Lx, double Lz, int n_h, const double *H1, double *c, double *kappa,
                                    double *f_s, double *gamma_flat, double *phi, double *h1_star);

/* ------------------------------------- measurement without allocation */

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: a framework or serving runtime whose own
 * pool allocator already owns the device, or a loop that cannot take the
 * implicit device synchronisation of cudaMalloc.  It computes the record
 * {sweep, B, M, M1, Mn, m(1..Lx)} of a packed film exactly as
 * ising_measure does, but allocates nothing.
 *   spins   device, caller-owned: the film in the library's packed layout
 *           (ising_packed_words() words, as written by
 *           ising_get_packed_device).
 *   Lx, Ly, Lz, y_mode, x_mode   the film's geometry (as for ising_create
 *           and ising_set_options).
 *   sweep   copied into record[0].
 *   record  device, caller-owned: 5 + Lx int64, written asynchronously.
 *   stream  cudaStream_t as void* (NULL = the default stream).
 * The per-block partial sums go to one fixed 128 KiB device array inside the
 * library (16384 int64), so the film may use at most 8192 measurement blocks,
 * Lx * ceil(Ly * ceil(Lz / 64) / 1024) <= 8192; larger films get EINVAL.
 * Each call looks up that array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing); the first call on a device
 * may load the library's device code there, so make it before any stream
 * capture.  All calls on a device share the array: each call overwrites
 * every partial it reads, so nothing needs clearing, but calls whose kernels
 * overlap on the GPU race on it -- serialise them on one stream or order
 * them with events. */
int ising_measure_packed_noalloc(const uint32_t *spins, int Lx, int Ly, int Lz, int y_mode, int x_mode,
                                 uint64_t sweep, int64_t *record, void *stream);

/* ------------------------------------------------------------- misc */

/* Bounds checking.  A library built with ISING_CHECKED tests every lattice
 * word index of the update, resident and record kernels (and of
 * ising_measure_packed_noalloc) against its plane:
 * an out-of-range index is counted and the first one kept (site id << 48 |
 * index), and the access is redirected (a load reads word 0, a store is
 * dropped) -- nothing traps.  *checked = 1 for such a build, with the totals
 * of the process so far; other builds give *checked = 0 and zeros.
 * ECUDA if the counters cannot be read. */
int ising_check_counters(int *checked, uint64_t *count, uint64_t *first);

const char *ising_strerror(int status);
const char *ising_last_error(void);
/* Library version and the compute capability it was built for (e.g. 103). */
int ising_version(int *major, int *minor, int *sm);

#ifdef __cplusplus
}
#endif
#endif /* ISING_GB300_H */
