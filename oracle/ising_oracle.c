/*
 * Ising-film oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU simulator of the checkerboard
 * single-spin-flip Metropolis sweep of the nearest-neighbour Ising film of
 * Block, Kim, Virnau & Binder (arXiv:1411.5588), used to check the CUDA path
 * bit for bit.  Only tests/, __graft_entry__.smoke() and the cpu_baseline leg
 * of bench.py may load it; the product library never does.  It shares no code
 * with the CUDA path: its own Philox4x32-10, its own acceptance thresholds,
 * its own int8 lattice in canonical order.
 *
 * What it follows:
 *   - Hamiltonian, Eq. 1 (Sec. II A): H = -J sum_<ij> S_i S_j - H sum S_i
 *     - H1 sum_{kx=1} S_i - Hn sum_{kx=Lx} S_i, with Hn = -H1.
 *   - Free surfaces at kx=1 and kx=Lx, periodic z (Sec. II A).
 *   - y boundary: the generalized antiperiodic rule of Eq. 11,
 *     S(kx, ky +- Ly, kz) = -S(Lx+1-kx, ky, kz); plain periodic and plain
 *     antiperiodic y are the other two modes used in Sec. II C (Eq. 20).
 *   - Checkerboard update (Appendix).  Reading: colour c = (kx+ky+kz) mod 2
 *     and four phases per sweep, P0 = {c=0, ky<Ly}, P1 = {c=0, ky=Ly},
 *     P2 = {c=1, ky<Ly}, P3 = {c=1, ky=Ly}; each phase is an independent set
 *     for every y mode (the Eq. 11 wrap bond joins equal colours when Lx+Ly is
 *     even, so two phases would not be).
 *   - Metropolis acceptance (the paper names no rule): accept iff dE <= 0 or
 *     u < floor(exp(-dE/T) * 2^32), u a 32-bit Philox word, with
 *     dE = 2*s*(J*sigma + h) evaluated in that order in binary64 and
 *     h = H, then += H1 on kx=1, then += Hn on kx=Lx.
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *     key = (lo32(seed) ^ hi32(seed), replica); site z0 = kz-1 of row
 *     (kx-1)*Ly + (ky-1) in sweep t uses counter (row, z0>>3, t, z0&1) and
 *     output word (z0>>1)&3.  Initialisation uses counter
 *     (row, z0>>3, 0xFFFFFFFF, 2 | (z0&1)).
 *   - Bond sum B = 1/2 sum_i sum_slots sigma S_i S_nb over the six neighbour
 *     slots of every site (a slot that wraps onto the same neighbour twice,
 *     e.g. Lz = 2, counts twice); M, M1 = sum over kx=1, Mn = sum over kx=Lx,
 *     and the layer sums m(kx) of Eq. 17.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_Y_GAPBC 0
#define ORC_Y_PBC 1
#define ORC_Y_APBC 2
#define ORC_X_FREE 0
#define ORC_X_PBC 1

#define ORC_INIT_RANDOM 0
#define ORC_INIT_SLAB_Y 1
#define ORC_INIT_ALL_UP 2

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds, from the published definition: each round
 * multiplies counter words 0 and 2 by fixed constants, swaps the halves and
 * mixes in the key; the key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Batch helper for tests: n counters (4 words each) under one key. */
void orc_philox4x32_10_n(const uint32_t *ctrs, const uint32_t key[2], uint32_t *outs, int64_t n)
{
    for (int64_t i = 0; i < n; i++) orc_philox4x32_10(ctrs + 4 * i, key, outs + 4 * i);
}

/* ------------------------------------------------------------------ film */

typedef struct {
    int Lx, Ly, Lz;
    double J, H, H1, T;
    int y_mode, x_mode;
    uint64_t seed;
    uint32_t replica;
    uint64_t sweep;   /* sweeps completed so far = index of the next sweep */
    int8_t *S;        /* ((kx-1)*Ly + (ky-1))*Lz + (kz-1) */
} orc_film;

static inline int8_t spin(const orc_film *f, int kx, int ky, int kz)
{
    return f->S[((int64_t)(kx - 1) * f->Ly + (ky - 1)) * f->Lz + (kz - 1)];
}

static inline void key_of(const orc_film *f, uint32_t key[2])
{
    key[0] = (uint32_t)f->seed ^ (uint32_t)(f->seed >> 32);
    key[1] = f->replica;
}

orc_film *orc_create(int Lx, int Ly, int Lz, double J, double H1, double T, uint64_t seed)
{
    if (Lx < 1 || Ly < 2 || Lz < 2 || (Lz & 1)) return NULL;
    if (!(T > 0.0)) return NULL;
    orc_film *f = (orc_film *)calloc(1, sizeof(orc_film));
    if (!f) return NULL;
    f->Lx = Lx; f->Ly = Ly; f->Lz = Lz;
    f->J = J; f->H = 0.0; f->H1 = H1; f->T = T;
    f->y_mode = ORC_Y_GAPBC; f->x_mode = ORC_X_FREE;
    f->seed = seed; f->replica = 0; f->sweep = 0;
    f->S = (int8_t *)malloc((size_t)Lx * Ly * Lz);
    if (!f->S) { free(f); return NULL; }
    for (int64_t i = 0; i < (int64_t)Lx * Ly * Lz; i++) f->S[i] = 1;
    return f;
}

int orc_set_options(orc_film *f, int y_mode, int x_mode, double H, uint32_t replica)
{
    if (y_mode < 0 || y_mode > 2 || x_mode < 0 || x_mode > 1) return 1;
    if (x_mode == ORC_X_PBC && (f->Lx < 2 || (f->Lx & 1))) return 1;
    f->y_mode = y_mode; f->x_mode = x_mode; f->H = H; f->replica = replica;
    return 0;
}

void orc_destroy(orc_film *f)
{
    if (f) { free(f->S); free(f); }
}

void orc_set_spins(orc_film *f, const int8_t *s)
{
    memcpy(f->S, s, (size_t)f->Lx * f->Ly * f->Lz);
}

void orc_get_spins(const orc_film *f, int8_t *s)
{
    memcpy(s, f->S, (size_t)f->Lx * f->Ly * f->Lz);
}

void orc_set_sweep(orc_film *f, uint64_t sweep) { f->sweep = sweep; }
uint64_t orc_get_sweep(const orc_film *f) { return f->sweep; }

/* Spin seen through neighbour slot `slot` of site (kx,ky,kz), sign of the
 * boundary rule included; 0 where a free x surface leaves the slot empty.
 * Slots: 0 x-1, 1 x+1, 2 y-1, 3 y+1, 4 z-1, 5 z+1. */
static int across_y(const orc_film *f, int kx, int ky_target, int kz)
{
    /* Eq. 11: S(kx, ky +- Ly, kz) = -S(Lx+1-kx, ky, kz) */
    if (f->y_mode == ORC_Y_GAPBC) return -spin(f, f->Lx + 1 - kx, ky_target, kz);
    if (f->y_mode == ORC_Y_APBC) return -spin(f, kx, ky_target, kz);
    return spin(f, kx, ky_target, kz);
}

static int neighbour(const orc_film *f, int kx, int ky, int kz, int slot)
{
    const int Lx = f->Lx, Ly = f->Ly, Lz = f->Lz;
    switch (slot) {
    case 0:
        if (kx > 1) return spin(f, kx - 1, ky, kz);
        return f->x_mode == ORC_X_PBC ? spin(f, Lx, ky, kz) : 0;
    case 1:
        if (kx < Lx) return spin(f, kx + 1, ky, kz);
        return f->x_mode == ORC_X_PBC ? spin(f, 1, ky, kz) : 0;
    case 2:
        if (ky > 1) return spin(f, kx, ky - 1, kz);
        return across_y(f, kx, Ly, kz);
    case 3:
        if (ky < Ly) return spin(f, kx, ky + 1, kz);
        return across_y(f, kx, 1, kz);
    case 4:
        return spin(f, kx, ky, kz == 1 ? Lz : kz - 1);
    default:
        return spin(f, kx, ky, kz == Lz ? 1 : kz + 1);
    }
}

/* Field acting on layer kx: bulk H plus the surface fields of Eq. 1. */
static double layer_field(const orc_film *f, int kx)
{
    double h = f->H;
    if (kx == 1) h += f->H1;
    if (kx == f->Lx) h += -f->H1;
    return h;
}

/* Energy change of flipping site (kx,ky,kz), from Eq. 1. */
double orc_delta_e(const orc_film *f, int kx, int ky, int kz)
{
    int sigma = 0;
    for (int slot = 0; slot < 6; slot++) sigma += neighbour(f, kx, ky, kz, slot);
    int s = spin(f, kx, ky, kz);
    return 2.0 * (double)s * (f->J * (double)sigma + layer_field(f, kx));
}

/* Metropolis rule with a 32-bit uniform word: accept iff dE <= 0 or
 * u < floor(exp(-dE/T) * 2^32). */
int orc_accept(double dE, double T, uint32_t u)
{
    if (dE <= 0.0) return 1;
    double p = exp(-dE / T);
    uint64_t thr = (uint64_t)floor(ldexp(p, 32));
    return (uint64_t)u < thr;
}

static uint32_t site_uniform(const orc_film *f, int kx, int ky, int kz, uint32_t c2, uint32_t c3_base)
{
    uint32_t key[2], ctr[4], out[4];
    key_of(f, key);
    uint32_t z0 = (uint32_t)(kz - 1);
    ctr[0] = (uint32_t)((kx - 1) * f->Ly + (ky - 1));
    ctr[1] = z0 >> 3;
    ctr[2] = c2;
    ctr[3] = c3_base | (z0 & 1u);
    orc_philox4x32_10(ctr, key, out);
    return out[(z0 >> 1) & 3u];
}

int orc_init(orc_film *f, int kind, double flip_p)
{
    if (kind < 0 || kind > 2) return 1;
    uint64_t flip_thr = 0;
    if (kind == ORC_INIT_SLAB_Y) {
        if (!(flip_p >= 0.0 && flip_p <= 1.0)) return 1;
        flip_thr = (uint64_t)floor(ldexp(flip_p, 32));
    }
    for (int kx = 1; kx <= f->Lx; kx++)
        for (int ky = 1; ky <= f->Ly; ky++)
            for (int kz = 1; kz <= f->Lz; kz++) {
                int8_t s;
                if (kind == ORC_INIT_ALL_UP) {
                    s = 1;
                } else {
                    uint32_t u = site_uniform(f, kx, ky, kz, 0xFFFFFFFFu, 2u);
                    if (kind == ORC_INIT_RANDOM) {
                        s = (u < 0x80000000u) ? 1 : -1;
                    } else {
                        s = (ky <= f->Ly / 2) ? 1 : -1;
                        if ((uint64_t)u < flip_thr) s = (int8_t)-s;
                    }
                }
                f->S[((int64_t)(kx - 1) * f->Ly + (ky - 1)) * f->Lz + (kz - 1)] = s;
            }
    f->sweep = 0;
    return 0;
}

/* One phase: every site of colour `colour` whose row is (ky == Ly) == last. */
static void run_phase(orc_film *f, int colour, int last, uint32_t t)
{
    const int Lx = f->Lx, Ly = f->Ly, Lz = f->Lz;
    const int64_t nrows = (int64_t)Lx * Ly;
#pragma omp parallel for schedule(static) if (nrows * (int64_t)Lz >= 65536)
    for (int64_t row = 0; row < nrows; row++) {
        int kx = (int)(row / Ly) + 1, ky = (int)(row % Ly) + 1;
        if ((ky == Ly) != (last != 0)) continue;
        for (int kz = 1; kz <= Lz; kz++) {
            if (((kx + ky + kz) & 1) != colour) continue;
            double dE = orc_delta_e(f, kx, ky, kz);
            uint32_t u = site_uniform(f, kx, ky, kz, t, 0u);
            if (orc_accept(dE, f->T, u)) {
                int8_t *p = &f->S[(row)*Lz + (kz - 1)];
                *p = (int8_t)-*p;
            }
        }
    }
}

void orc_measure(const orc_film *f, int64_t *rec);

/* n sweeps; after every completed sweep whose count is a multiple of
 * measure_every (> 0) one record is appended to recs (5 + Lx int64 each:
 * sweeps completed, B, M, M1, Mn, m(1..Lx)).  Returns records written, or -1
 * if the sweep counter would reach 0xFFFFFFFF (reserved for initialisation). */
int64_t orc_sweep(orc_film *f, uint64_t n, uint32_t measure_every, int64_t *recs, int64_t cap)
{
    int64_t nrec = 0;
    if (f->sweep + n >= 0xFFFFFFFFull) return -1;
    for (uint64_t i = 0; i < n; i++) {
        uint32_t t = (uint32_t)f->sweep;
        run_phase(f, 0, 0, t);
        run_phase(f, 0, 1, t);
        run_phase(f, 1, 0, t);
        run_phase(f, 1, 1, t);
        f->sweep++;
        if (measure_every && f->sweep % measure_every == 0 && recs && nrec < cap) {
            orc_measure(f, recs + nrec * (5 + f->Lx));
            nrec++;
        }
    }
    return nrec;
}

/* One record: {sweeps completed, B, M, M1, Mn, m(1), ..., m(Lx)}.  The
 * layers are summed in parallel; every sum is an exact int64, so the record
 * does not depend on the order or the thread count. */
void orc_measure(const orc_film *f, int64_t *rec)
{
    const int Lx = f->Lx, Ly = f->Ly, Lz = f->Lz;
    int64_t twice_b = 0, M = 0;
#pragma omp parallel for schedule(static) reduction(+ : twice_b) if ((int64_t)Lx * Ly * Lz >= 65536)
    for (int kx = 1; kx <= Lx; kx++) {
        int64_t mk = 0;
        for (int ky = 1; ky <= Ly; ky++)
            for (int kz = 1; kz <= Lz; kz++) {
                int s = spin(f, kx, ky, kz);
                for (int slot = 0; slot < 6; slot++) twice_b += s * neighbour(f, kx, ky, kz, slot);
                mk += s;
            }
        rec[5 + kx - 1] = mk;
    }
    for (int kx = 1; kx <= Lx; kx++) M += rec[5 + kx - 1];
    rec[0] = (int64_t)f->sweep;
    rec[1] = twice_b / 2;
    rec[2] = M;
    rec[3] = rec[5];
    rec[4] = rec[5 + Lx - 1];
}

/* Eq. 1 energy of the current configuration. */
double orc_energy(const orc_film *f)
{
    int64_t *rec = (int64_t *)malloc(sizeof(int64_t) * (5 + f->Lx));
    orc_measure(f, rec);
    double E = -f->J * (double)rec[1] - f->H * (double)rec[2] - f->H1 * (double)rec[3] - (-f->H1) * (double)rec[4];
    free(rec);
    return E;
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
