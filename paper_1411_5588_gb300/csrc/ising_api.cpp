// C ABI of the Ising-film library: single films and static batches.
//
// Everything numerical runs in the CUDA kernels of ising_kernels.cu; this file
// validates arguments, owns device memory, builds the Metropolis threshold
// tables of Eq. 1 and enqueues launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "ising_host.h"

namespace isg {

namespace {
thread_local std::string g_err;
}

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  // a failed runtime call stays CUDA's last error; consume it here so that a
  // later launch check does not report it again (sticky errors persist)
  if (code == ISING_ECUDA || code == ISING_ENOMEM) cudaGetLastError();
  return code;
}

void clear_error() { g_err.clear(); }

const char* last_error() { return g_err.c_str(); }

int check_film(int Lx, int Ly, int Lz, double T, int y_mode, int x_mode) {
  if (Lx < 1) return fail(ISING_EINVAL, "Lx must be >= 1 (got %d)", Lx);
  if (Ly < 2) return fail(ISING_EINVAL, "Ly must be >= 2 (got %d)", Ly);
  if (Lz < 2 || (Lz & 1)) return fail(ISING_EINVAL, "Lz must be even and >= 2 (got %d)", Lz);
  if (!(T > 0.0)) return fail(ISING_EINVAL, "T must be > 0 (got %g)", T);
  if (y_mode < ISING_Y_GAPBC || y_mode > ISING_Y_APBC) return fail(ISING_EINVAL, "bad y_mode %d", y_mode);
  if (x_mode != ISING_X_FREE && x_mode != ISING_X_PBC) return fail(ISING_EINVAL, "bad x_mode %d", x_mode);
  if (x_mode == ISING_X_PBC && (Lx < 2 || (Lx & 1))) return fail(ISING_EINVAL, "periodic x needs even Lx >= 2");
  const double plane = (double)Lx * (double)Ly * ((Lz / 2 + 31) / 32);
  if (plane >= 2147483648.0) return fail(ISING_EINVAL, "film too large (2^31 words per parity plane at most)");
  return ISING_OK;
}

void fill_geometry(FilmDesc& d, int Lx, int Ly, int Lz, int y_mode, int x_mode, uint64_t seed, uint32_t replica) {
  d.Lx = (uint32_t)Lx;
  d.Ly = (uint32_t)Ly;
  d.Lz = (uint32_t)Lz;
  d.n = (uint32_t)Lz / 2;
  d.W = (d.n + 31) / 32;
  d.Wp = d.W;  // rows contiguous: no padding words
  d.nq = (d.Wp + 3) / 4;
  const uint32_t r = d.n - 32 * (d.W - 1);  // valid sites of the last word, 1..32
  uint32_t mask = 0;
  for (uint32_t l = 0; l < r; l++) mask |= 1u << bitpos(l);
  d.last_mask = mask;
  d.last_calls = (r + 3) / 4;
  d.y_mode = (uint32_t)y_mode;
  d.x_pbc = x_mode == ISING_X_PBC ? 1u : 0u;
  d.key0 = (uint32_t)seed ^ (uint32_t)(seed >> 32);
  d.key1 = replica;
  for (uint32_t k = 0; k < 10; k++) {  // round keys: key + k * Weyl constant
    d.rk0[k] = d.key0 + k * kWeyl0;
    d.rk1[k] = d.key1 + k * kWeyl1;
  }
  d.upd_items = d.Lx * (d.Ly - 1) * d.W;
  d.meas_bpl = std::max<uint32_t>(1, (d.Ly * d.W + kMeasureItemsPerBlock - 1) / kMeasureItemsPerBlock);
  d.meas_lpu = 1;
  if (2 * d.Ly * d.W <= kMeasureItemsPerBlock)
    d.meas_lpu = std::min<uint32_t>({kMeasureMaxLpu, d.Lx, kMeasureItemsPerBlock / (d.Ly * d.W)});
  d.active = 1;
  d.sweep_end = 0xFFFFFFFFu;
  fastdiv_magic(d.W, &d.divw_m, &d.divw_l);
  fastdiv_magic(d.Ly > 2 ? d.Ly - 2 : 1, &d.divy_m, &d.divy_l);  // rows ky = 2 .. Ly-1 of a layer
  // thin films: the one-word grid kernels update 4 (at most 8 sites per
  // array) or 2 (at most 16) rows per packed word; the first and the last
  // group of a layer must differ.  Two rows pay only on films of at least
  // kPack2Rows rows: packing halves a film's threads and doubles each one's
  // chain of Philox calls, which a small film's few waves cannot hide
  // (measured on GB300: the beta-integration set's films of 1200-3000 rows
  // lose 6%, the line-tension set's of 13824 rows gain)
  d.pack = 1;
  if (d.W == 1 && d.n <= 8 && d.Ly % 4 == 0 && d.Ly >= 8) d.pack = 4;
  else if (d.W == 1 && d.n <= 16 && d.Ly % 2 == 0 && d.Ly >= 4 && d.Lx * d.Ly >= kPack2Rows) d.pack = 2;
  const uint32_t groups = d.Ly / d.pack;
  d.pk_items = d.Lx * (groups - 1);
  fastdiv_magic(groups > 2 ? groups - 2 : 1, &d.pk_divm, &d.pk_divl);
}

void build_tables(FilmDesc& d, double J, double H, double H1, double T) {
  const int Lx = (int)d.Lx;
  d.has_never = 0;
  for (int cls = 0; cls < 4; cls++) {
    bool present = false;  // does some layer kx have this class?
    for (int kx = 1; kx <= Lx && !present; kx = (kx == 1 && Lx > 2) ? Lx - 1 : kx + 1)
      present = row_class((uint32_t)kx, (uint32_t)Lx) == (uint32_t)cls;
    const bool first = cls & 1, lastl = (cls & 2) != 0;
    uint32_t always = 0;
    // classes that cannot occur for this Lx keep a harmless table
    const int n_nb = 6 - (d.x_pbc ? 0 : ((first ? 1 : 0) + (lastl ? 1 : 0)));
    double h = H;
    if (first) h += H1;
    if (lastl) h += -H1;
    for (int idx = 0; idx < 16; idx++) {
      const int sbit = idx & 1, nal = idx >> 1;
      d.thr[cls][idx] = 0;
      if (nal > n_nb) continue;
      const int s = sbit ? 1 : -1;
      const int sigma = s * (2 * nal - n_nb);  // sum of the neighbour spins
      const double dE = 2.0 * (double)s * (J * (double)sigma + h);
      if (dE <= 0.0) {
        always |= 1u << idx;
        continue;
      }
      const double t = std::floor(std::ldexp(std::exp(-dE / T), 32));
      if (t >= 4294967296.0) {
        always |= 1u << idx;
        continue;
      }
      d.thr[cls][idx] = (uint32_t)t;
      if (t == 0.0 && present) d.has_never = 1;
    }
    d.always[cls] = always;
    (void)Lx;
  }
}

// ------------------------------------------------------------ FilmSet

int FilmSet::init_device() {
  ISG_CK(cudaGetDevice(&device));
  ISG_CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device));
  upd_per_sm = update_blocks_per_sm();
  meas_per_sm = measure_blocks_per_sm();
  if (upd_per_sm <= 0 || meas_per_sm <= 0) return fail(ISING_ECUDA, "occupancy query failed (no sm_103a device?)");
  if (!stream) {
    ISG_CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    own_stream = true;
  }
  return ISING_OK;
}

void FilmSet::layout(bool assign_part) {
  uint32_t ub = 0, mb = 0;
  size_t po = 0;
  for (auto& d : h) {
    d.upd_block_begin = ub;
    d.meas_block_begin = mb;
    if (assign_part) d.part_off = po;
    ub += (grid_items(d, items) + words_per_block(items) - 1) / words_per_block(items);
    mb += meas_units(d);
    po += part_len(d);
  }
  hh.n_films = (uint32_t)h.size();
  hh.upd_blocks = ub;
  hh.meas_blocks = mb;
}

int FilmSet::upload() {
  const size_t nf = h.size();
  const size_t bytes = sizeof(LaunchHdr) + nf * sizeof(FilmDesc) + (hh.upd_blocks + hh.meas_blocks) * sizeof(uint32_t);
  if (bytes > meta_bytes) {
    const size_t cap = std::max(bytes, meta_bytes * 2);
    if (d_meta) {
      ISG_CK(cudaStreamSynchronize(stream));
      const cudaError_t e = cudaFree(d_meta);
      d_meta = nullptr;
      meta_bytes = 0;  // nothing held until the new area is allocated
      if (e != cudaSuccess) return fail(ISING_ECUDA, "cudaFree: %s", cudaGetErrorString(e));
    }
    if (dev_alloc(&d_meta, cap) != cudaSuccess)
      return fail(ISING_ENOMEM, "cannot allocate %zu bytes of launch descriptors", cap);
    meta_bytes = cap;
  }
  staging.resize(bytes);
  char* p = staging.data();
  std::memcpy(p, &hh, sizeof hh);
  std::memcpy(p + sizeof hh, h.data(), nf * sizeof(FilmDesc));
  uint32_t* ou = reinterpret_cast<uint32_t*>(p + sizeof hh + nf * sizeof(FilmDesc));
  uint32_t* om = ou + hh.upd_blocks;
  for (size_t f = 0; f < nf; f++) {
    const FilmDesc& d = h[f];
    const uint32_t nb = (grid_items(d, items) + words_per_block(items) - 1) / words_per_block(items);
    for (uint32_t b = 0; b < nb; b++) ou[d.upd_block_begin + b] = (uint32_t)f;
    for (uint32_t b = 0; b < meas_units(d); b++) om[d.meas_block_begin + b] = (uint32_t)f;
  }
  L.hdr = reinterpret_cast<LaunchHdr*>(d_meta);
  L.films = reinterpret_cast<FilmDesc*>(d_meta + sizeof hh);
  L.owner_upd = reinterpret_cast<uint32_t*>(d_meta + sizeof hh + nf * sizeof(FilmDesc));
  L.owner_meas = L.owner_upd + hh.upd_blocks;
  ISG_CK(cudaMemcpyAsync(d_meta, p, bytes, cudaMemcpyHostToDevice, stream));
  ISG_CK(cudaStreamSynchronize(stream));
  return ISING_OK;
}

uint32_t FilmSet::upd_grid() const { return hh.upd_blocks; }
uint32_t FilmSet::meas_grid() const { return std::min<uint32_t>(hh.meas_blocks, meas_grid_max()); }
uint32_t FilmSet::fin_grid() const { return std::min<uint32_t>(hh.n_films, (uint32_t)(2 * n_sm)); }

int FilmSet::enqueue_sweeps(uint32_t k0, uint32_t n, bool all_meas, bool fixed_grid) {
  const uint32_t ug = fixed_grid ? upd_grid_max() : upd_grid();
  const uint32_t fg = fixed_grid ? (uint32_t)(2 * n_sm) : fin_grid();
  bool exact = false, pack = false;
  for (const auto& d : h) {
    exact = exact || (d.active && d.has_never);
    pack = pack || d.pack > 1;
  }
  bool prev_meas = false;
  for (uint32_t k = k0; k < k0 + n; k++) {
    bool meas = all_meas;
    if (!meas)
      for (const auto& d : h)
        if (d.active && d.measure_every && (uint64_t)(d.sweep + k + 1) % d.measure_every == 0 &&
            (uint64_t)d.sweep + k + 1 <= d.sweep_end) {
          meas = true;
          break;
        }
    // records: half-sweep 1 accumulates the sums; the next half-sweep 0
    // writes them, or, after the last sweep of the call, a small kernel
    ISG_CK(launch_update(L, ug, pool, 0, k, exact, items, pack, part, rec, false, prev_meas ? k : 0, stream));
    ISG_CK(launch_update(L, ug, pool, 1, k, exact, items, pack, part, rec, meas, 0, stream));
    if (meas && k + 1 == k0 + n) ISG_CK(launch_record(L, fg, part, rec, k + 1, stream));
    prev_meas = meas;
  }
  return ISING_OK;
}

int FilmSet::release() {
  if (stream) cudaStreamSynchronize(stream);
  if (d_meta) cudaFree(d_meta);
  if (pool) cudaFree(pool);
  if (part) cudaFree(part);
  if (rec) cudaFree(rec);
  d_meta = nullptr;
  pool = nullptr;
  part = nullptr;
  rec = nullptr;
  if (own_stream && stream) cudaStreamDestroy(stream);
  stream = nullptr;
  own_stream = false;
  return ISING_OK;
}

int wait_stream(cudaStream_t st, double timeout_s) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return ISING_OK;
    if (e != cudaErrorNotReady) return fail(ISING_ECUDA, "stream: %s", cudaGetErrorString(e));
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (dt > timeout_s) return fail(ISING_ETIMEOUT, "wait timed out after %.3f s", dt);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace isg

using namespace isg;

// ---------------------------------------------------------------- one film

struct ising {
  FilmSet fs;
  double J = 1.0, H = 0.0, H1 = 0.0, T = 1.0;
  uint64_t seed = 0;
  int y_mode = ISING_Y_GAPBC, x_mode = ISING_X_FREE;
  uint32_t replica = 0;
  uint64_t rec_written = 0, rec_read = 0;  // ring counters (mirror of the device's rec_next)
  int64_t* d_direct = nullptr;
  int8_t* d_stage = nullptr;
  bool dirty = true;
  int shape = ISING_SHAPE_AUTO;
  uint32_t* d_cl_list = nullptr;  // the cluster path's film list: one cluster, this film
  // cluster size of this film (film_cluster_size), cached for the table
  // variant it was found for (cl_exact: 0 fast, 1 exact, -1 none yet)
  uint32_t cl_size = 0;
  int cl_exact = -1;
  // asynchronous record copies (ising_read_series_async): records
  // [inflight_lo, inflight_hi) of the ring counters are still being copied
  // on copy_stream until ev_copied
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_copied = nullptr;
  bool inflight = false;
  uint64_t inflight_lo = 0, inflight_hi = 0;
  FilmDesc& d() { return fs.h[0]; }
};

namespace {

int ensure_stage(ising* h) {
  if (!h->d_stage && dev_alloc(&h->d_stage, (size_t)h->d().Lx * h->d().Ly * h->d().Lz) != cudaSuccess)
    return fail(ISING_ENOMEM, "cannot allocate the spin staging buffer");
  return ISING_OK;
}

// CTAs per cluster of a single film on the cluster path: the most (up to
// kClusterMaxSize) its layers and shared memory allow and the GPU can hold
// as one cluster, 0 if none.
uint32_t film_cluster_size(const FilmDesc& d) {
  const bool exact = d.has_never != 0;
  for (uint32_t C = kClusterMaxSize; C >= 1; C--) {
    const uint32_t m = cluster_smem_bytes(d, C);
    if (m && cluster_capacity(C, 1, m, cluster_threads(d, C, exact, 1), exact) > 0) return C;
  }
  return 0;
}

// film_cluster_size of the handle's film, looked up once per table variant
// (the geometry of a handle never changes; its table variant can).
uint32_t handle_cluster_size(ising* h) {
  const int exact = h->d().has_never != 0 ? 1 : 0;
  if (h->cl_exact != exact) {
    h->cl_size = film_cluster_size(h->d());
    h->cl_exact = exact;
  }
  return h->cl_size;
}

// The launch shape of an ising_sweep call: the pinned one, else the
// autotuner's choice for this film shape and record interval, else the
// resident kernel up to kResidentAutoSites spins and one word per thread above.
int resolve_shape(ising* h, uint32_t measure_every) {
  const FilmDesc& d = h->d();
  if (h->shape != ISING_SHAPE_AUTO) return h->shape;
  int s = 0;
  if (tune_lookup(tune_key(d, measure_every), &s) && (s != ISING_SHAPE_RESIDENT || resident_smem_bytes(d)) &&
      (s != ISING_SHAPE_CLUSTER || handle_cluster_size(h)))
    return s;
  const uint64_t sites = (uint64_t)d.Lx * d.Ly * d.Lz;
  return (sites <= kResidentAutoSites && resident_smem_bytes(d)) ? ISING_SHAPE_RESIDENT : ISING_SHAPE_GRID_1;
}

int sync_desc(ising* h) {
  if (!h->dirty) return ISING_OK;
  int rc = h->fs.upload();
  if (rc) return rc;
  h->dirty = false;
  return ISING_OK;
}

// Grow the record ring so that `extra` more records fit beside the pending ones.
int ensure_ring(ising* h, uint64_t extra) {
  FilmDesc& d = h->d();
  const uint64_t pending = h->rec_written - h->rec_read;
  if (pending + extra <= d.rec_cap) return ISING_OK;
  if (h->inflight) {  // the old ring is about to be freed
    ISG_CK(cudaEventSynchronize(h->ev_copied));
    h->inflight = false;
  }
  uint64_t cap = std::max<uint64_t>({64, 2 * (uint64_t)d.rec_cap, pending + extra});
  if (cap > 0xFFFFFFF0ull) return fail(ISING_ENOMEM, "record series too long; read it out first");
  const size_t rl = record_len(d);
  int64_t* nr = nullptr;
  if (dev_alloc(&nr, cap * rl * sizeof(int64_t)) != cudaSuccess)
    return fail(ISING_ENOMEM, "cannot allocate %llu records", (unsigned long long)cap);
  cudaError_t e = cudaStreamSynchronize(h->fs.stream);
  for (uint64_t i = 0; e == cudaSuccess && i < pending; i++) {
    const uint64_t slot = (h->rec_read + i) % d.rec_cap;
    e = cudaMemcpyAsync(nr + i * rl, h->fs.rec + slot * rl, rl * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                        h->fs.stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->fs.stream);
  if (e != cudaSuccess) {  // the old ring stays in place
    cudaStreamSynchronize(h->fs.stream);
    cudaFree(nr);
    return fail(ISING_ECUDA, "record ring copy: %s", cudaGetErrorString(e));
  }
  if (h->fs.rec) cudaFree(h->fs.rec);
  h->fs.rec = nr;
  h->fs.rec_words = cap * rl;
  d.rec_off = 0;
  d.rec_cap = (uint32_t)cap;
  d.rec_next = (uint32_t)pending;
  h->rec_read = 0;
  h->rec_written = pending;
  h->dirty = true;
  return ISING_OK;
}

}  // namespace

extern "C" {

int ising_create(int Lx, int Ly, int Lz, double J, double H1, double T, uint64_t seed, ising** out) {
  clear_error();
  if (!out) return fail(ISING_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_film(Lx, Ly, Lz, T, ISING_Y_GAPBC, ISING_X_FREE);
  if (rc) return rc;
  ising* h = new (std::nothrow) ising();
  if (!h) return fail(ISING_ENOMEM, "host allocation failed");
  h->J = J;
  h->H1 = H1;
  h->T = T;
  h->seed = seed;
  h->fs.h.resize(1);
  FilmDesc& d = h->fs.h[0];
  std::memset(&d, 0, sizeof d);
  fill_geometry(d, Lx, Ly, Lz, ISING_Y_GAPBC, ISING_X_FREE, seed, 0);
  build_tables(d, J, 0.0, H1, T);
  rc = h->fs.init_device();
  if (rc) { delete h; return rc; }
  h->fs.layout();
  const size_t words = film_words(d);
  if (dev_alloc(&h->fs.pool, words * sizeof(uint32_t)) != cudaSuccess ||
      dev_alloc(&h->fs.part, part_len(d) * sizeof(int64_t)) != cudaSuccess ||
      cudaMemset(h->fs.part, 0, part_len(d) * sizeof(int64_t)) != cudaSuccess ||
      dev_alloc(&h->d_direct, record_len(d) * sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h->d_direct);
    delete h;
    return fail(ISING_ENOMEM, "device allocation failed");
  }
  h->fs.pool_words = words;
  rc = ensure_ring(h, 64);
  if (!rc) rc = launch_init(d, h->fs.pool, ISING_INIT_ALL_UP, 0, 0, h->fs.stream) == cudaSuccess ? ISING_OK
                                                                                           : fail(ISING_ECUDA, "init launch failed");
  if (!rc) rc = sync_desc(h);
  if (rc) { ising_destroy(h); return rc; }
  *out = h;
  return ISING_OK;
}

int ising_set_options(ising* h, int y_mode, int x_mode, double H, uint32_t replica) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  FilmDesc& d = h->d();
  int rc = check_film((int)d.Lx, (int)d.Ly, (int)d.Lz, h->T, y_mode, x_mode);
  if (rc) return rc;
  h->y_mode = y_mode;
  h->x_mode = x_mode;
  h->H = H;
  h->replica = replica;
  d.y_mode = (uint32_t)y_mode;
  d.x_pbc = x_mode == ISING_X_PBC;
  d.key1 = replica;
  for (int r = 0; r < 10; r++) d.rk1[r] = replica + (uint32_t)r * kWeyl1;
  build_tables(d, h->J, H, h->H1, h->T);
  h->dirty = true;
  return ISING_OK;
}

int ising_set_params(ising* h, double J, double H1, double T) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  if (!(T > 0.0)) return fail(ISING_EINVAL, "T must be > 0");
  h->J = J;
  h->H1 = H1;
  h->T = T;
  build_tables(h->d(), J, h->H, H1, T);
  h->dirty = true;
  return ISING_OK;
}

int ising_set_stream(ising* h, void* s) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  ISG_CK(cudaStreamSynchronize(h->fs.stream));
  if (h->fs.own_stream) ISG_CK(cudaStreamDestroy(h->fs.stream));
  h->fs.own_stream = false;
  h->fs.stream = nullptr;
  if (s) {
    h->fs.stream = (cudaStream_t)s;
  } else {
    ISG_CK(cudaStreamCreateWithFlags(&h->fs.stream, cudaStreamNonBlocking));
    h->fs.own_stream = true;
  }
  return ISING_OK;
}

int ising_init(ising* h, int kind, double flip_p) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  if (kind < ISING_INIT_RANDOM || kind > ISING_INIT_ALL_UP) return fail(ISING_EINVAL, "bad init kind %d", kind);
  uint32_t flip_lo = 0;
  int flip_all = 0;
  if (kind == ISING_INIT_SLAB_Y) {
    if (!(flip_p >= 0.0 && flip_p <= 1.0)) return fail(ISING_EINVAL, "flip_p must be in [0,1]");
    const double t = std::floor(std::ldexp(flip_p, 32));
    if (t >= 4294967296.0) flip_all = 1; else flip_lo = (uint32_t)t;
  }
  FilmDesc& d = h->d();
  ISG_CK(launch_init(d, h->fs.pool, kind, flip_lo, flip_all, h->fs.stream));
  d.sweep = 0;
  d.rec_next = 0;
  h->rec_written = h->rec_read = 0;
  h->dirty = true;
  return sync_desc(h);
}

int ising_set_spins(ising* h, const int8_t* s) {
  clear_error();
  if (!h || !s) return fail(ISING_EINVAL, "NULL argument");
  int rc = ensure_stage(h);
  if (rc) return rc;
  const FilmDesc& d = h->d();
  ISG_CK(cudaMemcpyAsync(h->d_stage, s, (size_t)d.Lx * d.Ly * d.Lz, cudaMemcpyHostToDevice, h->fs.stream));
  ISG_CK(launch_pack(d, h->fs.pool, h->d_stage, h->fs.stream));
  ISG_CK(cudaStreamSynchronize(h->fs.stream));
  return ISING_OK;
}

int ising_get_spins(ising* h, int8_t* s) {
  clear_error();
  if (!h || !s) return fail(ISING_EINVAL, "NULL argument");
  int rc = ensure_stage(h);
  if (rc) return rc;
  const FilmDesc& d = h->d();
  ISG_CK(launch_unpack(d, h->fs.pool, h->d_stage, h->fs.stream));
  ISG_CK(cudaMemcpyAsync(s, h->d_stage, (size_t)d.Lx * d.Ly * d.Lz, cudaMemcpyDeviceToHost, h->fs.stream));
  ISG_CK(cudaStreamSynchronize(h->fs.stream));
  return ISING_OK;
}

int ising_set_spins_device(ising* h, const int8_t* s) {
  clear_error();
  if (!h || !s) return fail(ISING_EINVAL, "NULL argument");
  ISG_CK(launch_pack(h->d(), h->fs.pool, s, h->fs.stream));
  return ISING_OK;
}

int ising_get_spins_device(ising* h, int8_t* s) {
  clear_error();
  if (!h || !s) return fail(ISING_EINVAL, "NULL argument");
  ISG_CK(launch_unpack(h->d(), h->fs.pool, s, h->fs.stream));
  return ISING_OK;
}

size_t ising_packed_words(const ising* h) { return h ? film_words(const_cast<ising*>(h)->d()) : 0; }

int ising_get_packed_device(ising* h, uint32_t* dst) {
  clear_error();
  if (!h || !dst) return fail(ISING_EINVAL, "NULL argument");
  ISG_CK(cudaMemcpyAsync(dst, h->fs.pool, film_words(h->d()) * 4, cudaMemcpyDeviceToDevice, h->fs.stream));
  return ISING_OK;
}

int ising_set_packed_device(ising* h, const uint32_t* src) {
  clear_error();
  if (!h || !src) return fail(ISING_EINVAL, "NULL argument");
  ISG_CK(cudaMemcpyAsync(h->fs.pool, src, film_words(h->d()) * 4, cudaMemcpyDeviceToDevice, h->fs.stream));
  return ISING_OK;
}

int ising_get_sweep(const ising* h, uint64_t* sweep) {
  clear_error();
  if (!h || !sweep) return fail(ISING_EINVAL, "NULL argument");
  *sweep = const_cast<ising*>(h)->d().sweep;
  return ISING_OK;
}

int ising_set_sweep(ising* h, uint64_t sweep) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  if (sweep >= 0xFFFFFFFFull) return fail(ISING_EINVAL, "sweep index must stay below 0xFFFFFFFF");
  h->d().sweep = (uint32_t)sweep;
  h->dirty = true;
  return sync_desc(h);
}

int ising_check_counters(int* checked, uint64_t* count, uint64_t* first) {
  clear_error();
  if (!checked || !count || !first) return fail(ISING_EINVAL, "NULL argument");
  unsigned long long c = 0, f = 0, c2 = 0, f2 = 0;
  const int r = read_oob_counters(&c, &f);
  const int r2 = read_noalloc_oob_counters(&c2, &f2);
  if (r < 0 || r2 < 0) return fail(ISING_ECUDA, "cannot read the check counters");
  *checked = r;
  *count = c + c2;
  *first = f ? f : f2;
  return ISING_OK;
}

int ising_reserve_records(ising* h, uint64_t n_records) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  return ensure_ring(h, n_records);
}

int ising_set_shape(ising* h, int shape) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  if (shape < ISING_SHAPE_AUTO || shape > ISING_SHAPE_CLUSTER) return fail(ISING_EINVAL, "unknown shape %d", shape);
  if (shape == ISING_SHAPE_RESIDENT && !resident_smem_bytes(h->d()))
    return fail(ISING_EINVAL, "film too large for the resident kernel");
  if (shape == ISING_SHAPE_CLUSTER && !handle_cluster_size(h))
    return fail(ISING_EINVAL, "film too large for the cluster kernel");
  h->shape = shape;
  return ISING_OK;
}

int ising_get_shape(ising* h, uint32_t measure_every, int* shape) {
  clear_error();
  if (!h || !shape) return fail(ISING_EINVAL, "NULL argument");
  *shape = resolve_shape(h, measure_every);
  return ISING_OK;
}

int ising_autotune(ising* h, uint32_t measure_every, int* shape) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  const FilmDesc& d = h->d();
  // a scratch film of the same shape and parameters: the kernels do the same
  // work whatever the spins are, and the handle's own chain is not touched
  DeviceGuard dev(h->fs.device);
  ising* s = nullptr;
  int rc = ising_create(d.Lx, d.Ly, d.Lz, h->J, h->H1, h->T, h->seed, &s);
  if (rc) return rc;
  rc = ising_set_options(s, h->y_mode, h->x_mode, h->H, h->replica);
  if (!rc) rc = ising_init(s, ISING_INIT_RANDOM, 0.0);
  const double sites = (double)d.Lx * d.Ly * d.Lz;
  const uint64_t n = (uint64_t)std::min(400.0, std::max(4.0, std::round(4e8 / sites)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = fail(ISING_ECUDA, "event creation failed");
  int best = ISING_SHAPE_GRID_1;
  float best_ms = 3.0e38f;
  std::vector<int64_t> drain;
  for (int cand = ISING_SHAPE_RESIDENT; !rc && cand <= ISING_SHAPE_CLUSTER; cand++) {
    if (cand == ISING_SHAPE_RESIDENT && !resident_smem_bytes(d)) continue;
    if (cand == ISING_SHAPE_CLUSTER && !film_cluster_size(d)) continue;
    s->shape = cand;
    float ms = 3.0e38f;
    for (int rep = 0; !rc && rep < 3; rep++) {  // the first run warms up
      if (cudaEventRecord(e0, s->fs.stream) != cudaSuccess) rc = fail(ISING_ECUDA, "event record failed");
      if (!rc) rc = ising_sweep(s, n, measure_every);
      if (!rc && cudaEventRecord(e1, s->fs.stream) != cudaSuccess) rc = fail(ISING_ECUDA, "event record failed");
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(ISING_ECUDA, "event wait failed");
      float t = 0.f;
      if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = fail(ISING_ECUDA, "event time failed");
      if (!rc && rep > 0) ms = std::min(ms, t);
      drain.resize((size_t)(s->rec_written - s->rec_read) * record_len(s->d()) + 1);
      size_t got = 0;
      if (!rc) rc = ising_read_series(s, drain.data(), (size_t)(s->rec_written - s->rec_read), &got);
    }
    if (!rc && ms < kTuneMargin * best_ms) {  // a later shape must win clearly
      best_ms = ms;
      best = cand;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  ising_destroy(s);
  if (rc) return rc;
  tune_store(tune_key(d, measure_every), best);
  if (shape) *shape = best;
  return ISING_OK;
}

int ising_sweep(ising* h, uint64_t n, uint32_t measure_every) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  FilmDesc& d = h->d();
  if (n == 0) return ISING_OK;
  if ((uint64_t)d.sweep + n >= 0xFFFFFFFFull) return fail(ISING_EINVAL, "sweep counter would reach 0xFFFFFFFF");
  if (d.measure_every != measure_every) {
    d.measure_every = measure_every;
    h->dirty = true;
  }
  const uint64_t s0 = d.sweep;
  const uint64_t nrec = measure_every ? (s0 + n) / measure_every - s0 / measure_every : 0;
  int rc = ensure_ring(h, nrec);
  if (rc) return rc;
  // records of this call land on ring slots of records rec_written + nrec -
  // rec_cap and later: if any of those are still being copied out, wait
  if (h->inflight && cudaEventQuery(h->ev_copied) == cudaSuccess) h->inflight = false;
  if (h->inflight && nrec && h->rec_written + nrec > h->inflight_lo + d.rec_cap)
    ISG_CK(cudaStreamWaitEvent(h->fs.stream, h->ev_copied, 0));
  rc = sync_desc(h);
  if (rc) return rc;
  const int shape = resolve_shape(h, measure_every);
  if (shape == ISING_SHAPE_CLUSTER) {
    // every sweep of the call in one launch: one cluster holds the film in
    // distributed shared memory
    if (!h->d_cl_list) {
      const uint32_t list[3] = {0u, 1u, 0u};  // cluster 0 sweeps film 0
      if (dev_alloc(&h->d_cl_list, sizeof list) != cudaSuccess)
        return fail(ISING_ENOMEM, "cannot allocate the cluster film list");
      ISG_CK(cudaMemcpy(h->d_cl_list, list, sizeof list, cudaMemcpyHostToDevice));
    }
    const uint32_t C = handle_cluster_size(h);
    const bool exact = d.has_never != 0;
    if (C == 0) return fail(ISING_EINVAL, "film too large for the cluster kernel");
    for (uint64_t done = 0; done < n;) {
      const uint32_t k = (uint32_t)std::min<uint64_t>(n - done, 4096);
      ISG_CK(launch_cluster(h->fs.L.films, h->d_cl_list, 1, C, 1, cluster_smem_bytes(d, C),
                            cluster_threads(d, C, exact, 1), exact, h->fs.pool, h->fs.rec, k, h->fs.stream));
      done += k;
    }
    d.sweep = (uint32_t)(s0 + n);
    d.rec_next += (uint32_t)nrec;
    h->rec_written += nrec;
    return ISING_OK;
  }
  if (shape == ISING_SHAPE_RESIDENT) {
    const uint32_t smem = resident_smem_bytes(d);
    // small film: every sweep of the call in one launch, planes in shared memory
    ISG_CK(launch_resident(h->fs.L.films, 1, smem, resident_threads(d), d.has_never != 0, h->fs.pool, h->fs.rec,
                           (uint32_t)n, h->fs.stream));
    d.sweep = (uint32_t)(s0 + n);
    d.rec_next += (uint32_t)nrec;
    h->rec_written += nrec;
    return ISING_OK;
  }
  // single film: the descriptor travels as a kernel parameter
  const uint32_t items = shape_items(shape);
  for (uint64_t k = 0; k < n; k++) {
    const uint32_t t = (uint32_t)(s0 + k);
    const bool rec_now = measure_every && (s0 + k + 1) % measure_every == 0;
    ISG_CK(launch_update_film(d, h->fs.pool, 0, t, items, nullptr, h->fs.stream));
    ISG_CK(launch_update_film(d, h->fs.pool, 1, t, items, rec_now ? h->fs.part + acc_offset(d) : nullptr,
                              h->fs.stream));
    if (rec_now) ISG_CK(launch_record(h->fs.L, 1, h->fs.part, h->fs.rec, (uint32_t)(k + 1), h->fs.stream));
  }
  ISG_CK(launch_advance(h->fs.L, 1, (uint32_t)n, h->fs.stream));
  d.sweep = (uint32_t)(s0 + n);
  d.rec_next += (uint32_t)nrec;
  h->rec_written += nrec;
  return ISING_OK;
}

int ising_measure(ising* h, ising_obs* out) {
  clear_error();
  if (!h || !out) return fail(ISING_EINVAL, "NULL argument");
  int rc = sync_desc(h);
  if (rc) return rc;
  FilmDesc& d = h->d();
  ISG_CK(launch_measure(h->fs.L, h->fs.meas_grid(), 1, h->fs.pool, h->fs.part, h->fs.rec, 0, 1, h->d_direct,
                        h->fs.stream));
  std::vector<int64_t> r(record_len(d));
  ISG_CK(cudaMemcpyAsync(r.data(), h->d_direct, r.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, h->fs.stream));
  ISG_CK(cudaStreamSynchronize(h->fs.stream));
  out->sweep = (uint64_t)r[0];
  out->bond_sum = r[1];
  out->M = r[2];
  out->M1 = r[3];
  out->Mn = r[4];
  if (out->m_x) std::memcpy(out->m_x, r.data() + 5, d.Lx * sizeof(int64_t));
  return ISING_OK;
}

int ising_read_series(ising* h, int64_t* buf, size_t cap, size_t* n_records) {
  clear_error();
  if (!h || !n_records || (cap && !buf)) return fail(ISING_EINVAL, "NULL argument");
  ISG_CK(cudaStreamSynchronize(h->fs.stream));
  const FilmDesc& d = h->d();
  const size_t rl = record_len(d);
  const uint64_t pending = h->rec_written - h->rec_read;
  const uint64_t k = std::min<uint64_t>(pending, cap);
  uint64_t i = 0;
  while (i < k) {
    const uint64_t slot = (h->rec_read + i) % d.rec_cap;
    const uint64_t run = std::min<uint64_t>(k - i, d.rec_cap - slot);
    ISG_CK(cudaMemcpyAsync(buf + i * rl, h->fs.rec + d.rec_off + slot * rl, run * rl * sizeof(int64_t),
                           cudaMemcpyDeviceToHost, h->fs.stream));
    i += run;
  }
  ISG_CK(cudaStreamSynchronize(h->fs.stream));
  h->rec_read += k;
  *n_records = (size_t)k;
  return ISING_OK;
}

int ising_read_series_async(ising* h, int64_t* buf, size_t cap, size_t* n_records, void* cuda_stream) {
  clear_error();
  if (!h || !n_records || (cap && !buf)) return fail(ISING_EINVAL, "NULL argument");
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  if (!cs) {
    if (!h->copy_stream) ISG_CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    cs = h->copy_stream;
  }
  if (!h->ev_ready) ISG_CK(cudaEventCreateWithFlags(&h->ev_ready, cudaEventDisableTiming));
  if (!h->ev_copied) ISG_CK(cudaEventCreateWithFlags(&h->ev_copied, cudaEventDisableTiming));
  const FilmDesc& d = h->d();
  const size_t rl = record_len(d);
  const uint64_t k = std::min<uint64_t>(h->rec_written - h->rec_read, cap);
  *n_records = (size_t)k;
  if (k == 0) return ISING_OK;
  if (h->inflight && cudaEventQuery(h->ev_copied) == cudaSuccess) h->inflight = false;
  // the copy starts once everything enqueued on the handle so far is done
  ISG_CK(cudaEventRecord(h->ev_ready, h->fs.stream));
  ISG_CK(cudaStreamWaitEvent(cs, h->ev_ready, 0));
  if (h->inflight) ISG_CK(cudaStreamWaitEvent(cs, h->ev_copied, 0));  // one in-flight range at a time
  uint64_t i = 0;
  while (i < k) {
    const uint64_t slot = (h->rec_read + i) % d.rec_cap;
    const uint64_t run = std::min<uint64_t>(k - i, d.rec_cap - slot);
    ISG_CK(cudaMemcpyAsync(buf + i * rl, h->fs.rec + d.rec_off + slot * rl, run * rl * sizeof(int64_t),
                           cudaMemcpyDeviceToHost, cs));
    i += run;
  }
  ISG_CK(cudaEventRecord(h->ev_copied, cs));
  h->inflight_lo = h->inflight ? h->inflight_lo : h->rec_read;
  h->inflight_hi = h->rec_read + k;
  h->inflight = true;
  h->rec_read += k;
  return ISING_OK;
}

int ising_pending_records(const ising* h, size_t* n) {
  clear_error();
  if (!h || !n) return fail(ISING_EINVAL, "NULL argument");
  *n = (size_t)(h->rec_written - h->rec_read);
  return ISING_OK;
}

int ising_synchronize(ising* h, double timeout_s) {
  clear_error();
  if (!h) return fail(ISING_EINVAL, "NULL handle");
  return wait_stream(h->fs.stream, timeout_s);
}

int ising_destroy(ising* h) {
  if (!h) return ISING_OK;
  if (h->ev_copied) cudaEventSynchronize(h->ev_copied);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->ev_ready) cudaEventDestroy(h->ev_ready);
  if (h->ev_copied) cudaEventDestroy(h->ev_copied);
  h->fs.release();
  if (h->d_direct) cudaFree(h->d_direct);
  if (h->d_stage) cudaFree(h->d_stage);
  if (h->d_cl_list) cudaFree(h->d_cl_list);
  delete h;
  return ISING_OK;
}

const char* ising_strerror(int status) {
  switch (status) {
    case ISING_OK: return "ok";
    case ISING_EINVAL: return "invalid argument";
    case ISING_ENOMEM: return "out of memory";
    case ISING_ECUDA: return "CUDA error";
    case ISING_ETIMEOUT: return "timed out";
    case ISING_EBUSY: return "busy";
    case ISING_ENOTFOUND: return "not found";
    default: return "unknown status";
  }
}

const char* ising_last_error(void) { return last_error(); }

int ising_version(int* major, int* minor, int* sm) {
  if (major) *major = 0;
  if (minor) *minor = 1;
  if (sm) *sm = 103;
  return ISING_OK;
}

}  // extern "C"
