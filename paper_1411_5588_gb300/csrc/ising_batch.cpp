// Static batches: many independent films (different T, H1, shape, key) that
// share every launch -- the integration points of Eqs. 9, 19 and 22 run as one
// job.  A chunk of sweeps can be captured once in a CUDA graph and replayed;
// the films' sweep and record counters live on the device, so the same graph
// serves every chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>

#include "ising_host.h"

using namespace isg;

struct ising_batch {
  FilmSet fs;
  std::vector<ising_job> jobs;
  std::vector<uint64_t> rec_written, rec_read;
  uint64_t sweeps = 0;
  int8_t* d_stage = nullptr;
  size_t stage_bytes = 0;
  bool dirty = true;
  int shape = ISING_SHAPE_AUTO;  // pinned launch shape, or AUTO
  int tuned_shape = 0;           // ising_batch_autotune's choice (0: none yet)
  std::map<uint32_t, cudaGraphExec_t> graphs;  // chunk length -> executable graph

  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    graphs.clear();
  }
};

namespace {

int batch_sync_desc(ising_batch* b) {
  if (!b->dirty) return ISING_OK;
  int rc = b->fs.upload();
  if (rc) return rc;
  b->dirty = false;
  return ISING_OK;
}

// Make room for `extra[f]` more records of every film (rebuilds the ring area).
int batch_ensure_rings(ising_batch* b, const std::vector<uint64_t>& extra) {
  FilmSet& fs = b->fs;
  const size_t nf = fs.h.size();
  bool grow = false;
  for (size_t f = 0; f < nf; f++)
    if (b->rec_written[f] - b->rec_read[f] + extra[f] > fs.h[f].rec_cap) grow = true;
  if (!grow && fs.rec) return ISING_OK;
  std::vector<uint64_t> cap(nf);
  size_t total = 0;
  for (size_t f = 0; f < nf; f++) {
    const uint64_t pending = b->rec_written[f] - b->rec_read[f];
    uint64_t c = fs.h[f].rec_cap;
    if (pending + extra[f] > c) c = std::max<uint64_t>({16, 2 * c, pending + extra[f]});
    if (c > 0xFFFFFFF0ull) return fail(ISING_ENOMEM, "record series of film %zu too long", f);
    cap[f] = c;
    total += c * record_len(fs.h[f]);
  }
  int64_t* nr = nullptr;
  if (cudaMalloc(&nr, std::max<size_t>(total, 1) * sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ISING_ENOMEM, "cannot allocate %zu record words", total);
  }
  ISG_CK(cudaStreamSynchronize(fs.stream));
  size_t off = 0;
  for (size_t f = 0; f < nf; f++) {
    FilmDesc& d = fs.h[f];
    const size_t rl = record_len(d);
    const uint64_t pending = b->rec_written[f] - b->rec_read[f];
    for (uint64_t i = 0; i < pending; i++) {
      const uint64_t slot = (b->rec_read[f] + i) % d.rec_cap;
      ISG_CK(cudaMemcpyAsync(nr + off + i * rl, fs.rec + d.rec_off + slot * rl, rl * sizeof(int64_t),
                             cudaMemcpyDeviceToDevice, fs.stream));
    }
    d.rec_off = off;
    d.rec_cap = (uint32_t)cap[f];
    d.rec_next = (uint32_t)pending;
    b->rec_read[f] = 0;
    b->rec_written[f] = pending;
    off += cap[f] * rl;
  }
  ISG_CK(cudaStreamSynchronize(fs.stream));
  if (fs.rec) cudaFree(fs.rec);
  fs.rec = nr;
  fs.rec_words = total;
  b->dirty = true;
  b->drop_graphs();
  return ISING_OK;
}

uint64_t lcm_u64(uint64_t a, uint64_t b) { return a / std::gcd(a, b) * b; }

// Switch the grid kernels' words per thread: new block ranges and owner
// tables, and the captured graphs (which bake in the old ones) are dropped.
int apply_items(ising_batch* b, uint32_t items) {
  if (b->fs.items == items) return ISING_OK;
  ISG_CK(cudaStreamSynchronize(b->fs.stream));
  b->fs.items = items;
  b->fs.layout();
  b->dirty = true;
  b->drop_graphs();
  return ISING_OK;
}

int direct_sweeps(ising_batch* b, uint32_t n) {
  if (n == 0) return ISING_OK;
  FilmSet& fs = b->fs;
  int rc = fs.enqueue_sweeps(0, n, false, false);
  if (rc) return rc;
  ISG_CK(launch_advance(fs.L, (fs.hh.n_films + 127) / 128, n, fs.stream));
  for (auto& d : fs.h) d.sweep += n;
  b->sweeps += n;
  return ISING_OK;
}

}  // namespace

extern "C" {

int ising_batch_create(const ising_job* jobs, size_t n, ising_batch** out) {
  clear_error();
  if (!out || (!jobs && n)) return fail(ISING_EINVAL, "NULL argument");
  *out = nullptr;
  if (n == 0 || n > (1u << 24)) return fail(ISING_EINVAL, "batch needs 1..2^24 films");
  for (size_t i = 0; i < n; i++) {
    const ising_job& j = jobs[i];
    int rc = check_film(j.Lx, j.Ly, j.Lz, j.T, j.y_mode, j.x_mode);
    if (rc) return fail(rc, "job %zu: %s", i, ising_last_error());
    if (j.init_kind < ISING_INIT_RANDOM || j.init_kind > ISING_INIT_ALL_UP)
      return fail(ISING_EINVAL, "job %zu: bad init kind", i);
    if (j.init_kind == ISING_INIT_SLAB_Y && !(j.flip_p >= 0.0 && j.flip_p <= 1.0))
      return fail(ISING_EINVAL, "job %zu: flip_p must be in [0,1]", i);
  }
  ising_batch* b = new (std::nothrow) ising_batch();
  if (!b) return fail(ISING_ENOMEM, "host allocation failed");
  b->jobs.assign(jobs, jobs + n);
  b->rec_written.assign(n, 0);
  b->rec_read.assign(n, 0);
  FilmSet& fs = b->fs;
  fs.h.resize(n);
  size_t words = 0, stage = 0;
  for (size_t i = 0; i < n; i++) {
    const ising_job& j = jobs[i];
    FilmDesc& d = fs.h[i];
    std::memset(&d, 0, sizeof d);
    fill_geometry(d, j.Lx, j.Ly, j.Lz, j.y_mode, j.x_mode, j.seed, j.replica);
    build_tables(d, j.J, j.H, j.H1, j.T);
    d.measure_every = j.measure_every;
    d.spin_off = words;
    words += (film_words(d) + 63) / 64 * 64;
    stage = std::max(stage, (size_t)j.Lx * j.Ly * j.Lz);
  }
  int rc = fs.init_device();
  if (rc) { delete b; return rc; }
  fs.layout();
  size_t part = 0;
  for (auto& d : fs.h) part += part_len(d);
  if (cudaMalloc(&fs.pool, words * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&fs.part, part * sizeof(int64_t)) != cudaSuccess ||
      cudaMemset(fs.part, 0, part * sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    ising_batch_destroy(b);
    return fail(ISING_ENOMEM, "device allocation of %zu words failed", words);
  }
  fs.pool_words = words;
  fs.part_words = part;
  b->stage_bytes = stage;
  std::vector<uint64_t> extra(n, 0);
  for (size_t i = 0; i < n; i++) extra[i] = jobs[i].measure_every ? 64 : 0;
  rc = batch_ensure_rings(b, extra);
  for (size_t i = 0; !rc && i < n; i++) {
    const ising_job& j = jobs[i];
    uint32_t flip_lo = 0;
    int flip_all = 0;
    if (j.init_kind == ISING_INIT_SLAB_Y) {
      const double t = std::floor(std::ldexp(j.flip_p, 32));
      if (t >= 4294967296.0) flip_all = 1; else flip_lo = (uint32_t)t;
    }
    if (launch_init(fs.h[i], fs.pool, j.init_kind, flip_lo, flip_all, fs.stream) != cudaSuccess)
      rc = fail(ISING_ECUDA, "init launch failed");
  }
  if (!rc) rc = batch_sync_desc(b);
  if (rc) { ising_batch_destroy(b); return rc; }
  *out = b;
  return ISING_OK;
}

int ising_batch_set_stream(ising_batch* b, void* s) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  ISG_CK(cudaStreamSynchronize(b->fs.stream));
  if (b->fs.own_stream) ISG_CK(cudaStreamDestroy(b->fs.stream));
  b->fs.own_stream = false;
  b->fs.stream = nullptr;
  if (s) {
    b->fs.stream = (cudaStream_t)s;
  } else {
    ISG_CK(cudaStreamCreateWithFlags(&b->fs.stream, cudaStreamNonBlocking));
    b->fs.own_stream = true;
  }
  b->drop_graphs();
  return ISING_OK;
}

int ising_batch_sweep(ising_batch* b, uint64_t n, int use_graph) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  if (n == 0) return ISING_OK;
  if (b->sweeps + n >= 0xFFFFFFFFull) return fail(ISING_EINVAL, "sweep counter would reach 0xFFFFFFFF");
  FilmSet& fs = b->fs;
  const size_t nf = fs.h.size();
  std::vector<uint64_t> extra(nf);
  uint64_t G = 1;
  for (size_t f = 0; f < nf; f++) {
    const uint64_t m = fs.h[f].measure_every;
    extra[f] = m ? (b->sweeps + n) / m - b->sweeps / m : 0;
    if (m) G = lcm_u64(G, m);
  }
  int rc = batch_ensure_rings(b, extra);
  if (!rc) rc = batch_sync_desc(b);
  if (rc) return rc;
  if (G == 1) G = 64;
  while (G < 16) G *= 2;
  if (!use_graph || G > 4096 || n < 2 * G) {
    rc = direct_sweeps(b, (uint32_t)n);
  } else {
    const uint64_t prefix = (G - b->sweeps % G) % G;
    rc = direct_sweeps(b, (uint32_t)prefix);
    uint64_t left = n - prefix;
    const uint32_t g = (uint32_t)G;
    if (!rc && left >= G && !b->graphs.count(g)) {
      cudaGraph_t graph = nullptr;
      ISG_CK(cudaStreamBeginCapture(fs.stream, cudaStreamCaptureModeThreadLocal));
      int crc = fs.enqueue_sweeps(0, g, false, false);
      if (!crc && launch_advance(fs.L, (fs.hh.n_films + 127) / 128, g, fs.stream) != cudaSuccess)
        crc = fail(ISING_ECUDA, "advance launch failed");
      cudaError_t e = cudaStreamEndCapture(fs.stream, &graph);
      if (crc) { if (graph) cudaGraphDestroy(graph); return crc; }
      if (e != cudaSuccess) return fail(ISING_ECUDA, "graph capture: %s", cudaGetErrorString(e));
      cudaGraphExec_t exec = nullptr;
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(ISING_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
      b->graphs[g] = exec;
    }
    while (!rc && left >= G) {
      ISG_CK(cudaGraphLaunch(b->graphs[g], fs.stream));
      for (auto& d : fs.h) d.sweep += g;
      b->sweeps += g;
      left -= G;
    }
    if (!rc) rc = direct_sweeps(b, (uint32_t)left);
  }
  if (rc) return rc;
  for (size_t f = 0; f < nf; f++) {
    fs.h[f].rec_next += (uint32_t)extra[f];
    b->rec_written[f] += extra[f];
  }
  return ISING_OK;
}

int ising_batch_reserve_records(ising_batch* b, uint64_t n_records) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  std::vector<uint64_t> extra(b->fs.h.size());
  for (size_t f = 0; f < extra.size(); f++) extra[f] = b->fs.h[f].measure_every ? n_records : 0;
  return batch_ensure_rings(b, extra);
}

int ising_batch_set_shape(ising_batch* b, int shape) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  if (shape != ISING_SHAPE_AUTO && shape != ISING_SHAPE_GRID_1 && shape != ISING_SHAPE_GRID_2 &&
      shape != ISING_SHAPE_GRID_Q)
    return fail(ISING_EINVAL, "batches take AUTO, GRID_1, GRID_2 or GRID_Q");
  b->shape = shape;
  const uint32_t items = shape == ISING_SHAPE_AUTO ? (b->tuned_shape ? shape_items(b->tuned_shape) : 1u)
                                                   : shape_items(shape);
  return apply_items(b, items);
}

int ising_batch_get_shape(ising_batch* b, int* shape) {
  clear_error();
  if (!b || !shape) return fail(ISING_EINVAL, "NULL argument");
  *shape = items_shape(b->fs.items);
  return ISING_OK;
}

int ising_batch_autotune(ising_batch* b, int* shape) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  // a scratch batch of the same films from their initial states: the kernels
  // do the same work whatever the spins are, and this batch is not touched
  DeviceGuard dev(b->fs.device);
  ising_batch* s = nullptr;
  int rc = ising_batch_create(b->jobs.data(), b->jobs.size(), &s);
  if (rc) return rc;
  double sites = 0;
  for (const auto& d : b->fs.h) sites += (double)d.Lx * d.Ly * d.Lz;
  const uint64_t n = (uint64_t)std::min(1024.0, std::max(64.0, std::round(4e8 / sites)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = fail(ISING_ECUDA, "event creation failed");
  int best = ISING_SHAPE_GRID_1;
  float best_ms = 3.0e38f;
  for (int cand = ISING_SHAPE_GRID_1; !rc && cand <= ISING_SHAPE_GRID_Q; cand++) {
    rc = apply_items(s, shape_items(cand));
    float ms = 3.0e38f;
    for (int rep = 0; !rc && rep < 3; rep++) {  // the first run captures the graph
      if (cudaEventRecord(e0, s->fs.stream) != cudaSuccess) rc = fail(ISING_ECUDA, "event record failed");
      if (!rc) rc = ising_batch_sweep(s, n, 1);
      if (!rc && cudaEventRecord(e1, s->fs.stream) != cudaSuccess) rc = fail(ISING_ECUDA, "event record failed");
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(ISING_ECUDA, "event wait failed");
      float t = 0.f;
      if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = fail(ISING_ECUDA, "event time failed");
      if (!rc && rep > 0) ms = std::min(ms, t);
      for (size_t f = 0; f < s->fs.h.size(); f++) s->rec_read[f] = s->rec_written[f];  // drop the records
    }
    if (!rc && ms < kTuneMargin * best_ms) {  // a later shape must win clearly
      best_ms = ms;
      best = cand;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  ising_batch_destroy(s);
  if (rc) return rc;
  b->tuned_shape = best;
  if (b->shape == ISING_SHAPE_AUTO) rc = apply_items(b, shape_items(best));
  if (!rc && shape) *shape = best;
  return rc;
}

int ising_batch_get_spins(ising_batch* b, size_t i, int8_t* s) {
  clear_error();
  if (!b || !s) return fail(ISING_EINVAL, "NULL argument");
  if (i >= b->fs.h.size()) return fail(ISING_ENOTFOUND, "film %zu out of range", i);
  if (!b->d_stage) ISG_CK(cudaMalloc(&b->d_stage, b->stage_bytes));
  const FilmDesc& d = b->fs.h[i];
  ISG_CK(launch_unpack(d, b->fs.pool, b->d_stage, b->fs.stream));
  ISG_CK(cudaMemcpyAsync(s, b->d_stage, (size_t)d.Lx * d.Ly * d.Lz, cudaMemcpyDeviceToHost, b->fs.stream));
  ISG_CK(cudaStreamSynchronize(b->fs.stream));
  return ISING_OK;
}

int ising_batch_read_series(ising_batch* b, size_t i, int64_t* buf, size_t cap, size_t* n_records) {
  clear_error();
  if (!b || !n_records || (cap && !buf)) return fail(ISING_EINVAL, "NULL argument");
  if (i >= b->fs.h.size()) return fail(ISING_ENOTFOUND, "film %zu out of range", i);
  ISG_CK(cudaStreamSynchronize(b->fs.stream));
  const FilmDesc& d = b->fs.h[i];
  const size_t rl = record_len(d);
  const uint64_t pending = b->rec_written[i] - b->rec_read[i];
  const uint64_t k = std::min<uint64_t>(pending, cap);
  uint64_t t = 0;
  while (t < k) {
    const uint64_t slot = (b->rec_read[i] + t) % d.rec_cap;
    const uint64_t run = std::min<uint64_t>(k - t, d.rec_cap - slot);
    ISG_CK(cudaMemcpyAsync(buf + t * rl, b->fs.rec + d.rec_off + slot * rl, run * rl * sizeof(int64_t),
                           cudaMemcpyDeviceToHost, b->fs.stream));
    t += run;
  }
  ISG_CK(cudaStreamSynchronize(b->fs.stream));
  b->rec_read[i] += k;
  *n_records = (size_t)k;
  return ISING_OK;
}

int ising_batch_pending_records(const ising_batch* b, size_t i, size_t* n) {
  clear_error();
  if (!b || !n) return fail(ISING_EINVAL, "NULL argument");
  if (i >= b->fs.h.size()) return fail(ISING_ENOTFOUND, "film %zu out of range", i);
  *n = (size_t)(b->rec_written[i] - b->rec_read[i]);
  return ISING_OK;
}

int ising_batch_synchronize(ising_batch* b, double timeout_s) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  return wait_stream(b->fs.stream, timeout_s);
}

int ising_batch_destroy(ising_batch* b) {
  if (!b) return ISING_OK;
  if (b->fs.stream) cudaStreamSynchronize(b->fs.stream);
  b->drop_graphs();
  if (b->d_stage) cudaFree(b->d_stage);
  b->fs.release();
  delete b;
  return ISING_OK;
}

}  // extern "C"
