// Static batches: many independent films (different T, H1, shape, key) that
// share launches -- the integration points of Eqs. 9, 19 and 22 run as one
// job.  The films are spread over lanes, each a film set on its own stream;
// the lanes run concurrently, so one lane's launch boundaries overlap another
// lane's work.  A chunk of sweeps can be captured once in a CUDA graph per
// lane and replayed; the films' sweep and record counters live on the device,
// so the same graph serves every chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "ising_host.h"

using namespace isg;

namespace {

// One lane of a batch: a film set with its own stream, record rings and
// captured graphs.  The lanes of a batch run concurrently.
struct Lane {
  FilmSet fs;
  std::vector<ising_job> jobs;
  std::vector<uint64_t> rec_written, rec_read;
  uint64_t sweeps = 0;
  int8_t* d_stage = nullptr;
  size_t stage_bytes = 0;
  bool dirty = true;
  std::map<uint32_t, cudaGraphExec_t> graphs;  // chunk length -> executable graph
  cudaEvent_t ev_done = nullptr;               // the lane's last sweep call has finished
  // cluster-resident path (CTAs per film; 0: the grid kernels), with the
  // launch's shared memory and threads per CTA and its table variant
  uint32_t cl_size = 0, cl_per_sm = 1, cl_smem = 0, cl_threads = 0;
  bool cl_exact = false;
  uint32_t cl_clusters = 0;        // clusters of the lane's launch
  uint32_t* d_cl_list = nullptr;   // their film lists (launch_cluster's list)

  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    graphs.clear();
  }
};

int lane_sync_desc(Lane* b) {
  if (!b->dirty) return ISING_OK;
  int rc = b->fs.upload();
  if (rc) return rc;
  b->dirty = false;
  return ISING_OK;
}

// Make room for `extra[f]` more records of every film (rebuilds the ring area).
int lane_ensure_rings(Lane* b, const std::vector<uint64_t>& extra) {
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
  if (dev_alloc(&nr, std::max<size_t>(total, 1) * sizeof(int64_t)) != cudaSuccess)
    return fail(ISING_ENOMEM, "cannot allocate %zu record words", total);
  // copy the unread records first; the films move to the new rings only once
  // every copy has finished, so a failure leaves the old rings in place
  cudaError_t e = cudaStreamSynchronize(fs.stream);
  std::vector<size_t> off(nf);
  size_t o = 0;
  for (size_t f = 0; f < nf; f++) {
    const FilmDesc& d = fs.h[f];
    const size_t rl = record_len(d);
    const uint64_t pending = b->rec_written[f] - b->rec_read[f];
    for (uint64_t i = 0; e == cudaSuccess && i < pending; i++) {
      const uint64_t slot = (b->rec_read[f] + i) % d.rec_cap;
      e = cudaMemcpyAsync(nr + o + i * rl, fs.rec + d.rec_off + slot * rl, rl * sizeof(int64_t),
                          cudaMemcpyDeviceToDevice, fs.stream);
    }
    off[f] = o;
    o += cap[f] * rl;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(fs.stream);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(fs.stream);
    cudaFree(nr);
    return fail(ISING_ECUDA, "record ring copy: %s", cudaGetErrorString(e));
  }
  for (size_t f = 0; f < nf; f++) {
    FilmDesc& d = fs.h[f];
    const uint64_t pending = b->rec_written[f] - b->rec_read[f];
    d.rec_off = off[f];
    d.rec_cap = (uint32_t)cap[f];
    d.rec_next = (uint32_t)pending;
    b->rec_read[f] = 0;
    b->rec_written[f] = pending;
  }
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
int lane_apply_items(Lane* b, uint32_t items) {
  if (b->fs.items == items) return ISING_OK;
  ISG_CK(cudaStreamSynchronize(b->fs.stream));
  b->fs.items = items;
  b->fs.layout();
  b->dirty = true;
  b->drop_graphs();
  return ISING_OK;
}

// Launch parameters of the cluster path with C CTAs per film, per_sm CTAs per
// SM, for every film of the lane; EINVAL if some film does not qualify.
int lane_cluster_params(const Lane* b, uint32_t C, uint32_t per_sm, uint32_t* smem, uint32_t* threads, bool* exact) {
  *smem = 0;
  *threads = 0;
  *exact = false;
  for (const FilmDesc& d : b->fs.h) *exact = *exact || d.has_never != 0;
  for (const FilmDesc& d : b->fs.h) {
    const uint32_t m = cluster_smem_bytes(d, C);
    if (m == 0) return fail(ISING_EINVAL, "film %ux%ux%u does not fit clusters of %u CTAs", d.Lx, d.Ly, d.Lz, C);
    *smem = std::max(*smem, m);
    *threads = std::max(*threads, cluster_threads(d, C, *exact, per_sm));
  }
  const int cap = cluster_capacity(C, per_sm, *smem, *threads, *exact);
  if (cap < 0) return fail(ISING_ECUDA, "cluster occupancy query failed");
  if (cap == 0) return fail(ISING_EINVAL, "this GPU cannot hold a cluster of %u CTAs of this size", C);
  return ISING_OK;
}

// Work of one sweep of film d in units of about one Philox call: a row's
// words' calls plus a few per word for the fetch and the neighbour count.
double cluster_film_work(const FilmDesc& d) {
  return (double)d.Lx * d.Ly * (8.0 * (d.W - 1) + d.last_calls + 3.0 * d.W);
}

// Switch the lane to the cluster path with C CTAs per film (C = 0: back to
// the grid kernels), on n_clusters clusters of one CTA per SM: the films go
// to clusters largest first, each to the cluster with the least work so far.
int lane_apply_cluster(Lane* b, uint32_t C, uint32_t n_clusters) {
  const uint32_t per_sm = 1;
  uint32_t smem = 0, threads = 0;
  bool exact = false;
  const size_t nf = b->fs.h.size();
  if (C) {
    int rc = lane_cluster_params(b, C, per_sm, &smem, &threads, &exact);
    if (rc) return rc;
    n_clusters = (uint32_t)std::min<size_t>(std::max<uint32_t>(n_clusters, 1), nf);
  }
  if (b->cl_size == C && (C == 0 || b->cl_clusters == n_clusters)) return ISING_OK;
  std::vector<uint32_t> list;
  if (C) {
    std::vector<size_t> order(nf);
    std::iota(order.begin(), order.end(), (size_t)0);
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
      return cluster_film_work(b->fs.h[x]) > cluster_film_work(b->fs.h[y]);
    });
    std::vector<double> load(n_clusters, 0.0);
    std::vector<std::vector<uint32_t>> members(n_clusters);
    for (size_t f : order) {
      const size_t c = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
      members[c].push_back((uint32_t)f);
      load[c] += cluster_film_work(b->fs.h[f]);
    }
    list.resize(n_clusters + 1 + nf);
    uint32_t o = 0;
    for (uint32_t c = 0; c < n_clusters; c++) {
      list[c] = o;
      for (uint32_t f : members[c]) list[n_clusters + 1 + o++] = f;
    }
    list[n_clusters] = o;
  }
  ISG_CK(cudaStreamSynchronize(b->fs.stream));
  if (b->d_cl_list) {
    cudaFree(b->d_cl_list);
    b->d_cl_list = nullptr;
  }
  if (C) {
    if (dev_alloc(&b->d_cl_list, list.size() * sizeof(uint32_t)) != cudaSuccess) {
      b->cl_size = 0;
      return fail(ISING_ENOMEM, "cannot allocate the cluster film lists");
    }
    ISG_CK(cudaMemcpy(b->d_cl_list, list.data(), list.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  }
  b->cl_size = C;
  b->cl_clusters = C ? n_clusters : 0;
  b->cl_per_sm = per_sm;
  b->cl_smem = smem;
  b->cl_threads = threads;
  b->cl_exact = exact;
  b->drop_graphs();
  return ISING_OK;
}

// n sweeps of every film on the cluster path, in launches of at most 4096
// sweeps; each launch advances the films' counters on the device.
int lane_cluster_sweeps(Lane* b, uint64_t n) {
  FilmSet& fs = b->fs;
  while (n) {
    const uint32_t k = (uint32_t)std::min<uint64_t>(n, 4096);
    ISG_CK(launch_cluster(fs.L.films, b->d_cl_list, b->cl_clusters, b->cl_size, b->cl_per_sm, b->cl_smem,
                          b->cl_threads, b->cl_exact, fs.pool, fs.rec, k, fs.stream));
    for (auto& d : fs.h) d.sweep += k;
    b->sweeps += k;
    n -= k;
  }
  return ISING_OK;
}

int lane_direct_sweeps(Lane* b, uint32_t n) {
  if (n == 0) return ISING_OK;
  FilmSet& fs = b->fs;
  int rc = fs.enqueue_sweeps(0, n, false, false);
  if (rc) return rc;
  ISG_CK(launch_advance(fs.L, (fs.hh.n_films + 127) / 128, n, fs.stream));
  for (auto& d : fs.h) d.sweep += n;
  b->sweeps += n;
  return ISING_OK;
}

void lane_destroy(Lane* b);

// A lane of the given films (caller's order within the lane), initial
// states drawn, descriptors uploaded.
int lane_create(const std::vector<ising_job>& jobs, Lane** out) {
  *out = nullptr;
  const size_t n = jobs.size();
  Lane* b = new (std::nothrow) Lane();
  if (!b) return fail(ISING_ENOMEM, "host allocation failed");
  b->jobs = jobs;
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
  auto drop = [&](int rc) {
    lane_destroy(b);
    return rc;
  };
  int rc = fs.init_device();
  if (rc) return drop(rc);
  if (cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) != cudaSuccess) {
    b->ev_done = nullptr;
    return drop(fail(ISING_ECUDA, "event creation failed"));
  }
  fs.layout();
  size_t part = 0;
  for (auto& d : fs.h) part += part_len(d);
  if (dev_alloc(&fs.pool, words * sizeof(uint32_t)) != cudaSuccess ||
      dev_alloc(&fs.part, part * sizeof(int64_t)) != cudaSuccess ||
      cudaMemset(fs.part, 0, part * sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    return drop(fail(ISING_ENOMEM, "device allocation of %zu words failed", words));
  }
  fs.pool_words = words;
  fs.part_words = part;
  b->stage_bytes = stage;
  std::vector<uint64_t> extra(n, 0);
  for (size_t i = 0; i < n; i++) extra[i] = jobs[i].measure_every ? 64 : 0;
  rc = lane_ensure_rings(b, extra);
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
  if (!rc) rc = lane_sync_desc(b);
  if (rc) return drop(rc);
  *out = b;
  return ISING_OK;
}

void lane_destroy(Lane* b) {
  if (!b) return;
  if (b->fs.stream) cudaStreamSynchronize(b->fs.stream);
  b->drop_graphs();
  if (b->d_stage) cudaFree(b->d_stage);
  if (b->d_cl_list) cudaFree(b->d_cl_list);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  b->fs.release();
  delete b;
}

// n sweeps of every film of the lane, on its stream.
int lane_sweep(Lane* b, uint64_t n, int use_graph) {
  FilmSet& fs = b->fs;
  const size_t nf = fs.h.size();
  std::vector<uint64_t> extra(nf);
  uint64_t G = 1;
  for (size_t f = 0; f < nf; f++) {
    const uint64_t m = fs.h[f].measure_every;
    extra[f] = m ? (b->sweeps + n) / m - b->sweeps / m : 0;
    if (m) G = lcm_u64(G, m);
  }
  int rc = lane_ensure_rings(b, extra);
  if (!rc) rc = lane_sync_desc(b);
  if (rc) return rc;
  if (G == 1) G = 64;
  while (G < 16) G *= 2;
  if (b->cl_size) {
    rc = lane_cluster_sweeps(b, n);  // one launch holds every sweep: nothing to capture
  } else if (!use_graph || G > 4096 || n < 2 * G) {
    rc = lane_direct_sweeps(b, (uint32_t)n);
  } else {
    const uint64_t prefix = (G - b->sweeps % G) % G;
    rc = lane_direct_sweeps(b, (uint32_t)prefix);
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
    if (!rc) rc = lane_direct_sweeps(b, (uint32_t)left);
  }
  if (rc) return rc;
  for (size_t f = 0; f < nf; f++) {
    fs.h[f].rec_next += (uint32_t)extra[f];
    b->rec_written[f] += extra[f];
  }
  return ISING_OK;
}

// Films to lanes: the largest first, each to the lane with the fewest sites
// so far (the lanes' sweeps take about equally long).
std::vector<uint32_t> assign_lanes(const ising_job* jobs, size_t n, uint32_t lanes) {
  std::vector<size_t> order(n);
  std::iota(order.begin(), order.end(), (size_t)0);
  auto sites = [&](size_t i) { return (double)jobs[i].Lx * jobs[i].Ly * jobs[i].Lz; };
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return sites(a) > sites(b); });
  std::vector<double> load(lanes, 0.0);
  std::vector<uint32_t> lane_of(n);
  for (size_t i : order) {
    const uint32_t l = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
    lane_of[i] = l;
    load[l] += sites(i);
  }
  return lane_of;
}

}  // namespace

// A batch: its films spread over lanes that sweep concurrently, each on its
// own stream.  Lane 0's stream is the batch's stream; a sweep forks from it
// to the other lanes and joins back, so work queued on it afterwards sees
// every film swept.
struct ising_batch {
  std::vector<Lane*> lanes;
  std::vector<std::pair<uint32_t, uint32_t>> where;  // film -> (lane, index in the lane)
  std::vector<ising_job> jobs;                        // in the caller's order
  cudaEvent_t ev_fork = nullptr;
  int device = 0;
  int shape = ISING_SHAPE_AUTO;  // pinned launch shape, or AUTO
  int tuned_shape = 0;           // ising_batch_autotune's choice (0: none yet)
  uint32_t cl_pinned = 0;        // CTAs per film pinned for the CLUSTER shape (0: automatic)
  uint32_t tuned_cl = 0;         // the autotuner's CTAs per film when it chose CLUSTER

  cudaStream_t stream() const { return lanes[0]->fs.stream; }
  Lane* lane_of(size_t i) const { return lanes[where[i].first]; }
  size_t index_in_lane(size_t i) const { return where[i].second; }
};

namespace {

int batch_apply_items(ising_batch* b, uint32_t items) {
  for (Lane* l : b->lanes) {
    int rc = lane_apply_cluster(l, 0, 0);
    if (!rc) rc = lane_apply_items(l, items);
    if (rc) return rc;
  }
  return ISING_OK;
}

// Every lane on the cluster path with C CTAs per film, the GPU's SMs shared
// out among the lanes (one CTA each, so a lane has n_SM / (C lanes) clusters,
// at least one); on EINVAL (some film does not qualify) every lane is back on
// the grid kernels.
int batch_apply_cluster(ising_batch* b, uint32_t C) {
  const uint32_t n_sm = (uint32_t)std::max(1, b->lanes[0]->fs.n_sm);
  const uint32_t per_lane = std::max<uint32_t>(1, n_sm / (C * (uint32_t)b->lanes.size()));
  for (Lane* l : b->lanes) {
    int rc = lane_apply_cluster(l, C, per_lane);
    if (rc) {
      for (Lane* m : b->lanes) lane_apply_cluster(m, 0, 0);
      return rc;
    }
  }
  return ISING_OK;
}

// CTAs per film of the CLUSTER shape when none is pinned: the most (up to
// kClusterMaxSize) for which every film qualifies and all films' clusters fit
// on the GPU's SMs at once, one CTA each; 1 when the films outnumber the
// SMs; 0 when no size qualifies.
uint32_t batch_auto_cluster(const ising_batch* b) {
  const size_t nf = b->jobs.size();
  const size_t n_sm = (size_t)std::max(1, b->lanes[0]->fs.n_sm);
  for (uint32_t C = kClusterMaxSize; C >= 1; C--) {
    if (C > 1 && nf * C > n_sm) continue;
    bool ok = true;
    for (const Lane* l : b->lanes)
      for (const FilmDesc& d : l->fs.h) ok = ok && cluster_smem_bytes(d, C) != 0;
    if (ok) return C;
  }
  return 0;
}

int batch_sweep(ising_batch* b, uint64_t n, int use_graph) {
  const size_t nl = b->lanes.size();
  if (nl > 1) {
    ISG_CK(cudaEventRecord(b->ev_fork, b->stream()));
    for (size_t l = 1; l < nl; l++) ISG_CK(cudaStreamWaitEvent(b->lanes[l]->fs.stream, b->ev_fork, 0));
  }
  for (Lane* l : b->lanes) {
    int rc = lane_sweep(l, n, use_graph);
    if (rc) return rc;
  }
  for (size_t l = 1; l < nl; l++) {
    ISG_CK(cudaEventRecord(b->lanes[l]->ev_done, b->lanes[l]->fs.stream));
    ISG_CK(cudaStreamWaitEvent(b->stream(), b->lanes[l]->ev_done, 0));
  }
  return ISING_OK;
}

int batch_create(const ising_job* jobs, size_t n, uint32_t lanes, ising_batch** out) {
  ising_batch* b = new (std::nothrow) ising_batch();
  if (!b) return fail(ISING_ENOMEM, "host allocation failed");
  b->jobs.assign(jobs, jobs + n);
  const std::vector<uint32_t> lane_of = assign_lanes(jobs, n, lanes);
  std::vector<std::vector<ising_job>> per(lanes);
  b->where.resize(n);
  for (size_t i = 0; i < n; i++) {
    b->where[i] = {lane_of[i], (uint32_t)per[lane_of[i]].size()};
    per[lane_of[i]].push_back(jobs[i]);
  }
  int rc = ISING_OK;
  for (uint32_t l = 0; !rc && l < lanes; l++) {
    Lane* ln = nullptr;
    rc = lane_create(per[l], &ln);
    if (!rc) b->lanes.push_back(ln);
  }
  if (!rc && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    b->ev_fork = nullptr;
    rc = fail(ISING_ECUDA, "event creation failed");
  }
  if (!rc) b->device = b->lanes[0]->fs.device;
  if (rc) {
    ising_batch_destroy(b);
    return rc;
  }
  *out = b;
  return ISING_OK;
}

}  // namespace

extern "C" {

int ising_batch_create(const ising_job* jobs, size_t n, ising_batch** out) {
  return ising_batch_create_lanes(jobs, n, 0, out);
}

int ising_batch_create_lanes(const ising_job* jobs, size_t n, uint32_t lanes, ising_batch** out) {
  clear_error();
  if (!out || (!jobs && n)) return fail(ISING_EINVAL, "NULL argument");
  *out = nullptr;
  if (n == 0 || n > (1u << 24)) return fail(ISING_EINVAL, "batch needs 1..2^24 films");
  if (lanes > ISING_MAX_LANES) return fail(ISING_EINVAL, "at most %d lanes", ISING_MAX_LANES);
  for (size_t i = 0; i < n; i++) {
    const ising_job& j = jobs[i];
    int rc = check_film(j.Lx, j.Ly, j.Lz, j.T, j.y_mode, j.x_mode);
    if (rc) return fail(rc, "job %zu: %s", i, ising_last_error());
    if (j.init_kind < ISING_INIT_RANDOM || j.init_kind > ISING_INIT_ALL_UP)
      return fail(ISING_EINVAL, "job %zu: bad init kind", i);
    if (j.init_kind == ISING_INIT_SLAB_Y && !(j.flip_p >= 0.0 && j.flip_p <= 1.0))
      return fail(ISING_EINVAL, "job %zu: flip_p must be in [0,1]", i);
  }
  if (lanes == 0) lanes = n >= 2 ? 2u : 1u;
  if (lanes > n) lanes = (uint32_t)n;
  return batch_create(jobs, n, lanes, out);
}

int ising_batch_get_lanes(const ising_batch* b, uint32_t* lanes) {
  clear_error();
  if (!b || !lanes) return fail(ISING_EINVAL, "NULL argument");
  *lanes = (uint32_t)b->lanes.size();
  return ISING_OK;
}

int ising_batch_set_stream(ising_batch* b, void* s) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  FilmSet& fs = b->lanes[0]->fs;
  for (Lane* l : b->lanes) ISG_CK(cudaStreamSynchronize(l->fs.stream));
  if (fs.own_stream) ISG_CK(cudaStreamDestroy(fs.stream));
  fs.own_stream = false;
  fs.stream = nullptr;
  if (s) {
    fs.stream = (cudaStream_t)s;
  } else {
    ISG_CK(cudaStreamCreateWithFlags(&fs.stream, cudaStreamNonBlocking));
    fs.own_stream = true;
  }
  b->lanes[0]->drop_graphs();
  return ISING_OK;
}

int ising_batch_sweep(ising_batch* b, uint64_t n, int use_graph) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  if (n == 0) return ISING_OK;
  if (b->lanes[0]->sweeps + n >= 0xFFFFFFFFull) return fail(ISING_EINVAL, "sweep counter would reach 0xFFFFFFFF");
  return batch_sweep(b, n, use_graph);
}

int ising_batch_reserve_records(ising_batch* b, uint64_t n_records) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  for (Lane* l : b->lanes) {
    std::vector<uint64_t> extra(l->fs.h.size());
    for (size_t f = 0; f < extra.size(); f++) extra[f] = l->fs.h[f].measure_every ? n_records : 0;
    int rc = lane_ensure_rings(l, extra);
    if (rc) return rc;
  }
  return ISING_OK;
}

int ising_batch_set_shape(ising_batch* b, int shape) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  if (shape != ISING_SHAPE_AUTO && shape != ISING_SHAPE_GRID_1 && shape != ISING_SHAPE_GRID_2 &&
      shape != ISING_SHAPE_GRID_Q && shape != ISING_SHAPE_CLUSTER)
    return fail(ISING_EINVAL, "batches take AUTO, GRID_1, GRID_2, GRID_Q or CLUSTER");
  if (shape == ISING_SHAPE_CLUSTER) {
    const uint32_t C = b->cl_pinned ? b->cl_pinned : batch_auto_cluster(b);
    if (C == 0) return fail(ISING_EINVAL, "some film of the batch fits no cluster size");
    int rc = batch_apply_cluster(b, C);
    if (!rc) b->shape = shape;
    return rc;
  }
  b->shape = shape;
  if (shape == ISING_SHAPE_AUTO && b->tuned_shape == ISING_SHAPE_CLUSTER) return batch_apply_cluster(b, b->tuned_cl);
  const uint32_t items = shape == ISING_SHAPE_AUTO ? (b->tuned_shape ? shape_items(b->tuned_shape) : 1u)
                                                   : shape_items(shape);
  return batch_apply_items(b, items);
}

int ising_batch_get_shape(ising_batch* b, int* shape) {
  clear_error();
  if (!b || !shape) return fail(ISING_EINVAL, "NULL argument");
  *shape = b->lanes[0]->cl_size ? ISING_SHAPE_CLUSTER : items_shape(b->lanes[0]->fs.items);
  return ISING_OK;
}

int ising_batch_set_cluster_size(ising_batch* b, uint32_t cluster_size) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  if (cluster_size > kClusterMaxSize) return fail(ISING_EINVAL, "clusters hold at most %u CTAs", kClusterMaxSize);
  if (cluster_size) {  // every film must qualify before anything changes
    uint32_t smem, threads;
    bool exact;
    for (Lane* l : b->lanes) {
      int rc = lane_cluster_params(l, cluster_size, 1, &smem, &threads, &exact);
      if (rc) return rc;
    }
  }
  b->cl_pinned = cluster_size;
  if (b->lanes[0]->cl_size)  // on the cluster path now (pinned, or the autotuner's pick)
    return batch_apply_cluster(b, cluster_size ? cluster_size
                                               : (b->shape == ISING_SHAPE_CLUSTER ? batch_auto_cluster(b)
                                                                                  : b->tuned_cl));
  return ISING_OK;
}

int ising_batch_get_cluster_size(const ising_batch* b, uint32_t* cluster_size) {
  clear_error();
  if (!b || !cluster_size) return fail(ISING_EINVAL, "NULL argument");
  *cluster_size = b->lanes[0]->cl_size;
  return ISING_OK;
}

int ising_batch_autotune(ising_batch* b, int* shape) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  // a scratch batch of the same films in the same lanes, from their initial
  // states: the kernels do the same work whatever the spins are, and this
  // batch is not touched; every candidate is timed with all lanes running
  DeviceGuard dev(b->device);
  ising_batch* s = nullptr;
  int rc = ising_batch_create_lanes(b->jobs.data(), b->jobs.size(), (uint32_t)b->lanes.size(), &s);
  if (rc) return rc;
  double sites = 0;
  for (const auto& j : b->jobs) sites += (double)j.Lx * j.Ly * j.Lz;
  uint64_t n = (uint64_t)std::min(1024.0, std::max(64.0, std::round(4e8 / sites)));
  // the grid shapes replay captured chunks only in calls of two chunks or
  // more (lane_sweep), as long runs do: where launch overhead matters (small
  // sets), time calls that long
  uint64_t G = 1;
  for (const auto& j : b->jobs)
    if (j.measure_every) G = lcm_u64(G, j.measure_every);
  if (G == 1) G = 64;
  while (G < 16) G *= 2;
  if (G <= 4096 && sites * 2.0 * (double)G <= 4e10) n = std::max<uint64_t>(n, 2 * G);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = fail(ISING_ECUDA, "event creation failed");
  int best = ISING_SHAPE_GRID_1;
  uint32_t best_cl = 0;
  float best_ms = 3.0e38f;
  // grid shapes, then the cluster path at each cluster size for which every
  // film qualifies
  std::vector<std::pair<int, uint32_t>> cands = {
      {ISING_SHAPE_GRID_1, 0}, {ISING_SHAPE_GRID_2, 0}, {ISING_SHAPE_GRID_Q, 0}};
  {
    const size_t n_sm = (size_t)std::max(1, b->lanes[0]->fs.n_sm);
    for (uint32_t C = 1; C <= kClusterMaxSize && C * b->lanes.size() <= n_sm; C++) {
      const uint32_t per_sm = 1;
      bool ok = true;
      for (const Lane* l : b->lanes) {
        uint32_t smem = 0, threads = 0;
        bool exact = false;
        ok = ok && lane_cluster_params(l, C, per_sm, &smem, &threads, &exact) == ISING_OK;
      }
      clear_error();
      if (ok) cands.push_back({ISING_SHAPE_CLUSTER, C});
    }
  }
  for (size_t ci = 0; !rc && ci < cands.size(); ci++) {
    const int cand = cands[ci].first;
    rc = cand == ISING_SHAPE_CLUSTER ? batch_apply_cluster(s, cands[ci].second) : batch_apply_items(s, shape_items(cand));
    float ms = 3.0e38f;
    for (int rep = 0; !rc && rep < 3; rep++) {  // the first run captures the graphs
      if (cudaEventRecord(e0, s->stream()) != cudaSuccess) rc = fail(ISING_ECUDA, "event record failed");
      if (!rc) rc = batch_sweep(s, n, 1);
      if (!rc && cudaEventRecord(e1, s->stream()) != cudaSuccess) rc = fail(ISING_ECUDA, "event record failed");
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(ISING_ECUDA, "event wait failed");
      float t = 0.f;
      if (!rc && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = fail(ISING_ECUDA, "event time failed");
      if (!rc && rep > 0) ms = std::min(ms, t);
      for (Lane* l : s->lanes)  // drop the records
        for (size_t f = 0; f < l->fs.h.size(); f++) l->rec_read[f] = l->rec_written[f];
    }
    if (!rc && ms < kTuneMargin * best_ms) {  // a later shape must win clearly
      best_ms = ms;
      best = cand;
      best_cl = cands[ci].second;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  ising_batch_destroy(s);
  if (rc) return rc;
  b->tuned_shape = best;
  b->tuned_cl = best_cl;
  if (b->shape == ISING_SHAPE_AUTO)
    rc = best == ISING_SHAPE_CLUSTER ? batch_apply_cluster(b, best_cl) : batch_apply_items(b, shape_items(best));
  if (!rc && shape) *shape = best;
  return rc;
}

int ising_batch_get_spins(ising_batch* b, size_t i, int8_t* s) {
  clear_error();
  if (!b || !s) return fail(ISING_EINVAL, "NULL argument");
  if (i >= b->jobs.size()) return fail(ISING_ENOTFOUND, "film %zu out of range", i);
  Lane* l = b->lane_of(i);
  if (!l->d_stage && dev_alloc(&l->d_stage, l->stage_bytes) != cudaSuccess)
    return fail(ISING_ENOMEM, "cannot allocate the spin staging buffer");
  const FilmDesc& d = l->fs.h[b->index_in_lane(i)];
  ISG_CK(launch_unpack(d, l->fs.pool, l->d_stage, l->fs.stream));
  ISG_CK(cudaMemcpyAsync(s, l->d_stage, (size_t)d.Lx * d.Ly * d.Lz, cudaMemcpyDeviceToHost, l->fs.stream));
  ISG_CK(cudaStreamSynchronize(l->fs.stream));
  return ISING_OK;
}

int ising_batch_read_series(ising_batch* b, size_t i, int64_t* buf, size_t cap, size_t* n_records) {
  clear_error();
  if (!b || !n_records || (cap && !buf)) return fail(ISING_EINVAL, "NULL argument");
  if (i >= b->jobs.size()) return fail(ISING_ENOTFOUND, "film %zu out of range", i);
  Lane* l = b->lane_of(i);
  const size_t j = b->index_in_lane(i);
  ISG_CK(cudaStreamSynchronize(l->fs.stream));
  const FilmDesc& d = l->fs.h[j];
  const size_t rl = record_len(d);
  const uint64_t pending = l->rec_written[j] - l->rec_read[j];
  const uint64_t k = std::min<uint64_t>(pending, cap);
  uint64_t t = 0;
  while (t < k) {
    const uint64_t slot = (l->rec_read[j] + t) % d.rec_cap;
    const uint64_t run = std::min<uint64_t>(k - t, d.rec_cap - slot);
    ISG_CK(cudaMemcpyAsync(buf + t * rl, l->fs.rec + d.rec_off + slot * rl, run * rl * sizeof(int64_t),
                           cudaMemcpyDeviceToHost, l->fs.stream));
    t += run;
  }
  ISG_CK(cudaStreamSynchronize(l->fs.stream));
  l->rec_read[j] += k;
  *n_records = (size_t)k;
  return ISING_OK;
}

int ising_batch_pending_records(const ising_batch* b, size_t i, size_t* n) {
  clear_error();
  if (!b || !n) return fail(ISING_EINVAL, "NULL argument");
  if (i >= b->jobs.size()) return fail(ISING_ENOTFOUND, "film %zu out of range", i);
  const Lane* l = b->lane_of(i);
  const size_t j = b->index_in_lane(i);
  *n = (size_t)(l->rec_written[j] - l->rec_read[j]);
  return ISING_OK;
}

int ising_batch_synchronize(ising_batch* b, double timeout_s) {
  clear_error();
  if (!b) return fail(ISING_EINVAL, "NULL batch");
  for (Lane* l : b->lanes) {  // the batch's stream has joined the others; wait on each all the same
    int rc = wait_stream(l->fs.stream, timeout_s);
    if (rc) return rc;
  }
  return ISING_OK;
}

int ising_batch_destroy(ising_batch* b) {
  if (!b) return ISING_OK;
  for (Lane* l : b->lanes) lane_destroy(l);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
  return ISING_OK;
}

}  // extern "C"
