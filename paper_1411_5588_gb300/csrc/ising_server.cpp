// Continuous-batching job server.
//
// Jobs (film shape, T, H1, key, sweeps) are queued by ising_batch_submit.  A
// host thread repeatedly (1) admits queued jobs whose packed lattice, record
// series, partial sums and unpack staging fit in a device arena of fixed size,
// (2) runs one chunk of sweeps over every admitted job in shared launches --
// a job that reaches its last sweep inside a chunk simply stops (sweep_end),
// (3) retires finished jobs, copying their records and final spins to the
// host and returning their arena space.  Each job's random stream depends only
// on its own key, so its result is the same alone or in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>

#include "ising_host.h"

using namespace isg;

namespace {

constexpr size_t kAlign = 256;

// First-fit allocator over [0, size) bytes.
struct Arena {
  std::map<size_t, size_t> free_;  // offset -> length
  size_t size = 0, used = 0;
  void reset(size_t n) {
    free_.clear();
    free_[0] = n;
    size = n;
    used = 0;
  }
  bool alloc(size_t n, size_t* off) {
    n = (n + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, at = it->first + n;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + kAlign - 1) / kAlign * kAlign;
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

enum JobState { kQueued, kRunning, kDone };

struct Job {
  ising_job p{};
  JobState state = kQueued;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  FilmDesc d{};
  uint64_t n_records = 0;
  size_t off_spin = 0, off_rec = 0, off_part = 0, off_stage = 0;
  size_t b_spin = 0, b_rec = 0, b_part = 0, b_stage = 0;
  bool inited = false;
  std::vector<int64_t> records;
  std::vector<int8_t> spins;
};

size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

}  // namespace

struct ising_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  int error = ISING_OK;
  std::string error_msg;
  size_t budget = 0;
  uint32_t chunk = 100;
  char* arena_dev = nullptr;
  Arena arena;
  FilmSet fs;
  std::deque<ising_ticket> queue;
  std::unordered_map<ising_ticket, Job> jobs;
  std::vector<ising_ticket> running;
  ising_ticket next_ticket = 1;
  uint64_t n_finished = 0, n_chunks = 0, attempts = 0;
  std::chrono::steady_clock::time_point t0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  void loop();
  int run_chunk(std::unique_lock<std::mutex>& lk);
};

namespace {

void job_footprint(Job& j) {
  const FilmDesc& d = j.d;
  j.b_spin = round_up(film_words(d) * sizeof(uint32_t));
  j.b_rec = round_up(std::max<uint64_t>(j.n_records, 1) * record_len(d) * sizeof(int64_t));
  j.b_part = round_up(part_len(d) * sizeof(int64_t));
  j.b_stage = round_up((size_t)d.Lx * d.Ly * d.Lz);
}

size_t footprint_bytes(const Job& j) { return j.b_spin + j.b_rec + j.b_part + j.b_stage; }

}  // namespace

// Runs one chunk over the running jobs; called with the lock held, releases it
// while the device works.
int ising_server::run_chunk(std::unique_lock<std::mutex>& lk) {
  // descriptors of the running jobs
  fs.h.clear();
  std::vector<ising_ticket> films = running;
  for (ising_ticket t : films) fs.h.push_back(jobs[t].d);
  std::vector<Job*> fresh;
  for (ising_ticket t : films)
    if (!jobs[t].inited) fresh.push_back(&jobs[t]);
  lk.unlock();
  fs.layout(false);  // partial sums stay in each job's own arena area
  for (Job* j : fresh) {
    uint32_t flip_lo = 0;
    int flip_all = 0;
    if (j->p.init_kind == ISING_INIT_SLAB_Y) {
      const double t = std::floor(std::ldexp(j->p.flip_p, 32));
      if (t >= 4294967296.0) flip_all = 1; else flip_lo = (uint32_t)t;
    }
    ISG_CK(launch_init(j->d, fs.pool, j->p.init_kind, flip_lo, flip_all, fs.stream));
  }
  int rc = fs.upload();
  if (rc) return rc;
  uint32_t K = chunk;
  uint64_t work = 0;
  for (const auto& d : fs.h) {
    const uint32_t left = d.sweep_end - d.sweep;
    work += (uint64_t)std::min(left, K) * d.Lx * d.Ly * d.Lz;
  }
  rc = fs.enqueue_sweeps(0, K, false, false);
  if (rc) return rc;
  ISG_CK(launch_advance(fs.L, (fs.hh.n_films + 127) / 128, K, fs.stream));
  // finished jobs: final spins into their staging areas
  std::vector<size_t> done_idx;
  for (size_t f = 0; f < fs.h.size(); f++) {
    FilmDesc& d = fs.h[f];
    const uint32_t left = d.sweep_end - d.sweep;
    d.sweep = left <= K ? d.sweep_end : d.sweep + K;
    if (d.measure_every) d.rec_next = d.sweep / d.measure_every;
    if (d.sweep == d.sweep_end) {
      done_idx.push_back(f);
      Job* j = nullptr;
      {
        lk.lock();
        j = &jobs[films[f]];
        lk.unlock();
      }
      ISG_CK(launch_unpack(d, fs.pool, reinterpret_cast<int8_t*>(arena_dev + j->off_stage), fs.stream));
    }
  }
  rc = wait_stream(fs.stream, 600.0);
  if (rc) return rc;
  std::vector<std::pair<ising_ticket, Job*>> fin;
  lk.lock();
  for (ising_ticket t : films) jobs[t].inited = true;
  for (size_t f = 0; f < fs.h.size(); f++) jobs[films[f]].d = fs.h[f];
  for (size_t f : done_idx) fin.push_back({films[f], &jobs[films[f]]});
  n_chunks++;
  attempts += work;
  lk.unlock();
  for (auto& pr : fin) {
    Job* j = pr.second;
    const size_t rl = record_len(j->d);
    j->records.resize(j->n_records * rl);
    if (j->n_records)
      ISG_CK(cudaMemcpy(j->records.data(), arena_dev + j->off_rec, j->n_records * rl * sizeof(int64_t),
                        cudaMemcpyDeviceToHost));
    j->spins.resize((size_t)j->d.Lx * j->d.Ly * j->d.Lz);
    ISG_CK(cudaMemcpy(j->spins.data(), arena_dev + j->off_stage, j->spins.size(), cudaMemcpyDeviceToHost));
  }
  lk.lock();
  const double tf = now();
  for (auto& pr : fin) {
    Job* j = pr.second;
    arena.release(j->off_spin, j->b_spin);
    arena.release(j->off_rec, j->b_rec);
    arena.release(j->off_part, j->b_part);
    arena.release(j->off_stage, j->b_stage);
    j->state = kDone;
    j->t_finish = tf;
    n_finished++;
    running.erase(std::find(running.begin(), running.end(), pr.first));
  }
  if (!fin.empty()) cv_done.notify_all();
  return ISING_OK;
}

void ising_server::loop() {
  cudaSetDevice(fs.device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    // admission in arrival order while the arena has room
    while (!queue.empty()) {
      Job& j = jobs[queue.front()];
      size_t o1, o2, o3, o4;
      if (!arena.alloc(j.b_spin, &o1)) break;
      if (!arena.alloc(j.b_rec, &o2)) { arena.release(o1, j.b_spin); break; }
      if (!arena.alloc(j.b_part, &o3)) { arena.release(o1, j.b_spin); arena.release(o2, j.b_rec); break; }
      if (!arena.alloc(j.b_stage, &o4)) {
        arena.release(o1, j.b_spin); arena.release(o2, j.b_rec); arena.release(o3, j.b_part);
        break;
      }
      j.off_spin = o1; j.off_rec = o2; j.off_part = o3; j.off_stage = o4;
      j.d.spin_off = o1 / sizeof(uint32_t);
      j.d.rec_off = o2 / sizeof(int64_t);
      j.d.part_off = o3 / sizeof(int64_t);
      j.state = kRunning;
      j.t_admit = now();
      running.push_back(queue.front());
      queue.pop_front();
    }
    if (running.empty()) {
      cv_work.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    int rc = run_chunk(lk);
    if (!lk.owns_lock()) lk.lock();
    if (rc) {
      error = rc;
      error_msg = last_error();
      stop = true;
      cv_done.notify_all();
    }
  }
}

extern "C" {

int ising_server_create(size_t hbm_budget_bytes, uint32_t chunk_sweeps, ising_server** out) {
  clear_error();
  if (!out) return fail(ISING_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes < (1u << 20)) return fail(ISING_EINVAL, "budget must be at least 1 MiB");
  if (chunk_sweeps == 0) return fail(ISING_EINVAL, "chunk_sweeps must be > 0");
  ising_server* s = new (std::nothrow) ising_server();
  if (!s) return fail(ISING_ENOMEM, "host allocation failed");
  s->budget = hbm_budget_bytes / kAlign * kAlign;
  s->chunk = chunk_sweeps;
  int rc = s->fs.init_device();
  if (rc) { delete s; return rc; }
  if (cudaMalloc(&s->arena_dev, s->budget) != cudaSuccess) {
    cudaGetLastError();
    s->fs.release();
    delete s;
    return fail(ISING_ENOMEM, "cannot allocate the %zu-byte device arena", hbm_budget_bytes);
  }
  s->arena.reset(s->budget);
  s->fs.pool = reinterpret_cast<uint32_t*>(s->arena_dev);
  s->fs.rec = reinterpret_cast<int64_t*>(s->arena_dev);
  s->fs.part = reinterpret_cast<int64_t*>(s->arena_dev);
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return ISING_OK;
}

int ising_batch_submit(ising_server* s, const ising_job* jobs, size_t n, ising_ticket* first) {
  clear_error();
  if (!s || !first || (n && !jobs)) return fail(ISING_EINVAL, "NULL argument");
  std::vector<Job> nj(n);
  for (size_t i = 0; i < n; i++) {
    const ising_job& p = jobs[i];
    int rc = check_film(p.Lx, p.Ly, p.Lz, p.T, p.y_mode, p.x_mode);
    if (rc) return fail(rc, "job %zu: %s", i, last_error());
    if (p.n_sweeps == 0 || p.n_sweeps >= 0xFFFFFFFFull) return fail(ISING_EINVAL, "job %zu: bad n_sweeps", i);
    if (p.init_kind < ISING_INIT_RANDOM || p.init_kind > ISING_INIT_ALL_UP)
      return fail(ISING_EINVAL, "job %zu: bad init kind", i);
    if (p.init_kind == ISING_INIT_SLAB_Y && !(p.flip_p >= 0.0 && p.flip_p <= 1.0))
      return fail(ISING_EINVAL, "job %zu: flip_p must be in [0,1]", i);
    Job& j = nj[i];
    j.p = p;
    std::memset(&j.d, 0, sizeof j.d);
    fill_geometry(j.d, p.Lx, p.Ly, p.Lz, p.y_mode, p.x_mode, p.seed, p.replica);
    build_tables(j.d, p.J, p.H, p.H1, p.T);
    j.d.measure_every = p.measure_every;
    j.d.sweep = 0;
    j.d.sweep_end = (uint32_t)p.n_sweeps;
    j.n_records = p.measure_every ? p.n_sweeps / p.measure_every : 0;
    j.d.rec_cap = (uint32_t)std::max<uint64_t>(j.n_records, 1);
    job_footprint(j);
    if (footprint_bytes(j) > s->budget)
      return fail(ISING_EINVAL, "job %zu needs %zu bytes, more than the %zu-byte budget", i, footprint_bytes(j),
                  s->budget);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->error) return fail(s->error, "server stopped: %s", s->error_msg.c_str());
  *first = s->next_ticket;
  const double t = s->now();
  for (size_t i = 0; i < n; i++) {
    nj[i].t_submit = t;
    const ising_ticket tk = s->next_ticket++;
    s->jobs.emplace(tk, std::move(nj[i]));
    s->queue.push_back(tk);
  }
  s->cv_work.notify_all();
  return ISING_OK;
}

int ising_batch_poll(ising_server* s, ising_ticket t, int* done) {
  clear_error();
  if (!s || !done) return fail(ISING_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(t);
  if (it == s->jobs.end()) return fail(ISING_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
  *done = it->second.state == kDone;
  if (!*done && s->error) return fail(s->error, "server stopped: %s", s->error_msg.c_str());
  return ISING_OK;
}

int ising_batch_wait(ising_server* s, ising_ticket t, double timeout_s) {
  clear_error();
  if (!s) return fail(ISING_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    auto it = s->jobs.find(t);
    if (it == s->jobs.end()) return fail(ISING_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
    if (it->second.state == kDone) return ISING_OK;
    if (s->error) return fail(s->error, "server stopped: %s", s->error_msg.c_str());
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout) {
      auto it2 = s->jobs.find(t);
      if (it2 != s->jobs.end() && it2->second.state == kDone) return ISING_OK;
      return fail(ISING_ETIMEOUT, "job %llu not finished after %.3f s", (unsigned long long)t, timeout_s);
    }
  }
}

int ising_batch_result(ising_server* s, ising_ticket t, int64_t* buf, size_t cap, int8_t* spins,
                       ising_job_info* info) {
  clear_error();
  if (!s) return fail(ISING_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(t);
  if (it == s->jobs.end()) return fail(ISING_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
  Job& j = it->second;
  if (j.state != kDone) return fail(ISING_EBUSY, "job %llu still running", (unsigned long long)t);
  const size_t rl = record_len(j.d);
  const size_t k = std::min<size_t>(cap, j.n_records);
  if (k && !buf) return fail(ISING_EINVAL, "NULL record buffer");
  if (k) std::memcpy(buf, j.records.data(), k * rl * sizeof(int64_t));
  if (spins) std::memcpy(spins, j.spins.data(), j.spins.size());
  if (info) {
    info->t_submit = j.t_submit;
    info->t_admit = j.t_admit;
    info->t_finish = j.t_finish;
    info->n_records = j.n_records;
  }
  s->jobs.erase(it);
  return ISING_OK;
}

int ising_server_get_stats(ising_server* s, ising_server_stats* st) {
  clear_error();
  if (!s || !st) return fail(ISING_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  st->bytes_in_use = s->arena.used;
  st->bytes_budget = s->budget;
  st->queued = s->queue.size();
  st->running = s->running.size();
  st->finished = s->n_finished;
  st->chunks = s->n_chunks;
  st->attempts = s->attempts;
  return ISING_OK;
}

int ising_server_destroy(ising_server* s) {
  if (!s) return ISING_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->fs.stream) cudaStreamSynchronize(s->fs.stream);
  s->fs.pool = nullptr;
  s->fs.rec = nullptr;
  s->fs.part = nullptr;
  if (s->arena_dev) cudaFree(s->arena_dev);
  s->fs.release();
  delete s;
  return ISING_OK;
}

}  // extern "C"
