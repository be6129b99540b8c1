// Continuous-batching job server.
//
// Jobs (film shape, T, H1, key, sweeps) are queued by ising_batch_submit.  A
// host thread keeps the device busy with chunks of `chunk` sweeps over every
// admitted job, two chunks in flight:
//   1. before reusing a slot (one of two), wait for the chunk that last used
//      it and retire the jobs that finished in it: copy their records and
//      final spins out of pinned staging, return their arena space;
//   2. admit queued jobs, in arrival order, while their packed lattice, record
//      series, partial sums and unpack staging fit in a fixed device arena;
//   3. split the running jobs between two lanes (by sites), write each
//      lane's descriptors into the slot's pinned staging and copy them to the
//      slot's device buffer, enqueue each lane's update/record launches and
//      the advance of its sweep counters on the lane's own stream (the lanes
//      run concurrently: one's launch boundaries overlap the other's work),
//      join them, and queue the unpack + copy-out of the jobs that finish
//      inside the chunk.
// The host prepares chunk i+1 while chunk i runs.
// A job that reaches its last sweep inside a chunk stops there (sweep_end).
// Each job's random stream depends only on its own key, so its result is the
// same alone or in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>

#include "ising_host.h"

using namespace isg;

namespace {

constexpr size_t kAlign = 256;
constexpr double kWaitLimit = 600.0;  // seconds a chunk may take before the server gives up

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
  uint64_t first_chunk = 0, last_chunk = 0;  // chunks that ran its sweeps
  FilmDesc d{};  // host mirror; d.sweep = sweeps enqueued so far
  uint64_t n_records = 0;
  size_t off_spin = 0, off_rec = 0, off_part = 0, off_stage = 0;
  size_t b_spin = 0, b_rec = 0, b_part = 0, b_stage = 0;
  bool inited = false;
  std::vector<int64_t> records;
  std::vector<int8_t> spins;
};

size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

void job_footprint(Job& j) {
  const FilmDesc& d = j.d;
  j.b_spin = round_up(film_words(d) * sizeof(uint32_t));
  j.b_rec = round_up(std::max<uint64_t>(j.n_records, 1) * record_len(d) * sizeof(int64_t));
  j.b_part = round_up(part_len(d) * sizeof(int64_t));
  j.b_stage = round_up((size_t)d.Lx * d.Ly * d.Lz);
}

size_t footprint_bytes(const Job& j) { return j.b_spin + j.b_rec + j.b_part + j.b_stage; }

// One of the two chunk slots: device descriptors, pinned staging for them, the
// event that marks the chunk done, and pinned space for finished results.
struct Slot {
  char* d_meta = nullptr;   // [lane 0 | lane 1], meta_bytes each
  char* h_stage = nullptr;
  cudaEvent_t done = nullptr;
  LaunchSet L, L2;          // lane 0, lane 1
  bool busy = false;
  std::vector<ising_ticket> finishing;
  std::vector<size_t> res_off;
  char* h_res = nullptr;
  size_t res_cap = 0;
};

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
  FilmSet fs;   // lane 0: device, stream, occupancy; pool/part/rec point into the arena
  FilmSet fs2;  // lane 1: its own stream, the same arena
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::deque<ising_ticket> queue;
  std::unordered_map<ising_ticket, Job> jobs;
  std::vector<ising_ticket> running;
  ising_ticket next_ticket = 1;
  uint64_t n_finished = 0, n_chunks = 0, attempts = 0;
  std::chrono::steady_clock::time_point t0;

  // chunk slots and the capacities their descriptor buffers were sized for
  Slot slot[2];
  uint32_t cap_films = 0, cap_upd = 0, cap_meas = 0;
  size_t meta_bytes = 0;  // one lane's share of a slot's descriptor buffer
  uint32_t grid_upd = 0, grid_meas = 0, grid_fin = 0, grid_adv = 0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  void loop();
  int ensure_capacity(uint32_t nf, uint32_t nu, uint32_t nm);
  int wait_slot(Slot& s);
  void retire(Slot& s);  // with the lock held
  void release_slots();
  void release_lanes();  // both film sets, the fork/join events and the arena
};

// Descriptor buffers large enough for nf films, nu update and nm measurement
// blocks (grown only between chunks, once no chunk uses them).
int ising_server::ensure_capacity(uint32_t nf, uint32_t nu, uint32_t nm) {
  bool held = true;  // every slot's areas (a failed allocation leaves some out)
  for (const Slot& s : slot) held = held && s.d_meta && s.h_stage;
  if (nf <= cap_films && nu <= cap_upd && nm <= cap_meas && held) return ISING_OK;
  for (Slot& s : slot) {
    int rc = wait_slot(s);
    if (rc) return rc;
  }
  auto grow = [](uint32_t cap, uint32_t need, uint32_t floor_) {
    if (cap >= need && cap >= floor_) return cap;
    return std::max<uint32_t>({floor_, need, 2 * cap});
  };
  cap_films = grow(cap_films, nf, 1024);
  cap_upd = grow(cap_upd, nu, 1u << 16);
  cap_meas = grow(cap_meas, nm, 1u << 16);
  meta_bytes = sizeof(LaunchHdr) + (size_t)cap_films * sizeof(FilmDesc) + ((size_t)cap_upd + cap_meas) * 4;
  meta_bytes = (meta_bytes + kAlign - 1) / kAlign * kAlign;
  auto carve = [&](char* base, LaunchSet& L) {
    L.hdr = reinterpret_cast<LaunchHdr*>(base);
    L.films = reinterpret_cast<FilmDesc*>(base + sizeof(LaunchHdr));
    L.owner_upd = reinterpret_cast<uint32_t*>(base + sizeof(LaunchHdr) + (size_t)cap_films * sizeof(FilmDesc));
    L.owner_meas = L.owner_upd + cap_upd;
  };
  for (Slot& s : slot) {
    if (s.d_meta) cudaFree(s.d_meta);
    if (s.h_stage) cudaFreeHost(s.h_stage);
    s.d_meta = nullptr;
    s.h_stage = nullptr;
    if (dev_alloc(&s.d_meta, 2 * meta_bytes) != cudaSuccess)
      return fail(ISING_ENOMEM, "cannot allocate %zu bytes of launch descriptors", 2 * meta_bytes);
    if (host_alloc(&s.h_stage, 2 * meta_bytes) != cudaSuccess)
      return fail(ISING_ENOMEM, "cannot allocate %zu bytes of pinned staging", 2 * meta_bytes);
    carve(s.d_meta, s.L);
    carve(s.d_meta + meta_bytes, s.L2);
  }
  return ISING_OK;
}

int ising_server::wait_slot(Slot& s) {
  if (!s.busy) return ISING_OK;
  const auto t = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(s.done);
    if (e == cudaSuccess) return ISING_OK;
    if (e != cudaErrorNotReady) return fail(ISING_ECUDA, "chunk: %s", cudaGetErrorString(e));
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count() > kWaitLimit)
      return fail(ISING_ETIMEOUT, "a chunk ran longer than %.0f s", kWaitLimit);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void ising_server::retire(Slot& s) {
  const double tf = now();
  for (size_t i = 0; i < s.finishing.size(); i++) {
    Job& j = jobs[s.finishing[i]];
    const size_t rl = record_len(j.d);
    const size_t rb = j.n_records * rl * sizeof(int64_t);
    j.records.resize(j.n_records * rl);
    if (rb) std::memcpy(j.records.data(), s.h_res + s.res_off[i], rb);
    j.spins.resize((size_t)j.d.Lx * j.d.Ly * j.d.Lz);
    std::memcpy(j.spins.data(), s.h_res + s.res_off[i] + rb, j.spins.size());
    arena.release(j.off_spin, j.b_spin);
    arena.release(j.off_rec, j.b_rec);
    arena.release(j.off_part, j.b_part);
    arena.release(j.off_stage, j.b_stage);
    j.state = kDone;
    j.t_finish = tf;
    n_finished++;
  }
  if (!s.finishing.empty()) {
    running.erase(std::remove_if(running.begin(), running.end(),
                                 [&](ising_ticket t) { return jobs[t].state == kDone; }),
                  running.end());
    cv_done.notify_all();
  }
  s.finishing.clear();
  s.res_off.clear();
  s.busy = false;
}

void ising_server::loop() {
  cudaSetDevice(fs.device);
  std::unique_lock<std::mutex> lk(mu);
  uint64_t chunk_id = 0;
  auto stop_with = [&](int rc) {
    error = rc;
    error_msg = last_error();
    stop = true;
    cv_done.notify_all();
  };
  while (!stop) {
    Slot& S = slot[chunk_id % 2];
    Slot& O = slot[(chunk_id + 1) % 2];
    if (S.busy) {
      lk.unlock();
      const int rc = wait_slot(S);
      lk.lock();
      if (rc) { stop_with(rc); break; }
      retire(S);
    }
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
    // jobs with sweeps left to enqueue
    std::vector<ising_ticket> films;
    for (ising_ticket t : running)
      if (jobs[t].d.sweep < jobs[t].d.sweep_end) films.push_back(t);
    if (films.empty()) {
      if (O.busy) {  // let the other chunk finish and retire it
        lk.unlock();
        const int rc = wait_slot(O);
        lk.lock();
        if (rc) { stop_with(rc); break; }
        retire(O);
        continue;
      }
      cv_work.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    // descriptors of the two lanes (the largest job first, each to the lane
    // with the fewer sites so far), and the jobs finishing in this chunk
    fs.h.clear();
    fs2.h.clear();
    std::vector<Job*> fresh, fin;
    {
      std::vector<ising_ticket> order(films);
      auto sites = [&](ising_ticket t) { return (double)jobs[t].d.Lx * jobs[t].d.Ly * jobs[t].d.Lz; };
      std::stable_sort(order.begin(), order.end(), [&](ising_ticket a, ising_ticket b) { return sites(a) > sites(b); });
      double load0 = 0, load1 = 0;
      for (ising_ticket t : order) {
        const bool first = load0 <= load1;
        (first ? fs.h : fs2.h).push_back(jobs[t].d);
        (first ? load0 : load1) += sites(t);
      }
    }
    for (ising_ticket t : films) {
      Job& j = jobs[t];
      if (!j.inited) fresh.push_back(&j);
      if (j.d.sweep_end - j.d.sweep <= chunk) fin.push_back(&j);
    }
    S.finishing.clear();
    for (ising_ticket t : films)
      if (jobs[t].d.sweep_end - jobs[t].d.sweep <= chunk) S.finishing.push_back(t);
    lk.unlock();
    fs2.items = fs.items;
    fs.layout(false);  // partial sums stay in each job's own arena area
    fs2.layout(false);
    int rc = ensure_capacity(std::max(fs.hh.n_films, fs2.hh.n_films), std::max(fs.hh.upd_blocks, fs2.hh.upd_blocks),
                             std::max(fs.hh.meas_blocks, fs2.hh.meas_blocks));
    // [hdr | films | owner_upd | owner_meas] of one lane into pinned staging
    auto stage = [&](const FilmSet& F, char* p) {
      std::memcpy(p, &F.hh, sizeof F.hh);
      std::memcpy(p + sizeof(LaunchHdr), F.h.data(), F.h.size() * sizeof(FilmDesc));
      uint32_t* ou = reinterpret_cast<uint32_t*>(p + sizeof(LaunchHdr) + (size_t)cap_films * sizeof(FilmDesc));
      uint32_t* om = ou + cap_upd;
      for (size_t f = 0; f < F.h.size(); f++) {
        const FilmDesc& d = F.h[f];
        const uint32_t nb = (grid_items(d, F.items) + words_per_block(F.items) - 1) / words_per_block(F.items);
        for (uint32_t b = 0; b < nb; b++) ou[d.upd_block_begin + b] = (uint32_t)f;
        for (uint32_t b = 0; b < meas_units(d); b++) om[d.meas_block_begin + b] = (uint32_t)f;
      }
    };
    // the used parts of one lane's buffer, on lane 0's stream
    auto upload = [&](const FilmSet& F, char* dev, const char* host) {
      const size_t off_u = sizeof(LaunchHdr) + (size_t)cap_films * sizeof(FilmDesc);
      const size_t off_m = off_u + (size_t)cap_upd * 4;
      const size_t b0 = sizeof(LaunchHdr) + F.h.size() * sizeof(FilmDesc);
      if (cudaMemcpyAsync(dev, host, b0, cudaMemcpyHostToDevice, fs.stream) != cudaSuccess ||
          cudaMemcpyAsync(dev + off_u, host + off_u, (size_t)F.hh.upd_blocks * 4, cudaMemcpyHostToDevice,
                          fs.stream) != cudaSuccess ||
          cudaMemcpyAsync(dev + off_m, host + off_m, (size_t)F.hh.meas_blocks * 4, cudaMemcpyHostToDevice,
                          fs.stream) != cudaSuccess)
        return fail(ISING_ECUDA, "descriptor upload failed");
      return (int)ISING_OK;
    };
    if (!rc) {
      stage(fs, S.h_stage);
      if (!fs2.h.empty()) stage(fs2, S.h_stage + meta_bytes);
      // pinned space for the results of the jobs finishing in this chunk
      size_t need = 0;
      S.res_off.clear();
      for (Job* j : fin) {
        S.res_off.push_back(need);
        need += j->n_records * record_len(j->d) * sizeof(int64_t) + (size_t)j->d.Lx * j->d.Ly * j->d.Lz;
        need = (need + 15) / 16 * 16;
      }
      if (need > S.res_cap) {
        if (S.h_res) cudaFreeHost(S.h_res);
        S.h_res = nullptr;
        S.res_cap = std::max(need, 2 * S.res_cap);
        if (host_alloc(&S.h_res, S.res_cap) != cudaSuccess) {
          S.res_cap = 0;
          rc = fail(ISING_ENOMEM, "cannot allocate %zu bytes of pinned result staging", need);
        }
      }
    }
    for (Job* j : fresh) {
      if (rc) break;
      // the record accumulators start at zero (the area may hold an earlier job's data)
      if (cudaMemsetAsync(arena_dev + j->off_part, 0, j->b_part, fs.stream) != cudaSuccess) {
        rc = fail(ISING_ECUDA, "partial-sum clear failed");
        break;
      }
      uint32_t flip_lo = 0;
      int flip_all = 0;
      if (j->p.init_kind == ISING_INIT_SLAB_Y) {
        const double t = std::floor(std::ldexp(j->p.flip_p, 32));
        if (t >= 4294967296.0) flip_all = 1; else flip_lo = (uint32_t)t;
      }
      if (launch_init(j->d, fs.pool, j->p.init_kind, flip_lo, flip_all, fs.stream) != cudaSuccess)
        rc = fail(ISING_ECUDA, "init launch failed");
    }
    if (!rc) rc = upload(fs, S.d_meta, S.h_stage);
    if (!rc && !fs2.h.empty()) rc = upload(fs2, S.d_meta + meta_bytes, S.h_stage + meta_bytes);
    // the chunk: lane 1 forks from lane 0's stream after the uploads and
    // initial states, and lane 0 joins it before the copy-outs; exact grids,
    // records only after sweeps where some job takes one
    const bool two = !rc && !fs2.h.empty();
    if (two && (cudaEventRecord(ev_fork, fs.stream) != cudaSuccess ||
                cudaStreamWaitEvent(fs2.stream, ev_fork, 0) != cudaSuccess))
      rc = fail(ISING_ECUDA, "lane fork failed");
    if (!rc) {
      fs.L = S.L;
      rc = fs.enqueue_sweeps(0, chunk, false, false);
      if (!rc && launch_advance(S.L, grid_adv, chunk, fs.stream) != cudaSuccess)
        rc = fail(ISING_ECUDA, "advance launch failed");
    }
    if (!rc && two) {
      fs2.L = S.L2;
      rc = fs2.enqueue_sweeps(0, chunk, false, false);
      if (!rc && launch_advance(S.L2, grid_adv, chunk, fs2.stream) != cudaSuccess)
        rc = fail(ISING_ECUDA, "advance launch failed");
      if (!rc && (cudaEventRecord(ev_join, fs2.stream) != cudaSuccess ||
                  cudaStreamWaitEvent(fs.stream, ev_join, 0) != cudaSuccess))
        rc = fail(ISING_ECUDA, "lane join failed");
    }
    for (size_t i = 0; !rc && i < fin.size(); i++) {
      Job* j = fin[i];
      FilmDesc d = j->d;  // geometry and offsets of the finished film
      const size_t rb = j->n_records * record_len(d) * sizeof(int64_t);
      if (rb && cudaMemcpyAsync(S.h_res + S.res_off[i], arena_dev + j->off_rec, rb, cudaMemcpyDeviceToHost,
                                fs.stream) != cudaSuccess)
        rc = fail(ISING_ECUDA, "record copy-out failed");
      if (!rc && launch_unpack(d, fs.pool, reinterpret_cast<int8_t*>(arena_dev + j->off_stage), fs.stream) !=
                     cudaSuccess)
        rc = fail(ISING_ECUDA, "unpack launch failed");
      if (!rc && cudaMemcpyAsync(S.h_res + S.res_off[i] + rb, arena_dev + j->off_stage,
                                 (size_t)d.Lx * d.Ly * d.Lz, cudaMemcpyDeviceToHost, fs.stream) != cudaSuccess)
        rc = fail(ISING_ECUDA, "spin copy-out failed");
    }
    if (!rc && cudaEventRecord(S.done, fs.stream) != cudaSuccess) rc = fail(ISING_ECUDA, "event record failed");
    lk.lock();
    if (rc) { stop_with(rc); break; }
    uint64_t work = 0;
    for (ising_ticket t : films) {
      Job& j = jobs[t];
      if (!j.inited) j.first_chunk = n_chunks;
      j.last_chunk = n_chunks;
      j.inited = true;
      const uint32_t left = j.d.sweep_end - j.d.sweep;
      work += (uint64_t)std::min(left, chunk) * j.d.Lx * j.d.Ly * j.d.Lz;
      j.d.sweep = left <= chunk ? j.d.sweep_end : j.d.sweep + chunk;
      if (j.d.measure_every) j.d.rec_next = j.d.sweep / j.d.measure_every;
    }
    S.busy = true;
    n_chunks++;
    attempts += work;
    chunk_id++;
  }
}

void ising_server::release_lanes() {
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  ev_fork = ev_join = nullptr;
  for (FilmSet* f : {&fs, &fs2}) {  // the arena is freed once, below, not by the film sets
    f->pool = nullptr;
    f->rec = nullptr;
    f->part = nullptr;
  }
  if (arena_dev) cudaFree(arena_dev);
  arena_dev = nullptr;
  fs2.release();
  fs.release();
}

void ising_server::release_slots() {
  for (Slot& s : slot) {
    if (s.done) cudaEventDestroy(s.done);
    if (s.d_meta) cudaFree(s.d_meta);
    if (s.h_stage) cudaFreeHost(s.h_stage);
    if (s.h_res) cudaFreeHost(s.h_res);
    s = Slot();
  }
}

extern "C" {

int ising_server_create(size_t hbm_budget_bytes, uint32_t chunk_sweeps, ising_server** out) {
  clear_error();
  if (!out) return fail(ISING_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes < (1u << 20)) return fail(ISING_EINVAL, "budget must be at least 1 MiB");
  if (chunk_sweeps == 0 || chunk_sweeps > 4096) return fail(ISING_EINVAL, "chunk_sweeps must be in 1..4096");
  ising_server* s = new (std::nothrow) ising_server();
  if (!s) return fail(ISING_ENOMEM, "host allocation failed");
  s->budget = hbm_budget_bytes / kAlign * kAlign;
  s->chunk = chunk_sweeps;
  int rc = s->fs.init_device();
  if (!rc) rc = s->fs2.init_device();
  if (rc) {
    s->fs2.release();
    s->fs.release();
    delete s;
    return rc;
  }
  if (dev_alloc(&s->arena_dev, s->budget) != cudaSuccess) {
    s->fs2.release();
    s->fs.release();
    delete s;
    return fail(ISING_ENOMEM, "cannot allocate the %zu-byte device arena", hbm_budget_bytes);
  }
  s->arena.reset(s->budget);
  for (FilmSet* f : {&s->fs, &s->fs2}) {
    f->pool = reinterpret_cast<uint32_t*>(s->arena_dev);
    f->rec = reinterpret_cast<int64_t*>(s->arena_dev);
    f->part = reinterpret_cast<int64_t*>(s->arena_dev);
  }
  s->grid_upd = s->fs.upd_grid_max();
  s->grid_meas = s->fs.meas_grid_max();
  s->grid_fin = (uint32_t)(2 * s->fs.n_sm);
  s->grid_adv = 64;
  for (Slot& sl : s->slot)
    if (!rc && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
      rc = fail(ISING_ECUDA, "event creation failed");
  if (!rc && (cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
              cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess))
    rc = fail(ISING_ECUDA, "event creation failed");
  if (!rc) rc = s->ensure_capacity(1, 1, 1);
  if (rc) {
    s->release_slots();
    s->release_lanes();
    delete s;
    return rc;
  }
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
    info->first_chunk = j.first_chunk;
    info->last_chunk = j.last_chunk;
  }
  s->running.erase(std::remove(s->running.begin(), s->running.end(), t), s->running.end());
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
  uint64_t run = 0;
  for (ising_ticket t : s->running)
    if (s->jobs.count(t) && s->jobs[t].state == kRunning) run++;
  st->running = run;
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
  if (s->fs2.stream) cudaStreamSynchronize(s->fs2.stream);
  s->release_slots();
  s->release_lanes();
  delete s;
  return ISING_OK;
}

}  // extern "C"
