// Host-side internals shared by the API translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "ising.h"
#include "ising_device.cuh"
#include "ising_launch.h"

namespace isg {

int fail(int code, const char* fmt, ...);
void clear_error();
const char* last_error();

// Polls a stream until it is idle or timeout_s passes (ETIMEOUT).
int wait_stream(cudaStream_t st, double timeout_s);

// cudaMalloc / cudaMallocHost that leave no error pending when they fail: a
// failed allocation stays CUDA's last error, and the next launch check would
// report it again against an unrelated call.  *p is null after a failure.
template <typename T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
  }
  return e;
}
template <typename T>
inline cudaError_t host_alloc(T** p, size_t bytes) {
  const cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
  }
  return e;
}

#define ISG_CK(call)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return ::isg::fail(ISING_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Validates a film's sizes and parameters; EINVAL with a message otherwise.
int check_film(int Lx, int Ly, int Lz, double T, int y_mode, int x_mode);

// Geometry, key and work sizes of a descriptor (no offsets, no tables).
void fill_geometry(FilmDesc& d, int Lx, int Ly, int Lz, int y_mode, int x_mode, uint64_t seed, uint32_t replica);

// Metropolis thresholds of Eq. 1 for the four row classes (binary64, libm exp).
void build_tables(FilmDesc& d, double J, double H, double H1, double T);

// Packed words of one film (both parity planes).
inline size_t film_words(const FilmDesc& d) { return 2 * (size_t)d.Lx * d.Ly * d.Wp; }
inline size_t record_len(const FilmDesc& d) { return 5 + (size_t)d.Lx; }
// Measurement partial sums, then the record accumulators (acc_offset).
inline size_t part_len(const FilmDesc& d) { return 2 * (size_t)d.Lx * d.meas_bpl + 2 * (size_t)d.Lx; }

// Films updated by the same launches: descriptors, owner tables and the
// device buffers they point into.
struct FilmSet {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_sm = 0, upd_per_sm = 0, meas_per_sm = 0;
  uint32_t items = 1;  // words per thread of the grid update kernel (1, 2; 0 = four threads per word)

  std::vector<FilmDesc> h;  // host mirror (counters tracked on the host too)
  LaunchHdr hh{};
  LaunchSet L;
  char* d_meta = nullptr;   // [hdr | films | owner_upd | owner_meas]
  size_t meta_bytes = 0;
  std::vector<char> staging;

  uint32_t* pool = nullptr;
  size_t pool_words = 0;
  int64_t* part = nullptr;
  size_t part_words = 0;
  int64_t* rec = nullptr;
  size_t rec_words = 0;

  int init_device();          // device, stream, occupancy
  void layout(bool assign_part = true);  // block ranges, owner tables, partial offsets
  int upload();               // copies hdr/films/owners to the device (synchronous)
  uint32_t upd_grid() const;  // grid of a direct launch
  uint32_t meas_grid() const;
  uint32_t fin_grid() const;
  uint32_t upd_grid_max() const { return (uint32_t)(n_sm * upd_per_sm); }
  uint32_t meas_grid_max() const { return (uint32_t)(n_sm * meas_per_sm); }
  // Kernels of sweeps k0..k0+n-1 of the current chunk, with measurements
  // where some film's measure_every divides (sweep + k + 1) (all_meas: after
  // every sweep, films decide on the device).
  int enqueue_sweeps(uint32_t k0, uint32_t n, bool all_meas, bool fixed_grid);
  int release();
  ~FilmSet() { release(); }
};

// A candidate launch shape replaces the autotuner's current best only when it
// is this much faster (candidates are tried in the order RESIDENT, GRID_1,
// GRID_2, GRID_Q), so that shapes within timing noise of each other resolve
// the same way on every run.
constexpr float kTuneMargin = 0.98f;

// Grid kernel words-per-thread code of a grid shape, and back.
inline uint32_t shape_items(int shape) {
  return shape == ISING_SHAPE_GRID_2 ? 2u : shape == ISING_SHAPE_GRID_Q ? 0u : 1u;
}
inline int items_shape(uint32_t items) {
  return items == 2 ? ISING_SHAPE_GRID_2 : items == 0 ? ISING_SHAPE_GRID_Q : ISING_SHAPE_GRID_1;
}

// Makes `device` current for the guard's lifetime (the scratch objects of
// the autotuners live on the tuned object's device).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess || prev == device || cudaSetDevice(device) != cudaSuccess) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Autotuner cache, shared by every handle of the process: the fastest launch
// shape (ISING_SHAPE_*) measured for a film shape, boundary, table variant
// and record interval.
struct TuneKey {
  uint32_t Lx, Ly, Lz, y_mode, x_pbc, exact, m_class;
  bool operator<(const TuneKey& o) const;
};
TuneKey tune_key(const FilmDesc& d, uint32_t measure_every);
bool tune_lookup(const TuneKey& k, int* shape);
void tune_store(const TuneKey& k, int shape);

}  // namespace isg
