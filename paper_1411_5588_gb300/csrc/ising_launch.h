// Host-side launchers of the Ising-film kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ising_device.cuh"

namespace isg {

// Grid update kernels: threads per block and blocks per SM.  A block updates
// items * kFilmThreads consecutive words of one film, items (words per
// thread, 1 or 2) being the launch shape the autotuner picks per film or
// film set: one word per thread halves the dependency chain of a launch
// (small and medium films are latency bound), two let each thread overlap
// the loads of its second word with the first word's arithmetic.
constexpr uint32_t kFilmThreads = 128;
constexpr int kFilmMinBlocks = 6;
constexpr int kMultiMinBlocks = 6;
constexpr int kMultiMinBlocks1 = 7;  // multi-film kernel, one word per thread, not summing records
// items = 0 is the quarter shape: four lanes share each word (they split its
// eight Philox calls), so a block covers kFilmThreads / 4 words.
__host__ __device__ constexpr uint32_t words_per_block(uint32_t items) {
  return items == 0 ? kFilmThreads / 4 : kFilmThreads * items;
}
constexpr int kMeasureBlock = 256;

// Items a measurement block covers per layer before another block is added;
// layers of fewer than kMeasureItemsPerBlock / 2 words are grouped, up to
// kMeasureMaxLpu of them per block.
constexpr uint32_t kMeasureItemsPerBlock = 4 * kMeasureBlock;
constexpr uint32_t kMeasureMaxLpu = 64;

// The film's per-layer record accumulators (int64 pairs: magnetisation,
// bonds; Lx of them) follow its measurement partial sums in the same area.
__host__ __device__ inline uint64_t acc_offset(const FilmDesc& d) {
  return d.part_off + 2ull * d.Lx * d.meas_bpl;
}

// Films of at least this many rows pack two rows per word when they qualify
// (fill_geometry); four rows pack at any size.
constexpr uint32_t kPack2Rows = 8192;

// Items of a film in the grid update kernels with `items` words per thread:
// thin films pack rows at one item per thread only.
__host__ __device__ inline uint32_t grid_items(const FilmDesc& d, uint32_t items) {
  return (items == 1 && d.pack > 1) ? d.pk_items : d.upd_items;
}

// Measurement blocks of one film.
inline uint32_t meas_units(const FilmDesc& d) {
  return d.meas_lpu > 1 ? (d.Lx + d.meas_lpu - 1) / d.meas_lpu : d.Lx * d.meas_bpl;
}

// Resident path: one block per film holds the film's packed planes in shared
// memory (row stride W) for a whole run of sweeps, records included.  Films
// up to kResidentMaxSites spins whose planes and layer sums fit in
// kResidentMaxSmem bytes qualify; larger ones use the per-half-sweep grid.
// Chosen automatically up to kResidentAutoSites: beyond that one SM's issue
// rate loses to the grid kernels (about 16 us per sweep there without
// records, 27 us with one every sweep).
constexpr uint32_t kResidentThreads = 512;
constexpr uint64_t kResidentMaxSites = 1ull << 16;
constexpr uint64_t kResidentAutoSites = 1ull << 15;
constexpr uint32_t kResidentMaxSmem = 48u * 1024u;

// Cluster-resident path: a thread-block cluster of C CTAs (C <= kClusterMaxSize)
// holds one film in distributed shared memory for a whole call of sweeps,
// each CTA a slab of ceil(Lx / C) layers or one fewer.  kClusterThreads is the
// most threads a CTA runs (one CTA per SM at the update body's registers);
// kClusterMaxSmem the most dynamic shared memory a CTA takes.  The exact-table
// variant (a strict compare and a mux tree per site) needs more registers, so
// it runs at most kClusterThreadsExact.
constexpr uint32_t kClusterThreads = 704;
constexpr uint32_t kClusterThreadsExact = 512;
__host__ __device__ constexpr uint32_t cluster_max_threads(bool exact) {
  return exact ? kClusterThreadsExact : kClusterThreads;
}
constexpr uint32_t kClusterMaxSize = 8;
constexpr uint32_t kClusterMaxSmem = 200u * 1024u;

// Device arrays describing the films of a launch.
struct LaunchSet {
  FilmDesc* films = nullptr;         // n_films descriptors
  uint32_t* owner_upd = nullptr;     // virtual update block -> film
  uint32_t* owner_meas = nullptr;    // virtual measurement block -> film
  LaunchHdr* hdr = nullptr;          // sizes
};

// exact: some film of the launch has a reachable thr = 0 entry (has_never);
// items: words per thread (1 or 2, or 0 for four lanes per word), matching the
// owner table's block size.  Records: with accumulate (colour 1) the films
// that record after sweep k add their record sums into their accumulators in
// part; with rec_done > 0 (colour 0) the films that recorded after rec_done
// sweeps have that record written into their rings in records by this
// launch (the chunk's last record goes through launch_record instead).
// pack: some film of the launch packs rows (FilmDesc::pack > 1; with items
// 1 its owner table counts groups of rows, grid_items).
cudaError_t launch_update(const LaunchSet& L, uint32_t grid, uint32_t* pool, uint32_t colour, uint32_t k, bool exact,
                          uint32_t items, bool pack, int64_t* part, int64_t* records, bool accumulate,
                          uint32_t rec_done, cudaStream_t st);
// One half-sweep of a single film whose descriptor (with `sweep` absolute) is
// passed by value; acc (colour 1 of a recorded sweep, else null): the film's
// accumulators.
cudaError_t launch_update_film(const FilmDesc& d, uint32_t* pool, uint32_t colour, uint32_t sweep, uint32_t items,
                               int64_t* acc, cudaStream_t st);
// Records of the films that record after `done` sweeps of the chunk, from the
// accumulators the half-sweep 1 launch filled (which it clears).
cudaError_t launch_record(const LaunchSet& L, uint32_t grid, int64_t* part, int64_t* records, uint32_t done,
                          cudaStream_t st);
cudaError_t launch_measure(const LaunchSet& L, uint32_t grid, uint32_t fin_grid, const uint32_t* pool,
                           int64_t* part, int64_t* records, uint32_t done, int force, int64_t* direct,
                           cudaStream_t st);
cudaError_t launch_advance(const LaunchSet& L, uint32_t grid, uint32_t n_sweeps, cudaStream_t st);
cudaError_t launch_init(const FilmDesc& f, uint32_t* pool, int kind, uint32_t flip_lo, int flip_all,
                        cudaStream_t st);
cudaError_t launch_pack(const FilmDesc& f, uint32_t* pool, const int8_t* s, cudaStream_t st);
cudaError_t launch_unpack(const FilmDesc& f, const uint32_t* pool, int8_t* s, cudaStream_t st);
// Dynamic shared memory of a film on the resident path, 0 if it does not qualify.
uint32_t resident_smem_bytes(const FilmDesc& d);
// Threads per block for a film on the resident path (a multiple of 32).
uint32_t resident_threads(const FilmDesc& d);
// n_sweeps sweeps (with their records) of films[0..n_films) on the resident
// path, one block each; every film must qualify, smem_bytes and threads cover
// the largest.  The kernel advances each descriptor's sweep and rec_next.
cudaError_t launch_resident(FilmDesc* films, uint32_t n_films, uint32_t smem_bytes, uint32_t threads, bool exact,
                            uint32_t* pool, int64_t* records, uint32_t n_sweeps, cudaStream_t st);
// Dynamic shared memory of a CTA of film d on the cluster-resident path with
// clusters of C CTAs, 0 if the film does not qualify (C out of range, fewer
// layers than C, or too large).
uint32_t cluster_smem_bytes(const FilmDesc& d, uint32_t C);
// CTAs of the cluster path that share one SM (1..kClusterMaxPerSm): a CTA's
// half-sweep ends at a cluster barrier where its warps wait for the slowest,
// and CTAs of other films on the same SM fill that wait.  per_sm divides the
// threads a CTA may run, and the launch pads each CTA's shared memory so
// that no more than per_sm CTAs fit on an SM.
constexpr uint32_t kClusterMaxPerSm = 3;
// Threads per CTA for film d with clusters of C CTAs, per_sm CTAs per SM: the
// slab's update items spread over as few full rounds as
// cluster_max_threads(exact) / per_sm allows (a multiple of 32).
uint32_t cluster_threads(const FilmDesc& d, uint32_t C, bool exact, uint32_t per_sm);
// Clusters of C CTAs (smem_bytes of dynamic shared memory needed and threads
// each, per_sm of them per SM) that one GPU can hold at once (0: such a
// launch cannot run), or -1 on a CUDA error.
int cluster_capacity(uint32_t C, uint32_t per_sm, uint32_t smem_bytes, uint32_t threads, bool exact);
// n_sweeps sweeps (with their records) of films on the cluster path:
// n_clusters clusters of C CTAs, per_sm CTAs per SM, cluster i sweeping the
// films list[n_clusters + 1 + j], j in [list[i], list[i + 1]), one after
// another (list: device memory).  Every listed film must qualify for C, and
// smem_bytes and threads cover the largest.  The kernel advances each
// descriptor's sweep and rec_next.
cudaError_t launch_cluster(FilmDesc* films, const uint32_t* list, uint32_t n_clusters, uint32_t C, uint32_t per_sm,
                           uint32_t smem_bytes, uint32_t threads, bool exact, uint32_t* pool, int64_t* records,
                           uint32_t n_sweeps, cudaStream_t st);
// Checked builds: the out-of-range access counters (returns 1); other
// builds return 0 with both zero; -1 on a CUDA error.
int read_oob_counters(unsigned long long* count, unsigned long long* first);
// The same for the allocation-free measurement kernel (ising_noalloc.cu).
int read_noalloc_oob_counters(unsigned long long* count, unsigned long long* first);
int update_blocks_per_sm();
int measure_blocks_per_sm();

}  // namespace isg
