// Host-side launchers of the Ising-film kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ising_device.cuh"

namespace isg {

// Update kernels: threads per block, words per thread, blocks per SM; one
// block updates kItemsPerBlock consecutive words of one film.
constexpr uint32_t kFilmThreads = 128;
constexpr uint32_t kFilmItems = 2;
constexpr int kFilmMinBlocks = 6;
constexpr int kMultiMinBlocks = 5;  // the multi-film kernel carries both table paths
constexpr uint32_t kItemsPerBlock = kFilmThreads * kFilmItems;
constexpr int kMeasureBlock = 256;

// Items a measurement block covers per layer before another block is added.
constexpr uint32_t kMeasureItemsPerBlock = 4 * kMeasureBlock;

// Device arrays describing the films of a launch.
struct LaunchSet {
  FilmDesc* films = nullptr;         // n_films descriptors
  uint32_t* owner_upd = nullptr;     // virtual update block -> film
  uint32_t* owner_meas = nullptr;    // virtual measurement block -> film
  LaunchHdr* hdr = nullptr;          // sizes
};

cudaError_t launch_update(const LaunchSet& L, uint32_t grid, uint32_t* pool, uint32_t colour, uint32_t k,
                          cudaStream_t st);
// One half-sweep of a single film whose descriptor (with `sweep` absolute) is
// passed by value.
cudaError_t launch_update_film(const FilmDesc& d, uint32_t* pool, uint32_t colour, uint32_t sweep,
                               cudaStream_t st);
cudaError_t launch_measure(const LaunchSet& L, uint32_t grid, uint32_t fin_grid, const uint32_t* pool,
                           int64_t* part, int64_t* records, uint32_t done, int force, int64_t* direct,
                           cudaStream_t st);
cudaError_t launch_advance(const LaunchSet& L, uint32_t grid, uint32_t n_sweeps, cudaStream_t st);
cudaError_t launch_init(const FilmDesc& f, uint32_t* pool, int kind, uint32_t flip_lo, int flip_all,
                        cudaStream_t st);
cudaError_t launch_pack(const FilmDesc& f, uint32_t* pool, const int8_t* s, cudaStream_t st);
cudaError_t launch_unpack(const FilmDesc& f, const uint32_t* pool, int8_t* s, cudaStream_t st);
int update_blocks_per_sm();
int measure_blocks_per_sm();

}  // namespace isg
