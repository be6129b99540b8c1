// ising_measure_packed_noalloc: the observable record of a packed film,
// computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a framework or serving runtime that has
// already handed the whole device to its own pool allocator, or a loop that
// cannot afford cudaMalloc's implicit device synchronisation.  This entry point
// serves them: the caller passes the packed spins and the output record, and
// the per-block partial sums of the two-pass reduction live in a fixed
// file-scope device array instead of memory obtained at run time.
//
// Limits and sharing: the scratch holds kNoAllocScratchWords int64 partials
// (two per measurement block), so a film may use at most
// kNoAllocScratchWords / 2 measurement blocks (Lx * ceil(Ly * W / 1024)
// blocks, W = ceil(Lz / 64)).  Every call on a device uses the same array and
// leaves its partials there; each call overwrites every partial it later
// reads, so nothing needs clearing, but two calls whose kernels overlap on the
// GPU (different streams without ordering) race on the array and may produce
// wrong records.
#include <cuda_runtime.h>

#include <cstring>

#include "ising_host.h"

namespace isg {

constexpr uint32_t kNoAllocScratchWords = 16384;  // 128 KiB of int64 partials

static __device__ __align__(256) int64_t g_noalloc_scratch[kNoAllocScratchWords];

namespace {

constexpr int kNaBlock = 256;

__device__ __forceinline__ int64_t na_block_sum(int64_t v, int64_t* s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  int64_t t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += s_red[i];
  __syncthreads();
  return t;
}

// Checked builds (-DISING_CHECKED) count out-of-range word indices of this
// file's kernel the way the other kernels do (ising_check_counters adds them
// in): the first one is kept and the access reads word 0 instead.
#ifdef ISING_CHECKED
__device__ unsigned long long g_na_oob_count;
__device__ unsigned long long g_na_oob_first;
#endif

struct NaLoad {
  __device__ __forceinline__ uint32_t operator()(const uint32_t* p, size_t idx, size_t lim, uint32_t site) const {
#ifdef ISING_CHECKED
    if (idx >= lim) {
      atomicAdd(&g_na_oob_count, 1ull);
      atomicCAS(&g_na_oob_first, 0ull, ((unsigned long long)site << 48) | (idx & 0xFFFFFFFFFFFFull));
      return p[0];
    }
#else
    (void)lim;
    (void)site;
#endif
    return p[idx];
  }
};

// First pass: block (layer kx, chunk c) sums m and the +x/+y/+z bonds of its
// rows (measure_word, the record arithmetic every measurement kernel shares)
// into part[2 * (kx * bpl + c) + {0, 1}].
__global__ void __launch_bounds__(kNaBlock)
na_partial_kernel(const __grid_constant__ FilmDesc F, const uint32_t* __restrict__ spins,
                  int64_t* __restrict__ part) {
  __shared__ int64_t s_red[kNaBlock / 32];
  const uint32_t Lx = F.Lx, Ly = F.Ly, W = F.W, Wp = F.Wp, bpl = F.meas_bpl;
  const uint32_t kxm1 = blockIdx.x / bpl, chunk = blockIdx.x % bpl;
  const uint32_t* A = spins;
  const uint32_t* B = A + (size_t)Lx * Ly * Wp;
  int64_t msum = 0, bsum = 0;
  for (uint32_t it = chunk * blockDim.x + threadIdx.x; it < Ly * W; it += bpl * blockDim.x) {
    const uint32_t kym1 = it / W, w = it % W;
    int m, bb;
    measure_word(NaLoad{}, A, B, Wp, Lx, Ly, W, F.n, F.last_mask, F.x_pbc, F.y_mode, kxm1, kym1, w, m, bb);
    msum += m;
    bsum += bb;
  }
  const int64_t tm = na_block_sum(msum, s_red);
  const int64_t tb = na_block_sum(bsum, s_red);
  if (threadIdx.x == 0) {
    int64_t* p = part + 2 * ((size_t)kxm1 * bpl + chunk);
    p[0] = tm;
    p[1] = tb;
  }
}

// Second pass (one block): the record {sweep, B, M, M1, Mn, m(1..Lx)}.
__global__ void __launch_bounds__(kNaBlock)
na_finalize_kernel(const __grid_constant__ FilmDesc F, const int64_t* __restrict__ part, int64_t* __restrict__ rec,
                   uint64_t sweep) {
  __shared__ int64_t s_red[kNaBlock / 32];
  const uint32_t Lx = F.Lx, bpl = F.meas_bpl;
  int64_t M = 0, Bs = 0;
  for (uint32_t kx = threadIdx.x; kx < Lx; kx += blockDim.x) {
    int64_t m = 0;
    for (uint32_t c = 0; c < bpl; c++) {
      m += part[2 * ((size_t)kx * bpl + c)];
      Bs += part[2 * ((size_t)kx * bpl + c) + 1];
    }
    rec[5 + kx] = m;
    M += m;
  }
  const int64_t tM = na_block_sum(M, s_red);
  const int64_t tB = na_block_sum(Bs, s_red);
  if (threadIdx.x == 0) {
    rec[0] = (int64_t)sweep;
    rec[1] = tB;
    rec[2] = tM;
    rec[3] = rec[5];
    rec[4] = rec[5 + Lx - 1];
  }
}

// Device address of the scratch array on the current device.  Host code
// sees only a stand-in for the symbol, so the address is looked up on every
// call (no allocation; the runtime keeps it per loaded module), which also
// stays right after a device reset reloads the module.
int noalloc_scratch(int64_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return fail(ISING_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  *out = static_cast<int64_t*>(p);
  return ISING_OK;
}

}  // namespace

int read_noalloc_oob_counters(unsigned long long* count, unsigned long long* first) {
#ifdef ISING_CHECKED
  if (cudaMemcpyFromSymbol(count, g_na_oob_count, sizeof *count) != cudaSuccess) return -1;
  if (cudaMemcpyFromSymbol(first, g_na_oob_first, sizeof *first) != cudaSuccess) return -1;
  return 1;
#else
  *count = 0;
  *first = 0;
  return 0;
#endif
}

}  // namespace isg

using namespace isg;

extern "C" int ising_measure_packed_noalloc(const uint32_t* spins, int Lx, int Ly, int Lz, int y_mode, int x_mode,
                                            uint64_t sweep, int64_t* record, void* stream) {
  clear_error();
  if (!spins || !record) return fail(ISING_EINVAL, "NULL argument");
  int rc = check_film(Lx, Ly, Lz, 1.0, y_mode, x_mode);
  if (rc) return rc;
  FilmDesc d;
  std::memset(&d, 0, sizeof d);
  fill_geometry(d, Lx, Ly, Lz, y_mode, x_mode, 0, 0);
  const uint64_t blocks = (uint64_t)d.Lx * d.meas_bpl;
  if (2 * blocks > kNoAllocScratchWords)
    return fail(ISING_EINVAL, "film needs %llu measurement blocks; the fixed scratch holds %u",
                (unsigned long long)blocks, kNoAllocScratchWords / 2);
  int64_t* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  na_partial_kernel<<<(unsigned)blocks, kNaBlock, 0, st>>>(d, spins, scratch);
  ISG_CK(cudaGetLastError());
  na_finalize_kernel<<<1, kNaBlock, 0, st>>>(d, scratch, record, sweep);
  ISG_CK(cudaGetLastError());
  return ISING_OK;
}
