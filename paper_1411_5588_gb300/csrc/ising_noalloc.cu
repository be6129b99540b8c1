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
#include <mutex>

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

__device__ __forceinline__ int na_bonds(uint32_t a, uint32_t b, uint32_t valid, int nv) {
  return nv - 2 * __popc((a ^ b) & valid);
}

// First pass: block (layer kx, chunk c) sums m and the +x/+y/+z bonds of its
// rows into part[2 * (kx * bpl + c) + {0, 1}].
__global__ void __launch_bounds__(kNaBlock)
na_partial_kernel(const __grid_constant__ FilmDesc F, const uint32_t* __restrict__ spins,
                  int64_t* __restrict__ part) {
  __shared__ int64_t s_red[kNaBlock / 32];
  const uint32_t Lx = F.Lx, Ly = F.Ly, W = F.W, Wp = F.Wp, bpl = F.meas_bpl;
  const uint32_t kxm1 = blockIdx.x / bpl, chunk = blockIdx.x % bpl;
  const uint32_t* A = spins;
  const uint32_t* B = A + (size_t)Lx * Ly * Wp;
  const bool neg = F.y_mode != kYPbc;
  const uint32_t gkx = (F.y_mode == kYGapbc) ? (Lx - 1 - kxm1) : kxm1;
  int64_t msum = 0, bsum = 0;
  for (uint32_t it = chunk * blockDim.x + threadIdx.x; it < Ly * W; it += bpl * blockDim.x) {
    const uint32_t kym1 = it / W, w = it % W;
    const uint32_t row = kxm1 * Ly + kym1;
    const size_t base = (size_t)row * Wp + w;
    const bool last = (w + 1 == W);
    const uint32_t valid = last ? F.last_mask : 0xFFFFFFFFu;
    const int nv = __popc(valid);
    const uint32_t a = A[base], b = B[base];
    const int m = 2 * (__popc(a & valid) + __popc(b & valid)) - 2 * nv;
    int bb = 0;
    if (kxm1 + 1 < Lx) {
      const size_t nb = base + (size_t)Ly * Wp;
      bb += na_bonds(a, A[nb], valid, nv) + na_bonds(b, B[nb], valid, nv);
    } else if (F.x_pbc) {
      const size_t nb = base - (size_t)(Lx - 1) * Ly * Wp;
      bb += na_bonds(a, A[nb], valid, nv) + na_bonds(b, B[nb], valid, nv);
    }
    if (kym1 + 1 < Ly) {
      bb += na_bonds(a, A[base + Wp], valid, nv) + na_bonds(b, B[base + Wp], valid, nv);
    } else {
      const size_t g = ((size_t)gkx * Ly) * Wp + w;
      const int y = na_bonds(a, A[g], valid, nv) + na_bonds(b, B[g], valid, nv);
      bb += neg ? -y : y;
    }
    bb += na_bonds(a, b, valid, nv);
    const size_t rbase = (size_t)row * Wp;
    uint32_t an = shift_next(a, last ? A[rbase] : A[base + 1]);
    if (last && F.last_mask != 0xFFFFFFFFu) an |= (A[rbase] & 1u) << bitpos((F.n - 1) & 31u);
    bb += na_bonds(b, an, valid, nv);
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

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
int64_t* g_na_ptr[kMaxDevices] = {};

int noalloc_scratch(int64_t** out) {
  int dev = 0;
  ISG_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ISING_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(ISING_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_na_ptr[dev] = static_cast<int64_t*>(p);
  }
  *out = g_na_ptr[dev];
  return ISING_OK;
}

}  // namespace
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
