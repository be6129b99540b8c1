// CUDA kernels of the Ising-film sweep for sm_103a.
//
//  - update_kernel: one half-sweep (colour c) of every film of a launch.  The
//    four phases of a sweep (Appendix checkerboard, split by the Eq. 11 wrap
//    rows) run as two launches: a thread updates one word of row (kx, ky<Ly)
//    and, when ky = 1, then the word of row (kx', Ly) whose wrap neighbour is
//    (kx, 1) -- kx' = Lx+1-kx for the Eq. 11 rule, kx' = kx otherwise.  That
//    row depends on nothing else updated in the half-sweep, so the thread-local
//    order reproduces "all of {c, ky<Ly}, then all of {c, ky=Ly}" exactly.
//  - measure_partial_kernel / measure_finalize_kernel: the int64 sums B, M,
//    M1, Mn and m(kx) of Eqs. 1, 7, 9, 17 and 19, per-block partials in a
//    scratch area, then one block per film writes the record.
//  - init_kernel, pack_kernel, unpack_kernel, advance_kernel.
#include <cuda_runtime.h>

#include "ising_device.cuh"
#include "ising_launch.h"

namespace isg {

namespace {

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (c & (a ^ b));
}

// Per-launch constants of one film, kept in registers.
struct FilmCtx {
  uint32_t* plane0;
  uint32_t* plane1;
  uint32_t Lx, Ly, n, W, y_mode, x_pbc, key0, key1, last_mask, last_calls;
  uint32_t colour, sweep;
};

// Update word w of row (kx, ky): Metropolis decisions for its up to 32 sites.
__device__ __forceinline__ void update_word(const FilmCtx& c, uint32_t kx, uint32_t ky, uint32_t w,
                                            const uint32_t* __restrict__ s_thr,
                                            const uint32_t* __restrict__ s_alw) {
  const uint32_t Lx = c.Lx, Ly = c.Ly, W = c.W;
  const uint32_t row = (kx - 1) * Ly + (ky - 1);
  const uint32_t X = (kx + ky + 1 + c.colour) & 1u;
  uint32_t* __restrict__ P = X ? c.plane1 : c.plane0;
  const uint32_t* __restrict__ Q = X ? c.plane0 : c.plane1;
  const size_t rowW = (size_t)W;
  const size_t base = (size_t)row * rowW + w;
  const uint32_t S = P[base];

  // x neighbours (free surfaces: an empty slot counts as not aligned)
  uint32_t a0, a1, a2, a3, a4, a5;
  if (kx > 1) a0 = ~(S ^ P[base - (size_t)Ly * rowW]);
  else a0 = c.x_pbc ? ~(S ^ P[base + (size_t)(Lx - 1) * Ly * rowW]) : 0u;
  if (kx < Lx) a1 = ~(S ^ P[base + (size_t)Ly * rowW]);
  else a1 = c.x_pbc ? ~(S ^ P[base - (size_t)(Lx - 1) * Ly * rowW]) : 0u;
  // y neighbours; the wrap rows follow Eq. 11 (reflected layer, sign reversed)
  const bool neg = c.y_mode != kYPbc;
  const uint32_t gkx = (c.y_mode == kYGapbc) ? (Lx - kx) : (kx - 1);  // 0-based layer of the wrap row
  if (ky > 1) {
    a2 = ~(S ^ P[base - rowW]);
  } else {
    uint32_t N = P[((size_t)gkx * Ly + (Ly - 1)) * rowW + w];
    a2 = neg ? (S ^ N) : ~(S ^ N);
  }
  if (ky < Ly) {
    a3 = ~(S ^ P[base + rowW]);
  } else {
    uint32_t N = P[((size_t)gkx * Ly) * rowW + w];
    a3 = neg ? (S ^ N) : ~(S ^ N);
  }
  // z neighbours from the other parity of the same row (periodic in z)
  const size_t rbase = (size_t)row * rowW;
  const uint32_t Z0 = Q[base];
  uint32_t Zs;
  if (X == 0) {
    uint32_t pw;
    if (w > 0) {
      pw = Q[base - 1];
    } else {
      const uint32_t lastw = Q[rbase + W - 1];
      pw = ((lastw >> bitpos((c.n - 1) & 31u)) & 1u) << 31;
    }
    Zs = shift_prev(Z0, pw);
  } else {
    const uint32_t nw = (w + 1 < W) ? Q[base + 1] : Q[rbase];
    Zs = shift_next(Z0, nw);
    if (w + 1 == W && c.last_mask != 0xFFFFFFFFu) {
      const uint32_t r = (c.n - 1) & 31u;  // last valid local site of the last word
      Zs |= (Q[rbase] & 1u) << bitpos(r);
    }
  }
  a4 = ~(S ^ Z0);
  a5 = ~(S ^ Zs);

  // bit-sliced count of aligned neighbours: n = c0 + 2 c1 + 4 c2
  const uint32_t s1 = a0 ^ a1 ^ a2, k1 = maj3(a0, a1, a2);
  const uint32_t s2 = a3 ^ a4 ^ a5, k2 = maj3(a3, a4, a5);
  const uint32_t c0 = s1 ^ s2, k3 = s1 & s2;
  const uint32_t c1 = k1 ^ k2 ^ k3, c2 = maj3(k1, k2, k3);

  const uint32_t cls = row_class(kx, Lx);
  // "always accept" (dE <= 0) as a 4-input function of (S, c0, c1, c2)
  const uint32_t* m = s_alw + cls * 16;
  uint32_t v0 = (S & m[1]) | (~S & m[0]);
  uint32_t v1 = (S & m[3]) | (~S & m[2]);
  uint32_t v2 = (S & m[5]) | (~S & m[4]);
  uint32_t v3 = (S & m[7]) | (~S & m[6]);
  uint32_t v4 = (S & m[9]) | (~S & m[8]);
  uint32_t v5 = (S & m[11]) | (~S & m[10]);
  uint32_t v6 = (S & m[13]) | (~S & m[12]);
  uint32_t v7 = (S & m[15]) | (~S & m[14]);
  uint32_t w0 = (c0 & v1) | (~c0 & v0);
  uint32_t w1 = (c0 & v3) | (~c0 & v2);
  uint32_t w2 = (c0 & v5) | (~c0 & v4);
  uint32_t w3 = (c0 & v7) | (~c0 & v6);
  uint32_t x0 = (c1 & w1) | (~c1 & w0);
  uint32_t x1 = (c1 & w3) | (~c1 & w2);
  const uint32_t alw = (c2 & x1) | (~c2 & x0);

  // transpose the planes (S, c0, c1, c2) into nibbles: nibble r of U[a] holds
  // the 4-bit table index S + 2*n of bit position 4r + a
  const uint32_t T0 = (S & 0x55555555u) | ((c0 & 0x55555555u) << 1);
  const uint32_t T1 = ((S >> 1) & 0x55555555u) | (c0 & 0xAAAAAAAAu);
  const uint32_t T2 = (c1 & 0x55555555u) | ((c2 & 0x55555555u) << 1);
  const uint32_t T3 = ((c1 >> 1) & 0x55555555u) | (c2 & 0xAAAAAAAAu);
  uint32_t U[4];
  U[0] = (T0 & 0x33333333u) | ((T2 & 0x33333333u) << 2);
  U[1] = (T1 & 0x33333333u) | ((T3 & 0x33333333u) << 2);
  U[2] = ((T0 >> 2) & 0x33333333u) | (T2 & 0xCCCCCCCCu);
  U[3] = ((T1 >> 2) & 0x33333333u) | (T3 & 0xCCCCCCCCu);

  const bool last = (w + 1 == W);
  const uint32_t ncalls = last ? c.last_calls : 8u;
  const uint32_t valid = last ? c.last_mask : 0xFFFFFFFFu;
  const uint32_t clsb = (cls * 64u) * 0x01010101u;  // byte offset of this class's table
  const char* tb = reinterpret_cast<const char*>(s_thr);
  const PhiloxRow pr(row, c.sweep, X, c.key0, c.key1);
  uint32_t lt = 0;
#pragma unroll
  for (uint32_t q = 0; q < 8; q++) {
    if (q < ncalls) {
      uint32_t u[4];
      pr.draw(8u * w + q, u);
      const uint32_t Y = (q < 4 ? ((U[q & 3] << 2) & 0x3C3C3C3Cu) : ((U[q & 3] >> 2) & 0x3C3C3C3Cu)) | clsb;
#pragma unroll
      for (uint32_t i = 0; i < 4; i++) {
        const uint32_t off = (Y >> (8 * i)) & 0xFFu;
        const uint32_t t = *reinterpret_cast<const uint32_t*>(tb + off);
        if (u[i] < t) lt |= 1u << (q + 8 * i);
      }
    }
  }
  const uint32_t flip = (lt | alw) & valid;
  P[base] = S ^ flip;
}

}  // namespace

__global__ void __launch_bounds__(kUpdateBlock)
update_kernel(const FilmDesc* __restrict__ films, const uint32_t* __restrict__ owner,
              const LaunchHdr* __restrict__ hdr, uint32_t* __restrict__ pool, uint32_t colour, uint32_t k) {
  __shared__ uint32_t s_thr[64];
  __shared__ uint32_t s_alw[64];
  const uint32_t nvb = hdr->upd_blocks;
  uint32_t cur = 0xFFFFFFFFu;
  for (uint32_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const uint32_t f = owner[vb];  // the same for every thread of the block
    const FilmDesc& F = films[f];
    if (f != cur) {
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) {
        s_thr[i] = F.thr[i >> 4][i & 15];
        s_alw[i] = ((F.always[i >> 4] >> (i & 15)) & 1u) ? 0xFFFFFFFFu : 0u;
      }
      __syncthreads();
      cur = f;
    }
    if (!F.active || F.sweep + k >= F.sweep_end) continue;
    const uint32_t item = (vb - F.upd_block_begin) * blockDim.x + threadIdx.x;
    if (item >= F.upd_items) continue;
    FilmCtx c;
    c.Lx = F.Lx; c.Ly = F.Ly; c.n = F.n; c.W = F.W;
    c.y_mode = F.y_mode; c.x_pbc = F.x_pbc; c.key0 = F.key0; c.key1 = F.key1;
    c.last_mask = F.last_mask; c.last_calls = F.last_calls;
    c.colour = colour; c.sweep = F.sweep + k;
    c.plane0 = pool + F.spin_off;
    c.plane1 = c.plane0 + (size_t)F.Lx * F.Ly * F.W;
    const uint32_t w = item % c.W;
    const uint32_t rp = item / c.W;
    const uint32_t kx = rp / (c.Ly - 1) + 1;
    const uint32_t ky = rp % (c.Ly - 1) + 1;
    update_word(c, kx, ky, w, s_thr, s_alw);
    if (ky == 1) {
      const uint32_t kx2 = (c.y_mode == kYGapbc) ? (c.Lx + 1 - kx) : kx;
      update_word(c, kx2, c.Ly, w, s_thr, s_alw);
    }
  }
}

// ------------------------------------------------------------ measurement

namespace {

__device__ __forceinline__ int64_t block_sum(int64_t v, int64_t* s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  int64_t t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += s_red[i];
  __syncthreads();
  return t;  // valid in thread 0
}

__device__ __forceinline__ int bonds(uint32_t a, uint32_t b, uint32_t valid, int nv) {
  return nv - 2 * __popc((a ^ b) & valid);
}

__device__ __forceinline__ bool measured_now(const FilmDesc& F, uint32_t done, int force) {
  if (force) return true;
  if (F.measure_every == 0 || done == 0 || F.sweep_end - F.sweep < done) return false;
  return ((F.sweep + done) % F.measure_every) == 0;
}

}  // namespace

__global__ void __launch_bounds__(kMeasureBlock)
measure_partial_kernel(const FilmDesc* __restrict__ films, const uint32_t* __restrict__ owner,
                       const LaunchHdr* __restrict__ hdr, const uint32_t* __restrict__ pool,
                       int64_t* __restrict__ part, uint32_t done, int force) {
  __shared__ int64_t s_red[kMeasureBlock / 32];
  const uint32_t nvb = hdr->meas_blocks;
  for (uint32_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const FilmDesc& F = films[owner[vb]];
    if (!F.active || !measured_now(F, done, force)) continue;
    const uint32_t Lx = F.Lx, Ly = F.Ly, W = F.W, bpl = F.meas_bpl;
    const uint32_t local = vb - F.meas_block_begin;
    const uint32_t kxm1 = local / bpl, chunk = local % bpl;
    const uint32_t* A = pool + F.spin_off;
    const uint32_t* B = A + (size_t)Lx * Ly * W;
    const bool neg = F.y_mode != kYPbc;
    const uint32_t gkx = (F.y_mode == kYGapbc) ? (Lx - 1 - kxm1) : kxm1;
    int64_t msum = 0, bsum = 0;
    for (uint32_t it = chunk * blockDim.x + threadIdx.x; it < Ly * W; it += bpl * blockDim.x) {
      const uint32_t kym1 = it / W, w = it % W;
      const uint32_t row = kxm1 * Ly + kym1;
      const size_t base = (size_t)row * W + w;
      const bool last = (w + 1 == W);
      const uint32_t valid = last ? F.last_mask : 0xFFFFFFFFu;
      const int nv = __popc(valid);
      const uint32_t a = A[base], b = B[base];
      int m = 2 * (__popc(a & valid) + __popc(b & valid)) - 2 * nv;
      int bb = 0;
      // +x bond
      if (kxm1 + 1 < Lx) {
        const size_t nb = base + (size_t)Ly * W;
        bb += bonds(a, A[nb], valid, nv) + bonds(b, B[nb], valid, nv);
      } else if (F.x_pbc) {
        const size_t nb = base - (size_t)(Lx - 1) * Ly * W;
        bb += bonds(a, A[nb], valid, nv) + bonds(b, B[nb], valid, nv);
      }
      // +y bond (wrap: the Eq. 11 partner row, sign -1 unless PBC)
      if (kym1 + 1 < Ly) {
        bb += bonds(a, A[base + W], valid, nv) + bonds(b, B[base + W], valid, nv);
      } else {
        const size_t g = ((size_t)gkx * Ly) * W + w;
        const int y = bonds(a, A[g], valid, nv) + bonds(b, B[g], valid, nv);
        bb += neg ? -y : y;
      }
      // +z bonds: (2j, 2j+1) inside the word pair, (2j+1, 2j+2) through a shift
      bb += bonds(a, b, valid, nv);
      const size_t rbase = (size_t)row * W;
      uint32_t an = shift_next(a, last ? A[rbase] : A[base + 1]);
      if (last && F.last_mask != 0xFFFFFFFFu) an |= (A[rbase] & 1u) << bitpos((F.n - 1) & 31u);
      bb += bonds(b, an, valid, nv);
      msum += m;
      bsum += bb;
    }
    const int64_t tm = block_sum(msum, s_red);
    const int64_t tb = block_sum(bsum, s_red);
    if (threadIdx.x == 0) {
      int64_t* p = part + F.part_off + 2 * ((size_t)kxm1 * bpl + chunk);
      p[0] = tm;
      p[1] = tb;
    }
  }
}

__global__ void __launch_bounds__(kMeasureBlock)
measure_finalize_kernel(FilmDesc* __restrict__ films, const LaunchHdr* __restrict__ hdr,
                        const int64_t* __restrict__ part, int64_t* __restrict__ records, uint32_t done, int force,
                        int64_t* __restrict__ direct) {
  __shared__ int64_t s_red[kMeasureBlock / 32];
  __shared__ uint32_t s_slot;
  const uint32_t nf = hdr->n_films;
  for (uint32_t f = blockIdx.x; f < nf; f += gridDim.x) {
    FilmDesc& F = films[f];
    if (!F.active || !measured_now(F, done, force)) continue;
    const uint32_t Lx = F.Lx, bpl = F.meas_bpl;
    __syncthreads();
    if (threadIdx.x == 0) s_slot = F.rec_cap ? (F.rec_next % F.rec_cap) : 0u;
    __syncthreads();
    int64_t* rec = direct ? direct : records + F.rec_off + (size_t)s_slot * (5 + Lx);
    const int64_t* p = part + F.part_off;
    int64_t M = 0, Bs = 0;
    for (uint32_t kx = threadIdx.x; kx < Lx; kx += blockDim.x) {
      int64_t m = 0;
      for (uint32_t c = 0; c < bpl; c++) {
        m += p[2 * ((size_t)kx * bpl + c)];
        Bs += p[2 * ((size_t)kx * bpl + c) + 1];
      }
      rec[5 + kx] = m;
      M += m;
    }
    const int64_t tM = block_sum(M, s_red);
    const int64_t tB = block_sum(Bs, s_red);
    if (threadIdx.x == 0) {
      rec[0] = (int64_t)F.sweep + done;
      rec[1] = tB;
      rec[2] = tM;
      rec[3] = rec[5];
      rec[4] = rec[5 + Lx - 1];
      if (!direct) F.rec_next = F.rec_next + 1;
    }
  }
}

__global__ void advance_kernel(FilmDesc* __restrict__ films, const LaunchHdr* __restrict__ hdr, uint32_t n_sweeps) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < hdr->n_films && films[f].active) {
    const uint32_t s = films[f].sweep, e = films[f].sweep_end;
    films[f].sweep = (e - s < n_sweeps) ? e : s + n_sweeps;
  }
}

// ------------------------------------------------------------- set-up

__global__ void init_kernel(FilmDesc F, uint32_t* __restrict__ pool, int kind, uint32_t flip_lo, int flip_all) {
  const size_t words = (size_t)F.Lx * F.Ly * F.W;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * words) return;
  const uint32_t X = (uint32_t)(i / words);
  const size_t rem = i % words;
  const uint32_t row = (uint32_t)(rem / F.W), w = (uint32_t)(rem % F.W);
  const uint32_t ky = row % F.Ly + 1;
  const bool last = (w + 1 == F.W);
  const uint32_t valid = last ? F.last_mask : 0xFFFFFFFFu;
  uint32_t word = 0;
  if (kind == 2) {
    word = 0xFFFFFFFFu;
  } else {
    const bool up_half = ky <= F.Ly / 2;
    for (uint32_t q = 0; q < 8; q++) {
      uint32_t u[4];
      philox10(row, 8u * w + q, kInitSweep, 2u | X, F.key0, F.key1, u);
      for (uint32_t t = 0; t < 4; t++) {
        bool up;
        if (kind == 0) up = u[t] < 0x80000000u;
        else up = up_half != (flip_all || u[t] < flip_lo);
        if (up) word |= 1u << (q + 8 * t);
      }
    }
  }
  pool[F.spin_off + i] = word & valid;
}

// int8 canonical order -> packed planes
__global__ void pack_kernel(FilmDesc F, uint32_t* __restrict__ pool, const int8_t* __restrict__ s) {
  const size_t words = (size_t)F.Lx * F.Ly * F.W;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * words) return;
  const uint32_t X = (uint32_t)(i / words);
  const size_t rem = i % words;
  const size_t row = rem / F.W;
  const uint32_t w = (uint32_t)(rem % F.W);
  uint32_t word = 0;
  for (uint32_t l = 0; l < 32; l++) {
    const uint32_t j = 32u * w + l;
    if (j >= F.n) break;
    const uint32_t z0 = 2u * j + X;
    if (s[row * F.Lz + z0] > 0) word |= 1u << bitpos(l);
  }
  pool[F.spin_off + i] = word;
}

__global__ void unpack_kernel(FilmDesc F, const uint32_t* __restrict__ pool, int8_t* __restrict__ s) {
  const size_t total = (size_t)F.Lx * F.Ly * F.Lz;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const size_t row = i / F.Lz;
  const uint32_t z0 = (uint32_t)(i % F.Lz);
  const uint32_t X = z0 & 1u, j = z0 >> 1;
  const size_t words = (size_t)F.Lx * F.Ly * F.W;
  const uint32_t word = pool[F.spin_off + X * words + row * F.W + (j >> 5)];
  s[i] = ((word >> bitpos(j & 31u)) & 1u) ? (int8_t)1 : (int8_t)-1;
}

// ------------------------------------------------------ host launchers

cudaError_t launch_update(const LaunchSet& L, uint32_t grid, uint32_t* pool, uint32_t colour, uint32_t k,
                          cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  update_kernel<<<grid, kUpdateBlock, 0, st>>>(L.films, L.owner_upd, L.hdr, pool, colour, k);
  return cudaGetLastError();
}

cudaError_t launch_measure(const LaunchSet& L, uint32_t grid, uint32_t fin_grid, const uint32_t* pool,
                           int64_t* part, int64_t* records, uint32_t done, int force, int64_t* direct,
                           cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  measure_partial_kernel<<<grid, kMeasureBlock, 0, st>>>(L.films, L.owner_meas, L.hdr, pool, part, done, force);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  measure_finalize_kernel<<<fin_grid, kMeasureBlock, 0, st>>>(L.films, L.hdr, part, records, done, force, direct);
  return cudaGetLastError();
}

cudaError_t launch_advance(const LaunchSet& L, uint32_t grid, uint32_t n_sweeps, cudaStream_t st) {
  if (grid == 0 || n_sweeps == 0) return cudaSuccess;
  advance_kernel<<<grid, 128, 0, st>>>(L.films, L.hdr, n_sweeps);
  return cudaGetLastError();
}

cudaError_t launch_init(const FilmDesc& f, uint32_t* pool, int kind, uint32_t flip_lo, int flip_all,
                        cudaStream_t st) {
  const size_t n = 2 * (size_t)f.Lx * f.Ly * f.W;
  init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, pool, kind, flip_lo, flip_all);
  return cudaGetLastError();
}

cudaError_t launch_pack(const FilmDesc& f, uint32_t* pool, const int8_t* s, cudaStream_t st) {
  const size_t n = 2 * (size_t)f.Lx * f.Ly * f.W;
  pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, pool, s);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const FilmDesc& f, const uint32_t* pool, int8_t* s, cudaStream_t st) {
  const size_t n = (size_t)f.Lx * f.Ly * f.Lz;
  unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, pool, s);
  return cudaGetLastError();
}

int update_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, update_kernel, kUpdateBlock, 0) != cudaSuccess) return 0;
  return nb;
}

int measure_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, measure_partial_kernel, kMeasureBlock, 0) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace isg
