// Device-side definitions shared by the Ising-film kernels (sm_103a).
//
// Lattice store.  A film Lx x Ly x Lz has Lx*Ly rows (kx,ky), row index
// (kx-1)*Ly + (ky-1).  Each row is split by the parity X = z0 & 1 of
// z0 = kz-1 into two arrays of n = Lz/2 sites, site j of array X being
// z0 = 2j + X.  An array is W = ceil(n/32) 32-bit words, stored with a row
// stride of Wp = W words (no padding: every kernel moves single words).  The
// film's words are laid out [X][row][w] (one "plane" per parity, rows
// contiguous, z fastest).
// Inside a word, local site l (0..31) sits at bit (l >> 2) + 8*(l & 3), so the
// four sites l = 4q..4q+3 served by one Philox call occupy bit q of each of
// the four bytes.  Bit = 1 means S = +1.  Padding bits (j >= n) stay 0.
//
// Checkerboard (Appendix) with colour c = (kx+ky+kz) mod 2: in half-sweep c a
// row (kx,ky) updates array X = (kx + ky + 1 + c) & 1 and reads the same array
// of its x/y neighbour rows (which update the other array) and both
// z-neighbours from its own other array.
#pragma once
#include <cstdint>

namespace isg {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u;
constexpr uint32_t kWeyl1 = 0xBB67AE85u;
constexpr uint32_t kInitSweep = 0xFFFFFFFFu;

enum : uint32_t { kYGapbc = 0, kYPbc = 1, kYApbc = 2 };

// One film of a launch.  Lives in device memory; counters `sweep` and
// `rec_next` are advanced by kernels so that captured graphs can be replayed.
struct FilmDesc {
  uint32_t Lx, Ly, Lz, n, W;   // n = Lz/2 sites per array, W words per array
  uint32_t Wp, nq;             // row stride in words (= W), nq = ceil(Wp / 4)
  uint32_t y_mode, x_pbc;
  uint32_t key0, key1;         // Philox key
  uint32_t last_mask;          // valid bits of word W-1
  uint32_t last_calls;         // Philox calls needed by word W-1 (1..8)
  uint32_t upd_block_begin;    // first block of this film in the update grid
  uint32_t upd_items;          // Lx*(Ly-1)*W (one item = one word of a row)
  uint32_t meas_block_begin;   // first block in the measurement grid
  uint32_t meas_bpl;           // measurement blocks per layer
  uint32_t measure_every;      // 0 = never
  uint32_t sweep;              // absolute index of chunk sweep 0
  uint32_t sweep_end;          // the film stops before this sweep index
  uint32_t rec_next;           // records written so far
  uint32_t rec_cap;            // ring capacity (records)
  uint32_t active;             // 0 = skip this film
  uint64_t spin_off;           // word offset of plane X=0 in the spin pool
  uint64_t rec_off;            // int64 offset of the record ring
  uint64_t part_off;           // int64 offset of this film's partial sums
  uint32_t divw_m, divw_l;     // n / W = (umulhi(n, m) + n) >> l  (n < 2^31)
  uint32_t divy_m, divy_l;     // the same for Ly - 2 (for 1 when Ly = 2)
  uint32_t thr[4][16];         // Metropolis thresholds [class][s + 2*n_aligned]
  uint32_t always[4];          // bit (s + 2*n_aligned): accept without a draw
  uint32_t has_never;          // some reachable entry has dE > 0 and thr = 0
  uint32_t meas_lpu;           // layers per measurement block (> 1 only when meas_bpl = 1)
  uint32_t rk0[10], rk1[10];   // Philox round keys: key + r * Weyl constant
  uint32_t pack;               // rows per packed word in the one- and two-word grid kernels (1, 2, 4)
  uint32_t pk_items;           // their items when pack > 1: Lx * (Ly / pack - 1) groups of pack rows
  uint32_t pk_divm, pk_divl;   // division by Ly / pack - 2 (by 1 when that is 0)
};

// Division by a runtime constant d < 2^31 for numerators n < 2^31 (round-up
// multiplier: l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1).
inline void fastdiv_magic(uint32_t d, uint32_t* m, uint32_t* l) {
  uint32_t k = 0;
  while ((1ull << k) < d) k++;
  *l = k;
  *m = (uint32_t)(((1ull << 32) * ((1ull << k) - d)) / d + 1);
}

// Work sizes of a launch, read by the kernels from device memory so that a
// captured chunk can be replayed while films come and go.
struct LaunchHdr {
  uint32_t n_films;
  uint32_t upd_blocks;   // virtual update blocks (owner table length)
  uint32_t meas_blocks;  // virtual measurement blocks
  uint32_t pad;
};

// Row class of layer kx: 0 bulk, 1 first layer, 2 last layer, 3 both (Lx=1).
__host__ __device__ inline uint32_t row_class(uint32_t kx, uint32_t Lx) {
  return (kx == 1 ? 1u : 0u) | (kx == Lx ? 2u : 0u);
}

// Bit position of local site l inside its word.
__host__ __device__ inline uint32_t bitpos(uint32_t l) { return (l >> 2) + 8u * (l & 3u); }

#ifdef __CUDACC__

__device__ __forceinline__ uint32_t mulhi(uint32_t a, uint32_t b) { return __umulhi(a, b); }

__device__ __forceinline__ uint32_t fastdiv(uint32_t n, uint32_t m, uint32_t l) { return (__umulhi(n, m) + n) >> l; }

// Philox4x32-10 (Salmon et al., SC'11) for counter (c0,c1,c2,c3), key (k0,k1).
__device__ __forceinline__ void philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                         uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    uint32_t lo0 = kPhiloxM0 * c0, hi0 = mulhi(kPhiloxM0, c0);
    uint32_t lo1 = kPhiloxM1 * c2, hi1 = mulhi(kPhiloxM1, c2);
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += kWeyl0;
    k1 += kWeyl1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Philox calls that share the row, sweep and parity words of the counter:
// the first round and half of the second depend only on those, so they are
// computed once per row and reused for the calls of a word.  rk0/rk1 are the
// round keys (key + r * Weyl constant, r = 0..9).
struct PhiloxRow {
  uint32_t r1_hi1, r1_c3, r2_c0, r2_c1;
  uint32_t r1_x2;
  const uint32_t* rk0;
  const uint32_t* rk1;
  __device__ __forceinline__ PhiloxRow(uint32_t row, uint32_t sweep, uint32_t parity, const uint32_t* k0,
                                       const uint32_t* k1)
      : rk0(k0), rk1(k1) {
    // round 1 with counter (row, c1, sweep, parity): words 1..3 of the result
    // do not depend on c1.
    const uint64_t p0 = (uint64_t)kPhiloxM0 * row, p1 = (uint64_t)kPhiloxM1 * sweep;
    r1_hi1 = (uint32_t)(p1 >> 32);  // x0 = hi1 ^ c1 ^ k0
    const uint32_t x1 = (uint32_t)p1;
    r1_x2 = (uint32_t)(p0 >> 32) ^ parity ^ rk1[0];
    r1_c3 = (uint32_t)p0;
    // round 2: the products of x2 are c1-independent
    const uint64_t q1 = (uint64_t)kPhiloxM1 * r1_x2;
    r2_c0 = (uint32_t)(q1 >> 32) ^ x1 ^ rk0[1];
    r2_c1 = (uint32_t)q1;
  }
  // Full Philox4x32-10 output for counter word 1 = c1.
  __device__ __forceinline__ void draw(uint32_t c1, uint32_t out[4]) const {
    const uint32_t x0 = r1_hi1 ^ c1 ^ rk0[0];  // end of round 1 (x1 = lo1, x2 = r1_x2, x3 = r1_c3)
    const uint64_t pp = (uint64_t)kPhiloxM0 * x0;
    uint32_t c0 = r2_c0, c1w = r2_c1, c2 = (uint32_t)(pp >> 32) ^ r1_c3 ^ rk1[1], c3 = (uint32_t)pp;
#pragma unroll
    for (int r = 2; r < 10; r++) {
      const uint64_t p0 = (uint64_t)kPhiloxM0 * c0, p1 = (uint64_t)kPhiloxM1 * c2;
      c0 = (uint32_t)(p1 >> 32) ^ c1w ^ rk0[r];
      c1w = (uint32_t)p1;
      c2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
      c3 = (uint32_t)p0;
    }
    out[0] = c0; out[1] = c1w; out[2] = c2; out[3] = c3;
  }
  // Two Philox calls (counter words 1 = c1a and c1b) computed side by side.
  __device__ __forceinline__ void draw2(uint32_t c1a, uint32_t c1b, uint32_t oa[4], uint32_t ob[4]) const {
    const uint32_t xa = r1_hi1 ^ c1a ^ rk0[0], xb = r1_hi1 ^ c1b ^ rk0[0];
    const uint64_t pa = (uint64_t)kPhiloxM0 * xa, pb = (uint64_t)kPhiloxM0 * xb;
    uint32_t a0 = r2_c0, a1 = r2_c1, a2 = (uint32_t)(pa >> 32) ^ r1_c3 ^ rk1[1], a3 = (uint32_t)pa;
    uint32_t b0 = r2_c0, b1 = r2_c1, b2 = (uint32_t)(pb >> 32) ^ r1_c3 ^ rk1[1], b3 = (uint32_t)pb;
#pragma unroll
    for (int r = 2; r < 10; r++) {
      const uint64_t pa0 = (uint64_t)kPhiloxM0 * a0, pa1 = (uint64_t)kPhiloxM1 * a2;
      const uint64_t pb0 = (uint64_t)kPhiloxM0 * b0, pb1 = (uint64_t)kPhiloxM1 * b2;
      a0 = (uint32_t)(pa1 >> 32) ^ a1 ^ rk0[r];
      a1 = (uint32_t)pa1;
      a2 = (uint32_t)(pa0 >> 32) ^ a3 ^ rk1[r];
      a3 = (uint32_t)pa0;
      b0 = (uint32_t)(pb1 >> 32) ^ b1 ^ rk0[r];
      b1 = (uint32_t)pb1;
      b2 = (uint32_t)(pb0 >> 32) ^ b3 ^ rk1[r];
      b3 = (uint32_t)pb0;
    }
    oa[0] = a0; oa[1] = a1; oa[2] = a2; oa[3] = a3;
    ob[0] = b0; ob[1] = b1; ob[2] = b2; ob[3] = b3;
  }
};

// The same calls with one more product hoisted: round 2's word 0 does not
// depend on c1 either, so neither does round 3's product of it.  Each call
// then starts at round 2 with one product there and one in round 3 (16 wide
// multiplies per call instead of 17).  It keeps two more words live across
// the calls, which the single-film kernel has room for.
struct PhiloxRow3 {
  uint32_t r1_hi1, r1_c3;  // round 1: hi(M1 * sweep) (x0 before the c1 and key xor), x3
  uint32_t r2_c1;          // round 2: y1
  uint32_t r3_x2, r3_c3;   // round 3: hi(M0 * y0) ^ key (z2 before the y3 xor), z3
  const uint32_t* rk0;
  const uint32_t* rk1;
  __device__ __forceinline__ PhiloxRow3(uint32_t row, uint32_t sweep, uint32_t parity, const uint32_t* k0,
                                       const uint32_t* k1)
      : rk0(k0), rk1(k1) {
    // round 1 with counter (row, c1, sweep, parity)
    const uint64_t p0 = (uint64_t)kPhiloxM0 * row, p1 = (uint64_t)kPhiloxM1 * sweep;
    r1_hi1 = (uint32_t)(p1 >> 32);
    const uint32_t x1 = (uint32_t)p1;
    const uint32_t x2 = (uint32_t)(p0 >> 32) ^ parity ^ rk1[0];
    r1_c3 = (uint32_t)p0;
    // round 2: word 0 and word 1 come from the product of x2
    const uint64_t q1 = (uint64_t)kPhiloxM1 * x2;
    const uint32_t y0 = (uint32_t)(q1 >> 32) ^ x1 ^ rk0[1];
    r2_c1 = (uint32_t)q1;
    // round 3: the product of y0
    const uint64_t q0 = (uint64_t)kPhiloxM0 * y0;
    r3_x2 = (uint32_t)(q0 >> 32) ^ rk1[2];
    r3_c3 = (uint32_t)q0;
  }
  // Rounds 2 and 3 of the call with counter word 1 = c1: (z0, z1, z2, z3).
  __device__ __forceinline__ void head(uint32_t c1, uint32_t& z0, uint32_t& z1, uint32_t& z2, uint32_t& z3) const {
    const uint32_t x0 = r1_hi1 ^ c1 ^ rk0[0];  // end of round 1
    const uint64_t pp = (uint64_t)kPhiloxM0 * x0;
    const uint32_t y2 = (uint32_t)(pp >> 32) ^ r1_c3 ^ rk1[1], y3 = (uint32_t)pp;
    const uint64_t qq = (uint64_t)kPhiloxM1 * y2;
    z0 = (uint32_t)(qq >> 32) ^ r2_c1 ^ rk0[2];
    z1 = (uint32_t)qq;
    z2 = r3_x2 ^ y3;
    z3 = r3_c3;
  }
  // Full Philox4x32-10 output for counter word 1 = c1.
  __device__ __forceinline__ void draw(uint32_t c1, uint32_t out[4]) const {
    uint32_t c0, c1w, c2, c3;
    head(c1, c0, c1w, c2, c3);
#pragma unroll
    for (int r = 3; r < 10; r++) {
      const uint64_t p0 = (uint64_t)kPhiloxM0 * c0, p1 = (uint64_t)kPhiloxM1 * c2;
      c0 = (uint32_t)(p1 >> 32) ^ c1w ^ rk0[r];
      c1w = (uint32_t)p1;
      c2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
      c3 = (uint32_t)p0;
    }
    out[0] = c0; out[1] = c1w; out[2] = c2; out[3] = c3;
  }
  // Two Philox calls (counter words 1 = c1a and c1b) computed side by side.
  __device__ __forceinline__ void draw2(uint32_t c1a, uint32_t c1b, uint32_t oa[4], uint32_t ob[4]) const {
    uint32_t a0, a1, a2, a3, b0, b1, b2, b3;
    head(c1a, a0, a1, a2, a3);
    head(c1b, b0, b1, b2, b3);
#pragma unroll
    for (int r = 3; r < 10; r++) {
      const uint64_t pa0 = (uint64_t)kPhiloxM0 * a0, pa1 = (uint64_t)kPhiloxM1 * a2;
      const uint64_t pb0 = (uint64_t)kPhiloxM0 * b0, pb1 = (uint64_t)kPhiloxM1 * b2;
      a0 = (uint32_t)(pa1 >> 32) ^ a1 ^ rk0[r];
      a1 = (uint32_t)pa1;
      a2 = (uint32_t)(pa0 >> 32) ^ a3 ^ rk1[r];
      a3 = (uint32_t)pa0;
      b0 = (uint32_t)(pb1 >> 32) ^ b1 ^ rk0[r];
      b1 = (uint32_t)pb1;
      b2 = (uint32_t)(pb0 >> 32) ^ b3 ^ rk1[r];
      b3 = (uint32_t)pb0;
    }
    oa[0] = a0; oa[1] = a1; oa[2] = a2; oa[3] = a3;
    ob[0] = b0; ob[1] = b1; ob[2] = b2; ob[3] = b3;
  }
};

// Word whose local site l holds site l-1 of the array (z-1 neighbour of
// parity-0 sites), `prev` being the word before (its bit 31 = local site 31).
__device__ __forceinline__ uint32_t shift_prev(uint32_t v, uint32_t prev) {
  return (v << 8) | ((v >> 23) & 0xFEu) | (prev >> 31);
}
// Word whose local site l holds site l+1 (z+1 neighbour of parity-1 sites).
__device__ __forceinline__ uint32_t shift_next(uint32_t v, uint32_t next) {
  return (v >> 8) | ((v << 23) & 0x7F000000u) | (next << 31);
}

// Sum of S_i S_j over the valid sites of two words (nv = popc(valid)).
__device__ __forceinline__ int word_bonds(uint32_t a, uint32_t b, uint32_t valid, int nv) {
  return nv - 2 * __popc((a ^ b) & valid);
}

// Record contributions (Eqs. 1, 17) of word w of row (kxm1, kym1) (0-based)
// of the planes A (z0 even) and B (z0 odd) with row stride Wp: the
// magnetisation of its sites and their +x, +y (Eq. 11 wrap: partner row, sign
// -1 unless PBC) and +z bonds, so that summing over all words counts every
// bond once.  ld(plane, index, limit, site id) loads one word; the kernels'
// checked builds test the index there.
template <class Load>
__device__ __forceinline__ void measure_word(Load ld, const uint32_t* A, const uint32_t* B, uint32_t Wp, uint32_t Lx,
                                             uint32_t Ly, uint32_t W, uint32_t n, uint32_t last_mask, uint32_t x_pbc,
                                             uint32_t y_mode, uint32_t kxm1, uint32_t kym1, uint32_t w, int& m,
                                             int& bb) {
  const uint32_t row = kxm1 * Ly + kym1;
  const size_t base = (size_t)row * Wp + w;
  const size_t lim = (size_t)Lx * Ly * Wp;
  const bool last = (w + 1 == W);
  const uint32_t valid = last ? last_mask : 0xFFFFFFFFu;
  const int nv = __popc(valid);
  const uint32_t a = ld(A, base, lim, 21), b = ld(B, base, lim, 22);
  m = 2 * (__popc(a & valid) + __popc(b & valid)) - 2 * nv;
  bb = 0;
  // +x bond
  if (kxm1 + 1 < Lx) {
    const size_t nb = base + (size_t)Ly * Wp;
    bb += word_bonds(a, ld(A, nb, lim, 23), valid, nv) + word_bonds(b, ld(B, nb, lim, 24), valid, nv);
  } else if (x_pbc) {
    const size_t nb = base - (size_t)(Lx - 1) * Ly * Wp;
    bb += word_bonds(a, ld(A, nb, lim, 25), valid, nv) + word_bonds(b, ld(B, nb, lim, 26), valid, nv);
  }
  // +y bond
  if (kym1 + 1 < Ly) {
    bb += word_bonds(a, ld(A, base + Wp, lim, 27), valid, nv) + word_bonds(b, ld(B, base + Wp, lim, 28), valid, nv);
  } else {
    const uint32_t gkx = (y_mode == kYGapbc) ? (Lx - 1 - kxm1) : kxm1;
    const size_t g = ((size_t)gkx * Ly) * Wp + w;
    const int y = word_bonds(a, ld(A, g, lim, 29), valid, nv) + word_bonds(b, ld(B, g, lim, 30), valid, nv);
    bb += (y_mode != kYPbc) ? -y : y;
  }
  // +z bonds: (2j, 2j+1) inside the word pair, (2j+1, 2j+2) through a shift
  bb += word_bonds(a, b, valid, nv);
  const size_t rbase = (size_t)row * Wp;
  uint32_t an = shift_next(a, last ? ld(A, rbase, lim, 31) : ld(A, base + 1, lim, 32));
  if (last && last_mask != 0xFFFFFFFFu) an |= (ld(A, rbase, lim, 33) & 1u) << bitpos((n - 1) & 31u);
  bb += word_bonds(b, an, valid, nv);
}

#endif  // __CUDACC__

}  // namespace isg
