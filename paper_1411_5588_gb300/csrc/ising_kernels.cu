// CUDA kernels of the Ising-film sweep for sm_103a.
//
//  - update_kernel: one half-sweep (colour c) of every film of a launch.  The
//    four phases of a sweep (Appendix checkerboard, split by the Eq. 11 wrap
//    rows) run as two launches: a thread updates one word of row (kx, ky<Ly)
//    and, when ky = 1, then the word of row (kx', Ly) whose wrap neighbour is
//    (kx, 1) -- kx' = Lx+1-kx for the Eq. 11 rule, kx' = kx otherwise.  That
//    row depends on nothing else updated in the half-sweep, so the thread-local
//    order reproduces "all of {c, ky<Ly}, then all of {c, ky=Ly}" exactly.
//    The half-sweep 1 launch of a sweep after which films record also sums
//    their int64 record quantities B, M, M1, Mn and m(kx) (Eqs. 1, 7, 9, 17,
//    19) from the words it holds in registers, into per-layer accumulators.
//  - record_kernel: writes those records and clears the accumulators.
//  - measure_partial_kernel / measure_finalize_kernel: the same sums from the
//    lattice alone (an on-demand measurement), per-block partials in a
//    scratch area, then one block per film writes the record.
//  - init_kernel, pack_kernel, unpack_kernel, advance_kernel.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "ising_device.cuh"

#include "ising_launch.h"

namespace isg {

namespace cg = cooperative_groups;

namespace {

// Programmatic dependent launch: every kernel of the sweep path lets the next
// launch of its stream start early (its blocks then sit in pdl_wait) and
// waits, before it touches any film state, for the previous grid to complete
// and its writes to be visible.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Checked builds (-DISING_CHECKED) test every lattice word index against its
// plane before the access: an index out of range is counted, the first one
// is kept (site << 48 | index), and the access goes to word 0 instead (a
// store is dropped).  Normal builds compile the checks away.
#ifdef ISING_CHECKED
__device__ unsigned long long g_oob_count;
__device__ unsigned long long g_oob_first;
__device__ __forceinline__ bool oob(uint64_t idx, uint64_t lim, uint32_t site) {
  if (idx < lim) return false;
  atomicAdd(&g_oob_count, 1ull);
  atomicCAS(&g_oob_first, 0ull, ((unsigned long long)site << 48) | (idx & 0xFFFFFFFFFFFFull));
  return true;
}
#define ISG_LD(p, idx, lim, site) ((p)[oob((idx), (lim), (site)) ? 0 : (idx)])
#define ISG_ST(p, idx, lim, site, v) \
  do {                               \
    if (!oob((idx), (lim), (site))) (p)[(idx)] = (v); \
  } while (0)
#else
#define ISG_LD(p, idx, lim, site) ((void)(lim), (p)[(idx)])
#define ISG_ST(p, idx, lim, site, v) ((void)(lim), (p)[(idx)] = (v))
#endif

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (c & (a ^ b));
}

// acc | bit when u <= t: one compare setting a predicate and one predicated OR.
__device__ __forceinline__ void or_if_le(uint32_t& acc, uint32_t u, uint32_t t, uint32_t bit) {
  asm("{\n\t.reg .pred p;\n\tsetp.le.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
      : "+r"(acc) : "r"(u), "r"(t), "r"(bit));
}

// The same with the bit as an immediate operand.
template <uint32_t BIT>
__device__ __forceinline__ void or_if_le_c(uint32_t& acc, uint32_t u, uint32_t t) {
  asm("{\n\t.reg .pred p;\n\tsetp.le.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
      : "+r"(acc) : "r"(u), "r"(t), "n"(BIT));
}
template <uint32_t BIT>
__device__ __forceinline__ void or_if_lt_c(uint32_t& acc, uint32_t u, uint32_t t) {
  asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
      : "+r"(acc) : "r"(u), "r"(t), "n"(BIT));
}

// acc | bit when u < t.
__device__ __forceinline__ void or_if_lt(uint32_t& acc, uint32_t u, uint32_t t, uint32_t bit) {
  asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
      : "+r"(acc) : "r"(u), "r"(t), "r"(bit));
}

// Decisions of the sites at bits Q + 8I (Philox call Q, word u[I]) and
// Q + 4 + 8I (call Q + 4, word v[I]) of a word.
template <bool FAST, uint32_t Q, uint32_t I>
__device__ __forceinline__ void site_pair(uint32_t& lt, const char* tb, uint32_t Y, uint32_t Y2, uint32_t u,
                                          uint32_t v, bool two) {
  uint32_t t, t2;
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(tb);
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t) : "r"(base + __byte_perm(Y, 0, 0x4440 + I)));
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t2) : "r"(base + __byte_perm(Y2, 0, 0x4440 + I)));
  if (FAST) {
    // table word thr - 1, or 0xFFFFFFFF for "always" (dE <= 0)
    or_if_le_c<1u << (Q + 8 * I)>(lt, u, t);
    if (two) or_if_le_c<1u << (Q + 4 + 8 * I)>(lt, v, t2);
  } else {
    or_if_lt_c<1u << (Q + 8 * I)>(lt, u, t);
    if (two) or_if_lt_c<1u << (Q + 4 + 8 * I)>(lt, v, t2);
  }
}

// Decision of the site at bit Q + 8I (Philox call Q, word u).
template <bool FAST, uint32_t Q, uint32_t I>
__device__ __forceinline__ void site_one(uint32_t& lt, const char* tb, uint32_t Y, uint32_t u) {
  uint32_t t;
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(tb);
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t) : "r"(base + __byte_perm(Y, 0, 0x4440 + I)));
  if (FAST) or_if_le_c<1u << (Q + 8 * I)>(lt, u, t);
  else or_if_lt_c<1u << (Q + 8 * I)>(lt, u, t);
}

// Per-launch constants of one film, kept in registers.
struct FilmCtx {
  uint32_t* plane0;
  uint32_t* plane1;
  uint32_t Lx, Ly, n, W, Wp, y_mode, x_pbc, last_mask, last_calls;
  uint32_t plane_words;  // words of one plane (Lx * Ly * Wp), for checked builds
  uint32_t seam_same;    // the y-wrap bonds join sites of one colour (Lx+Ly even under Eq. 11, Ly odd otherwise)
  uint32_t pack;         // rows per packed word (1, 2 or 4) in the grid kernels' items
  // decision path of the film's words (kFull, kPartial, kSingle or kMixed)
  __device__ __forceinline__ uint32_t path() const;
  const uint32_t* rk0;  // Philox round keys (constant bank or shared memory)
  const uint32_t* rk1;
  uint32_t colour, sweep;
};

__host__ __device__ inline uint32_t seam_joins_one_colour(uint32_t Lx, uint32_t Ly, uint32_t y_mode) {
  return y_mode == kYGapbc ? ((Lx + Ly) % 2 == 0) : (Ly % 2 == 1);
}

// Whether film F, at chunk start sweep `sweep`, records after `done` sweeps
// of the chunk.
__device__ __forceinline__ bool records_after(const FilmDesc& F, uint32_t sweep, uint32_t done) {
  if (F.measure_every == 0 || done == 0 || F.sweep_end - sweep < done) return false;
  return ((sweep + done) % F.measure_every) == 0;
}

__device__ __forceinline__ bool measured_now(const FilmDesc& F, uint32_t done, int force) {
  return force || records_after(F, F.sweep, done);
}

// The words one thread needs to update word w of row (kx, ky), loaded ahead
// of the arithmetic so that the loads of the next word overlap the current
// word's Philox draws.
struct Fetched {
  uint32_t S, xm, xp, ym, yp, z0, za, zf;
  uint32_t kx, ky, w;
};

__device__ __forceinline__ void fetch_word(const FilmCtx& c, uint32_t kx, uint32_t ky, uint32_t w, Fetched& f) {
  const uint32_t Lx = c.Lx, Ly = c.Ly, W = c.W, Wp = c.Wp;
  const uint32_t row = (kx - 1) * Ly + (ky - 1);
  const uint32_t X = (kx + ky + 1 + c.colour) & 1u;
  const uint32_t* __restrict__ P = X ? c.plane1 : c.plane0;
  const uint32_t* __restrict__ Q = X ? c.plane0 : c.plane1;
  const uint32_t rbase = row * Wp;  // planes hold < 2^31 words
  const uint32_t base = rbase + w;
  const uint32_t LyWp = Ly * Wp;
  const uint32_t gkx = (c.y_mode == kYGapbc) ? (Lx - kx) : (kx - 1);  // 0-based layer of the wrap row
  f.kx = kx; f.ky = ky; f.w = w;
  const uint32_t lim = c.plane_words;
  f.S = ISG_LD(P, base, lim, 1);
  f.xm = (kx > 1) ? ISG_LD(P, base - LyWp, lim, 2)
                  : (c.x_pbc ? ISG_LD(P, base + (Lx - 1) * LyWp, lim, 3) : 0u);
  f.xp = (kx < Lx) ? ISG_LD(P, base + LyWp, lim, 4)
                   : (c.x_pbc ? ISG_LD(P, base - (Lx - 1) * LyWp, lim, 5) : 0u);
  f.ym = (ky > 1) ? ISG_LD(P, base - Wp, lim, 6) : ISG_LD(P, (gkx * Ly + (Ly - 1)) * Wp + w, lim, 7);
  f.yp = (ky < Ly) ? ISG_LD(P, base + Wp, lim, 8) : ISG_LD(P, gkx * LyWp + w, lim, 9);
  f.z0 = ISG_LD(Q, base, lim, 10);
  if (X == 0)  // previous word, or the row's last
    f.za = (w > 0) ? ISG_LD(Q, base - 1, lim, 11) : ISG_LD(Q, rbase + W - 1, lim, 12);
  else  // next word, or the row's first
    f.za = (w + 1 < W) ? ISG_LD(Q, base + 1, lim, 13) : ISG_LD(Q, rbase, lim, 14);
  f.zf = ISG_LD(Q, rbase, lim, 15);
}

// Metropolis decisions for the up to 32 sites of the fetched word; returns
// the mask of sites that flip.  QUARTER: only Philox calls qsel and qsel + 4
// (the sites at bits qsel and qsel + 4 of each byte), for a word shared by
// four lanes.
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

// The record of film Fg after `done` sweeps of the chunk (chunk-start sweep
// `sweep`), from the per-layer accumulators half-sweep 1 filled, which it
// clears; advances the film's ring counter.  F holds the film's static
// fields (a staged copy or Fg itself).  The whole block calls it; s_red holds
// one int64 per warp.
__device__ __noinline__ void write_record(FilmDesc* Fg, const FilmDesc& F, uint32_t sweep, int64_t* part,
                                             int64_t* records, uint32_t done, int64_t* s_red, uint32_t* s_slot) {
  const uint32_t Lx = F.Lx;
  uint32_t rn = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    rn = __ldcg(&Fg->rec_next);  // written by an earlier kernel
    *s_slot = F.rec_cap ? rn % F.rec_cap : 0u;
  }
  __syncthreads();
  int64_t* rec = records + F.rec_off + (size_t)*s_slot * (5 + Lx);
  int64_t* acc = part + acc_offset(F);
  int64_t M = 0, Bs = 0;
  for (uint32_t kx = threadIdx.x; kx < Lx; kx += blockDim.x) {
    const int64_t m = acc[2 * kx], b = acc[2 * kx + 1];
    acc[2 * kx] = 0;
    acc[2 * kx + 1] = 0;
    rec[5 + kx] = m;
    M += m;
    Bs += b;
  }
  const int64_t tM = block_sum(M, s_red);
  const int64_t tB = block_sum(Bs, s_red);
  if (threadIdx.x == 0) {
    rec[0] = (int64_t)sweep + done;
    rec[1] = tB;
    rec[2] = tM;
    rec[3] = rec[5];
    rec[4] = rec[5 + Lx - 1];
    Fg->rec_next = rn + 1;
  }
}

// Record sums of half-sweep 1.  After its update every neighbour word a
// thread loaded is final -- it holds the other colour -- except the -y word
// of a ky = 1 row when the seam joins one colour: that is its wrap partner,
// which the same thread updates right after it.  So each thread can add up,
// for its word, the magnetisation of the row's two words w and
// sum sigma_b S_i S_j over the bonds from the word's sites to their
// neighbours (an empty x slot is no bond), and every bond of the film is
// counted once; the seam cases are settled in the partner step.
//
// The bonds come from the bit-sliced aligned-neighbour count (c0, c1, c2) of
// the decision: a flip toggles every aligned mask of its site, so over the
// D bond slots of the word
//   sum_d popc(a'_d) = n_old + D popc(fl) - 2 n_fl,
// n_old and n_fl being the aligned counts summed over the valid and over the
// flipped sites.  decide_word parks c0, c1, c2 and the row's other word z0 in
// slots 0-3 of the thread's kStashSlots consecutive shared-memory words
// (thread-major; the odd stride keeps a warp's accesses on distinct banks)
// across the Philox draws, so the sums cost no registers there; slot 4 holds
// a partner word's seam adjustment across its draws.
constexpr uint32_t kStashSlots = 5;

struct LayerSums {
  uint32_t layer = 0xFFFFFFFFu;  // 0-based kx, none when 0xFFFFFFFF
  int m = 0, b = 0;
};

__device__ __forceinline__ void stash_counts(uint32_t* stash, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t z0) {
  stash[0] = c0;
  stash[1] = c1;
  stash[2] = c2;
  stash[3] = z0;
}

// Sums of the word of layer kx (1-based) whose flips were fl and whose new
// value is v, from the counts decide_word parked.
__device__ __forceinline__ LayerSums word_sums(const FilmCtx& c, uint32_t kx, uint32_t w, uint32_t fl, uint32_t v,
                                               const uint32_t* stash) {
  const uint32_t valid = (w + 1 == c.W) ? c.last_mask : 0xFFFFFFFFu;
  const int nv = __popc(valid);
  const uint32_t c0 = stash[0], c1 = stash[1], c2 = stash[2];
  const uint32_t z0 = stash[3];
  const int D = 4 + ((kx > 1 || c.x_pbc) ? 1 : 0) + ((kx < c.Lx || c.x_pbc) ? 1 : 0);
  const int n_old = __popc(c0 & valid) + 2 * __popc(c1 & valid) + 4 * __popc(c2 & valid);
  const int n_fl = __popc(c0 & fl) + 2 * __popc(c1 & fl) + 4 * __popc(c2 & fl);
  LayerSums r;
  r.layer = kx - 1;
  r.b = 2 * (n_old + D * __popc(fl) - 2 * n_fl) - D * nv;
  r.m = 2 * (__popc(v & valid) + __popc(z0 & valid)) - 2 * nv;
  return r;
}

// Seam correction of a ky = 1 word (new value v, other word z0f) and its
// partner word g (just fetched) when the seam joins one colour: the word's
// -y count used the partner's old word, so it comes out again (the partner
// counts that bond from its +y side with both final words), and the seam
// bonds between the two rows' other arrays, which no one else holds, go in.
__device__ __forceinline__ int seam_adjust(const FilmCtx& c, uint32_t w, uint32_t v, uint32_t z0f,
                                           const Fetched& g) {
  const uint32_t valid = (w + 1 == c.W) ? c.last_mask : 0xFFFFFFFFu;
  const int nv = __popc(valid);
  const bool neg = c.y_mode != kYPbc;
  const int stale = 2 * __popc(~(v ^ g.S ^ (neg ? 0xFFFFFFFFu : 0u)) & valid) - nv;
  const int other = nv - 2 * __popc((z0f ^ g.z0) & valid);
  return (neg ? -other : other) - stale;
}

// Adds the sums of every lane that has some into the film's per-layer int64
// accumulators [2 kx (magnetisation), 2 kx + 1 (bonds)].  All 32 lanes call
// it.  The lanes in the first active lane's layer add with two warp
// reductions and two atomics; any other lane adds its own.  Integer atomics
// are exact in any order.
__device__ __forceinline__ void add_layer_sums(unsigned long long* acc, const LayerSums& r) {
  const bool on = r.layer != 0xFFFFFFFFu;
  const uint32_t act = __ballot_sync(0xFFFFFFFFu, on);
  if (act == 0) return;
  const int lead = __ffs(act) - 1;
  const uint32_t l0 = __shfl_sync(0xFFFFFFFFu, r.layer, lead);
  const bool in0 = on && r.layer == l0;
  const int m = __reduce_add_sync(0xFFFFFFFFu, in0 ? r.m : 0);
  const int b = __reduce_add_sync(0xFFFFFFFFu, in0 ? r.b : 0);
  if ((int)(threadIdx.x & 31u) == lead) {
    atomicAdd(acc + 2 * (size_t)l0, (unsigned long long)(long long)m);
    atomicAdd(acc + 2 * (size_t)l0 + 1, (unsigned long long)(long long)b);
  } else if (on && !in0) {
    atomicAdd(acc + 2 * (size_t)r.layer, (unsigned long long)(long long)r.m);
    atomicAdd(acc + 2 * (size_t)r.layer + 1, (unsigned long long)(long long)r.b);
  }
}

// A lane's own sums, without a warp reduction (partner words: a few lanes).
__device__ __forceinline__ void add_lane_sums(unsigned long long* acc, const LayerSums& r) {
  if (r.layer == 0xFFFFFFFFu) return;
  atomicAdd(acc + 2 * (size_t)r.layer, (unsigned long long)(long long)r.m);
  atomicAdd(acc + 2 * (size_t)r.layer + 1, (unsigned long long)(long long)r.b);
}

// The same into a block's shared counters (resident films: int32 suffices
// below 2^16 sites): layer sums s_m[kx], and the totals s_tot = {B, M}.  All
// 32 lanes call it.
__device__ __forceinline__ void add_layer_sums_shared(int* s_m, int* s_tot, const LayerSums& r) {
  const bool on = r.layer != 0xFFFFFFFFu;
  const uint32_t act = __ballot_sync(0xFFFFFFFFu, on);
  if (act == 0) return;
  const int lead = __ffs(act) - 1;
  const uint32_t l0 = __shfl_sync(0xFFFFFFFFu, r.layer, lead);
  const bool in0 = on && r.layer == l0;
  const int m0 = __reduce_add_sync(0xFFFFFFFFu, in0 ? r.m : 0);
  const int b = __reduce_add_sync(0xFFFFFFFFu, on ? r.b : 0);
  const int m = __reduce_add_sync(0xFFFFFFFFu, on ? r.m : 0);
  if ((int)(threadIdx.x & 31u) == lead) {
    atomicAdd(&s_m[l0], m0);
    atomicAdd(&s_tot[0], b);
    atomicAdd(&s_tot[1], m);
  } else if (on && !in0) {
    atomicAdd(&s_m[r.layer], r.m);
  }
}

// The other array's word w shifted by one site onto this word's sites, so
// that each site meets its second z-neighbour: site j of array 0 meets site
// j - 1 of array 1, site j of array 1 meets site j + 1 of array 0, and the
// row's ends meet through the periodic z wrap.
template <bool FULL>
__device__ __forceinline__ uint32_t z_shifted(const FilmCtx& c, const Fetched& f, uint32_t X, bool partial) {
  if (X == 0) {
    const uint32_t pw = (f.w > 0) ? f.za : (((f.za >> bitpos((c.n - 1) & 31u)) & 1u) << 31);
    return shift_prev(f.z0, pw);
  }
  uint32_t Zs = shift_next(f.z0, f.za);
  if (!FULL && partial) Zs |= (f.zf & 1u) << bitpos((c.n - 1) & 31u);
  return Zs;
}

// Decision paths of a word, chosen per film (so that a warp issues one):
//   kFull     32 valid sites, eight Philox calls;
//   kPartial  the row's only word (W = 1), partial: the film's last_mask and
//             last_calls (5..7 calls: calls Q and Q + 4 drawn together);
//   kSingle   the same with at most four calls, each drawn alone;
//   kMixed    rows of full words and a partial last word (W >= 2): each
//             word's own mask and call count.
enum : uint32_t { kFull = 0, kPartial = 1, kSingle = 2, kMixed = 3 };

__device__ __forceinline__ uint32_t FilmCtx::path() const {
  if (last_mask == 0xFFFFFFFFu) return kFull;
  if (W >= 2) return kMixed;
  return last_calls <= 4 ? kSingle : kPartial;
}

template <uint32_t PATH, bool FAST, bool QUARTER, bool MEAS = false, bool H3 = false>
__device__ __forceinline__ uint32_t decide_word(const FilmCtx& c, const Fetched& f,
                                                const uint32_t* __restrict__ s_thr,
                                                const uint32_t* __restrict__ s_alw, uint32_t qsel,
                                                uint32_t* stash = nullptr) {
  const uint32_t Lx = c.Lx, Ly = c.Ly;
  const uint32_t kx = f.kx, ky = f.ky, w = f.w;
  const uint32_t row = (kx - 1) * Ly + (ky - 1);
  const uint32_t X = (kx + ky + 1 + c.colour) & 1u;
  const uint32_t S = f.S;
  // aligned-with-S masks of the six neighbour slots (free x surface: empty
  // slot, mask 0; Eq. 11 wrap: the partner's spin enters with reversed sign)
  const uint32_t xm_on = (kx > 1 || c.x_pbc) ? 0xFFFFFFFFu : 0u;
  const uint32_t xp_on = (kx < Lx || c.x_pbc) ? 0xFFFFFFFFu : 0u;
  const uint32_t negm = (c.y_mode != kYPbc) ? 0xFFFFFFFFu : 0u;
  const uint32_t a0 = ~(S ^ f.xm) & xm_on;
  const uint32_t a1 = ~(S ^ f.xp) & xp_on;
  const uint32_t a2 = ~(S ^ f.ym ^ (ky > 1 ? 0u : negm));
  const uint32_t a3 = ~(S ^ f.yp ^ (ky < Ly ? 0u : negm));
  constexpr bool FULL = PATH == kFull, SINGLE = PATH == kSingle;
  const bool partial = PATH == kMixed ? (w + 1 == c.W) : !FULL;  // the word holds fewer than 32 sites
  const uint32_t Zs = z_shifted<FULL>(c, f, X, partial);
  const uint32_t a4 = ~(S ^ f.z0);
  const uint32_t a5 = ~(S ^ Zs);

  // bit-sliced count of aligned neighbours: n = c0 + 2 c1 + 4 c2
  const uint32_t s1 = a0 ^ a1 ^ a2, k1 = maj3(a0, a1, a2);
  const uint32_t s2 = a3 ^ a4 ^ a5, k2 = maj3(a3, a4, a5);
  const uint32_t c0 = s1 ^ s2, k3 = s1 & s2;
  const uint32_t c1 = k1 ^ k2 ^ k3, c2 = maj3(k1, k2, k3);
  if (MEAS) stash_counts(stash, c0, c1, c2, f.z0);  // for word_sums after the draws

  const uint32_t cls = row_class(kx, Lx);
  uint32_t alw = 0;
  if (!FAST) {
  // "always accept" (dE <= 0) as a 4-input function of (S, c0, c1, c2)
  const uint4* m4 = reinterpret_cast<const uint4*>(s_alw + cls * 16);
  const uint4 ma = m4[0], mb = m4[1], mc = m4[2], md = m4[3];
  const uint32_t v0 = (S & ma.y) | (~S & ma.x);
  const uint32_t v1 = (S & ma.w) | (~S & ma.z);
  const uint32_t v2 = (S & mb.y) | (~S & mb.x);
  const uint32_t v3 = (S & mb.w) | (~S & mb.z);
  const uint32_t v4 = (S & mc.y) | (~S & mc.x);
  const uint32_t v5 = (S & mc.w) | (~S & mc.z);
  const uint32_t v6 = (S & md.y) | (~S & md.x);
  const uint32_t v7 = (S & md.w) | (~S & md.z);
  const uint32_t w0 = (c0 & v1) | (~c0 & v0);
  const uint32_t w1 = (c0 & v3) | (~c0 & v2);
  const uint32_t w2 = (c0 & v5) | (~c0 & v4);
  const uint32_t w3 = (c0 & v7) | (~c0 & v6);
  const uint32_t x0 = (c1 & w1) | (~c1 & w0);
  const uint32_t x1 = (c1 & w3) | (~c1 & w2);
  alw = (c2 & x1) | (~c2 & x0);
  }

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

  const uint32_t ncalls = FULL ? 8u : PATH == kMixed ? (partial ? c.last_calls : 8u) : c.last_calls;
  const uint32_t clsb = (cls * 64u) * 0x01010101u;  // byte offset of this class's table
  const char* tb = reinterpret_cast<const char*>(s_thr);
  using Row = typename std::conditional<H3, PhiloxRow3, PhiloxRow>::type;
  const Row pr(row, c.sweep, X, c.rk0, c.rk1);
  uint32_t lt = 0;
  // calls Q and Q + 4 are drawn together (two independent Philox chains),
  // except on the kSingle path
  auto calls = [&](auto qc, uint32_t Uq) {
    constexpr uint32_t Q = decltype(qc)::value;
    if (FULL || Q < ncalls) {
      uint32_t u[4], v[4];
      if (SINGLE) {
        // a partial word of at most four calls: call Q alone
        pr.draw(8u * w + Q, u);
        const uint32_t Y = ((Uq << 2) & 0x3C3C3C3Cu) | clsb;
        site_one<FAST, Q, 0>(lt, tb, Y, u[0]);
        site_one<FAST, Q, 1>(lt, tb, Y, u[1]);
        site_one<FAST, Q, 2>(lt, tb, Y, u[2]);
        site_one<FAST, Q, 3>(lt, tb, Y, u[3]);
      } else {
        pr.draw2(8u * w + Q, 8u * w + Q + 4, u, v);
        const bool two = FULL || Q + 4 < ncalls;
        const uint32_t Y = ((Uq << 2) & 0x3C3C3C3Cu) | clsb;
        const uint32_t Y2 = ((Uq >> 2) & 0x3C3C3C3Cu) | clsb;
        site_pair<FAST, Q, 0>(lt, tb, Y, Y2, u[0], v[0], two);
        site_pair<FAST, Q, 1>(lt, tb, Y, Y2, u[1], v[1], two);
        site_pair<FAST, Q, 2>(lt, tb, Y, Y2, u[2], v[2], two);
        site_pair<FAST, Q, 3>(lt, tb, Y, Y2, u[3], v[3], two);
      }
    }
  };
  using Q0 = std::integral_constant<uint32_t, 0>;
  using Q1 = std::integral_constant<uint32_t, 1>;
  using Q2 = std::integral_constant<uint32_t, 2>;
  using Q3 = std::integral_constant<uint32_t, 3>;
  if (QUARTER) {
    // one code path for the four lanes (a switch on qsel would run all four
    // bodies one after another): runtime call index, bit in a register
    const uint32_t Uq = qsel == 0 ? U[0] : qsel == 1 ? U[1] : qsel == 2 ? U[2] : U[3];
    if (FULL || qsel < ncalls) {
      uint32_t u[4], v[4];
      pr.draw2(8u * w + qsel, 8u * w + qsel + 4, u, v);
      const bool two = FULL || qsel + 4 < ncalls;
      const uint32_t Y = ((Uq << 2) & 0x3C3C3C3Cu) | clsb;
      const uint32_t Y2 = ((Uq >> 2) & 0x3C3C3C3Cu) | clsb;
      const uint32_t base = (uint32_t)__cvta_generic_to_shared(tb);
#pragma unroll
      for (uint32_t i = 0; i < 4; i++) {
        uint32_t t, t2;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t) : "r"(base + __byte_perm(Y, 0, 0x4440 + i)));
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(t2) : "r"(base + __byte_perm(Y2, 0, 0x4440 + i)));
        if (FAST) {
          or_if_le(lt, u[i], t, 1u << (qsel + 8 * i));
          if (two) or_if_le(lt, v[i], t2, 1u << (qsel + 4 + 8 * i));
        } else {
          or_if_lt(lt, u[i], t, 1u << (qsel + 8 * i));
          if (two) or_if_lt(lt, v[i], t2, 1u << (qsel + 4 + 8 * i));
        }
      }
    }
  } else {
    calls(Q0{}, U[0]);
    calls(Q1{}, U[1]);
    calls(Q2{}, U[2]);
    calls(Q3{}, U[3]);
  }
  const uint32_t valid = FULL ? 0xFFFFFFFFu : PATH == kMixed ? (partial ? c.last_mask : 0xFFFFFFFFu) : c.last_mask;
  return (lt | alw) & valid;
}

// decide_word on the film's path (uniform across the film, so across a
// warp).  PATHS4 = false keeps two bodies only (for the kernel whose register
// budget has no room for more): full words on kFull, a partial last word on
// kPartial, chosen per word.
template <bool FAST, bool QUARTER, bool MEAS, bool PATHS4, bool H3 = false>
__device__ __forceinline__ uint32_t decide_any(const FilmCtx& c, const Fetched& f, const uint32_t* s_thr,
                                               const uint32_t* s_alw, uint32_t qsel, uint32_t* stash) {
  if (!PATHS4) {
    if (f.w + 1 < c.W || c.last_mask == 0xFFFFFFFFu)
      return decide_word<kFull, FAST, QUARTER, MEAS, H3>(c, f, s_thr, s_alw, qsel, stash);
    return decide_word<kPartial, FAST, QUARTER, MEAS, H3>(c, f, s_thr, s_alw, qsel, stash);
  }
  const uint32_t path = c.path();
  if (path == kFull) return decide_word<kFull, FAST, QUARTER, MEAS, H3>(c, f, s_thr, s_alw, qsel, stash);
  if (path == kMixed) return decide_word<kMixed, FAST, QUARTER, MEAS, H3>(c, f, s_thr, s_alw, qsel, stash);
  if (!QUARTER && path == kSingle)
    return decide_word<kSingle, FAST, QUARTER, MEAS, H3>(c, f, s_thr, s_alw, qsel, stash);
  return decide_word<kPartial, FAST, QUARTER, MEAS, H3>(c, f, s_thr, s_alw, qsel, stash);
}

__device__ __forceinline__ void store_word(const FilmCtx& c, const Fetched& f, uint32_t v) {
  const uint32_t row = (f.kx - 1) * c.Ly + (f.ky - 1);
  const uint32_t X = (f.kx + f.ky + 1 + c.colour) & 1u;
  uint32_t* __restrict__ P = X ? c.plane1 : c.plane0;
  ISG_ST(P, row * c.Wp + f.w, c.plane_words, 16, v);
}

// Word of update item `item`.  The first Lx * W items are the words of the
// ky = 1 rows, whose threads then also update the wrap partner's word: kept
// together, they fill whole warps instead of putting one lane that does twice
// the work into a third of the warps of a small film.  The other items are
// the rows ky = 2 .. Ly-1, layer by layer.  (dym, dyl) divide by Ly - 2 (by 1
// when Ly = 2, which has no such rows).
__device__ __forceinline__ void item_word(const FilmCtx& c, uint32_t item, uint32_t dwm, uint32_t dwl,
                                          uint32_t dym, uint32_t dyl, uint32_t& kx, uint32_t& ky, uint32_t& w) {
  const uint32_t rp = fastdiv(item, dwm, dwl);  // the region boundary Lx * W is a whole number of rows
  w = item - rp * c.W;
  const bool pair = rp < c.Lx;
  const uint32_t rq = pair ? 0u : rp - c.Lx;
  const uint32_t q = fastdiv(rq, dym, dyl);
  kx = (pair ? rp : q) + 1;
  ky = pair ? 1u : rq - q * (c.Ly - 2) + 2;
}

// MEAS: also return the record sums of the word (r1) and of its partner word
// (r2, ky = 1 only), using the thread's stash slots.
template <bool FAST, bool MEAS = false, bool PATHS4 = true, bool H3 = false>
__device__ __forceinline__ void update_fetched(const FilmCtx& c, const Fetched& f, const uint32_t* s_thr,
                                               const uint32_t* s_alw, uint32_t* stash = nullptr,
                                               LayerSums* r1 = nullptr, LayerSums* r2 = nullptr) {
  const uint32_t fl = decide_any<FAST, false, MEAS, PATHS4, H3>(c, f, s_thr, s_alw, 0, stash);
  const uint32_t v = f.S ^ fl;
  store_word(c, f, v);
  if (MEAS) *r1 = word_sums(c, f.kx, f.w, fl, v, stash);
  // ky = 1 rows then update their wrap partner row (kx', Ly); its wrap
  // neighbour is the word just written, so it is fetched only now
  if (f.ky == 1) {
    const uint32_t kx2 = (c.y_mode == kYGapbc) ? (c.Lx + 1 - f.kx) : f.kx;
    Fetched g;
    fetch_word(c, kx2, c.Ly, f.w, g);
    if (MEAS) stash[4] = c.seam_same ? (uint32_t)seam_adjust(c, f.w, v, stash[3], g) : 0u;
    const uint32_t fl2 = decide_any<FAST, false, MEAS, PATHS4, H3>(c, g, s_thr, s_alw, 0, stash);
    const uint32_t v2 = g.S ^ fl2;
    store_word(c, g, v2);
    if (MEAS) {
      *r2 = word_sums(c, kx2, g.w, fl2, v2, stash);
      r2->b += (int)stash[4];
    }
  }
}

// The same for a word shared by the four lanes 4j..4j+3 of a warp (lane qsel
// draws Philox calls qsel and qsel + 4); gmask holds the lanes whose group has
// a word.  The lanes merge their flip masks and the group's lane 0 stores
// (and, MEAS, takes the record sums).
template <bool FAST, bool MEAS>
__device__ __forceinline__ void update_fetched_quarter(const FilmCtx& c, const Fetched& f, bool on, uint32_t qsel,
                                                       uint32_t gmask, const uint32_t* s_thr,
                                                       const uint32_t* s_alw, uint32_t* stash, LayerSums& r1,
                                                       LayerSums& r2) {
  uint32_t fl = 0;
  if (on) fl = decide_any<FAST, true, MEAS, true>(c, f, s_thr, s_alw, qsel, stash);
  if (!on) return;
  fl |= __shfl_xor_sync(gmask, fl, 1);
  fl |= __shfl_xor_sync(gmask, fl, 2);
  const uint32_t v = f.S ^ fl;
  if (qsel == 0) store_word(c, f, v);
  if (MEAS && qsel == 0) r1 = word_sums(c, f.kx, f.w, fl, v, stash);
  // ky = 1 words then update their wrap partner word (see update_fetched)
  const uint32_t pmask = __ballot_sync(gmask, f.ky == 1);
  if (f.ky != 1) return;
  __syncwarp(pmask);  // the partner's wrap neighbour is the word stored above
  const uint32_t kx2 = (c.y_mode == kYGapbc) ? (c.Lx + 1 - f.kx) : f.kx;
  Fetched g;
  fetch_word(c, kx2, c.Ly, f.w, g);
  if (MEAS) stash[4] = c.seam_same ? (uint32_t)seam_adjust(c, f.w, v, stash[3], g) : 0u;
  uint32_t fl2 = decide_any<FAST, true, MEAS, true>(c, g, s_thr, s_alw, qsel, stash);
  fl2 |= __shfl_xor_sync(pmask, fl2, 1);
  fl2 |= __shfl_xor_sync(pmask, fl2, 2);
  const uint32_t v2 = g.S ^ fl2;
  if (qsel == 0) store_word(c, g, v2);
  if (MEAS && qsel == 0) {
    r2 = word_sums(c, kx2, g.w, fl2, v2, stash);
    r2.b += (int)stash[4];
  }
}

// ---- thin films: several rows per register
//
// A film whose rows hold one partial word per parity array (W = 1) with at
// most 8 sites (R = 4) or 16 sites (R = 2) per array spends the per-word work
// -- neighbour count, table indices, stores -- on a quarter or a half of a
// word's 32 sites.  The grid kernels then update R rows (kx, ky0 .. ky0+R-1)
// of one layer at once: row j's bits, which sit in the low B = 8/R bits of
// each byte, move up by j*B bits into one register, and the decision runs
// once on the packed word.  Packed bit j*B + q + 8*I is row j's site
// 4q + I, served by that row's Philox call q: the bit-to-call rule of a full
// word holds with "call" Q = j*B + q and the row's own counter.  The
// checkerboard is unchanged: consecutive rows update opposite arrays, and
// none reads an array another updates in the same half-sweep.  The memory
// layout is the same as for every other film; only the grid update kernels
// (one or two items per thread) pack.

// Packed operands of R rows (wrap signs folded into ym, yp).
struct Packed {
  uint32_t S, xm, xp, ym, yp, z0, Zs;
  uint32_t kx, ky0;
};

// Row mask of the low B bits of each byte.
template <uint32_t R>
__device__ __forceinline__ constexpr uint32_t slot_mask() {
  return 0x01010101u * ((1u << (8 / R)) - 1u);
}

template <uint32_t R>
__device__ __forceinline__ void fetch_packed(const FilmCtx& c, uint32_t kx, uint32_t ky0, Packed& p) {
  constexpr uint32_t B = 8 / R;
  p.kx = kx;
  p.ky0 = ky0;
  p.S = p.xm = p.xp = p.ym = p.yp = p.z0 = p.Zs = 0;
  const uint32_t valid = c.last_mask;  // the row's sites, all in the low B bits of each byte
  const uint32_t negm = (c.y_mode != kYPbc) ? valid : 0u;
#pragma unroll
  for (uint32_t j = 0; j < R; j++) {
    const uint32_t ky = ky0 + j;
    Fetched f;
    fetch_word(c, kx, ky, 0, f);
    const uint32_t X = (kx + ky + 1 + c.colour) & 1u;
    const uint32_t zs = z_shifted<false>(c, f, X, true) & valid;
    const uint32_t sh = j * B;
    p.S |= f.S << sh;
    p.xm |= f.xm << sh;
    p.xp |= f.xp << sh;
    p.ym |= (f.ym ^ (ky > 1 ? 0u : negm)) << sh;
    p.yp |= (f.yp ^ (ky < c.Ly ? 0u : negm)) << sh;
    p.z0 |= f.z0 << sh;
    p.Zs |= zs << sh;
  }
}

// The word of each of the R rows back into its own array.
template <uint32_t R>
__device__ __forceinline__ void store_packed(const FilmCtx& c, const Packed& p, uint32_t v) {
  constexpr uint32_t B = 8 / R;
#pragma unroll
  for (uint32_t j = 0; j < R; j++) {
    const uint32_t ky = p.ky0 + j;
    const uint32_t row = (p.kx - 1) * c.Ly + (ky - 1);
    const uint32_t X = (p.kx + ky + 1 + c.colour) & 1u;
    uint32_t* __restrict__ P = X ? c.plane1 : c.plane0;
    ISG_ST(P, row * c.Wp, c.plane_words, 17, (v >> (j * B)) & slot_mask<R>());
  }
}

// Metropolis decisions of the packed word: the flip mask (packed).
template <uint32_t R, bool FAST>
__device__ __forceinline__ uint32_t decide_packed(const FilmCtx& c, const Packed& p,
                                                  const uint32_t* __restrict__ s_thr,
                                                  const uint32_t* __restrict__ s_alw) {
  constexpr uint32_t B = 8 / R;
  const uint32_t Lx = c.Lx, kx = p.kx;
  const uint32_t S = p.S;
  const uint32_t xm_on = (kx > 1 || c.x_pbc) ? 0xFFFFFFFFu : 0u;
  const uint32_t xp_on = (kx < Lx || c.x_pbc) ? 0xFFFFFFFFu : 0u;
  const uint32_t a0 = ~(S ^ p.xm) & xm_on;
  const uint32_t a1 = ~(S ^ p.xp) & xp_on;
  const uint32_t a2 = ~(S ^ p.ym);
  const uint32_t a3 = ~(S ^ p.yp);
  const uint32_t a4 = ~(S ^ p.z0);
  const uint32_t a5 = ~(S ^ p.Zs);
  const uint32_t s1 = a0 ^ a1 ^ a2, k1 = maj3(a0, a1, a2);
  const uint32_t s2 = a3 ^ a4 ^ a5, k2 = maj3(a3, a4, a5);
  const uint32_t c0 = s1 ^ s2, k3 = s1 & s2;
  const uint32_t c1 = k1 ^ k2 ^ k3, c2 = maj3(k1, k2, k3);

  const uint32_t cls = row_class(kx, Lx);
  uint32_t alw = 0;
  if (!FAST) {
    const uint4* m4 = reinterpret_cast<const uint4*>(s_alw + cls * 16);
    const uint4 ma = m4[0], mb = m4[1], mc = m4[2], md = m4[3];
    const uint32_t v0 = (S & ma.y) | (~S & ma.x);
    const uint32_t v1 = (S & ma.w) | (~S & ma.z);
    const uint32_t v2 = (S & mb.y) | (~S & mb.x);
    const uint32_t v3 = (S & mb.w) | (~S & mb.z);
    const uint32_t v4 = (S & mc.y) | (~S & mc.x);
    const uint32_t v5 = (S & mc.w) | (~S & mc.z);
    const uint32_t v6 = (S & md.y) | (~S & md.x);
    const uint32_t v7 = (S & md.w) | (~S & md.z);
    const uint32_t w0 = (c0 & v1) | (~c0 & v0);
    const uint32_t w1 = (c0 & v3) | (~c0 & v2);
    const uint32_t w2 = (c0 & v5) | (~c0 & v4);
    const uint32_t w3 = (c0 & v7) | (~c0 & v6);
    const uint32_t x0 = (c1 & w1) | (~c1 & w0);
    const uint32_t x1 = (c1 & w3) | (~c1 & w2);
    alw = (c2 & x1) | (~c2 & x0);
  }
  const uint32_t T0 = (S & 0x55555555u) | ((c0 & 0x55555555u) << 1);
  const uint32_t T1 = ((S >> 1) & 0x55555555u) | (c0 & 0xAAAAAAAAu);
  const uint32_t T2 = (c1 & 0x55555555u) | ((c2 & 0x55555555u) << 1);
  const uint32_t T3 = ((c1 >> 1) & 0x55555555u) | (c2 & 0xAAAAAAAAu);
  uint32_t U[4];
  U[0] = (T0 & 0x33333333u) | ((T2 & 0x33333333u) << 2);
  U[1] = (T1 & 0x33333333u) | ((T3 & 0x33333333u) << 2);
  U[2] = ((T0 >> 2) & 0x33333333u) | (T2 & 0xCCCCCCCCu);
  U[3] = ((T1 >> 2) & 0x33333333u) | (T3 & 0xCCCCCCCCu);

  const uint32_t clsb = (cls * 64u) * 0x01010101u;
  const char* tb = reinterpret_cast<const char*>(s_thr);
  const uint32_t ncalls = c.last_calls;  // calls of one row (q < ncalls)
  const uint32_t rowb = (kx - 1) * c.Ly + (p.ky0 - 1);
  uint32_t lt = 0;
  // call Q (0..7) of the packed word: row Q / B's call Q % B, whose sites sit
  // at bits Q + 8 I; their table indices are nibbles of U[Q & 3] (the low or
  // high nibble of each byte for Q < 4 or Q >= 4)
  auto call = [&](auto qc) {
    constexpr uint32_t Q = decltype(qc)::value;
    constexpr uint32_t j = Q / B, q = Q % B;
    if (q < ncalls) {
      const uint32_t X = (kx + p.ky0 + j + 1 + c.colour) & 1u;
      uint32_t u[4];
      PhiloxRow(rowb + j, c.sweep, X, c.rk0, c.rk1).draw(q, u);
      const uint32_t Uq = U[Q & 3];
      const uint32_t Y = (Q < 4 ? ((Uq << 2) & 0x3C3C3C3Cu) : ((Uq >> 2) & 0x3C3C3C3Cu)) | clsb;
      site_one<FAST, Q, 0>(lt, tb, Y, u[0]);
      site_one<FAST, Q, 1>(lt, tb, Y, u[1]);
      site_one<FAST, Q, 2>(lt, tb, Y, u[2]);
      site_one<FAST, Q, 3>(lt, tb, Y, u[3]);
    }
  };
  call(std::integral_constant<uint32_t, 0>{});
  call(std::integral_constant<uint32_t, 4>{});
  call(std::integral_constant<uint32_t, 1>{});
  call(std::integral_constant<uint32_t, 5>{});
  call(std::integral_constant<uint32_t, 2>{});
  call(std::integral_constant<uint32_t, 6>{});
  call(std::integral_constant<uint32_t, 3>{});
  call(std::integral_constant<uint32_t, 7>{});
  uint32_t valid = 0;
#pragma unroll
  for (uint32_t j = 0; j < R; j++) valid |= c.last_mask << (j * B);
  return (lt | alw) & valid;
}

// The R rows of a group, and, for the group holding ky = 1, then the group
// holding ky = Ly of the wrap partner layer (fetched after the first group is
// stored, as update_fetched does with single rows).  Plain launches only: the
// summing launches take a group's rows one at a time (sweep_block_rows).
template <uint32_t R, bool FAST>
__device__ __forceinline__ void update_packed(const FilmCtx& c, const Packed& p, const uint32_t* s_thr,
                                              const uint32_t* s_alw) {
  const uint32_t fl = decide_packed<R, FAST>(c, p, s_thr, s_alw);
  store_packed<R>(c, p, p.S ^ fl);
  if (p.ky0 != 1) return;
  const uint32_t kx2 = (c.y_mode == kYGapbc) ? (c.Lx + 1 - p.kx) : p.kx;
  Packed g;
  fetch_packed<R>(c, kx2, c.Ly - R + 1, g);
  const uint32_t fl2 = decide_packed<R, FAST>(c, g, s_thr, s_alw);
  store_packed<R>(c, g, g.S ^ fl2);
}

// Group of packed update item `item`: the first Lx items are the groups
// holding ky = 1 (whose threads then update the wrap partner's last group),
// the others the middle groups of each layer.  (dm, dl) divide by
// Ly / R - 2 (by 1 when that is 0).
template <uint32_t R>
__device__ __forceinline__ void item_group(const FilmCtx& c, uint32_t item, uint32_t dm, uint32_t dl, uint32_t& kx,
                                           uint32_t& ky0) {
  const bool pair = item < c.Lx;
  const uint32_t r = pair ? 0u : item - c.Lx;
  const uint32_t q = fastdiv(r, dm, dl);
  kx = (pair ? item : q) + 1;
  ky0 = pair ? 1u : (r - q * (c.Ly / R - 2) + 1) * R + 1;
}

// The packed items of one block (as sweep_block's word items) in a plain
// launch.
template <uint32_t R, bool FAST>
__device__ __forceinline__ void sweep_block_packed(const FilmCtx& c, uint32_t first, uint32_t items, uint32_t dm,
                                                   uint32_t dl, const uint32_t* __restrict__ s_thr,
                                                   const uint32_t* __restrict__ s_alw) {
  const uint32_t item = first + threadIdx.x;
  if (item >= items) return;
  uint32_t kx, ky0;
  item_group<R>(c, item, dm, dl, kx, ky0);
  Packed p;
  fetch_packed<R>(c, kx, ky0, p);
  update_packed<R, FAST>(c, p, s_thr, s_alw);
}

// The packed items of one block, each group's rows decided one at a time
// with the single-row body (update_fetched): rows ky0 .. ky0+R-1 of layer
// kx, and for the group holding ky = 1 (whose row 1 then updates its wrap
// partner, row Ly of layer kx') the other rows of the partner's group.  The
// record sums of a group's rows (one layer) and of the partner's rows
// (another) are added up in registers and then added like a single word's.
template <bool FAST, bool MEAS, bool PATHS4, typename AccOf>
__device__ __forceinline__ void sweep_block_rows(const FilmCtx& c, uint32_t first, uint32_t items, uint32_t dm,
                                                 uint32_t dl, const uint32_t* __restrict__ s_thr,
                                                 const uint32_t* __restrict__ s_alw, bool meas, AccOf acc_of,
                                                 uint32_t* stash) {
  const uint32_t R = c.pack;
  const uint32_t item = first + threadIdx.x;
  const bool mine = item < items;
  LayerSums g1, g2;
  if (mine) {
    uint32_t kx, ky0;
    const uint32_t G2 = c.Ly / R - 2;
    const bool pair = item < c.Lx;
    const uint32_t r = pair ? 0u : item - c.Lx;
    const uint32_t q = fastdiv(r, dm, dl);
    kx = (pair ? item : q) + 1;
    ky0 = pair ? 1u : (r - q * G2 + 1) * R + 1;
    const uint32_t kx2 = (c.y_mode == kYGapbc) ? (c.Lx + 1 - kx) : kx;
    if (MEAS) {
      g1.layer = kx - 1;
      if (pair) g2.layer = kx2 - 1;
    }
    const uint32_t nrows = pair ? 2 * R - 1 : R;  // the partner row itself comes with row 1
#pragma unroll 1
    for (uint32_t i = 0; i < nrows; i++) {
      const bool own = i < R;
      const uint32_t rkx = own ? kx : kx2, rky = own ? ky0 + i : c.Ly - R + 1 + (i - R);
      Fetched f;
      fetch_word(c, rkx, rky, 0, f);
      if (MEAS && meas) {
        LayerSums a, b;
        update_fetched<FAST, true, PATHS4>(c, f, s_thr, s_alw, stash, &a, &b);
        LayerSums& g = own ? g1 : g2;
        g.m += a.m;
        g.b += a.b;
        if (b.layer != 0xFFFFFFFFu) {  // the partner row of row 1
          g2.m += b.m;
          g2.b += b.b;
        }
      } else {
        update_fetched<FAST, false, PATHS4>(c, f, s_thr, s_alw);
      }
    }
  }
  if (MEAS && meas) {
    add_layer_sums(acc_of(), g1);
    add_lane_sums(acc_of(), g2);
  }
}

}  // namespace

// The words of one block of words_per_block(ITEMS) consecutive words: each
// thread fetches its ITEMS words (kFilmThreads apart) before deciding any;
// ITEMS = 0: four lanes per word (kFilmThreads / 4 words).  MEAS and meas
// (half-sweep 1 of a sweep after which the film records): the words' record
// sums go into the film's per-layer accumulators acc_of() (a pointer made
// where it is used, not kept across the draws); s_stash holds kStashSlots
// words per thread.
template <bool FAST, uint32_t ITEMS, bool MEAS, bool PATHS4, bool H3, bool PK, typename AccOf>
__device__ __forceinline__ void sweep_block(const FilmCtx& c, uint32_t first, uint32_t items, uint32_t dwm,
                                            uint32_t dwl, uint32_t dym, uint32_t dyl,
                                            const uint32_t* __restrict__ s_thr, const uint32_t* __restrict__ s_alw,
                                            bool meas, AccOf acc_of, uint32_t* s_stash) {
  uint32_t* stash = s_stash + threadIdx.x * kStashSlots;
  if (ITEMS == 0) {
    const uint32_t item = first + (threadIdx.x >> 2);
    const bool on = item < items;
    const uint32_t gmask = __ballot_sync(0xFFFFFFFFu, on);
    Fetched f;
    if (on) {
      uint32_t kx, ky, w;
      item_word(c, item, dwm, dwl, dym, dyl, kx, ky, w);
      fetch_word(c, kx, ky, w, f);
    }
    LayerSums r1, r2;
    if (MEAS && meas) {
      update_fetched_quarter<FAST, true>(c, f, on, threadIdx.x & 3u, gmask, s_thr, s_alw, stash, r1, r2);
      add_layer_sums(acc_of(), r1);
      add_lane_sums(acc_of(), r2);
    } else {
      update_fetched_quarter<FAST, false>(c, f, on, threadIdx.x & 3u, gmask, s_thr, s_alw, stash, r1, r2);
    }
    return;
  }
  constexpr uint32_t NI = ITEMS == 0 ? 1 : ITEMS;
  if (PK && ITEMS == 1 && c.pack > 1) {  // the same for the whole film (the block)
    // fast-table plain launches decide a group's rows at once; the summing
    // and exact-table launches, whose registers have no room for the packed
    // body, take the group's rows one after another
    if (FAST && !MEAS) {
      if (c.pack == 4) sweep_block_packed<4, FAST>(c, first, items, dym, dyl, s_thr, s_alw);
      else sweep_block_packed<2, FAST>(c, first, items, dym, dyl, s_thr, s_alw);
    } else {
      sweep_block_rows<FAST, MEAS, PATHS4>(c, first, items, dym, dyl, s_thr, s_alw, meas, acc_of, stash);
    }
    return;
  }
  Fetched fw[NI];
  bool mine[NI];
#pragma unroll
  for (uint32_t it = 0; it < NI; it++) {
    const uint32_t item = first + threadIdx.x + it * kFilmThreads;
    mine[it] = item < items;
    if (mine[it]) {
      uint32_t kx, ky, w;
      item_word(c, item, dwm, dwl, dym, dyl, kx, ky, w);
      fetch_word(c, kx, ky, w, fw[it]);
    }
  }
  if (MEAS && meas) {
#pragma unroll
    for (uint32_t it = 0; it < NI; it++) {
      LayerSums r1, r2;
      if (mine[it]) update_fetched<FAST, true, PATHS4, H3>(c, fw[it], s_thr, s_alw, stash, &r1, &r2);
      add_layer_sums(acc_of(), r1);
      add_lane_sums(acc_of(), r2);
    }
    return;
  }
#pragma unroll
  for (uint32_t it = 0; it < NI; it++)
    if (mine[it]) update_fetched<FAST, false, PATHS4, H3>(c, fw[it], s_thr, s_alw);
}

// Half-sweep of every film of a launch: block b handles words_per_block(ITEMS)
// words of film owner[b], whose descriptor is staged in shared memory.  FAST:
// no film of the launch has a reachable thr = 0 entry (the compare-only
// table); otherwise every film takes the exact variant (which, at two words
// per thread, needs the registers of one block per SM fewer, and so does its
// recording form at one word).  At one word per thread the plain and
// record-writing forms fit one block per SM more (kMultiMinBlocks1), so that a
// small film set's half-sweep is one wave where it would spill into a second.
// MODE kUpdAccumulate: the half-sweep 1 launch
// of a sweep after which some film records; those films add their record
// sums into their accumulators in `part`.  MODE kUpdWriteRecord: a half-sweep
// 0 launch right after such a sweep; the last block of each film that
// recorded after `rec_done` sweeps writes that record (write_record) before
// its update, so the write overlaps the launch's other blocks.  The last
// block holds the film's ragged end, so it has the fewest words; the first
// ones hold the pair items, whose threads also update the wrap partner.
enum : uint32_t { kUpdPlain = 0, kUpdAccumulate = 1, kUpdWriteRecord = 2 };

template <uint32_t ITEMS>
__device__ __forceinline__ uint32_t last_update_block(const FilmDesc& d) {
  return d.upd_block_begin + (grid_items(d, ITEMS) + words_per_block(ITEMS) - 1) / words_per_block(ITEMS) - 1;
}

template <bool FAST, uint32_t ITEMS, uint32_t MODE, bool PK = false>
__global__ void __launch_bounds__(kFilmThreads, PK ? (MODE == kUpdAccumulate ? (FAST ? kMultiMinBlocks - 1
                                                                                    : kMultiMinBlocks - 2)
                                                                           : kMultiMinBlocks)
                                                : (ITEMS == 1 && MODE != kUpdAccumulate) ? kMultiMinBlocks1
                                                : (FAST || (ITEMS < 2 && MODE != kUpdAccumulate))
                                                    ? kMultiMinBlocks : kMultiMinBlocks - 1)
update_kernel(const FilmDesc* __restrict__ films, const uint32_t* __restrict__ owner,
              const LaunchHdr* __restrict__ hdr, uint32_t* __restrict__ pool, uint32_t colour, uint32_t k,
              int64_t* __restrict__ part, int64_t* __restrict__ records, uint32_t rec_done) {
  constexpr bool MEAS = MODE == kUpdAccumulate;
  constexpr uint32_t kDescWords = sizeof(FilmDesc) / 4;
  static_assert(sizeof(FilmDesc) % 16 == 0, "descriptor copied as uint4");
  __shared__ __align__(16) FilmDesc s_d;
  __shared__ __align__(16) uint32_t s_alw[FAST ? 1 : 64];
  __shared__ __align__(16) uint32_t s_lo[64];
  __shared__ uint32_t s_stash[MEAS ? kStashSlots * kFilmThreads : 1];
  __shared__ int64_t s_red[MODE == kUpdWriteRecord ? kFilmThreads / 32 : 1];
  __shared__ uint32_t s_slot;
  pdl_trigger();
  const uint32_t nvb = hdr->upd_blocks;
  for (uint32_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const uint32_t f = owner[vb];  // the same for every thread of the block
    __syncthreads();
    const uint4* src = reinterpret_cast<const uint4*>(films + f);
    uint4* dst = reinterpret_cast<uint4*>(&s_d);
    for (uint32_t i = threadIdx.x; i < kDescWords / 4; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) {
      const bool a = (s_d.always[i >> 4] >> (i & 15)) & 1u;
      if (!FAST) s_alw[i] = a ? 0xFFFFFFFFu : 0u;
      s_lo[i] = FAST ? (a ? 0xFFFFFFFFu : s_d.thr[i >> 4][i & 15] - 1u) : s_d.thr[i >> 4][i & 15];
    }
    __syncthreads();
    if (!s_d.active) continue;
    // The owner table, the descriptor and the table above are written by the
    // host before the launch; the lattice and the film's sweep counter may
    // still be written by the previous kernel of the stream (its blocks run
    // while these stage).  Wait for it (a no-op after the first time), then
    // read the counter again, around L1 (the staged copy may predate the
    // wait).
    pdl_wait();
    if (threadIdx.x == 0) s_d.sweep = __ldcg(&films[f].sweep);
    __syncthreads();
    if (MODE == kUpdWriteRecord && vb == last_update_block<ITEMS>(s_d) && records_after(s_d, s_d.sweep, rec_done))
      write_record(const_cast<FilmDesc*>(films + f), s_d, s_d.sweep, part, records, rec_done, s_red, &s_slot);
    if (s_d.sweep + k >= s_d.sweep_end) continue;
    FilmCtx c;
    c.Lx = s_d.Lx; c.Ly = s_d.Ly; c.n = s_d.n; c.W = s_d.W; c.Wp = s_d.Wp;
    c.plane_words = s_d.Lx * s_d.Ly * s_d.Wp;
    c.y_mode = s_d.y_mode; c.x_pbc = s_d.x_pbc; c.rk0 = s_d.rk0; c.rk1 = s_d.rk1;
    c.last_mask = s_d.last_mask; c.last_calls = s_d.last_calls;
    c.colour = colour; c.sweep = s_d.sweep + k;
    c.plane0 = pool + s_d.spin_off;
    c.plane1 = c.plane0 + (size_t)c.Lx * c.Ly * c.Wp;
    c.seam_same = seam_joins_one_colour(c.Lx, c.Ly, c.y_mode);
    const bool meas = MEAS && colour == 1 && measured_now(s_d, k + 1, 0);
    const FilmDesc* sd = &s_d;
    auto acc_of = [part, sd]() { return reinterpret_cast<unsigned long long*>(part + acc_offset(*sd)); };
    const uint32_t first = (vb - s_d.upd_block_begin) * words_per_block(ITEMS);
    // two words per thread, and the exact table: the register budget keeps
    // the two-path decision
    // packed thin films: group items and their divisor
    c.pack = PK ? s_d.pack : 1u;
    const bool pk = c.pack > 1;
    sweep_block<FAST, ITEMS, MEAS, FAST && ITEMS != 2, false, PK>(
        c, first, pk ? s_d.pk_items : s_d.upd_items, s_d.divw_m, s_d.divw_l, pk ? s_d.pk_divm : s_d.divy_m,
        pk ? s_d.pk_divl : s_d.divy_l, s_lo, s_alw, meas, acc_of, s_stash);
  }
}

// Single-film half-sweep.  The descriptor is a __grid_constant__ kernel
// parameter, so every per-film constant (round keys included) is read straight
// from the constant bank; block b updates words b * words_per_block(ITEMS)
// onwards.  MEAS: half-sweep 1 before a record, whose sums go into the
// film's accumulators acc.
template <bool FAST, uint32_t ITEMS, bool MEAS, bool PK = false>
__global__ void __launch_bounds__(kFilmThreads, PK && MEAS ? kFilmMinBlocks - 1 : kFilmMinBlocks)
update_film_kernel(const __grid_constant__ FilmDesc d, uint32_t* __restrict__ pool, uint32_t colour,
                   uint32_t sweep, int64_t* __restrict__ acc) {
  pdl_trigger();
  __shared__ __align__(16) uint32_t s_thr[64];
  __shared__ __align__(16) uint32_t s_alw[64];
  __shared__ uint32_t s_stash[MEAS ? kStashSlots * kFilmThreads : 1];
  for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) {
    const bool a = (d.always[i >> 4] >> (i & 15)) & 1u;
    s_thr[i] = FAST ? (a ? 0xFFFFFFFFu : d.thr[i >> 4][i & 15] - 1u) : d.thr[i >> 4][i & 15];
    s_alw[i] = a ? 0xFFFFFFFFu : 0u;
  }
  __syncthreads();
  pdl_wait();  // the table above needs nothing from the previous grid
  FilmCtx c;
  c.Lx = d.Lx; c.Ly = d.Ly; c.n = d.n; c.W = d.W; c.Wp = d.Wp;
  c.plane_words = d.Lx * d.Ly * d.Wp;
  c.y_mode = d.y_mode; c.x_pbc = d.x_pbc; c.rk0 = d.rk0; c.rk1 = d.rk1;
  c.last_mask = d.last_mask; c.last_calls = d.last_calls;
  c.colour = colour; c.sweep = sweep;
  c.plane0 = pool + d.spin_off;
  c.plane1 = c.plane0 + (size_t)d.Lx * d.Ly * d.Wp;
  c.seam_same = seam_joins_one_colour(d.Lx, d.Ly, d.y_mode);
  auto acc_of = [acc]() { return reinterpret_cast<unsigned long long*>(acc); };
  // the Philox head with round 3's product hoisted (PhiloxRow3) wherever the
  // registers allow it: not in the recording launch
  c.pack = PK ? d.pack : 1u;
  const bool pk = c.pack > 1;
  sweep_block<FAST, ITEMS, MEAS, true, !MEAS, PK>(c, blockIdx.x * words_per_block(ITEMS), pk ? d.pk_items : d.upd_items,
                                              d.divw_m, d.divw_l, pk ? d.pk_divm : d.divy_m,
                                              pk ? d.pk_divl : d.divy_l, s_thr, s_alw, MEAS, acc_of, s_stash);
}

// ------------------------------------------------------------ measurement

namespace {

// One lattice word for measure_word, its index tested in checked builds.
struct CheckedLoad {
  __device__ __forceinline__ uint32_t operator()(const uint32_t* p, size_t idx, size_t lim, uint32_t site) const {
    return ISG_LD(p, idx, lim, site);
  }
};

}  // namespace

__global__ void __launch_bounds__(kMeasureBlock)
measure_partial_kernel(const FilmDesc* __restrict__ films, const uint32_t* __restrict__ owner,
                       const LaunchHdr* __restrict__ hdr, const uint32_t* __restrict__ pool,
                       int64_t* __restrict__ part, uint32_t done, int force) {
  __shared__ int64_t s_red[kMeasureBlock / 32];
  __shared__ int s_m[kMeasureMaxLpu];
  pdl_trigger();
  pdl_wait();
  const uint32_t nvb = hdr->meas_blocks;
  for (uint32_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const FilmDesc& F = films[owner[vb]];
    if (!F.active || !measured_now(F, done, force)) continue;
    const uint32_t Lx = F.Lx, Ly = F.Ly, W = F.W, bpl = F.meas_bpl;
    if (F.meas_lpu > 1) {
      // several small layers per block: layer sums by shared atomics, one
      // bond-sum reduction; the bond sum goes to the first layer's slot
      const uint32_t* A = pool + F.spin_off;
      const uint32_t* B = A + (size_t)Lx * Ly * F.Wp;
      const uint32_t kx0 = (vb - F.meas_block_begin) * F.meas_lpu;
      const uint32_t nl = min(F.meas_lpu, Lx - kx0);
      const uint32_t per = Ly * W, total = nl * per;
      for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x) s_m[i] = 0;
      __syncthreads();
      int64_t bsum = 0;
      for (uint32_t base = 0; base < total; base += blockDim.x) {
        const uint32_t it = base + threadIdx.x;
        const bool on = it < total;
        int m = 0, bb = 0;
        uint32_t l = 0xFFFFFFFFu;
        if (on) {
          l = it / per;
          const uint32_t r = it - l * per, kym1 = r / W;
          measure_word(CheckedLoad{}, A, B, F.Wp, Lx, Ly, W, F.n, F.last_mask, F.x_pbc, F.y_mode, kx0 + l, kym1,
                       r - kym1 * W, m, bb);
          bsum += bb;
        }
        const uint32_t l0 = __shfl_sync(0xFFFFFFFFu, l, 0);
        if (__all_sync(0xFFFFFFFFu, !on || l == l0)) {
          int v = m;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
          if ((threadIdx.x & 31u) == 0 && l0 != 0xFFFFFFFFu) atomicAdd(&s_m[l0], v);
        } else if (on) {
          atomicAdd(&s_m[l], m);
        }
      }
      const int64_t tb = block_sum(bsum, s_red);  // its barriers also complete s_m
      for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x) {
        int64_t* p = part + F.part_off + 2 * (size_t)(kx0 + i);
        p[0] = s_m[i];
        if (i != 0) p[1] = 0;
      }
      if (threadIdx.x == 0) part[F.part_off + 2 * (size_t)kx0 + 1] = tb;
      __syncthreads();  // s_m is read above before the next block clears it
      continue;
    }
    const uint32_t local = vb - F.meas_block_begin;
    const uint32_t kxm1 = local / bpl, chunk = local % bpl;
    const uint32_t Wp = F.Wp;
    const uint32_t* A = pool + F.spin_off;
    const uint32_t* B = A + (size_t)Lx * Ly * Wp;
    int64_t msum = 0, bsum = 0;
    for (uint32_t it = chunk * blockDim.x + threadIdx.x; it < Ly * W; it += bpl * blockDim.x) {
      const uint32_t kym1 = it / W, w = it % W;
      int m, bb;
      measure_word(CheckedLoad{}, A, B, Wp, Lx, Ly, W, F.n, F.last_mask, F.x_pbc, F.y_mode, kxm1, kym1, w, m, bb);
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
  pdl_trigger();
  pdl_wait();
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

// Records of the films that record after `done` sweeps of the chunk, from
// the per-layer sums half-sweep 1 accumulated; the accumulators are cleared
// for the next record.
__global__ void __launch_bounds__(kMeasureBlock)
record_kernel(FilmDesc* __restrict__ films, const LaunchHdr* __restrict__ hdr, int64_t* __restrict__ part,
              int64_t* __restrict__ records, uint32_t done) {
  __shared__ int64_t s_red[kMeasureBlock / 32];
  __shared__ uint32_t s_slot;
  pdl_trigger();
  pdl_wait();
  const uint32_t nf = hdr->n_films;
  for (uint32_t f = blockIdx.x; f < nf; f += gridDim.x) {
    FilmDesc& F = films[f];
    if (!F.active || !measured_now(F, done, 0)) continue;
    write_record(&F, F, F.sweep, part, records, done, s_red, &s_slot);
  }
}

__global__ void advance_kernel(FilmDesc* __restrict__ films, const LaunchHdr* __restrict__ hdr, uint32_t n_sweeps) {
  pdl_trigger();
  pdl_wait();
  for (uint32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < hdr->n_films; f += gridDim.x * blockDim.x) {
    if (!films[f].active) continue;
    const uint32_t s = films[f].sweep, e = films[f].sweep_end;
    films[f].sweep = (e - s < n_sweeps) ? e : s + n_sweeps;
  }
}

// ------------------------------------------------------------ resident path

// All sweeps of a run for one small film per block.  The planes are copied
// into shared memory once (row stride W), each half-sweep is the same block
// body as the grid kernels followed by a block barrier (the next colour reads
// what this one wrote), the records of the run go straight into the film's
// ring, and the planes, sweep and rec_next are written back at the end.
template <bool FAST>
__global__ void __launch_bounds__(kResidentThreads, 1)
resident_kernel(FilmDesc* __restrict__ films, uint32_t* __restrict__ pool, int64_t* __restrict__ records,
                uint32_t n_sweeps) {
  extern __shared__ __align__(16) uint32_t s_planes[];
  constexpr uint32_t kDescWords = sizeof(FilmDesc) / 4;
  __shared__ __align__(16) FilmDesc s_d;
  __shared__ __align__(16) uint32_t s_thr[64];
  __shared__ __align__(16) uint32_t s_alw[64];
  __shared__ uint32_t s_stash[kStashSlots * kResidentThreads];
  __shared__ int s_tot[2];  // B and M of the record being summed
  pdl_trigger();
  pdl_wait();
  FilmDesc* Fg = films + blockIdx.x;
  {
    const uint4* src = reinterpret_cast<const uint4*>(Fg);
    uint4* dst = reinterpret_cast<uint4*>(&s_d);
    for (uint32_t i = threadIdx.x; i < kDescWords / 4; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) {
    const bool a = (s_d.always[i >> 4] >> (i & 15)) & 1u;
    s_thr[i] = FAST ? (a ? 0xFFFFFFFFu : s_d.thr[i >> 4][i & 15] - 1u) : s_d.thr[i >> 4][i & 15];
    s_alw[i] = a ? 0xFFFFFFFFu : 0u;
  }
  if (!s_d.active) return;  // the same for the whole block
  const uint32_t Lx = s_d.Lx, Ly = s_d.Ly, W = s_d.W, Wp = s_d.Wp;
  const uint32_t words = Lx * Ly * W;  // one plane in shared memory
  int* s_m = reinterpret_cast<int*>(s_planes + 2 * words);
  uint32_t* g0 = pool + s_d.spin_off;
  uint32_t* g1 = g0 + (size_t)Lx * Ly * Wp;
  for (uint32_t i = threadIdx.x; i < 2 * words; i += blockDim.x) {
    const uint32_t X = i >= words ? 1u : 0u;
    const uint32_t rw = i - X * words, r = rw / W, w = rw - r * W;
    s_planes[i] = ISG_LD(X ? g1 : g0, (size_t)r * Wp + w, (size_t)Lx * Ly * Wp, 41);
  }
  for (uint32_t kx = threadIdx.x; kx < Lx; kx += blockDim.x) s_m[kx] = 0;
  if (threadIdx.x < 2) s_tot[threadIdx.x] = 0;
  __syncthreads();
  FilmCtx c;
  c.Lx = Lx; c.Ly = Ly; c.n = s_d.n; c.W = W; c.Wp = W;
  c.plane_words = words;
  c.y_mode = s_d.y_mode; c.x_pbc = s_d.x_pbc; c.rk0 = s_d.rk0; c.rk1 = s_d.rk1;
  c.last_mask = s_d.last_mask; c.last_calls = s_d.last_calls;
  c.plane0 = s_planes;
  c.plane1 = s_planes + words;
  c.seam_same = seam_joins_one_colour(Lx, Ly, s_d.y_mode);
  c.pack = 1;  // the resident kernel updates single rows
  const uint32_t items = s_d.upd_items;
  const uint32_t m_every = s_d.measure_every;
  uint32_t rec_next = s_d.rec_next;
  uint32_t done = 0;
  for (uint32_t k = 0; k < n_sweeps; k++) {
    const uint32_t t = s_d.sweep + k;
    if (t >= s_d.sweep_end) break;
    c.sweep = t;
    // half-sweep 1 of a sweep after which the film records also sums the
    // record (as the grid kernels do) into s_m and s_tot
    const bool rec_now = m_every != 0 && (t + 1) % m_every == 0;
    for (uint32_t colour = 0; colour < 2; colour++) {
      c.colour = colour;
      if (colour == 1 && rec_now) {
        uint32_t* stash = s_stash + threadIdx.x * kStashSlots;
        for (uint32_t base = 0; base < items; base += blockDim.x) {
          const uint32_t item = base + threadIdx.x;
          LayerSums r1, r2;
          if (item < items) {
            uint32_t kx, ky, w;
            item_word(c, item, s_d.divw_m, s_d.divw_l, s_d.divy_m, s_d.divy_l, kx, ky, w);
            Fetched f;
            fetch_word(c, kx, ky, w, f);
            update_fetched<FAST, true>(c, f, s_thr, s_alw, stash, &r1, &r2);
          }
          add_layer_sums_shared(s_m, s_tot, r1);
          add_layer_sums_shared(s_m, s_tot, r2);
        }
      } else {
        for (uint32_t item = threadIdx.x; item < items; item += blockDim.x) {
          uint32_t kx, ky, w;
          item_word(c, item, s_d.divw_m, s_d.divw_l, s_d.divy_m, s_d.divy_l, kx, ky, w);
          Fetched f;
          fetch_word(c, kx, ky, w, f);
          update_fetched<FAST>(c, f, s_thr, s_alw);
        }
      }
      __syncthreads();
    }
    done = k + 1;
    if (!rec_now) continue;
    // record of sweep t + 1; every thread clears what it read, and the next
    // sweep's first barrier orders that before the next sums
    const uint32_t slot = s_d.rec_cap ? rec_next % s_d.rec_cap : 0u;
    int64_t* rec = records + s_d.rec_off + (size_t)slot * (5 + Lx);
    for (uint32_t kx = threadIdx.x; kx < Lx; kx += blockDim.x) {
      const int v = s_m[kx];
      s_m[kx] = 0;
      rec[5 + kx] = v;
      if (kx == 0) rec[3] = v;
      if (kx == Lx - 1) rec[4] = v;
    }
    if (threadIdx.x == 0) {
      rec[0] = (int64_t)t + 1;
      rec[1] = s_tot[0];
      rec[2] = s_tot[1];
      s_tot[0] = 0;
      s_tot[1] = 0;
    }
    rec_next++;
  }
  for (uint32_t i = threadIdx.x; i < 2 * words; i += blockDim.x) {
    const uint32_t X = i >= words ? 1u : 0u;
    const uint32_t rw = i - X * words, r = rw / W, w = rw - r * W;
    ISG_ST(X ? g1 : g0, (size_t)r * Wp + w, (size_t)Lx * Ly * Wp, 42, s_planes[i]);
  }
  if (threadIdx.x == 0) {
    Fg->sweep = s_d.sweep + done;
    Fg->rec_next = rec_next;
  }
}

// ------------------------------------------------------------- cluster-resident path

// Films held in distributed shared memory.  One thread-block cluster of C
// CTAs keeps one film for every sweep of a call: CTA r holds layers
// kx - 1 in [r Lx / C, (r + 1) Lx / C) of both planes (row stride W), and
// the cluster barrier between half-sweeps is the only synchronisation, so
// films never wait for one another and no launch boundary falls between
// half-sweeps.  A word's x-neighbour layer across a slab boundary, and the
// mirrored layer of an Eq. 11 partner row, sit in a peer CTA: every access
// goes through a table of the generic addresses of all layers of the film
// (the own CTA's shared window, or a peer's mapped into the cluster window),
// so such a word is a distributed-shared-memory load, and the partner's
// update a remote store.  Within a half-sweep no word is read that another
// thread writes (the checkerboard; the partner row reads the ky = 1 word its
// own thread has just written), so plain loads suffice, and the barrier's
// release/acquire orders one half-sweep's stores before the next one's loads.

// The words of fetch_word for word w of row (kx, ky), from the layer table
// lp[X * Lx + kx - 1] (plane X, 0-based layer kx - 1).
__device__ __forceinline__ void fetch_word_cl(const FilmCtx& c, uint32_t* const* lp, uint32_t kx, uint32_t ky,
                                              uint32_t w, Fetched& f) {
  const uint32_t Lx = c.Lx, Ly = c.Ly, W = c.W;
  const uint32_t X = (kx + ky + 1 + c.colour) & 1u;
  uint32_t* const* LP = lp + X * Lx;
  uint32_t* const* LQ = lp + (X ^ 1u) * Lx;
  const uint32_t rbase = (ky - 1) * W, base = rbase + w;
  const uint32_t lim = Ly * W;  // words of one layer
  const uint32_t* P = LP[kx - 1];
  const uint32_t* Q = LQ[kx - 1];
  const uint32_t gkx = (c.y_mode == kYGapbc) ? (Lx - kx) : (kx - 1);  // 0-based layer of the wrap row
  f.kx = kx; f.ky = ky; f.w = w;
  f.S = ISG_LD(P, base, lim, 61);
  f.xm = (kx > 1) ? ISG_LD(LP[kx - 2], base, lim, 62) : (c.x_pbc ? ISG_LD(LP[Lx - 1], base, lim, 63) : 0u);
  f.xp = (kx < Lx) ? ISG_LD(LP[kx], base, lim, 64) : (c.x_pbc ? ISG_LD(LP[0], base, lim, 65) : 0u);
  f.ym = (ky > 1) ? ISG_LD(P, base - W, lim, 66) : ISG_LD(LP[gkx], (Ly - 1) * W + w, lim, 67);
  f.yp = (ky < Ly) ? ISG_LD(P, base + W, lim, 68) : ISG_LD(LP[gkx], w, lim, 69);
  f.z0 = ISG_LD(Q, base, lim, 70);
  if (X == 0)  // previous word, or the row's last
    f.za = (w > 0) ? ISG_LD(Q, base - 1, lim, 71) : ISG_LD(Q, rbase + W - 1, lim, 72);
  else  // next word, or the row's first
    f.za = (w + 1 < W) ? ISG_LD(Q, base + 1, lim, 73) : ISG_LD(Q, rbase, lim, 74);
  f.zf = ISG_LD(Q, rbase, lim, 75);
}

__device__ __forceinline__ void store_word_cl(const FilmCtx& c, uint32_t* const* lp, const Fetched& f, uint32_t v) {
  const uint32_t X = (f.kx + f.ky + 1 + c.colour) & 1u;
  ISG_ST(lp[X * c.Lx + f.kx - 1], (f.ky - 1) * c.W + f.w, c.Ly * c.W, 76, v);
}

// update_fetched over the layer table.
template <bool FAST, bool MEAS>
__device__ __forceinline__ void update_fetched_cl(const FilmCtx& c, uint32_t* const* lp, const Fetched& f,
                                                  const uint32_t* s_thr, const uint32_t* s_alw,
                                                  uint32_t* stash = nullptr, LayerSums* r1 = nullptr,
                                                  LayerSums* r2 = nullptr) {
  const uint32_t fl = decide_any<FAST, false, MEAS, true>(c, f, s_thr, s_alw, 0, stash);
  const uint32_t v = f.S ^ fl;
  store_word_cl(c, lp, f, v);
  if (MEAS) *r1 = word_sums(c, f.kx, f.w, fl, v, stash);
  if (f.ky == 1) {
    const uint32_t kx2 = (c.y_mode == kYGapbc) ? (c.Lx + 1 - f.kx) : f.kx;
    Fetched g;
    fetch_word_cl(c, lp, kx2, c.Ly, f.w, g);
    if (MEAS) stash[4] = c.seam_same ? (uint32_t)seam_adjust(c, f.w, v, stash[3], g) : 0u;
    const uint32_t fl2 = decide_any<FAST, false, MEAS, true>(c, g, s_thr, s_alw, 0, stash);
    const uint32_t v2 = g.S ^ fl2;
    store_word_cl(c, lp, g, v2);
    if (MEAS) {
      *r2 = word_sums(c, kx2, g.w, fl2, v2, stash);
      r2->b += (int)stash[4];
    }
  }
}

// Word of the CTA's update item `item`: its nl layers from layer a + 1 on,
// the ky = 1 words first (their threads also update the wrap partner), then
// rows ky = 2 .. Ly-1 layer by layer (item_word on a slab of layers).
__device__ __forceinline__ void slab_item_word(const FilmDesc& d, uint32_t a, uint32_t nl, uint32_t item,
                                               uint32_t& kx, uint32_t& ky, uint32_t& w) {
  const uint32_t rp = fastdiv(item, d.divw_m, d.divw_l);
  w = item - rp * d.W;
  const bool pair = rp < nl;
  const uint32_t rq = pair ? 0u : rp - nl;
  const uint32_t q = fastdiv(rq, d.divy_m, d.divy_l);
  kx = a + (pair ? rp : q) + 1;
  ky = pair ? 1u : rq - q * (d.Ly - 2) + 2;
}

// Rounds of a CTA's half-sweep: a pair item (a ky = 1 word and its wrap
// partner) is two words of work, so its thread spends two rounds on it and
// takes one regular item fewer, and no warp runs a round longer than the
// others.  With P = q T + s pair items over T threads, thread t draws pair
// items t, t + T, ... (q + [t < s] of them) in rounds 0, 2, ..., and the
// P' regular items fill the remaining (thread, round) slots round by round:
// R = max(2 ceil(P / T), ceil((P' + 2 P) / T)) rounds hold them all.
struct SlabRounds {
  uint32_t P, q, s, R;
};

__device__ __forceinline__ SlabRounds slab_rounds(uint32_t P, uint32_t P2, uint32_t T) {
  SlabRounds o;
  o.P = P;
  o.q = P / T;
  o.s = P - o.q * T;
  const uint32_t rp = 2 * ((P + T - 1) / T), rw = (P2 + 2 * P + T - 1) / T;
  o.R = rp > rw ? rp : rw;
  return o;
}

// Item of thread t in round j: the pair item's index (< P) at the round that
// starts it, 0xFFFFFFFF at the round its partner takes, else P + the regular
// item's index (which may be >= P + P': nothing to do).
__device__ __forceinline__ uint32_t slab_round_item(const SlabRounds& r, uint32_t t, uint32_t j, uint32_t T) {
  const uint32_t kt = r.q + (t < r.s ? 1u : 0u);  // this thread's pair items
  if (j < 2 * kt) return (j & 1u) ? 0xFFFFFFFFu : t + (j >> 1) * T;
  const uint32_t j0 = 2 * r.q;
  const uint32_t reg = (j < j0 + 2) ? (j - j0) * (T - r.s) + (t - r.s) : 2 * (T - r.s) + (j - j0 - 2) * T + t;
  return r.P + reg;
}

// The record of sweep t (records-ring slot `slot`) from the layer sums the
// cluster's CTAs left in buffer `buf`: this CTA writes m(kx) of its own
// layers [a, b), rank 0 the totals.
__device__ __forceinline__ void cluster_record(cg::cluster_group& cl, const FilmDesc& d, int64_t* records, int* s_m,
                                               int (*s_tot)[2], uint32_t buf, uint32_t a, uint32_t b, uint32_t C,
                                               uint32_t t, uint32_t slot) {
  const uint32_t Lx = d.Lx;
  int64_t* rec = records + d.rec_off + (size_t)slot * (5 + Lx);
  for (uint32_t kx = a + threadIdx.x; kx < b; kx += blockDim.x) {
    int v = 0;
    for (uint32_t q = 0; q < C; q++) v += cl.map_shared_rank(s_m + buf * Lx, q)[kx];
    rec[5 + kx] = v;
    if (kx == 0) rec[3] = v;
    if (kx == Lx - 1) rec[4] = v;
  }
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    int B = 0, M = 0;
    for (uint32_t q = 0; q < C; q++) {
      const int* p = cl.map_shared_rank(&s_tot[buf][0], q);
      B += p[0];
      M += p[1];
    }
    rec[0] = (int64_t)t;
    rec[1] = B;
    rec[2] = M;
  }
}

// n_sweeps sweeps of film Fg on this cluster (C = its size), records into
// its ring, sweep and rec_next advanced at the end.  Dynamic shared memory
// s_dyn: planes [2][ceil(Lx / C)][Ly][W] words, the layer table (2 Lx
// generic addresses), and two buffers of Lx layer sums.  Ends with a cluster
// barrier, after which the CTA's shared memory is free for the next film.
template <bool FAST>
__device__ __forceinline__ void cluster_film(cg::cluster_group& cl, FilmDesc* Fg, uint32_t* __restrict__ pool,
                                             int64_t* __restrict__ records, uint32_t n_sweeps, FilmDesc& s_d,
                                             uint32_t* s_thr, uint32_t* s_alw, uint32_t* s_stash, int (*s_tot)[2],
                                             uint32_t* s_dyn) {
  constexpr uint32_t kDescWords = sizeof(FilmDesc) / 4;
  const uint32_t C = cl.num_blocks();
  const uint32_t r = cl.block_rank();
  {
    const uint4* src = reinterpret_cast<const uint4*>(Fg);
    uint4* dst = reinterpret_cast<uint4*>(&s_d);
    for (uint32_t i = threadIdx.x; i < kDescWords / 4; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < 64; i += blockDim.x) {
    const bool al = (s_d.always[i >> 4] >> (i & 15)) & 1u;
    s_thr[i] = FAST ? (al ? 0xFFFFFFFFu : s_d.thr[i >> 4][i & 15] - 1u) : s_d.thr[i >> 4][i & 15];
    s_alw[i] = al ? 0xFFFFFFFFu : 0u;
  }
  if (!s_d.active) return;  // the same for the whole cluster
  const uint32_t Lx = s_d.Lx, Ly = s_d.Ly, W = s_d.W;
  const uint32_t a = r * Lx / C, b = (r + 1) * Lx / C, nl = b - a;
  const uint32_t lw = Ly * W;                    // words of one layer
  const uint32_t pw = (Lx + C - 1) / C * lw;     // words of one local plane
  uint32_t* s_planes = s_dyn;
  uint32_t** s_lp = reinterpret_cast<uint32_t**>(s_dyn + 2 * pw);  // 8-byte aligned: 2 pw is even
  int* s_m = reinterpret_cast<int*>(s_lp + 2 * Lx);
  const size_t gpl = (size_t)Lx * lw;  // words of one plane in the pool (row stride W)
  uint32_t* g = pool + s_d.spin_off;
  for (uint32_t i = threadIdx.x; i < 2 * nl * lw; i += blockDim.x) {
    const uint32_t X = i >= nl * lw ? 1u : 0u;
    const uint32_t j = i - X * nl * lw;
    s_planes[X * pw + j] = ISG_LD(g, X * gpl + (size_t)a * lw + j, 2 * gpl, 77);
  }
  for (uint32_t i = threadIdx.x; i < 2 * Lx; i += blockDim.x) {
    const uint32_t X = i >= Lx ? 1u : 0u, k = i - X * Lx;
    uint32_t q = 0;
    while (q + 1 < C && (q + 1) * Lx / C <= k) q++;
    uint32_t* base = q == r ? s_planes : cl.map_shared_rank(s_planes, q);
    s_lp[i] = base + X * pw + (k - q * Lx / C) * lw;
    s_m[i] = 0;
  }
  if (threadIdx.x < 4) s_tot[threadIdx.x >> 1][threadIdx.x & 1] = 0;
  FilmCtx c;
  c.Lx = Lx; c.Ly = Ly; c.n = s_d.n; c.W = W; c.Wp = W;
  c.plane_words = lw;
  c.y_mode = s_d.y_mode; c.x_pbc = s_d.x_pbc; c.rk0 = s_d.rk0; c.rk1 = s_d.rk1;
  c.last_mask = s_d.last_mask; c.last_calls = s_d.last_calls;
  c.plane0 = nullptr;
  c.plane1 = nullptr;
  c.seam_same = seam_joins_one_colour(Lx, Ly, s_d.y_mode);
  c.pack = 1;
  const uint32_t items = nl * (Ly - 1) * W;
  const SlabRounds rounds = slab_rounds(nl * W, nl * (Ly - 2) * W, blockDim.x);
  const uint32_t m_every = s_d.measure_every;
  uint32_t rec_next = s_d.rec_next, nrec = 0, done = 0;
  // a record's sums are read in the half-sweep after the one that took them
  // and cleared in the next; two buffers alternate between records
  int read_buf = -1, clear_buf = -1;
  uint32_t read_t = 0, read_slot = 0;
  cl.sync();  // every CTA's planes are in place
  for (uint32_t k = 0; k < n_sweeps; k++) {
    const uint32_t t = s_d.sweep + k;
    if (t >= s_d.sweep_end) break;
    c.sweep = t;
    const bool rec_now = m_every != 0 && (t + 1) % m_every == 0;
    for (uint32_t colour = 0; colour < 2; colour++) {
      c.colour = colour;
      if (clear_buf >= 0) {
        for (uint32_t i = threadIdx.x; i < Lx; i += blockDim.x) s_m[clear_buf * Lx + i] = 0;
        if (threadIdx.x < 2) s_tot[clear_buf][threadIdx.x] = 0;
        clear_buf = -1;
      }
      if (read_buf >= 0) {
        cluster_record(cl, s_d, records, s_m, s_tot, (uint32_t)read_buf, a, b, C, read_t, read_slot);
        clear_buf = read_buf;
        read_buf = -1;
      }
      if (colour == 1 && rec_now) {
        int* sm = s_m + (nrec & 1u) * Lx;
        int* st = s_tot[nrec & 1u];
        uint32_t* stash = s_stash + threadIdx.x * kStashSlots;
        for (uint32_t j = 0; j < rounds.R; j++) {  // the same count for every thread (warp-wide sums)
          const uint32_t item = slab_round_item(rounds, threadIdx.x, j, blockDim.x);
          LayerSums r1, r2;
          if (item < items) {
            uint32_t kx, ky, w;
            slab_item_word(s_d, a, nl, item, kx, ky, w);
            Fetched f;
            fetch_word_cl(c, s_lp, kx, ky, w, f);
            update_fetched_cl<FAST, true>(c, s_lp, f, s_thr, s_alw, stash, &r1, &r2);
          }
          add_layer_sums_shared(sm, st, r1);
          add_layer_sums_shared(sm, st, r2);
        }
      } else {
        for (uint32_t j = 0; j < rounds.R; j++) {
          const uint32_t item = slab_round_item(rounds, threadIdx.x, j, blockDim.x);
          if (item >= items) continue;
          uint32_t kx, ky, w;
          slab_item_word(s_d, a, nl, item, kx, ky, w);
          Fetched f;
          fetch_word_cl(c, s_lp, kx, ky, w, f);
          update_fetched_cl<FAST, false>(c, s_lp, f, s_thr, s_alw);
        }
      }
      cl.sync();
    }
    done = k + 1;
    if (rec_now) {
      read_buf = (int)(nrec & 1u);
      read_t = t + 1;
      read_slot = s_d.rec_cap ? rec_next % s_d.rec_cap : 0u;
      rec_next++;
      nrec++;
    }
  }
  if (read_buf >= 0) cluster_record(cl, s_d, records, s_m, s_tot, (uint32_t)read_buf, a, b, C, read_t, read_slot);
  for (uint32_t i = threadIdx.x; i < 2 * nl * lw; i += blockDim.x) {
    const uint32_t X = i >= nl * lw ? 1u : 0u;
    const uint32_t j = i - X * nl * lw;
    ISG_ST(g, X * gpl + (size_t)a * lw + j, 2 * gpl, 78, s_planes[X * pw + j]);
  }
  if (r == 0 && threadIdx.x == 0) {
    Fg->sweep = s_d.sweep + done;
    Fg->rec_next = rec_next;
  }
  cl.sync();  // peers may still be reading this CTA's layer sums
}

// Clusters of C CTAs, cluster i sweeping films list[n_clusters + 1 + j] for j
// in [list[i], list[i + 1]) one after another (all n_sweeps sweeps of one,
// then the next): films never wait for one another, and the host packs them
// so that the clusters' loads are about equal.
template <bool FAST>
__global__ void __launch_bounds__(cluster_max_threads(!FAST), 1)
cluster_kernel(FilmDesc* __restrict__ films, const uint32_t* __restrict__ list, uint32_t n_clusters,
               uint32_t* __restrict__ pool, int64_t* __restrict__ records, uint32_t n_sweeps) {
  extern __shared__ __align__(16) uint32_t s_dyn[];
  __shared__ __align__(16) FilmDesc s_d;
  __shared__ __align__(16) uint32_t s_thr[64];
  __shared__ __align__(16) uint32_t s_alw[64];
  __shared__ uint32_t s_stash[kStashSlots * kClusterThreads];
  __shared__ int s_tot[2][2];  // {B, M} of the record being summed, two buffers
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t ci = blockIdx.x / cl.num_blocks();
  if (ci >= n_clusters) return;  // the same for the whole cluster
  const uint32_t j1 = list[ci + 1];
  for (uint32_t j = list[ci]; j < j1; j++) {
    __syncthreads();  // every thread is done with the previous film's descriptor
    cluster_film<FAST>(cl, films + list[n_clusters + 1 + j], pool, records, n_sweeps, s_d, s_thr, s_alw, s_stash,
                       s_tot, s_dyn);
  }
}

// ------------------------------------------------------------- set-up

__global__ void init_kernel(FilmDesc F, uint32_t* __restrict__ pool, int kind, uint32_t flip_lo, int flip_all) {
  const size_t words = (size_t)F.Lx * F.Ly * F.Wp;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * words) return;
  const uint32_t X = (uint32_t)(i / words);
  const size_t rem = i % words;
  const uint32_t row = (uint32_t)(rem / F.Wp), w = (uint32_t)(rem % F.Wp);
  if (w >= F.W) {
    pool[F.spin_off + i] = 0u;
    return;
  }
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
  const size_t words = (size_t)F.Lx * F.Ly * F.Wp;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * words) return;
  const uint32_t X = (uint32_t)(i / words);
  const size_t rem = i % words;
  const size_t row = rem / F.Wp;
  const uint32_t w = (uint32_t)(rem % F.Wp);
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
  const size_t words = (size_t)F.Lx * F.Ly * F.Wp;
  const uint32_t word = pool[F.spin_off + X * words + row * F.Wp + (j >> 5)];
  s[i] = ((word >> bitpos(j & 31u)) & 1u) ? (int8_t)1 : (int8_t)-1;
}

// ------------------------------------------------------ host launchers

namespace {

// Launch on st with programmatic stream serialisation: the kernel may begin
// while the previous kernel of the stream is still running and orders itself
// after it with pdl_wait.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), uint32_t grid, uint32_t block, uint32_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

namespace {

// pk: one item per thread and some film of the launch packs rows
template <uint32_t MODE>
auto update_variant(bool exact, uint32_t items, bool pk) {
  if (pk) return exact ? update_kernel<false, 1, MODE, true> : update_kernel<true, 1, MODE, true>;
  return exact ? (items == 2 ? update_kernel<false, 2, MODE>
                             : items == 1 ? update_kernel<false, 1, MODE> : update_kernel<false, 0, MODE>)
               : (items == 2 ? update_kernel<true, 2, MODE>
                             : items == 1 ? update_kernel<true, 1, MODE> : update_kernel<true, 0, MODE>);
}

template <bool MEAS>
auto update_film_variant(bool exact, uint32_t items, bool pk) {
  if (pk) return exact ? update_film_kernel<false, 1, MEAS, true> : update_film_kernel<true, 1, MEAS, true>;
  return exact ? (items == 2 ? update_film_kernel<false, 2, MEAS>
                             : items == 1 ? update_film_kernel<false, 1, MEAS> : update_film_kernel<false, 0, MEAS>)
               : (items == 2 ? update_film_kernel<true, 2, MEAS>
                             : items == 1 ? update_film_kernel<true, 1, MEAS> : update_film_kernel<true, 0, MEAS>);
}

}  // namespace

cudaError_t launch_update(const LaunchSet& L, uint32_t grid, uint32_t* pool, uint32_t colour, uint32_t k, bool exact,
                          uint32_t items, bool pack, int64_t* part, int64_t* records, bool accumulate,
                          uint32_t rec_done, cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  const bool pk = pack && items == 1;
  auto* kern = (accumulate && colour == 1) ? update_variant<kUpdAccumulate>(exact, items, pk)
               : (rec_done && colour == 0) ? update_variant<kUpdWriteRecord>(exact, items, pk)
                                           : update_variant<kUpdPlain>(exact, items, pk);
  return launch_pdl(kern, grid, kFilmThreads, 0, st, (const FilmDesc*)L.films, (const uint32_t*)L.owner_upd,
                    (const LaunchHdr*)L.hdr, pool, colour, k, part, records, rec_done);
}

cudaError_t launch_update_film(const FilmDesc& d, uint32_t* pool, uint32_t colour, uint32_t sweep, uint32_t items,
                               int64_t* acc, cudaStream_t st) {
  const uint32_t ipb = words_per_block(items);
  const uint32_t grid = (grid_items(d, items) + ipb - 1) / ipb;
  if (grid == 0) return cudaSuccess;
  const bool exact = d.has_never != 0;
  const bool pk = items == 1 && d.pack > 1;
  auto* kern = acc ? update_film_variant<true>(exact, items, pk) : update_film_variant<false>(exact, items, pk);
  return launch_pdl(kern, grid, kFilmThreads, 0, st, d, pool, colour, sweep, acc);
}

cudaError_t launch_record(const LaunchSet& L, uint32_t grid, int64_t* part, int64_t* records, uint32_t done,
                          cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  return launch_pdl(record_kernel, grid, kMeasureBlock, 0, st, L.films, (const LaunchHdr*)L.hdr, part, records,
                    done);
}

cudaError_t launch_measure(const LaunchSet& L, uint32_t grid, uint32_t fin_grid, const uint32_t* pool,
                           int64_t* part, int64_t* records, uint32_t done, int force, int64_t* direct,
                           cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  cudaError_t e = launch_pdl(measure_partial_kernel, grid, kMeasureBlock, 0, st, (const FilmDesc*)L.films,
                             (const uint32_t*)L.owner_meas, (const LaunchHdr*)L.hdr, pool, part, done, force);
  if (e != cudaSuccess) return e;
  return launch_pdl(measure_finalize_kernel, fin_grid, kMeasureBlock, 0, st, L.films, (const LaunchHdr*)L.hdr,
                    (const int64_t*)part, records, done, force, direct);
}

cudaError_t launch_advance(const LaunchSet& L, uint32_t grid, uint32_t n_sweeps, cudaStream_t st) {
  if (grid == 0 || n_sweeps == 0) return cudaSuccess;
  return launch_pdl(advance_kernel, grid, 128, 0, st, L.films, (const LaunchHdr*)L.hdr, n_sweeps);
}

cudaError_t launch_init(const FilmDesc& f, uint32_t* pool, int kind, uint32_t flip_lo, int flip_all,
                        cudaStream_t st) {
  const size_t n = 2 * (size_t)f.Lx * f.Ly * f.Wp;
  init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, pool, kind, flip_lo, flip_all);
  return cudaGetLastError();
}

cudaError_t launch_pack(const FilmDesc& f, uint32_t* pool, const int8_t* s, cudaStream_t st) {
  const size_t n = 2 * (size_t)f.Lx * f.Ly * f.Wp;
  pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, pool, s);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const FilmDesc& f, const uint32_t* pool, int8_t* s, cudaStream_t st) {
  const size_t n = (size_t)f.Lx * f.Ly * f.Lz;
  unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, pool, s);
  return cudaGetLastError();
}

uint32_t resident_smem_bytes(const FilmDesc& d) {
  const uint64_t sites = (uint64_t)d.Lx * d.Ly * d.Lz;
  const uint64_t bytes = 4ull * (2ull * d.Lx * d.Ly * d.W + d.Lx);
  if (sites > kResidentMaxSites || bytes > kResidentMaxSmem) return 0;
  return (uint32_t)bytes;
}

uint32_t resident_threads(const FilmDesc& d) {
  const uint32_t t = ((d.upd_items + 31u) / 32u) * 32u;
  return t < 32u ? 32u : (t > kResidentThreads ? kResidentThreads : t);
}

cudaError_t launch_resident(FilmDesc* films, uint32_t n_films, uint32_t smem_bytes, uint32_t threads, bool exact,
                            uint32_t* pool, int64_t* records, uint32_t n_sweeps, cudaStream_t st) {
  if (n_films == 0 || n_sweeps == 0) return cudaSuccess;
  if (smem_bytes > kResidentMaxSmem || threads == 0 || threads > kResidentThreads || threads % 32u)
    return cudaErrorInvalidValue;
  auto* kern = exact ? resident_kernel<false> : resident_kernel<true>;
  return launch_pdl(kern, n_films, threads, smem_bytes, st, films, pool, records, n_sweeps);
}

uint32_t cluster_smem_bytes(const FilmDesc& d, uint32_t C) {
  if (C == 0 || C > kClusterMaxSize || d.Lx < C || d.Ly < 2 || d.Wp != d.W) return 0;
  const uint64_t nlm = (d.Lx + C - 1) / C;
  const uint64_t bytes = 8ull * nlm * d.Ly * d.W + 24ull * d.Lx;
  if (bytes > kClusterMaxSmem) return 0;
  return (uint32_t)bytes;
}

uint32_t cluster_threads(const FilmDesc& d, uint32_t C, bool exact, uint32_t per_sm) {
  // a pair item (ky = 1 word and its wrap partner) is two words of work
  const uint64_t tmax = std::max<uint64_t>(32, cluster_max_threads(exact) / std::max<uint32_t>(per_sm, 1) / 32 * 32);
  const uint64_t nlm = (d.Lx + C - 1) / C;
  const uint64_t work = nlm * d.Ly * d.W;
  const uint64_t rounds = std::max<uint64_t>(1, (work + tmax - 1) / tmax);
  const uint64_t t = ((work + rounds - 1) / rounds + 31) / 32 * 32;
  return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(t, 32), tmax);
}

namespace {

// Dynamic shared memory of a launch with per_sm CTAs per SM: at least what the
// films need, and enough that per_sm + 1 CTAs (with the kernel's static
// shared memory and the per-block reserve) do not fit in one SM.
template <typename K>
cudaError_t cluster_launch_smem(K kern, uint32_t needed, uint32_t per_sm, uint32_t* out) {
  int dev = 0, per_smp = 0, reserve = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_smp, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const uint64_t fixed = (uint64_t)fa.sharedSizeBytes + (uint64_t)reserve;
  uint64_t pad = (uint64_t)per_smp / (per_sm + 1) + 1;  // per_sm + 1 CTAs of this size overflow the SM
  pad = pad > fixed ? (pad - fixed + 127) / 128 * 128 : 0;
  uint64_t smem = std::max<uint64_t>(needed, pad);
  if (smem > kClusterMaxSmem) smem = std::max<uint64_t>(needed, kClusterMaxSmem);
  *out = (uint32_t)smem;
  return cudaSuccess;
}

template <typename K>
cudaLaunchConfig_t cluster_config(K kern, uint32_t grid, uint32_t C, uint32_t smem, uint32_t threads,
                                  cudaStream_t st, cudaLaunchAttribute* attr, cudaError_t* e) {
  *e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterMaxSmem);
  // the whole unified L1 as shared memory, so that per_sm padded CTAs fit
  if (*e == cudaSuccess)
    *e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

int cluster_capacity(uint32_t C, uint32_t per_sm, uint32_t smem_bytes, uint32_t threads, bool exact) {
  if (C == 0 || C > kClusterMaxSize || per_sm == 0 || per_sm > kClusterMaxPerSm || smem_bytes > kClusterMaxSmem ||
      threads == 0 || threads > cluster_max_threads(exact) || threads % 32u)
    return 0;
  auto* kern = exact ? cluster_kernel<false> : cluster_kernel<true>;
  uint32_t smem = 0;
  if (cluster_launch_smem(kern, smem_bytes, per_sm, &smem) != cudaSuccess) return -1;
  cudaLaunchAttribute attr[1];
  cudaError_t e;
  cudaLaunchConfig_t cfg = cluster_config(kern, C, C, smem, threads, nullptr, attr, &e);
  if (e != cudaSuccess) return -1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) return -1;
  return n;
}

cudaError_t launch_cluster(FilmDesc* films, const uint32_t* list, uint32_t n_clusters, uint32_t C, uint32_t per_sm,
                           uint32_t smem_bytes, uint32_t threads, bool exact, uint32_t* pool, int64_t* records,
                           uint32_t n_sweeps, cudaStream_t st) {
  if (n_clusters == 0 || n_sweeps == 0) return cudaSuccess;
  if (C == 0 || C > kClusterMaxSize || per_sm == 0 || per_sm > kClusterMaxPerSm || smem_bytes > kClusterMaxSmem ||
      threads == 0 || threads > cluster_max_threads(exact) || threads % 32u)
    return cudaErrorInvalidValue;
  auto* kern = exact ? cluster_kernel<false> : cluster_kernel<true>;
  uint32_t smem = 0;
  cudaError_t e = cluster_launch_smem(kern, smem_bytes, per_sm, &smem);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config(kern, n_clusters * C, C, smem, threads, st, attr, &e);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, kern, films, list, n_clusters, pool, records, n_sweeps);
}

int read_oob_counters(unsigned long long* count, unsigned long long* first) {
#ifdef ISING_CHECKED
  if (cudaMemcpyFromSymbol(count, g_oob_count, sizeof *count) != cudaSuccess) return -1;
  if (cudaMemcpyFromSymbol(first, g_oob_first, sizeof *first) != cudaSuccess) return -1;
  return 1;
#else
  *count = 0;
  *first = 0;
  return 0;
#endif
}

int update_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, update_kernel<true, 1, kUpdPlain>, kFilmThreads, 0) !=
      cudaSuccess)
    return 0;
  return nb;
}

int measure_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, measure_partial_kernel, kMeasureBlock, 0) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace isg
