// Device multi-precision core: warp-cooperative Montgomery arithmetic on
// 32-bit limbs for sm_103a.
//
// One "instance" (one modular product chain) is held by a group of T
// consecutive lanes of a warp; lane k of the group owns limbs k*S .. k*S+S-1
// of every operand (S limbs per lane, NL = S*T limbs in all).  A Montgomery
// product t = a b R^-1 mod N (R = 2^(32 NL)) is the coarsely integrated
// operand-scanning method (CIOS): for each limb b_i of b,
//     t += a b_i ;  m = t_0 N' mod 2^32 ;  t += m N ;  t /= 2^32.
// Distribution across the group:
//   * b_i is read from shared memory, where the group staged b (a broadcast:
//     every lane of the group reads the same word);
//   * m is computed from the lowest limb, owned by lane 0, and broadcast with
//     a shuffle;
//   * the shift by one limb moves each lane's lowest limb to the lane below
//     (one shuffle); inside a lane the shift is a renaming of registers,
//     because the S steps of a block are unrolled with a rotating index;
//   * carries that leave a lane's top limb are not propagated step by step:
//     they stay in two per-lane carry words (x1, x2) that are folded into the
//     limb shifted in from the lane above, and the remaining carries are
//     resolved once at the end with a ballot-based carry-lookahead over the
//     group, followed by the conditional subtraction of N (borrows resolved
//     the same way).
// Row updates t += a * b_i use the PTX carry chain (mad.lo.cc / madc.hi.cc),
// split into the even and odd products so that each chain writes every limb
// once.
//
// The exponentiations run their schedules through a second form, mont_sos
// (separated operand scanning): the whole product is formed first as chunk
// products spread evenly over the lanes (a square forms each cross product
// once), then reduced by the second half of the CIOS steps; it is defined
// with its description further down.
#pragma once

#include <cstdint>
#include <utility>

namespace pl {

#define PL_DEV __device__ __forceinline__

// ---------------------------------------------------------------------------
// PTX carry-chain primitives.  Consecutive calls form one chain through the
// carry flag; nothing else touches the flag in between.
PL_DEV void mad_lo_cc(uint32_t& d, uint32_t a, uint32_t b) {
  asm volatile("mad.lo.cc.u32 %0, %1, %2, %0;" : "+r"(d) : "r"(a), "r"(b));
}
PL_DEV void madc_lo_cc(uint32_t& d, uint32_t a, uint32_t b) {
  asm volatile("madc.lo.cc.u32 %0, %1, %2, %0;" : "+r"(d) : "r"(a), "r"(b));
}
PL_DEV void madc_hi_cc(uint32_t& d, uint32_t a, uint32_t b) {
  asm volatile("madc.hi.cc.u32 %0, %1, %2, %0;" : "+r"(d) : "r"(a), "r"(b));
}
PL_DEV void add_cc(uint32_t& d, uint32_t a) { asm volatile("add.cc.u32 %0, %0, %1;" : "+r"(d) : "r"(a)); }
PL_DEV void addc_cc(uint32_t& d, uint32_t a) { asm volatile("addc.cc.u32 %0, %0, %1;" : "+r"(d) : "r"(a)); }
PL_DEV void addc(uint32_t& d, uint32_t a) { asm volatile("addc.u32 %0, %0, %1;" : "+r"(d) : "r"(a)); }
PL_DEV uint32_t carry_out() { uint32_t c; asm volatile("addc.u32 %0, 0, 0;" : "=r"(c)); return c; }
PL_DEV void sub_cc(uint32_t& d, uint32_t a) { asm volatile("sub.cc.u32 %0, %0, %1;" : "+r"(d) : "r"(a)); }
PL_DEV void subc_cc(uint32_t& d, uint32_t a) { asm volatile("subc.cc.u32 %0, %0, %1;" : "+r"(d) : "r"(a)); }
// sets the carry flag to c (0 or 1)
PL_DEV void set_carry(uint32_t c) {
  uint32_t z;  // only the carry flag is wanted
  asm volatile("add.cc.u32 %0, %1, 0xffffffff;" : "=r"(z) : "r"(c));
  (void)z;
}
// sets the borrow flag to b (0 or 1)
PL_DEV void set_borrow(uint32_t b) {
  uint32_t z;  // only the borrow flag is wanted
  asm volatile("sub.cc.u32 %0, 0, %1;" : "=r"(z) : "r"(b));
  (void)z;
}
// borrow flag of the chain as 0/1
PL_DEV uint32_t borrow_out() { uint32_t c; asm volatile("subc.u32 %0, 0, 0;" : "=r"(c)); return c & 1u; }

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// t += a * b over S limbs; t's logical limb j lives in physical register
// (j + ROT) % S; the carry out of logical limb S-1 goes to (x1, x2).
template <int S, int ROT>
PL_DEV void row(uint32_t (&t)[S], uint32_t& x1, uint32_t& x2, const uint32_t (&a)[S], uint32_t b) {
  static_assert(S % 2 == 0, "S must be even");
#define PL_T(j) t[((j) + ROT) % S]
  // even products: lo into limb j, hi into limb j+1
  mad_lo_cc(PL_T(0), a[0], b);
  madc_hi_cc(PL_T(1), a[0], b);
#pragma unroll
  for (int j = 2; j < S; j += 2) {
    madc_lo_cc(PL_T(j), a[j], b);
    madc_hi_cc(PL_T(j + 1), a[j], b);
  }
  addc_cc(x1, 0u);
  addc(x2, 0u);
  // odd products: lo into limb j, hi into limb j+1 (limb S is x1)
  mad_lo_cc(PL_T(1), a[1], b);
#pragma unroll
  for (int j = 1; j < S - 1; j += 2) {
    madc_hi_cc(PL_T(j + 1), a[j], b);
    madc_lo_cc(PL_T(j + 2), a[j + 2], b);
  }
  madc_hi_cc(x1, a[S - 1], b);
  addc(x2, 0u);
#undef PL_T
}

// One CIOS step (limb b_i) at rotation U.
template <int S, int T, int U>
PL_DEV void mont_step(uint32_t (&t)[S], uint32_t& x1, uint32_t& x2, const uint32_t (&a)[S],
                      const uint32_t (&n)[S], uint32_t np, uint32_t bi, int k, unsigned mask) {
  row<S, U>(t, x1, x2, a, bi);
  uint32_t m = t[U % S] * np;
  if constexpr (T > 1) m = __shfl_sync(mask, m, 0, T);
  row<S, U>(t, x1, x2, n, m);
  uint32_t nb = 0;
  if constexpr (T > 1) {
    nb = __shfl_down_sync(mask, t[U % S], 1, T);
    if (k == T - 1) nb = 0;
  }
  // logical limb 0 (physical U % S) leaves; the new top limb takes its register
  uint32_t top = x1;
  add_cc(top, nb);
  uint32_t nx1 = x2;
  addc(nx1, 0u);
  t[U % S] = top;
  x1 = nx1;
  x2 = 0;
}

template <int S, int T, int... U>
PL_DEV void mont_block(uint32_t (&t)[S], uint32_t& x1, uint32_t& x2, const uint32_t (&a)[S],
                       const uint32_t (&n)[S], uint32_t np, const uint32_t* bp, int bstride, int k,
                       unsigned mask, std::integer_sequence<int, U...>) {
  (mont_step<S, T, U>(t, x1, x2, a, n, np, bp[U * bstride], k, mask), ...);
}

// Carry-lookahead over the T lanes of a group: given per-lane generate and
// propagate bits, returns the carry into this lane; *out gets the carry out of
// the group's top lane.
template <int T>
PL_DEV uint32_t group_lookahead(bool gen, bool prop, int k, unsigned mask, uint32_t* out) {
  const int lane = threadIdx.x & 31;
  const int gb = lane - k;
  const uint32_t gm = (T == 32) ? 0xffffffffu : ((1u << T) - 1u);
  const uint32_t G = (__ballot_sync(mask, gen) >> gb) & gm;
  const uint32_t P = (__ballot_sync(mask, prop) >> gb) & gm;
  const uint64_t s = (uint64_t)(G | P) + G;
  const uint32_t cm = (uint32_t)s ^ (G | P) ^ G;
  *out = (uint32_t)(s >> T) & 1u;
  return (cm >> k) & 1u;
}

// Fold the per-lane carry words into the limbs and reduce once:
// V = sum_k 2^(32 S k) (t_k + x1_k 2^(32 S)) + inject (at limb 0), V < 2N;
// on return t holds V mod N, canonical.
template <int S, int T>
PL_DEV void normalize(uint32_t (&t)[S], uint32_t x1, uint32_t inject, const uint32_t (&n)[S], int k,
                      unsigned mask) {
  uint32_t cin = inject;
  if constexpr (T > 1) {
    const uint32_t up = __shfl_up_sync(mask, x1, 1, T);
    if (k != 0) cin = up;
  }
  add_cc(t[0], cin);
#pragma unroll
  for (int j = 1; j < S; ++j) addc_cc(t[j], 0u);
  const uint32_t g = carry_out();
  uint32_t top;
  if constexpr (T > 1) {
    uint32_t all = t[0];
#pragma unroll
    for (int j = 1; j < S; ++j) all &= t[j];
    uint32_t cout;
    const uint32_t c = group_lookahead<T>(g != 0, all == 0xffffffffu, k, mask, &cout);
    if (c) {
      add_cc(t[0], 1u);
#pragma unroll
      for (int j = 1; j < S; ++j) addc_cc(t[j], 0u);
    }
    top = __shfl_sync(mask, x1, T - 1, T) + cout;
  } else {
    top = x1 + g;
  }
  // borrow of t - n (per lane, no borrow in), and equality for propagation
  uint32_t z = t[0];
  sub_cc(z, n[0]);
  uint32_t eq = t[0] ^ n[0];
#pragma unroll
  for (int j = 1; j < S; ++j) {
    z = t[j];
    subc_cc(z, n[j]);
    eq |= t[j] ^ n[j];
  }
  const uint32_t b = borrow_out();
  uint32_t bin = 0, bout;
  if constexpr (T > 1) {
    bin = group_lookahead<T>(b != 0, eq == 0, k, mask, &bout);
  } else {
    bout = b;
  }
  if (top != 0 || bout == 0) {  // V >= N: subtract N (with this lane's borrow in)
    set_borrow(bin);
#pragma unroll
    for (int j = 0; j < S; ++j) subc_cc(t[j], n[j]);
  }
}

// r = a * b * R^-1 mod N (canonical); a, n in registers (this lane's slice),
// limb i of b at bs[i * bstride] in shared memory.  a and b < R, a b < N R.
template <int S, int T>
PL_DEV void mont_mul(uint32_t (&r)[S], const uint32_t (&a)[S], const uint32_t* bs, int bstride,
                     const uint32_t (&n)[S], uint32_t np, int k, unsigned mask = kFull) {
  uint32_t x1 = 0, x2 = 0;
#pragma unroll
  for (int j = 0; j < S; ++j) r[j] = 0;
#pragma unroll 1
  for (int blk = 0; blk < T; ++blk) {
    mont_block<S, T>(r, x1, x2, a, n, np, bs + blk * S * bstride, bstride, k, mask,
                     std::make_integer_sequence<int, S>{});
  }
  normalize<S, T>(r, x1, 0u, n, k, mask);
}

// ---------------------------------------------------------------------------
// Montgomery products and squarings in separated form (SOS), one code body
// for both: r = a b R^-1 mod N, or r = a^2 R^-1 mod N with every cross product
// a_i a_j (i != j) formed once.
//
// First the product P (2 NL limbs) is built in chunks of S limbs; lane k ends
// with chunk k ("lo", a part of P mod R) and chunk k + T ("hi", a part of
// P div R).  With A_k, B_k lane k's chunks of a and b and X = 2^(32 S), P is a
// sum of chunk products A_k B_l X^(k + l), formed in rounds in which every
// lane does the same work:
//   * product: rounds D = 0 .. T - 1, lane k forming A_k B_((k + D) mod T);
//   * square: P = sum_k A_k^2 X^(2k) + 2 sum_{k < l} A_k A_l X^(k + l):
//     rounds D = 1 .. T/2 - 1 (lane k forms A_k A_((k + D) mod T): every pair
//     at cyclic distance d once), the round "half" (the pair {k, k + T/2}
//     split between its two lanes by the halves of the upper chunk: the lower
//     lane multiplies the lower chunk by its low half, the upper lane by its
//     high half, S^2 / 2 each), then the sum so far is doubled and the round
//     D = 0 adds the diagonal chunks A_k^2.
// A square forms (T / 2 + 1/2) S^2 limb products per lane against T S^2 for a
// product.  A round's 2S-limb result lands at chunk c (low half) and c + 1
// (high half) with c = 2k + D mod T, so each lane receives exactly two halves
// of the same kind, with two shuffles in which every sending lane serves one
// receiver (a lane below T/2 sends its low half first, a lane above its high
// half).  Carries out of a chunk stay in that chunk's carry word.
// The reduction is the second half of the CIOS steps (m = t_0 N'; t += m N;
// shift) on the low half of P, after which the high half is added: the value
// (P + M N) / R is below 2N (P < N^2), and one conditional subtraction makes it
// canonical.  The rounds run in a loop, so an exponentiation's loop holds one
// routine's code whether an op squares or multiplies.

// t += a[j] * b for j = J, J + 2, ... < S: lo into logical limb j, hi into
// j + 1 (logical limb S is x1); the carry out of the chain goes into x1, x2.
template <int S, int ROT, int J>
PL_DEV void chain_from(uint32_t (&t)[S], uint32_t& x1, uint32_t& x2, const uint32_t (&a)[S], uint32_t b) {
  if constexpr (J < S) {
#define PL_T(j) t[((j) + ROT) % S]
    mad_lo_cc(PL_T(J), a[J], b);
    if constexpr (J + 1 < S) {
      madc_hi_cc(PL_T(J + 1), a[J], b);
    } else {
      madc_hi_cc(x1, a[J], b);
    }
#pragma unroll
    for (int j = J + 2; j < S; j += 2) {
      madc_lo_cc(PL_T(j), a[j], b);
      if (j + 1 < S) {
        madc_hi_cc(PL_T(j + 1), a[j], b);
      } else {
        madc_hi_cc(x1, a[j], b);
      }
    }
    constexpr int last = J + 2 * ((S - 1 - J) / 2);
    if constexpr (last + 1 == S) {
      addc(x2, 0u);
    } else {
      addc_cc(x1, 0u);
      addc(x2, 0u);
    }
#undef PL_T
  }
}

// t += a[j] * b for J0 <= j < S (logical limbs, rotation ROT), carry into x1, x2
template <int S, int ROT, int J0>
PL_DEV void row_from(uint32_t (&t)[S], uint32_t& x1, uint32_t& x2, const uint32_t (&a)[S], uint32_t b) {
  chain_from<S, ROT, J0>(t, x1, x2, a, b);
  chain_from<S, ROT, J0 + 1>(t, x1, x2, a, b);
}

// shift of a lane-local window of SW limbs by one limb: logical limb I leaves into out
template <int SW, int I>
PL_DEV void leave_w(uint32_t (&w)[SW], uint32_t& x1, uint32_t& x2, uint32_t& out) {
  out = w[I % SW];
  w[I % SW] = x1;
  x1 = x2;
  x2 = 0;
}

// v, made to depend on dep for the compiler: an operand computed from the
// result is not moved above the instructions that produce dep (it keeps a
// row's shuffle next to its row instead of every shuffle of a round being
// hoisted to the top of the round, each holding a register)
PL_DEV int after(int v, uint32_t dep) {
  asm volatile("" : "+r"(v) : "r"(dep));
  return v;
}

// z: zero, computed from the previous round's carry words (a carry word counts
// a few carries, far below 2^31).  Adding it to a round's shuffle lane makes the
// round wait for the previous one: otherwise the compiler may overlap the
// rounds' independent rows and hold all their limbs at once.
PL_DEV int seq_zero(uint32_t carry_word) { return (int)(carry_word >> 31); }

// lo, w = A_k * (partner p's chunk of src): S rows over this lane's a, the
// multiplier limbs arriving from lane p by shuffle, row by row
template <int S, int T, int... I>
PL_DEV void sos_pair(uint32_t (&lo)[S], uint32_t (&w)[S], const uint32_t (&a)[S], const uint32_t (&src)[S], int p,
                     unsigned mask, std::integer_sequence<int, I...>) {
  uint32_t x1 = 0, x2 = 0;
#pragma unroll
  for (int j = 0; j < S; ++j) w[j] = 0;
  ((row_from<S, I % S, 0>(w, x1, x2, a, __shfl_sync(mask, src[I], after(p, x1), T)),
    leave_w<S, I>(w, x1, x2, lo[I])),
   ...);
}

// row I of sos_half: multiplier = limb I of the pair's lower chunk (this lane's
// own limb on the lower lane, the partner's on the upper lane; every lane
// takes part in the shuffle)
template <int S, int T, int I>
PL_DEV void half_row(uint32_t (&w)[S / 2], uint32_t& x1, uint32_t& x2, uint32_t (&lo)[S], const uint32_t (&m)[S / 2],
                     const uint32_t (&a)[S], int p, bool up, unsigned mask) {
  const uint32_t v = __shfl_sync(mask, a[I], after(p, x1), T);
  const uint32_t b = up ? v : a[I];
  row_from<S / 2, I % (S / 2), 0>(w, x1, x2, m, b);
  leave_w<S / 2, I>(w, x1, x2, lo[I]);
}

// lo, hi = this lane's share of A_j A_(j + T/2), j = k mod T/2 (the pair's
// lower and upper chunks): the lower lane forms A_j times the low half of the
// upper chunk, the upper lane A_j times its high half (then shifted up by S/2
// limbs); both are S rows (the limbs of A_j) over an S/2-limb multiplicand.
template <int S, int T, int... I>
PL_DEV void sos_half(uint32_t (&lo)[S], uint32_t (&hi)[S], const uint32_t (&a)[S], int k, int z, unsigned mask,
                     std::integer_sequence<int, I...>) {
  constexpr int H = S / 2;
  const int p = (k ^ (T / 2)) + z;
  const bool up = k >= T / 2;
  uint32_t m[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const uint32_t v = __shfl_sync(mask, a[j], p, T);
    m[j] = up ? a[H + j] : v;
  }
  uint32_t w[H];
  uint32_t x1 = 0, x2 = 0;
#pragma unroll
  for (int j = 0; j < H; ++j) w[j] = 0;
  (half_row<S, T, I>(w, x1, x2, lo, m, a, p, up, mask), ...);
  // the product is lo (S limbs) then w (S/2 limbs); the upper lane's share sits S/2 limbs higher
#pragma unroll
  for (int j = 0; j < S; ++j) {
    const uint32_t h_lower = j < H ? w[j] : 0u;
    const uint32_t h_upper = j < H ? lo[j + H] : w[j - H];
    hi[j] = up ? h_upper : h_lower;
  }
#pragma unroll
  for (int j = S - 1; j >= 0; --j) lo[j] = up ? (j >= H ? lo[j - H] : 0u) : lo[j];
}

// R += v & msk over S limbs, the carry out into c
template <int S>
PL_DEV void add_masked(uint32_t (&R)[S], uint32_t& c, const uint32_t (&v)[S], uint32_t msk) {
  add_cc(R[0], v[0] & msk);
#pragma unroll
  for (int j = 1; j < S; ++j) addc_cc(R[j], v[j] & msk);
  addc(c, 0u);
}

// Chunk of lane s's product in a round: pair rounds at distance D (D = 0: the
// diagonal chunks), or the half round.
template <int T>
PL_DEV int sos_chunk(int s, bool half, int D) {
  return half ? 2 * (s & (T / 2 - 1)) + T / 2 : s + ((s + D) & (T - 1));
}

// Adds to this lane's chunks (Rl: chunk k, Rh: chunk k + T) the halves of the
// round's products (lo, w of every lane) that land there; lo, w are clobbered.
// D is the round's distance (T/2 for the half round).
template <int S, int T>
PL_DEV void sos_route(uint32_t (&lo)[S], uint32_t (&w)[S], uint32_t (&Rl)[S], uint32_t& cl, uint32_t (&Rh)[S],
                      uint32_t& ch, int k, bool half, int D, unsigned mask) {
  const int r = (k - D) & (T - 1);
  const int high = r & 1;  // this lane receives high halves (else low halves)
  const int base = r >> 1;
  const int sx = base + (high ? T / 2 : 0);
  const int sy = base + (high ? 0 : T / 2);
  const bool xhi = sos_chunk<T>(sx, half, D) + high >= T;
  const bool yhi = sos_chunk<T>(sy, half, D) + high >= T;
  const bool lowside = k < T / 2;
#pragma unroll
  for (int u = 0; u < S; ++u) {
    const uint32_t x = lowside ? lo[u] : w[u];
    const uint32_t y = lowside ? w[u] : lo[u];
    lo[u] = __shfl_sync(mask, x, sx, T);
    w[u] = __shfl_sync(mask, y, sy, T);
  }
  const uint32_t mxl = xhi ? 0u : 0xffffffffu, myl = yhi ? 0u : 0xffffffffu;
  add_masked<S>(Rl, cl, lo, mxl);
  add_masked<S>(Rl, cl, w, myl);
  add_masked<S>(Rh, ch, lo, ~mxl);
  add_masked<S>(Rh, ch, w, ~myl);
}

// R, c = 2 (R + c X) in carry-save form
template <int S>
PL_DEV void dbl(uint32_t (&R)[S], uint32_t& c) {
  c = (c << 1) | (R[S - 1] >> 31);
#pragma unroll
  for (int j = S - 1; j > 0; --j) R[j] = __funnelshift_l(R[j - 1], R[j], 1);
  R[0] <<= 1;
}

// one reduction step at rotation U: m = t_0 N'; t += m N; shift by one limb
template <int S, int T, int U>
PL_DEV void redc_step(uint32_t (&t)[S], uint32_t& x1, uint32_t& x2, const uint32_t (&n)[S], uint32_t np, int k,
                      unsigned mask) {
  uint32_t m = t[U % S] * np;
  if constexpr (T > 1) m = __shfl_sync(mask, m, 0, T);
  row<S, U>(t, x1, x2, n, m);
  uint32_t nb = 0;
  if constexpr (T > 1) {
    nb = __shfl_down_sync(mask, t[U % S], 1, T);
    if (k == T - 1) nb = 0;
  }
  uint32_t top = x1;
  add_cc(top, nb);
  uint32_t nx1 = x2;
  addc(nx1, 0u);
  t[U % S] = top;
  x1 = nx1;
  x2 = 0;
}

template <int S, int T, int... U>
PL_DEV void redc_block(uint32_t (&t)[S], uint32_t& x1, uint32_t& x2, const uint32_t (&n)[S], uint32_t np, int k,
                       unsigned mask, std::integer_sequence<int, U...>) {
  (redc_step<S, T, U>(t, x1, x2, n, np, k, mask), ...);
}

// Whether mont_sos is compiled for this shape (the half round's S/2-limb rows
// need an even S/2; it holds about 7 S limbs per lane at once, so wider slices
// keep to mont_mul).
template <int S, int T>
constexpr bool kHaveSos = (S % 4 == 0) && (S <= 24) && (T >= 2) && (T <= 16) && ((T & (T - 1)) == 0);

// Whether the exponentiations use it at this shape: from 4 lanes up.  On 2
// lanes a square saves only a quarter of the multiplication rows and, measured
// on a B300, the separated form was slower there (1024-bit encryption 1.70M
// against 1.86M/s, the first stage of 2048-bit encryption 397 against 391 ms).
template <int S, int T>
constexpr bool kUseSos = kHaveSos<S, T> && (T >= 4);

// r = a src R^-1 mod N (square: src is a, and r = a^2 R^-1 mod N), canonical;
// a, src canonical (this lane's slices).  r may alias a or src.
template <int S, int T>
PL_DEV void mont_sos(uint32_t (&r)[S], const uint32_t (&a)[S], const uint32_t (&src)[S], const uint32_t (&n)[S],
                     uint32_t np, int k, bool square, unsigned mask = kFull) {
  static_assert(kHaveSos<S, T>, "no SOS product for this shape");
  uint32_t Rl[S], Rh[S], cl = 0, ch = 0;
#pragma unroll
  for (int j = 0; j < S; ++j) {
    Rl[j] = 0;
    Rh[j] = 0;
  }
  const int nround = square ? T / 2 + 1 : T;
#pragma unroll 1
  for (int rd = 0; rd < nround; ++rd) {
    // square: rounds D = 1 .. T/2 - 1, the half round, then (after doubling) D = 0; product: D = rd
    const bool half = square && rd == T / 2 - 1;
    const int D = square ? (half ? T / 2 : (rd == T / 2 ? 0 : rd + 1)) : rd;
    if (square && rd == T / 2) {
      dbl<S>(Rl, cl);
      dbl<S>(Rh, ch);
    }
    const int z = seq_zero(cl | ch);
    uint32_t lo[S], w[S];
    if (half) {
      sos_half<S, T>(lo, w, a, k, z, mask, std::make_integer_sequence<int, S>{});
    } else {
      sos_pair<S, T>(lo, w, a, src, ((k + D) & (T - 1)) + z, mask, std::make_integer_sequence<int, S>{});
    }
    sos_route<S, T>(lo, w, Rl, cl, Rh, ch, k, half, D, mask);
  }
  // reduction of the low half, then the high half added
  uint32_t x1 = cl, x2 = 0;
#pragma unroll 1
  for (int blk = 0; blk < T; ++blk) {
    redc_block<S, T>(Rl, x1, x2, n, np, k, mask, std::make_integer_sequence<int, S>{});
  }
  add_cc(Rl[0], Rh[0]);
#pragma unroll
  for (int j = 1; j < S; ++j) addc_cc(Rl[j], Rh[j]);
  addc(x1, ch);
  normalize<S, T>(Rl, x1, 0u, n, k, mask);
#pragma unroll
  for (int j = 0; j < S; ++j) r[j] = Rl[j];
}

// r = (a + b) mod N for canonical a, b (this lane's slices)
template <int S, int T>
PL_DEV void mod_add(uint32_t (&r)[S], const uint32_t (&a)[S], const uint32_t (&b)[S], const uint32_t (&n)[S],
                    int k, unsigned mask = kFull) {
#pragma unroll
  for (int j = 0; j < S; ++j) r[j] = a[j];
  add_cc(r[0], b[0]);
#pragma unroll
  for (int j = 1; j < S; ++j) addc_cc(r[j], b[j]);
  const uint32_t c = carry_out();
  normalize<S, T>(r, c, 0u, n, k, mask);
}

// ---------------------------------------------------------------------------
// Moving slices between registers, shared and global memory.

// stage this lane's slice v into the group's b column (limb i at bs[i * stride])
template <int S>
PL_DEV void stage(uint32_t* bs, int stride, const uint32_t (&v)[S], int k) {
#pragma unroll
  for (int j = 0; j < S; ++j) bs[(k * S + j) * stride] = v[j];
}

// load limbs k*S .. k*S+S-1 of a row (16-byte aligned rows)
template <int S>
PL_DEV void load_slice(uint32_t (&v)[S], const uint32_t* row, int k) {
  const uint32_t* p = row + k * S;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int j = 0; j < S; j += 4) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(p + j));
      v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < S; j += 2) {
      const uint2 q = __ldg(reinterpret_cast<const uint2*>(p + j));
      v[j] = q.x; v[j + 1] = q.y;
    }
  }
}

// load from memory this kernel also writes (no read-only path)
template <int S>
PL_DEV void load_slice_rw(uint32_t (&v)[S], const uint32_t* row, int k) {
  const uint32_t* p = row + k * S;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int j = 0; j < S; j += 4) {
      const uint4 q = *reinterpret_cast<const uint4*>(p + j);
      v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < S; j += 2) {
      const uint2 q = *reinterpret_cast<const uint2*>(p + j);
      v[j] = q.x; v[j + 1] = q.y;
    }
  }
}

template <int S>
PL_DEV void store_slice(uint32_t* row, const uint32_t (&v)[S], int k) {
  uint32_t* p = row + k * S;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int j = 0; j < S; j += 4) *reinterpret_cast<uint4*>(p + j) = make_uint4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < S; j += 2) *reinterpret_cast<uint2*>(p + j) = make_uint2(v[j], v[j + 1]);
  }
}

// this lane's slice of a constant array (parameter space)
template <int S>
PL_DEV void const_slice(uint32_t (&v)[S], const uint32_t* c, int k) {
#pragma unroll
  for (int j = 0; j < S; ++j) v[j] = c[k * S + j];
}

// ---------------------------------------------------------------------------
// Single-thread helpers for the once-per-item finishing steps (CRT
// recombination, exact division).  Plain loops over s limbs in local memory;
// their cost is a few thousand limb products per item, against millions in the
// exponentiations.

// r = a b R^-1 mod N, R = 2^(32 s), a, b < N; r may alias neither a nor b.
PL_DEV void mm_1t(uint32_t* r, const uint32_t* a, const uint32_t* b, const uint32_t* N, uint32_t np, int s) {
  // the accumulator lives in r plus two extra words (hi, hi2)
  uint32_t hi = 0, hi2 = 0;
  for (int j = 0; j < s; ++j) r[j] = 0;
  for (int i = 0; i < s; ++i) {
    const uint32_t bi = b[i];
    uint64_t c = 0;
    for (int j = 0; j < s; ++j) {
      c += (uint64_t)a[j] * bi + r[j];
      r[j] = (uint32_t)c;
      c >>= 32;
    }
    c += hi;
    hi = (uint32_t)c;
    hi2 = (uint32_t)(c >> 32);
    const uint32_t m = r[0] * np;
    c = ((uint64_t)m * N[0] + r[0]) >> 32;
    for (int j = 1; j < s; ++j) {
      c += (uint64_t)m * N[j] + r[j];
      r[j - 1] = (uint32_t)c;
      c >>= 32;
    }
    c += hi;
    r[s - 1] = (uint32_t)c;
    hi = hi2 + (uint32_t)(c >> 32);
  }
  // conditional subtraction: value = hi 2^(32 s) + r < 2N
  bool ge = hi != 0;
  if (!ge) {
    ge = true;
    for (int j = s - 1; j >= 0; --j) {
      if (r[j] != N[j]) { ge = r[j] > N[j]; break; }
    }
  }
  if (ge) {
    int64_t br = 0;
    for (int j = 0; j < s; ++j) {
      const int64_t d = (int64_t)r[j] - N[j] - br;
      br = d < 0;
      r[j] = (uint32_t)d;
    }
  }
}

// returns a >= b over s limbs
PL_DEV bool ge_1t(const uint32_t* a, const uint32_t* b, int s) {
  for (int j = s - 1; j >= 0; --j)
    if (a[j] != b[j]) return a[j] > b[j];
  return true;
}

// a += b over s limbs, returns the carry
PL_DEV uint32_t add_1t(uint32_t* a, const uint32_t* b, int s) {
  uint64_t c = 0;
  for (int j = 0; j < s; ++j) { c += (uint64_t)a[j] + b[j]; a[j] = (uint32_t)c; c >>= 32; }
  return (uint32_t)c;
}

// a -= b over s limbs, returns the borrow
PL_DEV uint32_t sub_1t(uint32_t* a, const uint32_t* b, int s) {
  int64_t br = 0;
  for (int j = 0; j < s; ++j) {
    const int64_t d = (int64_t)a[j] - b[j] - br;
    br = d < 0;
    a[j] = (uint32_t)d;
  }
  return (uint32_t)br;
}

// r[0 .. sa+sb) = a * b (schoolbook)
PL_DEV void mul_1t(uint32_t* r, const uint32_t* a, int sa, const uint32_t* b, int sb) {
  for (int j = 0; j < sa + sb; ++j) r[j] = 0;
  for (int i = 0; i < sb; ++i) {
    uint64_t c = 0;
    const uint32_t bi = b[i];
    for (int j = 0; j < sa; ++j) {
      c += (uint64_t)a[j] * bi + r[i + j];
      r[i + j] = (uint32_t)c;
      c >>= 32;
    }
    r[i + sa] = (uint32_t)c;
  }
}

// r[0 .. s) = a * b mod 2^(32 s)
PL_DEV void mul_lo_1t(uint32_t* r, const uint32_t* a, const uint32_t* b, int s) {
  for (int j = 0; j < s; ++j) r[j] = 0;
  for (int i = 0; i < s; ++i) {
    uint64_t c = 0;
    const uint32_t bi = b[i];
    for (int j = 0; i + j < s; ++j) {
      c += (uint64_t)a[j] * bi + r[i + j];
      r[i + j] = (uint32_t)c;
      c >>= 32;
    }
  }
}

}  // namespace pl
