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
