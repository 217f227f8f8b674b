// Key-holder kernels: fixed-point encode/decode, encryption and CRT
// decryption (Sec. III.B: the active party encrypts g/h and decrypts the
// returned histograms; Sec. III.C: one single-number encryption per g and h).
//
// Both encryption and decryption are dominated by one batched sliding-window
// exponentiation in the two CRT halves (mod p^2 and mod q^2, L limbs each),
// run by k_modexp with T lanes per instance.  The once-per-item steps around
// it (CRT recombination, exact division L_p) are one thread per item.
#include <cuda_runtime.h>

#include <cstring>

#include "check.cuh"
#include "internal.h"
#include "mp.cuh"

namespace pl {
namespace {

constexpr int kBlock = 128;

// m = rint(v 2^24) + 2^24, v in [-1, 2^15] (x 2^24 is exact in float32).
__global__ void k_encode(const float* __restrict__ v, size_t count, uint64_t* __restrict__ m, int* status) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float x = v[i];
    if (x >= -1.0f && x <= 32768.0f) {
      m[i] = (uint64_t)(__float2ll_rn(x * 16777216.0f) + (1ll << 24));
    } else {
      m[i] = 0;
      atomicOr(status, kStatusEncode);
    }
  }
}

// g/h packing: m = enc(g) + 2^B enc(h) as two little-endian 64-bit words
// (enc as k_encode), 26 <= B <= 64.
__global__ void k_encode_gh(const float* __restrict__ g, const float* __restrict__ h, size_t count, int B,
                            uint64_t* __restrict__ m, int* status) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float x = g[i], y = h[i];
    uint64_t eg = 0, eh = 0;
    if (x >= -1.0f && x <= 32768.0f && y >= -1.0f && y <= 32768.0f) {
      eg = (uint64_t)(__float2ll_rn(x * 16777216.0f) + (1ll << 24));
      eh = (uint64_t)(__float2ll_rn(y * 16777216.0f) + (1ll << 24));
      if (B < 64 && (eg >> B) != 0) atomicOr(status, kStatusRange);
    } else {
      atomicOr(status, kStatusEncode);
    }
    // eg + eh 2^B, eg < 2^B
    m[2 * i] = eg | (B < 64 ? eh << B : 0);
    m[2 * i + 1] = B < 64 ? eh >> (64 - B) : eh;
  }
}

__global__ void k_decode(const uint64_t* __restrict__ s, const int32_t* __restrict__ cnt, size_t count,
                         double* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const int64_t d = (int64_t)(s[i] - ((uint64_t)(uint32_t)cnt[i] << 24));
    out[i] = (double)d * (1.0 / 16777216.0);
  }
}

// Sliding-window exponentiation of one instance held by a group of T lanes.
// acc: the base in Montgomery form on entry, base^e in Montgomery form on exit,
// e given by its schedule op[0..nop) (layout in ModexpParams).  tbl: this
// group's table of 2^(w-1) entries of S*T limbs (the odd powers); bs: its
// shared-memory column.  Every op is one Montgomery product: at 4 lanes and up,
// the separated-form body mont_sos for squarings and products alike
// (one routine's code in the loop; a square forms each cross product once),
// else mont_mul with the multiplier staged in shared memory.  The table build
// runs once per exponentiation and keeps mont_mul.
template <int S, int T>
PL_DEV void window_exp(uint32_t (&acc)[S], const uint32_t (&n)[S], uint32_t np, const uint8_t* op, int nop, int w,
                       uint32_t* tbl, uint32_t* bs, int st, int k) {
  constexpr int NL = S * T;
  const int nent = 1 << (w - 1);
  uint32_t a[S], t[S];
  store_slice<S>(tbl, acc, k);  // base^1
  // base^2, staged as the multiplier of the table build
  __syncwarp();
  stage<S>(bs, st, acc, k);
  __syncwarp();
  mont_mul<S, T>(t, acc, bs, st, n, np, k);
  __syncwarp();
  stage<S>(bs, st, t, k);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < S; ++j) a[j] = acc[j];
  for (int e = 1; e < nent; ++e) {  // base^(2e + 1) = base^(2e - 1) base^2
    mont_mul<S, T>(t, a, bs, st, n, np, k);
    store_slice<S>(tbl + e * NL, t, k);
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = t[j];
  }
  // most significant window first; an entry past the table (checked builds)
  // reads entry 0 instead
  auto entry = [&](int v) { return PL_BOUNDS((v >> 1) < nent, kBoundsTable) ? (v >> 1) : 0; };
  load_slice_rw<S>(a, tbl + (size_t)entry(op[0]) * NL, k);
  for (int i = 1; i < nop; ++i) {
    const int v = op[i];  // the same for every instance of the warp
    if constexpr (kUseSos<S, T>) {
      if (v != 0) {
        load_slice_rw<S>(t, tbl + (size_t)entry(v) * NL, k);
      } else {
#pragma unroll
        for (int j = 0; j < S; ++j) t[j] = a[j];
      }
      mont_sos<S, T>(a, a, t, n, np, k, v == 0);
      continue;
    }
    __syncwarp();
    if (v == 0) {
      stage<S>(bs, st, a, k);
    } else {
      load_slice_rw<S>(t, tbl + (size_t)entry(v) * NL, k);
      stage<S>(bs, st, t, k);
    }
    __syncwarp();
    mont_mul<S, T>(t, a, bs, st, n, np, k);
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = t[j];
  }
#pragma unroll
  for (int j = 0; j < S; ++j) acc[j] = a[j];
}

// The first encryption stage of one instance on a group of T lanes holding S
// limbs each of the prime x (S T = L/2 limbs): z = (r mod x)^(x' mod (x - 1))
// mod x, canonical, returned in z; r is the L-limb row rrow.  A zero residue r
// mod x (gcd(r, n) != 1) sets kStatusNonUnit when status is given.
template <int S, int T>
PL_DEV void enc_stage1(uint32_t (&z)[S], const HalfConst& H, const uint8_t* op1, int nop1, int w,
                       const uint32_t* rrow, uint32_t* mytbl, uint32_t* bs, int st, int k, bool valid, int gw,
                       int* status) {
  constexpr int NLh = S * T;
  uint32_t nx[S], tx[S];
  const_slice<S>(nx, H.Nx, k);
  const uint32_t npx = H.npx;
  // r = r_lo + r_hi Rx: Montgomery form (r mod x) Rx = mont(r_lo, Rx^2) + mont(r_hi, Rx^3)
  load_slice<S>(z, rrow, k);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < S; ++j) bs[(k * S + j) * st] = H.R2x[k * S + j];
  __syncwarp();
  mont_mul<S, T>(tx, z, bs, st, nx, npx, k);
  store_slice<S>(mytbl, tx, k);
  load_slice<S>(z, rrow + NLh, k);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < S; ++j) bs[(k * S + j) * st] = H.R3x[k * S + j];
  __syncwarp();
  mont_mul<S, T>(tx, z, bs, st, nx, npx, k);
  load_slice_rw<S>(z, mytbl, k);
  add_cc(tx[0], z[0]);
#pragma unroll
  for (int j = 1; j < S; ++j) addc_cc(tx[j], z[j]);
  const uint32_t c = carry_out();
  normalize<S, T>(tx, c, 0u, nx, k, kFull);
  if (status != nullptr) {
    // gcd(r, n) = 1 exactly when r mod p and r mod q are both non-zero
    uint32_t any = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) any |= tx[j];
    const unsigned nz = __ballot_sync(kFull, any != 0u);
    const unsigned gm = (T == 32) ? kFull : ((1u << T) - 1u);
    if (valid && k == 0 && ((nz >> (gw * T)) & gm) == 0u) atomicOr(status, kStatusNonUnit);
  }
  window_exp<S, T>(tx, nx, npx, op1, nop1, w, mytbl, bs, st, k);
  // leave Montgomery form mod x
  __syncwarp();
#pragma unroll
  for (int j = 0; j < S; ++j) bs[(k * S + j) * st] = (k * S + j == 0) ? 1u : 0u;
  __syncwarp();
  mont_mul<S, T>(z, tx, bs, st, nx, npx, k);
}

// Batched exponentiation in the CRT halves.  Instance (h, i): half h (prime
// x = p or q), item i.  A warp takes 32/T consecutive items of one half, so the
// exponent schedules are warp-uniform.
//   ENC: y[h][i] = (1 + m_i n) r_i^n mod x^2          (in = r [count][L])
//        with r^n mod x^2 = ((r mod x)^(x' mod (x - 1)) mod x)^x mod x^2, x' the
//        other prime: Fermat gives r^x' = r^(x' mod (x-1)) mod x, and z^x mod x^2
//        depends only on z mod x (every term of (z + k x)^x after the first has
//        x^2 as a factor).  One exponent of n_bits/2 bits mod x (L/2 limbs) and
//        one of n_bits/2 bits mod x^2 replace one of n_bits bits mod x^2.
//   DEC: y[h][i] = c_i^(x - 1) mod x^2                (in = c [count][2L])
// Every value is canonical.  tbl: per-group window table, 2^(w-1) entries of
// L limbs for each group of the grid.
// STAGE (encryption only) splits the two exponentiations over two launches so
// that each runs at its own lanes per instance: STAGE 1 computes z = (r mod
// x)^(x' mod (x - 1)) mod x alone (S T = L/2 limbs; out = z [2][count][L/2]),
// STAGE 2 the rest from z (in = z; S T = L limbs); STAGE 0 does both.
template <int S, int T, bool DEC, int STAGE = 0>
__global__ void __launch_bounds__(kBlock) k_modexp(const __grid_constant__ ModexpParams P,
                                                   const uint32_t* __restrict__ in, const uint64_t* __restrict__ msg,
                                                   int mw, uint32_t* __restrict__ out, uint32_t* __restrict__ tbl,
                                                   size_t count, int* status) {
  constexpr int NL = S * T;
  constexpr int IPW = 32 / T;
  extern __shared__ uint32_t smem[];
  const int ipb = blockDim.x / T;
  const int lane = threadIdx.x & 31;
  const int k = lane % T;
  const int gw = lane / T;
  const int g = threadIdx.x / T;
  uint32_t* bs = smem + g;
  const int st = ipb;
  const int w = P.w;
  uint32_t* mytbl = tbl + ((size_t)blockIdx.x * ipb + g) * table_entries(w) * NL;
  const size_t nchunk = (count + IPW - 1) / IPW;
  const size_t nitems = 2 * nchunk;
  const size_t warp0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;

  for (size_t item = warp0; item < nitems; item += nwarps) {
    const int h = (int)(item & 1);
    const size_t i = (item >> 1) * IPW + gw;
    const bool valid = i < count;
    const size_t ii = valid ? i : count - 1;
    const HalfConst& H = P.half[h];
    if constexpr (STAGE == 1) {
      uint32_t z[S];
      enc_stage1<S, T>(z, H, P.op1[h], P.nop1[h], w, in + ii * 2 * NL, mytbl, bs, st, k, valid, gw, status);
      if (valid) store_slice<S>(out + ((size_t)h * count + ii) * NL, z, k);
      continue;
    }
    uint32_t n[S], a[S], t[S];
    const_slice<S>(n, H.N, k);
    const uint32_t np = H.np;
    uint32_t* yrow = out + ((size_t)h * count + ii) * NL;

    if constexpr (!DEC) {
      // post-factor (1 + m n) mod x^2 = mont(nR, m) + 1, parked in the output row;
      // m has mw (1 or 2) little-endian 64-bit words
      const uint64_t m = msg[ii * mw];
      const uint64_t mh = mw == 2 ? msg[ii * 2 + 1] : 0;
      __syncwarp();
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const int idx = k * S + j;
        const uint64_t word = idx < 2 ? m : mh;
        bs[idx * st] = idx < 4 ? (uint32_t)(word >> (32 * (idx & 1))) : 0u;
      }
      __syncwarp();
      const_slice<S>(a, H.nR, k);
      mont_mul<S, T>(t, a, bs, st, n, np, k);
      normalize<S, T>(t, 0u, 1u, n, k, kFull);
      if (valid) store_slice<S>(yrow, t, k);

      if constexpr (STAGE == 0) {
        // stage 1, mod x on L/2 limbs; z (< x) into the L-limb layout of stage 2, zero-extended
        constexpr int S2 = S / 2;
        constexpr int NLh = S2 * T;
        uint32_t z[S2];
        enc_stage1<S2, T>(z, H, P.op1[h], P.nop1[h], w, in + ii * NL, mytbl, bs, st, k, valid, gw, status);
        __syncwarp();
        stage<S2>(bs, st, z, k);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < S; ++j) {
          const int idx = k * S + j;
          a[j] = idx < NLh ? bs[idx * st] : 0u;
        }
      } else {
        // z from the first-stage launch: lanes below T/2 hold its L/2 limbs, the rest zero
        static_assert(STAGE != 2 || T % 2 == 0, "the second stage needs an even number of lanes");
        if (k < T / 2) {
          load_slice<S>(a, in + ((size_t)h * count + ii) * (NL / 2), k);
        } else {
#pragma unroll
          for (int j = 0; j < S; ++j) a[j] = 0u;
        }
      }
      // stage 2 base: z R mod x^2
      __syncwarp();
#pragma unroll
      for (int j = 0; j < S; ++j) bs[(k * S + j) * st] = H.R2[k * S + j];
      __syncwarp();
      mont_mul<S, T>(t, a, bs, st, n, np, k);
    } else {
      // c = c_lo + c_hi R: Montgomery form c R = mont(c_lo, R^2) + mont(c_hi, R^3)
      load_slice<S>(a, in + ii * 2 * NL, k);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < S; ++j) bs[(k * S + j) * st] = H.R2[k * S + j];
      __syncwarp();
      mont_mul<S, T>(t, a, bs, st, n, np, k);
      store_slice<S>(mytbl, t, k);
      load_slice<S>(a, in + ii * 2 * NL + NL, k);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < S; ++j) bs[(k * S + j) * st] = H.R3[k * S + j];
      __syncwarp();
      mont_mul<S, T>(t, a, bs, st, n, np, k);
      load_slice_rw<S>(a, mytbl, k);
      add_cc(t[0], a[0]);
#pragma unroll
      for (int j = 1; j < S; ++j) addc_cc(t[j], a[j]);
      const uint32_t c = carry_out();
      normalize<S, T>(t, c, 0u, n, k, kFull);
    }

    // exponentiation mod x^2: exponent x (ENC) or x - 1 (DEC)
    window_exp<S, T>(t, n, np, P.op[h], P.nop[h], w, mytbl, bs, st, k);
#pragma unroll
    for (int j = 0; j < S; ++j) a[j] = t[j];

    // leave Montgomery form: times the post factor (ENC) or times 1 (DEC)
    __syncwarp();
    if constexpr (!DEC) {
      load_slice_rw<S>(t, yrow, k);
      stage<S>(bs, st, t, k);
    } else {
#pragma unroll
      for (int j = 0; j < S; ++j) bs[(k * S + j) * st] = (k * S + j == 0) ? 1u : 0u;
    }
    __syncwarp();
    mont_mul<S, T>(t, a, bs, st, n, np, k);
    if (valid) store_slice<S>(yrow, t, k);
  }
}

// c = y_q + q^2 ((y_p - y_q) (q^2)^-1 mod p^2), one thread per ciphertext.
__global__ void __launch_bounds__(kBlock) k_enc_crt(const __grid_constant__ EncCrtParams P,
                                                    const uint32_t* __restrict__ y, size_t count,
                                                    uint32_t* __restrict__ ct) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int L = P.L;
  const uint32_t* yp = y + i * L;
  const uint32_t* yq = y + (count + i) * L;
  uint32_t d[kMaxL], u[kMaxL], c[2 * kMaxL];
  for (int j = 0; j < L; ++j) d[j] = yp[j];
  if (sub_1t(d, yq, L)) {  // y_q may exceed y_p (and p^2): add p^2 until non-negative
    if (!add_1t(d, P.p2, L)) add_1t(d, P.p2, L);
  }
  mm_1t(u, d, P.QinvR, P.p2, P.p2_np, L);
  mul_1t(c, P.q2, L, u, L);
  uint64_t cy = 0;
  for (int j = 0; j < 2 * L; ++j) {
    cy += (uint64_t)c[j] + (j < L ? yq[j] : 0u);
    c[j] = (uint32_t)cy;
    cy >>= 32;
  }
  uint32_t* o = ct + i * 2 * L;
  for (int j = 0; j < 2 * L; j += 4) *reinterpret_cast<uint4*>(o + j) = make_uint4(c[j], c[j + 1], c[j + 2], c[j + 3]);
}

// m_p = L_p(y_p) h_p mod p (L_p an exact division done as a product with
// p^-1 mod 2^(32 Lh)), m_q likewise, m = m_q + q ((m_p - m_q) q^-1 mod p).
template <bool U64>
__global__ void __launch_bounds__(kBlock) k_dec_crt(const __grid_constant__ DecCrtParams P,
                                                    const uint32_t* __restrict__ y, size_t count, int L,
                                                    void* __restrict__ outp, int* status) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int Lh = P.Lh;
  uint32_t x[kMaxLh], lx[kMaxLh], mp[kMaxLh], mq[kMaxLh], u[kMaxLh], m[kMaxL];
  for (int half = 0; half < 2; ++half) {
    const uint32_t* yr = y + ((size_t)half * count + i) * L;
    for (int j = 0; j < Lh; ++j) x[j] = yr[j];
    // x - 1 mod 2^(32 Lh)
    for (int j = 0; j < Lh; ++j) {
      const uint32_t old = x[j];
      x[j] = old - 1u;
      if (old != 0) break;
    }
    mul_lo_1t(lx, x, half ? P.qinv2k : P.pinv, Lh);
    if (half == 0)
      mm_1t(mp, lx, P.hpR, P.p, P.p_np, Lh);
    else
      mm_1t(mq, lx, P.hqR, P.q, P.q_np, Lh);
  }
  // (m_p - m_q) mod p, with m_q < q < 2p
  for (int j = 0; j < Lh; ++j) x[j] = mp[j];
  if (sub_1t(x, mq, Lh)) {
    if (!add_1t(x, P.p, Lh)) add_1t(x, P.p, Lh);
  }
  mm_1t(u, x, P.qinvR, P.p, P.p_np, Lh);
  mul_1t(m, P.q, Lh, u, Lh);
  uint64_t cy = 0;
  for (int j = 0; j < L; ++j) {
    cy += (uint64_t)m[j] + (j < Lh ? mq[j] : 0u);
    m[j] = (uint32_t)cy;
    cy >>= 32;
  }
  if constexpr (U64) {
    uint32_t hi = 0;
    for (int j = 2; j < L; ++j) hi |= m[j];
    uint64_t* o = reinterpret_cast<uint64_t*>(outp);
    if (hi) {
      o[i] = ~0ull;
      atomicOr(status, kStatusRange);
    } else {
      o[i] = (uint64_t)m[0] | ((uint64_t)m[1] << 32);
    }
  } else {
    uint32_t* o = reinterpret_cast<uint32_t*>(outp) + i * L;
    for (int j = 0; j < L; j += 4) *reinterpret_cast<uint4*>(o + j) = make_uint4(m[j], m[j + 1], m[j + 2], m[j + 3]);
  }
}

// ---------------------------------------------------------------------------
// launch helpers

template <int S, int T, bool DEC, int STAGE = 0>
pl_status run_modexp(const ModexpParams* P, const uint32_t* in, const uint64_t* msg, int mw, uint32_t* y,
                     uint32_t* tbl, int grid, size_t count, int* status, cudaStream_t s) {
  const int ipb = kBlock / T;
  const size_t smem = (size_t)S * T * ipb * sizeof(uint32_t);
  {
    ProfScope _ps(DEC ? "modexp_dec" : (STAGE == 1 ? "modexp_enc1" : "modexp_enc"), s);
    k_modexp<S, T, DEC, STAGE><<<grid, kBlock, smem, s>>>(*P, in, msg, mw, y, tbl, count, status);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

template <int S, int T, bool DEC, int STAGE = 0>
int modexp_grid() {
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    const int ipb = kBlock / T;
    const size_t smem = (size_t)S * T * ipb * sizeof(uint32_t);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_modexp<S, T, DEC, STAGE>, kBlock, smem) !=
            cudaSuccess ||
        b < 1)
      b = 1;
    blocks_per_sm = b;
  }
  return blocks_per_sm * sm_count();
}

// dispatch on (limbs per half L, lanes per instance T)
template <bool DEC>
pl_status modexp_dispatch(int L, int T, int* grid_out, bool launch, const ModexpParams* P, const uint32_t* in,
                          const uint64_t* msg, uint32_t* y, uint32_t* tbl, size_t count, cudaStream_t s,
                          int mw = 1, int* status = nullptr) {
#define PL_CASE(LL, TT)                                                            \
  if (L == LL && T == TT) {                                                        \
    if (!launch) { *grid_out = modexp_grid<LL / TT, TT, DEC>(); return PL_OK; }     \
    return run_modexp<LL / TT, TT, DEC>(P, in, msg, mw, y, tbl, *grid_out, count, status, s); \
  }
  PL_CASE(32, 2)
  PL_CASE(32, 4)
  PL_CASE(64, 2)
  PL_CASE(64, 4)
  PL_CASE(64, 8)
  PL_CASE(96, 4)
  PL_CASE(96, 8)
  if constexpr (DEC) {  // 6 limbs per lane: decryption only (encryption's first stage needs an even half)
    PL_CASE(96, 16)
  }
#undef PL_CASE
  return fail(PL_EINVAL, "no exponentiation kernel for this (limbs, lanes) pair");
}

// Encryption split over two launches (STAGE 1, then 2) where both kernels
// exist: the first stage at half the lanes of the second (2048-bit: 2 lanes of
// 16 limbs mod x, then 4 of 16 mod x^2; 3072-bit: 4 of 12, then 8 of 12).
bool enc_split(int L, int T) { return (L == 64 && T == 4) || (L == 96 && T == 8); }

// STAGE 1 dispatch on (limbs of x, lanes) and STAGE 2 on (limbs of x^2, lanes)
template <int STAGE>
pl_status enc_stage_dispatch(int L, int T, int* grid_out, bool launch, const ModexpParams* P, const uint32_t* in,
                             const uint64_t* msg, uint32_t* y, uint32_t* tbl, size_t count, cudaStream_t s, int mw,
                             int* status) {
#define PL_CASE(LL, TT)                                                                            \
  if (L == LL && T == TT) {                                                                        \
    if (!launch) { *grid_out = modexp_grid<LL / TT, TT, false, STAGE>(); return PL_OK; }            \
    return run_modexp<LL / TT, TT, false, STAGE>(P, in, msg, mw, y, tbl, *grid_out, count, status, s); \
  }
  if constexpr (STAGE == 1) {
    PL_CASE(32, 2)
    PL_CASE(48, 4)
  } else {
    PL_CASE(64, 4)
    PL_CASE(96, 8)
  }
#undef PL_CASE
  return fail(PL_EINVAL, "no split encryption kernel for this (limbs, lanes) pair");
}

}  // namespace

bool modexp_supported(int L, int T) {
  return (L == 32 && (T == 2 || T == 4)) || (L == 64 && (T == 2 || T == 4 || T == 8)) ||
         (L == 96 && (T == 4 || T == 8));
}

pl_status launch_encode(const float* d_v, size_t count, uint64_t* d_m, int* st, cudaStream_t s) {
  if (count == 0) return PL_OK;
  const int grid = (int)std::min<size_t>((count + 255) / 256, (size_t)sm_count() * 8);
  {
    ProfScope _ps("encode", s);
    k_encode<<<grid, 256, 0, s>>>(d_v, count, d_m, st);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status launch_encode_gh(const float* d_g, const float* d_h, size_t count, int B, uint64_t* d_m, int* st,
                           cudaStream_t s) {
  if (count == 0) return PL_OK;
  const int grid = (int)std::min<size_t>((count + 255) / 256, (size_t)sm_count() * 8);
  {
    ProfScope _ps("encode", s);
    k_encode_gh<<<grid, 256, 0, s>>>(d_g, d_h, count, B, d_m, st);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status launch_decode(const uint64_t* d_s, const int32_t* d_cnt, size_t count, double* d_out, cudaStream_t s) {
  if (count == 0) return PL_OK;
  const int grid = (int)std::min<size_t>((count + 255) / 256, (size_t)sm_count() * 8);
  {
    ProfScope _ps("decode", s);
    k_decode<<<grid, 256, 0, s>>>(d_s, d_cnt, count, d_out);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

// Shared by encrypt and decrypt: scratch = y [2][count][L] + window tables.
// Lanes per instance for a call on `count` items: the configured lanes, or twice
// as many when the call is too small to keep the GPU's multiply-add pipes busy
// and that kernel exists (fewer, faster instances: shorter latency for small
// calls; the results do not depend on it).
template <bool DEC>
ModexpCfg lanes_for_count(int L, ModexpCfg cfg, size_t count) {
  const bool have = modexp_supported(L, 2 * cfg.T) || (DEC && L == 96 && 2 * cfg.T == 16);
  // 2 count instances: the two CRT halves
  if (have && double_lanes_pays(2 * count, cfg.T)) cfg.T *= 2;
  return cfg;
}

// grid of a launch on `count` items at T lanes: no more blocks than items need
static int trim_grid(int grid, size_t count, int T) {
  const size_t ipw = 32 / (size_t)T;
  const size_t warps_needed = 2 * ((count + ipw - 1) / ipw);
  const size_t blocks_needed = (warps_needed + (kBlock / 32) - 1) / (kBlock / 32);
  return (size_t)grid > blocks_needed ? (int)blocks_needed : grid;
}

// Encryption as two launches (enc_split): z [2][count][L/2], then y.
static pl_status enc_phase_split(pl_key* key, ModexpCfg cfg, const ModexpParams* P, const uint32_t* d_r,
                                 const uint64_t* msg, size_t count, uint32_t** y_out, cudaStream_t s,
                                 Scratch* scratch, int mw, int* st) {
  const int L = key->L, T1 = cfg.T / 2;
  int g1 = 0, g2 = 0;
  pl_status rc = enc_stage_dispatch<1>(L / 2, T1, &g1, false, P, nullptr, nullptr, nullptr, nullptr, 0, s, mw, st);
  if (rc) return rc;
  rc = enc_stage_dispatch<2>(L, cfg.T, &g2, false, P, nullptr, nullptr, nullptr, nullptr, 0, s, mw, st);
  if (rc) return rc;
  g1 = trim_grid(g1, count, T1);
  g2 = trim_grid(g2, count, cfg.T);
  // the window tables of the two launches share one region
  const size_t tb1 = (size_t)g1 * (kBlock / T1) * table_entries(cfg.w) * (L / 2);
  const size_t tb2 = (size_t)g2 * (kBlock / cfg.T) * table_entries(cfg.w) * L;
  Carve cv;
  const size_t off_y = cv.take((size_t)2 * count * L * sizeof(uint32_t));
  const size_t off_z = cv.take((size_t)count * L * sizeof(uint32_t));
  const size_t off_t = cv.take(std::max(tb1, tb2) * sizeof(uint32_t));
  Scratch* sc = scratch ? scratch : key->scratch_for_current_device();
  if (!sc) return fail(PL_ECUDA, "no current device");
  char* base = static_cast<char*>(sc->get(cv.off, s));
  if (!base) return fail(PL_ENOMEM, "scratch allocation failed");
  uint32_t* y = reinterpret_cast<uint32_t*>(base + off_y);
  uint32_t* z = reinterpret_cast<uint32_t*>(base + off_z);
  uint32_t* tbl = reinterpret_cast<uint32_t*>(base + off_t);
  rc = enc_stage_dispatch<1>(L / 2, T1, &g1, true, P, d_r, msg, z, tbl, count, s, mw, st);
  if (rc) return rc;
  rc = enc_stage_dispatch<2>(L, cfg.T, &g2, true, P, z, msg, y, tbl, count, s, mw, st);
  *y_out = y;
  return rc;
}

template <bool DEC>
static pl_status modexp_phase(pl_key* key, ModexpCfg cfg, const uint32_t* in, const uint64_t* msg,
                              size_t count, uint32_t** y_out, cudaStream_t s, Scratch* scratch, int mw = 1,
                              int* st = nullptr) {
  cfg = lanes_for_count<DEC>(key->L, cfg, count);
  const ModexpParams* P = key->modexp_params(DEC, cfg.w);
  if (!P) return fail(PL_EINVAL, "unsupported window width");
  const int L = key->L;
  if constexpr (!DEC) {
    if (enc_split(L, cfg.T)) return enc_phase_split(key, cfg, P, in, msg, count, y_out, s, scratch, mw, st);
  }
  int grid = 0;
  pl_status rc = modexp_dispatch<DEC>(L, cfg.T, &grid, false, P, nullptr, nullptr, nullptr, nullptr, 0, s);
  if (rc) return rc;
  grid = trim_grid(grid, count, cfg.T);
  const size_t ipb = kBlock / cfg.T;
  Carve cv;
  const size_t off_y = cv.take((size_t)2 * count * L * sizeof(uint32_t));
  const size_t off_t = cv.take((size_t)grid * ipb * table_entries(cfg.w) * L * sizeof(uint32_t));
  Scratch* sc = scratch ? scratch : key->scratch_for_current_device();
  if (!sc) return fail(PL_ECUDA, "no current device");
  char* base = static_cast<char*>(sc->get(cv.off, s));
  if (!base) return fail(PL_ENOMEM, "scratch allocation failed");
  uint32_t* y = reinterpret_cast<uint32_t*>(base + off_y);
  uint32_t* tbl = reinterpret_cast<uint32_t*>(base + off_t);
  rc = modexp_dispatch<DEC>(L, cfg.T, &grid, true, P, in, msg, y, tbl, count, s, mw, st);
  *y_out = y;
  return rc;
}

pl_status launch_encrypt(pl_key* key, const uint64_t* d_m, const uint32_t* d_r, size_t count, uint32_t* d_ct,
                         int* st, cudaStream_t s, Scratch* scratch, int mw) {
  if (count == 0) return PL_OK;
  uint32_t* y = nullptr;
  pl_status rc = modexp_phase<false>(key, key->enc_cfg, d_r, d_m, count, &y, s, scratch, mw, st);
  if (rc) return rc;
  {
    ProfScope _ps("enc_crt", s);
    k_enc_crt<<<(unsigned)((count + kBlock - 1) / kBlock), kBlock, 0, s>>>(key->enc, y, count, d_ct);
  }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

size_t decrypt_scratch_bytes(const pl_key* key, size_t count) {
  // the same carve as modexp_phase<true>: y [2][count][L] plus the window
  // tables of the grid that launch will use
  const int L = key->L;
  const ModexpCfg cfg = lanes_for_count<true>(L, key->dec_cfg, count);
  int grid = 0;
  if (modexp_dispatch<true>(L, cfg.T, &grid, false, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr)) return 0;
  grid = trim_grid(grid, count, cfg.T);
  const size_t ipb = kBlock / cfg.T;
  Carve cv;
  cv.take((size_t)2 * count * L * sizeof(uint32_t));
  cv.take((size_t)grid * ipb * table_entries(cfg.w) * L * sizeof(uint32_t));
  return cv.off;
}

pl_status launch_decrypt(pl_key* key, const uint32_t* d_ct, size_t count, void* d_out, bool u64, int* st,
                         cudaStream_t s, Scratch* scratch) {
  if (count == 0) return PL_OK;
  uint32_t* y = nullptr;
  pl_status rc = modexp_phase<true>(key, key->dec_cfg, d_ct, nullptr, count, &y, s, scratch);
  if (rc) return rc;
  const unsigned grid = (unsigned)((count + kBlock - 1) / kBlock);
  if (u64)
    {
      ProfScope _ps("dec_crt", s);
      k_dec_crt<true><<<grid, kBlock, 0, s>>>(key->dec, y, count, key->L, d_out, st);
    }
  else
    {
      ProfScope _ps("dec_crt", s);
      k_dec_crt<false><<<grid, kBlock, 0, s>>>(key->dec, y, count, key->L, d_out, st);
    }
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

}  // namespace pl

// ---------------------------------------------------------------------------
// Allocation-free CRT decryption to uint64 (paillier_decrypt_u64_noalloc).
//
// For callers that must not allocate device memory, the scratch this path
// needs (the two CRT half results and the per-instance window tables) lives in
// one file-scope device array instead of the key's scratch buffer.  The array
// is part of the library's device image: every GPU that loads the library
// holds it (about 21 MB) until the process exits.
namespace pl {
namespace {

constexpr size_t kNaMaxCount = 8192;  // ciphertexts per call
constexpr int kNaWindow = 4;          // window bits
constexpr size_t kNaYWords = 2 * kNaMaxCount * kMaxL;  // y[2][count][L]
// Window tables for this many instances running at once (each instance owns
// table_entries(kNaWindow) = 8 entries of up to kMaxL limbs); the launch grid
// is cut so that no more instances than this are resident, whatever the GPU.
constexpr size_t kNaTableSlots = 4736;
constexpr size_t kNaTblWords = kNaTableSlots * table_entries(kNaWindow) * kMaxL;
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) uint32_t g_na_scratch[kNaYWords + kNaTblWords];
static __device__ int g_na_status;  // range errors of this path (write-only sink)

std::mutex g_na_mu;
uint32_t* g_na_scratch_ptr[kNaMaxDevices] = {};
int* g_na_status_ptr[kNaMaxDevices] = {};

// Once per device, with that device current: device addresses of the arrays.
pl_status na_setup(int dev, uint32_t** scratch, int** status) {
  if (dev < 0 || dev >= kNaMaxDevices) return fail(PL_EINVAL, "device ordinal out of range for the allocation-free path");
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_na_status);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(status)");
    g_na_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    g_na_status_ptr[dev] = static_cast<int*>(q);
  }
  *scratch = g_na_scratch_ptr[dev];
  *status = g_na_status_ptr[dev];
  return PL_OK;
}

}  // namespace
}  // namespace pl

extern "C" pl_status paillier_decrypt_u64_noalloc(const pl_key* key, const uint32_t* d_ct, size_t count,
                                                  uint64_t* d_m, void* stream) {
  using namespace pl;
  clear_error();
  if (!key) return fail(PL_EINVAL, "key is NULL");
  if (!key->priv) return fail(PL_EINVAL, "decryption needs the private key");
  if (count == 0) return PL_OK;
  if (count > kNaMaxCount)
    return fail(PL_EINVAL, "count exceeds the allocation-free maximum of 8192 ciphertexts per call");
  if (!d_ct || !d_m) return fail(PL_EINVAL, "NULL buffer");
  if ((reinterpret_cast<uintptr_t>(d_ct) & 15u) || (reinterpret_cast<uintptr_t>(d_m) & 15u))
    return fail(PL_EINVAL, "buffers must be 16-byte aligned");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
  uint32_t* scratch = nullptr;
  int* status = nullptr;
  pl_status rc = na_setup(dev, &scratch, &status);
  if (rc) return rc;
  const int L = key->L;
  const int T = key->dec_cfg.T;
  // schedules of p - 1 and q - 1 at this path's window width, built on the stack
  ModexpParams P;
  std::memset(&P, 0, sizeof(P));
  for (int h = 0; h < 2; ++h) {
    P.half[h] = key->half[h];
    P.nop[h] = sliding_schedule(key->e_dec[h], kNaWindow, P.op[h], kMaxOps);
    if (P.nop[h] < 0) return fail(PL_EINVAL, "exponent too long");
  }
  P.w = kNaWindow;
  int grid = 0;
  rc = modexp_dispatch<true>(L, T, &grid, false, &P, nullptr, nullptr, nullptr, nullptr, 0, nullptr);
  if (rc) return rc;
  // the table slots the array holds for this key size bound the grid
  const size_t ipb = kBlock / T;
  const size_t slots = kNaTblWords / (table_entries(kNaWindow) * L);
  const size_t ipw = 32 / (size_t)T;
  const size_t warps_needed = 2 * ((count + ipw - 1) / ipw);
  const size_t blocks_needed = (warps_needed + (kBlock / 32) - 1) / (kBlock / 32);
  size_t g = std::min<size_t>((size_t)grid, slots / ipb);
  g = std::min(g, blocks_needed);
  grid = (int)std::max<size_t>(g, 1);
  uint32_t* y = scratch;
  uint32_t* tbl = scratch + kNaYWords;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = modexp_dispatch<true>(L, T, &grid, true, &P, d_ct, nullptr, y, tbl, count, s);
  if (rc) return rc;
  k_dec_crt<true><<<(unsigned)((count + kBlock - 1) / kBlock), kBlock, 0, s>>>(key->dec, y, count, L, d_m, status);
  note_launch();
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_fail(ce, "k_dec_crt");
  return PL_OK;
}
