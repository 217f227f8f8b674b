// CKKS for the secure horizontal pattern: negacyclic NTT over one 62-bit prime,
// canonical-embedding encoding/decoding, public-key encryption, addition and
// decryption (see include/ckks.h).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/ckks.h"
#include "check.cuh"
#include "internal.h"

namespace {

using u64 = uint64_t;
using u128 = unsigned __int128;

// ---- host modular arithmetic (set-up only) ---------------------------------
u64 h_mul(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 h_pow(u64 a, u64 e, u64 q) {
  u64 r = 1;
  a %= q;
  while (e) {
    if (e & 1) r = h_mul(r, a, q);
    a = h_mul(a, a, q);
    e >>= 1;
  }
  return r;
}
bool h_prime(u64 n) {  // deterministic Miller-Rabin for 64-bit n
  if (n < 2) return false;
  for (u64 p : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull})
    if (n % p == 0) return n == p;
  u64 d = n - 1;
  int s = 0;
  while (!(d & 1)) { d >>= 1; ++s; }
  for (u64 a : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
    u64 x = h_pow(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool ok = false;
    for (int r = 1; r < s; ++r) {
      x = h_mul(x, x, n);
      if (x == n - 1) { ok = true; break; }
    }
    if (!ok) return false;
  }
  return true;
}
int bitrev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// ---- device arithmetic mod q < 2^62, Montgomery with R = 2^64 ---------------
__device__ __forceinline__ u64 mmul(u64 a, u64 b, u64 q, u64 qn) {  // a b 2^-64 mod q
  const u64 lo = a * b, hi = __umul64hi(a, b);
  const u64 m = lo * qn;
  const u64 t = hi + __umul64hi(m, q) + (lo != 0 ? 1ull : 0ull);
  return t >= q ? t - q : t;
}
__device__ __forceinline__ u64 addm(u64 a, u64 b, u64 q) { const u64 s = a + b; return s >= q ? s - q : s; }
__device__ __forceinline__ u64 subm(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
__device__ __forceinline__ u64 smod(long long x, u64 q) {  // signed small or large -> [0, q)
  const long long r = x % (long long)q;
  return r < 0 ? (u64)(r + (long long)q) : (u64)r;
}
// the same for a 64-bit value that is usually smaller than q in magnitude
// (encoded plaintext coefficients): one conditional add then, else the remainder
__device__ __forceinline__ u64 smod64(long long x, u64 q) {
  const u64 ax = x < 0 ? (u64)(-(x + 1)) + 1u : (u64)x;  // |x|, also for INT64_MIN
  if (ax < q) return x < 0 ? q - ax : ax;
  return smod(x, q);
}
// the same for a 32-bit value: one conditional add when |x| < q is certain
// (q > 2^31; q is the same for every thread, so the branch is uniform)
__device__ __forceinline__ u64 smod32(int32_t x, u64 q) {
  if (q > 0x80000000ull) return x < 0 ? q - (u64)(-(long long)x) : (u64)x;
  return smod(x, q);
}

struct NttConst {
  u64 q, qn, r2;
  u64 ninv;    // N^-1, Montgomery form
  u64 last;    // inverse twiddle of the last Gentleman-Sande stage times N^-1, Montgomery form
  int log_n;
};

constexpr int kMaxLogN = 13;  // one polynomial (or two) resident in shared memory per CTA
constexpr int kThreads = 1024;

// ---- negacyclic NTT on a shared-memory polynomial (all threads of the CTA) --
// Forward: Cooley-Tukey, natural order in, bit-reversed order out; the stage
// with butterfly distance t has N/(2t) blocks, block i using psi^bitrev(N/(2t)+i)
// (table tw, Montgomery form).  Inverse: Gentleman-Sande with psi^-bitrev
// (table itw) back to natural order, the factor N^-1 folded into the last
// stage.  Three consecutive stages run in registers on 8 elements per thread
// (one barrier per three stages); the one or two stages left over run as plain
// radix-2 stages.  Both expect the input visible to all threads and end with a
// barrier.

__device__ __forceinline__ void ct_bfly(u64& x, u64& y, u64 w, const NttConst& C) {
  const u64 v = mmul(y, w, C.q, C.qn);
  y = subm(x, v, C.q);
  x = addm(x, v, C.q);
}

__device__ __forceinline__ void gs_bfly(u64& x, u64& y, u64 w, const NttConst& C) {
  const u64 s = addm(x, y, C.q);
  y = mmul(subm(x, y, C.q), w, C.q, C.qn);
  x = s;
}

// the last inverse stage: both outputs times N^-1 (C.last = psi^-bitrev(1) N^-1)
__device__ __forceinline__ void gs_last(u64& x, u64& y, const NttConst& C) {
  const u64 s = addm(x, y, C.q);
  y = mmul(subm(x, y, C.q), C.last, C.q, C.qn);
  x = mmul(s, C.ninv, C.q, C.qn);
}

// L: log2 of the transformed length (C.log_n for a whole polynomial; less for
// the slice of one CTA of a cluster, see below).
__device__ void ntt_fwd8(u64* a, const u64* tw, const NttConst& C, int L) {
  const int N = 1 << L;
  int lt = L - 1;  // log2 of the butterfly distance of the next stage
  for (; lt >= 2; lt -= 3) {
    // distances t, t/2, t/4 on e_k = 2t i + j + k t/4 (k < 8, j < t/4)
    const int q4 = lt - 2, m = N >> (lt + 1);
    for (int g = threadIdx.x; g < N / 8; g += blockDim.x) {
      const int i = g >> q4, j = g & ((1 << q4) - 1);
      const int base = (i << (lt + 1)) + j;
      u64 x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = a[base + (k << q4)];
      const u64 w1 = tw[m + i];
#pragma unroll
      for (int k = 0; k < 4; ++k) ct_bfly(x[k], x[k + 4], w1, C);
      const u64 w2a = tw[2 * m + 2 * i], w2b = tw[2 * m + 2 * i + 1];
      ct_bfly(x[0], x[2], w2a, C);
      ct_bfly(x[1], x[3], w2a, C);
      ct_bfly(x[4], x[6], w2b, C);
      ct_bfly(x[5], x[7], w2b, C);
#pragma unroll
      for (int k = 0; k < 4; ++k) ct_bfly(x[2 * k], x[2 * k + 1], tw[4 * m + 4 * i + k], C);
#pragma unroll
      for (int k = 0; k < 8; ++k) a[base + (k << q4)] = x[k];
    }
    __syncthreads();
  }
  for (; lt >= 0; --lt) {
    const int m = N >> (lt + 1);
    for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
      const int i = b >> lt, idx = (i << (lt + 1)) + (b & ((1 << lt) - 1));
      u64 x = a[idx], y = a[idx + (1 << lt)];
      ct_bfly(x, y, tw[m + i], C);
      a[idx] = x;
      a[idx + (1 << lt)] = y;
    }
    __syncthreads();
  }
}

// inverse transform of one or two polynomials (b may be NULL); the work items
// of both polynomials are spread over the threads together
__device__ void ntt_inv8(u64* a, u64* b, const u64* itw, const NttConst& C, int L) {
  const int N = 1 << L;
  const int two = b ? 1 : 0;  // log2 of the number of polynomials
  int lt = 0;
  for (; lt < L % 3; ++lt) {  // leading radix-2 stages (never the last one: L >= 4)
    const int h = N >> (lt + 1);
    for (int task = threadIdx.x; task < (N / 2) << two; task += blockDim.x) {
      u64* p = (task >= N / 2) ? b : a;
      const int k = task & (N / 2 - 1);
      const int i = k >> lt, idx = (i << (lt + 1)) + (k & ((1 << lt) - 1));
      u64 x = p[idx], y = p[idx + (1 << lt)];
      gs_bfly(x, y, itw[h + i], C);
      p[idx] = x;
      p[idx + (1 << lt)] = y;
    }
    __syncthreads();
  }
  for (; lt < L; lt += 3) {
    // distances t, 2t, 4t on e_k = 8t I + j + k t (k < 8, j < t)
    const int h1 = N >> (lt + 1), h2 = N >> (lt + 2), h3 = N >> (lt + 3);
    const bool last = (lt + 3 == L);
    for (int task = threadIdx.x; task < (N / 8) << two; task += blockDim.x) {
      u64* p = (task >= N / 8) ? b : a;
      const int g = task & (N / 8 - 1);
      const int I = g >> lt, base = (I << (lt + 3)) + (g & ((1 << lt) - 1));
      const u64 w1[4] = {itw[h1 + 4 * I], itw[h1 + 4 * I + 1], itw[h1 + 4 * I + 2], itw[h1 + 4 * I + 3]};
      const u64 w2a = itw[h2 + 2 * I], w2b = itw[h2 + 2 * I + 1], w3 = itw[h3 + I];
      u64 x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = p[base + (k << lt)];
#pragma unroll
      for (int k = 0; k < 4; ++k) gs_bfly(x[2 * k], x[2 * k + 1], w1[k], C);
      gs_bfly(x[0], x[2], w2a, C);
      gs_bfly(x[1], x[3], w2a, C);
      gs_bfly(x[4], x[6], w2b, C);
      gs_bfly(x[5], x[7], w2b, C);
      if (last) {
#pragma unroll
        for (int k = 0; k < 4; ++k) gs_last(x[k], x[k + 4], C);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) gs_bfly(x[k], x[k + 4], w3, C);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) p[base + (k << lt)] = x[k];
    }
    __syncthreads();
  }
}

// Radix-4 forms (two stages per barrier, N/4 work items) for one polynomial
// when the radix-8 forms would leave half of the CTA's threads idle; the one
// stage left over (odd L) runs as a radix-2 stage: last for the forward
// transform, first for the inverse (so that N^-1 folds into a radix-4 stage).
__device__ void ntt_fwd4(u64* a, const u64* tw, const NttConst& C, int L) {
  const int N = 1 << L;
  int lt = L - 1;
  for (; lt >= 1; lt -= 2) {
    // distances t, t/2 on e_k = 2t i + j + k t/2 (k < 4, j < t/2)
    const int m = N >> (lt + 1), q2 = lt - 1;
    for (int g = threadIdx.x; g < N / 4; g += blockDim.x) {
      const int i = g >> q2, base = (i << (lt + 1)) + (g & ((1 << q2) - 1));
      u64 x0 = a[base], x1 = a[base + (1 << q2)], x2 = a[base + (2 << q2)], x3 = a[base + (3 << q2)];
      const u64 w1 = tw[m + i];
      ct_bfly(x0, x2, w1, C);
      ct_bfly(x1, x3, w1, C);
      ct_bfly(x0, x1, tw[2 * m + 2 * i], C);
      ct_bfly(x2, x3, tw[2 * m + 2 * i + 1], C);
      a[base] = x0;
      a[base + (1 << q2)] = x1;
      a[base + (2 << q2)] = x2;
      a[base + (3 << q2)] = x3;
    }
    __syncthreads();
  }
  if (lt == 0) {
    for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
      u64 x = a[2 * b], y = a[2 * b + 1];
      ct_bfly(x, y, tw[N / 2 + b], C);
      a[2 * b] = x;
      a[2 * b + 1] = y;
    }
    __syncthreads();
  }
}

__device__ void ntt_inv4(u64* a, const u64* itw, const NttConst& C, int L) {
  const int N = 1 << L;
  int lt = 0;
  if (L & 1) {
    for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
      u64 x = a[2 * k], y = a[2 * k + 1];
      gs_bfly(x, y, itw[N / 2 + k], C);
      a[2 * k] = x;
      a[2 * k + 1] = y;
    }
    __syncthreads();
    lt = 1;
  }
  for (; lt < L; lt += 2) {
    // distances t, 2t on e_k = 4t I + j + k t (k < 4, j < t)
    const int h1 = N >> (lt + 1), h2 = N >> (lt + 2);
    const bool last = (lt + 2 == L);
    for (int g = threadIdx.x; g < N / 4; g += blockDim.x) {
      const int I = g >> lt, base = (I << (lt + 2)) + (g & ((1 << lt) - 1));
      u64 x0 = a[base], x1 = a[base + (1 << lt)], x2 = a[base + (2 << lt)], x3 = a[base + (3 << lt)];
      gs_bfly(x0, x1, itw[h1 + 2 * I], C);
      gs_bfly(x2, x3, itw[h1 + 2 * I + 1], C);
      if (last) {
        gs_last(x0, x2, C);
        gs_last(x1, x3, C);
      } else {
        const u64 w2 = itw[h2 + I];
        gs_bfly(x0, x2, w2, C);
        gs_bfly(x1, x3, w2, C);
      }
      a[base] = x0;
      a[base + (1 << lt)] = x1;
      a[base + (2 << lt)] = x2;
      a[base + (3 << lt)] = x3;
    }
    __syncthreads();
  }
}

// Dispatch: radix-8 unless it would leave half of the threads idle.
__device__ __forceinline__ void ntt_fwd(u64* a, const u64* tw, const NttConst& C, int L) {
  if ((int)blockDim.x >= (1 << L) / 4 && L >= 2)
    ntt_fwd4(a, tw, C, L);
  else
    ntt_fwd8(a, tw, C, L);
}
__device__ __forceinline__ void ntt_inv(u64* a, u64* b, const u64* itw, const NttConst& C, int L) {
  if (!b && (int)blockDim.x >= (1 << L) / 4 && L >= 2)
    ntt_inv4(a, itw, C, L);
  else
    ntt_inv8(a, b, itw, C, L);
}

__device__ __forceinline__ u64 to_q(u64 x, u64) { return x; }  // already in [0, q)
__device__ __forceinline__ u64 to_q(int8_t x, u64 q) { return smod32(x, q); }

// Every kernel below keeps its twiddle table in shared memory (copied once at
// entry with 16-byte loads): one DRAM/L2 round trip instead of one per stage.
__device__ __forceinline__ void stage_table(u64* dst, const u64* __restrict__ src, int N) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < N / 2; i += blockDim.x) d4[i] = s4[i];
}

// forward transforms of one or two polynomials: CTA b reads src[b] (reduced
// into [0, q)) and writes dst + b N.  smem: poly [N] + twiddles [N]
// With mont = 1 the outputs are in Montgomery form (x R mod q), so that one
// Montgomery product with them is a plain product mod q.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_ntt(const T* __restrict__ src0, const T* __restrict__ src1, u64* __restrict__ dst, const u64* __restrict__ tw,
          NttConst C, int mont) {
  extern __shared__ u64 sm[];
  const int N = 1 << C.log_n;
  u64* t = sm + N;
  const T* src = blockIdx.x == 0 ? src0 : src1;
  stage_table(t, tw, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = to_q(src[i], C.q);
  __syncthreads();
  ntt_fwd(sm, t, C, C.log_n);
  u64* p = dst + (size_t)blockIdx.x * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) p[i] = mont ? mmul(sm[i], C.r2, C.q, C.qn) : sm[i];
}

// Encryption of one plaintext per CTA: v -> NTT -> (v b^, v a^) -> inverse NTT
// (both at once) -> c0 = b v + e0 + m, c1 = a v + e1.  pk = [b^ | a^], the
// public key in the transform domain, Montgomery form.  smem: x, y,
// twiddles [N] each.
__global__ void __launch_bounds__(kThreads)
    k_encrypt(const u64* __restrict__ pk, const int64_t* __restrict__ m, const int8_t* __restrict__ v,
              const int32_t* __restrict__ e0, const int32_t* __restrict__ e1, const u64* __restrict__ tw,
              const u64* __restrict__ itw, NttConst C, u64* __restrict__ c) {
  extern __shared__ u64 sm[];
  const int N = 1 << C.log_n;
  const size_t p = blockIdx.x;
  u64 *x = sm, *y = sm + N, *t = sm + 2 * N;
  stage_table(t, tw, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = smod32(v[p * N + i], C.q);
  __syncthreads();
  ntt_fwd(x, t, C, C.log_n);
  stage_table(t, itw, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const u64 xv = x[i];
    x[i] = mmul(xv, pk[i], C.q, C.qn);
    y[i] = mmul(xv, pk[N + i], C.q, C.qn);
  }
  __syncthreads();
  ntt_inv(x, y, t, C, C.log_n);
  u64* c0 = c + p * 2 * N;
  u64* c1 = c0 + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    c0[i] = addm(addm(x[i], smod32(e0[p * N + i], C.q), C.q), smod64(m[p * N + i], C.q), C.q);
    c1[i] = addm(y[i], smod32(e1[p * N + i], C.q), C.q);
  }
}

// Decryption of one ciphertext per CTA: m = c0 + InvNTT(NTT(c1) s^), s^ in
// Montgomery form.
// smem: poly + twiddles [N] each.
__global__ void __launch_bounds__(kThreads)
    k_decrypt(const u64* __restrict__ c, const u64* __restrict__ shat, const u64* __restrict__ tw,
              const u64* __restrict__ itw, NttConst C, u64* __restrict__ m) {
  extern __shared__ u64 sm[];
  const int N = 1 << C.log_n;
  const size_t p = blockIdx.x;
  u64* t = sm + N;
  const u64* c0 = c + p * 2 * N;
  stage_table(t, tw, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = c0[N + i];
  __syncthreads();
  ntt_fwd(sm, t, C, C.log_n);
  stage_table(t, itw, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    sm[i] = mmul(sm[i], shat[i], C.q, C.qn);
  __syncthreads();
  ntt_inv(sm, nullptr, t, C, C.log_n);
  for (int i = threadIdx.x; i < N; i += blockDim.x) m[p * N + i] = addm(c0[i], sm[i], C.q);
}

// b = -(a s) + e, from a^ (Montgomery form) and s^ (transform domain).
// smem: poly + twiddles.
__global__ void __launch_bounds__(kThreads)
    k_keygen(const u64* __restrict__ ahat, const u64* __restrict__ shat, const int32_t* __restrict__ e,
             const u64* __restrict__ itw, NttConst C, u64* __restrict__ b) {
  extern __shared__ u64 sm[];
  const int N = 1 << C.log_n;
  u64* t = sm + N;
  stage_table(t, itw, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    sm[i] = mmul(ahat[i], shat[i], C.q, C.qn);
  __syncthreads();
  ntt_inv(sm, nullptr, t, C, C.log_n);
  for (int i = threadIdx.x; i < N; i += blockDim.x) b[i] = addm(subm(0, sm[i], C.q), smod32(e[i], C.q), C.q);
}

constexpr int kMaxSum = 256;  // operands of one ckks_sum (kernel parameter space)
struct SumArgs {
  const u64* p[kMaxSum];
};

__global__ void k_sum(const __grid_constant__ SumArgs a, int count, size_t n, u64 q, u64* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    u64 s = 0;
    for (int k = 0; k < count; ++k) s = addm(s, a.p[k][i], q);
    out[i] = s;
  }
}

// ---- canonical embedding by FFT ---------------------------------------------
// With omega = exp(i pi / N) and n = N / 2: every slot root zeta_j = omega^r_j
// has r_j = 5^j = 1 mod 4, so zeta_j^n = i and, for a real m of degree < N,
//   m(zeta_j) = w(zeta_j),  w_k = m_k + i m_(k+n)  (k < n),
// a complex polynomial of degree < n.  The r_j run over all residues 1 mod 4 in
// [0, 2N), so zeta_j = omega W^t with W = omega^4 = exp(2 pi i / n) and
// t = pos_j = (r_j - 1) / 4 a permutation of [0, n):
//   decode:  z_j = Z[pos_j] / scale,  Z[t] = sum_k (w_k omega^k) W^(t k)
//   encode:  w_k = omega^-k (1/n) sum_t Y[t] W^(-t k),  Y[pos_j] = scale z_j,
//            m_k = round(Re w_k), m_(k+n) = round(Im w_k)
// Length-n radix-2 decimation in time on a bit-reversed load, in shared memory,
// with the stage twiddles W^j (j < n/2) staged in shared memory too.

// DIT stages; a bit-reversed on entry, natural order on exit; w[j] = W^j
__device__ void fft_stages(double2* a, const double2* w, int log_m, double sign) {
  const int n = 1 << log_m;
  for (int lg = 1; lg <= log_m; ++lg) {
    const int half = 1 << (lg - 1);
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int g = b >> (lg - 1), j = b & (half - 1);
      const int i0 = (g << lg) + j;
      const double2 t = w[j << (log_m - lg)];
      const double wr = t.x, wi = sign * t.y;
      const double2 u = a[i0], x = a[i0 + half];
      const double vr = x.x * wr - x.y * wi, vi = x.x * wi + x.y * wr;
      a[i0] = make_double2(u.x + vr, u.y + vi);
      a[i0 + half] = make_double2(u.x - vr, u.y - vi);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int brev(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

// smem: a [n] + w [n/2] double2
__global__ void __launch_bounds__(kThreads)
    k_encode(const double* __restrict__ re, const double* __restrict__ im, int log_n,
             const int32_t* __restrict__ pos, const double2* __restrict__ fftw, const double2* __restrict__ twist,
             double scale, int64_t* __restrict__ m) {
  extern __shared__ double2 z[];
  const int log_m = log_n - 1, n = 1 << log_m, N = 2 * n;
  double2* w = z + n;
  const size_t p = blockIdx.x;
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) w[j] = fftw[j];
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (PL_BOUNDS(pos[j] >= 0 && pos[j] < n, pl::kBoundsSlot))
      z[brev(pos[j], log_m)] = make_double2(re[p * n + j], im[p * n + j]);
  __syncthreads();
  fft_stages(z, w, log_m, -1.0);
  const double f = scale / n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double2 t = twist[k], v = z[k];  // v * conj(omega^k)
    m[p * N + k] = (int64_t)rint((v.x * t.x + v.y * t.y) * f);
    m[p * N + k + n] = (int64_t)rint((v.y * t.x - v.x * t.y) * f);
  }
}

__global__ void __launch_bounds__(kThreads)
    k_decode(const u64* __restrict__ m, int log_n, u64 q, const int32_t* __restrict__ pos,
             const double2* __restrict__ fftw, const double2* __restrict__ twist, double scale, double inv,
             double* __restrict__ re, double* __restrict__ im) {
  extern __shared__ double2 z[];
  const int log_m = log_n - 1, n = 1 << log_m, N = 2 * n;
  double2* w = z + n;
  const size_t p = blockIdx.x;
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) w[j] = fftw[j];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const u64 a = m[p * N + k], b = m[p * N + k + n];
    const double x = a > q / 2 ? -(double)(q - a) : (double)a;
    const double y = b > q / 2 ? -(double)(q - b) : (double)b;
    const double2 t = twist[k];
    z[brev(k, log_m)] = make_double2(x * t.x - y * t.y, x * t.y + y * t.x);
  }
  __syncthreads();
  fft_stages(z, w, log_m, 1.0);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double2 v = z[PL_BOUNDS(pos[j] >= 0 && pos[j] < n, pl::kBoundsSlot) ? pos[j] : 0];
    // inv = 1 / scale when scale is a power of two (the product is then exact
    // and equals the quotient), else 0
    re[p * n + j] = inv != 0.0 ? v.x * inv : v.x / scale;
    im[p * n + j] = inv != 0.0 ? v.y * inv : v.y / scale;
  }
}

// ---- one polynomial per cluster of kCl CTAs (distributed shared memory) ----
// For a small batch, one CTA per polynomial leaves most SMs idle.  The cluster
// kernels split each polynomial over kCl CTAs.  With M = (length) / kCl:
//   cyclic layout: CTA r holds global indices r + kCl u (u < M);
//   block layout:  CTA r holds global indices r M + v (v < M).
// Forward NTT (distances t = N/2 .. 1): the stages with t >= kCl pair indices of
// one residue class mod kCl, and on the cyclic slice they are exactly the stages
// of a length-M transform with the same twiddle entries tw[m + i], m < M; the
// last log2 kCl stages (t < kCl <= M) are local in the block layout.  One
// exchange through distributed shared memory (cyclic -> block) sits between
// them.  The inverse runs the mirror image (block stages t = 1 .. kCl/2, block
// -> cyclic, then a length-M inverse on the cyclic slice, N^-1 folded into its
// last stage as for a whole polynomial).  The canonical-embedding FFT (decimation
// in time on a bit-reversed load) does its small distances in the block layout
// and its large ones in the cyclic layout.  Every cluster barrier is a hardware
// barrier (no polling).
namespace cg = cooperative_groups;

constexpr int kCl = 8, kClLog = 3;
constexpr int kClNttThreads = 256, kClFftThreads = 256;

// offset of the block-stage twiddles of distance 2^lt in a CTA's packed table
// (t = 4, 2, 1 at 0, M/8, M/8 + M/4)
__device__ __forceinline__ int tail_off(int lt, int M) { return lt == 2 ? 0 : (lt == 1 ? M / 8 : M / 8 + M / 4); }

// forward stages t = kCl/2 .. 1 on the block slice of CTA r; tw: this CTA's
// packed block-stage twiddles (global entry N/2t + r M/2t + i at tail_off + i).
// The three stages stay inside groups of 8 consecutive entries: one work item
// per group, in registers, one barrier.
static_assert(kCl == 8, "the block-layout stages are written for clusters of 8");
__device__ void ntt_fwd_tail(u64* a, const u64* tw, const NttConst& C, int logM) {
  const int M = 1 << logM;
  const u64 *w4 = tw + tail_off(2, M), *w2 = tw + tail_off(1, M), *w1 = tw + tail_off(0, M);
  for (int g = threadIdx.x; g < M / 8; g += blockDim.x) {
    u64 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = a[8 * g + k];
    const u64 t4 = w4[g];
#pragma unroll
    for (int k = 0; k < 4; ++k) ct_bfly(x[k], x[k + 4], t4, C);
    const u64 t2a = w2[2 * g], t2b = w2[2 * g + 1];
    ct_bfly(x[0], x[2], t2a, C);
    ct_bfly(x[1], x[3], t2a, C);
    ct_bfly(x[4], x[6], t2b, C);
    ct_bfly(x[5], x[7], t2b, C);
#pragma unroll
    for (int m = 0; m < 4; ++m) ct_bfly(x[2 * m], x[2 * m + 1], w1[4 * g + m], C);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[8 * g + k] = x[k];
  }
  __syncthreads();
}

// inverse stages t = 1 .. kCl/2 on the block slice (one or two polynomials,
// spread over the threads together); itw: packed like ntt_fwd_tail's; the
// mirror image of ntt_fwd_tail (groups of 8, one barrier)
__device__ void ntt_inv_head(u64* a, u64* b, const u64* itw, const NttConst& C, int logM) {
  const int M = 1 << logM;
  const int two = b ? 1 : 0;
  const u64 *w1 = itw + tail_off(0, M), *w2 = itw + tail_off(1, M), *w4 = itw + tail_off(2, M);
  for (int task = threadIdx.x; task < (M / 8) << two; task += blockDim.x) {
    u64* p = (task >= M / 8) ? b : a;
    const int g = task & (M / 8 - 1);
    u64 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = p[8 * g + k];
#pragma unroll
    for (int m = 0; m < 4; ++m) gs_bfly(x[2 * m], x[2 * m + 1], w1[4 * g + m], C);
    const u64 t2a = w2[2 * g], t2b = w2[2 * g + 1];
    gs_bfly(x[0], x[2], t2a, C);
    gs_bfly(x[1], x[3], t2a, C);
    gs_bfly(x[4], x[6], t2b, C);
    gs_bfly(x[5], x[7], t2b, C);
    const u64 t4 = w4[g];
#pragma unroll
    for (int k = 0; k < 4; ++k) gs_bfly(x[k], x[k + 4], t4, C);
#pragma unroll
    for (int k = 0; k < 8; ++k) p[8 * g + k] = x[k];
  }
  __syncthreads();
}

// block slice of CTA r <- the cluster's cyclic slices (global index r M + v
// lives in CTA (r M + v) mod kCl at (r M + v) / kCl)
template <typename E>
__device__ void gather_block(cg::cluster_group& cl, E* dst, E* cyc, int r, int logM) {
  for (int v = threadIdx.x; v < (1 << logM); v += blockDim.x) {
    const int idx = (r << logM) + v;
    const int src = idx & (kCl - 1), li = idx >> kClLog;
    if (PL_BOUNDS(src < (int)cl.num_blocks() && li < (1 << logM), pl::kBoundsCluster))
      dst[v] = cl.map_shared_rank(cyc, src)[li];
  }
}

// cyclic slice of CTA r <- the cluster's block slices (global index r + kCl u
// lives in CTA (r + kCl u) / M at (r + kCl u) mod M)
template <typename E>
__device__ void gather_cyclic(cg::cluster_group& cl, E* dst, E* blk, int r, int logM) {
  for (int u = threadIdx.x; u < (1 << logM); u += blockDim.x) {
    const int idx = r + (u << kClLog);
    const int src = idx >> logM;
    if (PL_BOUNDS(src < (int)cl.num_blocks(), pl::kBoundsCluster))
      dst[u] = cl.map_shared_rank(blk, src)[idx & ((1 << logM) - 1)];
  }
}

// Asynchronous global -> shared copies (cp.async; completion is awaited with
// cp.async.wait_all, a hardware wait on the thread's own copies).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// waits until at most P of this thread's committed groups are still in flight
template <int P>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(P) : "memory"); }

// 16-byte copies of n words (n even, both ends 16-byte aligned)
__device__ __forceinline__ void cp_async_words(u64* dst, const u64* src, int n) {
  for (int i = threadIdx.x; i < n / 2; i += blockDim.x) cp_async16(dst + 2 * i, src + 2 * i);
}

// The twiddles of the block-layout stages of CTA r: for t = 4, 2, 1 the
// M / 2t consecutive entries tab[N / 2t + r M / 2t ..], packed at offsets
// 0, M/8, M/8 + M/4 (7M/8 words in all).
__device__ __forceinline__ void cp_async_tail(u64* dst, const u64* tab, int N, int r, int logM) {
  const int M = 1 << logM;
  for (int lt = 0; lt < kClLog; ++lt)
    cp_async_words(dst + tail_off(lt, M), tab + (N >> (lt + 1)) + ((r << logM) >> (lt + 1)), M >> (lt + 1));
}

// smem (M words each unless noted): x0, x1 (cyclic), y0, y1 (block), t
// (length-M twiddles), pk0, pk1 (this CTA's key slices), twf, twi (block-stage
// twiddles, 7M/8 each), em (epilogue m), ee (epilogue e0 | e1, int32)
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClNttThreads)
    k_encrypt_cl(const u64* __restrict__ pk, const int64_t* __restrict__ m, const int8_t* __restrict__ v,
                 const int32_t* __restrict__ e0, const int32_t* __restrict__ e1, const u64* __restrict__ tw,
                 const u64* __restrict__ itw, NttConst C, u64* __restrict__ c) {
  extern __shared__ u64 sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const size_t p = blockIdx.x / kCl;
  const int N = 1 << C.log_n, logM = C.log_n - kClLog, M = 1 << logM;
  u64 *x0 = sm, *x1 = sm + M, *y0 = sm + 2 * M, *y1 = sm + 3 * M, *t = sm + 4 * M;
  u64 *pk0 = sm + 5 * M, *pk1 = sm + 6 * M, *twf = sm + 7 * M, *twi = sm + 8 * M, *em = sm + 9 * M;
  int32_t* ee = reinterpret_cast<int32_t*>(sm + 10 * M);
  // asynchronous copies in three groups: the forward length-M twiddles (needed
  // first), everything needed after the first transform, and (issued once the
  // forward transform is done with t) the inverse length-M twiddles
  cp_async_words(t, tw, M);
  cp_async_commit();
  cp_async_words(pk0, pk + (r << logM), M);
  cp_async_words(pk1, pk + N + (r << logM), M);
  cp_async_tail(twf, tw, N, r, logM);
  cp_async_tail(twi, itw, N, r, logM);
  for (int u = threadIdx.x; u < M; u += blockDim.x) {
    const size_t g = p * N + r + ((size_t)u << kClLog);
    cp_async8(em + u, m + g);
    cp_async4(ee + u, e0 + g);
    cp_async4(ee + M + u, e1 + g);
  }
  cp_async_commit();
  for (int u = threadIdx.x; u < M; u += blockDim.x) x0[u] = smod32(v[p * N + r + (u << kClLog)], C.q);
  cp_async_wait_group<1>();
  __syncthreads();
  ntt_fwd(x0, t, C, logM);  // stages t >= kCl
  cl.sync();
  cp_async_words(t, itw, M);
  cp_async_commit();
  gather_block(cl, y0, x0, r, logM);
  cp_async_wait_group<1>();
  __syncthreads();
  ntt_fwd_tail(y0, twf, C, logM);  // stages t < kCl
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const u64 xv = y0[i];
    y0[i] = mmul(xv, pk0[i], C.q, C.qn);
    y1[i] = mmul(xv, pk1[i], C.q, C.qn);
  }
  __syncthreads();
  ntt_inv_head(y0, y1, twi, C, logM);
  cl.sync();  // every block slice done; every read of the cyclic slices done
  gather_cyclic(cl, x0, y0, r, logM);
  gather_cyclic(cl, x1, y1, r, logM);
  cl.sync();  // no CTA reads another's block slice after this
  cp_async_wait();  // the inverse twiddles
  __syncthreads();
  ntt_inv(x0, x1, t, C, logM);
  u64* c0 = c + p * 2 * N;
  u64* c1 = c0 + N;
  for (int u = threadIdx.x; u < M; u += blockDim.x) {
    const size_t g = (size_t)r + ((size_t)u << kClLog);
    c0[g] = addm(addm(x0[u], smod32(ee[u], C.q), C.q), smod64((long long)em[u], C.q), C.q);
    c1[g] = addm(x1[u], smod32(ee[M + u], C.q), C.q);
  }
}

// smem: x (cyclic), y (block), t, sh (this CTA's slice of s^), ec0 (epilogue
// c0): M words each; twf, twi: 7M/8 each (M reserved)
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClNttThreads)
    k_decrypt_cl(const u64* __restrict__ c, const u64* __restrict__ shat, const u64* __restrict__ tw,
                 const u64* __restrict__ itw, NttConst C, u64* __restrict__ m) {
  extern __shared__ u64 sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const size_t p = blockIdx.x / kCl;
  const int N = 1 << C.log_n, logM = C.log_n - kClLog, M = 1 << logM;
  u64 *x = sm, *y = sm + M, *t = sm + 2 * M, *sh = sm + 3 * M, *ec0 = sm + 4 * M, *twf = sm + 5 * M,
      *twi = sm + 6 * M;
  const u64* c0 = c + p * 2 * N;
  // copy groups as in k_encrypt_cl
  cp_async_words(t, tw, M);
  cp_async_commit();
  cp_async_words(sh, shat + (r << logM), M);
  cp_async_tail(twf, tw, N, r, logM);
  cp_async_tail(twi, itw, N, r, logM);
  for (int u = threadIdx.x; u < M; u += blockDim.x) cp_async8(ec0 + u, c0 + r + ((size_t)u << kClLog));
  cp_async_commit();
  for (int u = threadIdx.x; u < M; u += blockDim.x) x[u] = c0[N + r + (u << kClLog)];
  cp_async_wait_group<1>();
  __syncthreads();
  ntt_fwd(x, t, C, logM);
  cl.sync();
  cp_async_words(t, itw, M);
  cp_async_commit();
  gather_block(cl, y, x, r, logM);
  cp_async_wait_group<1>();
  __syncthreads();
  ntt_fwd_tail(y, twf, C, logM);
  for (int i = threadIdx.x; i < M; i += blockDim.x) y[i] = mmul(y[i], sh[i], C.q, C.qn);
  __syncthreads();
  ntt_inv_head(y, nullptr, twi, C, logM);
  cl.sync();
  gather_cyclic(cl, x, y, r, logM);
  cl.sync();
  cp_async_wait();  // the inverse twiddles
  __syncthreads();
  ntt_inv(x, nullptr, t, C, logM);
  for (int u = threadIdx.x; u < M; u += blockDim.x) {
    const size_t g = (size_t)r + ((size_t)u << kClLog);
    m[p * N + g] = addm(ec0[u], x[u], C.q);
  }
}

// One DIT butterfly: u + t x, u - t x (t = W^j, conjugated for sign -1), the
// same operations in the same order as the radix-2 stages.
__device__ __forceinline__ void dit_bfly(double2& u, double2& x, double2 t, double sign) {
  const double wr = t.x, wi = sign * t.y;
  const double vr = x.x * wr - x.y * wi, vi = x.x * wi + x.y * wr;
  x = make_double2(u.x - vr, u.y - vi);
  u = make_double2(u.x + vr, u.y + vi);
}

// FFT stages in the block layout: lg = 1 .. logM (half size h = 2^(lg-1) < M);
// w[j] = W^j of the length-n transform (log_n2 = log2 n).  Two consecutive
// stages run in registers on four elements per work item (one barrier per
// pair), the last one alone when logM is odd.
__device__ void fft_block_stages(double2* a, const double2* w, int logM, int log_n2, double sign) {
  const int M = 1 << logM;
  int lg0 = 1;
  for (; lg0 + 1 <= logM; lg0 += 2) {
    const int half = 1 << (lg0 - 1);
    for (int b = threadIdx.x; b < M / 4; b += blockDim.x) {
      const int j = b & (half - 1);
      const int i0 = ((b >> (lg0 - 1)) << (lg0 + 1)) + j;
      double2 x0 = a[i0], x1 = a[i0 + half], x2 = a[i0 + 2 * half], x3 = a[i0 + 3 * half];
      const double2 t1 = w[j << (log_n2 - lg0)];
      dit_bfly(x0, x1, t1, sign);
      dit_bfly(x2, x3, t1, sign);
      dit_bfly(x0, x2, w[j << (log_n2 - lg0 - 1)], sign);
      dit_bfly(x1, x3, w[(j + half) << (log_n2 - lg0 - 1)], sign);
      a[i0] = x0;
      a[i0 + half] = x1;
      a[i0 + 2 * half] = x2;
      a[i0 + 3 * half] = x3;
    }
    __syncthreads();
  }
  for (int lg = lg0; lg <= logM; ++lg) {
    const int half = 1 << (lg - 1);
    for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
      const int g = b >> (lg - 1), j = b & (half - 1);
      const int i0 = (g << lg) + j;
      const double2 t = w[j << (log_n2 - lg)];
      const double wr = t.x, wi = sign * t.y;
      const double2 u = a[i0], x = a[i0 + half];
      const double vr = x.x * wr - x.y * wi, vi = x.x * wi + x.y * wr;
      a[i0] = make_double2(u.x + vr, u.y + vi);
      a[i0 + half] = make_double2(u.x - vr, u.y - vi);
    }
    __syncthreads();
  }
}

// FFT stages in the cyclic layout of CTA r: lg = logM + 1 .. log_n2 (global half
// size h >= M, local half size h / kCl; the pair's global offset in its group
// is r + kCl j'), two stages per barrier as in the block layout
__device__ void fft_cyclic_stages(double2* a, const double2* w, int r, int logM, int log_n2, double sign) {
  const int M = 1 << logM;
  int lg0 = logM + 1;
  for (; lg0 + 1 <= log_n2; lg0 += 2) {
    const int lh = lg0 - 1 - kClLog;  // log2 of the local half size of stage lg0
    for (int b = threadIdx.x; b < M / 4; b += blockDim.x) {
      const int jl = b & ((1 << lh) - 1);
      const int i0 = ((b >> lh) << (lh + 2)) + jl;
      const int hl = 1 << lh;
      double2 x0 = a[i0], x1 = a[i0 + hl], x2 = a[i0 + 2 * hl], x3 = a[i0 + 3 * hl];
      const double2 t1 = w[(r + (jl << kClLog)) << (log_n2 - lg0)];
      dit_bfly(x0, x1, t1, sign);
      dit_bfly(x2, x3, t1, sign);
      dit_bfly(x0, x2, w[(r + (jl << kClLog)) << (log_n2 - lg0 - 1)], sign);
      dit_bfly(x1, x3, w[(r + ((jl + hl) << kClLog)) << (log_n2 - lg0 - 1)], sign);
      a[i0] = x0;
      a[i0 + hl] = x1;
      a[i0 + 2 * hl] = x2;
      a[i0 + 3 * hl] = x3;
    }
    __syncthreads();
  }
  for (int lg = lg0; lg <= log_n2; ++lg) {
    const int lh = lg - 1 - kClLog;  // log2 of the local half size
    for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
      const int g = b >> lh, jl = b & ((1 << lh) - 1);
      const int i0 = (g << (lh + 1)) + jl;
      const double2 t = w[(r + (jl << kClLog)) << (log_n2 - lg)];
      const double wr = t.x, wi = sign * t.y;
      const double2 u = a[i0], x = a[i0 + (1 << lh)];
      const double vr = x.x * wr - x.y * wi, vi = x.x * wi + x.y * wr;
      a[i0] = make_double2(u.x + vr, u.y + vi);
      a[i0 + (1 << lh)] = make_double2(u.x - vr, u.y - vi);
    }
    __syncthreads();
  }
}

// smem: block [M] + cyclic [M] + twiddles [n/2] double2 (n = N/2, M = n / kCl)
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClFftThreads)
    k_encode_cl(const double* __restrict__ re, const double* __restrict__ im, int log_n,
                const int32_t* __restrict__ invpos, const double2* __restrict__ fftw,
                const double2* __restrict__ twist, double scale, int64_t* __restrict__ m) {
  extern __shared__ double2 z[];
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const size_t p = blockIdx.x / kCl;
  const int log_m = log_n - 1, n = 1 << log_m, N = 2 * n, logM = log_m - kClLog, M = 1 << logM;
  double2 *blk = z, *cyc = z + M, *w = z + 2 * M;
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) cp_async16(w + j, fftw + j);  // in flight during the load
  cp_async_commit();
  for (int v = threadIdx.x; v < M; v += blockDim.x) {  // bit-reversed load: Y[t] = z_j at t = pos_j
    int j = invpos[brev((r << logM) + v, log_m)];
    if (!PL_BOUNDS(j >= 0 && j < n, pl::kBoundsSlot)) j = 0;
    blk[v] = make_double2(re[p * n + j], im[p * n + j]);
  }
  cp_async_wait();
  __syncthreads();
  fft_block_stages(blk, w, logM, log_m, -1.0);
  cl.sync();
  gather_cyclic(cl, cyc, blk, r, logM);
  cl.sync();
  fft_cyclic_stages(cyc, w, r, logM, log_m, -1.0);
  const double f = scale / n;
  for (int u = threadIdx.x; u < M; u += blockDim.x) {
    const int k = r + (u << kClLog);
    const double2 t = twist[k], v = cyc[u];
    m[p * N + k] = (int64_t)rint((v.x * t.x + v.y * t.y) * f);
    m[p * N + k + n] = (int64_t)rint((v.y * t.x - v.x * t.y) * f);
  }
}

__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClFftThreads)
    k_decode_cl(const u64* __restrict__ mq, int log_n, u64 q, const int32_t* __restrict__ invpos,
                const double2* __restrict__ fftw, const double2* __restrict__ twist, double scale, double inv,
                double* __restrict__ re, double* __restrict__ im) {
  extern __shared__ double2 z[];
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const size_t p = blockIdx.x / kCl;
  const int log_m = log_n - 1, n = 1 << log_m, N = 2 * n, logM = log_m - kClLog, M = 1 << logM;
  double2 *blk = z, *cyc = z + M, *w = z + 2 * M;
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) cp_async16(w + j, fftw + j);  // in flight during the load
  cp_async_commit();
  for (int v = threadIdx.x; v < M; v += blockDim.x) {  // bit-reversed load of the twisted w_k
    const int k = brev((r << logM) + v, log_m);
    const u64 a = mq[p * N + k], b = mq[p * N + k + n];
    const double x = a > q / 2 ? -(double)(q - a) : (double)a;
    const double y = b > q / 2 ? -(double)(q - b) : (double)b;
    const double2 t = twist[k];
    blk[v] = make_double2(x * t.x - y * t.y, x * t.y + y * t.x);
  }
  cp_async_wait();
  __syncthreads();
  fft_block_stages(blk, w, logM, log_m, 1.0);
  cl.sync();
  gather_cyclic(cl, cyc, blk, r, logM);
  cl.sync();
  fft_cyclic_stages(cyc, w, r, logM, log_m, 1.0);
  for (int u = threadIdx.x; u < M; u += blockDim.x) {
    int j = invpos[r + (u << kClLog)];
    if (!PL_BOUNDS(j >= 0 && j < n, pl::kBoundsSlot)) continue;
    const double2 v = cyc[u];
    re[p * n + j] = inv != 0.0 ? v.x * inv : v.x / scale;
    im[p * n + j] = inv != 0.0 ? v.y * inv : v.y / scale;
  }
}

int ew_grid(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)pl::sm_count() * 8); }

template <typename K>
cudaError_t allow_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)((3u << kMaxLogN) * sizeof(u64)));
}

}  // namespace

struct ckks_ctx {
  int log_n = 0, N = 0, device = 0;
  double scale = 1.0, inv_scale = 0.0;  // inv_scale: 1 / scale if scale is a power of two, else 0
  NttConst C{};
  u64* d_tw = nullptr;   // forward twiddles psi^bitrev(i), Montgomery form
  u64* d_itw = nullptr;  // inverse twiddles psi^-bitrev(i), Montgomery form
  int32_t* d_pos = nullptr;    // slot j -> (r_j - 1) / 4
  int32_t* d_invpos = nullptr; // (r_j - 1) / 4 -> slot j
  double2* d_fftw = nullptr;   // W^j = exp(2 pi i j / n), j < n / 2
  double2* d_twist = nullptr;  // omega^k = exp(i pi k / N), k < n
  pl::Scratch scratch;
  u64* d_pk = nullptr;    // prepared [b^ | a^], Montgomery form (NULL until prepared)
  u64* d_shat = nullptr;  // prepared s^, Montgomery form

  ~ckks_ctx() {
    cudaFree(d_pk);
    cudaFree(d_shat);
    cudaFree(d_tw);
    cudaFree(d_itw);
    cudaFree(d_pos);
    cudaFree(d_invpos);
    cudaFree(d_fftw);
    cudaFree(d_twist);
  }
  int threads() const { return std::min(N / 2, kThreads); }
  // a small batch spreads each polynomial over a cluster of kCl CTAs; a large
  // one (or a small N) keeps one polynomial per CTA
  size_t cluster_max_batch = 64;
  bool clustered(size_t batch) const { return log_n >= 10 && batch <= cluster_max_batch; }

  pl_status launch_encrypt(const u64* pk, const int64_t* d_m, const int8_t* d_v, const int32_t* d_e0,
                           const int32_t* d_e1, size_t batch, u64* d_c, cudaStream_t s) {
    if (clustered(batch))
      k_encrypt_cl<<<(unsigned)(batch * kCl), kClNttThreads, 11 * poly_bytes() / kCl, s>>>(pk, d_m, d_v, d_e0, d_e1,
                                                                                         d_tw, d_itw, C, d_c);
    else
      k_encrypt<<<(unsigned)batch, threads(), 3 * poly_bytes(), s>>>(pk, d_m, d_v, d_e0, d_e1, d_tw, d_itw, C, d_c);
    pl::note_launch();
    PL_CUDA_TRY(cudaGetLastError());
    return PL_OK;
  }
  pl_status launch_decrypt(const u64* d_c, const u64* shat, size_t batch, u64* d_m, cudaStream_t s) {
    if (clustered(batch))
      k_decrypt_cl<<<(unsigned)(batch * kCl), kClNttThreads, 7 * poly_bytes() / kCl, s>>>(d_c, shat, d_tw, d_itw, C,
                                                                                         d_m);
    else
      k_decrypt<<<(unsigned)batch, threads(), 2 * poly_bytes(), s>>>(d_c, shat, d_tw, d_itw, C, d_m);
    pl::note_launch();
    PL_CUDA_TRY(cudaGetLastError());
    return PL_OK;
  }
  int fft_threads() const { return std::min(N / 4, kThreads); }
  size_t fft_smem() const { return (size_t)(N / 2 + N / 4) * sizeof(double2); }
  size_t fft_cl_smem() const { return (size_t)(2 * (N / 2 / kCl) + N / 4) * sizeof(double2); }
  size_t poly_bytes() const { return (size_t)N * sizeof(u64); }

  // dst [2][N] = NTT(src0), NTT(src1) (src1 may be NULL: one polynomial),
  // in Montgomery form if mont
  template <typename T>
  pl_status ntt(const T* src0, const T* src1, u64* dst, bool mont, cudaStream_t s) {
    k_ntt<T><<<src1 ? 2 : 1, threads(), 2 * poly_bytes(), s>>>(src0, src1, dst, d_tw, C, mont ? 1 : 0);
    pl::note_launch();
    PL_CUDA_TRY(cudaGetLastError());
    return PL_OK;
  }
};

extern "C" {

pl_status ckks_create(int log_n, uint64_t q, double scale, ckks_ctx** out) {
  using namespace pl;
  clear_error();
  if (!out || log_n < 4 || log_n > kMaxLogN || !(scale > 0)) return fail(PL_EINVAL, "need 4 <= log_n <= 13, scale > 0");
  const int N = 1 << log_n;
  if (q >= (1ull << 62) || q < 3 || q % (2ull * N) != 1 || !h_prime(q))
    return fail(PL_EINVAL, "q must be a prime < 2^62 with q = 1 mod 2N");
  auto* c = new (std::nothrow) ckks_ctx();
  if (!c) return fail(PL_ENOMEM, "host allocation failed");
  c->log_n = log_n;
  c->N = N;
  c->scale = scale;
  int ex = 0;
  if (std::frexp(scale, &ex) == 0.5) c->inv_scale = std::ldexp(1.0, 1 - ex);
  cudaGetDevice(&c->device);
  // primitive 2N-th root of unity: psi^N = -1
  u64 psi = 0;
  for (u64 g = 2; g < 1000 && !psi; ++g) {
    const u64 x = h_pow(g, (q - 1) / (2ull * N), q);
    if (h_pow(x, (u64)N, q) == q - 1) psi = x;
  }
  if (!psi) { delete c; return fail(PL_EINVAL, "no primitive 2N-th root found"); }
  const u64 R = (u64)(((u128)1 << 64) % q);
  u64 qinv = 1;
  for (int i = 0; i < 6; ++i) qinv *= 2 - q * qinv;
  const u64 ninv = h_pow((u64)N, q - 2, q);
  std::vector<u64> tw(N), itw(N);
  const u64 ipsi = h_pow(psi, q - 2, q);
  for (int i = 0; i < N; ++i) {
    const int e = bitrev(i, log_n);
    tw[i] = h_mul(h_pow(psi, (u64)e, q), R, q);
    itw[i] = h_mul(h_pow(ipsi, (u64)e, q), R, q);
  }
  c->C.q = q;
  c->C.qn = (u64)0 - qinv;
  c->C.r2 = h_mul(R, R, q);
  c->C.ninv = h_mul(ninv, R, q);
  c->C.last = h_mul(itw[1], ninv, q);
  c->C.log_n = log_n;
  const int n = N / 2;
  std::vector<int32_t> pos(n), invpos(n);
  u64 x = 1;  // r_j = 5^j mod 2N
  for (int j = 0; j < n; ++j) { pos[j] = (int32_t)((x - 1) / 4); x = x * 5 % (2ull * N); }
  for (int j = 0; j < n; ++j) invpos[pos[j]] = j;
  std::vector<double2> fftw(n / 2), twist(n);
  for (int j = 0; j < n / 2; ++j) fftw[j] = make_double2(std::cos(M_PI * 4 * j / N), std::sin(M_PI * 4 * j / N));
  for (int k = 0; k < n; ++k) twist[k] = make_double2(std::cos(M_PI * k / N), std::sin(M_PI * k / N));
  cudaError_t e = cudaSuccess;
  auto up = [&](void** d, const void* h, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(d, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice);
  };
  up((void**)&c->d_tw, tw.data(), N * sizeof(u64));
  up((void**)&c->d_itw, itw.data(), N * sizeof(u64));
  up((void**)&c->d_pos, pos.data(), pos.size() * sizeof(int32_t));
  up((void**)&c->d_invpos, invpos.data(), invpos.size() * sizeof(int32_t));
  up((void**)&c->d_fftw, fftw.data(), fftw.size() * sizeof(double2));
  up((void**)&c->d_twist, twist.data(), twist.size() * sizeof(double2));
  for (cudaError_t a : {allow_smem(k_ntt<u64>), allow_smem(k_ntt<int8_t>), allow_smem(k_encrypt),
                        allow_smem(k_decrypt), allow_smem(k_keygen), allow_smem(k_encode), allow_smem(k_decode),
                        allow_smem(k_encrypt_cl), allow_smem(k_decrypt_cl), allow_smem(k_encode_cl),
                        allow_smem(k_decode_cl)})
    if (e == cudaSuccess) e = a;
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "ckks tables"); }
  c->scratch.device = c->device;
  *out = c;
  return PL_OK;
}

void ckks_free(ckks_ctx* ctx) { delete ctx; }

pl_status ckks_set_cluster_limit(ckks_ctx* ctx, size_t max_batch) {
  using namespace pl;
  clear_error();
  if (!ctx) return fail(PL_EINVAL, "ctx is NULL");
  ctx->cluster_max_batch = max_batch;
  return PL_OK;
}

int ckks_slots(const ckks_ctx* ctx) { return ctx ? ctx->N / 2 : 0; }

pl_status ckks_encode(ckks_ctx* ctx, const double* d_re, const double* d_im, size_t batch, int64_t* d_m,
                      void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx) return fail(PL_EINVAL, "ctx is NULL");
  if (!batch) return PL_OK;
  if (!d_re || !d_im || !d_m) return fail(PL_EINVAL, "NULL buffer");
  if (batch > 0x7fffffff) return fail(PL_ERANGE, "batch too large");
  if (ctx->clustered(batch))
    k_encode_cl<<<(unsigned)(batch * kCl), kClFftThreads, ctx->fft_cl_smem(), static_cast<cudaStream_t>(stream)>>>(
        d_re, d_im, ctx->log_n, ctx->d_invpos, ctx->d_fftw, ctx->d_twist, ctx->scale, d_m);
  else
    k_encode<<<(unsigned)batch, ctx->fft_threads(), ctx->fft_smem(), static_cast<cudaStream_t>(stream)>>>(
        d_re, d_im, ctx->log_n, ctx->d_pos, ctx->d_fftw, ctx->d_twist, ctx->scale, d_m);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status ckks_decode(ckks_ctx* ctx, const uint64_t* d_m, size_t batch, double* d_re, double* d_im, void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx) return fail(PL_EINVAL, "ctx is NULL");
  if (!batch) return PL_OK;
  if (!d_re || !d_im || !d_m) return fail(PL_EINVAL, "NULL buffer");
  if (batch > 0x7fffffff) return fail(PL_ERANGE, "batch too large");
  if (ctx->clustered(batch))
    k_decode_cl<<<(unsigned)(batch * kCl), kClFftThreads, ctx->fft_cl_smem(), static_cast<cudaStream_t>(stream)>>>(
        d_m, ctx->log_n, ctx->C.q, ctx->d_invpos, ctx->d_fftw, ctx->d_twist, ctx->scale, ctx->inv_scale, d_re, d_im);
  else
    k_decode<<<(unsigned)batch, ctx->fft_threads(), ctx->fft_smem(), static_cast<cudaStream_t>(stream)>>>(
        d_m, ctx->log_n, ctx->C.q, ctx->d_pos, ctx->d_fftw, ctx->d_twist, ctx->scale, ctx->inv_scale, d_re, d_im);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status ckks_keygen(ckks_ctx* ctx, const int8_t* d_s, const uint64_t* d_a, const int32_t* d_e, uint64_t* d_b,
                      void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_s || !d_a || !d_e || !d_b) return fail(PL_EINVAL, "NULL argument");
  const size_t N = (size_t)ctx->N;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* t = static_cast<u64*>(ctx->scratch.get(2 * N * sizeof(u64), s));
  if (!t) return fail(PL_ENOMEM, "scratch");
  pl_status rc = ctx->ntt<u64>(d_a, nullptr, t, true, s);  // a^ (Montgomery form)
  if (!rc) rc = ctx->ntt<int8_t>(d_s, nullptr, t + N, false, s);  // s^
  if (rc) return rc;
  k_keygen<<<1, ctx->threads(), 2 * ctx->poly_bytes(), s>>>(t, t + N, d_e, ctx->d_itw, ctx->C, d_b);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status ckks_encrypt(ckks_ctx* ctx, const uint64_t* d_b, const uint64_t* d_a, const int64_t* d_m,
                       const int8_t* d_v, const int32_t* d_e0, const int32_t* d_e1, size_t batch, uint64_t* d_c,
                       void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_b || !d_a || !d_m || !d_v || !d_e0 || !d_e1 || !d_c) return fail(PL_EINVAL, "NULL argument");
  if (!batch) return PL_OK;
  if (batch > 0x7fffffff) return fail(PL_ERANGE, "batch too large");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* pk = static_cast<u64*>(ctx->scratch.get(2 * ctx->poly_bytes(), s));
  if (!pk) return fail(PL_ENOMEM, "scratch");
  pl_status rc = ctx->ntt<u64>(d_b, d_a, pk, true, s);  // [b^ | a^], Montgomery form
  if (rc) return rc;
  return ctx->launch_encrypt(pk, d_m, d_v, d_e0, d_e1, batch, d_c, s);
}

pl_status ckks_sum(ckks_ctx* ctx, const uint64_t* const* d_cts, int count, size_t batch, uint64_t* d_out,
                   void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_cts || count < 1 || count > kMaxSum || !d_out) return fail(PL_EINVAL, "need 1 <= count <= 256");
  if (!batch) return PL_OK;
  SumArgs a{};
  for (int k = 0; k < count; ++k) {
    if (!d_cts[k]) return fail(PL_EINVAL, "NULL operand");
    a.p[k] = d_cts[k];
  }
  const size_t n = batch * 2 * (size_t)ctx->N;
  k_sum<<<ew_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, count, n, ctx->C.q, d_out);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status ckks_decrypt(ckks_ctx* ctx, const uint64_t* d_c, const int8_t* d_s, size_t batch, uint64_t* d_m,
                       void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_c || !d_s || !d_m) return fail(PL_EINVAL, "NULL argument");
  if (!batch) return PL_OK;
  if (batch > 0x7fffffff) return fail(PL_ERANGE, "batch too large");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* shat = static_cast<u64*>(ctx->scratch.get(ctx->poly_bytes(), s));
  if (!shat) return fail(PL_ENOMEM, "scratch");
  pl_status rc = ctx->ntt<int8_t>(d_s, nullptr, shat, true, s);
  if (rc) return rc;
  return ctx->launch_decrypt(d_c, shat, batch, d_m, s);
}

pl_status ckks_prepare_public_key(ckks_ctx* ctx, const uint64_t* d_b, const uint64_t* d_a, void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_b || !d_a) return fail(PL_EINVAL, "NULL argument");
  if (!ctx->d_pk) PL_CUDA_TRY(cudaMalloc(&ctx->d_pk, 2 * ctx->poly_bytes()));
  return ctx->ntt<u64>(d_b, d_a, ctx->d_pk, true, static_cast<cudaStream_t>(stream));
}

pl_status ckks_prepare_secret_key(ckks_ctx* ctx, const int8_t* d_s, void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_s) return fail(PL_EINVAL, "NULL argument");
  if (!ctx->d_shat) PL_CUDA_TRY(cudaMalloc(&ctx->d_shat, ctx->poly_bytes()));
  return ctx->ntt<int8_t>(d_s, nullptr, ctx->d_shat, true, static_cast<cudaStream_t>(stream));
}

pl_status ckks_encrypt_prepared(ckks_ctx* ctx, const int64_t* d_m, const int8_t* d_v, const int32_t* d_e0,
                                const int32_t* d_e1, size_t batch, uint64_t* d_c, void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_m || !d_v || !d_e0 || !d_e1 || !d_c) return fail(PL_EINVAL, "NULL argument");
  if (!ctx->d_pk) return fail(PL_EINVAL, "no public key prepared");
  if (!batch) return PL_OK;
  if (batch > 0x7fffffff) return fail(PL_ERANGE, "batch too large");
  return ctx->launch_encrypt(ctx->d_pk, d_m, d_v, d_e0, d_e1, batch, d_c, static_cast<cudaStream_t>(stream));
}

pl_status ckks_decrypt_prepared(ckks_ctx* ctx, const uint64_t* d_c, size_t batch, uint64_t* d_m, void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_c || !d_m) return fail(PL_EINVAL, "NULL argument");
  if (!ctx->d_shat) return fail(PL_EINVAL, "no secret key prepared");
  if (!batch) return PL_OK;
  if (batch > 0x7fffffff) return fail(PL_ERANGE, "batch too large");
  return ctx->launch_decrypt(d_c, ctx->d_shat, batch, d_m, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
