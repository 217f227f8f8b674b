// CKKS for the secure horizontal pattern: negacyclic NTT over one 62-bit prime,
// canonical-embedding encoding/decoding, public-key encryption, addition and
// decryption (see include/ckks.h).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/ckks.h"
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

struct NttConst {
  u64 q, qn, r2, ninv;  // ninv in Montgomery form
  int log_n;
};

// In-place negacyclic NTT of one polynomial per block (shared memory).
// Forward: Cooley-Tukey, natural order in, bit-reversed order out, twiddles
// psi^bitrev(i) (Montgomery form).  Inverse: Gentleman-Sande back to natural
// order, then the factor N^-1.
__global__ void k_ntt(u64* __restrict__ data, const u64* __restrict__ tw, NttConst C, int inverse) {
  extern __shared__ u64 a[];
  const int N = 1 << C.log_n;
  u64* p = data + (size_t)blockIdx.x * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) a[i] = p[i];
  __syncthreads();
  const u64 q = C.q, qn = C.qn;
  if (!inverse) {
    for (int m = 1, t = N >> 1; m < N; m <<= 1, t >>= 1) {
      for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
        const int i = b / t, j = b - i * t, idx = 2 * i * t + j;
        const u64 U = a[idx], V = mmul(a[idx + t], tw[m + i], q, qn);
        a[idx] = addm(U, V, q);
        a[idx + t] = subm(U, V, q);
      }
      __syncthreads();
    }
  } else {
    for (int m = N, t = 1; m > 1; m >>= 1, t <<= 1) {
      const int h = m >> 1;
      for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
        const int i = b / t, j = b - i * t, idx = 2 * i * t + j;
        const u64 U = a[idx], V = a[idx + t];
        a[idx] = addm(U, V, q);
        a[idx + t] = mmul(subm(U, V, q), tw[h + i], q, qn);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) a[i] = mmul(a[i], C.ninv, q, qn);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) p[i] = a[i];
}

// out[i] = x[i] y[i mod period] mod q  (period = N broadcasts one polynomial)
// (out may alias x)
__global__ void k_pointwise(const u64* x, const u64* __restrict__ y, size_t period, size_t count, NttConst C,
                            u64* out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = mmul(mmul(x[i], y[i % period], C.q, C.qn), C.r2, C.q, C.qn);
}

template <typename T>
__global__ void k_to_modq(const T* __restrict__ x, size_t count, u64 q, u64* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = smod((long long)x[i], q);
}

// b = -(a s) + e
__global__ void k_keygen_finish(const u64* __restrict__ as, const int32_t* __restrict__ e, int N, u64 q,
                                u64* __restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    b[i] = addm(subm(0, as[i], q), smod(e[i], q), q);
}

// c0 = bv + e0 + m, c1 = av + e1 for every message (bv, av [batch][N])
__global__ void k_encrypt_finish(const u64* __restrict__ bv, const u64* __restrict__ av,
                                 const int32_t* __restrict__ e0, const int32_t* __restrict__ e1,
                                 const int64_t* __restrict__ m, size_t batch, int N, u64 q, u64* __restrict__ c) {
  const size_t count = batch * (size_t)N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / N, k = i % N;
    c[(p * 2) * N + k] = addm(addm(bv[i], smod(e0[i], q), q), smod(m[i], q), q);
    c[(p * 2 + 1) * N + k] = addm(av[i], smod(e1[i], q), q);
  }
}

// m = c0 + (c1 s)
__global__ void k_decrypt_finish(const u64* __restrict__ c, const u64* __restrict__ c1s, size_t batch, int N, u64 q,
                                 u64* __restrict__ m) {
  const size_t count = batch * (size_t)N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / N, k = i % N;
    m[i] = addm(c[(p * 2) * N + k], c1s[i], q);
  }
}

// gather c1 of every ciphertext into a contiguous [batch][N] array
__global__ void k_take_c1(const u64* __restrict__ c, size_t batch, int N, u64* __restrict__ out) {
  const size_t count = batch * (size_t)N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = c[(i / N * 2 + 1) * N + i % N];
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

// m_k = rint((2 scale / N) sum_j (cos(pi r_j k / N) re_j + sin(pi r_j k / N) im_j))
__global__ void k_encode(const double* __restrict__ re, const double* __restrict__ im, size_t batch, int log_n,
                         const int32_t* __restrict__ r, const double* __restrict__ cs, const double* __restrict__ sn,
                         double scale, int64_t* __restrict__ m) {
  const int N = 1 << log_n, n = N / 2, mask = 2 * N - 1;
  const size_t count = batch * (size_t)N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / N;
    const long long k = (long long)(i % N);
    const double* zr = re + p * n;
    const double* zi = im + p * n;
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      const int t = (int)((k * r[j]) & mask);
      s += cs[t] * zr[j] + sn[t] * zi[j];
    }
    m[i] = (int64_t)rint(s * (2.0 * scale / N));
  }
}

// z_j = sum_k m_k exp(i pi r_j k / N) / scale, m centred
__global__ void k_decode(const u64* __restrict__ m, size_t batch, int log_n, u64 q, const int32_t* __restrict__ r,
                         const double* __restrict__ cs, const double* __restrict__ sn, double scale,
                         double* __restrict__ re, double* __restrict__ im) {
  const int N = 1 << log_n, n = N / 2, mask = 2 * N - 1;
  const size_t count = batch * (size_t)n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / n, j = i % n;
    const u64* mp = m + p * N;
    const long long rj = r[j];
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < N; ++k) {
      const u64 x = mp[k];
      const double v = x > q / 2 ? -(double)(q - x) : (double)x;
      const int t = (int)((rj * k) & mask);
      sr += v * cs[t];
      si += v * sn[t];
    }
    re[i] = sr / scale;
    im[i] = si / scale;
  }
}

int ew_grid(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)pl::sm_count() * 8); }

}  // namespace

struct ckks_ctx {
  int log_n = 0, N = 0, device = 0;
  double scale = 1.0;
  NttConst C{};
  u64* d_tw = nullptr;   // forward twiddles psi^bitrev(i), Montgomery form
  u64* d_itw = nullptr;  // inverse twiddles psi^-bitrev(i), Montgomery form
  int32_t* d_r = nullptr;
  double* d_cos = nullptr;
  double* d_sin = nullptr;
  pl::Scratch scratch;

  ~ckks_ctx() {
    cudaFree(d_tw);
    cudaFree(d_itw);
    cudaFree(d_r);
    cudaFree(d_cos);
    cudaFree(d_sin);
  }

  pl_status ntt(u64* polys, size_t count, bool inverse, cudaStream_t s) {
    const int threads = std::min(N / 2, 1024);
    k_ntt<<<(unsigned)count, threads, (size_t)N * sizeof(u64), s>>>(polys, inverse ? d_itw : d_tw, C, inverse);
    pl::note_launch();
    PL_CUDA_TRY(cudaGetLastError());
    return PL_OK;
  }
};

extern "C" {

pl_status ckks_create(int log_n, uint64_t q, double scale, ckks_ctx** out) {
  using namespace pl;
  clear_error();
  if (!out || log_n < 4 || log_n > 14 || !(scale > 0)) return fail(PL_EINVAL, "need 4 <= log_n <= 14, scale > 0");
  const int N = 1 << log_n;
  if (q >= (1ull << 62) || q < 3 || q % (2ull * N) != 1 || !h_prime(q))
    return fail(PL_EINVAL, "q must be a prime < 2^62 with q = 1 mod 2N");
  auto* c = new (std::nothrow) ckks_ctx();
  if (!c) return fail(PL_ENOMEM, "host allocation failed");
  c->log_n = log_n;
  c->N = N;
  c->scale = scale;
  cudaGetDevice(&c->device);
  // primitive 2N-th root of unity
  u64 psi = 0;
  for (u64 g = 2; g < 1000 && !psi; ++g) {
    const u64 x = h_pow(g, (q - 1) / (2ull * N), q);
    if (h_pow(x, (u64)N, q) == q - 1) psi = x;
  }
  if (!psi) { delete c; return fail(PL_EINVAL, "no primitive 2N-th root found"); }
  const u64 R = (u64)(((u128)1 << 64) % q);
  u64 qinv = 1;
  for (int i = 0; i < 6; ++i) qinv *= 2 - q * qinv;
  c->C.q = q;
  c->C.qn = (u64)0 - qinv;
  c->C.r2 = h_mul(R, R, q);
  c->C.ninv = h_mul(h_pow((u64)N, q - 2, q), R, q);
  c->C.log_n = log_n;
  std::vector<u64> tw(N), itw(N);
  const u64 ipsi = h_pow(psi, q - 2, q);
  for (int i = 0; i < N; ++i) {
    const int e = bitrev(i, log_n);
    tw[i] = h_mul(h_pow(psi, (u64)e, q), R, q);
    itw[i] = h_mul(h_pow(ipsi, (u64)e, q), R, q);
  }
  std::vector<int32_t> r(N / 2);
  u64 x = 1;
  for (int j = 0; j < N / 2; ++j) { r[j] = (int32_t)x; x = x * 5 % (2ull * N); }
  std::vector<double> cs(2 * N), sn(2 * N);
  for (int t = 0; t < 2 * N; ++t) {
    cs[t] = std::cos(M_PI * t / N);
    sn[t] = std::sin(M_PI * t / N);
  }
  cudaError_t e = cudaSuccess;
  auto up = [&](void** d, const void* h, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(d, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice);
  };
  up((void**)&c->d_tw, tw.data(), N * sizeof(u64));
  up((void**)&c->d_itw, itw.data(), N * sizeof(u64));
  up((void**)&c->d_r, r.data(), r.size() * sizeof(int32_t));
  up((void**)&c->d_cos, cs.data(), cs.size() * sizeof(double));
  up((void**)&c->d_sin, sn.data(), sn.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ntt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((1 << 14) * sizeof(u64)));
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "ckks tables"); }
  c->scratch.device = c->device;
  *out = c;
  return PL_OK;
}

void ckks_free(ckks_ctx* ctx) { delete ctx; }

int ckks_slots(const ckks_ctx* ctx) { return ctx ? ctx->N / 2 : 0; }

pl_status ckks_encode(ckks_ctx* ctx, const double* d_re, const double* d_im, size_t batch, int64_t* d_m,
                      void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx) return fail(PL_EINVAL, "ctx is NULL");
  if (!batch) return PL_OK;
  if (!d_re || !d_im || !d_m) return fail(PL_EINVAL, "NULL buffer");
  const size_t n = batch * (size_t)ctx->N;
  k_encode<<<ew_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_re, d_im, batch, ctx->log_n, ctx->d_r,
                                                                      ctx->d_cos, ctx->d_sin, ctx->scale, d_m);
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
  const size_t n = batch * (size_t)(ctx->N / 2);
  k_decode<<<ew_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_m, batch, ctx->log_n, ctx->C.q, ctx->d_r,
                                                                      ctx->d_cos, ctx->d_sin, ctx->scale, d_re, d_im);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

pl_status ckks_keygen(ckks_ctx* ctx, const int8_t* d_s, const uint64_t* d_a, const int32_t* d_e, uint64_t* d_b,
                      void* stream) {
  using namespace pl;
  clear_error();
  if (!ctx || !d_s || !d_a || !d_e || !d_b) return fail(PL_EINVAL, "NULL argument");
  const int N = ctx->N;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* t = static_cast<u64*>(ctx->scratch.get(2 * (size_t)N * sizeof(u64), s));
  if (!t) return fail(PL_ENOMEM, "scratch");
  u64 *ta = t, *ts = t + N;
  PL_CUDA_TRY(cudaMemcpyAsync(ta, d_a, N * sizeof(u64), cudaMemcpyDeviceToDevice, s));
  k_to_modq<int8_t><<<ew_grid(N), 256, 0, s>>>(d_s, N, ctx->C.q, ts);
  note_launch();
  pl_status rc = ctx->ntt(ta, 1, false, s);
  if (!rc) rc = ctx->ntt(ts, 1, false, s);
  if (rc) return rc;
  k_pointwise<<<ew_grid(N), 256, 0, s>>>(ta, ts, N, N, ctx->C, ta);
  note_launch();
  rc = ctx->ntt(ta, 1, true, s);
  if (rc) return rc;
  k_keygen_finish<<<ew_grid(N), 256, 0, s>>>(ta, d_e, N, ctx->C.q, d_b);
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
  const size_t N = (size_t)ctx->N, n = batch * N;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // tb, ta: the key in the transform domain; tv: v; bv, av: products
  auto* t = static_cast<u64*>(ctx->scratch.get((2 * N + 3 * n) * sizeof(u64), s));
  if (!t) return fail(PL_ENOMEM, "scratch");
  u64 *tb = t, *ta = t + N, *tv = t + 2 * N, *bv = tv + n, *av = bv + n;
  PL_CUDA_TRY(cudaMemcpyAsync(tb, d_b, N * sizeof(u64), cudaMemcpyDeviceToDevice, s));
  PL_CUDA_TRY(cudaMemcpyAsync(ta, d_a, N * sizeof(u64), cudaMemcpyDeviceToDevice, s));
  k_to_modq<int8_t><<<ew_grid(n), 256, 0, s>>>(d_v, n, ctx->C.q, tv);
  note_launch();
  pl_status rc = ctx->ntt(tb, 1, false, s);
  if (!rc) rc = ctx->ntt(ta, 1, false, s);
  if (!rc) rc = ctx->ntt(tv, batch, false, s);
  if (rc) return rc;
  k_pointwise<<<ew_grid(n), 256, 0, s>>>(tv, tb, N, n, ctx->C, bv);
  k_pointwise<<<ew_grid(n), 256, 0, s>>>(tv, ta, N, n, ctx->C, av);
  note_launch();
  note_launch();
  rc = ctx->ntt(bv, batch, true, s);
  if (!rc) rc = ctx->ntt(av, batch, true, s);
  if (rc) return rc;
  k_encrypt_finish<<<ew_grid(n), 256, 0, s>>>(bv, av, d_e0, d_e1, d_m, batch, (int)N, ctx->C.q, d_c);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
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
  const size_t N = (size_t)ctx->N, n = batch * N;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* t = static_cast<u64*>(ctx->scratch.get((N + n) * sizeof(u64), s));
  if (!t) return fail(PL_ENOMEM, "scratch");
  u64 *ts = t, *c1 = t + N;
  k_to_modq<int8_t><<<ew_grid(N), 256, 0, s>>>(d_s, N, ctx->C.q, ts);
  k_take_c1<<<ew_grid(n), 256, 0, s>>>(d_c, batch, (int)N, c1);
  note_launch();
  note_launch();
  pl_status rc = ctx->ntt(ts, 1, false, s);
  if (!rc) rc = ctx->ntt(c1, batch, false, s);
  if (rc) return rc;
  k_pointwise<<<ew_grid(n), 256, 0, s>>>(c1, ts, N, n, ctx->C, c1);
  note_launch();
  rc = ctx->ntt(c1, batch, true, s);
  if (rc) return rc;
  k_decrypt_finish<<<ew_grid(n), 256, 0, s>>>(d_c, c1, batch, (int)N, ctx->C.q, d_m);
  note_launch();
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

}  // extern "C"
