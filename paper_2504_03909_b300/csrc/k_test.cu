// The Montgomery core on its own, for limb-exact unit tests.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/paillier_testing.h"
#include "check.cuh"
#include "internal.h"
#include "mp.cuh"

namespace pl {
namespace {

constexpr int kBlock = 128;

template <int S, int T>
__global__ void __launch_bounds__(kBlock) k_test_mont_mul(const __grid_constant__ N2Const P,
                                                          const uint32_t* __restrict__ A,
                                                          const uint32_t* __restrict__ B, size_t count,
                                                          uint32_t* __restrict__ out) {
  constexpr int NL = S * T;
  constexpr int IPW = 32 / T;
  extern __shared__ uint32_t smem[];
  const int ipb = blockDim.x / T;
  const int lane = threadIdx.x & 31, k = lane % T, gw = lane / T, g = threadIdx.x / T;
  uint32_t* bs = smem + g;
  uint32_t n[S], a[S], t[S];
  const_slice<S>(n, P.N, k);
  const size_t nchunk = (count + IPW - 1) / IPW;
  const size_t warp0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t c = warp0; c < nchunk; c += nwarps) {
    const size_t i = c * IPW + gw;
    const bool valid = i < count;
    const size_t ii = valid ? i : count - 1;
    load_slice<S>(a, A + ii * NL, k);
    load_slice<S>(t, B + ii * NL, k);
    __syncwarp();
    stage<S>(bs, ipb, t, k);
    __syncwarp();
    mont_mul<S, T>(t, a, bs, ipb, n, P.np, k);
    if (valid) store_slice<S>(out + ii * NL, t, k);
  }
}

// d_out = a b R^-1 mod N (or a^2 R^-1 mod N when B is null) through the SOS
// body of the exponentiations (mont_sos)
template <int S, int T>
__global__ void __launch_bounds__(kBlock) k_test_mont_sos(const __grid_constant__ N2Const P,
                                                          const uint32_t* __restrict__ A,
                                                          const uint32_t* __restrict__ B, size_t count,
                                                          uint32_t* __restrict__ out) {
  constexpr int NL = S * T;
  constexpr int IPW = 32 / T;
  const int lane = threadIdx.x & 31, k = lane % T, gw = lane / T;
  uint32_t n[S], a[S], b[S];
  const_slice<S>(n, P.N, k);
  const bool square = B == nullptr;
  const size_t nchunk = (count + IPW - 1) / IPW;
  const size_t warp0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t c = warp0; c < nchunk; c += nwarps) {
    const size_t i = c * IPW + gw;
    const bool valid = i < count;
    const size_t ii = valid ? i : count - 1;
    load_slice<S>(a, A + ii * NL, k);
    if (square) {
#pragma unroll
      for (int j = 0; j < S; ++j) b[j] = a[j];
    } else {
      load_slice<S>(b, B + ii * NL, k);
    }
    mont_sos<S, T>(a, a, b, n, P.np, k, square);
    if (valid) store_slice<S>(out + ii * NL, a, k);
  }
}

template <int S, int T>
int run_sos(const N2Const& P, const uint32_t* a, const uint32_t* b, size_t count, uint32_t* out, cudaStream_t s) {
  const size_t ipw = 32 / T;
  const size_t blocks = ((count + ipw - 1) / ipw + (kBlock / 32) - 1) / (kBlock / 32);
  const int grid = (int)std::min<size_t>(blocks, 4096);
  k_test_mont_sos<S, T><<<grid, kBlock, 0, s>>>(P, a, b, count, out);
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

template <int S, int T>
int run(const N2Const& P, const uint32_t* a, const uint32_t* b, size_t count, uint32_t* out, cudaStream_t s) {
  const size_t ipw = 32 / T;
  const size_t blocks = ((count + ipw - 1) / ipw + (kBlock / 32) - 1) / (kBlock / 32);
  const int grid = (int)std::min<size_t>(blocks, 4096);
  const size_t smem = (size_t)S * T * (kBlock / T) * sizeof(uint32_t);
  k_test_mont_mul<S, T><<<grid, kBlock, smem, s>>>(P, a, b, count, out);
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
}

}  // namespace
}  // namespace pl

extern "C" int paillier_test_mont_mul(int limbs, int lanes, const uint32_t* h_N, const uint32_t* d_a,
                                      const uint32_t* d_b, size_t count, uint32_t* d_out, void* stream) {
  using namespace pl;
  clear_error();
  if (!h_N || limbs < 1 || limbs > 2 * kMaxL || !(h_N[0] & 1u) || h_N[limbs - 1] == 0)
    return fail(PL_EINVAL, "modulus must be odd with a non-zero top limb");
  if (count == 0) return PL_OK;
  if (!d_a || !d_b || !d_out) return fail(PL_EINVAL, "NULL buffer");
  N2Const P;
  std::memset(&P, 0, sizeof(P));
  std::memcpy(P.N, h_N, sizeof(uint32_t) * (size_t)limbs);
  P.np = plh::neg_inv32(h_N[0]);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
#define PL_CASE(LL, TT) \
  if (limbs == LL && lanes == TT) return run<LL / TT, TT>(P, d_a, d_b, count, d_out, s);
  PL_CASE(32, 2) PL_CASE(32, 4) PL_CASE(64, 2) PL_CASE(64, 4) PL_CASE(64, 8) PL_CASE(96, 4) PL_CASE(96, 8)
  PL_CASE(128, 4) PL_CASE(128, 8) PL_CASE(192, 8) PL_CASE(192, 16)
#undef PL_CASE
  return fail(PL_EINVAL, "no compiled kernel for this (limbs, lanes) pair");
}

extern "C" int paillier_test_mont_sos(int limbs, int lanes, const uint32_t* h_N, const uint32_t* d_a,
                                      const uint32_t* d_b, size_t count, uint32_t* d_out, void* stream) {
  using namespace pl;
  clear_error();
  if (!h_N || limbs < 1 || limbs > kMaxL || !(h_N[0] & 1u) || h_N[limbs - 1] == 0)
    return fail(PL_EINVAL, "modulus must be odd with a non-zero top limb");
  if (count == 0) return PL_OK;
  if (!d_a || !d_out) return fail(PL_EINVAL, "NULL buffer");
  N2Const P;
  std::memset(&P, 0, sizeof(P));
  std::memcpy(P.N, h_N, sizeof(uint32_t) * (size_t)limbs);
  P.np = plh::neg_inv32(h_N[0]);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
#define PL_CASE(LL, TT) \
  if (limbs == LL && lanes == TT) return run_sos<LL / TT, TT>(P, d_a, d_b, count, d_out, s);
  PL_CASE(32, 2) PL_CASE(32, 4) PL_CASE(64, 4) PL_CASE(64, 8) PL_CASE(96, 4) PL_CASE(96, 8)
#undef PL_CASE
  return fail(PL_EINVAL, "no compiled SOS kernel for this (limbs, lanes) pair");
}

#ifdef PL_CHECKED
namespace {
__global__ void k_bounds_report(int site) { PL_BOUNDS(false, site); }
}  // namespace
#endif

extern "C" int paillier_test_bounds_report(int site, void* stream) {
  using namespace pl;
  clear_error();
  if (site < 0 || site > 30) return fail(PL_EINVAL, "site must be 0..30");
#ifdef PL_CHECKED
  k_bounds_report<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(site);
  PL_CUDA_TRY(cudaGetLastError());
  return PL_OK;
#else
  (void)stream;
  return fail(PL_EINVAL, "not a checked build");
#endif
}

extern "C" int paillier_test_schedule_ops(const pl_key* key, int dec, int w, int* nop, int* nop1) {
  using namespace pl;
  clear_error();
  if (!key || !nop) return fail(PL_EINVAL, "NULL argument");
  if (!key->priv) return fail(PL_EINVAL, "a public key has no exponentiation schedules");
  const ModexpParams* P = const_cast<pl_key*>(key)->modexp_params(dec != 0, w);
  if (!P) return fail(PL_EINVAL, "unsupported window width");
  for (int h = 0; h < 2; ++h) {
    nop[h] = P->nop[h];
    if (nop1) nop1[h] = dec ? 0 : P->nop1[h];
  }
  return PL_OK;
}
