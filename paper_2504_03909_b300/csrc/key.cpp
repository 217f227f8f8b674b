// Key generation, import/export and the per-key precomputation: Montgomery
// constants of n^2, p^2, q^2, the CRT constants of encryption and of
// decryption (Paillier 1999, Sec. 7), and the sliding-window exponentiation schedules.
#include <cstring>

#include "internal.h"

using plh::Big;

namespace {

bool supported_bits(int n_bits) { return n_bits == 1024 || n_bits == 2048 || n_bits == 3072; }

void put(uint32_t* dst, const Big& v, int limbs) {
  std::vector<uint32_t> x = v.to_limbs((size_t)limbs);
  std::memcpy(dst, x.data(), sizeof(uint32_t) * (size_t)limbs);
}

Big pow2(int bits) { return plh::shl_bits(Big(1), bits); }

// Montgomery constants of an odd modulus N with R = 2^(32 limbs)
void mont_consts(const Big& N, int limbs, uint32_t* np, Big* R1, Big* R2) {
  *np = plh::neg_inv32(N.d[0]);
  *R1 = plh::mod(pow2(32 * limbs), N);
  *R2 = plh::mod(plh::mul(*R1, *R1), N);
}

void fill_public(pl_key* k) {
  const int L = k->L;
  k->n2 = plh::mul(k->n, k->n);
  Big R1, R2;
  mont_consts(k->n2, 2 * L, &k->n2c.np, &R1, &R2);
  put(k->n2c.N, k->n2, 2 * L);
  put(k->n2c.R2, R2, 2 * L);
}

// lanes x tile of the histogram products: 8x16 for 1024 and 2048 bits, 16x16 for 3072
pl::AggCfg default_agg(int L) { return {L == 96 ? 16 : 8, 16}; }

// Everything the key holder's kernels need.
void fill_private(pl_key* k) {
  const int L = k->L, Lh = k->Lh;
  const Big& p = k->p;
  const Big& q = k->q;
  const Big g = plh::add(k->n, Big(1));
  const Big P2[2] = {plh::mul(p, p), plh::mul(q, q)};
  const Big X[2] = {p, q};
  Big R1s[2];
  for (int h = 0; h < 2; ++h) {
    pl::HalfConst& H = k->half[h];
    Big R1, R2;
    mont_consts(P2[h], L, &H.np, &R1, &R2);
    const Big R3 = plh::mod(plh::mul(R2, R1), P2[h]);
    const Big nR = plh::mod(plh::mul(plh::mod(k->n, P2[h]), R1), P2[h]);
    put(H.N, P2[h], L);
    put(H.R1, R1, L);
    put(H.R2, R2, L);
    put(H.R3, R3, L);
    put(H.nR, nR, L);
    R1s[h] = R1;
    // arithmetic mod the prime x itself (L/2 limbs)
    Big R1x, R2x;
    mont_consts(X[h], Lh, &H.npx, &R1x, &R2x);
    const Big R3x = plh::mod(plh::mul(R2x, R1x), X[h]);
    put(H.Nx, X[h], Lh);
    put(H.R1x, R1x, Lh);
    put(H.R2x, R2x, Lh);
    put(H.R3x, R3x, Lh);
    // r^n mod x^2 = ((r mod x)^(x' mod (x - 1)) mod x)^x mod x^2, x' the other prime
    k->e_enc1[h] = plh::mod(X[1 - h], plh::sub(X[h], Big(1)));
    k->e_enc2[h] = X[h];
  }
  k->e_dec[0] = plh::sub(p, Big(1));
  k->e_dec[1] = plh::sub(q, Big(1));

  // encryption CRT: c = c_q + q^2 ((c_p - c_q) (q^2)^-1 mod p^2)
  {
    plh::Mont Mp2(P2[0]);
    // (q^2)^-1 mod p^2 by Euler: x^(phi(p^2) - 1), phi(p^2) = p (p - 1)
    const Big phi = plh::mul(p, plh::sub(p, Big(1)));
    const Big q2inv = Mp2.pow(P2[1], plh::sub(phi, Big(1)));
    const Big QinvR = plh::mod(plh::mul(q2inv, R1s[0]), P2[0]);
    put(k->enc.p2, P2[0], L);
    put(k->enc.q2, P2[1], L);
    put(k->enc.QinvR, QinvR, L);
    k->enc.p2_np = k->half[0].np;
    k->enc.L = L;
  }
  // decryption CRT constants
  {
    const Big pr[2] = {p, q};
    Big hR[2];
    for (int h = 0; h < 2; ++h) {
      plh::Mont Mx2(P2[h]);
      const Big gx = Mx2.pow(g, plh::sub(pr[h], Big(1)));  // g^(x-1) mod x^2
      Big Lx, rem;
      plh::divmod(plh::sub(gx, Big(1)), pr[h], &Lx, &rem);  // L_x(g^(x-1) mod x^2)
      plh::Mont Mx(pr[h]);
      const Big hx = Mx.pow(Lx, plh::sub(pr[h], Big(2)));   // inverse mod the prime x
      hR[h] = plh::mod(plh::mul(hx, Mx.R1), pr[h]);
    }
    plh::Mont Mp(p);
    const Big qinv = Mp.pow(plh::mod(q, p), plh::sub(p, Big(2)));
    const Big qinvR = plh::mod(plh::mul(qinv, Mp.R1), p);
    put(k->dec.p, p, Lh);
    put(k->dec.q, q, Lh);
    put(k->dec.pinv, plh::inv_pow2(p, (size_t)Lh), Lh);
    put(k->dec.qinv2k, plh::inv_pow2(q, (size_t)Lh), Lh);
    put(k->dec.hpR, hR[0], Lh);
    put(k->dec.hqR, hR[1], Lh);
    put(k->dec.qinvR, qinvR, Lh);
    k->dec.p_np = plh::neg_inv32(p.d[0]);
    k->dec.q_np = plh::neg_inv32(q.d[0]);
    k->dec.Lh = Lh;
  }
  // default launch configuration by key size, from measurements on B300 (148
  // SMs): lanes 2 / 4 / 8 for 1024 / 2048 / 3072 bits; sliding windows of 6 bits
  // from 2048 bits up (32 odd powers per instance; +0.4 % / +1.1 % over 5 bits
  // at 2048 / 3072 bits, full-size launches), 5 bits for 1024
  const int T_half = (L == 32) ? 2 : (L == 64 ? 4 : 8);
  const int w = (L == 32) ? 5 : 6;
  k->enc_cfg = {T_half, w};
  k->dec_cfg = {T_half, w};
  k->agg_cfg = default_agg(L);
}

bool check_prime_shape(const Big& x, int half_bits) {
  return x.bits() == half_bits && x.bit(half_bits - 1) && x.bit(half_bits - 2) && x.is_odd();
}

pl_status make_private(int n_bits, const Big& p, const Big& q, pl_key** out) {
  const int half = n_bits / 2;
  if (!check_prime_shape(p, half) || !check_prime_shape(q, half))
    return pl::fail(PL_EINVAL, "p and q must be odd n_bits/2-bit numbers with the top two bits set");
  if (plh::cmp(p, q) == 0) return pl::fail(PL_EINVAL, "p == q");
  auto* k = new (std::nothrow) pl_key();
  if (!k) return pl::fail(PL_ENOMEM, "host allocation failed");
  k->n_bits = n_bits;
  k->L = n_bits / 32;
  k->Lh = k->L / 2;
  k->priv = true;
  k->p = p;
  k->q = q;
  k->n = plh::mul(p, q);
  if (k->n.bits() != n_bits) {
    delete k;
    return pl::fail(PL_EINVAL, "p q does not have n_bits bits");
  }
  fill_public(k);
  fill_private(k);
  *out = k;
  return PL_OK;
}

}  // namespace

const pl::ModexpParams* pl_key::modexp_params(bool dec, int w) {
  if (w < 2 || w > 7) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  auto& cache = dec ? dec_params : enc_params;
  auto it = cache.find(w);
  if (it != cache.end()) return it->second.get();
  auto P = std::make_unique<pl::ModexpParams>();
  std::memset(P.get(), 0, sizeof(pl::ModexpParams));
  for (int h = 0; h < 2; ++h) {
    P->half[h] = half[h];
    P->nop[h] = pl::sliding_schedule(dec ? e_dec[h] : e_enc2[h], w, P->op[h], pl::kMaxOps);
    if (P->nop[h] < 0) return nullptr;
    if (!dec) {
      P->nop1[h] = pl::sliding_schedule(e_enc1[h], w, P->op1[h], pl::kMaxOps);
      if (P->nop1[h] < 0) return nullptr;
    }
  }
  P->w = w;
  const pl::ModexpParams* raw = P.get();
  cache[w] = std::move(P);
  return raw;
}

namespace pl {

int sliding_schedule(const plh::Big& e, int w, uint8_t* op, int maxops) {
  int i = e.bits() - 1;  // the top bit is set
  if (i < 0 || w < 1 || w > 8) return -1;
  int n = 0;
  while (i >= 0) {
    if (!e.bit(i)) {  // a zero outside a window: one squaring
      if (n >= maxops) return -1;
      op[n++] = 0;
      --i;
      continue;
    }
    // the window: bits i .. j, at most w of them, ending in a set bit
    int j = i - w + 1 > 0 ? i - w + 1 : 0;
    while (!e.bit(j)) ++j;
    int v = 0;
    for (int b = i; b >= j; --b) v = (v << 1) | (int)e.bit(b);
    const int len = i - j + 1;
    if (n == 0) {
      op[n++] = (uint8_t)v;  // start from base^v
    } else {
      if (n + len + 1 > maxops) return -1;
      for (int s = 0; s < len; ++s) op[n++] = 0;
      op[n++] = (uint8_t)v;
    }
    i = j - 1;
  }
  return n;
}

}  // namespace pl

pl::Scratch* pl_key::scratch_for_current_device(bool aux) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  auto& s = aux ? scratch_aux[dev] : scratch[dev];
  if (!s) {
    s = std::make_unique<pl::Scratch>();
    s->device = dev;
  }
  return s.get();
}

extern "C" {

pl_status paillier_keygen(int n_bits, uint64_t seed, pl_key** out) {
  pl::clear_error();
  if (!out) return pl::fail(PL_EINVAL, "out is NULL");
  if (!supported_bits(n_bits)) return pl::fail(PL_EINVAL, "n_bits must be 1024, 2048 or 3072");
  const int half = n_bits / 2;
  plh::SplitMix64 rng(seed ^ 0x5041494c4c494552ull);
  auto draw = [&]() {
    for (;;) {
      Big x;
      x.d.resize((size_t)half / 32);
      for (auto& w : x.d) w = (uint32_t)rng.next();
      x.d.back() |= 0xC0000000u;  // top two bits set
      x.d[0] |= 1u;
      x.trim();
      if (plh::probable_prime(x, 64, rng)) return x;
    }
  };
  for (;;) {
    Big p = draw(), q = draw();
    if (plh::cmp(p, q) == 0) continue;
    Big n = plh::mul(p, q);
    if (n.bits() != n_bits) continue;
    Big phi = plh::mul(plh::sub(p, Big(1)), plh::sub(q, Big(1)));
    Big gg = plh::gcd(n, phi);
    if (plh::cmp(gg, Big(1)) != 0) continue;
    return make_private(n_bits, p, q, out);
  }
}

pl_status paillier_key_import(int n_bits, const uint32_t* h_p, const uint32_t* h_q, pl_key** out) {
  pl::clear_error();
  if (!out || !h_p || !h_q) return pl::fail(PL_EINVAL, "NULL argument");
  if (!supported_bits(n_bits)) return pl::fail(PL_EINVAL, "n_bits must be 1024, 2048 or 3072");
  const size_t lh = (size_t)n_bits / 64;
  return make_private(n_bits, Big::from_limbs(h_p, lh), Big::from_limbs(h_q, lh), out);
}

pl_status paillier_key_import_public(int n_bits, const uint32_t* h_n, pl_key** out) {
  pl::clear_error();
  if (!out || !h_n) return pl::fail(PL_EINVAL, "NULL argument");
  if (!supported_bits(n_bits)) return pl::fail(PL_EINVAL, "n_bits must be 1024, 2048 or 3072");
  Big n = Big::from_limbs(h_n, (size_t)n_bits / 32);
  if (n.bits() != n_bits || !n.is_odd()) return pl::fail(PL_EINVAL, "n must be odd with exactly n_bits bits");
  auto* k = new (std::nothrow) pl_key();
  if (!k) return pl::fail(PL_ENOMEM, "host allocation failed");
  k->n_bits = n_bits;
  k->L = n_bits / 32;
  k->Lh = k->L / 2;
  k->priv = false;
  k->n = n;
  fill_public(k);
  k->agg_cfg = default_agg(k->L);
  *out = k;
  return PL_OK;
}

pl_status paillier_key_export(const pl_key* key, uint32_t* h_n, uint32_t* h_p, uint32_t* h_q) {
  pl::clear_error();
  if (!key) return pl::fail(PL_EINVAL, "key is NULL");
  if (h_n) put(h_n, key->n, key->L);
  if ((h_p || h_q) && !key->priv) return pl::fail(PL_EINVAL, "public key has no p, q");
  if (h_p) put(h_p, key->p, key->Lh);
  if (h_q) put(h_q, key->q, key->Lh);
  return PL_OK;
}

int paillier_key_bits(const pl_key* key) { return key ? key->n_bits : 0; }
int paillier_key_is_private(const pl_key* key) { return key && key->priv ? 1 : 0; }

void paillier_key_free(pl_key* key) { delete key; }

}  // extern "C"
