// Host multi-precision integers for key set-up only (prime search, the
// Montgomery constants and the CRT constants of a key).  Nothing here runs per
// ciphertext; the device kernels carry their own arithmetic.
#pragma once

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace plh {

// Unsigned integer, little-endian 32-bit limbs, no leading zero limbs
// (zero is the empty vector).
struct Big {
  std::vector<uint32_t> d;

  Big() = default;
  explicit Big(uint64_t v) {
    while (v) { d.push_back((uint32_t)v); v >>= 32; }
  }
  static Big from_limbs(const uint32_t* p, size_t n) {
    Big b; b.d.assign(p, p + n); b.trim(); return b;
  }
  void trim() { while (!d.empty() && d.back() == 0) d.pop_back(); }
  bool is_zero() const { return d.empty(); }
  size_t limbs() const { return d.size(); }
  uint32_t limb(size_t i) const { return i < d.size() ? d[i] : 0u; }
  int bits() const {
    if (d.empty()) return 0;
    return 32 * (int)(d.size() - 1) + (32 - __builtin_clz(d.back()));
  }
  bool bit(int i) const { return (limb((size_t)i / 32) >> (i % 32)) & 1u; }
  bool is_odd() const { return !d.empty() && (d[0] & 1u); }
  // fixed-width little-endian export (the value must fit)
  std::vector<uint32_t> to_limbs(size_t n) const {
    std::vector<uint32_t> out(n, 0);
    for (size_t i = 0; i < d.size() && i < n; ++i) out[i] = d[i];
    return out;
  }
};

inline int cmp(const Big& a, const Big& b) {
  if (a.d.size() != b.d.size()) return a.d.size() < b.d.size() ? -1 : 1;
  for (size_t i = a.d.size(); i-- > 0;)
    if (a.d[i] != b.d[i]) return a.d[i] < b.d[i] ? -1 : 1;
  return 0;
}

inline Big add(const Big& a, const Big& b) {
  Big r; size_t n = a.d.size() > b.d.size() ? a.d.size() : b.d.size();
  r.d.resize(n + 1);
  uint64_t c = 0;
  for (size_t i = 0; i < n; ++i) { c += (uint64_t)a.limb(i) + b.limb(i); r.d[i] = (uint32_t)c; c >>= 32; }
  r.d[n] = (uint32_t)c; r.trim(); return r;
}

// a - b, requires a >= b
inline Big sub(const Big& a, const Big& b) {
  Big r; r.d.resize(a.d.size());
  int64_t br = 0;
  for (size_t i = 0; i < a.d.size(); ++i) {
    int64_t t = (int64_t)a.d[i] - (int64_t)b.limb(i) - br;
    br = t < 0; r.d[i] = (uint32_t)(t + (br ? (int64_t)1 << 32 : 0));
  }
  r.trim(); return r;
}

inline Big mul(const Big& a, const Big& b) {
  if (a.is_zero() || b.is_zero()) return Big();
  Big r; r.d.assign(a.d.size() + b.d.size(), 0);
  for (size_t i = 0; i < a.d.size(); ++i) {
    uint64_t c = 0;
    for (size_t j = 0; j < b.d.size(); ++j) {
      c += (uint64_t)a.d[i] * b.d[j] + r.d[i + j];
      r.d[i + j] = (uint32_t)c; c >>= 32;
    }
    r.d[i + b.d.size()] = (uint32_t)c;
  }
  r.trim(); return r;
}

inline Big shl_bits(const Big& a, int s) {
  if (a.is_zero()) return Big();
  int w = s / 32, b = s % 32;
  Big r; r.d.assign(a.d.size() + w + 1, 0);
  for (size_t i = 0; i < a.d.size(); ++i) {
    uint64_t v = (uint64_t)a.d[i] << b;
    r.d[i + w] |= (uint32_t)v;
    r.d[i + w + 1] |= (uint32_t)(v >> 32);
  }
  r.trim(); return r;
}

inline Big shr_bits(const Big& a, int s) {
  int w = s / 32, b = s % 32;
  if ((size_t)w >= a.d.size()) return Big();
  Big r; r.d.assign(a.d.size() - w, 0);
  for (size_t i = 0; i < r.d.size(); ++i) {
    uint64_t v = a.limb(i + w) | ((uint64_t)a.limb(i + w + 1) << 32);
    r.d[i] = (uint32_t)(v >> b);
  }
  r.trim(); return r;
}

// Binary long division: q = a / m, r = a mod m (m != 0).  O(bits * limbs);
// used only a handful of times per key.
inline void divmod(const Big& a, const Big& m, Big* q, Big* r) {
  Big rem, quo;
  int nb = a.bits();
  if (q) quo.d.assign((size_t)(nb + 31) / 32 + 1, 0);
  for (int i = nb - 1; i >= 0; --i) {
    rem = shl_bits(rem, 1);
    if (a.bit(i)) { if (rem.d.empty()) rem.d.push_back(1); else rem.d[0] |= 1u; }
    if (cmp(rem, m) >= 0) {
      rem = sub(rem, m);
      if (q) quo.d[(size_t)i / 32] |= 1u << (i % 32);
    }
  }
  if (q) { quo.trim(); *q = quo; }
  if (r) *r = rem;
}

inline Big mod(const Big& a, const Big& m) { Big r; divmod(a, m, nullptr, &r); return r; }

// -m^-1 mod 2^32 for odd m (Newton iteration)
inline uint32_t neg_inv32(uint32_t m0) {
  uint32_t x = 1;
  for (int i = 0; i < 5; ++i) x *= 2u - m0 * x;
  return (uint32_t)(0u - x);
}

// Montgomery context for an odd modulus N of s limbs, R = 2^(32 s).
struct Mont {
  Big N; size_t s = 0; uint32_t np = 0; Big R1, R2;
  explicit Mont(const Big& n) : N(n), s(n.limbs()), np(neg_inv32(n.d[0])) {
    Big R = shl_bits(Big(1), 32 * (int)s);
    R1 = mod(R, N);
    R2 = mod(mul(R1, R1), N);
  }
  // a * b * R^-1 mod N for a, b < N (textbook CIOS)
  Big mm(const Big& a, const Big& b) const {
    std::vector<uint32_t> t(s + 2, 0);
    for (size_t i = 0; i < s; ++i) {
      uint64_t c = 0; uint32_t bi = b.limb(i);
      for (size_t j = 0; j < s; ++j) { c += (uint64_t)a.limb(j) * bi + t[j]; t[j] = (uint32_t)c; c >>= 32; }
      c += t[s]; t[s] = (uint32_t)c; t[s + 1] = (uint32_t)(c >> 32);
      uint32_t m = t[0] * np;
      c = ((uint64_t)m * N.d[0] + t[0]) >> 32;
      for (size_t j = 1; j < s; ++j) { c += (uint64_t)m * N.d[j] + t[j]; t[j - 1] = (uint32_t)c; c >>= 32; }
      c += t[s]; t[s - 1] = (uint32_t)c; c >>= 32;
      t[s] = t[s + 1] + (uint32_t)c; t[s + 1] = 0;
    }
    Big r; r.d.assign(t.begin(), t.begin() + s + 1); r.trim();
    if (cmp(r, N) >= 0) r = sub(r, N);
    return r;
  }
  Big to(const Big& a) const { return mm(mod(a, N), R2); }
  Big from(const Big& a) const { return mm(a, Big(1)); }
  Big pow(const Big& base, const Big& e) const {
    Big x = to(base), acc = R1;
    for (int i = e.bits() - 1; i >= 0; --i) {
      acc = mm(acc, acc);
      if (e.bit(i)) acc = mm(acc, x);
    }
    return from(acc);
  }
};

// a^-1 mod 2^(32 s) for odd a (Newton iteration)
inline Big inv_pow2(const Big& a, size_t s) {
  Big x(1), two(2);
  Big P = shl_bits(Big(1), 32 * (int)s);
  for (int bits = 1; bits < 32 * (int)s; bits *= 2) {
    Big ax = mod(mul(a, x), P);
    Big t = mod(sub(add(two, P), ax), P);  // 2 - a x mod 2^k, kept non-negative
    x = mod(mul(x, t), P);
  }
  return x;
}

// Deterministic 64-bit generator (SplitMix64) for key generation.
struct SplitMix64 {
  uint64_t s;
  explicit SplitMix64(uint64_t seed) : s(seed) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

// Miller-Rabin with `rounds` random witnesses after trial division.
inline bool probable_prime(const Big& x, int rounds, SplitMix64& rng) {
  static const uint32_t small[] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61, 67, 71,
                                   73, 79, 83, 89, 97, 101, 103, 107, 109, 113, 127, 131, 137, 139, 149, 151,
                                   157, 163, 167, 173, 179, 181, 191, 193, 197, 199, 211, 223, 227, 229, 233};
  if (!x.is_odd()) return cmp(x, Big(2)) == 0;
  for (uint32_t p : small) {
    uint64_t r = 0;
    for (size_t i = x.d.size(); i-- > 0;) r = ((r << 32) | x.d[i]) % p;
    if (r == 0) return cmp(x, Big(p)) == 0;
  }
  Big xm1 = sub(x, Big(1));
  int s = 0;
  while (!xm1.bit(s)) ++s;
  Big d = shr_bits(xm1, s);
  Mont M(x);
  Big one_m = M.R1, mone_m = M.to(xm1);
  Big range = sub(x, Big(3));
  for (int r = 0; r < rounds; ++r) {
    Big a;  // witness in [2, x - 2]
    a.d.resize(x.d.size());
    for (auto& w : a.d) w = (uint32_t)rng.next();
    a.trim();
    a = add(mod(a, range), Big(2));
    Big am = M.to(a), y = M.R1;
    for (int i = d.bits() - 1; i >= 0; --i) {
      y = M.mm(y, y);
      if (d.bit(i)) y = M.mm(y, am);
    }
    if (cmp(y, one_m) == 0 || cmp(y, mone_m) == 0) continue;
    bool ok = false;
    for (int j = 1; j < s; ++j) {
      y = M.mm(y, y);
      if (cmp(y, mone_m) == 0) { ok = true; break; }
    }
    if (!ok) return false;
  }
  return true;
}

inline Big gcd(Big a, Big b) {
  while (!b.is_zero()) { Big r = mod(a, b); a = b; b = r; }
  return a;
}

}  // namespace plh
