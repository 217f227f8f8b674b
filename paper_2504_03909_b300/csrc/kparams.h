// Kernel parameter blocks shared by the host launchers and the kernels.  They
// are passed by value (__grid_constant__), so every constant a kernel needs
// sits in the constant bank and warp-uniform reads of it are broadcasts.
#pragma once

#include <cstdint>

namespace pl {

constexpr int kMaxL = 96;                 // limbs of n for the largest key (3072-bit)
constexpr int kMaxLh = kMaxL / 2;         // limbs of p, q
// Sliding-window schedules (see ModexpParams): at most one squaring per
// exponent bit and one product per set bit, for exponents of at most 1536 bits
// (the primes of a 3072-bit key).
constexpr int kMaxOps = 2 * 1536 + 2;

// Device status word bits (OR-ed by kernels, read by paillier_sync)
constexpr int kStatusBadBin = 1;       // bin >= K
constexpr int kStatusBadNode = 2;      // node >= num_nodes
constexpr int kStatusRange = 4;        // plaintext does not fit the output type
constexpr int kStatusEncode = 8;       // value outside the encodable range
constexpr int kStatusTimeout = 16;     // a bounded wait ran out
constexpr int kStatusCapacity = 32;    // a work list was larger than its buffer
constexpr int kStatusNonUnit = 64;     // encryption randomness r with gcd(r, n) != 1
constexpr int kStatusBadSplit = 128;   // a split feature >= F

// One half of the key holder's CRT split: arithmetic mod N = x^2 for the
// prime x = p (or q), L limbs, R = 2^(32 L); and mod x itself, L/2 limbs,
// Rx = 2^(16 L).
struct HalfConst {
  uint32_t N[kMaxL];    // x^2
  uint32_t R1[kMaxL];   // R mod N (Montgomery one)
  uint32_t R2[kMaxL];   // R^2 mod N
  uint32_t R3[kMaxL];   // R^3 mod N (reduces a 2L-limb value into Montgomery form)
  uint32_t nR[kMaxL];   // n R mod N (so that mont(m, nR) = m n mod N)
  uint32_t Nx[kMaxLh];  // x
  uint32_t R1x[kMaxLh]; // Rx mod x
  uint32_t R2x[kMaxLh]; // Rx^2 mod x
  uint32_t R3x[kMaxLh]; // Rx^3 mod x (reduces an L-limb value into Montgomery form mod x)
  uint32_t np;          // -N^-1 mod 2^32
  uint32_t npx;         // -x^-1 mod 2^32
  uint32_t pad[2];
};

// Batched left-to-right sliding-window exponentiation over both halves.
//   decryption: c^(x-1) mod x^2, schedule in op;
//   encryption: r^n mod x^2 = ((r mod x)^(x' mod (x-1)) mod x)^x mod x^2, where x'
//   is the other prime (y^x mod x^2 depends only on y mod x):
//   schedule of x' mod (x-1) in op1 (mod x), of x in op (mod x^2).
// A schedule for exponent e and window w: op[0] is the odd value v of the
// leading window (start from base^v); then, most significant bits first, 0 =
// square, odd v = multiply by base^v (v < 2^w).  The table holds the odd powers
// base^1, base^3, .., base^(2^w - 1).  The exponents are the key's, so every
// instance of a launch runs the same schedule.
struct ModexpParams {
  HalfConst half[2];
  uint8_t op[2][kMaxOps];
  int nop[2];
  uint8_t op1[2][kMaxOps];   // encryption, first exponentiation (mod x)
  int nop1[2];
  int w;                     // window width in bits
  int pad;
};

// Montgomery arithmetic mod n^2 (2L limbs, R = 2^(64 L)).
struct N2Const {
  uint32_t N[2 * kMaxL];
  uint32_t R2[2 * kMaxL];   // R^2 mod n^2
  uint32_t np;
  uint32_t pad[3];
};

// Single-thread finishing step of encrypt (CRT recombination mod n^2).
struct EncCrtParams {
  uint32_t p2[kMaxL], q2[kMaxL];
  uint32_t QinvR[kMaxL];    // (q^2)^-1 R mod p^2
  uint32_t p2_np;
  int L;
};

// Single-thread finishing step of CRT decryption.
struct DecCrtParams {
  uint32_t p[kMaxLh], q[kMaxLh];
  uint32_t pinv[kMaxLh], qinv2k[kMaxLh];  // p^-1, q^-1 mod 2^(32 Lh) (exact division)
  uint32_t hpR[kMaxLh], hqR[kMaxLh];      // h_p Rh mod p, h_q Rh mod q
  uint32_t qinvR[kMaxLh];                 // q^-1 Rh mod p
  uint32_t p_np, q_np;
  int Lh;
  int pad;
};

// Size of one histogram pass, read by the kernels from device memory so that a
// captured launch set can be replayed for levels with different node counts.
struct HistDesc {
  int num_nodes;  // nodes of the level (valid node ids are 0 .. num_nodes-1)
  int NK;         // keys per feature: num_nodes * K, or K when only_node >= 0
  int only_node;  // -1: all nodes; otherwise only this node (per-node comparator)
  int pad;
};

}  // namespace pl
