// The random draws of the method, made by the library from a seed.
//
// Eq. 1 needs L*K hash vectors with N(0,1) entries and Alg. 1 a uniform
// sample of the points; the paper fixes no generator. Both come from one
// counter-based generator, splitmix64 (Steele, Lea and Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014): the state
// advances by the odd constant 0x9E3779B97F4A7C15 and each output is the
// state passed through a fixed 64-bit mixing function.
//
// * Hash vectors: the entries of A [L*K][d] (row r = i*K + j) in row-major
//   order, two at a time, by the Box-Muller transform (Box and Muller, 1958)
//   in FP64 from two consecutive outputs: u1 = (top 53 bits + 1) / 2^53 in
//   (0, 1], u2 = (top 53 bits) / 2^53 in [0, 1), rho = sqrt(-2 ln u1),
//   theta = 2*pi*u2; the pair is (rho cos theta, rho sin theta), each rounded
//   once to FP32. The stream starts at state = seed.
// * Sample: a partial Fisher-Yates shuffle (Durstenfeld's in-place form) of
//   the positions 0..n-1: for i = 0..n_s-1 the swap partner is
//   j = i + floor(z * (n - i) / 2^64) with z the next output (the high word
//   of a 128-bit product); the sample is the first n_s positions, sorted
//   ascending. The stream starts at state = seed XOR 0x5A.
//
// Only products, quotients by powers of two and single library calls occur
// (no multiply-add to contract), so the values are reproducible wherever the
// C library's log, sin and cos agree.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "../../include/detlsh.h"

namespace detlsh {

namespace {

struct SplitMix64 {
  uint64_t x;
  explicit SplitMix64(uint64_t seed) : x(seed) {}
  uint64_t next() {
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

constexpr double kTwoPi = 2.0 * 3.14159265358979323846;
constexpr double kInv53 = 1.0 / 9007199254740992.0;  // 2^-53

}  // namespace

void draw_hashes(uint64_t seed, int64_t count, float* A) {
  SplitMix64 g(seed);
  for (int64_t e = 0; e < count; e += 2) {
    const double u1 = (double)((g.next() >> 11) + 1) * kInv53;
    const double u2 = (double)(g.next() >> 11) * kInv53;
    const double rho = std::sqrt(-2.0 * std::log(u1));
    const double theta = kTwoPi * u2;
    const double z0 = rho * std::cos(theta);
    const double z1 = rho * std::sin(theta);
    A[e] = (float)z0;
    if (e + 1 < count) A[e + 1] = (float)z1;
  }
}

void draw_sample(uint64_t seed, int64_t n, int64_t n_s, int64_t* ids) {
  SplitMix64 g(seed ^ 0x5Aull);
  auto partner = [&](int64_t i) {
    const unsigned __int128 p = (unsigned __int128)g.next() * (unsigned __int128)(uint64_t)(n - i);
    return i + (int64_t)(uint64_t)(p >> 64);
  };
  if (n_s * 16 >= n) {
    // dense positions
    std::vector<uint32_t> pos((size_t)n);
    for (int64_t i = 0; i < n; ++i) pos[(size_t)i] = (uint32_t)i;
    for (int64_t i = 0; i < n_s; ++i) std::swap(pos[(size_t)i], pos[(size_t)partner(i)]);
    for (int64_t i = 0; i < n_s; ++i) ids[i] = pos[(size_t)i];
  } else {
    // only the positions a swap has touched differ from the identity
    std::unordered_map<int64_t, int64_t> moved;
    moved.reserve((size_t)(2 * n_s));
    auto at = [&](int64_t i) {
      const auto it = moved.find(i);
      return it == moved.end() ? i : it->second;
    };
    for (int64_t i = 0; i < n_s; ++i) {
      const int64_t j = partner(i);
      const int64_t vi = at(i), vj = at(j);
      moved[i] = vj;
      moved[j] = vi;
      ids[i] = vj;
    }
  }
  std::sort(ids, ids + n_s);
}

}  // namespace detlsh

extern "C" {

int detlsh_draw_hashes(uint64_t seed, int32_t LK, int32_t d, float* A) {
  if (!A || LK < 1 || LK > 256 || d < 1 || d > 65536) return DETLSH_EINVAL;
  detlsh::draw_hashes(seed, (int64_t)LK * d, A);
  return DETLSH_OK;
}

int detlsh_draw_sample(uint64_t seed, int64_t n, int64_t n_s, int64_t* ids) {
  if (!ids || n < 1 || n >= ((int64_t)1 << 32) || n_s < 1 || n_s > n) return DETLSH_EINVAL;
  detlsh::draw_sample(seed, n, n_s, ids);
  return DETLSH_OK;
}

}  // extern "C"
