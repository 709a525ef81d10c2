// 256-bit unsigned integers for exact contraction costs.
//
// Tensor sizes of cut circuits grow as 6^(gate cuts) * 4^(wire cuts) * batch
// (section 2.1: O(6^k) and O(4^k) per cut kind), so sizes of poor pairwise
// orders overflow 64 and even 128 bits.  The planner compares costs exactly;
// anything at or above 2^255 is reported as unsupported.
#pragma once
#include <cstdint>
#include <string>

namespace qtpu {

struct U256 {
  uint64_t w[4] = {0, 0, 0, 0};  // little-endian limbs

  U256() = default;
  explicit U256(uint64_t v) { w[0] = v; }

  bool top_bit() const { return (w[3] >> 63) != 0; }
  bool is_zero() const { return !(w[0] | w[1] | w[2] | w[3]); }

  friend bool operator<(const U256& a, const U256& b) {
    for (int i = 3; i >= 0; --i)
      if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
    return false;
  }
  friend bool operator==(const U256& a, const U256& b) {
    return a.w[0] == b.w[0] && a.w[1] == b.w[1] && a.w[2] == b.w[2] && a.w[3] == b.w[3];
  }
  friend bool operator!=(const U256& a, const U256& b) { return !(a == b); }

  // a + b; sets *ovf if the result reaches 2^255
  static U256 add(const U256& a, const U256& b, bool* ovf) {
    U256 r;
    unsigned __int128 c = 0;
    for (int i = 0; i < 4; ++i) {
      c += (unsigned __int128)a.w[i] + b.w[i];
      r.w[i] = (uint64_t)c;
      c >>= 64;
    }
    if (c || r.top_bit()) *ovf = true;
    return r;
  }

  // a * b; sets *ovf if the exact product reaches 2^255
  static U256 mul(const U256& a, const U256& b, bool* ovf) {
    uint64_t t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 4; ++i) {
      unsigned __int128 c = 0;
      for (int j = 0; j < 4; ++j) {
        c += (unsigned __int128)a.w[i] * b.w[j] + t[i + j];
        t[i + j] = (uint64_t)c;
        c >>= 64;
      }
      t[i + 4] = (uint64_t)c;
    }
    U256 r;
    for (int i = 0; i < 4; ++i) r.w[i] = t[i];
    if (t[4] | t[5] | t[6] | t[7] || r.top_bit()) *ovf = true;
    return r;
  }

  static U256 mul_u64(const U256& a, uint64_t b, bool* ovf) { return mul(a, U256(b), ovf); }

  double to_double() const {
    double r = 0.0;
    for (int i = 3; i >= 0; --i) r = r * 18446744073709551616.0 + (double)w[i];
    return r;
  }

  bool fits_u64() const { return !(w[1] | w[2] | w[3]); }

  std::string str() const {
    if (is_zero()) return "0";
    U256 v = *this;
    std::string s;
    while (!v.is_zero()) {
      // divide by 10, collect remainder
      unsigned __int128 rem = 0;
      for (int i = 3; i >= 0; --i) {
        unsigned __int128 cur = (rem << 64) | v.w[i];
        v.w[i] = (uint64_t)(cur / 10);
        rem = cur % 10;
      }
      s.push_back(char('0' + (int)rem));
    }
    return std::string(s.rbegin(), s.rend());
  }
};

}  // namespace qtpu
