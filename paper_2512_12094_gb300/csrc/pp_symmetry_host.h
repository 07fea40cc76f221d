// Symmetry groups on host-side Pauli strings (x words, then z words): the
// group codes, each group's generators as maps of sites, and the invariance
// tests pp_create and pp_apply_layer use to reject a layer, an observable or
// a state the declared group does not map onto itself (PP_ERR_SYMMETRY).
// Plain C++ with no CUDA, so the same code is compiled into the library and
// into a CPU test driver.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <vector>

#include "../../include/pp.h"

namespace ppsym {

inline void get_bit(const uint64_t* m, int q, int& b) { b = (int)((m[q >> 6] >> (q & 63)) & 1ull); }

inline void permute_string(const uint64_t* x, const uint64_t* z, int n, int W,
                           const std::vector<int>& to, uint64_t* ox, uint64_t* oz) {
  for (int j = 0; j < W; ++j) ox[j] = oz[j] = 0;
  for (int q = 0; q < n; ++q) {
    int xb, zb;
    get_bit(x, q, xb);
    get_bit(z, q, zb);
    int t = to[q];
    ox[t >> 6] |= (uint64_t)xb << (t & 63);
    oz[t >> 6] |= (uint64_t)zb << (t & 63);
  }
}

// Group codes: kind in the low byte (pp_symmetry), torus width above it.
inline int group_kind(int code) { return code & 0xFF; }
inline int group_lx(int code) { return code >> 8; }

inline bool valid_group(int code, int n) {
  const int kind = group_kind(code), lx = group_lx(code);
  if (code < 0 || kind > PP_SYM_TORUS) return false;
  if (kind == PP_SYM_TORUS) return lx >= 1 && lx <= n && n % lx == 0;
  return lx == 0;
}

// Generators of the group as site maps (the letter of q moves to to[q]).
inline std::vector<std::vector<int>> generators(int group, int n) {
  std::vector<std::vector<int>> gens;
  const int kind = group_kind(group);
  if (n < 2 || kind == PP_SYM_NONE) return gens;
  if (kind == PP_SYM_TORUS) {
    const int lx = group_lx(group), ly = n / lx;
    std::vector<int> sx(n), sy(n);
    for (int q = 0; q < n; ++q) {
      const int x = q % lx, y = q / lx;
      sx[q] = (x + 1) % lx + lx * y;
      sy[q] = x + lx * ((y + 1) % ly);
    }
    gens.push_back(sx);
    gens.push_back(sy);
    return gens;
  }
  std::vector<int> shift(n);
  for (int q = 0; q < n; ++q) shift[q] = (q + n - 1) % n;  // T: qubit q -> q-1
  gens.push_back(shift);
  if (kind == PP_SYM_SN) {
    std::vector<int> swap01(n);
    for (int q = 0; q < n; ++q) swap01[q] = q;
    std::swap(swap01[0], swap01[1]);
    gens.push_back(swap01);
  }
  if (kind == PP_SYM_DN) {
    std::vector<int> refl(n);
    for (int q = 0; q < n; ++q) refl[q] = n - 1 - q;
    gens.push_back(refl);
  }
  return gens;
}

typedef std::vector<uint64_t> HKey;

// Is the multiset {(string_i, value_i)} mapped onto itself by every generator?
inline bool multiset_invariant(int group, int n, int W, const std::vector<HKey>& keys,
                               const std::vector<double>& vals, double rel_tol) {
  std::map<HKey, std::vector<double>> base;
  for (size_t i = 0; i < keys.size(); ++i) base[keys[i]].push_back(vals[i]);
  for (auto& kv : base) std::sort(kv.second.begin(), kv.second.end());
  for (const auto& g : generators(group, n)) {
    std::map<HKey, std::vector<double>> img;
    for (size_t i = 0; i < keys.size(); ++i) {
      HKey k(2 * W);
      permute_string(keys[i].data(), keys[i].data() + W, n, W, g, k.data(), k.data() + W);
      img[k].push_back(vals[i]);
    }
    if (img.size() != base.size()) return false;
    for (auto& kv : img) {
      auto it = base.find(kv.first);
      if (it == base.end() || it->second.size() != kv.second.size()) return false;
      std::sort(kv.second.begin(), kv.second.end());
      for (size_t t = 0; t < kv.second.size(); ++t) {
        double a = kv.second[t], b = it->second[t];
        if (std::fabs(a - b) > rel_tol * std::max(1.0, std::max(std::fabs(a), std::fabs(b))))
          return false;
      }
    }
  }
  return true;
}

inline bool bloch_invariant(int group, int n, const double* bloch) {
  for (const auto& g : generators(group, n))
    for (int q = 0; q < n; ++q)
      for (int a = 0; a < 3; ++a)
        if (bloch[3 * q + a] != bloch[3 * g[q] + a]) return false;
  return true;
}

}  // namespace ppsym
