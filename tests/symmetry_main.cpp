// Test driver for the host-side symmetry checks (csrc/pp_symmetry_host.h):
// compiled with g++ on the CPU, it reads one request per line on standard
// input and prints one line per request.
//
//   multiset group n K   then K lines "x_0 .. x_{W-1} z_0 .. z_{W-1} value"
//                        (words as unsigned decimals): prints 1 if the
//                        multiset of (string, value) is invariant, else 0
//   bloch group n        then 3n numbers: prints 1 if the product state is
//                        invariant, else 0
//   valid code n         prints 1 if the group code is valid for n qubits
//   gens group n         prints the number of generators, then one line per
//                        generator: the site each site's letter moves to
#include <cstdint>
#include <iostream>
#include <string>
#include <vector>

#include "../paper_2512_12094_gb300/csrc/pp_symmetry_host.h"

int main() {
  std::string cmd;
  while (std::cin >> cmd) {
    if (cmd == "multiset") {
      int group = 0, n = 0, k = 0;
      std::cin >> group >> n >> k;
      const int W = (n + 63) / 64;
      std::vector<ppsym::HKey> keys(k, ppsym::HKey(2 * W));
      std::vector<double> vals(k);
      for (int i = 0; i < k; ++i) {
        for (auto& w : keys[i]) std::cin >> w;
        std::cin >> vals[i];
      }
      std::cout << (ppsym::multiset_invariant(group, n, W, keys, vals, 0.0) ? 1 : 0) << "\n";
    } else if (cmd == "bloch") {
      int group = 0, n = 0;
      std::cin >> group >> n;
      std::vector<double> b(3 * (size_t)n);
      for (double& v : b) std::cin >> v;
      std::cout << (ppsym::bloch_invariant(group, n, b.data()) ? 1 : 0) << "\n";
    } else if (cmd == "valid") {
      int code = 0, n = 0;
      std::cin >> code >> n;
      std::cout << (ppsym::valid_group(code, n) ? 1 : 0) << "\n";
    } else if (cmd == "gens") {
      int group = 0, n = 0;
      std::cin >> group >> n;
      const auto gens = ppsym::generators(group, n);
      std::cout << gens.size() << "\n";
      for (const auto& g : gens) {
        for (size_t q = 0; q < g.size(); ++q) std::cout << g[q] << (q + 1 < g.size() ? " " : "\n");
      }
    } else {
      std::cerr << "unknown request " << cmd << "\n";
      return 2;
    }
  }
  return 0;
}
