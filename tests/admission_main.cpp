// Test driver for the job server's host-side rules (csrc/pp_admission.h):
// compiled with g++ on the CPU, it reads one request per line on standard
// input and prints one line of results per request.
//
//   fit N            then N lines "f0 .. f7 y": add the samples to a new cost
//                    model; prints its 8 coefficients
//   pick Q           then Q lines "key fits bypassed": prints the admitted
//                    index and every job's bypass count afterwards
//   share slots running wanted free
//                    prints the units a layer takes (0 = wait)
//   key predicted waited_s gave_back
//                    prints the admission key
//   features n_qubits symmetry noise_mode eps n_layers n_gates
//                    prints the 8 features
#include <cstdio>
#include <cstring>
#include <iostream>
#include <string>
#include <vector>

#include "../paper_2512_12094_gb300/csrc/pp_admission.h"

int main() {
  std::string cmd;
  std::cout.precision(17);
  while (std::cin >> cmd) {
    if (cmd == "fit") {
      int n = 0;
      std::cin >> n;
      ppadm::CostModel m;
      for (int i = 0; i < n; ++i) {
        double f[ppadm::kFeat], y;
        for (double& v : f) std::cin >> v;
        std::cin >> y;
        m.add(f, y);
      }
      for (int i = 0; i < ppadm::kFeat; ++i) std::cout << m.beta[i] << (i + 1 < ppadm::kFeat ? " " : "\n");
    } else if (cmd == "pick") {
      int q = 0;
      std::cin >> q;
      std::vector<double> key(q);
      std::vector<char> fits(q);
      std::vector<int> bypassed(q);
      for (int k = 0; k < q; ++k) {
        int f = 0;
        std::cin >> key[k] >> f >> bypassed[k];
        fits[k] = (char)(f != 0);
      }
      std::cout << ppadm::pick_admission(key, fits, bypassed);
      for (int b : bypassed) std::cout << " " << b;
      std::cout << "\n";
    } else if (cmd == "share") {
      int slots = 0, freeu = 0;
      long long running = 0;
      double wanted = 0.0;
      std::cin >> slots >> running >> wanted >> freeu;
      std::cout << ppadm::share_units(slots, running, wanted, freeu) << "\n";
    } else if (cmd == "key") {
      double predicted = 0.0, waited = 0.0;
      int gave_back = 0;
      std::cin >> predicted >> waited >> gave_back;
      std::cout << ppadm::admission_key(predicted, waited, gave_back != 0) << "\n";
    } else if (cmd == "features") {
      pp_config cfg;
      std::memset(&cfg, 0, sizeof(cfg));
      int n_layers = 0, n_gates = 0;
      std::cin >> cfg.n_qubits >> cfg.symmetry >> cfg.noise_mode >> cfg.coeff_eps >> n_layers >>
          n_gates;
      double f[ppadm::kFeat];
      ppadm::job_features(cfg, n_layers, n_gates, f);
      for (int i = 0; i < ppadm::kFeat; ++i) std::cout << f[i] << (i + 1 < ppadm::kFeat ? " " : "\n");
    } else {
      std::cerr << "unknown request " << cmd << "\n";
      return 2;
    }
  }
  return 0;
}
