// Test driver: runs the oracle's C interface through propagation, merging,
// truncation, noise, overlaps and batched rows, for one- and two-word
// strings, so that a build with AddressSanitizer and UndefinedBehaviorSanitizer
// can check every path for invalid memory accesses and undefined behaviour.
// Prints the expectation values it computes, one per line, for comparison
// with the same calls through the Python binding.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

extern "C" {
void* orc_create(int n, long long n_terms, const uint64_t* x, const uint64_t* z,
                 const double* coef, int group, double eps, int wmax);
void orc_destroy(void* h);
long long orc_size(void* h);
void orc_export(void* h, uint64_t* x, uint64_t* z, double* coef);
int orc_apply_layer(void* h, int n_gates, const uint64_t* gx, const uint64_t* gz,
                    const double* theta, int noise_mode, double p, double eps, int wmax,
                    int group);
int orc_truncate(void* h, double eps, int wmax);
double orc_expect(void* h, const double* bloch, int group);
void orc_canonical(int n, long long m, int group, const uint64_t* x, const uint64_t* z,
                   uint64_t* ox, uint64_t* oz);
void* orcb_create(int n, long long n_terms, int B, const uint64_t* x, const uint64_t* z,
                  const double* coef, int group, double eps, int wmax);
void orcb_destroy(void* h);
long long orcb_size(void* h);
int orcb_apply_layer(void* h, int n_gates, const uint64_t* gx, const uint64_t* gz,
                     const double* theta, int noise_mode, double p, double eps, int wmax,
                     int group);
void orcb_expect(void* h, const double* bloch, int group, double* out);
void orcb_export(void* h, uint64_t* x, uint64_t* z, double* coef);
}

namespace {

void set_bit(std::vector<uint64_t>& m, int W, int row, int q) {
  m[(size_t)row * W + (q >> 6)] |= 1ull << (q & 63);
}

// The ring layer in time order: ZZ on every bond, then X, then Z on every
// qubit; masks [3n][W].
void ring_layer(int n, std::vector<uint64_t>& gx, std::vector<uint64_t>& gz) {
  const int W = (n + 63) / 64;
  gx.assign((size_t)3 * n * W, 0);
  gz.assign((size_t)3 * n * W, 0);
  for (int q = 0; q < n; ++q) {
    set_bit(gz, W, q, q);
    set_bit(gz, W, q, (q + 1) % n);
    set_bit(gx, W, n + q, q);
    set_bit(gz, W, 2 * n + q, q);
  }
}

// (1/n) sum Z_q
void mean_z(int n, std::vector<uint64_t>& x, std::vector<uint64_t>& z, std::vector<double>& c) {
  const int W = (n + 63) / 64;
  x.assign((size_t)n * W, 0);
  z.assign((size_t)n * W, 0);
  c.assign(n, 1.0 / n);
  for (int q = 0; q < n; ++q) set_bit(z, W, q, q);
}

double run_single(int n, int group, int noise_mode, double p, double eps, int wmax, int layers) {
  std::vector<uint64_t> x, z, gx, gz;
  std::vector<double> c;
  mean_z(n, x, z, c);
  ring_layer(n, gx, gz);
  std::vector<double> theta(3 * n);
  for (int q = 0; q < n; ++q) {
    theta[q] = 0.4;
    theta[n + q] = 0.6;
    theta[2 * n + q] = 0.3;
  }
  void* h = orc_create(n, n, x.data(), z.data(), c.data(), group, eps, wmax);
  for (int l = 0; l < layers; ++l)
    orc_apply_layer(h, 3 * n, gx.data(), gz.data(), theta.data(), noise_mode, p, eps, wmax, group);
  orc_truncate(h, eps, wmax);
  const int W = (n + 63) / 64;
  const long long m = orc_size(h);
  std::vector<uint64_t> ex((size_t)m * W + 1), ez((size_t)m * W + 1);
  std::vector<double> ec((size_t)m + 1);
  orc_export(h, ex.data(), ez.data(), ec.data());
  std::vector<uint64_t> cx((size_t)m * W + 1), cz((size_t)m * W + 1);
  if (m > 0) orc_canonical(n, m, group == 0 ? 1 : group, ex.data(), ez.data(), cx.data(), cz.data());
  std::vector<double> bloch((size_t)3 * n, 0.0);
  for (int q = 0; q < n; ++q) bloch[3 * q + 2] = (q % 2) ? -1.0 : 1.0;  // Neel
  const double v = orc_expect(h, bloch.data(), group);
  orc_destroy(h);
  return v;
}

void run_batched(int n, int B, int group, double eps, int layers, std::vector<double>& out) {
  std::vector<uint64_t> x, z, gx, gz;
  std::vector<double> c1;
  mean_z(n, x, z, c1);
  std::vector<double> c((size_t)n * B);
  for (int i = 0; i < n; ++i)
    for (int b = 0; b < B; ++b) c[(size_t)i * B + b] = c1[i];
  ring_layer(n, gx, gz);
  std::vector<double> theta((size_t)3 * n * B);
  for (int g = 0; g < 3 * n; ++g)
    for (int b = 0; b < B; ++b) theta[(size_t)g * B + b] = 0.1 + 0.2 * b + 0.01 * (g % 7);
  void* h = orcb_create(n, n, B, x.data(), z.data(), c.data(), group, eps, -1);
  for (int l = 0; l < layers; ++l)
    orcb_apply_layer(h, 3 * n, gx.data(), gz.data(), theta.data(), 0, 0.0, eps, -1, group);
  const int W = (n + 63) / 64;
  const long long m = orcb_size(h);
  std::vector<uint64_t> ex((size_t)m * W + 1), ez((size_t)m * W + 1);
  std::vector<double> ec((size_t)m * B + 1);
  orcb_export(h, ex.data(), ez.data(), ec.data());
  std::vector<double> bloch((size_t)3 * n, 0.0);
  for (int q = 0; q < n; ++q) bloch[3 * q + 2] = 1.0;
  out.assign(B, 0.0);
  orcb_expect(h, bloch.data(), group, out.data());
  orcb_destroy(h);
}

}  // namespace

int main() {
  std::printf("%.17g\n", run_single(10, 0, 0, 0.0, 1e-4, 6, 3));
  std::printf("%.17g\n", run_single(10, 1, 0, 0.0, 1e-4, 6, 3));
  std::printf("%.17g\n", run_single(8, 2, 1, 0.02, 1e-5, -1, 2));
  std::printf("%.17g\n", run_single(8, 3, 2, 0.05, 1e-5, -1, 2));
  std::printf("%.17g\n", run_single(8, 4 | (4 << 8), 0, 0.0, 1e-4, -1, 2));
  std::printf("%.17g\n", run_single(70, 1, 0, 0.0, 1e-3, 4, 2));
  std::vector<double> out;
  run_batched(9, 3, 1, 1e-4, 2, out);
  for (double v : out) std::printf("%.17g\n", v);
  return 0;
}
