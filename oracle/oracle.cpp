// Plain CPU oracle for symmetry-merging Pauli propagation.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
// restatement of the method that the tests, the smoke check and the CPU
// baseline leg of the benchmark compare the CUDA library against.  Nothing in
// the product path links, loads or calls it, and it shares no code, header,
// table or helper with the CUDA library.
//
// Representation: a Pauli string over n qubits is a std::string of n bytes,
// one letter per qubit with values 0 = I, 1 = X, 2 = Y, 3 = Z.  These are the
// base-4 digit values of the "lowest integer representation" (Appendix E,
// Definition "Lowest integer representation": I -> 00, X -> 01, Y -> 10,
// Z -> 11).  Operators are stored unnormalised, O = sum_s c_s s, with real
// coefficients (Appendix A: the Pauli transfer matrix of a unitary is real).
// The only bit masks in this file are the I/O format (x, z words), converted
// to letters on entry and back on exit.
//
// Parity status: every function here is pinned by a "not gpu" test against a
// dense state-vector / density-matrix simulation, a closed form, a count from
// Burnside's lemma, or brute force over group elements.  No function is
// "parity unpinned".

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

namespace {

// Single-qubit Pauli products a*b = i^phase * letter, written out from the
// Pauli algebra XY = iZ, YZ = iX, ZX = iY (reversed order gives -i).
struct Prod {
  uint8_t letter;
  uint8_t phase;  // exponent of i, mod 4
};
const Prod kMul[4][4] = {
    /* I * {I,X,Y,Z} */ {{0, 0}, {1, 0}, {2, 0}, {3, 0}},
    /* X * {I,X,Y,Z} */ {{1, 0}, {0, 0}, {3, 1}, {2, 3}},
    /* Y * {I,X,Y,Z} */ {{2, 0}, {3, 3}, {0, 0}, {1, 1}},
    /* Z * {I,X,Y,Z} */ {{3, 0}, {2, 1}, {1, 3}, {0, 0}},
};

bool site_anticommutes(uint8_t a, uint8_t b) { return a != 0 && b != 0 && a != b; }

int weight(const std::string& s) {
  int w = 0;
  for (char ch : s) w += (ch != 0);
  return w;
}

std::string letters_from_masks(int n, int W, const uint64_t* x, const uint64_t* z) {
  std::string s(n, '\0');
  for (int q = 0; q < n; ++q) {
    int xb = (x[q / 64] >> (q % 64)) & 1;
    int zb = (z[q / 64] >> (q % 64)) & 1;
    uint8_t l = 0;
    if (xb && !zb) l = 1;
    if (xb && zb) l = 2;
    if (!xb && zb) l = 3;
    s[q] = (char)l;
  }
  (void)W;
  return s;
}

void masks_from_letters(const std::string& s, int W, uint64_t* x, uint64_t* z) {
  for (int w = 0; w < W; ++w) x[w] = z[w] = 0;
  for (size_t q = 0; q < s.size(); ++q) {
    uint8_t l = (uint8_t)s[q];
    if (l == 1 || l == 2) x[q / 64] |= (uint64_t)1 << (q % 64);
    if (l == 2 || l == 3) z[q / 64] |= (uint64_t)1 << (q % 64);
  }
}

// int(s) comparison of Definition "Lowest integer representation": qubit q is
// the base-4 digit of weight 4^q, so the most significant digit is qubit n-1.
bool int_less(const std::string& a, const std::string& b) {
  for (int q = (int)a.size() - 1; q >= 0; --q) {
    if (a[q] != b[q]) return (uint8_t)a[q] < (uint8_t)b[q];
  }
  return false;
}

// T^j shifts every letter j sites to the left (Example B.1: T(IZI..) = ZII..).
std::string translate(const std::string& s, int j) {
  int n = (int)s.size();
  std::string r(n, '\0');
  for (int q = 0; q < n; ++q) r[q] = s[(q + j) % n];
  return r;
}

// Algorithm 2: lowest integer representative under Z_n by enumerating all n
// translations.
std::string canonical_zn(const std::string& s) {
  std::string best = s;
  for (int j = 1; j < (int)s.size(); ++j) {
    std::string t = translate(s, j);
    if (int_less(t, best)) best = t;
  }
  return best;
}

// Algorithm 3: count (n_X, n_Y, n_Z) and write Z^{n_Z} Y^{n_Y} X^{n_X} I...
std::string canonical_sn(const std::string& s) {
  int nx = 0, ny = 0, nz = 0;
  for (char ch : s) {
    if (ch == 1) ++nx;
    if (ch == 2) ++ny;
    if (ch == 3) ++nz;
  }
  std::string r(s.size(), '\0');
  int q = 0;
  for (int k = 0; k < nz; ++k) r[q++] = 3;
  for (int k = 0; k < ny; ++k) r[q++] = 2;
  for (int k = 0; k < nx; ++k) r[q++] = 1;
  return r;
}

// Group codes: 1 = Z_n, 2 = S_n, 3 = D_n (the n rotations and n reflections of
// a ring, Sec. "Symmetry" / Appendix B: dihedral symmetry), 4 | (Lx << 8) =
// translations of an Lx x Ly torus with qubit q = x + Lx y (the 2D
// translations used for the XXZ figure).
int group_kind(int group) { return group & 0xFF; }
int group_lx(int group) { return group >> 8; }

// Every element of D_n or of the torus translations as a map of sites: the
// letter of site q moves to site m[q].
std::vector<std::vector<int>> group_elements(int group, int n) {
  std::vector<std::vector<int>> out;
  if (group_kind(group) == 3) {
    for (int j = 0; j < n; ++j) {
      std::vector<int> rot(n), ref(n);
      for (int q = 0; q < n; ++q) {
        rot[q] = (q + j) % n;
        ref[q] = (n - 1 - q + j) % n;
      }
      out.push_back(rot);
      out.push_back(ref);
    }
  } else if (group_kind(group) == 4) {
    const int lx = group_lx(group), ly = n / lx;
    for (int dy = 0; dy < ly; ++dy)
      for (int dx = 0; dx < lx; ++dx) {
        std::vector<int> m(n);
        for (int q = 0; q < n; ++q) {
          const int x = q % lx, y = q / lx;
          m[q] = (x + dx) % lx + lx * ((y + dy) % ly);
        }
        out.push_back(m);
      }
  }
  return out;
}

const std::vector<std::vector<int>>& cached_elements(int group, int n) {
  static std::map<std::pair<int, int>, std::vector<std::vector<int>>> cache;
  auto key = std::make_pair(group, n);
  auto it = cache.find(key);
  if (it == cache.end()) it = cache.emplace(key, group_elements(group, n)).first;
  return it->second;
}

std::string apply_map(const std::string& s, const std::vector<int>& m) {
  std::string r(s.size(), '\0');
  for (size_t q = 0; q < s.size(); ++q) r[m[q]] = s[q];
  return r;
}

// Lowest integer representative by enumerating every group element.
std::string canonical_by_elements(const std::string& s, int group) {
  std::string best = s;
  for (const auto& m : cached_elements(group, (int)s.size())) {
    std::string t = apply_map(s, m);
    if (int_less(t, best)) best = t;
  }
  return best;
}

std::string canonical(const std::string& s, int group) {
  if (group == 1) return canonical_zn(s);
  if (group == 2) return canonical_sn(s);
  if (group_kind(group) == 3 || group_kind(group) == 4) return canonical_by_elements(s, group);
  return s;
}

double bloch_value(const double* bloch, int q, uint8_t letter) {
  if (letter == 0) return 1.0;
  return bloch[3 * q + (letter - 1)];
}

// Tr[rho s] for rho = prod_q (I + bx X + by Y + bz Z)/2 and an unnormalised
// Pauli string s: the product of the per-site Bloch components.
double product_overlap(const std::string& s, const double* bloch) {
  double v = 1.0;
  for (int q = 0; q < (int)s.size(); ++q) v *= bloch_value(bloch, q, (uint8_t)s[q]);
  return v;
}

struct State {
  int n = 0;
  int W = 1;
  std::unordered_map<std::string, double> terms;
  double updates = 0.0;  // sum over gates of the live terms entering the gate
  // cache of S_n orbit-averaged overlaps, keyed by (n_X, n_Y, n_Z)
  std::vector<double> sn_table;
  std::vector<double> sn_bloch;
};

bool keep(double c, const std::string& s, double eps, int wmax) {
  if (eps > 0.0 && !(std::fabs(c) >= eps)) return false;
  if (wmax >= 0 && weight(s) > wmax) return false;
  return true;
}

void truncate_all(State* st, double eps, int wmax) {
  for (auto it = st->terms.begin(); it != st->terms.end();) {
    if (!keep(it->second, it->first, eps, wmax))
      it = st->terms.erase(it);
    else
      ++it;
  }
}

void symmetry_merge(State* st, int group) {
  std::unordered_map<std::string, double> merged;
  for (const auto& kv : st->terms) merged[canonical(kv.first, group)] += kv.second;
  st->terms.swap(merged);
}

// One Pauli rotation exp(-i theta P / 2) in the Heisenberg picture (App. A,
// Prop. 1 proof): Q -> Q if [P, Q] = 0, otherwise
// Q -> cos(theta) Q + sin(theta) (i P Q), with i P Q = +-R a Hermitian string.
// Per-gate depolarising damping multiplies each term by (1-p)^k, k = number
// of non-identity letters of Q on the gate's support; in the Heisenberg
// picture the noise that follows the gate in time acts before the conjugation.
void apply_gate(State* st, const std::string& P, double theta, int noise_mode, double p,
                double eps, int wmax) {
  const double c = std::cos(theta);
  const double s = std::sin(theta);
  std::vector<int> support;
  for (int q = 0; q < st->n; ++q)
    if (P[q] != 0) support.push_back(q);
  std::vector<double> damp(support.size() + 1, 1.0);
  for (size_t k = 1; k < damp.size(); ++k) damp[k] = damp[k - 1] * (1.0 - p);

  st->updates += (double)st->terms.size();
  std::unordered_map<std::string, double> next;
  next.reserve(st->terms.size() * 2);
  for (const auto& kv : st->terms) {
    const std::string& Q = kv.first;
    double d = kv.second;
    if (noise_mode == 1) {
      int k = 0;
      for (int q : support) k += (Q[q] != 0);
      if (k > 0) d = d * damp[k];
    }
    int anti = 0;
    for (int q : support) anti += site_anticommutes((uint8_t)P[q], (uint8_t)Q[q]);
    if (anti % 2 == 0) {
      next[Q] += d;
      continue;
    }
    std::string R = Q;
    int phase = 0;
    for (int q : support) {
      const Prod& pr = kMul[(uint8_t)P[q]][(uint8_t)Q[q]];
      R[q] = (char)pr.letter;
      phase += pr.phase;
    }
    // P Q = i^phase R, so i P Q = i^(phase+1) R; phase+1 is even here.
    int e = (phase + 1) % 4;
    double sign = (e == 0) ? 1.0 : -1.0;
    next[Q] += c * d;
    next[R] += sign * (s * d);
  }
  st->terms.swap(next);
  truncate_all(st, eps, wmax);
}

// Orbit average of Tr[rho g.s] over S_n for a string with counts
// (nx, ny, nz): the arrangement of the letters over the sites is uniform over
// all distinct arrangements, so assign sites 0, 1, ... in turn; site k draws
// each remaining letter with probability (remaining count)/(remaining sites).
// E_k(x, y, z) is the expected product over sites k..n-1 given the remaining
// counts.  Every step is a convex combination, so no cancellation occurs.
void build_sn_table(State* st, const double* bloch) {
  int n = st->n;
  int S = n + 1;
  auto at = [S](int x, int y, int z) { return ((size_t)x * S + y) * S + z; };
  std::vector<double> next((size_t)S * S * S, 0.0), cur((size_t)S * S * S, 0.0);
  next[at(0, 0, 0)] = 1.0;  // k = n: nothing left
  for (int k = n - 1; k >= 0; --k) {
    int left = n - k;
    std::fill(cur.begin(), cur.end(), 0.0);
    for (int x = 0; x <= left; ++x)
      for (int y = 0; x + y <= left; ++y)
        for (int z = 0; x + y + z <= left; ++z) {
          int i = left - x - y - z;
          double v = 0.0;
          if (i > 0) v += (double)i * bloch_value(bloch, k, 0) * next[at(x, y, z)];
          if (x > 0) v += (double)x * bloch_value(bloch, k, 1) * next[at(x - 1, y, z)];
          if (y > 0) v += (double)y * bloch_value(bloch, k, 2) * next[at(x, y - 1, z)];
          if (z > 0) v += (double)z * bloch_value(bloch, k, 3) * next[at(x, y, z - 1)];
          cur[at(x, y, z)] = v / (double)left;
        }
    cur.swap(next);
  }
  st->sn_table = next;
  st->sn_bloch.assign(bloch, bloch + 3 * n);
}

double sym_overlap(State* st, const std::string& s, const double* bloch, int group) {
  if (group == 1) {
    double acc = 0.0;
    for (int j = 0; j < st->n; ++j) acc += product_overlap(translate(s, j), bloch);
    return acc / (double)st->n;
  }
  if (group == 2) {
    if (st->sn_bloch.size() != (size_t)(3 * st->n) ||
        !std::equal(st->sn_bloch.begin(), st->sn_bloch.end(), bloch))
      build_sn_table(st, bloch);
    int nx = 0, ny = 0, nz = 0;
    for (char ch : s) {
      nx += (ch == 1);
      ny += (ch == 2);
      nz += (ch == 3);
    }
    int S = st->n + 1;
    return st->sn_table[((size_t)nx * S + ny) * S + nz];
  }
  if (group_kind(group) == 3 || group_kind(group) == 4) {
    const auto& els = cached_elements(group, st->n);
    double acc = 0.0;
    for (const auto& m : els) acc += product_overlap(apply_map(s, m), bloch);
    return acc / (double)els.size();
  }
  return product_overlap(s, bloch);
}

}  // namespace

extern "C" {

// Ingest O = sum c_s s (duplicates accumulate).  With group != 0 the terms
// are replaced by their orbit representatives and merged (Algorithm 1, step
// 1).  Truncation rules are applied at the end.
void* orc_create(int n, long long n_terms, const uint64_t* x, const uint64_t* z,
                 const double* coef, int group, double eps, int wmax) {
  State* st = new State();
  st->n = n;
  st->W = (n + 63) / 64;
  for (long long i = 0; i < n_terms; ++i) {
    std::string s = letters_from_masks(n, st->W, x + i * st->W, z + i * st->W);
    st->terms[s] += coef[i];
  }
  if (group != 0) symmetry_merge(st, group);
  truncate_all(st, eps, wmax);
  return st;
}

void orc_destroy(void* h) { delete (State*)h; }

long long orc_size(void* h) { return (long long)((State*)h)->terms.size(); }

double orc_updates(void* h) { return ((State*)h)->updates; }

// Terms are written in ascending order of the (x words, z words) tuple so the
// output is reproducible.
void orc_export(void* h, uint64_t* x, uint64_t* z, double* coef) {
  State* st = (State*)h;
  std::vector<std::tuple<std::vector<uint64_t>, double>> rows;
  rows.reserve(st->terms.size());
  for (const auto& kv : st->terms) {
    std::vector<uint64_t> key(2 * st->W);
    masks_from_letters(kv.first, st->W, key.data(), key.data() + st->W);
    rows.emplace_back(std::move(key), kv.second);
  }
  std::sort(rows.begin(), rows.end(),
            [](const auto& a, const auto& b) { return std::get<0>(a) < std::get<0>(b); });
  for (size_t i = 0; i < rows.size(); ++i) {
    const auto& key = std::get<0>(rows[i]);
    for (int w = 0; w < st->W; ++w) {
      x[i * st->W + w] = key[w];
      z[i * st->W + w] = key[st->W + w];
    }
    coef[i] = std::get<1>(rows[i]);
  }
}

int orc_apply_gate(void* h, const uint64_t* px, const uint64_t* pz, double theta,
                   int noise_mode, double p, double eps, int wmax) {
  State* st = (State*)h;
  std::string P = letters_from_masks(st->n, st->W, px, pz);
  apply_gate(st, P, theta, noise_mode, p, eps, wmax);
  return 0;
}

// Per-layer depolarising damping c <- c exp(-gamma |Q|) (Fig. 2 caption),
// followed by truncation.
int orc_damp_layer(void* h, double gamma, double eps, int wmax) {
  State* st = (State*)h;
  for (auto& kv : st->terms) kv.second = kv.second * std::exp(-gamma * (double)weight(kv.first));
  truncate_all(st, eps, wmax);
  return 0;
}

int orc_symmetry_merge(void* h, int group, double eps, int wmax) {
  State* st = (State*)h;
  symmetry_merge(st, group);
  truncate_all(st, eps, wmax);
  return 0;
}

int orc_truncate(void* h, double eps, int wmax) {
  truncate_all((State*)h, eps, wmax);
  return 0;
}

// One Heisenberg layer O_{l-1} = U_l^dag O_l U_l (App. A) for a layer given
// in time order: per-layer noise first (it follows the layer in time), then
// the gates from last to first, then the symmetry merge of Eq. (O-merging)
// when `group` is non-zero.
int orc_apply_layer(void* h, int n_gates, const uint64_t* gx, const uint64_t* gz,
                    const double* theta, int noise_mode, double p, double eps, int wmax,
                    int group) {
  State* st = (State*)h;
  if (noise_mode == 2) orc_damp_layer(h, p, eps, wmax);
  for (int g = n_gates - 1; g >= 0; --g) {
    std::string P = letters_from_masks(st->n, st->W, gx + (size_t)g * st->W, gz + (size_t)g * st->W);
    apply_gate(st, P, theta[g], noise_mode, p, eps, wmax);
  }
  if (group != 0) orc_symmetry_merge(h, group, eps, wmax);
  return 0;
}

// Tr[rho O] for a product state (bloch = [n][3]).  With group != 0 each term
// contributes c_r times the orbit average of Tr[rho g.r]; for a symmetric rho
// that average equals Tr[rho r] (Eq. 2).
double orc_expect(void* h, const double* bloch, int group) {
  State* st = (State*)h;
  double acc = 0.0;
  for (const auto& kv : st->terms) acc += kv.second * sym_overlap(st, kv.first, bloch, group);
  return acc;
}

void orc_canonical(int n, long long m, int group, const uint64_t* x, const uint64_t* z,
                   uint64_t* ox, uint64_t* oz) {
  int W = (n + 63) / 64;
  for (long long i = 0; i < m; ++i) {
    std::string s = letters_from_masks(n, W, x + i * W, z + i * W);
    masks_from_letters(canonical(s, group), W, ox + i * W, oz + i * W);
  }
}

// Orbit-averaged overlap of single strings (used to pin the S_n table).
void orc_sym_overlap(int n, long long m, int group, const uint64_t* x, const uint64_t* z,
                     const double* bloch, double* out) {
  State st;
  st.n = n;
  st.W = (n + 63) / 64;
  for (long long i = 0; i < m; ++i) {
    std::string s = letters_from_masks(n, st.W, x + i * st.W, z + i * st.W);
    out[i] = sym_overlap(&st, s, bloch, group);
  }
}

}  // extern "C"

namespace {

// ------------------------------------------------------------------------
// Batched angles: B angle sets share one circuit structure, so every string
// carries a row of B coefficients.  A term is kept iff some column has
// |c_b| >= eps (and its weight is allowed).  Each column follows exactly the
// single-set rules above with its own angles.
// ------------------------------------------------------------------------

struct BState {
  int n = 0, W = 1, B = 1;
  std::unordered_map<std::string, std::vector<double>> terms;
  double updates = 0.0;
  State helper;  // for overlaps (S_n table cache)
};

bool keep_row(const std::vector<double>& c, const std::string& s, double eps, int wmax) {
  if (wmax >= 0 && weight(s) > wmax) return false;
  if (eps <= 0.0) return true;
  for (double v : c)
    if (std::fabs(v) >= eps) return true;
  return false;
}

void btruncate(BState* st, double eps, int wmax) {
  for (auto it = st->terms.begin(); it != st->terms.end();) {
    if (!keep_row(it->second, it->first, eps, wmax))
      it = st->terms.erase(it);
    else
      ++it;
  }
}

void bmerge(BState* st, int group) {
  std::unordered_map<std::string, std::vector<double>> merged;
  for (const auto& kv : st->terms) {
    auto& row = merged[canonical(kv.first, group)];
    if (row.empty()) row.assign(st->B, 0.0);
    for (int b = 0; b < st->B; ++b) row[b] += kv.second[b];
  }
  st->terms.swap(merged);
}

void bapply_gate(BState* st, const std::string& P, const double* theta, int noise_mode, double p,
                 double eps, int wmax) {
  const int B = st->B;
  std::vector<double> c(B), s(B);
  for (int b = 0; b < B; ++b) {
    c[b] = std::cos(theta[b]);
    s[b] = std::sin(theta[b]);
  }
  std::vector<int> support;
  for (int q = 0; q < st->n; ++q)
    if (P[q] != 0) support.push_back(q);
  std::vector<double> damp(support.size() + 1, 1.0);
  for (size_t k = 1; k < damp.size(); ++k) damp[k] = damp[k - 1] * (1.0 - p);
  st->updates += (double)st->terms.size();
  std::unordered_map<std::string, std::vector<double>> next;
  auto row_of = [&](const std::string& key) -> std::vector<double>& {
    auto& r = next[key];
    if (r.empty()) r.assign(B, 0.0);
    return r;
  };
  for (const auto& kv : st->terms) {
    const std::string& Q = kv.first;
    std::vector<double> d = kv.second;
    if (noise_mode == 1) {
      int k = 0;
      for (int q : support) k += (Q[q] != 0);
      if (k > 0)
        for (int b = 0; b < B; ++b) d[b] = d[b] * damp[k];
    }
    int anti = 0;
    for (int q : support) anti += site_anticommutes((uint8_t)P[q], (uint8_t)Q[q]);
    if (anti % 2 == 0) {
      auto& r = row_of(Q);
      for (int b = 0; b < B; ++b) r[b] += d[b];
      continue;
    }
    std::string R = Q;
    int phase = 0;
    for (int q : support) {
      const Prod& pr = kMul[(uint8_t)P[q]][(uint8_t)Q[q]];
      R[q] = (char)pr.letter;
      phase += pr.phase;
    }
    double sign = ((phase + 1) % 4 == 0) ? 1.0 : -1.0;
    auto& rq = row_of(Q);
    for (int b = 0; b < B; ++b) rq[b] += c[b] * d[b];
    auto& rr = row_of(R);
    for (int b = 0; b < B; ++b) rr[b] += sign * (s[b] * d[b]);
  }
  st->terms.swap(next);
  btruncate(st, eps, wmax);
}

}  // namespace

extern "C" {

void* orcb_create(int n, long long n_terms, int B, const uint64_t* x, const uint64_t* z,
                  const double* coef, int group, double eps, int wmax) {
  BState* st = new BState();
  st->n = n;
  st->W = (n + 63) / 64;
  st->B = B;
  st->helper.n = n;
  st->helper.W = st->W;
  for (long long i = 0; i < n_terms; ++i) {
    std::string s = letters_from_masks(n, st->W, x + i * st->W, z + i * st->W);
    auto& r = st->terms[s];
    if (r.empty()) r.assign(B, 0.0);
    for (int b = 0; b < B; ++b) r[b] += coef[i * B + b];
  }
  if (group != 0) bmerge(st, group);
  btruncate(st, eps, wmax);
  return st;
}

void orcb_destroy(void* h) { delete (BState*)h; }
long long orcb_size(void* h) { return (long long)((BState*)h)->terms.size(); }
double orcb_updates(void* h) { return ((BState*)h)->updates; }

// Layer in time order, theta = [n_gates][B]; applied last gate first, then
// the symmetry merge when group != 0.
int orcb_apply_layer(void* h, int n_gates, const uint64_t* gx, const uint64_t* gz,
                     const double* theta, int noise_mode, double p, double eps, int wmax,
                     int group) {
  BState* st = (BState*)h;
  for (int g = n_gates - 1; g >= 0; --g) {
    std::string P = letters_from_masks(st->n, st->W, gx + (size_t)g * st->W, gz + (size_t)g * st->W);
    bapply_gate(st, P, theta + (size_t)g * st->B, noise_mode, p, eps, wmax);
  }
  if (group != 0) {
    bmerge(st, group);
    btruncate(st, eps, wmax);
  }
  return 0;
}

void orcb_expect(void* h, const double* bloch, int group, double* out) {
  BState* st = (BState*)h;
  for (int b = 0; b < st->B; ++b) out[b] = 0.0;
  for (const auto& kv : st->terms) {
    double ov = sym_overlap(&st->helper, kv.first, bloch, group);
    for (int b = 0; b < st->B; ++b) out[b] += kv.second[b] * ov;
  }
}

void orcb_export(void* h, uint64_t* x, uint64_t* z, double* coef) {
  BState* st = (BState*)h;
  std::vector<std::pair<std::vector<uint64_t>, const std::vector<double>*>> rows;
  for (const auto& kv : st->terms) {
    std::vector<uint64_t> key(2 * st->W);
    masks_from_letters(kv.first, st->W, key.data(), key.data() + st->W);
    rows.emplace_back(std::move(key), &kv.second);
  }
  std::sort(rows.begin(), rows.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  for (size_t i = 0; i < rows.size(); ++i) {
    for (int w = 0; w < st->W; ++w) {
      x[i * st->W + w] = rows[i].first[w];
      z[i * st->W + w] = rows[i].first[st->W + w];
    }
    for (int b = 0; b < st->B; ++b) coef[i * st->B + b] = (*rows[i].second)[b];
  }
}

}  // extern "C"
