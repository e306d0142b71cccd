// Bond form-factor basis (Sec. 3, footnote: one bond length per function,
// C4v irreps s, p, d, g; Sec. 2.3: real functions on a Bravais lattice).
//
// Each function is stored as a short sum of cos/sin plane waves
// trig(k . R), which also gives its exact bond coefficients
// c_m(R) in f_m(k) = sum_R c_m(R) exp(i k . R).
#include <cmath>
#include <map>
#include <utility>

#include "internal.h"

namespace tufrg {
namespace {

// squared length of each shell 0..6
const int kShellR2[7] = {0, 1, 2, 4, 5, 8, 9};
const int kShellSize[7] = {1, 4, 4, 4, 8, 4, 4};

int shell_of(int x, int y) {
  int r2 = x * x + y * y;
  for (int s = 0; s < 7; ++s)
    if (kShellR2[s] == r2) return s;
  return -1;
}

FormFactor make(int shell, const char* irrep, std::vector<TrigTerm> terms) {
  FormFactor f;
  f.shell = shell;
  f.irrep = irrep;
  f.terms = std::move(terms);
  f.parity = f.terms.front().is_sin ? -1 : 1;
  return f;
}

// Functions of one shell in canonical order (A1, B1/B2/A2, E pairs).
std::vector<FormFactor> shell_functions(int s) {
  const double r2 = std::sqrt(2.0), h = std::sqrt(2.0) / 2.0;
  std::vector<FormFactor> v;
  auto C = [](double c, int x, int y) { return TrigTerm{c, false, x, y}; };
  auto S = [](double c, int x, int y) { return TrigTerm{c, true, x, y}; };
  if (s == 0) {
    v.push_back(make(0, "A1", {C(1.0, 0, 0)}));
  } else if (s == 1 || s == 3 || s == 6) {  // axial bonds (n, 0), (0, n)
    int n = s == 1 ? 1 : (s == 3 ? 2 : 3);
    v.push_back(make(s, "A1", {C(1.0, n, 0), C(1.0, 0, n)}));
    v.push_back(make(s, "B1", {C(1.0, n, 0), C(-1.0, 0, n)}));
    v.push_back(make(s, "E", {S(r2, n, 0)}));
    v.push_back(make(s, "E", {S(r2, 0, n)}));
  } else if (s == 2 || s == 5) {  // diagonal bonds (n, +-n)
    int n = s == 2 ? 1 : 2;
    // 2 c c = cos(a+b) + cos(a-b); 2 s s = cos(a-b) - cos(a+b)
    // 2 s c = sin(a+b) + sin(a-b); 2 c s = sin(a+b) - sin(a-b)
    v.push_back(make(s, "A1", {C(1.0, n, n), C(1.0, n, -n)}));
    v.push_back(make(s, "B2", {C(1.0, n, -n), C(-1.0, n, n)}));
    v.push_back(make(s, "E", {S(1.0, n, n), S(1.0, n, -n)}));
    v.push_back(make(s, "E", {S(1.0, n, n), S(-1.0, n, -n)}));
  } else if (s == 4) {  // knight bonds (2, 1), (1, 2)
    v.push_back(make(4, "A1", {C(h, 2, 1), C(h, 2, -1), C(h, 1, 2), C(h, 1, -2)}));
    v.push_back(make(4, "B1", {C(h, 2, 1), C(h, 2, -1), C(-h, 1, 2), C(-h, 1, -2)}));
    v.push_back(make(4, "B2", {C(h, 2, -1), C(-h, 2, 1), C(h, 1, -2), C(-h, 1, 2)}));
    v.push_back(make(4, "A2", {C(h, 2, -1), C(-h, 2, 1), C(-h, 1, -2), C(h, 1, 2)}));
    v.push_back(make(4, "E", {S(1.0, 2, 1), S(1.0, 2, -1)}));   // 2 s2x cy
    v.push_back(make(4, "E", {S(1.0, 1, 2), S(-1.0, 1, -2)}));  // 2 cx s2y
    v.push_back(make(4, "E", {S(1.0, 1, 2), S(1.0, 1, -2)}));   // 2 sx c2y
    v.push_back(make(4, "E", {S(1.0, 2, 1), S(-1.0, 2, -1)}));  // 2 c2x sy
  }
  return v;
}

}  // namespace

tufrg_status Basis::build(int n_bonds, const int32_t* bonds) {
  if (n_bonds <= 0 || bonds == nullptr) return TUFRG_ERR_ARG;
  std::map<std::pair<int, int>, int> index;
  int count[7] = {0, 0, 0, 0, 0, 0, 0};
  n_shells = -1;
  bx.assign(n_bonds, 0);
  by.assign(n_bonds, 0);
  max_component = 0;
  for (int b = 0; b < n_bonds; ++b) {
    int x = bonds[2 * b], y = bonds[2 * b + 1];
    int s = shell_of(x, y);
    if (s < 0) return TUFRG_ERR_ARG;
    if (!index.emplace(std::make_pair(x, y), b).second) return TUFRG_ERR_ARG;  // duplicate
    ++count[s];
    if (s > n_shells) n_shells = s;
    bx[b] = x;
    by[b] = y;
    max_component = std::max(max_component, std::max(std::abs(x), std::abs(y)));
  }
  for (int s = 0; s <= n_shells; ++s)
    if (count[s] != kShellSize[s]) return TUFRG_ERR_ARG;  // shells must be complete
  nb = n_bonds;
  ff.clear();
  for (int s = 0; s <= n_shells; ++s)
    for (auto& f : shell_functions(s)) ff.push_back(f);
  nff = (int)ff.size();
  if (nff != nb) return TUFRG_ERR_ARG;
  coef.assign((size_t)nff * nb, std::complex<double>(0.0, 0.0));
  for (int m = 0; m < nff; ++m) {
    for (const TrigTerm& t : ff[m].terms) {
      auto plus = index.find({t.rx, t.ry});
      auto minus = index.find({-t.rx, -t.ry});
      if (plus == index.end() || minus == index.end()) return TUFRG_ERR_ARG;
      // cos(kR) = (e^{ikR} + e^{-ikR})/2, sin(kR) = (e^{ikR} - e^{-ikR})/(2i)
      std::complex<double> cp = t.is_sin ? std::complex<double>(0.0, -0.5 * t.coef)
                                         : std::complex<double>(0.5 * t.coef, 0.0);
      coef[(size_t)m * nb + plus->second] += cp;
      coef[(size_t)m * nb + minus->second] += std::conj(cp);
    }
  }
  return TUFRG_OK;
}

// The eight elements g of C4v as integer matrices acting on momenta k:
// identity, rotations by 90, 180, 270 degrees, mirrors y -> -y, x -> -x,
// the diagonal and the antidiagonal.
const int kC4v[8][2][2] = {{{1, 0}, {0, 1}},  {{0, -1}, {1, 0}}, {{-1, 0}, {0, -1}},
                           {{0, 1}, {-1, 0}}, {{1, 0}, {0, -1}}, {{-1, 0}, {0, 1}},
                           {{0, 1}, {1, 0}},  {{0, -1}, {-1, 0}}};

// f_m(g k) = sum_n R^g_mn f_n(k).  With f_m(k) = sum_b c_m(b) e^{i k.R_b}
// and g orthogonal, f_m(g k) = sum_b c_m(b) e^{i k.(g^T R_b)}, so
// R^g_mn = sum_b c_m(b) conj(c_n(b')), R_b' = g^T R_b (plane waves of distinct
// bonds are orthonormal under the zone average).  For a basis adapted to
// C4v every R^g is a signed permutation; returns false otherwise.
bool Basis::point_group(std::vector<int>& perm, std::vector<int>& sign) const {
  std::map<std::pair<int, int>, int> index;
  for (int b = 0; b < nb; ++b) index[{bx[b], by[b]}] = b;
  perm.assign(8 * (size_t)nff, 0);
  sign.assign(8 * (size_t)nff, 0);
  for (int g = 0; g < 8; ++g) {
    std::vector<int> bmap(nb);
    for (int b = 0; b < nb; ++b) {
      // g^T R_b
      const int x = kC4v[g][0][0] * bx[b] + kC4v[g][1][0] * by[b];
      const int y = kC4v[g][0][1] * bx[b] + kC4v[g][1][1] * by[b];
      auto it = index.find({x, y});
      if (it == index.end()) return false;
      bmap[b] = it->second;
    }
    for (int m = 0; m < nff; ++m) {
      int found = -1;
      for (int n = 0; n < nff; ++n) {
        std::complex<double> r(0.0, 0.0);
        for (int b = 0; b < nb; ++b)
          r += coef[(size_t)m * nb + b] * std::conj(coef[(size_t)n * nb + bmap[b]]);
        if (std::abs(r.imag()) > 1e-9) return false;
        if (std::abs(r.real()) < 1e-9) continue;
        if (found >= 0 || std::abs(std::abs(r.real()) - 1.0) > 1e-9) return false;
        found = n;
        sign[(size_t)g * nff + m] = r.real() > 0 ? 1 : -1;
      }
      if (found < 0) return false;
      perm[(size_t)g * nff + m] = found;
    }
  }
  return true;
}

double Basis::eval(int m, double kx, double ky) const {
  double v = 0.0;
  for (const TrigTerm& t : ff[m].terms) {
    double a = kx * t.rx + ky * t.ry;
    v += t.coef * (t.is_sin ? std::sin(a) : std::cos(a));
  }
  return v;
}

}  // namespace tufrg
